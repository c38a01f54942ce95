"""GPU parity of the batched launch: every image against the single-image
path in the same configuration (bit for bit: both run the same tile body for
r <= 8 and the same streaming sweeps above) and against the FP64 oracle on
sampled pixels."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
TOL = 0.05


@pytest.fixture(scope="module")
def bf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_4204_gb300 import build
    build.build()
    import paper_1105_4204_gb300 as pkg
    return pkg


def _single(bf, plan, img, batch=None):
    """bf_forward of one image in the configuration the batch runs for its
    radius bucket (tile shape and term split; by default 32 x 64 tiles with all
    terms in one block -- bf_forward alone would cut the terms of a small
    image into groups, which sums them in another order)."""
    r = plan.radius // 3
    if r <= 8:
        shape, split = batch.config()[r] if batch is not None else ("32x64", 1)
        bf.set_shape(plan, img, shape, split=split)
    return bf.forward(plan, img)


def _setup(bf, specs, seed):
    import torch
    imgs = synth.batch_images(specs, noise=10.0, seed=seed)
    plans = [bf.Plan(ss, sr, 255.0, kind="box") for (_, _, ss, sr) in specs]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.empty_like(t) for t in ins]
    b = bf.Batch(plans, [(h, w) for (h, w, _, _) in specs])
    b.bind(ins, outs)
    return imgs, plans, ins, outs, b


def test_small_batch_against_single_and_oracle(bf, oracle):
    import torch
    specs = synth.batch_specs(12, seed=7, w_range=(40, 300), h_range=(30, 200))
    imgs, plans, ins, outs, b = _setup(bf, specs, seed=7)
    b.forward()
    assert b.check() == 0
    for i, (h, w, ss, sr) in enumerate(specs):
        got = outs[i].cpu().numpy()
        single = _single(bf, plans[i], ins[i]).cpu().numpy()
        r = plans[i].radius // 3
        np.testing.assert_array_equal(got, single)
        idx = synth.sample_indices(h, w, 300, seed=i)
        w1 = oracle.spatial_w1("box", ss)
        ref = oracle.bf_brute_at(imgs[i].astype(np.float64), idx, sigma_r=sr, w1=w1, N=plans[i].N)
        assert np.abs(got.ravel()[idx] - ref).max() <= TOL, (i, r, plans[i].N)


def test_config4_batch_matches_single_image_path(bf, oracle):
    # 64 images, W ~ U[128, 1920], H ~ U[128, 1080], sigma_s ~ U[2, 16],
    # sigma_r ~ U[15, 60]; rectangles + noise 10
    import torch
    specs = synth.batch_specs(64, seed=0)
    imgs, plans, ins, outs, b = _setup(bf, specs, seed=0)
    Ns = sorted(p.N for p in plans)
    assert Ns[0] >= 8 and Ns[-1] <= 118
    rs = [p.radius // 3 for p in plans]
    assert min(rs) <= 8 < max(rs)  # both the persistent tiles and the streaming sweeps
    b.forward()
    torch.cuda.synchronize()
    assert b.check() == 0
    worst = 0.0
    for i, (h, w, ss, sr) in enumerate(specs):
        got = outs[i]
        single = _single(bf, plans[i], ins[i])
        worst = max(worst, float((got - single).abs().max()))
        if i % 16 == 0:  # oracle on a sample of a few images
            idx = synth.sample_indices(h, w, 64, seed=i, border=False)
            ref = oracle.bf_brute_at(imgs[i].astype(np.float64), idx, sigma_r=sr,
                                     w1=oracle.spatial_w1("box", ss), N=plans[i].N)
            assert np.abs(got.cpu().numpy().ravel()[idx] - ref).max() <= TOL
    assert worst == 0.0


def test_replay_tune_and_rebind(bf):
    import torch
    specs = synth.batch_specs(10, seed=3, w_range=(64, 256), h_range=(64, 256))
    imgs, plans, ins, outs, b = _setup(bf, specs, seed=3)
    b.forward()
    before = [o.clone() for o in outs]
    info = b.tune(reps=2)
    assert info["grid"] >= 1 and info["ms"] > 0
    b.forward()
    first = [o.clone() for o in outs]
    # the tuned configuration may sum the terms in groups: equal to rounding
    for a, c in zip(before, first):
        torch.testing.assert_close(a, c, rtol=0, atol=1e-3)
    for o in outs:
        o.zero_()
    b.forward()
    b.forward()  # replays are idempotent
    assert b.check() == 0
    for a, c in zip(first, outs):
        torch.testing.assert_close(a, c, rtol=0, atol=0)
    # rebinding to new buffers
    outs2 = [torch.empty_like(t) for t in ins]
    b.bind(ins, outs2)
    b.forward()
    torch.cuda.synchronize()
    for a, c in zip(first, outs2):
        torch.testing.assert_close(a, c, rtol=0, atol=0)


def test_batch_rejects_unsupported_plans(bf):
    from paper_1105_4204_gb300._lib import BfError
    with pytest.raises(BfError):
        bf.Batch([bf.Plan(3.0, 30.0, kind="gauss")], [(32, 32)])


def test_batch_of_streaming_images_only(bf, oracle):
    # every image with r > 8: no persistent launch, only streaming sweeps
    import torch
    specs = [(70, 150, 12.0, 30.0), (130, 90, 20.0, 25.0), (40, 300, 40.0, 40.0)]
    imgs, plans, ins, outs, b = _setup(bf, specs, seed=4)
    assert all(p.radius // 3 > 8 for p in plans)
    b.forward()
    b.forward()
    assert b.check() == 0
    for i, (h, w, ss, sr) in enumerate(specs):
        got = outs[i].cpu().numpy()
        np.testing.assert_array_equal(got, _single(bf, plans[i], ins[i]).cpu().numpy())
        idx = synth.sample_indices(h, w, 200, seed=i)
        ref = oracle.bf_brute_at(imgs[i].astype(np.float64), idx, sigma_r=sr,
                                 w1=oracle.spatial_w1("box", ss), N=plans[i].N)
        assert np.abs(got.ravel()[idx] - ref).max() <= TOL


@pytest.mark.parametrize("split", [1, 2, 4])
def test_every_bucket_configuration_matches_single_image(bf, oracle, split):
    # every radius bucket in every tile shape it has, with its terms in 1, 2
    # or 4 groups per tile: each image bit for bit as bf_forward in the same
    # configuration, and within the bar against the oracle
    import torch
    specs = [(70 + 9 * r, 150 - 7 * r, float(r), 20.0 + 3 * r) for r in range(1, 9)]
    imgs, plans, ins, outs, b = _setup(bf, specs, seed=40 + split)
    assert [p.radius // 3 for p in plans] == list(range(1, 9))
    shapes = {r: ["32x64"] + (["32x96"] if r <= 4 else []) + (["64x64-seg32"] if r >= 7 else [])
              for r in range(1, 9)}
    for k in range(3):
        for r in range(1, 9):
            b.set_config(r, shapes[r][min(k, len(shapes[r]) - 1)], split)
        b.forward()
        assert b.check() == 0
        cfg = b.config()
        for i, (h, w, ss, sr) in enumerate(specs):
            got = outs[i].cpu().numpy()
            np.testing.assert_array_equal(got, _single(bf, plans[i], ins[i], b).cpu().numpy())
            idx = synth.sample_indices(h, w, 60, seed=i + k)
            ref = oracle.bf_brute_at(imgs[i].astype(np.float64), idx, sigma_r=sr,
                                     w1=oracle.spatial_w1("box", ss), N=plans[i].N)
            assert np.abs(got.ravel()[idx] - ref).max() <= TOL, (i, cfg[i + 1])


def test_tuner_picks_a_configuration_per_bucket(bf):
    import torch
    specs = synth.batch_specs(20, seed=5, w_range=(100, 700), h_range=(100, 500))
    imgs, plans, ins, outs, b = _setup(bf, specs, seed=5)
    info = b.tune(reps=1)
    assert set(info["buckets"]) == set(range(1, 9))
    for r, (shape, split) in info["buckets"].items():
        assert shape in ("32x64", "32x96", "64x64-seg32") and split in (1, 2, 4)
    b.forward()
    assert b.check() == 0
    for i in range(len(plans)):
        np.testing.assert_array_equal(outs[i].cpu().numpy(),
                                      _single(bf, plans[i], ins[i], b).cpu().numpy())
    with pytest.raises(Exception):
        b.set_config(5, "32x96", 1)   # 32 x 96 tiles serve r <= 4
    with pytest.raises(Exception):
        b.set_config(3, "32x64", 3)   # splits 1, 2, 4
