"""GPU parity of the recursive O(1) Gaussian spatial filter (the one the
paper's experiments use, Section 3; Young and van Vliet's third-order
recursion) against the FP64 oracle's Algorithm 1 with the same recursion.
Bar: max abs error <= 0.05 gray levels."""
import math

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


def _run(bf, img, plan):
    import torch
    out = bf.forward(plan, torch.from_numpy(np.ascontiguousarray(img)).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("ss", [0.5, 1.0, 2.4, 2.5, 5.0, 20.0])
@pytest.mark.parametrize("sr", [20.0, 60.0])
def test_against_oracle(bf, oracle, ss, sr):
    img = synth.smooth_field(83, 117, noise=6.0, seed=int(ss * 10) + int(sr))
    plan = bf.Plan(ss, sr, kind="recursive")
    out = _run(bf, img, plan)
    ref = oracle.bf_trig_rg(img.astype(np.float64), sigma_s=ss, sigma_r=sr, N=plan.N)
    err = np.abs(out - ref).max()
    print("recursive sigma_s=%g sigma_r=%g N=%d max abs err %.3e" % (ss, sr, plan.N, err))
    assert err <= TOL


@pytest.mark.parametrize("H,W", [(1, 1), (1, 50), (50, 1), (17, 3), (3, 40), (33, 16)])
def test_degenerate_sizes(bf, oracle, H, W):
    img = synth.rectangles(H, W, n_rect=3, noise=8.0, seed=H * 7 + W)
    plan = bf.Plan(3.0, 30.0, kind="recursive")
    ref = oracle.bf_trig_rg(img.astype(np.float64), sigma_s=3.0, sigma_r=30.0, N=plan.N)
    assert np.abs(_run(bf, img, plan) - ref).max() <= TOL


def test_more_terms_than_one_vertical_launch(bf, oracle):
    # N = 200: the terms pass through the scratch in two rounds (64 + the rest)
    N = 200
    sr = 1.001 * 2 * 255.0 / (math.pi * math.sqrt(N))
    img = synth.rectangles(40, 60, n_rect=5, noise=8.0, seed=5)
    plan = bf.Plan(2.0, sr, kind="recursive", N=N)
    assert plan.n_terms > 64
    ref = oracle.bf_trig_rg(img.astype(np.float64), sigma_s=2.0, sigma_r=sr, N=N)
    assert np.abs(_run(bf, img, plan) - ref).max() <= TOL


def test_u8_channels_and_stack(bf, oracle):
    import torch
    img = synth.rect_disk_u8(45, 70, C=3, n_shapes=6, seed=3)
    plan = bf.Plan(4.0, 30.0, kind="recursive")
    ref = oracle.bf_trig_rg(img.astype(np.float64), sigma_s=4.0, sigma_r=30.0, N=plan.N)
    assert np.abs(_run(bf, img, plan) - ref).max() <= TOL
    stack = np.stack([synth.rectangles(30, 50, seed=s) for s in range(3)])
    got = bf.forward_stack(plan, torch.from_numpy(stack).cuda()).cpu().numpy()
    for k in range(3):
        r = oracle.bf_trig_rg(stack[k].astype(np.float64), sigma_s=4.0, sigma_r=30.0, N=plan.N)
        assert np.abs(got[k] - r).max() <= TOL


@pytest.mark.parametrize("ss", [10.0, 100.0])
def test_paper_timing_image_size(bf, oracle, ss):
    # the 720 x 540 image of the paper's timing table, sigma_s = 10 and 100, sigma_r = 30
    img = synth.rectangles(540, 720, n_rect=20, noise=10.0, seed=int(ss))
    plan = bf.Plan(ss, 30.0, kind="recursive")
    ref = oracle.bf_trig_rg(img.astype(np.float64), sigma_s=ss, sigma_r=30.0, N=plan.N)
    err = np.abs(_run(bf, img, plan) - ref).max()
    print("720x540 sigma_s=%g max abs err %.3e" % (ss, err))
    assert err <= TOL


def test_batch_with_recursive_and_box_images(bf):
    # recursive-Gaussian images run on the batch's streaming chains beside box
    # images on tiles and on chains: each streaming image equals its
    # single-image call bit for bit (the tile image up to the summation order
    # of the single call's own configuration); the adjoint is tested with the
    # others in test_gpu_backward.py
    import torch
    specs = [("recursive", 3.0, 30.0, 70, 90), ("box", 2.0, 25.0, 64, 80),
             ("recursive", 10.0, 20.0, 130, 50), ("box", 12.0, 20.0, 40, 100),
             ("recursive", 0.8, 40.0, 1, 33)]
    plans = [bf.Plan(ss, sr, kind=k) for k, ss, sr, _, _ in specs]
    imgs = [torch.from_numpy(synth.rectangles(h, w, seed=i)).cuda()
            for i, (_, _, _, h, w) in enumerate(specs)]
    outs = [torch.empty_like(t) for t in imgs]
    batch = bf.Batch(plans, [tuple(t.shape) for t in imgs])
    batch.bind(imgs, outs)
    batch.forward()
    torch.cuda.synchronize()
    assert batch.check() == 0
    for (k, ss, _, _, _), p, t, o in zip(specs, plans, imgs, outs):
        ref = bf.forward(p, t)
        if k == "recursive" or p.radius // 3 > 8:
            assert torch.equal(o, ref)
        else:
            torch.testing.assert_close(o, ref, rtol=0, atol=1e-3)
