"""GPU parity for general trigonometric range kernels (Section 2.2,
phi(s) = a_0 + a_1 cos(gamma s) + ... + a_N cos(N gamma s)) against the FP64
oracle's term-by-term brute force: every kernel path (tile kernels, the
large-radius streaming sweeps, interleaved channels, stacks, batches) and the
adjoint for dL/df.  Bars as for the raised cosine: max abs error <= 0.05 gray
levels; gradients within 1e-3 relative."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
TOL = 0.05
REL = 1e-3
GAMMA = math.pi / 510  # the paper's gamma = pi / 2T for T = 255


def _fejer(N):
    # Fejer kernel: sum_{|n|<=N} (1 - |n|/(N+1)) e^{j n x} >= 0 everywhere, in real form
    return np.array([1.0] + [2.0 * (1.0 - n / (N + 1.0)) for n in range(1, N + 1)]) / (N + 1.0)


KERNELS = {
    "fejer6": _fejer(6),
    "fejer20": _fejer(20),
    "decaying": np.array([1.0, 0.8, 0.5, 0.3, 0.1]),
    "sparse": np.array([0.6, 0.0, 0.0, 0.4]),
}


@pytest.fixture(scope="module")
def bf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_4204_gb300 import build
    build.build()
    import paper_1105_4204_gb300 as pkg
    return pkg


def _w1(oracle, plan):
    if plan.kind == "gauss":
        return oracle.spatial_w1("gauss", plan.sigma_s, radius=plan.radius)
    return oracle.spatial_w1("box", plan.sigma_s, radius=plan.radius // 3, passes=3)


def _run(bf, img, plan):
    import torch
    out = bf.forward(plan, torch.from_numpy(np.ascontiguousarray(img)).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_kernels_are_positive_on_the_range(oracle):
    s = np.linspace(-255, 255, 2041)
    for a in KERNELS.values():
        assert oracle.phi_cos(s, GAMMA, a).min() > 0


@pytest.mark.parametrize("name", sorted(KERNELS))
@pytest.mark.parametrize("kind,ss,rad", [("gauss", 3.0, 9), ("gauss", 1.0, 3), ("box", 2.0, 2),
                                         ("box", 8.0, 8), ("box", 12.0, 12)])
def test_forward_every_path(bf, oracle, name, kind, ss, rad):
    # tile kernels (Gaussian, box r <= 8) and the streaming sweeps (box r = 12)
    img = synth.smooth_field(70, 131, noise=6.0, seed=rad + len(name))
    plan = bf.Plan.cosine(ss, GAMMA, KERNELS[name], kind=kind, radius=rad)
    out = _run(bf, img, plan)
    ref = oracle.bf_brute_cos(img.astype(np.float64), GAMMA, KERNELS[name], w1=_w1(oracle, plan))
    err = np.abs(out - ref).max()
    print("%s %s rad=%d max abs err %.3e" % (name, kind, rad, err))
    assert err <= TOL


def test_raised_cosine_coefficients_match_the_raised_cosine_plan(bf):
    # the raised cosine written as a cosine polynomial runs the same kernels
    N, sr = 30, 30.0
    a = np.zeros(N + 1)
    for n in range(N + 1):
        a[abs(N - 2 * n)] += math.comb(N, n) / 2.0 ** N
    img = synth.rectangles(90, 110, seed=4)
    p1 = bf.Plan(3.0, sr, kind="gauss")
    p2 = bf.Plan.cosine(3.0, 1.0 / (sr * math.sqrt(N)), a, kind="gauss")
    assert p1.N == p2.N == N and p1.n_terms == p2.n_terms
    assert np.abs(_run(bf, img, p1) - _run(bf, img, p2)).max() <= 1e-3


def test_u8_channels_and_stack(bf, oracle):
    import torch
    a = KERNELS["decaying"]
    img = synth.rect_disk_u8(50, 67, C=3, n_shapes=8, seed=2)
    plan = bf.Plan.cosine(2.0, GAMMA, a, kind="gauss")
    out = _run(bf, img, plan)
    ref = oracle.bf_brute_cos(img.astype(np.float64), GAMMA, a, w1=_w1(oracle, plan))
    assert np.abs(out - ref).max() <= TOL
    stack = np.stack([synth.rectangles(40, 56, seed=s) for s in range(3)])
    got = bf.forward_stack(plan, torch.from_numpy(stack).cuda()).cpu().numpy()
    for k in range(3):
        r = oracle.bf_brute_cos(stack[k].astype(np.float64), GAMMA, a, w1=_w1(oracle, plan))
        assert np.abs(got[k] - r).max() <= TOL


def test_batch_with_cosine_plans(bf, oracle):
    # a batch mixing cosine-polynomial and raised-cosine box plans, tile and streaming radii
    import torch
    sizes = [(60, 90), (45, 130), (80, 70), (33, 47)]
    plans = [bf.Plan.cosine(2.0, GAMMA, KERNELS["fejer6"], kind="box"),
             bf.Plan(4.0, 30.0, kind="box"),
             bf.Plan.cosine(10.0, GAMMA, KERNELS["decaying"], kind="box"),
             bf.Plan.cosine(6.0, GAMMA, KERNELS["sparse"], kind="box")]
    imgs = [synth.rectangles(h, w, seed=i) for i, (h, w) in enumerate(sizes)]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.empty_like(t) for t in ins]
    b = bf.Batch(plans, sizes)
    b.bind(ins, outs)
    b.forward()
    assert b.check() == 0
    for i, p in enumerate(plans):
        if p.radius // 3 <= 8:  # the batch's configuration: 32 x 64 tiles, all terms per block
            bf.set_shape(p, ins[i], "32x64", split=1)
        single = bf.forward(p, ins[i]).cpu().numpy()
        got = outs[i].cpu().numpy()
        assert np.array_equal(got, single)
        if p.sigma_r is None:
            ref = oracle.bf_brute_cos(imgs[i].astype(np.float64), GAMMA, p.coefs,
                                      w1=_w1(oracle, p))
            assert np.abs(got - ref).max() <= TOL


@pytest.mark.parametrize("name,kind,ss,rad", [("decaying", "gauss", 2.0, 6),
                                              ("fejer6", "gauss", 1.5, 5),
                                              ("sparse", "box", 2.0, 2)])
def test_backward_image_gradient(bf, oracle, name, kind, ss, rad):
    import torch
    a = KERNELS[name]
    img = synth.rectangles(48, 72, n_rect=6, noise=8.0, seed=rad)
    u = synth.upstream(img.shape, seed=rad + 1)
    plan = bf.Plan.cosine(ss, GAMMA, a, kind=kind, radius=rad)
    f = torch.from_numpy(img).cuda()
    out, q = bf.forward(plan, f, return_q=True)
    g, gs = bf.backward(plan, f, out, q, torch.from_numpy(u).cuda(), need_sigma=False)
    assert gs is None
    g = g.cpu().numpy().astype(np.float64)
    w1 = _w1(oracle, plan)
    gref = oracle.bf_grad_cos(img.astype(np.float64), u.astype(np.float64), GAMMA, a, w1=w1)
    scale = np.abs(gref).max()
    assert np.abs(g - gref).max() <= REL * scale
    assert np.linalg.norm(g - gref) <= REL * np.linalg.norm(gref)
    idx = synth.sample_indices(48, 72, 60, seed=9)
    fd = oracle.fd_grad_f_cos(img.astype(np.float64), u.astype(np.float64), idx, GAMMA, a,
                              h=1e-3, w1=w1)
    assert np.abs(g.ravel()[idx] - fd).max() <= REL * np.abs(fd).max()
    with pytest.raises(Exception):
        bf.backward(plan, f, out, q, torch.from_numpy(u).cuda(), need_sigma=True)
