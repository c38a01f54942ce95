"""bf_backward_noalloc: the backward entry point for callers that cannot
allocate device memory (real-time loops, fixed memory pools, plug-in hosts
that own every allocation).  It runs the same kernel and the same
fixed-order reduction as bf_backward with a caller workspace, so its results
must be the same bits, call after call, although every call reuses one fixed
device array for its partial sums.  This file is named to be collected last,
so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_4204_gb300 import build
    build.build()
    import paper_1105_4204_gb300 as bf
    from paper_1105_4204_gb300 import _lib
    l = ctypes.CDLL(_lib.LIB_PATH)  # same library object the binding loaded
    fn = l.bf_backward_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 7 + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    return torch, bf, fn, l


def _noalloc(torch, fn, plan, f, out, q, u, need_sigma=True):
    g = torch.empty_like(f)
    gs = torch.full((), float("nan"), dtype=torch.float64, device=f.device)
    st = fn(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(u.data_ptr()),
            ctypes.c_void_p(g.data_ptr()),
            ctypes.c_void_p(gs.data_ptr() if need_sigma else 0), f.shape[0], f.shape[1],
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return g, gs


def _inputs(torch, bf, plan, H, W, seed):
    f = torch.from_numpy(synth.rectangles(H, W, seed=seed)).cuda()
    u = torch.from_numpy(synth.upstream((H, W), seed=seed + 1)).cuda()
    out, q = bf.forward(plan, f, return_q=True)
    return f, out, q, u


@pytest.mark.parametrize("kind,ss,sr,H,W", [("gauss", 4.0, 25.0, 512, 512),
                                              ("box", 2.0, 20.0, 300, 170)])
def test_noalloc_matches_workspace_backward_bit_for_bit(env, kind, ss, sr, H, W):
    torch, bf, fn, _ = env
    plan = bf.Plan(ss, sr, kind=kind)
    f, out, q, u = _inputs(torch, bf, plan, H, W, seed=11)
    g_ref, gs_ref = bf.backward(plan, f, out, q, u)  # caller-provided workspace
    torch.cuda.synchronize()
    # a call on other data, at least as large, fills the shared array with
    # other partials first; the next call must overwrite every one it reads
    f2, out2, q2, u2 = _inputs(torch, bf, plan, H + 64, W + 64, seed=21)
    g2_ref, gs2_ref = bf.backward(plan, f2, out2, q2, u2)
    for call in range(3):
        if call == 1:
            g2, gs2 = _noalloc(torch, fn, plan, f2, out2, q2, u2)
            assert torch.equal(g2, g2_ref)
            assert torch.equal(gs2, gs2_ref)
            assert float(gs2) != float(gs_ref)
            continue
        g, gs = _noalloc(torch, fn, plan, f, out, q, u)
        assert torch.equal(g, g_ref)
        assert torch.equal(gs, gs_ref)


def test_noalloc_image_gradient_alone(env):
    # grad_sigma_r = NULL: no partials, the no-dsigma_r kernel; same bits as
    # bf_backward without grad_sigma_r
    torch, bf, fn, _ = env
    plan = bf.Plan(3.0, 30.0, kind="gauss")
    f, out, q, u = _inputs(torch, bf, plan, 200, 333, seed=31)
    g_ref, _ = bf.backward(plan, f, out, q, u, need_sigma=False)
    torch.cuda.synchronize()
    for _ in range(2):
        g, _ = _noalloc(torch, fn, plan, f, out, q, u, need_sigma=False)
        assert torch.equal(g, g_ref)


def test_noalloc_without_sigma_has_no_size_limit(env):
    # ceil(8192/64) * ceil(4128/32) = 16512 blocks: more partials than the
    # fixed array holds, accepted when no dL/dsigma_r is asked for
    torch, bf, fn, _ = env
    plan = bf.Plan(2.0, 20.0, kind="box")
    H, W = 4128, 8192
    f, out, q, u = _inputs(torch, bf, plan, H, W, seed=41)
    g_ref, _ = bf.backward(plan, f, out, q, u, need_sigma=False)
    torch.cuda.synchronize()
    g, _ = _noalloc(torch, fn, plan, f, out, q, u, need_sigma=False)
    assert torch.equal(g, g_ref)
    assert bool(torch.isfinite(g).all())


def test_noalloc_rejects_images_beyond_the_fixed_array(env):
    torch, bf, fn, l = env
    l.bf_last_error.restype = ctypes.c_char_p
    plan = bf.Plan(3.0, 30.0)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the size check comes first
    # ceil(8192/64) * ceil(4128/32) = 128 * 129 = 16512 > 16384 partials
    st = fn(plan.handle, fake, fake, fake, fake, fake, fake, 4128, 8192, None)
    assert st == 2  # BF_EUNSUPPORTED
    assert b"16384" in l.bf_last_error()
