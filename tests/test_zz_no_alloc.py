"""bf_backward_noalloc: the backward entry point for callers that cannot
allocate device memory (real-time loops, fixed memory pools, plug-in hosts
that own every allocation).  It must give what bf_backward gives with a
caller workspace, call after call, although every call reuses one fixed
device array for its partial sums.  This file is named to be collected last,
so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL = 1e-3


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


def _noalloc(torch, fn, plan, f, out, q, u):
    g = torch.empty_like(f)
    gs = torch.empty((), dtype=torch.float64, device=f.device)
    st = fn(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(u.data_ptr()),
            ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(gs.data_ptr()), f.shape[0], f.shape[1],
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return g, gs


@pytest.mark.parametrize("kind,ss,sr,H,W", [("gauss", 4.0, 25.0, 512, 512),
                                              ("box", 2.0, 20.0, 300, 170)])
def test_noalloc_matches_workspace_backward_twice(env, kind, ss, sr, H, W):
    torch, bf, fn, _ = env
    img = synth.rectangles(H, W, seed=11)
    u_np = synth.upstream((H, W), seed=12)
    f = torch.from_numpy(img).cuda()
    u = torch.from_numpy(u_np).cuda()
    plan = bf.Plan(ss, sr, kind=kind)
    out, q = bf.forward(plan, f, return_q=True)
    g_ref, gs_ref = bf.backward(plan, f, out, q, u)  # caller-provided workspace
    torch.cuda.synchronize()
    g_ref = g_ref.cpu().numpy()
    gs_ref = float(gs_ref)
    scale = np.abs(g_ref).max()
    for _ in range(2):  # the second call reuses the array the first one filled
        g, gs = _noalloc(torch, fn, plan, f, out, q, u)
        assert np.abs(g.cpu().numpy() - g_ref).max() <= REL * scale
        assert abs(float(gs) - gs_ref) <= REL * abs(gs_ref)


def test_noalloc_rejects_images_beyond_the_fixed_array(env):
    torch, bf, fn, l = env
    l.bf_last_error.restype = ctypes.c_char_p
    plan = bf.Plan(3.0, 30.0)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the size check comes first
    # ceil(8192/64) * ceil(4128/32) = 128 * 129 = 16512 > 16384 partials
    st = fn(plan.handle, fake, fake, fake, fake, fake, fake, 4128, 8192, None)
    assert st == 2  # BF_EUNSUPPORTED
    assert b"16384" in l.bf_last_error()
