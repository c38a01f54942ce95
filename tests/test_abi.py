"""Host-side tests of libbf: it builds, loads, exports what include/bf.h
declares, and its plan (pure host code) follows the paper.  No GPU needed."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bf.h")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def bf():
    from paper_1105_4204_gb300 import build
    build.build()
    import paper_1105_4204_gb300 as pkg
    from paper_1105_4204_gb300 import _lib
    _lib.lib()
    return pkg


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(bf_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["bf_plan_create", "bf_plan_destroy", "bf_plan_info", "bf_forward",
                     "bf_backward", "bf_batch_forward", "bf_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(bf):
    from paper_1105_4204_gb300 import _lib
    l = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(l, n)]
    assert not missing, missing


def test_plan_degree_rule_matches_table1(bf):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_degree.txt"))
            if l.strip() and not l.startswith("#")]
    for sigma, _n0, n_rule in rows:
        assert bf.Plan(3.0, float(sigma), 255.0).N == int(n_rule)


def test_plan_table1_degree_rule_matches_the_oracle(bf, oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_degree.txt"))
            if l.strip() and not l.startswith("#")]
    for sigma, n0, _n_rule in rows:
        assert bf.Plan(3.0, float(sigma), 255.0, degree_rule="table1").N == int(n0)
    for T in [100.0, 255.0, 4095.0]:
        for sr in np.linspace(0.05, 1.0, 97) * T:
            p = bf.Plan(2.0, float(sr), T, kind="box", degree_rule="table1")
            assert p.N == oracle.n_table1(float(sr), T), (T, sr)
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    h = ctypes.c_void_p()
    bad = _lib.PlanOpts(0, 0, 0, 2)
    assert l.bf_plan_create(ctypes.byref(h), 2.0, 40.0, 255.0, 0, ctypes.byref(bad)) == 1
    assert b"degree_rule" in l.bf_last_error()
    a = np.array([1.0, 0.5])
    cos_opts = _lib.PlanOpts(0, 0, 0, 1)
    assert l.bf_plan_create_cosine(ctypes.byref(h), 2.0, 0.01,
                                   a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2, 0,
                                   ctypes.byref(cos_opts)) == 1


@pytest.mark.parametrize("sr,N", [(10.0, 264), (15.0, 118), (20.0, 66), (25.0, 43), (30.0, 30),
                                  (50.0, 11), (60.0, 8)])
def test_plan_degree_at_workload_sigmas(bf, sr, N):
    assert bf.Plan(3.0, sr).N == N


@pytest.mark.parametrize("sr", [10.0, 20.0, 25.0, 30.0, 50.0, 200.0])
def test_plan_terms_reproduce_raised_cosine(bf, sr):
    # Section 2.3: cos^N(x) = sum_n 2^-N C(N,n) exp(j (2n-N) x); the plan folds
    # conjugate pairs into real cosines.  Check against the direct power.
    p = bf.Plan(3.0, sr)
    a, w = p.terms()
    s = np.linspace(-255.0, 255.0, 2001)
    phi = np.sum(a[:, None] * np.cos(w[:, None] * s[None, :]), axis=0)
    ref = np.cos(s / (sr * math.sqrt(p.N))) ** p.N
    # terms dropped because their FP32 weight is 0 are below 1e-38 each
    np.testing.assert_allclose(phi, ref, atol=1e-12)
    # accumulation order: nondecreasing weight, constant term last for even N
    assert np.all(np.diff(a[:-1] if p.N % 2 == 0 else a) >= 0)
    if p.N % 2 == 0:
        assert w[-1] == 0.0
    assert p.n_terms == len(a)


def test_plan_terms_exact_binomials_small_n(bf):
    for N in range(1, 14):
        p = bf.Plan(3.0, 30.0, N=N)
        a, w = p.terms()
        k = 1.0 / (30.0 * math.sqrt(N))
        for n in range((N + 1) // 2):
            m = N - 2 * n
            idx = int(np.argmin(np.abs(w - m * k)))
            assert w[idx] == pytest.approx(m * k, rel=1e-15)
            assert a[idx] == pytest.approx(2 * math.comb(N, n) / 2.0 ** N, rel=1e-14)
        if N % 2 == 0:
            assert a[-1] == pytest.approx(math.comb(N, N // 2) / 2.0 ** N, rel=1e-14)


def test_plan_zero_weights_dropped_at_large_degree(bf):
    p = bf.Plan(6.0, 10.0)  # N = 264
    a, _ = p.terms()
    assert p.N == 264
    # 132 folded frequencies + constant; 50 of the 265 binomial weights (25
    # conjugate pairs) round to 0 in FP32
    assert p.n_terms == 133 - 25
    assert np.all(a.astype(np.float32) > 0)


def test_plan_spatial_weights(bf):
    g = bf.Plan(3.0, 30.0, kind="gauss")
    w = g.weights()
    assert g.radius == 9 and len(w) == 19
    k = np.arange(-9, 10)
    np.testing.assert_allclose(w / w[9], np.exp(-k * k / 18.0), rtol=1e-14)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    for ss, r in [(2.0, 2), (8.0, 8), (32.0, 32)]:
        b = bf.Plan(ss, 20.0, kind="box")
        assert b.radius == 3 * r
        ref = np.ones(1)
        for _ in range(3):
            ref = np.convolve(ref, np.ones(2 * r + 1) / (2 * r + 1))
        np.testing.assert_allclose(b.weights(), ref, atol=1e-15)
        assert b.achieved_sigma_s == pytest.approx(math.sqrt((2 * r + 1) ** 2 - 1) / 2, rel=1e-12)


def test_plan_rejects_bad_arguments(bf):
    from paper_1105_4204_gb300._lib import BfError
    for args in [(0.0, 30.0), (3.0, 0.0), (3.0, -1.0), (float("nan"), 30.0)]:
        with pytest.raises(BfError) as e:
            bf.Plan(*args)
        assert e.value.status == 1  # BF_EINVAL
    with pytest.raises(BfError) as e:
        bf.Plan(3.0, 2.0)  # N = 4121 > 1024
    assert e.value.status == 2  # BF_EUNSUPPORTED
    with pytest.raises(BfError) as e:
        bf.Plan(3.0, 20.0, kind="box", passes=2)
    assert e.value.status == 2


def test_forward_rejects_bad_arguments_without_touching_a_gpu(bf):
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    p = bf.Plan(3.0, 30.0)
    null = ctypes.c_void_p(0)
    st = l.bf_forward(p.handle, null, 0, null, 16, 16, 1, 16, null, null)
    assert st == 1 and b"NULL" in l.bf_last_error()
    fake = ctypes.c_void_p(0x1000)
    assert l.bf_forward(p.handle, fake, 0, fake, 0, 16, 1, 16, null, null) == 1
    assert l.bf_forward(p.handle, fake, 0, fake, 16, 16, 1, 8, null, null) == 1   # stride < W
    assert l.bf_forward(p.handle, fake, 0, fake, 16, 16, 5, 80, null, null) == 2  # C > 4
    assert l.bf_forward(p.handle, fake, 7, fake, 16, 16, 1, 16, null, null) == 1  # dtype
    assert l.bf_forward(None, fake, 0, fake, 16, 16, 1, 16, null, null) == 1


def test_set_shape_accepts_only_the_supports_shapes(bf):
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    box2, box8 = bf.Plan(2.0, 20.0, kind="box"), bf.Plan(8.0, 20.0, kind="box")
    assert l.bf_forward_set_shape(box2.handle, 64, 64, 1, 1) == 0   # 32 x 96
    assert l.bf_forward_set_shape(box2.handle, 64, 64, 1, 2) == 1   # 64 x 64 needs r >= 3
    assert l.bf_forward_set_shape(box8.handle, 64, 64, 1, 2) == 0
    assert l.bf_forward_set_shape(box8.handle, 64, 64, 1, 1) == 1   # 32 x 96 needs r <= 4
    assert l.bf_forward_set_shape(box8.handle, 64, 64, 1, 3) == 0   # 64 x 64, 32-px segments
    assert l.bf_forward_set_shape(box2.handle, 64, 64, 1, 3) == 1   # needs r >= 7
    assert l.bf_forward_set_shape(box8.handle, 64, 64, 1, 7) == 1
    assert l.bf_forward_set_shape(box8.handle, 0, 64, 1, 0) == 1
    big = bf.Plan(32.0, 20.0, kind="box")                          # streaming kernels
    assert l.bf_forward_set_shape(big.handle, 64, 64, 1, 0) == 1
    assert b"streaming" in l.bf_last_error()


def test_set_shape_term_split(bf):
    # configuration = shape | split << 8; split a power of two up to 8 and no
    # more groups than terms
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    g = bf.Plan(3.0, 30.0, kind="gauss")                           # 16 terms
    for split in (0, 1, 2, 4, 8, 16):
        assert l.bf_forward_set_shape(g.handle, 64, 64, 1, split << 8) == 0
    for split in (3, 32):
        assert l.bf_forward_set_shape(g.handle, 64, 64, 1, split << 8) == 1
        assert b"split" in l.bf_last_error()
    one = bf.Plan(3.0, 200.0, kind="gauss")                        # N = 1: one term
    assert one.n_terms == 1
    assert l.bf_forward_set_shape(one.handle, 64, 64, 1, 2 << 8) == 1
    assert l.bf_forward_set_shape(g.handle, 64, 64, 1, (2 << 8) | 7) == 1


def test_cosine_plan_terms_reproduce_the_polynomial(bf):
    # Section 2.2: phi(s) = sum_n a_n cos(n gamma s); the plan's folded term table must give
    # the same function (terms of zero FP32 weight dropped, constant last)
    gamma = math.pi / 510
    coefs = [1.0, 0.8, 0.0, 0.3, 1e-50, 0.1]
    p = bf.Plan.cosine(3.0, gamma, coefs, kind="gauss")
    assert p.N == 3 + 2 and p.n_terms == 4 and p.radius == 9
    a, w = p.terms()
    assert w[-1] == 0.0 and a[-1] == 1.0
    assert list(np.abs(a[:-1])) == sorted(np.abs(a[:-1]))
    s = np.linspace(-255, 255, 101)
    got = sum(ak * np.cos(wk * s) for ak, wk in zip(a, w))
    ref = sum(c * np.cos(n * gamma * s) for n, c in enumerate(coefs) if n != 4)
    np.testing.assert_allclose(got, ref, atol=1e-15)
    box = bf.Plan.cosine(8.0, gamma, coefs, kind="box")
    assert box.radius == 24


def test_cosine_plan_rejects_bad_arguments(bf):
    from paper_1105_4204_gb300._lib import BfError
    gamma = math.pi / 510
    for args in [(0.0, gamma, [1.0]), (3.0, 0.0, [1.0]), (3.0, -gamma, [1.0]),
                 (3.0, gamma, [0.0, 0.0]), (3.0, gamma, [1.0, float("nan")]),
                 (3.0, gamma, [])]:
        with pytest.raises(BfError) as e:
            bf.Plan.cosine(*args)
        assert e.value.status == 1  # BF_EINVAL
    with pytest.raises(BfError) as e:
        bf.Plan.cosine(3.0, gamma, np.ones(1026))
    assert e.value.status == 2  # BF_EUNSUPPORTED


def test_cosine_plan_backward_has_no_sigma_r(bf):
    # dL/dsigma_r is refused before any launch: a cosine-polynomial plan has no sigma_r
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    p = bf.Plan.cosine(2.0, math.pi / 510, [1.0, 0.5])
    fake = ctypes.c_void_p(0x1000)
    st = l.bf_backward(p.handle, fake, fake, fake, fake, fake, fake, 16, 16, fake, 1 << 20, None)
    assert st == 1 and b"sigma_r" in l.bf_last_error()


def test_size_limits_are_checked_on_the_host(bf):
    # 2^29 pixels is the largest image; one more pixel is refused before any launch
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    p = bf.Plan(2.0, 20.0, kind="box")
    fake = ctypes.c_void_p(0x1000)
    null = ctypes.c_void_p(0)
    H, W = 16384, 32768 + 1
    assert l.bf_forward(p.handle, fake, 0, fake, H, W, 1, W, null, null) == 2
    assert b"too large" in l.bf_last_error()
    assert l.bf_backward(p.handle, fake, fake, fake, fake, fake, null, H, W, null, 0, null) == 2


def test_tall_images_are_refused_on_the_host(bf):
    # 2^22 x 128 is within the pixel limit but has more 32-row tiles than a
    # grid's y dimension holds: refused with a message, before any launch
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    l.bf_backward_noalloc.restype = ctypes.c_int
    l.bf_backward_noalloc.argtypes = [ctypes.c_void_p] * 7 + [ctypes.c_int, ctypes.c_int,
                                                              ctypes.c_void_p]
    fake = ctypes.c_void_p(0x1000)
    null = ctypes.c_void_p(0)
    H, W = 1 << 22, 128
    for kind, ss in (("gauss", 3.0), ("box", 2.0)):
        p = bf.Plan(ss, 20.0, kind=kind)
        assert l.bf_forward(p.handle, fake, 0, fake, H, W, 1, W, null, null) == 2
        assert b"taller than" in l.bf_last_error()
        assert l.bf_backward(p.handle, fake, fake, fake, fake, fake, null, H, W, null, 0,
                             null) == 2
        assert b"taller than" in l.bf_last_error()
        assert l.bf_backward_stack(p.handle, fake, fake, fake, fake, fake, null, H, W, 1, null,
                                   0, null) == 2
        assert b"taller than" in l.bf_last_error()
        assert l.bf_backward_noalloc(p.handle, fake, fake, fake, fake, fake, null, H, W,
                                     null) == 2
        assert b"taller than" in l.bf_last_error()
    # the tallest accepted height is stated in the message
    assert str(65535 * 32).encode() in l.bf_last_error()


def test_backward_supports_on_the_host(bf):
    # the box with 8 < r <= 64 (the largest box a plan takes) and the
    # recursive Gaussian have adjoints through device scratch, which the
    # no-alloc entry point refuses before any pointer is read
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    l.bf_backward_noalloc.restype = ctypes.c_int
    l.bf_backward_noalloc.argtypes = [ctypes.c_void_p] * 7 + [ctypes.c_int, ctypes.c_int,
                                                              ctypes.c_void_p]
    fake = ctypes.c_void_p(0x1000)
    null = ctypes.c_void_p(0)
    big = bf.Plan(12.0, 20.0, kind="box")
    assert big.radius // 3 == 12
    assert l.bf_backward_noalloc(big.handle, fake, fake, fake, fake, fake, null, 64, 64,
                                 null) == 2
    assert b"scratch" in l.bf_last_error()
    with pytest.raises(Exception):  # no plan beyond the largest supported box
        bf.Plan(65.0, 20.0, kind="box", radius=65)
    rec = bf.Plan(10.0, 20.0, kind="recursive")
    assert l.bf_backward_noalloc(rec.handle, fake, fake, fake, fake, fake, null, 64, 64,
                                 null) == 2
    assert b"recursive" in l.bf_last_error()


def test_recursive_gaussian_plan(bf, oracle):
    # radius reports the extension P = ceil(6 sigma_s); achieved sigma is the cascade's
    # (closed form from the coefficients), equal to the oracle's measured impulse response
    for ss in (0.5, 2.4, 2.5, 10.0, 100.0):
        p = bf.Plan(ss, 30.0, kind="recursive")
        assert p.radius == math.ceil(6 * ss) and p.N == 30
        n = int(40 * ss) + 81
        x = np.zeros((1, n))
        x[0, n // 2] = 1.0
        y = oracle.rg_filter(x, ss)[0]
        k = np.arange(n) - n // 2
        assert p.achieved_sigma_s == pytest.approx(math.sqrt((y * k * k).sum()), rel=1e-5)
    from paper_1105_4204_gb300._lib import BfError
    with pytest.raises(BfError) as e:
        bf.Plan(0.4, 30.0, kind="recursive")
    assert e.value.status == 2
    with pytest.raises(BfError) as e:
        bf.Plan(3.0, 30.0, kind="recursive", radius=5)
    assert e.value.status == 1


def test_fp32_pipe_rate_rejects_null_output_without_touching_a_gpu(bf):
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    assert l.bf_fp32_pipe_rate(0, None, None) == 1
    assert b"NULL" in l.bf_last_error()


def test_forward_host_rejects_bad_arguments_without_touching_a_gpu(bf):
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    p = bf.Plan(2.0, 20.0, kind="box")
    fake = ctypes.c_void_p(0x1000)
    null = ctypes.c_void_p(0)
    assert l.bf_forward_host(p.handle, fake, 0, null, fake, fake, 16, 16, 1, 16, null) == 1
    assert b"dev_in" in l.bf_last_error()
    assert l.bf_forward_host(p.handle, fake, 0, fake, fake, fake, 16, 16, 1, 8, null) == 1
    assert l.bf_forward_host(p.handle, fake, 0, fake, fake, fake, 16, 16, 5, 80, null) == 2
    # the overlapping form needs a copy stream other than the filter's
    l.bf_forward_host_overlap.restype = ctypes.c_int
    assert l.bf_forward_host_overlap(p.handle, fake, 0, fake, fake, fake, 16, 16, 1, 16, null,
                                     null) == 1
    assert b"copy_stream" in l.bf_last_error()


def test_space_variant_rejects_bad_arguments_without_touching_a_gpu(bf):
    from paper_1105_4204_gb300 import _lib
    l = _lib.lib()
    p = bf.Plan(2.0, 20.0)
    fake = ctypes.c_void_p(0x1000)
    null = ctypes.c_void_p(0)
    assert l.bf_forward_space_variant(p.handle, fake, 0, null, 4, fake, 16, 16, 16, null) == 1
    assert l.bf_forward_space_variant(p.handle, fake, 0, fake, 17, fake, 16, 16, 16, null) == 1
    assert b"r_max" in l.bf_last_error()
    assert l.bf_forward_space_variant(p.handle, fake, 0, fake, -1, fake, 16, 16, 16, null) == 1
    assert l.bf_forward_space_variant(p.handle, fake, 0, fake, 4, fake, 16, 16, 8, null) == 1
    assert l.bf_forward_space_variant(p.handle, fake, 0, fake, 4, fake, 16384, 32769, 32769,
                                      null) == 2
    # channels 1 .. 4 with rows of at least W C elements; spatial 0 or 1
    l.bf_forward_space_variant_ex.restype = ctypes.c_int
    assert l.bf_forward_space_variant_ex(p.handle, fake, 0, fake, 4, 0, fake, 16, 16, 5, 80,
                                         null) == 1
    assert l.bf_forward_space_variant_ex(p.handle, fake, 0, fake, 4, 0, fake, 16, 16, 3, 47,
                                         null) == 1
    assert b"W * C" in l.bf_last_error()
    assert l.bf_forward_space_variant_ex(p.handle, fake, 0, fake, 4, 2, fake, 16, 16, 1, 16,
                                         null) == 1
    # the hat takes half-widths up to 8
    assert l.bf_forward_space_variant_hat(p.handle, fake, 0, fake, 9, fake, 16, 16, 16, null) == 1
    assert b"[0, 8]" in l.bf_last_error()
    assert l.bf_forward_space_variant_hat(p.handle, fake, 0, null, 4, fake, 16, 16, 16, null) == 1
