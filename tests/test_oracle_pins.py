"""Pins of the FP64 oracle to things other than itself.

Each test ties one part of the oracle to a value printed in the paper, a
closed form worked by hand from eq. (BF), a mathematical identity, an
invariant of the filter, or an independent library routine (scipy, numpy,
torch autograd).  Together they are chosen so that a dropped term, a wrong
sign, a wrong clamp index or a transposed operand in the oracle fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_image(H=23, W=19, seed=3):
    return synth.rectangles(H, W, n_rect=5, noise=6.0, seed=seed).astype(np.float64)


# ---------------------------------------------------------------- degree rule

def test_degree_rule_matches_table1(oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_degree.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 7
    for sigma, _n0, n_rule in rows:
        assert oracle.n_rule(float(sigma), 255.0) == int(n_rule), sigma


def test_table1_lookup_reproduces_the_printed_degrees(oracle):
    # Table 1's N_0 row at its own sigmas; the look-up reading in between
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_degree.txt"))
            if l.strip() and not l.startswith("#")]
    for sigma, n0, _n_rule in rows:
        assert oracle.n_table1(float(sigma), 255.0) == int(n0), sigma
    # between listed sigmas: the next smaller listed sigma's N_0, capped by the estimate
    assert oracle.n_table1(45.0) == 9 and oracle.n_table1(55.0) == 7
    assert oracle.n_table1(90.0) == 4 and oracle.n_table1(180.0) == 1
    grid = np.linspace(1.0, 400.0, 4000)
    ns = [oracle.n_table1(float(s)) for s in grid]
    assert all(a >= b for a, b in zip(ns, ns[1:]))            # non-increasing in sigma
    for s, n in zip(grid, ns):
        assert 1 <= n <= oracle.n_rule(float(s))
        if s < 40.0:
            assert n == oracle.n_rule(float(s))                # below the table: the estimate
    for T in [1.0, 100.0, 1000.0, 65535.0]:                   # sigma / T is what matters
        for s in [45.0, 52.0, 75.0, 130.0, 300.0]:
            assert oracle.n_table1(s * T / 255.0, T) == oracle.n_table1(s, 255.0)


def test_table1_degrees_keep_the_kernel_nearly_non_negative(oracle):
    # Section 2.5: below the estimate the phase passes pi / 2 and cos^N can dip
    # below 0; over the look-up's whole range the dip stays under 3.6e-3 (the
    # deepest at sigma = 60, N = 5: cos(1.9007)^5 = -3.566e-3), and it is absent
    # wherever the look-up returns the estimate
    s = np.linspace(-255.0, 255.0, 20001)
    worst = 0.0
    for sigma in np.linspace(30.0, 400.0, 741):
        N = oracle.n_table1(float(sigma))
        phi_min = (np.cos(s / (sigma * math.sqrt(N))) ** N).min()
        worst = min(worst, phi_min)
        if N == oracle.n_rule(float(sigma)):
            assert phi_min >= -1e-15, sigma
    assert -3.6e-3 <= worst < -3.5e-3


def test_degree_rule_keeps_phase_in_half_period(oracle):
    # Section 2.5: N must make the argument of cos stay in [-pi/2, pi/2] on
    # [-T, T], i.e. T / (sigma_r sqrt N) <= pi / 2.
    for sr in [5.0, 10.0, 15.0, 20.0, 25.0, 30.0, 47.3, 60.0, 100.0, 161.0]:
        N = oracle.n_rule(sr, 255.0)
        assert 255.0 / (sr * math.sqrt(N)) <= math.pi / 2 + 1e-12
        if N > 1:  # and N is the smallest such degree
            assert 255.0 / (sr * math.sqrt(N - 1)) > math.pi / 2


# ------------------------------------------------------------- spatial kernel

@pytest.mark.parametrize("r,passes", [(1, 1), (1, 3), (2, 3), (5, 3), (4, 2)])
def test_box_weights_are_repeated_box_convolution(oracle, r, passes):
    w = oracle.spatial_w1("box", 1.0, radius=r, passes=passes)
    ref = np.ones(1)
    for _ in range(passes):
        ref = np.convolve(ref, np.ones(2 * r + 1) / (2 * r + 1))
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-15)
    # variance of the sum of `passes` uniform integers on [-r, r]
    k = np.arange(-passes * r, passes * r + 1)
    var = float(np.sum(w * k * k))
    assert var == pytest.approx(passes * ((2 * r + 1) ** 2 - 1) / 12.0, rel=1e-12)


@pytest.mark.parametrize("sigma_s,expect_r", [(2.0, 2), (8.0, 8), (32.0, 32)])
def test_box_radius_from_sigma(oracle, sigma_s, expect_r):
    w = oracle.spatial_w1("box", sigma_s, passes=3)
    assert (len(w) - 1) // 2 == 3 * expect_r


def test_gauss_weights(oracle):
    for s, R in [(3.0, 9), (4.0, 12), (6.0, 18)]:
        w = oracle.spatial_w1("gauss", s)
        assert len(w) == 2 * R + 1
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        k = np.arange(-R, R + 1)
        np.testing.assert_allclose(w / w[R], np.exp(-k * k / (2 * s * s)), rtol=1e-14)


# --------------------------------------------------------- hand-worked examples

def _golden_hand():
    vals = {}
    for l in open(os.path.join(GOLDEN, "hand_examples.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            vals[k] = float(v)
    return vals


def test_hand_examples(oracle):
    g = _golden_hand()
    c = math.cos(0.5)
    # closed forms worked by hand from eq. (BF)
    assert g["1d_p0"] == pytest.approx(100 * c / (2 + c), abs=5e-8)
    assert g["2d_00"] == pytest.approx(400 * c / (5 + 4 * c), abs=5e-8)
    w1 = oracle.spatial_w1("box", 1.0, radius=1, passes=1)
    assert oracle.n_rule(200.0, 255.0) == 1
    out1 = oracle.bf_brute(np.array([[0.0, 100.0]]), sigma_r=200.0, w1=w1)
    np.testing.assert_allclose(out1[0], [100 * c / (2 + c), 200 / (2 + c)], atol=1e-12)
    np.testing.assert_allclose(out1[0], [g["1d_p0"], g["1d_p1"]], atol=1e-7)
    out2 = oracle.bf_brute(np.array([[0.0, 100.0], [100.0, 0.0]]), sigma_r=200.0, w1=w1)
    np.testing.assert_allclose(out2, [[g["2d_00"], g["2d_01"]], [g["2d_10"], g["2d_11"]]],
                               atol=1e-7)
    # the complex form of Algorithm 1 gives the same numbers
    out3 = oracle.bf_trig(np.array([[0.0, 100.0], [100.0, 0.0]]), sigma_r=200.0, w1=w1)
    np.testing.assert_allclose(out3, out2, atol=1e-10)


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("kind,ss", [("gauss", 2.0), ("box", 1.0)])
def test_constant_image_preserved(oracle, kind, ss):
    f = np.full((9, 13), 117.25)
    out = oracle.bf_brute(f, sigma_s=ss, sigma_r=20.0, kind=kind)
    np.testing.assert_allclose(out, 117.25, rtol=1e-13)


def test_shift_equivariance(oracle):
    f = _small_image()
    a = oracle.bf_brute(f, sigma_s=2.0, sigma_r=25.0)
    b = oracle.bf_brute(f + 31.5, sigma_s=2.0, sigma_r=25.0)
    np.testing.assert_allclose(b, a + 31.5, atol=1e-9)


def test_flip_and_transpose_equivariance(oracle):
    f = _small_image()
    kw = dict(sigma_s=1.5, sigma_r=30.0)
    a = oracle.bf_brute(f, **kw)
    np.testing.assert_allclose(oracle.bf_brute(f[::-1], **kw), a[::-1], atol=1e-10)
    np.testing.assert_allclose(oracle.bf_brute(f[:, ::-1], **kw), a[:, ::-1], atol=1e-10)
    np.testing.assert_allclose(oracle.bf_brute(f.T.copy(), **kw), a.T, atol=1e-10)


def test_output_inside_neighbourhood_range(oracle):
    f = _small_image()
    R = 3
    out = oracle.bf_brute(f, sigma_s=1.0, sigma_r=15.0)  # R = ceil(3 * 1) = 3
    H, W = f.shape
    for i in range(H):
        for j in range(W):
            nb = f[max(0, i - R):i + R + 1, max(0, j - R):j + R + 1]
            assert nb.min() - 1e-9 <= out[i, j] <= nb.max() + 1e-9


def test_linear_limit_is_clamped_convolution(oracle):
    # sigma_r -> infinity: phi -> 1 and eq. (BF) reduces to eq. (averaging).
    from scipy.ndimage import convolve1d
    f = _small_image()
    for kind, ss in [("gauss", 2.0), ("box", 1.0)]:
        w1 = oracle.spatial_w1(kind, ss)
        out = oracle.bf_brute(f, sigma_r=1e9, w1=w1)
        ref = convolve1d(convolve1d(f, w1, axis=0, mode="nearest"), w1, axis=1,
                         mode="nearest")
        np.testing.assert_allclose(out, ref, atol=1e-9)


# ------------------------------------------------ raised cosine and its expansion

@pytest.mark.parametrize("N", [1, 2, 3, 4, 11, 30, 66])
def test_raised_cosine_binomial_identity(oracle, N):
    # Section 2.3: cos^N(x) = sum_n 2^-N C(N,n) exp(j (2n-N) x), exact integers.
    sr = 20.0
    s = np.linspace(-255, 255, 1021)
    x = s / (sr * math.sqrt(N))
    expansion = sum(math.comb(N, n) * np.cos((2 * n - N) * x) for n in range(N + 1))
    expansion = expansion / 2.0 ** N
    np.testing.assert_allclose(oracle.phi(s, sr, N=N), expansion, atol=1e-13)


def test_raised_cosine_approaches_gaussian(oracle):
    # eq. (convergence1): cos^N(s / (sigma sqrt N)) -> exp(-s^2 / 2 sigma^2).
    s = np.linspace(-255, 255, 2041)
    sr = 40.0
    g = oracle.phi(s, sr, range_mode="gaussian")
    errs = [np.max(np.abs(oracle.phi(s, sr, N=N) - g)) for N in [17, 34, 68, 136, 272]]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 2e-3
    # and the filter output follows
    f = _small_image(17, 15)
    out_g = oracle.bf_brute(f, sigma_s=1.5, sigma_r=sr, range_mode="gaussian")
    diffs = [np.max(np.abs(oracle.bf_brute(f, sigma_s=1.5, sigma_r=sr, N=N) - out_g))
             for N in [17, 68, 272]]
    assert diffs[2] < diffs[0]


@pytest.mark.parametrize("kind,ss,sr,N", [
    ("gauss", 2.0, 30.0, None),   # N = 30 (even)
    ("gauss", 1.0, 50.0, None),   # N = 11 (odd)
    ("box", 1.0, 20.0, None),     # N = 66
    ("box", 2.0, 200.0, None),    # N = 1
    ("gauss", 1.0, 25.0, 2),      # N override
])
def test_algorithm1_complex_form_matches_definition(oracle, kind, ss, sr, N):
    # Section 2.2 says eq. (final-form) is exact for trigonometric kernels.
    f = _small_image(21, 18, seed=7)
    w1 = oracle.spatial_w1(kind, ss)
    a = oracle.bf_brute(f, sigma_r=sr, w1=w1, N=N)
    b, worst_imag = oracle.bf_trig(f, sigma_r=sr, w1=w1, N=N, return_imag=True)
    np.testing.assert_allclose(b, a, atol=1e-8)
    assert worst_imag < 1e-9


def test_brute_at_matches_full(oracle):
    f = _small_image()
    w1 = oracle.spatial_w1("box", 1.0)
    full, q = oracle.bf_brute(f, sigma_r=30.0, w1=w1, return_q=True)
    idx = synth.sample_indices(*f.shape, 20, seed=1)
    o, qq = oracle.bf_brute_at(f, idx, sigma_r=30.0, w1=w1, return_q=True)
    np.testing.assert_array_equal(o, full.ravel()[idx])
    np.testing.assert_array_equal(qq, q.ravel()[idx])


def test_multichannel_is_per_channel(oracle):
    img = synth.rect_disk_u8(14, 11, C=3, n_shapes=6, seed=2).astype(np.float64)
    out = oracle.bf_brute(img, sigma_s=1.0, sigma_r=30.0)
    for c in range(3):
        np.testing.assert_array_equal(out[:, :, c],
                                      oracle.bf_brute(img[:, :, c], sigma_s=1.0, sigma_r=30.0))


# ------------------------------------------------------------------- gradient

def test_gradient_matches_finite_differences(oracle):
    f = _small_image(16, 14, seed=11)
    u = synth.upstream(f.shape, seed=5).astype(np.float64)
    kw = dict(sigma_s=1.3, sigma_r=25.0)  # R = 4, N = 43
    g, gs = oracle.bf_grad(f, u, **kw)
    idx = np.arange(f.size)  # every pixel: all of them touch a border here
    fd = oracle.fd_grad_f(f, u, idx, h=1e-4, **kw)
    np.testing.assert_allclose(g.ravel(), fd, atol=1e-6 * np.abs(fd).max())
    fds = oracle.fd_grad_sigma_r(f, u, h=1e-4, **kw)
    assert gs == pytest.approx(fds, rel=1e-6)


def test_gradient_box_and_gaussian_range(oracle):
    f = _small_image(12, 15, seed=4)
    u = synth.upstream(f.shape, seed=8).astype(np.float64)
    for kw in [dict(kind="box", sigma_s=1.0, sigma_r=40.0),
               dict(kind="gauss", sigma_s=1.0, sigma_r=35.0, range_mode="gaussian")]:
        g, gs = oracle.bf_grad(f, u, **kw)
        idx = np.arange(f.size)
        fd = oracle.fd_grad_f(f, u, idx, h=1e-4, **kw)
        np.testing.assert_allclose(g.ravel(), fd, atol=1e-6 * np.abs(fd).max())
        assert gs == pytest.approx(oracle.fd_grad_sigma_r(f, u, h=1e-4, **kw), rel=1e-6)


def test_gradient_matches_torch_autograd(oracle):
    # An independent derivative: torch's reverse-mode autodiff of eq. (BF)
    # evaluated with gathers over the clamp-extended image.
    torch = pytest.importorskip("torch")
    f = _small_image(9, 8, seed=9)
    u = synth.upstream(f.shape, seed=1).astype(np.float64)
    sr, ss = 22.0, 0.9
    w1 = oracle.spatial_w1("gauss", ss)
    R = (len(w1) - 1) // 2
    N = oracle.n_rule(sr)
    H, W = f.shape
    ft = torch.tensor(f, dtype=torch.float64, requires_grad=True)
    srt = torch.tensor(sr, dtype=torch.float64, requires_grad=True)
    ii = torch.arange(H)[:, None, None, None]
    jj = torch.arange(W)[None, :, None, None]
    aa = torch.arange(-R, R + 1)[None, None, :, None]
    bb = torch.arange(-R, R + 1)[None, None, None, :]
    zi = (ii - aa).clamp(0, H - 1)
    zj = (jj - bb).clamp(0, W - 1)
    nb = ft[zi, zj]                                   # H x W x (2R+1) x (2R+1)
    wt = torch.tensor(np.outer(w1, w1))[None, None]
    ph = torch.cos((nb - ft[:, :, None, None]) / (srt * math.sqrt(N))) ** N
    out = (wt * ph * nb).sum((2, 3)) / (wt * ph).sum((2, 3))
    (out * torch.tensor(u)).sum().backward()
    g, gs = oracle.bf_grad(f, u, sigma_s=ss, sigma_r=sr, w1=w1)
    np.testing.assert_allclose(g, ft.grad.numpy(), atol=1e-11)
    assert gs == pytest.approx(float(srt.grad), rel=1e-10)


# ------------------------------------- general trigonometric range kernel (Section 2.2)

def _raised_cosine_as_cosine_polynomial(N, sr):
    # cos^N(k s) = 2^-N sum_n C(N, n) cos((N - 2n) k s), k = 1 / (sr sqrt N), written as
    # a[m] cos(m k s): a[0] = 2^-N C(N, N/2) (N even), a[m] = 2^(1-N) C(N, (N-m)/2), m ≡ N mod 2
    a = np.zeros(N + 1)
    for n in range(N + 1):
        a[abs(N - 2 * n)] += math.comb(N, n) / 2.0 ** N
    return 1.0 / (sr * math.sqrt(N)), a


def test_cosine_kernel_hand_examples(oracle):
    g = {}
    for l in open(os.path.join(os.path.dirname(__file__), "golden", "cosine_kernel_examples.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            g[k] = float(v)
    # closed forms worked by hand from eq. (BF) with phi(0) = 1, phi(100) = 1/2
    assert g["1d_p0"] == pytest.approx(50 / 2.5, abs=5e-8)
    assert g["2d_00"] == pytest.approx(200 / 7, abs=5e-8)
    w1 = oracle.spatial_w1("box", 1.0, radius=1, passes=1)
    gam, a = math.pi / 200, [0.5, 0.5]
    out1 = oracle.bf_brute_cos(np.array([[0.0, 100.0]]), gam, a, w1=w1)
    np.testing.assert_allclose(out1[0], [g["1d_p0"], g["1d_p1"]], atol=1e-7)
    out2 = oracle.bf_brute_cos(np.array([[0.0, 100.0], [100.0, 0.0]]), gam, a, w1=w1)
    np.testing.assert_allclose(out2, [[g["2d_00"], g["2d_01"]], [g["2d_10"], g["2d_11"]]],
                               atol=1e-7)


@pytest.mark.parametrize("N", [1, 4, 7, 30])
def test_cosine_kernel_reproduces_raised_cosine(oracle, N):
    # the raised cosine is one cosine polynomial: its binomial coefficients (exact integers)
    # fed to the general kernel give the power-form brute force
    sr = 1.001 * 2 * 255.0 / (math.pi * math.sqrt(N))
    gam, a = _raised_cosine_as_cosine_polynomial(N, sr)
    s = np.linspace(-255, 255, 511)
    np.testing.assert_allclose(oracle.phi_cos(s, gam, a), oracle.phi(s, sr, N=N), atol=1e-13)
    f = _small_image()
    w1 = oracle.spatial_w1("gauss", 1.5)
    np.testing.assert_allclose(oracle.bf_brute_cos(f, gam, a, w1=w1),
                               oracle.bf_brute(f, sigma_r=sr, N=N, w1=w1), atol=1e-9)


def test_constant_cosine_kernel_is_the_clamped_convolution(oracle):
    # phi = a0 (any a0 > 0): eq. (BF) reduces to eq. (averaging)
    from scipy.ndimage import convolve1d
    f = _small_image()
    for kind, ss in [("gauss", 2.0), ("box", 1.0)]:
        w1 = oracle.spatial_w1(kind, ss)
        ref = convolve1d(convolve1d(f, w1, axis=0, mode="nearest"), w1, axis=1, mode="nearest")
        np.testing.assert_allclose(oracle.bf_brute_cos(f, 0.01, [2.5], w1=w1), ref, atol=1e-9)


def test_cosine_kernel_gradient(oracle):
    # exact gradient against central differences, and against the raised-cosine gradient
    # when the coefficients are the raised cosine's
    f = _small_image()[:12, :14].copy()
    u = synth.upstream(f.shape, seed=5).astype(np.float64)
    w1 = oracle.spatial_w1("gauss", 1.0)
    gam, a = math.pi / 510, [1.0, 0.8, 0.5, 0.3, 0.1]
    g = oracle.bf_grad_cos(f, u, gam, a, w1=w1)
    idx = np.arange(0, f.size, 7)
    fd = oracle.fd_grad_f_cos(f, u, idx, gam, a, h=1e-4, w1=w1)
    np.testing.assert_allclose(g.ravel()[idx], fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max())
    N, sr = 6, 60.0
    gam2, a2 = _raised_cosine_as_cosine_polynomial(N, sr)
    g2 = oracle.bf_grad_cos(f, u, gam2, a2, w1=w1)
    g3, _ = oracle.bf_grad(f, u, sigma_r=sr, N=N, w1=w1)
    np.testing.assert_allclose(g2, g3, atol=1e-10 * np.abs(g3).max())


# ------------------------------------------------ recursive Gaussian (Section 3)

def _impulse_response(oracle, sigma, n=None):
    n = n or int(24 * sigma) + 61
    x = np.zeros((1, n))
    x[0, n // 2] = 1.0
    return oracle.rg_filter(x, sigma)[0], np.arange(n) - n // 2


@pytest.mark.parametrize("sigma,bound", [(0.5, 0.08), (1.0, 0.10), (3.0, 0.05), (10.0, 0.025),
                                         (50.0, 0.025)])
def test_recursive_gaussian_approximates_the_gaussian(oracle, sigma, bound):
    # unit mass, symmetric, and within a few percent of the sampled Gaussian of the same
    # sigma (the third-order recursion approximates it; its tails are heavier)
    y, k = _impulse_response(oracle, sigma)
    g = np.exp(-k * k / (2 * sigma * sigma))
    g /= g.sum()
    assert abs(y.sum() - 1.0) < 1e-5
    np.testing.assert_allclose(y, y[::-1], atol=1e-12)
    assert np.abs(y - g).max() <= bound * g.max()
    assert int(np.argmax(y)) == len(y) // 2


def _yvv_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "young_van_vliet_design.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


def test_recursive_gaussian_design_matches_the_published_coefficients(oracle):
    # the oracle's (B, b1/b0, b2/b0, b3/b0) at seven sigma on both branches of
    # the published q(sigma), against the design worked out from Young and van
    # Vliet's equations in tests/golden: one wrong digit of a published constant
    # moves some ratio by far more than 1e-9
    for s, q, b0, b1, b2, b3, B in _yvv_golden():
        c, P = oracle.rg_coefs(s)
        assert P == math.ceil(6 * s)
        for got, want in zip(c, (B, b1 / b0, b2 / b0, b3 / b0)):
            assert got == pytest.approx(want, rel=1e-9, abs=1e-15), (s, got, want)


def test_recursive_gaussian_variance_closed_form(oracle):
    # the cascade's variance from the cumulants of the causal recursion
    # (2 (S''/B + (S'/B)^2), S' = sum k a_k, S'' = sum k^2 a_k) equals the measured one
    for sigma in (0.7, 2.0, 6.0, 20.0):
        c, _ = oracle.rg_coefs(sigma)
        B, a = c[0], c[1:]
        kk = np.array([1.0, 2.0, 3.0])
        var = 2 * ((kk * kk * a).sum() / B + ((kk * a).sum() / B) ** 2)
        y, k = _impulse_response(oracle, sigma, int(40 * sigma) + 81)
        assert (y * k * k).sum() == pytest.approx(var, rel=1e-6)
        assert c.sum() == pytest.approx(1.0, abs=1e-12)


def test_recursive_gaussian_borders(oracle):
    # constant rows and columns stay constant (unit gain, steady-state starts); a signal
    # that is constant near the first sample is filtered there as if extended forever
    f = np.full((7, 40), 42.0)
    np.testing.assert_allclose(oracle.rg_filter(f, 3.0), 42.0, atol=1e-9)
    x = np.concatenate([np.full(60, 10.0), np.linspace(10, 200, 40)])[None, :]
    ext = np.concatenate([np.full(300, 10.0), x[0]])[None, :]
    np.testing.assert_allclose(oracle.rg_filter(x, 4.0)[0, :30], oracle.rg_filter(ext, 4.0)[0, 300:330],
                               atol=1e-9)


def test_algorithm1_with_the_recursive_filter(oracle):
    # sigma_r -> infinity: the bilateral filter is the spatial averaging itself; and in the
    # interior, Algorithm 1 with the recursive filter equals eq. (BF) with the recursive
    # filter's impulse response as w (a separable kernel there)
    f = synth.rectangles(70, 80, n_rect=6, noise=6.0, seed=2).astype(np.float64)
    np.testing.assert_allclose(oracle.bf_trig_rg(f, sigma_s=2.0, sigma_r=1e9, N=1),
                               oracle.rg_filter(f, 2.0), atol=1e-8)
    sigma = 1.5
    y, k = _impulse_response(oracle, sigma, 161)
    keep = np.abs(y) > 1e-13 * y.max()
    w1 = y[keep] / y[keep].sum()
    R = (len(w1) - 1) // 2
    assert R < 40
    f = synth.rectangles(120, 130, n_rect=8, noise=6.0, seed=4).astype(np.float64)
    out = oracle.bf_trig_rg(f, sigma_s=sigma, sigma_r=30.0)
    idx = [i * 130 + j for i in range(R, 120 - R, 3) for j in range(R, 130 - R, 3)]
    ref = oracle.bf_brute_at(f, idx, sigma_r=30.0, w1=w1)
    np.testing.assert_allclose(out.ravel()[idx], ref, atol=1e-6)


def test_recursive_filter_matrix_is_the_line_filter(oracle):
    # rg_matrix's columns are the line's unit responses: applying the matrix is the
    # filter (a 1-row image filters its row alone), rows sum to 1 (unit DC gain),
    # and the interior rows are shifts of one impulse response
    W, sigma = 37, 2.5
    M = oracle.rg_matrix(W, sigma)
    x = np.random.default_rng(3).uniform(0, 255, W)
    np.testing.assert_allclose(M @ x, oracle.rg_filter(x[None, :], sigma)[0], atol=1e-10)
    np.testing.assert_allclose(M.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(M[18, 18 - 5:18 + 6], M[19, 19 - 5:19 + 6], atol=1e-6)
    assert oracle.rg_matrix(1, sigma)[0, 0] == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("sigma_s", [0.8, 3.0, 7.0])
def test_recursive_filter_gradient_matches_finite_differences(oracle, sigma_s):
    # the exact gradient with the recursive filter (its matrices in the chain rule)
    # against central differences of Algorithm 1 with the recursion, at corner,
    # edge and interior pixels, and for sigma_r with N held fixed
    f = synth.rectangles(13, 17, n_rect=4, noise=8.0, seed=5).astype(np.float64)
    u = np.random.default_rng(6).standard_normal(f.shape)
    N = oracle.n_rule(25.0)
    g, gs = oracle.bf_grad_rg(f, u, sigma_s=sigma_s, sigma_r=25.0, N=N)
    h = 1e-4

    def L(ff, sr=25.0):
        return float((u * oracle.bf_trig_rg(ff, sigma_s=sigma_s, sigma_r=sr, N=N)).sum())
    for (i, j) in [(0, 0), (0, 16), (12, 0), (12, 16), (6, 8), (3, 0), (0, 9)]:
        fp, fm = f.copy(), f.copy()
        fp[i, j] += h
        fm[i, j] -= h
        fd = (L(fp) - L(fm)) / (2 * h)
        assert g[i, j] == pytest.approx(fd, rel=2e-5, abs=2e-6)
    fd_s = (L(f, 25.0 + h) - L(f, 25.0 - h)) / (2 * h)
    assert gs == pytest.approx(fd_s, rel=1e-6, abs=1e-7)


# ------------------------------------------------------ space-variant (Section 4)

def _golden_sv():
    vals = {}
    for l in open(os.path.join(GOLDEN, "space_variant_examples.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            vals[k] = float(v)
    return vals


def test_space_variant_hand_examples(oracle):
    g = _golden_sv()
    c, c2 = math.cos(0.5), math.cos(0.25)
    # closed forms worked by hand from eq. (BF) over each pixel's own box
    assert g["sv1d_0"] == pytest.approx((500 * c + 250 * c2) / (15 + 5 * c + 5 * c2), abs=5e-8)
    assert g["sv1d_1"] == pytest.approx((300 + 150 * c2) / (3 * c + 3 + 3 * c2), abs=5e-8)
    out = oracle.bf_brute_sv(np.array([[0.0, 100.0], [100.0, 0.0]]), [[1, 0], [0, 1]],
                             sigma_r=200.0)
    np.testing.assert_allclose(out, [[g["sv2d_00"], g["sv2d_01"]], [g["sv2d_10"], g["sv2d_11"]]],
                               atol=1e-7)
    out1 = oracle.bf_brute_sv(np.array([[0.0, 100.0, 50.0]]), [[2, 1, 0]], sigma_r=200.0)
    np.testing.assert_allclose(out1[0], [g["sv1d_0"], g["sv1d_1"], g["sv1d_2"]], atol=1e-7)


def test_space_variant_constant_radius_is_the_one_box_filter(oracle):
    # r(x) = r0 everywhere is the plain filter with one box of half-width r0
    f = _small_image(17, 23, seed=8)
    for r0 in (0, 1, 3):
        w1 = oracle.spatial_w1("box", 1.0, radius=max(r0, 1), passes=1) if r0 else np.ones(1)
        ref = oracle.bf_brute(f, sigma_r=25.0, w1=w1)
        out = oracle.bf_brute_sv(f, np.full(f.shape, r0), sigma_r=25.0)
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-10)
    np.testing.assert_array_equal(oracle.bf_brute_sv(f, np.zeros(f.shape, int), sigma_r=25.0), f)


def test_space_variant_wide_range_kernel_is_the_box_mean(oracle):
    # sigma_r -> infinity: phi -> 1, so out(x) is the mean of the clamp-extended image
    # over x's box; the means here come from a summed-area table of the padded image
    f = _small_image(19, 26, seed=9)
    rng = np.random.default_rng(4)
    rad = rng.integers(0, 5, size=f.shape)
    out = oracle.bf_brute_sv(f, rad, sigma_r=1e9)
    R = 4
    fp = np.pad(f, R, mode="edge")
    sat = np.zeros((fp.shape[0] + 1, fp.shape[1] + 1))
    sat[1:, 1:] = fp.cumsum(0).cumsum(1)
    H, W = f.shape
    ref = np.empty_like(f)
    for i in range(H):
        for j in range(W):
            r = rad[i, j]
            a0, a1, b0, b1 = i + R - r, i + R + r + 1, j + R - r, j + R + r + 1
            ref[i, j] = (sat[a1, b1] - sat[a0, b1] - sat[a1, b0] + sat[a0, b0]) / (2 * r + 1) ** 2
    np.testing.assert_allclose(out, ref, rtol=1e-9)


def test_space_variant_matches_a_python_loop(oracle):
    # tiny mixed-radius case against plain Python loops of eq. (BF)
    f = _small_image(6, 7, seed=10)
    rad = np.random.default_rng(5).integers(0, 4, size=f.shape)
    sr, N = 30.0, oracle.n_rule(30.0)
    k = 1.0 / (sr * math.sqrt(N))
    H, W = f.shape
    out = oracle.bf_brute_sv(f, rad, sigma_r=sr)
    for i in range(H):
        for j in range(W):
            r = int(rad[i, j])
            p = q = 0.0
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    v = f[min(max(i + a, 0), H - 1), min(max(j + b, 0), W - 1)]
                    ph = math.cos(k * (v - f[i, j])) ** N
                    p += ph * v
                    q += ph
            assert out[i, j] == pytest.approx(p / q, rel=1e-12)
    # the sampled form gives the same values at the same pixels
    idx = np.array([0, 5, 17, H * W - 1])
    np.testing.assert_array_equal(oracle.bf_brute_sv_at(f, rad, idx, int(rad.max()), sigma_r=sr),
                                  out.ravel()[idx])
    # radii are clamped into [0, r_max]
    np.testing.assert_array_equal(oracle.bf_brute_sv(f, rad + 10, sigma_r=sr, r_max=3),
                                  oracle.bf_brute_sv(f, np.full(f.shape, 3), sigma_r=sr))


def test_space_variant_hat_hand_examples(oracle):
    # Section 4's hat: closed forms worked by hand from eq. (BF) with the hat's
    # weights (r + 1 - |a|)(r + 1 - |b|)
    g = _golden_sv()
    c, c2 = math.cos(0.5), math.cos(0.25)
    assert g["svhat2d_00"] == pytest.approx(600 * c / (10 + 6 * c), abs=5e-8)
    assert g["svhat1d_0"] == pytest.approx((1800 * c + 450 * c2) / (54 + 18 * c + 9 * c2),
                                           abs=5e-8)
    assert g["svhat1d_1"] == pytest.approx((800 + 200 * c2) / (4 * c + 8 + 4 * c2), abs=5e-8)
    out = oracle.bf_brute_sv(np.array([[0.0, 100.0], [100.0, 0.0]]), [[1, 0], [0, 1]],
                             sigma_r=200.0, spatial="hat")
    np.testing.assert_allclose(out, [[g["svhat2d_00"], g["svhat2d_01"]],
                                     [g["svhat2d_10"], g["svhat2d_11"]]], atol=1e-7)
    out1 = oracle.bf_brute_sv(np.array([[0.0, 100.0, 50.0]]), [[2, 1, 0]], sigma_r=200.0,
                              spatial="hat")
    np.testing.assert_allclose(out1[0], [g["svhat1d_0"], g["svhat1d_1"], g["svhat1d_2"]],
                               atol=1e-7)


def test_space_variant_hat_constant_radius_is_the_triangle_filter(oracle):
    # r(x) = r0 everywhere is the plain filter with separable triangle taps
    # (r0 + 1 - |k|) / (r0 + 1)^2, the 1-D hat
    f = _small_image(17, 23, seed=18)
    for r0 in (1, 2, 5):
        k = np.arange(-r0, r0 + 1)
        w1 = (r0 + 1 - np.abs(k)) / float((r0 + 1) ** 2)
        ref = oracle.bf_brute(f, sigma_r=25.0, w1=w1)
        out = oracle.bf_brute_sv(f, np.full(f.shape, r0), sigma_r=25.0, spatial="hat")
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-10)
    # r = 0: a one-pixel hat returns the image
    np.testing.assert_array_equal(
        oracle.bf_brute_sv(f, np.zeros(f.shape, int), sigma_r=25.0, spatial="hat"), f)


def test_space_variant_hat_wide_range_kernel_is_the_hat_mean(oracle):
    # sigma_r -> infinity: out(x) is the hat-weighted mean of the clamp-extended
    # image around x, here summed with numpy from the padded image
    f = _small_image(15, 21, seed=19)
    rad = np.random.default_rng(14).integers(0, 5, size=f.shape)
    out = oracle.bf_brute_sv(f, rad, sigma_r=1e9, spatial="hat")
    R = 4
    fp = np.pad(f, R, mode="edge")
    H, W = f.shape
    ref = np.empty_like(f)
    for i in range(H):
        for j in range(W):
            r = rad[i, j]
            t = r + 1 - np.abs(np.arange(-r, r + 1))
            w = np.outer(t, t).astype(np.float64)
            win = fp[i + R - r:i + R + r + 1, j + R - r:j + R + r + 1]
            ref[i, j] = (w * win).sum() / w.sum()
    np.testing.assert_allclose(out, ref, rtol=1e-9)
    idx = np.array([0, 7, 100, H * W - 1])
    np.testing.assert_array_equal(
        oracle.bf_brute_sv_at(f, rad, idx, 4, sigma_r=1e9, spatial="hat"), out.ravel()[idx])


def test_space_variant_cosine_kernel_agrees_with_the_power_form(oracle):
    # the raised cosine written as its cosine polynomial gives the power-form
    # space-variant filter; a constant radius gives the one-box cosine filter
    f = _small_image(14, 17, seed=12)
    rad = np.random.default_rng(6).integers(0, 4, size=f.shape)
    sr = 40.0
    N = oracle.n_rule(sr)
    gamma = 1.0 / (sr * math.sqrt(N))
    coefs = np.zeros(N + 1)
    for n in range(N + 1):  # cos^N x = 2^-N sum_n C(N,n) cos((2n - N) x)
        k = abs(2 * n - N)
        coefs[k] += math.comb(N, n) / 2.0 ** N
    np.testing.assert_allclose(oracle.bf_brute_sv_cos(f, rad, gamma, coefs),
                               oracle.bf_brute_sv(f, rad, sigma_r=sr), rtol=1e-11)
    w1 = oracle.spatial_w1("box", 1.0, radius=2, passes=1)
    np.testing.assert_allclose(oracle.bf_brute_sv_cos(f, np.full(f.shape, 2), gamma, coefs),
                               oracle.bf_brute_cos(f, gamma, coefs, w1=w1), rtol=1e-11)


def test_sampled_and_scalar_forms_agree_with_the_whole_image(oracle):
    # the sampled cosine-kernel brute force and the scalar loss are the whole-image
    # filter read at pixels / summed against u
    f = _small_image(12, 15, seed=15)
    gamma = math.pi / 510
    coefs = np.array([1.0, 0.8, 0.5, 0.3, 0.1])
    whole = oracle.bf_brute_cos(f, gamma, coefs, sigma_s=1.5)
    idx = np.array([0, 7, 33, 12 * 15 - 1])
    np.testing.assert_array_equal(oracle.bf_brute_cos_at(f, idx, gamma, coefs, sigma_s=1.5),
                                  whole.ravel()[idx])
    u = np.random.default_rng(3).standard_normal(f.shape)
    out = oracle.bf_brute(f, sigma_s=2.0, sigma_r=25.0, kind="gauss")
    assert oracle.loss(f, u, sigma_s=2.0, sigma_r=25.0) == pytest.approx(float((u * out).sum()),
                                                                        rel=1e-12)
