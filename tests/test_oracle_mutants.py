"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of the oracle's C source (a dropped range factor, a wrong clamp
bound, a wrong frequency or sign, floor for ceil, an off-by-one box or hat, a
flipped gradient term, a wrong coefficient of the recursive filter), builds it with gcc on the CPU and checks that at least one of
the pin checks below fails on it -- while all of them pass on the oracle as
committed."""
import importlib.util
import math
import os
import subprocess

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "bf_oracle.c")
INIT = os.path.join(ROOT, "oracle", "__init__.py")
GOLDEN = os.path.join(HERE, "golden")

MUTANTS = {
    "dropped range factor in P": ("p += wt * ph * v;", "p += wt * v;"),
    "clamp bound W-2": ("int zj = or_clamp(j - b, 0, W - 1);\n            double wt = w1[a + R] * "
                        "w1[b + R];\n            double v = f[(size_t)zi * W + zj];\n"
                        "            double ph = or_phi(rg, v - fx);",
                        "int zj = or_clamp(j - b, 0, W - 2);\n            double wt = w1[a + R] * "
                        "w1[b + R];\n            double v = f[(size_t)zi * W + zj];\n"
                        "            double ph = or_phi(rg, v - fx);"),
    "doubled frequency in phi": ("return pow(cos(r->k * s), r->N);",
                                 "return pow(cos(2.0 * r->k * s), r->N);"),
    "sign of the range argument": ("double ph = or_phi(rg, v - fx);\n            p += wt * ph * v;",
                                   "double ph = or_phi(rg, v + fx);\n            p += wt * ph * v;"),
    "floor for ceil in the degree rule": ("double n = ceil(x * (1.0 - 1e-12));",
                                          "double n = floor(x * (1.0 - 1e-12));"),
    "flipped gradient term": ("g[(size_t)i * W + j] -= alpha * wt * dph * (v - o);",
                              "g[(size_t)i * W + j] += alpha * wt * dph * (v - o);"),
    "space-variant box one row short": ("for (int a = -r; a <= r; a++) {\n        int zi = "
                                        "or_clamp(i + a, 0, H - 1);",
                                        "for (int a = -r; a < r; a++) {\n        int zi = "
                                        "or_clamp(i + a, 0, H - 1);"),
    "box taps one short": ("for (int d = -r; d <= r; d++) tmp[k + d + R] += cnt[k + R];",
                           "for (int d = -r; d < r; d++) tmp[k + d + R] += cnt[k + R];"),
    "wrong scale in Algorithm 1": ("double sigma_r, double T, int N, double *out, double *q_out)\n"
                                   "{\n    size_t n = (size_t)H * W;\n"
                                   "    double gamma = OR_PI / (2.0 * T);\n"
                                   "    double rho = gamma * sigma_r;",
                                   "double sigma_r, double T, int N, double *out, double *q_out)\n"
                                   "{\n    size_t n = (size_t)H * W;\n"
                                   "    double gamma = OR_PI / (2.0 * T);\n"
                                   "    double rho = 1.05 * gamma * sigma_r;"),
    "cosine kernel frequency shifted": ("v += r->a[n] * cos((double)n * r->gamma * s);",
                                        "v += r->a[n] * cos((double)(n + 1) * r->gamma * s);"),
    "recursive design coefficient": ("double b2 = -(1.4281 * q * q + 1.26661 * q * q * q);",
                                     "double b2 = -(1.4281 * q * q + 1.26661 * q * q);"),
    "recursive design digits transposed": ("double b1 = 2.44413 * q",
                                           "double b1 = 2.44431 * q"),
    "recursive design digit of the small-sigma branch": (": 3.97156 - 4.14554 * sqrt",
                                                         ": 3.97156 - 4.14545 * sqrt"),
    "space-variant hat weight off by one": ("double wa = hat ? (double)(r + 1 - abs(a)) : 1.0;",
                                            "double wa = hat ? (double)(r + 2 - abs(a)) : 1.0;"),
    "matrix weights transposed": ("double weight = wv * Mh[(size_t)j * W + zj];",
                                  "double weight = wv * Mh[(size_t)zj * W + j];"),
    "matrix-form gradient term flipped": ("g[px] -= aw * dk * dv;", "g[px] += aw * dk * dv;"),
}


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _load(src_text, tag, tmp):
    c = os.path.join(tmp, "bf_oracle_%s.c" % tag)
    so = os.path.join(tmp, "liboracle_%s.so" % tag)
    with open(c, "w") as fh:
        fh.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", so, c,
                    "-lm"], check=True)
    spec = importlib.util.spec_from_file_location("oracle_%s" % tag, INIT)
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    m._SRC, m._LIB_PATH, m._lib = c, so, None
    return m


def _checks(o):
    """Pin checks; returns the names of those that fail."""
    failed = []
    c = math.cos(0.5)
    g = _golden("hand_examples.txt")
    w1 = o.spatial_w1("box", 1.0, radius=1, passes=1)
    out2 = o.bf_brute(np.array([[0.0, 100.0], [100.0, 0.0]]), sigma_r=200.0, w1=w1)
    if not np.allclose(out2, [[g["2d_00"], g["2d_01"]], [g["2d_10"], g["2d_11"]]], atol=1e-7) \
            or abs(g["2d_00"] - 400 * c / (5 + 4 * c)) > 5e-8:
        failed.append("hand examples")
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_degree.txt"))
            if l.strip() and not l.startswith("#")]
    if any(o.n_rule(float(s), 255.0) != int(n) for s, _n0, n in rows):
        failed.append("Table 1 degrees")
    box3 = np.convolve(np.convolve(np.ones(3), np.ones(3)), np.ones(3)) / 27.0
    if not np.allclose(o.spatial_w1("box", 1.0, radius=1, passes=3), box3, atol=1e-15):
        failed.append("box taps")
    f = synth.rectangles(11, 13, n_rect=4, noise=6.0, seed=2).astype(np.float64)
    wg = o.spatial_w1("gauss", 1.5)
    if not np.allclose(o.bf_trig(f, sigma_r=30.0, w1=wg), o.bf_brute(f, sigma_r=30.0, w1=wg),
                       rtol=0, atol=1e-8):
        failed.append("Algorithm 1 = brute force")
    u = np.random.default_rng(1).standard_normal(f.shape)
    gf, _ = o.bf_grad(f, u, sigma_s=1.5, sigma_r=30.0)
    idx = np.array([0, 20, 77, 11 * 13 - 1])
    fd = o.fd_grad_f(f, u, idx, sigma_s=1.5, sigma_r=30.0)
    if not np.allclose(gf.ravel()[idx], fd, rtol=1e-5, atol=1e-7):
        failed.append("gradient = differences")
    gs = _golden("space_variant_examples.txt")
    sv = o.bf_brute_sv(np.array([[0.0, 100.0, 50.0]]), [[2, 1, 0]], sigma_r=200.0)
    if not np.allclose(sv[0], [gs["sv1d_0"], gs["sv1d_1"], gs["sv1d_2"]], atol=1e-7):
        failed.append("space-variant examples")
    svh = o.bf_brute_sv(np.array([[0.0, 100.0, 50.0]]), [[2, 1, 0]], sigma_r=200.0,
                        spatial="hat")
    svh2 = o.bf_brute_sv(np.array([[0.0, 100.0], [100.0, 0.0]]), [[1, 0], [0, 1]],
                         sigma_r=200.0, spatial="hat")
    if not np.allclose(svh[0], [gs["svhat1d_0"], gs["svhat1d_1"], gs["svhat1d_2"]], atol=1e-7) \
            or not np.allclose(svh2, [[gs["svhat2d_00"], gs["svhat2d_01"]],
                                      [gs["svhat2d_10"], gs["svhat2d_11"]]], atol=1e-7):
        failed.append("space-variant hat examples")
    gc = _golden("cosine_kernel_examples.txt")
    outc = o.bf_brute_cos(np.array([[0.0, 100.0], [100.0, 0.0]]), math.pi / 200, [0.5, 0.5],
                          w1=w1)
    if not np.allclose(outc, [[gc["2d_00"], gc["2d_01"]], [gc["2d_10"], gc["2d_11"]]],
                       atol=1e-7) or abs(gc["2d_00"] - 200 / 7) > 5e-8:
        failed.append("cosine kernel examples")
    sigma, n = 3.0, 133
    x = np.zeros((1, n))
    x[0, n // 2] = 1.0
    y = o.rg_filter(x, sigma)[0]
    k = np.arange(n) - n // 2
    gauss = np.exp(-k * k / (2 * sigma * sigma))
    gauss /= gauss.sum()
    if abs(y.sum() - 1.0) > 1e-5 or np.abs(y - gauss).max() > 0.05 * gauss.max():
        failed.append("recursive Gaussian impulse response")
    for line in open(os.path.join(GOLDEN, "young_van_vliet_design.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        s, _q, b0, b1, b2, b3, B = [float(x) for x in line.split()]
        c, _ = o.rg_coefs(s)
        if not np.allclose(c, [B, b1 / b0, b2 / b0, b3 / b0], rtol=1e-9, atol=1e-15):
            failed.append("recursive Gaussian published design")
            break
    # the filter and gradient with explicit per-axis weight matrices: the
    # clamp-extended Gaussian's matrices give the tap-based results, and the
    # recursive filter's give Algorithm 1 with the recursion
    def clamp_matrix(nn, taps):
        R = (len(taps) - 1) // 2
        M = np.zeros((nn, nn))
        for a in range(nn):
            for d in range(-R, R + 1):
                M[a, min(max(a - d, 0), nn - 1)] += taps[d + R]
        return M
    fm = f[:9, :10]
    um = u[:9, :10]
    Mv, Mh = clamp_matrix(9, wg), clamp_matrix(10, wg)
    g_taps, s_taps = o.bf_grad(fm, um, sigma_s=1.5, sigma_r=30.0)
    g_mat, s_mat = o.bf_grad_mat(fm, um, Mv, Mh, sigma_r=30.0)
    if not np.allclose(g_mat, g_taps, rtol=0, atol=1e-10) or abs(s_mat - s_taps) > 1e-9 \
            or not np.allclose(o.bf_brute_mat(fm, Mv, Mh, sigma_r=30.0),
                               o.bf_brute(fm, sigma_r=30.0, w1=wg), rtol=0, atol=1e-9):
        failed.append("matrix form = taps")
    Rv, Rh = o.rg_matrix(9, 3.0), o.rg_matrix(10, 3.0)
    if not np.allclose(o.bf_brute_mat(fm, Rv, Rh, sigma_r=30.0),
                       o.bf_trig_rg(fm, sigma_s=3.0, sigma_r=30.0), rtol=0, atol=1e-8):
        failed.append("matrix form = Algorithm 1 with the recursive filter")
    return failed


def test_checks_pass_on_the_oracle(tmp_path):
    src = open(SRC).read()
    assert _checks(_load(src, "committed", str(tmp_path))) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_planted_mistake_fails_a_pin(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "the mutation site must be unique"
    mutant = _load(src.replace(old, new), "m%d" % sorted(MUTANTS).index(name), str(tmp_path))
    failed = _checks(mutant)
    print("%s: fails %s" % (name, failed))
    assert failed, name
