"""The recursive Gaussian's line filter W and the steps its adjoint takes for
W^T (the recursions from zero starts, the steady-state starts' adjoints at the
line's ends, the extension folded onto the last sample), written out in FP64
numpy and checked against the transpose of the oracle's matrix of the line
filter: the derivation the GPU adjoint follows, pinned on the CPU."""
import numpy as np
import pytest


def _causal(x, B, a, w0=0.0):
    # w(k) = B x(k) + a1 w(k-1) + a2 w(k-2) + a3 w(k-3), w(-1..-3) = w0
    w = np.empty(len(x))
    h = [w0, w0, w0]
    for k, v in enumerate(x):
        w[k] = B * v + a[0] * h[0] + a[1] * h[1] + a[2] * h[2]
        h = [w[k], h[0], h[1]]
    return w


def _anticausal(x, B, a, y0=0.0):
    return _causal(x[::-1], B, a, y0)[::-1]


def _w_line(x, c, P):
    # the forward line: steady-state starts, P samples of the last one
    B, a = c[0], c[1:]
    ext = np.concatenate([x, np.full(P, x[-1])])
    w = _causal(ext, B, a, x[0])
    return _anticausal(w, B, a, w[-1])[:len(x)]


def _wt_line(g, c, P):
    # the adjoint's steps, in the order the GPU takes them
    B, a = c[0], c[1:]
    n = len(g)
    E = n + P
    ybar = np.concatenate([g, np.zeros(P)])
    z = _causal(ybar, B, a)                       # the anticausal pass's transpose
    zz = lambda k: z[k] if k >= 0 else 0.0
    wbar = z.copy()
    wbar[E - 1] += ((1 - B) * zz(E - 1) + (a[1] + a[2]) * zz(E - 2) + a[2] * zz(E - 3)) / B
    v = _anticausal(wbar, B, a)                   # the causal pass's transpose
    xbar = v[:n].copy()
    xbar[0] += ((1 - B) * v[0] + (a[1] + a[2]) * v[1] + a[2] * v[2]) / B
    xbar[n - 1] += v[n:].sum()
    return xbar


@pytest.mark.parametrize("sigma", [0.8, 3.0, 10.0])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 40])
def test_line_filter_and_its_transpose(oracle, sigma, n):
    c, P = oracle.rg_coefs(sigma)
    M = oracle.rg_matrix(n, sigma)
    rng = np.random.default_rng(n + int(10 * sigma))
    x = rng.uniform(0, 255, n)
    g = rng.standard_normal(n)
    # the restated forward line is the oracle's, and the adjoint's steps give
    # the matrix's transpose
    np.testing.assert_allclose(_w_line(x, c, P), M @ x, rtol=1e-10, atol=1e-9)
    scale = np.abs(M.T @ g).max()
    np.testing.assert_allclose(_wt_line(g, c, P), M.T @ g, rtol=0, atol=1e-9 * max(scale, 1.0))
    # the adjoint identity <W x, g> = <x, W^T g>
    assert float(_w_line(x, c, P) @ g) == pytest.approx(float(x @ _wt_line(g, c, P)),
                                                       rel=1e-10, abs=1e-9)
