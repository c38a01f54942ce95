"""FP64 CPU oracle for the trigonometric O(1) bilateral filter.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_1105_4204_gb300``) and neither imports the
other; they meet only through the seeded generators in ``synth``.

The arithmetic lives in ``bf_oracle.c`` (plain C, double precision, OpenMP):

* ``bf_brute`` / ``bf_brute_at`` -- eq. (BF) and eq. (normalization) summed
  directly over the support, clamp-to-edge extension, range kernel
  ``cos(s/(sigma_r sqrt N))^N`` evaluated as a power (Algorithm 1 step 3 with
  ``rho = gamma sigma_r``), or the Gaussian ``exp(-s^2/2 sigma_r^2)`` of
  eq. (convergence1).
* ``bf_trig`` -- Algorithm 1 steps 3-5 with the N+1 complex auxiliary images
  of the raised-cosine expansion (Section 2.3) and eq. (final-form).
* ``bf_grad`` -- exact gradient of ``sum(u * out)`` w.r.t. the image and
  sigma_r (N fixed), by the chain rule on eq. (BF).
* ``fd_grad_f`` / ``loss`` -- central finite differences of the brute force.
* ``rg_filter`` / ``bf_trig_rg`` -- the recursive O(1) Gaussian of Young and
  van Vliet (the paper's spatial filter in Section 3) and Algorithm 1 with it.
* ``bf_brute_cos`` / ``bf_brute_cos_at`` / ``bf_grad_cos`` / ``fd_grad_f_cos``
  / ``phi_cos`` -- the same for a general trigonometric range kernel of
  Section 2.2, ``phi(s) = a_0 + a_1 cos(gamma s) + ... + a_N cos(N gamma s)``,
  evaluated term by term.
* ``bf_brute_sv`` -- the space-variant extension of Section 4: each pixel's
  own box of half-width r(x), eq. (BF) summed directly over it.

This module only marshals numpy arrays into that library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAUSS = 0
BOX = 1
RAISED_COSINE = 0
GAUSSIAN_RANGE = 1

_dp = ctypes.POINTER(ctypes.c_double)
_llp = ctypes.POINTER(ctypes.c_longlong)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile ``bf_oracle.c`` into ``liboracle.so`` beside it (gcc, OpenMP)."""
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.or_n_rule.restype = ctypes.c_int
        lib.or_n_rule.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_spatial_w1.restype = ctypes.c_int
        lib.or_spatial_w1.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, _dp, ctypes.c_int]
        lib.or_bf_brute.restype = None
        lib.or_bf_brute.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]
        lib.or_bf_brute_at.restype = None
        lib.or_bf_brute_at.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int, _llp,
                                       ctypes.c_longlong, _dp, _dp]
        lib.or_bf_trig.restype = ctypes.c_double
        lib.or_bf_trig.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp]
        lib.or_bf_grad.restype = None
        lib.or_bf_grad.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]
        lib.or_bf_fd_grad_f.restype = None
        lib.or_bf_fd_grad_f.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, _llp, ctypes.c_longlong,
                                        ctypes.c_double, _dp]
        lib.or_bf_loss.restype = ctypes.c_double
        lib.or_bf_loss.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_int]
        lib.or_bf_brute_cos.restype = None
        lib.or_bf_brute_cos.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                        ctypes.c_double, _dp, ctypes.c_int, _dp, _dp]
        lib.or_bf_brute_cos_at.restype = None
        lib.or_bf_brute_cos_at.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                           ctypes.c_double, _dp, ctypes.c_int, _llp,
                                           ctypes.c_longlong, _dp, _dp]
        lib.or_bf_grad_cos.restype = None
        lib.or_bf_grad_cos.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                       ctypes.c_double, _dp, ctypes.c_int, _dp]
        lib.or_bf_fd_grad_f_cos.restype = None
        lib.or_bf_fd_grad_f_cos.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp,
                                            ctypes.c_int, ctypes.c_double, _dp, ctypes.c_int,
                                            _llp, ctypes.c_longlong, ctypes.c_double, _dp]
        lib.or_phi_cos_table.restype = None
        lib.or_phi_cos_table.argtypes = [ctypes.c_double, _dp, ctypes.c_int, _dp,
                                         ctypes.c_longlong, _dp]
        lib.or_rg_coefs.restype = ctypes.c_int
        lib.or_rg_coefs.argtypes = [ctypes.c_double, _dp]
        lib.or_rg_filter.restype = None
        lib.or_rg_filter.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
        lib.or_rg_matrix.restype = None
        lib.or_rg_matrix.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        lib.or_bf_brute_mat.restype = None
        lib.or_bf_brute_mat.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, _dp]
        lib.or_bf_grad_mat.restype = None
        lib.or_bf_grad_mat.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]
        lib.or_bf_trig_rg.restype = ctypes.c_double
        lib.or_bf_trig_rg.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp]
        lib.or_bf_brute_sv.restype = None
        lib.or_bf_brute_sv.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp]
        lib.or_bf_brute_sv_cos.restype = None
        lib.or_bf_brute_sv_cos.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int,
                                           ctypes.c_double, _dp, ctypes.c_int, _dp]
        lib.or_bf_brute_sv_at.restype = None
        lib.or_bf_brute_sv_at.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, _llp,
                                          ctypes.c_longlong, _dp]
        lib.or_bf_brute_sv_shape.restype = None
        lib.or_bf_brute_sv_shape.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, _dp, _dp]
        lib.or_bf_brute_sv_shape_at.restype = None
        lib.or_bf_brute_sv_shape_at.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _ip,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_int, _llp,
                                                ctypes.c_longlong, _dp]
        lib.or_phi_table.restype = None
        lib.or_phi_table.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp,
                                     ctypes.c_longlong, _dp]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS or all cores)."""
    return int(_load().or_num_threads())


def n_rule(sigma_r: float, T: float = 255.0) -> int:
    """Degree N = max(1, ceil((gamma sigma_r)^-2)), gamma = pi/(2T) (Alg. 1, Table 1)."""
    return int(_load().or_n_rule(float(sigma_r), float(T)))


# Table 1 (Section 2.5): empirical minimum degrees N_0 of the raised cosine
# for T = 255, listed for these sigma values.
_TABLE1 = ((200.0, 1), (150.0, 2), (100.0, 3), (80.0, 4), (60.0, 5), (50.0, 7), (40.0, 9))


def n_table1(sigma_r: float, T: float = 255.0) -> int:
    """Degree by the look-up table Algorithm 1 step 2 allows: Table 1's N_0
    read at sigma' = 255 sigma_r / T (the same approximation problem after
    scaling s by 255 / T).  Between listed sigmas, the N_0 of the next smaller
    listed sigma; never above the estimate n_rule; below the smallest listed
    sigma the table says nothing and the estimate is used."""
    est = n_rule(sigma_r, T)
    sp = float(sigma_r) * 255.0 / float(T)
    listed = [n0 for sig, n0 in _TABLE1 if sig <= sp]
    if not listed:
        return est
    return min(listed[0], est)


def _kind(kind) -> int:
    if isinstance(kind, str):
        return {"gauss": GAUSS, "box": BOX}[kind]
    return int(kind)


def spatial_w1(kind, sigma_s: float, radius: int = 0, passes: int = 3) -> np.ndarray:
    """1-D spatial weights w1[-R..R] (unit sum); the 2-D kernel is w1 x w1."""
    cap = 1 << 16
    buf = np.zeros(cap, dtype=np.float64)
    R = _load().or_spatial_w1(_kind(kind), float(sigma_s), int(radius), int(passes),
                              _ptr(buf), cap)
    if R < 0:
        raise ValueError("spatial support too large")
    return buf[: 2 * R + 1].copy()


def _range_mode(mode) -> int:
    if isinstance(mode, str):
        return {"raised_cosine": RAISED_COSINE, "gaussian": GAUSSIAN_RANGE}[mode]
    return int(mode)


def _channels(f: np.ndarray):
    f = np.asarray(f)
    if f.ndim == 2:
        return [f], False
    if f.ndim == 3:
        return [f[:, :, c] for c in range(f.shape[2])], True
    raise ValueError("image must be H x W or H x W x C")


def _setup(sigma_s, sigma_r, T, kind, radius, passes, N, w1):
    if w1 is None:
        w1 = spatial_w1(kind, sigma_s, radius, passes)
    w1 = _f64(w1)
    R = (len(w1) - 1) // 2
    if N is None:
        N = n_rule(sigma_r, T)
    return w1, R, int(N)


def bf_brute(f, sigma_s=3.0, sigma_r=30.0, T=255.0, kind="gauss", radius=0, passes=3,
             range_mode="raised_cosine", N=None, w1=None, return_q=False):
    """Brute-force FP64 bilateral filter, eq. (BF); f is H x W or H x W x C
    (channels filtered independently)."""
    lib = _load()
    w1, R, N = _setup(sigma_s, sigma_r, T, kind, radius, passes, N, w1)
    chans, multi = _channels(f)
    outs, qs = [], []
    for ch in chans:
        x = _f64(ch)
        H, W = x.shape
        o = np.empty((H, W), dtype=np.float64)
        q = np.empty((H, W), dtype=np.float64)
        lib.or_bf_brute(_ptr(x), H, W, _ptr(w1), R, _range_mode(range_mode),
                        float(sigma_r), N, _ptr(o), _ptr(q))
        outs.append(o)
        qs.append(q)
    out = np.stack(outs, axis=2) if multi else outs[0]
    q = np.stack(qs, axis=2) if multi else qs[0]
    return (out, q) if return_q else out


def bf_brute_sv(f, radius, sigma_r=30.0, T=255.0, r_max=None, N=None,
                range_mode="raised_cosine", return_q=False, spatial="box"):
    """Space-variant brute force (Section 4): at each pixel a box (or, with
    spatial="hat", the separable hat, weight (r + 1 - |a|)(r + 1 - |b|) at
    offset (a, b)) of half-width radius[i, j] (clamped into [0, r_max]; r_max
    defaults to radius.max()), eq. (BF) summed directly over it; single-channel
    H x W."""
    lib = _load()
    if N is None:
        N = n_rule(sigma_r, T)
    x = _f64(f)
    H, W = x.shape
    rad = np.ascontiguousarray(np.asarray(radius, dtype=np.int32))
    if rad.shape != (H, W):
        raise ValueError("radius must be H x W")
    if r_max is None:
        r_max = int(rad.max()) if rad.size else 0
    o = np.empty((H, W), dtype=np.float64)
    q = np.empty((H, W), dtype=np.float64)
    if spatial == "box":
        lib.or_bf_brute_sv(_ptr(x), H, W, rad.ctypes.data_as(_ip), int(r_max),
                           _range_mode(range_mode), float(sigma_r), int(N), _ptr(o), _ptr(q))
    elif spatial == "hat":
        lib.or_bf_brute_sv_shape(_ptr(x), H, W, rad.ctypes.data_as(_ip), int(r_max), 1,
                                 _range_mode(range_mode), float(sigma_r), int(N), _ptr(o),
                                 _ptr(q))
    else:
        raise ValueError("spatial must be 'box' or 'hat'")
    return (o, q) if return_q else o


def bf_brute_sv_cos(f, radius, gamma, coefs, r_max=None):
    """Space-variant brute force with a general cosine kernel (Section 2.2),
    phi(s) = sum_n coefs[n] cos(n gamma s)."""
    lib = _load()
    x = _f64(f)
    H, W = x.shape
    rad = np.ascontiguousarray(np.asarray(radius, dtype=np.int32))
    a = np.ascontiguousarray(np.asarray(coefs, dtype=np.float64).ravel())
    if r_max is None:
        r_max = int(rad.max()) if rad.size else 0
    o = np.empty((H, W), dtype=np.float64)
    lib.or_bf_brute_sv_cos(_ptr(x), H, W, rad.ctypes.data_as(_ip), int(r_max), float(gamma),
                           _ptr(a), len(a), _ptr(o))
    return o


def bf_brute_sv_at(f, radius, idx, r_max, sigma_r=30.0, T=255.0, N=None,
                   range_mode="raised_cosine", spatial="box"):
    """bf_brute_sv at flat pixel indices ``idx`` only."""
    lib = _load()
    if N is None:
        N = n_rule(sigma_r, T)
    x = _f64(f)
    H, W = x.shape
    rad = np.ascontiguousarray(np.asarray(radius, dtype=np.int32))
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    o = np.empty(len(ix), dtype=np.float64)
    if spatial == "box":
        lib.or_bf_brute_sv_at(_ptr(x), H, W, rad.ctypes.data_as(_ip), int(r_max),
                              _range_mode(range_mode), float(sigma_r), int(N),
                              ix.ctypes.data_as(_llp), len(ix), _ptr(o))
    elif spatial == "hat":
        lib.or_bf_brute_sv_shape_at(_ptr(x), H, W, rad.ctypes.data_as(_ip), int(r_max), 1,
                                    _range_mode(range_mode), float(sigma_r), int(N),
                                    ix.ctypes.data_as(_llp), len(ix), _ptr(o))
    else:
        raise ValueError("spatial must be 'box' or 'hat'")
    return o


def bf_brute_at(f, idx, sigma_s=3.0, sigma_r=30.0, T=255.0, kind="gauss", radius=0,
                passes=3, range_mode="raised_cosine", N=None, w1=None, return_q=False):
    """Brute force at flat pixel indices ``idx`` of a single-channel H x W image."""
    lib = _load()
    w1, R, N = _setup(sigma_s, sigma_r, T, kind, radius, passes, N, w1)
    x = _f64(f)
    if x.ndim != 2:
        raise ValueError("bf_brute_at takes one channel")
    H, W = x.shape
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    o = np.empty(len(idx), dtype=np.float64)
    q = np.empty(len(idx), dtype=np.float64)
    lib.or_bf_brute_at(_ptr(x), H, W, _ptr(w1), R, _range_mode(range_mode),
                       float(sigma_r), N, idx.ctypes.data_as(_llp), len(idx),
                       _ptr(o), _ptr(q))
    return (o, q) if return_q else o


def bf_trig(f, sigma_s=3.0, sigma_r=30.0, T=255.0, kind="gauss", radius=0, passes=3,
            N=None, w1=None, return_q=False, return_imag=False):
    """Algorithm 1 in the paper's complex form (N+1 terms), single channel."""
    lib = _load()
    w1, R, N = _setup(sigma_s, sigma_r, T, kind, radius, passes, N, w1)
    x = _f64(f)
    H, W = x.shape
    o = np.empty((H, W), dtype=np.float64)
    q = np.empty((H, W), dtype=np.float64)
    worst = lib.or_bf_trig(_ptr(x), H, W, _ptr(w1), R, float(sigma_r), float(T), N,
                           _ptr(o), _ptr(q))
    res = [o]
    if return_q:
        res.append(q)
    if return_imag:
        res.append(worst)
    return res[0] if len(res) == 1 else tuple(res)


def bf_grad(f, u, sigma_s=4.0, sigma_r=25.0, T=255.0, kind="gauss", radius=0, passes=3,
            range_mode="raised_cosine", N=None, w1=None):
    """Exact FP64 gradient of sum(u * out) w.r.t. f (H x W) and sigma_r (N fixed)."""
    lib = _load()
    w1, R, N = _setup(sigma_s, sigma_r, T, kind, radius, passes, N, w1)
    x = _f64(f)
    uu = _f64(u)
    H, W = x.shape
    g = np.empty((H, W), dtype=np.float64)
    gs = ctypes.c_double(0.0)
    lib.or_bf_grad(_ptr(x), _ptr(uu), H, W, _ptr(w1), R, _range_mode(range_mode),
                   float(sigma_r), N, _ptr(g), ctypes.byref(gs))
    return g, float(gs.value)


def fd_grad_f(f, u, idx, h=1e-3, sigma_s=4.0, sigma_r=25.0, T=255.0, kind="gauss",
              radius=0, passes=3, range_mode="raised_cosine", N=None, w1=None):
    """Central finite differences of sum(u * out) at flat pixel indices ``idx``."""
    lib = _load()
    w1, R, N = _setup(sigma_s, sigma_r, T, kind, radius, passes, N, w1)
    x = _f64(f)
    uu = _f64(u)
    H, W = x.shape
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.empty(len(idx), dtype=np.float64)
    lib.or_bf_fd_grad_f(_ptr(x), _ptr(uu), H, W, _ptr(w1), R, _range_mode(range_mode),
                        float(sigma_r), N, idx.ctypes.data_as(_llp), len(idx), float(h),
                        _ptr(out))
    return out


def loss(f, u, sigma_s=4.0, sigma_r=25.0, T=255.0, kind="gauss", radius=0, passes=3,
         range_mode="raised_cosine", N=None, w1=None):
    """sum(u * out) of the brute force (single channel)."""
    lib = _load()
    w1, R, N = _setup(sigma_s, sigma_r, T, kind, radius, passes, N, w1)
    x = _f64(f)
    uu = _f64(u)
    H, W = x.shape
    return float(lib.or_bf_loss(_ptr(x), _ptr(uu), H, W, _ptr(w1), R,
                                _range_mode(range_mode), float(sigma_r), N))


def fd_grad_sigma_r(f, u, h=1e-4, sigma_s=4.0, sigma_r=25.0, T=255.0, kind="gauss",
                    radius=0, passes=3, range_mode="raised_cosine", N=None, w1=None):
    """Central difference of sum(u * out) in sigma_r with N held fixed."""
    if N is None:
        N = n_rule(sigma_r, T)
    kw = dict(sigma_s=sigma_s, T=T, kind=kind, radius=radius, passes=passes,
              range_mode=range_mode, N=N, w1=w1)
    lp = loss(f, u, sigma_r=sigma_r + h, **kw)
    lm = loss(f, u, sigma_r=sigma_r - h, **kw)
    return (lp - lm) / (2.0 * h)


def phi(s, sigma_r, N=None, T=255.0, range_mode="raised_cosine"):
    """The range kernel the brute force uses, at the points ``s``."""
    lib = _load()
    if N is None:
        N = n_rule(sigma_r, T)
    s = _f64(s).ravel()
    out = np.empty_like(s)
    lib.or_phi_table(_range_mode(range_mode), float(sigma_r), int(N), _ptr(s), len(s),
                     _ptr(out))
    return out


# ---- general trigonometric range kernel (Section 2.2) ----------------------

def _cos_setup(sigma_s, kind, radius, passes, w1, coefs):
    if w1 is None:
        w1 = spatial_w1(kind, sigma_s, radius, passes)
    w1 = _f64(w1)
    a = _f64(coefs).ravel()
    if len(a) < 1:
        raise ValueError("at least one coefficient")
    return w1, (len(w1) - 1) // 2, a


def bf_brute_cos(f, gamma, coefs, sigma_s=3.0, kind="gauss", radius=0, passes=3, w1=None,
                 return_q=False):
    """Brute-force FP64 bilateral filter, eq. (BF), with the range kernel
    phi(s) = sum_n coefs[n] cos(n gamma s); f is H x W or H x W x C."""
    lib = _load()
    w1, R, a = _cos_setup(sigma_s, kind, radius, passes, w1, coefs)
    chans, multi = _channels(f)
    outs, qs = [], []
    for ch in chans:
        x = _f64(ch)
        H, W = x.shape
        o = np.empty((H, W), dtype=np.float64)
        q = np.empty((H, W), dtype=np.float64)
        lib.or_bf_brute_cos(_ptr(x), H, W, _ptr(w1), R, float(gamma), _ptr(a), len(a),
                            _ptr(o), _ptr(q))
        outs.append(o)
        qs.append(q)
    out = np.stack(outs, axis=2) if multi else outs[0]
    q = np.stack(qs, axis=2) if multi else qs[0]
    return (out, q) if return_q else out


def bf_brute_cos_at(f, idx, gamma, coefs, sigma_s=3.0, kind="gauss", radius=0, passes=3,
                    w1=None):
    """bf_brute_cos at flat pixel indices ``idx`` of a single-channel image."""
    lib = _load()
    w1, R, a = _cos_setup(sigma_s, kind, radius, passes, w1, coefs)
    x = _f64(f)
    H, W = x.shape
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    o = np.empty(len(idx), dtype=np.float64)
    lib.or_bf_brute_cos_at(_ptr(x), H, W, _ptr(w1), R, float(gamma), _ptr(a), len(a),
                           idx.ctypes.data_as(_llp), len(idx), _ptr(o), None)
    return o


def bf_grad_cos(f, u, gamma, coefs, sigma_s=4.0, kind="gauss", radius=0, passes=3, w1=None):
    """Exact FP64 gradient of sum(u * out) w.r.t. f for the cosine-polynomial kernel."""
    lib = _load()
    w1, R, a = _cos_setup(sigma_s, kind, radius, passes, w1, coefs)
    x = _f64(f)
    uu = _f64(u)
    H, W = x.shape
    g = np.empty((H, W), dtype=np.float64)
    lib.or_bf_grad_cos(_ptr(x), _ptr(uu), H, W, _ptr(w1), R, float(gamma), _ptr(a), len(a),
                       _ptr(g))
    return g


def fd_grad_f_cos(f, u, idx, gamma, coefs, h=1e-3, sigma_s=4.0, kind="gauss", radius=0,
                  passes=3, w1=None):
    """Central finite differences of sum(u * out) for the cosine-polynomial kernel."""
    lib = _load()
    w1, R, a = _cos_setup(sigma_s, kind, radius, passes, w1, coefs)
    x = _f64(f)
    uu = _f64(u)
    H, W = x.shape
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.empty(len(idx), dtype=np.float64)
    lib.or_bf_fd_grad_f_cos(_ptr(x), _ptr(uu), H, W, _ptr(w1), R, float(gamma), _ptr(a),
                            len(a), idx.ctypes.data_as(_llp), len(idx), float(h), _ptr(out))
    return out


def phi_cos(s, gamma, coefs):
    """The cosine polynomial sum_n coefs[n] cos(n gamma s) at the points ``s``."""
    lib = _load()
    a = _f64(coefs).ravel()
    s = _f64(s).ravel()
    out = np.empty_like(s)
    lib.or_phi_cos_table(float(gamma), _ptr(a), len(a), _ptr(s), len(s), _ptr(out))
    return out


# ---- recursive Gaussian (Young and van Vliet) -------------------------------

def rg_coefs(sigma: float):
    """(B, b1/b0, b2/b0, b3/b0) of the recursive Gaussian and the extension P."""
    c = np.zeros(4, dtype=np.float64)
    P = _load().or_rg_coefs(float(sigma), _ptr(c))
    return c, int(P)


def rg_filter(img, sigma: float) -> np.ndarray:
    """The separable recursive Gaussian of an H x W image (columns, then rows)."""
    x = _f64(img)
    H, W = x.shape
    y = np.empty_like(x)
    _load().or_rg_filter(_ptr(x), H, W, float(sigma), _ptr(y))
    return y


def rg_matrix(n: int, sigma: float) -> np.ndarray:
    """The recursive Gaussian of one line of n samples as an n x n matrix
    (row a: the weights of the inputs in output a)."""
    M = np.empty((n, n), dtype=np.float64)
    _load().or_rg_matrix(int(n), float(sigma), _ptr(M))
    return M


def bf_brute_mat(f, Mv, Mh, sigma_r=30.0, T=255.0, N=None, range_mode="raised_cosine"):
    """eq. (BF) with explicit per-axis weight matrices: pixel (zi, zj) weighs
    Mv[i, zi] Mh[j, zj] in the output at (i, j)."""
    if N is None:
        N = n_rule(sigma_r, T)
    x = _f64(f)
    H, W = x.shape
    Mv, Mh = _f64(Mv), _f64(Mh)
    assert Mv.shape == (H, H) and Mh.shape == (W, W)
    out = np.empty((H, W), dtype=np.float64)
    _load().or_bf_brute_mat(_ptr(x), H, W, _ptr(Mv), _ptr(Mh), _range_mode(range_mode),
                            float(sigma_r), int(N), _ptr(out))
    return out


def bf_grad_mat(f, u, Mv, Mh, sigma_r=25.0, T=255.0, N=None, range_mode="raised_cosine"):
    """Exact FP64 gradient of sum(u * out) w.r.t. f and sigma_r (N fixed) for
    the filter of bf_brute_mat."""
    if N is None:
        N = n_rule(sigma_r, T)
    x, uu = _f64(f), _f64(u)
    H, W = x.shape
    Mv, Mh = _f64(Mv), _f64(Mh)
    assert Mv.shape == (H, H) and Mh.shape == (W, W)
    g = np.empty((H, W), dtype=np.float64)
    gs = ctypes.c_double(0.0)
    _load().or_bf_grad_mat(_ptr(x), _ptr(uu), H, W, _ptr(Mv), _ptr(Mh), _range_mode(range_mode),
                           float(sigma_r), int(N), _ptr(g), ctypes.byref(gs))
    return g, float(gs.value)


def bf_grad_rg(f, u, sigma_s=4.0, sigma_r=25.0, T=255.0, N=None):
    """Exact FP64 gradient of sum(u * out) for the recursive Gaussian spatial
    filter (Section 3): bf_grad_mat with the line filter's matrices."""
    x = _f64(f)
    H, W = x.shape
    return bf_grad_mat(x, u, rg_matrix(H, sigma_s), rg_matrix(W, sigma_s), sigma_r=sigma_r,
                       T=T, N=N)


def bf_trig_rg(f, sigma_s=10.0, sigma_r=30.0, T=255.0, N=None, return_q=False):
    """Algorithm 1 (complex form) with the recursive Gaussian as the averaging;
    f is H x W or H x W x C (channels filtered independently)."""
    lib = _load()
    if N is None:
        N = n_rule(sigma_r, T)
    chans, multi = _channels(f)
    outs, qs = [], []
    for ch in chans:
        x = _f64(ch)
        H, W = x.shape
        o = np.empty((H, W), dtype=np.float64)
        q = np.empty((H, W), dtype=np.float64)
        lib.or_bf_trig_rg(_ptr(x), H, W, float(sigma_s), float(sigma_r), float(T), int(N),
                          _ptr(o), _ptr(q))
        outs.append(o)
        qs.append(q)
    out = np.stack(outs, axis=2) if multi else outs[0]
    q = np.stack(qs, axis=2) if multi else qs[0]
    return (out, q) if return_q else out
