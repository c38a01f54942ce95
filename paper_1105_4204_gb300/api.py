"""Python binding of libbf: argument marshalling only.

Every step of the filter runs in the CUDA library; torch provides device
memory and the current stream.  Images are torch CUDA tensors, row-major,
H x W (one channel) or H x W x C (interleaved channels).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import PlanOpts, check, lib

GAUSS = 0
BOX = 1
RECURSIVE = 2
_KINDS = {"gauss": GAUSS, "box": BOX, "recursive": RECURSIVE}


def _kind(kind) -> int:
    return _KINDS[kind] if isinstance(kind, str) else int(kind)


def _stream_ptr(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """Host-side plan: degree N, folded binomial term table, spatial taps
    (Algorithm 1 steps 1-3).  Creating it never touches the GPU."""

    DEGREE_RULES = {"estimate": 0, "table1": 1}

    def __init__(self, sigma_s: float, sigma_r: float, T: float = 255.0, kind="gauss",
                 N: int = 0, radius: int = 0, passes: int = 0, degree_rule: str = "estimate"):
        """``degree_rule`` (when N is 0): "estimate" N = max(1, ceil((gamma
        sigma_r)^-2)), or "table1", the empirical minimum degrees of Table 1."""
        self._lib = lib()
        self._h = ctypes.c_void_p()
        opts = PlanOpts(int(N), int(radius), int(passes), self.DEGREE_RULES[degree_rule])
        check(self._lib.bf_plan_create(ctypes.byref(self._h), float(sigma_s), float(sigma_r),
                                       float(T), _kind(kind), ctypes.byref(opts)))
        self.sigma_s, self.sigma_r, self.T, self.kind = float(sigma_s), float(sigma_r), float(T), kind
        self._info()

    @classmethod
    def cosine(cls, sigma_s: float, gamma: float, coefs, kind="gauss", radius: int = 0,
               passes: int = 0) -> "Plan":
        """Plan for the general trigonometric range kernel of Section 2.2,
        phi(s) = sum_n coefs[n] cos(n gamma s) (gamma in radians per gray
        level).  The spatial kernel is as for the raised cosine."""
        self = cls.__new__(cls)
        self._lib = lib()
        self._h = ctypes.c_void_p()
        a = np.ascontiguousarray(np.asarray(coefs, dtype=np.float64).ravel())
        opts = PlanOpts(0, int(radius), int(passes))
        check(self._lib.bf_plan_create_cosine(
            ctypes.byref(self._h), float(sigma_s), float(gamma),
            a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(a), _kind(kind),
            ctypes.byref(opts)))
        self.sigma_s, self.sigma_r, self.T, self.kind = float(sigma_s), None, None, kind
        self.gamma, self.coefs = float(gamma), a.copy()
        self._info()
        return self

    def _info(self):
        n, nf, rad = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        sig = ctypes.c_double()
        check(self._lib.bf_plan_info(self._h, ctypes.byref(n), ctypes.byref(nf),
                                     ctypes.byref(rad), ctypes.byref(sig)))
        self.N, self.n_terms, self.radius = n.value, nf.value, rad.value
        self.achieved_sigma_s = sig.value

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def terms(self):
        """(a, omega): FP64 weights and angular frequencies (rad per gray level)
        in the kernels' accumulation order."""
        a = np.zeros(self.n_terms, dtype=np.float64)
        w = np.zeros(self.n_terms, dtype=np.float64)
        cnt = ctypes.c_int()
        check(self._lib.bf_plan_terms(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      self.n_terms, ctypes.byref(cnt)))
        return a, w

    def weights(self) -> np.ndarray:
        """1-D spatial taps w1[-R..R] (unit sum)."""
        w = np.zeros(2 * self.radius + 1, dtype=np.float64)
        cnt = ctypes.c_int()
        check(self._lib.bf_plan_weights(self._h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        len(w), ctypes.byref(cnt)))
        return w

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                self._lib.bf_plan_destroy(h)
            except Exception:
                pass
            self._h = ctypes.c_void_p()


def _image_args(img: torch.Tensor, where: str = "cuda"):
    if where == "cuda" and not img.is_cuda:
        raise ValueError("image must be a CUDA tensor")
    if where == "host" and img.is_cuda:
        raise ValueError("image must be a host tensor")
    if img.dtype == torch.float32:
        dt = 0
    elif img.dtype == torch.uint8:
        dt = 1
    else:
        raise ValueError("image dtype must be float32 or uint8")
    if img.dim() == 2:
        H, W = img.shape
        C = 1
        if img.stride(1) != 1:
            raise ValueError("rows must be contiguous")
        row_stride = img.stride(0)
    elif img.dim() == 3:
        H, W, C = img.shape
        if img.stride(2) != 1 or img.stride(1) != C:
            raise ValueError("H x W x C image must have interleaved, contiguous rows")
        row_stride = img.stride(0)
    else:
        raise ValueError("image must be H x W or H x W x C")
    return dt, H, W, C, row_stride


def forward(plan: Plan, img: torch.Tensor, return_q: bool = False, out: torch.Tensor | None = None,
            q: torch.Tensor | None = None, stream=None):
    """Fused forward filter; returns a float32 tensor of img's shape (and the
    normaliser Q when ``return_q``)."""
    dt, H, W, C, rs = _image_args(img)
    shape = tuple(img.shape)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=img.device)
    if return_q and q is None:
        q = torch.empty(shape, dtype=torch.float32, device=img.device)
    check(lib().bf_forward(plan.handle, ctypes.c_void_p(img.data_ptr()), dt,
                           ctypes.c_void_p(out.data_ptr()), H, W, C, rs,
                           ctypes.c_void_p(q.data_ptr() if return_q else 0), _stream_ptr(stream)))
    return (out, q) if return_q else out


def tune(plan: Plan, img: torch.Tensor, reps: int = 3, stream=None):
    """Pick the fused kernel's tile shape for this plan and image size by
    timing the candidates on ``img`` (cached for later ``forward`` calls)."""
    dt, H, W, C, rs = _image_args(img)
    out = torch.empty(tuple(img.shape), dtype=torch.float32, device=img.device)
    shape, ms = ctypes.c_int(), ctypes.c_float()
    check(lib().bf_forward_tune(plan.handle, ctypes.c_void_p(img.data_ptr()), dt,
                                ctypes.c_void_p(out.data_ptr()), H, W, C, rs, int(reps),
                                _stream_ptr(stream), ctypes.byref(shape), ctypes.byref(ms)))
    v = shape.value
    names = {-1: "streaming", 0: "32x64", 1: "32x96", 2: "64x64", 3: "64x64-seg32"}
    return {"shape": names[v if v < 0 else v & 0xFF],
            "split": 1 if v < 0 else max(1, v >> 8), "ms": ms.value}


SHAPES = {"32x64": 0, "32x96": 1, "64x64": 2, "64x64-seg32": 3}


def set_shape(plan: Plan, img: torch.Tensor, shape: str, split: int = 1):
    """Pin the fused kernel's tile shape ("32x64", "32x96", "64x64" or
    "64x64-seg32") and term split (1, 2, 4 or 8 groups of terms, one block
    each per tile) for this plan at img's size, as ``tune`` would after
    timing."""
    dt, H, W, C, rs = _image_args(img)
    check(lib().bf_forward_set_shape(plan.handle, H, W, C, SHAPES[shape] | (int(split) << 8)))


def forward_space_variant(plan: Plan, img: torch.Tensor, radius: torch.Tensor, r_max: int = 16,
                          out: torch.Tensor | None = None, stream=None,
                          spatial: str = "box") -> torch.Tensor:
    """Space-variant filter (Section 4): pixel x averages over its own box
    (spatial="box", r_max <= 16) or separable hat (spatial="hat", r_max <= 8)
    of half-width radius[x] (int32 H x W on the device, clamped into
    [0, r_max]), with the plan's range kernel.  H x W, or H x W x C with
    interleaved channels (C <= 4, each filtered with the same radius map); a
    smaller r_max reads less halo."""
    if spatial not in ("box", "hat"):
        raise ValueError("spatial must be 'box' or 'hat'")
    dt, H, W, C, rs = _image_args(img)
    if radius.dtype != torch.int32 or tuple(radius.shape) != (H, W) or not radius.is_contiguous() \
            or radius.device != img.device:
        raise ValueError("radius must be a contiguous int32 H x W tensor on the image's device")
    if out is None:
        out = torch.empty(tuple(img.shape), dtype=torch.float32, device=img.device)
    check(lib().bf_forward_space_variant_ex(plan.handle, ctypes.c_void_p(img.data_ptr()), dt,
                                            ctypes.c_void_p(radius.data_ptr()), int(r_max),
                                            0 if spatial == "box" else 1,
                                            ctypes.c_void_p(out.data_ptr()), H, W, C, rs,
                                            _stream_ptr(stream)))
    return out


def fp32_pipe_rate(paired: bool = False, stream=None) -> float:
    """Measured FP32 lane operations per second of the current device (an FMA
    counts as one; ``paired`` issues them as FFMA2).  Synchronises the
    stream; about 10 ms of GPU time.  A measuring aid for the ALU roofline."""
    r = ctypes.c_double()
    check(lib().bf_fp32_pipe_rate(int(bool(paired)), ctypes.byref(r), _stream_ptr(stream)))
    return r.value


def forward_host(plan: Plan, img_host: torch.Tensor | None, out_host: torch.Tensor | None = None,
                 stream=None, dev_in: torch.Tensor | None = None,
                 dev_out: torch.Tensor | None = None, copy_stream=None) -> torch.Tensor | None:
    """End-to-end call for a host image (``bf_forward_host``): copies img_host
    (pinned for asynchrony) into ``dev_in``, filters it into ``dev_out`` and
    copies the result into ``out_host`` (a new pinned tensor when None), in
    order on the stream.  ``img_host=None`` filters what ``dev_in`` already
    holds (no copy in); the device buffers are allocated when not given.
    With ``copy_stream`` (``bf_forward_host_overlap``) the copy back runs on
    that stream after this call's filter, so that ``stream`` can go on.
    Returns out_host; it is complete once the stream that copies it reaches
    the call's end."""
    src = img_host if img_host is not None else dev_in
    if src is None:
        raise ValueError("forward_host needs img_host or a filled dev_in")
    dt, H, W, C, rs = _image_args(src, "host" if img_host is not None else "cuda")
    dev = torch.device("cuda", torch.cuda.current_device())
    shape = tuple(src.shape)
    if dev_in is None:
        dev_in = torch.empty(shape, dtype=src.dtype, device=dev)
    if dev_out is None:
        dev_out = torch.empty(shape, dtype=torch.float32, device=dev)
    if out_host is None:
        out_host = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    if img_host is not None and (tuple(dev_in.stride()) != tuple(img_host.stride())
                                 or dev_in.dtype != img_host.dtype):
        raise ValueError("dev_in must have img_host's dtype and strides")
    if not out_host.is_contiguous() or not dev_out.is_contiguous():
        raise ValueError("out_host and dev_out must be contiguous")
    args = (plan.handle, ctypes.c_void_p(img_host.data_ptr() if img_host is not None else 0), dt,
            ctypes.c_void_p(dev_in.data_ptr()), ctypes.c_void_p(dev_out.data_ptr()),
            ctypes.c_void_p(out_host.data_ptr()), H, W, C, rs, _stream_ptr(stream))
    if copy_stream is None:
        check(lib().bf_forward_host(*args))
    else:
        check(lib().bf_forward_host_overlap(*args, _stream_ptr(copy_stream)))
    return out_host


def forward_unfused(plan: Plan, img: torch.Tensor, out: torch.Tensor | None = None,
                    workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Unfused per-term baseline (single-channel float32 only)."""
    dt, H, W, C, rs = _image_args(img)
    if dt != 0 or C != 1 or rs != W:
        raise ValueError("unfused baseline takes a contiguous H x W float32 image")
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    nbytes = lib().bf_forward_unfused_workspace(H, W)
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=img.device)
    check(lib().bf_forward_unfused(plan.handle, ctypes.c_void_p(img.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), H, W,
                                   ctypes.c_void_p(workspace.data_ptr()), nbytes,
                                   _stream_ptr(stream)))
    return out


def backward(plan: Plan, f: torch.Tensor, out: torch.Tensor, q: torch.Tensor,
             grad_out: torch.Tensor, need_sigma: bool = True, grad_in: torch.Tensor | None = None,
             workspace: torch.Tensor | None = None, stream=None):
    """Adjoint of ``forward`` for one H x W float32 image.  Returns (dL/df,
    dL/dsigma_r as a 0-dim float64 device tensor or None)."""
    for t in (f, out, q, grad_out):
        if not t.is_cuda or t.dtype != torch.float32 or t.dim() != 2 or not t.is_contiguous():
            raise ValueError("backward takes contiguous H x W float32 CUDA tensors")
    H, W = f.shape
    if grad_in is None:
        grad_in = torch.empty((H, W), dtype=torch.float32, device=f.device)
    gs = None
    ws_ptr, nbytes = 0, 0
    if need_sigma:
        gs = torch.empty((), dtype=torch.float64, device=f.device)
        nbytes = lib().bf_backward_workspace(plan.handle, H, W)
        if workspace is None or workspace.numel() * workspace.element_size() < nbytes:
            workspace = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=f.device)
        ws_ptr = workspace.data_ptr()
    check(lib().bf_backward(plan.handle, ctypes.c_void_p(f.data_ptr()),
                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                            ctypes.c_void_p(grad_out.data_ptr()),
                            ctypes.c_void_p(grad_in.data_ptr()),
                            ctypes.c_void_p(gs.data_ptr() if gs is not None else 0), H, W,
                            ctypes.c_void_p(ws_ptr), nbytes, _stream_ptr(stream)))
    return grad_in, gs


def forward_stack(plan: Plan, imgs: torch.Tensor, return_q: bool = False,
                  out: torch.Tensor | None = None, q: torch.Tensor | None = None, stream=None):
    """Filter a contiguous B x H x W stack (float32 or uint8) in one launch."""
    if not imgs.is_cuda or imgs.dim() != 3 or not imgs.is_contiguous():
        raise ValueError("stack must be a contiguous B x H x W CUDA tensor")
    dt = {torch.float32: 0, torch.uint8: 1}.get(imgs.dtype)
    if dt is None:
        raise ValueError("stack dtype must be float32 or uint8")
    B, H, W = imgs.shape
    if out is None:
        out = torch.empty((B, H, W), dtype=torch.float32, device=imgs.device)
    if return_q and q is None:
        q = torch.empty((B, H, W), dtype=torch.float32, device=imgs.device)
    check(lib().bf_forward_stack(plan.handle, ctypes.c_void_p(imgs.data_ptr()), dt,
                                 ctypes.c_void_p(out.data_ptr()), H, W, B,
                                 ctypes.c_void_p(q.data_ptr() if return_q else 0),
                                 _stream_ptr(stream)))
    return (out, q) if return_q else out


def backward_stack(plan: Plan, f: torch.Tensor, out: torch.Tensor, q: torch.Tensor,
                   grad_out: torch.Tensor, need_sigma: bool = True,
                   grad_in: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                   stream=None):
    """Adjoint over a contiguous B x H x W float32 stack in one launch; returns
    (dL/df, sum over the stack of dL/dsigma_r or None)."""
    for t in (f, out, q, grad_out):
        if not t.is_cuda or t.dtype != torch.float32 or t.dim() != 3 or not t.is_contiguous():
            raise ValueError("backward_stack takes contiguous B x H x W float32 CUDA tensors")
    B, H, W = f.shape
    if grad_in is None:
        grad_in = torch.empty_like(f)
    gs = None
    ws_ptr, nbytes = 0, 0
    if need_sigma:
        gs = torch.empty((), dtype=torch.float64, device=f.device)
        nbytes = lib().bf_backward_stack_workspace(plan.handle, H, W, B)
        if workspace is None or workspace.numel() * workspace.element_size() < nbytes:
            workspace = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=f.device)
        ws_ptr = workspace.data_ptr()
    check(lib().bf_backward_stack(plan.handle, ctypes.c_void_p(f.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                  ctypes.c_void_p(grad_out.data_ptr()),
                                  ctypes.c_void_p(grad_in.data_ptr()),
                                  ctypes.c_void_p(gs.data_ptr() if gs is not None else 0), H, W, B,
                                  ctypes.c_void_p(ws_ptr), nbytes, _stream_ptr(stream)))
    return grad_in, gs


class BilateralFunction(torch.autograd.Function):
    """Differentiable filter: forward through the fused kernel, backward through
    the fused adjoint kernel (gradients w.r.t. the image and sigma_r; N is held
    at the degree the rule gives for the forward's sigma_r)."""

    @staticmethod
    def forward(ctx, f, sigma_r, sigma_s, T, kind, radius):
        sr = float(sigma_r)
        plan = Plan(sigma_s, sr, T, kind=kind, radius=radius)
        imgs = (f if f.dim() == 3 else f.unsqueeze(0)).contiguous()
        out, q = forward_stack(plan, imgs, return_q=True)
        ctx.plan = plan
        ctx.squeeze = f.dim() == 2
        ctx.sigma_is_tensor = isinstance(sigma_r, torch.Tensor)
        ctx.save_for_backward(imgs, out, q)
        return out[0] if ctx.squeeze else out

    @staticmethod
    def backward(ctx, grad_out):
        imgs, out, q = ctx.saved_tensors
        g = (grad_out if grad_out.dim() == 3 else grad_out.unsqueeze(0)).contiguous()
        need_sigma = ctx.sigma_is_tensor and ctx.needs_input_grad[1]
        gf, gs = backward_stack(ctx.plan, imgs, out, q, g, need_sigma=need_sigma)
        if ctx.squeeze:
            gf = gf[0]
        gsig = gs.to(torch.float32) if gs is not None else None
        return gf, gsig, None, None, None, None


def bilateral(f: torch.Tensor, sigma_s: float, sigma_r, T: float = 255.0, kind="gauss",
              radius: int = 0) -> torch.Tensor:
    """Differentiable bilateral filter of an H x W or B x H x W float32 CUDA
    tensor; ``sigma_r`` may be a float or a 0-dim tensor requiring grad."""
    return BilateralFunction.apply(f, sigma_r, float(sigma_s), float(T), kind, int(radius))


class Batch:
    """Many float32 H x W images, each with its own plan, filtered by one
    persistent launch replayed from a CUDA graph."""

    def __init__(self, plans, sizes):
        self._lib = lib()
        self.plans = list(plans)
        self.sizes = [(int(h), int(w)) for h, w in sizes]
        n = len(self.plans)
        arr = (ctypes.c_void_p * n)(*[p.handle.value for p in self.plans])
        Hs = (ctypes.c_int * n)(*[h for h, _ in self.sizes])
        Ws = (ctypes.c_int * n)(*[w for _, w in self.sizes])
        self._h = ctypes.c_void_p()
        check(self._lib.bf_batch_create(ctypes.byref(self._h), arr, Hs, Ws, n))
        self._bound = None

    def bind(self, ins, outs, stream=None):
        n = len(self.plans)
        for t, (h, w) in zip(list(ins) + list(outs), self.sizes + self.sizes):
            if not t.is_cuda or t.dtype != torch.float32 or tuple(t.shape) != (h, w) \
                    or not t.is_contiguous():
                raise ValueError("batch images must be contiguous float32 CUDA tensors of their size")
        pin = (ctypes.c_void_p * n)(*[t.data_ptr() for t in ins])
        pout = (ctypes.c_void_p * n)(*[t.data_ptr() for t in outs])
        check(self._lib.bf_batch_bind(self._h, pin, pout, _stream_ptr(stream)))
        self._bound = (list(ins), list(outs))  # keep the buffers alive while bound

    def forward(self, stream=None):
        check(self._lib.bf_batch_forward(self._h, _stream_ptr(stream)))

    def check(self, stream=None) -> int:
        err = ctypes.c_int()
        check(self._lib.bf_batch_check(self._h, _stream_ptr(stream), ctypes.byref(err)))
        return err.value

    def tune(self, reps: int = 3, stream=None):
        """Pick each radius bucket's tile shape and term split, then the
        persistent grid and queue order, by timing the whole batch."""
        g, o, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        check(self._lib.bf_batch_tune(self._h, _stream_ptr(stream), int(reps), ctypes.byref(g),
                                      ctypes.byref(o), ctypes.byref(ms)))
        return {"grid": g.value, "order": "largest-cost-first" if o.value == 0 else "image",
                "ms": ms.value, "buckets": self.config()}

    def config(self):
        """{r: (shape name, split)} of the radius buckets r = 1 .. 8."""
        names = {0: "32x64", 1: "32x96", 3: "64x64-seg32"}
        out = {}
        for r in range(1, 9):
            sh, sp = ctypes.c_int(), ctypes.c_int()
            check(self._lib.bf_batch_config(self._h, r, ctypes.byref(sh), ctypes.byref(sp)))
            out[r] = (names[sh.value], sp.value)
        return out

    def set_config(self, r: int, shape: str, split: int = 1, stream=None):
        """Pin radius bucket r's tile shape ("32x64", "32x96" for r <= 4,
        "64x64-seg32" for r = 7, 8) and term split (1, 2 or 4)."""
        ids = {"32x64": 0, "32x96": 1, "64x64-seg32": 3}
        check(self._lib.bf_batch_set_config(self._h, int(r), ids[shape], int(split),
                                            _stream_ptr(stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                self._lib.bf_batch_destroy(h)
            except Exception:
                pass
            self._h = ctypes.c_void_p()
