"""ctypes loader for libbf.so.

There is no fallback: if the library is not built, or cannot be loaded, every
entry point raises.  torch is imported first so that libbf binds to the same
CUDA runtime instance torch uses (same SONAME, already loaded), which keeps
the current device and stream handles consistent between the two.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbf.so")
_lock = threading.Lock()
_lib = None

c_int = ctypes.c_int
c_double = ctypes.c_double
c_void_p = ctypes.c_void_p
c_size_t = ctypes.c_size_t
c_ll = ctypes.c_longlong
c_char_p = ctypes.c_char_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class BfError(RuntimeError):
    """A libbf call returned a status other than BF_OK."""

    def __init__(self, status: int, message: str):
        super().__init__("libbf status %d: %s" % (status, message))
        self.status = status


class PlanOpts(ctypes.Structure):
    _fields_ = [("N_override", c_int), ("radius_override", c_int), ("box_passes", c_int),
                ("degree_rule", c_int)]


def _declare(lib):
    sig = {
        "bf_plan_create": (c_int, [ctypes.POINTER(c_void_p), c_double, c_double, c_double, c_int,
                                   ctypes.POINTER(PlanOpts)]),
        "bf_plan_create_cosine": (c_int, [ctypes.POINTER(c_void_p), c_double, c_double, _dp,
                                          c_int, c_int, ctypes.POINTER(PlanOpts)]),
        "bf_plan_destroy": (None, [c_void_p]),
        "bf_plan_info": (c_int, [c_void_p, _ip, _ip, _ip, _dp]),
        "bf_plan_terms": (c_int, [c_void_p, _dp, _dp, c_int, _ip]),
        "bf_plan_weights": (c_int, [c_void_p, _dp, c_int, _ip]),
        "bf_forward": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_int, c_int, c_ll,
                               c_void_p, c_void_p]),
        "bf_forward_stack": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_int, c_int,
                                     c_void_p, c_void_p]),
        "bf_backward_stack_workspace": (c_size_t, [c_void_p, c_int, c_int, c_int]),
        "bf_backward_stack": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_int, c_int, c_int, c_void_p, c_size_t, c_void_p]),
        "bf_forward_tune": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_int, c_int, c_ll,
                                    c_int, c_void_p, _ip, ctypes.POINTER(ctypes.c_float)]),
        "bf_forward_set_shape": (c_int, [c_void_p, c_int, c_int, c_int, c_int]),
        "bf_forward_unfused_workspace": (c_size_t, [c_int, c_int]),
        "bf_forward_unfused": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p,
                                       c_size_t, c_void_p]),
        "bf_backward_workspace": (c_size_t, [c_void_p, c_int, c_int]),
        "bf_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_int, c_int, c_void_p, c_size_t, c_void_p]),
        "bf_batch_create": (c_int, [ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), _ip, _ip,
                                    c_int]),
        "bf_batch_bind": (c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                  c_void_p]),
        "bf_batch_forward": (c_int, [c_void_p, c_void_p]),
        "bf_batch_check": (c_int, [c_void_p, c_void_p, _ip]),
        "bf_batch_destroy": (None, [c_void_p]),
        "bf_batch_tune": (c_int, [c_void_p, c_void_p, c_int, _ip, _ip,
                                  ctypes.POINTER(ctypes.c_float)]),
        "bf_batch_config": (c_int, [c_void_p, c_int, _ip, _ip]),
        "bf_batch_set_config": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p]),
        "bf_release_scratch": (None, []),
        "bf_last_error": (c_char_p, []),
        "bf_version": (c_int, []),
        "bf_forward_space_variant": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p,
                                             c_int, c_int, ctypes.c_longlong, c_void_p]),
        "bf_forward_space_variant_hat": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int,
                                                 c_void_p, c_int, c_int, ctypes.c_longlong,
                                                 c_void_p]),
        "bf_forward_space_variant_ex": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_int,
                                                c_void_p, c_int, c_int, c_int, ctypes.c_longlong,
                                                c_void_p]),
        "bf_forward_host": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int,
                                    c_int, c_int, ctypes.c_longlong, c_void_p]),
        "bf_forward_host_overlap": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p,
                                            c_void_p, c_int, c_int, c_int, ctypes.c_longlong,
                                            c_void_p, c_void_p]),
        "bf_fp32_pipe_rate": (c_int, [c_int, ctypes.POINTER(ctypes.c_double), c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def lib():
    """The loaded library; raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            import torch  # noqa: F401  (load torch's CUDA runtime first)
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    "libbf.so is not built (%s); run paper_1105_4204_gb300.build.build() -- "
                    "there is no CPU fallback" % LIB_PATH)
            l = ctypes.CDLL(LIB_PATH)
            _declare(l)
            _lib = l
    return _lib


def check(status: int) -> None:
    if status != 0:
        msg = lib().bf_last_error()
        raise BfError(status, msg.decode() if msg else "")
