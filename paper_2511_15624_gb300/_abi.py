"""Thin ctypes binding of ``include/ibp.h`` (argument marshalling only).

Every step of a bound runs in the CUDA library ``_lib/libibp_gb300.so``; this
module only converts arrays to pointers.  Host arrays (numpy) use the
synchronous host-pointer mode; CUDA tensors (torch) use the device-pointer
mode on the caller's current stream.  If the library is missing the import
fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# IBP_LIB=check loads the checked build (index guards; see build.py)
LIB_PATH = os.path.join(_PKG, "_lib", "libibp_gb300_check.so" if os.environ.get("IBP_LIB") == "check"
                        else "libibp_gb300.so")

IBP_OK, IBP_EINVAL, IBP_EISLAND, IBP_ESINGULAR, IBP_ENOMEM, IBP_ECUDA, IBP_ETIMEOUT, \
    IBP_EUNSOUND, IBP_ENOTSUP = range(9)

EXPORTED = (
    "ibp_case_create", "ibp_case_destroy", "ibp_bound", "ibp_bound_backward", "ibp_bound_multi",
    "ibp_case_sync", "ibp_case_info", "ibp_case_set_variant", "ibp_kernel_variants",
    "ibp_case_set_timing", "ibp_case_last_timing", "ibp_selftest_wait_timeout", "ibp_last_error",
    "ibp_status_string", "ibp_bound_noalloc", "ibp_case_set_screen", "ibp_case_last_live",
    "ibp_case_set_reduction", "ibp_case_set_refine", "ibp_case_reduction", "ibp_bound_paper",
    "ibp_set_alloc_limit", "ibp_bound_backward_lo", "ibp_case_set_ratings", "ibp_bound_linear",
    "ibp_case_linear_slopes", "ibp_case_linear_inherit", "ibp_bound_multi_backward",
)


class IBPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


class CaseInfo(ctypes.Structure):
    _fields_ = [("n_bus", ctypes.c_int32), ("n_line", ctypes.c_int32), ("n_ctg", ctypes.c_int32),
                ("n_gen", ctypes.c_int32), ("n_load", ctypes.c_int32),
                ("n_active", ctypes.c_int32), ("n_active_pad", ctypes.c_int32),
                ("device", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("build_seconds", ctypes.c_double), ("max_abs_lodf", ctypes.c_double),
                ("n_bus_classes", ctypes.c_int32), ("n_bridges", ctypes.c_int32)]


_lib = None


def lib():
    """Load the CUDA library (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library not built: {LIB_PATH} is missing "
                "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        L.ibp_case_create.argtypes = [I32, I32, I32, P, P, P, P, P, I32, P, P, P, P, I32, P, P, P, P,
                                      D, D, I32, P, I32, ctypes.POINTER(P)]
        L.ibp_case_create.restype = ctypes.c_int
        L.ibp_case_destroy.argtypes = [P]
        L.ibp_case_destroy.restype = None
        L.ibp_bound.argtypes = [P, I32, P, P, P, P, P, P, P, I32, P]
        L.ibp_bound.restype = ctypes.c_int
        L.ibp_set_alloc_limit.argtypes = [ctypes.c_int64]
        L.ibp_set_alloc_limit.restype = ctypes.c_int
        L.ibp_bound_paper.argtypes = [P, I32, P, P, P, P, P, I32, P]
        L.ibp_bound_paper.restype = ctypes.c_int
        L.ibp_bound_backward.argtypes = [P, I32, P, P, P, P, P, P, I32, P]
        L.ibp_bound_backward.restype = ctypes.c_int
        L.ibp_bound_backward_lo.argtypes = [P, I32, P, P, P, P, P, P, I32, P]
        L.ibp_bound_backward_lo.restype = ctypes.c_int
        L.ibp_case_set_ratings.argtypes = [P, P, P, I32, P]
        L.ibp_case_set_ratings.restype = ctypes.c_int
        L.ibp_bound_linear.argtypes = [P, I32, P, P, I32, D, I32, P, P, P, I32, P]
        L.ibp_case_linear_inherit.argtypes = [P, I32, P]
        L.ibp_case_linear_inherit.restype = ctypes.c_int
        L.ibp_bound_linear.restype = ctypes.c_int
        L.ibp_case_linear_slopes.argtypes = [P, I32, P, P, P]
        L.ibp_case_linear_slopes.restype = ctypes.c_int
        L.ibp_bound_multi.argtypes = [I32, P, P, P, P, P, P, P, P]
        L.ibp_bound_multi.restype = ctypes.c_int
        L.ibp_bound_multi_backward.argtypes = [I32, P, P, P, P, P, P, P, P, I32, P]
        L.ibp_bound_multi_backward.restype = ctypes.c_int
        L.ibp_bound_noalloc.argtypes = [P, P, P, P, P, P, P]
        L.ibp_bound_noalloc.restype = ctypes.c_int
        L.ibp_case_sync.argtypes = [P]
        L.ibp_case_sync.restype = ctypes.c_int
        L.ibp_case_info.argtypes = [P, ctypes.POINTER(CaseInfo)]
        L.ibp_case_info.restype = ctypes.c_int
        L.ibp_case_set_variant.argtypes = [P, I32]
        L.ibp_case_set_variant.restype = ctypes.c_int
        L.ibp_kernel_variants.argtypes = [P, I32, I32]
        L.ibp_kernel_variants.restype = I32
        L.ibp_case_set_timing.argtypes = [P, I32]
        L.ibp_case_set_timing.restype = ctypes.c_int
        L.ibp_case_last_timing.argtypes = [P, P, I32]
        L.ibp_case_last_timing.restype = ctypes.c_int
        L.ibp_case_set_screen.argtypes = [P, I32]
        L.ibp_case_set_screen.restype = ctypes.c_int
        L.ibp_case_last_live.argtypes = [P, P, P]
        L.ibp_case_set_reduction.argtypes = [P, I32]
        L.ibp_case_set_reduction.restype = ctypes.c_int
        L.ibp_case_set_refine.argtypes = [P, I32]
        L.ibp_case_set_refine.restype = ctypes.c_int
        L.ibp_case_reduction.argtypes = [P, P, P]
        L.ibp_case_reduction.restype = ctypes.c_int
        L.ibp_case_last_live.restype = ctypes.c_int
        L.ibp_selftest_wait_timeout.argtypes = [I32, I32]
        L.ibp_selftest_wait_timeout.restype = ctypes.c_int
        L.ibp_last_error.argtypes = []
        L.ibp_last_error.restype = ctypes.c_char_p
        L.ibp_status_string.argtypes = [ctypes.c_int]
        L.ibp_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _status_name(s: int) -> str:
    names = ["IBP_OK", "IBP_EINVAL", "IBP_EISLAND", "IBP_ESINGULAR", "IBP_ENOMEM", "IBP_ECUDA",
             "IBP_ETIMEOUT", "IBP_EUNSOUND", "IBP_ENOTSUP"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _check(status: int):
    if status != IBP_OK:
        raise IBPError(status, lib().ibp_last_error().decode())


def ibp_last_error() -> str:
    return lib().ibp_last_error().decode()


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _is_cuda_tensor(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def ibp_case_create(n_bus, slack_bus, line_from, line_to, reactance, rating, rating_ctg,
                    gen_bus, gen_nseg, gen_slope, gen_bkpt, load_bus, load_nseg, load_slope,
                    load_bkpt, zeta_inj, zeta_f, ctg_line, device=0) -> int:
    """Returns the opaque case handle (an int)."""
    keep = dict(
        fr=_host(line_from, np.int32), to=_host(line_to, np.int32), x=_host(reactance, np.float64),
        r=_host(rating, np.float64),
        rc=None if rating_ctg is None else _host(rating_ctg, np.float64),
        gb=_host(gen_bus, np.int32), gn=_host(gen_nseg, np.int32), gs=_host(gen_slope, np.float64),
        gk=_host(gen_bkpt, np.float64), lb=_host(load_bus, np.int32), ln=_host(load_nseg, np.int32),
        ls=_host(load_slope, np.float64), lk=_host(load_bkpt, np.float64),
        ctg=_host(ctg_line, np.int32))
    out = ctypes.c_void_p()
    st = lib().ibp_case_create(
        int(n_bus), int(slack_bus), keep["fr"].size, _ptr(keep["fr"]), _ptr(keep["to"]),
        _ptr(keep["x"]), _ptr(keep["r"]), _ptr(keep["rc"]), keep["gb"].size, _ptr(keep["gb"]),
        _ptr(keep["gn"]), _ptr(keep["gs"]), _ptr(keep["gk"]), keep["lb"].size, _ptr(keep["lb"]),
        _ptr(keep["ln"]), _ptr(keep["ls"]), _ptr(keep["lk"]), float(zeta_inj), float(zeta_f),
        keep["ctg"].size, _ptr(keep["ctg"]), int(device), ctypes.byref(out))
    _check(st)
    return out.value


def ibp_case_destroy(handle: int):
    lib().ibp_case_destroy(ctypes.c_void_p(handle))


def ibp_bound(handle, n_box, box_lo, box_hi, obj_lo, obj_hi, obj_err, flow_lo=None, flow_hi=None,
              ptr_mode=0, stream=None):
    st = lib().ibp_bound(ctypes.c_void_p(handle), int(n_box), _ptr(box_lo), _ptr(box_hi),
                         _ptr(obj_lo), _ptr(obj_hi), _ptr(obj_err), _ptr(flow_lo), _ptr(flow_hi),
                         int(ptr_mode), stream)
    _check(st)


def ibp_set_alloc_limit(nbytes: int):
    _check(lib().ibp_set_alloc_limit(int(nbytes)))


def ibp_bound_paper(handle, n_box, box_lo, box_hi, obj_lo, obj_hi, obj_err, ptr_mode=0, stream=None):
    st = lib().ibp_bound_paper(ctypes.c_void_p(handle), int(n_box), _ptr(box_lo), _ptr(box_hi),
                               _ptr(obj_lo), _ptr(obj_hi), _ptr(obj_err), int(ptr_mode), stream)
    _check(st)


def ibp_bound_backward(handle, n_box, box_lo, box_hi, grad_obj_hi, grad_lo, grad_hi,
                       grad_rating=None, ptr_mode=0, stream=None):
    st = lib().ibp_bound_backward(ctypes.c_void_p(handle), int(n_box), _ptr(box_lo), _ptr(box_hi),
                                  _ptr(grad_obj_hi), _ptr(grad_lo), _ptr(grad_hi),
                                  _ptr(grad_rating), int(ptr_mode), stream)
    _check(st)


def ibp_bound_backward_lo(handle, n_box, box_lo, box_hi, grad_obj_lo, grad_lo, grad_hi,
                          grad_rating=None, ptr_mode=0, stream=None):
    _check(lib().ibp_bound_backward_lo(ctypes.c_void_p(handle), int(n_box), _ptr(box_lo), _ptr(box_hi),
                                       _ptr(grad_obj_lo), _ptr(grad_lo), _ptr(grad_hi),
                                       _ptr(grad_rating), int(ptr_mode), stream))


def ibp_case_set_ratings(handle, rating, rating_ctg=None, ptr_mode=0, stream=None):
    _check(lib().ibp_case_set_ratings(ctypes.c_void_p(handle), _ptr(rating), _ptr(rating_ctg),
                                      int(ptr_mode), stream))


def ibp_bound_multi(handles, n_box, box_lo, box_hi, obj_lo, obj_hi, obj_err, stream=None):
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[ctypes.c_void_p(h) for h in handles])
    NB = (ctypes.c_int32 * n)(*[int(b) for b in n_box])

    def arr(xs):
        return (ctypes.c_void_p * n)(*[ctypes.c_void_p(_ptr(x)) for x in xs])
    st = lib().ibp_bound_multi(n, H, NB, arr(box_lo), arr(box_hi), arr(obj_lo), arr(obj_hi),
                               arr(obj_err), stream)
    _check(st)


def ibp_bound_multi_backward(handles, n_box, box_lo, box_hi, grad_obj, grad_lo, grad_hi,
                             grad_rating=None, side=0, stream=None):
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[ctypes.c_void_p(h) for h in handles])
    NB = (ctypes.c_int32 * n)(*[int(b) for b in n_box])

    def arr(xs):
        return (ctypes.c_void_p * n)(*[ctypes.c_void_p(_ptr(x)) for x in xs])
    GR = None if grad_rating is None else arr(grad_rating)
    st = lib().ibp_bound_multi_backward(n, H, NB, arr(box_lo), arr(box_hi), arr(grad_obj), arr(grad_lo),
                                        arr(grad_hi), GR, int(side), stream)
    _check(st)


def ibp_bound_noalloc(handle, box_lo, box_hi, obj_lo, obj_hi, obj_err, stream=None):
    """One-box bound with no device allocation; all pointers are device pointers."""
    st = lib().ibp_bound_noalloc(ctypes.c_void_p(handle), _ptr(box_lo), _ptr(box_hi), _ptr(obj_lo),
                                 _ptr(obj_hi), _ptr(obj_err), stream)
    _check(st)


def ibp_case_sync(handle):
    _check(lib().ibp_case_sync(ctypes.c_void_p(handle)))


def ibp_case_info(handle) -> CaseInfo:
    info = CaseInfo()
    _check(lib().ibp_case_info(ctypes.c_void_p(handle), ctypes.byref(info)))
    return info


def ibp_case_set_variant(handle, variant: int):
    _check(lib().ibp_case_set_variant(ctypes.c_void_p(handle), int(variant)))


def ibp_kernel_variants(batched: bool):
    n = lib().ibp_kernel_variants(None, 0, int(batched))
    ids = (ctypes.c_int32 * max(n, 1))()
    lib().ibp_kernel_variants(ids, n, int(batched))
    return [ids[i] for i in range(n)]


def ibp_case_set_timing(handle, enable: bool):
    _check(lib().ibp_case_set_timing(ctypes.c_void_p(handle), int(bool(enable))))


def ibp_case_last_timing(handle):
    ms = (ctypes.c_float * 6)()
    _check(lib().ibp_case_last_timing(ctypes.c_void_p(handle), ms, 6))
    return {"box_to_bus": ms[0], "base_flow": ms[1], "screen": ms[2], "contingency": ms[3],
            "refine": ms[4], "assemble": ms[5]}


def ibp_case_set_screen(handle, enable: bool):
    _check(lib().ibp_case_set_screen(ctypes.c_void_p(handle), int(bool(enable))))


def ibp_case_set_reduction(handle, enable: bool):
    _check(lib().ibp_case_set_reduction(ctypes.c_void_p(handle), int(bool(enable))))


def ibp_case_set_refine(handle, enable: bool):
    _check(lib().ibp_case_set_refine(ctypes.c_void_p(handle), int(bool(enable))))


def ibp_case_reduction(handle, n_active: int, n_line: int):
    """(class of each active column or -1, bridge flag of each line)."""
    cls = np.empty(max(n_active, 1), np.int32)
    br = np.empty(max(n_line, 1), np.int32)
    _check(lib().ibp_case_reduction(ctypes.c_void_p(handle), cls.ctypes.data_as(ctypes.c_void_p),
                                    br.ctypes.data_as(ctypes.c_void_p)))
    return cls[:n_active].copy(), br[:n_line].copy()


def ibp_case_last_live(handle, n_line: int):
    """(count, ascending line indices) kept by the last screened call, or (-1, None)."""
    n = ctypes.c_int32(0)
    buf = np.empty(max(n_line, 1), np.int32)
    _check(lib().ibp_case_last_live(ctypes.c_void_p(handle), ctypes.byref(n),
                                    buf.ctypes.data_as(ctypes.c_void_p)))
    if n.value < 0:
        return -1, None
    return int(n.value), buf[: n.value].copy()


def ibp_selftest_wait_timeout(device: int, limit_us: int) -> int:
    """Returns the status code (IBP_ETIMEOUT is the expected outcome)."""
    return int(lib().ibp_selftest_wait_timeout(int(device), int(limit_us)))


def ibp_bound_linear(handle, n_box, box_lo, box_hi, n_iter, primal_weight, obj_hi, obj_err,
                     x_point=None, ptr_mode=0, stream=None, warm=0):
    """warm: 0 cold, 1 + f to continue the held boxes [f, f + n_box)."""
    _check(lib().ibp_bound_linear(ctypes.c_void_p(handle), int(n_box), _ptr(box_lo), _ptr(box_hi),
                                  int(n_iter), float(primal_weight), int(warm), _ptr(obj_hi),
                                  _ptr(obj_err), _ptr(x_point), int(ptr_mode), stream))


def ibp_case_linear_inherit(handle, parent):
    par = np.ascontiguousarray(parent, np.int32)
    _check(lib().ibp_case_linear_inherit(ctypes.c_void_p(handle), par.size, _ptr(par)))


def ibp_case_linear_slopes(handle, n_box, n_ctg, n_line):
    a_c = np.empty((n_box, n_ctg, n_line), np.float32)
    a_b = np.empty((n_box, n_line), np.float32)
    a0 = np.empty(n_box)
    _check(lib().ibp_case_linear_slopes(ctypes.c_void_p(handle), int(n_box), _ptr(a_c), _ptr(a_b), _ptr(a0)))
    return a_c, a_b, a0
