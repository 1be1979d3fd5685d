"""Thin Python binding of the C ABI in include/csrk.h (argument marshalling only).

Every function here has the C entry point's name without the ``csrk_`` prefix and does
nothing but convert arguments: numpy arrays become host pointers, torch tensors device
pointers, ``stream=None`` becomes the current torch stream of the tensors' device.  All
computation runs in libcsrk.so; if the library is missing or fails to load, ``lib()``
raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

F64, F32, BF16 = 0, 1, 2
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16, F64: F64, F32: F32, BF16: BF16}
VEC_PERMUTED, ACC_F32, X_F32, HOST_VECTORS, X_PERMUTED = 1, 2, 4, 8, 16
REORDER = {"none": 0, "rcm": 1, 0: 0, 1: 1}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_MATRIX", 3: "ERR_STATE", 4: "ERR_ALLOC",
          5: "ERR_CUDA", 6: "ERR_UNSUPPORTED", 7: "ERR_TIMEOUT", 8: "ERR_NOT_CONVERGED"}


class CsrkError(RuntimeError):
    def __init__(self, code: int, message: str, func: str):
        self.code = code
        self.status = STATUS.get(code, str(code))
        super().__init__(f"{func}: {self.status}: {message}")


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_d = ctypes.c_double
_u = ctypes.c_uint
_pi32 = ctypes.POINTER(ctypes.c_int32)
_pi64 = ctypes.POINTER(ctypes.c_int64)

_PROTOS = {
    "csrk_create": [_i32, _vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(_vp)],
    "csrk_reorder": [_vp, ctypes.c_int, _vp],
    "csrk_reorder_bandk": [_vp, _i32, _i32, _vp],
    "csrk_index_bits": [_vp, _pi32],
    "csrk_split_long_rows": [_vp, _i32, _pi32],
    "csrk_set_sizes": [_vp, _i32, _i32],
    "csrk_set_pointers": [_vp, _i32, _vp, _i32, _vp],
    "csrk_spmv": [_vp, _d, _vp, _d, _vp, _u, _vp],
    "csrk_spmm": [_vp, _i32, _d, _vp, _i64, _d, _vp, _i64, _u, _vp],
    "csrk_destroy": [_vp],
    "csrk_permute": [_vp, ctypes.c_int, _i32, _vp, _i64, _vp, _i64, _u, _vp],
    "csrk_info": [_vp, _pi32, _pi64, _pi32, _pi32, _pi32, _pi32, _pi32],
    "csrk_export": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "csrk_export_values": [_vp, ctypes.c_int, _vp],
    "csrk_model_sizes": [_d, ctypes.c_int, _pi32, _pi32],
    "csrk_tuned_config": [_vp, _pi32, _pi32, _pi32, _pi32, _pi32, _pi32],
    "csrk_set_config": [_vp, _i32, _i32, _i32, _i32, _i32, _i32],
    "csrk_device_status": [_vp, _vp, _pi32],
    "csrk_cg": [_vp, _vp, _vp, _d, _i32, ctypes.c_int, _i32, _i32, _u, _pi32, ctypes.POINTER(_d), _vp],
    "csrk_selftest_bounded_wait": [_vp, ctypes.c_uint64, _vp, _pi32],
    "csrk_selftest_narrow": [_vp, _i64, _vp, _vp, _vp],
    "csrk_batch_create": [_vp, _i32, _vp, ctypes.POINTER(_vp)],
    "csrk_batch_spmm": [_vp, _d, _vp, _d, _vp, _u, _vp],
    "csrk_batch_cg": [_vp, _vp, _vp, _i32, _d, _vp, _vp, _vp],
    "csrk_batch_info": [_vp, _pi32, _pi32, _pi32, _pi64],
    "csrk_batch_plan": [_vp, _pi32, _pi32, _pi32],
    "csrk_batch_cg_solve": [_vp, _vp, _vp, _d, _i32, ctypes.c_int, _i32, ctypes.c_int, _vp, _vp, _pi32, _vp],
    "csrk_batch_device_status": [_vp, _pi32],
    "csrk_batch_destroy": [_vp],
    "csrk_spmv_static_scratch": [_i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _d, _vp, _d, _vp, _vp],
    "csrk_xwin_info": [_vp, _vp, _vp, _vp, _vp],
    "csrk_xwin_export": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "csrk_col16_export": [_vp, _vp, _vp],
    "csrk_selftest_stage_plan": [_i32, _i32, _i64, _i32, _i32, _i32, _i32, _i64, _i32, _vp],
}


def lib(build_if_missing: bool = True):
    """Load libcsrk.so (building it first when the sources are newer); with the environment
    variable CSRK_CHECKS=1, the bounds-checked build libcsrk_checks.so instead."""
    global _LIB
    if _LIB is None:
        checks = os.environ.get("CSRK_CHECKS") == "1"
        path = _build.LIB_CHECKS if checks else _build.LIB
        if build_if_missing:
            path = _build.build(checks=checks)
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not found at {path}; run __graft_entry__.build()")
        h = ctypes.CDLL(path)
        for name, args in _PROTOS.items():
            fn = getattr(h, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        h.csrk_last_error.argtypes = []
        h.csrk_last_error.restype = ctypes.c_char_p
        h.csrk_build_info.argtypes = []
        h.csrk_build_info.restype = ctypes.c_char_p
        _LIB = h
    return _LIB


def _check(rc: int, func: str):
    if rc != 0:
        msg = lib().csrk_last_error().decode(errors="replace")
        raise CsrkError(rc, msg, func)


def _host(a, dtype):
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(_vp)


def _ptr(t):
    """Device (torch tensor) or host (numpy array) pointer of a vector argument."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("host vectors must be C-contiguous")
        return t.ctypes.data
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return int(t)


def _stream(stream, *tensors):
    if stream is not None:
        return int(stream) if not hasattr(stream, "cuda_stream") else stream.cuda_stream
    for t in tensors:
        if hasattr(t, "is_cuda") and t.is_cuda:
            import torch
            return torch.cuda.current_stream(t.device).cuda_stream
    return None


# ------------------------------------------------------------------ entry points
def create(n, rowptr, colidx, vals, dtype="f64"):
    rp, prp = _host(rowptr, np.int32)
    ci, pci = _host(colidx, np.int32)
    va, pva = _host(vals, np.float64)
    if rp.size != n + 1:
        raise ValueError("rowptr must have n + 1 entries")
    out = _vp()
    _check(lib().csrk_create(int(n), prp, pci, pva, DTYPES[dtype], ctypes.byref(out)), "csrk_create")
    return out.value


def reorder(h, method="rcm", want_perm=True):
    n = info(h)["n"]
    perm = np.empty(n, dtype=np.int32) if want_perm else None
    _check(lib().csrk_reorder(h, REORDER[method], None if perm is None else perm.ctypes.data_as(_vp)),
           "csrk_reorder")
    return perm


def split_long_rows(h, min_len):
    """Move rows with at least min_len entries behind the super-rows; returns their count."""
    v = ctypes.c_int32()
    _check(lib().csrk_split_long_rows(h, int(min_len), ctypes.byref(v)), "csrk_split_long_rows")
    return v.value


def reorder_bandk(h, sr, ssr, want_perm=True):
    """Band-k ordering with its variable super-row / super-super-row pointers."""
    n = info(h)["n"]
    perm = np.empty(n, dtype=np.int32) if want_perm else None
    _check(lib().csrk_reorder_bandk(h, int(sr), int(ssr), None if perm is None else perm.ctypes.data_as(_vp)),
           "csrk_reorder_bandk")
    return perm


def set_sizes(h, sr, ssr):
    _check(lib().csrk_set_sizes(h, int(sr), int(ssr)), "csrk_set_sizes")


def index_bits(h):
    v = ctypes.c_int32()
    _check(lib().csrk_index_bits(h, ctypes.byref(v)), "csrk_index_bits")
    return v.value


def set_pointers(h, sr_ptr, ssr_ptr):
    a, pa = _host(sr_ptr, np.int32)
    b, pb = _host(ssr_ptr, np.int32)
    _check(lib().csrk_set_pointers(h, a.size - 1, pa, b.size - 1, pb), "csrk_set_pointers")


def spmv(h, alpha, x, beta, y, flags=0, stream=None):
    _check(lib().csrk_spmv(h, float(alpha), _ptr(x), float(beta), _ptr(y), int(flags),
                           _stream(stream, x, y)), "csrk_spmv")


def spmm(h, k, alpha, X, ldx, beta, Y, ldy, flags=0, stream=None):
    _check(lib().csrk_spmm(h, int(k), float(alpha), _ptr(X), int(ldx), float(beta), _ptr(Y),
                           int(ldy), int(flags), _stream(stream, X, Y)), "csrk_spmm")


def permute(h, direction, k, inp, ldi, out, ldo, flags=0, stream=None):
    _check(lib().csrk_permute(h, int(direction), int(k), _ptr(inp), int(ldi), _ptr(out), int(ldo),
                              int(flags), _stream(stream, inp, out)), "csrk_permute")


def destroy(h):
    if h:
        _check(lib().csrk_destroy(h), "csrk_destroy")


def info(h):
    v = [ctypes.c_int32() for _ in range(6)]
    nnz = ctypes.c_int64()
    _check(lib().csrk_info(h, ctypes.byref(v[0]), ctypes.byref(nnz), ctypes.byref(v[1]),
                           ctypes.byref(v[2]), ctypes.byref(v[3]), ctypes.byref(v[4]),
                           ctypes.byref(v[5])), "csrk_info")
    return dict(n=v[0].value, nnz=nnz.value, nsr=v[1].value, nssr=v[2].value, sr=v[3].value,
                ssr=v[4].value, dtype=v[5].value)


def export(h, with_pointers=True):
    d = info(h)
    n, nnz = d["n"], d["nnz"]
    perm = np.empty(n, np.int32)
    rowptr = np.empty(n + 1, np.int32)
    colidx = np.empty(nnz, np.int32)
    vals = np.empty(nnz, np.float64)
    srp = np.empty(d["nsr"] + 1, np.int32) if with_pointers else None
    ssrp = np.empty(d["nssr"] + 1, np.int32) if with_pointers else None
    p = lambda a: None if a is None else a.ctypes.data_as(_vp)
    _check(lib().csrk_export(h, p(perm), p(rowptr), p(colidx), p(vals), p(srp), p(ssrp)), "csrk_export")
    return dict(perm=perm, rowptr=rowptr, colidx=colidx, vals=vals, sr_ptr=srp, ssr_ptr=ssrp)


def export_values(h, dtype):
    nnz = info(h)["nnz"]
    dt = {F64: np.float64, F32: np.float32, BF16: np.uint16}[DTYPES[dtype]]
    out = np.empty(nnz, dt)
    _check(lib().csrk_export_values(h, DTYPES[dtype], out.ctypes.data_as(_vp)), "csrk_export_values")
    return out


def model_sizes(rdensity, arch="ampere"):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().csrk_model_sizes(float(rdensity), {"volta": 0, "ampere": 1}.get(arch, arch),
                                  ctypes.byref(a), ctypes.byref(b)), "csrk_model_sizes")
    return a.value, b.value


def tuned_config(h):
    v = [ctypes.c_int32() for _ in range(6)]
    _check(lib().csrk_tuned_config(h, *[ctypes.byref(t) for t in v]), "csrk_tuned_config")
    return dict(zip(("kernel", "lanes", "unroll", "warps", "stages", "ctas"), (t.value for t in v)))


def xwin_info(h):
    """The x windows of kernels 5 and 6: dict(available, runs, max_window, row_order)."""
    av, mw, ro = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    runs = ctypes.c_int64()
    _check(lib().csrk_xwin_info(h, ctypes.byref(av), ctypes.byref(runs), ctypes.byref(mw), ctypes.byref(ro)),
           "csrk_xwin_info")
    return dict(available=bool(av.value), runs=runs.value, max_window=mw.value, row_order=bool(ro.value))


def xwin_export(h):
    """The x windows and rows' length order, built on the host (csrk_xwin_export): dict(available,
    wptr, win (runs x 2), cover, codes, ord, slots=(natural, ordered))."""
    d = info(h)
    av, nr = ctypes.c_int32(), ctypes.c_int64()
    p = lambda a: a.ctypes.data_as(_vp)
    _check(lib().csrk_xwin_export(h, ctypes.byref(av), ctypes.byref(nr), None, None, None, None, None, None),
           "csrk_xwin_export")
    wptr = np.zeros(d["nssr"] + 1, np.int32)
    win = np.zeros((max(nr.value, 0), 2), np.int32)
    cover = np.zeros(d["nssr"], np.int32)
    codes = np.zeros(d["nnz"], np.uint16)
    covered = int(export(h)["sr_ptr"][-1]) if d["nsr"] else 0
    ord_ = np.zeros(covered, np.uint16)
    slots = np.zeros(2, np.int64)
    _check(lib().csrk_xwin_export(h, ctypes.byref(av), ctypes.byref(nr), p(wptr), p(win), p(cover), p(codes),
                                  p(ord_), p(slots)), "csrk_xwin_export")
    return dict(available=bool(av.value), wptr=wptr, win=win, cover=cover, codes=codes, ord=ord_,
                slots=(int(slots[0]), int(slots[1])))


def col16_export(h):
    """Kernel 4's delta-coded columns built on the host (csrk_col16_export): dict(codes, cbase)."""
    d = info(h)
    codes = np.zeros(d["nnz"], np.uint16)
    cbase = np.zeros(d["nssr"], np.int32)
    _check(lib().csrk_col16_export(h, codes.ctypes.data_as(_vp), cbase.ctypes.data_as(_vp)), "csrk_col16_export")
    return dict(codes=codes, cbase=cbase)


def stage_plan(max_srs, max_rows, max_nnz, val_bytes, col_bytes, max_smem, want_stages=0, x_bytes=0,
               with_ord=False):
    """The TMA kernels' shared-memory stage layout (csrk_selftest_stage_plan) as a dict."""
    out = np.zeros(10, np.uint32)
    _check(lib().csrk_selftest_stage_plan(int(max_srs), int(max_rows), int(max_nnz), int(val_bytes),
                                          int(col_bytes), int(max_smem), int(want_stages), int(x_bytes),
                                          int(bool(with_ord)), out.ctypes.data_as(_vp)), "csrk_selftest_stage_plan")
    keys = ("off_srp", "off_rp", "off_col", "off_val", "off_x", "off_perm", "off_ord", "stage_bytes",
            "header_bytes", "stages")
    return dict(zip(keys, (int(v) for v in out)))


def set_config(h, kernel=-1, lanes=-1, unroll=-1, warps=-1, stages=-1, ctas=-1):
    _check(lib().csrk_set_config(h, kernel, lanes, unroll, warps, stages, ctas), "csrk_set_config")


def device_status(h, stream=None):
    st = ctypes.c_int32()
    rc = lib().csrk_device_status(h, _stream(stream), ctypes.byref(st))
    if rc not in (0, 7):
        _check(rc, "csrk_device_status")
    return st.value


def cg(h, b, x, rtol=1e-10, maxit=10000, inner="f64", replace_every=20, restart=0, flags=0,
       stream=None, check=True):
    """Solve A x = b; returns (status, iterations, true relative residual)."""
    it = ctypes.c_int32()
    rel = ctypes.c_double()
    rc = lib().csrk_cg(h, _ptr(b), _ptr(x), float(rtol), int(maxit), DTYPES[inner], int(replace_every),
                       int(restart), int(flags), ctypes.byref(it), ctypes.byref(rel), _stream(stream, b, x))
    if check and rc not in (0, 8):
        _check(rc, "csrk_cg")
    return rc, it.value, rel.value


def batch_create(handles, ks):
    hs = (_vp * len(handles))(*handles)
    k, pk = _host(ks, np.int32)
    out = _vp()
    _check(lib().csrk_batch_create(hs, len(handles), pk, ctypes.byref(out)), "csrk_batch_create")
    return out.value


def _ptr_array(ts):
    return (_vp * len(ts))(*[_ptr(t) for t in ts])


def batch_spmm(b, alpha, Xs, beta, Ys, flags=VEC_PERMUTED, stream=None):
    _check(lib().csrk_batch_spmm(b, float(alpha), _ptr_array(Xs), float(beta), _ptr_array(Ys), int(flags),
                                 _stream(stream, *Xs)), "csrk_batch_spmm")


def batch_info(b):
    v = [ctypes.c_int32() for _ in range(3)]
    t = ctypes.c_int64()
    _check(lib().csrk_batch_info(b, *[ctypes.byref(x) for x in v], ctypes.byref(t)), "csrk_batch_info")
    return dict(nmat=v[0].value, nsys=v[1].value, ntiles=v[2].value, total=t.value)


def batch_plan(b):
    v = [ctypes.c_int32() for _ in range(3)]
    _check(lib().csrk_batch_plan(b, *[ctypes.byref(x) for x in v]), "csrk_batch_plan")
    return dict(items=v[0].value, stages=v[1].value, stage_bytes=v[2].value)


def batch_device_status(b):
    v = ctypes.c_int32()
    _check(lib().csrk_batch_device_status(b, ctypes.byref(v)), "csrk_batch_device_status")
    return v.value


def batch_cg(b, Bs, Xs, iters, rtol=1e-10, stream=None):
    """Returns (relres per system, iterations per system)."""
    nsys = batch_info(b)["nsys"]
    rel = np.empty(nsys, np.float64)
    its = np.empty(nsys, np.int32)
    _check(lib().csrk_batch_cg(b, _ptr_array(Bs), _ptr_array(Xs), int(iters), float(rtol),
                               rel.ctypes.data_as(_vp), its.ctypes.data_as(_vp), _stream(stream, *Bs)),
           "csrk_batch_cg")
    return rel, its


def batch_cg_solve(b, Bs, Xs, rtol=1e-10, maxit=2000, inner="f64", replace_every=20, restart=0,
                   stream=None, check=True):
    """CG to rtol for every system of the batch; returns (status, relres, iterations, cycles)
    with one relres / iteration count per system (matrix-major, then column)."""
    nsys = batch_info(b)["nsys"]
    rel = np.empty(nsys, np.float64)
    its = np.empty(nsys, np.int32)
    cyc = ctypes.c_int32()
    rc = lib().csrk_batch_cg_solve(b, _ptr_array(Bs), _ptr_array(Xs), float(rtol), int(maxit), DTYPES[inner],
                                   int(replace_every), int(restart), rel.ctypes.data_as(_vp),
                                   its.ctypes.data_as(_vp), ctypes.byref(cyc), _stream(stream, *Bs))
    if check and rc not in (0, 8):
        _check(rc, "csrk_batch_cg_solve")
    return rc, rel, its, cyc.value


def batch_destroy(b):
    if b:
        _check(lib().csrk_batch_destroy(b), "csrk_batch_destroy")


def spmv_static_scratch(n, nssr, ssr_ptr, sr_ptr, rowptr, colidx, vals, perm, alpha, x, beta, y,
                        stream=None):
    """Allocation-free SpMV (all arrays device tensors, e.g. from csrk.export)."""
    _check(lib().csrk_spmv_static_scratch(int(n), int(nssr), _ptr(ssr_ptr), _ptr(sr_ptr),
                                          _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(perm),
                                          float(alpha), _ptr(x), float(beta), _ptr(y),
                                          _stream(stream, x, y)), "csrk_spmv_static_scratch")


def selftest_bounded_wait(h, timeout_ns=20_000_000, stream=None):
    """Returns (status code, status word) of a wait that nothing completes."""
    st = ctypes.c_int32()
    rc = lib().csrk_selftest_bounded_wait(h, int(timeout_ns), _stream(stream), ctypes.byref(st))
    return rc, st.value


def selftest_narrow(x, by_int, by_cvt, stream=None):
    """Device FP64 -> FP32 narrowing of x two ways (integer rounding, conversion instruction)."""
    _check(lib().csrk_selftest_narrow(_ptr(x), int(x.numel()), _ptr(by_int), _ptr(by_cvt),
                                      _stream(stream, x)), "csrk_selftest_narrow")


def build_info() -> str:
    return lib().csrk_build_info().decode()


class Matrix:
    """Owning wrapper: ``Matrix(csr, dtype)``; frees the handle when collected."""

    def __init__(self, n, rowptr, colidx, vals, dtype="f64"):
        self.h = create(n, rowptr, colidx, vals, dtype)

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h and _LIB is not None:
            _LIB.csrk_destroy(h)

    def close(self):
        destroy(self.h)
        self.h = None
