"""ctypes binding of ``include/flycoo.h``: one Python function per C entry
point, same name, argument marshalling only (torch tensors -> device
pointers, the current torch stream -> cudaStream_t).  Every computation runs
in the CUDA library; there is no fallback.  A missing library raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np
import torch  # loads the CUDA runtime the library shares

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libflycoo.so")
MAX_MODES = 8

OK = 0
STATUS_NAMES = {
    0: "FLYCOO_OK", 1: "FLYCOO_ERR_INVALID_ARG", 2: "FLYCOO_ERR_INDEX_RANGE", 3: "FLYCOO_ERR_OOM",
    4: "FLYCOO_ERR_LAYOUT", 5: "FLYCOO_ERR_NOT_SPD", 6: "FLYCOO_ERR_TIMEOUT", 7: "FLYCOO_ERR_CUDA",
    8: "FLYCOO_ERR_UNSUPPORTED",
}
F32 = 0
BF16 = 1


class FlycooError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.status_name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{self.status_name}: {message}")


class flycoo_params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64 * MAX_MODES), ("g", ctypes.c_uint64), ("bins", ctypes.c_uint32),
                ("schedule", ctypes.c_uint32), ("order", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class flycoo_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("layout_mode", ctypes.c_int32), ("nnz", ctypes.c_uint64),
                ("dims", ctypes.c_uint64 * MAX_MODES), ("m", ctypes.c_uint64 * MAX_MODES),
                ("g", ctypes.c_uint64), ("bins", ctypes.c_uint32), ("elem_bytes", ctypes.c_uint32),
                ("schedule", ctypes.c_uint32), ("order", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("super_shards", ctypes.c_uint64 * MAX_MODES), ("shards", ctypes.c_uint64 * MAX_MODES),
                ("segments", ctypes.c_uint64 * MAX_MODES),
                ("fixup_super_shards", ctypes.c_uint64 * MAX_MODES), ("device_bytes", ctypes.c_uint64)]


_lib = None


def lib():
    """Load ``libflycoo.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libflycoo.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I, U64, U32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32
        sigs = {
            "flycoo_create": [I, P, U64, P, P, P, P, P],
            "flycoo_destroy": [P],
            "flycoo_spmttkrp": [P, I, P, I, I, P, I, P],
            "flycoo_spmttkrp_static_scratch": [P, I, P, I, I, P, I, P],
            "flycoo_remap": [P, I, P],
            "flycoo_sync": [P, P],
            "flycoo_all_modes_host": [P, P, I, I, P, P],
            "flycoo_mttkrp_adjoint": [P, I, P, I, I, P, P, P, P],
            "flycoo_cpopt_grad": [P, P, I, P, P, P],
            "flycoo_cp_als_step": [P, P, I, I, P, P, P],
            "flycoo_cp_als": [P, P, I, I, I, P, P, P],
            "flycoo_get_info": [P, P],
            "flycoo_export_layout": [P, P, P, P],
            "flycoo_export_partition": [P, I, P, P, P],
            "flycoo_export_schedule": [P, I, I, P, P],
            "flycoo_export_next": [P, I, P, P],
            "flycoo_export_tile_order": [P, I, I, P, P],
            "flycoo_timing_enable": [P, I],
            "flycoo_timing_read": [P, P, P],
            "flycoo_last_error": [],
            "flycoo_debug_set_wait_limit": [P, ctypes.c_int64],
            "flycoo_debug_fail_alloc_after": [ctypes.c_int64],
            "flycoo_plan_create": [U64, U64, P, U64, U32, U32, P],
            "flycoo_plan_get": [P, I, P, P],
            "flycoo_plan_destroy": [P],
        }
        for name, args in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.flycoo_destroy.restype = None
        L.flycoo_plan_destroy.restype = None
        L.flycoo_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def flycoo_last_error() -> str:
    return lib().flycoo_last_error().decode()


def _check(status: int):
    if status != OK:
        raise FlycooError(status, flycoo_last_error())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev_ptr(t: torch.Tensor, dtypes, what: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise TypeError(f"{what} has dtype {t.dtype}, expected one of {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


SCHEDULE_LPT = 0
SCHEDULE_BLOCK_CYCLIC = 1
ORDER_KEY = 0
ORDER_MORTON = 1


def make_params(m: Optional[Sequence[int]] = None, g: int = 0, bins: int = 0,
                schedule: int = SCHEDULE_LPT, order: int = ORDER_KEY) -> flycoo_params:
    p = flycoo_params()
    for i, v in enumerate(m or []):
        p.m[i] = int(v)
    p.g = int(g)
    p.bins = int(bins)
    p.schedule = int(schedule)
    p.order = int(order)
    return p


def flycoo_create(N: int, dims: Sequence[int], nnz: int, idx: torch.Tensor, vals: torch.Tensor,
                  params: Optional[flycoo_params] = None, stream=None) -> ctypes.c_void_p:
    """``idx``: int32/uint32 CUDA tensor [N, nnz] (mode-major); ``vals`` float32 [nnz]."""
    h = ctypes.c_void_p()
    d = (ctypes.c_uint64 * len(dims))(*[int(x) for x in dims])
    pi = _dev_ptr(idx, (torch.int32, getattr(torch, "uint32", torch.int32)), "idx") if nnz else None
    pv = _dev_ptr(vals, (torch.float32,), "vals") if nnz else None
    if nnz and (idx.numel() != N * nnz or vals.numel() != nnz):
        raise ValueError("idx must hold N*nnz coordinates and vals nnz values")
    _check(lib().flycoo_create(int(N), d, int(nnz), pi, pv,
                               ctypes.byref(params) if params is not None else None, _stream(stream),
                               ctypes.byref(h)))
    return h


def flycoo_destroy(h) -> None:
    if h:
        lib().flycoo_destroy(h)


def flycoo_spmttkrp(h, mode: int, factors: Sequence[Optional[torch.Tensor]], out: torch.Tensor,
                    next_mode: int = -1, stream=None) -> None:
    """``factors``: one CUDA tensor [I_w, R] per mode (float32 or bfloat16; the
    entry of ``mode`` may be None); ``out``: float32 [I_mode, R]."""
    N = len(factors)
    ptrs = (ctypes.c_void_p * N)()
    fdt = None
    R = None
    for w, f in enumerate(factors):
        if w == mode or f is None:
            continue
        ptrs[w] = _dev_ptr(f, (torch.float32, torch.bfloat16), f"factor {w}")
        dt = BF16 if f.dtype == torch.bfloat16 else F32
        if fdt is not None and dt != fdt:
            raise TypeError("all factors must share one dtype")
        fdt = dt
        if f.dim() != 2 or (R is not None and f.shape[1] != R):
            raise ValueError("factors must be 2-D with a common rank")
        R = f.shape[1]
    if R is None:
        raise ValueError("no input factor given")
    po = _dev_ptr(out, (torch.float32,), "out")
    if out.dim() != 2 or out.shape[1] != R:
        raise ValueError("out must be [I_mode, R]")
    _check(lib().flycoo_spmttkrp(h, int(mode), ptrs, int(fdt), int(R), po, int(next_mode), _stream(stream)))


def flycoo_spmttkrp_static_scratch(h, mode: int, factors: Sequence[Optional[torch.Tensor]],
                                   out: torch.Tensor, next_mode: int = -1, stream=None) -> None:
    """As ``flycoo_spmttkrp``, with the partial rows in the library's fixed
    8 MiB device array; the call allocates nothing (see include/flycoo.h)."""
    ptrs, fdt, R, po = _spmttkrp_args(mode, factors, out)
    _check(lib().flycoo_spmttkrp_static_scratch(h, int(mode), ptrs, int(fdt), int(R), po, int(next_mode),
                                                _stream(stream)))


def _spmttkrp_args(mode, factors, out):
    N = len(factors)
    ptrs = (ctypes.c_void_p * N)()
    fdt = None
    R = None
    for w, f in enumerate(factors):
        if w == mode or f is None:
            continue
        ptrs[w] = _dev_ptr(f, (torch.float32, torch.bfloat16), f"factor {w}")
        dt = BF16 if f.dtype == torch.bfloat16 else F32
        if fdt is not None and dt != fdt:
            raise TypeError("all factors must share one dtype")
        fdt = dt
        if f.dim() != 2 or (R is not None and f.shape[1] != R):
            raise ValueError("factors must be 2-D with a common rank")
        R = f.shape[1]
    if R is None:
        raise ValueError("no input factor given")
    po = _dev_ptr(out, (torch.float32,), "out")
    if out.dim() != 2 or out.shape[1] != R:
        raise ValueError("out must be [I_mode, R]")
    return ptrs, fdt, R, po


def _ptr_array(tensors, dtypes, what, skip=-1, allow_none=False):
    arr = (ctypes.c_void_p * len(tensors))()
    for w, t in enumerate(tensors):
        if w == skip or (allow_none and t is None):
            continue
        arr[w] = _dev_ptr(t, dtypes, f"{what} {w}")
    return arr


def flycoo_mttkrp_adjoint(h, mode: int, factors: Sequence[Optional[torch.Tensor]], gout: torch.Tensor,
                          gfactors: Sequence[Optional[torch.Tensor]], gvals: Optional[torch.Tensor] = None,
                          stream=None) -> None:
    """dY_w = spMTTKRP_w(X, Y with Y_mode := gout) into ``gfactors[w]`` (FP32;
    None entries skipped) and, when ``gvals`` is given (float32 [nnz]), the
    gradient with respect to each nonzero value in the input COO order.
    ``factors`` and ``gout`` share one dtype, float32 or bfloat16."""
    R = gout.shape[1]
    dt = gout.dtype
    if dt not in (torch.float32, torch.bfloat16):
        raise TypeError("gout must be float32 or bfloat16")
    F = _ptr_array(factors, (dt,), "factor", skip=mode, allow_none=True)
    Gp = _dev_ptr(gout, (dt,), "gout")
    GF = _ptr_array(gfactors, (torch.float32,), "gradient", skip=mode, allow_none=True)
    Vp = _dev_ptr(gvals, (torch.float32,), "gvals") if gvals is not None else None
    _check(lib().flycoo_mttkrp_adjoint(h, int(mode), F, BF16 if dt == torch.bfloat16 else F32, int(R), Gp, GF,
                                       Vp, _stream(stream)))


def flycoo_cpopt_grad(h, factors: Sequence[torch.Tensor], grads: Sequence[torch.Tensor], stream=None,
                      want_loss: bool = True):
    """CP-OPT loss 1/2 sum (x - m_x)^2 over the nonzeros and its gradients
    (written to ``grads``); returns the loss (float) or None."""
    R = factors[0].shape[1]
    F = _ptr_array(factors, (torch.float32,), "factor")
    Gr = _ptr_array(grads, (torch.float32,), "gradient")
    loss = ctypes.c_double()
    _check(lib().flycoo_cpopt_grad(h, F, int(R), Gr, ctypes.byref(loss) if want_loss else None,
                                   _stream(stream)))
    return loss.value if want_loss else None


def flycoo_cp_als_step(h, factors: Sequence[torch.Tensor], lam: torch.Tensor, stream=None) -> float:
    """One CP-ALS iteration: updates ``factors`` (all FP32 or all BF16) in
    place, writes the last mode's column norms to ``lam`` (R float64 on the
    device) and returns the fit."""
    R = factors[0].shape[1]
    dt = factors[0].dtype
    if dt not in (torch.float32, torch.bfloat16) or any(f.dtype != dt for f in factors):
        raise TypeError("factors must all be float32 or all bfloat16")
    F = _ptr_array(factors, (dt,), "factor")
    Lp = _dev_ptr(lam, (torch.float64,), "lambda")
    if lam.numel() < R:
        raise ValueError(f"lambda holds {lam.numel()} values, R = {R}")
    fit = ctypes.c_double()
    _check(lib().flycoo_cp_als_step(h, F, BF16 if dt == torch.bfloat16 else F32, int(R), Lp, ctypes.byref(fit),
                                    _stream(stream)))
    return fit.value


def flycoo_cp_als(h, factors: Sequence[torch.Tensor], lam: torch.Tensor, iters: int, stream=None) -> List[float]:
    """``iters`` CP-ALS iterations in one call (the Gram matrices carried from
    one iteration to the next); returns the fit after each iteration."""
    R = factors[0].shape[1]
    dt = factors[0].dtype
    if dt not in (torch.float32, torch.bfloat16) or any(f.dtype != dt for f in factors):
        raise TypeError("factors must all be float32 or all bfloat16")
    F = _ptr_array(factors, (dt,), "factor")
    Lp = _dev_ptr(lam, (torch.float64,), "lambda")
    if lam.numel() < R:
        raise ValueError(f"lambda holds {lam.numel()} values, R = {R}")
    fits = (ctypes.c_double * int(iters))()
    _check(lib().flycoo_cp_als(h, F, BF16 if dt == torch.bfloat16 else F32, int(R), int(iters), Lp, fits,
                               _stream(stream)))
    return list(fits)


def flycoo_debug_set_wait_limit(h, polls: int) -> None:
    """Test hook: barrier polls before a fused pass gives up (negative = default)."""
    _check(lib().flycoo_debug_set_wait_limit(h, int(polls)))


def flycoo_debug_fail_alloc_after(n: int) -> None:
    """Test hook: the allocation after the next ``n`` fails (negative = off)."""
    _check(lib().flycoo_debug_fail_alloc_after(int(n)))


def flycoo_remap(h, next_mode: int, stream=None) -> None:
    _check(lib().flycoo_remap(h, int(next_mode), _stream(stream)))


def flycoo_all_modes_host(h, factors: Sequence[torch.Tensor], outs: Sequence[torch.Tensor], stream=None) -> None:
    """All-mode spMTTKRP from host memory: ``factors`` are CPU tensors
    [I_w, R] (float32 or bfloat16, pinned for asynchronous copies), ``outs``
    CPU float32 tensors [I_n, R], overwritten.  Waits for the stream."""
    N = len(factors)
    dt = factors[0].dtype
    R = factors[0].shape[1]
    F = (ctypes.c_void_p * N)()
    O = (ctypes.c_void_p * N)()
    for w in range(N):
        f, o = factors[w], outs[w]
        if f.is_cuda or o.is_cuda or f.dtype != dt or o.dtype != torch.float32:
            raise TypeError("factors (one dtype) and float32 outputs must be CPU tensors")
        if not f.is_contiguous() or not o.is_contiguous() or f.shape[1] != R or o.shape[1] != R:
            raise ValueError("contiguous [I, R] tensors with one rank are required")
        F[w] = ctypes.c_void_p(f.data_ptr())
        O[w] = ctypes.c_void_p(o.data_ptr())
    _check(lib().flycoo_all_modes_host(h, F, BF16 if dt == torch.bfloat16 else F32, int(R), O, _stream(stream)))


def flycoo_sync(h, stream=None) -> None:
    """Wait for the stream; raise FLYCOO_ERR_TIMEOUT if a bounded device wait gave up."""
    _check(lib().flycoo_sync(h, _stream(stream)))


def flycoo_get_info(h) -> dict:
    info = flycoo_info()
    _check(lib().flycoo_get_info(h, ctypes.byref(info)))
    N = info.N
    return dict(N=N, layout_mode=info.layout_mode, nnz=info.nnz, dims=list(info.dims[:N]),
                m=list(info.m[:N]), g=info.g, bins=info.bins, elem_bytes=info.elem_bytes,
                super_shards=list(info.super_shards[:N]), shards=list(info.shards[:N]),
                segments=list(info.segments[:N]),
                fixup_super_shards=list(info.fixup_super_shards[:N]), device_bytes=info.device_bytes,
                schedule=info.schedule, order=info.order)


def flycoo_export_layout(h, stream=None):
    inf = flycoo_get_info(h)
    N, nnz = inf["N"], inf["nnz"]
    idx = torch.empty((N, nnz), dtype=torch.int32, device="cuda")
    vals = torch.empty(nnz, dtype=torch.float32, device="cuda")
    _check(lib().flycoo_export_layout(h, ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                      _stream(stream)))
    return idx, vals


def flycoo_export_partition(h, mode: int):
    """``(ss_ptr, shard_ptr, shard_ss)`` of ``mode`` (Section III-A)."""
    inf = flycoo_get_info(h)
    k, S = inf["super_shards"][mode], inf["shards"][mode]
    ss = np.empty(k + 1, dtype=np.uint64)
    sp = np.empty(S + 1, dtype=np.uint64)
    sss = np.empty(S, dtype=np.uint32)
    _check(lib().flycoo_export_partition(h, int(mode), ss.ctypes.data, sp.ctypes.data, sss.ctypes.data))
    return ss, sp, sss


def flycoo_export_schedule(h, mode: int, which: int):
    inf = flycoo_get_info(h)
    n_items = inf["super_shards"][mode] if which == 0 else inf["shards"][mode]
    bp = np.empty(inf["bins"] + 1, dtype=np.uint64)
    it = np.empty(n_items, dtype=np.uint64)
    _check(lib().flycoo_export_schedule(h, int(mode), int(which), bp.ctypes.data, it.ctypes.data))
    return bp, it


def flycoo_export_next(h, mode: int, stream=None) -> torch.Tensor:
    nnz = flycoo_get_info(h)["nnz"]
    nx = torch.empty(nnz, dtype=torch.int32, device="cuda")
    _check(lib().flycoo_export_next(h, int(mode), ctypes.c_void_p(nx.data_ptr()), _stream(stream)))
    return nx


def flycoo_export_tile_order(h, mode: int, stage: int, stream=None) -> torch.Tensor:
    """Compute order of the stage tiles of ``mode`` for stage size 512 or
    1024 (int16 holding uint16 tile-local indexes, one per position)."""
    nnz = flycoo_get_info(h)["nnz"]
    out = torch.empty(nnz, dtype=torch.int16, device="cuda")
    _check(lib().flycoo_export_tile_order(h, int(mode), int(stage), ctypes.c_void_p(out.data_ptr()),
                                          _stream(stream)))
    return out


def flycoo_timing_enable(h, enable: bool = True) -> None:
    _check(lib().flycoo_timing_enable(h, 1 if enable else 0))


def flycoo_timing_read(h):
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(lib().flycoo_timing_read(h, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


PLAN_G = 0
PLAN_SHARD_PTR = 1
PLAN_SHARD_SS = 2
PLAN_SS_SHARD_PTR = 3
PLAN_SS_BIN_PTR = 4
PLAN_SS_ITEMS = 5
PLAN_SHARD_BIN_PTR = 6
PLAN_SHARD_ITEMS = 7
PLAN_K4_ITEMS = 8
PLAN_TILE_BIN_PTR_512 = 9
PLAN_TILES_512 = 10
PLAN_TILE_BIN_PTR_1024 = 11
PLAN_TILES_1024 = 12
PLAN_SEG_SS = 13
PLAN_SS_SEG_PTR = 14
PLAN_K4_ORDER = 15
PLAN_K4_NLIGHT = 16


def flycoo_plan_create(nnz: int, ss_ptr, g: int = 0, bins: int = 1, schedule: int = SCHEDULE_LPT):
    """Host-only plan of one mode from its super-shard pointers (no device)."""
    ss = np.ascontiguousarray(ss_ptr, dtype=np.uint64)
    if ss.ndim != 1 or ss.size < 2:
        raise ValueError("ss_ptr needs k + 1 >= 2 entries")
    out = ctypes.c_void_p()
    _check(lib().flycoo_plan_create(int(nnz), int(ss.size - 1), ss.ctypes.data, int(g), int(bins),
                                    int(schedule), ctypes.byref(out)))
    return out


def flycoo_plan_get(plan, which: int) -> np.ndarray:
    n = ctypes.c_uint64(0)
    _check(lib().flycoo_plan_get(plan, int(which), None, ctypes.byref(n)))
    buf = np.empty(n.value, dtype=np.uint64)
    _check(lib().flycoo_plan_get(plan, int(which), buf.ctypes.data, ctypes.byref(n)))
    return buf


def flycoo_plan_destroy(plan) -> None:
    lib().flycoo_plan_destroy(plan)


def header_functions(header: Optional[str] = None) -> List[str]:
    """Names of the functions ``include/flycoo.h`` declares."""
    import re
    header = header or os.path.join(os.path.dirname(HERE), "include", "flycoo.h")
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(flycoo_[a-z_0-9]+)\s*\(", src)))
