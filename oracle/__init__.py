"""FP64 CPU oracle for FLYCOO spMTTKRP -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and it imports nothing from the product.
It is written from the paper (Wijeratne, Kannan, Prasanna, "Dynasor: A
Dynamic Memory Layout for Accelerating Sparse MTTKRP for Tensor Decomposition
on Multi-core CPU", arXiv 2309.09131); each function names the passage it
follows.

The arithmetic loops live in ``flycoo_oracle.c`` (plain C, FP64, sequential
in COO order); this module loads it with ctypes and adds the definitions that
are plain array bookkeeping (inverse permutations, CSR lists of bins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flycoo_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

__all__ = [
    "build", "mttkrp", "mttkrp_threads", "mttkrp_rows", "sampled", "layout_order", "layout_order_qsort", "layout_order_morton",
    "morton_code", "inverse", "partition",
    "lpt", "lpt_bins", "round_bf16", "factors_f64", "flycoo_layout", "remap",
]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (plain gcc, no CUDA)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        U64 = ctypes.c_uint64
        I = ctypes.c_int
        lib.oracle_mttkrp.argtypes = [I, P, U64, P, P, P, I, I, P]
        lib.oracle_mttkrp_rows.argtypes = [I, P, U64, P, P, P, I, I, U64, P, P]
        lib.oracle_mttkrp_threads.argtypes = [I, P, U64, P, P, P, I, I, I, P]
        lib.oracle_sampled.argtypes = [I, U64, P, P, I, P]
        lib.oracle_layout_order.argtypes = [I, U64, P, P, I, P]
        lib.oracle_partition.argtypes = [U64, U64, P, U64, U64, P, P, U64, P]
        lib.oracle_lpt.argtypes = [U64, P, U64, P, P, P]
        lib.oracle_round_bf16.argtypes = [U64, P, P]
        lib.oracle_round_bf16.restype = None
        for f in ("oracle_mttkrp", "oracle_mttkrp_rows", "oracle_mttkrp_threads", "oracle_sampled", "oracle_layout_order",
                  "oracle_partition", "oracle_lpt"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _coo(idx):
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    assert idx.ndim == 2
    return idx


def _dims(idx, dims):
    if dims is None:
        dims = [int(idx[w].max()) + 1 if idx.shape[1] else 1 for w in range(idx.shape[0])]
    return np.ascontiguousarray(dims, dtype=np.uint64)


def _fptrs(F):
    F = [np.ascontiguousarray(f, dtype=np.float64) for f in F]
    arr = (ctypes.c_void_p * len(F))(*[f.ctypes.data for f in F])
    return F, arr


def factors_f64(factors: Sequence[np.ndarray], bf16: bool = False) -> List[np.ndarray]:
    """Widen float32 factors to float64 exactly; with ``bf16`` round them to
    bfloat16 first (round-to-nearest-even), as BF16 factor storage does."""
    out = []
    for f in factors:
        f = np.ascontiguousarray(f, dtype=np.float32)
        if bf16:
            f = round_bf16(f)
        out.append(f.astype(np.float64))
    return out


def mttkrp(idx, vals, factors, mode: int, dims=None) -> np.ndarray:
    """spMTTKRP of ``mode`` (Section II-C; the elementwise equation of Section IV, Eq. 4).

    ``factors`` are ``[I_w, R]`` arrays (float64 after exact widening); the
    factor of ``mode`` itself is not read.  Returns ``[I_mode, R]`` float64.
    """
    lib = _load()
    idx = _coo(idx)
    N, nnz = idx.shape
    d = _dims(idx, dims)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    F, arr = _fptrs(factors)
    R = F[0].shape[1]
    M = np.empty((int(d[mode]), R), dtype=np.float64)
    rc = lib.oracle_mttkrp(N, _ptr(d), nnz, _ptr(idx), _ptr(vals), arr, R, mode, _ptr(M))
    if rc:
        raise ValueError(f"oracle_mttkrp failed ({rc})")
    return M


def mttkrp_threads(idx, vals, factors, mode: int, threads: int, dims=None) -> np.ndarray:
    """``mttkrp`` split over ``threads`` threads (fixed contiguous chunks of
    the nonzeros, private FP64 outputs added in thread order): the timed
    multi-threaded CPU baseline.  Equal to ``mttkrp`` up to FP64 rounding."""
    lib = _load()
    idx = _coo(idx)
    N, nnz = idx.shape
    d = _dims(idx, dims)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    F, arr = _fptrs(factors)
    R = F[0].shape[1]
    M = np.empty((int(d[mode]), R), dtype=np.float64)
    rc = lib.oracle_mttkrp_threads(N, _ptr(d), nnz, _ptr(idx), _ptr(vals), arr, R, mode, int(threads), _ptr(M))
    if rc:
        raise ValueError(f"oracle_mttkrp_threads failed ({rc})")
    return M


def mttkrp_rows(idx, vals, factors, mode: int, rows, dims=None) -> np.ndarray:
    """Rows ``rows`` of the spMTTKRP of ``mode`` (same sums as ``mttkrp``)."""
    lib = _load()
    idx = _coo(idx)
    N, nnz = idx.shape
    d = _dims(idx, dims)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    F, arr = _fptrs(factors)
    R = F[0].shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    out = np.empty((rows.size, R), dtype=np.float64)
    rc = lib.oracle_mttkrp_rows(N, _ptr(d), nnz, _ptr(idx), _ptr(vals), arr, R, mode, rows.size,
                                _ptr(rows), _ptr(out))
    if rc:
        raise ValueError(f"oracle_mttkrp_rows failed ({rc})")
    return out


def sampled(idx, F) -> np.ndarray:
    """``out[e] = sum_r prod_w F_w[c_w(e), r]`` over all modes (CPD model value
    at each nonzero, Eq. 1)."""
    lib = _load()
    idx = _coo(idx)
    N, nnz = idx.shape
    F, arr = _fptrs(F)
    out = np.empty(nnz, dtype=np.float64)
    rc = lib.oracle_sampled(N, nnz, _ptr(idx), arr, F[0].shape[1], _ptr(out))
    if rc:
        raise ValueError(f"oracle_sampled failed ({rc})")
    return out


def morton_code(ids: Sequence[np.ndarray], widths: Sequence[int]) -> np.ndarray:
    """Z-Morton code of id tuples: bit levels from the most significant down;
    at each level, the bit of every id whose width exceeds the level, in the
    order the ids are given.  ``widths[t]`` is the bit width of ``ids[t]``.
    The code is built one bit at a time (at most 64 bits in all)."""
    assert sum(widths) <= 64
    n = ids[0].size if ids else 0
    code = np.zeros(n, dtype=np.uint64)
    for level in range(max(widths, default=0) - 1, -1, -1):
        for v, b in zip(ids, widths):
            if level < b:
                code = (code << np.uint64(1)) | ((v.astype(np.uint64) >> np.uint64(level)) & np.uint64(1))
    return code


def layout_order_morton(idx, mode: int, m, dims) -> np.ndarray:
    """pi_n of the Z-Morton variant of L_n (the Z-Morton ordering of
    super-shards among the preprocessing stages of Section V-J).  Reading:
    the nonzeros are ordered by the output mode's super-shard id ss_n, then
    by the Z-Morton code of the other modes' super-shard ids taken in the
    order n+1, n+2, ..., n-1 (mode indices mod N, each id with the bit width
    of its mode's largest id, ceil(I_w / m_w) - 1), ties kept in input order."""
    idx = _coo(idx)
    N, nnz = idx.shape
    mm = np.asarray(m, dtype=np.uint64)
    if nnz == 0:
        return np.empty(0, dtype=np.uint32)
    others = [(mode + t) % N for t in range(1, N)]
    ids = [idx[w].astype(np.uint64) // mm[w] for w in others]
    widths = [max(1, int((int(dims[w]) + int(mm[w]) - 1) // int(mm[w]) - 1).bit_length()) for w in others]
    code = morton_code(ids, widths)
    ssn = idx[mode].astype(np.uint64) // mm[mode]
    return np.lexsort((code, ssn)).astype(np.uint32)


def layout_order(idx, mode: int, m=None) -> np.ndarray:
    """pi_n: position -> original element of layout L_n.

    Section III-B orders the tensor by the shard ids of the output mode and
    Section III-A gives every element a super-shard in each mode.  Reading:
    with ss_w = c_w div m_w, L_n is the input sorted by the key
    ``(ss_n, ss_{n-1}, ..., ss_{n+1})`` (mode indices mod N), ties kept in
    input order.  A stable library sort of that key tuple is the definition:
    the ids are packed into one integer when they fit in 63 bits, else
    ``np.lexsort`` takes them as separate keys.  ``m`` defaults to all ones
    (order by coordinates)."""
    idx = _coo(idx)
    N, nnz = idx.shape
    mm = np.ones(N, dtype=np.uint64) if m is None else np.asarray(m, dtype=np.uint64)
    if nnz == 0:
        return np.empty(0, dtype=np.uint32)
    # keys[0] is the primary key ss_n, keys[t] = ss_{n-t}
    keys = [idx[(mode - t) % N].astype(np.uint64) // mm[(mode - t) % N] for t in range(N)]
    widths = [max(1, int(k.max()).bit_length()) for k in keys]
    if sum(widths) <= 63:
        packed = np.zeros(nnz, dtype=np.uint64)
        for k, b in zip(keys, widths):
            packed = (packed << np.uint64(b)) | k
        order = np.argsort(packed, kind="stable")
    else:
        order = np.lexsort(keys[::-1])      # lexsort: the last key is the primary one
    return order.astype(np.uint32)


def layout_order_qsort(idx, mode: int, m=None) -> np.ndarray:
    """The same order by the C library's qsort with an explicit comparator
    on the key tuple and then the input position (a second, independent
    coding of ``layout_order``'s definition, for small inputs)."""
    lib = _load()
    idx = _coo(idx)
    N, nnz = idx.shape
    mm = np.ascontiguousarray(np.ones(N) if m is None else m, dtype=np.uint64)
    order = np.empty(nnz, dtype=np.uint32)
    rc = lib.oracle_layout_order(N, nnz, _ptr(idx), _ptr(mm), mode, _ptr(order))
    if rc:
        raise ValueError(f"oracle_layout_order failed ({rc})")
    return order


def inverse(perm: np.ndarray) -> np.ndarray:
    """Inverse permutation: ``inv[perm[p]] = p``."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size, dtype=perm.dtype)
    return inv


def partition(rows, I: int, m: int, g: int):
    """Super-shard and shard pointers of one mode (Section III-A)."""
    lib = _load()
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    nnz = rows.size
    k = (I + m - 1) // m
    ss_ptr = np.empty(k + 1, dtype=np.uint64)
    cap = nnz // max(g, 1) + k + 2
    shard_ptr = np.empty(cap, dtype=np.uint64)
    S = np.zeros(1, dtype=np.uint64)
    rc = lib.oracle_partition(I, nnz, _ptr(rows), m, g, _ptr(ss_ptr), _ptr(shard_ptr), cap, _ptr(S))
    if rc:
        raise ValueError(f"oracle_partition failed ({rc})")
    return ss_ptr, shard_ptr[: int(S[0]) + 1].copy()


def lpt(sizes, nbins: int):
    """Algorithm 3: returns ``(order, bin_of, load)``."""
    lib = _load()
    sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
    n = sizes.size
    order = np.empty(n, dtype=np.uint64)
    bin_of = np.empty(n, dtype=np.uint64)
    load = np.empty(nbins, dtype=np.uint64)
    rc = lib.oracle_lpt(n, _ptr(sizes), nbins, _ptr(order), _ptr(bin_of), _ptr(load))
    if rc:
        raise ValueError(f"oracle_lpt failed ({rc})")
    return order, bin_of, load


def lpt_bins(sizes, nbins: int):
    """Algorithm 3 as CSR lists: ``bin_ptr[nbins+1]`` and ``items`` where bin b
    holds ``items[bin_ptr[b]:bin_ptr[b+1]]`` in the order they were appended."""
    order, bin_of, load = lpt(sizes, nbins)
    per_bin: List[List[int]] = [[] for _ in range(nbins)]
    for it in order.tolist():
        per_bin[int(bin_of[it])].append(int(it))
    bin_ptr = np.zeros(nbins + 1, dtype=np.uint64)
    bin_ptr[1:] = np.cumsum([len(b) for b in per_bin])
    items = np.array([i for b in per_bin for i in b], dtype=np.uint64)
    return bin_ptr, items, load


def round_bf16(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 (round to nearest, ties to even), widened back."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    lib.oracle_round_bf16(x.size, _ptr(x), _ptr(out))
    return out


def flycoo_layout(idx, dims, m: Sequence[int], g: int, nbins: int, order: str = "key"
                  ) -> List[Dict[str, np.ndarray]]:
    """Everything the FLYCOO format fixes for each mode n, from the definitions:

    ``order`` (pi_n: the order of L_n, the super-shard key order of
    ``layout_order``, or with ``order="morton"`` the Z-Morton variant of
    ``layout_order_morton``), ``pos`` (its inverse: slot of each element in L_n),
    ``ss_ptr`` and ``shard_ptr`` (Section III-A), ``shard_ss`` (super-shard
    of every shard), ``next`` (slot in L_{(n+1) mod N} of the element at each
    position of L_n: the dynamic remap of Section III-B and Algorithm 2),
    ``ss_bins`` (Algorithm 3 over super-shards, load = shard count) and
    ``shard_bins`` (Algorithm 3 over shards, load = element count).
    """
    idx = _coo(idx)
    N, nnz = idx.shape
    modes = []
    for n in range(N):
        ss_ptr, shard_ptr = partition(idx[n], int(dims[n]), int(m[n]), int(g))
        order_n = layout_order(idx, n, m) if order == "key" else layout_order_morton(idx, n, m, dims)
        starts = shard_ptr[:-1].astype(np.int64)
        ends = shard_ptr[1:].astype(np.int64)
        ss_sizes = ss_ptr[1:] - ss_ptr[:-1]
        ss_shards = (ss_sizes + np.uint64(g) - np.uint64(1)) // np.uint64(g)
        shard_ss = np.repeat(np.arange(ss_sizes.size, dtype=np.uint32), ss_shards.astype(np.int64))
        modes.append(dict(
            order=order_n,
            pos=inverse(order_n),
            ss_ptr=ss_ptr,
            shard_ptr=shard_ptr,
            shard_ss=shard_ss,
            ss_bins=lpt_bins(ss_shards, nbins)[:2],
            shard_bins=lpt_bins(ends - starts, nbins)[:2],
        ))
    for n in range(N):
        nx = modes[(n + 1) % N]
        modes[n]["next"] = nx["pos"][modes[n]["order"]]
    return modes


def remap(buf: np.ndarray, order_from: np.ndarray, pos_to: np.ndarray) -> np.ndarray:
    """Dynamic tensor remapping (Section III-B): the element at position p of
    the current layout is stored at its slot in the target layout."""
    out = np.empty_like(buf)
    out[pos_to[order_from]] = buf
    return out
