"""Seeded synthetic COO tensors shaped like the FROSTT workloads of the paper.

Every draw comes from numpy's PCG64 bit generator.  The tensor and the
factors use two independent streams derived from one integer seed:
``SeedSequence([seed, 0])`` for the tensor and ``SeedSequence([seed, 1])``
for the factors.

Recipe (``make_coo``):

1. Draw coordinates per mode, independently, from the mode's distribution:
   uniform over ``[0, I)``, a bounded Zipf law ``P(i) ~ (i+1)^-s`` over
   ``[0, I)`` (index 0 is the most frequent), or a "hot slice" law that
   puts a fixed share of the draws on a few ids and spreads the rest
   uniformly over the other ids.
2. If the workload asks for distinct coordinates, merge duplicates and keep
   drawing batches until at least ``nnz`` distinct coordinates exist, then
   keep a seeded random subset of exactly ``nnz`` of them.  The subset is
   also a random order, so the COO order is shuffled.
3. Draw the values last, one per kept coordinate.  Values are independent
   of coordinates, so drawing them after the merge leaves their
   distribution exactly the stated one.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "zipf_cdf",
    "draw_zipf",
    "make_coo",
    "make_factors",
    "make_workload",
    "random_coo",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """A synthetic workload: tensor shape, index and value laws, rank."""

    name: str
    dims: Tuple[int, ...]
    nnz: int
    # per mode: ("uniform",) | ("zipf", s) | ("hot", n_hot, share)
    index_laws: Tuple[tuple, ...]
    # "uniform01" | "lognormal" | "int1to5" | "normal"
    value_law: str
    rank: int
    # "normal" = N(0,1); "normal_over_sqrt_r" = N(0,1)/sqrt(R)
    factor_law: str
    factor_dtype: str = "f32"
    distinct: bool = True
    seed: int = 0
    stands_in_for: str = ""


WORKLOADS: Dict[str, Workload] = {
    # Correctness case: 100K distinct uniform coordinates, R=16.
    "uniform_1000x800x600_100k_r16": Workload(
        name="uniform_1000x800x600_100k_r16",
        dims=(1000, 800, 600),
        nnz=100_000,
        index_laws=(("uniform",),) * 3,
        value_law="uniform01",
        rank=16,
        factor_law="normal",
    ),
    # Nell-2-sized (12.1K x 9.2K x 28.8K, 76.9M nnz): Zipf(1.1) per mode.
    "nell2like_12000x9000x29000_77m_r32": Workload(
        name="nell2like_12000x9000x29000_77m_r32",
        dims=(12_000, 9_000, 29_000),
        nnz=77_000_000,
        index_laws=(("zipf", 1.1),) * 3,
        value_law="lognormal",
        rank=32,
        factor_law="normal_over_sqrt_r",
        stands_in_for="Nell-2 (FROSTT)",
    ),
    # The same laws at 16M nonzeros: a profiling case that still exceeds L2
    # (two 256 MB element buffers) but keeps an ncu capture to ~1 GB.
    "nell2like_12000x9000x29000_16m_r32": Workload(
        name="nell2like_12000x9000x29000_16m_r32",
        dims=(12_000, 9_000, 29_000),
        nnz=16_000_000,
        index_laws=(("zipf", 1.1),) * 3,
        value_law="lognormal",
        rank=32,
        factor_law="normal_over_sqrt_r",
        stands_in_for="Nell-2 (FROSTT), reduced for profiling",
    ),
    # Delicious-like 4-mode tensor for the BF16-vs-FP32 precision study.
    "delicious4d_1.2mx1.2mx50kx10k_140m_r32": Workload(
        name="delicious4d_1.2mx1.2mx50kx10k_140m_r32",
        dims=(1_200_000, 1_200_000, 50_000, 10_000),
        nnz=140_000_000,
        index_laws=(("zipf", 1.3), ("zipf", 1.3), ("uniform",), ("uniform",)),
        value_law="uniform01",
        rank=32,
        factor_law="normal_over_sqrt_r",
        factor_dtype="bf16",
        stands_in_for="Delicious (FROSTT, 4 modes)",
    ),
    # Nell-1-sized 3-mode tensor for the CP-OPT gradient study.
    "nell1like_4.8mx1.8mx1.8m_140m_r32": Workload(
        name="nell1like_4.8mx1.8mx1.8m_140m_r32",
        dims=(4_800_000, 1_800_000, 1_800_000),
        nnz=140_000_000,
        index_laws=(("zipf", 1.2),) * 3,
        value_law="int1to5",
        rank=32,
        factor_law="normal_over_sqrt_r",
        stands_in_for="Nell-1 (FROSTT)",
    ),
    # Skew stress for CP-ALS: 10 mode-0 slices hold half of the nonzeros.
    "skewed_20kx200kx500k_200m_r64": Workload(
        name="skewed_20kx200kx500k_200m_r64",
        dims=(20_000, 200_000, 500_000),
        nnz=200_000_000,
        index_laws=(("hot", 10, 0.5), ("uniform",), ("uniform",)),
        value_law="normal",
        rank=64,
        factor_law="normal_over_sqrt_r",
        factor_dtype="bf16",
        stands_in_for="Vast-like load imbalance",
    ),
}


def _streams(seed: int):
    ss_t = np.random.SeedSequence([seed, 0])
    ss_f = np.random.SeedSequence([seed, 1])
    return (np.random.Generator(np.random.PCG64(ss_t)),
            np.random.Generator(np.random.PCG64(ss_f)))


def zipf_cdf(I: int, s: float) -> np.ndarray:
    """Cumulative distribution of the bounded Zipf law P(i) ~ (i+1)^-s, i < I."""
    k = np.arange(1, I + 1, dtype=np.float64)
    c = np.cumsum(k ** (-float(s)))
    c /= c[-1]
    c[-1] = 1.0
    return c


class _InverseCdf:
    """Inverse-CDF sampler with a guide table.

    ``sample(u)`` equals ``np.searchsorted(cdf, u, side='right')`` for
    ``u`` in [0, 1): the guide table only gives a start index that is never
    past the answer, and a short forward walk finishes the search.
    """

    def __init__(self, cdf: np.ndarray):
        self.cdf = cdf
        n = len(cdf)
        self.M = int(min(max(16 * n, 1024), 1 << 24))
        grid = np.arange(self.M, dtype=np.float64) / self.M
        self.guide = np.searchsorted(cdf, grid, side="right").astype(np.int64)

    def sample(self, u: np.ndarray) -> np.ndarray:
        j = np.floor(u * self.M).astype(np.int64) - 1
        np.clip(j, 0, self.M - 1, out=j)
        k = self.guide[j]
        n = len(self.cdf)
        active = np.nonzero(k < n)[0]
        active = active[self.cdf[np.minimum(k[active], n - 1)] <= u[active]]
        while active.size:
            k[active] += 1
            ka = k[active]
            keep = ka < n
            active = active[keep]
            active = active[self.cdf[k[active]] <= u[active]]
        return k


_SAMPLERS: Dict[Tuple[int, float], _InverseCdf] = {}


def draw_zipf(rng: np.random.Generator, size: int, I: int, s: float) -> np.ndarray:
    key = (int(I), float(s))
    smp = _SAMPLERS.get(key)
    if smp is None:
        smp = _InverseCdf(zipf_cdf(I, s))
        if I <= 4_000_000:
            _SAMPLERS[key] = smp
    return smp.sample(rng.random(size))


def _draw_mode(rng, law: tuple, I: int, size: int, hot_ids: Optional[np.ndarray]) -> np.ndarray:
    kind = law[0]
    if kind == "uniform":
        return rng.integers(0, I, size=size, dtype=np.int64)
    if kind == "zipf":
        return draw_zipf(rng, size, I, law[1])
    if kind == "hot":
        n_hot, share = int(law[1]), float(law[2])
        assert hot_ids is not None and len(hot_ids) == n_hot
        cold = np.setdiff1d(np.arange(I, dtype=np.int64), hot_ids, assume_unique=True)
        is_hot = rng.random(size) < share
        out = cold[rng.integers(0, len(cold), size=size)]
        nh = int(is_hot.sum())
        out[is_hot] = hot_ids[rng.integers(0, n_hot, size=nh)]
        return out
    raise ValueError(f"unknown index law {law!r}")


def _split_point(dims: Sequence[int]) -> int:
    """Largest k such that every key of the first k modes fits in an unsigned
    64-bit integer, i.e. prod(dims[:k]) <= 2^64 (at least 1)."""
    p = 1
    for k, d in enumerate(dims):
        if p * d > (1 << 64):
            return max(k, 1)
        p *= d
    return len(dims)


def _linear(coords: List[np.ndarray], dims: Sequence[int], lo: int, hi: int) -> np.ndarray:
    key = np.zeros(len(coords[0]), dtype=np.uint64)
    for m in range(lo, hi):
        key *= np.uint64(dims[m])
        key += coords[m].astype(np.uint64)
    return key


def _unique_sorted(hi: np.ndarray, lo: Optional[np.ndarray]):
    """Distinct (hi, lo) pairs, lexicographically sorted."""
    if lo is None:
        s = np.sort(hi)
        if s.size == 0:
            return s, None
        keep = np.empty(s.size, dtype=bool)
        keep[0] = True
        np.not_equal(s[1:], s[:-1], out=keep[1:])
        return s[keep], None
    order = np.argsort(hi)
    hs = hi[order]
    ls = lo[order]
    if hs.size:
        same = hs[1:] == hs[:-1]
        in_run = np.zeros(hs.size, dtype=bool)
        in_run[1:] |= same
        in_run[:-1] |= same
        idx = np.nonzero(in_run)[0]
        if idx.size:
            sub = np.lexsort((ls[idx], hs[idx]))
            ls[idx] = ls[idx][sub]
    keep = np.ones(hs.size, dtype=bool)
    if hs.size:
        keep[1:] = (hs[1:] != hs[:-1]) | (ls[1:] != ls[:-1])
    return hs[keep], ls[keep]


def _decode(key: np.ndarray, dims: Sequence[int], lo: int, hi: int, out: List[np.ndarray]):
    k = key.copy()
    for m in range(hi - 1, lo - 1, -1):
        d = np.uint64(dims[m])
        out[m] = (k % d).astype(np.uint32)
        k //= d


def make_coo(dims: Sequence[int], nnz: int, index_laws: Sequence[tuple], value_law: str,
             seed: int = 0, distinct: bool = True) -> Tuple[np.ndarray, np.ndarray]:
    """Return ``(idx, vals)``: ``idx`` is uint32 ``[N, nnz]`` (mode-major),
    ``vals`` float32 ``[nnz]``."""
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    assert len(index_laws) == N
    rng, _ = _streams(seed)
    hot_ids = [None] * N
    for m, law in enumerate(index_laws):
        if law[0] == "hot":
            hot_ids[m] = np.sort(rng.choice(dims[m], size=int(law[1]), replace=False)).astype(np.int64)

    def draw(size):
        return [_draw_mode(rng, index_laws[m], dims[m], size, hot_ids[m]) for m in range(N)]

    if not distinct:
        cols = draw(nnz)
        idx = np.stack([c.astype(np.uint32) for c in cols]) if nnz else np.zeros((N, 0), np.uint32)
    else:
        cells = math.prod(dims)
        if nnz > cells:
            raise ValueError("more distinct nonzeros than cells")
        k = _split_point(dims)
        hi_key = None
        lo_key = None
        need = nnz
        batch = nnz + 1024
        while True:
            cols = draw(batch)
            h = _linear(cols, dims, 0, k)
            l = _linear(cols, dims, k, N) if k < N else None
            del cols
            if hi_key is not None:
                h = np.concatenate([hi_key, h])
                if l is not None:
                    l = np.concatenate([lo_key, l])
            before = 0 if hi_key is None else hi_key.size
            hi_key, lo_key = _unique_sorted(h, l)
            del h, l
            have = hi_key.size
            if have >= nnz:
                break
            gained = max(have - before, 1)
            rate = gained / batch
            need = nnz - have
            batch = int(min(max(need / max(rate, 1e-3) * 1.2, 4096), 4 * nnz + 4096))
        pick = rng.permutation(hi_key.size)[:nnz]
        out: List[np.ndarray] = [None] * N  # type: ignore[list-item]
        _decode(hi_key[pick], dims, 0, k, out)
        if lo_key is not None:
            _decode(lo_key[pick], dims, k, N, out)
        idx = np.stack(out) if nnz else np.zeros((N, 0), np.uint32)

    if value_law == "uniform01":
        vals = rng.random(nnz, dtype=np.float32)
    elif value_law == "lognormal":
        vals = rng.lognormal(0.0, 1.0, nnz).astype(np.float32)
    elif value_law == "int1to5":
        vals = rng.integers(1, 6, size=nnz).astype(np.float32)
    elif value_law == "normal":
        vals = rng.standard_normal(nnz, dtype=np.float32)
    else:
        raise ValueError(f"unknown value law {value_law!r}")
    return np.ascontiguousarray(idx, dtype=np.uint32), vals


def make_factors(dims: Sequence[int], rank: int, law: str = "normal", seed: int = 0) -> List[np.ndarray]:
    """One float32 ``[I_w, R]`` row-major matrix per mode."""
    _, rng = _streams(seed)
    out = []
    for I in dims:
        a = rng.standard_normal((int(I), int(rank)), dtype=np.float32)
        if law == "normal_over_sqrt_r":
            a /= np.float32(math.sqrt(rank))
        elif law != "normal":
            raise ValueError(f"unknown factor law {law!r}")
        out.append(a)
    return out


def make_workload(w: Workload, seed: Optional[int] = None):
    """Return ``(idx, vals, factors)`` for a named workload."""
    s = w.seed if seed is None else seed
    idx, vals = make_coo(w.dims, w.nnz, w.index_laws, w.value_law, seed=s, distinct=w.distinct)
    facs = make_factors(w.dims, w.rank, w.factor_law, seed=s)
    return idx, vals, facs


def random_coo(dims: Sequence[int], nnz: int, seed: int = 0, distinct: bool = True,
               law: str = "uniform", value_law: str = "uniform01", zipf_s: float = 1.2):
    """Small helper for tests: every mode uses the same index law."""
    if law == "uniform":
        laws = tuple(("uniform",) for _ in dims)
    elif law == "zipf":
        laws = tuple(("zipf", zipf_s) for _ in dims)
    else:
        raise ValueError(law)
    return make_coo(dims, nnz, laws, value_law, seed=seed, distinct=distinct)
