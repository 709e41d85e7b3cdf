"""The library's host-side planning on CPU, through the C ABI (no device):
the Section III-A shard split, the Algorithm 3 schedules and the block-cyclic
alternative, the default shard size, the K4 list and the fused kernel's tile
descriptors, bit-exact against the oracle's partition and LPT (and the
hand-worked Algorithm 3 run), on Zipf and uniform tensors and the degenerate
cases.  flycoo_create runs the same planner for every mode."""
import os
import shutil

import numpy as np
import pytest

import oracle
from synth import random_coo

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STAGE_TILES = (512, 1024)


@pytest.fixture(scope="module")
def P():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2309_09131_gb300 import build as B
    B.build()
    import paper_2309_09131_gb300 as pkg
    return pkg


def _plan(P, nnz, ss_ptr, g, bins, schedule=0):
    from paper_2309_09131_gb300 import _native as nat
    h = P.flycoo_plan_create(nnz, ss_ptr, g=g, bins=bins, schedule=schedule)
    try:
        names = [n for n in dir(nat) if n.startswith("PLAN_")]
        return {n[5:].lower(): P.flycoo_plan_get(h, getattr(nat, n)) for n in names}
    finally:
        P.flycoo_plan_destroy(h)


def _expected_segments(shard_ss, k, bin_ptr, items):
    """Segments as the header defines them: maximal runs of shards of one
    super-shard that follow each other in one bin, numbered by super-shard and
    then in schedule order.  Returns (segment of each schedule position,
    seg_ss, ss_seg_ptr)."""
    tmp, seg_tmp = [], np.zeros(items.size, dtype=np.int64)
    for b in range(bin_ptr.size - 1):
        for pos in range(int(bin_ptr[b]), int(bin_ptr[b + 1])):
            j = int(shard_ss[items[pos]])
            if pos == bin_ptr[b] or int(shard_ss[items[pos - 1]]) != j:
                tmp.append(j)
            seg_tmp[pos] = len(tmp) - 1
    order = sorted(range(len(tmp)), key=lambda q: (tmp[q], q))
    renum = np.empty(len(tmp), dtype=np.int64)
    renum[order] = np.arange(len(tmp))
    seg_ss = np.array([tmp[q] for q in order], dtype=np.int64)
    ss_seg_ptr = np.concatenate([[0], np.cumsum(np.bincount(seg_ss, minlength=k))]).astype(np.int64)
    return seg_tmp, renum, seg_ss, ss_seg_ptr


def _expected_tiles(shard_ptr, shard_ss, k, bin_ptr, items, tile):
    """Descriptors as the header defines them: the shards of each bin in
    schedule order, each cut into runs of `tile` positions, flagged at the
    first and last tile of each segment."""
    seg_tmp, renum, seg_ss, ss_seg_ptr = _expected_segments(shard_ss, k, bin_ptr, items)
    nseg = np.diff(ss_seg_ptr)
    desc, tbp = [], [0]
    for b in range(bin_ptr.size - 1):
        i0, i1 = int(bin_ptr[b]), int(bin_ptr[b + 1])
        for pos in range(i0, i1):
            sh = int(items[pos])
            lo, hi = int(shard_ptr[sh]), int(shard_ptr[sh + 1])
            j = int(shard_ss[sh])
            begin = pos == i0 or seg_tmp[pos - 1] != seg_tmp[pos]
            end = pos + 1 == i1 or seg_tmp[pos + 1] != seg_tmp[pos]
            for p in range(lo, hi, tile):
                ln = min(tile, hi - p)
                flags = (1 if begin and p == lo else 0) | (2 if end and p + ln == hi else 0) | \
                        (4 if nseg[j] == 1 else 0)
                desc += [p, ln | (flags << 16), j, int(renum[seg_tmp[pos]])]
        tbp.append(len(desc) // 4)
    return np.array(desc, dtype=np.uint64), np.array(tbp, dtype=np.uint64)


def _check_against_oracle(P, rows, I, m, g, bins):
    ss_ptr, shard_ptr = oracle.partition(rows, I, m, g)
    nnz = rows.size
    got = _plan(P, nnz, ss_ptr, g, bins)
    assert got["g"].tolist() == [g]
    assert np.array_equal(got["shard_ptr"], shard_ptr)
    ss_sizes = (ss_ptr[1:] - ss_ptr[:-1]).astype(np.int64)
    ss_shards = (ss_sizes + g - 1) // g
    shard_ss = np.repeat(np.arange(ss_sizes.size), ss_shards)
    assert np.array_equal(got["shard_ss"], shard_ss)
    assert np.array_equal(got["ss_shard_ptr"], np.concatenate([[0], np.cumsum(ss_shards)]))
    bp, it, _ = oracle.lpt_bins(ss_shards, bins)
    assert np.array_equal(got["ss_bin_ptr"], bp) and np.array_equal(got["ss_items"], it)
    bp, it, _ = oracle.lpt_bins(np.diff(shard_ptr.astype(np.int64)), bins)
    assert np.array_equal(got["shard_bin_ptr"], bp) and np.array_equal(got["shard_items"], it)
    k = ss_sizes.size
    _, _, seg_ss, ss_seg_ptr = _expected_segments(shard_ss, k, bp, it)
    assert np.array_equal(got["seg_ss"], seg_ss)
    assert np.array_equal(got["ss_seg_ptr"], ss_seg_ptr)
    assert np.array_equal(got["k4_items"], np.nonzero(np.diff(ss_seg_ptr) != 1)[0])
    # the fixup kernel's launch order: super-shards of at most 16 segments (one
    # block each) first, then the others, each group in ascending order
    k4 = np.nonzero(np.diff(ss_seg_ptr) != 1)[0]
    nseg = np.diff(ss_seg_ptr)[k4]
    light, heavy = k4[nseg <= 16], k4[nseg > 16]
    assert got["k4_nlight"].tolist() == [light.size]
    assert np.array_equal(got["k4_order"], np.concatenate([light, heavy]))
    # every shard of a super-shard lies in one of its segments: at most as many
    # segments as shards, and a super-shard with shards has at least one
    assert np.all(np.diff(ss_seg_ptr) <= ss_shards) and np.all((np.diff(ss_seg_ptr) > 0) == (ss_shards > 0))
    for z, tile in enumerate(STAGE_TILES):
        desc, tbp = _expected_tiles(shard_ptr, shard_ss, k, bp, it, tile)
        assert np.array_equal(got[f"tiles_{tile}"], desc), tile
        assert np.array_equal(got[f"tile_bin_ptr_{tile}"], tbp), tile
    return got


@pytest.mark.parametrize("law", ["zipf", "uniform"])
@pytest.mark.parametrize("g,bins", [(1024, 7), (700, 17), (4096, 3)])
def test_plan_matches_oracle(P, law, g, bins):
    dims = (900, 300, 5000)
    idx, _ = random_coo(dims, 60_000, seed=11, law=law)
    for n, I in enumerate(dims):
        _check_against_oracle(P, idx[n], I, min(I, 128), g, bins)


def test_plan_reproduces_hand_worked_lpt(P):
    # six super-shards of one shard each (g above every size): the shard
    # schedule is Algorithm 3 over the golden sizes
    gold = {}
    with open(os.path.join(GOLDEN, "lpt_6items_2bins.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                tag, *v = line.split()
                gold[tag] = [int(x) for x in v]
    sizes = gold["sizes"]
    ss_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    got = _plan(P, int(ss_ptr[-1]), ss_ptr, g=max(sizes), bins=gold["nbins"][0])
    bp, it = got["shard_bin_ptr"], got["shard_items"]
    assert it[bp[0]:bp[1]].tolist() == gold["bin0"]
    assert it[bp[1]:bp[2]].tolist() == gold["bin1"]
    assert got["k4_items"].size == 0


def test_block_cyclic(P):
    rows = np.sort(np.random.default_rng(2).integers(0, 1000, size=20_000)).astype(np.uint32)
    ss_ptr, shard_ptr = oracle.partition(rows, 1000, 64, 300)
    bins = 9
    got = _plan(P, rows.size, ss_ptr, 300, bins, schedule=1)
    for key, n_items in (("ss", ss_ptr.size - 1), ("shard", shard_ptr.size - 1)):
        bp, it = got[f"{key}_bin_ptr"], got[f"{key}_items"]
        for b in range(bins):
            assert it[bp[b]:bp[b + 1]].tolist() == list(range(b, n_items, bins))


@pytest.mark.parametrize("nnz,bins", [(0, 456), (5000, 456), (10_000_000, 456), (200_000_000, 456),
                                      (77_000_000, 456), (3_000_000, 17)])
def test_default_shard_size(P, nnz, bins):
    g = int(_plan(P, nnz, [0, nnz], 0, bins)["g"][0])
    # the largest power of two in [1024, 32768] leaving at least sixteen shards per bin
    cands = [1 << e for e in range(10, 16) if (1 << e) == 1024 or nnz // (1 << e) >= 16 * bins]
    assert g == max(cands)


def test_degenerate_plans(P):
    # no nonzeros: no shards, nothing scheduled, K4 writes every super-shard
    got = _plan(P, 0, [0, 0, 0, 0], 1024, 5)
    assert got["shard_ptr"].tolist() == [0] and got["shard_ss"].size == 0
    assert got["shard_items"].size == 0 and got["shard_bin_ptr"].tolist() == [0] * 6
    assert got["k4_items"].tolist() == [0, 1, 2]
    assert got["tiles_512"].size == 0 and got["tile_bin_ptr_1024"].tolist() == [0] * 6
    # one super-shard, one shard smaller than a tile: a single first+last+alone tile
    got = _plan(P, 37, [0, 37], 1024, 4)
    assert got["tiles_1024"].tolist() == [0, 37 | (7 << 16), 0, 0]
    assert got["k4_items"].size == 0
    # one super-shard of three shards in one bin: one segment, so its tiles are
    # flagged first (shard 0) and last (shard 2) only, and it writes the output
    got = _plan(P, 3000, [0, 3000], 1024, 1)
    assert got["seg_ss"].tolist() == [0] and got["k4_items"].size == 0
    t = got["tiles_1024"].reshape(-1, 4)
    assert [int(x >> 16) for x in t[:, 1]] == [1 | 4, 4, 2 | 4]
    assert t[:, 3].tolist() == [0, 0, 0]
    # the same over two bins: shards 0, 2 in bin 0 and shard 1 in bin 1 form two
    # segments (numbered bin 0 first), and K4 sums them
    got = _plan(P, 3000, [0, 3000], 1024, 2)
    assert got["seg_ss"].tolist() == [0, 0] and got["k4_items"].tolist() == [0]
    t = got["tiles_1024"].reshape(-1, 4)
    assert t[:, 0].tolist() == [0, 2048, 1024] and t[:, 3].tolist() == [0, 0, 1]
    assert [int(x >> 16) for x in t[:, 1]] == [1, 2, 1 | 2]
    # more bins than shards: the extra bins stay empty
    got = _plan(P, 3000, [0, 3000], 1024, 8)
    assert np.diff(got["shard_bin_ptr"].astype(np.int64)).tolist() == [1, 1, 1, 0, 0, 0, 0, 0]
    # g = 1: one shard per nonzero
    got = _plan(P, 10, [0, 4, 10], 1, 3)
    assert got["shard_ptr"].tolist() == list(range(11))


def test_plan_argument_errors(P):
    E = P.FlycooError
    cases = [
        dict(nnz=10, ss_ptr=[0, 10], g=4, bins=0),              # no bins
        dict(nnz=10, ss_ptr=[0, 10], g=4, bins=(1 << 20) + 1),  # too many bins
        dict(nnz=10, ss_ptr=[0, 10], g=4, bins=2, schedule=7),  # unknown schedule
        dict(nnz=10, ss_ptr=[1, 10], g=4, bins=2),              # does not start at 0
        dict(nnz=10, ss_ptr=[0, 9], g=4, bins=2),               # does not end at nnz
        dict(nnz=10, ss_ptr=[0, 6, 5, 10], g=4, bins=2),        # decreasing
        dict(nnz=10, ss_ptr=[0, 10], g=1 << 32, bins=2),        # g too large
    ]
    for c in cases:
        with pytest.raises(E) as ei:
            P.flycoo_plan_create(**c)
        assert ei.value.status_name == "FLYCOO_ERR_INVALID_ARG", c
    with pytest.raises(E) as ei:
        P.flycoo_plan_create((1 << 32) - 1, [0, (1 << 32) - 1], bins=2)
    assert ei.value.status_name == "FLYCOO_ERR_UNSUPPORTED"


def test_plan_get_errors(P):
    import ctypes
    from paper_2309_09131_gb300 import _native as nat
    h = P.flycoo_plan_create(100, [0, 60, 100], g=16, bins=2)
    try:
        L = nat.lib()
        n = ctypes.c_uint64(2)
        buf = (ctypes.c_uint64 * 2)()
        # capacity 2 for S + 1 = 8 shard pointers: refused, the length reported
        assert L.flycoo_plan_get(h, nat.PLAN_SHARD_PTR, buf, ctypes.byref(n)) == 1
        assert n.value == 8
        assert L.flycoo_plan_get(h, 99, None, ctypes.byref(n)) == 1
        assert L.flycoo_plan_get(h, nat.PLAN_G, None, None) == 1
        assert L.flycoo_plan_get(None, nat.PLAN_G, None, ctypes.byref(n)) == 1
    finally:
        P.flycoo_plan_destroy(h)
    P.flycoo_plan_destroy(None)


def test_fixup_order_light_then_heavy(P):
    # super-shard 0 spread over 40 bins (40 segments: heavy), super-shard 1 over
    # a few (light), super-shard 2 in one segment (no fixup), super-shard 3 empty
    ss_ptr = np.array([0, 40 * 64, 40 * 64 + 3 * 64, 40 * 64 + 3 * 64 + 10, 40 * 64 + 3 * 64 + 10],
                      dtype=np.uint64)
    got = _plan(P, int(ss_ptr[-1]), ss_ptr, 64, 40)
    nseg = np.diff(got["ss_seg_ptr"].astype(np.int64))
    assert nseg[0] > 16 and 1 < nseg[1] <= 16 and nseg[2] == 1 and nseg[3] == 0
    assert got["k4_items"].tolist() == [0, 1, 3]
    assert got["k4_nlight"].tolist() == [2]
    assert got["k4_order"].tolist() == [1, 3, 0]
