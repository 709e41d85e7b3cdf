"""Pins of the oracle's FLYCOO layout, partition, remap and schedule
(Sections III-A, III-B; Algorithms 2 and 3) to properties that hold by
construction of the format and to a hand-worked schedule."""
import itertools
import os

import numpy as np
import pytest

import oracle
from synth import random_coo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

CASES = [((30, 20, 10), 500, 0), ((6, 5, 4, 3), 200, 1), ((4, 3, 3, 2, 2), 120, 2),
         ((50, 2, 3), 150, 3)]


@pytest.mark.parametrize("dims,nnz,seed", CASES)
def test_layout_is_sorted_permutation(dims, nnz, seed):
    idx, _ = random_coo(dims, nnz, seed=seed, distinct=False)
    N = len(dims)
    for n in range(N):
        order = oracle.layout_order(idx, n)
        assert np.array_equal(np.sort(order), np.arange(nnz))
        # rows are contiguous: the output index never decreases
        assert np.all(np.diff(idx[n][order].astype(np.int64)) >= 0)


@pytest.mark.parametrize("dims,nnz,seed", CASES)
@pytest.mark.parametrize("widths", ["ones", "mixed"])
def test_next_layout_is_stable_counting_sort(dims, nnz, seed, widths):
    # Under the cyclic key, L_{n+1} is L_n stably sorted by the super-shard id
    # of mode n+1 alone: the remap of Algorithm 2 is a stable bucket scatter
    # into the next mode's super-shards.
    idx, _ = random_coo(dims, nnz, seed=seed, distinct=False)
    N = len(dims)
    m = [1] * N if widths == "ones" else [max(1, d // 3) for d in dims]
    ss = [idx[w] // m[w] for w in range(N)]
    orders = [oracle.layout_order(idx, n, m) for n in range(N)]
    for n in range(N):
        nx = (n + 1) % N
        prev = orders[n]
        stable = prev[np.argsort(ss[nx][prev], kind="stable")]
        assert np.array_equal(stable, orders[nx])
        # super-shards of mode n are contiguous and ascending in L_n
        assert np.all(np.diff(ss[n][orders[n]].astype(np.int64)) >= 0)
    # and L_0 is the input order stably sorted by modes 1, 2, ..., N-1, 0 in turn
    cur = np.arange(nnz, dtype=np.uint32)
    for w in list(range(1, N)) + [0]:
        cur = cur[np.argsort(ss[w][cur], kind="stable")]
    assert np.array_equal(cur, orders[0])


@pytest.mark.parametrize("dims,nnz,seed", CASES + [((70000, 3, 90000), 400, 5)])
@pytest.mark.parametrize("widths", ["ones", "mixed"])
def test_layout_order_matches_comparator_sort(dims, nnz, seed, widths):
    # two codings of the key order: a stable library sort of the key tuple
    # (packed, or lexsort when the ids need more than 63 bits) and a qsort with
    # an explicit comparator on (key tuple, input position)
    idx, _ = random_coo(dims, nnz, seed=seed, distinct=False)
    N = len(dims)
    m = [1] * N if widths == "ones" else [max(1, d // 3) for d in dims]
    for n in range(N):
        assert np.array_equal(oracle.layout_order(idx, n, m), oracle.layout_order_qsort(idx, n, m))


def test_layout_order_wide_keys_use_separate_sort_keys():
    # 3 modes of ~2^31 ids each need 93 bits: the lexsort branch; its order is
    # checked against the comparator sort and by direct key comparison
    rng = np.random.default_rng(9)
    idx = rng.integers(0, 2**31 - 1, size=(3, 500), dtype=np.int64).astype(np.uint32)
    idx[:, 100:200] = idx[:, :100]          # exact ties: input order decides
    for n in range(3):
        o = oracle.layout_order(idx, n)
        assert np.array_equal(o, oracle.layout_order_qsort(idx, n))
        keys = list(zip(idx[n][o].tolist(), idx[(n - 1) % 3][o].tolist(), idx[(n + 1) % 3][o].tolist(), o.tolist()))
        assert keys == sorted(keys)


def test_layout_order_with_unit_widths_sorts_by_coordinates():
    # with m_w = 1 every super-shard id is the coordinate: L_n is ordered by
    # (c_n, c_{n-1}, ..., c_{n+1}) and rows are contiguous
    idx, _ = random_coo((9, 8, 7), 300, seed=4, distinct=True)
    for n in range(3):
        o = oracle.layout_order(idx, n, [1, 1, 1])
        keys = list(zip(idx[n][o], idx[(n - 1) % 3][o], idx[(n + 1) % 3][o]))
        assert keys == sorted(keys)


@pytest.mark.parametrize("dims,nnz,seed", CASES)
def test_remap_cycle_returns_to_mode0(dims, nnz, seed):
    idx, vals = random_coo(dims, nnz, seed=seed, distinct=False)
    N = len(dims)
    modes = oracle.flycoo_layout(idx, dims, [3] * N, 7, 4)
    buf = np.stack([*idx, vals.view(np.uint32)], axis=1)[modes[0]["order"]]
    start = buf.copy()
    for n in range(N):
        nxt = oracle.remap(buf, modes[n]["order"], modes[(n + 1) % N]["pos"])
        # the next map is the same permutation the remap applies
        check = np.empty_like(buf)
        check[modes[n]["next"]] = buf
        assert np.array_equal(check, nxt)
        assert np.array_equal(np.sort(nxt[:, -1]), np.sort(buf[:, -1]))   # value multiset kept
        assert np.array_equal(nxt, np.stack([*idx, vals.view(np.uint32)], 1)[modes[(n + 1) % N]["order"]])
        buf = nxt
    assert np.array_equal(buf, start)
    comp = np.arange(nnz)
    for n in range(N):
        comp = modes[n]["next"][comp]
    assert np.array_equal(comp, np.arange(nnz))


@pytest.mark.parametrize("m,g", [(1, 1), (3, 4), (7, 16), (100, 1000), (4, 5)])
def test_partition_invariants(m, g):
    dims = (37, 11, 13)
    idx, _ = random_coo(dims, 400, seed=12, law="zipf")
    for n in range(3):
        I = dims[n]
        ss_ptr, shard_ptr = oracle.partition(idx[n], I, m, g)
        k = -(-I // m)
        assert ss_ptr.size == k + 1 and ss_ptr[0] == 0 and ss_ptr[-1] == 400
        rows_sorted = np.sort(idx[n])
        for j in range(k):
            seg = rows_sorted[ss_ptr[j]:ss_ptr[j + 1]]
            assert np.all((seg >= j * m) & (seg < (j + 1) * m))
            # ss_ptr[j] counts the elements below the interval
            assert ss_ptr[j] == np.count_nonzero(idx[n] < j * m)
        sizes = ss_ptr[1:] - ss_ptr[:-1]
        S = int(sum(-(-int(s) // g) for s in sizes))
        assert shard_ptr.size == S + 1 and shard_ptr[-1] == 400
        # shards tile each super-shard: g each, the last one of a super-shard shorter
        starts = set(shard_ptr[:-1].tolist())
        for j in range(k):
            lo, hi = int(ss_ptr[j]), int(ss_ptr[j + 1])
            assert [p for p in range(lo, hi) if p in starts] == list(range(lo, hi, g))


def test_partition_small_modes_use_unit_intervals():
    # with m = 1 every super-shard is one output index
    idx, _ = random_coo((5, 5, 5), 60, seed=3, distinct=False)
    ss_ptr, _ = oracle.partition(idx[0], 5, 1, 8)
    np.testing.assert_array_equal(np.diff(ss_ptr), np.bincount(idx[0], minlength=5))


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                tag, *v = line.split()
                rows[tag] = [int(x) for x in v]
    return rows


def test_lpt_hand_worked():
    g = _read_golden("lpt_6items_2bins.txt")
    bin_ptr, items, load = oracle.lpt_bins(g["sizes"], g["nbins"][0])
    assert items[bin_ptr[0]:bin_ptr[1]].tolist() == g["bin0"]
    assert items[bin_ptr[1]:bin_ptr[2]].tolist() == g["bin1"]
    assert load.tolist() == g["load"]


@pytest.mark.parametrize("nbins", [2, 3, 4, 5])
def test_lpt_graham_tight_instance(nbins):
    # Graham's worst case: jobs 2m-1, 2m-1, 2m-2, 2m-2, ..., m+1, m+1, m, m, m on m
    # machines; LPT makes 4m-1 while the optimum is 3m.
    m = nbins
    sizes = [s for s in range(2 * m - 1, m, -1) for _ in range(2)] + [m, m, m]
    _, _, load = oracle.lpt(sizes, m)
    assert int(load.max()) == 4 * m - 1


def test_lpt_within_four_thirds_of_optimum():
    rng = np.random.default_rng(0)
    for trial in range(40):
        nb = int(rng.integers(2, 4))
        n = int(rng.integers(1, 9))
        sizes = rng.integers(0, 20, size=n)
        _, bin_of, load = oracle.lpt(sizes, nb)
        assert int(load.sum()) == int(sizes.sum())
        assert np.array_equal(np.bincount(bin_of.astype(np.int64), weights=sizes, minlength=nb), load)
        opt = min(max(np.bincount(np.array(a), weights=sizes, minlength=nb))
                  for a in itertools.product(range(nb), repeat=n))
        assert load.max() <= (4.0 / 3.0 - 1.0 / (3 * nb)) * opt + 1e-9


def test_flycoo_layout_shards_lie_in_their_super_shard():
    dims = (40, 9, 8)
    m = [5, 2, 3]
    idx, _ = random_coo(dims, 300, seed=21, law="zipf")
    modes = oracle.flycoo_layout(idx, dims, m, 16, 6)
    for n, md in enumerate(modes):
        ss = idx[n][md["order"]] // m[n]
        sp = md["shard_ptr"].astype(np.int64)
        for q in range(sp.size - 1):
            assert np.all(ss[sp[q]:sp[q + 1]] == md["shard_ss"][q])
            assert sp[q + 1] - sp[q] <= 16
        ptr, items = md["shard_bins"]
        assert np.array_equal(np.sort(items), np.arange(sp.size - 1))
        ptr, items = md["ss_bins"]
        assert np.array_equal(np.sort(items), np.arange(md["ss_ptr"].size - 1))


def test_morton_code_hand_worked():
    g = {"pairs": [], "w31": []}
    with open(os.path.join(GOLDEN, "morton_4x4_ids.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t = line.split()
            if t[0] == "W31":
                g["w31"].append([int(x) for x in t[1:]])
            else:
                g["pairs"].append([int(x) for x in t])
    a, b, z = (np.array(c, dtype=np.uint64) for c in zip(*g["pairs"]))
    np.testing.assert_array_equal(oracle.morton_code([a, b], [2, 2]), z)
    a, b, z = (np.array(c, dtype=np.uint64) for c in zip(*g["w31"]))
    np.testing.assert_array_equal(oracle.morton_code([a, b], [3, 1]), z)


def test_morton_code_single_id_is_the_id():
    v = np.arange(1000, dtype=np.uint64)
    np.testing.assert_array_equal(oracle.morton_code([v], [10]), v)


@pytest.mark.parametrize("dims,nnz,seed", [((40, 30, 20), 800, 0), ((9, 8, 7, 6), 500, 1)])
def test_morton_layout_properties(dims, nnz, seed):
    idx, _ = random_coo(dims, nnz, seed=seed, distinct=False)
    N = len(dims)
    m = [3] * N
    for n in range(N):
        o = oracle.layout_order_morton(idx, n, m, dims)
        assert np.array_equal(np.sort(o), np.arange(nnz))
        ssn = idx[n][o] // m[n]
        assert np.all(np.diff(ssn.astype(np.int64)) >= 0)     # super-shards of mode n contiguous
        others = [(n + t) % N for t in range(1, N)]
        widths = [max(1, ((dims[w] + m[w] - 1) // m[w] - 1).bit_length()) for w in others]
        code = oracle.morton_code([idx[w][o].astype(np.uint64) // m[w] for w in others], widths).astype(np.int64)
        same = np.diff(ssn.astype(np.int64)) == 0
        dc = np.diff(code)
        assert np.all(dc[same] >= 0)                         # Z order inside a super-shard
        assert np.all(np.diff(o.astype(np.int64))[same & (dc == 0)] > 0)   # ties in input order
        # the top bit of every other mode's id is the leading part of the code:
        # within a super-shard the tuple of top bits never decreases
        top = np.zeros(nnz, dtype=np.int64)
        L = max(widths)
        for w, b in zip(others, widths):
            if b == L:
                top = top * 2 + ((idx[w][o] // m[w]) >> (L - 1)).astype(np.int64)
        assert np.all(np.diff(top)[same] >= 0)


def test_morton_layout_with_one_other_mode_varying_is_the_key_order():
    # when all but one of the other modes have a single super-shard, the Z code
    # is that mode's id and the Morton layout equals the key order
    rng = np.random.default_rng(3)
    dims = (20, 50, 4)
    idx = np.stack([rng.integers(0, 20, 300), rng.integers(0, 50, 300), rng.integers(0, 4, 300)]).astype(np.uint32)
    m = [5, 5, 4]
    np.testing.assert_array_equal(oracle.layout_order_morton(idx, 0, m, dims), oracle.layout_order(idx, 0, m))
