"""Pins of the oracle's spMTTKRP (Section II-C; elementwise equation of
Section IV) to results fixed by mathematics, not by the oracle itself."""
import os

import numpy as np
import pytest

import oracle
from synth import make_factors, random_coo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def densify(idx, vals, dims):
    X = np.zeros(dims)
    np.add.at(X, tuple(idx.astype(np.int64)), vals.astype(np.float64))
    return X


def unfold(X, n):
    """Kolda-Bader mode-n unfolding: remaining modes in increasing order, the
    lowest one varying fastest."""
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1, order="F")


def khatri_rao_excluding(Y, n):
    """Y_{N-1} (.) ... (.) Y_{n+1} (.) Y_{n-1} (.) ... (.) Y_0, column by column."""
    R = Y[0].shape[1]
    mats = [Y[w] for w in range(len(Y) - 1, -1, -1) if w != n]
    cols = []
    for r in range(R):
        v = np.ones(1)
        for A in mats:
            v = np.kron(v, A[:, r])
        cols.append(v)
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("dims,nnz,R,seed", [
    ((7, 6, 5), 40, 3, 0),
    ((5, 4, 3, 3), 60, 4, 1),
    ((3, 4, 2, 3, 2), 50, 2, 2),
    ((9, 1, 4), 20, 5, 3),
])
def test_dense_bruteforce(dims, nnz, R, seed):
    # densify -> unfold -> explicit Khatri-Rao -> dense GEMM, all in FP64
    idx, vals = random_coo(dims, nnz, seed=seed, distinct=False)
    Y = [f.astype(np.float64) for f in make_factors(dims, R, seed=seed)]
    X = densify(idx, vals, dims)
    for n in range(len(dims)):
        ref = unfold(X, n) @ khatri_rao_excluding(Y, n)
        got = oracle.mttkrp(idx, vals, Y, n, dims)
        assert got.shape == ref.shape
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_rank1_closed_form():
    # X = lam * a o b o c with every cell a nonzero:
    # M_n[i, r] = lam * y_n[i] * prod_{w != n} (y_w^T Y_w)[r]
    rng = np.random.default_rng(7)
    dims = (6, 5, 4)
    lam = 1.75
    vecs = [rng.standard_normal(d) for d in dims]
    grid = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), 0).reshape(3, -1)
    idx = grid.astype(np.uint32)
    vals = lam * vecs[0][grid[0]] * vecs[1][grid[1]] * vecs[2][grid[2]]
    Y = [rng.standard_normal((d, 3)) for d in dims]
    for n in range(3):
        scale = np.ones(3)
        for w in range(3):
            if w != n:
                scale *= vecs[w] @ Y[w]
        ref = lam * np.outer(vecs[n], scale)
        np.testing.assert_allclose(oracle.mttkrp(idx, vals, Y, n, dims), ref, rtol=1e-12, atol=1e-12)


def test_slice_sums_with_unit_factors():
    # all factors = 1: every column of M_n is the sum of the values in each slice
    dims = (11, 7, 5)
    idx, vals = random_coo(dims, 200, seed=4, distinct=False, value_law="int1to5")
    Y = [np.ones((d, 4)) for d in dims]
    for n in range(3):
        ref = np.bincount(idx[n], weights=vals.astype(np.float64), minlength=dims[n])
        got = oracle.mttkrp(idx, vals, Y, n, dims)
        for r in range(4):
            np.testing.assert_array_equal(got[:, r], ref)


def test_cross_mode_scalar_invariant():
    # sum_{i,r} M_n[i,r] Y_n[i,r] = sum_x val_x sum_r prod_w Y_w[c_w, r] for every n
    dims = (9, 8, 7, 6)
    idx, vals = random_coo(dims, 300, seed=5)
    Y = [f.astype(np.float64) for f in make_factors(dims, 5, seed=5)]
    s = [float(np.sum(oracle.mttkrp(idx, vals, Y, n, dims) * Y[n])) for n in range(4)]
    np.testing.assert_allclose(s, s[0], rtol=1e-12)


def test_linearity_and_duplicates():
    dims = (8, 6, 5)
    idx1, v1 = random_coo(dims, 50, seed=8, distinct=False)
    idx2, v2 = random_coo(dims, 70, seed=9, distinct=False)
    Y = [f.astype(np.float64) for f in make_factors(dims, 3, seed=8)]
    both_idx = np.concatenate([idx1, idx2], axis=1)
    both_v = np.concatenate([v1, v2])
    for n in range(3):
        a = oracle.mttkrp(idx1, v1, Y, n, dims) + oracle.mttkrp(idx2, v2, Y, n, dims)
        b = oracle.mttkrp(both_idx, both_v, Y, n, dims)
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    # a duplicated coordinate acts like one nonzero holding the sum of its values
    dup_idx = np.array([[1, 1, 2], [2, 2, 0], [3, 3, 4]], dtype=np.uint32)
    dup_v = np.array([0.25, 0.5, 2.0], dtype=np.float32)
    merged_idx = np.array([[1, 2], [2, 0], [3, 4]], dtype=np.uint32)
    merged_v = np.array([0.75, 2.0], dtype=np.float32)
    for n in range(3):
        np.testing.assert_allclose(oracle.mttkrp(dup_idx, dup_v, Y, n, dims),
                                   oracle.mttkrp(merged_idx, merged_v, Y, n, dims), rtol=1e-15)


def test_empty_rows_and_empty_tensor():
    dims = (10, 3, 3)
    idx = np.array([[2, 2, 7], [0, 1, 2], [1, 1, 0]], dtype=np.uint32)
    vals = np.array([1.0, 2.0, 3.0], dtype=np.float32)
    Y = [np.full((d, 2), 1.5) for d in dims]
    M = oracle.mttkrp(idx, vals, Y, 0, dims)
    assert np.all(M[[0, 1, 3, 4, 5, 6, 8, 9]] == 0.0)
    z = oracle.mttkrp(np.zeros((3, 0), np.uint32), np.zeros(0, np.float32), Y, 1, dims)
    assert z.shape == (3, 2) and np.all(z == 0.0)


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, *vals = line.split()
            rows.setdefault(tag, []).append([float(v) for v in vals])
    return rows


def test_hand_worked_example():
    g = _read_golden("mttkrp_2x2x2_r2.txt")
    nz = np.array(g["nnz"])
    idx = nz[:, :3].T.astype(np.uint32)
    vals = nz[:, 3].astype(np.float32)
    Y = [np.array(g[f"Y{w}"]) for w in range(3)]
    for n in range(3):
        np.testing.assert_array_equal(oracle.mttkrp(idx, vals, Y, n, (2, 2, 2)), np.array(g[f"M{n}"]))


def test_rows_subset_matches_full():
    dims = (13, 9, 7)
    idx, vals = random_coo(dims, 400, seed=11, law="zipf")
    Y = [f.astype(np.float64) for f in make_factors(dims, 4, seed=11)]
    for n in range(3):
        full = oracle.mttkrp(idx, vals, Y, n, dims)
        rows = np.array([dims[n] - 1, 0, 3], dtype=np.uint32)
        np.testing.assert_array_equal(oracle.mttkrp_rows(idx, vals, Y, n, rows, dims), full[rows])


def test_bf16_rounding_pins():
    x = np.array([1.0, 0.5, -2.0, 1.5,                       # exactly representable
                  1.0 + 2.0 ** -8,                          # tie -> even (1.0)
                  1.0 + 3 * 2.0 ** -8,                      # tie -> even (1 + 2^-6)
                  1.0 + 2.0 ** -8 + 2.0 ** -20,             # above the tie -> up
                  np.inf, -np.inf, -0.0, 3.0e38], dtype=np.float32)
    want = np.array([1.0, 0.5, -2.0, 1.5, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7,
                     np.inf, -np.inf, -0.0], dtype=np.float32)
    got = oracle.round_bf16(x)
    np.testing.assert_array_equal(got[:10], want)
    assert np.signbit(got[9])
    assert np.isnan(oracle.round_bf16(np.array([np.nan], np.float32)))[0]
    # the result always has its low 16 bits clear and is within half an ulp of bf16
    r = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 100
    b = oracle.round_bf16(r)
    assert np.all(b.view(np.uint32) & 0xFFFF == 0)
    assert np.all(np.abs(b - r) <= np.abs(r) * 2.0 ** -8)


def test_bf16_rounding_agrees_with_torch():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(1).standard_normal(50000).astype(np.float32) * 37
    ref = torch.from_numpy(r).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(r), ref)


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_threaded_oracle_equals_sequential(threads):
    # the threaded baseline is the same sum split into fixed chunks: bit-equal
    # with one thread, equal to FP64 rounding otherwise, and repeatable
    dims = (40, 30, 20)
    idx, vals = random_coo(dims, 5000, seed=7, law="zipf", distinct=False, value_law="normal")
    facs = [np.random.default_rng(w).standard_normal((d, 8)) for w, d in enumerate(dims)]
    for n in range(3):
        ref = oracle.mttkrp(idx, vals, facs, n, dims)
        got = oracle.mttkrp_threads(idx, vals, facs, n, threads, dims)
        if threads == 1:
            np.testing.assert_array_equal(got, ref)
        else:
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(got, oracle.mttkrp_threads(idx, vals, facs, n, threads, dims))
