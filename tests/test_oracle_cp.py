"""Pins of the oracle's CP layers (Algorithm 1 with the least-squares update,
CP-OPT loss and gradient, spMTTKRP adjoint) to mathematics: exact
recovery, dense brute force, finite differences and adjoint identities."""
import numpy as np
import pytest

import oracle
from oracle import cp
from synth import make_factors, random_coo


def dense_model(Y, lam=None):
    R = Y[0].shape[1]
    lam = np.ones(R) if lam is None else lam
    X = np.zeros([y.shape[0] for y in Y])
    for r in range(R):
        t = lam[r]
        for y in Y:
            t = np.multiply.outer(t, y[:, r])
        X += t
    return X


def all_cells(dims):
    g = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), 0)
    return g.reshape(len(dims), -1).astype(np.uint32)


def test_cholesky_and_solve():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((9, 9))
    V = A @ A.T + 9 * np.eye(9)
    L = cp.cholesky(V)
    assert np.allclose(np.triu(L, 1), 0.0)
    np.testing.assert_allclose(L @ L.T, V, rtol=1e-13, atol=1e-12)
    X = rng.standard_normal((5, 9))
    np.testing.assert_allclose(cp.chol_solve_rows(L, X @ V), X, rtol=1e-10, atol=1e-10)
    with pytest.raises(cp.NotSPD):
        cp.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))
    with pytest.raises(cp.NotSPD):
        cp.cholesky(np.zeros((3, 3)))


def test_fit_matches_dense_residual():
    # fit = 1 - ||X - Xhat||_F / ||X||_F over ALL cells, X sparse
    dims = (5, 4, 6)
    idx, vals = random_coo(dims, 40, seed=3)
    Y = [f.astype(np.float64) for f in make_factors(dims, 3, seed=3)]
    lam = np.array([0.5, 2.0, 1.25])
    X = np.zeros(dims)
    X[tuple(idx.astype(np.int64))] = vals
    ref = 1.0 - np.linalg.norm(X - dense_model(Y, lam)) / np.linalg.norm(X)
    M_last = oracle.mttkrp(idx, vals, Y, 2, dims)
    assert cp.cp_fit(vals, Y, lam, M_last) == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_als_recovers_exact_cp_tensor():
    # dense exact rank-R tensor: one ALS step from the exact (column-normalised)
    # factors is a fixed point with fit 1
    dims = (6, 5, 4)
    R = 3
    rng = np.random.default_rng(5)
    Y = [rng.standard_normal((d, R)) for d in dims]
    lam_true = np.array([3.0, 2.0, 1.0])
    Yn = [y / np.linalg.norm(y, axis=0) for y in Y]
    X = dense_model(Yn, lam_true)
    idx = all_cells(dims)
    vals = X.reshape(-1)
    Y1, lam, fit = cp.cp_als_step(idx, vals, dims, Yn)
    # the fit takes a square root of ||X||^2 + ||Xhat||^2 - 2<X,Xhat>, a
    # difference of equal terms here, so FP64 resolves it to ~sqrt(eps)
    assert fit == pytest.approx(1.0, abs=1e-7)
    np.testing.assert_allclose(dense_model(Y1, lam), X, rtol=1e-9, atol=1e-9)


def test_als_fit_increases_monotonically():
    dims = (8, 7, 6)
    R = 2
    rng = np.random.default_rng(9)
    Yt = [rng.standard_normal((d, R)) for d in dims]
    X = dense_model(Yt) + 0.01 * rng.standard_normal(dims)
    idx = all_cells(dims)
    vals = X.reshape(-1)
    Y = [rng.standard_normal((d, R)) for d in dims]
    fits = []
    for _ in range(15):
        Y, lam, fit = cp.cp_als_step(idx, vals, dims, Y)
        fits.append(fit)
    # ALS never lowers the fit (each mode update is an exact least-squares solve)
    assert all(b >= a - 1e-10 for a, b in zip(fits, fits[1:]))
    assert fits[-1] > fits[0] + 0.1
    # started near the generating factors it converges to the noise floor
    Y = [y + 0.05 * rng.standard_normal(y.shape) for y in Yt]
    for _ in range(10):
        Y, lam, fit = cp.cp_als_step(idx, vals, dims, Y)
    assert fit > 0.99


def test_sampled_matches_dense_model():
    dims = (4, 3, 5, 2)
    idx, _ = random_coo(dims, 30, seed=2)
    Y = [f.astype(np.float64) for f in make_factors(dims, 3, seed=2)]
    X = dense_model(Y)
    np.testing.assert_allclose(oracle.sampled(idx, Y), X[tuple(idx.astype(np.int64))], rtol=1e-12)


def test_cpopt_gradient_central_differences():
    dims = (4, 3, 5)
    idx, vals = random_coo(dims, 25, seed=6, value_law="int1to5")
    Y = [f.astype(np.float64) for f in make_factors(dims, 2, seed=6)]
    loss, e, grads = cp.cpopt_loss_grad(idx, vals, dims, Y)
    eps = 1e-6
    for w in range(3):
        for i in range(dims[w]):
            for r in range(2):
                Yp = [y.copy() for y in Y]
                Ym = [y.copy() for y in Y]
                Yp[w][i, r] += eps
                Ym[w][i, r] -= eps
                fd = (cp.cpopt_loss_grad(idx, vals, dims, Yp)[0]
                      - cp.cpopt_loss_grad(idx, vals, dims, Ym)[0]) / (2 * eps)
                assert grads[w][i, r] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_adjoint_identities():
    # M is linear in vals and in each Y_w (w != n):
    # <G, M(v)> = <dvals, v> and <G, M(Y)> = <dY_w, Y_w>
    dims = (6, 5, 4, 3)
    idx, vals = random_coo(dims, 80, seed=13)
    Y = [f.astype(np.float64) for f in make_factors(dims, 3, seed=13)]
    rng = np.random.default_rng(13)
    for n in range(4):
        G = rng.standard_normal((dims[n], 3))
        M = oracle.mttkrp(idx, vals, Y, n, dims)
        lhs = float(np.sum(G * M))
        dvals, dY = cp.mttkrp_adjoint(idx, vals, dims, Y, n, G)
        assert float(dvals @ vals.astype(np.float64)) == pytest.approx(lhs, rel=1e-12)
        for w in range(4):
            if w == n:
                assert dY[w] is None
            else:
                assert float(np.sum(dY[w] * Y[w])) == pytest.approx(lhs, rel=1e-12)
