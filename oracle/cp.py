"""FP64 oracle for the CP layers above spMTTKRP -- TEST INFRASTRUCTURE ONLY.

* ``cp_als_step``: one iteration of CP-ALS (Algorithm 1).  Algorithm 1
  writes the factor update as "A <- spMTTKRP(...)" followed by "Normalize";
  the paper leaves out the least-squares solve, so the update follows the
  Kolda-Bader CP-ALS it cites: Y_n <- M_n (hadamard_{w != n} Y_w^T Y_w)^{-1},
  then the columns of Y_n are scaled to unit 2-norm and the norms kept in
  lambda.  Modes are updated in order 0..N-1, each with the newest factors.
* ``cpopt_loss_grad``: weighted CP (CP-OPT) loss on the observed entries,
  L = 1/2 sum_x (x - m_x)^2 with m_x the CPD model value (Eq. 1) at x, and
  its gradient dL/dY_n = -spMTTKRP_n(residuals).
* ``mttkrp_adjoint``: adjoint of spMTTKRP of mode n with respect to the
  nonzero values and to every other factor.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this module.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import mttkrp, round_bf16, sampled

__all__ = ["NotSPD", "cholesky", "chol_solve_rows", "cp_als_step", "cp_fit", "cpopt_loss_grad",
           "mttkrp_adjoint"]


class NotSPD(ValueError):
    """The R x R system of the ALS update is not symmetric positive definite."""


def cholesky(V: np.ndarray) -> np.ndarray:
    """Lower-triangular L with L L^T = V, by the textbook column algorithm.

    Raises ``NotSPD`` when a pivot is not positive."""
    V = np.asarray(V, dtype=np.float64)
    R = V.shape[0]
    L = np.zeros_like(V)
    for j in range(R):
        d = V[j, j] - sum(L[j, k] * L[j, k] for k in range(j))
        if not d > 0.0:
            raise NotSPD(f"pivot {j} is {d!r}")
        L[j, j] = math.sqrt(d)
        for i in range(j + 1, R):
            L[i, j] = (V[i, j] - sum(L[i, k] * L[j, k] for k in range(j))) / L[j, j]
    return L


def chol_solve_rows(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = B V^{-1} for V = L L^T (V symmetric): solve V x_i = b_i per row i
    by forward then backward substitution, vectorised over the rows (the
    rows are held transposed so each substitution step is a contiguous
    matrix-vector product)."""
    Bt = np.ascontiguousarray(np.asarray(B, dtype=np.float64).T)
    R = L.shape[0]
    Zt = np.empty_like(Bt)
    for j in range(R):
        Zt[j] = (Bt[j] - L[j, :j] @ Zt[:j]) / L[j, j]
    Xt = np.empty_like(Bt)
    for j in range(R - 1, -1, -1):
        Xt[j] = (Zt[j] - L[j + 1:, j] @ Xt[j + 1:]) / L[j, j]
    return np.ascontiguousarray(Xt.T)


def _store(Y: np.ndarray, store: str) -> np.ndarray:
    if store == "f64":
        return Y
    if store == "f32":
        return Y.astype(np.float32).astype(np.float64)
    if store == "bf16":
        return round_bf16(Y.astype(np.float32)).astype(np.float64)
    raise ValueError(store)


def cp_fit(vals, factors: Sequence[np.ndarray], lam: np.ndarray, M_last: np.ndarray) -> float:
    """fit = 1 - ||X - Xhat|| / ||X|| with ||Xhat||^2 = lam^T (hadamard_w G_w) lam
    and <X, Xhat> = sum_r lam_r sum_i M_{N-1}[i,r] Y_{N-1}[i,r], where M_{N-1}
    is the spMTTKRP of the last mode taken with the final other factors."""
    vals = np.asarray(vals, dtype=np.float64)
    normx2 = float(vals @ vals)
    V = np.ones((lam.size, lam.size))
    for Y in factors:
        V *= Y.T @ Y
    normxh2 = float(lam @ V @ lam)
    inner = float(lam @ np.sum(M_last * factors[-1], axis=0))
    resid2 = max(normx2 + normxh2 - 2.0 * inner, 0.0)
    return 1.0 - math.sqrt(resid2) / math.sqrt(normx2)


def cp_als_step(idx, vals, dims, factors: Sequence[np.ndarray], store: str = "f64"
                ) -> Tuple[List[np.ndarray], np.ndarray, float]:
    """One CP-ALS iteration over all modes.  ``store`` rounds each updated
    factor to the storage precision ("f64", "f32" or "bf16") before it is used
    again, as factor storage in that precision does.  Returns
    ``(factors, lambda, fit)``."""
    Y = [np.asarray(f, dtype=np.float64).copy() for f in factors]
    N = len(Y)
    R = Y[0].shape[1]
    G = [y.T @ y for y in Y]
    lam = np.ones(R)
    M = None
    for n in range(N):
        M = mttkrp(idx, vals, Y, n, dims)
        V = np.ones((R, R))
        for w in range(N):
            if w != n:
                V *= G[w]
        Yn = chol_solve_rows(cholesky(V), M)
        lam = np.sqrt(np.sum(Yn * Yn, axis=0))
        safe = np.where(lam > 0.0, lam, 1.0)
        Yn = _store(Yn / safe, store)
        Y[n] = Yn
        G[n] = Yn.T @ Yn
    fit = cp_fit(vals, Y, lam, M)
    return Y, lam, fit


def cpopt_loss_grad(idx, vals, dims, factors: Sequence[np.ndarray]):
    """CP-OPT on observed entries: ``(loss, residuals, grads)`` with
    residual e_x = x - m_x and dL/dY_n = -spMTTKRP_n with values e."""
    Y = [np.asarray(f, dtype=np.float64) for f in factors]
    m = sampled(idx, Y)
    e = np.asarray(vals, dtype=np.float64) - m
    loss = 0.5 * float(e @ e)
    grads = [-mttkrp(idx, e, Y, n, dims) for n in range(len(Y))]
    return loss, e, grads


def mttkrp_adjoint(idx, vals, dims, factors: Sequence[np.ndarray], mode: int, G: np.ndarray,
                   wrt_vals: bool = True):
    """Adjoint of M = spMTTKRP_mode(vals, Y) against an upstream ``G`` (I_mode x R).

    d<G,M>/d val_x = sum_r G[c_mode, r] prod_{w != mode} Y_w[c_w, r];
    d<G,M>/d Y_w   = spMTTKRP_w(vals, Y with Y_mode replaced by G), w != mode.
    Returns ``(dvals or None, [dY_w or None for each w])``."""
    Y = [np.asarray(f, dtype=np.float64) for f in factors]
    F = list(Y)
    F[mode] = np.asarray(G, dtype=np.float64)
    dvals = sampled(idx, F) if wrt_vals else None
    dY: List[Optional[np.ndarray]] = []
    for w in range(len(Y)):
        dY.append(None if w == mode else mttkrp(idx, vals, F, w, dims))
    return dvals, dY
