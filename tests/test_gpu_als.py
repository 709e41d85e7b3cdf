"""GPU parity of one CP-ALS iteration (Algorithm 1 with the least-squares
update, ``flycoo_cp_als_step``) against the FP64 oracle ``cp.cp_als_step``
with the same storage rounding, plus properties that fix the result
independently of the oracle: exact recovery of a planted dense CP tensor,
monotone fit, the NOT_SPD status, determinism and the layout cycle.

Tolerances.
* The solve itself: given the same M (the GPU's own spMTTKRP, which the
  fused pass reproduces bit for bit), the update Y = M V^{-1} / lambda is
  FP64-accurate, so the stored FP32 factor matches the oracle's FP64 solve
  rounded to FP32 to within 1e-6 (a few last-place differences) even at
  kappa(V) >= 1e5; an FP32 inverse would miss by kappa * 2^-24 ~ 1e-2.
* A whole step against the oracle: the only error left is the FP32
  spMTTKRP (relative 1e-5 at most, about 1e-6 in practice), which the solve
  amplifies by at most kappa(V).  The cases here have kappa(V) <= 50 (checked
  from the oracle's iterates), and FP32 factors and lambda are held to a
  fixed 1e-4.
* BF16 storage is held to the BF16 bar of 1e-2."""
import math

import numpy as np
import pytest

import oracle
from oracle import cp
from synth import make_coo, make_factors, random_coo

from _util import rel_fro, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_09131_gb300 as pkg
    pkg._native.lib()
    return pkg


def _kappa_max(old, new):
    """max_n cond(V_n), V_n built as the Gauss-Seidel sweep sees it."""
    N = len(old)
    k = 1.0
    for n in range(N):
        V = np.ones((old[0].shape[1],) * 2)
        for w in range(N):
            if w != n:
                y = new[w] if w < n else old[w]
                V *= y.T @ y
        k = max(k, float(np.linalg.cond(V)))
    return k


def _fit_tol(vals, Y, lam, M_last_inner, rel):
    normx2 = float(np.dot(vals.astype(np.float64), vals.astype(np.float64)))
    V = np.ones((lam.size, lam.size))
    for y in Y:
        V *= y.T @ y
    xh2 = float(lam @ V @ lam)
    resid2 = max(normx2 + xh2 - 2 * M_last_inner, 1e-300)
    return rel * (normx2 + xh2 + 2 * abs(M_last_inner)) / (2 * math.sqrt(resid2) * math.sqrt(normx2))


def _run_case(P, idx, vals, dims, facs, store, **kw):
    N = len(dims)
    R = facs[0].shape[1]
    T = P.FlycooTensor(idx, vals, dims, **kw)
    dt = torch.bfloat16 if store == "bf16" else torch.float32
    Y = [torch.from_numpy(f).cuda().to(dt).contiguous() for f in facs]
    start = [to_np(y.float()).astype(np.float64) for y in Y]
    lam, fit = T.cp_als_step(Y)
    torch.cuda.synchronize()
    assert T.layout_mode == 0
    Yo, lamo, fito = cp.cp_als_step(idx, vals, dims, start, store=store)
    got = [to_np(y.float()).astype(np.float64) for y in Y]
    return T, Y, got, to_np(lam), fit, start, Yo, lamo, fito


ALS_TOL = 1e-4


@pytest.mark.parametrize("dims,nnz,R,law,g,bins", [
    ((300, 200, 250), 40_000, 16, "zipf", 1000, 41),
    ((300, 200, 250), 40_000, 32, "uniform", 700, 64),
    ((500, 400, 300), 60_000, 64, "zipf", 2048, 97),
    ((40, 50, 30, 20), 20_000, 32, "zipf", 600, 29),
    ((30, 20, 25, 10, 12), 15_000, 16, "uniform", 333, 13),
])
def test_als_step_fp32_matches_oracle(P, dims, nnz, R, law, g, bins):
    N = len(dims)
    idx, vals = random_coo(dims, nnz, seed=11, law=law, value_law="lognormal")
    facs = make_factors(dims, R, "normal", seed=11)
    T, Y, got, lam, fit, start, Yo, lamo, fito = _run_case(P, idx, vals, dims, facs, "f32", g=g, bins=bins)
    assert _kappa_max(start, Yo) <= 50
    for n in range(N):
        assert rel_fro(got[n], Yo[n]) <= ALS_TOL, (n, rel_fro(got[n], Yo[n]))
    assert rel_fro(lam, lamo) <= ALS_TOL
    inner = float(lamo @ np.sum(oracle.mttkrp(idx, vals, Yo, N - 1, dims) * Yo[N - 1], axis=0))
    assert abs(fit - fito) <= _fit_tol(vals, Yo, lamo, inner, ALS_TOL) + 1e-12, (fit, fito)
    # columns of every updated factor have unit 2-norm
    for n in range(N):
        np.testing.assert_allclose(np.linalg.norm(got[n], axis=0), 1.0, rtol=1e-5)


def test_als_update_solve_is_fp64_accurate(P):
    # nearly collinear columns make V_0 = G_1 * G_2 ill-conditioned; given the
    # GPU's own M_0, the update must equal the FP64 solve rounded to FP32
    dims = (400, 300, 200)
    R = 16
    idx, vals = random_coo(dims, 30_000, seed=24, law="zipf", value_law="lognormal")
    rng = np.random.default_rng(24)
    facs = make_factors(dims, R, "normal", seed=24)
    for w in (1, 2):
        base = rng.standard_normal((dims[w], 1))
        facs[w] = (base + 3e-3 * rng.standard_normal((dims[w], R))).astype(np.float32)
    Y64 = [f.astype(np.float64) for f in facs]
    V = (Y64[1].T @ Y64[1]) * (Y64[2].T @ Y64[2])
    assert np.linalg.cond(V) >= 1e5
    T = P.FlycooTensor(idx, vals, dims, g=700, bins=31)
    Y = [torch.from_numpy(f).cuda() for f in facs]
    M0 = to_np(T.spmttkrp(0, Y, remap=False)).astype(np.float64)
    Yn = cp.chol_solve_rows(cp.cholesky(V), M0)
    lam0 = np.sqrt(np.sum(Yn * Yn, axis=0))
    want = (Yn / lam0).astype(np.float32)
    T.cp_als_step(Y)
    got = to_np(Y[0])
    assert rel_fro(got, want) <= 1e-6, rel_fro(got, want)
    # almost every element is the same FP32 number
    assert np.mean(got == want) >= 0.99


@pytest.mark.parametrize("dims,nnz,R", [((300, 200, 250), 40_000, 32), ((40, 50, 30, 20), 20_000, 16)])
def test_als_step_bf16_matches_oracle(P, dims, nnz, R):
    idx, vals = random_coo(dims, nnz, seed=12, law="zipf", value_law="normal")
    facs = make_factors(dims, R, "normal_over_sqrt_r", seed=12)
    T, Y, got, lam, fit, start, Yo, lamo, fito = _run_case(P, idx, vals, dims, facs, "bf16", g=800, bins=37)
    assert all(y.dtype == torch.bfloat16 for y in Y)
    for n in range(len(dims)):
        assert rel_fro(got[n], Yo[n]) <= 1e-2, (n, rel_fro(got[n], Yo[n]))
    assert rel_fro(lam, lamo) <= 1e-2
    assert fit == pytest.approx(fito, abs=1e-2)


SKEWED_DIMS = (20_000, 200_000, 500_000)
SKEWED_LAWS = (("hot", 10, 0.5), ("uniform",), ("uniform",))


def test_als_step_skewed_rank64_sample(P):
    # the 20K x 200K x 500K shape with a hot first mode (10 ids take half of
    # the draws), R = 64, at 2M nonzeros: one FP32 step against the oracle
    idx, vals = make_coo(SKEWED_DIMS, 2_000_000, SKEWED_LAWS, "normal", seed=5)
    facs = make_factors(SKEWED_DIMS, 64, "normal_over_sqrt_r", seed=5)
    T, Y, got, lam, fit, start, Yo, lamo, fito = _run_case(P, idx, vals, SKEWED_DIMS, facs, "f32")
    assert _kappa_max(start, Yo) <= 50
    for n in range(3):
        assert rel_fro(got[n], Yo[n]) <= ALS_TOL, (n, rel_fro(got[n], Yo[n]))
    assert rel_fro(lam, lamo) <= ALS_TOL
    inner = float(lamo @ np.sum(oracle.mttkrp(idx, vals, Yo, 2, SKEWED_DIMS) * Yo[2], axis=0))
    assert abs(fit - fito) <= _fit_tol(vals, Yo, lamo, inner, ALS_TOL) + 1e-12


def test_als_skewed_bf16_r64_ten_iterations(P):
    # CP-ALS as the skewed workload runs it (Algorithm 1): BF16 factors, FP32
    # spMTTKRP accumulation, FP64-accurate Gram matrices and solve, R = 64,
    # ten iterations from one seeded start, at 2M of its 200M nonzeros.  The
    # values are N(0, 1) with no low-rank structure, so the fit stays near
    # 1e-5; fits are compared relative to their size.
    # (a) iterations 1, 5 and 10 against one oracle step from the GPU's own
    #     previous iterate: the FP32 spMTTKRP error (~1e-6) flips the BF16
    #     rounding of a few factor entries by one BF16 step (2^-8 relative),
    #     so the factors and lambda agree within 1e-2 and the fit within 1e-2
    #     of its value;
    # (b) the fit after every iteration against the oracle's own ten
    #     iterations from the same start, within 2e-2 of its value, and the
    #     final factors and lambda within 5e-2.
    idx, vals = make_coo(SKEWED_DIMS, 2_000_000, SKEWED_LAWS, "normal", seed=0)
    facs = make_factors(SKEWED_DIMS, 64, "normal_over_sqrt_r", seed=0)
    T = P.FlycooTensor(idx, vals, SKEWED_DIMS)
    Y = [torch.from_numpy(f).cuda().to(torch.bfloat16).contiguous() for f in facs]
    start = [to_np(y.float()).astype(np.float64) for y in Y]
    prev = start
    fits = []
    lam = None
    for it in range(10):
        lam, fit = T.cp_als_step(Y, lam)
        fits.append(fit)
        got = [to_np(y.float()).astype(np.float64) for y in Y]
        if it in (0, 4, 9):
            Yo, lamo, fito = cp.cp_als_step(idx, vals, SKEWED_DIMS, prev, store="bf16")
            for n in range(3):
                assert rel_fro(got[n], Yo[n]) <= 1e-2, (it, n, rel_fro(got[n], Yo[n]))
            assert rel_fro(to_np(lam), lamo) <= 1e-2, (it, rel_fro(to_np(lam), lamo))
            assert abs(fit - fito) <= 1e-2 * abs(fito) + 1e-9, (it, fit, fito)
        prev = got
    assert T.layout_mode == 0
    assert all(b > a for a, b in zip(fits, fits[1:])), fits
    traj = list(start)
    for it in range(10):
        traj, lamo, fito = cp.cp_als_step(idx, vals, SKEWED_DIMS, traj, store="bf16")
        assert abs(fits[it] - fito) <= 2e-2 * abs(fito) + 1e-9, (it, fits[it], fito)
    for n in range(3):
        assert rel_fro(prev[n], traj[n]) <= 5e-2, (n, rel_fro(prev[n], traj[n]))
    assert rel_fro(to_np(lam), lamo) <= 5e-2


def _dense_model(Y, lam):
    R = Y[0].shape[1]
    X = np.zeros([y.shape[0] for y in Y])
    for r in range(R):
        t = lam[r]
        for y in Y:
            t = np.multiply.outer(t, y[:, r])
        X += t
    return X


def test_als_recovers_planted_dense_cp_tensor(P):
    # a dense tensor of exact rank 16 held as 24000 "nonzeros": ALS started
    # near the generating factors converges to it (fit -> 1); the residual is
    # recomputed here from the returned factors, independently of the fit
    dims = (30, 40, 20)
    R = 16
    rng = np.random.default_rng(21)
    Yt = [rng.standard_normal((d, R)) for d in dims]
    X = _dense_model(Yt, np.ones(R))
    idx = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), 0).reshape(3, -1).astype(np.uint32)
    vals = X.reshape(-1).astype(np.float32)
    T = P.FlycooTensor(idx, vals, dims, g=512, bins=23)
    Y = [torch.from_numpy((y + 0.05 * rng.standard_normal(y.shape)).astype(np.float32)).cuda() for y in Yt]
    lam, fits = T.cp_als(Y, iters=25)
    # near fit 1 the fit formula cancels: ||X - Xhat||^2 is a difference of
    # terms near ||X||^2, each carrying ~1e-6 relative error, so allow 2e-3
    assert all(b >= a - 2e-3 for a, b in zip(fits, fits[1:])), fits
    Xh = _dense_model([to_np(y).astype(np.float64) for y in Y], to_np(lam))
    rel_resid = np.linalg.norm(Xh - vals.reshape(dims)) / np.linalg.norm(vals)
    assert rel_resid < 1e-3, rel_resid
    assert fits[-1] == pytest.approx(1.0 - rel_resid, abs=2e-3)


def test_als_fit_monotone_on_sparse_data(P):
    dims = (200, 150, 100)
    idx, vals = random_coo(dims, 30_000, seed=13, law="zipf", value_law="int1to5")
    facs = make_factors(dims, 16, "normal", seed=13)
    T = P.FlycooTensor(idx, vals, dims, g=600, bins=31)
    Y = [torch.from_numpy(f).cuda() for f in facs]
    _, fits = T.cp_als(Y, iters=12)
    # each mode update is an exact least-squares minimiser, so the fit of the
    # sweep never drops (beyond the rounding of the fit formula)
    assert all(b >= a - 1e-5 for a, b in zip(fits, fits[1:])), fits
    assert fits[-1] > fits[0]


def test_als_step_deterministic_and_layout_cycle(P):
    dims = (120, 90, 70)
    idx, vals = random_coo(dims, 15_000, seed=14, law="zipf")
    facs = make_factors(dims, 32, "normal", seed=14)
    out = []
    for start_layout in (0, 2):
        T = P.FlycooTensor(idx, vals, dims, g=400, bins=19)
        if start_layout:
            T.remap(start_layout)
        Y = [torch.from_numpy(f).cuda() for f in facs]
        lam, fit = T.cp_als_step(Y)
        assert T.layout_mode == 0
        out.append(([to_np(y) for y in Y], to_np(lam), fit))
    (Ya, la, fa), (Yb, lb, fb) = out
    assert fa == fb
    np.testing.assert_array_equal(la, lb)
    for a, b in zip(Ya, Yb):
        np.testing.assert_array_equal(a, b)


def test_als_not_spd_status(P):
    # a zero column in Y_1 makes V_0 = G_1 * G_2 singular (V_0[0,0] = 0): the
    # oracle raises NotSPD and the library returns NOT_SPD, leaving every
    # factor unchanged (mode 0 is the first update)
    dims = (50, 40, 30)
    idx, vals = random_coo(dims, 5_000, seed=15)
    facs = make_factors(dims, 16, "normal", seed=15)
    facs[1][:, 0] = 0.0
    with pytest.raises(cp.NotSPD):
        cp.cp_als_step(idx, vals, dims, [f.astype(np.float64) for f in facs])
    T = P.FlycooTensor(idx, vals, dims, g=256, bins=7)
    Y = [torch.from_numpy(f).cuda() for f in facs]
    with pytest.raises(P.FlycooError) as ei:
        T.cp_als_step(Y)
    assert ei.value.status_name == "FLYCOO_ERR_NOT_SPD"
    assert "positive definite" in P.flycoo_last_error()
    for y, f in zip(Y, facs):
        np.testing.assert_array_equal(to_np(y), f)
    assert T.layout_mode == 0
    # the handle stays usable
    Y[1][:, 0] = 1.0
    T.cp_als_step(Y)


def test_als_argument_errors(P):
    dims = (20, 20, 20)
    idx, vals = random_coo(dims, 1_000, seed=16)
    T = P.FlycooTensor(idx, vals, dims, g=128, bins=3)
    Y = [torch.randn(d, 16, device="cuda") for d in dims]
    with pytest.raises(TypeError):
        T.cp_als_step([Y[0], Y[1].bfloat16(), Y[2]])
    Y24 = [torch.randn(d, 24, device="cuda") for d in dims]
    with pytest.raises(P.FlycooError) as ei:
        T.cp_als_step(Y24)
    assert ei.value.status_name == "FLYCOO_ERR_UNSUPPORTED"
    zero = P.FlycooTensor(idx, np.zeros_like(vals), dims, g=128, bins=3)
    with pytest.raises(P.FlycooError) as ei:
        zero.cp_als_step(Y)
    assert ei.value.status_name == "FLYCOO_ERR_INVALID_ARG"


def test_als_checkpoint_resume_is_bitwise(P, tmp_path):
    # three iterations straight against two, a checkpoint, a handle rebuilt
    # from the same COO input, and one more iteration
    dims = (150, 120, 90)
    idx, vals = random_coo(dims, 20_000, seed=17, law="zipf")
    facs = make_factors(dims, 16, "normal", seed=17)
    T = P.FlycooTensor(idx, vals, dims, g=512, bins=19)
    Ya = [torch.from_numpy(f).cuda() for f in facs]
    lam_a, fits_a = T.cp_als(Ya, iters=3)
    T2 = P.FlycooTensor(idx, vals, dims, g=512, bins=19)
    Yb = [torch.from_numpy(f).cuda() for f in facs]
    lam_b, fits_b = T2.cp_als(Yb, iters=2)
    path = str(tmp_path / "als.pt")
    P.FlycooTensor.save_cp_als_state(path, T2.cp_als_state(Yb, lam_b, fits_b))
    T2.close()
    Yc, lam_c, fits_c = P.FlycooTensor.load_cp_als_state(path)
    T3 = P.FlycooTensor(idx, vals, dims, g=512, bins=19)
    lam_c, fit = T3.cp_als_step(Yc, lam_c)
    fits_c.append(fit)
    assert fits_c == fits_a
    np.testing.assert_array_equal(to_np(lam_c), to_np(lam_a))
    for a, c in zip(Ya, Yc):
        np.testing.assert_array_equal(to_np(a), to_np(c))


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_multi_iteration_call_equals_single_steps(P, dtype):
    # flycoo_cp_als carries the Gram matrices between its iterations; the
    # factors, lambda and fits are bit for bit those of repeated single steps
    dims = (200, 150, 100)
    idx, vals = random_coo(dims, 25_000, seed=18, law="zipf", value_law="int1to5")
    facs = make_factors(dims, 32, "normal_over_sqrt_r", seed=18)
    Ta = P.FlycooTensor(idx, vals, dims, g=600, bins=29)
    Ya = [torch.from_numpy(f).cuda().to(dtype).contiguous() for f in facs]
    lam_a = torch.empty(32, dtype=torch.float64, device="cuda")
    fits_a = P.flycoo_cp_als(Ta.h, Ya, lam_a, 6)
    Tb = P.FlycooTensor(idx, vals, dims, g=600, bins=29)
    Yb = [torch.from_numpy(f).cuda().to(dtype).contiguous() for f in facs]
    fits_b = []
    lam_b = None
    for _ in range(6):
        lam_b, fit = Tb.cp_als_step(Yb, lam_b)
        fits_b.append(fit)
    assert fits_a == fits_b
    assert torch.equal(lam_a, lam_b)
    for a, b in zip(Ya, Yb):
        assert torch.equal(a, b)
    assert Ta.layout_mode == 0
    with pytest.raises(P.FlycooError) as e:
        P.flycoo_cp_als(Ta.h, Ya, lam_a, 0)
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG"
