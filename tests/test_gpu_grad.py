"""GPU parity of the differentiation path: the spMTTKRP adjoint, the
``SpMTTKRP`` autograd function, and the fused CP-OPT loss / gradient sweep,
against the FP64 oracle, adjoint identities and central finite differences
(eps = 1e-3, FP64)."""
import numpy as np
import pytest

import oracle
from oracle import cp
from synth import make_factors, random_coo

from _util import rel_fro, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_09131_gb300 as pkg
    pkg._native.lib()
    return pkg


def _fac(facs):
    return [torch.from_numpy(f).cuda().contiguous() for f in facs]


@pytest.mark.parametrize("dims,nnz,R,g", [((300, 200, 250), 40_000, 32, 1000), ((40, 50, 30, 20), 20_000, 16, 600),
                                          ((30, 20, 25, 10, 12), 15_000, 64, 333)])
def test_adjoint_matches_oracle_and_identity(P, dims, nnz, R, g):
    N = len(dims)
    idx, vals = random_coo(dims, nnz, seed=3, law="zipf", value_law="lognormal")
    facs = make_factors(dims, R, "normal", seed=3)
    T = P.FlycooTensor(idx, vals, dims, g=g, bins=41)
    Y = _fac(facs)
    Y64 = oracle.factors_f64(facs)
    rng = np.random.default_rng(3)
    for mode in range(N):
        G = rng.standard_normal((dims[mode], R)).astype(np.float32)
        grads = [torch.full_like(y, float("nan")) if w != mode else None for w, y in enumerate(Y)]
        gv = torch.full((nnz,), float("nan"), device="cuda")
        P.flycoo_mttkrp_adjoint(T.h, mode, Y, torch.from_numpy(G).cuda(), grads, gv)
        torch.cuda.synchronize()
        assert T.layout_mode == mode
        dv, dY = cp.mttkrp_adjoint(idx, vals, dims, Y64, mode, G.astype(np.float64), wrt_vals=True)
        M = oracle.mttkrp(idx, vals, Y64, mode, dims)
        lhs = float(np.sum(G.astype(np.float64) * M))
        for w in range(N):
            if w == mode:
                continue
            got = to_np(grads[w])
            assert rel_fro(got, dY[w]) <= TOL, (mode, w, rel_fro(got, dY[w]))
            # <G, M_mode(Y)> = <dY_w, Y_w>
            assert abs(float(np.sum(got.astype(np.float64) * Y64[w])) - lhs) <= 1e-5 * abs(lhs) + 1e-6
        # the value gradient, in input order, and <dvals, vals> = <G, M> (M is linear in the values)
        gvn = to_np(gv).astype(np.float64)
        assert rel_fro(gvn, dv) <= TOL, (mode, rel_fro(gvn, dv))
        assert abs(float(gvn @ vals.astype(np.float64)) - lhs) <= 1e-5 * np.abs(dv) @ np.abs(vals) + 1e-6


def test_adjoint_bf16_factors(P):
    # BF16 factors and a BF16 upstream gradient, FP32 accumulation: within 1e-5
    # of the oracle on the same BF16 values, within the 1e-2 bar of the FP32 ones
    dims = (200, 150, 120)
    nnz, R, mode = 25_000, 32, 1
    idx, vals = random_coo(dims, nnz, seed=8, law="zipf", value_law="lognormal")
    facs = make_factors(dims, R, "normal", seed=8)
    G = np.random.default_rng(8).standard_normal((dims[mode], R)).astype(np.float32)
    T = P.FlycooTensor(idx, vals, dims, g=512, bins=23)
    Yb = [y.bfloat16() for y in _fac(facs)]
    grads = [torch.empty((d, R), device="cuda") if w != mode else None for w, d in enumerate(dims)]
    gv = torch.empty(nnz, device="cuda")
    P.flycoo_mttkrp_adjoint(T.h, mode, Yb, torch.from_numpy(G).cuda().bfloat16(), grads, gv)
    torch.cuda.synchronize()
    Yb64 = oracle.factors_f64(facs, bf16=True)
    Gb64 = oracle.factors_f64([G], bf16=True)[0]
    dvb, dYb = cp.mttkrp_adjoint(idx, vals, dims, Yb64, mode, Gb64, wrt_vals=True)
    dv, dY = cp.mttkrp_adjoint(idx, vals, dims, oracle.factors_f64(facs), mode, G.astype(np.float64), wrt_vals=True)
    for w in (0, 2):
        assert rel_fro(to_np(grads[w]), dYb[w]) <= TOL
        assert rel_fro(to_np(grads[w]), dY[w]) <= 1e-2
    assert rel_fro(to_np(gv), dvb) <= TOL
    assert rel_fro(to_np(gv), dv) <= 1e-2


def test_value_gradient_central_differences(P):
    # L(v) = <G, M_mode(v)>: central differences (eps = 1e-3) of the FP64 oracle
    # along random unit directions V of the values against <dvals_gpu, V>
    dims = (60, 50, 40)
    nnz, R = 6_000, 16
    idx, vals = random_coo(dims, nnz, seed=9, value_law="normal")
    facs = make_factors(dims, R, "normal", seed=9)
    Y64 = oracle.factors_f64(facs)
    rng = np.random.default_rng(9)
    T = P.FlycooTensor(idx, vals, dims, g=256, bins=11)
    for mode in range(3):
        G = rng.standard_normal((dims[mode], R)).astype(np.float32)
        gv = torch.empty(nnz, device="cuda")
        P.flycoo_mttkrp_adjoint(T.h, mode, _fac(facs), torch.from_numpy(G).cuda(), [None] * 3, gv)
        g64 = to_np(gv).astype(np.float64)
        eps = 1e-3
        for _ in range(4):
            V = rng.standard_normal(nnz)
            V /= np.linalg.norm(V)
            Lp = float(np.sum(G * oracle.mttkrp(idx, vals + eps * V, Y64, mode, dims)))
            Lm = float(np.sum(G * oracle.mttkrp(idx, vals - eps * V, Y64, mode, dims)))
            assert float(g64 @ V) == pytest.approx((Lp - Lm) / (2 * eps), rel=1e-4, abs=1e-5)


def test_spmttkrp_autograd_backward(P):
    dims = (120, 90, 70)
    idx, vals = random_coo(dims, 15_000, seed=4, law="zipf")
    facs = make_factors(dims, 16, "normal", seed=4)
    T = P.FlycooTensor(idx, vals, dims, g=512, bins=17)
    Y = [y.clone().requires_grad_(True) for y in _fac(facs)]
    v = torch.from_numpy(vals).cuda().requires_grad_(True)
    G = torch.randn((dims[1], 16), device="cuda")
    M = P.spmttkrp(T, 1, Y, vals=v)
    (M * G).sum().backward()
    assert Y[1].grad is None
    Y64 = oracle.factors_f64(facs)
    dv, dY = cp.mttkrp_adjoint(idx, vals, dims, Y64, 1, to_np(G).astype(np.float64), wrt_vals=True)
    for w in (0, 2):
        assert rel_fro(to_np(Y[w].grad), dY[w]) <= TOL
    assert rel_fro(to_np(v.grad), dv) <= TOL
    np.testing.assert_allclose(to_np(M.detach()), oracle.mttkrp(idx, vals, Y64, 1, dims), rtol=1e-4, atol=1e-4)
    # without values only the factors get gradients; BF16 factors give BF16 gradients
    Yb = [y.detach().bfloat16().requires_grad_(True) for y in Y]
    (P.spmttkrp(T, 0, Yb) * torch.randn((dims[0], 16), device="cuda")).sum().backward()
    assert Yb[0].grad is None and Yb[1].grad.dtype == torch.bfloat16 and Yb[2].grad is not None


@pytest.mark.parametrize("dims,nnz,R", [((200, 150, 180), 30_000, 32), ((30, 40, 20, 25), 12_000, 16)])
def test_cpopt_loss_and_gradient_vs_oracle(P, dims, nnz, R):
    N = len(dims)
    idx, vals = random_coo(dims, nnz, seed=5, law="zipf", value_law="int1to5")
    facs = make_factors(dims, R, "normal_over_sqrt_r", seed=5)
    T = P.FlycooTensor(idx, vals, dims, g=700, bins=29)
    Y = _fac(facs)
    grads = [torch.full_like(y, float("nan")) for y in Y]
    loss = P.flycoo_cpopt_grad(T.h, Y, grads)
    torch.cuda.synchronize()
    assert T.layout_mode == 0
    L64, e, G64 = cp.cpopt_loss_grad(idx, vals, dims, oracle.factors_f64(facs))
    assert loss == pytest.approx(L64, rel=TOL)
    for n in range(N):
        assert rel_fro(to_np(grads[n]), G64[n]) <= TOL, (n, rel_fro(to_np(grads[n]), G64[n]))


def test_cpopt_gradient_central_differences(P):
    # directional derivative of the FP64 oracle loss by central differences
    # (eps = 1e-3) against <grad_gpu, V> along random unit directions V (unit
    # Frobenius norm over all factors, so the eps^2 truncation term stays small)
    dims = (60, 50, 40)
    idx, vals = random_coo(dims, 6_000, seed=6, value_law="int1to5")
    facs = make_factors(dims, 16, "normal_over_sqrt_r", seed=6)
    T = P.FlycooTensor(idx, vals, dims, g=256, bins=11)
    grads = [torch.empty_like(y) for y in _fac(facs)]
    P.flycoo_cpopt_grad(T.h, _fac(facs), grads)
    gg = [to_np(g).astype(np.float64) for g in grads]
    Y64 = oracle.factors_f64(facs)
    rng = np.random.default_rng(6)
    eps = 1e-3
    for _ in range(8):
        V = [rng.standard_normal(y.shape) for y in Y64]
        nv = np.sqrt(sum(float(np.sum(v * v)) for v in V))
        V = [v / nv for v in V]
        Lp = cp.cpopt_loss_grad(idx, vals, dims, [y + eps * v for y, v in zip(Y64, V)])[0]
        Lm = cp.cpopt_loss_grad(idx, vals, dims, [y - eps * v for y, v in zip(Y64, V)])[0]
        fd = (Lp - Lm) / (2 * eps)
        an = sum(float(np.sum(g * v)) for g, v in zip(gg, V))
        assert an == pytest.approx(fd, rel=1e-4, abs=1e-5)


def test_cpopt_autograd_descent(P):
    dims = (80, 70, 60)
    idx, vals = random_coo(dims, 10_000, seed=7, value_law="int1to5")
    facs = make_factors(dims, 16, "normal_over_sqrt_r", seed=7)
    T = P.FlycooTensor(idx, vals, dims, g=512, bins=13)
    Y = [y.clone().requires_grad_(True) for y in _fac(facs)]
    opt = torch.optim.Adam(Y, lr=0.02)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        L = P.cpopt_loss(T, Y)
        L.backward()
        opt.step()
        losses.append(float(L.detach()))
    assert losses[-1] < 0.75 * losses[0]
    assert sum(b < a for a, b in zip(losses, losses[1:])) >= 25
    # the autograd loss equals the oracle's at the final factors
    L64 = cp.cpopt_loss_grad(idx, vals, dims, [to_np(y).astype(np.float64) for y in Y])[0]
    assert float(P.cpopt_loss(T, Y)) == pytest.approx(L64, rel=1e-5)


def test_cpopt_nell1_shaped_sample(P):
    # the Nell-1-sized shape (4.8M x 1.8M x 1.8M, Zipf(1.2), values 1..5) at 3M nonzeros
    dims = (4_800_000, 1_800_000, 1_800_000)
    idx, vals = random_coo(dims, 3_000_000, seed=0, law="zipf", zipf_s=1.2, value_law="int1to5")
    facs = make_factors(dims, 32, "normal_over_sqrt_r", seed=0)
    T = P.FlycooTensor(idx, vals, dims)
    Y = _fac(facs)
    grads = [torch.empty_like(y) for y in Y]
    loss = P.flycoo_cpopt_grad(T.h, Y, grads)
    L64, e, G64 = cp.cpopt_loss_grad(idx, vals, dims, oracle.factors_f64(facs))
    assert loss == pytest.approx(L64, rel=TOL)
    for n in range(3):
        assert rel_fro(to_np(grads[n]), G64[n]) <= TOL
