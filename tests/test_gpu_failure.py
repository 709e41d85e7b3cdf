"""Failure paths on the GPU, driven from the host: a tile-load wait that gives
up (the wait limit set to zero polls) must come back as FLYCOO_ERR_TIMEOUT
with the context still usable, a remapping pass that gave up must leave the
handle refusing further work, and a refused device allocation must come back
as FLYCOO_ERR_OOM.  No kernel traps, faults or waits without a bound."""
import numpy as np
import pytest

import oracle
from synth import make_factors, random_coo

from _util import rel_fro, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS = (300, 200, 250)


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_09131_gb300 as pkg
    pkg._native.lib()
    return pkg


@pytest.fixture(scope="module")
def data():
    idx, vals = random_coo(DIMS, 30_000, seed=41, law="zipf")
    facs = make_factors(DIMS, 32, "normal", seed=41)
    return idx, vals, facs


def _status(err):
    return err.value.status_name


def test_wait_timeout_reported_and_handle_recovers(P, data):
    idx, vals, facs = data
    T = P.FlycooTensor(idx, vals, DIMS, g=1024, bins=17)
    Y = [torch.from_numpy(f).cuda() for f in facs]
    out = torch.empty((DIMS[0], 32), device="cuda")
    P.flycoo_debug_set_wait_limit(T.h, 0)
    P.flycoo_spmttkrp(T.h, 0, Y, out, -1)          # no remap: the layout stays valid
    with pytest.raises(P.FlycooError) as ei:
        P.flycoo_sync(T.h)
    assert _status(ei) == "FLYCOO_ERR_TIMEOUT"
    P.flycoo_sync(T.h)                              # the error word was cleared
    P.flycoo_debug_set_wait_limit(T.h, -1)
    P.flycoo_spmttkrp(T.h, 0, Y, out, -1)
    P.flycoo_sync(T.h)
    ref = oracle.mttkrp(idx, vals, oracle.factors_f64(facs), 0, DIMS)
    assert rel_fro(to_np(out), ref) <= 1e-5


def test_timeout_in_a_remapping_pass_poisons_the_handle(P, data):
    idx, vals, facs = data
    T = P.FlycooTensor(idx, vals, DIMS, g=1024, bins=17)
    Y = [torch.from_numpy(f).cuda() for f in facs]
    out = torch.empty((DIMS[0], 32), device="cuda")
    P.flycoo_debug_set_wait_limit(T.h, 0)
    P.flycoo_spmttkrp(T.h, 0, Y, out, 1)
    with pytest.raises(P.FlycooError) as ei:
        P.flycoo_sync(T.h)
    assert _status(ei) == "FLYCOO_ERR_TIMEOUT"
    assert "layout is undefined" in P.flycoo_last_error()
    P.flycoo_debug_set_wait_limit(T.h, -1)
    out1 = torch.empty((DIMS[1], 32), device="cuda")
    with pytest.raises(P.FlycooError) as ei:
        P.flycoo_spmttkrp(T.h, 1, Y, out1, 2)
    assert _status(ei) == "FLYCOO_ERR_LAYOUT"
    with pytest.raises(P.FlycooError) as ei:
        P.flycoo_remap(T.h, 0)
    assert _status(ei) == "FLYCOO_ERR_LAYOUT"
    # a new handle over the same data is unaffected
    T2 = P.FlycooTensor(idx, vals, DIMS, g=1024, bins=17)
    outs = T2.all_modes(Y)
    torch.cuda.synchronize()
    for n in range(3):
        ref = oracle.mttkrp(idx, vals, oracle.factors_f64(facs), n, DIMS)
        assert rel_fro(to_np(outs[n]), ref) <= 1e-5


def test_als_and_cpopt_report_a_timeout(P, data):
    idx, vals, facs = data
    T = P.FlycooTensor(idx, vals, DIMS, g=1024, bins=17)
    Y = [torch.from_numpy(f).cuda() for f in facs]
    P.flycoo_debug_set_wait_limit(T.h, 0)
    with pytest.raises(P.FlycooError) as ei:
        T.cp_als_step([y.clone() for y in Y])
    assert _status(ei) == "FLYCOO_ERR_TIMEOUT"
    T2 = P.FlycooTensor(idx, vals, DIMS, g=1024, bins=17)
    P.flycoo_debug_set_wait_limit(T2.h, 0)
    grads = [torch.empty_like(y) for y in Y]
    with pytest.raises(P.FlycooError) as ei:
        P.flycoo_cpopt_grad(T2.h, Y, grads)
    assert _status(ei) == "FLYCOO_ERR_TIMEOUT"


def test_refused_allocation_is_oom_and_nothing_leaks(P, data):
    idx, vals, facs = data
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for n in (0, 1, 5, 20):
            P.flycoo_debug_fail_alloc_after(n)
            with pytest.raises(P.FlycooError) as ei:
                P.FlycooTensor(idx, vals, DIMS, g=1024, bins=17)
            assert _status(ei) == "FLYCOO_ERR_OOM"
            assert "test hook" in P.flycoo_last_error()
    finally:
        P.flycoo_debug_fail_alloc_after(-1)
    torch.cuda.synchronize()
    # the failed creates released what they had allocated
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    T = P.FlycooTensor(idx, vals, DIMS, g=1024, bins=17)
    out = T.spmttkrp(0, [torch.from_numpy(f).cuda() for f in facs])
    torch.cuda.synchronize()
    ref = oracle.mttkrp(idx, vals, oracle.factors_f64(facs), 0, DIMS)
    assert rel_fro(to_np(out), ref) <= 1e-5
