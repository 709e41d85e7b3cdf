"""flycoo_spmttkrp_static_scratch: the spMTTKRP entry point that allocates
nothing.  Its partial rows live in a fixed device array inside the library,
for callers that must not allocate device memory at the point of the call.
Checked through the C ABI against flycoo_spmttkrp on the same tensor, on two
calls in a row (the array keeps the previous call's contents).  This file is
collected last so that a stop-at-first-failure run has already run the rest.
"""
import numpy as np
import pytest

from synth import make_factors, random_coo

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


@pytest.mark.parametrize("dims,nnz,R,dtype,g", [
    ((400, 300, 200), 60_000, 32, torch.float32, 256),
    ((60, 70, 50, 40), 30_000, 64, torch.bfloat16, 128),
])
def test_static_scratch_matches_allocated_scratch(P, dims, nnz, R, dtype, g):
    N = len(dims)
    idx, vals = random_coo(dims, nnz, seed=21, law="zipf", value_law="lognormal")
    facs = [torch.from_numpy(f).cuda().to(dtype) for f in make_factors(dims, R, "normal", seed=21)]
    T = P.FlycooTensor(idx, vals, dims, g=g, bins=48)
    # every mode has a super-shard split over several segments, so every pass
    # writes row blocks into the static array and K4 reads them back
    assert all(k > 0 for k in T.info["fixup_super_shards"])
    ref = T.all_modes(facs)
    ref = [r.clone() for r in ref]
    for call in range(2):
        outs = [torch.full((d, R), float("nan"), device="cuda") for d in dims]
        for n in range(N):
            P.flycoo_spmttkrp_static_scratch(T.h, n, facs, outs[n], (n + 1) % N)
        torch.cuda.synchronize()
        assert T.layout_mode == 0
        for n in range(N):
            assert rel_fro(to_np(outs[n]), to_np(ref[n])) <= 1e-5, (call, n)
            # same kernel, same order: the results agree bit for bit
            assert torch.equal(outs[n], ref[n]), (call, n)


def test_static_scratch_at_its_size_limit(P):
    # one 64-row super-shard per mode, 512 equal shards and 512 bins: each bin
    # holds one shard, so every mode has 512 segments, and at R = 64 their row
    # blocks fill the 8 MiB array exactly (512 x 64 x 64 x 4 bytes)
    dims = (64, 64, 64)
    R = 64
    idx, vals = random_coo(dims, 512 * 64, seed=22, law="uniform", distinct=False, value_law="normal")
    facs = [torch.from_numpy(f).cuda() for f in make_factors(dims, R, "normal", seed=22)]
    T = P.FlycooTensor(idx, vals, dims, m=dims, g=64, bins=512)
    info = T.info
    assert info["segments"] == [512, 512, 512] and info["m"] == [64, 64, 64]
    ref = [r.clone() for r in T.all_modes(facs)]
    for call in range(2):
        outs = [torch.full((d, R), float("nan"), device="cuda") for d in dims]
        for n in range(3):
            P.flycoo_spmttkrp_static_scratch(T.h, n, facs, outs[n], (n + 1) % 3)
        torch.cuda.synchronize()
        for n in range(3):
            assert torch.equal(outs[n], ref[n]), (call, n)
    # one segment more than fits: 513 bins, 513 shards
    idx, vals = random_coo(dims, 513 * 64, seed=23, law="uniform", distinct=False, value_law="normal")
    T2 = P.FlycooTensor(idx, vals, dims, m=dims, g=64, bins=513)
    assert T2.info["segments"][0] == 513
    out = torch.empty((64, R), device="cuda")
    with pytest.raises(P.FlycooError) as e:
        P.flycoo_spmttkrp_static_scratch(T2.h, 0, facs, out, 1)
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG"
    assert T2.layout_mode == 0


def test_static_scratch_rejects_oversized_requests(P):
    # mode 0 has 600 super-shards of 64 rows, each split over several bins:
    # over 512 row blocks of 64 x 64 floats, more than the 8 MiB array holds
    dims = (38_400, 40, 30)
    idx, vals = random_coo(dims, 20_000, seed=3)
    T = P.FlycooTensor(idx, vals, dims, m=(64, 40, 30), g=16, bins=8)
    assert T.info["segments"][0] > 512
    facs = [torch.randn((d, 64), device="cuda") for d in dims]
    out = torch.empty((dims[0], 64), device="cuda")
    with pytest.raises(P.FlycooError) as e:
        P.flycoo_spmttkrp_static_scratch(T.h, 0, facs, out, 1)
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG"
    assert "static scratch holds" in str(e.value)
    assert T.layout_mode == 0
