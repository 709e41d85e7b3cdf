"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer structures (layouts, pointers, remap permutations, schedules) must
match bit for bit.  FP32 spMTTKRP must match within relative Frobenius error
1e-5 per mode; BF16 factor storage within 1e-2 against the FP32 factors (and
1e-5 against the same BF16-rounded factors, which isolates the FP32
accumulation).  Where the data make every FP32 operation exact (unit factors,
small integer values) the result must be bitwise equal.
"""
import numpy as np
import pytest

import oracle
from synth import make_factors, random_coo

from _util import rel_fro, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
BF16_TOL = 1e-2


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_09131_gb300 as pkg
    pkg._native.lib()
    return pkg


def _cuda_factors(facs, dtype):
    return [torch.from_numpy(f).to("cuda").to(dtype).contiguous() for f in facs]


LAYOUT_CASES = [
    # dims, nnz, seed, law, distinct, m, g, bins
    ((30, 20, 10), 500, 0, "uniform", False, (3, 2, 4), 7, 5),
    ((6, 5, 4, 3), 300, 1, "zipf", False, (1, 1, 1, 1), 16, 3),
    ((4, 3, 3, 2, 2), 100, 2, "uniform", False, (2, 1, 1, 1, 1), 5, 4),
    ((50, 2, 3), 150, 3, "zipf", True, (7, 1, 1), 1, 2),
    ((1000, 800, 600), 20000, 4, "zipf", True, (0, 0, 0), 0, 0),
    ((300, 200, 250), 30000, 6, "zipf", True, (64, 5, 1), 777, 13),
    ((3, 1, 700), 700, 5, "uniform", True, (1, 1, 10), 64, 9),
]


def tile_ids(shard_ptr, stage, nnz):
    """Stage tile of every position: runs of `stage` positions from each shard
    start (the last run of a shard shorter).  Returns (tile id, tile start)."""
    starts = np.concatenate([np.arange(a, b, stage) for a, b in zip(shard_ptr[:-1], shard_ptr[1:])] +
                            [np.zeros(0)]).astype(np.int64)
    tid = np.zeros(nnz, dtype=np.int64)
    tid[starts[1:]] = 1
    tid = np.cumsum(tid)
    return tid, starts[tid] if nnz else np.zeros(0, dtype=np.int64)


def expected_tile_order(rows, shard_ptr, stage):
    """The compute order of every stage tile, from its definition: the
    tile-local indexes of the tile's nonzeros sorted stably by output row."""
    nnz = rows.size
    tid, tstart = tile_ids(shard_ptr, stage, nnz)
    local = np.arange(nnz, dtype=np.int64) - tstart
    return local[np.lexsort((local, rows, tid))]


def check_tile_orders(T, order, rows_of_elem, mode):
    """Exported compute orders of both stage sizes equal their definition."""
    _, sp, _ = T.export_partition(mode)
    rows = rows_of_elem[order]
    for stage in (512, 1024):
        got = to_np(T.export_tile_order(mode, stage)).view(np.uint16).astype(np.int64)
        np.testing.assert_array_equal(got, expected_tile_order(rows, sp.astype(np.int64), stage))


@pytest.mark.parametrize("order", ["key", "morton"])
@pytest.mark.parametrize("case", LAYOUT_CASES, ids=lambda c: f"{c[0]}-{c[1]}")
def test_layout_partition_schedule_bitexact(P, case, order):
    dims, nnz, seed, law, distinct, m, g, bins = case
    idx, vals = random_coo(dims, nnz, seed=seed, law=law, distinct=distinct)
    T = P.FlycooTensor(idx, vals, dims, m=m, g=g, bins=bins,
                       order=P.ORDER_MORTON if order == "morton" else P.ORDER_KEY)
    info = T.info
    N = len(dims)
    assert info["nnz"] == nnz and info["layout_mode"] == 0 and info["order"] == (order == "morton")
    ref = oracle.flycoo_layout(idx, dims, info["m"], info["g"], info["bins"], order=order)
    for n in range(N):
        ss, sp, sss = T.export_partition(n)
        np.testing.assert_array_equal(ss, ref[n]["ss_ptr"])
        np.testing.assert_array_equal(sp, ref[n]["shard_ptr"])
        np.testing.assert_array_equal(sss, ref[n]["shard_ss"])
        for which, key in ((0, "ss_bins"), (1, "shard_bins")):
            bp, items = T.export_schedule(n, which)
            np.testing.assert_array_equal(bp, ref[n][key][0])
            np.testing.assert_array_equal(items, ref[n][key][1])
        np.testing.assert_array_equal(to_np(T.export_next(n)).view(np.uint32), ref[n]["next"])
        check_tile_orders(T, ref[n]["order"], idx[n], n)

    def layout_is(n):
        li, lv = T.export_layout()
        order = ref[n]["order"]
        np.testing.assert_array_equal(to_np(li).view(np.uint32), idx[:, order])
        np.testing.assert_array_equal(to_np(lv).view(np.uint32), vals[order].view(np.uint32))
        assert T.layout_mode == n

    layout_is(0)
    # the standalone remap walks L_0 -> L_1 -> ... -> L_0 exactly
    for step in range(1, N + 1):
        T.remap(step % N)
        layout_is(step % N)
    # and so does the remap fused into each spMTTKRP pass (Algorithm 2)
    facs = [torch.randn((d, 16), device="cuda") for d in dims]
    for n in range(N):
        T.spmttkrp(n, facs, remap=True)
        torch.cuda.synchronize()
        layout_is((n + 1) % N)


MTTKRP_CASES = [
    # dims, nnz, law, R, g, bins
    ((1000, 800, 600), 100_000, "uniform", 16, 0, 0),
    ((5000, 3000, 2000), 80_000, "zipf", 32, 2048, 50),
    ((200, 150, 120), 30_000, "zipf", 32, 512, 37),
    ((300, 50, 400), 25_000, "zipf", 64, 1000, 64),
    ((60, 70, 50, 40), 20_000, "zipf", 32, 700, 20),
    ((40, 30, 20, 10, 9), 12_000, "uniform", 16, 300, 11),
    ((40, 30, 20, 10, 9), 12_000, "zipf", 64, 333, 7),
]


@pytest.mark.parametrize("case", MTTKRP_CASES, ids=lambda c: f"{c[0]}-{c[1]}-R{c[3]}")
def test_all_modes_fp32_and_bf16(P, case):
    dims, nnz, law, R, g, bins = case
    N = len(dims)
    idx, vals = random_coo(dims, nnz, seed=11, law=law, distinct=True, value_law="lognormal")
    facs = make_factors(dims, R, "normal", seed=11)
    T = P.FlycooTensor(idx, vals, dims, g=g, bins=bins)
    Y64 = oracle.factors_f64(facs)
    Yb64 = oracle.factors_f64(facs, bf16=True)
    for dtype in (torch.float32, torch.bfloat16):
        outs = T.all_modes(_cuda_factors(facs, dtype))
        torch.cuda.synchronize()
        assert T.layout_mode == 0
        for n in range(N):
            got = to_np(outs[n])
            ref = oracle.mttkrp(idx, vals, Y64, n, dims)
            if dtype == torch.float32:
                assert rel_fro(got, ref) <= FP32_TOL, (n, rel_fro(got, ref))
            else:
                refb = oracle.mttkrp(idx, vals, Yb64, n, dims)
                assert rel_fro(got, refb) <= FP32_TOL, (n, rel_fro(got, refb))
                assert rel_fro(got, ref) <= BF16_TOL, (n, rel_fro(got, ref))


def test_unit_factors_integer_values_are_exact(P):
    # every product is 1 * val and every partial sum an integer below 2^24
    dims = (64, 48, 40)
    idx, vals = random_coo(dims, 40_000, seed=3, law="zipf", distinct=False, value_law="int1to5")
    T = P.FlycooTensor(idx, vals, dims, g=97, bins=13)
    for dtype in (torch.float32, torch.bfloat16):
        Y = [torch.ones((d, 32), dtype=dtype, device="cuda") for d in dims]
        outs = T.all_modes(Y)
        Y64 = [np.ones((d, 32)) for d in dims]
        for n in range(3):
            np.testing.assert_array_equal(to_np(outs[n]), oracle.mttkrp(idx, vals, Y64, n, dims))


def test_heavy_row_spanning_many_shards(P):
    # one output row holds most nonzeros: many shards, long fixed-order combine
    rng = np.random.default_rng(5)
    dims = (50, 400, 300)
    nnz = 60_000
    idx = np.stack([np.where(rng.random(nnz) < 0.8, 7, rng.integers(0, 50, nnz)),
                    rng.integers(0, 400, nnz), rng.integers(0, 300, nnz)]).astype(np.uint32)
    vals = rng.standard_normal(nnz).astype(np.float32)
    facs = make_factors(dims, 32, "normal", seed=5)
    T = P.FlycooTensor(idx, vals, dims, g=64, bins=40)
    outs = T.all_modes(_cuda_factors(facs, torch.float32))
    Y64 = oracle.factors_f64(facs)
    for n in range(3):
        got = to_np(outs[n])
        ref = oracle.mttkrp(idx, vals, Y64, n, dims)
        assert rel_fro(got, ref) <= FP32_TOL
        mag = oracle.mttkrp(idx, np.abs(vals), [np.abs(y) for y in Y64], n, dims)
        assert np.all(np.abs(got - ref) <= 1e-5 * mag + 1e-30)


@pytest.mark.parametrize("nnz,g,bins", [(0, 0, 4), (1, 0, 4), (5, 1, 1), (33, 1, 64), (1000, 3, 2)])
def test_edge_cases(P, nnz, g, bins):
    dims = (9, 1, 13)
    idx, vals = random_coo(dims, nnz, seed=nnz, distinct=False, value_law="normal")
    facs = make_factors(dims, 16, "normal", seed=1)
    T = P.FlycooTensor(idx, vals, dims, g=g, bins=bins)
    outs = T.all_modes(_cuda_factors(facs, torch.float32))
    Y64 = oracle.factors_f64(facs)
    A64 = [np.abs(y) for y in Y64]
    for n in range(3):
        got = to_np(outs[n])
        ref = oracle.mttkrp(idx, vals, Y64, n, dims)
        # FP32 summation error is bounded by a multiple of eps32 * sum |terms|
        mag = oracle.mttkrp(idx, np.abs(vals), A64, n, dims)
        assert np.all(np.abs(got - ref) <= 1e-5 * mag + 1e-30)
        assert rel_fro(got, ref) <= FP32_TOL
        assert np.all(got[mag.sum(1) == 0] == 0.0)


def test_single_row_tensor(P):
    dims = (1, 1, 5000)
    idx = np.stack([np.zeros(5000), np.zeros(5000), np.arange(5000)]).astype(np.uint32)
    vals = np.linspace(-1, 1, 5000).astype(np.float32)
    facs = make_factors(dims, 16, "normal", seed=2)
    T = P.FlycooTensor(idx, vals, dims, g=128, bins=8)
    outs = T.all_modes(_cuda_factors(facs, torch.float32))
    Y64 = oracle.factors_f64(facs)
    for n in range(3):
        assert rel_fro(to_np(outs[n]), oracle.mttkrp(idx, vals, Y64, n, dims)) <= FP32_TOL


def test_without_remap_and_determinism(P):
    dims = (120, 90, 70)
    idx, vals = random_coo(dims, 20_000, seed=8, law="zipf")
    facs = _cuda_factors(make_factors(dims, 32, seed=8), torch.float32)
    T = P.FlycooTensor(idx, vals, dims, g=256, bins=17)
    a = T.spmttkrp(0, facs, remap=False)
    assert T.layout_mode == 0
    b = T.spmttkrp(0, facs, remap=True)
    assert T.layout_mode == 1
    assert torch.equal(a, b)
    first = [o.clone() for o in T.all_modes(facs)]
    second = T.all_modes(facs)
    for x, y in zip(first, second):
        assert torch.equal(x, y)


def test_error_statuses(P):
    dims = (10, 10, 10)
    idx, vals = random_coo(dims, 100, seed=1)
    T = P.FlycooTensor(idx, vals, dims, g=16, bins=4)
    facs = _cuda_factors(make_factors(dims, 32, seed=1), torch.float32)
    out = torch.empty((10, 32), device="cuda")
    nat = P._native
    with pytest.raises(P.FlycooError) as e:
        nat.flycoo_spmttkrp(T.h, 1, facs, out, -1)
    assert e.value.status_name == "FLYCOO_ERR_LAYOUT"
    with pytest.raises(P.FlycooError) as e:
        nat.flycoo_spmttkrp(T.h, 3, facs + [facs[0]], out, -1)
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG"
    with pytest.raises(P.FlycooError) as e:
        nat.flycoo_spmttkrp(T.h, 0, facs, out, 2)
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG"
    with pytest.raises(P.FlycooError) as e:
        nat.flycoo_spmttkrp(T.h, 0, [f[:, :24].contiguous() for f in facs], out[:, :24].contiguous(), -1)
    assert e.value.status_name == "FLYCOO_ERR_UNSUPPORTED"
    flat = torch.empty(10 * 32 + 1, device="cuda")
    with pytest.raises(P.FlycooError) as e:
        nat.flycoo_spmttkrp(T.h, 0, facs, flat[1:].view(10, 32), -1)
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG"
    bad = idx.copy()
    bad[2, 17] = 10
    with pytest.raises(P.FlycooError) as e:
        P.FlycooTensor(bad, vals, dims)
    assert e.value.status_name == "FLYCOO_ERR_INDEX_RANGE"
    # the context is still usable after the rejected calls
    T.all_modes(facs)
    torch.cuda.synchronize()


def test_block_cyclic_schedule(P):
    # the block-cyclic baseline of Section V-D: item i in bin i mod bins, ascending;
    # the schedule changes which block does the work, never the result
    dims = (300, 200, 250)
    idx, vals = random_coo(dims, 40_000, seed=31, law="zipf")
    facs = make_factors(dims, 32, "normal", seed=31)
    bins = 13
    T = P.FlycooTensor(idx, vals, dims, g=700, bins=bins, schedule=1)
    info = T.info
    assert info["schedule"] == 1
    for mode in range(3):
        for which, count in ((0, info["super_shards"][mode]), (1, info["shards"][mode])):
            bp, items = T.export_schedule(mode, which)
            ref_items = np.concatenate([np.arange(b, count, bins) for b in range(bins)]).astype(np.uint64)
            ref_bp = np.concatenate([[0], np.cumsum([len(range(b, count, bins)) for b in range(bins)])])
            np.testing.assert_array_equal(items, ref_items)
            np.testing.assert_array_equal(bp, ref_bp.astype(np.uint64))
    Y = [torch.from_numpy(f).cuda() for f in facs]
    outs = T.all_modes(Y)
    torch.cuda.synchronize()
    Y64 = oracle.factors_f64(facs)
    for n in range(3):
        assert rel_fro(to_np(outs[n]), oracle.mttkrp(idx, vals, Y64, n, dims)) <= FP32_TOL
    with pytest.raises(P.FlycooError) as e:
        P.FlycooTensor(idx, vals, dims, schedule=7)
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG"


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_all_modes_from_host_buffers(P, dtype):
    # flycoo_all_modes_host: pinned host factors in, host outputs back, the same
    # kernels in the same order as the device path, so the results are identical
    dims = (300, 200, 250)
    idx, vals = random_coo(dims, 40_000, seed=32, law="zipf", value_law="lognormal")
    facs = make_factors(dims, 32, "normal", seed=32)
    T = P.FlycooTensor(idx, vals, dims, g=700, bins=29)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    hY = [torch.from_numpy(f).to(tdt).pin_memory() for f in facs]
    hO = [torch.full((d, 32), float("nan")).pin_memory() for d in dims]
    T.remap(2)   # the call starts by bringing the tensor back to L_0
    P.flycoo_all_modes_host(T.h, hY, hO)
    assert T.layout_mode == 0
    ref = T.all_modes([y.cuda() for y in hY])
    for n in range(3):
        assert torch.equal(hO[n], ref[n].cpu()), n
    Y64 = oracle.factors_f64(facs, bf16=dtype == "bf16")
    for n in range(3):
        assert rel_fro(hO[n].numpy(), oracle.mttkrp(idx, vals, Y64, n, dims)) <= FP32_TOL


@pytest.mark.parametrize("dims,nnz,law,m,g,bins", [
    ((1000, 800, 600), 100_000, "uniform", (64, 64, 64), 0, 0),
    ((5000, 3000, 2000), 80_000, "zipf", (64, 32, 64), 2048, 50),
    ((200, 150, 40), 30_000, "zipf", (50, 64, 40), 333, 37),
])
def test_rank128_all_modes(P, dims, nnz, law, m, g, bins):
    # rank 128 on 3-mode tensors whose super-shards have at most 64 rows
    idx, vals = random_coo(dims, nnz, seed=12, law=law, distinct=True, value_law="lognormal")
    facs = make_factors(dims, 128, "normal", seed=12)
    T = P.FlycooTensor(idx, vals, dims, m=m, g=g, bins=bins)
    Y64 = oracle.factors_f64(facs)
    Yb64 = oracle.factors_f64(facs, bf16=True)
    for dtype in (torch.float32, torch.bfloat16):
        outs = T.all_modes(_cuda_factors(facs, dtype))
        torch.cuda.synchronize()
        assert T.layout_mode == 0
        for n in range(3):
            ref = oracle.mttkrp(idx, vals, Yb64 if dtype == torch.bfloat16 else Y64, n, dims)
            assert rel_fro(to_np(outs[n]), ref) <= FP32_TOL, (dtype, n, rel_fro(to_np(outs[n]), ref))


def test_super_shard_width_limit_and_rank128_modes(P):
    # the accumulator holds at most 64 rows of a super-shard: wider m is
    # rejected at creation; rank 128 is built for 3-mode tensors only
    dims = (300, 200, 100)
    idx, vals = random_coo(dims, 5_000, seed=13)
    with pytest.raises(P.FlycooError) as e:
        P.FlycooTensor(idx, vals, dims, m=(65, 32, 32))
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG" and "exceeds 64 rows" in str(e.value)
    T = P.FlycooTensor(idx, vals, dims)          # default m = min(I_n, 32)
    assert T.info["m"] == [32, 32, 32]
    facs = [torch.randn((d, 128), device="cuda") for d in dims]
    outs = T.all_modes(facs)
    torch.cuda.synchronize()
    Y64 = [to_np(f).astype(np.float64) for f in facs]
    for n in range(3):
        assert rel_fro(to_np(outs[n]), oracle.mttkrp(idx, vals, Y64, n, dims)) <= FP32_TOL, n
    dims4 = (30, 20, 10, 8)
    idx4, vals4 = random_coo(dims4, 2_000, seed=14)
    T4 = P.FlycooTensor(idx4, vals4, dims4, m=(16, 16, 8, 8))
    f4 = [torch.randn((d, 128), device="cuda") for d in dims4]
    with pytest.raises(P.FlycooError) as e:
        P.flycoo_spmttkrp(T4.h, 0, f4, torch.empty((30, 128), device="cuda"), 1)
    assert e.value.status_name == "FLYCOO_ERR_UNSUPPORTED" and "3-mode" in str(e.value)
    assert T4.layout_mode == 0
    # the handle stays usable at a built rank
    T4.all_modes([f[:, :64].contiguous() for f in f4])
    torch.cuda.synchronize()


@pytest.mark.parametrize("R", [16, 32, 64])
def test_all_modes_widest_super_shards(P, R):
    # 64-row super-shards fill the kernel's accumulator (the default width of
    # tensors with many rows); FP32 and BF16 factors against the FP64 oracle
    dims = (3000, 2000, 1000)
    idx, vals = random_coo(dims, 200_000, seed=41, law="zipf", distinct=True, value_law="lognormal")
    facs = make_factors(dims, R, "normal", seed=41)
    T = P.FlycooTensor(idx, vals, dims, m=(64, 64, 64), g=2048, bins=61)
    assert T.info["m"] == [64, 64, 64]
    for dtype, bf in ((torch.float32, False), (torch.bfloat16, True)):
        outs = T.all_modes(_cuda_factors(facs, dtype))
        torch.cuda.synchronize()
        Y64 = oracle.factors_f64(facs, bf16=bf)
        for n in range(3):
            ref = oracle.mttkrp(idx, vals, Y64, n, dims)
            assert rel_fro(to_np(outs[n]), ref) <= FP32_TOL, (R, dtype, n, rel_fro(to_np(outs[n]), ref))


@pytest.mark.parametrize("case", MTTKRP_CASES[1:5], ids=lambda c: f"{c[0]}-{c[1]}-R{c[3]}")
def test_all_modes_morton_order(P, case):
    # the Z-Morton variant changes the order inside super-shards, never the result
    dims, nnz, law, R, g, bins = case
    N = len(dims)
    idx, vals = random_coo(dims, nnz, seed=11, law=law, distinct=True, value_law="lognormal")
    facs = make_factors(dims, R, "normal", seed=11)
    T = P.FlycooTensor(idx, vals, dims, g=g, bins=bins, order=P.ORDER_MORTON)
    outs = T.all_modes(_cuda_factors(facs, torch.float32))
    torch.cuda.synchronize()
    assert T.layout_mode == 0
    Y64 = oracle.factors_f64(facs)
    for n in range(N):
        assert rel_fro(to_np(outs[n]), oracle.mttkrp(idx, vals, Y64, n, dims)) <= FP32_TOL


def test_morton_code_width_limit(P):
    # 3 other modes of 2^22 super-shards each need 66 bits: refused at create
    dims = (4, 1 << 29, 1 << 29, 1 << 29)
    idx = np.zeros((4, 10), dtype=np.uint32)
    vals = np.ones(10, dtype=np.float32)
    with pytest.raises(P.FlycooError) as e:
        P.FlycooTensor(idx, vals, dims, order=P.ORDER_MORTON)
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG" and "64" in str(e.value)
    with pytest.raises(P.FlycooError) as e:
        P.FlycooTensor(idx, vals, (4, 4, 4, 4), order=7)
    assert e.value.status_name == "FLYCOO_ERR_INVALID_ARG"
