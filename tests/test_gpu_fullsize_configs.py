"""Full-size parity on the other benchmark workloads, in the launch
configuration the benchmark times (default partition parameters): the
4-mode Delicious-like tensor (140M nonzeros), the Nell-1-like tensor (140M)
and the skewed R = 64 tensor (200M, ten hot mode-0 slices holding half the
nonzeros).  Sampled output rows (the heaviest, empty ones, random ones and
both ends) against the oracle row by row, FP32 and BF16 factors, after a
full all-mode sweep with the fused remaps; the sweep must end in L_0."""
import numpy as np
import pytest

import oracle
from synth import WORKLOADS, make_workload

from _util import rel_fro, to_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ["delicious4d_1.2mx1.2mx50kx10k_140m_r32", "nell1like_4.8mx1.8mx1.8m_140m_r32",
         "skewed_20kx200kx500k_200m_r64"]


def _sample_rows(idx_n, I, rng):
    counts = np.bincount(idx_n, minlength=I)
    heavy = np.argsort(counts)[-6:]
    empty = np.nonzero(counts == 0)[0][:4]
    rand = rng.choice(I, size=12, replace=False)
    return np.unique(np.concatenate([heavy, empty, rand, [0, I - 1]])).astype(np.uint32)


@pytest.mark.parametrize("name", NAMES)
def test_sampled_rows_full_size(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_09131_gb300 as P
    wl = WORKLOADS[name]
    N = len(wl.dims)
    idx, vals, facs = make_workload(wl)
    T = P.FlycooTensor(idx, vals, wl.dims)
    rng = np.random.default_rng(1)
    rows = [_sample_rows(idx[n], wl.dims[n], rng) for n in range(N)]
    Y64 = oracle.factors_f64(facs)
    Yb64 = oracle.factors_f64(facs, bf16=True)
    try:
        for dtype in (torch.float32, torch.bfloat16):
            Y = [torch.from_numpy(f).cuda().to(dtype) for f in facs]
            outs = T.all_modes(Y)
            torch.cuda.synchronize()
            assert T.layout_mode == 0
            for n in range(N):
                got = to_np(outs[n])[rows[n]]
                ref = oracle.mttkrp_rows(idx, vals, Y64, n, rows[n], wl.dims)
                if dtype == torch.float32:
                    assert rel_fro(got, ref) <= 1e-5, (name, n, rel_fro(got, ref))
                else:
                    refb = oracle.mttkrp_rows(idx, vals, Yb64, n, rows[n], wl.dims)
                    assert rel_fro(got, refb) <= 1e-5, (name, n, rel_fro(got, refb))
                    assert rel_fro(got, ref) <= 1e-2, (name, n, rel_fro(got, ref))
            del Y, outs
    finally:
        T.close()
        torch.cuda.empty_cache()
