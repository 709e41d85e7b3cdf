#!/usr/bin/env python3
"""All-mode spMTTKRP benchmark (FLYCOO layout, remap fused into each pass).

One step = spMTTKRP of every mode n = 0..N-1 in turn, each fused with the
dynamic remap of the tensor to the next mode's layout (Algorithm 2), so the
tensor is back in layout L_0 after the step.  The default workload is the
Nell-2-sized synthetic tensor (12,000 x 9,000 x 29,000, 77M nonzeros,
Zipf(1.1) indices, lognormal values, R = 32, FP32 factors).

``value`` is whole-job algorithmic HBM throughput in GB/s: the compulsory
bytes of one step (every stored nonzero read and written once, its remap slot
read once, every input factor row read once, every output row written once)
times the replicas, divided by the max-over-ranks step time.  Multi-GPU runs
are independent replicas (the path does not shard across GPUs here).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl flycoo|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "all-mode spMTTKRP ms & HBM GB/s (% of peak); BF16 vs FP32 at stated err"
DEFAULT_WORKLOAD = "nell2like_12000x9000x29000_77m_r32"
PRECISION_WORKLOAD = "delicious4d_1.2mx1.2mx50kx10k_140m_r32"
FALLBACK_HBM_GBS = 6800.0


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["flycoo", "reference"], default="flycoo")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--g", type=int, default=0, help="shard size (0: the library default)")
    ap.add_argument("--bins", type=int, default=0, help="schedule bins (0: the library default)")
    ap.add_argument("--m", type=int, default=0, help="super-shard width of every mode (0: the library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-als", action="store_true")
    ap.add_argument("--no-cpopt", action="store_true")
    ap.add_argument("--ablations", action="store_true",
                    help="also time passes without the fused remap and the sweep at R = 16, 32, 64")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the FP32-vs-BF16 section on the 4-mode 140M-nonzero tensor")
    ap.add_argument("--no-oracle-err", action="store_true",
                    help="skip the per-mode errors against the FP64 oracle on sampled rows")
    ap.add_argument("--cpu-sample", type=int, default=40_000_000, help="nonzeros in the CPU baseline sample")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    return args


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def step_bytes(dims, nnz, R, factor_bytes, elem_bytes):
    """Compulsory bytes of each mode's fused pass and of the whole step."""
    per_mode = []
    for n in range(len(dims)):
        b = nnz * (2 * elem_bytes + 4)                       # read + remap-write the nonzero, read its slot
        b += sum(dims[w] * R * factor_bytes for w in range(len(dims)) if w != n)  # input factor rows
        b += dims[n] * R * 4                                  # output rows (FP32)
        per_mode.append(b)
    return per_mode, sum(per_mode)


def _all_reduce(x, world, op, device):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op))
    return float(t.item())


def reduce_max(x, world, device="cuda"):
    return _all_reduce(x, world, "MAX", device)


def whole_job_gbps(bytes_local, ms_local, world, device="cuda"):
    """Whole-job throughput: the bytes all ranks processed in one step divided
    by the slowest rank's step time.  Returns ``(GB/s, max-over-ranks ms)``."""
    ms = reduce_max(ms_local, world, device)
    total = _all_reduce(bytes_local, world, "SUM", device)
    return total / (ms * 1e-3) / 1e9, ms


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=None):
        self.proc = None
        self.path = None
        self.gpu_index = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            if self.gpu_index is not None:
                cmd += ["-i", str(self.gpu_index)]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


def cpu_oracle_pass(idx, vals, facs, dims, sample, threads=1):
    """The FP64 oracle over the first ``sample`` nonzeros (COO order is random),
    all modes, on ``threads`` host threads; returns (seconds, algorithmic bytes
    of the sample, nonzeros in the sample)."""
    import oracle
    S = min(sample, idx.shape[1])
    sidx = idx[:, :S].copy()
    svals = vals[:S].copy()
    Y64 = oracle.factors_f64(facs)
    t0 = time.perf_counter()
    for n in range(len(dims)):
        if threads == 1:
            oracle.mttkrp(sidx, svals, Y64, n, dims)
        else:
            oracle.mttkrp_threads(sidx, svals, Y64, n, threads, dims)
    sec = time.perf_counter() - t0
    _, b = step_bytes(dims, S, facs[0].shape[1], 4, 16)
    return sec, b, S


def sample_rows(idx_n, I, rng, heavy=64, rand=192):
    """Rows of one mode for the error against the oracle: the heaviest ones
    (they carry most of the Frobenius norm) and uniformly random ones."""
    counts = np.bincount(idx_n, minlength=I)
    h = np.argsort(counts, kind="stable")[-heavy:]
    r = rng.choice(I, size=min(rand, I), replace=False)
    return np.unique(np.concatenate([h, r])).astype(np.uint32)


def oracle_row_errors(idx, vals, facs, dims, outs, seed=0):
    """Relative Frobenius error per mode, on sampled rows, of each named set
    of GPU outputs against the FP64 oracle on the original FP32 factors.
    ``outs`` maps a name to N host arrays.  Returns (errors, rows per mode)."""
    import oracle
    rng = np.random.default_rng(seed)
    Y64 = oracle.factors_f64(facs)
    errs = {k: [] for k in outs}
    nrows = []
    for n in range(len(dims)):
        rows = sample_rows(idx[n], dims[n], rng)
        ref = oracle.mttkrp_rows(idx, vals, Y64, n, rows, dims)
        den = float(np.linalg.norm(ref))
        for k, o in outs.items():
            d = o[n][rows].astype(np.float64) - ref
            errs[k].append(float(np.linalg.norm(d)) / den if den else float(np.linalg.norm(d)))
        nrows.append(int(rows.size))
    return errs, nrows


def _generate_to_dir(name, path):
    """Child process: draw a named workload and save it as .npy files."""
    from synth import WORKLOADS, make_workload
    idx, vals, facs = make_workload(WORKLOADS[name])
    np.save(os.path.join(path, "idx.npy"), idx)
    np.save(os.path.join(path, "vals.npy"), vals)
    for w, f in enumerate(facs):
        np.save(os.path.join(path, f"f{w}.npy"), f)


class BackgroundWorkload:
    """Draws a workload in a spawned process (started before the first GPU
    call) while the main benchmark runs; ``get()`` waits and loads it."""

    def __init__(self, name):
        import multiprocessing as mp
        self.name = name
        self.dir = tempfile.mkdtemp(prefix="flycoo_wl_")
        self.proc = mp.get_context("spawn").Process(target=_generate_to_dir, args=(name, self.dir))
        self.proc.start()

    def get(self):
        self.proc.join()
        if self.proc.exitcode != 0:
            raise RuntimeError(f"generating {self.name} failed (exit {self.proc.exitcode})")
        idx = np.load(os.path.join(self.dir, "idx.npy"))
        vals = np.load(os.path.join(self.dir, "vals.npy"))
        facs = []
        w = 0
        while os.path.exists(os.path.join(self.dir, f"f{w}.npy")):
            facs.append(np.load(os.path.join(self.dir, f"f{w}.npy")))
            w += 1
        self.cleanup()
        return idx, vals, facs

    def cleanup(self):
        import shutil
        if self.proc.is_alive():
            self.proc.terminate()
            self.proc.join()
        shutil.rmtree(self.dir, ignore_errors=True)


def time_all_modes(P, T, Y, outs, steps, warmup=3):
    """Mean all-mode step time (ms) and per-mode times of ``steps`` sweeps."""
    import torch
    N = len(Y)
    for _ in range(warmup):
        T.all_modes(Y, outs)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(N + 1)] for _ in range(steps)]
    for s in range(steps):
        ev[s][0].record()
        for n in range(N):
            P.flycoo_spmttkrp(T.h, n, Y, outs[n], (n + 1) % N)
            ev[s][n + 1].record()
    ev[-1][-1].synchronize()
    total = ev[0][0].elapsed_time(ev[-1][-1]) / steps
    per_mode = [statistics.mean(ev[s][n].elapsed_time(ev[s][n + 1]) for s in range(steps)) for n in range(N)]
    return total, per_mode


def workload_config(wl):
    """The workload description both arms report (shape, laws, rank, seed)."""
    return {"workload": wl.name, "dims": list(wl.dims), "nnz": wl.nnz, "rank": wl.rank,
            "index_laws": [" ".join(str(x) for x in law) for law in wl.index_laws],
            "values": wl.value_law, "factor_law": wl.factor_law, "seed": wl.seed,
            "duplicates": "merged" if wl.distinct else "kept"}


def run_reference(args):
    rank, local_rank, world = dist_env()
    if rank != 0:
        return 0
    from synth import WORKLOADS, make_workload
    wl = WORKLOADS[args.workload]
    idx, vals, facs = make_workload(wl)
    sample = min(2_000_000, wl.nnz)
    times = []
    for s in range(args.warmup + args.steps):
        sec, b, S = cpu_oracle_pass(idx, vals, facs, wl.dims, sample)
        if s >= args.warmup:
            times.append(sec)
    sec = statistics.mean(times)
    gbs = b / sec / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wl),
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {S} nonzeros (random COO order) of the workload, all "
                                   f"{len(wl.dims)} modes, FP64 single-threaded C oracle, per step"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def traffic_from_profiles(kernel_sha, g):
    """DRAM bytes per 77M-nonzero launch of the fused kernel from the
    committed ncu summary at shard size g, if it was taken on this exact kernel
    source; else None."""
    p = os.path.join(ROOT, "profiles", f"fused_mttkrp_remap_f32_nell2like_16m_g{int(g)}.md")
    try:
        kv = {}
        with open(p) as f:
            for line in f:
                if line.startswith("- ") and ":" in line:
                    k, v = line[2:].split(":", 1)
                    kv[k.strip()] = v.strip().strip("`")
        if kv.get("kernel_source_sha256") == kernel_sha:
            return float(kv["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def kernel_source_sha():
    """SHA-256 of the fused kernel's sources with comments and blank space
    removed, so that a comment edit keeps a capture valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2309_09131_gb300", "csrc")
    for f in ("fused.cuh", "internal.cuh"):
        with open(os.path.join(csrc, f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(" ".join(line.split()) for line in text.splitlines() if line.strip()).encode())
    return h.hexdigest()


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)

    rank, local_rank, world = dist_env()
    # the precision workload is drawn in a spawned process while the main
    # benchmark runs (started before the first GPU call)
    bg = None
    if rank == 0 and world == 1 and not args.no_precision and args.workload == DEFAULT_WORKLOAD:
        bg = BackgroundWorkload(PRECISION_WORKLOAD)

    import torch

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    import paper_2309_09131_gb300 as P
    from synth import WORKLOADS, make_factors, make_workload

    wl = WORKLOADS[args.workload]
    t0 = time.perf_counter()
    idx, vals, facs = make_workload(wl)
    gen_s = time.perf_counter() - t0
    N, R = len(wl.dims), wl.rank

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    T = P.FlycooTensor(idx, vals, wl.dims, g=args.g, bins=args.bins,
                       m=[min(args.m, d) for d in wl.dims] if args.m else None)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    info = T.info
    elem_bytes = info["elem_bytes"]

    Yf = [torch.from_numpy(f).cuda() for f in facs]
    outs = [torch.empty((d, R), dtype=torch.float32, device="cuda") for d in wl.dims]
    per_mode_b, step_b = step_bytes(wl.dims, wl.nnz, R, 4, elem_bytes)
    launches_per_step = sum(1 + (1 if info["fixup_super_shards"][n] else 0) for n in range(N))

    # ---- warm-up
    for _ in range(args.warmup):
        T.all_modes(Yf, outs)
    torch.cuda.synchronize()

    # ---- timed region: K steps, inputs (2 x 1.23 GB element buffers) far larger than L2;
    # no events between the passes but the library's own around each fused launch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler()
    if rank == 0:
        clocks.start()
    T.timing_enable(True)
    barrier()
    torch.cuda.synchronize()
    start.record()
    for s in range(args.steps):
        for n in range(N):
            P.flycoo_spmttkrp(T.h, n, Yf, outs[n], (n + 1) % N)
    end.record()
    end.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if rank == 0 else None
    total_ms = start.elapsed_time(end)
    k2_ms, k2_launches = T.timing_read()
    T.timing_enable(False)
    value, step_ms = whole_job_gbps(step_b, total_ms / args.steps, world)
    # per-mode times from a separate sweep with an event after every pass
    per_mode_ms = time_all_modes(P, T, Yf, outs, args.steps, warmup=1)[1]

    peak, peak_kind = hbm_peak()
    achieved = (step_b * args.steps) / (k2_ms * 1e-3) / 1e9 if k2_ms > 0 else None
    sha = kernel_source_sha()
    # the committed capture (a 16M-nonzero case of the same shape at the bench's
    # shard size, scaled to 77M nonzeros) describes the bench workload only
    traffic = traffic_from_profiles(sha, T.info["g"]) if wl.name == DEFAULT_WORKLOAD else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "peak_kind": peak_kind, "kernel": f"fused_mttkrp_remap_kernel<{N},{R},fp32>",
                "algorithmic_bytes_per_launch": step_b / N, "avg_launch_ms": k2_ms / max(k2_launches, 1),
                "kernel_source_sha256": sha}

    # ---- BF16 factor storage, same sweep
    bf16 = None
    if not args.no_bf16:
        Yb = [y.to(torch.bfloat16) for y in Yf]
        outs_b = [torch.empty_like(o) for o in outs]
        for _ in range(3):
            T.all_modes(Yb, outs_b)
        torch.cuda.synchronize()
        sb = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        sb.record()
        for _ in range(args.steps):
            T.all_modes(Yb, outs_b)
        eb.record()
        eb.synchronize()
        _, step_bb = step_bytes(wl.dims, wl.nnz, R, 2, elem_bytes)
        gbps_b, ms_b = whole_job_gbps(step_bb, sb.elapsed_time(eb) / args.steps, world)
        T.all_modes(Yf, outs)
        torch.cuda.synchronize()
        diff = [float(torch.linalg.norm(outs_b[n] - outs[n]) / torch.linalg.norm(outs[n])) for n in range(N)]
        bf16 = {"ms_per_step": ms_b, "gbps": gbps_b,
                "speedup_vs_f32": step_ms / ms_b, "rel_fro_diff_vs_f32_gpu_per_mode": diff}
        host_outs = {"f32": [o.cpu().numpy() for o in outs], "bf16": [o.cpu().numpy() for o in outs_b]}
        del outs_b, Yb
    else:
        T.all_modes(Yf, outs)
        host_outs = {"f32": [o.cpu().numpy() for o in outs]}

    # ---- per-mode error of the timed outputs against the FP64 oracle (sampled rows)
    oracle_err = None
    if rank == 0 and not args.no_oracle_err:
        errs, nrows = oracle_row_errors(idx, vals, facs, wl.dims, host_outs)
        oracle_err = {"rows_per_mode": nrows, "reference": "FP64 oracle on the FP32 factors",
                      "rows": "the 64 heaviest rows of each mode and up to 192 uniformly random ones",
                      **{f"{k}_rel_fro_per_mode": v for k, v in errs.items()}}
        if bf16 is not None:
            bf16["rel_fro_err_vs_oracle_per_mode"] = errs["bf16"]
    del host_outs

    # ---- CP-ALS iterations (Algorithm 1 with the least-squares update) on the same tensor
    als = None
    if not args.no_als:
        adt = torch.bfloat16 if wl.factor_dtype == "bf16" else torch.float32
        Ya = [y.to(adt).clone() for y in Yf]
        lam = torch.empty(R, dtype=torch.float64, device="cuda")
        fits = [T.cp_als_step(Ya, lam)[1] for _ in range(2)]
        torch.cuda.synchronize()
        iters = max(3, min(args.steps, 10))
        sa = torch.cuda.Event(enable_timing=True)
        ea = torch.cuda.Event(enable_timing=True)
        sa.record()
        fits += P.flycoo_cp_als(T.h, Ya, lam, iters)   # the iterations in one call
        ea.record()
        ea.synchronize()
        ms_a = reduce_max(sa.elapsed_time(ea) / iters, world)
        sweep_ms = bf16["ms_per_step"] if (adt == torch.bfloat16 and bf16) else step_ms
        als = {"ms_per_iter": ms_a, "iters_timed": iters, "spmttkrp_share": sweep_ms / ms_a,
               "fits": fits, "factor_dtype": wl.factor_dtype}

    # ---- CP-OPT loss and gradient sweep (N fused passes forming residuals on the fly), FP32
    cpopt = None
    if not args.no_cpopt:
        grads = [torch.empty_like(y) for y in Yf]
        loss = P.flycoo_cpopt_grad(T.h, Yf, grads)
        for _ in range(2):
            P.flycoo_cpopt_grad(T.h, Yf, grads, want_loss=False)
        torch.cuda.synchronize()
        sc = torch.cuda.Event(enable_timing=True)
        ec = torch.cuda.Event(enable_timing=True)
        sc.record()
        for _ in range(args.steps):
            P.flycoo_cpopt_grad(T.h, Yf, grads, want_loss=False)
        ec.record()
        ec.synchronize()
        cp_b = step_b + sum(wl.dims) * R * 4  # the output mode's own rows are gathered too
        gbps_c, ms_c = whole_job_gbps(cp_b, sc.elapsed_time(ec) / args.steps, world)
        cpopt = {"ms_per_sweep": ms_c, "gbps": gbps_c, "loss": loss, "bytes_per_sweep": cp_b}

    # ---- optional: per-mode passes without the fused remap, and other ranks
    extra = {}
    if args.ablations:
        T.remap(0)
        nr = []
        for n in range(N):
            T.remap(n)
            for _ in range(3):
                P.flycoo_spmttkrp(T.h, n, Yf, outs[n], -1)
            torch.cuda.synchronize()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record()
            for _ in range(args.steps):
                P.flycoo_spmttkrp(T.h, n, Yf, outs[n], -1)
            s1.record()
            s1.synchronize()
            nr.append(s0.elapsed_time(s1) / args.steps)
        T.remap(0)
        extra["no_remap_ms_per_mode"] = nr
        ranks = {}
        for R2 in (16, 32, 64) + ((128,) if N == 3 else ()):
            Y2 = [torch.from_numpy(f).cuda() for f in make_factors(wl.dims, R2, wl.factor_law, seed=wl.seed)]
            o2 = [torch.empty((d, R2), dtype=torch.float32, device="cuda") for d in wl.dims]
            for _ in range(2):
                T.all_modes(Y2, o2)
            torch.cuda.synchronize()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record()
            for _ in range(args.steps):
                T.all_modes(Y2, o2)
            s1.record()
            s1.synchronize()
            ranks[str(R2)] = s0.elapsed_time(s1) / args.steps
            del Y2, o2
        extra["all_mode_ms_by_rank_fp32"] = ranks
        # super-shard width m_n (Section III-A): the default min(I_n, 32) against
        # 16 and 64 rows, FP32 at the workload's rank
        widths = {}
        for mw in (16, 64):
            Tm = P.FlycooTensor(idx, vals, wl.dims, m=[min(mw, d) for d in wl.dims])
            widths[str(mw)] = time_all_modes(P, Tm, Yf, outs, args.steps)[0]
            Tm.close()
        widths[str(32)] = time_all_modes(P, T, Yf, outs, args.steps)[0]
        extra["all_mode_ms_by_super_shard_rows_fp32"] = widths
        # the same sweep with the block-cyclic schedule instead of Algorithm 3 (LPT)
        Tb = P.FlycooTensor(idx, vals, wl.dims, schedule=P._native.SCHEDULE_BLOCK_CYCLIC)
        for _ in range(2):
            Tb.all_modes(Yf, outs)
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(args.steps):
            Tb.all_modes(Yf, outs)
        s1.record()
        s1.synchronize()
        extra["all_mode_ms_block_cyclic_schedule"] = s0.elapsed_time(s1) / args.steps
        Tb.close()
        # the Z-Morton order inside super-shards instead of the key order
        Tz = P.FlycooTensor(idx, vals, wl.dims, order=P.ORDER_MORTON)
        zm = {"f32": time_all_modes(P, Tz, Yf, outs, args.steps)[0]}
        Yz = [y.to(torch.bfloat16) for y in Yf]
        zm["bf16"] = time_all_modes(P, Tz, Yz, outs, args.steps)[0]
        extra["all_mode_ms_morton_order"] = zm
        Tz.close()
        del Yz

    # ---- end to end through the C ABI with host buffers: flycoo_all_modes_host
    # copies the pinned host factors in, runs the N fused passes and copies
    # every output back, then waits for the stream
    e2e = None
    if not args.no_e2e:
        hY = [torch.from_numpy(f).pin_memory() for f in facs]
        hO = [torch.empty((d, R), dtype=torch.float32).pin_memory() for d in wl.dims]
        h2d = sum(y.numel() * 4 for y in hY)
        d2h = sum(o.numel() * 4 for o in hO)
        for _ in range(3):
            P.flycoo_all_modes_host(T.h, hY, hO)
        torch.cuda.synchronize()
        barrier()
        se = torch.cuda.Event(enable_timing=True)
        ee = torch.cuda.Event(enable_timing=True)
        se.record()
        for _ in range(args.steps):
            P.flycoo_all_modes_host(T.h, hY, hO)
        ee.record()
        ee.synchronize()
        value_e, ms_e = whole_job_gbps(step_b, se.elapsed_time(ee) / args.steps, world)
        e2e = {"value": value_e, "unit": "GB/s", "ms_per_step": ms_e, "api": "flycoo_all_modes_host",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, single GPU only)
    cpu = None
    cpu_threads = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sec, b, S = cpu_oracle_pass(idx, vals, facs, wl.dims, args.cpu_sample)
        cpu = {"value": b / sec / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"first {S} nonzeros (random COO order) of the workload, all {N} modes, "
                         f"FP64 single-threaded C oracle, {sec:.2f} s"}
        nthr = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        if nthr > 1:
            sec_t, b_t, S_t = cpu_oracle_pass(idx, vals, facs, wl.dims, args.cpu_sample, threads=nthr)
            cpu_threads = {"value": b_t / sec_t / 1e9, "unit": "GB/s", "cores": nthr, "kind": "oracle",
                           "sample": f"the same {S_t} nonzeros, FP64 C oracle split over {nthr} threads "
                                     f"(fixed chunks, private outputs added in thread order), {sec_t:.2f} s"}

    # ---- precision: FP32 against BF16 factor storage on the 4-mode 140M-nonzero
    # tensor, all modes, each with its per-mode error against the FP64 oracle
    precision = None
    if bg is not None:
        pwl = WORKLOADS[PRECISION_WORKLOAD]
        t0 = time.perf_counter()
        pidx, pvals, pfacs = bg.get()
        wait_s = time.perf_counter() - t0
        T3 = P.FlycooTensor(pidx, pvals, pwl.dims)
        info3 = T3.info
        N3, R3 = len(pwl.dims), pwl.rank
        o3 = [torch.empty((d, R3), dtype=torch.float32, device="cuda") for d in pwl.dims]
        psteps = max(5, min(args.steps, 10))
        sec = {}
        hout = {}
        for name, dt, fb in (("f32", torch.float32, 4), ("bf16", torch.bfloat16, 2)):
            Y3 = [torch.from_numpy(f).cuda().to(dt) for f in pfacs]
            ms, pm = time_all_modes(P, T3, Y3, o3, psteps)
            _, b3 = step_bytes(pwl.dims, pwl.nnz, R3, fb, info3["elem_bytes"])
            hout[name] = [o.cpu().numpy() for o in o3]
            sec[name] = {"all_mode_ms": ms, "per_mode_ms": pm, "gbps": b3 / (ms * 1e-3) / 1e9,
                         "frac_of_hbm_peak": b3 / (ms * 1e-3) / 1e9 / hbm_peak()[0], "bytes_per_step": b3}
            del Y3
        errs, nrows = oracle_row_errors(pidx, pvals, pfacs, pwl.dims, hout)
        for name in sec:
            sec[name]["rel_fro_err_vs_oracle_per_mode"] = errs[name]
        precision = {"config": {**workload_config(pwl), "g": info3["g"], "bins": info3["bins"],
                                "elem_bytes": info3["elem_bytes"]},
                     "steps": psteps, **sec, "bf16_speedup_vs_f32": sec["f32"]["all_mode_ms"] / sec["bf16"]["all_mode_ms"],
                     "bf16_within_1e-2": all(e <= 1e-2 for e in errs["bf16"]),
                     "oracle_rows_per_mode": nrows, "generation_wait_s": wait_s}
        T3.close()
        del hout, o3

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**workload_config(wl), "factor_dtype": "f32", "g": info["g"], "bins": info["bins"],
                       "elem_bytes": elem_bytes,
                       "l2": f"no flush: inputs larger than L2 (two {wl.nnz * elem_bytes / 1e9:.2f} GB element "
                             f"buffers and {N * wl.nnz * 4 / 1e9:.2f} GB of remap slots streamed per step)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "all_mode_ms": step_ms, "per_mode_ms": per_mode_ms, "bytes_per_step": step_b,
            "frac_of_hbm_peak": value / world / peak, "bf16": bf16, "preprocess_ms": create_s * 1e3,
            "generate_s": gen_s, "oracle_err": oracle_err, "precision": precision,
            "cp_als": als, "cpopt": cpopt, **extra,
            "memory": {"device_bytes": info["device_bytes"], "tensor_bytes": wl.nnz * elem_bytes,
                       "device_over_tensor": info["device_bytes"] / max(1, wl.nnz * elem_bytes)},
            "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_threads": cpu_threads, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    T.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
