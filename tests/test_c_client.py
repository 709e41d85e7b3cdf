"""The C ABI from a plain C99 program (tests/c_client/flycoo_all_modes.c), no
Python in between: on the CPU it compiles, links against libflycoo.so and the
CUDA runtime, and answers a bad command line; on the GPU it runs an all-mode
sweep (3- and 4-mode tensors) whose outputs must match the oracle, and checks
that the host-only planner reproduces the handle's schedule."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from synth import make_factors, random_coo

from _util import rel_fro

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "flycoo_all_modes.c")
OUT_DIR = os.path.join(ROOT, "_build", "c_client")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _env():
    from paper_2309_09131_gb300 import _native
    lib_dirs = [os.path.dirname(_native.LIB_PATH), os.path.join(CUDA, "lib64")]
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = ":".join(lib_dirs + [env.get("LD_LIBRARY_PATH", "")])
    return env


@pytest.fixture(scope="module")
def client():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime_api.h")):
        pytest.skip("no C compiler or CUDA headers")
    if shutil.which("nvcc") is None and not os.path.exists(os.path.join(CUDA, "bin", "nvcc")):
        pytest.skip("nvcc not available")
    from paper_2309_09131_gb300 import build as B
    lib = B.build()
    os.makedirs(OUT_DIR, exist_ok=True)
    exe = os.path.join(OUT_DIR, "flycoo_all_modes")
    lib_dir = os.path.dirname(lib)
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), SRC, "-L", lib_dir, "-lflycoo", "-L", os.path.join(CUDA, "lib64"),
           "-lcudart", f"-Wl,-rpath,{lib_dir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_builds_and_answers_usage(client):
    r = subprocess.run([client], capture_output=True, text=True, env=_env(), timeout=60)
    assert r.returncode == 2 and "usage" in r.stderr


def _write_input(path, idx, vals, dims, facs, R):
    with open(path, "wb") as f:
        f.write(np.array([len(dims), R], dtype="<u4").tobytes())
        f.write(np.array([idx.shape[1]], dtype="<u8").tobytes())
        f.write(np.asarray(dims, dtype="<u8").tobytes())
        f.write(np.ascontiguousarray(idx, dtype="<u4").tobytes())
        f.write(np.ascontiguousarray(vals, dtype="<f4").tobytes())
        for F in facs:
            f.write(np.ascontiguousarray(F, dtype="<f4").tobytes())


@pytest.mark.gpu
@pytest.mark.parametrize("dims,nnz,R", [((300, 200, 250), 30_000, 32), ((40, 30, 20, 25), 8_000, 16)])
def test_c_client_all_modes_matches_oracle(client, dims, nnz, R):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    idx, vals = random_coo(dims, nnz, seed=7, law="zipf", value_law="lognormal")
    facs = make_factors(dims, R, "normal", seed=7)
    tag = "x".join(map(str, dims))
    inp, outp = os.path.join(OUT_DIR, f"in_{tag}.bin"), os.path.join(OUT_DIR, f"out_{tag}.bin")
    _write_input(inp, idx, vals, dims, facs, R)
    r = subprocess.run([client, inp, outp], capture_output=True, text=True, env=_env(), timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    got = np.fromfile(outp, dtype="<f4")
    assert got.size == sum(d * R for d in dims)
    Y64 = oracle.factors_f64(facs)
    off = 0
    for n, d in enumerate(dims):
        M = got[off:off + d * R].reshape(d, R)
        off += d * R
        ref = oracle.mttkrp(idx, vals, Y64, n, dims)
        assert rel_fro(M, ref) <= 1e-5, (n, rel_fro(M, ref))
