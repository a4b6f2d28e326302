"""The C ABI used from C: tests/c_abi/abi_check.c includes include/slab.h and links libslab.so.

CPU: the program compiles and links with gcc against the header and the built library (the
header is valid C, every symbol it calls resolves).  GPU: it factors a 2-D diffusion problem
with opts == NULL and with a slab_opts struct pre-filled with 0xFF bytes and then passed to
slab_default_opts, solves, runs the adjoint with the gradient, and its results are compared
with the oracle's banded-LU solution and the oracle's gradient formula.
"""
import os
import subprocess

import numpy as np
import pytest

from paper_2211_07572_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "abi_check.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build_program(tmp_path):
    from paper_2211_07572_gb300 import _lib
    _lib.load()                                     # builds libslab.so if it is missing
    libdir = os.path.dirname(_lib.library_path())
    exe = str(tmp_path / "abi_check")
    cmd = ["gcc", "-std=c11", "-O1", "-Wall", "-Werror", SRC, "-o", exe,
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           "-L", libdir, "-lslab", f"-Wl,-rpath,{libdir}",
           "-L", os.path.join(CUDA, "lib64"), f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_compiles_and_links(tmp_path):
    assert os.path.exists(_build_program(tmp_path))


@pytest.mark.gpu
def test_c_caller_defaults_solve_adjoint_match_oracle(tmp_path, oracle_mod):
    n, b = 64, 8
    exe = _build_program(tmp_path)
    p = inputs.diffusion(n, b, k=1, n_modes=8, field_seed=21, rhs_seed=22)
    kp, fp, op = tmp_path / "kappa.bin", tmp_path / "f.bin", tmp_path / "out.bin"
    np.ascontiguousarray(p.kappa, dtype=np.float64).tofile(kp)
    np.ascontiguousarray(p.f[0], dtype=np.float64).tofile(fp)
    r = subprocess.run([exe, str(n), str(b), str(kp), str(fp), str(op)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    N, NN = (n - 1) ** 2, (n + 1) ** 2
    raw = op.read_bytes()
    status = np.frombuffer(raw[:24], dtype=np.int32)
    vals = np.frombuffer(raw[24:], dtype=np.float64)
    relres, rest = vals[:2], vals[2:]
    u_null, lam, grad, u_def = rest[:N], rest[N:2 * N], rest[2 * N:2 * N + NN], rest[2 * N + NN:]
    assert (status == 0).all(), status
    assert relres.max() <= 1e-10, relres              # the default rtol
    uo = oracle_mod.solve(p)[0]
    for u in (u_null, u_def):
        assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo)
    lo = oracle_mod.solve(p, p.f)[0]                   # A symmetric: lambda = A^-1 dL/du with dL/du = f
    assert np.linalg.norm(lam - lo) <= 1e-8 * np.linalg.norm(lo)
    go = oracle_mod.kappa_gradient(2, n, uo, lo)
    assert np.linalg.norm(grad.reshape(go.shape) - go) <= 1e-8 * np.linalg.norm(go)
