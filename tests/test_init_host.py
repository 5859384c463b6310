"""The library's seeded initialisation on the host (no GPU): builds
tests/init_check.cpp against libmera.so and compares its normals and
isometries (real, complex, Z2 charge blocks) with oracle/rng.py, which
restates the generator and the sign-fixed QR from their definitions."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import rng
from paper_2007_03638_gb300 import inputs as inp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_init_matches_oracle(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    from paper_2007_03638_gb300 import build as b
    lib = b.build()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = str(tmp_path / "init_check")
    cmd = [cxx, "-std=c++17", "-O1", os.path.join(ROOT, "tests", "init_check.cpp"),
           "-I", os.path.join(ROOT, "paper_2007_03638_gb300", "csrc"), "-I", os.path.join(cuda, "include"),
           lib, "-Wl,-rpath," + os.path.dirname(lib), "-L", os.path.join(cuda, "lib64"), "-lcudart", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    n_gauss = n_iso = 0
    for line in r.stdout.splitlines():
        head, vals = line.split(":")
        v = np.array([float(x) for x in vals.split()])
        f = head.split()
        if f[0] == "gauss":
            seed, stream, count = int(f[1]), int(f[2]), int(f[3])
            want = rng.gaussians(seed, stream, count)
            assert np.abs(v - want).max() < 1e-14 * max(1.0, np.abs(want).max()), line
            n_gauss += 1
        else:
            seed, stream, n, p, cplx, z2 = (int(x) for x in f[1:])
            rq, cq = (inp.fused_parities(2, 2, 2), inp.z2_parities(4)) if z2 else (None, None)
            want = rng.random_isometry(seed, stream, n, p, bool(cplx), rq, cq)
            got = (v[0::2] + 1j * v[1::2]).reshape(n, p) if cplx else v.reshape(n, p)
            assert np.abs(got - want).max() < 1e-12, (line[:40], np.abs(got - want).max())
            n_iso += 1
    assert (n_gauss, n_iso) == (3, 6)
