"""include/mera.h is a C ABI: a plain C99 program (tests/c_abi_example.c)
compiles against it with every warning an error and links against
libmera.so (CPU); on a GPU it runs an optimisation through the ABI alone."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2007_03638_gb300 import build as b
    lib = b.build()
    exe = str(tmp_path / "c_abi_example")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", os.path.join(ROOT, "tests", "c_abi_example.c"),
           "-I", os.path.join(ROOT, "include"), lib, "-Wl,-rpath," + os.path.dirname(lib), "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_header_is_c99_and_links(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_program_optimises(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([_build(tmp_path)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    fields = r.stdout.split()
    e = float(fields[1])
    assert -4 / 3.141592653589793 < e < -1.2, r.stdout  # variational, and well below the product state's -1
