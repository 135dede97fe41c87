"""The C ABI used from plain C: tests/c/abi_example.c compiled with gcc against include/ and linked
against the built library (no torch, no CUDA headers).  On a machine without a GPU the program
runs its argument-validation checks and reports that no device is usable (exit 3)."""
import os
import shutil
import subprocess

import pytest

from paper_1909_05423_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _compile(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    lib = build.build()
    exe = str(tmp_path / "abi_example")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "c", "abi_example.c"), "-L", libdir, "-lpittpack_gb", "-Wl,-rpath," + libdir,
           "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_validation_without_gpu(tmp_path):
    exe = _compile(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode in (0, 3), r.stdout + r.stderr  # 3: no usable GPU here


@pytest.mark.gpu
def test_c_program_solves_on_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _compile(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")
