"""A plain C program (tests/c_api_example.c) using the library through
include/atlas_gb.h only: compiled with gcc and linked against libatlasgb.so
and the CUDA runtime.  Without a GPU the operator call must fail with
ATLAS_ECUDA (exit code 2); on a GB300 the program checks exact zeros and the
vanishing total circulation on the device results (exit code 0)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PKG = os.path.join(ROOT, "paper_1908_07038_gb300")


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime_api.h")):
            return c
    nvcc = shutil.which("nvcc")
    return os.path.dirname(os.path.dirname(nvcc)) if nvcc else None


@pytest.fixture(scope="module")
def example(product, tmp_path_factory):
    cuda = _cuda_home()
    if cuda is None or shutil.which("gcc") is None:
        pytest.skip("gcc or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("capi") / "c_api_example")
    libdirs = [os.path.join(cuda, d) for d in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib")]
    libdirs = [d for d in libdirs if os.path.exists(d)]
    cmd = ["gcc", "-std=c11", "-O1", "-Wall", "-o", exe, os.path.join(HERE, "c_api_example.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"), "-L", PKG, "-latlasgb"]
    for d in libdirs:
        cmd += ["-L", d]
    cmd += ["-lcudart", "-lm", "-Wl,-rpath," + PKG] + ["-Wl,-rpath," + d for d in libdirs]
    subprocess.check_call(cmd)
    return exe


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_c_program_without_a_gpu_gets_ecuda(example):
    if _has_gpu():
        pytest.skip("a GPU is present (the GPU test runs the program)")
    p = subprocess.run([example, "8", example + ".geom"], capture_output=True, text=True, timeout=120)
    assert p.returncode == 2, p.stdout + p.stderr
    assert "returned -3" in p.stdout
    assert "regional 13 x 9: 117 nodes" in p.stdout and "reloaded 117 nodes" in p.stdout


@pytest.mark.gpu
def test_c_program_on_the_gpu(example):
    if not _has_gpu():
        pytest.skip("no CUDA device")
    for N in ("16", "80"):
        p = subprocess.run([example, N, example + ".geom"], capture_output=True, text=True, timeout=300)
        assert p.returncode == 0, p.stdout + p.stderr
        assert "exactly 0" in p.stdout and p.stdout.rstrip().endswith("ok")
