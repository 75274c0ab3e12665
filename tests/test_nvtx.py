"""Tracing: every ABI call of libdsps opens an NVTX range named after itself.
A small NVTX tool (tests/nvtx_inject.c, loaded through NVTX_INJECTION64_PATH,
the hook profilers use) records the ranges of calls made in a child process;
no GPU is needed, since the range opens before any argument check."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        inc = os.path.join(d, "include")
        if d and os.path.exists(os.path.join(inc, "nvtx3", "nvToolsExt.h")):
            return inc
    return None


def test_abi_calls_open_named_nvtx_ranges(tmp_path):
    from paper_2112_06830_gb300 import dsps
    inc = _cuda_include()
    if inc is None or shutil.which("gcc") is None:
        pytest.skip("needs gcc and the CUDA toolkit's NVTX 3 headers")
    lib = dsps.library_path()
    if not os.path.exists(lib):
        pytest.skip("libdsps.so is not built")
    so = tmp_path / "libnvtx_probe.so"
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-I", inc, os.path.join(ROOT, "tests", "nvtx_inject.c"),
                    "-o", str(so)], check=True)
    log = tmp_path / "ranges.log"
    code = (
        "import ctypes, sys; sys.path.insert(0, %r)\n"
        "from paper_2112_06830_gb300 import dsps\n"
        "lib = dsps.load()\n"
        "assert lib.dsps_photometry(None, 0, None, 0, 0, None, None) == dsps.DSPS_ERR_INVALID_ARG\n"
        "assert lib.dsps_photometry_vjp(None, 0, None, 0, 0, None, None, None, None) == dsps.DSPS_ERR_INVALID_ARG\n"
        "lib.dsps_poll(None, 1, 0, None)\n"
        "lib.dsps_photometry_fp32_static(None, 0, None, 0, None, None)\n"
    ) % ROOT
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(so), DSPS_NVTX_LOG=str(log))
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=ROOT, timeout=300)
    lines = log.read_text().split("\n")
    pushes = [ln[5:] for ln in lines if ln.startswith("push ")]
    pops = sum(ln == "pop" for ln in lines)
    assert pushes == ["dsps_photometry", "dsps_photometry_vjp", "dsps_poll", "dsps_photometry_fp32_static"], pushes
    assert pops == len(pushes)
