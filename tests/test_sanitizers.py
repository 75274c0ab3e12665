"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer, on the CPU:

* the FP64 oracle (oracle/oracle.c), rebuilt with -fsanitize=address,undefined
  and driven in a child process (libasan preloaded) through every entry point
  on small grids with every model option: weights, magnitudes and their
  adjoint, spectra and line widths, the nebular axis, age-dependent dust,
  tabulated histories, rest-frame filters, both MDF kernels;
* the request loop's host-only logic (paper_2112_06830_gb300/csrc/serve_host.h:
  the HBM arena, the batch choice, the fault switch), built with the same
  sanitizers into tests/sanitize_host.cpp's driver.

Any invalid access, leak-free misuse or undefined operation aborts the child
(-fno-sanitize-recover=all) and fails the test."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g", "-O1"]


def _need(tool):
    if shutil.which(tool) is None:
        pytest.skip(f"needs {tool}")


def test_serve_host_logic_under_sanitizers(tmp_path):
    _need("g++")
    exe = tmp_path / "sanitize_host"
    subprocess.run(["g++", "-std=c++17", *SAN, "-I", os.path.join(ROOT, "paper_2112_06830_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "sanitize_host.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 failures" in r.stdout


_DRIVER = r"""
import sys
sys.path.insert(0, %(root)r)
import numpy as np
import oracle
oracle._LIB = %(lib)r
oracle.build = lambda force=False: oracle._LIB
from paper_2112_06830_gb300 import synth

spec = synth.GridSpec(9, 5, 120, 1e3, 1e5)
g = synth.make_ssp(spec, 0)
F = oracle.Filters(synth.make_filters(3))
Fr = oracle.Filters(synth.make_filters(2), rest=True)
n = 5
rng = np.random.default_rng(0)
for sfh in (0, 1):
    for kernel in (0, 1):
        grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, sfh_model=sfh, mdf_kernel=kernel,
                           dust_bump=1, dust_law=kernel)
        p = synth.make_population(sfh, n, 1)
        w = oracle.weights(grid, p, nthreads=2)
        m = oracle.mags(grid, F, p, nthreads=2)
        m2, pb = oracle.mags_vjp(grid, F, p, rng.standard_normal((n, 3)), nthreads=2)
        mr = oracle.mags(grid, Fr, p)
        sp = oracle.spectra(grid, p)
        ew = oracle.line_ew(grid, p, 5007.0, 40.0, 300.0)
        assert np.isfinite(m).all() and np.isfinite(pb).all() and np.isfinite(mr).all()
# nebular axis
gn = synth.make_ssp_nebular(spec, 0)
grid = oracle.Grid(gn.log_age_yr, gn.lgz, gn.lam, gn.l_ssp, sfh_model=1, lgu=gn.lgu)
p = synth.with_nebular(synth.make_population(1, n, 2), 2)
oracle.mags_vjp(grid, F, p, rng.standard_normal((n, 3)))
oracle.weights(grid, p)
# age-dependent dust, T_erf MDF mean
grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, sfh_model=1, dust_agedep=1, mdf_mean=1)
p = synth.with_agedep_dust(synth.with_terf_mdf(synth.make_population(1, n, 3), 3), 3)
oracle.mags_vjp(grid, F, p, rng.standard_normal((n, 3)))
oracle.line_ew(grid, p, 5007.0, 40.0, 300.0)
# tabulated histories, with an invalid galaxy
grid = oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, sfh_model=oracle.SFH_TABLE)
p = synth.with_sfr_table(synth.make_population(1, n, 4), g.n_t, 4)
p[11, 2] = -1.0
oracle.mags_vjp(grid, F, p, rng.standard_normal((n, 3)))
# scalar entry points
for z in (-3.5, -3.0, 0.0, 1.7, 3.0, 4.0):
    oracle.triweight_cdf(z); oracle.triweight_pdf(z); oracle.gauss_cdf(z)
oracle.age_gyr(0.5); oracle.dist_mod(2.0)
print("oracle under sanitizers: ok")
"""


def test_oracle_under_sanitizers(tmp_path):
    _need("gcc")
    lib = tmp_path / "liboracle_san.so"
    subprocess.run(["gcc", "-std=gnu11", "-fPIC", "-shared", *SAN, "-o", str(lib),
                    os.path.join(ROOT, "oracle", "oracle.c"), "-lm", "-lpthread"], check=True)
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("libasan.so not found")
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", _DRIVER % {"root": ROOT, "lib": str(lib)}], capture_output=True,
                       text=True, env=env, timeout=900, cwd=ROOT)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    assert "oracle under sanitizers: ok" in r.stdout
