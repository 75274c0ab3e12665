"""Shared helpers of the test-suite: builds oracle and library views of the same
seeded synthetic inputs (paper_2112_06830_gb300.synth)."""
import functools

import numpy as np

import oracle
from paper_2112_06830_gb300 import synth

TOL_FP32 = 1e-4      # mag, FP32 contraction against the FP64 oracle
TOL_BF16X3 = 1e-3    # mag, split-bf16 tensor contraction against the FP64 oracle


@functools.lru_cache(maxsize=None)
def ssp(kind: str):
    spec = synth.SMALL_GRID if kind == "small" else synth.FULL_GRID
    return synth.make_ssp(spec, 0 if kind == "small" else 1)


@functools.lru_cache(maxsize=None)
def oracle_grid(kind: str, sfh_model: int, mdf_kernel: int = 0):
    g = ssp(kind)
    return oracle.Grid(g.log_age_yr, g.lgz, g.lam, g.l_ssp, t0=g.t0, t1=g.t1, n_t=g.n_t,
                       sfh_model=sfh_model, mdf_kernel=mdf_kernel)


def params_f32(p):
    """The library takes float32 parameters; the oracle gets the very same
    (float32-rounded) values in float64."""
    p32 = np.ascontiguousarray(p, dtype=np.float32)
    return p32, p32.astype(np.float64)
