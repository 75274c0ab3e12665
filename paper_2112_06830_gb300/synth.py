"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method: it only draws the stand-in data
(SSP grid, filter tables, galaxy parameters) that the paper's experiments take
from FSPS/MILES, LSST filter curves and Diffstar, none of which is available.
Both sides (oracle and CUDA library) read exactly these arrays.

Workloads (sizes and distributions of the paper's benchmark, Sec. 5.1 and its
synthetic stand-ins):

* ``small``   64 galaxies; SSP grid 94 ages x 12 metallicities x 1000 wavelengths
              (log-spaced 1e3..1e5 A); 6 Gaussian filters; delayed-tau SFH.
* ``full``    1e5 galaxies; grid 107 x 22 x 5994 (log-spaced 900..1e5 A);
              12 Gaussian filters; double power-law SFH with a quench drop;
              age-dependent MDF mean.  ``million`` is the same with 1e6 galaxies,
              ``grad`` the same with 1e5 galaxies and magnitude targets.
* ``serve``   Poisson request stream over the ``full`` grid.

Parameter rows (structure of arrays, ``params[12, G]`` float):
    0..4 SFH, 5 mdf_mu, 6 mdf_sigma, 7 mdf_slope, 8 Av, 9 delta, 10 logM, 11 z;
    with a nebular axis ``params[14, G]``: 12 u_mean, 13 u_sigma.
"""
from __future__ import annotations

import dataclasses

import numpy as np

NPAR = 12
NGRAD = 11
PARAM_NAMES = ("sfh0", "sfh1", "sfh2", "sfh3", "sfh4", "mdf_mu", "mdf_sigma", "mdf_slope",
               "Av", "delta", "logM", "z")

SFH_DELAYED_TAU = 0
SFH_DPL_QUENCH = 1
SFH_TABLE = 2          # SFR tabulated at the n_t time nodes (the last n_t parameter rows)
MDF_TRIWEIGHT = 0
MDF_GAUSSIAN = 1

_H = 6.62607015e-34
_C = 2.99792458e8
_KB = 1.380649e-23


@dataclasses.dataclass(frozen=True)
class GridSpec:
    n_age: int
    n_z: int
    n_lam: int
    lam_min: float
    lam_max: float
    log_age_min: float = 5.5
    log_age_max: float = 10.15
    lgz_min: float = -2.0
    lgz_max: float = 0.3
    n_t: int = 200
    t0: float = 0.05
    t1: float = 13.8


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    grid: GridSpec
    n_gal: int
    n_filt: int
    sfh_model: int
    seed: int


SMALL_GRID = GridSpec(94, 12, 1000, 1e3, 1e5)
FULL_GRID = GridSpec(107, 22, 5994, 900.0, 1e5)

WORKLOADS = {
    "small": Workload("small", SMALL_GRID, 64, 6, SFH_DELAYED_TAU, 0),
    "full": Workload("full", FULL_GRID, 100_000, 12, SFH_DPL_QUENCH, 1),
    "million": Workload("million", FULL_GRID, 1_000_000, 12, SFH_DPL_QUENCH, 2),
    "grad": Workload("grad", FULL_GRID, 100_000, 12, SFH_DPL_QUENCH, 3),
}


@dataclasses.dataclass
class SSPGrid:
    log_age_yr: np.ndarray   # [n_age] float64
    lgz: np.ndarray          # [n_z]   float64, log10(Z/0.019)
    lam: np.ndarray          # [n_lam] float64, Angstrom
    l_ssp: np.ndarray        # [n_age, n_z, n_lam] (or [n_age, n_z, n_u, n_lam]) float32, Lsun/Hz/Msun
    t0: float
    t1: float
    n_t: int
    lgu: np.ndarray | None = None   # [n_u] log10 U of the nebular axis, or None


def _planck_lambda(lam_aa: np.ndarray, T: np.ndarray) -> np.ndarray:
    lam = lam_aa * 1e-10
    x = _H * _C / (lam * _KB * T)
    return 2.0 * _H * _C ** 2 / lam ** 5 / np.expm1(x)


def make_ssp(spec: GridSpec, seed: int) -> SSPGrid:
    """Synthetic SSP block: L = C (age/1e6 yr)^-0.9 B_lambda(T) exp(0.05 N(0,1)),
    T = 4000 K + 36000 K (1e6 yr/age)^0.3 (Z/0.019)^-0.05, C such that the
    noiseless value at (age nearest 1 Gyr, Z nearest 0.019, lambda nearest 5500 A)
    is 3e-15."""
    log_age = np.linspace(spec.log_age_min, spec.log_age_max, spec.n_age)
    lgz = np.linspace(spec.lgz_min, spec.lgz_max, spec.n_z)
    lam = np.geomspace(spec.lam_min, spec.lam_max, spec.n_lam)
    age = 10.0 ** log_age
    T = 4000.0 + 36000.0 * (1e6 / age[:, None]) ** 0.3 * (10.0 ** lgz[None, :]) ** -0.05
    base = (age[:, None, None] / 1e6) ** -0.9 * _planck_lambda(lam[None, None, :], T[:, :, None])
    i0 = int(np.argmin(np.abs(log_age - 9.0)))
    j0 = int(np.argmin(np.abs(lgz - 0.0)))
    n0 = int(np.argmin(np.abs(lam - 5500.0)))
    base *= 3e-15 / base[i0, j0, n0]
    rng = np.random.default_rng(seed)
    noise = np.exp(0.05 * rng.standard_normal(base.shape))
    return SSPGrid(log_age, lgz, lam, (base * noise).astype(np.float32), spec.t0, spec.t1, spec.n_t)


def with_emission_line(ssp: SSPGrid, lam_line: float = 5007.0, sigma: float = 8.0, amp: float = 30.0,
                       age_scale: float = 5e6) -> SSPGrid:
    """The same SSP block with a Gaussian emission line of width ``sigma`` [A] at
    ``lam_line`` added to the young populations, as the stand-in for the nebular
    lines the paper's SSPs carry: row (i, j) gains
    a_i L_ij(lam_line) exp(-(lam - lam_line)^2 / (2 sigma^2)) with
    a_i = amp / (1 + (age_i / age_scale)^2), L_ij(lam_line) the row's value at the
    grid point nearest the line."""
    lam = ssp.lam
    n_l = int(np.argmin(np.abs(lam - lam_line)))
    age = 10.0 ** ssp.log_age_yr
    a = amp / (1.0 + (age / age_scale) ** 2)
    prof = np.exp(-0.5 * ((lam - lam_line) / sigma) ** 2)
    base = ssp.l_ssp.astype(np.float64)
    add = a[:, None, None] * base[:, :, n_l:n_l + 1] * prof[None, None, :]
    return SSPGrid(ssp.log_age_yr, ssp.lgz, lam, (base + add).astype(np.float32), ssp.t0, ssp.t1, ssp.n_t)


# Nebular axis (Sec. 3.3): log U grid of the stand-in SSPs (FSPS's range and step).
LGU_GRID = np.linspace(-4.0, -1.0, 7)
NPAR_NEB = NPAR + 2


def make_ssp_nebular(spec: GridSpec, seed: int, lgu=LGU_GRID, age_scale: float = 5e6) -> SSPGrid:
    """SSP block with a nebular axis, l_ssp [n_age, n_z, n_u, n_lam]: the
    continuum of ``make_ssp`` (the same for every U) plus Gaussian emission
    lines on the young populations whose strengths depend on the ionisation
    parameter u = log10 U, standing in for FSPS's nebular lines: a 5007 A line
    growing with u (amplitude 10 * 10^(0.6 (u + 2.5))), a 3727 A line falling
    with u (8 * 10^(-0.4 (u + 2.5))) and a 6563 A line independent of u (20),
    each times a_i = 1 / (1 + (age_i / age_scale)^2) and the row's continuum at
    the line (sigma 8 A)."""
    base = make_ssp(spec, seed)
    lam = base.lam
    lgu = np.asarray(lgu, dtype=np.float64)
    age = 10.0 ** base.log_age_yr
    a = 1.0 / (1.0 + (age / age_scale) ** 2)
    cont = base.l_ssp.astype(np.float64)
    out = np.repeat(cont[:, :, None, :], len(lgu), axis=2)
    for lam_l, amp in ((5007.0, 10.0 * 10.0 ** (0.6 * (lgu + 2.5))), (3727.0, 8.0 * 10.0 ** (-0.4 * (lgu + 2.5))),
                       (6563.0, np.full(len(lgu), 20.0))):
        n_l = int(np.argmin(np.abs(lam - lam_l)))
        prof = np.exp(-0.5 * ((lam - lam_l) / 8.0) ** 2)
        out += (a[:, None, None, None] * amp[None, None, :, None] * cont[:, :, None, n_l:n_l + 1]
                * prof[None, None, None, :])
    return SSPGrid(base.log_age_yr, base.lgz, lam, out.astype(np.float32), base.t0, base.t1, base.n_t, lgu)


def with_nebular(params: np.ndarray, seed: int, start: int = 0) -> np.ndarray:
    """The same galaxies with the nebular rows appended: row 12 u_mean ~
    U[-3.5, -1.5], row 13 u_sigma = 0.25 dex (the paper's Sec. 3.3 example
    scatter); galaxy i's draw depends only on (seed, i)."""
    p = np.asarray(params, dtype=np.float64)
    n = p.shape[1]
    out = np.zeros((NPAR_NEB, n))
    out[:NPAR] = p
    if n == 0:
        return out
    b0, b1 = start // _BLOCK, (start + n - 1) // _BLOCK
    draws = [np.random.default_rng([seed, b, 13]).uniform(-3.5, -1.5, _BLOCK) for b in range(b0, b1 + 1)]
    out[12] = np.concatenate(draws)[start - b0 * _BLOCK:start - b0 * _BLOCK + n]
    out[13] = 0.25
    return out


def with_agedep_dust(params: np.ndarray, seed: int, start: int = 0) -> np.ndarray:
    """The same galaxies with age-dependent dust (Sec. 3.4.1): rows 8, 9 become
    the young-star values Av_young ~ U[0.4, 2.0], delta_young ~ U[-0.6, 0.0],
    and two rows are appended, Av_old ~ U[0, 0.8], delta_old ~ U[-0.4, 0.3];
    galaxy i's draw depends only on (seed, i)."""
    p = np.asarray(params, dtype=np.float64)
    n = p.shape[1]
    out = np.zeros((p.shape[0] + 2, n))
    out[:p.shape[0]] = p
    if n == 0:
        return out
    b0, b1 = start // _BLOCK, (start + n - 1) // _BLOCK
    draws = []
    for b in range(b0, b1 + 1):
        rng = np.random.default_rng([seed, b, 17])
        draws.append(np.stack([rng.uniform(0.4, 2.0, _BLOCK), rng.uniform(-0.6, 0.0, _BLOCK),
                               rng.uniform(0.0, 0.8, _BLOCK), rng.uniform(-0.4, 0.3, _BLOCK)]))
    d = np.concatenate(draws, axis=1)[:, start - b0 * _BLOCK:start - b0 * _BLOCK + n]
    out[8], out[9], out[-2], out[-1] = d
    return out


def with_sfr_table(params: np.ndarray, n_t: int, seed: int, start: int = 0) -> np.ndarray:
    """The same galaxies with a tabulated star formation history appended as
    the last n_t rows (the SFR at the n_t time nodes, in arbitrary units) and
    rows 0-4 set to 0 (unused).  The histories are random, not of any
    parametric form, standing in for tabulated ones such as simulation
    outputs: log SFR is a rise-and-fall curve (peak at a random node) plus a
    Gaussian random walk of 0.08 dex per node, with two bursts of up to 10x
    lasting one to three nodes, and a third of the galaxies drop to exactly 0
    after a random node in the second half of the grid.  Galaxy i's draw
    depends only on (seed, i)."""
    p = np.asarray(params, dtype=np.float64)
    n = p.shape[1]
    out = np.zeros((p.shape[0] + n_t, n))
    out[:p.shape[0]] = p
    out[:5] = 0.0
    if n == 0:
        return out
    b0, b1 = start // _BLOCK, (start + n - 1) // _BLOCK
    x = np.arange(n_t) / (n_t - 1)
    tabs = []
    for b in range(b0, b1 + 1):
        rng = np.random.default_rng([seed, b, 19])
        xp = rng.uniform(0.1, 0.8, _BLOCK)[:, None]
        wd = rng.uniform(0.15, 0.5, _BLOCK)[:, None]
        lg = -((x[None, :] - xp) / wd) ** 2 * 0.5
        lg = lg + np.cumsum(rng.normal(0.0, 0.08, (_BLOCK, n_t)), axis=1)
        t = 10.0 ** np.clip(lg, -4.0, 2.0)
        for _ in range(2):
            at = rng.integers(0, n_t, _BLOCK)
            ln = rng.integers(1, 4, _BLOCK)
            amp = rng.uniform(1.0, 10.0, _BLOCK)
            m = (np.arange(n_t)[None, :] >= at[:, None]) & (np.arange(n_t)[None, :] < (at + ln)[:, None])
            t = np.where(m, t * amp[:, None], t)
        cut = rng.integers(n_t // 2, n_t, _BLOCK)
        quench = rng.uniform(0.0, 1.0, _BLOCK) < 1.0 / 3.0
        t = np.where(quench[:, None] & (np.arange(n_t)[None, :] > cut[:, None]), 0.0, t)
        tabs.append(t)
    tab = np.concatenate(tabs, axis=0)[start - b0 * _BLOCK:start - b0 * _BLOCK + n]
    out[p.shape[0]:] = tab.T
    return out


# Line-strength workload: [OIII] 5007 A (the line of the paper's Sec. 3.3 example),
# line window +-30 A, continuum 100 A on each side.
EW_LINE = (5007.0, 30.0, 100.0)


def gaussian_filter(center: float, fwhm: float = 800.0, step: float = 2.0):
    """Gaussian transmission curve with unit peak, tabulated every ``step`` A and
    truncated at center +- 4 FWHM."""
    sig = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    n = int(round(8.0 * fwhm / step)) + 1
    lam = center - 4.0 * fwhm + step * np.arange(n)
    return lam, np.exp(-0.5 * ((lam - center) / sig) ** 2)


def make_filters(n_filt: int, lo: float = 3500.0, hi: float = 9000.0, fwhm: float = 800.0):
    """``n_filt`` Gaussian filters with centres evenly spaced on [lo, hi]."""
    return [gaussian_filter(c, fwhm) for c in np.linspace(lo, hi, n_filt)]


_BLOCK = 4096


def _draw_block(sfh_model: int, seed: int, block: int) -> np.ndarray:
    rng = np.random.default_rng([seed, block])
    n = _BLOCK
    p = np.zeros((NPAR, n))
    if sfh_model == SFH_DELAYED_TAU:
        p[0] = rng.uniform(0.5, 5.0, n)            # tau [Gyr]
        p[10] = rng.uniform(9.0, 11.5, n)          # logM
        p[5] = rng.uniform(-1.0, 0.2, n)           # mdf mu
        p[6] = 0.2                                 # mdf sigma
        p[7] = 0.0                                 # uncorrelated MDF
        p[8] = rng.uniform(0.0, 1.0, n)            # Av
        p[9] = rng.uniform(-0.4, 0.3, n)           # delta
        p[11] = rng.uniform(0.1, 1.5, n)           # z
    else:
        p[0] = rng.uniform(1.0, 10.0, n)           # t_peak [Gyr]
        p[1] = rng.uniform(1.0, 3.0, n)            # rising slope
        p[2] = rng.uniform(-3.0, -0.5, n)          # falling slope
        p[3] = rng.uniform(5.0, 13.8, n)           # t_q [Gyr]
        p[4] = rng.uniform(0.0, 3.0, n)            # q_drop [dex]
        p[10] = rng.uniform(9.0, 11.5, n)
        p[5] = rng.uniform(-1.0, 0.2, n)
        p[6] = 0.2
        p[7] = rng.uniform(-0.3, 0.0, n)           # MDF slope
        p[8] = rng.uniform(0.0, 1.0, n)
        p[9] = rng.uniform(-0.4, 0.3, n)
        p[11] = np.maximum(rng.uniform(0.0, 3.0, n), 1e-3)
    return p


def make_population(sfh_model: int, n: int, seed: int, start: int = 0) -> np.ndarray:
    """Galaxy parameters ``[12, n]`` (float64) for galaxies [start, start+n).
    Galaxy i depends only on (seed, i), so any slice is a prefix-consistent
    sample of the full population."""
    if n <= 0:
        return np.zeros((NPAR, 0))
    b0, b1 = start // _BLOCK, (start + n - 1) // _BLOCK
    blocks = [_draw_block(sfh_model, seed, b) for b in range(b0, b1 + 1)]
    allp = np.concatenate(blocks, axis=1)
    off = start - b0 * _BLOCK
    return np.ascontiguousarray(allp[:, off:off + n])


def with_terf_mdf(params: np.ndarray, seed: int, start: int = 0) -> np.ndarray:
    """The same galaxies with the paper's age-dependent MDF in its T_erf form:
    row 5 becomes mu_young ~ U[-0.5, 0.4] and row 7 mu_old ~ U[-1.6, -0.4]
    (old stars metal-poor), galaxy i's draw depending only on (seed, i)."""
    p = np.array(params, dtype=np.float64, copy=True)
    n = p.shape[1]
    if n == 0:
        return p
    b0, b1 = start // _BLOCK, (start + n - 1) // _BLOCK
    draws = []
    for b in range(b0, b1 + 1):
        rng = np.random.default_rng([seed, b, 7])
        draws.append(np.stack([rng.uniform(-0.5, 0.4, _BLOCK), rng.uniform(-1.6, -0.4, _BLOCK)]))
    d = np.concatenate(draws, axis=1)[:, start - b0 * _BLOCK:start - b0 * _BLOCK + n]
    p[5], p[7] = d[0], d[1]
    return p


def workload_inputs(name: str, n_gal: int | None = None, start: int = 0):
    """(grid, filters, params) for a named workload."""
    w = WORKLOADS[name]
    grid = make_ssp(w.grid, w.seed if name in ("small",) else 1)
    filters = make_filters(w.n_filt)
    params = make_population(w.sfh_model, w.n_gal if n_gal is None else n_gal, w.seed, start)
    return grid, filters, params


@dataclasses.dataclass
class Request:
    t_arrive: float
    n_gal: int
    n_filt: int
    want_grad: bool
    seed: int


def make_request_stream(rate: float = 200.0, duration: float = 60.0, seed: int = 4,
                        median: float = 3e3, sigma_ln: float = 1.5, lo: int = 100,
                        hi: int = 200_000, grad_frac: float = 0.3):
    """Poisson arrivals; population sizes lognormal(median, sigma_ln) clipped to
    [lo, hi]; filter sets of 4, 8 or 12 filters with equal probability; a
    fraction ``grad_frac`` of requests also asks for gradients."""
    rng = np.random.default_rng(seed)
    t, out, i = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(np.clip(np.round(median * np.exp(sigma_ln * rng.standard_normal())), lo, hi))
        q = int(rng.choice([4, 8, 12]))
        g = bool(rng.uniform() < grad_frac)
        out.append(Request(t, n, q, g, 1000 + i))
        i += 1
    return out
