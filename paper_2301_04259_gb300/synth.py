"""Seeded synthetic inputs shaped like the workloads of SOAP-GPU (arXiv 2301.04259).

The paper integrates Kitt Peak FTS / PHOENIX local spectra (Sect. 2.1, Sect. 4.3)
which are not available here.  These generators stand in for them with
Gaussian-line spectra on a log-uniform wavelength grid; they feed BOTH the CUDA
library and the CPU oracle and contain none of the method's arithmetic (no
Doppler shift, no interpolation, no limb darkening, no disk sum).

Every draw comes from ``numpy.random.default_rng(seed)``.

Line model, per local spectrum (one per centre-to-limb angle mu):
    S(lambda) = prod_l [1 - d_l(mu) * exp(-(lambda - lambda_l(mu))^2 / (2 sigma_l^2))]
truncated at +-8 sigma, with d_l(mu) = d_l * (0.8 + 0.2 mu) (line depth grows to disk
centre) and, for the quiet photosphere only, lambda_l(mu) = lambda_l * (1 + v_cb(mu)/c)
with v_cb(mu) = -0.3 km/s * mu (convective blueshift, strongest at disk centre).  The
active-region spectrum carries no blueshift (convection inhibited, Sect. 4.3.2), lines
1.2x deeper, and extra weak "molecular" lines (Sect. 4.3.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

C_KMS = 299792.458          # speed of light, km/s
SPOT, FACULA = 1, 2         # region types (InfoMap values, Sect. 3.3)


@dataclass
class Star:
    """Stellar parameters that fix the disk geometry (Sect. 2.1, Fig. 0)."""
    grid_n: int
    vsini_kms: float
    incl_deg: float
    u1: float
    u2: float
    lambda_start_A: float
    lambda_end_A: float
    n_px: int
    mu_values: np.ndarray
    t_quiet_K: float = 5778.0
    diff_rot_alpha: float = 0.0

    @property
    def n_mu(self) -> int:
        return int(len(self.mu_values))


@dataclass
class Region:
    """One active region: type (1 spot, 2 facula), centre, radius (R*), temperature."""
    type: int
    lat_deg: float
    lon_deg: float
    radius_rstar: float
    temp_K: float


@dataclass
class Case:
    """A complete synthetic workload: star, local spectra, regions, phases, CCF mask."""
    name: str
    star: Star
    quiet: np.ndarray                      # [n_mu, n_px] float64
    active: Dict[int, np.ndarray]          # type -> [n_mu, n_px] float64
    regions: List[Region]
    phases: np.ndarray                     # [n_phases] float64, in rotations
    mask_lambda: np.ndarray                # rest wavelengths (A)
    mask_weight: np.ndarray                # CCF weights (line depth)
    mask_width_kms: float = 0.82
    seed: int = 0
    extra: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------------
# wavelength grid and line spectra (input construction only)
# ----------------------------------------------------------------------------------

def wavelength_grid(lambda_start: float, lambda_end: float, n_px: int) -> np.ndarray:
    """Log-uniform grid with both ends included: lambda_n = lambda_start * exp(n * Delta)."""
    delta = np.log1p((lambda_end - lambda_start) / lambda_start) / (n_px - 1)
    return lambda_start * np.exp(np.arange(n_px, dtype=np.float64) * delta)


def _line_product(lam: np.ndarray, centers, depths, sigmas, trunc: float = 8.0) -> np.ndarray:
    """prod_l (1 - d_l g_l(lambda)) over lines, each truncated at +-trunc sigma."""
    centers = np.asarray(centers, np.float64)
    depths = np.asarray(depths, np.float64)
    sigmas = np.asarray(sigmas, np.float64)
    lo = np.searchsorted(lam, centers - trunc * sigmas)
    hi = np.searchsorted(lam, centers + trunc * sigmas)
    counts = hi - lo
    total = int(counts.sum())
    if total == 0:
        return np.ones_like(lam)
    starts = np.repeat(lo, counts)
    offs = np.arange(total) - np.repeat(np.cumsum(counts) - counts, counts)
    idx = starts + offs
    li = np.repeat(np.arange(len(centers)), counts)
    g = np.exp(-0.5 * ((lam[idx] - centers[li]) / sigmas[li]) ** 2)
    log_s = np.bincount(idx, weights=np.log1p(-depths[li] * g), minlength=lam.size)
    return np.exp(log_s)


def local_spectra(lam, centers, depths, sigmas, mu_values, *, cb_kms_at_disk_centre=-0.3,
                  depth_scale=1.0, extra_lines=None) -> np.ndarray:
    """[n_mu, n_px] local spectra following the line model in the module docstring."""
    out = np.empty((len(mu_values), lam.size), np.float64)
    for b, mu in enumerate(mu_values):
        d = np.minimum(depths * depth_scale * (0.8 + 0.2 * mu), 0.99)
        c = centers * (1.0 + cb_kms_at_disk_centre * mu / C_KMS)
        s = _line_product(lam, c, d, sigmas)
        if extra_lines is not None:
            ec, ed, es = extra_lines
            s = s * _line_product(lam, ec, np.minimum(ed * (0.8 + 0.2 * mu), 0.99), es)
        out[b] = s
    return out


def _mask(centers, depths, min_depth=0.05):
    keep = depths > min_depth
    order = np.argsort(centers[keep])
    return centers[keep][order].copy(), depths[keep][order].copy()


# ----------------------------------------------------------------------------------
# generic case builder
# ----------------------------------------------------------------------------------

def make_case(seed: int, *, name: str, grid_n: int, lambda_start: float, lambda_end: float,
              n_px: int, mu_values, n_lines: int, depth_law: str, sigma_law: str,
              n_molecular: Optional[int] = None, molecular_from: float = 0.0,
              vsini_kms: float = 2.0, incl_deg: float = 90.0, u1: float = 0.29, u2: float = 0.34,
              regions: Optional[List[Region]] = None, n_phases: int = 25,
              region_draw=None, t_quiet: float = 5778.0, diff_rot_alpha: float = 0.0) -> Case:
    rng = np.random.default_rng(seed)
    lam = wavelength_grid(lambda_start, lambda_end, n_px)
    centers = rng.uniform(lambda_start, lambda_end, n_lines)
    if depth_law == "uniform":          # d ~ U(0.1, 0.8)
        depths = rng.uniform(0.1, 0.8, n_lines)
    else:                               # d log-uniform in [0.01, 0.9]
        depths = np.exp(rng.uniform(np.log(0.01), np.log(0.9), n_lines))
    if sigma_law == "angstrom":         # sigma ~ U(0.03, 0.08) A
        sigmas = rng.uniform(0.03, 0.08, n_lines)
    else:                               # sigma ~ U(1.5, 4) km/s in velocity
        sigmas = centers * rng.uniform(1.5, 4.0, n_lines) / C_KMS
    n_mol = n_lines // 3 if n_molecular is None else n_molecular
    mol_lo = lambda_start + molecular_from * (lambda_end - lambda_start)
    mc = rng.uniform(mol_lo, lambda_end, n_mol)
    md = rng.uniform(0.01, 0.1, n_mol)
    if sigma_law == "angstrom":
        ms = rng.uniform(0.03, 0.08, n_mol)
    else:
        ms = mc * rng.uniform(1.5, 4.0, n_mol) / C_KMS
    mu_values = np.asarray(mu_values, np.float64)
    quiet = local_spectra(lam, centers, depths, sigmas, mu_values)
    active = local_spectra(lam, centers, depths, sigmas, mu_values, cb_kms_at_disk_centre=0.0,
                           depth_scale=1.2, extra_lines=(mc, md, ms))
    if regions is None:
        regions = region_draw(rng) if region_draw is not None else []
    star = Star(grid_n=grid_n, vsini_kms=vsini_kms, incl_deg=incl_deg, u1=u1, u2=u2,
                lambda_start_A=lambda_start, lambda_end_A=lambda_end, n_px=n_px,
                mu_values=mu_values, t_quiet_K=t_quiet, diff_rot_alpha=diff_rot_alpha)
    ml, mw = _mask(centers, depths)
    phases = np.arange(n_phases, dtype=np.float64) / n_phases
    return Case(name=name, star=star, quiet=quiet, active={SPOT: active, FACULA: active},
                regions=list(regions), phases=phases, mask_lambda=ml, mask_weight=mw, seed=seed,
                extra={"line_centers": centers, "line_depths": depths, "line_sigmas": sigmas})


# ----------------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------------

def config1(seed: int = 0) -> Case:
    """Disk 50x50, 6000-6010 A at 4096 px, 30 lines, 11 mu values, one 0.1 R* spot at
    latitude 20 deg, 25 phases, vsini 2 km/s, i = 90 deg."""
    return make_case(seed, name="disk50_4096px_1spot_25ph", grid_n=50, lambda_start=6000.0,
                     lambda_end=6010.0, n_px=4096, mu_values=0.1 + 0.09 * np.arange(11),
                     n_lines=30, depth_law="uniform", sigma_law="angstrom", n_molecular=10,
                     regions=[Region(SPOT, 20.0, 0.0, 0.1, 4800.0)], n_phases=25)


def _cfg2_regions(rng):
    # one facula (0.15 R*, 6100 K) listed first, then two spots (0.05-0.1 R*, 4800 K);
    # the facula surrounds the first spot (a complex region, Sect. 4.2.2).
    lat1, lon1 = rng.uniform(-60, 60), rng.uniform(0, 360)
    lat2, lon2 = rng.uniform(-60, 60), rng.uniform(0, 360)
    r1, r2 = rng.uniform(0.05, 0.1), rng.uniform(0.05, 0.1)
    return [Region(FACULA, lat1, lon1, 0.15, 6100.0),
            Region(SPOT, lat1, lon1, r1, 4800.0),
            Region(SPOT, lat2, lon2, r2, 4800.0)]


CFG2_N_PX = 205800   # 3800-6900 A at 3 px per R=115000 resolution element


def config2(seed: int = 0, *, grid_n: int = 300, n_px: int = CFG2_N_PX,
            lambda_start: float = 3800.0, lambda_end: float = 6900.0,
            n_lines: Optional[int] = None, n_phases: int = 100) -> Case:
    """Disk 300x300, 3800-6900 A log-uniform at 3 px per R=115000 element (205,800 px),
    20 mu bins, 20k lines (depth log-uniform 0.01-0.9), 2 spots + 1 facula, 100 phases,
    vsini 2 km/s, i = 90 deg.  Smaller grids / ranges keep the same line density."""
    if n_lines is None:
        n_lines = int(round(20000 * (lambda_end - lambda_start) / 3100.0))
    return make_case(seed, name=f"disk{grid_n}_{n_px}px_2spot1fac_{n_phases}ph", grid_n=grid_n,
                     lambda_start=lambda_start, lambda_end=lambda_end, n_px=n_px,
                     mu_values=(np.arange(20) + 0.5) / 20.0, n_lines=n_lines,
                     depth_law="loguniform", sigma_law="velocity", molecular_from=0.4,
                     region_draw=_cfg2_regions, n_phases=n_phases)


def n_px_for_sampling(lambda_start: float, lambda_end: float, resolution: float = 115000.0,
                      px_per_element: float = 3.0) -> int:
    """Pixels of a log-uniform grid with px_per_element pixels per lambda/R element."""
    return int(round(np.log(lambda_end / lambda_start) * resolution * px_per_element)) + 1


@dataclass
class BatchConfig:
    """One independent active-region configuration of the batched workload."""
    vsini_kms: float
    incl_deg: float
    regions: List[Region]
    n_phases: int


def batch_configs(seed: int, n_configs: int) -> List[BatchConfig]:
    """Per config: 1-4 spots of radius U(0.01,0.2) R*, latitude U(-60,60), longitude
    U(0,360), 10-200 phases, vsini U(1,10) km/s, inclination U(30,90) deg."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_configs):
        ns = int(rng.integers(1, 5))
        regs = [Region(SPOT, float(rng.uniform(-60, 60)), float(rng.uniform(0, 360)),
                       float(rng.uniform(0.01, 0.2)), 4800.0) for _ in range(ns)]
        out.append(BatchConfig(vsini_kms=float(rng.uniform(1, 10)),
                               incl_deg=float(rng.uniform(30, 90)), regions=regs,
                               n_phases=int(rng.integers(10, 201))))
    return out


def batch_layout(configs: List[BatchConfig]):
    """Flatten configs into (items, regions, phases): item k = (vsini, incl, first_region,
    n_regions, first_phase, n_phases); config k's phases are j / n_phases, j = 0 .. n_phases-1
    (one rotation)."""
    items, regions, phases = [], [], []
    for c in configs:
        items.append((c.vsini_kms, c.incl_deg, len(regions), len(c.regions), len(phases), c.n_phases))
        regions.extend(c.regions)
        phases.extend((np.arange(c.n_phases) / c.n_phases).tolist())
    return items, regions, np.asarray(phases, dtype=np.float64)


def batch_spectra(seed: int, *, grid_n: int = 150, n_px: Optional[int] = None,
                  lambda_start: float = 6000.0, lambda_end: float = 6300.0) -> Case:
    """Shared local spectra for the batched workload (6000-6300 A, R=115000 x3 sampling)."""
    if n_px is None:
        n_px = n_px_for_sampling(lambda_start, lambda_end)
    n_lines = int(round(20000 * (lambda_end - lambda_start) / 3100.0))
    return make_case(seed, name=f"batch_disk{grid_n}_{n_px}px", grid_n=grid_n,
                     lambda_start=lambda_start, lambda_end=lambda_end, n_px=n_px,
                     mu_values=(np.arange(20) + 0.5) / 20.0, n_lines=n_lines,
                     depth_law="loguniform", sigma_law="velocity", molecular_from=0.4,
                     regions=[], n_phases=1, vsini_kms=10.0)


def velocity_grid(vsini_kms: float, step_kms: float = 0.25, margin_kms: float = 20.0):
    """CCF velocity grid -(vsini+margin) .. +(vsini+margin) in steps of step_kms."""
    half = vsini_kms + margin_kms
    n_v = int(np.floor(2 * half / step_kms + 1e-9)) + 1
    return -half, step_kms, n_v


# ----------------------------------------------------------------------------------
# learned surrogate: query parameters, their batch layout, initial weights
# ----------------------------------------------------------------------------------
# inputs: spot latitude (deg), spot longitude (deg), spot radius (R*), spot temperature (K),
# phase, inclination (deg), vsini (km/s), facula filling (facula area / spot area around it)
SURROGATE_INPUTS = ("lat_deg", "lon_deg", "radius_rstar", "spot_temp_K", "phase", "incl_deg", "vsini_kms",
                    "facula_filling")
SURROGATE_LO = np.array([-60.0, 0.0, 0.01, 3800.0, 0.0, 30.0, 1.0, 0.0])
SURROGATE_HI = np.array([60.0, 360.0, 0.2, 5600.0, 1.0, 90.0, 10.0, 3.0])
SURROGATE_FACULA_TEMP = 6100.0


def surrogate_params(seed: int, n: int) -> np.ndarray:
    """n query vectors drawn uniformly inside the surrogate's input ranges, float32 [n, 8]."""
    rng = np.random.default_rng(seed)
    return (SURROGATE_LO + (SURROGATE_HI - SURROGATE_LO) * rng.uniform(size=(n, 8))).astype(np.float32)


def surrogate_layout(params):
    """(items, regions, phases) of the batched method for query vectors: one item per query with
    one phase; a facula of area (1 + filling) x the spot's, centred on it and listed first (the
    spot keeps its cells), when filling > 0, then the spot."""
    items, regions, phases = [], [], []
    for k, q in enumerate(np.asarray(params, np.float64)):
        lat, lon, r, t_spot, ph, inc, vs, fill = q
        regs = []
        if fill > 0:
            regs.append(Region(FACULA, lat, lon, min(1.0, r * np.sqrt(1.0 + fill)), SURROGATE_FACULA_TEMP))
        regs.append(Region(SPOT, lat, lon, r, t_spot))
        items.append((vs, inc, len(regions), len(regs), k, 1))
        regions.extend(regs)
        phases.append(ph)
    return items, regions, np.asarray(phases, np.float64)


def surrogate_layout_columns(params):
    """surrogate_layout() as numpy columns (for many queries): a dict with item columns vsini,
    incl, first_region, n_regions, first_phase, n_phases, region columns type, lat, lon, radius,
    temp, and phases."""
    q = np.asarray(params, np.float64)
    n = q.shape[0]
    lat, lon, r, t_spot, ph, inc, vs, fill = (q[:, i] for i in range(8))
    has_fac = fill > 0
    n_reg = np.where(has_fac, 2, 1)
    first = np.concatenate([[0], np.cumsum(n_reg)[:-1]])
    total = int(n_reg.sum())
    rtype = np.full(total, SPOT, np.int32)
    rlat, rlon = np.empty(total), np.empty(total)
    rrad, rtemp = np.empty(total), np.empty(total)
    fac_idx = first[has_fac]
    spot_idx = first + has_fac.astype(np.int64)
    rtype[fac_idx] = FACULA
    for idx, sel in ((fac_idx, has_fac), (spot_idx, np.ones(n, bool))):
        rlat[idx], rlon[idx] = lat[sel], lon[sel]
    rrad[fac_idx] = np.minimum(1.0, r[has_fac] * np.sqrt(1.0 + fill[has_fac]))
    rtemp[fac_idx] = SURROGATE_FACULA_TEMP
    rrad[spot_idx], rtemp[spot_idx] = r, t_spot
    return dict(vsini=vs, incl=inc, first_region=first.astype(np.int32), n_regions=n_reg.astype(np.int32),
                first_phase=np.arange(n, dtype=np.int32), n_phases=np.ones(n, np.int32),
                type=rtype, lat=rlat, lon=rlon, radius=rrad, temp=rtemp, phases=ph.copy())


def surrogate_init(seed: int, shapes=((256, 8), (256, 256), (256, 256), (256, 256), (129, 256))) -> np.ndarray:
    """Initial weights, flat [W1 | b1 | ... ]: normal with variance 2/in (hidden layers) and
    1/in (output layer), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (o, i) in enumerate(shapes):
        sd = np.sqrt((1.0 if l == len(shapes) - 1 else 2.0) / i)
        parts += [rng.normal(0.0, sd, o * i), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)


def gaussian_test_matrix(seed: int, p: int, l: int) -> np.ndarray:
    """Standard normal test matrix [p, l] (float32) for the randomized PCA."""
    return np.random.default_rng(seed).standard_normal((p, l)).astype(np.float32)
