"""Seeded synthetic workloads for the two-grid triple-porosity Navier-Stokes solver.

This module holds problem *inputs* only: mesh sizes, grading, subdomain layout,
physical parameters and the seeded random draws that some workloads use.  It
contains none of the method's arithmetic, so both the CPU oracle (``oracle/``)
and the GPU path (``paper_2311_05170_gb300``) may import it.

Notation follows the paper (Sec. 2): macro-fracture ``F``, micro-fracture ``f``
and matrix ``m`` pressures; ``k`` are permeabilities, ``phiC`` the storage
coefficients phi_i*C_i, ``sigma`` / ``sigma_star`` the shape factors of the
f-m and F-f exchange terms, ``mu`` the dynamic viscosity (mu tilde), ``rho``,
``eta`` (rescaling factor), ``nu`` and the Beavers-Joseph ``alpha``.

Manufactured solutions (``mms``):
  1  the 2D trigonometric field  u = (sin(pi x) cos(pi y), -cos(pi x) sin(pi y)) e^-t,
     p = cos(pi x) cos(pi y) e^-t,  (p_m, p_f, p_F) = (1, 2, 3) cos(pi x) cos(pi y) e^-t
  3  the steady polynomial patch field  u = (x^2, -2xy), p = x + y,
     p_i = c_i (x^2 + y^2) with c = (3, 2, 1) for (F, f, m).
"""
import math
from dataclasses import dataclass, field, asdict
from typing import List, Tuple

import numpy as np


@dataclass
class Params:
    nu: float = 1.0
    eta: float = 1.0
    rho: float = 1.0
    mu: float = 1.0
    alpha: float = 1.0
    sigma: float = 1.0
    sigma_star: float = 1.0
    # order of the three Darcy fields everywhere: F (macro), f (micro), m (matrix)
    phiC: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    k: Tuple[float, float, float] = (1.0, 1.0, 1.0)


@dataclass
class Workload:
    """One 2D run: fluid region [0,1]x[1,2] over porous region [0,1]x[0,1], Gamma at y=1."""
    name: str
    nx_coarse: int                 # coarse cells in x (uniform, H = 1/nx_coarse)
    ny_coarse: int                 # coarse rows per region in y
    fine_per_coarse_x: int         # fine columns per coarse column (uniform)
    # fine rows per coarse row, listed from Gamma outwards (same on both sides of Gamma)
    fine_rows_from_gamma: List[int]
    nsub: Tuple[int, int]          # subdomains per region (x, y)
    overlap: int                   # overlap in fine layers beyond D_j
    dt: float
    nsteps: int
    mms: int
    params: Params = field(default_factory=Params)

    def to_dict(self):
        d = asdict(self)
        return d


def _fine_rows_uniform(ny_coarse, r):
    return [r] * ny_coarse


def config_small(nsteps=10) -> Workload:
    """2D uniform: H=1/4, h=1/16, 2x2 subdomains per region, overlap 2h, dt=0.01, all parameters 1."""
    return Workload("2d_uniform_H4_h16", 4, 4, 4, _fine_rows_uniform(4, 4), (2, 2), 2,
                    0.01, nsteps, 1, Params())


def graded_rows_8():
    """Fine rows per coarse row of height 1/8, from Gamma outwards: 16, 8, then 4 (h from 1/128 to 1/32)."""
    return [16, 8, 4, 4, 4, 4, 4, 4]


def draw_permeabilities(seed: int):
    """k_m, k_mi, k_M drawn in that order, log-uniform on [1e-4, 1]."""
    rng = np.random.default_rng(seed)
    ks = np.exp(rng.uniform(math.log(1e-4), math.log(1.0), size=3))
    k_m, k_mi, k_M = (float(v) for v in ks)
    return (k_M, k_mi, k_m)    # returned in (F, f, m) order


def config_graded(nsteps=200) -> Workload:
    """2D graded toward Gamma: H=1/8, h_x=1/128, h_y from 1/128 (at Gamma) to 1/32,
    4x4 subdomains per region, overlap 2 fine layers, log-uniform permeabilities (seed 0),
    dt=0.005, 200 steps."""
    p = Params(k=draw_permeabilities(0))
    return Workload("2d_graded_H8_h128", 8, 8, 16, graded_rows_8(), (4, 4), 2,
                    0.005, nsteps, 1, p)


def config_patch(nx_coarse=2, r=2, nsub=(2, 2), nsteps=3, dt=0.1) -> Workload:
    """Steady polynomial patch field (P2 velocity, P1 pressure, P2 Darcy pressures)."""
    p = Params(nu=0.7, eta=1.0, rho=1.3, mu=1.1, alpha=0.9, sigma=0.8, sigma_star=1.2,
               phiC=(0.5, 0.7, 0.9), k=(1.5, 0.6, 0.25))
    return Workload(f"2d_patch_H{nx_coarse}_r{r}", nx_coarse, nx_coarse, r,
                    [r] * nx_coarse, nsub, 1, dt, nsteps, 3, p)


def config_uniform(nx_coarse, r, nsub=(2, 2), overlap=2, dt=0.01, nsteps=10, mms=1,
                   params=None) -> Workload:
    """Uniform 2D run with H = 1/nx_coarse and h = H/r."""
    return Workload(f"2d_uniform_H{nx_coarse}_h{nx_coarse * r}", nx_coarse, nx_coarse, r,
                    [r] * nx_coarse, nsub, overlap, dt, nsteps, mms, params or Params())


def as_algorithm1(w: Workload) -> Workload:
    """The same run with the coarse mesh equal to the fine mesh (H = h) and one subdomain per
    region: the two-grid scheme then reduces to the global fine-grid partitioned time stepping
    of Algorithm 1 (the local corrections vanish).  Uniform fine rows only."""
    rows = w.fine_rows_from_gamma[: w.ny_coarse]
    if len(set(rows)) != 1:
        raise ValueError("Algorithm 1 workloads need uniform fine rows")
    r = rows[0]
    return Workload(w.name + "_alg1", w.nx_coarse * w.fine_per_coarse_x, w.ny_coarse * r, 1,
                    [1] * (w.ny_coarse * r), (1, 1), 0, w.dt, w.nsteps, w.mms, w.params)


def serving_requests(n=512, seed_arrivals=3, rate=20.0):
    """Serving workload: Poisson arrivals (exponential gaps, rate per second); per request a
    seeded h in {1/32, 1/64, 1/128}, H = sqrt(h) rounded (up, finer) to a power of 1/2, a
    subdomain count in {4, 16, 64} per region with D_j at least one coarse cell, and seeded
    physical parameters.  Returns a list of (arrival_time, Workload)."""
    rng = np.random.default_rng(seed_arrivals)
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    out = []
    for r in range(n):
        g = np.random.default_rng(1000 + r)
        inv_h = int(g.choice([32, 64, 128]))
        inv_H = {32: 8, 64: 8, 128: 16}[inv_h]
        ks = np.exp(g.uniform(math.log(1e-4), 0.0, size=3))
        phis = g.uniform(0.05, 0.3, size=3)
        sig = np.exp(g.uniform(math.log(1e-2), math.log(10.0), size=2))
        choices = [s for s in (2, 4, 8) if s <= inv_H]
        ns = int(g.choice(choices))
        p = Params(k=(float(ks[2]), float(ks[1]), float(ks[0])),
                   phiC=(float(phis[2]), float(phis[1]), float(phis[0])),
                   sigma=float(sig[0]), sigma_star=float(sig[1]))
        r_f = inv_h // inv_H
        w = Workload(f"req{r}_H{inv_H}_h{inv_h}", inv_H, inv_H, r_f, [r_f] * inv_H,
                     (ns, ns), 2, 0.01, 100, 1, p)
        out.append((float(t[r]), w))
    return out


def serving_requests_small(n=6, seed=7, rate=200.0, nsteps=4):
    """A small serving mix for tests: Poisson arrivals, h in {1/16, 1/32}, H in {1/4, 1/8},
    2 or 4 subdomains per direction, seeded permeabilities, porosities and exchange
    coefficients (same distributions as serving_requests).  Returns (arrival, Workload, nsteps)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for r in range(n):
        g = np.random.default_rng(2000 + r)
        inv_H = int(g.choice([4, 8]))
        ratio = int(g.choice([2, 4]))
        ns = int(g.choice([2, 4]))
        ks = np.exp(g.uniform(math.log(1e-4), 0.0, size=3))
        phis = g.uniform(0.05, 0.3, size=3)
        sig = np.exp(g.uniform(math.log(1e-2), math.log(10.0), size=2))
        p = Params(k=(float(ks[2]), float(ks[1]), float(ks[0])),
                   phiC=(float(phis[2]), float(phis[1]), float(phis[0])),
                   sigma=float(sig[0]), sigma_star=float(sig[1]))
        w = Workload(f"sreq{r}_H{inv_H}_h{inv_H * ratio}", inv_H, inv_H, ratio, [ratio] * inv_H,
                     (ns, ns), 2, 0.01, nsteps, 1, p)
        out.append((float(t[r]), w, nsteps))
    return out


# ---------------------------------------------------------------------------------- 3D
@dataclass
class Workload3D:
    """One 3D run: fluid region [0,1]^2 x [1,2] over porous region [0,1]^3, Gamma at z=1,
    uniform Kuhn tetrahedral meshes with H = 1/n_coarse and h = H / fine_per_coarse."""
    name: str
    n_coarse: int                  # coarse cells per axis and region
    fine_per_coarse: int           # fine cells per coarse cell and axis
    nsub: Tuple[int, int, int]     # subdomains per region (x, y, z)
    overlap: int                   # overlap in fine layers beyond D_j
    dt: float
    nsteps: int
    mms: int                       # 2: 3D trigonometric field, 4: steady polynomial patch field, 0: zero
    params: Params = field(default_factory=Params)
    dim: int = 3

    def to_dict(self):
        return asdict(self)


def config_3d(nsteps=50) -> Workload3D:
    """3D plain vs mixed precision: H=1/4, h=1/24, 2x2x2 subdomains per region, overlap 2h,
    3D trigonometric manufactured solution, all parameters 1, dt=0.01, 50 steps."""
    return Workload3D("3d_H4_h24_2x2x2sub_overlap2h_dt0.01", 4, 6, (2, 2, 2), 2, 0.01, nsteps, 2, Params())


def config_3d_small(n_coarse=2, r=2, nsub=(2, 2, 1), overlap=1, nsteps=2, dt=0.01, mms=2, params=None) -> Workload3D:
    """Small 3D runs for tests (H = 1/n_coarse, h = H/r)."""
    return Workload3D(f"3d_H{n_coarse}_h{n_coarse * r}_{nsub[0]}x{nsub[1]}x{nsub[2]}sub", n_coarse, r, nsub, overlap,
                      dt, nsteps, mms, params or Params())


def config_3d_patch(n_coarse=2, r=2, nsub=(2, 1, 1), nsteps=2, dt=0.1) -> Workload3D:
    """Steady polynomial patch field in 3D (P2 velocity, P1 pressure, P2 Darcy pressures)."""
    p = Params(nu=0.7, eta=1.0, rho=1.3, mu=1.1, alpha=0.9, sigma=0.8, sigma_star=1.2,
               phiC=(0.5, 0.7, 0.9), k=(1.5, 0.6, 0.25))
    return Workload3D(f"3d_patch_H{n_coarse}_r{r}", n_coarse, r, nsub, 1, dt, nsteps, 4, p)
