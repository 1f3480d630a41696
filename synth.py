"""Seeded synthetic inputs for the quasi-static wake march (shared by the oracle and the CUDA path).

This module holds no arithmetic of the method itself.  It only

* names the workloads (parameter sets in normalised units: lengths in k_p^-1, densities in n_p,
  momenta in m c), with the two-bunch driver of Eq. 12 and the warm plasma of Sec. II.A;
* draws the random numbers the method consumes, as standard normals, from NumPy's PCG64:
  - plasma: one (u_r, u_theta, u_z) triple per macroparticle, drawn in mirrored pairs
    (particle 2p+1 carries the negated draw of particle 2p), so that each pair has zero net
    momentum;
  - beam: five normals per macroparticle (x, y, u_x, u_y, xi).

Both the oracle and the CUDA library scale these normals themselves (u = u_th * n,
x = sigma_r * n, ...), so the two sides share the draws and nothing else.

Workload shapes follow the paper's parameter sets: the single-bunch OSIRIS comparison
(Sec. III, uniform plasma, bi-Gaussian driver) and the Table I two-bunch FACET driver
(Sec. II.B, Eq. 12), in a warm plasma (Sec. II.A).  No dataset is involved.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20141112


@dataclasses.dataclass
class WakeConfig:
    """One simulation's parameters, normalised units (k_p^-1, n_p, m c)."""

    nr: int              # radial cells; nodes r_i = i*dr, i = 0..nr
    nxi: int             # xi cells; nodes xi_k = k*dxi, k = 0..nxi
    ppc: int             # plasma macroparticles per radial cell (even when u_th > 0)
    rmax: float          # wall radius R
    ximax: float         # box length L
    u_th: float = 0.0    # plasma thermal momentum (Maxwellian, per component)
    n_d: float = 0.1     # drive peak density (Eq. 12)
    n_w: float = 0.0     # witness peak density (Eq. 12)
    sigma_r: float = 0.5
    sigma_zd: float = 1.0
    sigma_zw: float = 0.5625
    xi_d: float = 4.0
    xi_w: float = 8.5
    gamma_b: float = 4.0e4
    eps_n: float = 1.0e-2   # normalised emittance; sigma_u_perp = eps_n / sigma_r
    n_beam: int = 0         # beam macroparticles (0: frozen analytic driver)
    n_drive: int = 0        # first n_drive beam particles belong to the drive bunch
    ds: float = 5.0         # beam time step
    n_steps: int = 0        # beam steps in one run
    seed: int = SEED_BASE
    geometry: int = 0       # 0: cylindrical (r, xi); 1: slab (x, xi), mirror plane x = 0

    @property
    def np_plasma(self) -> int:
        return self.nr * self.ppc


def two_bunch(cfg: WakeConfig, q_ratio: float, delay: float, n_beam: int) -> WakeConfig:
    """Fill in the witness bunch of Eq. 12: sigma_zw = 0.5625 sigma_zd (the Table I ratio
    0.81/1.44), xi_w = xi_d + delay, and n_w such that Q_w = q_ratio * Q_d (charge of a
    bi-Gaussian bunch scales as n sigma_z sigma_r^2; both bunches share sigma_r).  Beam
    macroparticles are split in proportion to charge."""
    cfg.sigma_zw = 0.5625 * cfg.sigma_zd
    cfg.xi_w = cfg.xi_d + delay
    cfg.n_w = q_ratio * cfg.n_d * cfg.sigma_zd / cfg.sigma_zw
    cfg.n_beam = int(n_beam)
    cfg.n_drive = int(n_beam) - int(round(n_beam * q_ratio / (1.0 + q_ratio)))
    return cfg


def config_linear(nr=128, nxi=256, n0=0.1) -> WakeConfig:
    """Plain FP64, frozen driver: Nr=128 over r in [0,6], Nxi=256 over 10, cold plasma with
    4 particles per cell, single bi-Gaussian driver n_b/n_p=n0, sigma_r=0.5, sigma_z=1
    (linear regime)."""
    return WakeConfig(nr=nr, nxi=nxi, ppc=4, rmax=6.0, ximax=10.0, u_th=0.0, n_d=n0, n_w=0.0,
                      sigma_r=0.5, sigma_zd=1.0, xi_d=4.0, seed=SEED_BASE + 1)


def config_slab_linear(nr=128, nxi=256, n0=0.1) -> WakeConfig:
    """Slab geometry (x, xi), mirror plane x = 0, conducting wall at x = 6: the linear case's
    grid and sheet driver n_b = n0 exp(-x^2/2 sigma^2) f(xi), sigma = 0.5, sigma_z = 1."""
    cfg = config_linear(nr=nr, nxi=nxi, n0=n0)
    cfg.geometry = 1
    cfg.seed = SEED_BASE + 21
    return cfg


def config_slab_blowout(n_beam=1 << 20, n_steps=200, nr=512, nxi=2048) -> WakeConfig:
    """The blowout workload in slab geometry: the same box, warm plasma and two sheet bunches
    (drive n_b/n_p = 8 peaked on the mirror plane x = 0, witness 4.5 behind)."""
    cfg = config_blowout(n_beam=n_beam, n_steps=n_steps, nr=nr, nxi=nxi)
    cfg.geometry = 1
    cfg.seed = SEED_BASE + 22
    return cfg


def config_blowout(n_beam=1 << 20, n_steps=200, nr=512, nxi=2048) -> WakeConfig:
    """Nonlinear blowout, two bunches: Nr=512 over 8, Nxi=2048 over 12, warm plasma with
    8 particles per cell and u_th=0.01 (about 51 eV); drive n_b/n_p=8, sigma_r=0.2,
    sigma_z=0.6, gamma=4e4, xi_d = 4 sigma_zd; witness 4.5 behind with 30% of the drive
    charge; normalised emittance 1e-2; beam step 5."""
    cfg = WakeConfig(nr=nr, nxi=nxi, ppc=8, rmax=8.0, ximax=12.0, u_th=0.01, n_d=8.0,
                     sigma_r=0.2, sigma_zd=0.6, xi_d=2.4, gamma_b=4.0e4, eps_n=1.0e-2,
                     ds=5.0, n_steps=n_steps, seed=SEED_BASE + 2)
    return two_bunch(cfg, 0.3, 4.5, n_beam)


def config_large(n_beam=1 << 24, n_steps=1000) -> WakeConfig:
    """Large: Nr=2048 over 10, Nxi=8192 over 16, 32 particles per cell, u_th=0.02, the
    blowout two-bunch driver with 16M beam macroparticles, 1000 beam steps."""
    cfg = WakeConfig(nr=2048, nxi=8192, ppc=32, rmax=10.0, ximax=16.0, u_th=0.02, n_d=8.0,
                     sigma_r=0.2, sigma_zd=0.6, xi_d=2.4, gamma_b=4.0e4, eps_n=1.0e-2,
                     ds=5.0, n_steps=n_steps, seed=SEED_BASE + 5)
    return two_bunch(cfg, 0.3, 4.5, n_beam)


def config_table1(nr=256, nxi=1024, u_th=0.0, n_beam=0) -> WakeConfig:
    """Table I two-bunch FACET parameters in normalised units: n_d=3.56, n_w=2.85,
    sigma_r=0.42, sigma_zd=1.44, sigma_zw=0.81, xi_w - xi_d = 5.48, 23 GeV (gamma=45000).
    xi_d = 4 sigma_zd; box 6 x 16."""
    return WakeConfig(nr=nr, nxi=nxi, ppc=4 if u_th == 0 else 8, rmax=6.0, ximax=16.0,
                      u_th=u_th, n_d=3.56, n_w=2.85, sigma_r=0.42, sigma_zd=1.44,
                      sigma_zw=0.81, xi_d=5.76, xi_w=5.76 + 5.48, gamma_b=23.0e3 / 0.511,
                      n_beam=n_beam, n_drive=n_beam, seed=SEED_BASE + 11)


def config_facet(n_beam=1 << 20, te_ev=0.0, nr=256, nxi=1024, ds=5.0) -> WakeConfig:
    """The Table I two-bunch beam as macroparticles in a plasma of temperature te_ev
    (u_th = sqrt(T_e / m c^2)), with zero initial emittance as in the paper's FACET runs
    (Sec. III).  Macroparticles are split between the bunches in proportion to their charge
    (n sigma_z sigma_r^2, both bunches sharing sigma_r)."""
    cfg = config_table1(nr=nr, nxi=nxi, u_th=math.sqrt(te_ev / 511.0e3))
    q_ratio = (cfg.n_w * cfg.sigma_zw) / (cfg.n_d * cfg.sigma_zd)
    cfg.n_beam = int(n_beam)
    cfg.n_drive = int(n_beam) - int(round(n_beam * q_ratio / (1.0 + q_ratio)))
    cfg.eps_n = 0.0
    cfg.ds = ds
    return cfg


def config_osiris(n_beam=2_500_000, nr=200, nxi=500, ds=5.0) -> WakeConfig:
    """The single-bunch parameter set of the paper's OSIRIS comparison (Sec. III): box
    10 x 25 with 200 x 500 cells, cold plasma with 9 macroparticles per cell, driver
    n_d = 3.6, sigma_r = 0.19, sigma_zd = 1.72 at 30 GeV, 2.5e6 beam macroparticles, no
    witness.  Readings: the driver centred at xi_d = 4 sigma_zd, and zero emittance (the
    paper states none for this run)."""
    return WakeConfig(nr=nr, nxi=nxi, ppc=9, rmax=10.0, ximax=25.0, u_th=0.0, n_d=3.6, n_w=0.0,
                      sigma_r=0.19, sigma_zd=1.72, xi_d=4 * 1.72, xi_w=4 * 1.72, gamma_b=30.0e3 / 0.511,
                      eps_n=0.0, n_beam=int(n_beam), n_drive=int(n_beam), ds=ds, seed=SEED_BASE + 12)


def config_batch(n_sims=256, n_steps=50, seed=SEED_BASE + 3) -> list[WakeConfig]:
    """Batched sweep of the linear-driver physics plus a witness: Nr in {128..1024} and
    Nxi in {512..4096}, each log-uniform over powers of two; R=6, L=10, ppc=4;
    u_th ~ U[0, 0.02]; witness delay ~ U[3.5, 5.5]; beam macroparticles log-uniform in
    [65536, 262144]; 50 steps of 5."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_sims):
        nr = int(2 ** rng.integers(7, 11))
        nxi = int(2 ** rng.integers(9, 13))
        u_th = float(rng.uniform(0.0, 0.02))
        delay = float(rng.uniform(3.5, 5.5))
        nb = int(round(math.exp(rng.uniform(math.log(65536), math.log(262144)))))
        cfg = WakeConfig(nr=nr, nxi=nxi, ppc=4, rmax=6.0, ximax=10.0, u_th=u_th, n_d=0.1,
                         sigma_r=0.5, sigma_zd=1.0, xi_d=4.0, gamma_b=4.0e4, eps_n=1.0e-2,
                         ds=5.0, n_steps=n_steps, seed=seed * 1000 + s)
        out.append(two_bunch(cfg, 0.3, delay, nb))
    return out


def config_adjoint(n_steps=100, seed=SEED_BASE + 4) -> WakeConfig:
    """Differentiation workload: the linear-driver grid (Nr=128 over 6, 4 particles per cell)
    at Nxi=1024 over 10, the batched sweep's first witness delay, 262,144 beam
    macroparticles split by charge, u_th = 0.005, n_steps beam steps of 5."""
    cfg = config_batch(n_sims=1, seed=seed)[0]
    cfg.nr, cfg.nxi, cfg.ppc = 128, 1024, 4
    cfg = two_bunch(cfg, 0.3, cfg.xi_w - cfg.xi_d, 262144)
    cfg.u_th = 0.005
    cfg.n_steps = n_steps
    return cfg


def plasma_normals(cfg: WakeConfig) -> np.ndarray | None:
    """Standard normals for the warm-plasma momenta, shape (np_plasma, 3) holding
    (u_r, u_theta, u_z) draws, mirrored in pairs.  None for a cold plasma."""
    if cfg.u_th == 0.0:
        return None
    n = cfg.np_plasma
    if n % 2:
        raise ValueError("a warm plasma needs an even particle count per cell")
    rng = np.random.default_rng(cfg.seed)
    half = rng.standard_normal((n // 2, 3))
    out = np.empty((n, 3))
    out[0::2] = half
    out[1::2] = -half
    return np.ascontiguousarray(out)


def beam_normals(cfg: WakeConfig) -> np.ndarray:
    """Standard normals for the beam, shape (5, n_beam): x, y, u_x, u_y, xi."""
    rng = np.random.default_rng(cfg.seed + 7919)
    return np.ascontiguousarray(rng.standard_normal((5, cfg.n_beam)))
