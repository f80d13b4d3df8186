"""Physical-to-lattice unit conversion and the paper's experiment set-ups.

The paper states its experiments in SI units (Section 4). In lattice units
(dx = dt = 1, c = 1, c_s^2 = 1/3, rho0 = 1):

* ``nu_eff = (tau - 1/2) / 3``                      (Section 2.1, below Eq. 1)
* ``nu_l = nu dt / dx^2``, ``kappa_l = kappa / dx^2``
* ``G_l = G dt^2 / dx``, ``u_l = u dt / dx``

The conversions only rescale inputs; they do not touch the method.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fields


@dataclass(frozen=True)
class LatticeUnits:
    dx: float
    dt: float

    def nu(self, nu_si: float) -> float:
        return nu_si * self.dt / (self.dx * self.dx)

    def kappa(self, k_si):
        return np.asarray(k_si, dtype=np.float64) / (self.dx * self.dx) if not np.isscalar(k_si) \
            else k_si / (self.dx * self.dx)

    def force(self, g_si):
        return g_si * self.dt * self.dt / self.dx

    def tau_from_nu_eff(self, nu_eff_si: float) -> float:
        return 0.5 + 3.0 * nu_eff_si * self.dt / (self.dx * self.dx)


def paper_experiment(name: str, **kw) -> dict:
    """Lattice-unit set-up of one of the paper's experiments.

    ``name``: ``"E1"`` (Eq. 22, Section 4.1), ``"E2"`` series layers (Table 1),
    ``"E3"`` parallel layers (Table 2), ``"E4"`` checkerboard (Table 3; ``n`` = 100
    or 1000), ``"E5_local"``/``"E6_local"`` (one 10x10 sinusoidal block of Eq. 23,
    Sections 4.3.1/4.3.2), ``"E5_fine"``, ``"E6_fine"`` (400x400, Eq. 23 with
    G = (sin pi x, sin pi y)). Keyword ``ratio`` selects kappa2/kappa1 for E2-E4.

    Returns a dict with ``tau, nu, eps, kappa [ny, nx], g (gx, gy) or gfield [2, ny, nx]``.
    """
    eps = 0.8
    nu_si = 2e-6
    if name == "E1":
        u = LatticeUnits(0.01, 1e-4)
        return dict(tau=0.53, nu=u.nu(nu_si), eps=eps,
                    kappa=u.kappa(fields.block_kappa_eq22(100, 1e-6, 1e-5)),
                    g=(u.force(2.0), 0.0))
    if name in ("E2", "E3"):
        u = LatticeUnits(0.01, 1e-4)
        k1 = 1e-12
        k2 = kw.get("ratio", 2.0) * k1
        ny = kw.get("ny", 100)
        kap = fields.layered_kappa(100, ny, k1, k2)
        if name == "E2":
            return dict(tau=0.53, nu=u.nu(nu_si), eps=eps, kappa=u.kappa(kap), g=(u.force(2.0), 0.0))
        return dict(tau=0.5, nu=u.nu(nu_si), eps=eps, kappa=u.kappa(kap), g=(0.0, u.force(2.0)))
    if name == "E4":
        n = kw.get("n", 100)
        u = LatticeUnits(0.01, 1e-4) if n == 100 else LatticeUnits(1e-3, 1e-5)
        k1 = 1e-12
        k2 = kw.get("ratio", 2.0) * k1
        kap = fields.checkerboard_kappa(n, k1, k2)
        return dict(tau=0.5, nu=u.nu(nu_si), eps=eps, kappa=u.kappa(kap), g=(u.force(2.0), 0.0))
    if name in ("E5_local", "E6_local", "E5_fine", "E6_fine"):
        u = LatticeUnits(0.0025, 2.5e-5)
        k_const = 1e-13 if name.startswith("E5") else 1e-7
        tau = 0.5 if name.startswith("E5") or kw.get("nu_eff_zero", False) \
            else u.tau_from_nu_eff(1e-5)
        if name.endswith("local"):
            # one 10x10 block of the sinusoidal region: the sinusoid has exactly one
            # period per block, so any such block is the same local problem
            full = fields.fiveblock_kappa_eq23(400, k_const)
            kap = full[:10, :10]
            return dict(tau=tau, nu=u.nu(nu_si), eps=eps, kappa=u.kappa(kap),
                        g_const=u.force(2.0), k_const=u.kappa(k_const))
        kap = fields.fiveblock_kappa_eq23(400, k_const)
        return dict(tau=tau, nu=u.nu(nu_si), eps=eps, kappa=u.kappa(kap),
                    gfield=fields.sinusoidal_g_field(400, u.force(1.0)), k_const=u.kappa(k_const))
    raise ValueError(f"unknown experiment {name!r}")
