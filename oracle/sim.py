"""End-to-end FP64 forward model, call-for-call with the library's entry points
(TEST INFRASTRUCTURE ONLY).

    sim = Simulation(**workload)     # pm_init: cosmology tables, schedule
    sim.ic(noise)                    # pm_ic:  LPT state at a0 and F(x0)
    for i in range(nsteps):
        sim.step(i)                  # pm_step: kick, drift, force at a_{i+1}
        sim.lens_project(i)          # lens_project: shell i onto the maps
    kappa = sim.kappa_maps()         # kappa_maps: subtract the mean term
"""
from __future__ import annotations

import numpy as np

from .cosmology import Cosmology
from .lightcone import LensGeometry
from .lpt import linear_modes, lpt_displacements, lpt_state
from .nbody import PMState, Stepper, compute_force, kdk_step, pgd_displacement


class Simulation:
    def __init__(self, nc, nmesh, box, a_init, nsteps, zs, map_npix, map_fov_deg,
                 omega_m, sigma8, h=0.6774, n_s=0.9667, omega_b=0.0486, t_cmb=2.7255,
                 lpt_order=1, sub_evolution=1, pgd=0, pgd_params=(0.0, 0.0, 0.1, 1.0, 4.0),
                 rotate=1, rotation_seed=42, cosmo=None, source_nz=None, **_ignored):
        self.nc, self.nmesh, self.box = int(nc), int(nmesh), float(box)
        self.nsteps, self.lpt_order = int(nsteps), int(lpt_order)
        self.cosmo = cosmo or Cosmology(omega_m, sigma8, h, n_s, omega_b, t_cmb,
                                        a_min=min(0.02, 0.5 * a_init))
        self.stepper = Stepper(self.cosmo, a_init, nsteps)
        self.geom = LensGeometry(self.cosmo, self.stepper, zs, map_npix, map_fov_deg,
                                 box, nc, nmesh, rotate=rotate, seed=rotation_seed,
                                 sub_evolution=sub_evolution)
        # source_nz: {plane index: (z, n)} -- those planes become distributions n(z)
        for s_, (z, n) in (source_nz or {}).items():
            self.geom.set_source_nz(int(s_), z, n)
        self.pgd = bool(pgd)
        self.pgd_params = tuple(pgd_params)
        self.maps = np.zeros((len(self.geom.zs), self.geom.npix, self.geom.npix))
        self.state = None
        self.hits = 0

    def ic(self, noise):
        dk = linear_modes(noise, self.cosmo, self.box)
        psi1, psi2 = lpt_displacements(dk, self.nc, self.box, self.lpt_order)
        x, p = lpt_state(psi1, psi2, self.cosmo, self.stepper.a[0], self.nc, self.box,
                            self.nmesh)
        self.set_state(x, p)
        return psi1, psi2

    def set_state(self, x, p):
        f = compute_force(x, self.nc, self.nmesh, self.box, self.cosmo.omega_m)
        self.state = PMState(np.mod(x, self.box), p, f)

    def step(self, i):
        self.state = kdk_step(self.state, i, self.stepper, self.nc, self.nmesh, self.box)

    def pgd_at(self, i):
        """PGD displacement at x(a_{i+1}) (None when PGD is off)."""
        if not self.pgd:
            return None
        return pgd_displacement(self.state.x, self.stepper.a[i + 1], self.nc, self.nmesh,
                                self.box, self.pgd_params)

    def lens_project(self, i):
        if not self.geom.active(i):
            return
        S = self.pgd_at(i)
        inc, hits = self.geom.project(i, self.state.x, self.state.p, S)
        self.maps += inc
        self.hits += hits

    def kappa_maps(self):
        return self.maps - self.geom.mean_term()[:, None, None]

    def run(self, noise):
        self.ic(noise)
        for i in range(self.nsteps):
            self.step(i)
            self.lens_project(i)
        return self.kappa_maps()
