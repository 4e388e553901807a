"""FastPM kick-drift-kick stepping in FP64 (TEST INFRASTRUCTURE ONLY).

Sec. 3: particles are evolved "through a kick and drift scheme enforcing correct
linear displacement in each step", with forces from a particle-mesh solver.

Schedule (reading; steps linear in a, a_i = a0 + i (1 - a0) / n,
a_{i+1/2} = (a_i + a_{i+1}) / 2, a_{-1/2} = a0):
* initial conditions at a0 give x_0, p_0 and the force F_0 = F(x_0);
* step i (i = 0 .. n-1):
    kick   p <- p + F_i  [g_p(a_{i+1/2}) - g_p(a_{i-1/2})] / g_f(a_i)
    drift  x <- x + p    [D1(a_{i+1}) - D1(a_i)] / g_p(a_{i+1/2})
    force  F_{i+1} = F(x_{i+1})
  so that after step i the state is x(a_{i+1}), p(a_{i+1/2}) and F_{i+1}; the
  lightcone shell of step i is projected from exactly that state.
"""
from __future__ import annotations

import numpy as np

from .cosmology import Cosmology, time_grid
from .mesh import density, pm_forces, cic_readout, pgd_mesh


class Stepper:
    """Per-step kick and drift coefficients (FP64)."""

    def __init__(self, cosmo: Cosmology, a_init: float, nsteps: int):
        self.cosmo = cosmo
        self.a, self.ah = time_grid(a_init, nsteps)
        self.nsteps = nsteps
        a_prev_half = np.concatenate([[self.a[0]], self.ah[:-1]])
        self.kick = (cosmo.gp(self.ah) - cosmo.gp(a_prev_half)) / cosmo.gf(self.a[:-1])
        self.drift = (cosmo.D1(self.a[1:]) - cosmo.D1(self.a[:-1])) / cosmo.gp(self.ah)


class PMState:
    """Particle state and the force at the current positions."""

    def __init__(self, x, p, force):
        self.x = x
        self.p = p
        self.force = force


def compute_force(x, nc, nmesh, box, omega_m):
    f, _, _ = pm_forces(x, nc, nmesh, box, omega_m)
    return f


def kdk_step(state: PMState, i: int, stepper: Stepper, nc, nmesh, box):
    """One kick-drift step followed by the force at the new positions."""
    p = state.p + state.force * stepper.kick[i]
    x = np.mod(state.x + p * stepper.drift[i], box)
    f = compute_force(x, nc, nmesh, box, stepper.cosmo.omega_m)
    return PMState(x, p, f)


def pgd_displacement(x, a, nc, nmesh, box, pgd_params):
    """PGD displacement S at the particles from the density of x at time a."""
    alpha0, mu, k_l, k_s, n_s = pgd_params
    rho = density(x, nc, nmesh, box)
    sm = pgd_mesh(rho - 1.0, box, alpha0 * a ** mu, k_l, k_s, n_s)
    return np.stack([cic_readout(m, x, box) for m in sm], axis=1)
