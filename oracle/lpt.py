"""Initial conditions: Gaussian modes and Lagrangian perturbation theory
(TEST INFRASTRUCTURE ONLY).

Sec. 4 / Appendix A: the model is differentiable in the initial Gaussian modes,
the linear power is Eisenstein-Hu, and the initial conditions are LPT.

Readings (the paper is silent on each):
* the "initial modes" are a real-space N(0,1) white-noise field w on the
  Nc^3 particle lattice; delta_L(k) = DFT(w)(k) * sqrt(P(k) Nc^3 / V) with
  V = L^3, P the z = 0 linear power, and k = 0 set to 0;
* Psi1 = IDFT[i k / k^2 delta_L]  (div Psi1 = -delta_L), Nyquist planes of the
  odd factor zeroed;
* 2LPT: div Psi2 = sum_{i<j} (Psi1_{i,i} Psi1_{j,j} - Psi1_{i,j}^2), so that
  Psi2 = IDFT[-i k / k^2 DFT(source)], with x = q + D1 Psi1 + D2 Psi2 and
  D2 -> -(3/7) D1^2 (this sign reproduces the Eulerian second-order kernel);
* lattice position q_j = (jx, jy, jz) L / Nc + L / (2 M): offset by half a
  force-mesh cell, so that for integer B = M / Nc the unperturbed lattice
  paints to an exactly uniform CIC density (particles on mesh nodes would put
  order-one power into the aliased lattice modes and bias the force even in
  the linear regime); particle index j = (jz Nc + jy) Nc + jx;
* p = g_p(a) Psi1 + g_p2(a) Psi2 with g_p = a^3 E dD1/da, g_p2 = a^3 E dD2/da.
"""
from __future__ import annotations

import numpy as np

from .mesh import gradient_multipliers, wavevectors
from . import dft


def lattice(nc, box, nmesh):
    """Lagrangian lattice positions q (N, 3), x fastest."""
    j = np.arange(nc, dtype=np.float64) * (box / nc) + 0.5 * box / nmesh
    qz, qy, qx = np.meshgrid(j, j, j, indexing="ij")
    return np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)


def linear_modes(noise, cosmo, box):
    """delta_L(k) (half spectrum) of the z = 0 linear field from white noise."""
    nc = noise.shape[0]
    kx, ky, kz = wavevectors(nc, box)
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    amp = np.sqrt(cosmo.pk_lin(k) * nc ** 3 / box ** 3)
    dk = dft.rfftn(noise) * amp
    dk[0, 0, 0] = 0.0
    return dk


def _odd(k, nc, box):
    kny = np.pi * nc / box
    return np.where(np.abs(np.abs(k) - kny) < 1e-9 * kny, 0.0, k)


def lpt_displacements(delta_k, nc, box, order=1):
    """Psi1 (and Psi2 when order == 2) on the lattice, each (N, 3)."""
    shape = (nc, nc, nc)
    mult = gradient_multipliers(nc, box)
    psi1 = np.stack([dft.irfftn(m * delta_k, s=shape, axes=(0, 1, 2)).ravel() for m in mult], axis=1)
    if order == 1:
        return psi1, None
    kx, ky, kz = wavevectors(nc, box)
    kk = (kx, ky, kz)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0, 1.0 / k2, 0.0)
    # Psi1_{i,j} = d_j Psi1_i = -k_i k_j / k^2 delta; the diagonal k_i^2 is
    # even and kept, off-diagonal terms are odd in both axes.
    d = {}
    for i in range(3):
        for j in range(i, 3):
            if i == j:
                mult_ij = -kk[i] * kk[i] * inv
            else:
                mult_ij = -_odd(kk[i], nc, box) * _odd(kk[j], nc, box) * inv
            d[(i, j)] = dft.irfftn(mult_ij * delta_k, s=shape, axes=(0, 1, 2))
    src = (d[(0, 0)] * d[(1, 1)] + d[(0, 0)] * d[(2, 2)] + d[(1, 1)] * d[(2, 2)]
           - d[(0, 1)] ** 2 - d[(0, 2)] ** 2 - d[(1, 2)] ** 2)
    sk = dft.rfftn(src)
    psi2 = np.stack([dft.irfftn(-m * sk, s=shape, axes=(0, 1, 2)).ravel() for m in mult], axis=1)
    return psi1, psi2


def lpt_state(psi1, psi2, cosmo, a, nc, box, nmesh):
    """Particle positions (wrapped to [0, L)) and momenta at scale factor a."""
    q = lattice(nc, box, nmesh)
    x = q + cosmo.D1(a) * psi1
    p = cosmo.gp(a) * psi1
    if psi2 is not None:
        x = x + cosmo.D2(a) * psi2
        p = p + cosmo.gp2(a) * psi2
    return np.mod(x, box), p
