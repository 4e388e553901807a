"""FP64 mesh operations of the particle-mesh solver (TEST INFRASTRUCTURE ONLY).

Conventions (the paper fixes none of them; Sec. 3 only says particles are
"painted" to a force mesh of resolution B x the particle grid):

* mesh arrays are float64 of shape (M, M, M) indexed [iz, iy, ix] (x fastest);
  node (ix, iy, iz) sits at position (ix, iy, iz) * L / M;
* cloud-in-cell (CIC) assignment to the 8 nearest nodes, periodic;
* forward DFT with sign -1, unnormalised (numpy.fft.rfftn over all axes);
* exact spectral operators: k_j = 2 pi n_j / L with n_j in [-M/2, M/2),
  k^2 = |k|^2, the k = 0 mode set to 0, and every factor odd in k_j
  (i k_j) set to 0 on the Nyquist plane of axis j so that real fields stay real.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import dft

def cic_paint(pos, nmesh, box, weight=1.0):
    """Cloud-in-cell paint of particles at pos (N, 3) [x, y, z] in Mpc/h."""
    pos = np.asarray(pos, dtype=np.float64)
    g = pos * (nmesh / box)
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    w = np.broadcast_to(np.asarray(weight, dtype=np.float64), (pos.shape[0],))
    out = np.zeros(nmesh ** 3, dtype=np.float64)
    for dx, dy, dz in itertools.product((0, 1), repeat=3):
        wx = f[:, 0] if dx else 1.0 - f[:, 0]
        wy = f[:, 1] if dy else 1.0 - f[:, 1]
        wz = f[:, 2] if dz else 1.0 - f[:, 2]
        ix = (i0[:, 0] + dx) % nmesh
        iy = (i0[:, 1] + dy) % nmesh
        iz = (i0[:, 2] + dz) % nmesh
        flat = (iz * nmesh + iy) * nmesh + ix
        out += np.bincount(flat, weights=w * wx * wy * wz, minlength=nmesh ** 3)
    return out.reshape(nmesh, nmesh, nmesh)


def cic_readout(mesh, pos, box):
    """Cloud-in-cell interpolation of a mesh [iz, iy, ix] at positions (N, 3)."""
    nmesh = mesh.shape[0]
    pos = np.asarray(pos, dtype=np.float64)
    g = pos * (nmesh / box)
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    out = np.zeros(pos.shape[0], dtype=np.float64)
    for dx, dy, dz in itertools.product((0, 1), repeat=3):
        wx = f[:, 0] if dx else 1.0 - f[:, 0]
        wy = f[:, 1] if dy else 1.0 - f[:, 1]
        wz = f[:, 2] if dz else 1.0 - f[:, 2]
        out += wx * wy * wz * mesh[(i0[:, 2] + dz) % nmesh,
                                   (i0[:, 1] + dy) % nmesh,
                                   (i0[:, 0] + dx) % nmesh]
    return out


def cic_readout_grad(mesh, pos, box):
    """d/dx_d of the CIC interpolation of a mesh, shape (N, 3), per Mpc/h.

    The CIC weight is piecewise linear; at a node the derivative is taken from
    the cell that contains the particle (floor convention), as in cic_readout.
    """
    nmesh = mesh.shape[0]
    pos = np.asarray(pos, dtype=np.float64)
    g = pos * (nmesh / box)
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    out = np.zeros_like(pos)
    for dx, dy, dz in itertools.product((0, 1), repeat=3):
        w = [f[:, 0] if dx else 1.0 - f[:, 0],
             f[:, 1] if dy else 1.0 - f[:, 1],
             f[:, 2] if dz else 1.0 - f[:, 2]]
        dw = [1.0 if dx else -1.0, 1.0 if dy else -1.0, 1.0 if dz else -1.0]
        v = mesh[(i0[:, 2] + dz) % nmesh, (i0[:, 1] + dy) % nmesh, (i0[:, 0] + dx) % nmesh]
        out[:, 0] += dw[0] * w[1] * w[2] * v
        out[:, 1] += w[0] * dw[1] * w[2] * v
        out[:, 2] += w[0] * w[1] * dw[2] * v
    return out * (nmesh / box)


def wavevectors(nmesh, box):
    """(kx, ky, kz) broadcastable to the rfftn half-spectrum shape (M, M, M/2+1)."""
    kf = 2.0 * np.pi / box
    n_full = np.fft.fftfreq(nmesh, d=1.0 / nmesh)       # 0..M/2-1, -M/2..-1
    n_half = np.arange(nmesh // 2 + 1, dtype=np.float64)  # 0..M/2
    kz = (kf * n_full)[:, None, None]
    ky = (kf * n_full)[None, :, None]
    kx = (kf * n_half)[None, None, :]
    return kx, ky, kz


def _odd_factor(kj, nmesh, box, axis_len_half=False):
    """i*k_j with the Nyquist plane of axis j zeroed."""
    kny = np.pi * nmesh / box
    return np.where(np.abs(np.abs(kj) - kny) < 1e-9 * kny, 0.0, kj) * 1j


def gradient_multipliers(nmesh, box):
    """i k_j / k^2 for j = x, y, z (Nyquist planes of axis j zeroed, k=0 -> 0)."""
    kx, ky, kz = wavevectors(nmesh, box)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0, 1.0 / k2, 0.0)
    return [_odd_factor(k, nmesh, box) * inv for k in (kx, ky, kz)]


def force_mesh(delta_real, box, omega_m):
    """Force meshes F_j = IDFT[(3/2) Om (i k_j / k^2) DFT(delta)], j = x, y, z.

    This is F = -(3/2) Om grad(phi) with lap(phi) = delta (Sec. 3 PM force);
    the mean of delta is irrelevant (k = 0 is dropped).
    """
    nmesh = delta_real.shape[0]
    dk = dft.rfftn(delta_real)
    return [dft.irfftn(1.5 * omega_m * m * dk, s=delta_real.shape, axes=(0, 1, 2))
            for m in gradient_multipliers(nmesh, box)]


def pgd_filter(nmesh, box, k_l, k_s, n_s):
    """O_L(k) O_S(k) = exp(-(k_l/k)^2) exp(-(k/k_s)^n) (PGD long/short filters)."""
    kx, ky, kz = wavevectors(nmesh, box)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k = np.sqrt(k2)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ol = np.where(k2 > 0, np.exp(-(k_l * k_l) / np.where(k2 > 0, k2, 1.0)), 0.0)
    os_ = np.exp(-(k / k_s) ** n_s)
    return ol * os_


def pgd_mesh(delta_real, box, alpha, k_l, k_s, n_s):
    """PGD displacement meshes S_j = IDFT[alpha O_L O_S (i k_j / k^2) DFT(delta)].

    Reading of the sharpening step (Sec. 3, PGD of Dai, Feng & Seljak): the
    displacement is alpha * (-grad) of the filtered potential, which moves
    particles towards density peaks; alpha = alpha0 a^mu, and the fifth
    parameter is the exponent n of the short-range filter.
    """
    nmesh = delta_real.shape[0]
    dk = dft.rfftn(delta_real)
    filt = pgd_filter(nmesh, box, k_l, k_s, n_s)
    return [dft.irfftn(alpha * filt * m * dk, s=delta_real.shape, axes=(0, 1, 2))
            for m in gradient_multipliers(nmesh, box)]


def particle_mass(nc, nmesh):
    """Mass per particle in units of the mean density per mesh cell: (M/Nc)^3."""
    return (nmesh / nc) ** 3


def density(pos, nc, nmesh, box):
    """CIC density rho (mean 1) of nc^3 equal-mass particles."""
    return cic_paint(pos, nmesh, box, particle_mass(nc, nmesh))


def pm_forces(pos, nc, nmesh, box, omega_m):
    """PM forces (N, 3) at the particles: paint, Poisson + gradient, readout."""
    rho = density(pos, nc, nmesh, box)
    fm = force_mesh(rho - 1.0, box, omega_m)
    return np.stack([cic_readout(m, pos, box) for m in fm], axis=1), fm, rho
