"""Shot-noise runs and the flat-sky angular power spectrum in FP64
(TEST INFRASTRUCTURE ONLY).

Sec. 4 (Fig. accuracy): the shot noise of the convergence maps, which comes from
sampling the matter field with a finite number of particles, is estimated by
projecting particles at uniformly random positions through the same lightcone
and averaging the power spectra of those maps over several such runs; the
average is subtracted from the simulated spectrum.

Readings (the paper gives no details of the random runs): one run draws the
Nc^3 particle positions i.i.d. uniform in the box, with zero momentum and
without PGD, and projects every shell exactly as a simulation's state would be
projected (same replicas, rotations, source planes or distributions, mean-term
subtraction).  Coordinate k of particle j is output 3j + k of the SplitMix64
sequence seeded with the run's seed, its top 24 bits r giving x = L r / 2^24.

The spectrum of a map on n x n pixels of a field of view FOV (flat sky):
    kappa~(l) = Omega_pix sum_j kappa_j exp(-i l . theta_j),
    C(l) = |kappa~(l)|^2 / Omega_map = Omega_pix |DFT(kappa)(m)|^2 / n^2,
at l = (2 pi / FOV) m, m = (m_x, m_y) on the DFT grid (-n/2 .. n/2 - 1 per
axis), averaged over the modes of each bin edges[b] <= |l| < edges[b+1].
|l| is (2 pi / FOV_rad) sqrt(m_x^2 + m_y^2) with FOV_rad = FOV_deg (pi / 180),
evaluated in that order in IEEE double, so that a mode on a bin edge falls in
the same bin on every implementation that follows the same order.
"""
from __future__ import annotations

import numpy as np

from . import dft
GAMMA = np.uint64(0x9E3779B97F4A7C15)


def splitmix64_stream(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 seeded with `seed` (Steele,
    Lea & Flood 2014): output n mixes the state seed + (n + 1) gamma mod 2^64."""
    with np.errstate(over="ignore"):
        n = np.arange(start, start + count, dtype=np.uint64)
        z = np.uint64(seed) + (n + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform_positions(seed: int, nc: int, box: float) -> np.ndarray:
    """(Nc^3, 3) positions uniform in [0, L)^3, particle j's coordinate k from
    output 3j + k: x = L r / 2^24 with r the output's top 24 bits."""
    npart = nc ** 3
    r = (splitmix64_stream(seed, 0, 3 * npart) >> np.uint64(40)).astype(np.float64)
    return (box * (r / 2.0 ** 24)).reshape(npart, 3)


def shot_noise_maps(sim, seed: int, shells=None) -> np.ndarray:
    """Convergence maps (n_zs, npix, npix) of one random-position run through the
    lightcone of `sim` (an oracle Simulation, whose geometry and sources are
    used; its particle state is not touched).  `shells` restricts the projection
    to the given shells (default: all), for tests of the noise's distance
    dependence; the mean term is always subtracted."""
    geom = sim.geom
    x = uniform_positions(seed, sim.nc, sim.box)
    p = np.zeros_like(x)
    maps = np.zeros((len(geom.zs), geom.npix, geom.npix))
    for i in range(sim.nsteps) if shells is None else shells:
        if geom.active(i):
            maps += geom.project(i, x, p, None)[0]
    return maps - geom.mean_term()[:, None, None]


def multipole_of_modes(n: int, fov_deg: float) -> np.ndarray:
    """|l| of every DFT mode of an n x n map, [my, mx] as numpy's fft2 orders them."""
    m = np.fft.fftfreq(n, d=1.0 / n)                    # 0, 1, .., n/2 - 1, -n/2, .., -1
    k2 = m[:, None] ** 2 + m[None, :] ** 2
    fov_rad = fov_deg * (np.pi / 180.0)
    return (2.0 * np.pi / fov_rad) * np.sqrt(k2)


def angular_cl(maps, fov_deg: float, edges):
    """Binned flat-sky C(l) of maps (..., n, n): returns (cl (..., nbins), counts
    (nbins,)); an empty bin reads 0."""
    maps = np.asarray(maps, dtype=np.float64)
    edges = np.asarray(edges, dtype=np.float64)
    n = maps.shape[-1]
    fov_rad = fov_deg * (np.pi / 180.0)
    omega_pix = (fov_rad / n) ** 2
    power = omega_pix * np.abs(dft.fft2(maps)) ** 2 / n ** 2
    ell = multipole_of_modes(n, fov_deg)
    nb = len(edges) - 1
    cl = np.zeros(maps.shape[:-2] + (nb,))
    counts = np.zeros(nb, dtype=np.int64)
    for b in range(nb):
        sel = (ell >= edges[b]) & (ell < edges[b + 1])
        counts[b] = int(sel.sum())
        if counts[b]:
            cl[..., b] = power[..., sel].mean(axis=-1)
    return cl, counts


def shot_noise_cl(sim, edges, seeds):
    """Average C(l) of the random-position runs with the given seeds (Sec. 4)."""
    acc = None
    for s in seeds:
        cl, _ = angular_cl(shot_noise_maps(sim, s), sim.geom.fov_deg, edges)
        acc = cl if acc is None else acc + cl
    return acc / len(seeds)
