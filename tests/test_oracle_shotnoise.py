"""Pins of the oracle's shot-noise runs and angular power spectrum (Sec. 4,
Fig. accuracy): the counter-based generator against the published SplitMix64
sequence, the uniform positions against their moments, the spectrum estimator
against Parseval's identity, a single Fourier mode and white noise, and the
maps of random-position runs against the closed-form Poisson variance and mean
of projected unclustered particles."""
import os

import numpy as np
from scipy.integrate import quad

from oracle.cosmology import C_OVER_H0
from oracle.lightcone import splitmix64
from oracle.shotnoise import angular_cl, shot_noise_maps, splitmix64_stream, uniform_positions
from oracle.sim import Simulation
from pm_inputs import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_stream_published_sequence():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and not l.startswith("#")]
    assert [int(v) for v in splitmix64_stream(0, 0, len(vals))] == vals
    gamma = 0x9E3779B97F4A7C15
    for seed in (1, 12345, 2 ** 63 + 7):
        out = splitmix64_stream(seed, 1000, 5)
        for k in range(5):
            assert int(out[k]) == splitmix64((seed + (1000 + k) * gamma) % 2 ** 64)


def test_uniform_positions_moments():
    nc, L = 32, 100.0
    x = uniform_positions(7, nc, L)
    n = x.shape[0]
    assert x.shape == (nc ** 3, 3) and x.min() >= 0.0 and x.max() < L
    r = x * 2.0 ** 24 / L
    assert np.all(r == np.round(r))                       # 24-bit grid
    assert np.all(np.abs(x.mean(0) - L / 2) < 4 * L / np.sqrt(12 * n))
    var_sd = L ** 2 * np.sqrt(1 / 80 - 1 / 144) / np.sqrt(n)   # sd of the sample variance
    assert np.all(np.abs(x.var(0) - L ** 2 / 12) < 4 * var_sd)
    h = np.stack([np.histogram(x[:, k], bins=16, range=(0, L))[0] for k in range(3)])
    chi2 = ((h - n / 16) ** 2 / (n / 16)).sum(1)
    assert np.all(chi2 < 45)                              # 15 dof, p ~ 1e-4
    assert np.abs(np.corrcoef(x.T)[np.triu_indices(3, 1)]).max() < 4 / np.sqrt(n)


def test_cl_parseval():
    rng = np.random.default_rng(3)
    n, fov = 32, 3.0
    maps = rng.standard_normal((2, n, n)) + 0.1
    cl, counts = angular_cl(maps, fov, [0.0, np.inf])
    omega_pix = np.deg2rad(fov / n) ** 2
    assert counts[0] == n * n
    assert np.allclose(cl[:, 0] / omega_pix, (maps ** 2).mean(axis=(1, 2)), rtol=1e-12, atol=0)


def test_cl_single_mode():
    n, fov, A = 64, 4.0, 0.7
    iy, ix = np.mgrid[0:n, 0:n]
    kappa = A * np.cos(2 * np.pi * (3 * ix + 5 * iy) / n)
    lscale = 2 * np.pi / np.deg2rad(fov)
    edges = lscale * np.array([0.0, 5.8, 5.9, 50.0])
    cl, counts = angular_cl(kappa, fov, edges)
    k2 = [mx * mx + my * my for mx in range(-n // 2, n // 2) for my in range(-n // 2, n // 2)]
    brute = [sum(1 for k in k2 if lo <= np.sqrt(k) < hi) for lo, hi in zip(edges[:-1] / lscale, edges[1:] / lscale)]
    assert list(counts) == brute and counts[1] == 8      # (+-3, +-5) and (+-5, +-3)
    omega_pix = np.deg2rad(fov / n) ** 2
    assert abs(cl[1] - 2 * omega_pix * (A * n * n / 2) ** 2 / n ** 2 / 8) < 1e-12 * cl[1]
    assert abs(cl[0]) < 1e-25 and abs(cl[2]) < 1e-25


def test_cl_white_noise_is_flat():
    rng = np.random.default_rng(4)
    n, fov, sig = 128, 5.0, 0.3
    maps = sig * rng.standard_normal((4, n, n))
    lscale = 2 * np.pi / np.deg2rad(fov)
    edges = lscale * np.array([1.0, 8.0, 16.0, 32.0, 45.0])
    cl, counts = angular_cl(maps, fov, edges)
    omega_pix = np.deg2rad(fov / n) ** 2
    # each mode's power is exponential about sig^2 Omega_pix; +-l pairs are equal
    err = sig ** 2 * omega_pix / np.sqrt(4 * counts / 2)
    assert np.all(np.abs(cl.mean(0) - sig ** 2 * omega_pix) < 4 * err)


def _random_run_sim():
    w = workload("pm64", nc=64, nmesh=64, box=128.0, nsteps=10, map_npix=64, map_fov_deg=2.0, zs=(1.0,))
    return Simulation(**w)


def _poisson_integrals(sim, chi_a, chi_b):
    """(4/9)-free pieces of the Poisson variance of projected unclustered
    particles: K^2 V_p / Omega_pix int q^2 / a^2 dchi and K int chi q / a dchi,
    with the mean flat-sky Jacobian (1 + theta^2)^(-3/2) over the pixel centres."""
    g = sim.geom
    c = sim.cosmo
    K = 1.5 * c.omega_m / C_OVER_H0 ** 2
    cs = g.chi_s[0]
    th = (np.arange(g.npix) + 0.5) * g.dtheta - 0.5 * g.fov
    J = float(np.mean((1 + th[:, None] ** 2 + th[None, :] ** 2) ** -1.5))
    vp, opix = g.vp, g.dtheta ** 2
    b = min(chi_b, cs)
    var = K ** 2 * vp / opix * J * quad(lambda x: ((cs - x) / cs / c.a_of_chi(x)) ** 2, chi_a, b,
                                        epsrel=1e-10)[0]
    mean = K * quad(lambda x: x * (cs - x) / cs / c.a_of_chi(x), 0.0, cs, epsrel=1e-10)[0]
    return var, mean, J, K


def test_shot_noise_pixel_variance_closed_form():
    """Pixel variance of random-position maps against the Poisson value
    (4/9) K^2 V_p/Omega_pix J int q^2/a^2 dchi (the 4/9 from the squared CIC tent
    integrated over a pixel), over the shells beyond 300 Mpc/h (the nearest
    particles' weights have a heavy tail that makes the full-range sample
    variance too noisy to pin)."""
    sim = _random_run_sim()
    g = sim.geom
    shells = [i for i in range(sim.nsteps) if g.shell(i)[0] >= 300.0]
    chi_a = g.shell(shells[-1])[0]
    chi_b = g.shell(shells[0])[1]
    var_th, _, _, _ = _poisson_integrals(sim, chi_a, chi_b)
    v = [shot_noise_maps(sim, seed, shells)[0].var() for seed in (11, 12, 13)]
    assert abs(np.mean(v) / (4.0 / 9.0 * var_th) - 1) < 0.06


def test_shot_noise_map_mean():
    """All shells: the map mean is the Poisson mean K int chi q J / a dchi minus
    the subtracted mean term, zero up to the flat-sky Jacobian, within four
    standard deviations K^2 V_p J / (Omega_pix N_pix) int q^2 / a^2 dchi."""
    sim = _random_run_sim()
    g = sim.geom
    var_th, mean_term, J, _ = _poisson_integrals(sim, 0.0, g.chi_s[0])
    sd = np.sqrt(var_th / g.npix ** 2)
    m = shot_noise_maps(sim, 21)[0].mean()
    assert abs(m - (J - 1) * mean_term) < 4 * sd
    # the mean term matters: without it the mean is off by many deviations
    assert mean_term > 20 * sd


def test_cl_against_direct_sum():
    """The estimator against its definition written out on a tiny map: kappa~(l) =
    Omega_pix sum_j kappa_j exp(-i l . theta_j) over the pixel-centre angles theta_j,
    C(l) = |kappa~(l)|^2 / Omega_map, at l = (2 pi / FOV) m; bins one |m| shell wide."""
    rng = np.random.default_rng(5)
    n, fov = 8, 1.5
    kappa = rng.standard_normal((n, n))
    fr = np.deg2rad(fov)
    dth = fr / n
    th = (np.arange(n) + 0.5) * dth - 0.5 * fr
    lscale = 2 * np.pi / fr
    k2s = sorted({mx * mx + my * my for mx in range(-n // 2, n // 2) for my in range(-n // 2, n // 2)})
    edges = [lscale * (np.sqrt(k) - 1e-9) for k in k2s] + [lscale * n]
    sums, cnt = np.zeros(len(k2s)), np.zeros(len(k2s))
    for mx in range(-n // 2, n // 2):
        for my in range(-n // 2, n // 2):
            acc = 0j
            for iy in range(n):
                for ix in range(n):
                    acc += kappa[iy, ix] * np.exp(-1j * lscale * (mx * th[ix] + my * th[iy]))
            c = abs(acc * dth * dth) ** 2 / fr ** 2
            b = k2s.index(mx * mx + my * my)
            sums[b] += c
            cnt[b] += 1
    cl, counts = angular_cl(kappa, fov, edges)
    assert list(counts) == list(cnt.astype(int))
    assert np.allclose(cl, sums / cnt, rtol=1e-11, atol=0)
