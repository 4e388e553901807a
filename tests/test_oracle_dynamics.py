"""Pins of the oracle's initial conditions and kick-drift-kick stepping."""
import numpy as np
import pytest

from oracle import mesh
from oracle.cosmology import Cosmology
from oracle.lpt import lattice, linear_modes, lpt_displacements, lpt_state
from oracle.sim import Simulation
from pm_inputs import white_noise, workload


def _field_from_real(f):
    return np.fft.rfftn(f)


def test_lpt_single_plane_wave():
    """One plane wave: Psi1 closed form and Psi2 = 0 (2LPT source vanishes)."""
    nc, L, A = 16, 80.0, 0.3
    k = 2 * np.pi * np.array([1.0, 2.0, 0.0]) / L
    g = np.arange(nc) * L / nc
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z
    delta = -A * np.cos(ph)
    psi1, psi2 = lpt_displacements(_field_from_real(delta), nc, L, order=2)
    k2 = np.sum(k * k)
    for j in range(3):
        # div Psi1 = -delta = A cos(k.x)  =>  Psi1 = A k sin(k.x) / k^2
        assert np.allclose(psi1[:, j], (A * k[j] / k2 * np.sin(ph)).ravel(), atol=1e-12)
    assert np.allclose(psi2, 0.0, atol=1e-12)


def test_2lpt_two_orthogonal_waves_closed_form():
    """Psi1 = (A sin(k1 x)/k1, B sin(k2 y)/k2, 0) gives
    Psi2 = AB (k1 sin(k1x)cos(k2y), k2 cos(k1x) sin(k2y), 0) / (k1^2 + k2^2)."""
    nc, L, A, B = 16, 64.0, 0.2, 0.35
    k1, k2 = 2 * np.pi * 1 / L, 2 * np.pi * 3 / L
    g = np.arange(nc) * L / nc
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    delta = -(A * np.cos(k1 * x) + B * np.cos(k2 * y))   # = -div Psi1
    psi1, psi2 = lpt_displacements(_field_from_real(delta), nc, L, order=2)
    assert np.allclose(psi1[:, 0], (A * np.sin(k1 * x) / k1).ravel(), atol=1e-12)
    assert np.allclose(psi1[:, 1], (B * np.sin(k2 * y) / k2).ravel(), atol=1e-12)
    den = k1 * k1 + k2 * k2
    assert np.allclose(psi2[:, 0], (A * B * k1 * np.sin(k1 * x) * np.cos(k2 * y) / den).ravel(), atol=1e-12)
    assert np.allclose(psi2[:, 1], (A * B * k2 * np.cos(k1 * x) * np.sin(k2 * y) / den).ravel(), atol=1e-12)
    assert np.allclose(psi2[:, 2], 0.0, atol=1e-12)


def test_linear_modes_power_normalisation():
    """<|delta_L(k)|^2> = Nc^6 P(k) / V for the DFT convention (shell average)."""
    nc, L = 32, 200.0
    c = Cosmology()
    dk = linear_modes(white_noise(nc, 11), c, L)
    kx, ky, kz = mesh.wavevectors(nc, L)
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2) * np.ones(dk.shape)
    sel = (k > 0.1) & (k < 0.3)
    ratio = np.abs(dk[sel]) ** 2 / (nc ** 6 * c.pk_lin(k[sel]) / L ** 3)
    assert abs(ratio.mean() - 1.0) < 0.05   # ~ 1/sqrt(#modes)
    assert dk[0, 0, 0] == 0


def _za_run(nc, nmesh, A, nsteps=10):
    w = workload("pm64", nc=nc, nmesh=nmesh, nsteps=nsteps, map_npix=8)
    sim = Simulation(**w)
    L = sim.box
    k = 2 * np.pi / L
    q = lattice(nc, L, nmesh)
    psi = np.zeros_like(q)
    psi[:, 0] = A / k * np.sin(k * q[:, 0])
    c, a0 = sim.cosmo, sim.stepper.a[0]
    sim.set_state(q + c.D1(a0) * psi, c.gp(a0) * psi)
    for i in range(sim.nsteps):
        sim.step(i)
    xe = q + c.D1(1.0) * psi
    d = (sim.state.x - xe + L / 2) % L - L / 2
    return np.abs(d).max() / np.abs(psi).max()


def test_zeldovich_sinusoid_before_shell_crossing():
    """A 1D sinusoidal mode (D1 A = 0.5 at a = 1, before shell crossing) follows
    x = q + D1(a) Psi exactly in the continuum; the PM error must converge with M."""
    e32 = _za_run(32, 32, 0.5)
    e64 = _za_run(64, 64, 0.5)
    assert e64 < 0.02 and e64 < 0.6 * e32


def test_kdk_exact_linear_growth_small_mode():
    """Tiny amplitude: the FastPM factors reproduce D1 growth to the PM force
    accuracy (~CIC window, second order in k Delta)."""
    e32 = _za_run(32, 32, 1e-3)
    e64 = _za_run(64, 64, 1e-3)
    assert e64 < 2.5e-3 and e64 < 0.35 * e32


def _growth_deviation(nc, L=256.0, kmax=0.1 * np.pi * 32 / 256.0):
    w = workload("pm64", nc=nc, nmesh=nc, box=L, nsteps=10, a_init=0.05, map_npix=8)
    sim = Simulation(**w)
    sim.ic(1e-3 * white_noise(nc, 5))   # scaled: linear regime
    d0 = np.fft.rfftn(mesh.density(sim.state.x, nc, nc, L) - 1)
    for i in range(4):
        sim.step(i)
    d1 = np.fft.rfftn(mesh.density(sim.state.x, nc, nc, L) - 1)
    c = sim.cosmo
    g = c.D1(sim.stepper.a[4]) / c.D1(sim.stepper.a[0])
    kx, ky, kz = mesh.wavevectors(nc, L)
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2) * np.ones(d0.shape)
    sel = (k > 0) & (k < kmax)
    ratio = np.abs(d1[sel]) ** 2 / np.abs(d0[sel]) ** 2 / g ** 2
    return np.abs(ratio - 1).max(), sel.sum()


def test_linear_growth_of_modes_early_steps():
    """Low-k density modes grow as D1(a)/D1(a0): P(k, a)/P(k, a0) = [D1(a)/D1(a0)]^2
    mode by mode, up to the PM force error that is second order in k Delta
    (halving Delta must cut the deviation by about 4)."""
    dev32, n32 = _growth_deviation(32)
    dev64, n64 = _growth_deviation(64)
    assert n32 == n64 and n32 > 5
    assert dev32 < 0.04 and dev64 < 0.01 and dev64 < 0.35 * dev32


def test_ic_state_wraps_and_momentum():
    w = workload("pm64", nc=16, nmesh=32, map_npix=8, lpt_order=2)
    sim = Simulation(**w)
    psi1, psi2 = sim.ic(white_noise(16, 3))
    x, p = sim.state.x, sim.state.p
    assert np.all((x >= 0) & (x < sim.box))
    c, a0 = sim.cosmo, sim.stepper.a[0]
    assert np.allclose(p, c.gp(a0) * psi1 + c.gp2(a0) * psi2)
    assert np.allclose(psi1.mean(axis=0), 0, atol=1e-12)
