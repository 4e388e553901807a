"""Pins of the oracle's lightcone projection (Eq. conv, Sec. 3)."""
import os

import numpy as np

from oracle.cosmology import Cosmology
from oracle.lightcone import (LensGeometry, apply_rotation, apply_transform, replica_transform,
                              splitmix64)
from oracle.lpt import lattice
from oracle.nbody import Stepper
from oracle.sim import Simulation
from pm_inputs import white_noise, workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_sequence():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and not l.startswith("#")]
    state, out = 0, []
    for _ in vals:
        out.append(splitmix64(state))
        state = (state + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
    assert out == vals


def test_replica_transform_is_torus_isometry():
    rng = np.random.default_rng(0)
    L, M = 100.0, 50
    x = rng.uniform(0, L, size=(200, 3))
    seen_perm, seen_flip = set(), set()
    for n in [(i, j, k) for i in (-2, 0, 1) for j in (-1, 0, 3) for k in range(12)]:
        tr = replica_transform(n, 42, True, M)
        seen_perm.add(tr[0])
        seen_flip.add(tr[1])
        y = apply_transform(x, tr, L, M)
        assert np.all((y >= 0) & (y < L))
        for a, b in [(0, 1), (5, 17), (33, 150)]:
            d0 = (x[a] - x[b] + L / 2) % L - L / 2
            d1 = (y[a] - y[b] + L / 2) % L - L / 2
            assert np.isclose(np.linalg.norm(d0), np.linalg.norm(d1))
            # the separation vector itself rotates like a momentum
            assert np.allclose(apply_rotation(d0[None], tr)[0], d1, atol=1e-9)
    assert len(seen_perm) == 6 and len(seen_flip) >= 6
    assert replica_transform((3, 1, 2), 42, False, M) == ((0, 1, 2), (0, 0, 0), (0, 0, 0))


def _geometry(nc=32, nmesh=32, box=128.0, nsteps=10, npix=32, fov=2.0, sub=True, rotate=False):
    c = Cosmology()
    st = Stepper(c, 0.1, nsteps)
    return LensGeometry(c, st, [1.0], npix, fov, box, nc, nmesh, rotate=rotate,
                        sub_evolution=sub), c, st


def test_single_particle_on_axis_splits_over_four_centre_pixels():
    """theta = 0 lies on the corner shared by the four central pixels, which
    share every on-axis copy of the particle equally (angle convention)."""
    g, c, st = _geometry(sub=False)
    i = 7
    lo, hi = g.shell(i)
    chi = 0.5 * (lo + hi)
    box = g.box
    nz = int(chi // box)
    x = np.array([[0.0, 0.0, chi - nz * box]])
    maps, hits = g.project(i, x, np.zeros((1, 3)))
    assert hits >= 1        # other replicas of the particle may share the shell
    m = maps[0]
    n = g.npix
    assert np.isclose(m[n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1].sum(), m.sum(), rtol=1e-14)
    assert np.allclose(m[n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1], m.sum() / 4)
    assert m.sum() > 0


def test_uniform_lattice_matches_born_integral():
    """A uniform particle lattice (delta = 0) projected through every shell
    reproduces the continuum Born integral of the mean density (the term that
    is subtracted), so the map mean of kappa vanishes: pins the weight
    (3/2) Om (H0/c)^2 (chi_s - chi)/(chi_s chi a) V_p / Omega_pix against Eq. conv."""
    nc, box = 64, 128.0
    g, c, st = _geometry(nc=nc, nmesh=nc, box=box, nsteps=10, npix=16, fov=2.0, sub=False)
    x = lattice(nc, box, nc)
    p = np.zeros_like(x)
    maps = np.zeros((1, g.npix, g.npix))
    for i in range(st.nsteps):
        maps += g.project(i, x, p)[0]
    mean = g.mean_term()[0]
    assert abs(maps.mean() / mean - 1.0) < 5e-3


def _lowpass_noise(nc, seed, frac=0.1, amp=1e-3):
    w = np.fft.rfftn(white_noise(nc, seed))
    n = np.fft.fftfreq(nc, 1.0 / nc)
    nz, ny, nx = np.meshgrid(n, n, np.arange(nc // 2 + 1), indexing="ij")
    w[np.sqrt(nx ** 2 + ny ** 2 + nz ** 2) > frac * nc / 2] = 0
    return amp * np.fft.irfftn(w, s=(nc, nc, nc), axes=(0, 1, 2))


def test_subevolution_of_linear_state_is_zeldovich_at_crossing_time():
    """In the linear regime, moving x(a_{i+1}) with p(a_{i+1/2}) by the
    sub-evolution factor lands on q + D1(a_c) Psi1 for any a_c in the step
    (long-wavelength field, where the PM force is linear theory to ~1%), and
    on x(a_i) exactly for a_c = a_i (the drift trajectory of the step)."""
    w = workload("pm64", nc=32, nmesh=32, nsteps=10, map_npix=8)
    sim = Simulation(**w)
    psi1, _ = sim.ic(_lowpass_noise(32, 9))
    i = 5
    for j in range(i):
        sim.step(j)
    x_prev = sim.state.x.copy()
    sim.step(i)
    q = lattice(32, sim.box, 32)
    for a_c in (sim.stepper.a[i] + 1e-3, sim.stepper.ah[i], sim.stepper.a[i + 1]):
        dt = sim.geom.subevolve_factor(i, a_c)
        xc = sim.state.x + sim.state.p * dt
        expect = q + sim.cosmo.D1(a_c) * psi1
        d = (xc - expect + sim.box / 2) % sim.box - sim.box / 2
        assert np.abs(d).max() < 0.015 * np.abs(sim.cosmo.D1(a_c) * psi1).max()
    dt = sim.geom.subevolve_factor(i, sim.stepper.a[i])
    d = (sim.state.x + sim.state.p * dt - x_prev + sim.box / 2) % sim.box - sim.box / 2
    assert np.abs(d).max() < 1e-12


def test_shells_tile_the_lightcone():
    g, c, st = _geometry(nsteps=10)
    edges = [g.shell(i) for i in range(st.nsteps)]
    for (lo0, hi0), (lo1, hi1) in zip(edges[:-1], edges[1:]):
        assert lo0 == hi1 and lo0 > lo1
    assert edges[-1][0] == 0.0 or abs(edges[-1][0]) < 1e-9
    assert edges[0][1] > g.chi_s.max()


def test_end_to_end_small_run_statistics():
    """Whole forward model at 32^3: kappa has ~zero mean (mean term cancels the
    particle sum) and a positive skewness (non-Gaussian tail, Fig. hist)."""
    w = workload("pm64", nc=32, nmesh=64, map_npix=32)
    sim = Simulation(**w)
    kappa = sim.run(white_noise(32, 1))
    assert np.all(np.isfinite(kappa))
    assert abs(kappa.mean()) < 0.1 * kappa.std()
    k = kappa.ravel() - kappa.mean()
    assert np.mean(k ** 3) > 0
