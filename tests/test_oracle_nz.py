"""Pins of the oracle's general source distribution n(z) (Eq. conv with a
distribution of source distances): the lensing efficiency q(chi) against its
closed form for sources uniform in comoving distance, the plane-source limit
of a narrow distribution, the mean-density term against the closed form, and
the reverse and forward derivatives of a pipeline with a distribution against
finite differences and against each other (dot-product identity)."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import adjoint as adj
from oracle import jvp as ojvp
from oracle.sim import Simulation
from pm_inputs import white_noise, workload


def _geom(**over):
    w = workload("pm64", nc=16, nmesh=32, box=128.0, nsteps=6, map_npix=16, zs=(1.0,), **over)
    return Simulation(**w)


def _uniform_in_chi(cosmo, za, zb, npts=2001):
    """n(z) proportional to dchi/dz on [za, zb]: uniform in comoving distance."""
    z = np.linspace(za, zb, npts)
    return z, 1.0 / cosmo.E(1.0 / (1.0 + z))


def test_q_closed_form_uniform_in_chi():
    sim = _geom()
    c = sim.cosmo
    za, zb = 0.6, 1.2
    z, n = _uniform_in_chi(c, za, zb)
    sim.geom.set_source_nz(0, z, n)
    ca, cb = float(c.chi_z(za)), float(c.chi_z(zb))
    chi = np.array([50.0, 0.5 * ca, ca, 0.5 * (ca + cb), 0.9 * cb])
    m = np.maximum(chi, ca)
    q_exact = ((cb - m) - chi * np.log(cb / m)) / (cb - ca)
    dq_exact = -np.log(cb / m) / (cb - ca)
    q, dq = sim.geom.source_weight(0, chi)
    assert np.allclose(q, q_exact, rtol=2e-6, atol=0)
    assert np.allclose(dq, dq_exact, rtol=2e-6, atol=0)
    q_far, _ = sim.geom.source_weight(0, np.array([cb * 1.01]))
    assert q_far[0] == 0.0


def test_narrow_distribution_is_the_plane():
    sim = _geom()
    c = sim.cosmo
    zs = 1.0
    z = np.linspace(zs - 5e-3, zs + 5e-3, 201)
    n = np.exp(-0.5 * ((z - zs) / 1e-3) ** 2)
    sim.geom.set_source_nz(0, z, n)
    cs = float(c.chi_z(zs))
    chi = np.linspace(10.0, 0.95 * cs, 7)
    q, _ = sim.geom.source_weight(0, chi)
    # q = 1 - chi <1/chi'>: the 1e-3 width shifts <1/chi'> at second order (~3e-7 relative)
    assert np.allclose(q, (cs - chi) / cs, rtol=0, atol=2e-6)


def test_mean_term_uniform_in_chi():
    sim = _geom()
    c = sim.cosmo
    za, zb = 0.6, 1.2
    z, n = _uniform_in_chi(c, za, zb)
    sim.geom.set_source_nz(0, z, n)
    ca, cb = float(c.chi_z(za)), float(c.chi_z(zb))

    def q(x):
        m = max(x, ca)
        return ((cb - m) - x * np.log(cb / m)) / (cb - ca)
    exact = 1.5 * c.omega_m / (299792.458 / 100.0) ** 2 * quad(
        lambda x: x * q(x) / c.a_of_chi(x), 0.0, cb, points=[ca], limit=500, epsrel=1e-12)[0]
    assert abs(sim.geom.mean_term()[0] - exact) < 2e-6 * abs(exact)


def _nz_work(**over):
    base = dict(nc=16, nmesh=32, box=128.0, nsteps=6, map_npix=16, zs=(0.8, 1.0), lpt_order=2, pgd=1)
    base.update(over)
    w = workload("pm64", **base)
    z = np.linspace(0.5, 1.1, 61)
    w["source_nz"] = {1: (z, np.exp(-0.5 * ((z - 0.8) / 0.12) ** 2))}
    return w


def test_pipeline_with_distribution_vjp_and_jvp():
    """Reverse mode against central differences, and forward mode against the
    reverse mode (dot-product identity), with one source plane replaced by n(z)."""
    w = _nz_work()
    noise = white_noise(16, 60)
    rng = np.random.default_rng(61)
    lam = rng.standard_normal((2, 16, 16))
    d = rng.standard_normal(noise.shape)
    _, g, _, _ = adj.vjp(Simulation(**w), noise, lam)
    eps = 1e-6

    def loss(nz):
        return float(np.sum(lam * Simulation(**w).run(nz)))
    fd = (loss(noise + eps * d) - loss(noise - eps * d)) / (2 * eps)
    assert abs(np.sum(g * d) - fd) < 1e-5 * abs(fd)
    _, dk = ojvp.jvp(Simulation(**w), noise, d)
    assert abs(np.sum(lam * dk) - np.sum(g * d)) < 1e-9 * abs(np.sum(g * d))


@pytest.mark.parametrize("h", [1e-8])
def test_pipeline_with_distribution_omega_m(h):
    """d/d Omega_m with a distribution: the coefficient finite differences of the
    reverse sweep against the whole-model difference at a step small enough that
    no particle changes shell (in this two-source configuration h = 1e-6 already
    moves particles across shell boundaries; from 1e-7 down the difference is
    smooth and converged)."""
    w = _nz_work(lpt_order=1, pgd=0)
    noise = white_noise(16, 62)
    lam = np.random.default_rng(63).standard_normal((2, 16, 16))
    _, _, dom, _ = adj.vjp(Simulation(**w), noise, lam, h_om=1e-4)
    wp, wm = dict(w), dict(w)
    wp["omega_m"] += h
    wm["omega_m"] -= h
    fd = (float(np.sum(lam * Simulation(**wp).run(noise))) - float(np.sum(lam * Simulation(**wm).run(noise)))) / (2 * h)
    assert abs(dom - fd) < 1e-2 * abs(fd)
