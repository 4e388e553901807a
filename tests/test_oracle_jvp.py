"""Pins of the oracle's forward-mode derivative (JVP): each tangent against
central finite differences of the forward operation it linearises, and the
whole pipeline against (i) the oracle's reverse-mode derivative through the
dot-product identity <lam, J d> = <J^T lam, d> and (ii) finite differences of
the whole forward model, along a random direction and along one noise pixel
(the paper's check of its Jacobian-vector product, Sec. 4.1 / Fig. 8)."""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import jvp as ojvp
from oracle import mesh
from oracle.lpt import lattice, linear_modes, lpt_displacements
from oracle.nbody import pgd_displacement
from oracle.sim import Simulation
from pm_inputs import white_noise, workload


def _pos(nc, M, L, seed, spread=2.0):
    rng = np.random.default_rng(seed)
    return np.mod(lattice(nc, L, M) + rng.normal(0, spread, size=(nc ** 3, 3)), L)


def test_paint_tangent_finite_difference():
    nc, M, L = 8, 16, 40.0
    rng = np.random.default_rng(30)
    x = _pos(nc, M, L, 31)
    d = rng.standard_normal(x.shape)
    t = ojvp.cic_paint_tangent(x, d, M, L, 2.0)
    eps = 1e-7
    fd = (mesh.cic_paint(x + eps * d, M, L, 2.0) - mesh.cic_paint(x - eps * d, M, L, 2.0)) / (2 * eps)
    assert np.linalg.norm(t - fd) < 1e-6 * np.linalg.norm(fd)


def test_force_and_pgd_tangent_finite_difference():
    nc, M, L, om = 8, 16, 40.0, 0.3
    params = (0.05, -0.3, 0.3, 1.5, 4.0)
    rng = np.random.default_rng(32)
    x = _pos(nc, M, L, 33)
    d = rng.standard_normal(x.shape)
    eps = 1e-6
    t = ojvp.force_tangent(x, d, nc, M, L, om)
    fd = (mesh.pm_forces(x + eps * d, nc, M, L, om)[0] - mesh.pm_forces(x - eps * d, nc, M, L, om)[0]) / (2 * eps)
    assert np.linalg.norm(t - fd) < 1e-6 * np.linalg.norm(fd)
    t = ojvp.pgd_tangent(x, d, 0.7, nc, M, L, params)
    fd = (pgd_displacement(x + eps * d, 0.7, nc, M, L, params)
          - pgd_displacement(x - eps * d, 0.7, nc, M, L, params)) / (2 * eps)
    assert np.linalg.norm(t - fd) < 1e-6 * np.linalg.norm(fd)


def test_lpt_tangent_finite_difference():
    w = workload("pm64", nc=16, nmesh=16, box=128.0)
    sim = Simulation(**w)
    rng = np.random.default_rng(34)
    w0 = white_noise(16, 35)
    d = rng.standard_normal(w0.shape)
    c, L = sim.cosmo, sim.box
    dk, ddk = linear_modes(w0, c, L), linear_modes(d, c, L)
    t1, t2 = ojvp.lpt_tangent(dk, ddk, 16, L, 2)
    eps = 1e-4    # Psi2 is quadratic: the central difference is exact up to rounding
    p1p, p2p = lpt_displacements(linear_modes(w0 + eps * d, c, L), 16, L, 2)
    p1m, p2m = lpt_displacements(linear_modes(w0 - eps * d, c, L), 16, L, 2)
    assert np.linalg.norm(t1 - (p1p - p1m) / (2 * eps)) < 1e-9 * np.linalg.norm(t1)
    assert np.linalg.norm(t2 - (p2p - p2m) / (2 * eps)) < 1e-8 * np.linalg.norm(t2)


@pytest.mark.parametrize("sub,pgd", [(1, 0), (1, 1), (0, 0)])
def test_projection_tangent_finite_difference(sub, pgd):
    w = workload("pm64", nc=16, nmesh=16, box=128.0, nsteps=10, map_npix=24, zs=(0.7, 1.0),
                 sub_evolution=sub, pgd=pgd, rotate=1)
    sim = Simulation(**w)
    sim.ic(white_noise(16, 36))
    i = 6
    for j in range(i + 1):
        sim.step(j)
    x, p = sim.state.x, sim.state.p
    S = sim.pgd_at(i)
    rng = np.random.default_rng(37)
    dx, dp = rng.standard_normal(x.shape), rng.standard_normal(p.shape)
    dS = rng.standard_normal(x.shape) if S is not None else None
    t = ojvp.project_tangent(sim.geom, i, x, p, S, dx, dp, dS)
    eps = 1e-7
    # the margin (replica candidates) is held at the central state, as the selection is
    geom = sim.geom
    mp = geom.project(i, np.mod(x + eps * dx, geom.box), p + eps * dp,
                      None if S is None else S + eps * dS)[0]
    mm = geom.project(i, np.mod(x - eps * dx, geom.box), p - eps * dp,
                      None if S is None else S - eps * dS)[0]
    fd = (mp - mm) / (2 * eps)
    assert np.linalg.norm(t - fd) < 1e-5 * np.linalg.norm(fd)


def _pipeline(**over):
    base = dict(nc=16, nmesh=32, box=128.0, nsteps=6, map_npix=16, zs=(1.0,))
    base.update(over)
    return workload("pm64", **base)


@pytest.mark.parametrize("over", [dict(lpt_order=1), dict(lpt_order=2, pgd=1, zs=(0.8, 1.0))])
def test_pipeline_jvp_dot_product_with_vjp(over):
    """<lam, J d> from the tangent-linear model equals <J^T lam, d> from the
    independent reverse sweep (both FP64, same trajectory)."""
    w = _pipeline(**over)
    noise = white_noise(16, 40)
    rng = np.random.default_rng(41)
    d = rng.standard_normal(noise.shape)
    lam = rng.standard_normal((len(w["zs"]), 16, 16))
    kappa, dk = ojvp.jvp(Simulation(**w), noise, d)
    _, g, _, _ = adj.vjp(Simulation(**w), noise, lam)
    lhs, rhs = float(np.sum(lam * dk)), float(np.sum(g * d))
    assert abs(lhs - rhs) < 1e-9 * abs(rhs)
    assert np.allclose(kappa, Simulation(**w).run(noise), rtol=0, atol=1e-14)


@pytest.mark.parametrize("pixel", [False, True])
def test_pipeline_jvp_finite_difference(pixel):
    """J d against central differences of the whole forward model, along a random
    direction and along a single noise pixel (the paper's check, Fig. 8)."""
    w = _pipeline(lpt_order=2, pgd=1)
    noise = white_noise(16, 42)
    rng = np.random.default_rng(43)
    if pixel:
        d = np.zeros_like(noise)
        d[5, 7, 9] = 1.0
    else:
        d = rng.standard_normal(noise.shape)
    _, dk = ojvp.jvp(Simulation(**w), noise, d)
    eps = 1e-6
    fd = (Simulation(**w).run(noise + eps * d) - Simulation(**w).run(noise - eps * d)) / (2 * eps)
    assert np.linalg.norm(dk - fd) < 1e-5 * np.linalg.norm(fd)
