"""GPU source distributions n(z) (pm_set_source_nz) through the C ABI: maps,
reverse-mode and forward-mode derivatives against the FP64 oracle, with one of
two source planes replaced by a Gaussian n(z).  Tolerances as the plane-source
tests (maps 1e-6 / 1e-3, gradients 1e-6 / 2e-3, Omega_m at equal step 1e-6 /
5e-3); the q tables of the two sides come from different quadrature grids
(agreement ~1e-8)."""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle import jvp as ojvp
from oracle.sim import Simulation as OSim
from pm_inputs import white_noise, workload

pytestmark = pytest.mark.gpu


def gsim(precision=0, **w):
    from paper_2012_07266_gb300.api import Simulation
    return Simulation(device="cuda:0", precision=precision, **w)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _work(**over):
    base = dict(nc=32, nmesh=64, box=128.0, nsteps=6, map_npix=16, zs=(0.8, 1.0), lpt_order=2, pgd=1)
    base.update(over)
    w = workload("pm64", **base)
    z = np.linspace(0.5, 1.1, 61)
    w["source_nz"] = {1: (z, np.exp(-0.5 * ((z - 0.8) / 0.12) ** 2))}
    return w


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (0, 1e-3)])
def test_maps_with_distribution(cuda_lib, prec, tol):
    w = _work()
    noise = white_noise(w["nc"], 70)
    kappa = gsim(prec, **w).run(torch.from_numpy(noise)).cpu().numpy()
    ref = OSim(**w).run(noise)
    assert rel(kappa, ref) < tol
    # the distribution's map differs from the plane it replaced
    w_plane = dict(w)
    w_plane.pop("source_nz")
    plane = OSim(**w_plane).run(noise)
    assert rel(plane[1], ref[1]) > 1e-2


@pytest.mark.parametrize("prec,tol,tol_om", [(1, 1e-6, 1e-6), (0, 2e-3, 5e-3)])
def test_vjp_with_distribution(cuda_lib, prec, tol, tol_om):
    w = _work(ckpt_every=2)
    noise = white_noise(w["nc"], 71)
    lam = np.random.default_rng(72).standard_normal((2, w["map_npix"], w["map_npix"]))
    s = gsim(prec, **w)
    s.run(torch.from_numpy(noise))
    dn, (dom, ds8) = s.vjp(torch.from_numpy(lam))
    _, on, oom, os8 = oadj.vjp(OSim(**w), noise, lam, h_om=1e-3)
    assert rel(dn.cpu().numpy(), on) < tol
    assert abs(ds8 - os8) < tol * abs(os8)
    assert abs(dom - oom) < tol_om * abs(oom)


def test_jvp_with_distribution_fp64(cuda_lib):
    w = _work(jvp=1, ckpt_every=6)
    noise = white_noise(w["nc"], 73)
    rng = np.random.default_rng(74)
    d = rng.standard_normal(noise.shape)
    lam = rng.standard_normal((2, w["map_npix"], w["map_npix"]))
    s = gsim(1, **w)
    _, dk = s.jvp(torch.from_numpy(noise), torch.from_numpy(d))
    _, odk = ojvp.jvp(OSim(**w), noise, d)
    assert rel(dk.cpu().numpy(), odk) < 1e-6
    dn, _ = s.vjp(torch.from_numpy(lam))
    lhs, rhs = float(np.sum(lam * dk.cpu().numpy())), float(np.sum(dn.cpu().numpy() * d))
    assert abs(lhs - rhs) < 1e-8 * abs(rhs)


def test_set_source_nz_checks(cuda_lib):
    from paper_2012_07266_gb300 import lib
    w = _work()
    w.pop("source_nz")
    s = gsim(0, **w)
    for z, n in [([0.5, 0.4], [1.0, 1.0]),      # not ascending
                 ([0.0, 0.5], [1.0, 1.0]),      # z = 0
                 ([0.5, 20.0], [1.0, 1.0]),     # beyond the initial redshift
                 ([0.5, 0.6], [0.0, 0.0])]:     # no weight
        with pytest.raises(lib.PMError) as ei:
            s.set_source_nz(0, z, n)
        assert ei.value.status == 1  # PM_ERR_ARG
    noise = torch.from_numpy(white_noise(w["nc"], 75))
    s.ic(noise)
    s.step(0)
    s.lens_project(0)
    with pytest.raises(lib.PMError) as ei:
        s.set_source_nz(0, [0.5, 0.6], [1.0, 1.0])
    assert ei.value.status == 5  # PM_ERR_STATE
