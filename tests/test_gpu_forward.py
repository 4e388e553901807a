"""GPU parity of the forward path against the FP64 oracle, through the C ABI.

Tolerances: FFT relative L2 1e-6 (FP32) / 1e-12 (FP64); CIC density and
single-step forces relative L2 <= 1e-5; positions after a run within 1e-3 of a
mesh cell RMS; kappa maps relative L2 <= 1e-3 per map and power-spectrum
bins within 0.1%.
"""
import numpy as np
import pytest
import torch

from oracle import mesh as omesh
from oracle.lpt import lattice
from oracle.nbody import pgd_displacement
from oracle.sim import Simulation as OSim
from pm_inputs import white_noise, workload

pytestmark = pytest.mark.gpu


def gsim(precision=0, **w):
    from paper_2012_07266_gb300.api import Simulation
    return Simulation(device="cuda:0", precision=precision, **w)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def periodic_diff(a, b, L):
    return (np.asarray(a) - np.asarray(b) + L / 2) % L - L / 2


@pytest.mark.parametrize("M,prec,tol", [(64, 0, 1e-6), (96, 0, 1e-6), (32, 1, 1e-12), (192, 0, 1e-6)])
def test_fft_r2c_vs_numpy(cuda_lib, M, prec, tol):
    w = workload("pm64", nc=32, nmesh=M, map_npix=8)
    s = gsim(prec, **w)
    rng = np.random.default_rng(M)
    f = rng.standard_normal((M, M, M))
    g = s.fft_r2c(torch.from_numpy(f)).cpu().numpy()
    ref = np.fft.rfftn(f)
    assert rel(g, ref) < tol


@pytest.mark.parametrize("nc,M,prec", [(32, 64, 0), (32, 96, 0), (32, 32, 1)])
def test_density_and_forces_vs_oracle(cuda_lib, nc, M, prec):
    """Random particle positions: CIC density and PM forces (paint, r2c,
    Poisson + gradient, c2r, readout) against the oracle, relative L2 <= 1e-5."""
    w = workload("pm64", nc=nc, nmesh=M, box=100.0, map_npix=8)
    s = gsim(prec, **w)
    rng = np.random.default_rng(nc + M)
    q = lattice(nc, w["box"], M)
    x = np.mod(q + rng.normal(0, 3.0, size=q.shape), w["box"])
    p = rng.normal(0, 1.0, size=q.shape)
    s.set_particles(torch.from_numpy(x), torch.from_numpy(p), 0)
    rho = s.density().cpu().numpy()
    ref_rho = omesh.density(x, nc, M, w["box"])
    assert rel(rho, ref_rho) < 1e-6
    assert abs(rho.sum() / M ** 3 - 1.0) < 1e-6
    f = s.forces().cpu().numpy()
    ref_f, _, _ = omesh.pm_forces(x, nc, M, w["box"], w["omega_m"])
    assert rel(f, ref_f) < 1e-5
    gx, gp = s.particles()
    assert np.abs(periodic_diff(gx.cpu().numpy(), x, w["box"])).max() < 1e-5 * w["box"] / M
    assert rel(gp.cpu().numpy(), p) < 1e-6


@pytest.mark.parametrize("order", [1, 2])
def test_ic_vs_oracle(cuda_lib, order):
    nc, M = 32, 64
    w = workload("pm64", nc=nc, nmesh=M, lpt_order=order, map_npix=8)
    noise = white_noise(nc, 3)
    s = gsim(0, **w)
    s.ic(torch.from_numpy(noise))
    x, p = [t.cpu().numpy() for t in s.particles()]
    o = OSim(**w)
    o.ic(noise)
    cell = w["box"] / M
    dx = periodic_diff(x, o.state.x, w["box"]) / cell
    assert np.sqrt(np.mean(dx ** 2)) < 1e-5
    assert rel(p, o.state.p) < 1e-5
    assert rel(s.forces().cpu().numpy(), o.state.force) < 1e-5


def test_pgd_vs_oracle(cuda_lib):
    nc, M = 32, 64
    w = workload("pm64", nc=nc, nmesh=M, pgd=1, map_npix=8)
    noise = white_noise(nc, 4)
    o = OSim(**w)
    o.ic(noise)
    for i in range(7):
        o.step(i)
    s = gsim(0, **w)
    s.set_particles(torch.from_numpy(o.state.x), torch.from_numpy(o.state.p), 7)
    S = s.pgd().cpu().numpy()
    ref = pgd_displacement(o.state.x, o.stepper.a[7], nc, M, w["box"], w["pgd_params"])
    assert rel(S, ref) < 1e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_run_positions_and_kappa_vs_oracle(cuda_lib, prec):
    """Whole forward run (1LPT, 10 steps, sub-evolution, rotated replicas):
    final positions within 1e-3 cell RMS and kappa within 1e-3 relative L2."""
    nc, M = 32, 64
    w = workload("pm64", nc=nc, nmesh=M, map_npix=32)
    noise = white_noise(nc, 1)
    s = gsim(prec, **w)
    kappa = s.run(torch.from_numpy(noise)).cpu().numpy()
    x, _ = [t.cpu().numpy() for t in s.particles()]
    o = OSim(**w)
    ref = o.run(noise)
    dx = periodic_diff(x, o.state.x, w["box"]) / (w["box"] / M)
    assert np.sqrt(np.mean(dx ** 2)) < 1e-3
    assert rel(kappa, ref) < 1e-3


def test_lens_projection_vs_oracle_with_pgd(cuda_lib):
    """Projection of one shell from an identical state (sub-evolution, PGD,
    rotation, two source planes)."""
    nc, M = 32, 64
    w = workload("pm64", nc=nc, nmesh=M, pgd=1, zs=(0.6, 1.0), map_npix=48)
    noise = white_noise(nc, 5)
    o = OSim(**w)
    o.ic(noise)
    i = 7
    for j in range(i + 1):
        o.step(j)
    o.lens_project(i)
    s = gsim(0, **w)
    s.set_particles(torch.from_numpy(o.state.x), torch.from_numpy(o.state.p), i + 1)
    s.lens_project(i)
    k = s.kappa_maps().cpu().numpy() + o.geom.mean_term()[:, None, None]
    assert o.maps.sum() > 0
    for m in range(2):
        assert rel(k[m], o.maps[m]) < 1e-4


def test_power_spectrum_bins_vs_oracle(cuda_lib):
    """Particle P(k) after a run: bins within 0.1% of the oracle."""
    nc, M = 32, 64
    w = workload("pm64", nc=nc, nmesh=M, map_npix=16)
    noise = white_noise(nc, 2)
    s = gsim(0, **w)
    s.run(torch.from_numpy(noise))
    x, _ = [t.cpu().numpy() for t in s.particles()]
    o = OSim(**w)
    o.run(noise)
    def pk(pos):
        d = np.fft.rfftn(omesh.density(pos, nc, nc, w["box"]) - 1)
        kx, ky, kz = omesh.wavevectors(nc, w["box"])
        k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2) * np.ones(d.shape)
        edges = np.linspace(0, np.pi * nc / w["box"], 9)
        idx = np.digitize(k.ravel(), edges)
        pw = np.abs(d.ravel()) ** 2
        return np.array([pw[idx == b].mean() for b in range(2, 9)])
    assert np.all(np.abs(pk(x) / pk(o.state.x) - 1) < 1e-3)


def test_state_errors(cuda_lib):
    from paper_2012_07266_gb300.lib import PMError
    w = workload("pm64", nc=32, nmesh=32, map_npix=8)
    s = gsim(0, **w)
    with pytest.raises(PMError):
        s.step(0)           # before pm_ic
    s.ic(torch.from_numpy(white_noise(32, 1)))
    with pytest.raises(PMError):
        s.step(1)           # out of order
    s.step(0)
    with pytest.raises(PMError):
        s.lens_project(1)   # not the last step
    s.lens_project(0)
    with pytest.raises(PMError):
        s.lens_project(0)   # twice
    s.sync()
