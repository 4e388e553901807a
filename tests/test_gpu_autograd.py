"""torch.autograd through the whole forward model (KappaModel / KappaFn): the
gradients of a Gaussian likelihood of the maps with respect to the white noise
and to [Omega_m, sigma_8] reach the library's reverse sweep (pm_vjp) and match
the oracle's FP64 adjoint (Sec. 3; Appendix A for the cosmology derivatives).

Loss: L = 1/2 sum ((kappa - d) / sigma)^2 with data d drawn far from the model
(d ~ 100 rms(kappa) N(0, 1), sigma = 1), so that dL/dkappa = kappa - d is set
by the data and the oracle's own dL/dkappa (from its own maps) differs from the
GPU's by the map error divided by ~100: well inside the tolerances.
Tolerances as the direct pm_vjp tests: noise 1e-6 (FP64) / 2e-3 (FP32),
sigma_8 1e-6 / 2e-3, Omega_m 1e-6 / 5e-3 (both sides difference the
cosmology-dependent coefficients with the step 1e-3).
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle.sim import Simulation as OSim
from pm_inputs import white_noise, workload

pytestmark = pytest.mark.gpu


def _work(**over):
    base = dict(nc=32, nmesh=64, box=128.0, nsteps=6, map_npix=16, zs=(0.8, 1.0), lpt_order=2, pgd=1)
    base.update(over)
    return workload("pm64", **base)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("prec,ckpt,tol,tol_om", [(1, 2, 1e-6, 1e-6), (0, 2, 2e-3, 5e-3), (0, None, 2e-3, 5e-3)])
def test_autograd_gaussian_loss_vs_oracle(cuda_lib, prec, ckpt, tol, tol_om):
    from paper_2012_07266_gb300.api import KappaModel
    over = {} if ckpt is None else {"ckpt_every": ckpt}  # None: the model's default (resident)
    w = _work(**over)
    noise_np = white_noise(w["nc"], 31)
    cosmo_np = np.array([w["omega_m"], w["sigma8"]])
    model = KappaModel(device="cuda:0", precision=prec, **w)
    noise = torch.from_numpy(noise_np).cuda().requires_grad_()
    cosmo = torch.tensor(cosmo_np, dtype=torch.float64, requires_grad=True)
    kappa = model(noise, cosmo)
    rng = np.random.default_rng(32)
    scale = 100.0 * float(kappa.detach().pow(2).mean().sqrt())
    d = torch.from_numpy(scale * rng.standard_normal(tuple(kappa.shape))).cuda()
    loss = 0.5 * ((kappa - d) ** 2).sum()
    gn, gc = torch.autograd.grad(loss, [noise, cosmo])
    assert gn.shape == noise.shape and gn.dtype == noise.dtype and gn.is_cuda
    assert gc.shape == (2,) and gc.device.type == "cpu"

    osim = OSim(**w)
    ok = osim.run(noise_np)
    lam = ok - d.cpu().numpy()
    _, on, oom, os8 = oadj.vjp(OSim(**w), noise_np, lam, h_om=1e-3)
    assert rel(kappa.detach().cpu().numpy(), ok) < (1e-6 if prec else 1e-3)
    assert rel(gn.cpu().numpy(), on) < tol
    assert abs(float(gc[1]) - os8) < tol * abs(os8)
    assert abs(float(gc[0]) - oom) < tol_om * abs(oom)


def test_autograd_backward_needs_its_own_forward(cuda_lib):
    """A model differentiates its latest run once: a backward after another
    forward, or a second backward, raises instead of returning wrong gradients."""
    from paper_2012_07266_gb300.api import KappaModel
    w = _work(nsteps=4, pgd=0, lpt_order=1, zs=(1.0,))
    model = KappaModel(device="cuda:0", **w)
    cosmo = torch.tensor([w["omega_m"], w["sigma8"]], dtype=torch.float64, requires_grad=True)
    n1 = torch.from_numpy(white_noise(32, 1)).cuda().requires_grad_()
    n2 = torch.from_numpy(white_noise(32, 2)).cuda().requires_grad_()
    k1 = model(n1, cosmo)
    k2 = model(n2, cosmo)
    with pytest.raises(RuntimeError):
        k1.sum().backward()
    loss = k2.sum()
    loss.backward(retain_graph=True)
    assert n2.grad is not None and torch.isfinite(n2.grad).all()
    with pytest.raises(RuntimeError):
        loss.backward()


def test_autograd_cosmology_change_rebuilds_tables(cuda_lib):
    """A new (Omega_m, sigma_8) gives the maps of that cosmology (the model
    replaces its simulation), equal to a Simulation built for it directly."""
    from paper_2012_07266_gb300.api import KappaModel, Simulation
    w = _work(nsteps=4, pgd=0, lpt_order=1, zs=(1.0,))
    model = KappaModel(device="cuda:0", precision=1, **w)
    noise = torch.from_numpy(white_noise(32, 3)).cuda()
    k_a = model(noise, torch.tensor([0.30, 0.80], dtype=torch.float64))
    k_b = model(noise, torch.tensor([0.32, 0.85], dtype=torch.float64))
    ref = Simulation(device="cuda:0", precision=1, **dict(w, omega_m=0.32, sigma8=0.85)).run(noise)
    assert float((k_b - ref).norm() / ref.norm()) < 1e-12
    assert float((k_a - k_b).norm() / k_b.norm()) > 1e-2
