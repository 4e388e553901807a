"""GPU forward-mode derivative (pm_jvp) through the C ABI: against the oracle's
FP64 tangent-linear model, against the GPU reverse sweep of the same trajectory
through the dot-product identity <lam, J d> = <J^T lam, d>, and along one noise
pixel (the paper's check, Fig. 8).

Tolerances: the map derivative matches the oracle to relative L2 1e-6 on the
FP64 path and 2e-3 on the FP32 path (FP32 particle state and meshes, as the
reverse-mode tests); the dot-product identity to 1e-8 (FP64: the two sides are
different exact derivatives of one trajectory, differing by rounding order).
Six steps include a re-sort of the particle state (the tangent follows it).
"""
import numpy as np
import pytest
import torch

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
    base = dict(nc=32, nmesh=64, box=128.0, nsteps=6, map_npix=16, zs=(1.0,), jvp=1)
    base.update(over)
    return workload("pm64", **base)


CASES = [
    (1, dict(), 1e-6),
    (0, dict(), 2e-3),
    (1, dict(lpt_order=2, pgd=1, zs=(0.8, 1.0)), 1e-6),
    (0, dict(lpt_order=2, pgd=1, zs=(0.8, 1.0)), 2e-3),
]


@pytest.mark.parametrize("prec,over,tol", CASES)
def test_jvp_vs_oracle(cuda_lib, prec, over, tol):
    w = _work(**over)
    noise = white_noise(w["nc"], 51)
    d = np.random.default_rng(52).standard_normal(noise.shape)
    kappa, dk = gsim(prec, **w).jvp(torch.from_numpy(noise), torch.from_numpy(d))
    ok, odk = ojvp.jvp(OSim(**w), noise, d)
    assert rel(kappa.cpu().numpy(), ok) < (1e-6 if prec else 1e-3)
    assert rel(dk.cpu().numpy(), odk) < tol


def test_jvp_single_pixel_fp64(cuda_lib):
    """The paper's test direction: one pixel of the initial field (Fig. 8)."""
    w = _work(lpt_order=2, pgd=1)
    noise = white_noise(w["nc"], 53)
    d = np.zeros_like(noise)
    d[3, 17, 29] = 1.0
    _, dk = gsim(1, **w).jvp(torch.from_numpy(noise), torch.from_numpy(d))
    _, odk = ojvp.jvp(OSim(**w), noise, d)
    assert rel(dk.cpu().numpy(), odk) < 1e-6


@pytest.mark.parametrize("ckpt", [2, 6])
def test_jvp_vjp_dot_product_fp64(cuda_lib, ckpt):
    """<lam, J d> (forward mode) against <J^T lam, d> (reverse sweep, checkpointed
    or resident) on the GPU, for the trajectory pm_jvp ran."""
    w = _work(lpt_order=2, pgd=1, zs=(0.8, 1.0), ckpt_every=ckpt)
    noise = white_noise(w["nc"], 54)
    rng = np.random.default_rng(55)
    d = rng.standard_normal(noise.shape)
    lam = rng.standard_normal((2, w["map_npix"], w["map_npix"]))
    s = gsim(1, **w)
    _, dk = s.jvp(torch.from_numpy(noise), torch.from_numpy(d))
    dn, _ = s.vjp(torch.from_numpy(lam))
    lhs = float(np.sum(lam * dk.cpu().numpy()))
    rhs = float(np.sum(dn.cpu().numpy() * d))
    assert abs(lhs - rhs) < 1e-8 * abs(rhs)


def test_jvp_needs_the_tangent_workspace(cuda_lib):
    from paper_2012_07266_gb300 import lib
    w = _work(jvp=0)
    noise = torch.from_numpy(white_noise(w["nc"], 56))
    with pytest.raises(lib.PMError) as ei:
        gsim(0, **w).jvp(noise, noise)
    assert ei.value.status == 6  # PM_ERR_UNSUPPORTED
