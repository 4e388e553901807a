"""GPU reverse-mode derivative (pm_vjp) against the oracle's FP64 adjoint and
against finite differences of the GPU forward model, through the C ABI.

Checkpointed (ckpt_every < nsteps: segments recomputed from checkpoints) and
resident (ckpt_every >= nsteps: nothing recomputed) reverse sweeps.

Tolerances: the noise gradient matches the oracle to relative L2 1e-6 on the
FP64 path and 2e-3 on the FP32 path (FP32 particle state and meshes);
dL/dsigma_8 to 1e-6 / 2e-3; dL/dOmega_m to 1e-6 / 5e-3, both sides taking the
central difference of the cosmology-dependent coefficients with the same
step (1e-3; the difference to the h -> 0 limit is ~0.1% because the map's CIC
weights have kinks at pixel centres).
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as oadj
from oracle.sim import Simulation as OSim
from pm_inputs import white_noise, workload

pytestmark = pytest.mark.gpu


def gsim(precision=0, **w):
    from paper_2012_07266_gb300.api import Simulation
    return Simulation(device="cuda:0", precision=precision, **w)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _work(**over):
    base = dict(nc=32, nmesh=64, box=128.0, nsteps=6, map_npix=16, zs=(1.0,), ckpt_every=2)
    base.update(over)
    return workload("pm64", **base)


CASES = [
    (1, dict(), 1e-6, 1e-6),
    (0, dict(), 2e-3, 5e-3),
    (1, dict(lpt_order=2, pgd=1, zs=(0.8, 1.0), ckpt_every=4), 1e-6, 1e-6),
    (0, dict(lpt_order=2, pgd=1, zs=(0.8, 1.0), ckpt_every=4), 2e-3, 5e-3),
    # resident adjoint (ckpt_every >= nsteps): every state, force and PGD mesh kept by the forward,
    # no recompute; the state is re-sorted after step 3, inside the single segment
    (1, dict(lpt_order=2, pgd=1, zs=(0.8, 1.0), ckpt_every=6), 1e-6, 1e-6),
    (0, dict(lpt_order=2, pgd=1, zs=(0.8, 1.0), ckpt_every=100), 2e-3, 5e-3),
    (0, dict(ckpt_every=6), 2e-3, 5e-3),
    # as many particles as mesh cells: runs of sorted particles then cover ~1000-2000 cells, so
    # both forms of the cotangent paint and of the readout gradient run in the same sweep (the
    # shared-memory tile for the runs whose box fits it -- about half of the readout gradient's
    # runs of 1024 particles, 10-15% of the paired ones -- and per-corner global reductions and
    # gathers for the others)
    (0, dict(nc=32, nmesh=32, lpt_order=2, pgd=1, zs=(0.8, 1.0), ckpt_every=2), 2e-3, 5e-3),
]


@pytest.mark.parametrize("prec,over,tol,tol_om", CASES)
def test_vjp_vs_oracle(cuda_lib, prec, over, tol, tol_om):
    w = _work(**over)
    noise = white_noise(w["nc"], 21)
    rng = np.random.default_rng(22)
    lam = rng.standard_normal((len(w["zs"]), w["map_npix"], w["map_npix"]))
    s = gsim(prec, **w)
    kappa = s.run(torch.from_numpy(noise))
    dn, (dom, ds8) = s.vjp(torch.from_numpy(lam))
    dn = dn.cpu().numpy()
    ok, on, oom, os8 = oadj.vjp(OSim(**w), noise, lam, h_om=1e-3)
    assert rel(kappa.cpu().numpy(), ok) < (1e-6 if prec else 1e-3)
    assert rel(dn, on) < tol
    assert abs(ds8 - os8) < tol * abs(os8)
    assert abs(dom - oom) < tol_om * abs(oom)


def test_vjp_directional_derivative_fp64(cuda_lib):
    """<dL/dnoise, d> against a central difference of the GPU forward (FP64)."""
    w = _work(lpt_order=2, pgd=1)
    noise = white_noise(w["nc"], 23)
    rng = np.random.default_rng(24)
    lam = rng.standard_normal((1, w["map_npix"], w["map_npix"]))
    d = rng.standard_normal(noise.shape)
    s = gsim(1, **w)
    s.run(torch.from_numpy(noise))
    dn, _ = s.vjp(torch.from_numpy(lam))
    eps = 1e-6

    def loss(nz):
        return float(np.sum(lam * gsim(1, **w).run(torch.from_numpy(nz)).cpu().numpy()))
    fd = (loss(noise + eps * d) - loss(noise - eps * d)) / (2 * eps)
    an = float(np.sum(dn.cpu().numpy() * d))
    # 32^3 particles: a 1e-6 step already crosses a few CIC cell boundaries
    assert abs(an - fd) < 1e-4 * abs(fd)


def test_vjp_state_checks(cuda_lib):
    from paper_2012_07266_gb300.lib import PMError
    w = _work(ckpt_every=0)
    s = gsim(0, **w)
    s.run(torch.from_numpy(white_noise(32, 1)))
    with pytest.raises(PMError):      # no checkpoints configured
        s.vjp(torch.zeros((1, 16, 16), dtype=torch.float64))
    w = _work()
    s = gsim(0, **w)
    s.ic(torch.from_numpy(white_noise(32, 1)))
    with pytest.raises(PMError):      # forward run not finished
        s.vjp(torch.zeros((1, 16, 16), dtype=torch.float64))
