"""The reverse-mode derivative at the differentiable workload's full size
(128^3 particles, 256^3 mesh, 200 Mpc/h, 20 steps, a z = 1 source on a
1024^2 map over 4 degrees, every 4th step checkpointed) against central
finite differences of the GPU's own FP64 forward model (Sec. 3; Fig. vjp for
single initial modes, Appendix A for Omega_m and sigma_8).

Loss L = sum(lam * kappa) with lam ~ N(0, 1) per pixel (the gradient of a
Gaussian likelihood with unit noise, for data lam away from the model).

The forward model is smooth only piecewise: a particle that moves across a
shell boundary is projected from the next step's state, and one that crosses
the box boundary reappears in a neighbouring, differently rotated replica.
A central difference whose step moves particles across such boundaries
measures those jumps too, not only the derivative the reverse sweep computes.
Measured at this size: with step 1e-3 the sigma_8 difference even changes
sign between 1e-3 and 1e-4 and single modes scatter from 1e-4 to ~1 relative;
with step 1e-5 single modes agree to ~1e-6 (a few to 4e-3), and Omega_m and
sigma_8 agree to 2e-4 and 2e-7 with step 1e-9, where no particle crosses (the
FP64 forward's roundoff then limits the modes, whose derivatives are ~1e4
times smaller).  The test asserts at those steps and prints the 1e-3 record.
"""
import numpy as np
import pytest
import torch

from pm_inputs import white_noise, workload

pytestmark = pytest.mark.gpu

N_MODES = 16


def _sim(w, **over):
    from paper_2012_07266_gb300.api import Simulation
    return Simulation(device="cuda:0", precision=1, **dict(w, **over))


@pytest.fixture(scope="module")
def config3():
    w = workload("pm128_vjp")
    noise = white_noise(w["nc"], w["noise_seed"])
    rng = np.random.default_rng(5)
    lam = torch.from_numpy(rng.standard_normal((1, w["map_npix"], w["map_npix"]))).cuda()
    s = _sim(w)
    s.run(torch.from_numpy(noise))
    dn, (dom, ds8) = s.vjp(lam)
    modes = rng.choice(noise.size, N_MODES, replace=False)
    return w, noise, lam, dn.cpu().numpy().ravel(), dom, ds8, modes


def _loss(w, lam, noise, **over):
    k = _sim(w, ckpt_every=0, **over).run(torch.from_numpy(noise))
    return float((k * lam).sum())


def _fd_mode(w, lam, noise, j, eps):
    e = np.zeros(noise.size)
    e[j] = eps
    e = e.reshape(noise.shape)
    return (_loss(w, lam, noise + e) - _loss(w, lam, noise - e)) / (2 * eps)


def _fd_param(w, lam, noise, name, eps):
    return (_loss(w, lam, noise, **{name: w[name] + eps}) - _loss(w, lam, noise, **{name: w[name] - eps})) / (2 * eps)


def test_vjp_modes_vs_central_differences(cuda_lib, config3):
    """16 random initial modes, step 1e-5: median relative error below 1e-4,
    every mode below 3e-2 (a mode whose step moves a particle across a shell
    or box boundary keeps that jump)."""
    w, noise, lam, dn, _, _, modes = config3
    errs = []
    for j in modes:
        fd = _fd_mode(w, lam, noise, j, 1e-5)
        errs.append(abs(dn[j] - fd) / abs(dn[j]))
    errs = np.array(errs)
    print(f"\nconfig 3, 16 modes, step 1e-5: relative errors median {np.median(errs):.2e}, max {errs.max():.2e}")
    assert np.median(errs) < 1e-4
    assert errs.max() < 3e-2


def test_vjp_cosmology_vs_central_differences(cuda_lib, config3):
    """sigma_8 and Omega_m with step 1e-9 (no particle crosses a boundary): 1e-4
    and 3e-3 (the reverse sweep differences the Omega_m-dependent coefficients
    with step 1e-3, ~0.1% from the limit because of the CIC kinks)."""
    w, noise, lam, _, dom, ds8, _ = config3
    fd_s8 = _fd_param(w, lam, noise, "sigma8", 1e-9)
    fd_om = _fd_param(w, lam, noise, "omega_m", 1e-9)
    print(f"\nconfig 3, step 1e-9: sigma_8 vjp {ds8:.6e} fd {fd_s8:.6e}; Omega_m vjp {dom:.6e} fd {fd_om:.6e}")
    assert abs(ds8 - fd_s8) < 1e-4 * abs(ds8)
    assert abs(dom - fd_om) < 3e-3 * abs(dom)


def test_record_at_the_stated_step(cuda_lib, config3):
    """The stated check, step 1e-3 on the 16 modes and both parameters: printed
    for the record; asserted only to be finite and, for the modes, of the right
    sign in most cases (the differences straddle the model's jumps)."""
    w, noise, lam, dn, dom, ds8, modes = config3
    fds = np.array([_fd_mode(w, lam, noise, j, 1e-3) for j in modes])
    rel = np.abs(dn[modes] - fds) / np.abs(dn[modes])
    fd_s8 = _fd_param(w, lam, noise, "sigma8", 1e-3)
    fd_om = _fd_param(w, lam, noise, "omega_m", 1e-3)
    print(f"\nconfig 3, step 1e-3: modes relative error median {np.median(rel):.2e} max {rel.max():.2e}; "
          f"sigma_8 vjp {ds8:.4e} fd {fd_s8:.4e}; Omega_m vjp {dom:.4e} fd {fd_om:.4e}")
    assert np.all(np.isfinite(fds)) and np.isfinite(fd_s8) and np.isfinite(fd_om)
    assert np.mean(np.sign(fds) == np.sign(dn[modes])) >= 0.75
