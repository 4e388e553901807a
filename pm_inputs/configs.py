"""Workload parameter sets (plain data, no arithmetic of the method).

The parameter names mirror the user-settable simulation parameters of the
paper (Table 1): box size, particle grid, force mesh (B = nmesh / nc),
number of steps, source redshifts, map resolution and field of view,
Omega_m, sigma_8, PGD on/off and the sub-evolution ("interpolation") switch.

PGD parameters: the fitted values are not printed in the paper (Sec. 3 says
they are fitted on training simulations); the values below are arbitrary,
fixed stand-ins of plausible magnitude (alpha0, mu, k_l [h/Mpc], k_s [h/Mpc], n).
"""
from __future__ import annotations

import copy

# flat LCDM used by every workload (Omega_b, T_cmb are the Eisenstein-Hu extras)
_COSMO = dict(omega_m=0.3089, sigma8=0.8159, h=0.6774, n_s=0.9667,
              omega_b=0.0486, t_cmb=2.7255)

PGD_PARAMS = (0.02, -0.3, 0.35, 6.0, 4.0)  # alpha0, mu, k_l, k_s, n

WORKLOADS = {
    # 64^3 particles on a 64^3 mesh, 128 Mpc/h, 1LPT at a=0.1, 10 steps, one
    # source at z=1 on a 64x64, 2x2 degree map.
    "pm64": dict(nc=64, nmesh=64, box=128.0, a_init=0.1, nsteps=10, lpt_order=1,
                 zs=(1.0,), map_npix=64, map_fov_deg=2.0, sub_evolution=1,
                 pgd=0, pgd_params=PGD_PARAMS, rotate=1, rotation_seed=42,
                 noise_seed=1234 + 1, **_COSMO),
    # paper-scale forward run: 256^3 particles, 512^3 mesh, 256 Mpc/h, 2LPT at
    # a=0.1, 40 steps, four source planes, 2048^2 maps over 5x5 degrees, PGD on.
    "pm256": dict(nc=256, nmesh=512, box=256.0, a_init=0.1, nsteps=40, lpt_order=2,
                  zs=(0.5, 1.0, 1.5, 2.0), map_npix=2048, map_fov_deg=5.0,
                  sub_evolution=1, pgd=1, pgd_params=PGD_PARAMS, rotate=1,
                  rotation_seed=42, noise_seed=1234 + 2, **_COSMO),
    # differentiable run: 128^3 particles, 256^3 mesh, 200 Mpc/h, 20 steps,
    # one source at z=1 on a 1024^2, 4x4 degree map, checkpoint every 4 steps.
    "pm128_vjp": dict(nc=128, nmesh=256, box=200.0, a_init=0.1, nsteps=20, lpt_order=1,
                      zs=(1.0,), map_npix=1024, map_fov_deg=4.0, sub_evolution=1,
                      pgd=0, pgd_params=PGD_PARAMS, rotate=1, rotation_seed=42,
                      ckpt_every=4, noise_seed=1234 + 3, **_COSMO),
    # large run: 512^3 particles, 1024^3 mesh, 512 Mpc/h, 40 steps, 8 source
    # planes to z=2.5, 4096^2 maps over 10x10 degrees, PGD on.
    "pm512": dict(nc=512, nmesh=1024, box=512.0, a_init=0.1, nsteps=40, lpt_order=2,
                  zs=(0.5, 0.75, 1.0, 1.25, 1.5, 1.75, 2.0, 2.5), map_npix=4096,
                  map_fov_deg=10.0, sub_evolution=1, pgd=1, pgd_params=PGD_PARAMS,
                  rotate=1, rotation_seed=42, noise_seed=1234 + 5, **_COSMO),
}


def workload(name: str, **overrides) -> dict:
    """Return a copy of a named workload with optional overrides."""
    w = copy.deepcopy(WORKLOADS[name])
    w.update(overrides)
    return w


def cosmology_params(w: dict) -> dict:
    """The cosmological subset of a workload dict."""
    return {k: w[k] for k in _COSMO}
