"""Seeded random draws (numpy PCG64), handed unchanged to both implementations."""
from __future__ import annotations

import numpy as np


def white_noise(nc: int, seed: int) -> np.ndarray:
    """Real-space N(0,1) white-noise field on the nc^3 particle lattice.

    float64, C order, shape (nc, nc, nc) indexed [z, y, x] (x fastest).
    The GPU path receives the same values cast to float32.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((nc, nc, nc))


def serving_arrivals(n: int, rate_hz: float = 20.0, seed: int = 7):
    """Poisson arrival times and per-request parameters for the serving mix.

    Mesh per side from {64, 128, 192} with nc = mesh / 2, Omega_m ~ U(0.25, 0.35),
    sigma_8 ~ U(0.7, 0.9), 10-30 steps, one source z_s ~ U(0.8, 1.6), 512^2 maps;
    half the requests ask for forward + adjoint.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(n):
        mesh = int(rng.choice([64, 128, 192]))
        reqs.append(dict(
            t_arrive=float(t[i]), nmesh=mesh, nc=mesh // 2,
            omega_m=float(rng.uniform(0.25, 0.35)), sigma8=float(rng.uniform(0.7, 0.9)),
            nsteps=int(rng.integers(10, 31)), zs=(float(rng.uniform(0.8, 1.6)),),
            adjoint=bool(rng.integers(0, 2)), noise_seed=int(rng.integers(0, 2**31 - 1)),
        ))
    return reqs
