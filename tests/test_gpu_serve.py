"""Serving loop: requests that overlap on the GPU give the same maps and
gradients as the same requests run alone -- only the order of floating-point
atomic additions differs: maps within relative L2 1e-4, FP32 noise gradients
within 1e-3 (the adjoint's sensitivity amplifies the summation-order noise; the
FP32 gradient tolerance against the oracle is 2e-3) -- and admission respects
the HBM budget and the slot count."""
import numpy as np
import pytest
import torch

from pm_inputs import workload

pytestmark = pytest.mark.gpu

BASE = workload("pm64", box=256.0, map_npix=64, map_fov_deg=5.0, pgd=0, lpt_order=1)


def _specs():
    rng = np.random.default_rng(3)
    out = []
    for i, mesh in enumerate([64, 128, 64, 128, 64, 192]):
        out.append(dict(t_arrive=0.002 * i, nmesh=mesh, nc=mesh // 2,
                        omega_m=float(rng.uniform(0.25, 0.35)), sigma8=float(rng.uniform(0.7, 0.9)),
                        nsteps=int(rng.integers(8, 13)), zs=(float(rng.uniform(0.8, 1.6)),),
                        adjoint=bool(i % 2), noise_seed=100 + i))
    return out


def test_mix_equals_alone(cuda_lib):
    from paper_2012_07266_gb300.serve import Server, make_requests
    mix = make_requests(_specs(), BASE)
    stats = Server(max_slots=6).serve(mix)
    assert stats.completed == len(mix) and stats.max_active > 1
    for r in mix:
        assert r.error is None, r.error
        alone = make_requests([_specs()[r.rid]], BASE)[0]
        alone.t_arrive = 0.0
        Server(max_slots=1).serve([alone])
        a, b = r.kappa.cpu().numpy(), alone.kappa.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-4
        if r.adjoint:
            ga, gb = r.grad_noise.cpu().numpy(), alone.grad_noise.cpu().numpy()
            assert np.linalg.norm(ga - gb) / np.linalg.norm(gb) < 1e-3


def test_admission_by_footprint(cuda_lib):
    from paper_2012_07266_gb300.serve import Server, footprint, make_requests
    specs = [dict(_specs()[1], noise_seed=200 + i, t_arrive=0.0) for i in range(3)]  # three 128^3 meshes
    reqs = make_requests(specs, BASE)
    one = footprint(reqs[0].params)
    stats = Server(budget_bytes=int(1.5 * one), max_slots=8).serve(reqs)
    assert stats.completed == 3 and stats.max_active == 1      # a second one never fits
    assert stats.peak_bytes <= 1.5 * one
    reqs = make_requests(specs, BASE)
    stats = Server(budget_bytes=int(10 * one), max_slots=2).serve(reqs)
    assert stats.completed == 3 and stats.max_active == 2      # slot limit
    big = make_requests(_specs()[:1], BASE)[0]
    srv = Server(budget_bytes=footprint(big.params) - 1)
    st = srv.serve([big])
    assert st.completed == 0 and big.error is not None
