"""The lightcone projection and a whole run at the benchmark workloads' own
geometry against the oracle (Eq. conv; Sec. 3 box replication, rotation and
sub-evolution).

pm256 geometry: 5 x 5 degree maps of 2048^2 pixels, four source planes to
z = 2, a 256 Mpc/h box on a 512^3 force mesh with PGD: the field of view is
wider than the box beyond z ~ 1.4, so shells are tiled across the line of
sight as well as along it, which is where the projection's per-warp replica
culling decides most.  pm512 geometry: 10 x 10 degrees, 4096^2 pixels, eight
sources to z = 2.5, a 512 Mpc/h box.  64^3 particles (set from an oracle
state through pm_set_particles) keep the oracle's projection to seconds; the
culling works on whatever particles are there.

Tolerances: one shell, relative L2 per map, 1.5 npix 2^-24 on the FP32 path
(1.8e-4 at 2048^2, 3.7e-4 at 4096^2): the FP32 pixel coordinate u in [0, npix)
keeps npix 2^-24 of a pixel at best, and its rounding moves CIC weight between
neighbouring pixels (measured 1.2e-4 and 2.8e-4, both in the shell that holds
the farthest source; shell membership itself is decided in FP64 near the shell
boundaries); 1e-6 on the FP64 path (the library's 16384-point distance tables
against the oracle's splines).  The whole run: 1e-3 (FP32) / 1e-6 (FP64) per
map and final positions 1e-3 of a force-mesh cell RMS.
"""
import numpy as np
import pytest
import torch

from oracle.lightcone import candidate_replicas
from oracle.sim import Simulation as OSim
from pm_inputs import white_noise, workload

pytestmark = pytest.mark.gpu


def gsim(precision=0, **w):
    from paper_2012_07266_gb300.api import Simulation
    return Simulation(device="cuda:0", precision=precision, **w)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def periodic_diff(a, b, box):
    d = a - b
    return d - box * np.round(d / box)


def transverse_replicas(o, i):
    lo, hi = o.geom.shell(i)
    reps = candidate_replicas(lo, hi, o.geom.box, 0.5 * o.geom.fov + o.geom.dtheta, 2.0 * o.geom.box / o.geom.nmesh)
    return {(n[0], n[1]) for n in reps}


def oracle_state(w, seed):
    o = OSim(**w)
    o.ic(white_noise(w["nc"], seed))
    return o


@pytest.fixture(scope="module")
def pm256_geometry():
    return oracle_state(workload("pm256", nc=64), 41)


@pytest.fixture(scope="module")
def pm512_geometry():
    return oracle_state(workload("pm512", nc=64, nmesh=256), 42)


def check_shells(w, o, shells, prec, tol):
    """Project the oracle state as the state after each step of `shells` in turn;
    compare each shell's map increments with the oracle's."""
    x, p = o.state.x, o.state.p
    s = gsim(prec, **w)
    prev = np.zeros((len(w["zs"]), w["map_npix"], w["map_npix"]))
    mean = o.geom.mean_term()[:, None, None]
    for i in shells:
        inc, hits = o.geom.project(i, x, p, o.pgd_at(i))
        assert hits > 0
        s.set_particles(torch.from_numpy(x), torch.from_numpy(p), i + 1)
        s.lens_project(i)
        raw = s.kappa_maps().cpu().numpy() + mean
        got, prev = raw - prev, raw
        for m in range(len(w["zs"])):
            if np.any(inc[m]):
                assert rel(got[m], inc[m]) < tol, (i, m, rel(got[m], inc[m]))
            else:
                assert np.max(np.abs(got[m])) <= 1e-12 * np.max(np.abs(raw))


def fp32_map_tol(npix):
    return 1.5 * npix * 2.0 ** -24


@pytest.mark.parametrize("prec,tol", [(0, fp32_map_tol(2048)), (1, 1e-6)])
def test_shells_at_pm256_geometry_vs_oracle(cuda_lib, pm256_geometry, prec, tol):
    """Shells at z ~ 1.9 (holding the farthest source, z = 2), ~0.8 and ~0.3."""
    w, o = workload("pm256", nc=64), pm256_geometry
    assert len(transverse_replicas(o, 10)) >= 4   # tiled across the line of sight
    check_shells(w, o, (10, 20, 30), prec, tol)


@pytest.mark.parametrize("prec,tol", [(0, fp32_map_tol(4096)), (1, 1e-6)])
def test_shells_at_pm512_geometry_vs_oracle(cuda_lib, pm512_geometry, prec, tol):
    """Shells at z ~ 2.5 (the farthest source) and ~0.8, 10 degrees over 4096^2
    (the field of view, +-360 Mpc/h at z = 2.5, spans 2 x 2 replicas of the box)."""
    w, o = workload("pm512", nc=64, nmesh=256), pm512_geometry
    assert len(transverse_replicas(o, 8)) >= 4
    check_shells(w, o, (8, 20), prec, tol)


@pytest.fixture(scope="module")
def pm256_short_run():
    """The oracle's whole run at pm256 geometry with 64^3 particles and 10 steps
    (2LPT, PGD; shells 2..9 lie inside the lightcone of the z = 2 source), on a
    256^3 force mesh to keep the FP64 oracle to minutes (the 512^3 mesh's FFT
    and force kernels are checked at full size elsewhere)."""
    w = workload("pm256", nc=64, nmesh=256, nsteps=10)
    noise = white_noise(64, 43)
    o = OSim(**w)
    kappa = o.run(noise)
    return w, noise, kappa, o.state.x


@pytest.mark.parametrize("prec,tol", [(0, 1e-3), (1, 1e-6)])
def test_run_at_pm256_geometry_vs_oracle(cuda_lib, pm256_short_run, prec, tol):
    w, noise, ok, ox = pm256_short_run
    s = gsim(prec, **w)
    kappa = s.run(torch.from_numpy(noise)).cpu().numpy()
    x, _ = [t.cpu().numpy() for t in s.particles()]
    dx = periodic_diff(x, ox, w["box"]) / (w["box"] / w["nmesh"])
    pos_rms = float(np.sqrt(np.mean(dx ** 2)))
    errs = [rel(kappa[m], ok[m]) for m in range(len(w["zs"]))]
    print(f"\npm256 geometry, 64^3 on 256^3, 10 steps, precision {prec}: position RMS {pos_rms:.3e} cells, "
          f"kappa rel L2 per source {['%.3e' % e for e in errs]}")
    assert pos_rms < 1e-3
    assert max(errs) < tol


def test_pm512_fp32_vs_fp64_first_steps(cuda_lib):
    """Config 5 at its full size (512^3 particles, 1024^3 mesh, 8 sources to z =
    2.5, 4096^2 maps, PGD): the FP32 path against the FP64 path through IC and
    the first ten steps, whose last two shells hold the z = 2.5 source (positions
    1e-3 cell RMS, forces 1e-5 relative L2, maps 2e-3 per map)."""
    w = workload("pm512")
    noise = torch.from_numpy(white_noise(512, w["noise_seed"]))
    nsteps = 10
    ref = {}
    for prec in (1, 0):
        s = gsim(prec, **w)
        s.ic(noise)
        for i in range(nsteps):
            s.step(i)
            s.lens_project(i)
        x, _ = s.particles()
        f = s.forces()
        k = s.kappa_maps()
        if prec == 1:
            ref = dict(x=x, f=f, k=k)
            del s, x, f, k
            torch.cuda.empty_cache()
            continue
        cell = w["box"] / w["nmesh"]
        d = x - ref["x"]
        d = d - w["box"] * torch.round(d / w["box"])
        pos_rms = float((d / cell).pow(2).mean().sqrt())
        ferr = float((f - ref["f"]).norm() / ref["f"].norm())
        kerr = [float((k[m] - ref["k"][m]).norm() / ref["k"][m].norm())
                for m in range(len(w["zs"])) if float(ref["k"][m].abs().max()) > 0]
        print(f"\npm512 FP32 vs FP64 after {nsteps} steps: position RMS {pos_rms:.3e} cells, force rel L2 "
              f"{ferr:.3e}, kappa rel L2 {['%.2e' % e for e in kerr]}")
        assert len(kerr) > 0
        assert pos_rms < 1e-3
        assert ferr < 1e-5
        assert max(kerr) < 2e-3
