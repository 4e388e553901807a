"""GPU shot-noise runs (pm_shot_noise_maps) and the binned angular power
spectrum (pm_map_cl) through the C ABI (Sec. 4, Fig. accuracy).

Small sizes: the random-run maps against the oracle's (same counter-based
positions; relative L2 1e-6 FP64, 1e-3 FP32, as the simulation maps), the
spectrum against the oracle's estimator (relative 1e-11 per bin; the mode
counts bit-exact, including modes that sit exactly on a bin edge), the
alpha/beta accumulation, and the whole "C(l) minus mean shot noise" pipeline.
Full size (pm256: 256^3 particles, four 2048^2 maps over 5 deg, the configuration
the benchmark times): the estimator against the oracle on the GPU's maps,
Parseval's identity, and each map's pixel variance and mean against the
closed-form Poisson values of projected unclustered particles.
"""
import numpy as np
import pytest
import torch
from scipy.integrate import quad

from oracle.cosmology import C_OVER_H0
from oracle.shotnoise import angular_cl, shot_noise_cl, shot_noise_maps
from oracle.sim import Simulation as OSim
from pm_inputs import white_noise, workload

pytestmark = pytest.mark.gpu


def gsim(precision=0, **w):
    from paper_2012_07266_gb300.api import Simulation
    return Simulation(device="cuda:0", precision=precision, **w)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _work(**over):
    base = dict(nc=32, nmesh=64, box=128.0, nsteps=10, map_npix=32, map_fov_deg=2.0, zs=(0.8, 1.0))
    base.update(over)
    w = workload("pm64", **base)
    z = np.linspace(0.5, 1.1, 61)
    w["source_nz"] = {1: (z, np.exp(-0.5 * ((z - 0.8) / 0.12) ** 2))}
    return w


def _edges(fov, nb, lmax_modes):
    lscale = 2 * np.pi / (fov * (np.pi / 180.0))
    return lscale * np.linspace(0.0, lmax_modes, nb + 1)    # edges on whole modes: ties exist


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (0, 1e-3)])
def test_shot_noise_maps_vs_oracle(cuda_lib, prec, tol):
    w = _work()
    s = gsim(prec, **w)
    for seed in (5, 2 ** 63 + 11):
        g = s.shot_noise_maps(seed).cpu().numpy()
        o = shot_noise_maps(OSim(**w), seed)
        assert rel(g, o) < tol


def test_map_cl_vs_oracle(cuda_lib):
    from paper_2012_07266_gb300.api import map_cl
    rng = np.random.default_rng(8)
    for n, fov, nb in [(8, 1.0, 3), (64, 2.0, 20), (256, 5.0, 37)]:
        maps = rng.standard_normal((3, n, n)) + np.linspace(0, 1, n)[None, None, :]
        edges = _edges(fov, nb, n / 2 * 1.2)
        gm = torch.from_numpy(maps).cuda()
        cl, counts = map_cl(gm, fov, edges, return_counts=True)
        ocl, ocounts = angular_cl(maps, fov, edges)
        assert counts == list(ocounts)
        ok = ocounts > 0
        assert np.all(np.abs(cl.cpu().numpy()[:, ok] - ocl[:, ok]) <= 1e-11 * np.abs(ocl[:, ok]))
        assert np.all(cl.cpu().numpy()[:, ~ok] == 0.0)
    # a mode on an edge: |m| = 5 from (3, 4) lands in the bin that starts at 5
    n, fov = 16, 3.0
    iy, ix = np.mgrid[0:n, 0:n]
    m = np.cos(2 * np.pi * (3 * ix + 4 * iy) / n)[None]
    edges = _edges(fov, 2, 10.0)                              # [0, 5 lscale), [5 lscale, 10 lscale)
    cl, counts = map_cl(torch.from_numpy(m).cuda(), fov, edges, return_counts=True)
    ocl, ocounts = angular_cl(m, fov, edges)
    assert counts == list(ocounts) and ocl[0, 0] < 1e-25 * ocl[0, 1]
    assert abs(cl[0, 1].item() - ocl[0, 1]) < 1e-12 * ocl[0, 1]


def test_map_cl_accumulation(cuda_lib):
    from paper_2012_07266_gb300.api import map_cl
    rng = np.random.default_rng(9)
    a, b = rng.standard_normal((2, 64, 64)), rng.standard_normal((2, 64, 64))
    edges = _edges(2.0, 8, 40)
    out = torch.full((2, 8), float("nan"), dtype=torch.float64, device="cuda")
    map_cl(torch.from_numpy(a).cuda(), 2.0, edges, out=out)                      # beta = 0 ignores the NaNs
    map_cl(torch.from_numpy(b).cuda(), 2.0, edges, alpha=-0.5, beta=2.0, out=out)
    ref = 2.0 * angular_cl(a, 2.0, edges)[0] - 0.5 * angular_cl(b, 2.0, edges)[0]
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-11, atol=0)


def test_cl_minus_shot_noise_fp64(cuda_lib):
    w = _work()
    noise = white_noise(w["nc"], 80)
    edges = _edges(w["map_fov_deg"], 6, 16)
    s = gsim(1, **w)
    kappa = s.run(torch.from_numpy(noise))
    got = s.cl_minus_shot_noise(kappa, edges, seeds=(3, 4)).cpu().numpy()
    o = OSim(**w)
    ok = o.run(noise)
    ref = angular_cl(ok, w["map_fov_deg"], edges)[0] - shot_noise_cl(OSim(**w), edges, (3, 4))
    assert rel(got, ref) < 1e-6
    # the runs replaced the state: stepping needs a new IC, after which a run is unchanged
    from paper_2012_07266_gb300 import lib
    with pytest.raises(lib.PMError) as ei:
        s.step(0)
    assert ei.value.status == 5
    assert rel(s.run(torch.from_numpy(noise)).cpu().numpy(), kappa.cpu().numpy()) < 1e-12


def test_map_cl_argument_checks(cuda_lib):
    import ctypes as C

    from paper_2012_07266_gb300 import lib
    so = lib.load()
    n = C.c_size_t(0)
    assert so.pm_map_cl_workspace_size(48, 1, 4, C.byref(n)) == 1       # not a power of two
    assert so.pm_map_cl_workspace_size(8192, 1, 4, C.byref(n)) == 1     # too large
    assert so.pm_map_cl_workspace_size(64, 1, 4096, C.byref(n)) == 1    # too many bins
    assert so.pm_map_cl_workspace_size(64, 2, 4, C.byref(n)) == 0
    maps = torch.zeros(2, 64, 64, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, 4, dtype=torch.float64, device="cuda")
    ws = torch.empty(n.value, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream

    def call(edges, nbytes, fov=2.0):
        e = (C.c_double * len(edges))(*edges)
        return so.pm_map_cl(C.c_void_p(maps.data_ptr()), 2, 64, fov, C.cast(e, C.c_void_p), len(edges) - 1, 1.0,
                            0.0, C.c_void_p(out.data_ptr()), None, C.c_void_p(ws.data_ptr()), nbytes,
                            C.c_void_p(st))
    assert call([0, 1, 2, 3, 4], n.value) == 0
    assert call([0, 2, 1, 3, 4], n.value) == 1           # not ascending
    assert call([0, 1, 2, 3, float("nan")], n.value) == 1
    assert call([0, 1, 2, 3, 4], n.value, fov=0.0) == 1
    assert call([0, 1, 2, 3, 4], n.value - 256) == 2     # workspace too small


def _poisson(w, s_index, g):
    """Closed-form pixel variance (4/9) K^2 V_p/Omega_pix J int q^2/a^2 dchi, the
    expected map mean (J - 1) K int chi q / a dchi (the particles' flat-sky
    density J against the subtracted mean term) and its standard deviation, for
    source plane s_index of the oracle geometry g (J = (1 + theta^2)^(-3/2)
    averaged over the pixel centres)."""
    c = g.cosmo
    K = 1.5 * c.omega_m / C_OVER_H0 ** 2
    cs = g.chi_s[s_index]
    th = (np.arange(g.npix) + 0.5) * g.dtheta - 0.5 * g.fov
    J = float(np.mean((1 + th[:, None] ** 2 + th[None, :] ** 2) ** -1.5))
    I = quad(lambda x: ((cs - x) / cs / c.a_of_chi(x)) ** 2, 0.0, cs, epsrel=1e-10, limit=500)[0]
    var = K ** 2 * g.vp / g.dtheta ** 2 * J * I
    mt = K * quad(lambda x: x * (cs - x) / cs / c.a_of_chi(x), 0.0, cs, epsrel=1e-10, limit=500)[0]
    return 4.0 / 9.0 * var, (J - 1.0) * mt, np.sqrt(var / g.npix ** 2)


def test_shot_noise_full_size_pm256(cuda_lib):
    """pm256 random run: each map's pixel variance within 3% of the closed-form
    Poisson value (the nearest particles' weights add ~0.3% at this resolution),
    the mean within 5 standard deviations of its flat-sky offset, the
    spectrum against the oracle's estimator and Parseval's identity."""
    from paper_2012_07266_gb300.api import map_cl
    w = workload("pm256")
    s = gsim(0, **w)
    maps = s.shot_noise_maps(1234)
    g = OSim(**w).geom
    m = maps.cpu().numpy()
    for k in range(len(w["zs"])):
        var_th, mean_th, sd_mean = _poisson(w, k, g)
        assert abs(m[k].var() / var_th - 1) < 0.03
        assert abs(m[k].mean() - mean_th) < 5 * sd_mean
    fov = w["map_fov_deg"]
    edges = np.concatenate([[0.0], np.geomspace(100.0, 40000.0, 30)])
    cl, counts = map_cl(maps, fov, edges, return_counts=True)
    ocl, ocounts = angular_cl(m, fov, edges)
    assert counts == list(ocounts)
    assert np.allclose(cl.cpu().numpy(), ocl, rtol=1e-10, atol=0)
    one = map_cl(maps, fov, [0.0, np.inf]).cpu().numpy()[:, 0]
    opix = (fov * np.pi / 180.0 / w["map_npix"]) ** 2
    assert np.allclose(one / opix, (m ** 2).mean(axis=(1, 2)), rtol=1e-10, atol=0)
