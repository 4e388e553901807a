"""The allocation-free force entry point (pm_forces_static) against the
workspace path (pm_set_particles + pm_get_forces), on calls in a row.

pm_forces_static serves callers that cannot allocate device memory; its
scratch lives in a static device array shared by every call, so a call must
not see anything left over from the one before, including one of the other
mesh size (32^3 and 64^3 use different half-spectrum pitches in the same
array).  This file is collected last so that a failure here comes after every
other test has run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative L2, the single-step force tolerance of the other tests
BOX = 100.0
NC = {32: 32, 64: 32}  # particles per side for each mesh (the IC lattice FFT needs nc >= 32)


def _static(so, x, M, omega_m, f):
    return so.pm_forces_static(C.c_void_p(x.data_ptr()), C.c_int64(x.shape[0]), M, C.c_double(BOX),
                               C.c_double(omega_m), C.c_void_p(f.data_ptr()),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _positions(M, seed):
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.uniform(0, BOX, size=(NC[M] ** 3, 3))).cuda()


def test_forces_static_matches_workspace_path_in_a_row(cuda_lib):
    from paper_2012_07266_gb300 import lib
    from paper_2012_07266_gb300.api import Simulation
    from pm_inputs import workload

    so = lib.load()
    sims = {M: Simulation(device="cuda:0", **workload("pm64", nc=NC[M], nmesh=M, box=BOX, map_npix=8))
            for M in (32, 64)}
    om = sims[64].cfg.omega_m
    # two calls of each size in a row, the sizes alternating
    for M, seed in ((64, 11), (64, 12), (32, 13), (32, 14), (64, 15), (32, 16)):
        x = _positions(M, seed)
        f = torch.full_like(x, float("nan"))
        st = _static(so, x, M, om, f)
        assert st == 0, lib.STATUS.get(st)
        sims[M].set_particles(x, torch.zeros_like(x), 0)
        ref = sims[M].forces()
        torch.cuda.synchronize()
        assert torch.isfinite(f).all()
        err = float((f - ref).norm() / ref.norm())
        assert err < TOL, (M, seed, err)


def test_forces_static_allocates_nothing(cuda_lib):
    """After a first call (which may load the library's device code), further
    calls leave the device's free memory unchanged."""
    from paper_2012_07266_gb300 import lib
    so = lib.load()
    xs = {M: _positions(M, 20 + M) for M in (32, 64)}
    fs = {M: torch.empty_like(xs[M]) for M in (32, 64)}
    for M in (32, 64):
        assert _static(so, xs[M], M, 0.3, fs[M]) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        for M in (32, 64):
            assert _static(so, xs[M], M, 0.3, fs[M]) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_forces_static_rejects_oversized_mesh(cuda_lib):
    from paper_2012_07266_gb300 import lib
    so = lib.load()
    x = torch.zeros((8, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros_like(x)
    st = so.pm_forces_static(C.c_void_p(x.data_ptr()), C.c_int64(8), 128, C.c_double(100.0),
                             C.c_double(0.3), C.c_void_p(f.data_ptr()), None)
    assert st == 6  # PM_ERR_UNSUPPORTED, before any device work
