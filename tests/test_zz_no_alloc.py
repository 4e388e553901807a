"""The allocation-free force entry point (pm_forces_static) against the
workspace path (pm_set_particles + pm_get_forces), on two calls in a row.

pm_forces_static serves callers that cannot allocate device memory; its
scratch lives in a static device array shared by every call, so the second
call must not see anything left over from the first.  This file is collected
last so that a failure here comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative L2, the single-step force tolerance of the other tests


def test_forces_static_matches_workspace_path_twice(cuda_lib):
    from paper_2012_07266_gb300 import lib
    from paper_2012_07266_gb300.api import Simulation
    from pm_inputs import workload

    so = lib.load()
    nc, M, L = 32, 64, 100.0
    w = workload("pm64", nc=nc, nmesh=M, box=L, map_npix=8)
    sim = Simulation(device="cuda:0", **w)
    stream = torch.cuda.current_stream()
    for seed in (11, 12):
        rng = np.random.default_rng(seed)
        x = torch.from_numpy(rng.uniform(0, L, size=(nc ** 3, 3))).cuda()
        f = torch.full_like(x, float("nan"))
        st = so.pm_forces_static(C.c_void_p(x.data_ptr()), C.c_int64(nc ** 3), M, C.c_double(L),
                                 C.c_double(w["omega_m"]), C.c_void_p(f.data_ptr()),
                                 C.c_void_p(stream.cuda_stream))
        assert st == 0, lib.STATUS.get(st)
        sim.set_particles(x, torch.zeros_like(x), 0)
        ref = sim.forces()
        torch.cuda.synchronize()
        assert torch.isfinite(f).all()
        err = float((f - ref).norm() / ref.norm())
        assert err < TOL, err


def test_forces_static_rejects_oversized_mesh(cuda_lib):
    from paper_2012_07266_gb300 import lib
    so = lib.load()
    x = torch.zeros((8, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros_like(x)
    st = so.pm_forces_static(C.c_void_p(x.data_ptr()), C.c_int64(8), 128, C.c_double(100.0),
                             C.c_double(0.3), C.c_void_p(f.data_ptr()), None)
    assert st == 6  # PM_ERR_UNSUPPORTED, before any device work
