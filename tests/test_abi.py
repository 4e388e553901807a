"""Host-side checks of the C ABI: the library loads, exports every symbol
include/pm.h declares, and validates configurations before any device work."""
import ctypes as C
import os
import re

import pytest

from pm_inputs import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2012_07266_gb300 import lib
    if not os.path.exists(lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return lib


def header_functions():
    src = open(os.path.join(ROOT, "include", "pm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:pm_status|const char\*|int32_t)\s+(\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert len(names) >= 16
    so = L.load()
    for n in names:
        assert hasattr(so, n), n
    assert sorted(L.EXPORTS) == names


def test_workspace_size_host_only(L):
    n32 = L.workspace_size(L.make_config(workload("pm64")))
    n64 = L.workspace_size(L.make_config(workload("pm64"), precision=L.PM_FP64))
    assert 0 < n32 < n64
    big = L.workspace_size(L.make_config(workload("pm256")))
    assert big > 4e9


def test_config_validation_returns_errors_before_device_work(L):
    so = L.load()
    h = C.c_void_p()
    cfg = L.make_config(workload("pm64"))
    assert so.pm_init(C.byref(h), C.byref(cfg), None, 0, None) == 2       # PM_ERR_WORKSPACE
    bad = L.make_config(workload("pm64", nmesh=100))                       # no FFT plan for 100
    n = C.c_size_t()
    assert so.pm_workspace_size(C.byref(bad), C.byref(n)) == 6           # PM_ERR_UNSUPPORTED
    bad = L.make_config(workload("pm64", nc=128, nmesh=64))                # B < 1
    assert so.pm_workspace_size(C.byref(bad), C.byref(n)) == 1
    bad = L.make_config(workload("pm64", zs=(12.0,)))                      # source beyond a_init
    assert so.pm_workspace_size(C.byref(bad), C.byref(n)) == 1
    assert so.pm_step(None, 0) == 1 and so.kappa_maps(None, None) == 1
    assert so.pm_strerror(5) == b"entry point called out of order"
    assert so.pm_strerror(7) == b"device-side wait for a bulk copy timed out"
    assert L.STATUS[7] == "PM_ERR_TIMEOUT"


def test_map_cl_host_validation(L):
    """pm_map_cl and its workspace query refuse bad sizes, edges and workspaces before any
    device work (the device pointers below are never dereferenced)."""
    so = L.load()
    n = C.c_size_t(0)
    assert so.pm_map_cl_workspace_size(64, 2, 8, C.byref(n)) == 0
    # work (64^2 complex) + twiddles + edges + sums + counts, each 256-byte aligned
    expect = sum(-(-b // 256) * 256 for b in (64 * 64 * 16, 32 * 16, 9 * 8, 2 * 8 * 8, 8 * 8))
    assert n.value == expect
    for args in [(48, 1, 4), (4, 1, 4), (8192, 1, 4), (64, 0, 4), (64, 1, 0), (64, 1, 2049)]:
        assert so.pm_map_cl_workspace_size(*args, C.byref(n)) == 1, args
    assert so.pm_map_cl_workspace_size(64, 1, 4, None) == 1
    fake = C.c_void_p(0x1000)

    def call(edges, npix=64, nmaps=1, fov=2.0, alpha=1.0, beta=0.0, ws=fake, nbytes=1 << 20, out=fake):
        e = (C.c_double * len(edges))(*edges)
        return so.pm_map_cl(fake, nmaps, npix, fov, C.cast(e, C.c_void_p), len(edges) - 1, alpha, beta, out,
                            None, ws, nbytes, None)
    good = [0.0, 1.0, 2.0, float("inf")]
    assert call(good, npix=96) == 1                       # not a power of two
    assert call([0.0, 2.0, 1.0]) == 1                     # not ascending
    assert call([0.0, 1.0, 1.0]) == 1                     # repeated edge
    assert call([0.0, float("nan"), 2.0]) == 1
    assert call(good, fov=-1.0) == 1
    assert call(good, alpha=float("inf")) == 1
    assert call(good, out=None) == 1
    assert call(good, ws=None) == 1
    assert call(good, nbytes=1024) == 2                   # workspace too small
    assert call(good, ws=C.c_void_p(0x1010)) == 2         # workspace not 256-byte aligned
    assert so.pm_shot_noise_maps(None, 1, fake) == 1
