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
