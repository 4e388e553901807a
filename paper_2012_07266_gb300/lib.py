"""ctypes binding of the C ABI declared in include/pm.h (argument marshalling only).

Every function here forwards to libpmlens.so; no step of the model runs in
Python.  Loading fails loudly when the CUDA library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmlens.so")

PM_FP32, PM_FP64 = 0, 1
PM_MAX_ZS = 16

STATUS = {0: "PM_OK", 1: "PM_ERR_ARG", 2: "PM_ERR_WORKSPACE", 3: "PM_ERR_CUDA",
          4: "PM_ERR_NONFINITE", 5: "PM_ERR_STATE", 6: "PM_ERR_UNSUPPORTED", 7: "PM_ERR_TIMEOUT"}

# every symbol include/pm.h declares
EXPORTS = ["pm_workspace_size", "pm_init", "pm_ic", "pm_step", "lens_project", "kappa_maps",
           "pm_vjp", "pm_jvp", "pm_set_source_nz", "pm_shot_noise_maps", "pm_map_cl_workspace_size",
           "pm_map_cl", "pm_destroy", "pm_strerror", "pm_get_particles", "pm_set_particles",
           "pm_get_forces", "pm_get_pgd", "pm_fft_r2c", "pm_get_density", "pm_sync_status",
           "pm_profile", "pm_profile_read", "pm_kernel_kinds", "pm_kernel_name",
           "pm_forces_static"]


class PMConfig(C.Structure):
    """Mirror of pm_config (include/pm.h)."""
    _fields_ = [
        ("nc", C.c_int32), ("nmesh", C.c_int32), ("box", C.c_double),
        ("omega_m", C.c_double), ("sigma8", C.c_double),
        ("h", C.c_double), ("n_s", C.c_double), ("omega_b", C.c_double), ("t_cmb", C.c_double),
        ("a_init", C.c_double), ("nsteps", C.c_int32), ("lpt_order", C.c_int32),
        ("n_zs", C.c_int32), ("zs", C.c_double * PM_MAX_ZS),
        ("map_npix", C.c_int32), ("map_fov_deg", C.c_double),
        ("sub_evolution", C.c_int32), ("pgd", C.c_int32), ("pgd_params", C.c_double * 5),
        ("rotation_seed", C.c_uint64), ("rotate", C.c_int32), ("precision", C.c_int32),
        ("ckpt_every", C.c_int32), ("jvp", C.c_int32),
    ]


class PMError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} -> {STATUS.get(status, status)}")


def make_config(w: dict, precision=PM_FP32) -> PMConfig:
    """pm_config from a workload dict (names of pm_inputs.configs)."""
    c = PMConfig()
    c.nc, c.nmesh, c.box = int(w["nc"]), int(w["nmesh"]), float(w["box"])
    c.omega_m, c.sigma8 = float(w["omega_m"]), float(w["sigma8"])
    c.h, c.n_s = float(w.get("h", 0.6774)), float(w.get("n_s", 0.9667))
    c.omega_b, c.t_cmb = float(w.get("omega_b", 0.0486)), float(w.get("t_cmb", 2.7255))
    c.a_init, c.nsteps = float(w["a_init"]), int(w["nsteps"])
    c.lpt_order = int(w.get("lpt_order", 1))
    zs = list(w["zs"])
    if not 1 <= len(zs) <= PM_MAX_ZS:
        raise ValueError("1..16 source redshifts")
    c.n_zs = len(zs)
    for i, z in enumerate(zs):
        c.zs[i] = float(z)
    c.map_npix, c.map_fov_deg = int(w["map_npix"]), float(w["map_fov_deg"])
    c.sub_evolution, c.pgd = int(w.get("sub_evolution", 1)), int(w.get("pgd", 0))
    for i, v in enumerate(w.get("pgd_params", (0.0, 0.0, 0.1, 1.0, 4.0))):
        c.pgd_params[i] = float(v)
    c.rotation_seed = int(w.get("rotation_seed", 42))
    c.rotate = int(w.get("rotate", 1))
    c.precision = int(w.get("precision", precision))
    c.ckpt_every = int(w.get("ckpt_every", 0))
    c.jvp = int(w.get("jvp", 0))
    return c


_lib = None


def load():
    """Load libpmlens.so and declare the prototypes; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    import torch  # noqa: F401  (loads the same CUDA runtime the library links against)
    lib = C.CDLL(LIB_PATH)
    vp, i32, st = C.c_void_p, C.c_int32, C.c_int
    proto = {
        "pm_workspace_size": [C.POINTER(PMConfig), C.POINTER(C.c_size_t)],
        "pm_init": [C.POINTER(vp), C.POINTER(PMConfig), vp, C.c_size_t, vp],
        "pm_ic": [vp, vp],
        "pm_step": [vp, i32],
        "lens_project": [vp, i32],
        "kappa_maps": [vp, vp],
        "pm_vjp": [vp, vp, vp, vp],
        "pm_jvp": [vp, vp, vp, vp, vp],
        "pm_set_source_nz": [vp, i32, vp, vp, i32],
        "pm_shot_noise_maps": [vp, C.c_uint64, vp],
        "pm_map_cl_workspace_size": [i32, i32, i32, C.POINTER(C.c_size_t)],
        "pm_map_cl": [vp, i32, i32, C.c_double, vp, i32, C.c_double, C.c_double, vp, vp, vp, C.c_size_t, vp],
        "pm_destroy": [vp],
        "pm_get_particles": [vp, vp, vp],
        "pm_set_particles": [vp, vp, vp, i32],
        "pm_get_forces": [vp, vp],
        "pm_get_pgd": [vp, vp],
        "pm_fft_r2c": [vp, vp, vp],
        "pm_get_density": [vp, vp],
        "pm_sync_status": [vp],
        "pm_profile": [vp, i32],
        "pm_profile_read": [vp, vp, vp, vp, i32],
        "pm_forces_static": [vp, C.c_int64, i32, C.c_double, C.c_double, vp, vp],
    }
    for name, args in proto.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = st
    lib.pm_strerror.argtypes = [st]
    lib.pm_strerror.restype = C.c_char_p
    lib.pm_kernel_kinds.argtypes = []
    lib.pm_kernel_kinds.restype = i32
    lib.pm_kernel_name.argtypes = [i32]
    lib.pm_kernel_name.restype = C.c_char_p
    _lib = lib
    return lib


def check(fn: str, status: int):
    if status != 0:
        raise PMError(fn, status)


def call(fn: str, *args):
    """Call an entry point and raise PMError on a non-zero status."""
    check(fn, getattr(load(), fn)(*args))


def workspace_size(cfg: PMConfig) -> int:
    n = C.c_size_t(0)
    call("pm_workspace_size", C.byref(cfg), C.byref(n))
    return int(n.value)


def kernel_names():
    so = load()
    return [so.pm_kernel_name(k).decode() for k in range(so.pm_kernel_kinds())]
