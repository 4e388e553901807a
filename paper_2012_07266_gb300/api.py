"""Python API over the C ABI: PyTorch supplies device memory and the stream.

    sim = Simulation(**workload)           # pm_init on torch-allocated workspace
    kappa = sim.run(noise)                 # pm_ic, pm_step / lens_project, kappa_maps

All arithmetic runs in libpmlens.so kernels; this module only allocates
buffers, marshals pointers and sequences the calls.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import lib
from .lib import PM_FP32, PM_FP64, make_config  # noqa: F401


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class Simulation:
    """One forward (and optionally adjoint) lensing simulation on one GPU."""

    def __init__(self, device=None, stream=None, precision=PM_FP32, **workload):
        lib.load()
        self.device = torch.device(device or "cuda")
        self.w = dict(workload)
        self.cfg = make_config(workload, precision)
        self.nbytes = lib.workspace_size(self.cfg)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        lib.call("pm_init", C.byref(h), C.byref(self.cfg), _ptr(self.workspace), C.c_size_t(self.nbytes),
                 C.c_void_p(self.stream.cuda_stream))
        self.ctx = h
        self.nc = self.cfg.nc
        self.np = self.nc ** 3
        self.nsteps = self.cfg.nsteps
        self.n_zs = self.cfg.n_zs
        self.npix = self.cfg.map_npix
        # source planes replaced by distributions n(z): {plane index: (z, n)}
        for s, (z, n) in (workload.get("source_nz") or {}).items():
            self.set_source_nz(int(s), z, n)

    def set_source_nz(self, s: int, z, n):
        """Source plane s becomes the distribution n(z) (host arrays; see pm_set_source_nz)."""
        z = [float(v) for v in z]
        n = [float(v) for v in n]
        if len(z) != len(n):
            raise ValueError("z and n(z) differ in length")
        zt, nt = (C.c_double * len(z))(*z), (C.c_double * len(n))(*n)
        lib.call("pm_set_source_nz", self.ctx, int(s), C.cast(zt, C.c_void_p), C.cast(nt, C.c_void_p), len(z))

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and ctx.value:
            try:
                lib.load().pm_destroy(ctx)
            except Exception:
                pass
            self.ctx = None

    def _f64(self, *shape):
        return torch.empty(*shape, dtype=torch.float64, device=self.device)

    # -- the method's entry points
    def ic(self, noise: torch.Tensor):
        noise = noise.to(device=self.device, dtype=torch.float64).contiguous()
        self._noise = noise  # kept alive until the stream has consumed it
        lib.call("pm_ic", self.ctx, _ptr(noise))

    def step(self, i: int):
        lib.call("pm_step", self.ctx, int(i))

    def lens_project(self, i: int):
        lib.call("lens_project", self.ctx, int(i))

    def kappa_maps(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = self._f64(self.n_zs, self.npix, self.npix)
        lib.call("kappa_maps", self.ctx, _ptr(out))
        return out

    def run(self, noise: torch.Tensor) -> torch.Tensor:
        self.ic(noise)
        for i in range(self.nsteps):
            self.step(i)
            self.lens_project(i)
        return self.kappa_maps()

    def jvp(self, noise: torch.Tensor, dnoise: torch.Tensor):
        """(kappa, dkappa): a whole forward run from `noise` and the derivative of
        the maps along the noise direction `dnoise` (needs jvp=1 in the workload)."""
        noise = noise.to(device=self.device, dtype=torch.float64).contiguous()
        dnoise = dnoise.to(device=self.device, dtype=torch.float64).contiguous()
        self._noise = (noise, dnoise)  # kept alive until the stream has consumed them
        kappa = self._f64(self.n_zs, self.npix, self.npix)
        dkappa = self._f64(self.n_zs, self.npix, self.npix)
        lib.call("pm_jvp", self.ctx, _ptr(noise), _ptr(dnoise), _ptr(kappa), _ptr(dkappa))
        return kappa, dkappa

    def vjp(self, dL_dkappa: torch.Tensor, want_noise=True):
        g = dL_dkappa.to(device=self.device, dtype=torch.float64).contiguous()
        dn = self._f64(self.nc, self.nc, self.nc) if want_noise else None
        hp = (C.c_double * 2)()
        lib.call("pm_vjp", self.ctx, _ptr(g), _ptr(dn), C.cast(hp, C.c_void_p))
        return dn, (hp[0], hp[1])

    # -- state transfer / inspection
    def particles(self):
        x, p = self._f64(self.np, 3), self._f64(self.np, 3)
        lib.call("pm_get_particles", self.ctx, _ptr(x), _ptr(p))
        return x, p

    def set_particles(self, x: torch.Tensor, p: torch.Tensor, next_step: int):
        x = x.to(device=self.device, dtype=torch.float64).contiguous()
        p = p.to(device=self.device, dtype=torch.float64).contiguous()
        self._keep = (x, p)
        lib.call("pm_set_particles", self.ctx, _ptr(x), _ptr(p), int(next_step))

    def forces(self):
        f = self._f64(self.np, 3)
        lib.call("pm_get_forces", self.ctx, _ptr(f))
        return f

    def pgd(self):
        s = self._f64(self.np, 3)
        lib.call("pm_get_pgd", self.ctx, _ptr(s))
        return s

    def density(self):
        m = self.cfg.nmesh
        r = self._f64(m, m, m)
        lib.call("pm_get_density", self.ctx, _ptr(r))
        return r

    def fft_r2c(self, field: torch.Tensor) -> torch.Tensor:
        m = self.cfg.nmesh
        f = field.to(device=self.device, dtype=torch.float64).contiguous()
        out = self._f64(m, m, m // 2 + 1, 2)
        lib.call("pm_fft_r2c", self.ctx, _ptr(f), _ptr(out))
        return torch.view_as_complex(out)

    def sync(self):
        lib.call("pm_sync_status", self.ctx)

    def profile(self, enable: bool):
        lib.call("pm_profile", self.ctx, int(bool(enable)))

    def profile_read(self):
        """{kernel class: (ms, launches, algorithmic bytes)} since the last read (synchronises)."""
        names = lib.kernel_names()
        ms = (C.c_double * len(names))()
        n = (C.c_int64 * len(names))()
        b = (C.c_double * len(names))()
        lib.call("pm_profile_read", self.ctx, C.cast(ms, C.c_void_p), C.cast(n, C.c_void_p),
                 C.cast(b, C.c_void_p), len(names))
        return {k: (ms[i], int(n[i]), b[i]) for i, k in enumerate(names)}
