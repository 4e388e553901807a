"""Python API over the C ABI: PyTorch supplies device memory and the stream.

    sim = Simulation(**workload)           # pm_init on torch-allocated workspace
    kappa = sim.run(noise)                 # pm_ic, pm_step / lens_project, kappa_maps

    model = KappaModel(**workload)         # differentiable: torch.autograd reaches pm_vjp
    kappa = model(noise, cosmo)            # cosmo = tensor([Omega_m, sigma_8])
    loss(kappa).backward()                 # noise.grad, cosmo.grad

All arithmetic runs in libpmlens.so kernels; this module only allocates
buffers, marshals pointers and sequences the calls.

Streams: a Simulation enqueues its work on its own stream (given, or the
current stream at construction).  Every call that reads a caller's tensor first
makes that stream wait for the caller's current stream; every tensor it returns
is allocated on the caller's current stream, recorded as used by the
simulation's stream, and the current stream is made to wait for the
simulation's stream before the call returns.  So a caller may use the results
on its current stream at once, and free them whenever it likes.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import lib
from .lib import PM_FP32, PM_FP64, make_config  # noqa: F401


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def map_cl(maps: torch.Tensor, fov_deg: float, edges, alpha=1.0, beta=0.0, out=None, stream=None,
           return_counts=False):
    """Binned flat-sky angular power spectrum of maps (..., npix, npix) on their
    GPU (pm_map_cl): out = beta * out + alpha * C(l) per map and bin; with
    return_counts also the number of modes per bin.  Every device step (a float64
    copy of the maps when one is needed, the workspace, the output) runs on
    `stream` (default: the current stream), after the caller's current stream;
    the current stream waits for the result before this returns."""
    if not maps.is_cuda or maps.dim() < 2 or maps.shape[-1] != maps.shape[-2]:
        raise ValueError("map_cl: maps must be a CUDA tensor of shape (..., npix, npix)")
    if out is None and beta != 0.0:
        raise ValueError("map_cl: beta != 0 accumulates into out, which must then be given")
    cur = torch.cuda.current_stream(maps.device)
    stream = stream if stream is not None else cur
    if stream != cur:
        stream.wait_stream(cur)
    fresh = out is None
    with torch.cuda.stream(stream):
        m64 = maps.to(dtype=torch.float64).contiguous()
        m64.record_stream(stream)
        npix = int(m64.shape[-1])
        nmaps = m64.numel() // (npix * npix)
        edges = [float(e) for e in edges]
        nb = len(edges) - 1
        n = C.c_size_t(0)
        lib.call("pm_map_cl_workspace_size", npix, nmaps, nb, C.byref(n))
        ws = torch.empty(int(n.value), dtype=torch.uint8, device=m64.device)
        if fresh:
            # beta = 0: the library writes every entry
            out = torch.empty(tuple(m64.shape[:-2]) + (nb,), dtype=torch.float64, device=m64.device)
        elif (out.device != m64.device or out.dtype != torch.float64 or not out.is_contiguous()
              or out.numel() != nmaps * nb):
            raise ValueError("map_cl: out must be a contiguous float64 tensor of nmaps x nbins on the maps' device")
        else:
            out.record_stream(stream)
        eh = (C.c_double * (nb + 1))(*edges)
        counts = (C.c_int64 * nb)() if return_counts else None
        lib.call("pm_map_cl", _ptr(m64), nmaps, npix, float(fov_deg), C.cast(eh, C.c_void_p), nb, float(alpha),
                 float(beta), _ptr(out), C.cast(counts, C.c_void_p) if counts is not None else None, _ptr(ws),
                 C.c_size_t(n.value), C.c_void_p(stream.cuda_stream))
    if stream != cur:
        cur.wait_stream(stream)
        if fresh:
            out.record_stream(cur)
    return (out, [int(v) for v in counts]) if return_counts else out


class Simulation:
    """One forward (and optionally adjoint) lensing simulation on one GPU."""

    def __init__(self, device=None, stream=None, precision=PM_FP32, **workload):
        lib.load()
        self.device = torch.device(device or "cuda")
        self.w = dict(workload)
        self.cfg = make_config(workload, precision)
        self.nbytes = lib.workspace_size(self.cfg)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.runs = 0  # forward runs started (pm_ic calls); pm_vjp differentiates the latest
        # the workspace belongs to the simulation's stream (all its use is there)
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
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
                # kernels still queued on the stream use the workspace: let them finish
                # before the context and the workspace go
                self.stream.synchronize()
                lib.load().pm_destroy(ctx)
            except Exception:
                pass
            self.ctx = None

    def _after_caller(self):
        """The simulation's stream waits for the caller's current stream (inputs and
        freshly allocated outputs are ready before the library touches them)."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _before_caller(self):
        """The caller's current stream waits for the simulation's stream (results
        written by the library are complete for the caller's next work)."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def _call(self, fn, *args):
        """An entry point that reads or writes caller tensors, ordered both ways."""
        self._after_caller()
        lib.call(fn, *args)
        self._before_caller()

    def _f64(self, *shape):
        """An output buffer on the caller's current stream, marked as used by ours."""
        t = torch.empty(*shape, dtype=torch.float64, device=self.device)
        t.record_stream(self.stream)
        return t

    def _in64(self, t: torch.Tensor) -> torch.Tensor:
        """t as a contiguous float64 tensor on the device.  The conversion, when one
        is needed, runs on this simulation's stream after the caller's pending work;
        the result is marked as used by this stream, so that its memory is not
        reused while the library still reads it."""
        self._after_caller()
        with torch.cuda.stream(self.stream):
            u = t.to(device=self.device, dtype=torch.float64).contiguous()
        u.record_stream(self.stream)
        return u

    # -- the method's entry points
    def ic(self, noise: torch.Tensor):
        noise = self._in64(noise)
        self._noise = noise  # kept alive until the stream has consumed it
        self.runs += 1
        lib.call("pm_ic", self.ctx, _ptr(noise))

    def step(self, i: int):
        lib.call("pm_step", self.ctx, int(i))

    def lens_project(self, i: int):
        lib.call("lens_project", self.ctx, int(i))

    def kappa_maps(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = self._f64(self.n_zs, self.npix, self.npix)
        elif (not out.is_cuda or out.dtype != torch.float64 or not out.is_contiguous()
              or out.numel() != self.n_zs * self.npix * self.npix):
            raise ValueError("kappa_maps: out must be a contiguous float64 (n_zs, npix, npix) tensor on the device")
        else:
            out.record_stream(self.stream)
        self._call("kappa_maps", self.ctx, _ptr(out))
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
        noise = self._in64(noise)
        dnoise = self._in64(dnoise)
        self._noise = (noise, dnoise)  # kept alive until the stream has consumed them
        kappa = self._f64(self.n_zs, self.npix, self.npix)
        dkappa = self._f64(self.n_zs, self.npix, self.npix)
        self.runs += 1
        self._call("pm_jvp", self.ctx, _ptr(noise), _ptr(dnoise), _ptr(kappa), _ptr(dkappa))
        return kappa, dkappa

    def vjp(self, dL_dkappa: torch.Tensor, want_noise=True):
        g = self._in64(dL_dkappa)
        dn = self._f64(self.nc, self.nc, self.nc) if want_noise else None
        hp = (C.c_double * 2)()
        self._call("pm_vjp", self.ctx, _ptr(g), _ptr(dn), C.cast(hp, C.c_void_p))
        return dn, (hp[0], hp[1])

    # -- shot noise (Sec. 4)
    def shot_noise_maps(self, seed: int) -> torch.Tensor:
        """Maps of one shot-noise run with uniformly random particles; replaces the
        particle state (pm_ic starts the next simulation)."""
        out = self._f64(self.n_zs, self.npix, self.npix)
        self._call("pm_shot_noise_maps", self.ctx, C.c_uint64(int(seed)), _ptr(out))
        return out

    def cl(self, maps: torch.Tensor, edges, **kw) -> torch.Tensor:
        """Binned C(l) of maps of this field of view (see map_cl)."""
        return map_cl(maps, self.cfg.map_fov_deg, edges, stream=self.stream, **kw)

    def shot_noise_cl(self, edges, seeds) -> torch.Tensor:
        """Mean binned C(l) of the shot-noise runs with the given seeds."""
        seeds = list(seeds)
        out = None
        for k, sd in enumerate(seeds):
            out = self.cl(self.shot_noise_maps(sd), edges, alpha=1.0 / len(seeds), beta=0.0 if k == 0 else 1.0,
                          out=out)
        return out

    def cl_minus_shot_noise(self, kappa: torch.Tensor, edges, seeds) -> torch.Tensor:
        """C(l) of the maps kappa minus the mean C(l) of shot-noise runs (Sec. 4,
        Fig. accuracy); the runs replace the particle state."""
        seeds = list(seeds)
        out = self.cl(kappa, edges)
        for sd in seeds:
            self.cl(self.shot_noise_maps(sd), edges, alpha=-1.0 / len(seeds), beta=1.0, out=out)
        return out

    # -- state transfer / inspection
    def particles(self):
        x, p = self._f64(self.np, 3), self._f64(self.np, 3)
        self._call("pm_get_particles", self.ctx, _ptr(x), _ptr(p))
        return x, p

    def set_particles(self, x: torch.Tensor, p: torch.Tensor, next_step: int):
        x = self._in64(x)
        p = self._in64(p)
        self._keep = (x, p)
        self._call("pm_set_particles", self.ctx, _ptr(x), _ptr(p), int(next_step))

    def forces(self):
        f = self._f64(self.np, 3)
        self._call("pm_get_forces", self.ctx, _ptr(f))
        return f

    def pgd(self):
        s = self._f64(self.np, 3)
        self._call("pm_get_pgd", self.ctx, _ptr(s))
        return s

    def density(self):
        m = self.cfg.nmesh
        r = self._f64(m, m, m)
        self._call("pm_get_density", self.ctx, _ptr(r))
        return r

    def fft_r2c(self, field: torch.Tensor) -> torch.Tensor:
        m = self.cfg.nmesh
        f = self._in64(field)
        out = self._f64(m, m, m // 2 + 1, 2)
        self._call("pm_fft_r2c", self.ctx, _ptr(f), _ptr(out))
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


class KappaFn(torch.autograd.Function):
    """kappa = KappaFn.apply(noise, cosmo, model): the whole forward model as one
    differentiable operation (Sec. 3: the model is differentiable in the initial
    modes; Appendix A: and in Omega_m, sigma_8).

    noise: the nc^3 white-noise field (any float dtype, any device);
    cosmo: a tensor [Omega_m, sigma_8]; model: the KappaModel that owns the
    simulation.  Returns the float64 maps (n_zs, npix, npix) on the model's
    device.  backward runs the library's reverse sweep (pm_vjp) once: the
    gradient of the noise comes back in the noise's dtype, shape and device,
    that of cosmo as [dL/dOmega_m, dL/dsigma_8] in cosmo's dtype and device.
    A model differentiates only its latest forward run, once: a backward after
    the model has run again, or a second backward of the same run, raises."""

    @staticmethod
    def forward(ctx, noise, cosmo, model):
        om, s8 = (float(v) for v in cosmo.detach().reshape(-1).tolist())
        sim = model.simulation(om, s8)
        kappa = sim.run(noise.detach())
        ctx.model, ctx.sim, ctx.run = model, sim, sim.runs
        ctx.noise_like = (noise.shape, noise.dtype, noise.device)
        ctx.cosmo_like = (cosmo.dtype, cosmo.device)
        return kappa

    @staticmethod
    def backward(ctx, g):
        sim = ctx.sim
        if sim is None or ctx.model._sim is not sim or sim.runs != ctx.run:
            raise RuntimeError("KappaFn.backward: the model has run again since this forward (or this backward "
                               "already ran); the reverse sweep needs the state of its own forward run")
        ctx.sim = None
        want_noise = ctx.needs_input_grad[0]
        dn, (dom, ds8) = sim.vjp(g, want_noise=want_noise)
        sim.runs += 1  # the reverse sweep consumed the forward state
        dnoise = None
        if want_noise:
            shape, dtype, device = ctx.noise_like
            dnoise = dn.to(device=device, dtype=dtype).reshape(shape)
        dcosmo = None
        if ctx.needs_input_grad[1]:
            dtype, device = ctx.cosmo_like
            dcosmo = torch.tensor([dom, ds8], dtype=torch.float64).to(device=device, dtype=dtype)
        return dnoise, dcosmo, None


class KappaModel:
    """The differentiable lensing forward model of one workload on one GPU:
    kappa = model(noise, cosmo) with cosmo = [Omega_m, sigma_8] (see KappaFn).

    The library builds its cosmology tables at pm_init, so the model keeps one
    Simulation for the current (Omega_m, sigma_8) and replaces it when they
    change (the old workspace is released first).  ckpt_every defaults to the
    number of steps (the resident reverse sweep: no recompute, largest
    workspace); give a smaller interval to trade time for memory."""

    def __init__(self, device=None, stream=None, precision=PM_FP32, **workload):
        self.device = device
        self.stream = stream
        self.precision = precision
        self.w = dict(workload)
        self.w.setdefault("ckpt_every", int(self.w["nsteps"]))
        self._sim = None
        self._key = None

    def simulation(self, omega_m: float, sigma8: float) -> Simulation:
        key = (float(omega_m), float(sigma8))
        if self._sim is None or self._key != key:
            self._sim = None  # release the old context and workspace before the new one
            self._sim = Simulation(device=self.device, stream=self.stream, precision=self.precision,
                                   **dict(self.w, omega_m=key[0], sigma8=key[1]))
            self._key = key
        return self._sim

    def __call__(self, noise: torch.Tensor, cosmo: torch.Tensor) -> torch.Tensor:
        return KappaFn.apply(noise, cosmo, self)
