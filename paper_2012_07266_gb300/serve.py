"""Continuous-batching request loop for lensing simulations (forward or
forward + adjoint) on one GPU.

Requests (training-set generation, samplers) arrive over time with their own
mesh size, cosmology and number of steps.  The admission controller starts a
request as soon as a slot is free and its workspace (pm_workspace_size, the
HBM footprint of its particle state, meshes and maps) fits in the remaining
device-memory budget; each admitted request runs on its own CUDA stream from
its own host thread, so the kernels of all active requests overlap on the
device.  Particle state stays resident in the request's workspace for the
whole run.  Latency = completion - arrival; throughput = requests / wall time.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import lib
from .api import PM_FP32, Simulation


@dataclass
class Request:
    rid: int
    t_arrive: float
    params: dict                 # workload dict (pm_inputs names)
    noise: np.ndarray            # white noise on the nc^3 lattice (float64)
    adjoint: bool = False
    # filled by the server
    t_admit: float = 0.0
    t_done: float = 0.0
    kappa: torch.Tensor | None = None
    grad_noise: torch.Tensor | None = None
    grad_params: tuple | None = None
    error: str | None = None


@dataclass
class ServeStats:
    latencies: list = field(default_factory=list)
    wall: float = 0.0
    completed: int = 0
    max_active: int = 0
    peak_bytes: int = 0

    def summary(self):
        lat = np.asarray(self.latencies)
        return {"p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                "throughput_req_s": self.completed / self.wall if self.wall > 0 else None,
                "completed": self.completed, "max_active": self.max_active,
                "peak_workspace_gb": self.peak_bytes / 1e9}


def footprint(params: dict, precision=PM_FP32) -> int:
    """HBM bytes a request needs (its workspace)."""
    return lib.workspace_size(lib.make_config(params, precision))


class Server:
    """Admission by HBM footprint and slots; one stream + host thread per request."""

    def __init__(self, device="cuda:0", budget_bytes=None, max_slots=8, precision=PM_FP32):
        self.device = torch.device(device)
        self.precision = precision
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(0.8 * free)
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self._lock = threading.Lock()
        self._used = 0
        self._active = 0

    def _execute(self, req: Request):
        """The request's device work on its own stream: the forward run, and the
        reverse sweep when the request asks for gradients."""
        stream = torch.cuda.Stream(self.device)
        with torch.cuda.stream(stream):
            sim = Simulation(device=self.device, stream=stream, precision=self.precision, **req.params)
            noise = torch.from_numpy(req.noise).to(self.device, non_blocking=False)
            req.kappa = sim.run(noise)  # kappa_maps synchronises this request's stream
            if req.adjoint:
                # gradient of L = sum(kappa^2) / 2
                req.grad_noise, req.grad_params = sim.vjp(req.kappa)
            stream.synchronize()
            del sim

    def _run_one(self, req: Request, nbytes: int, t0: float, stats: ServeStats):
        try:
            self._execute(req)
        except Exception as e:  # the request fails, the server keeps serving
            req.error = repr(e)
        req.t_done = time.perf_counter() - t0
        with self._lock:
            self._used -= nbytes
            self._active -= 1
            if req.error is None:
                stats.latencies.append(req.t_done - req.t_arrive)
                stats.completed += 1

    def serve(self, requests: list[Request], time_scale=1.0) -> ServeStats:
        """Replay requests at their arrival times (seconds * time_scale)."""
        stats = ServeStats()
        pending = sorted(requests, key=lambda r: r.t_arrive)
        sizes = {r.rid: footprint(r.params, self.precision) for r in pending}
        for r in pending:
            if sizes[r.rid] > self.budget:
                r.error = "footprint exceeds the HBM budget"
        pending = [r for r in pending if r.error is None]
        threads = []
        t0 = time.perf_counter()
        while pending or any(t.is_alive() for t in threads):
            now = time.perf_counter() - t0
            while pending and pending[0].t_arrive * time_scale <= now:
                r = pending[0]
                with self._lock:
                    fits = self._active < self.max_slots and self._used + sizes[r.rid] <= self.budget
                    if fits:
                        self._used += sizes[r.rid]
                        self._active += 1
                        stats.max_active = max(stats.max_active, self._active)
                        stats.peak_bytes = max(stats.peak_bytes, self._used)
                if not fits:
                    break  # FIFO: wait for memory or a slot
                pending.pop(0)
                r.t_arrive *= time_scale
                r.t_admit = now
                th = threading.Thread(target=self._run_one, args=(r, sizes[r.rid], t0, stats), daemon=True)
                th.start()
                threads.append(th)
            time.sleep(0.0005)
        for t in threads:
            t.join()
        stats.wall = time.perf_counter() - t0
        return stats


def make_requests(specs: list[dict], base: dict) -> list[Request]:
    """Requests from pm_inputs.serving_arrivals specs on top of a base workload."""
    from pm_inputs import white_noise
    out = []
    for i, s in enumerate(specs):
        p = dict(base)
        p.update(nc=s["nc"], nmesh=s["nmesh"], omega_m=s["omega_m"], sigma8=s["sigma8"],
                 nsteps=s["nsteps"], zs=s["zs"])
        if s.get("adjoint"):
            p["ckpt_every"] = 4
        out.append(Request(rid=i, t_arrive=s["t_arrive"], params=p,
                           noise=white_noise(s["nc"], s["noise_seed"]), adjoint=bool(s.get("adjoint"))))
    return out
