#!/usr/bin/env python
"""Throughput of the GB300 particle-mesh lensing forward model.

One bench step = one whole forward simulation of the workload (initial
conditions, every kick-drift-kick step with PGD and lightcone projection, and
the final kappa maps): every row of the hot path.  The metric is particle-steps
per second = N_particles * N_steps / (seconds per simulation).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 runs under torchrun: one independent simulation per GPU (ensemble
sharding, no data-path collective; "scaling": "weak"), value = the particle
steps of all ranks / the slowest rank's time.  `--impl reference` times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s fwd and fwd+adjoint at 256^3 vs plain path; serve p50/p99 latency"
UNIT = "particle-steps/s"
WORKLOAD_DESC = {
    "pm256": "256^3 particles, 512^3 mesh, 256 Mpc/h, 2LPT at a=0.1, 40 KDK steps, PGD on, "
             "replicated lightcone to z_s in {0.5,1,1.5,2}, 2048^2 maps over 5x5 deg",
    "pm64": "64^3 particles, 64^3 mesh, 128 Mpc/h, 1LPT at a=0.1, 10 steps, z_s=1, 64^2 map over 2x2 deg",
    "pm128_vjp": "128^3 particles, 256^3 mesh, 200 Mpc/h, 20 steps, z_s=1, 1024^2 map over 4x4 deg",
    "pm512": "512^3 particles, 1024^3 mesh, 512 Mpc/h, 40 steps, 8 sources to z=2.5, 4096^2 maps, PGD on",
}


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="pm256")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nc", type=int, default=None, help="override particles per side (profiling cases)")
    ap.add_argument("--pgd", type=int, default=None, help="override PGD on/off (profiling cases)")
    ap.add_argument("--no-extra", action="store_true", help="skip the adjoint, FP64 and serving legs")
    ap.add_argument("--serve-requests", type=int, default=40)
    ap.add_argument("--cpu-single-thread", action="store_true",
                    help="also time the oracle baseline with one DFT thread")
    ap.add_argument("--leg", default="forward", choices=["forward", "adjoint"],
                    help="adjoint: each timed step is a forward run plus the reverse sweep (checkpoint "
                         "every 4 unless the workload sets one; a profiling case)")
    ap.add_argument("--large", action="store_true",
                    help="also time the 512^3-particle workload: forward, and forward + reverse sweep "
                         "checkpointed every 2 steps (269 GB of HBM)")
    return ap.parse_args()


def bench_workload(a):
    from pm_inputs import workload
    over = {}
    if a.nc is not None:
        over["nc"] = a.nc
    if a.pgd is not None:
        over["pgd"] = a.pgd
    w = workload(a.workload, **over)
    if getattr(a, "leg", "forward") == "adjoint" and not w.get("ckpt_every"):
        w["ckpt_every"] = 4
    return w


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"clocks_bench_{self.gpu}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.path:
                self.f.close()
                os.unlink(self.path)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------- CPU baseline
PROJ_SUBSET = 16          # the shell projection is timed on every 16th particle and scaled by 16
STEP_SUBSETS = (8, 16)    # kick-drift and PGD timed on every 8th and 16th particle, then fitted


class OracleSample:
    """The FP64 oracle as it stands on the work of one lightcone step of the
    workload (the metric's unit of work, particle-steps, comes from whole steps):
    a kick-drift step with the PM force on the workload's mesh, the PGD
    displacement at the new positions, and the projection of one mid-lightcone
    shell onto the workload's maps.  Kick-drift and PGD are timed with 1/8 and
    1/16 of the particles on the full mesh and extrapolated to all particles by
    the affine fit t = a + b N (the mesh work is the same, CIC paint and readout
    are linear in N; when noise makes the fit unphysical, the larger subset is
    scaled in proportion, an upper bound on the time); the projection is timed
    on 1/PROJ_SUBSET of the particles and scaled (linear in N).  `workers`: the
    threads the oracle's DFTs may use (its elementwise numpy work is
    single-threaded either way)."""

    def __init__(self, w, seed=0, workers=1):
        from oracle import dft
        from oracle.cosmology import Cosmology
        from oracle.lightcone import LensGeometry
        from oracle.lpt import lattice
        from oracle.nbody import PMState, Stepper, kdk_step, pgd_displacement
        self._kdk, self._pgd, self._state = kdk_step, pgd_displacement, PMState
        dft.set_workers(workers)
        self.w, self.workers = w, workers
        rng = np.random.default_rng(seed)
        self.nc, self.M, self.L = w["nc"], w["nmesh"], w["box"]
        self.npart = self.nc ** 3
        cosmo = Cosmology(w["omega_m"], w["sigma8"], w["h"], w["n_s"], w["omega_b"], w["t_cmb"])
        self.st = Stepper(cosmo, w["a_init"], w["nsteps"])
        self.geom = LensGeometry(cosmo, self.st, w["zs"], w["map_npix"], w["map_fov_deg"], self.L, self.nc, self.M,
                                 rotate=w.get("rotate", 1), seed=w.get("rotation_seed", 42),
                                 sub_evolution=w.get("sub_evolution", 1))
        self.active = [i for i in range(w["nsteps"]) if self.geom.active(i)]
        self.i = self.active[len(self.active) // 2]
        self.x = np.mod(lattice(self.nc, self.L, self.M) + rng.normal(0, 1.0, size=(self.npart, 3)), self.L)
        self.p = rng.normal(0, 1.0, size=(self.npart, 3))
        self.f = rng.normal(0, 1.0, size=(self.npart, 3))
        self.S = rng.normal(0, 0.1, size=(self.npart, 3))
        self.t = {}      # component -> extrapolated seconds
        self.fits = {}

    def _extrapolate(self, name, ts, ns):
        b = (ts[0] - ts[1]) / (ns[0] - ns[1])
        a = ts[0] - b * ns[0]
        if b > 0 and a > 0:
            self.fits[name] = "affine"
            return a + b * self.npart
        self.fits[name] = "proportional"
        return ts[0] * self.npart / ns[0]

    def kick_drift(self):
        i, ts, ns = self.i, [], []
        for sub in STEP_SUBSETS:
            sl = slice(0, None, sub)
            t0 = time.perf_counter()
            self._kdk(self._state(self.x[sl], self.p[sl], self.f[sl]), i, self.st, self.nc, self.M, self.L)
            ts.append(time.perf_counter() - t0)
            ns.append(len(self.x[sl]))
        self.t["kick_drift"] = self._extrapolate("kick_drift", ts, ns)

    def pgd(self):
        if not self.w.get("pgd"):
            self.t["pgd"] = 0.0
            return
        i, ts, ns = self.i, [], []
        for sub in STEP_SUBSETS:
            sl = slice(0, None, sub)
            t0 = time.perf_counter()
            self._pgd(self.x[sl], self.st.a[i + 1], self.nc, self.M, self.L, self.w["pgd_params"])
            ts.append(time.perf_counter() - t0)
            ns.append(len(self.x[sl]))
        self.t["pgd"] = self._extrapolate("pgd", ts, ns)

    def projection(self):
        sl = slice(0, None, PROJ_SUBSET)
        t0 = time.perf_counter()
        self.geom.project(self.i, self.x[sl], self.p[sl], self.S[sl] if self.w.get("pgd") else None)
        self.t["projection"] = PROJ_SUBSET * (time.perf_counter() - t0)

    def warm(self):
        """Untimed pass on 1/32 of the particles: the mesh-sized arrays' memory is touched once."""
        sl = slice(0, None, 32)
        self._kdk(self._state(self.x[sl], self.p[sl], self.f[sl]), self.i, self.st, self.nc, self.M, self.L)
        if self.w.get("pgd"):
            self._pgd(self.x[sl], self.st.a[self.i + 1], self.nc, self.M, self.L, self.w["pgd_params"])

    COMPONENTS = ("kick_drift", "pgd", "projection")

    def run(self, component):
        getattr(self, component)()

    def rate(self):
        """Particle-steps/s of a whole simulation: plain steps outside the lightcone, lightcone steps inside."""
        w = self.w
        t_sim = w["nsteps"] * self.t["kick_drift"] + len(self.active) * (self.t["pgd"] + self.t["projection"])
        return self.npart * w["nsteps"] / t_sim, t_sim

    def describe(self, dt):
        w, t = self.w, self.t
        return (f"FP64 oracle, the work of one lightcone step of {w['nc']}^3 particles on the {w['nmesh']}^3 mesh: "
                f"kick-drift with the PM force ({t.get('kick_drift', 0):.1f} s), PGD ({t.get('pgd', 0):.1f} s) and "
                f"one shell projected onto {len(w['zs'])} {w['map_npix']}^2 maps ({t.get('projection', 0):.1f} s), "
                f"extrapolated to all particles from timings with 1/8 and 1/16 of them (kick-drift, PGD: "
                f"{self.fits.get('kick_drift', '-')}/{self.fits.get('pgd', '-')}) or 1/{PROJ_SUBSET} (projection, "
                f"linear); rate for a whole simulation of {w['nsteps']} steps ({len(self.active)} in the lightcone); "
                f"DFTs on {self.workers} thread(s), elementwise numpy single-threaded; {dt:.1f} s of timing")


def cpu_baseline_sample(w, seed=0, workers=1):
    """One whole oracle sample (all three components); returns (particle-steps/s, seconds, sample)."""
    smp = OracleSample(w, seed, workers)
    smp.warm()
    t0 = time.perf_counter()
    for comp in OracleSample.COMPONENTS:
        smp.run(comp)
    dt = time.perf_counter() - t0
    return smp.rate()[0], dt, smp


def run_reference(a, rank, world):
    """The oracle on the host cores.  Each step times one component of the lightcone step's
    work in rotation (kick-drift, PGD, projection), so that a step stays at ~20 s; the rate
    combines the mean time of each component (components no timed step reached are timed
    once after the steps)."""
    if rank != 0:
        return
    w = bench_workload(a)
    cores = os.cpu_count() or 1
    smp = OracleSample(w, workers=cores)
    smp.warm()
    comps = OracleSample.COMPONENTS
    for k in range(a.warmup):
        smp.run(comps[k % 3])
    acc = {c: [] for c in comps}
    t0 = time.perf_counter()
    for k in range(a.steps):
        smp.run(comps[k % 3])
        acc[comps[k % 3]].append(smp.t[comps[k % 3]])
    for c in comps:
        if not acc[c]:
            smp.run(c)
            acc[c].append(smp.t[c])
    dt = time.perf_counter() - t0
    for c in comps:
        smp.t[c] = float(np.mean(acc[c]))
    v, t_sim = smp.rate()
    sample = smp.describe(dt)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_sim * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{a.workload}: {WORKLOAD_DESC.get(a.workload, '')}",
                       "sample": "each step one component of the lightcone step in rotation; " + sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------- ranks (replicas only)
def rank_noise_seed(w, rank):
    """Every rank runs its own independent simulation (ensemble sharding): rank r draws the
    white noise of seed noise_seed + r; nothing is exchanged on the data path."""
    return w["noise_seed"] + rank


def max_over_ranks(x, dist=None, device=None):
    """The slowest rank's time: an all-reduce MAX of one number (no-op on one rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, npart, nsteps, ms):
    """Whole-job particle-steps per second: all ranks' particle steps over the slowest rank's time."""
    return world * npart * nsteps / (ms * 1e-3)


# ------------------------------------------------------------- GPU arm
def run_gpu(a, rank, world, local_rank):
    import torch

    from paper_2012_07266_gb300.api import PM_FP32, PM_FP64, Simulation
    from pm_inputs import white_noise

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    w = bench_workload(a)
    prec = PM_FP64 if a.precision == "fp64" else PM_FP32
    stream = torch.cuda.Stream(dev)
    sim = Simulation(device=dev, stream=stream, precision=prec, **w)
    noise = torch.from_numpy(white_noise(w["nc"], rank_noise_seed(w, rank))).to(dev)
    npart, nsteps = w["nc"] ** 3, w["nsteps"]

    lam = None
    if a.leg == "adjoint":
        lam = torch.ones((sim.n_zs, sim.npix, sim.npix), dtype=torch.float64, device=dev)

    def one():
        sim.run(noise)  # kappa_maps synchronises the stream
        if lam is not None:
            sim.vjp(lam)

    for _ in range(a.warmup):
        one()
    sim.profile_read()
    sim.profile(True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(a.steps):
        one()
    ev1.record(stream)
    ev1.synchronize()
    barrier()
    clk = clocks.stop()
    sim.profile(False)
    prof = sim.profile_read()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / a.steps, dist, dev)
    value = aggregate_rate(world, npart, nsteps, ms)
    launches = sum(v[1] for v in prof.values())

    # end to end through the public API with host buffers (pinned)
    e2e = None
    if not a.no_e2e:
        h_noise = torch.from_numpy(white_noise(w["nc"], rank_noise_seed(w, rank))).pin_memory()
        h_kappa = torch.empty((sim.n_zs, sim.npix, sim.npix), dtype=torch.float64).pin_memory()
        d_noise = torch.empty_like(h_noise, device=dev)
        d_kappa = torch.empty((sim.n_zs, sim.npix, sim.npix), dtype=torch.float64, device=dev)

        def one_e2e():
            with torch.cuda.stream(stream):
                d_noise.copy_(h_noise, non_blocking=True)
                sim.ic(d_noise)
                for i in range(nsteps):
                    sim.step(i)
                    sim.lens_project(i)
                sim.kappa_maps(d_kappa)
                h_kappa.copy_(d_kappa, non_blocking=True)
            stream.synchronize()

        one_e2e()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            one_e2e()
        e1.record(stream)
        e1.synchronize()
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1) / a.steps, dist, dev)
        e2e = {"value": aggregate_rate(world, npart, nsteps, ems), "unit": UNIT,
               "h2d_bytes_per_step": h_noise.numel() * 8, "d2h_bytes_per_step": h_kappa.numel() * 8}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peak, peak_src = peaks()
    kern = {}
    for k, (kms, n, b) in prof.items():
        if n == 0:
            continue
        kern[k] = {"launches": n, "ms_total": round(kms, 3),
                   "ms_per_launch": round(kms / n, 4) if kms else None,
                   "gbs": round(b / (kms * 1e-3) / 1e9, 1) if kms > 0 and b > 0 else None,
                   "share": None}
    tot = sum(v["ms_total"] for v in kern.values())
    for v in kern.values():
        v["share"] = round(v["ms_total"] / tot, 4) if tot else None
    dom = max((k for k in kern if prof[k][2] > 0), key=lambda k: kern[k]["ms_total"])
    dms, dn, db = prof[dom]
    achieved = db / dn / (dms / dn * 1e-3) / 1e9
    traffic = read_traffic(dom, a.workload)
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_src,
            "algo_bytes_per_launch": db / dn, "traffic": traffic}
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        cores = os.cpu_count() or 1
        v, dt, smp = cpu_baseline_sample(w, workers=cores)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": smp.describe(dt)}
        if a.cpu_single_thread:
            v1, dt1, smp1 = cpu_baseline_sample(w, workers=1)
            cpu["single_thread"] = {"value": v1, "cores": 1, "sample": smp1.describe(dt1)}
    extra = {} if (a.no_extra or world > 1) else extra_legs(a, w, dev, rank, ms)
    ws_gb = sim.nbytes / 1e9
    if a.large and world == 1:
        del sim
        torch.cuda.empty_cache()
        extra["large"] = large_leg(dev)
    # whole-simulation roofline against the byte model of the path, R = 4 M^3, C = 8 M^2 (M/2 + 1):
    # every KDK step (paint, forward FFT, three inverse FFTs with the fused Poisson/gradient,
    # readout + kick, drift) 9 R + 20 C + 100 N_p; every lightcone step adds PGD (three inverse
    # FFTs and the readout of three meshes) 3 (5 C + R) + 3 R + 12 N_p and the projection's read
    # of the particle state 28 N_p
    M = w["nmesh"]
    R_, C_ = 4.0 * M ** 3, 8.0 * M * M * (M // 2 + 1)
    kdk_bytes = 9 * R_ + 20 * C_ + 100.0 * npart
    n_lens = prof.get("lens_project", (0, 0, 0))[1] // max(a.steps, 1)
    lens_bytes = (3 * (5 * C_ + R_) + 3 * R_ + 12.0 * npart if w.get("pgd") else 0.0) + 28.0 * npart
    sim_bytes = nsteps * kdk_bytes + n_lens * lens_bytes
    at_peak = peak * 1e9 / sim_bytes * npart * nsteps
    model = {"bytes_per_kdk_step_gb": round(kdk_bytes / 1e9, 2), "bytes_per_lightcone_step_extra_gb":
             round(lens_bytes / 1e9, 2), "lightcone_steps": n_lens, "bytes_per_simulation_gb": round(sim_bytes / 1e9, 1),
             "ms_per_simulation_at_peak": round(sim_bytes / (peak * 1e9) * 1e3, 2),
             "particle_steps_per_s_at_peak": at_peak, "frac": round(value / (world * at_peak), 4),
             "peak_gbs": peak, "peak_source": peak_src}
    maps_per_hour = world * 3600.0 / (ms * 1e-3) * len(w["zs"])  # one map per source plane
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == PM_FP32 else "f64", "data": "synthetic",
            "config": {"workload": f"{a.workload}: {WORKLOAD_DESC.get(a.workload, '')}",
                       "step": "one whole forward simulation (IC, all KDK steps, PGD, lightcone, kappa)"
                               + (" and its reverse sweep (profiling leg)" if a.leg == "adjoint" else ""),
                       "l2": "inputs larger than L2 (workspace %.1f GB)" % ws_gb,
                       "parallelism": f"replicas x{world}"},
            "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "cpu_baseline": cpu, "kernels": kern, "step_roofline_model": model,
            "kappa_maps_per_hour": maps_per_hour, **extra}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def extra_legs(a, w, dev, rank, forward_ms):
    """Forward + adjoint at the same workload, forward mode, the plain FP64
    path, the shot-noise estimate, and the serving mix (Poisson arrivals, mixed
    sizes and cosmologies)."""
    import torch

    from paper_2012_07266_gb300.api import PM_FP32, PM_FP64, Simulation
    from pm_inputs import serving_arrivals, white_noise, workload
    out = {}
    npart, nsteps = w["nc"] ** 3, w["nsteps"]
    noise = torch.from_numpy(white_noise(w["nc"], rank_noise_seed(w, rank))).to(dev)
    # forward + reverse-mode derivative: resident (every step's state and meshes kept in HBM,
    # no recompute) and checkpointed every 4 steps (one recompute of each segment)
    stream = torch.cuda.Stream(dev)

    def time_fwd_adj(ckpt):
        sim = Simulation(device=dev, stream=stream, precision=PM_FP32, **dict(w, ckpt_every=ckpt))
        k = sim.run(noise)
        lam = k.clone()
        sim.vjp(lam)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        reps = 2
        t_f = t_fa = 0.0
        for _ in range(reps):
            e0.record(stream)
            k = sim.run(noise)
            e1.record(stream)
            sim.vjp(lam)
            e2.record(stream)
            e2.synchronize()
            t_f += e0.elapsed_time(e1)
            t_fa += e0.elapsed_time(e2)
        t_f, t_fa = t_f / reps, t_fa / reps
        # kernel classes of one reverse sweep (library CUDA-event profile)
        sim.run(noise)
        sim.profile_read()
        sim.profile(True)
        sim.vjp(lam)
        sim.profile(False)
        classes = {kk: {"ms": round(v[0], 2), "launches": v[1]} for kk, v in sim.profile_read().items() if v[1]}
        gb = sim.nbytes / 1e9
        del sim
        torch.cuda.empty_cache()
        # the reverse sweep's time, against this leg's forward and against the main timed forward
        # (the leg times two runs only, so its forward carries more run-to-run spread)
        return {"value": npart * nsteps / (t_fa * 1e-3), "unit": UNIT, "ms_per_step": t_fa, "forward_ms": t_f,
                "adjoint_ms": t_fa - t_f, "adjoint_over_forward": (t_fa - t_f) / t_f,
                "adjoint_over_main_forward": (t_fa - t_f) / forward_ms, "checkpoint_every": ckpt,
                "workspace_gb": gb, "adjoint_kernel_classes": classes}, k

    out["fwd_adjoint"], k = time_fwd_adj(nsteps)
    out["fwd_adjoint_ckpt4"], _ = time_fwd_adj(4)
    # the differentiable workload at its own size (128^3 particles, 256^3 mesh, 20 steps, one
    # 1024^2 map, checkpoint every 4): forward + reverse sweep per request
    w3 = workload("pm128_vjp")
    sim3 = Simulation(device=dev, stream=stream, precision=PM_FP32, **w3)
    n3 = torch.from_numpy(white_noise(w3["nc"], w3["noise_seed"])).to(dev)
    lam3 = sim3.run(n3).clone()
    sim3.vjp(lam3)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t3f = t3a = 0.0
    for _ in range(3):
        e0.record(stream)
        sim3.run(n3)
        e1.record(stream)
        sim3.vjp(lam3)
        e2.record(stream)
        e2.synchronize()
        t3f += e0.elapsed_time(e1) / 3
        t3a += e0.elapsed_time(e2) / 3
    out["config3_fwd_adjoint"] = {"workload": "pm128_vjp: " + WORKLOAD_DESC["pm128_vjp"] + ", checkpoint every 4",
                                  "forward_ms": t3f, "forward_adjoint_ms": t3a, "workspace_gb": sim3.nbytes / 1e9,
                                  "value": w3["nc"] ** 3 * w3["nsteps"] / (t3a * 1e-3), "unit": UNIT}
    del sim3
    torch.cuda.empty_cache()
    # forward-mode derivative along a noise direction (one whole run with the tangent)
    sim = Simulation(device=dev, stream=stream, precision=PM_FP32, **dict(w, jvp=1))
    d = torch.from_numpy(white_noise(w["nc"], w["noise_seed"] + 1000)).to(dev)
    sim.jvp(noise, d)
    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
    e0.record(stream)
    for _ in range(2):
        sim.jvp(noise, d)
    e1.record(stream)
    e1.synchronize()
    t_j = e0.elapsed_time(e1) / 2
    out["fwd_jvp"] = {"value": npart * nsteps / (t_j * 1e-3), "unit": UNIT, "ms_per_step": t_j,
                      "jvp_over_forward": t_j / out["fwd_adjoint"]["forward_ms"], "workspace_gb": sim.nbytes / 1e9}
    del sim
    torch.cuda.empty_cache()
    kappa32 = k.clone()
    # plain FP64 path, one simulation at a time
    sim = Simulation(device=dev, stream=stream, precision=PM_FP64, **w)
    sim.run(noise)
    e0.record(stream)
    k64 = sim.run(noise)
    e1.record(stream)
    e1.synchronize()
    t64 = e0.elapsed_time(e1)
    err = float((kappa32 - k64).norm() / k64.norm())
    out["plain_fp64"] = {"value": npart * nsteps / (t64 * 1e-3), "unit": UNIT, "ms_per_step": t64,
                         "fp32_speedup": t64 / out["fwd_adjoint"]["forward_ms"], "kappa_rel_l2_fp32_vs_fp64": err}
    del sim
    torch.cuda.empty_cache()
    # shot-noise estimate (Sec. 4): random-position runs through the whole lightcone and the
    # binned spectra of their maps (30 logarithmic bins, 100 <= l < 40000, plus l < 100)
    sim = Simulation(device=dev, stream=stream, precision=PM_FP32, **w)
    edges = np.concatenate([[0.0], np.geomspace(100.0, 40000.0, 30)])
    m = sim.shot_noise_maps(0)
    sim.cl(m, edges)
    e2 = torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for r in range(reps):
        m = sim.shot_noise_maps(r + 1)
    e1.record(stream)
    for r in range(reps):
        sim.cl(m, edges)
    e2.record(stream)
    e2.synchronize()
    t_run, t_cl = e0.elapsed_time(e1) / reps, e1.elapsed_time(e2) / reps
    out["shot_noise"] = {"run_ms": t_run, "cl_ms": t_cl, "maps": len(w["zs"]),
                         "npix": w["map_npix"], "bins": len(edges) - 1,
                         "run_over_forward": t_run / out["fwd_adjoint"]["forward_ms"]}
    del sim
    torch.cuda.empty_cache()
    # serving mix: Poisson arrivals at 20/s, meshes 64/128/192 (nc = mesh/2)
    from paper_2012_07266_gb300.serve import Server, make_requests
    base = workload("pm64", box=256.0, map_npix=512, map_fov_deg=5.0, pgd=0, lpt_order=1)
    specs = serving_arrivals(a.serve_requests, rate_hz=20.0, seed=7)
    warm = make_requests(specs[:3], base)
    for r in warm:
        r.t_arrive = 0.0
    Server(device=dev, max_slots=8).serve(warm)
    reqs = make_requests(specs, base)
    st = Server(device=dev, max_slots=8).serve(reqs)
    out["serve"] = dict(st.summary(), requests=len(reqs), arrival_rate_hz=20.0,
                        adjoint_fraction=float(np.mean([r.adjoint for r in reqs])),
                        failed=sum(r.error is not None for r in reqs))
    return out


def large_leg(dev):
    """The 512^3-particle workload (1024^3 mesh, 8 sources to z = 2.5, 4096^2 maps, PGD): one
    timed forward after a warm-up run, then the forward + reverse sweep with a checkpoint every
    2 steps if its workspace fits the device."""
    import torch

    from paper_2012_07266_gb300.api import PM_FP32, Simulation
    from pm_inputs import white_noise, workload
    w = workload("pm512")
    out = {"workload": "pm512: " + WORKLOAD_DESC["pm512"]}
    stream = torch.cuda.Stream(dev)
    noise = torch.from_numpy(white_noise(w["nc"], w["noise_seed"])).to(dev)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    sim = Simulation(device=dev, stream=stream, precision=PM_FP32, **w)
    sim.run(noise)
    e0.record(stream)
    sim.run(noise)
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1)
    out["forward"] = {"ms": t, "value": w["nc"] ** 3 * w["nsteps"] / (t * 1e-3), "unit": UNIT,
                      "workspace_gb": sim.nbytes / 1e9}
    del sim
    torch.cuda.empty_cache()
    try:
        sim = Simulation(device=dev, stream=stream, precision=PM_FP32, **dict(w, ckpt_every=2))
        lam = sim.run(noise).clone()
        e0.record(stream)
        sim.run(noise)
        e1.record(stream)
        sim.vjp(lam)
        e2.record(stream)
        e2.synchronize()
        out["forward_adjoint_ckpt2"] = {"forward_ms": e0.elapsed_time(e1), "ms": e0.elapsed_time(e2),
                                        "workspace_gb": sim.nbytes / 1e9}
        del sim
    except (RuntimeError, torch.cuda.OutOfMemoryError) as err:
        out["forward_adjoint_ckpt2"] = {"failed": str(err).splitlines()[0][:200]}
    torch.cuda.empty_cache()
    return out


def read_traffic(kernel, workload):
    """Per-launch DRAM bytes of `kernel` from a committed ncu summary, if its
    source hash still matches the current kernels (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    want = source_hash(kernel)
    for line in open(path):
        parts = line.split()
        if len(parts) == 4 and parts[0] == kernel and parts[1] == workload and parts[3] == want:
            return float(parts[2])
    return None


# the sources a kernel's device code and launch come from; a kernel not listed is
# keyed on every source
KERNEL_SOURCES = {
    "fft_x_c2r": ("fft_impl.cuh", "fft.cu"),
    "kick_drift_paint": ("particles.cu", "cic.cuh"),
}


def source_hash(kernel=None):
    """SHA-1 prefix of the sources of `kernel` (all CUDA/C++ sources if None or unlisted):
    a committed DRAM-traffic figure is used only while it still matches."""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2012_07266_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) or [f for f in os.listdir(d) if f.endswith((".cu", ".cuh", ".h", ".cpp"))]
    for f in sorted(files):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:12]


def main():
    a = args_()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
    else:
        run_gpu(a, rank, world, local_rank)


if __name__ == "__main__":
    main()
