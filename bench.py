#!/usr/bin/env python
"""Benchmark of the fluctuating D2Q9 step on GB300: MLUPS and fraction of the HBM roofline.

Workload (one GPU): a single periodic 4096 x 4096 FP32 lattice, rho0 = 1, tau_s = 0.8,
tau_b = 1, tau_ghost = 1, kT = 1e-4, cs2 = 1/3, radially binned S(k) and velocity spectra
accumulated in FP64 on the device every 100 steps.  The main line runs the long-wavelength
noise at kappa = 0.01; the correlated (full FDT) noise at kappa = 0.05 is measured in the
same run and reported under "variants".  A step is one time step of every node (pull,
density stencil, equilibrium, MRT relaxation, noise, back-transform, store) plus, every
100th step, the spectra sample.  Inputs (2 x 614 MB of populations) are larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

(--n, --noise full, --no-variants, --no-cpu-baseline and --batched-only select smaller or
other runs for profiling.)

With N > 1 (launched by torch.distributed.run) every rank steps its own independent
lattice (replicas; the method has no exchange between independent runs): weak scaling.
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_NODE_STEP = 72          # 9 FP32 populations read + 9 written
BYTES_PER_NODE_STEP_FULL = 80     # + the (xi_4, xi_9) FP32 pair read by the step kernel
BYTES_PER_NODE_STEP_FP16 = 36     # 9 FP16 populations read + 9 written
PARAMS_LW = dict(kT=1e-4, kappa=0.01, tau_s=0.8, tau_b=1.0, tau_ghost=1.0)
PARAMS_FULL = dict(kT=1e-4, kappa=0.05, tau_s=0.8, tau_b=1.0, tau_ghost=1.0)


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's independent lattice: replicas differ only in their Philox key."""
    return base_seed + 1000 * rank


def whole_job_mlups(world: int, nodes: int, steps: int, ms_max: float) -> float:
    """Node updates of all ranks per second (MLUPS), timed by the slowest rank."""
    return world * nodes * steps / (ms_max / 1e3) / 1e6


def max_over_ranks(dist, value: float, device) -> float:
    """The largest value over all ranks (no collective when running alone)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=4096, help="lattice side")
    p.add_argument("--every", type=int, default=100)
    p.add_argument("--nbins", type=int, default=2048)
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--batched-only", action="store_true",
                   help="run only the batched-ensemble variant and print its JSON (profiling runs)")
    p.add_argument("--serve-study", action="store_true",
                   help="run only the serving comparison on traces of 500 requests at 5/s and 2/s "
                        "(served engine and measured plain path) and print its JSON (several minutes)")
    p.add_argument("--d3-only", type=int, default=0, metavar="N",
                   help="run only the three-dimensional variant on an N^3 lattice and print its JSON "
                        "(profiling runs; --lattice 19 or 27)")
    p.add_argument("--lattice", type=int, default=19, choices=[19, 27])
    p.add_argument("--d3-noise", default="lw", choices=["lw", "rs", "local"])
    p.add_argument("--noise", default="lw", choices=["lw", "full", "rs"],
                   help="noise of the main line (full: correlated via k-space, rs: correlated built in real "
                        "space, both at kappa=0.05; for profiling runs)")
    p.add_argument("--storage", default="fp32", choices=["fp32", "fp16"],
                   help="population storage of the main line (fp16: deviations; for profiling runs)")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash(names):
    """sha256 of the listed sources with // comments, trailing blanks and empty lines removed
    (a comment edit leaves the compiled kernel, and so its counters, unchanged)."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, name)) as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def step_kernel_traffic(nodes):
    """DRAM bytes per step-kernel launch from a committed ncu capture, scaled by nodes,
    or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if kernel_source_hash(d.get("sources", [])) != d.get("source_sha256"):
        return None
    return float(d["dram_bytes_per_launch"]) * nodes / float(d["nodes"])


class ClockSampler:
    """nvidia-smi samples (every 20 ms) of SM clock and throttle reasons during the timed
    region.  The sampler runs on until the whole bench has finished, so a timed region
    shorter than 0.1 s is widened by 0.1 s on either side (warm-up before it, the next
    measurement after it); the record says so."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if t1 - t0 >= 0.1:
            return self._summary(t0, t1)
        rec = self._summary(t0 - 0.1, t1 + 0.1)
        rec["window"] = ("timed region %.4f s; clocks sampled from 0.1 s before it to 0.1 s after it"
                         % (t1 - t0))
        return rec

    def _summary(self, t0, t1):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if ts < t0 or ts > t1 + 0.05:
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def _oracle_strip(n_side, h, steps, seed, warmup=1):
    """One oracle run of `steps` steps on a periodic n_side x h strip with the main line's
    parameters after `warmup` untimed steps; returns the seconds the timed steps took."""
    import oracle
    p = PARAMS_LW
    L = oracle.Lattice(n_side, h, seed=seed)
    L.set_params(p["kT"], p["kappa"], p["tau_s"], p["tau_b"], p["tau_ghost"], oracle.NOISE_LW)
    L.step(warmup)
    t0 = time.perf_counter()
    L.step(steps)
    return time.perf_counter() - t0


def _oracle_strip_task(job):
    return _oracle_strip(*job)


def cpu_baseline(seconds, n_side):
    """The FP64 oracle (as it stands, single-threaded) on periodic n_side x h strips of the
    workload with the main line's parameters: one process, sized for about `seconds` of
    work, then one independent strip per host core in as many processes (spawned, so no
    GPU state is inherited), timed by the slowest."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    oracle.build()
    steps = 5
    dt = _oracle_strip(n_side, 4, 2, 42)
    rate = n_side * 4 * 2 / max(dt, 1e-9)                   # node updates / s
    h = int(max(4, min(n_side, seconds * rate / (n_side * steps))))
    dt = _oracle_strip(n_side, h, steps, 42)
    single = n_side * h * steps / dt / 1e6
    cores = _host_cores()
    # ~3 s of work per core, at most 2^20 nodes per strip (bounded host memory)
    hp = int(max(4, min(h, 3.0 * rate / (n_side * steps), (1 << 20) // n_side)))
    jobs = [(n_side, hp, steps, 42 + 1000 * j) for j in range(cores)]
    try:
        with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
            times = [f.result(timeout=600) for f in [ex.submit(_oracle_strip_task, j) for j in jobs]]
    except Exception as e:                  # a broken worker pool must not hang the bench
        return {"value": single, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                "sample": "%d steps of a periodic %dx%d strip, one thread (all-core run failed: %s)"
                          % (steps, n_side, h, type(e).__name__), "seconds": dt}
    allc = cores * n_side * hp * steps / max(times) / 1e6
    return {"value": allc, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "%d independent periodic %dx%d strips (one per host core, one process each, "
                      "single-threaded), %d steps each, long-wavelength noise, kappa=%.2f; FP64 C core + numpy "
                      "noise; timed by the slowest" % (cores, n_side, hp, steps, PARAMS_LW["kappa"]),
            "seconds": max(times),
            "single_core": {"value": single, "unit": "MLUPS", "cores": 1, "seconds": dt,
                            "sample": "%d steps of a periodic %dx%d strip" % (steps, n_side, h)}}


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def reference_arm(args):
    """The oracle as it stands, on the host cores: one independent periodic strip of the
    workload per core (one single-threaded process each, spawned), each doing the warm-up
    and the timed steps; the step time is the slowest process's."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    oracle.build()
    n_side = args.n
    t = _oracle_strip(n_side, 4, 2, 42)
    rate = n_side * 4 * 2 / max(t, 1e-9)
    cores = _host_cores()
    budget = 100.0                                   # seconds of oracle work per process
    h = int(max(2, min(n_side, budget * rate / (n_side * max(1, args.steps + args.warmup)))))
    jobs = [(n_side, h, args.steps, 42 + 1000 * j, args.warmup) for j in range(cores)]
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        times = [f.result(timeout=1800) for f in [ex.submit(_oracle_strip_task, j) for j in jobs]]
    dt = max(times)
    mlups = cores * n_side * h * args.steps / dt / 1e6
    sample = ("each step: one oracle step of %d independent periodic %dx%d strips of the %dx%d workload, one "
              "per host core" % (cores, n_side, h, n_side, n_side))
    line = {"impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "D2Q9 fluctuating non-ideal LB, periodic %dx%d FP32 lattice, long-wavelength "
                                   "noise, kappa=0.01, tau_s=0.8, kT=1e-4" % (n_side, n_side),
                       "sample_rows": h, "processes": cores},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def timed_run(lbf, torch, L, steps, warmup, mode, params, dist):
    L.set_params(params["kT"], params["kappa"], params["tau_s"], params["tau_b"], params["tau_ghost"], mode)
    L.step(warmup)
    torch.cuda.synchronize()
    # CUDA events around a sample of the step-kernel launches spread over the timed region
    # (every launch would add the events' own cost, ~4 us a step, to the whole-run time)
    lbf.lb_set_kernel_timing(L.ctx, max(1, steps // 500))
    k0 = lbf.lb_launch_count(L.ctx)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    wall0 = time.time()
    ev0.record(L.stream)
    L.step(steps)
    ev1.record(L.stream)
    torch.cuda.synchronize()
    wall1 = time.time()
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    kms, kl = lbf.lb_kernel_time(L.ctx)
    launches = lbf.lb_launch_count(L.ctx) - k0
    lbf.lb_set_kernel_timing(L.ctx, 0)
    return ms, kms, kl, launches, wall0, wall1


# the two-phase variants: the Landau double well of Sec. II A, mean density in the spinodal
# region (the uniform state decomposes, seeded by the noise at the local density)
DOUBLE_WELL = (0.04, 0.5, 1.0)      # beta, rhoV, rhoL
RHO0_TWOPHASE = 0.75


def d3_variant(lbf, torch, hbm, lattice=19, n=256, steps=300, warmup=5, noise="lw"):
    """A three-dimensional lattice (the paper's model carried to D3Q19 or D3Q27): n^3 FP32
    (2 x 19 x 67 MB or 2 x 27 x 67 MB of populations at n = 256, larger than L2), cs2 = 1/3,
    uncorrelated noise of Xi(0) (noise="lw") or the correlated noise Xi(k) built in real space
    (noise="rs"), the PARAMS_LW relaxation times and kappa; or the two-phase model
    (noise="local": the double well DOUBLE_WELL at mean density RHO0_TWOPHASE, kappa = 0.03,
    noise at the local density); one kernel launch per step.  Algorithmic bytes: Q FP32
    populations read and Q written per node."""
    twophase = noise == "local"
    L = lbf.Lattice3(n, n, n, seed=42, rho0=RHO0_TWOPHASE if twophase else 1.0, cs2=1.0 / 3.0, lattice=lattice)
    p = dict(PARAMS_LW, kappa=0.03) if twophase else PARAMS_LW
    if twophase:
        L.set_eos(lbf.LB_EOS_DOUBLE_WELL, *DOUBLE_WELL)
    mode = {"rs": lbf.LB_NOISE_FULL_RS, "local": lbf.LB_NOISE_LW_LOCAL}.get(noise, lbf.LB_NOISE_LW)
    L.set_params(p["kT"], p["kappa"], p["tau_s"], p["tau_b"], p["tau_ghost"], mode)
    L.step(warmup)
    torch.cuda.synchronize()
    lbf.lb3_set_kernel_timing(L.ctx, max(1, steps // 100))
    k0 = lbf.lb3_launch_count(L.ctx)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(L.stream)
    L.step(steps)
    ev1.record(L.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    kms, kl = lbf.lb3_kernel_time(L.ctx)
    launches = lbf.lb3_launch_count(L.ctx) - k0
    lbf.lb3_set_kernel_timing(L.ctx, 0)
    nodes = n ** 3
    bpn = 2 * lattice * 4
    k_s = kms / max(kl, 1) / 1e3
    L.close()
    return {"lattice": "D3Q%d %d^3, FP32 deviations" % (lattice, n),
            "noise": {"rs": "correlated, built in real space (2x2x2 stencil of eight white corner fields; "
                            + ("the (4,16) block's 2-vectors)" if lattice == 19 else
                               "a white part plus two scalar fields along the rank-two slope)"),
                      "local": "uncorrelated at the local density and c_s^2 (two-phase: double well beta=%g, "
                               "rhoV=%g, rhoL=%g, rho0=%g)" % (DOUBLE_WELL + (RHO0_TWOPHASE,))}.get(
                noise, "long-wavelength"),
            "kappa": p["kappa"], "value": nodes * steps / (ms / 1e3) / 1e6, "unit": "MLUPS",
            "ms_per_step": ms / steps,
            "step_kernel": {"achieved": bpn * nodes / k_s / 1e9, "unit": "GB/s",
                            "frac": bpn * nodes / k_s / 1e9 / hbm, "avg_us": k_s * 1e6, "bytes_per_node": bpn},
            "gpu_launches": launches}


def twophase_variant(lbf, torch, hbm, n=4096, steps=1000, warmup=5):
    """The two-phase model on D2Q9: an n^2 FP32 lattice with the double well DOUBLE_WELL at
    mean density RHO0_TWOPHASE (spinodal decomposition from the uniform state), kappa = 0.03,
    the PARAMS_LW relaxation times and kT, noise at the local density (Sec. IV, V B); the step
    kernel that carries the double well's quartic.  Algorithmic bytes: 72 per node."""
    L = lbf.Lattice(n, n, seed=44, rho0=RHO0_TWOPHASE)
    L.set_eos(lbf.LB_EOS_DOUBLE_WELL, *DOUBLE_WELL)
    p = dict(PARAMS_LW, kappa=0.03)
    ms, kms, kl, launches, _, _ = timed_run(lbf, torch, L, steps, warmup, lbf.LB_NOISE_LW_LOCAL, p, None)
    k_s = kms / max(kl, 1) / 1e3
    rho = L.populations().sum(axis=0)
    L.close()
    return {"lattice": "D2Q9 %d^2, FP32 deviations" % n,
            "noise": "uncorrelated at the local density and c_s^2 (two-phase: double well beta=%g, rhoV=%g, "
                     "rhoL=%g, rho0=%g)" % (DOUBLE_WELL + (RHO0_TWOPHASE,)),
            "kappa": 0.03, "value": n * n * steps / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_step": ms / steps,
            "step_kernel": {"achieved": BYTES_PER_NODE_STEP * n * n / k_s / 1e9, "unit": "GB/s",
                            "frac": BYTES_PER_NODE_STEP * n * n / k_s / 1e9 / hbm, "avg_us": k_s * 1e6,
                            "bytes_per_node": BYTES_PER_NODE_STEP},
            "density_range_after": [float(rho.min()), float(rho.max())],
            "gpu_launches": launches}


def batched_variant(lbf, torch, steps=2000, graph_steps=100, plain_steps=20):
    """Batched ensemble: 512 replicas, 128 each of 32^2, 64^2, 128^2, 256^2, own seeds and kT
    uniform in [5e-5, 2e-4], long-wavelength noise, one persistent launch per step replayed
    from a CUDA graph of `graph_steps` steps, tile shape autotuned; against the plain path
    (one lb_step per lattice per step) on the same replicas."""
    rng = np.random.default_rng(2024)
    sizes = [(L, L) for L in (32, 64, 128, 256) for _ in range(128)]
    seeds = [int(x) for x in rng.integers(1, 2 ** 62, len(sizes))]
    kT = rng.uniform(5e-5, 2e-4, len(sizes))
    nodes = sum(a * b for a, b in sizes)
    ens = lbf.Ensemble(sizes, seeds)
    for r in range(len(sizes)):
        ens.set_params(r, float(kT[r]), 0.01, 0.8, 1.0, 1.0, lbf.LB_NOISE_LW)
    ens.autotune(20)
    ens.set_sampling(100, 64)
    ens.step(2 * graph_steps, graph_steps=graph_steps)        # warm-up, graph captured
    torch.cuda.synchronize()
    k0 = lbf.lb_batch_launch_count(ens.b)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(ens.stream)
    ens.step(steps, graph_steps=graph_steps)
    ev1.record(ens.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = lbf.lb_batch_launch_count(ens.b) - k0
    tx, ty, nt, _ = lbf.lb_batch_tuning(ens.b)
    # the same ensemble with the correlated (full FDT) noise of Sec. IV
    for r in range(len(sizes)):
        ens.set_params(r, float(kT[r]), 0.01, 0.8, 1.0, 1.0, lbf.LB_NOISE_FULL)
    fsteps = max(1, steps // 4)
    ens.step(graph_steps, graph_steps=graph_steps)
    torch.cuda.synchronize()
    ev0.record(ens.stream)
    ens.step(fsteps, graph_steps=graph_steps)
    ev1.record(ens.stream)
    torch.cuda.synchronize()
    fms = ev0.elapsed_time(ev1)
    # and with the correlated noise built in real space (no per-class synthesis launches)
    for r in range(len(sizes)):
        ens.set_params(r, float(kT[r]), 0.01, 0.8, 1.0, 1.0, lbf.LB_NOISE_FULL_RS)
    ens.step(graph_steps, graph_steps=graph_steps)
    torch.cuda.synchronize()
    ev0.record(ens.stream)
    ens.step(fsteps, graph_steps=graph_steps)
    ev1.record(ens.stream)
    torch.cuda.synchronize()
    rms = ev0.elapsed_time(ev1)
    ens.close()
    del ens
    # plain path: the same lattices as separate contexts, one step launch per lattice
    lats = []
    for r in range(len(sizes)):
        L = lbf.Lattice(*sizes[r], seed=seeds[r])
        L.set_params(float(kT[r]), 0.01, 0.8, 1.0, 1.0, lbf.LB_NOISE_LW)
        lats.append(L)
    for L in lats:
        L.step(2)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(plain_steps):
        for L in lats:
            L.step(1)
    ev1.record()
    torch.cuda.synchronize()
    pms = ev0.elapsed_time(ev1)
    for L in lats:
        L.close()
    value = nodes * steps / (ms / 1e3) / 1e6
    plain = nodes * plain_steps / (pms / 1e3) / 1e6
    return {"workload": "batched ensemble: 512 FP32 replicas (128 each of 32^2, 64^2, 128^2, 256^2), own Philox "
                        "seeds, kT uniform in [5e-5, 2e-4], kappa=0.01, tau_s=0.8, long-wavelength noise, "
                        "%d steps, S(k) every 100 steps into 64 bins" % steps,
            "value": value, "unit": "MLUPS", "ms_per_step": ms / steps,
            "launch": "one persistent launch per step, CUDA graph of %d steps" % graph_steps,
            "autotuned_tile": [tx, ty, nt], "gpu_launches": launches,
            "correlated_noise": {"value": nodes * fsteps / (fms / 1e3) / 1e6, "unit": "MLUPS",
                                 "ms_per_step": fms / fsteps, "steps": fsteps,
                                 "how": "same replicas with full FDT noise (k-space synthesis per replica)"},
            "correlated_noise_real_space": {"value": nodes * fsteps / (rms / 1e3) / 1e6, "unit": "MLUPS",
                                            "ms_per_step": rms / fsteps, "steps": fsteps,
                                            "how": "same replicas with full FDT noise built in real space "
                                                   "(2x2 stencil in the step kernel)"},
            "plain_path": {"value": plain, "unit": "MLUPS", "steps": plain_steps,
                           "how": "512 lb_step calls per step, one context per lattice"},
            "speedup_vs_plain": value / plain,
            "accuracy": "each replica steps exactly the trajectory it has alone (bitwise, tests/test_gpu_batch.py); "
                        "replicas vs FP64 oracle <= 1e-5, per-replica S(k) vs oracle rtol 1e-4"}


def _request_stream(rate, n_requests, seed):
    """Arrival times and parameters of a Poisson stream of simulation requests."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_requests)
    arrive = np.cumsum(gaps) - gaps[0]
    side = rng.choice([64, 128, 256, 512, 1024], n_requests)
    steps = np.exp(rng.uniform(np.log(1e3), np.log(1e5), n_requests)).astype(np.int64)
    kT = rng.uniform(5e-5, 2e-4, n_requests)
    kap = rng.uniform(0.005, 0.05, n_requests)
    ts = rng.uniform(0.6, 1.5, n_requests)
    return arrive, side, steps, kT, kap, ts


def _serve_stream(lbf, stream, budget, chunk, admission=None):
    """Submits the stream at its arrival times, waits for the drain; returns latencies
    (completion - submission, host clock) and the server's counters.  admission: optional
    (large_nodes, max_large) for lb_server_set_admission."""
    arrive, side, steps, kT, kap, ts = stream
    srv = lbf.Server(budget, max_active=4096, max_chunk_steps=chunk)
    if admission is not None:
        lbf.lb_server_set_admission(srv.srv, *admission)
    t0 = time.perf_counter()
    for k in range(len(arrive)):
        d = arrive[k] - (time.perf_counter() - t0)
        if d > 0:
            time.sleep(d)
        srv.submit(int(side[k]), int(side[k]), int(steps[k]), kT=float(kT[k]), kappa=float(kap[k]),
                   tau_s=float(ts[k]), seed=1000 + k)
    srv.wait(0)
    res = srv.poll(len(arrive) + 8)
    st = srv.stats()
    srv.close()
    lat = np.array([r.t_complete - r.t_submit for r in res])
    return lat, st


def _plain_server(lbf, torch, stream):
    """The plain path as a server: the same trace replayed on one host thread, each request
    run alone through lb_step in arrival order (FIFO) on a context of its size, completion =
    when the host sees its last step finish.  Returns latencies and the aggregate MLUPS
    (node updates / (last completion - first start))."""
    arrive, side, steps, kT, kap, ts = stream
    lat = np.zeros(len(arrive))
    updates = 0.0
    t0 = time.perf_counter()
    first = None
    for k in range(len(arrive)):
        now = time.perf_counter() - t0
        if arrive[k] > now:
            time.sleep(arrive[k] - now)
        L = int(side[k])
        start = time.perf_counter() - t0
        first = start if first is None else first
        lat_ = lbf.Lattice(L, L, seed=1000 + k)      # at rest, time 0 (as a served request)
        lat_.set_params(float(kT[k]), float(kap[k]), float(ts[k]), 1.0, 1.0, lbf.LB_NOISE_LW)
        lat_.step(int(steps[k]))
        torch.cuda.synchronize()
        done = time.perf_counter() - t0
        lat_.close()
        lat[k] = done - arrive[k]
        updates += float(L) * L * int(steps[k])
    wall = (time.perf_counter() - t0) - first
    return lat, updates / wall / 1e6, wall


def serve_compare(lbf, torch, r, n, seed, budget=120 * 10 ** 9, chunk=200, admission=None, plain=True):
    """One trace of n requests at r/s through the server and through the plain FIFO path."""
    stream = _request_stream(r, n, seed)
    lat, st = _serve_stream(lbf, stream, budget, chunk, admission)
    wall = st.t_last_complete - st.t_first_admit
    if not plain:
        return {"rate_per_s": r, "requests": n, "completed": int(st.completed), "admission": admission,
                "value": st.node_updates / wall / 1e6, "unit": "MLUPS (aggregate, first admission to last completion)",
                "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                              "max": float(lat.max())}}
    plat, pmlups, pwall = _plain_server(lbf, torch, stream)
    offered = float(np.sum(stream[1].astype(float) ** 2 * stream[2])) / max(stream[0][-1], 1e-9) / 1e6
    return {"rate_per_s": r, "requests": n, "completed": int(st.completed),
            "value": st.node_updates / wall / 1e6, "unit": "MLUPS (aggregate, first admission to last completion)",
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
            "offered_mlups_during_arrivals": offered, "node_updates": st.node_updates, "wall_s": wall,
            "gpu_busy_s": st.gpu_busy_s, "hbm_peak_gb": st.bytes_peak / 1e9,
            "plain_path": {"value": pmlups, "unit": "MLUPS (aggregate, first start to last completion)",
                           "wall_s": pwall,
                           "latency_s": {"p50": float(np.percentile(plat, 50)),
                                         "p99": float(np.percentile(plat, 99)), "max": float(plat.max())},
                           "how": "measured: the same trace replayed one request at a time through "
                                  "lb_step (FIFO, host clock)"}}


def served_variant(lbf, torch, n_requests=64, rate=200.0, budget=120 * 10 ** 9, chunk=200,
                   sweep=((5.0, 32), (2.0, 16))):
    """Serving: a Poisson stream of requests at `rate`/s (a bounded sample of n_requests),
    L uniform in {64, 128, 256, 512, 1024}, steps log-uniform in [1e3, 1e5], kT in
    [5e-5, 2e-4], kappa in [0.005, 0.05], tau_s in [0.6, 1.5], FP32, admitted under an HBM
    budget; latency = completion - submission on the host clock.  At 200/s the offered
    load is ~20x what one GPU sustains, so the sample is a finite trace that drains; the
    sweep repeats it at sustainable rates.  The plain path is measured on the same trace:
    one request at a time through lb_step, in arrival order."""

    def one(r, n, seed):
        return serve_compare(lbf, torch, r, n, seed, budget, chunk)

    line = one(rate, n_requests, 11)
    line["workload"] = ("served: Poisson arrivals at %.0f/s (sample of %d requests), L in {64..1024}^2, steps "
                        "log-uniform in [1e3, 1e5], kT in [5e-5, 2e-4], kappa in [0.005, 0.05], tau_s in [0.6, 1.5], "
                        "FP32, HBM budget %.0f GB" % (rate, n_requests, budget / 1e9))
    line["rate_sweep"] = [one(r, n, 12 + i) for i, (r, n) in enumerate(sweep)]
    line["accuracy"] = ("each served result is bitwise the same alone and in the mix (tests/test_gpu_serve.py); "
                        "served lattices vs FP64 oracle <= 1e-5")
    return line


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import paper_1009_0254_gb300 as lbf
    from paper_1009_0254_gb300 import build as lbbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        lbbuild.build()
    if dist is not None:
        dist.barrier()
    lbf.load()
    if args.batched_only:
        print(json.dumps(batched_variant(lbf, torch)))
        return 0
    if args.d3_only:
        print(json.dumps(d3_variant(lbf, torch, peaks()[0], args.lattice, n=args.d3_only, steps=args.steps,
                                    warmup=args.warmup, noise=args.d3_noise)))
        return 0
    if args.serve_study:
        big = (512 * 512, 1)      # lattices of 512^2 and more: one at a time
        print(json.dumps({"workload": "served request stream (config 5 mix) at sustainable rates, 500 requests "
                                      "per trace; served engine against the plain path measured on the same trace; "
                                      "the server also with lattices of 512^2 nodes and more admitted one at a time",
                          "rates": [serve_compare(lbf, torch, 5.0, 500, 31), serve_compare(lbf, torch, 2.0, 500, 32)],
                          "large_one_at_a_time": [serve_compare(lbf, torch, 5.0, 500, 31, admission=big, plain=False),
                                                  serve_compare(lbf, torch, 2.0, 500, 32, admission=big,
                                                                plain=False)]}))
        return 0

    n = args.n
    nodes = n * n
    main_fp16 = args.storage == "fp16"
    L = lbf.Lattice(n, n, seed=replica_seed(42, rank), precision=lbf.LB_FP16DEV if main_fp16 else lbf.LB_FP32)
    L.set_sampling(args.every, args.nbins)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_index = vis.split(",")[local] if vis else local
    clocks = ClockSampler(gpu_index)
    time.sleep(0.3)

    # main line: long-wavelength noise
    main_full = args.noise != "lw"
    main_mode = {"lw": lbf.LB_NOISE_LW, "full": lbf.LB_NOISE_FULL, "rs": lbf.LB_NOISE_FULL_RS}[args.noise]
    main_params = PARAMS_FULL if main_full else PARAMS_LW
    main_bpn = (BYTES_PER_NODE_STEP_FP16 if main_fp16 else BYTES_PER_NODE_STEP) + (8 if args.noise == "full" else 0)
    ms, kms, kl, launches, w0, w1 = timed_run(lbf, torch, L, args.steps, args.warmup, main_mode, main_params, dist)
    clk_window = (w0, w1)

    ms = max_over_ranks(dist, ms, "cuda")
    value = whole_job_mlups(world, nodes, args.steps, ms)
    hbm, peak_kind = peaks()
    k_avg_s = kms / max(kl, 1) / 1e3
    achieved = main_bpn * nodes / k_avg_s / 1e9
    traffic = None if (main_full or main_fp16) else step_kernel_traffic(nodes)

    # variants of config 2: the other (noise, kappa) combinations of the same lattice
    variants = []
    if not args.no_variants and not main_full and not main_fp16:
        for vmode, vkappa in ((lbf.LB_NOISE_FULL, 0.05), (lbf.LB_NOISE_FULL, 0.01), (lbf.LB_NOISE_LW, 0.05),
                              (lbf.LB_NOISE_FULL_RS, 0.05), (lbf.LB_NOISE_FULL_RS, 0.01)):
            vparams = dict(PARAMS_LW, kappa=vkappa)
            full = vmode == lbf.LB_NOISE_FULL
            bpn = BYTES_PER_NODE_STEP_FULL if full else BYTES_PER_NODE_STEP
            L.set_sampling(args.every, args.nbins)
            fms, fkms, fkl, flaunch, _, _ = timed_run(lbf, torch, L, args.steps, args.warmup, vmode, vparams, dist)
            fms = max_over_ranks(dist, fms, "cuda")
            fk = fkms / max(fkl, 1) / 1e3
            variants.append({"noise": {lbf.LB_NOISE_FULL: "full (correlated, k-space synthesis + FFT each step)",
                                       lbf.LB_NOISE_FULL_RS: "full (correlated, built in real space: 2x2 stencil of "
                                                             "four white fields, fused in the step kernel)",
                                       lbf.LB_NOISE_LW: "long-wavelength"}[vmode], "kappa": vkappa,
                             "value": whole_job_mlups(world, nodes, args.steps, fms), "unit": "MLUPS",
                             "ms_per_step": fms / args.steps,
                             "step_kernel": {"achieved": bpn * nodes / fk / 1e9, "unit": "GB/s",
                                             "frac": bpn * nodes / fk / 1e9 / hbm, "avg_us": fk * 1e6,
                                             "bytes_per_node": bpn},
                             "gpu_launches": flaunch})

    # variant: FP16 deviation storage, long-wavelength noise (the precision study's second arm)
    if not args.no_variants and not main_fp16:
        L16 = lbf.Lattice(n, n, seed=replica_seed(43, rank), precision=lbf.LB_FP16DEV)
        L16.set_sampling(args.every, args.nbins)
        hms, hkms, hkl, hlaunch, _, _ = timed_run(lbf, torch, L16, args.steps, args.warmup, lbf.LB_NOISE_LW,
                                                  PARAMS_LW, dist)
        hms = max_over_ranks(dist, hms, "cuda")
        hk = hkms / max(hkl, 1) / 1e3
        variants.append({"storage": "fp16 deviations (FP32 arithmetic)", "noise": "long-wavelength", "kappa": 0.01,
                         "value": whole_job_mlups(world, nodes, args.steps, hms), "unit": "MLUPS",
                         "ms_per_step": hms / args.steps,
                         "step_kernel": {"achieved": BYTES_PER_NODE_STEP_FP16 * nodes / hk / 1e9, "unit": "GB/s",
                                         "frac": BYTES_PER_NODE_STEP_FP16 * nodes / hk / 1e9 / hbm,
                                         "avg_us": hk * 1e6},
                         "gpu_launches": hlaunch})
        L16.close()
        del L16

    # the three-dimensional lattices
    if not args.no_variants and not main_fp16:
        variants.append(d3_variant(lbf, torch, hbm, 19))
        variants.append(d3_variant(lbf, torch, hbm, 19, noise="rs"))
        variants.append(d3_variant(lbf, torch, hbm, 27))
        variants.append(d3_variant(lbf, torch, hbm, 27, noise="rs"))

    # the two-phase model (double well, noise at the local density) on D2Q9, D3Q19, D3Q27
    if not args.no_variants and not main_fp16:
        variants.append(twophase_variant(lbf, torch, hbm))
        variants.append(d3_variant(lbf, torch, hbm, 19, noise="local"))
        variants.append(d3_variant(lbf, torch, hbm, 27, noise="local"))

    # batched ensemble and request server (rank 0 of a single-GPU run)
    if not args.no_variants and world == 1:
        variants.append(batched_variant(lbf, torch))
        variants.append(served_variant(lbf, torch))

    # end to end through the public API: host initial state in, spectra and sums out
    L.set_params(PARAMS_LW["kT"], PARAMS_LW["kappa"], PARAMS_LW["tau_s"], PARAMS_LW["tau_b"],
                 PARAMS_LW["tau_ghost"], lbf.LB_NOISE_LW)
    L.set_sampling(args.every, args.nbins)
    host_f = torch.empty((9, n, n), dtype=torch.float64, pin_memory=True)
    host_f.copy_(torch.from_numpy(L.populations()))
    S = np.zeros(args.nbins)
    Jl = np.zeros(args.nbins)
    Jt = np.zeros(args.nbins)
    cnt = np.zeros(args.nbins, dtype=np.int64)
    ns = np.zeros(1, dtype=np.int64)
    sums = np.zeros(3)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    lbf.lb_set_populations(L.ctx, host_f.data_ptr(), lbf.LB_HOST, 0)
    lbf.lb_step(L.ctx, args.steps)
    lbf.lb_structure_factor(L.ctx, args.nbins, S, Jl, Jt, cnt, ns)
    lbf.lb_moments(L.ctx, None, lbf.LB_HOST, sums)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(dist, e2e_s, "cuda")
    h2d = 9 * nodes * 8
    d2h = 3 * args.nbins * 8 + 3 * 8
    e2e = {"value": whole_job_mlups(world, nodes, args.steps, e2e_s * 1e3), "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "job": "lb_set_populations (host FP64) + lb_step(K) + lb_structure_factor + lb_moments sums"}

    clk = clocks.stop(*clk_window)
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(args.cpu_seconds, n)
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "D2Q9 fluctuating non-ideal LB (modified equilibrium), periodic %dx%d %s "
                               "lattice, %s noise, kappa=%.2f, tau_s=0.8, tau_b=1, tau_ghost=1, "
                               "kT=1e-4, cs2=1/3, S(k) every %d steps into %d bins (FP64)" % (
                                   n, n, "FP16-deviation" if main_fp16 else "FP32",
                                   {"lw": "long-wavelength", "full": "correlated (full FDT, k-space)",
                                    "rs": "correlated (full FDT, real space)"}[args.noise],
                                   main_params["kappa"], args.every, args.nbins),
                   "lattice": [n, n], "l2": "inputs larger than L2 (2 x %.0f MB populations)" % (
                       9 * (n + 64) * (n + 4) * 4 / 1e6), "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic, "kernel": "step_kernel (fused pull+collide+noise)",
                     "bytes_per_node": main_bpn, "avg_launch_us": k_avg_s * 1e6, "timed_launches": kl,
                     "peak_source": peak_kind},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "variants": variants,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
