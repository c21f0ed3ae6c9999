"""Benchmark of the resonant-line Monte Carlo hot path on GB300.

Workload: the static homogeneous sphere (H I + dust) -- 8^3 root octree
refined to 64^3 equivalent inside the sphere (R = 0.45 box), centre-to-edge
line-centre optical depth tau0 = 1e6 at T = 1e4 K (a = 4.7e-4), dust albedo
0.32, g = 0.73, centre-to-edge tau_dust = 1, packets emitted at the centre at
line centre.  One step propagates one batch of packets (distinct packet ids
every step) until each escapes or is absorbed, with the escape spectrum
(200 bins over x in [-60, 60]) accumulated on the device.

Metric: scatterings per second (and packets per second) on the GPU, the oracle
(plain FP64 C, host cores) as the reference arm.  Multi-GPU: packet ids are
sharded across ranks (weak scaling), no collective on the data path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--packets P] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "scatterings/sec & packets/sec on 1 GB300 vs oracle; batched vs plain speedup; HBM roofline %"
WORKLOAD = ("static H I + dust sphere: 8^3 root refined to 64^3-equivalent octree (172992 leaves), "
            "tau0=1e6 centre-to-edge, T=1e4 K, tau_dust=1, albedo 0.32, packets from the centre at x=0")
# Instruction counts of k_propagate per scattering on this workload, from one
# ncu capture of the kernel (an uncapped launch of 65536 packets of the same
# sphere; smsp__inst_executed.sum and smsp__inst_executed_pipe_*.sum divided
# by the launch's scatterings), and the active lanes per warp instruction of
# the same capture.  They are constants of the code and the workload, so the
# bench multiplies them by its own live scattering rate.
INST_PER_SCATT = 6044032067435 / 111923728554
LANES_PER_INST = 106529112851470 / 6044032067435
# pipe -> warp instructions per scattering of the same capture (FP32 FMA,
# FP64, special-function unit)
PIPE_PER_SCATT = {"fma": 2877856853460 / 111923728554, "fp64": 83386945512 / 111923728554,
                  "xu": 166026282325 / 111923728554}
# DRAM bytes per leaf visit of k_ray_tau on the synthetic galaxy
# (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of 2^18
# rays from emitting leaves, 59 732 805 leaf visits)
RAY_DRAM_BYTES_PER_VISIT = (4.107982e9 + 49.11232e6) / 59732805


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--packets", type=int, default=1_000_000,
                    help="packets per step (the workload's 1e6 packets: fewer leave the GPU idle while the last, "
                         "longest packets finish)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--batch-models", type=int, default=512,
                    help="models in the batched-vs-plain comparison (0 = skip it)")
    ap.add_argument("--batch-scale", type=float, default=0.01,
                    help="packets per batch model: log-uniform [1e3, 1e5] times this")
    ap.add_argument("--batch-plain", type=int, default=1,
                    help="also time one launch per model (1) or only the persistent launch (0)")
    ap.add_argument("--batch-cap", type=int, default=100000,
                    help="scatterings per packet cap in the batch comparison (CAPPED packets are reported)")
    ap.add_argument("--galaxy", type=int, default=1, help="run the synthetic-galaxy section (1) or not (0)")
    ap.add_argument("--c3-packets", type=int, default=1 << 17,
                    help="packets of the expanding-sphere configuration in --section configs")
    ap.add_argument("--peel-adjoint", action="store_true",
                    help="--section peel: run the adjoint of the cube instead of the forward propagation")
    ap.add_argument("--configs-only", default="",
                    help="comma-separated prefixes of the configurations --section configs runs (default: all)")
    ap.add_argument("--galaxy-rays", type=int, default=1 << 20)
    ap.add_argument("--galaxy-packets", type=int, default=1 << 18)
    ap.add_argument("--galaxy-cap", type=int, default=64, help="scatterings per packet in the galaxy section")
    ap.add_argument("--galaxy-thin", type=float, default=1e-12,
                    help="density scale of the lower-column copy of the galaxy used for peeling and its adjoint")
    ap.add_argument("--galaxy-all-packets", type=int, default=10_000_000,
                    help="packets of the core-skipped galaxy run (the configuration's 1e7)")
    ap.add_argument("--galaxy-core-skip", type=float, default=0.5,
                    help="core-skipping factor f (x_crit = f (a tau_cell)^(1/3)) of the uncapped galaxy run")
    ap.add_argument("--galaxy-cs-cap", type=int, default=1_000_000,
                    help="scatterings per packet cap of the core-skipped galaxy run (CAPPED packets are reported)")
    ap.add_argument("--section", default="all",
                    choices=["all", "main", "batch", "galaxy", "configs", "kernel", "peel"],
                    help="all (default): the headline line with the batch and galaxy sections; "
                         "batch / galaxy: that section alone, printed as its own JSON line; configs: GPU and "
                         "oracle rates of the other configurations (not part of the default run); kernel: one "
                         "launch over --packets packets of the headline workload (for profiling); peel: one "
                         "propagation with peeling of --galaxy-packets packets through the galaxy with densities "
                         "x --galaxy-thin (for profiling the peel kernel)")
    ap.add_argument("--voigt", default="tasitsiomi", choices=["tasitsiomi", "faddeeva"],
                    help="H(a,x) evaluation: Tasitsiomi's form (default, the paper's hot-path choice) or the "
                         "accurate Faddeeva function")
    ap.add_argument("--max-scatt", type=int, default=0,
                    help="cap scatterings per packet (profiling runs only; 0 = the full workload)")
    return ap.parse_args()


# H(a,x) method of every run (0: Tasitsiomi's form, the default and the
# headline; 1: the Faddeeva function), set from --voigt
VOIGT = 0


def host_cpu():
    """The host CPU the oracle ran on: model name where the kernel reports
    one, machine type, logical CPUs."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu": model or platform.machine(), "machine": platform.machine(), "nproc": os.cpu_count()}


def _with_voigt(wl):
    wl.physics.voigt = VOIGT
    return wl


def workload(n):
    import synth
    wl = synth.sphere(tau0=1e6, T=1e4, tau_dust=1.0, n_packets=n, recoil=0, isotropic=0)
    wl.physics.voigt = VOIGT
    return wl


def shard_first(rank, step, warmup, steps, n):
    """First packet id of `step` on `rank`: every rank owns its own id ranges
    (weak scaling: packets are independent, so ranks exchange nothing while
    they propagate)."""
    return (rank * (warmup + steps + 1) + step) * n


def reduce_over_ranks(dist, dev, t, counts):
    """(max of t, sums of counts) over the ranks; the identity on one rank."""
    if dist is None:
        return t, list(counts)
    import torch
    v = torch.tensor([t], dtype=torch.float64, device=dev)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    c = torch.tensor(list(counts), dtype=torch.float64, device=dev)
    dist.all_reduce(c)
    return float(v.item()), [float(x) for x in c.tolist()]


def packets(wl, first, n):
    import synth
    return synth.point_source(n, (0.5, 0.5, 0.5), wl.packets.nu[0], wl.physics.seed ^ 0xA5A5 ^ first, first_id=first)


# ------------------------------------------------------------------ clocks
class Clocks:
    def __init__(self, gpu=0):
        self.samples = []
        self.stop = threading.Event()
        self.gpu = gpu
        self.t = threading.Thread(target=self.run, daemon=True)

    def run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                self.samples.append([s.strip() for s in out.split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.t.join(timeout=10)

    def summary(self):
        sm = [float(s[0]) for s in self.samples if len(s) >= 7 and s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if len(s) >= 7 and s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples if len(s) >= 7 for i in range(4)
                          if s[3 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ reference arm
def cpu_oracle_rate(wl_fn, seconds, threads):
    """Oracle (as it stands) on a bounded sample of the workload: packets are
    run in growing batches until about `seconds` of CPU work are done."""
    import oracle
    done_p = done_s = 0
    t_tot = 0.0
    n = max(threads, 8)
    first = 10_000_000
    while t_tot < seconds:
        wl = wl_fn(n)
        pk = packets(wl, first, n)
        first += n
        t0 = time.perf_counter()
        out, tal = oracle.Oracle(wl).run(packets=pk, threads=threads, chunk=1)
        dt = time.perf_counter() - t0
        t_tot += dt
        done_p += n
        done_s += int(out["nscatt"].sum())
        if dt < seconds / 4:
            n *= 2
    return done_s / t_tot, done_p / t_tot, done_p, t_tot


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    per_step = max(2.0, args.cpu_seconds / max(1, args.steps))
    rates = []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(workload, per_step if i >= args.warmup else 0.5, threads)
        if i >= args.warmup:
            rates.append(r)
    sc = sum(r[0] * r[3] for r in rates) / sum(r[3] for r in rates)
    pk = sum(r[2] for r in rates) / sum(r[3] for r in rates)
    line = {"impl": "reference", "metric": METRIC, "value": sc, "unit": "scatterings/s",
            "packets_per_s": pk, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(r[3] for r in rates) / len(rates), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "voigt": args.voigt,
                       "sample": "oracle on %d packets per step" % int(np.mean([r[2] for r in rates]))},
            "cpu_baseline": {"value": sc, "unit": "scatterings/s", "cores": threads, "kind": "oracle",
                             "sample": "%d packets of the workload per step, %d threads" % (int(np.mean([r[2] for r in rates])), threads),
                             "host": host_cpu()},
            "e2e": {"value": sc, "unit": "scatterings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batch comparison
def run_batch(args):
    """Many uneven independent models: one persistent launch (CUDA graph,
    autotuned shape) against one launch per model on the same stream."""
    import paper_2001_11252_gb300 as rg
    import synth
    models = synth.batch_models(args.batch_models, packet_scale=args.batch_scale)
    ctx = rg.Context(0)
    w0 = models[0]
    ctx.set_lines(w0.lines, w0.dust)
    ph = w0.physics
    ctx.set_physics(ph.recoil, ph.isotropic, 0, ph.x_gauss, args.batch_cap, 0, ph.tau_stop, ph.seed)
    ctx.set_voigt(VOIGT)
    ctx.load_batch(models, nbin=200)
    tune_cap = max(1, min(args.batch_cap // 20, 20000))
    tune = ctx.autotune_batch(max_scatt=tune_cap)
    ctx.propagate_batch(rg.BATCH_PERSISTENT)           # warm-up (graph capture)
    t0 = time.perf_counter()
    stb = ctx.propagate_batch(rg.BATCH_PERSISTENT)
    tb = time.perf_counter() - t0
    tp = float("nan")
    if args.batch_plain:
        t0 = time.perf_counter()
        ctx.propagate_batch(rg.BATCH_PER_MODEL)
        tp = time.perf_counter() - t0
    sc = stb["nscatt_line"] + stb["nscatt_dust"]
    ctx.close()
    plain = tp == tp   # timed
    return {"models": len(models), "packets": stb["packets"], "scatterings": sc, "capped": stb["capped"],
            "cap_per_packet": args.batch_cap, "persistent_s": tb, "per_model_s": tp if plain else None,
            "persistent_scatt_per_s": sc / tb, "per_model_scatt_per_s": sc / tp if plain else None,
            "speedup": tp / tb if plain else None,
            "autotuned": {"block": tune["best"][0], "blocks_per_sm": tune["best"][1], "refill": tune["refill"],
                          "tune_cap": tune_cap},
            "workload": "512 homogeneous slab/sphere models: tau0 log-U[1e2,1e7], T log-U[1e2,1e5] K, "
                        "v_max U[0,300] km/s, (2^d)^3 grids d in 2..5, packets log-U[1e3,1e5] x %g" % args.batch_scale}


# ------------------------------------------------------------------ per-config rates
def _oracle_rate(wl, seconds, threads, chunk=1):
    """Oracle on the first packets of a workload, doubling the sample until
    about `seconds` of work: (scatterings/s, packets/s, packets, seconds).
    chunk: packets per task of the thread pool (None: n / (4 threads), for
    short packets whose per-task tallies would cost more than the packets)."""
    import oracle
    o = oracle.Oracle(wl)
    n = max(threads, 2)
    while True:
        n = min(n, wl.packets.n)
        t0 = time.perf_counter()
        out, _ = o.run(lo=0, hi=n, threads=threads, chunk=chunk)
        dt = time.perf_counter() - t0
        if dt >= seconds / 3 or n == wl.packets.n:
            return int(out["nscatt"].sum()) / dt, n / dt, n, dt
        n *= 2


def run_configs(args):
    """GPU and oracle rates per configuration, at equal work per packet: the
    oracle on a bounded sample, one thread and all host threads."""
    import torch
    import paper_2001_11252_gb300 as rg
    import synth
    dev = torch.device("cuda:0")
    threads = os.cpu_count() or 1
    cfgs = [
        ("C1 slab tau0=1e4, T=1e4 K, 2000 packets", lambda n: synth.slab(tau0=1e4, n_packets=n), 2000),
        ("C1-thick slab tau0=1e6, T=10 K, 2000 packets", lambda n: synth.slab(tau0=1e6, T=10.0, n_packets=n), 2000),
        ("C3 expanding sphere N_HI=1e20, v_max 200 km/s, tau_dust 0.5, peeling 3 x 100^2 x 200",
         lambda n: synth.expanding_sphere(n_packets=n), args.c3_packets),
        ("deuterium sphere N_HI=2e19, D/H 3e-5", lambda n: synth.deuterium_sphere(n_packets=n), 1 << 18),
        ("Fe II UV1 sphere tau0=1e4 (fluorescence)", lambda n: synth.feII_sphere(n_packets=n), 1 << 20),
    ]
    out = []
    only = [c.strip() for c in args.configs_only.split(",") if c.strip()]
    for name, fn0, n in cfgs:
        if only and not any(name.startswith(o) for o in only):
            continue
        fn = (lambda f: (lambda k: _with_voigt(f(k))))(fn0)
        wl = fn(n)
        ctx = rg.Context(0)
        ctx.setup(wl)
        pk = wl.packets
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
        args_d = (t(pk.pos, torch.float64), t(pk.dir, torch.float64), t(pk.nu, torch.float64),
                  t(pk.ids.view(np.int64), torch.int64))
        m = min(n, 1024)
        ctx.propagate(*[a[:m] for a in args_d], stats=False)
        ctx.zero_tallies()
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ctx.propagate(*args_d, stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        ctx.close()
        sc = st["nscatt_line"] + st["nscatt_dust"]
        o1 = _oracle_rate(fn(64), args.cpu_seconds / 6, 1)
        on = _oracle_rate(fn(max(64, 8 * threads)), args.cpu_seconds / 6, threads)
        out.append({"config": name, "packets": n, "gpu_s": sec, "gpu_scatt_per_s": sc / sec, "gpu_packets_per_s": n / sec,
                    "mean_scatterings": sc / n, "peel_rays": st["npeel_rays"],
                    "oracle_1_thread_scatt_per_s": o1[0], "oracle_threads": threads,
                    "oracle_all_threads_scatt_per_s": on[0], "oracle_sample_packets": [o1[2], on[2]],
                    "gpu_over_oracle_all_threads": (sc / sec) / on[0]})
    if not only or any(o.startswith("C4") for o in only):
        out.append(_config_batch(args, threads))
    if not only or any(o.startswith("C5") for o in only):
        out.extend(_config_galaxy(args, threads, adjoint=not only or "C5" in only or "C5-adjoint" in only))
    return out


def _oracle_models_rate(models, seconds, threads):
    """Oracle over several models, each on a bounded first sample of its
    packets: (scatterings/s, packets/s, packets, seconds) summed over them."""
    sc = dt = 0.0
    npk = 0
    for w in models:
        r = _oracle_rate(w, seconds / len(models), threads)
        sc += r[0] * r[3]
        dt += r[3]
        npk += r[2]
    return sc / dt, npk / dt, npk, dt


def _config_batch(args, threads):
    """C4 at equal work: every 16th of the 512 batch models (1 % of their
    packets, the bench's cap), one persistent launch on the GPU against the
    oracle on bounded samples of the same models."""
    import paper_2001_11252_gb300 as rg
    import synth
    cap = args.batch_cap
    sub = synth.batch_models(args.batch_models, packet_scale=args.batch_scale, max_scatt=cap)[::16]
    ctx = rg.Context(0)
    w0 = sub[0]
    ctx.set_lines(w0.lines, w0.dust)
    ph = w0.physics
    ctx.set_physics(ph.recoil, ph.isotropic, 0, ph.x_gauss, cap, 0, ph.tau_stop, ph.seed)
    ctx.set_voigt(VOIGT)
    ctx.load_batch(sub, nbin=200)
    ctx.autotune_batch(max_scatt=max(1, min(cap // 20, 20000)))
    ctx.propagate_batch(rg.BATCH_PERSISTENT)
    t0 = time.perf_counter()
    st = ctx.propagate_batch(rg.BATCH_PERSISTENT)
    sec = time.perf_counter() - t0
    ctx.close()
    sc = st["nscatt_line"] + st["nscatt_dust"]
    for w in sub:
        w.physics.voigt = VOIGT
    o1 = _oracle_models_rate(sub, args.cpu_seconds / 6, 1)
    on = _oracle_models_rate(sub, args.cpu_seconds / 6, threads)
    return {"config": "C4 batch: every 16th of the %d models (%d), %g of their packets, cap %d scatterings"
                      % (args.batch_models, len(sub), args.batch_scale, cap),
            "packets": st["packets"], "gpu_s": sec, "gpu_scatt_per_s": sc / sec,
            "gpu_packets_per_s": st["packets"] / sec, "mean_scatterings": sc / st["packets"], "capped": st["capped"],
            "oracle_1_thread_scatt_per_s": o1[0], "oracle_threads": threads, "oracle_all_threads_scatt_per_s": on[0],
            "oracle_sample_packets": [o1[2], on[2]], "gpu_over_oracle_all_threads": (sc / sec) / on[0]}


def _config_galaxy(args, threads, adjoint=True):
    """C5 at equal work: (a) the galaxy as generated, packets capped at the
    bench's cap, peeling into 4 directions; (b) the adjoint of the cube on a
    150 000-leaf galaxy with every density x 1e-12 (peeling rays cross many
    leaves).  The oracle's detector in (a) is 4 x 32^2 x 40: a peeling ray
    adds into one bin either way, and the oracle keeps FP64 tallies per chunk
    of packets, which at 256^2 x 400 would take 0.84 GB each."""
    import torch
    import paper_2001_11252_gb300 as rg
    import synth
    dev = torch.device("cuda:0")
    tp = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
    rows = []
    # (a) forward
    m = args.galaxy_packets
    wl = synth.galaxy(n_packets=m)
    wl.physics.voigt = VOIGT
    wl.physics.max_scatt = args.galaxy_cap
    ctx = rg.Context(0)
    ctx.setup(wl)
    pk = wl.packets
    packets = (tp(pk.pos, torch.float64), tp(pk.dir, torch.float64), tp(pk.nu, torch.float64),
               tp(pk.ids.view(np.int64), torch.int64))
    ctx.propagate(*[a[:4096] for a in packets], stats=False)
    ctx.zero_tallies()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ctx.propagate(*packets, stats=True)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    ctx.close()
    d = wl.detector
    wl.detector = synth.Detector(d.nu_lo, d.nu_hi, 40, dirs=d.dirs, npix=32, fov=d.fov, centre=d.centre, cube=d.cube)
    o1 = _oracle_rate(wl, args.cpu_seconds / 6, 1)
    on = _oracle_rate(wl, args.cpu_seconds / 6, threads, chunk=None)
    sc = st["nscatt_line"] + st["nscatt_dust"]
    rows.append({"config": "C5 galaxy as generated (%d leaves), cap %d scatterings, peeling 4 directions"
                           % (wl.medium.tree.nleaf, args.galaxy_cap),
                 "packets": m, "gpu_s": sec, "gpu_scatt_per_s": sc / sec, "gpu_packets_per_s": m / sec,
                 "mean_scatterings": sc / m, "peel_rays": st["npeel_rays"], "capped": st["capped"],
                 "oracle_1_thread_packets_per_s": o1[1], "oracle_threads": threads,
                 "oracle_all_threads_packets_per_s": on[1], "oracle_1_thread_scatt_per_s": o1[0],
                 "oracle_all_threads_scatt_per_s": on[0], "oracle_sample_packets": [o1[2], on[2]],
                 "gpu_over_oracle_all_threads": (m / sec) / on[1]})
    del wl
    if not adjoint:
        return rows
    # (b) adjoint on a cut-out
    import oracle
    n = 4096
    wl = synth.galaxy(n_leaf=150_000, grid_level=6, base_level=4, max_level=10, n_packets=n, npix=16, nchan=40)
    md = wl.medium
    for f in ("n_HI", "n_dust", "n_metal"):
        setattr(md, f, (np.asarray(getattr(md, f), np.float32) * np.float32(1e-12)).astype(np.float32))
    wl.physics.voigt = VOIGT
    wl.physics.max_scatt = 64
    ctx = rg.Context(0)
    ctx.setup(wl)
    pk = wl.packets
    packets = (tp(pk.pos, torch.float64), tp(pk.dir, torch.float64), tp(pk.nu, torch.float64),
               tp(pk.ids.view(np.int64), torch.int64))
    st = ctx.propagate(*packets, stats=True)
    g = torch.ones((len(wl.detector.dirs), wl.detector.npix, wl.detector.npix, wl.detector.nbin), device=dev)
    ctx.peel_adjoint(*packets, g_cube=g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.peel_adjoint(*packets, g_cube=g)
    torch.cuda.synchronize()
    gsec = time.perf_counter() - t0
    ctx.close()
    o = oracle.Oracle(wl)
    k = 64
    while True:
        _, tal = o.run(lo=0, hi=k, threads=1, record_events=1 << 21)
        ev = tal["events"]
        t0 = time.perf_counter()
        o.adjoint(ev, g_cube=np.ones((len(wl.detector.dirs), wl.detector.npix, wl.detector.npix,
                                      wl.detector.nbin)))
        osec = time.perf_counter() - t0
        if osec >= args.cpu_seconds / 12 or k >= n:
            break
        k *= 2
    rows.append({"config": "C5 adjoint of the 4 x 16^2 x 40 cube, 150 000-leaf galaxy, densities x 1e-12, cap 64",
                 "packets": n, "gpu_s": gsec, "gpu_peel_rays_per_s": st["npeel_rays"] / gsec,
                 "gpu_leaves_per_ray": st["npeel_cells"] / max(1, st["npeel_rays"]),
                 "oracle_1_thread_peel_rays_per_s": ev.size / osec, "oracle_sample_packets": k,
                 "oracle_events": int(ev.size),
                 "gpu_over_oracle_1_thread": (st["npeel_rays"] / gsec) / (ev.size / osec)})
    return rows


# ------------------------------------------------------------------ galaxy section
def run_galaxy(args, peaks):
    """Synthetic galaxy (~1e7 leaves, levels 6-12, three lines, dust,
    turbulence): (a) optical depths of rays from emitting leaves to the box
    border at Lya line centre (the peeling integral on its own, the
    HBM-bound walk), (b) propagation with peeling into 4 directions and
    256x256x400 cubes, (c) the adjoint of those cubes."""
    import torch
    import paper_2001_11252_gb300 as rg
    import synth
    t0 = time.perf_counter()
    wl = synth.galaxy(n_packets=max(args.galaxy_rays, args.galaxy_packets, args.galaxy_all_packets))
    wl.physics.voigt = VOIGT
    gen_s = time.perf_counter() - t0
    dev = torch.device("cuda:0")
    ctx = rg.Context(0)
    ctx.setup(wl)
    ph = wl.physics
    ctx.set_physics(ph.recoil, ph.isotropic, 0, ph.x_gauss, args.galaxy_cap, 0, ph.tau_stop, ph.seed)
    tree = wl.medium.tree
    out = {"leaves": tree.nleaf, "octs": tree.noct, "levels": [int(tree.leaf_level.min()), int(tree.leaf_level.max())],
           "generate_s": gen_s}
    # (a) ray casting
    n = args.galaxy_rays
    rng = np.random.default_rng(7)
    mu = 2 * rng.random(n) - 1
    phi = 2 * math.pi * rng.random(n)
    st = np.sqrt(1 - mu * mu)
    d = np.stack([st * np.cos(phi), st * np.sin(phi), mu], 1)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev, torch.float64)
    pos, dr = t(wl.packets.pos[:n]), t(d)
    nu = t(np.full(n, synth.nu_of(wl.lines[0].lambda_A)))
    ctx.ray_tau(pos, dr, nu)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tau, _, _, ncell = ctx.ray_tau(pos, dr, nu)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    cells = int(ncell.sum().item())
    alg = cells * 28.0   # n_HI, v(3), T, n_dust, n_Si per leaf visit
    hbm = peaks.get("hbm_gbs", 6671.9)
    out["ray_cast"] = {"rays": n, "cells": cells, "ms": ms, "rays_per_s": n / (ms * 1e-3),
                       "cells_per_s": cells / (ms * 1e-3),
                       "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                                    "frac": alg / (ms * 1e-3) / 1e9 / hbm,
                                    "traffic": RAY_DRAM_BYTES_PER_VISIT * cells,
                                    "note": "28 algorithmic bytes per leaf visit; peak = measured copy bandwidth; "
                                            "traffic = DRAM bytes per leaf visit of a 2^18-ray ncu capture x the "
                                            "visits of this launch"}}
    # (b) column densities along the same rays (12 algorithmic bytes per leaf
    # visit: n_HI, n_dust, n_metal)
    ctx.ray_columns(pos, dr, 6.3e-18, 4e-22)
    torch.cuda.synchronize()
    e0.record(stream)
    cols, ctau, cnc = ctx.ray_columns(pos, dr, 6.3e-18, 4e-22)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ccells = int(cnc.sum().item())
    alg = ccells * 12.0
    out["columns"] = {"rays": n, "cells": ccells, "ms": ms, "rays_per_s": n / (ms * 1e-3),
                      "cells_per_s": ccells / (ms * 1e-3),
                      "median_N_HI": float(cols[:, 0].median().item()),
                      "escape_fraction_13.6eV": float(torch.exp(-ctau).mean().item()),
                      "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                                   "frac": alg / (ms * 1e-3) / 1e9 / hbm, "traffic": None,
                                   "note": "12 algorithmic bytes per leaf visit (n_HI, n_dust, n_metal); the walk "
                                           "reads the leaf's 32-byte record (one sector)"}}
    # (c) propagation with peeling into the 4 x 256^2 x 400 cubes, (d) adjoint
    m = args.galaxy_packets
    pk = wl.packets
    tp = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
    packets = (tp(pk.pos[:m], torch.float64), tp(pk.dir[:m], torch.float64), tp(pk.nu[:m], torch.float64),
               tp(pk.ids[:m].view(np.int64), torch.int64))
    ph = wl.physics

    def peel_run(label, cap, core_skip_f=0.0, npk=None):
        args_p = packets
        if npk is not None:
            args_p = (tp(pk.pos[:npk], torch.float64), tp(pk.dir[:npk], torch.float64),
                      tp(pk.nu[:npk], torch.float64), tp(pk.ids[:npk].view(np.int64), torch.int64))
        ctx.set_physics(ph.recoil, ph.isotropic, 0, ph.x_gauss, cap, 0, ph.tau_stop, ph.seed, 0, 0.0, core_skip_f)
        ctx.zero_tallies()
        ctx.propagate(*[a[:4096] for a in args_p], stats=False)
        torch.cuda.synchronize()
        ctx.zero_tallies()
        t0 = time.perf_counter()
        stp = ctx.propagate(*args_p, stats=True)
        torch.cuda.synchronize()
        tprop = time.perf_counter() - t0
        rays, cells = stp["npeel_rays"], stp["npeel_cells"]
        n_p = args_p[0].shape[0]
        return stp, {"medium": label, "packets": n_p, "cap": cap, "core_skip_f": core_skip_f, "seconds": tprop,
                     "packets_per_s": n_p / tprop,
                     "scatterings": stp["nscatt_line"] + stp["nscatt_dust"],
                     "mean_scatterings": (stp["nscatt_line"] + stp["nscatt_dust"]) / n_p,
                     "peel_rays": rays, "peel_cells": cells,
                     "cells_per_ray": cells / max(1, rays), "peel_rays_per_s": rays / tprop,
                     "peel_cells_per_s": cells / tprop,
                     "peel_hbm_gbs_lower_bound": 28.0 * cells / tprop / 1e9,
                     "capped": stp["capped"], "escaped": stp["escaped"], "absorbed": stp["absorbed"]}

    # as generated: the sources sit in the densest leaves (line-centre tau to
    # the border >= 5e8, dust >= 4e4); with a 64-scattering cap most packets
    # end CAPPED, with core-skipping every packet ends uncapped
    _, out["peel_capped"] = peel_run("as generated, capped", args.galaxy_cap)
    nall = min(pk.n, args.galaxy_all_packets)
    _, out["core_skip"] = peel_run("as generated, core-skipping, %d packets" % nall, args.galaxy_cs_cap,
                                   args.galaxy_core_skip, npk=nall)
    # the same octree and fields with every density scaled down: peeling rays
    # cross the galaxy and the adjoint has work to do
    mm = wl.medium
    nm = getattr(mm, "n_metal", None)

    def scale_fields(sc):
        ctx.update_fields(np.asarray(mm.n_HI, np.float32) * sc, mm.vx, mm.vy, mm.vz, mm.T,
                          np.asarray(mm.n_dust, np.float32) * sc,
                          None if nm is None else np.asarray(nm, np.float32) * sc)

    sc = args.galaxy_thin
    scale_fields(sc)
    stp, out["peel_thin"] = peel_run("densities x %g" % sc, args.galaxy_cap)
    g = torch.randn((len(wl.detector.dirs), wl.detector.npix, wl.detector.npix, wl.detector.nbin), device=dev)
    ctx.peel_adjoint(*packets, g_cube=g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grad = ctx.peel_adjoint(*packets, g_cube=g)
    torch.cuda.synchronize()
    tadj = time.perf_counter() - t0
    out["adjoint"] = {"medium": "densities x %g" % sc, "seconds": tadj,
                      "peel_rays_per_s": stp["npeel_rays"] / tadj,
                      "cells_per_s_two_walks": 2 * stp["npeel_cells"] / tadj,
                      "grad_nonzero_leaves": int((grad[0] != 0).sum().item())}
    scale_fields(sc * 1e-2)
    _, out["peel_thinner"] = peel_run("densities x %g" % (sc * 1e-2), args.galaxy_cap)
    ctx.close()
    return out


# ------------------------------------------------------------------ one launch (profiling)
def run_kernel(args):
    """One propagation of --packets packets of the headline workload (capped
    at --max-scatt scatterings when given), timed with CUDA events: the
    command the kernel profiles are taken on."""
    import torch
    import paper_2001_11252_gb300 as rg
    dev = torch.device("cuda:0")
    wl = workload(8)
    ctx = rg.Context(0)
    ctx.setup(wl)
    ph = wl.physics
    if args.max_scatt:
        ctx.set_physics(ph.recoil, ph.isotropic, ph.keep_direction, ph.x_gauss, args.max_scatt, 0, ph.tau_stop,
                        ph.seed)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    pk = packets(wl, 0, args.packets)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
    args_d = (t(pk.pos, torch.float64), t(pk.dir, torch.float64), t(pk.nu, torch.float64),
              t(pk.ids.view(np.int64), torch.int64))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = ctx.propagate(*args_d, stats=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sc = st["nscatt_line"] + st["nscatt_dust"]
    return {"packets": args.packets, "cap": args.max_scatt, "ms": ms, "scatterings": sc,
            "scatt_per_s": sc / (ms * 1e-3), "stats": st}


def run_peel(args):
    """One propagation with peeling through the synthetic galaxy with every
    density scaled by --galaxy-thin: the command the peel-kernel profile is
    taken on."""
    import torch
    import paper_2001_11252_gb300 as rg
    import synth
    m = args.galaxy_packets
    wl = synth.galaxy(n_packets=m)
    wl.physics.voigt = VOIGT
    mm = wl.medium
    for f in ("n_HI", "n_dust", "n_metal"):
        setattr(mm, f, (np.asarray(getattr(mm, f), np.float32) * np.float32(args.galaxy_thin)).astype(np.float32))
    ctx = rg.Context(0)
    ctx.setup(wl)
    ph = wl.physics
    ctx.set_physics(ph.recoil, ph.isotropic, 0, ph.x_gauss, args.galaxy_cap, 0, ph.tau_stop, ph.seed)
    pk = wl.packets
    dev = torch.device("cuda:0")
    tp = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
    packets = (tp(pk.pos, torch.float64), tp(pk.dir, torch.float64), tp(pk.nu, torch.float64),
               tp(pk.ids.view(np.int64), torch.int64))
    torch.cuda.synchronize()
    if args.peel_adjoint:
        # the adjoint of the cube alone (its replay and the gradient walks)
        g = torch.randn((len(wl.detector.dirs), wl.detector.npix, wl.detector.npix, wl.detector.nbin), device=dev)
        t0 = time.perf_counter()
        grad = ctx.peel_adjoint(*packets, g_cube=g)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return {"packets": m, "thin": args.galaxy_thin, "adjoint_seconds": dt,
                "grad_nonzero_leaves": int((grad[0] != 0).sum().item())}
    t0 = time.perf_counter()
    st = ctx.propagate(*packets, stats=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"packets": m, "thin": args.galaxy_thin, "seconds": dt, "peel_rays": st["npeel_rays"],
            "peel_cells": st["npeel_cells"], "cells_per_ray": st["npeel_cells"] / max(1, st["npeel_rays"])}


# ------------------------------------------------------------------ our arm
def main():
    global VOIGT
    args = parse()
    VOIGT = 1 if args.voigt == "faddeeva" else 0
    if args.impl == "reference":
        return run_reference(args)
    if args.section in ("batch", "galaxy", "configs", "kernel", "peel"):
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        res = (run_batch(args) if args.section == "batch" else
               run_galaxy(args, peaks) if args.section == "galaxy" else
               run_kernel(args) if args.section == "kernel" else
               run_peel(args) if args.section == "peel" else run_configs(args))
        print(json.dumps({"section": args.section, args.section: res}), flush=True)
        return
    import torch
    import paper_2001_11252_gb300 as rg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    P = args.packets
    wl = workload(8)
    ctx = rg.Context(local)
    ctx.setup(wl)
    if args.max_scatt:
        ph = wl.physics
        ctx.set_physics(ph.recoil, ph.isotropic, ph.keep_direction, ph.x_gauss, args.max_scatt, 0, ph.tau_stop,
                        ph.seed)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    rates = None
    try:
        rates = ctx.probe_issue_rates()    # ~0.1 s, before the timed region
    except Exception as e:                 # the roofline then has no peak
        print("issue-rate probe failed: %s" % e, file=sys.stderr)

    def dev_packets(step):
        pk = packets(wl, shard_first(rank, step, args.warmup, args.steps, P), P)
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
        return pk, (t(pk.pos, torch.float64), t(pk.dir, torch.float64), t(pk.nu, torch.float64),
                    t(pk.ids.view(np.int64), torch.int64))

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    inputs = [dev_packets(s) for s in range(args.warmup + args.steps)]
    for s in range(args.warmup):
        ctx.propagate(*inputs[s][1], stats=False)
    torch.cuda.synchronize()

    # ---- device-resident timed region
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    scatt = pk_done = 0
    stats_all = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            e0, e1 = evs[i]
            e0.record(stream)
            st = ctx.propagate(*inputs[args.warmup + i][1], stats=True)
            e1.record(stream)
            stats_all.append(st)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = sum(step_ms)
    scatt = sum(s["nscatt_line"] + s["nscatt_dust"] for s in stats_all)
    pk_done = sum(s["packets"] for s in stats_all)
    loads = sum(s["leaf_loads"] for s in stats_all)
    sons = sum(s["son_loads"] for s in stats_all)
    nbrs = sum(s["nbor_loads"] for s in stats_all)
    tmax, (tot_scatt, tot_pk) = reduce_over_ranks(dist, dev, t_ms, (scatt, pk_done))

    # ---- end to end through the C ABI with host buffers (copies in the timed region)
    e2e_inputs = [packets(wl, shard_first(rank, args.warmup + i, args.warmup, args.steps, P), P)
                  for i in range(args.steps)]
    outs = [{"status": np.zeros(P, np.int32), "nscatt": np.zeros(P, np.int64), "nu": np.zeros(P)}
            for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_scatt = 0
    for i in range(args.steps):
        pk = e2e_inputs[i]
        st = ctx.propagate(pk.pos, pk.dir, pk.nu, pk.ids, out=outs[i], stats=True)
        e2e_scatt += st["nscatt_line"] + st["nscatt_dust"]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s, (e2e_scatt,) = reduce_over_ranks(dist, dev, e2e_s, (e2e_scatt,))
    h2d = P * (3 + 3 + 1 + 1) * 8
    d2h = P * (4 + 8 + 8)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = tot_scatt / (tmax * 1e-3)
    pk_rate = tot_pk / (tmax * 1e-3)
    clk = clk.summary()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_mhz = clk["sm_mhz"] or 1900.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # Issue roofline of the scattering loop: its warp instructions per second
    # against the measured issue rate of the FP32 FMA pipe (one warp
    # instruction per clock per scheduler), and each pipe the loop uses
    # against that pipe's own measured rate.
    roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "Gwarp-inst/s", "frac": None, "traffic": None}
    if rates and INST_PER_SCATT:
        ach = INST_PER_SCATT * scatt / (t_ms * 1e-3) / 1e9
        peak = rates["ffma"] / 1e9
        lane_peak = sms * 128 * sm_mhz * 1e6 / 1e12   # T lane-instructions / s
        lane_ach = INST_PER_SCATT * LANES_PER_INST * scatt / (t_ms * 1e-3) / 1e12
        roof.update({"achieved": ach, "peak": peak, "frac": ach / peak,
                     "peak_note": "measured: FP32 FMA warp-instructions/s of the issue-rate probe "
                                  "(rascas_probe_issue_rates) on this GPU before the timed region (%d SMs; "
                                  "nominal %d x 4 schedulers x %.0f MHz = %.0f G)"
                                  % (sms, sms, sm_mhz, sms * 4 * sm_mhz * 1e-3),
                     "lanes": {"achieved": lane_ach, "peak": lane_peak, "unit": "Tlane-inst/s",
                               "frac": lane_ach / lane_peak,
                               "note": "the same count x %.2f active lanes per warp instruction, against %d SMs x "
                                       "128 lanes x SM clock: divergence shows here" % (LANES_PER_INST, sms)}})
        pipes = {}
        rate_of = {"fma": rates["ffma"], "fp64": rates["dfma"], "xu": rates["mufu"]}
        for pipe, per in PIPE_PER_SCATT.items():
            if pipe in rate_of and rate_of[pipe] > 0:
                pipes[pipe] = {"warp_inst_per_scatt": per,
                               "frac": per * scatt / (t_ms * 1e-3) / rate_of[pipe]}
        if pipes:
            roof["pipes"] = pipes
        roof["measured_rates_gwarp_inst_s"] = {k: v / 1e9 for k, v in rates.items()}
    cell_bytes = loads * 24 + sons * 4 + nbrs * 28
    hbm = peaks.get("hbm_gbs", 6671.9)
    line = {"metric": METRIC, "value": value, "unit": "scatterings/s", "packets_per_s": pk_rate,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmax / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "voigt": args.voigt, "packets_per_step": P, "per_rank": True,
                       "l2": "256 MB buffer written between timed steps (L2 flush)",
                       "mean_scatterings_per_packet": scatt / max(1, pk_done)},
            "roofline": roof,
            "hbm_cell_bytes": {"achieved_gbs": cell_bytes / (t_ms * 1e-3) / 1e9, "peak_gbs": hbm,
                               "frac": cell_bytes / (t_ms * 1e-3) / 1e9 / hbm,
                               "note": "algorithmic leaf/tree bytes touched (24 B per leaf visit, 4 B per son, "
                                       "28 B per neighbour record) / time; of measured copy bandwidth"},
            "e2e": {"value": e2e_scatt / e2e_s, "unit": "scatterings/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps,
            "clocks": clk}
    if args.batch_models > 0 and world == 1 and args.section == "all":
        line["batch"] = run_batch(args)
    if args.galaxy and world == 1 and args.section == "all":
        line["galaxy"] = run_galaxy(args, peaks)
    if not args.no_cpu_baseline and world == 1:
        threads = os.cpu_count() or 1
        sc, pr, npk, secs = cpu_oracle_rate(workload, args.cpu_seconds, threads)
        line["cpu_baseline"] = {"value": sc, "unit": "scatterings/s", "cores": threads, "kind": "oracle",
                                "sample": "%d packets of the workload (%.1f s on %d threads), %.3g packets/s"
                                          % (npk, secs, threads, pr), "host": host_cpu()}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
