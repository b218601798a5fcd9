#!/usr/bin/env python
"""Benchmark of the fused bump-function LBM step on GB300.

One step = one pass of the whole hot path over the lattice: pull streaming,
moments, isotropic-gradient corrections, equilibrium + forcing, BGK, store,
and the FP64 mass/momentum/energy reduction of the state (recorded every
step).  Default workload: the 3D periodic D3Q19 256^3 solenoidal-turbulence
configuration in FP32 (the paper's own lattice, and the largest single-GPU
configuration); --workload tgv2d | sound1d | riemann1d select the others,
and --workload std3d times the standard-lattice comparator (BGK with the
Hermite equilibrium of Eq. 4) on the same lattice as a speed reference.

Prints one JSON line (rank 0).  Under torchrun each rank advances its own
copy of the workload (independent replicas, weak scaling, no collective on
the data path); timing is the max over ranks.

--impl reference times the FP64 CPU oracle (the reference arm) on a bounded
sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline at stated error vs FP64 oracle; serving p50/p99"

WORKLOAD_TEXT = {
    "turb3d": "D3Q19 256^3 periodic; seeded solenoidal u, E(k)~k^4 exp(-2k^2/k0^2), k0=8, "
              "Mach_rms 0.3; rho=1, T=T0=0.05; tau=0.52; isothermal",
    "tgv2d": "D2Q9 2048^2 periodic; Taylor-Green u0=0.1 + Gaussian rho/T pulse (amp 0.2, sigma 64); "
             "T0=0.1; tau=0.6; thermal",
    "std3d": "standard-lattice comparator (BGK, Hermite equilibrium of Eq. 4) on D3Q19 256^3 periodic; "
             "the turb3d velocity field (Mach 0.12 at cs2 = 1/3); T0=1/3; tau=0.52",
    "channel3d": "D3Q19 256^3 plane Poiseuille channel: half-way bounce-back walls normal to z, uniform "
                 "acceleration 1e-7 along x, from rest (rho=1, u=0, T=T0=0.1); tau=0.6; isothermal",
    "mrt3d": "the turb3d lattice and fields with the MRT collision of Appendix B (s3=1.2, s4=1.4)",
    "sound1d": "D1Q3 256 periodic sound wave, rho=1+1e-3 sin(2 pi x/256), T0=1/3, tau=0.8; isothermal",
    "riemann1d": "D1Q3 4096 two-state Riemann (rho 1:0.125, T 1.0:0.8 x 0.15), tau=0.55; thermal; "
                 "fixed-state ends",
    "serve": "serving mix: seeded Poisson arrivals at 200/s of 1000 requests, half D1Q3 (nx log-uniform "
             "64-65536), half D2Q9 (N^2, N log-uniform 64-1024), half sound waves (tau 0.8, T0 1/3), half "
             "Riemann (tau 0.55, T0 0.15, thermal, fixed-state x), steps uniform 100-5000; FP32, except FP64 for "
             "the 1D Riemann requests (the server's precision policy)",
}


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="turb3d", choices=sorted(WORKLOAD_TEXT))
    p.add_argument("--dtype", default=None, help="storage dtype override: f64 f32 f16 bf16")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--scale", type=int, default=0,
                   help="grid edge of a smaller instance of the workload (profiling captures); 0: full size")
    p.add_argument("--tile", type=int, default=-1, help="force a kernel tile variant (-1: autotuned)")
    p.add_argument("--chunk", type=int, default=0, help="force planes per block (0: autotuned)")
    p.add_argument("--steps-per-launch", type=int, default=0,
                   help="steps per cooperative launch (1D, small 2D; 0: autotuned, 1: single launches)")
    p.add_argument("--cluster", type=int, default=0,
                   help="small periodic 2D lattices: cluster-resident kernel (-1 never, 0 autotuned, 1+v variant v)")
    p.add_argument("--no-diagnostics", action="store_true",
                   help="steps without the per-step conservation sums (lbm_opts.diagnostics = 0)")
    p.add_argument("--inplace", action="store_true",
                   help="the in-place step (one population buffer, two passes per step)")
    p.add_argument("--no-others", action="store_true",
                   help="skip the short measurements of the other workloads that follow the default "
                        "(turb3d, one GPU) line's own measurement")
    p.add_argument("--requests", type=int, default=1000, help="serve: number of requests of the mix")
    p.add_argument("--rate", type=float, default=200.0,
                   help="serve: Poisson arrival rate (requests per second; the mix states 200)")
    p.add_argument("--no-sequential", action="store_true", help="serve: skip the one-at-a-time comparison")
    return p.parse_args(argv)


def max_over_ranks(x, dist, device="cuda"):
    """Largest value of x over all ranks -- the slowest rank's time decides a
    step of the whole job.  One all-reduce of a one-element tensor on
    `device` (cuda under NCCL, cpu under gloo); x itself without a process
    group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds_max):
    """Units all ranks processed per second when every rank does the same
    work (weak scaling) and the slowest rank's time counts."""
    return world * units_per_rank / seconds_max


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_uuid(dev):
    try:
        import torch
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


# ---------------------------------------------------------------------------
# roofline bookkeeping

def algorithmic_bytes_per_site(d, dtype, model="bump", inplace=False):
    Q = {1: 3, 2: 9, 3: 19}[d]
    NB = {1: 1, 2: 3, 3: 6}[d] if model == "bump" else 0
    fb = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[dtype]
    bb = 8 if dtype == "f64" else 4
    if inplace:
        # two passes: the state is read by both, written once; (u0, rho b)
        # (d + NB values) is written by the first and read by the second
        return 3 * (Q * fb + NB * bb) + 2 * (d + NB) * bb
    return 2 * (Q * fb + NB * bb)   # read + write of the emitted state


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


# the staged kernel's device code (it compiles from these headers alone) and its
# tile table
KERNEL_SOURCES = ("lbm_args.cuh", "lbm_lattice.cuh", "lbm_site.cuh", "lbm_tma.cuh", "lbm_lean.cuh", "lbm_mrt.cuh",
                  "lbm_step_fast.cuh", "lbm_fast_launch.cuh")


def _code_only(text):
    """C++ source without // and /* */ comments and blank lines: edits of
    comments do not change what is compiled."""
    out, i, n = [], 0, len(text)
    while i < n:
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif text[i] == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(text[i])
            i += 1
    return "\n".join(ln.rstrip() for ln in "".join(out).splitlines() if ln.strip())


# the comparator kernel's own sources
KERNEL_SOURCES_BY_KERNEL = {
    "std_step_kernel": ("lbm_args.cuh", "lbm_lattice.cuh", "lbm_site.cuh", "lbm_step.cuh", "lbm_mrt.cuh",
                        "lbm_std.cu"),
    "step_pair_kernel": ("lbm_args.cuh", "lbm_lattice.cuh", "lbm_site.cuh", "lbm_tma.cuh", "lbm_lean.cuh",
                         "lbm_f2.cuh", "lbm_step_pair.cuh", "lbm_pair_launch.cuh"),
}


def kernel_source_hash(kernel=None):
    """Hash of the code (comments stripped) of the device sources a step
    kernel is built from: an ncu figure taken from other code no longer
    describes the kernel."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES_BY_KERNEL.get(kernel, KERNEL_SOURCES):
        with open(os.path.join(ROOT, "paper_2501_00620_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload, dtype):
    """DRAM bytes per launch from the committed ncu summary of this kernel and
    workload, if it was captured from the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "%s_%s_%s.md" % (kernel, workload, dtype))
    try:
        text = open(p).read()
    except OSError:
        return None
    vals = {}
    for ln in text.splitlines():
        if ":" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha") != kernel_source_hash(kernel):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------

def workload_params(name, dtype_override):
    from paper_2501_00620_gb300 import workloads as W
    c = dict(W.CONFIGS[name])
    if dtype_override:
        c["dtype"] = dtype_override
    return c


def apply_settings(sim, c):
    """Body force and MRT rates of a workload, on the library's Simulation or
    the oracle's (the two share these method names)."""
    if c.get("force"):
        sim.set_force(list(c["force"]))
    if c.get("mrt"):
        sim.set_mrt(*c["mrt"])


def oracle_sample(name, budget_s, steps_total):
    """A bounded sample of the workload for the CPU oracle: a smaller lattice
    of the same generator, sized so that steps_total steps take ~budget_s."""
    import numpy as np
    import oracle
    from paper_2501_00620_gb300 import workloads as W
    c = W.CONFIGS[name]
    d = c["d"]
    threads = oracle.set_threads(os.cpu_count() or 1)
    # probe the oracle's rate on a small instance
    n_probe = {1: 4096, 2: 64, 3: 16}[d]
    sites_probe = n_probe ** (1 if d == 1 else d)
    rho, u, T = W.fields_for(name, scale=n_probe) if d > 1 else W.fields_for(name)
    if d == 1:
        sites_probe = c["nx"]
        n_probe = c["nx"]
    s = oracle.Sim(d, n_probe, n_probe if d >= 2 else 1, n_probe if d == 3 else 1, tau=c["tau"], T0=c["T0"],
                   thermal=c["thermal"], bc=c["bc"], model=c.get("model", "bump"))
    s.init(rho, u, T)
    apply_settings(s, c)
    t0 = time.perf_counter()
    s.step(2)
    rate = 2 * sites_probe / (time.perf_counter() - t0)
    if d == 1:
        return n_probe, threads, rate
    # at most 2M sites: the oracle keeps ~70 doubles per site
    target_sites = max(sites_probe, min(2.0e6, rate * budget_s / max(steps_total, 1)))
    n = int(target_sites ** (1.0 / d))
    n = max(8, min(n, c["nx"]))
    return n, threads, rate


def run_oracle(name, n, steps, warmup):
    import oracle
    from paper_2501_00620_gb300 import workloads as W
    c = W.CONFIGS[name]
    d = c["d"]
    rho, u, T = W.fields_for(name, scale=n) if d > 1 else W.fields_for(name)
    s = oracle.Sim(d, n, n if d >= 2 else 1, n if d == 3 else 1, tau=c["tau"], T0=c["T0"],
                   thermal=c["thermal"], bc=c["bc"], model=c.get("model", "bump"))
    s.init(rho, u, T)
    apply_settings(s, c)
    s.step(warmup)
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    sites = n ** d if d > 1 else n
    return sites * steps / dt / 1e6, dt, sites


def reference_serve_sample(budget_s):
    """The oracle over the serving mix in arrival order, each request run to
    its full step count, until about budget_s of CPU time: MLUPS."""
    import oracle
    from paper_2501_00620_gb300 import workloads as W
    t0 = time.perf_counter()
    updates, n = 0.0, 0
    for r in W.serving_requests(1000, 200.0, seed=0):
        rho, u, T = W.request_fields(r)
        tau, T0, thermal, bc = W.request_params(r)
        s = oracle.Sim(r["dim"], r["nx"], r["ny"], 1, tau=tau, T0=T0, thermal=thermal, bc=bc)
        s.init(rho, u, T)
        s.step(r["steps"])
        s.moments()
        updates += r["nx"] * r["ny"] * r["steps"]
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return updates / dt / 1e6, dt, n


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    name = args.workload
    if name == "serve":
        import oracle
        threads = oracle.set_threads(0)
        mlups, dt, n = reference_serve_sample(20.0)
        sample = "first %d requests of the serving mix, full step counts, %.1f s" % (n, dt)
        line = {
            "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": n, "warmup": 0, "ms_per_step": 1e3 * dt / max(n, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "serve: " + WORKLOAD_TEXT["serve"], "reference": "FP64 CPU oracle (oracle/)",
                       "step_unit": "one request"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    c = workload_params(name, None)
    n, threads, _ = oracle_sample(name, 120.0, args.steps + args.warmup)
    mlups, dt, sites = run_oracle(name, n, args.steps, args.warmup)
    d = c["d"]
    sample = ("%s sample: same generator on %s (%d sites), %d timed steps after %d warm-up"
              % (name, "x".join([str(n)] * d) if d > 1 else str(n), sites, args.steps, args.warmup))
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": name + ": " + WORKLOAD_TEXT[name], "reference": "FP64 CPU oracle (oracle/)"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def serve_measure(reqs, local, dist, world, sequential):
    """The requests through the continuous-batching server, submitted at their
    arrival times (after a few short warm-up requests); then, if
    `sequential`, the same requests one at a time through the plain entry
    points (create, init, step, moments, destroy)."""
    import numpy as np
    import torch
    from paper_2501_00620_gb300 import lbm
    from paper_2501_00620_gb300 import workloads as W

    sites = [r["nx"] * r["ny"] for r in reqs]
    updates = float(sum(n * r["steps"] for n, r in zip(sites, reqs)))
    # the server's precision policy: FP64 storage for 1D fixed-state (Riemann)
    # requests, FP32 for the rest
    def req_dtype(r):
        return "f64" if (r["dim"] == 1 and W.request_params(r)[3] == "fixed") else "f32"

    bytes_alg = float(sum(n * r["steps"] * algorithmic_bytes_per_site(r["dim"], req_dtype(r))
                          for n, r in zip(sites, reqs)))

    def submit(srv, r):
        rho, u, T = W.request_fields(r)
        tau, T0, thermal, bc = W.request_params(r)
        return srv.submit(r["dim"], r["nx"], r["ny"], tau, T0, thermal, bc, r["steps"], rho, u, T)

    srv = lbm.Server()
    for r in reqs[:8]:  # warm-up: kernel loading, first rounds
        srv.wait(submit(srv, dict(r, steps=min(r["steps"], 50))))
    base = srv.stats()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        delay = t0 + r["t_arrival"] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(submit(srv, r))
    results = [srv.wait(t, timeout=3600.0) for t in tickets]
    lat = np.array([r[3] for r in results])
    unstable = [dict(id=q["id"], kind=q["kind"], dim=q["dim"], nx=q["nx"], steps=q["steps"])
                for q, r in zip(reqs, results) if r.unstable]
    # requests on which the FP64 oracle itself leaves the physical range (a
    # list written by tests/golden/make_riemann_mix_oracle.py for the seeded
    # 1000-request mix)
    oracle_fatal = set()
    try:
        with open(os.path.join(ROOT, "tests", "golden", "riemann_mix_oracle.txt")) as fh:
            for ln in fh:
                if ln.strip() and not ln.startswith("#"):
                    rid, _, _, fatal = (int(v) for v in ln.split())
                    if fatal:
                        oracle_fatal.add(rid)
    except OSError:
        pass
    st = srv.stats()
    clocks = sampler.stop()
    srv.close()
    wall = max_over_ranks(st["last_done_s"] - max(st["first_submit_s"], base["last_done_s"]), dist)
    busy = st["busy_s"] - base["busy_s"]
    rounds = st["rounds"] - base["rounds"]
    launches = st["kernel_launches"] - base["kernel_launches"]
    value = whole_job_rate(updates, world, wall) / 1e6

    seq = None
    if sequential:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for r in reqs:
            rho, u, T = W.request_fields(r)
            tau, T0, thermal, bc = W.request_params(r)
            sim = lbm.Simulation(r["dim"], r["nx"], r["ny"], 1, tau=tau, T0=T0, bc=bc, dtype=req_dtype(r),
                                 thermal=thermal, device=local)
            sim.init(rho, u, T)
            sim.step(r["steps"])
            try:
                sim.moments()
            except lbm.LBMError as e:
                if e.status != lbm.LBM_EUNSTABLE:
                    raise
            sim.close()
        seq_s = time.perf_counter() - t1
        seq = {"value": updates / seq_s / 1e6, "unit": "MLUPS", "wall_s": seq_s,
               "how": "same requests in arrival order, one at a time: lbm_create, lbm_init, lbm_step, "
                      "lbm_moments, lbm_destroy (the server's storage per request, autotuned "
                      "single-simulation kernels)"}
    return dict(lat=lat, unstable=unstable, seq=seq, clocks=clocks, wall=wall, busy=busy, rounds=rounds,
                launches=launches, value=value, updates=updates, bytes_alg=bytes_alg, sites=sites,
                oracle_fatal=oracle_fatal)


def run_serve(args):
    """The serving mix through the continuous-batching server, submitted in
    real time; then, unless --no-sequential, the same requests one at a time
    through the plain entry points (create, init, step, moments, destroy)."""
    rank, world, local = dist_env()
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_00620_gb300 import lbm
    from paper_2501_00620_gb300 import workloads as W

    reqs = W.serving_requests(args.requests, args.rate, seed=0)
    m = serve_measure(reqs, local, dist, world, not args.no_sequential)
    lat, unstable, seq, clocks = m["lat"], m["unstable"], m["seq"], m["clocks"]
    wall, busy, rounds, launches, value = m["wall"], m["busy"], m["rounds"], m["launches"], m["value"]
    updates, bytes_alg, sites = m["updates"], m["bytes_alg"], m["sites"]
    oracle_fatal = m["oracle_fatal"]
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    peak, peak_src = hbm_peak()
    achieved = bytes_alg / busy / 1e9 if busy > 0 else None
    h2d = float(sum((2 + r["dim"]) * n * 8 for n, r in zip(sites, reqs)))
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": len(reqs),
        "warmup": 8, "ms_per_step": 1e3 * wall / len(reqs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (f64 for 1D fixed-state requests)", "data": "synthetic",
        "config": {"workload": "serve: " + WORKLOAD_TEXT["serve"], "requests": len(reqs), "rate_per_s": args.rate,
                   "site_updates": updates, "step_unit": "one request (steps and ms_per_step count requests)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "kernel": "serve_kernel (persistent cooperative kernel: rounds of K steps posted through a "
                             "mapped-memory mailbox, start states and moments of admitted and finishing requests "
                             "computed in their rounds; host loop pipelined one round deep)"},
        "serving": {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "max_s": float(lat.max()), "wall_s": wall, "busy_s": busy, "rounds": rounds,
                    "kernel_launches": launches,
                    "offered_mlups": updates / max(reqs[-1]["t_arrival"], 1e-9) / 1e6,
                    "unstable_requests": len(unstable),
                    "unstable_also_in_fp64_oracle": (sum(1 for q in unstable if q["id"] in oracle_fatal)
                                                     if len(reqs) == 1000 else None),
                    "fp64_oracle_unstable_in_mix": len(oracle_fatal) if len(reqs) == 1000 else None,
                    "unstable_examples": unstable[:5],
                    "sequential": seq},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": None, "peak_source": peak_src,
                     "kernel": "serve_kernel", "launches": launches, "rounds": rounds,
                     "duration": "device clock (%globaltimer) at the start and end of each round (busy_s)"},
        "cpu_baseline": None,
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": h2d / len(reqs),
                "d2h_bytes_per_step": h2d / len(reqs),
                "includes": "per request: fields copied in at submit, results copied out at completion; "
                            "time from first submit to last completion"},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# Short measurements of the other workloads, run after the headline one (outside
# its timed region) so that one default bench run reports every kernel family:
# (workload, storage, timed steps, warm-up steps).  Each is timed with CUDA
# events on its own stream after the autotuner has run, like the headline.
OTHER_WORKLOADS = (("tgv2d", "f32", 50, 5), ("tgv2d", "f16", 50, 5), ("tgv2d", "bf16", 50, 5),
                   ("std3d", "f32", 40, 5), ("channel3d", "f32", 40, 5), ("mrt3d", "f32", 40, 5),
                   ("sound1d", "f64", 2000, 5), ("riemann1d", "f64", 5000, 5), ("riemann1d", "f32", 1000, 5))


def measure_others(local, fields_cache):
    import numpy as np
    import torch
    from paper_2501_00620_gb300 import lbm
    from paper_2501_00620_gb300 import workloads as W
    peak, peak_src = hbm_peak()
    out = []
    for name, dtype, steps, warm in OTHER_WORKLOADS:
        c = workload_params(name, dtype)
        d, nx, ny, nz = c["d"], c["nx"], c["ny"], c["nz"]
        N = nx * ny * nz
        if name in ("mrt3d", "std3d") and "turb3d" in fields_cache:
            # the turb3d fields (std3d: at its own uniform T0)
            rho, u, T = fields_cache["turb3d"]
            if name == "std3d":
                T = np.full_like(rho, c["T0"])
        else:
            if name not in fields_cache:
                fields_cache[name] = W.fields_for(name)
            rho, u, T = fields_cache[name]
        stream = torch.cuda.Stream(device=local)
        sim = lbm.Simulation(d, nx, ny, nz, tau=c["tau"], T0=c["T0"], bc=c["bc"], dtype=dtype,
                             thermal=c["thermal"], device=local, stream=stream.cuda_stream,
                             model=c.get("model", "bump"))
        sim.init(rho, u, T)
        apply_settings(sim, c)
        sim.step(warm)
        sim.sync()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        sim.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        status = "ok"
        try:
            sim.moments()
        except lbm.LBMError as e:
            status = "unstable" if e.status == lbm.LBM_EUNSTABLE else "error %d" % e.status
        tile, chunk, kernel = sim.launch_config()
        sim.close()
        bps = algorithmic_bytes_per_site(d, dtype, c.get("model", "bump"))
        rec = {"workload": name, "storage": dtype, "sites": N, "steps": steps,
               "ms_per_step": ms / steps, "mlups": N * steps / (ms * 1e-3) / 1e6,
               "kernel": kernel, "tile": tile, "chunk": chunk, "final_state": status}
        if d > 1:
            ach = N * bps / (ms / steps * 1e-3) / 1e9
            rec["roofline"] = {"bytes_per_site": bps, "achieved_gbs": ach, "frac": ach / peak,
                               "peak_source": peak_src}
        else:
            rec["time_to_result_ms"] = ms
        out.append(rec)
    # the serving path: the first 200 requests of the seeded mix at its rate,
    # then the same requests one at a time
    reqs = W.serving_requests(200, 200.0, seed=0)
    m = serve_measure(reqs, local, None, 1, True)
    out.append({"workload": "serve: first 200 requests of the seeded mix at 200/s", "kernel": "serve_kernel",
                "mlups": m["value"], "p50_s": float(np.percentile(m["lat"], 50)),
                "p99_s": float(np.percentile(m["lat"], 99)),
                "offered_mlups": m["updates"] / max(reqs[-1]["t_arrival"], 1e-9) / 1e6,
                "sequential_mlups": m["seq"]["value"], "rounds": m["rounds"], "kernel_launches": m["launches"],
                "unstable_requests": len(m["unstable"]),
                "final_state": "ok" if not m["unstable"] else "%d flagged" % len(m["unstable"])})
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "serve":
        return run_serve(args)

    rank, world, local = dist_env()
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2501_00620_gb300 import lbm
    from paper_2501_00620_gb300 import workloads as W

    name = args.workload
    c = workload_params(name, args.dtype)
    if args.scale:
        c["nx"] = args.scale
        c["ny"] = args.scale if c["d"] >= 2 else 1
        c["nz"] = args.scale if c["d"] == 3 else 1
    d, nx, ny, nz = c["d"], c["nx"], c["ny"], c["nz"]
    N = nx * ny * nz
    rho, u, T = W.fields_for(name, scale=args.scale or None)

    stream = torch.cuda.Stream(device=local)
    sim = lbm.Simulation(d, nx, ny, nz, tau=c["tau"], T0=c["T0"], bc=c["bc"], dtype=c["dtype"],
                         thermal=c["thermal"], device=local, stream=stream.cuda_stream,
                         diagnostics=not args.no_diagnostics,
                         tile=args.tile, chunk=args.chunk, model=c.get("model", "bump"), inplace=args.inplace,
                         steps_per_launch=args.steps_per_launch, cluster=args.cluster)
    sim.init(rho, u, T)
    apply_settings(sim, c)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (includes autotuning and graph capture)
    sim.step(max(args.warmup, 3))
    sim.sync()
    barrier()

    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    sim.step(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    barrier()
    clocks = sampler.stop()
    sim.sync()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, dist)
    value = whole_job_rate(N * args.steps, world, ms_max * 1e-3) / 1e6
    ms_per_step = ms_max / args.steps

    # roofline of the step kernel (one launch per step)
    bps = algorithmic_bytes_per_site(d, c["dtype"], c.get("model", "bump"), args.inplace)
    # one buffer of the emitted state (the A-B form; the in-place form keeps
    # one population buffer and two variance buffers)
    state_b = N * algorithmic_bytes_per_site(d, c["dtype"], c.get("model", "bump")) / 2
    tile, chunk, kernel = sim.launch_config()
    if kernel in ("step_multi_kernel", "step_cluster_kernel"):
        launches = -(-args.steps // chunk)  # chunk = steps per launch
    else:
        launches = args.steps * (2 if args.inplace else 1)
    achieved = N * bps / (ms_per_step * 1e-3) / 1e9
    peak, peak_src = hbm_peak()
    traffic = profiled_traffic(kernel, name, c["dtype"])

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e and not args.no_diagnostics:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hr, hu, hT = pin(rho), pin(u), pin(T)
        orr = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
        ou = torch.empty(d * N, dtype=torch.float64).pin_memory().numpy()
        oT = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
        rec = np.empty(d + 3)
        # one untimed pass through the same host buffers first (the first DMA
        # from or to freshly pinned pages can cost far more than the copy)
        lbm.lbm_init(sim.h, hr, hu, hT)
        lbm.lbm_moments(sim.h, orr, ou, oT)
        barrier()
        t0 = time.perf_counter()
        lbm.lbm_init(sim.h, hr, hu, hT)
        t1 = time.perf_counter()
        for _ in range(args.steps):
            lbm.lbm_step(sim.h, 1)
            lbm.lbm_last_diagnostics(sim.h, rec)
        t2 = time.perf_counter()
        lbm.lbm_moments(sim.h, orr, ou, oT)
        t3 = time.perf_counter()
        te = max_over_ranks(t3 - t0, dist)
        h2d = (2 + d) * N * 8
        d2h = (d + 3) * 8 * args.steps + (2 + d) * N * 8
        e2e = {"value": whole_job_rate(N * args.steps, world, te) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "includes": "lbm_init from pinned host fields, per step lbm_step(1) + lbm_last_diagnostics "
                           "(d+3 doubles D2H), final lbm_moments (rho, u, T D2H); after one untimed "
                           "lbm_init + lbm_moments through the same host buffers",
               "phases_ms": {"init": 1e3 * (t1 - t0), "steps": 1e3 * (t2 - t1), "moments": 1e3 * (t3 - t2)}}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu_baseline:
        n, threads, _ = oracle_sample(name, 15.0, 4)
        steps_cpu = 4 if d > 1 else 200
        mlups, dt, sites = run_oracle(name, n, steps_cpu, 1)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": "%s on %d sites (%s), %d steps, %.1f s" % (
                   name, sites, "x".join([str(n)] * d) if d > 1 else str(n), steps_cpu, dt)}

    others = None
    if name == "turb3d" and world == 1 and not args.no_others and not args.scale and args.tile < 0:
        sim.close()
        others = measure_others(local, {"turb3d": (rho, u, T)})

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if c["dtype"] == "f64" else "f32",
        "data": "synthetic",
        "config": {"workload": name + ": " + WORKLOAD_TEXT[name], "storage": c["dtype"],
                   "sites": N, "l2": ("state of %.3f GB per buffer > 129 MB L2, no flush needed" % (state_b / 1e9))
                   if state_b > 129e6 else "flush not applied: state of %.1f MB per buffer fits in L2" % (state_b / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "kernel": kernel, "tile": tile, "chunk": chunk,
                   "edge": args.scale or None, "inplace": bool(args.inplace),
                   "diagnostics": not args.no_diagnostics},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_src, "bytes_per_site": bps, "kernel": kernel,
                     "launches": launches,
                     "duration": "CUDA events on the launching stream around the timed steps, "
                                 + ("two launches per step (aux pass, collide pass); bytes of both"
                                    if args.inplace else "one step-kernel launch per step")},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if others is not None:
        line["other_workloads"] = {
            "how": "after the headline measurement, same process and GPU: each workload created, "
                   "initialised, warmed up (autotuner), then its timed steps between CUDA events on its "
                   "own stream; diagnostics recorded every step; roofline frac of measured HBM on the "
                   "algorithmic bytes per site; 1D lattices report time to result; the serving record: "
                   "200 requests through the server at their arrival times (aggregate = site updates / "
                   "first submit to last completion), then one at a time",
            "results": others}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
