#!/usr/bin/env python
"""Throughput of checkerboard-overrelaxation Landau gauge fixing on one GB300.

Workload: SU(3), 32^4 periodic lattice, U_mu(x) = g(x) exp(i 0.3 H_mu(x)) g(x+mu)^+
with Haar-random g (seed 2), omega = 1.7. One step is a whole gauge fixing
through the library's handle: canonical links (resident in HBM) -> internal
layout, FP32 12-real sweeps until theta < 1e-8, switch to FP64 18-real, FP64
sweeps until theta < 1e-12 (theta every 10 sweeps, reunitarisation every 50),
internal -> canonical. value = site updates per second over the K timed steps.

Also reported: plain FP64 time to theta < 1e-12 on the same input, the
end-to-end rate through culgt_landau_fix_host (host buffers, copies inside),
the roofline of the dominant kernel (CUDA events, back-to-back launches) and
the FP64 CPU oracle on the host cores.

--impl reference times the FP64 CPU oracle instead (the only other
implementation of the method here): each step is one oracle sweep of the same
lattice on the host cores.

Multi-GPU (torchrun): the path does not shard across GPUs here; every rank
gauge-fixes its own replica and value sums the ranks' site updates over the
slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SU(3) OR site-updates/s, HBM GB/s; time to θ<1e-12 mixed vs plain FP64"
UNIT = "site-updates/s"

WORKLOADS = {
    # name: dims, nc, eps, seed, omega
    "su3_32x32x32x32": ((32, 32, 32, 32), 3, 0.3, 2, 1.7),
    "su3_4x4x4x4": ((4, 4, 4, 4), 3, 0.3, 1, 1.7),
}

# batched workloads (not the default line): Gribov copies of 16^4 plus uneven
# lattices in shared launches, and Coulomb gauge on 48^3 x 96 (one problem per
# time slice)
BATCHED = {
    "gribov_su3_16x16x16x16_64copies_uneven": [((16, 16, 16, 16), 64), ((8, 8, 8, 8), 8), ((12, 12, 12, 12), 8),
                                               ((32, 16, 16, 16), 8), ((24, 24, 24, 24), 8)],
    "coulomb_su3_48x48x48x96": None,
    "su3_64x64x64x64": None,
    "su2_64x64x64x64": None,
    "mag_su3_32x32x32x32": None,
}

# algorithmic bytes per site update: 8 links read + 8 written
# algorithmic FP64 flops per site update (FMA = 2): SU(3) = gather 126 +
# subgroup steps 108 + row rotations 336 + eight 3x3 complex products 1584
FLOPS_PER_SITE = {3: 2154, 2: 282}
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12
L2_BYTES = 129e6  # GB300 L2

BYTES_PER_SITE = {(3, 1, 12): 768, (3, 1, 18): 1152, (3, 0, 18): 2304, (3, 0, 12): 1536,
                  (2, 1, 4): 256, (2, 0, 4): 512,
                  # FP32 phase of the mixed schedule: plus the site's own accumulated g, read and written
                  (3, 1, 12, "acc"): 768 + 96, (2, 1, 4, "acc"): 256 + 32}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="culgt", choices=["culgt", "reference"])
    ap.add_argument("--workload", default="su3_32x32x32x32", choices=sorted(WORKLOADS) + sorted(BATCHED))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (64^4, Gribov batch, Coulomb, MAG, SU(2) 64^4) in the line")
    ap.add_argument("--profile-step", choices=["mixed", "fp64", "fp32", "df", "mixed_df"], default=None,
                    help="run one gauge fixing (or --profile-sweeps sweeps) of the workload and exit; "
                         "the command the ncu captures in profiles/ wrap")
    ap.add_argument("--profile-gauge", choices=["landau", "mag"], default="landau",
                    help="with --profile-step: the gauge functional of the handle")
    ap.add_argument("--profile-heatbath", type=float, default=0.0,
                    help="with --profile-step and --profile-sweeps: heat-bath sweeps at this temperature instead")
    ap.add_argument("--profile-sweeps", type=int, default=0,
                    help="with --profile-step: this many sweeps instead of a whole fix")
    ap.add_argument("--tps", type=int, default=0, help="with --profile-step: threads per site (0 = autotune)")
    ap.add_argument("--block", type=int, default=0, help="with --profile-step: threads per block (0 = autotune)")
    ap.add_argument("--minb", type=int, default=0, help="with --profile-step: min blocks per SM (0 = autotune)")
    ap.add_argument("--storage", type=int, default=0, help="with --profile-step: reals per link (0 = default)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(ms_local, units_local, world_size, device=None):
    """Whole-job figures over replicas: the slowest rank's time and the sum of
    the ranks' site updates (the ranks run independent replicas)."""
    if world_size <= 1:
        return ms_local, units_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


# the files that define each family of single-lattice kernels: a recorded ncu
# traffic figure holds only while its family's files are unchanged
_BASE_SOURCES = ("culgt_device.cuh", "dfloat.cuh", "kernels.cuh", "ops_impl.cuh")
KERNEL_SOURCES = {
    "halfsweep_": _BASE_SOURCES,
    "heatbath_": _BASE_SOURCES + ("anneal.cuh",),
    "mag_halfsweep_": _BASE_SOURCES + ("anneal.cuh", "mag.cuh"),
}


def _code_only(text):
    """The source without comments and blank space, so that a comment edit
    does not void a recorded figure."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.strip() for line in text.splitlines() if line.strip())


def source_hash(kernel_key):
    files = next(v for k, v in KERNEL_SOURCES.items() if kernel_key.startswith(k))
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1412_3655_gb300", "csrc")
    for name in files:
        with open(os.path.join(csrc, name)) as f:
            h.update(name.encode())
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    entry = rec.get(kernel_key)
    if not entry or entry.get("source_hash") != source_hash(kernel_key):
        return None
    return entry.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_index):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            ids = [v.strip() for v in vis.split(",") if v.strip()]
            self.index = ids[local_index] if local_index < len(ids) else str(local_index)
        else:
            self.index = str(local_index)
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) == 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(U, dims, nc, omega, budget_s=12.0):
    """The FP64 oracle, as it stands, on the host cores: whole-lattice sweeps
    until about budget_s seconds have passed; then one sweep on a single core
    (the paper compares against one CPU core)."""
    import oracle
    work = U.copy()
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.sweep(work, dims, nc, omega, 1)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 50:
            break
    dt = time.perf_counter() - t0
    V = int(dims[0] * dims[1] * dims[2] * dims[3])
    cores = oracle.get_threads()
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.sweep(work, dims, nc, omega, 1)
    one_core = V / (time.perf_counter() - t1)
    oracle.set_threads(cores)
    return {"value": n * V / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} FP64 sweeps of the {'x'.join(map(str, dims))} SU({nc}) lattice ({dt:.1f} s)",
            "one_core": {"value": one_core, "unit": UNIT, "sample": "1 FP64 sweep on one core"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401

    import oracle
    from paper_1412_3655_gb300 import synth
    dims, nc, eps, seed, omega = WORKLOADS[args.workload]
    oracle.build()
    U = synth.gauge_config(dims, nc, eps, seed)
    V = int(dims[0] * dims[1] * dims[2] * dims[3])
    work = U.copy()
    for _ in range(args.warmup):
        oracle.sweep(work, dims, nc, omega, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sweep(work, dims, nc, omega, 1)
    dt = time.perf_counter() - t0
    value = args.steps * V / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "dims": list(dims), "nc": nc, "eps": eps, "seed": seed,
                   "omega": omega, "step": "one FP64 oracle sweep of the whole lattice on the host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"{args.steps} FP64 sweeps of the {'x'.join(map(str, dims))} lattice"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_profile_step(args):
    """One step of the chosen schedule, nothing else: what the ncu captures wrap."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1412_3655_gb300 import culgt, synth
    dims, nc, eps, seed, omega = WORKLOADS[args.workload]
    U = synth.gauge_config(dims, nc, eps, seed)
    d_in = torch.from_numpy(U.view(np.float64).copy()).cuda()
    d_out = torch.empty_like(d_in)
    prec = {"mixed": culgt.MIXED, "fp64": culgt.FP64, "fp32": culgt.FP32, "df": culgt.DF,
            "mixed_df": culgt.MIXED_DF}[args.profile_step]
    p = culgt.Params.defaults(nc, dims, omega=omega, precision=prec, check_every=10, reunit_every=50,
                              max_sweeps=20000, threads_per_site=args.tps, block_size=args.block,
                              min_blocks_per_sm=args.minb, storage_reals=args.storage,
                              gauge=culgt.MAG if args.profile_gauge == "mag" else culgt.LANDAU)
    with culgt.Handle(p) as h:
        h.culgt_load(d_in)
        if args.profile_sweeps and args.profile_heatbath > 0:
            for k in range(args.profile_sweeps):
                h.culgt_handle_heatbath(args.profile_heatbath, 1, k)
            th, F = h.culgt_handle_theta()
            out = {"heatbath_sweeps": args.profile_sweeps, "T": args.profile_heatbath, "theta": th, "F": F}
        elif args.profile_sweeps:
            h.culgt_handle_sweep(args.profile_sweeps)
            th, F = h.culgt_handle_theta()
            out = {"sweeps": args.profile_sweeps, "theta": th, "F": F}
        else:
            r = h.culgt_handle_fix()
            out = {"sweeps_fp32": r.sweeps_fp32, "sweeps_fp64": r.sweeps_fp64, "theta": r.theta, "F": r.F}
        h.culgt_store(d_out)
        torch.cuda.synchronize()
    print(json.dumps({"profile_step": args.profile_step, "workload": args.workload, **out}), flush=True)
    return 0


class Background:
    """Generates the large inputs of the other workloads on the host cores, one
    after the other in a background thread, while the GPU measures; the
    generator itself runs in spawned worker processes (all cores but two)."""

    def __init__(self, jobs):
        from concurrent.futures import ThreadPoolExecutor
        self.ex = ThreadPoolExecutor(max_workers=1)
        self.futs = {name: self.ex.submit(fn) for name, fn in jobs}

    def get(self, name):
        return self.futs.pop(name).result()

    def close(self):
        self.ex.shutdown(wait=True)


def gen_workers():
    return max(1, min(os.cpu_count() or 1, 16) - 2)


def _gribov_copy(job):
    import numpy as np
    from paper_1412_3655_gb300 import synth
    dims, c = job
    return synth.gauge_config(dims, 3, 0.3, 4, copy=c, workers=1).view(np.float64).reshape(-1).copy()


def gribov_inputs(synth, workers=1):
    """C4: 64 Haar gauge copies of one SU(3) 16^4 field (eps 0.3, seed 4) and 8
    copies each of 8^4, 12^4, 16^3 x 32 and 24^4, as flat float64 arrays; the
    copies generated by `workers` spawned processes."""
    jobs, dims_list, groups = [], [], []
    for dims, copies in BATCHED["gribov_su3_16x16x16x16_64copies_uneven"]:
        for c in range(1, copies + 1):
            jobs.append((dims, c))
            dims_list.append(dims)
            groups.append("x".join(map(str, dims)))
    if workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            inputs = list(ex.map(_gribov_copy, jobs))
    else:
        inputs = [_gribov_copy(j) for j in jobs]
    return dims_list, groups, inputs


def _flat(U):
    import numpy as np
    return U.view(np.float64).reshape(-1)


def timed_fix(culgt, torch, stream, params, d_in, d_out):
    """(seconds, result) of one whole fix through a handle: load, fix, store;
    CUDA events on the launching stream."""
    with culgt.Handle(params, stream) as h:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.culgt_load(d_in)
        r = h.culgt_handle_fix()
        h.culgt_store(d_out)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, r


def sweep_rate(culgt, torch, stream, params, d_in, n_sweeps, warm=5):
    """ms per sweep of n_sweeps back-to-back sweeps through a handle (after
    warm sweeps, which also run the autotuner), and the mapping it used."""
    with culgt.Handle(params, stream) as h:
        h.culgt_load(d_in)
        h.culgt_handle_sweep(warm)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.culgt_handle_sweep(n_sweeps)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n_sweeps, h.culgt_handle_tuning()


def workload_mag(culgt, torch, stream, d_in, d_out, hbm, src):
    """Maximally Abelian gauge on the 32^4 SU(3) field: MAG half-sweeps timed
    back to back (FP32 12-real, FP64 18-real) and whole MAG fixes to
    theta_MAG < 1e-12, mixed FP32 -> FP64 and plain FP64."""
    dims, nc, eps, seed, omega = WORKLOADS["su3_32x32x32x32"]
    V = dims[0] * dims[1] * dims[2] * dims[3]
    kernels = {}
    for name, prec, bps, n in [("fp32_12", culgt.FP32, 768, 100), ("fp64_18", culgt.FP64, 2304, 20)]:
        p = culgt.Params.defaults(nc, dims, omega=omega, precision=prec, gauge=culgt.MAG)
        ms, _ = sweep_rate(culgt, torch, stream, p, d_in, n, warm=3)
        ms /= 2
        gbs = (V // 2) * bps / (ms / 1e3) / 1e9
        key = f"mag_halfsweep_su3_{name[:3]}_{name[4:]}_b128"
        tr = recorded_traffic(key)
        kernels[name] = {"launch_ms": ms, "algorithmic_GB_per_s": gbs, "hbm_frac": gbs / hbm,
                         "dram_frac": (tr / (ms / 1e3) / 1e9 / hbm) if tr else None,
                         "peak_source": f"{src} hbm_gbs", "traffic": tr}
    fixes = {}
    for name, prec in [("mixed", culgt.MIXED), ("fp64", culgt.FP64)]:
        p = culgt.Params.defaults(nc, dims, omega=omega, precision=prec, check_every=10, reunit_every=50,
                                  max_sweeps=20000, gauge=culgt.MAG)
        t, r = timed_fix(culgt, torch, stream, p, d_in, d_out)
        fixes[name] = {"s": t, "sweeps": [r.sweeps_fp32, r.sweeps_fp64], "theta": r.theta, "F": r.F,
                       "status": r.status}
    return {"workload": "SU(3) 32^4, eps 0.3, seed 2, omega 1.7, maximally Abelian gauge",
            "half_sweeps": kernels, "time_to_theta": fixes,
            "speedup_mixed_vs_fp64": fixes["fp64"]["s"] / fixes["mixed"]["s"]}


def workload_large(culgt, torch, stream, U, hbm, src, fixes=False):
    """C3, SU(3) 64^4 (eps 0.25, seed 3, omega 1.75): 200 timed sweeps in FP64
    18-real and in FP32 12-real; with fixes, whole fixes to theta < 1e-12,
    mixed FP32 -> FP64 and plain FP64 (about 11 minutes together)."""
    dims, nc, omega = (64, 64, 64, 64), 3, 1.75
    V = dims[0] * dims[1] * dims[2] * dims[3]
    d_in = torch.from_numpy(_flat(U)).cuda()
    out = {}
    for name, prec, bps in [("fp64_18", culgt.FP64, 2304), ("fp32_12", culgt.FP32, 768)]:
        p = culgt.Params.defaults(nc, dims, omega=omega, precision=prec)
        ms, m = sweep_rate(culgt, torch, stream, p, d_in, 200, warm=10)
        gbs = V * bps / (ms / 1e3) / 1e9
        out[name] = {"ms_per_sweep": ms, "site_updates_per_s": V / (ms / 1e3), "GB_per_s": gbs,
                     "hbm_frac": gbs / hbm, "peak_source": f"{src} hbm_gbs", "mapping": m}
    res = {"workload": "SU(3) 64^4, eps 0.25, seed 3, omega 1.75", "timed_sweeps_200": out,
           "l2": "working set far above L2 (FP32 links 3.2 GB, FP64 links 9.7 GB)"}
    if fixes:
        d_out = torch.empty_like(d_in)
        tt = {}
        for name, prec in [("mixed", culgt.MIXED), ("fp64", culgt.FP64)]:
            p = culgt.Params.defaults(nc, dims, omega=omega, precision=prec, check_every=10, reunit_every=50,
                                      max_sweeps=40000)
            t, r = timed_fix(culgt, torch, stream, p, d_in, d_out)
            tt[name] = {"s": t, "sweeps": [r.sweeps_fp32, r.sweeps_fp64], "theta": r.theta, "F": r.F,
                        "status": r.status}
        res["time_to_theta"] = tt
    return res


def workload_su2_large(culgt, torch, stream, U, hbm, src):
    """SU(2) 64^4 (eps 0.25, seed 3, omega 1.75), a working set well above L2
    (FP32 quaternion links 1.07 GB): the per-phase half-sweep rates of the
    mixed schedule and time to theta < 1e-12, mixed against plain FP64."""
    dims, nc, omega = (64, 64, 64, 64), 2, 1.75
    V = dims[0] * dims[1] * dims[2] * dims[3]
    d_in = torch.from_numpy(_flat(U)).cuda()
    d_out = torch.empty_like(d_in)
    mixed = culgt.Params.defaults(nc, dims, omega=omega, precision=culgt.MIXED, check_every=10, reunit_every=50,
                                  max_sweeps=40000)
    plain = culgt.Params(**{**mixed.__dict__, "precision": culgt.FP64})
    k = {}
    for name, p, key, n in [("fp32_phase", mixed, (2, 1, 4, "acc"), 200), ("fp64", plain, (2, 0, 4), 50)]:
        ms, m = sweep_rate(culgt, torch, stream, p, d_in, n)
        ms /= 2
        gbs = (V // 2) * BYTES_PER_SITE[key] / (ms / 1e3) / 1e9
        k[name] = {"launch_ms": ms, "algorithmic_GB_per_s": gbs, "hbm_frac": gbs / hbm,
                   "peak_source": f"{src} hbm_gbs", "mapping": m,
                   "working_set_bytes": V * 4 * (16 if name == "fp32_phase" else 32) + (V * 16 if name == "fp32_phase"
                                                                                       else 0)}
    tt = {}
    for name, p in [("mixed", mixed), ("fp64", plain)]:
        t, r = timed_fix(culgt, torch, stream, p, d_in, d_out)
        tt[name] = {"s": t, "sweeps": [r.sweeps_fp32, r.sweeps_fp64], "F": r.F, "status": r.status}
    return {"workload": "SU(2) 64^4, eps 0.25, seed 3, omega 1.75", "half_sweeps": k, "time_to_theta": tt}


def workload_gribov(culgt, torch, np, stream, dims_list, groups, inputs, anneal=True):
    """C4 through the batched engine: every copy in shared launches, mixed
    FP32 -> FP64 against plain FP64, time to theta < 1e-12 for every problem,
    max F per lattice size; with anneal, simulated annealing before the
    overrelaxation (copy j keyed by seed + j)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    nc, omega = 3, 1.7
    per = [int(np.prod(d)) for d in dims_list]

    def run(prec, switch=1e-8):
        ds = [torch.from_numpy(t).to(dev) for t in inputs]
        p = culgt.Params.defaults(nc, dims_list[0], omega=omega, precision=prec, check_every=10,
                                  reunit_every=50, max_sweeps=20000, switch_theta=switch)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = culgt.culgt_fix_batched(ds, dims_list, p, stream)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, res

    run(culgt.MIXED)  # warm-up (graph capture)
    t_mixed, r_mixed = run(culgt.MIXED)
    t_fp64, r_fp64 = run(culgt.FP64)
    t_auto, r_auto = run(culgt.MIXED, culgt.SWITCH_AUTO)
    maxF, maxF64 = {}, {}
    for g, r, q in zip(groups, r_mixed, r_fp64):
        maxF[g] = max(maxF.get(g, -1.0), r.F)
        maxF64[g] = max(maxF64.get(g, -1.0), q.F)
    updates = sum((r.sweeps_fp32 + r.sweeps_fp64) * n for r, n in zip(r_mixed, per))
    out = {
        "workload": "64 Haar copies of one SU(3) 16^4 field (eps 0.3, seed 4) + 8 copies each of 8^4, 12^4, "
                    "16^3x32, 24^4; 96 problems in shared launches",
        "problems": len(r_mixed), "sites": sum(per),
        "time_to_theta": {"mixed_s": t_mixed, "fp64_s": t_fp64, "mixed_auto_switch_s": t_auto,
                          "speedup_mixed_vs_fp64": t_fp64 / t_mixed},
        "site_updates_per_s_mixed": updates / t_mixed,
        "all_converged": {"mixed": all(r.status == culgt.OK for r in r_mixed),
                          "fp64": all(r.status == culgt.OK for r in r_fp64),
                          "mixed_auto": all(r.status == culgt.OK for r in r_auto)},
        "max_F": maxF, "max_F_fp64": maxF64,
        "mixed_vs_fp64_max_dF": max(abs(a.F - b.F) for a, b in zip(r_mixed, r_fp64)),
        "plaquette_drift_max": max(abs(r.plaq_after - r.plaq_before) for r in r_mixed),
    }
    if anneal:
        a = culgt.culgt_default_anneal_params()
        a.seed = 11
        ds = [torch.from_numpy(t).to(dev) for t in inputs]
        p = culgt.Params.defaults(nc, dims_list[0], omega=omega, precision=culgt.MIXED, check_every=10,
                                  reunit_every=50, max_sweeps=20000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r_ann = culgt.culgt_fix_batched_anneal(ds, dims_list, p, a, stream)
        torch.cuda.synchronize()
        t_ann = time.perf_counter() - t0
        best = {}
        for g, r1 in zip(groups, r_ann):
            best[g] = max(best.get(g, -1.0), r1.F)
        sa_sweeps = a.steps * (1 + a.micro_sweeps)
        out["anneal"] = {
            "schedule": {"t_start": a.t_start, "t_end": a.t_end, "steps": a.steps, "micro_sweeps": a.micro_sweeps,
                         "seed": a.seed},
            "s": t_ann, "all_converged": all(r.status == culgt.OK for r in r_ann),
            "site_updates_per_s": sum((sa_sweeps + r.sweeps_fp32 + r.sweeps_fp64) * n
                                      for r, n in zip(r_ann, per)) / t_ann,
            "max_F": best}
    return out


def workload_batched_cost(culgt, torch, np, stream, dims_list, groups, inputs, n1=60, n2=240):
    """What the batched engine's design (one launch per colour over the tiles
    of every active problem, each check interval replayed as a CUDA graph)
    costs on the C4 mix. Per lattice-size group, the engine's time per FP32
    12-real sweep of the whole group, taken as the difference of runs of n2
    and n1 sweeps (so the call's fixed cost, allocation and layout
    conversion, drops out), against the same sweeps of each lattice alone
    through a single-lattice handle (sweeps back to back, so a lattice whose
    links fit in L2 runs from L2 there). The fixed cost of a colour launch is
    the engine's time per sweep (two launches) of 64 lattices of 2^4 sites."""
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}
    order = []
    for g in groups:
        if g not in order:
            order.append(g)

    def per_sweep_s(ds, dl):
        ts = []
        for n in (n1, n2):
            p = culgt.Params.defaults(3, dl[0], precision=culgt.FP32, theta_target=0.0, max_sweeps=n,
                                      check_every=30, reunit_every=0)
            culgt.culgt_fix_batched(ds, dl, p, stream)  # warm-up (graph capture)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            culgt.culgt_fix_batched(ds, dl, p, stream)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return (ts[1] - ts[0]) / (n2 - n1)

    for g in order + ["all"]:
        idx = [i for i, gg in enumerate(groups) if gg == g or g == "all"]
        dl = [dims_list[i] for i in idx]
        ds = [torch.from_numpy(inputs[i]).to(dev) for i in idx]
        sites = sum(int(np.prod(d)) for d in dl)
        tb = per_sweep_s(ds, dl)
        rec = {"problems": len(idx), "sites": sites, "batched_ms_per_sweep": 1e3 * tb,
               "batched_site_updates_per_s": sites / tb,
               "batched_GB_per_s": sites * BYTES_PER_SITE[(3, 1, 12)] / tb / 1e9}
        if g != "all":
            p = culgt.Params.defaults(3, dl[0], precision=culgt.FP32)
            ts = 0.0
            for d in ds:
                ms, m = sweep_rate(culgt, torch, stream, p, d, n2, warm=3)
                ts += ms / 1e3
            one = int(np.prod(dl[0])) * 4 * 48
            rec.update({"single_ms_per_sweep": 1e3 * ts, "single_site_updates_per_s": sites / ts,
                        "batched_over_single": ts / tb, "single_mapping": m,
                        "single_lattice_links_bytes": one, "single_lattice_in_l2": one < L2_BYTES})
        out[g] = rec
    tiny = [(2, 2, 2, 2)] * 64
    from paper_1412_3655_gb300 import synth
    base = _flat(synth.gauge_config((2, 2, 2, 2), 3, 0.3, 4)).copy()
    out["fixed_cost_per_colour_launch_us"] = 1e6 * per_sweep_s([torch.from_numpy(base).to(dev) for _ in tiny],
                                                               tiny) / 2
    out["note"] = ("FP32 12-real sweeps, theta every 30 sweeps (one graph replay each), per-sweep time from "
                   "two run lengths; "
                   "single: each lattice alone through a handle, the group's lattices one after another")
    return out


def workload_coulomb(culgt, torch, stream, U):
    """C5: SU(3) Coulomb gauge on 48^3 x 96 (eps 0.3, seed 5, omega 1.7), one
    problem per time slice in shared launches, each retired at its own
    theta < 1e-12: mixed FP32 -> FP64 against plain FP64."""
    dims, nc, omega = (96, 48, 48, 48), 3, 1.7
    host = torch.from_numpy(_flat(U))
    dev = torch.device("cuda", torch.cuda.current_device())

    def run(prec, switch=1e-8):
        d = host.to(dev)
        p = culgt.Params.defaults(nc, dims, omega=omega, precision=prec, check_every=10, reunit_every=50,
                                  max_sweeps=20000, switch_theta=switch)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = culgt.culgt_coulomb_fix(d, p, stream)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, res

    t_mixed, r_mixed = run(culgt.MIXED)
    t_fp64, r_fp64 = run(culgt.FP64)
    t_auto, r_auto = run(culgt.MIXED, culgt.SWITCH_AUTO)
    V3 = 48 ** 3
    updates = sum((r.sweeps_fp32 + r.sweeps_fp64) * V3 for r in r_mixed)
    return {"workload": "SU(3) Coulomb gauge, 48^3 x 96, eps 0.3, seed 5, omega 1.7: 96 slices in shared launches",
            "time_to_theta": {"mixed_s": t_mixed, "fp64_s": t_fp64, "mixed_auto_switch_s": t_auto,
                              "speedup_mixed_vs_fp64": t_fp64 / t_mixed},
            "site_updates_per_s_mixed": updates / t_mixed,
            "all_converged": {"mixed": all(r.status == culgt.OK for r in r_mixed),
                              "fp64": all(r.status == culgt.OK for r in r_fp64),
                              "mixed_auto": all(r.status == culgt.OK for r in r_auto)},
            "sweeps_mixed": {"fp32_max": max(r.sweeps_fp32 for r in r_mixed),
                             "fp64_max": max(r.sweeps_fp64 for r in r_mixed)},
            "mixed_vs_fp64_max_dF": max(abs(a.F - b.F) for a, b in zip(r_mixed, r_fp64)),
            "plaquette_drift_max": abs(r_mixed[0].plaq_after - r_mixed[0].plaq_before)}


def run_workload(args):
    """One of the other workloads alone, as its own JSON line."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1412_3655_gb300 import culgt, synth
    stream = torch.cuda.current_stream()
    peaks, src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    w = args.workload
    if w == "mag_su3_32x32x32x32":
        dims, nc, eps, seed, _ = WORKLOADS["su3_32x32x32x32"]
        d_in = torch.from_numpy(_flat(synth.gauge_config(dims, nc, eps, seed)).copy()).cuda()
        res = workload_mag(culgt, torch, stream, d_in, torch.empty_like(d_in), hbm, src)
        value = sum(res["time_to_theta"]["mixed"]["sweeps"]) * 32 ** 4 / res["time_to_theta"]["mixed"]["s"]
    elif w == "su3_64x64x64x64":
        res = workload_large(culgt, torch, stream, synth.gauge_config((64,) * 4, 3, 0.25, 3), hbm, src, fixes=True)
        tt = res["time_to_theta"]["mixed"]
        value = sum(tt["sweeps"]) * 64 ** 4 / tt["s"]
    elif w == "su2_64x64x64x64":
        res = workload_su2_large(culgt, torch, stream, synth.gauge_config((64,) * 4, 2, 0.25, 3), hbm, src)
        tt = res["time_to_theta"]["mixed"]
        value = sum(tt["sweeps"]) * 64 ** 4 / tt["s"]
    elif w.startswith("gribov"):
        dl, groups, inputs = gribov_inputs(synth, gen_workers())
        res = workload_gribov(culgt, torch, np, stream, dl, groups, inputs)
        res["batched_engine_cost"] = workload_batched_cost(culgt, torch, np, stream, dl, groups, inputs)
        value = res["site_updates_per_s_mixed"]
    else:
        res = workload_coulomb(culgt, torch, stream, synth.gauge_config((96, 48, 48, 48), 3, 0.3, 5))
        value = res["site_updates_per_s_mixed"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32->f64 (mixed)",
            "data": "synthetic", "config": {"workload": w}, **res}
    print(json.dumps(line), flush=True)
    return 0


def run_culgt(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build_library()
    from paper_1412_3655_gb300 import culgt, synth

    dims, nc, eps, seed, omega = WORKLOADS[args.workload]
    V = int(dims[0] * dims[1] * dims[2] * dims[3])
    U = synth.gauge_config(dims, nc, eps, seed)
    host = torch.from_numpy(U.view(np.float64).copy())
    d_in = host.to(dev)
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream(dev)

    mixed = culgt.Params.defaults(nc, dims, omega=omega, precision=culgt.MIXED, check_every=10, reunit_every=50,
                                  max_sweeps=20000)
    plain = culgt.Params.defaults(nc, dims, omega=omega, precision=culgt.FP64, check_every=10, reunit_every=50,
                                  max_sweeps=20000)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    h = culgt.Handle(mixed, stream)

    def step():
        h.culgt_load(d_in)
        r = h.culgt_handle_fix()
        h.culgt_store(d_out)
        return r

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = culgt.culgt_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    e0.record(stream)
    for _ in range(args.steps):
        results.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = culgt.culgt_kernel_launches() - launches0
    clocks = sampler.stop()
    extras = ws == 1 and not args.no_extras
    bg = None
    if extras:
        # inputs of the other workloads, generated on the host while the GPU
        # measures what follows (the timed region above is over)
        w = gen_workers()
        bg = Background([
            ("gribov", lambda: gribov_inputs(synth, w)),
            ("su3_64", lambda: synth.gauge_config((64, 64, 64, 64), 3, 0.25, 3, workers=w)),
            ("su2_64", lambda: synth.gauge_config((64, 64, 64, 64), 2, 0.25, 3, workers=w)),
            ("coulomb", lambda: synth.gauge_config((96, 48, 48, 48), 3, 0.3, 5, workers=w)),
        ])
    ms = e0.elapsed_time(e1)
    updates = sum((r.sweeps_fp32 + r.sweeps_fp64) * V for r in results)
    ms, updates_all = aggregate(ms, updates, ws, dev)
    value = updates_all / (ms / 1e3)
    last = results[-1]

    # per-kernel launch times: back-to-back half-sweeps on the launching stream
    mapping = {}

    def kernel_ms(params, n_sweeps=100, links=None, prefix=""):
        with culgt.Handle(params, stream) as hk:
            hk.culgt_load(d_in if links is None else links)
            hk.culgt_handle_sweep(5)
            mapping[prefix + {culgt.MIXED: "fp32_phase", culgt.FP64: "fp64", culgt.DF: "double_float"}.get(
                params.precision, str(params.precision))] = hk.culgt_handle_tuning()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            hk.culgt_handle_sweep(n_sweeps)
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / (2 * n_sweeps)

    # the FP32 phase kernel of the mixed schedule (it also accumulates g)
    t32 = kernel_ms(mixed)
    t64 = kernel_ms(plain, 20)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    share32 = last.sweeps_fp32 * t32
    share64 = last.sweeps_fp64 * t64

    def roofline_hbm(key, t_ms, m):
        bytes_launch = (V // 2) * BYTES_PER_SITE[key]
        achieved = bytes_launch / (t_ms / 1e3) / 1e9
        name = (f"halfsweep_su{key[0]}_{'f32' if key[1] else 'f64'}_{key[2]}" + ("_acc" if len(key) > 3 else "")
                + f"_tps{m[0]}_b{m[1]}_mb{m[2]}")
        tr = recorded_traffic(name)
        return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": tr, "dram_frac": dram_frac(tr, t_ms), "kernel": name, "launch_ms": t_ms,
                "algorithmic_bytes_per_launch": bytes_launch, "peak_source": f"{peak_src} hbm_gbs"}

    def dram_frac(traffic, t_ms):
        # measured DRAM bytes of the kernel (ncu, per launch) over its launch time
        return traffic / (t_ms / 1e3) / 1e9 / hbm if traffic else None

    def roofline_fp64(key, t_ms, m):
        # FP64-ALU bound on GB300: algorithmic FP64 flops per site update
        # (FMA = 2) against 2 DFMA/clock/SM x 152 SMs x 2070 MHz
        flops_launch = (V // 2) * FLOPS_PER_SITE[key[0]]
        achieved = flops_launch / (t_ms / 1e3) / 1e12
        name = f"halfsweep_su{key[0]}_{'f32' if key[1] else 'f64'}_{key[2]}_tps{m[0]}_b{m[1]}_mb{m[2]}"
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": recorded_traffic(name),
                "dram_frac": dram_frac(recorded_traffic(name), t_ms), "kernel": name,
                "launch_ms": t_ms, "algorithmic_flops_per_launch": flops_launch,
                "algorithmic_bytes_per_launch": (V // 2) * BYTES_PER_SITE[key],
                "hbm_frac": (V // 2) * BYTES_PER_SITE[key] / (t_ms / 1e3) / 1e9 / hbm,
                "peak_source": "FP64: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (unit counts and max clock)"}

    # heat-bath (simulated annealing) half-sweeps: one thread per site, blocks of 128
    def heatbath_ms(params, n_sweeps=20):
        with culgt.Handle(params, stream) as hk:
            hk.culgt_load(d_in)
            hk.culgt_handle_heatbath(0.5, 1, 0)
            keep, minb = hk.culgt_handle_heatbath_tuning()
            mapping["heatbath_" + ("fp32_phase" if params.precision == culgt.MIXED else "fp64")] = (keep, 128, minb)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for k in range(n_sweeps):
                hk.culgt_handle_heatbath(0.5, 1, k + 1)
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / (2 * n_sweeps)

    thb32 = heatbath_ms(mixed)
    thb64 = heatbath_ms(plain, 10)
    rl32 = roofline_hbm((nc, 1, 12 if nc == 3 else 4, "acc"), t32, mapping["fp32_phase"])
    rl64 = roofline_fp64((nc, 0, 18 if nc == 3 else 4), t64, mapping["fp64"])
    dominant = rl32 if share32 >= share64 else rl64
    dominant = dict(dominant, time_share_in_step=max(share32, share64) / max(share32 + share64, 1e-30))

    # time to theta < 1e-12 on the same input: plain FP64, and the double-float
    # variants (FP64-size links as float pairs, FP32-pipe arithmetic, theta in FP64)
    def fix_time(params, links=None):
        hx = culgt.Handle(params, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hx.culgt_load(d_in if links is None else links)
        r = hx.culgt_handle_fix()
        hx.culgt_store(d_out if links is None else links_out[0])
        b.record(stream)
        torch.cuda.synchronize()
        hx.close()
        return a.elapsed_time(b) / 1e3, r

    links_out = [None]

    fp64_s, rp = fix_time(plain)
    mixed_df = culgt.Params(**{**mixed.__dict__, "precision": culgt.MIXED_DF})
    only_df = culgt.Params(**{**plain.__dict__, "precision": culgt.DF})
    mixed_df_s, rmd = fix_time(mixed_df)
    df_s, rdf = fix_time(only_df)
    tdf = kernel_ms(only_df, 20)
    rldf = roofline_hbm((nc, 0, 18 if nc == 3 else 4), tdf, mapping["double_float"])
    rldf["kernel"] = rldf["kernel"].replace("f64", "df")
    rldf["traffic"] = recorded_traffic(rldf["kernel"])
    rldf["dram_frac"] = dram_frac(rldf["traffic"], tdf)
    mk = mapping["heatbath_fp32_phase"]
    rlhb32 = roofline_hbm((nc, 1, 12 if nc == 3 else 4, "acc"), thb32, mk)
    rlhb32["kernel"] = rlhb32["kernel"].replace("halfsweep", "heatbath").replace(f"_tps{mk[0]}_", f"_keep{mk[0]}_")
    rlhb32["traffic"] = recorded_traffic(rlhb32["kernel"])
    rlhb32["dram_frac"] = dram_frac(rlhb32["traffic"], thb32)
    mk = mapping["heatbath_fp64"]
    rlhb64 = roofline_fp64((nc, 0, 18 if nc == 3 else 4), thb64, mk)
    rlhb64["kernel"] = rlhb64["kernel"].replace("halfsweep", "heatbath").replace(f"_tps{mk[0]}_", f"_keep{mk[0]}_")
    rlhb64["traffic"] = recorded_traffic(rlhb64["kernel"])
    rlhb64["dram_frac"] = dram_frac(rlhb64["traffic"], thb64)
    rlhb64["note"] = "flops counted as for the overrelaxation update; the draw adds its own"
    # the FP32 -> FP64 switch later: the orbit-exact switch keeps the FP32
    # rounding off the result, so the FP32 phase may run to a lower theta
    late = {}
    for sw in (1e-10, 1e-11):
        t_sw, r_sw = fix_time(culgt.Params(**{**mixed.__dict__, "switch_theta": sw}))
        late[f"{sw:g}"] = {"s": t_sw, "sweeps": [r_sw.sweeps_fp32, r_sw.sweeps_fp64], "F": r_sw.F, "theta": r_sw.theta}
    # the automatic switch (switch_theta = 0): the FP32 phase runs until a
    # check interval no longer lowers theta, FP64 or double-float polish after
    auto = {}
    for name, prec in [("mixed", culgt.MIXED), ("mixed_df", culgt.MIXED_DF)]:
        t_a, r_a = fix_time(culgt.Params(**{**mixed.__dict__, "precision": prec,
                                            "switch_theta": culgt.SWITCH_AUTO}))
        auto[name] = {"s": t_a, "sweeps": [r_a.sweeps_fp32, r_a.sweeps_fp64], "F": r_a.F, "theta": r_a.theta,
                      "status": r_a.status, "site_updates_per_s": (r_a.sweeps_fp32 + r_a.sweeps_fp64) * V / t_a}
    # FP64 with 12-real storage (third row rebuilt): 2/3 of the bytes, more FP64 arithmetic
    plain12 = culgt.Params(**{**plain.__dict__, "storage_reals": 12})
    t64_12 = kernel_ms(plain12, 20, prefix="s12_")
    rl64_12 = roofline_fp64((nc, 0, 12), t64_12, mapping["s12_fp64"])

    # SU(2) on the same generator (eps 0.3, Haar g, seed 2) and lattice: the
    # per-phase half-sweep rates and the time to theta < 1e-12, mixed vs FP64
    U2 = synth.gauge_config(dims, 2, eps, seed)
    d2 = torch.from_numpy(U2.view(np.float64).copy()).to(dev)
    del U2
    links_out[0] = torch.empty_like(d2)
    mixed2 = culgt.Params(**{**mixed.__dict__, "nc": 2})
    plain2 = culgt.Params(**{**plain.__dict__, "nc": 2})
    t2_32 = kernel_ms(mixed2, 100, d2, "su2_")
    t2_64 = kernel_ms(plain2, 50, d2, "su2_")
    su2_mixed_s, r2m = fix_time(mixed2, d2)
    su2_fp64_s, r2p = fix_time(plain2, d2)
    # FP32 quaternion links (4V x 16 B) and the g accumulator (V x 16 B) fit in
    # L2 at 32^4: that half-sweep runs from L2, so no HBM fraction is claimed
    rl2_32 = roofline_hbm((2, 1, 4, "acc"), t2_32, mapping["su2_fp32_phase"])
    su2_bytes = 5 * V * 16
    if su2_bytes < L2_BYTES:
        rl2_32.update({"bound": "l2-resident", "frac": None, "working_set_bytes": su2_bytes,
                       "note": f"working set {su2_bytes / 1e6:.0f} MB < L2 {L2_BYTES / 1e6:.0f} MB: "
                               "achieved is an L2 rate"})
    su2 = {
        "fp32_phase": rl2_32,
        "fp64": roofline_fp64((2, 0, 4), t2_64, mapping["su2_fp64"]),
        "time_to_theta": {"mixed_s": su2_mixed_s, "mixed_sweeps": [r2m.sweeps_fp32, r2m.sweeps_fp64],
                          "mixed_F": r2m.F, "fp64_s": su2_fp64_s, "fp64_sweeps": r2p.sweeps_fp64, "fp64_F": r2p.F},
    }
    del d2
    links_out[0] = None

    # end to end through the host entry point (pinned host buffer)
    pinned = host.pin_memory()
    n_e2e = max(1, min(args.steps, 2))
    culgt.culgt_landau_fix_host(pinned, mixed, stream)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_updates = 0
    for _ in range(n_e2e):
        pinned.copy_(host)
        r = culgt.culgt_landau_fix_host(pinned, mixed, stream)
        e2e_updates += (r.sweeps_fp32 + r.sweeps_fp64) * V
    e2e_s = time.perf_counter() - t0
    canon_bytes = host.numel() * host.element_size()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32->f64 (mixed)", "data": "synthetic",
        "config": {"workload": args.workload, "dims": list(dims), "nc": nc, "eps": eps, "seed": seed,
                   "omega": omega, "precision": "mixed: FP32 12-real to theta<1e-8, FP64 18-real to theta<1e-12",
                   "check_every": 10, "reunit_every": 50, "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (FP32 links 201 MB, FP64 links 604 MB)"},
        "sweeps": {"fp32": last.sweeps_fp32, "fp64": last.sweeps_fp64, "theta": last.theta, "F": last.F},
        "time_to_theta": {"mixed_s": ms / args.steps / 1e3, "fp64_s": fp64_s,
                          "fp64_sweeps": rp.sweeps_fp64, "fp64_F": rp.F, "mixed_F": last.F,
                          "mixed_df_s": mixed_df_s, "mixed_df_sweeps": [rmd.sweeps_fp32, rmd.sweeps_fp64],
                          "mixed_df_F": rmd.F, "df_s": df_s, "df_sweeps": rdf.sweeps_fp64, "df_F": rdf.F,
                          "mixed_switch_later": late,
                          "note": "mixed: FP32 to theta<1e-8, then IEEE FP64 sweeps (the value above); *_df: "
                                  "double-float sweeps (float pairs, ~48-bit) with theta/F in FP64; "
                                  "mixed_switch_later: the same schedule with the FP32 phase run to a lower theta"},
        "roofline": dominant,
        "roofline_kernels": {"fp32_phase": rl32, "fp64": rl64, "fp64_12": rl64_12, "double_float": rldf,
                             "heatbath_fp32_phase": rlhb32, "heatbath_fp64": rlhb64},
        "auto_switch": auto,
        "su2": su2,
        "gpu_launches": launches,
        "sweep_mapping": {k: ({"keep_links": v[0], "block": v[1], "min_blocks_per_sm": v[2]} if
                              k.startswith("heatbath") else
                              {"threads_per_site": v[0], "block": v[1], "min_blocks_per_sm": v[2]})
                          for k, v in mapping.items()},
        "e2e": {"value": e2e_updates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": canon_bytes,
                "d2h_bytes_per_step": canon_bytes, "steps": n_e2e},
        "clocks": clocks,
    }
    h.close()
    if extras:
        line["mag_su3_32x32x32x32"] = workload_mag(culgt, torch, stream, d_in, d_out, hbm, peak_src)
        dl, groups, inputs = bg.get("gribov")
        gr = workload_gribov(culgt, torch, np, stream, dl, groups, inputs)
        gr["batched_engine_cost"] = workload_batched_cost(culgt, torch, np, stream, dl, groups, inputs)
        line["gribov_batch"] = gr
        del inputs
        line["su3_64x64x64x64"] = workload_large(culgt, torch, stream, bg.get("su3_64"), hbm, peak_src)
        torch.cuda.empty_cache()
        line["su2_64x64x64x64"] = workload_su2_large(culgt, torch, stream, bg.get("su2_64"), hbm, peak_src)
        torch.cuda.empty_cache()
        line["coulomb_48x48x48x96"] = workload_coulomb(culgt, torch, stream, bg.get("coulomb"))
        bg.close()
        line["extras_note"] = ("other workloads, each measured once after the timed region: MAG on the same "
                               "field; the batched Gribov search (C4), 64^4 SU(3) sweep rates (C3; its whole "
                               "fixes, about 11 minutes, run with --workload su3_64x64x64x64), SU(2) 64^4 and "
                               "Coulomb 48^3x96 (C5)")
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(U, dims, nc, omega)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_step:
        return run_profile_step(args)
    if args.workload in BATCHED:
        return run_workload(args)
    return run_culgt(args)


if __name__ == "__main__":
    sys.exit(main())
