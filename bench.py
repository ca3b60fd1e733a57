#!/usr/bin/env python3
"""Benchmark: integral-direct J/K builds on one GB300 (or N independent replicas).

A step is one complete J/K build (screening, every class kernel, symmetrisation)
of the medium workload: 30 atoms on a jittered 1.8 A lattice, 3s2p1d per atom
with contraction depths 1..6, 450 Cartesian functions, one random PSD density
(60 columns), tau = 1e-12, FP64 throughout.  It stands in for the paper's
6-31G(d)-class Gly_n / RNA_n Fock builds (Sec. 5), whose inputs are not
available.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle
(OS/HGP, OpenMP) on a bounded random sample of the same build per step.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "J/K builds/s & ERI quartets/s (FP64 vs mixed @1e-6); served p50/p99 latency"
# split of the mixed mode: quartets whose transfer-aware Schwarz x density bound is <= 1e-4
# run their recurrences in FP32
MIXED_THRESH = 1e-4
def workload_name(natm):
    return (f"medium J/K build: {natm} atoms, jittered 1.8 A lattice, 3s2p1d per atom, depths 1-6, "
            f"{15 * natm} Cartesian functions, 1 PSD density (60 columns), tau 1e-12, FP64")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--natm", type=int, default=30, help="atoms of the medium recipe (30 = the benchmark)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision measurement")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-workload measurement")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target wall time of the oracle sample")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed plumbing

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    def __init__(self, backend):
        self.ws, self.rank, self.local = dist_env()
        self.pg = None
        if self.ws > 1:
            import torch.distributed as td
            td.init_process_group(backend=backend)
            self.td = td

    def barrier(self):
        if self.ws > 1:
            self.td.barrier()

    def max(self, x):
        if self.ws == 1:
            return x
        import torch
        dev = torch.device("cuda", self.local) if torch.cuda.is_available() else torch.device("cpu")
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.td.all_reduce(t, op=self.td.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.ws > 1:
            self.td.destroy_process_group()


def replica_throughput(steps, world_size, t_max):
    """Whole-job builds/s of independent replicas: every rank runs `steps` builds and the job
    lasts as long as its slowest rank."""
    return steps * world_size / t_max


# ---------------------------------------------------------------- clocks sampler

class Clocks:
    FIELDS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap", "power.draw"]

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + ",".join(self.FIELDS),
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return summarize_clock_lines(self.lines)


def summarize_clock_lines(lines):
    """Median SM clock, maximum SM clock, the throttle reasons seen active and the median power
    over nvidia-smi samples (clocks.sm, clocks.max.sm, hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap, power.draw per line); malformed lines are skipped."""
    sm, smax, reasons, power = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) != len(Clocks.FIELDS):
            continue
        try:
            sm.append(float(parts[0]))
            smax.append(float(parts[1]))
            power.append(float(parts[6]))
        except ValueError:
            continue
        for n, v in zip(names, parts[2:6]):
            if v.lower().startswith("active"):
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm),
            "power_w_median": statistics.median(power) if power else None}


def gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        if local < len(ids):
            return ids[local]
    return str(local)


# ---------------------------------------------------------------- CPU oracle sample

def oracle_sample_rate(mol, target_s, seed=0):
    """Time the CPU oracle on a seeded random sample of the build's unique shell quartets.

    Returns (builds_per_s, quartets_per_s, cores, description).  The sample grows until
    one timed run takes about target_s seconds of wall time."""
    import numpy as np

    import oracle
    b = oracle.OracleBasis(mol)
    npair = mol.nshell * (mol.nshell + 1) // 2
    total = npair * (npair + 1) // 2
    rng = np.random.default_rng(1234 + seed)
    n = 256
    while True:
        q = np.sort(rng.choice(total, size=min(n, total), replace=False))
        t0 = time.perf_counter()
        oracle.jk_sample(b, q)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * target_s or n >= total:
            break
        n = int(min(total, max(2 * n, n * target_s / max(dt, 1e-3))))
    frac = q.size / total
    builds = frac / dt
    desc = (f"{q.size} of {total} unique shell quartets drawn uniformly (seeded), evaluated and digested "
            f"by the OS/HGP oracle in {dt:.2f} s; builds/s = (sample fraction) / time")
    return builds, q.size / dt, oracle.max_threads(), desc


# ---------------------------------------------------------------- arms

def run_reference(args):
    from workloads import config_medium
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build_oracle()
    mol = config_medium(seed=args.seed, natm=args.natm)
    per_step = max(2.0, min(args.cpu_seconds, 20.0))
    for _ in range(args.warmup):
        oracle_sample_rate(mol, per_step / 4, seed=0)
    rates, qrates, desc, cores = [], [], "", 1
    for k in range(args.steps):
        b, qs, cores, desc = oracle_sample_rate(mol, per_step, seed=k + 1)
        rates.append(b)
        qrates.append(qs)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "J/K builds/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.natm), "seed": args.seed},
        "quartets_per_s": statistics.median(qrates),
        "cpu_baseline": {"value": value, "unit": "J/K builds/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "J/K builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_2407_09700_gb300 as pkg
    from workloads import config_medium

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = Dist("nccl")
    pkg.build()
    mol = config_medium(seed=args.seed, natm=args.natm)
    nbf = mol.nbf
    plan = pkg.Plan(mol)
    stream = torch.cuda.current_stream()
    D = torch.from_numpy(mol.D).cuda()
    J = torch.empty_like(D)
    K = torch.empty_like(D)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > L2
    fp64_peak, fp32_peak = pkg.probe_fma_peak()

    for _ in range(args.warmup):
        plan.jk(D, J, K)
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident, L2 flushed between steps
    plan.set_profiling(True)
    clk = Clocks(gpu_index(local))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    per_kernel = {}
    dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        plan.jk(D, J, K)
        ev[k][1].record(stream)
        recs = plan.launch_records()            # syncs this step's stream; outside the events
        for r in recs:
            prec = "float" if r["fp32"] else "double"
            if r["specialised"]:
                key = f"eri_small_kernel<{r['la']}, {r['lb']}, {r['lc']}, {r['ld']}, {prec}>"
            else:
                xy = "true" if r["shared_products"] else "false"
                key = f"eri_class_kernel<{r['team_size']}, {prec}, {xy}>"
            e = per_kernel.setdefault(key, {"ms": 0.0, "flops": 0.0, "launches": 0})
            e["ms"] += r["ms"]
            e["flops"] += r["model_flops"]
            e["launches"] += 1
    torch.cuda.synchronize()
    dist.barrier()
    clocks = clk.stop()
    plan.set_profiling(False)
    t_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    t_max = dist.max(t_s)
    st = plan.stats()
    nsteps_total = args.steps * ws
    value = replica_throughput(args.steps, ws, t_max)
    quartets_per_s = st["quartets_computed"] * nsteps_total / t_max
    # per build: the density-maxima kernel, the class kernels, three compaction kernels
    # (counts, scan, ordered writes) per FP64 class launch, and the two symmetrisations
    launches_per_step = 1 + st["nclasses_launched"] + 3 * st["nclasses_launched"] + 2

    # dominant kernel: the class-kernel instantiation with the most time in the region
    dom_name, dom = max(per_kernel.items(), key=lambda kv: kv[1]["ms"])
    achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
    all_ms = sum(v["ms"] for v in per_kernel.values())

    # ---- end to end: host buffers through the C-ABI (copies inside the timed call)
    Dh = torch.from_numpy(mol.D).pin_memory()
    Jh = torch.empty_like(Dh).pin_memory()
    Kh = torch.empty_like(Dh).pin_memory()
    lib = pkg.load_library()
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    sh = ctypes.c_void_p(stream.cuda_stream)

    def host_call():
        rc = lib.eri_jk_host(plan._h, ctypes.cast(Dh.data_ptr(), dp), 1, ctypes.cast(Jh.data_ptr(), dp),
                             ctypes.cast(Kh.data_ptr(), dp), 3, sh)
        if rc != 0:
            raise RuntimeError(lib.eri_last_error().decode())
    host_call()
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        host_call()
    te = dist.max(time.perf_counter() - t0)
    e2e = nsteps_total / te
    bytes_mat = 8 * nbf * nbf

    # parity spot check of the timed result against the e2e result (same algorithm, host copies)
    assert float((J.cpu() - Jh).abs().max()) < 1e-9

    # ---- mixed precision on the same workload (FP32 recurrences where the bound <= MIXED_THRESH)
    mixed = None
    if not args.no_mixed:
        plan_m = pkg.Plan(mol, precision=pkg.ERI_MIXED, mixed_thresh=MIXED_THRESH)
        Jm = torch.empty_like(D)
        Km = torch.empty_like(D)
        for _ in range(max(1, args.warmup - 2)):
            plan_m.jk(D, Jm, Km)
        torch.cuda.synchronize()
        evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        dist.barrier()
        for k in range(args.steps):
            flush.zero_()
            evm[k][0].record(stream)
            plan_m.jk(D, Jm, Km)
            evm[k][1].record(stream)
        torch.cuda.synchronize()
        tm = dist.max(sum(a_.elapsed_time(b_) for a_, b_ in evm) / 1e3)
        stm = plan_m.stats()
        mixed = {"value": nsteps_total / tm, "unit": "J/K builds/s", "ms_per_step": 1e3 * tm / args.steps,
                 "quartets_per_s": stm["quartets_computed"] * nsteps_total / tm,
                 "fp32_quartet_fraction": stm["quartets_fp32"] / max(1, stm["quartets_computed"]),
                 "mixed_thresh": MIXED_THRESH,
                 "max_abs_dJ_vs_fp64": float((Jm - J).abs().max()),
                 "max_abs_dK_vs_fp64": float((Km - K).abs().max()),
                 "speedup_vs_fp64": (nsteps_total / tm) / value}
        plan_m.close()

    # ---- J/K energy gradient (FP64) on the 12-atom cut of the same recipe, beside its J/K build
    grad = None
    if not args.no_grad:
        mg = config_medium(seed=args.seed, natm=12)
        plan_g = pkg.Plan(mg)
        Dg = torch.from_numpy(np.ascontiguousarray(mg.D[0])).cuda()
        gJ = torch.empty((mg.natm, 3), dtype=torch.float64, device="cuda")
        gK = torch.empty_like(gJ)
        plan_g.jk_grad(Dg, gJ, gK)
        plan_g.jk(Dg)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        flush.zero_()
        e0.record(stream)
        plan_g.jk_grad(Dg, gJ, gK)
        e1.record(stream)
        flush.zero_()
        e2.record(stream)
        plan_g.jk(Dg)
        e3 = torch.cuda.Event(enable_timing=True)
        e3.record(stream)
        torch.cuda.synchronize()
        gst = plan_g.grad_stats()
        tg, tj = e0.elapsed_time(e1) / 1e3, e2.elapsed_time(e3) / 1e3
        grad = {"workload": "E_J / E_K nuclear gradient, medium recipe cut to 12 atoms (180 functions), FP64",
                "value": 1.0 / tg, "unit": "gradients/s", "ms": 1e3 * tg, "jk_ms_same_molecule": 1e3 * tj,
                "quartets_per_s": gst["quartets"] / tg, "prim_quartets_per_s": gst["prim_quartets"] / tg,
                "max_abs_sum_over_atoms": float(max(gJ.sum(0).abs().max(), gK.sum(0).abs().max()))}
        plan_g.close()

    # ---- served workload (rank 0): continuous batching (mixed) against one-at-a-time FP64
    served = None
    if rank == 0 and not args.no_serve:
        from workloads import config_served_requests
        from paper_2407_09700_gb300.serve import Server, make_jobs, run_sequential
        reqs = config_served_requests(seed=args.seed, nreq=32, mean_interarrival_s=0.02, natm_range=(5, 15))
        Server().run(make_jobs(reqs[:1], natm_cap=5))        # warm kernels and allocator
        sv = Server(hbm_budget=64 << 30, max_slots=32).run(make_jobs(reqs))
        sq = run_sequential(make_jobs(reqs))
        served = {"workload": "32 requests, exponential inter-arrival mean 20 ms (50 req/s), atoms log-uniform "
                              "[5, 15], 30% RHF to 1e-8 Ha, 70% single J/K; heavy/light 3s2p1d/2s1p recipe",
                  "served_mixed": {k: sv[k] for k in ("throughput_req_s", "p50_latency_s", "p99_latency_s",
                                                      "makespan_s", "mean_batch")},
                  "sequential_fp64": {k: sq[k] for k in ("throughput_req_s", "p50_latency_s", "p99_latency_s",
                                                         "makespan_s")}}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        b, qs, cores, desc = oracle_sample_rate(mol, args.cpu_seconds)
        cpu = {"value": b, "unit": "J/K builds/s", "cores": cores, "kind": "oracle", "sample": desc,
               "quartets_per_s": qs}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "J/K builds/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.natm), "seed": args.seed, "nbf": nbf, "natm": mol.natm,
                       "nshell": mol.nshell, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "flushed (256 MB write) before every timed step; events exclude the flush"},
            "quartets_per_s": quartets_per_s,
            "quartets_per_build": st["quartets_computed"],
            "prim_quartets_per_build": st["prim_quartets"],
            "model_tflops": st["model_flops"] / (t_max / nsteps_total) / 1e12,
            "roofline": {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": None,
                         "peak_kind": "measured FP64 FMA loop on this GPU (nominal 152 SM x 4 flop/clk x "
                                      "2.07 GHz = 1.26 TFLOP/s)",
                         "share_of_kernel_time": dom["ms"] / all_ms,
                         "flops_kind": "FP64 operations of the class kernel's algorithm per class "
                                       "(FMA = 2), times primitive quartets / quartets counted on device"},
            "fp32_fma_peak_tflops": fp32_peak,
            "e2e": {"value": e2e, "unit": "J/K builds/s", "h2d_bytes_per_step": bytes_mat,
                    "d2h_bytes_per_step": 2 * bytes_mat},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "mixed": mixed,
            "grad": grad,
            "served": served,
            "kernel_shares": {k: round(v["ms"] / all_ms, 4) for k, v in sorted(per_kernel.items(), key=lambda kv: -kv[1]["ms"])[:8]},
        }
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
