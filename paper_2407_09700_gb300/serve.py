"""Serving loop with continuous batching for J/K builds and RHF jobs.

Requests (a single J/K build on a given density, or a full RHF run to a
convergence threshold) arrive over time.  The server

  * admits a waiting request when a slot is free and its estimated device
    footprint fits the HBM budget (plan, densities, J/K, SCF state); requests
    that arrive while others run are admitted as soon as slots and memory free up;
  * keeps every admitted job's plan, density, Fock/DIIS state and orbitals on
    the device;
  * advances all active jobs together: one eri_jk_batch call per tick evaluates
    the pending J/K build of every active job, with each angular-momentum class
    run as one launch over all jobs (the class kernels read each task's plan,
    D, J and K from a job table), then each job takes its own step (J/K jobs
    finish, RHF jobs update F, E, DIIS and D; RHF jobs build J and K of the
    density change after their first iteration, as PySCF's direct SCF does);
  * builds the plans (pair data, Schwarz factors) and RHF set-up of arrived
    requests ahead of admission on a worker thread with its own CUDA stream, so
    that plan creation does not hold up the tick, and frees retired jobs' plans
    only when no job is active or an admission needs the memory (freeing device
    memory waits for the whole device);
  * records arrival, admission and finish times, giving throughput and
    p50 / p99 latency (finish - arrival).

``run_sequential`` is the baseline: the same requests one at a time, in arrival
order, each with its own FP64 plan (RHF jobs with the same incremental builds).
"""

from __future__ import annotations

import concurrent.futures
import dataclasses
import math
import time
from typing import Dict, List, Optional

import numpy as np

from .eri import ERI_FP64, ERI_MIXED, Batch, Plan
from .scf import RHF


@dataclasses.dataclass
class Job:
    rid: int
    kind: str                 # "jk" or "scf"
    mol: object
    arrival: float
    footprint: int
    plan: Optional[Plan] = None
    scf: Optional[RHF] = None
    D: object = None
    J: object = None
    K: object = None
    admit: float = math.nan
    finish: float = math.nan
    iters: int = 0
    result: Dict = dataclasses.field(default_factory=dict)
    prepared: object = None       # future of the worker thread's preparation (plan, RHF set-up)
    ready: object = None          # CUDA event after the preparation's device work


def footprint_bytes(mol, kind: str) -> int:
    """Device memory a job holds while admitted: pair and primitive-pair records,
    density block maxima, D / J / K and (RHF) S, H, X, Fock and DIIS matrices."""
    nsh = int(mol.nshell)
    nbf = int(mol.nbf)
    K = np.asarray(mol.shell_nprim, dtype=np.int64)
    npairs = nsh * (nsh + 1) // 2
    nprim_pairs = int((K.sum() ** 2 + (K ** 2).sum()) // 2)
    mats = 3 + (4 + 2 * 8 + 2 if kind == "scf" else 0)
    return int(2 * 64 * npairs + (80 + 40) * nprim_pairs + 8 * nsh * nsh + 8 * mats * nbf * nbf + (1 << 20))


def _percentile(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else math.nan


class Server:
    def __init__(self, precision: int = ERI_MIXED, mixed_thresh: float = 1e-4, hbm_budget: int = 8 << 30,
                 max_slots: int = 32, scf_conv: float = 1e-8, scf_max_iter: int = 100, batch=None, sync=None,
                 prefetch: int = 4):
        """batch: the batched J/K engine (an eri_batch by default); sync: waits for the device
        (torch.cuda.synchronize by default).  Both are replaceable so that the admission and
        retirement policy can run against stand-ins.  prefetch: arrived requests whose plans
        are built ahead of admission (0: build at admission)."""
        import torch
        self.torch = torch
        self.precision = precision
        self.mixed_thresh = mixed_thresh
        self.hbm_budget = hbm_budget
        self.max_slots = max_slots
        self.scf_conv = scf_conv
        self.scf_max_iter = scf_max_iter
        self.batch = batch if batch is not None else Batch()
        self.sync = sync if sync is not None else torch.cuda.synchronize
        self.prefetch = int(prefetch)
        self.pool = concurrent.futures.ThreadPoolExecutor(1) if self.prefetch > 0 else None
        self.prep_stream = None
        self.ticks = 0
        self.batch_sizes: List[int] = []
        self.max_active = 0
        self.max_used = 0
        self.prepared_ahead = 0
        self.freed_deferred = 0

    # ---- preparation (worker thread): everything that does not need the job's turn
    def _prepare(self, job: Job):
        torch = self.torch
        if self.prep_stream is None:
            self.prep_stream = torch.cuda.Stream()
        with torch.cuda.stream(self.prep_stream):
            job.plan = Plan(job.mol, precision=self.precision, mixed_thresh=self.mixed_thresh,
                            stream=self.prep_stream)
            if job.kind == "scf":
                job.scf = RHF(job.mol, plan=job.plan, incremental=True)
            ev = torch.cuda.Event()
            ev.record(self.prep_stream)
            job.ready = ev

    def _admit(self, job: Job, now: float):
        torch = self.torch
        if job.prepared is not None:
            job.prepared.result()
            torch.cuda.current_stream().wait_event(job.ready)
        else:
            job.plan = Plan(job.mol, precision=self.precision, mixed_thresh=self.mixed_thresh)
            if job.kind == "scf":
                job.scf = RHF(job.mol, plan=job.plan, incremental=True)
        nbf = job.plan.nbf
        if job.kind == "scf":
            job.scf.start()
            job.D = job.scf.build_density().unsqueeze(0).contiguous()
        else:
            job.D = torch.from_numpy(np.ascontiguousarray(job.mol.D[:1])).cuda()
        job.J = torch.empty((1, nbf, nbf), dtype=torch.float64, device="cuda")
        job.K = torch.empty_like(job.J)
        job.admit = now

    def _retire(self, job: Job, now: float):
        job.finish = now
        if job.scf is not None:
            job.scf.plan = None
            job.scf = None
        job.D = job.J = job.K = None

    def _destroy(self, job: Job):
        """Free a retired job's plan (synchronises the device)."""
        if job.plan is not None:
            job.plan.close()
            job.plan = None

    def run(self, jobs: List[Job], keep_results: bool = False):
        """Serve jobs (sorted by arrival).  Wall-clock times are relative to the start."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        active: List[Job] = []
        retired: List[Job] = []       # plans still held (freed when idle or when memory is needed)
        used = 0                      # footprints of active, prepared and not yet freed jobs
        t0 = time.perf_counter()

        def free_retired():
            nonlocal used
            for j in retired:
                self._destroy(j)
                used -= j.footprint
                self.freed_deferred += 1
            retired.clear()

        while pending or active:
            now = time.perf_counter() - t0
            # ---- prepare arrived requests ahead of admission while the budget allows (their
            #      footprint is counted from then on)
            if self.pool is not None:
                n_prep = sum(1 for j in pending if j.prepared is not None)
                for j in pending:
                    if n_prep >= self.prefetch or j.arrival > now:
                        break
                    if j.prepared is None:
                        if used + j.footprint > self.hbm_budget:
                            break
                        j.prepared = self.pool.submit(self._prepare, j)
                        used += j.footprint
                        n_prep += 1
                        self.prepared_ahead += 1
                        self.max_used = max(self.max_used, used)
            # ---- continuous admission: arrived and a slot free; a prepared job joins once its
            #      preparation is done (waited for only when nothing else can run), otherwise the
            #      footprint must fit
            while pending and pending[0].arrival <= now and len(active) < self.max_slots:
                j = pending[0]
                if j.prepared is not None:
                    if not j.prepared.done() and active:
                        break
                    extra = 0
                else:
                    extra = j.footprint
                    if used + extra > self.hbm_budget:
                        if retired:
                            free_retired()
                            continue
                        break
                pending.pop(0)
                self._admit(j, now)
                active.append(j)
                used += extra
                self.max_active = max(self.max_active, len(active))
                self.max_used = max(self.max_used, used)
            if not active:
                free_retired()
                if pending:
                    if pending[0].footprint > self.hbm_budget:
                        raise RuntimeError(f"request {pending[0].rid} exceeds the HBM budget on its own")
                    if pending[0].arrival > time.perf_counter() - t0:
                        time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 0.005)))
                continue
            # ---- one batched J/K over every active job
            self.batch.jk([j.plan for j in active], [j.D for j in active], [j.J for j in active],
                          [j.K for j in active])
            self.ticks += 1
            self.batch_sizes.append(len(active))
            done = []
            for j in active:
                if j.kind == "jk":
                    if keep_results:
                        j.result = {"J": j.J[0].clone(), "K": j.K[0].clone()}
                    done.append(j)
                else:
                    e, conv = j.scf.update(j.J[0].clone(), j.K[0].clone(), self.scf_conv)
                    j.iters += 1
                    if conv or j.iters >= self.scf_max_iter:
                        j.result = {"energy": e, "converged": conv, "iterations": j.iters}
                        done.append(j)
                    else:
                        j.D = j.scf.build_density().unsqueeze(0).contiguous()
            if done:
                self.sync()
                now = time.perf_counter() - t0
                for j in done:
                    self._retire(j, now)
                    active.remove(j)
                    retired.append(j)
        free_retired()
        makespan = time.perf_counter() - t0
        if self.pool is not None:
            self.pool.shutdown(wait=True)
        return summarize(jobs, makespan, {"ticks": self.ticks, "mean_batch": float(np.mean(self.batch_sizes)),
                                          "prepared_ahead": self.prepared_ahead})


def run_sequential(jobs: List[Job], scf_conv: float = 1e-8, scf_max_iter: int = 100, keep_results=False):
    """Baseline: one request at a time in arrival order, FP64, each with its own plan."""
    import torch
    order = sorted(jobs, key=lambda j: j.arrival)
    t0 = time.perf_counter()
    for j in order:
        now = time.perf_counter() - t0
        if now < j.arrival:
            time.sleep(j.arrival - now)
        j.admit = time.perf_counter() - t0
        plan = Plan(j.mol, precision=ERI_FP64)
        if j.kind == "jk":
            D = torch.from_numpy(np.ascontiguousarray(j.mol.D[:1])).cuda()
            J, K = plan.jk(D)
            torch.cuda.synchronize()
            if keep_results:
                j.result = {"J": J[0].clone(), "K": K[0].clone()}
        else:
            r = RHF(j.mol, plan=plan, incremental=True).kernel(conv_tol=scf_conv, max_iter=scf_max_iter)
            j.result = {"energy": r.energy, "converged": r.converged, "iterations": r.iterations}
            j.iters = r.iterations
        plan.close()
        j.finish = time.perf_counter() - t0
    return summarize(jobs, time.perf_counter() - t0, {})


def summarize(jobs: List[Job], makespan: float, extra: Dict) -> Dict:
    lat = [j.finish - j.arrival for j in jobs]
    out = {"requests": len(jobs), "makespan_s": makespan, "throughput_req_s": len(jobs) / makespan,
           "p50_latency_s": _percentile(lat, 50), "p99_latency_s": _percentile(lat, 99),
           "mean_latency_s": float(np.mean(lat)) if lat else math.nan}
    out.update(extra)
    return out


def make_jobs(requests, natm_cap: Optional[int] = None) -> List[Job]:
    """Jobs of the served workload: molecules of the heavy/light recipe (3s2p1d / 2s1p,
    6-31G(d)-like depths) with each request's atom count and seed."""
    from workloads import config_scf
    jobs = []
    for r in requests:
        natm = r.natm if natm_cap is None else min(r.natm, natm_cap)
        mol = config_scf(seed=r.seed, natm=natm)
        jobs.append(Job(rid=r.rid, kind=r.kind, mol=mol, arrival=r.arrival_s, footprint=footprint_bytes(mol, r.kind)))
    return jobs


def main():
    """Served-workload benchmark: continuous batching in mixed precision and in FP64 against
    sequential FP64 on the same requests; prints one JSON line."""
    import argparse
    import json

    from workloads import config_served_requests
    from . import build

    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--mean-interarrival", type=float, default=0.02)
    ap.add_argument("--natm-min", type=int, default=5)
    ap.add_argument("--natm-max", type=int, default=80)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--slots", type=int, default=32)
    ap.add_argument("--hbm-gb", type=float, default=64.0)
    ap.add_argument("--no-sequential", action="store_true")
    ap.add_argument("--no-batched-fp64", action="store_true")
    args = ap.parse_args()
    build()
    reqs = config_served_requests(seed=args.seed, nreq=args.requests, mean_interarrival_s=args.mean_interarrival,
                                  natm_range=(args.natm_min, args.natm_max))
    # warm the kernels and the allocator on one small request
    Server().run(make_jobs(reqs[:1], natm_cap=5))

    def arm(fn):
        jobs = make_jobs(reqs)
        out = fn(jobs)
        scf = [j for j in jobs if j.kind == "scf"]
        out["scf_jobs"] = len(scf)
        out["scf_converged"] = sum(1 for j in scf if j.result.get("converged"))
        out["scf_iterations_mean"] = float(np.mean([j.iters for j in scf])) if scf else 0.0
        return out

    budget = int(args.hbm_gb * (1 << 30))
    out = {"workload": f"{args.requests} requests, exponential inter-arrival mean {args.mean_interarrival * 1e3:.0f} ms, "
                       f"atoms log-uniform [{args.natm_min}, {args.natm_max}], 30% RHF to 1e-8 Ha (at most 100 "
                       "iterations), 70% single J/K; heavy/light 3s2p1d/2s1p recipe",
           "batched_mixed": arm(lambda jobs: Server(hbm_budget=budget, max_slots=args.slots).run(jobs))}
    if not args.no_batched_fp64:
        out["batched_fp64"] = arm(lambda jobs: Server(precision=ERI_FP64, hbm_budget=budget,
                                                      max_slots=args.slots).run(jobs))
    if not args.no_sequential:
        out["sequential_fp64"] = arm(run_sequential)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
