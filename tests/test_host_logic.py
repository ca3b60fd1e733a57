"""Host-side logic without a GPU: the bench's multi-rank plumbing on two gloo ranks
(barrier, max over ranks, replica throughput) and the server's continuous-batching
policy (admission by slots and HBM footprint, requests admitted while others run,
retirement, latency summary) driven by stand-in jobs."""

import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    d = bench.Dist("gloo")
    d.barrier()
    t = 0.25 * (rank + 1)                      # each rank's timed region
    t_max = d.max(t)
    q.put((rank, t_max, bench.replica_throughput(3, ws, t_max)))
    d.barrier()
    d.close()


def test_two_gloo_ranks_barrier_and_max():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [0.5, 0.5]            # both ranks see the slowest rank's time
    assert all(o[2] == pytest.approx(3 * 2 / 0.5) for o in out)


# ---------------------------------------------------------------- server policy with stand-ins

class _FakeBatch:
    def __init__(self, delay):
        self.calls = []
        self.delay = delay

    def jk(self, plans, Ds, Js, Ks):
        import time
        self.calls.append(len(plans))
        time.sleep(self.delay)


class _FakeSCF:
    def __init__(self, iters):
        self.left = iters
        self.D = torch.zeros(1)

    def update(self, J, K, conv):
        self.left -= 1
        return -1.0, self.left <= 0

    def build_density(self):
        return self.D


def _server(**kw):
    from paper_2407_09700_gb300.serve import Server

    class S(Server):
        def _admit(self, job, now):
            job.plan = object()
            job.scf = _FakeSCF(job.mol) if job.kind == "scf" else None
            job.D = job.J = job.K = torch.zeros((1, 1, 1))
            job.admit = now

        def _retire(self, job, now):
            job.finish = now
            job.plan = job.scf = None

    return S(batch=_FakeBatch(kw.pop("delay", 0.002)), sync=lambda: None, prefetch=0, **kw)


def _jobs(spec):
    from paper_2407_09700_gb300.serve import Job
    return [Job(rid=i, kind=k, mol=it, arrival=a, footprint=f) for i, (k, it, a, f) in enumerate(spec)]


def test_server_admits_by_slots_and_footprint():
    # 6 J/K requests at t = 0 of footprint 4; budget 10 and 3 slots -> at most 2 together
    jobs = _jobs([("jk", 0, 0.0, 4)] * 6)
    srv = _server(hbm_budget=10, max_slots=3)
    out = srv.run(jobs)
    assert srv.max_active == 2 and srv.max_used <= 10
    assert srv.batch.calls == [2, 2, 2]
    assert out["requests"] == 6 and all(j.finish >= j.admit >= j.arrival for j in jobs)


def test_server_continuous_admission_and_latency():
    # a long RHF job (10 ticks) is running when J/K requests arrive: they are admitted into
    # the running batch and finish long before it
    jobs = _jobs([("scf", 10, 0.0, 1)] + [("jk", 0, 0.005 * (i + 1), 1) for i in range(4)])
    srv = _server(hbm_budget=100, max_slots=8, delay=0.004)
    out = srv.run(jobs)
    scf, jks = jobs[0], jobs[1:]
    assert srv.ticks == 10
    assert max(srv.batch.calls) >= 2                       # the J/K requests shared ticks with the RHF job
    assert all(j.finish < scf.finish for j in jks)
    lat = sorted(j.finish - j.arrival for j in jobs)
    assert out["p50_latency_s"] == pytest.approx(float(np.percentile(lat, 50)))
    assert out["p99_latency_s"] == pytest.approx(float(np.percentile(lat, 99)))
    assert math.isfinite(out["throughput_req_s"]) and out["throughput_req_s"] > 0


def test_server_prepares_ahead_and_frees_retired_plans_when_idle_or_needed():
    """Arrived requests are prepared on the worker thread before their admission, within the
    budget; retired plans are freed only when no job is active or an admission needs the
    memory, and every prepared plan is freed by the end."""
    from paper_2407_09700_gb300.serve import Server
    log = []

    class S(Server):
        def _prepare(self, job):
            log.append(("prepare", job.rid))
            job.plan = object()

        def _admit(self, job, now):
            assert job.prepared is None or job.prepared.done() or job.prepared.result() is None
            log.append(("admit", job.rid))
            job.scf = _FakeSCF(job.mol) if job.kind == "scf" else None
            job.D = job.J = job.K = torch.zeros((1, 1, 1))
            job.admit = now

        def _retire(self, job, now):
            job.finish = now

        def _destroy(self, job):
            log.append(("free", job.rid))
            job.plan = None

    # budget 10, footprint 4: two jobs at a time; the third needs the first one's memory
    jobs = _jobs([("scf", 3, 0.0, 4), ("jk", 0, 0.0, 4), ("jk", 0, 0.0, 4), ("jk", 0, 0.0, 4)])
    srv = S(batch=_FakeBatch(0.002), sync=lambda: None, prefetch=4, hbm_budget=10, max_slots=4)
    out = srv.run(jobs)
    assert out["requests"] == 4 and srv.max_used <= 10
    assert sorted(r for k, r in log if k == "prepare") == [0, 1, 2, 3][:len([1 for k, _ in log if k == "prepare"])]
    assert sorted(r for k, r in log if k == "free") == [0, 1, 2, 3]
    for rid in range(4):
        assert log.index(("admit", rid)) < log.index(("free", rid))
    assert all(j.plan is None for j in jobs)


def test_server_rejects_a_request_larger_than_the_budget():
    jobs = _jobs([("jk", 0, 0.0, 50)])
    with pytest.raises(RuntimeError, match="exceeds the HBM budget"):
        _server(hbm_budget=10, max_slots=2).run(jobs)


# ---------------------------------------------------------------- bench helpers

def test_clock_summary_flags_throttling_and_skips_bad_lines():
    import bench
    lines = ["2070, 2070, Not Active, Not Active, Not Active, Not Active, 290.5",
             "2070, 2070, Not Active, Not Active, Not Active, Active, 1399.0",
             "1980, 2070, Active, Not Active, Not Active, Not Active, 800.0",
             "garbage line", "[N/A], 2070, Not Active, Not Active, Not Active, Not Active, 300"]
    out = bench.summarize_clock_lines(lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert out["power_w_median"] == 800.0
    assert bench.summarize_clock_lines([])["sm_mhz"] is None


def test_gpu_index_follows_visible_devices(monkeypatch):
    import bench
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3,5")
    assert bench.gpu_index(0) == "3" and bench.gpu_index(1) == "5"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.gpu_index(2) == "2"


def test_replica_throughput_counts_every_rank():
    import bench
    assert bench.replica_throughput(2, 4, 8.0) == pytest.approx(1.0)


# ---------------------------------------------------------------- RHF driver host logic

def test_rhf_driver_steps_match_the_oracle_rhf_on_cpu():
    """The driver's Fock build, energy, DIIS and density update (the step-wise interface the
    server uses), run on CPU tensors with J and K from the oracle, against the oracle's own
    plain RHF iteration by iteration (one-electron integrals from the library's host routine
    on one side, quadrature on the other)."""
    import oracle
    from oracle import scf_ref
    from paper_2407_09700_gb300.scf import RHF
    from workloads import custom_molecule
    import paper_2407_09700_gb300 as pkg
    pkg.build()
    rng = np.random.default_rng(1)
    coords = np.array([[0.0, 0.0, 0.0], [1.9, 0.3, -0.2], [-0.7, 1.8, 0.4]])
    shells = []
    for a, ls in enumerate([(0, 0, 1, 2), (0, 1), (0, 1)]):
        for l in ls:
            K = int(rng.integers(1, 4))
            shells.append((a, l, np.sort(rng.uniform(0.2, 4.0, K))[::-1], rng.uniform(0.2, 1.0, K)))
    m = custom_molecule(coords, shells, charges=[6.0, 1.0, 1.0])
    for scheme in (dict(damp=0.5, damp_cycles=3, diis_start=3), dict(damp=0.0, damp_cycles=0, diis_start=1)):
        drv = RHF(m, plan=object(), device="cpu", **scheme)
        D = drv.start()
        energies = []
        for _ in range(10):
            J, K, _ = oracle.jk(m, D=D.numpy()[None])
            e, _ = drv.update(torch.from_numpy(J[0]), torch.from_numpy(K[0]), None)
            energies.append(e)
            D = drv.D
        _, ref_hist, _ = scf_ref.rhf(m, fixed_iters=10, **scheme)
        np.testing.assert_allclose(energies, ref_hist, atol=1e-8, rtol=0)


def test_reference_arm_under_two_ranks_prints_one_line():
    """`bench.py --impl reference` launched as two ranks: rank 0 times the oracle on a bounded
    sample and prints the one JSON line; rank 1 exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-seconds", "2", "--natm", "6"]
    out = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
