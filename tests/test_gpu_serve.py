"""Serving loop with continuous batching: every request's result is the same when it
runs alone and when it is batched with other requests (J/K within 1e-12 relative for
FP64 plans, 1e-9 for mixed; RHF energies within 1e-8 Ha), and admission by device
footprint queues requests instead of failing."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2407_09700_gb300 as pkg  # noqa: E402
from paper_2407_09700_gb300.eri import Plan  # noqa: E402
from paper_2407_09700_gb300.scf import RHF  # noqa: E402
from paper_2407_09700_gb300.serve import Server, make_jobs  # noqa: E402
from workloads import config_served_requests  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def _requests(n=10, seed=3):
    reqs = config_served_requests(seed=seed, nreq=n, mean_interarrival_s=0.005, natm_range=(3, 7),
                                  scf_fraction=0.5)
    return reqs


@pytest.mark.parametrize("precision", [pkg.ERI_FP64, pkg.ERI_MIXED])
def test_same_alone_and_in_the_mix(precision):
    reqs = _requests()
    jobs = make_jobs(reqs)
    stats = Server(precision=precision, max_slots=16).run(jobs, keep_results=True)
    assert stats["requests"] == len(reqs) and stats["mean_batch"] > 1.0
    assert stats["prepared_ahead"] > 0             # plans were built ahead of admission
    tol = 1e-12 if precision == pkg.ERI_FP64 else 1e-9
    for j in jobs:
        plan = Plan(j.mol, precision=precision)
        if j.kind == "jk":
            D = torch.from_numpy(np.ascontiguousarray(j.mol.D[:1])).cuda()
            J, K = plan.jk(D)
            torch.cuda.synchronize()
            assert float((J[0] - j.result["J"]).abs().max()) <= tol * float(J.abs().max())
            assert float((K[0] - j.result["K"]).abs().max()) <= tol * float(K.abs().max())
        else:
            r = RHF(j.mol, plan=plan, incremental=True).kernel(conv_tol=1e-8, max_iter=100)
            assert j.result["converged"] and r.converged
            assert abs(r.energy - j.result["energy"]) <= 1e-8
        plan.close()


def test_admission_by_footprint_queues():
    reqs = _requests(n=6, seed=5)
    jobs = make_jobs(reqs)
    budget = max(j.footprint for j in jobs)           # room for one job at a time
    stats = Server(precision=pkg.ERI_FP64, hbm_budget=budget).run(jobs)
    assert stats["requests"] == 6 and stats["mean_batch"] == 1.0
    assert all(j.admit >= prev.finish - 1e-9 for prev, j in zip(sorted(jobs, key=lambda x: x.admit),
                                                                  sorted(jobs, key=lambda x: x.admit)[1:]))
    with pytest.raises(RuntimeError):
        Server(hbm_budget=16).run(make_jobs(reqs[:1]))
