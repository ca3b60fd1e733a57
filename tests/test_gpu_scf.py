"""RHF driver on the GPU (J/K through the C-ABI) against the oracle's plain RHF."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2407_09700_gb300 as pkg  # noqa: E402
from oracle import scf_ref  # noqa: E402
from paper_2407_09700_gb300.scf import RHF  # noqa: E402
from workloads import config_scf, custom_molecule  # noqa: E402

STO3G_H = ([3.42525091, 0.62391373, 0.16885540], [0.15432897, 0.53532814, 0.44463454])


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def _small(seed=0):
    rng = np.random.default_rng(seed)
    coords = np.array([[0.0, 0.0, 0.0], [1.9, 0.3, -0.2], [-0.7, 1.8, 0.4]])
    shells = []
    for a, ls in enumerate([(0, 0, 1, 2), (0, 1), (0, 1)]):
        for l in ls:
            K = int(rng.integers(1, 4))
            shells.append((a, l, np.sort(rng.uniform(0.2, 4.0, K))[::-1], rng.uniform(0.2, 1.0, K)))
    return custom_molecule(coords, shells, charges=[6.0, 1.0, 1.0])


def test_h2_sto3g_on_gpu():
    e, c = STO3G_H
    m = custom_molecule([[0, 0, 0], [0, 0, 1.4]], [(0, 0, e, c), (1, 0, e, c)], charges=[1.0, 1.0])
    r = RHF(m).kernel(conv_tol=1e-10)
    assert r.converged
    assert r.energy == pytest.approx(-1.1167, abs=1e-4)


def test_heh_plus_sto3g_on_gpu():
    """The textbook HeH+ / STO-3G example (Szabo & Ostlund, App. B: -2.860662 Hartree)."""
    from test_onee_scf import heh_plus
    r = RHF(heh_plus(), charge=1).kernel(conv_tol=1e-12, max_iter=100)
    assert r.converged
    assert r.energy == pytest.approx(-2.860662, abs=1e-5)


def test_rhf_matches_oracle_rhf():
    m = _small(1)
    # plain DIIS from the second iteration (the default) and a damped start (three damped
    # densities, DIIS from the fourth iteration), each against the oracle's RHF with that scheme
    ref_E, ref_hist, _ = scf_ref.rhf(m, fixed_iters=12)
    r = RHF(m).kernel(fixed_iters=12)
    np.testing.assert_allclose(r.energies, ref_hist, atol=1e-8, rtol=0)
    ref_E, ref_hist, _ = scf_ref.rhf(m, fixed_iters=12, damp=0.5, damp_cycles=3, diis_start=3)
    r = RHF(m, damp=0.5, damp_cycles=3, diis_start=3).kernel(fixed_iters=12)
    np.testing.assert_allclose(r.energies, ref_hist, atol=1e-8, rtol=0)


def test_rhf_mixed_within_1e6_hartree():
    m = config_scf(seed=2, natm=6)
    e64 = RHF(m).kernel(conv_tol=1e-9, max_iter=60)
    emx = RHF(m, plan=pkg.Plan(m, precision=pkg.ERI_MIXED, mixed_thresh=1e-4, mixed_min_tasks=0)).kernel(
        conv_tol=1e-9, max_iter=60)
    assert e64.converged and emx.converged
    assert abs(e64.energy - emx.energy) <= 1e-6, (e64.energy, emx.energy)


def test_incremental_builds_match_full_builds():
    """PySCF-style incremental J/K (density changes after the first build) gives the energies
    of full rebuilds, iteration by iteration, in FP64; in mixed precision within 1e-6 Ha."""
    m = _small(1)
    full = RHF(m).kernel(fixed_iters=15)
    inc = RHF(m, incremental=True).kernel(fixed_iters=15)
    np.testing.assert_allclose(inc.energies, full.energies, atol=1e-9, rtol=0)
    mx = RHF(m, incremental=True, plan=pkg.Plan(m, precision=pkg.ERI_MIXED, mixed_min_tasks=0)).kernel(
        fixed_iters=15)
    assert abs(mx.energy - full.energy) <= 1e-6
    m2 = config_scf(seed=2, natm=6)
    a = RHF(m2).kernel(conv_tol=1e-9, max_iter=60)
    b = RHF(m2, precision=pkg.ERI_MIXED, incremental=True, plan=pkg.Plan(m2, precision=pkg.ERI_MIXED,
                                                                        mixed_min_tasks=0)).kernel(
        conv_tol=1e-9, max_iter=60)
    assert a.converged and b.converged
    assert abs(a.energy - b.energy) <= 1e-6, (a.energy, b.energy)
