"""Two-electron energy gradient on the GPU (eri_jk_grad through the C-ABI) against the
oracle's gradient by definition (shifted-shell derivative integrals, Sec. 4), and
properties that hold at any size: translational invariance, agreement with central
differences of the GPU's own J/K energies, independence of the plan precision."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2407_09700_gb300 as pkg  # noqa: E402
from oracle import grad_ref  # noqa: E402
from workloads import config_high_l, config_medium, custom_molecule, random_psd_density  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def _mol(seed, ls_per_atom, natm, kmax=3, spread=1.4):
    rng = np.random.default_rng(seed)
    coords = rng.uniform(-spread, spread, (natm, 3))
    shells = []
    for a in range(natm):
        for l in ls_per_atom[a % len(ls_per_atom)]:
            K = int(rng.integers(1, kmax + 1))
            shells.append((a, l, np.sort(rng.uniform(0.3, 3.0, K))[::-1], rng.uniform(0.2, 1.0, K)))
    m = custom_molecule(coords, shells)
    m.D = random_psd_density(m.nbf, max(2, m.nbf // 3), rng)
    return m


def _gpu_grad(m, D, tau=0.0, precision=pkg.ERI_FP64):
    plan = pkg.Plan(m, tau=tau, precision=precision)
    gJ, gK = plan.jk_grad(torch.from_numpy(np.ascontiguousarray(D)).cuda())
    torch.cuda.synchronize()
    st = plan.grad_stats()
    plan.close()
    return gJ.cpu().numpy(), gK.cpu().numpy(), st


def _close(got, ref, rel=1e-10):
    scale = max(1.0, float(np.abs(ref).max()))
    np.testing.assert_allclose(got, ref, atol=rel * scale, rtol=0)


@pytest.mark.parametrize("seed,ls,natm", [
    (0, [(0, 1), (1,), (0,)], 3),        # s, p on three centres, contracted
    (1, [(2,), (0, 1)], 2),              # d with s, p
    (2, [(1, 2), (3,)], 2),              # p, d, f
    (4, [(0,)], 4),                      # four distinct centres, s only
    (5, [(1,)], 1),                      # one centre: every derivative cancels
])
def test_grad_matches_oracle(seed, ls, natm):
    m = _mol(seed, ls, natm)
    gJr, gKr = grad_ref.jk_grad(m, m.D[0])
    gJ, gK, st = _gpu_grad(m, m.D[0])
    _close(gJ, gJr)
    _close(gK, gKr)
    assert st["quartets"] > 0


def test_grad_every_class_s_to_g():
    """Two centres with one shell of each l = 0..4: every class up to (gg|gg), whose
    derivative needs h functions and nine Rys roots."""
    rng = np.random.default_rng(5)
    coords = np.array([[0.0, 0.0, 0.0], [0.9, -0.4, 0.7]])
    shells = [(a, l, np.array([rng.uniform(0.4, 1.5)]), np.array([1.0])) for a in range(2) for l in range(5)]
    m = custom_molecule(coords, shells)
    D = random_psd_density(m.nbf, 6, rng)[0]
    gJr, gKr = grad_ref.jk_grad(m, D)
    gJ, gK, _ = _gpu_grad(m, D)
    _close(gJ, gJr)
    _close(gK, gKr)


def test_grad_translational_invariance_at_scale():
    """Screened medium workload (12 atoms, tau = 1e-12): the gradient sums to zero over
    atoms for every screening, since each quartet's four centre derivatives do."""
    m = config_medium(seed=0, nD=1, natm=12)
    gJ, gK, _ = _gpu_grad(m, m.D[0], tau=m.tau)
    for g in (gJ, gK):
        assert np.abs(g.sum(axis=0)).max() <= 1e-11 * np.abs(g).max()
        assert np.abs(g).max() > 0


def _energies(m, D, coords):
    md = m.translated([0.0, 0.0, 0.0])
    md.coords = np.ascontiguousarray(coords)
    plan = pkg.Plan(md, tau=0.0)
    J, K = plan.jk(torch.from_numpy(np.ascontiguousarray(D)).cuda())
    torch.cuda.synchronize()
    Dt = torch.from_numpy(D).cuda()
    eJ = 0.5 * float((Dt * J).sum())
    eK = -0.25 * float((Dt * K).sum())
    plan.close()
    return eJ, eK


@pytest.mark.parametrize("cfg", ["medium", "high_l"])
def test_grad_matches_central_differences_of_gpu_energies(cfg):
    if cfg == "medium":
        m = config_medium(seed=1, nD=1, natm=5)
    else:
        m = config_high_l(seed=1, nD=1, natm=3, nocc=10)
    D = m.D[0]
    gJ, gK, _ = _gpu_grad(m, D)
    h = 1e-4
    rng = np.random.default_rng(0)
    for _ in range(3):
        atom, ax = int(rng.integers(m.natm)), int(rng.integers(3))
        cp, cm = m.coords.copy(), m.coords.copy()
        cp[atom, ax] += h
        cm[atom, ax] -= h
        ejp, ekp = _energies(m, D, cp)
        ejm, ekm = _energies(m, D, cm)
        assert (ejp - ejm) / (2 * h) == pytest.approx(gJ[atom, ax], abs=2e-6 * max(1.0, abs(gJ[atom, ax])))
        assert (ekp - ekm) / (2 * h) == pytest.approx(gK[atom, ax], abs=2e-6 * max(1.0, abs(gK[atom, ax])))


def test_grad_independent_of_plan_precision():
    """The gradient path is FP64 for every plan: a mixed plan gives the same gradient up to
    the order of FP64 atomic additions."""
    m = _mol(7, [(0, 1, 2)], 3)
    a = _gpu_grad(m, m.D[0], tau=1e-12)
    b = _gpu_grad(m, m.D[0], tau=1e-12, precision=pkg.ERI_MIXED)
    _close(b[0], a[0], 1e-13)
    _close(b[1], a[1], 1e-13)
