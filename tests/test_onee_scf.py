"""One-electron integrals and the RHF driver's reference (no GPU).

* The library's host S, T, V (Obara-Saika recursions, Boys values from the Rys rule)
  against the oracle's quadrature (Gauss-Hermite per axis; Gaussian transform of 1/r).
* The oracle's quadrature against closed forms for s functions.
* The oracle's plain RHF against exact results: one basis function (E = 2 h + (11|11)
  + E_nuc), the textbook H2 / STO-3G energy at R = 1.4 bohr (Szabo & Ostlund,
  "Modern Quantum Chemistry", Sec. 3.5: -1.117 Hartree) and the book's HeH+ / STO-3G
  worked example at R = 1.4632 bohr (App. B: total energy -2.860662 Hartree, printed to
  6 decimals from integrals of that program's precision), plus translation invariance.
"""

import math

import numpy as np
import pytest

import oracle
from oracle import onee as O
from oracle import scf_ref
import paper_2407_09700_gb300 as pkg
from workloads import custom_molecule, random_psd_density


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def _mol(seed, ls=(0, 1, 2), natm=3, spread=1.5, K=2):
    rng = np.random.default_rng(seed)
    coords = rng.uniform(-spread, spread, (natm, 3))
    shells = []
    for a in range(natm):
        for l in ls:
            e = np.sort(rng.uniform(0.3, 3.0, K))[::-1]
            shells.append((a, l, e, rng.uniform(0.2, 1.0, K)))
    return custom_molecule(coords, shells, charges=rng.integers(1, 8, natm).astype(float))


@pytest.mark.parametrize("seed,ls", [(0, (0, 1)), (1, (0, 1, 2)), (2, (2, 3)), (3, (4, 1))])
def test_library_onee_matches_quadrature(seed, ls):
    m = _mol(seed, ls=ls, natm=2 if max(ls) > 2 else 3)
    S, T, V = pkg.one_electron(m)
    So, To, Vo = O.one_electron(m)
    for a, b in ((S, So), (T, To), (V, Vo)):
        assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max(), np.abs(a - b).max()


def test_quadrature_closed_forms_s():
    A, B, C = np.array([0.1, -0.4, 0.3]), np.array([1.0, 0.2, -0.5]), np.array([-0.3, 0.8, 0.6])
    a, b = 0.8, 1.7
    m = custom_molecule([A, B], [(0, 0, [a], [1.0]), (1, 0, [b], [1.0])])
    S, T, V = O.one_electron(m, charges=[2.5], charge_xyz=[C])
    na, nb = (2 * a / math.pi) ** 0.75, (2 * b / math.pi) ** 0.75
    zeta = a + b
    P = (a * A + b * B) / zeta
    R2 = np.sum((A - B) ** 2)
    K = math.exp(-a * b / zeta * R2)
    s_ab = (math.pi / zeta) ** 1.5 * K
    t_ab = a * b / zeta * (3 - 2 * a * b / zeta * R2) * s_ab
    Tc = zeta * np.sum((P - C) ** 2)
    F0 = 0.5 * math.sqrt(math.pi / Tc) * math.erf(math.sqrt(Tc))
    v_ab = -2.5 * 2 * math.pi / zeta * K * F0
    assert S[0, 1] == pytest.approx(na * nb * s_ab, rel=1e-13)
    assert T[0, 1] == pytest.approx(na * nb * t_ab, rel=1e-12)
    assert V[0, 1] == pytest.approx(na * nb * v_ab, rel=1e-11)
    assert S[0, 0] == pytest.approx(1.0, rel=1e-13)
    assert T[0, 0] == pytest.approx(1.5 * a, rel=1e-12)     # <g|-lap/2|g> = 3a/2 for a normalised s


def test_rhf_one_function_exact():
    m = custom_molecule([[0, 0, 0], [0, 0, 1.7]], [(0, 0, [1.3], [1.0])], charges=[1.0, 1.0])
    E, _, conv = scf_ref.rhf(m)
    S, T, V = O.one_electron(m)
    g = oracle.shell_quartet(m, 0, 0, 0, 0).item()
    assert E == pytest.approx(2 * (T + V)[0, 0] + g + 1.0 / 1.7, abs=1e-12)


STO3G_H = ([3.42525091, 0.62391373, 0.16885540], [0.15432897, 0.53532814, 0.44463454])


def test_rhf_h2_sto3g_textbook():
    e, c = STO3G_H
    m = custom_molecule([[0, 0, 0], [0, 0, 1.4]], [(0, 0, e, c), (1, 0, e, c)], charges=[1.0, 1.0])
    E, _, conv = scf_ref.rhf(m)
    assert conv
    assert E == pytest.approx(-1.1167, abs=1e-4)


def test_rhf_translation_invariance():
    m = _mol(5, ls=(0, 1), natm=3)
    if int(m.charges.sum()) % 2:
        m.charges[0] += 1
    E1, _, _ = scf_ref.rhf(m)
    E2, _, _ = scf_ref.rhf(m.translated([2.0, -1.0, 0.5]))
    assert E1 == pytest.approx(E2, abs=1e-9)


STO3G_1S = ([0.109818, 0.405771, 2.22766], [0.444635, 0.535328, 0.154329])   # zeta = 1 fit


def heh_plus():
    """HeH+ in STO-3G with zeta(He) = 2.0925, zeta(H) = 1.24 at R = 1.4632 bohr."""
    a, d = (np.array(x) for x in STO3G_1S)
    shells = [(0, 0, a * 2.0925 ** 2, d), (1, 0, a * 1.24 ** 2, d)]
    return custom_molecule([[0, 0, 0], [0, 0, 1.4632]], shells, charges=[2.0, 1.0])


def test_rhf_heh_plus_sto3g_textbook():
    E, hist, conv = scf_ref.rhf(heh_plus(), charge=1, conv_tol=1e-12, max_iter=100)
    assert conv
    assert E == pytest.approx(-2.860662, abs=1e-5)
