"""Pin the oracle's two-electron gradient: central finite differences of E_J and E_K
(computed from the oracle's J/K by definition, with D fixed) and translational
invariance (the gradient sums to zero over atoms)."""

import numpy as np
import pytest

from oracle import grad_ref
from workloads import custom_molecule, random_psd_density


def _mol(seed, ls_per_atom, natm=3):
    rng = np.random.default_rng(seed)
    coords = rng.uniform(-1.4, 1.4, (natm, 3))
    shells = []
    for a in range(natm):
        for l in ls_per_atom[a % len(ls_per_atom)]:
            K = int(rng.integers(1, 3))
            shells.append((a, l, np.sort(rng.uniform(0.3, 2.5, K))[::-1], rng.uniform(0.2, 1.0, K)))
    m = custom_molecule(coords, shells)
    m.D = random_psd_density(m.nbf, max(2, m.nbf // 3), rng)
    return m


@pytest.mark.parametrize("seed,ls", [(0, [(0, 1), (1,), (0,)]), (1, [(2,), (0, 1)]), (2, [(1, 2), (3,)]),
                                     (3, [(4,), (0,)])])
def test_gradient_matches_finite_differences(seed, ls):
    m = _mol(seed, ls, natm=3 if len(ls) > 2 else 2)
    gJ, gK = grad_ref.jk_grad(m, m.D)
    assert np.abs(gJ.sum(axis=0)).max() <= 1e-10 * np.abs(gJ).max()
    assert np.abs(gK.sum(axis=0)).max() <= 1e-10 * np.abs(gK).max()
    h = 1e-4
    for atom in range(m.natm):
        for ax in range(3):
            cp = m.coords.copy()
            cm = m.coords.copy()
            cp[atom, ax] += h
            cm[atom, ax] -= h
            ejp, ekp = grad_ref.jk_energies(m, m.D, coords=cp)
            ejm, ekm = grad_ref.jk_energies(m, m.D, coords=cm)
            assert (ejp - ejm) / (2 * h) == pytest.approx(gJ[atom, ax], abs=2e-7)
            assert (ekp - ekm) / (2 * h) == pytest.approx(gK[atom, ax], abs=2e-7)
