"""Pin the CPU oracle to results fixed by mathematics (no GPU).

Each check targets a class of plausible mistakes in the oracle:
  * closed-form (ss|ss) and the one-centre identity  -> prefactor, Boys, norms;
  * brute-force 6D integration up to g               -> OS VRR and HGP HRR terms,
                                                        signs, indices, operand order;
  * unit self-overlap of normalised x^l functions    -> normalisation;
  * 8-fold permutation symmetry (Sec. 3)             -> HRR direction, transposes;
  * Cauchy-Schwarz inequality (Eq. 7)                -> gross value errors;
  * positivity of tr(DJ), tr(DK) >= 0                -> digestion signs;
  * translation and atom-permutation invariance      -> centre handling;
  * J/K from the full ERI tensor                     -> symmetry expansion in digestion.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from workloads import config_tiny, custom_molecule, random_psd_density


def _rand_mol(rng, ls, nprim=1, spread=1.5, same_centre=False):
    coords = np.zeros((len(ls), 3)) if same_centre else rng.uniform(-spread, spread, (len(ls), 3))
    shells = []
    for i, l in enumerate(ls):
        e = np.sort(rng.uniform(0.25, 2.5, nprim))[::-1]
        c = rng.uniform(0.2, 1.0, nprim)
        shells.append((i, l, e, c))
    return custom_molecule(coords, shells)


# ---------------------------------------------------------------- closed forms

def test_one_centre_ss_identity():
    # four identical normalised s functions on one centre: (ss|ss) = 2 sqrt(a/pi)
    for a in (0.1, 1.0, 3.7, 42.0):
        m = custom_molecule([[0.3, -0.2, 0.5]], [(0, 0, [a], [0.77])])
        g = oracle.shell_quartet(m, 0, 0, 0, 0).item()
        assert g == pytest.approx(2.0 * math.sqrt(a / math.pi), rel=2e-15)


def _ss_closed(A, a, B, b, C, c, D, d):
    zeta, eta = a + b, c + d
    P = (a * A + b * B) / zeta
    Q = (c * C + d * D) / eta
    rho = zeta * eta / (zeta + eta)
    T = rho * np.sum((P - Q) ** 2)
    F0 = 1.0 if T < 1e-300 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    return (2 * math.pi ** 2.5 / (zeta * eta * math.sqrt(zeta + eta))
            * math.exp(-a * b / zeta * np.sum((A - B) ** 2))
            * math.exp(-c * d / eta * np.sum((C - D) ** 2)) * F0)


def test_contracted_ss_closed_form():
    rng = np.random.default_rng(3)
    for trial in range(20):
        m = _rand_mol(rng, [0, 0, 0, 0], nprim=3, spread=2.5)
        cn = oracle.normalise(m)
        ref = 0.0
        cen = [m.coords[int(m.shell_atom[s])] for s in range(4)]
        prim = [[(m.exps[int(m.shell_off[s]) + p], cn[int(m.shell_off[s]) + p])
                 for p in range(int(m.shell_nprim[s]))] for s in range(4)]
        for (a, ca), (b, cb), (c, cc), (d, cd) in itertools.product(*prim):
            ref += ca * cb * cc * cd * _ss_closed(cen[0], a, cen[1], b, cen[2], c, cen[3], d)
        g = oracle.shell_quartet(m, 0, 1, 2, 3).item()
        assert g == pytest.approx(ref, rel=1e-13)


def test_normalised_self_overlap():
    rng = np.random.default_rng(5)
    for l in range(5):
        e = np.sort(rng.uniform(0.1, 5.0, 3))
        c = rng.uniform(0.1, 1.0, 3)
        m = custom_molecule([[0, 0, 0]], [(0, l, e, c)])
        cn = oracle.normalise(m)
        assert brute.overlap_xl(l, e, cn) == pytest.approx(1.0, rel=1e-13)
        # raw coefficients are only defined up to a common factor
        m2 = custom_molecule([[0, 0, 0]], [(0, l, e, 3.5 * c)])
        np.testing.assert_allclose(oracle.normalise(m2), cn, rtol=1e-14)


# ---------------------------------------------------------------- brute force

LOW = [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (1, 1, 0, 0),
       (1, 0, 1, 0), (1, 1, 1, 1), (2, 0, 0, 0), (0, 2, 1, 0), (2, 1, 1, 0), (2, 2, 0, 0),
       (1, 2, 0, 2), (2, 1, 2, 1), (2, 2, 2, 2)]


@pytest.mark.parametrize("ls", LOW)
def test_brute_force_low_l(ls):
    rng = np.random.default_rng(hash(ls) % 2 ** 32)
    m = _rand_mol(rng, list(ls), nprim=1)
    cn = oracle.normalise(m)
    g = oracle.shell_quartet(m, 0, 1, 2, 3)
    b = brute.contracted_block(m, cn, 0, 1, 2, 3, ns=400)
    scale = np.abs(g).max()
    assert np.abs(g - b).max() <= 1e-11 * scale, (ls, np.abs(g - b).max(), scale)


@pytest.mark.parametrize("ls", [(0, 1, 1, 0), (1, 2, 0, 1)])
def test_brute_force_contracted(ls):
    rng = np.random.default_rng(17 + sum(ls))
    m = _rand_mol(rng, list(ls), nprim=2)
    cn = oracle.normalise(m)
    g = oracle.shell_quartet(m, 0, 1, 2, 3)
    b = brute.contracted_block(m, cn, 0, 1, 2, 3, ns=300)
    assert np.abs(g - b).max() <= 1e-11 * np.abs(g).max()


@pytest.mark.parametrize("ls", [(3, 0, 0, 0), (4, 0, 0, 0), (3, 1, 2, 0), (4, 2, 1, 1), (4, 4, 0, 0),
                                (3, 3, 3, 3), (4, 4, 4, 4)])
def test_brute_force_high_l(ls):
    rng = np.random.default_rng(101 + 7 * sum(ls))
    m = _rand_mol(rng, list(ls), nprim=1, spread=1.2)
    cn = oracle.normalise(m)
    g = oracle.shell_quartet(m, 0, 1, 2, 3)
    b = brute.contracted_block(m, cn, 0, 1, 2, 3, ns=300, nh=16)
    assert np.abs(g - b).max() <= 1e-10 * np.abs(g).max(), (ls, np.abs(g - b).max())


# ---------------------------------------------------------------- symmetry and bounds

def test_eightfold_symmetry_all_l():
    rng = np.random.default_rng(7)
    for ls in [(1, 0, 2, 1), (3, 2, 4, 1), (4, 3, 2, 0), (2, 2, 1, 1)]:
        m = _rand_mol(rng, list(ls), nprim=2)
        g = oracle.shell_quartet(m, 0, 1, 2, 3)
        perms = {(1, 0, 2, 3): (1, 0, 2, 3), (0, 1, 3, 2): (0, 1, 3, 2), (2, 3, 0, 1): (2, 3, 0, 1),
                 (3, 2, 1, 0): (3, 2, 1, 0), (1, 0, 3, 2): (1, 0, 3, 2), (2, 3, 1, 0): (2, 3, 1, 0),
                 (3, 2, 0, 1): (3, 2, 0, 1)}
        for sh, axes in perms.items():
            h = oracle.shell_quartet(m, *sh)
            # h[x_sh0, x_sh1, x_sh2, x_sh3]; bring back to (0,1,2,3) order
            back = np.transpose(h, np.argsort(axes))
            assert np.abs(back - g).max() <= 1e-12 * np.abs(g).max() + 1e-300


def test_schwarz_inequality():
    m = config_tiny(seed=2)
    b = oracle.OracleBasis(m)
    ns = m.nshell
    diag = {}
    for i in range(ns):
        for j in range(ns):
            g = oracle.shell_quartet(b, i, j, i, j)
            ni, nj = g.shape[0], g.shape[1]
            diag[(i, j)] = np.array([[g[a, c, a, c] for c in range(nj)] for a in range(ni)])
    rng = np.random.default_rng(0)
    for _ in range(40):
        i, j, k, l = rng.integers(0, ns, 4)
        g = oracle.shell_quartet(b, i, j, k, l)
        bound = np.sqrt(np.einsum("ab,cd->abcd", diag[(i, j)], diag[(k, l)]))
        assert np.all(np.abs(g) <= bound * (1 + 1e-13) + 1e-15)
    Q = oracle.schwarz(b)
    for (i, j), d in diag.items():
        assert Q[i, j] == pytest.approx(math.sqrt(np.abs(d).max()), rel=1e-15)


def _full_tensor(b, mol):
    nbf = b.nbf
    f0 = mol.shell_first_bf()
    G = np.zeros((nbf,) * 4)
    ns = mol.nshell
    for i, j, k, l in itertools.product(range(ns), repeat=4):
        g = oracle.shell_quartet(b, i, j, k, l)
        G[f0[i]:f0[i] + g.shape[0], f0[j]:f0[j] + g.shape[1],
          f0[k]:f0[k] + g.shape[2], f0[l]:f0[l] + g.shape[3]] = g
    return G


def test_jk_match_full_tensor_definition():
    m = config_tiny(seed=1, nD=2)
    b = oracle.OracleBasis(m)
    G = _full_tensor(b, m)
    J, K, n = oracle.jk(b, m.D, screen=False)
    ns = m.nshell
    npair = ns * (ns + 1) // 2
    assert n == npair * (npair + 1) // 2
    for x in range(2):
        Jr = np.einsum("ijkl,kl->ij", G, m.D[x])
        Kr = np.einsum("ijkl,jl->ik", G, m.D[x])
        assert np.abs(J[x] - Jr).max() <= 1e-13 * np.abs(Jr).max()
        assert np.abs(K[x] - Kr).max() <= 1e-13 * np.abs(Kr).max()
        assert np.abs(J[x] - J[x].T).max() <= 1e-14 * np.abs(J[x]).max()
        assert np.abs(K[x] - K[x].T).max() <= 1e-14 * np.abs(K[x]).max()


def test_jk_mixed_l_small_molecule_definition():
    rng = np.random.default_rng(11)
    shells = [(0, 0, [1.3, 0.4], [0.5, 0.6]), (0, 2, [0.8], [1.0]), (1, 1, [1.1, 0.3], [0.4, 0.7]),
              (1, 3, [0.6], [1.0]), (2, 4, [0.9], [1.0]), (2, 0, [0.5], [1.0])]
    m = custom_molecule(rng.uniform(-1.5, 1.5, (3, 3)), shells)
    m.D = random_psd_density(m.nbf, 4, rng)
    b = oracle.OracleBasis(m)
    G = _full_tensor(b, m)
    J, K, _ = oracle.jk(b, m.D, screen=False)
    Jr = np.einsum("ijkl,kl->ij", G, m.D[0])
    Kr = np.einsum("ijkl,jl->ik", G, m.D[0])
    assert np.abs(J[0] - Jr).max() <= 1e-13 * np.abs(Jr).max()
    assert np.abs(K[0] - Kr).max() <= 1e-13 * np.abs(Kr).max()
    # sampled blocks from the definition agree with the full build
    pairs = [(0, 0), (3, 1), (4, 2), (5, 4)]
    Jb, Kb = oracle.jk_blocks(b, pairs, D=m.D, screen=False)
    f0 = m.shell_first_bf()
    for s, (I, X) in enumerate(pairs):
        ni, nx = Jb[s].shape[1], Jb[s].shape[2]
        np.testing.assert_allclose(Jb[s][0], J[0][f0[I]:f0[I] + ni, f0[X]:f0[X] + nx],
                                   atol=1e-13 * np.abs(J).max(), rtol=0)
        np.testing.assert_allclose(Kb[s][0], K[0][f0[I]:f0[I] + ni, f0[X]:f0[X] + nx],
                                   atol=1e-13 * np.abs(K).max(), rtol=0)


def test_positivity():
    for seed in range(3):
        m = config_tiny(seed=seed)
        J, K, _ = oracle.jk(m, screen=False)
        D = m.D[0]
        assert np.sum(D * J[0]) > 0
        assert np.sum(D * K[0]) >= -1e-14
        # the Coulomb kernel is positive definite: any non-zero symmetric D gives tr(DJ) > 0
        rng = np.random.default_rng(seed)
        S = rng.standard_normal(D.shape)
        S = S + S.T
        J2, _, _ = oracle.jk(m, D=S, screen=False)
        assert np.sum(S * J2[0]) > 0


def test_translation_and_atom_permutation_invariance():
    m = config_tiny(seed=4)
    J, K, _ = oracle.jk(m, screen=False)
    J2, K2, _ = oracle.jk(m.translated([3.1, -7.2, 0.4]), screen=False)
    assert np.abs(J - J2).max() <= 1e-12
    assert np.abs(K - K2).max() <= 1e-12
    # reverse the atom order (shells follow their atoms); J and K permute accordingly
    order = [2, 1, 0]
    shells, perm_bf = [], []
    f0 = m.shell_first_bf()
    for new_a, old_a in enumerate(order):
        for s in range(m.nshell):
            if int(m.shell_atom[s]) == old_a:
                o, n = int(m.shell_off[s]), int(m.shell_nprim[s])
                shells.append((new_a, int(m.shell_l[s]), m.exps[o:o + n], m.coefs[o:o + n]))
                nc = (int(m.shell_l[s]) + 1) * (int(m.shell_l[s]) + 2) // 2
                perm_bf.extend(range(f0[s], f0[s] + nc))
    perm_bf = np.array(perm_bf)
    mp = custom_molecule(m.coords[order], shells)
    Dp = m.D[0][np.ix_(perm_bf, perm_bf)]
    J3, K3, _ = oracle.jk(mp, D=Dp, screen=False)
    assert np.abs(J3[0] - J[0][np.ix_(perm_bf, perm_bf)]).max() <= 1e-12
    assert np.abs(K3[0] - K[0][np.ix_(perm_bf, perm_bf)]).max() <= 1e-12


def test_screening_predicate_effect():
    m = config_tiny(seed=0)
    b = oracle.OracleBasis(m)
    J0, K0, n0 = oracle.jk(b, screen=False)
    J1, K1, n1 = oracle.jk(b, tau=1e-12, screen=True)
    assert n1 <= n0
    assert np.abs(J1 - J0).max() <= 1e-10 and np.abs(K1 - K0).max() <= 1e-10
    # a huge threshold drops every quartet, tau = 0 keeps every pair product > 0
    _, _, nbig = oracle.jk(b, tau=1e6, screen=True)
    assert nbig == 0
    assert oracle.count_quartets(b, tau=0.0, screen=True) == n0


def test_sampled_jk_partitions_the_full_build():
    # the unique quartets split into two disjoint samples add up to the full build
    m = config_tiny(seed=3)
    b = oracle.OracleBasis(m)
    J, K, n = oracle.jk(b, screen=True)
    npair = m.nshell * (m.nshell + 1) // 2
    allq = np.arange(npair * (npair + 1) // 2)
    rng = np.random.default_rng(0)
    rng.shuffle(allq)
    half = allq.size // 2
    J1, K1, n1 = oracle.jk_sample(b, allq[:half])
    J2, K2, n2 = oracle.jk_sample(b, allq[half:])
    assert n1 + n2 == n
    assert np.abs(J1 + J2 - J).max() <= 1e-13 and np.abs(K1 + K2 - K).max() <= 1e-13
