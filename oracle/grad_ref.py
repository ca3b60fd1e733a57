"""Two-electron energy gradient by definition (test infrastructure only).

E_J = 1/2 sum_abcd (ab|cd) D_ab D_cd and E_K = -1/4 sum_abcd (ab|cd) D_ac D_bd for a
fixed symmetric AO density D (the two-electron part of the RHF energy, Sec. 4, Eq. 9).
Their nuclear gradients sum, over every ordered shell quartet and each of its four
centres on the atom, the derivative integrals contracted with the density products.
The derivative of a contracted Cartesian ERI with respect to the centre of its first
function follows from differentiating each primitive (Obara & Saika):
    d/dA_x (ab|cd) = sum_p c_p [2 alpha_p (a+1_x b|cd)_p - a_x (a-1_x b|cd)_p],
evaluated here with the oracle's OS/HGP quartets over shells of angular momentum
l +- 1 whose coefficients are 2 alpha_p c_p and c_p.  Small molecules only.
"""

from __future__ import annotations

import itertools

import numpy as np

from workloads.molecules import _pack

from . import oracle as _orc
from .brute import cart_list


def _cart_index(l, v):
    return cart_list(l).index(tuple(v))


def _extended(mol):
    """A basis with every shell, then for each shell its l+1 (coefs 2a c) and l-1 (coefs c)
    companions.  Returns (OracleBasis, plus_index[shell], minus_index[shell])."""
    cn = _orc.normalise(mol)
    shells, coefs = [], []
    for s in range(mol.nshell):
        o, n = int(mol.shell_off[s]), int(mol.shell_nprim[s])
        shells.append((int(mol.shell_atom[s]), int(mol.shell_l[s]), mol.exps[o:o + n], cn[o:o + n]))
    ns = mol.nshell
    plus, minus = {}, {}
    for s in range(ns):
        a, l, e, c = shells[s]
        plus[s] = len(shells)
        shells.append((a, l + 1, e, 2.0 * e * c))
        if l > 0:
            minus[s] = len(shells)
            shells.append((a, l - 1, e, c))
    m = _pack("ext", mol.coords, mol.charges, shells)
    return _orc.OracleBasis(m, coefs=m.coefs), plus, minus


def _deriv_block(ob, plus, minus, ls, sh, pos):
    """d/dR_{centre of position pos} of (sh0 sh1|sh2 sh3): array [3, n0, n1, n2, n3]."""
    l = ls[pos]
    base = [int(x) for x in sh]
    up = list(base)
    up[pos] = plus[base[pos]]
    gp = _orc.shell_quartet(ob, *up)
    gm = None
    if l > 0:
        dn = list(base)
        dn[pos] = minus[base[pos]]
        gm = _orc.shell_quartet(ob, *dn)
    shape = [(x + 1) * (x + 2) // 2 for x in ls]
    out = np.zeros([3] + shape)
    comps = cart_list(l)
    for i, v in enumerate(comps):
        for ax in range(3):
            vp = list(v)
            vp[ax] += 1
            ip = _cart_index(l + 1, vp)
            sl_out = [ax] + [slice(None)] * 4
            sl_out[1 + pos] = i
            sl_p = [slice(None)] * 4
            sl_p[pos] = ip
            val = gp[tuple(sl_p)]
            if v[ax] > 0:
                vm = list(v)
                vm[ax] -= 1
                sl_m = [slice(None)] * 4
                sl_m[pos] = _cart_index(l - 1, vm)
                val = val - v[ax] * gm[tuple(sl_m)]
            out[tuple(sl_out)] = val
    return out


def jk_grad(mol, D):
    """(gJ, gK): [natm, 3] gradients of E_J and E_K with D held fixed."""
    D = np.asarray(D, dtype=np.float64)
    if D.ndim == 3:
        D = D[0]
    ob, plus, minus = _extended(mol)
    f0 = mol.shell_first_bf()
    nf = [(int(l) + 1) * (int(l) + 2) // 2 for l in mol.shell_l]
    gJ = np.zeros((mol.natm, 3))
    gK = np.zeros((mol.natm, 3))
    ns = mol.nshell
    for sh in itertools.product(range(ns), repeat=4):
        ls = [int(mol.shell_l[x]) for x in sh]
        blk = [slice(f0[x], f0[x] + nf[x]) for x in sh]
        Dab = D[blk[0], blk[1]]
        Dcd = D[blk[2], blk[3]]
        Dac = D[blk[0], blk[2]]
        Dbd = D[blk[1], blk[3]]
        WJ = 0.5 * np.einsum("ab,cd->abcd", Dab, Dcd)
        WK = -0.25 * np.einsum("ac,bd->abcd", Dac, Dbd)
        for pos in range(4):
            d = _deriv_block(ob, plus, minus, ls, sh, pos)
            atom = int(mol.shell_atom[sh[pos]])
            gJ[atom] += np.einsum("xabcd,abcd->x", d, WJ)
            gK[atom] += np.einsum("xabcd,abcd->x", d, WK)
    return gJ, gK


def jk_energies(mol, D, coords=None):
    """(E_J, E_K) = (1/2 tr D J, -1/4 tr D K) with the oracle's J/K (no screening)."""
    m = mol if coords is None else mol.translated([0, 0, 0])
    if coords is not None:
        m.coords = np.ascontiguousarray(coords)
    D = np.asarray(D, dtype=np.float64)
    J, K, _ = _orc.jk(m, D=D[None] if D.ndim == 2 else D, screen=False)
    Dm = D if D.ndim == 2 else D[0]
    return 0.5 * np.sum(Dm * J[0]), -0.25 * np.sum(Dm * K[0])
