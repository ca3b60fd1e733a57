"""One-electron integrals by quadrature (test infrastructure only).

Independent of recursions and of the Boys function:
  * overlap and kinetic: per Cartesian axis the integrand is a polynomial times
    a Gaussian, integrated exactly (up to rounding) by Gauss-Hermite nodes
    centred on the Gaussian product; the kinetic operator is applied to the
    ket analytically (d^2/dx^2 of (x-B)^j exp(-b (x-B)^2));
  * nuclear attraction: 1/|r - C| = (2/sqrt(pi)) int_0^inf exp(-s^2 |r-C|^2) ds, so
    for fixed s each axis is again a polynomial times one Gaussian (Gauss-Hermite),
    and the s integral uses Gauss-Legendre nodes mapped from [0, 1).
Used to pin the library's S, T, V and the RHF driver on small molecules.
"""

from __future__ import annotations

import math

import numpy as np

from .brute import cart_list
from .oracle import normalise


def _prim_1d(i, j, A, B, a, b, nh=20, kinetic=False):
    """int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) dx (or with -1/2 d^2/dx^2 on the ket)."""
    z, W = np.polynomial.hermite.hermgauss(nh)
    zeta = a + b
    P = (a * A + b * B) / zeta
    K = math.exp(-a * b / zeta * (A - B) ** 2)
    x = P + z / math.sqrt(zeta)
    bra = (x - A) ** i
    if not kinetic:
        ket = (x - B) ** j
    else:
        d = x - B
        ket = -0.5 * ((j * (j - 1) * d ** (j - 2) if j >= 2 else 0.0) - 2 * b * (2 * j + 1) * d ** j
                      + 4 * b * b * d ** (j + 2))
    return K * np.dot(W, bra * ket) / math.sqrt(zeta)


def _prim_nuc_1d(i, j, A, B, C, a, b, s, nh=20):
    """Per-axis factor of the s-transformed attraction at the s nodes."""
    z, W = np.polynomial.hermite.hermgauss(nh)
    zeta = a + b
    P = (a * A + b * B) / zeta
    K = math.exp(-a * b / zeta * (A - B) ** 2)
    s2 = s * s
    g = zeta + s2
    Pp = (zeta * P + s2 * C) / g
    pref = K * np.exp(-zeta * s2 / g * (P - C) ** 2) / np.sqrt(g)
    x = Pp[:, None] + z[None, :] / np.sqrt(g)[:, None]
    return pref * (((x - A) ** i * (x - B) ** j) @ W)


def one_electron(mol, charges=None, charge_xyz=None, ns=300):
    """(S, T, V) for a workloads.Molecule by quadrature."""
    cn = normalise(mol)
    if charges is None:
        charges, charge_xyz = mol.charges, mol.coords
    charge_xyz = np.asarray(charge_xyz, dtype=np.float64).reshape(-1, 3)
    f0 = mol.shell_first_bf()
    nbf = mol.nbf
    S = np.zeros((nbf, nbf))
    T = np.zeros((nbf, nbf))
    V = np.zeros((nbf, nbf))
    xg, wg = np.polynomial.legendre.leggauss(ns)
    u = 0.5 * (xg + 1.0)
    for I in range(mol.nshell):
        A = mol.coords[mol.shell_atom[I]]
        for J in range(mol.nshell):
            B = mol.coords[mol.shell_atom[J]]
            ca, cb = cart_list(int(mol.shell_l[I])), cart_list(int(mol.shell_l[J]))
            for p in range(int(mol.shell_nprim[I])):
                a = mol.exps[mol.shell_off[I] + p]
                c1 = cn[mol.shell_off[I] + p]
                for q in range(int(mol.shell_nprim[J])):
                    b = mol.exps[mol.shell_off[J] + q]
                    cc = c1 * cn[mol.shell_off[J] + q]
                    zeta = a + b
                    sc = math.sqrt(zeta)
                    s = sc * u / (1.0 - u)
                    ws = 0.5 * wg * sc / (1.0 - u) ** 2
                    for ia, av in enumerate(ca):
                        for ib, bv in enumerate(cb):
                            sx = [_prim_1d(av[k], bv[k], A[k], B[k], a, b) for k in range(3)]
                            tx = [_prim_1d(av[k], bv[k], A[k], B[k], a, b, kinetic=True) for k in range(3)]
                            S[f0[I] + ia, f0[J] + ib] += cc * sx[0] * sx[1] * sx[2]
                            T[f0[I] + ia, f0[J] + ib] += cc * (tx[0] * sx[1] * sx[2] + sx[0] * tx[1] * sx[2]
                                                               + sx[0] * sx[1] * tx[2])
                            v = 0.0
                            for Z, Cc in zip(charges, charge_xyz):
                                f = (_prim_nuc_1d(av[0], bv[0], A[0], B[0], Cc[0], a, b, s)
                                     * _prim_nuc_1d(av[1], bv[1], A[1], B[1], Cc[1], a, b, s)
                                     * _prim_nuc_1d(av[2], bv[2], A[2], B[2], Cc[2], a, b, s))
                                v -= Z * 2.0 / math.sqrt(math.pi) * np.dot(ws, f)
                            V[f0[I] + ia, f0[J] + ib] += cc * v
    return S, T, V


def nuclear_repulsion(coords, charges) -> float:
    e = 0.0
    n = len(charges)
    for i in range(n):
        for j in range(i):
            e += charges[i] * charges[j] / np.linalg.norm(np.asarray(coords[i]) - np.asarray(coords[j]))
    return float(e)
