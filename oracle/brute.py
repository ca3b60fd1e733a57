"""Brute-force numerical ERIs for small angular momentum (test infrastructure only).

Independent of the Boys function, of Obara-Saika and of Rys quadrature.  It
writes the Coulomb operator through the Gaussian transform

    1/r12 = (2/sqrt(pi)) * int_0^inf exp(-s^2 r12^2) ds,

so that, for a fixed s, the 6D integral of Eq. 1's primitive quartet (Sec. 2)
factorises into three 2D integrals (one per Cartesian axis) of a polynomial
times a Gaussian in (x1, x2).  Each 2D integral is done exactly (up to
rounding) by a Gauss-Hermite product rule after whitening the 2x2 quadratic
form; the remaining integral over s uses Gauss-Legendre nodes mapped from
[0, 1) with s = c * u / (1 - u), c = sqrt(zeta*eta/(zeta+eta)).

Used to pin the oracle on tiny inputs; it is slow and only meant for l <= 2.
"""

from __future__ import annotations

import math

import numpy as np


def cart_list(l: int):
    """Cartesian exponent triples in x-descending order (xx, xy, xz, yy, yz, zz for l=2)."""
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


def _axis_tables(la, lb, lc, ld, A, B, C, D, al, be, ga, de, s, nh):
    """2D integrals for one axis at the s nodes: shape (ns, la+1, lb+1, lc+1, ld+1)."""
    z, W = np.polynomial.hermite.hermgauss(nh)
    zeta, eta = al + be, ga + de
    P = (al * A + be * B) / zeta
    Q = (ga * C + de * D) / eta
    kab = math.exp(-al * be / zeta * (A - B) ** 2)
    kcd = math.exp(-ga * de / eta * (C - D) ** 2)
    d = P - Q
    s2 = s * s
    det = zeta * eta + s2 * (zeta + eta)
    y1s = -s2 * d * eta / det
    y2s = s2 * d * zeta / det
    r11 = np.sqrt(zeta + s2)
    r22 = np.sqrt(det / (zeta + s2))
    pref = kab * kcd * np.exp(-s2 * zeta * eta * d * d / det) / np.sqrt(det)
    # x1 = P + y1* + z1/r11 + z2 s^2/(r11^2 r22);  x2 = Q + y2* + z2/r22
    x1 = (P + y1s)[:, None, None] + z[None, :, None] / r11[:, None, None] \
        + z[None, None, :] * (s2 / (r11 * r11 * r22))[:, None, None]
    x2 = (Q + y2s)[:, None] + z[None, :] / r22[:, None]
    pa = np.stack([(x1 - A) ** k for k in range(la + 1)], axis=-1)   # (ns, i, j, a)
    pb = np.stack([(x1 - B) ** k for k in range(lb + 1)], axis=-1)
    pc = np.stack([(x2 - C) ** k for k in range(lc + 1)], axis=-1)   # (ns, j, c)
    pd = np.stack([(x2 - D) ** k for k in range(ld + 1)], axis=-1)
    t = np.einsum("i,j,sija,sijb,sjc,sjd->sabcd", W, W, pa, pb, pc, pd, optimize=True)
    return t * pref[:, None, None, None, None]


def primitive_block(la, A, al, lb, B, be, lc, C, ga, ld, D, de, ns=400, nh=14):
    """[ab|cd] for un-normalised Cartesian primitives (Eq. 2), shape (na, nb, nc, nd)."""
    A, B, C, D = (np.asarray(v, dtype=np.float64) for v in (A, B, C, D))
    zeta, eta = al + be, ga + de
    c = math.sqrt(zeta * eta / (zeta + eta))
    x, w = np.polynomial.legendre.leggauss(ns)
    u = 0.5 * (x + 1.0)
    s = c * u / (1.0 - u)
    ws = 0.5 * w * c / (1.0 - u) ** 2
    tabs = [_axis_tables(la, lb, lc, ld, A[k], B[k], C[k], D[k], al, be, ga, de, s, nh)
            for k in range(3)]
    ca, cb, cc, cd = cart_list(la), cart_list(lb), cart_list(lc), cart_list(ld)
    out = np.zeros((len(ca), len(cb), len(cc), len(cd)))
    for ia, a in enumerate(ca):
        for ib, b in enumerate(cb):
            for ic, cc_ in enumerate(cc):
                for id_, d in enumerate(cd):
                    f = tabs[0][:, a[0], b[0], cc_[0], d[0]] * tabs[1][:, a[1], b[1], cc_[1], d[1]] \
                        * tabs[2][:, a[2], b[2], cc_[2], d[2]]
                    out[ia, ib, ic, id_] = 2.0 / math.sqrt(math.pi) * np.dot(ws, f)
    return out


def contracted_block(mol, coefs_norm, i, j, k, l, ns=400, nh=14):
    """(ij|kl) for contracted shells, given normalised coefficients (one per primitive)."""
    sh = (i, j, k, l)
    ls = [int(mol.shell_l[x]) for x in sh]
    cen = [mol.coords[int(mol.shell_atom[x])] for x in sh]
    prims = []
    for x in sh:
        o, n = int(mol.shell_off[x]), int(mol.shell_nprim[x])
        prims.append([(mol.exps[o + p], coefs_norm[o + p]) for p in range(n)])
    out = 0.0
    for a_, ca in prims[0]:
        for b_, cb in prims[1]:
            for c_, cc in prims[2]:
                for d_, cd in prims[3]:
                    out = out + ca * cb * cc * cd * primitive_block(
                        ls[0], cen[0], a_, ls[1], cen[1], b_, ls[2], cen[2], c_, ls[3], cen[3], d_,
                        ns=ns, nh=nh)
    return out


def overlap_xl(l: int, exps, coefs, n=40) -> float:
    """<x^l g | x^l g> for a contracted one-centre function sum_p c_p x^l exp(-a_p r^2),
    by Gauss-Hermite quadrature in each axis (independent of any closed form)."""
    z, W = np.polynomial.hermite.hermgauss(n)
    tot = 0.0
    for ap, cp in zip(exps, coefs):
        for aq, cq in zip(exps, coefs):
            s = ap + aq
            # int x^(2l) e^{-s x^2} dx with x = z / sqrt(s)
            ix = np.dot(W, (z / math.sqrt(s)) ** (2 * l)) / math.sqrt(s)
            iy = np.dot(W, np.ones_like(z)) / math.sqrt(s)
            tot += cp * cq * ix * iy * iy
    return tot
