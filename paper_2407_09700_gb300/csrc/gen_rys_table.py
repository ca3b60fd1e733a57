#!/usr/bin/env python3
"""Generate the Rys root/weight interpolation table compiled into the library.

The N-point Rys rule integrates f(t^2) against exp(-T t^2) on t in [0, 1]
exactly for polynomials f of degree < 2N (Eq. 1, Sec. 2).  In u = t^2 it is
the Gauss rule of the weight exp(-T u) / (2 sqrt(u)) on [0, 1], whose moments
are the Boys functions F_k(T).  For each N = 1..9 this script

  1. computes the exact rule at 60 significant digits: Boys moments F_k(T)
     (positive series plus downward recursion), recurrence coefficients of the
     orthogonal polynomials by the Chebyshev algorithm (W. Gautschi,
     "Orthogonal Polynomials: Computation and Approximation", 2004, Sec. 2.1.7),
     then nodes and weights from the Jacobi matrix (Golub & Welsch, Math.
     Comp. 23, 221 (1969));
  2. interpolates every u_n(T) and w_n(T) on intervals [i/SUB, (i+1)/SUB) of T by a
     degree-DEG Chebyshev interpolant, re-expanded in powers of
     x = 2 (SUB T - i) - 1 so the device evaluates it by Horner's rule (SUB = 4,
     DEG = 7: 5e-15 worst relative error for 8 FMAs per value, against 12 FMAs per value
     for degree 11 on unit intervals);
  3. above a cutoff T_N uses the large-T limit u_n = v_n / T,
     w_n = W_n / (2 sqrt(T)), with (v_n, W_n) the N-point generalised
     Gauss-Laguerre rule for v^(-1/2) exp(-v) on [0, inf); T_N is the first
     integer beyond which that limit agrees with the exact rule to 2e-17
     relative in every node and weight.

Output: ``rys_table.cpp`` (host arrays; the library copies them to the device once).  The run
checks every interval at interior points, in float64 Horner arithmetic, and
prints the worst relative errors.  Needs mpmath; takes a minute on 8 cores.
"""

from __future__ import annotations

import multiprocessing as mproc
import os
import sys

import mpmath as mp

DPS = 60
NMAX = 9
DEG = 7             # polynomial degree on each interval
SUB = 4             # intervals per unit of T
ASYM_TOL = mp.mpf("2e-17")


def _setup():
    mp.mp.dps = DPS


def boys_all(kmax, T):
    T = mp.mpf(T)
    if T == 0:
        return [mp.mpf(1) / (2 * k + 1) for k in range(kmax + 1)]
    term = mp.mpf(1) / (2 * kmax + 1)
    s = term
    j = 1
    eps = mp.mpf(10) ** (-DPS - 5)
    while True:
        term *= 2 * T / (2 * kmax + 2 * j + 1)
        s += term
        j += 1
        if term < s * eps:
            break
    eT = mp.exp(-T)
    F = [mp.mpf(0)] * (kmax + 1)
    F[kmax] = eT * s
    for k in range(kmax, 0, -1):
        F[k - 1] = (2 * T * F[k] + eT) / (2 * k - 1)
    return F


def gauss_from_recurrence(a, b, mu0):
    N = len(a)
    J = mp.matrix(N, N)
    for i in range(N):
        J[i, i] = a[i]
        if i + 1 < N:
            J[i, i + 1] = J[i + 1, i] = mp.sqrt(b[i + 1])
    E, Q = mp.eigsy(J)
    nodes = [E[i] for i in range(N)]
    wts = [mu0 * Q[0, i] ** 2 for i in range(N)]
    order = sorted(range(N), key=lambda i: nodes[i])
    return [nodes[i] for i in order], [wts[i] for i in order]


def rys_exact(N, T):
    """(u[N], w[N]) of the Rys rule at T, ascending u."""
    mu = boys_all(2 * N - 1, T)
    a = [mp.mpf(0)] * N
    b = [mp.mpf(0)] * N
    sig_prev = [mp.mpf(0)] * (2 * N)
    sig = list(mu)
    a[0] = mu[1] / mu[0]
    b[0] = mu[0]
    for k in range(1, N):
        new = [mp.mpf(0)] * (2 * N)
        for l in range(k, 2 * N - k):
            new[l] = sig[l + 1] - a[k - 1] * sig[l] - b[k - 1] * sig_prev[l]
        a[k] = new[k + 1] / new[k] - sig[k] / sig[k - 1]
        b[k] = new[k] / sig[k - 1]
        sig_prev, sig = sig, new
    return gauss_from_recurrence(a, b, mu[0])


def laguerre_half(N):
    """N-point Gauss rule for v^(-1/2) exp(-v) on [0, inf): (v_n, W_n) with sum W = sqrt(pi)."""
    a = [2 * k + mp.mpf(1) / 2 for k in range(N)]
    b = [mp.mpf(0)] + [k * (k - mp.mpf(1) / 2) for k in range(1, N)]
    return gauss_from_recurrence(a, b, mp.sqrt(mp.pi))


def asym_cutoff(N):
    v, W = laguerre_half(N)
    T = 10
    while True:
        ok = True
        for TT in (T, T + 1, T + 3, T + 7):
            u, w = rys_exact(N, TT)
            for n in range(N):
                if abs(u[n] - v[n] / TT) > ASYM_TOL * u[n]:
                    ok = False
                if abs(w[n] - W[n] / (2 * mp.sqrt(TT))) > ASYM_TOL * w[n]:
                    ok = False
        if ok:
            return T, v, W
        T += 1


def cheb_to_monomial(c):
    """Coefficients of sum_j c_j T_j(x) in powers of x (exact in mp)."""
    d = len(c) - 1
    # T_0 = 1, T_1 = x, T_{j+1} = 2x T_j - T_{j-1}
    Tp = [[mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]]
    for j in range(1, d):
        nxt = [mp.mpf(0)] * (j + 2)
        for k, v in enumerate(Tp[j]):
            nxt[k + 1] += 2 * v
        for k, v in enumerate(Tp[j - 1]):
            nxt[k] -= v
        Tp.append(nxt)
    m = [mp.mpf(0)] * (d + 1)
    for j in range(d + 1):
        for k, v in enumerate(Tp[j]):
            m[k] += c[j] * v
    return m


def horner64(m, x):
    acc = 0.0
    for v in reversed(m):
        acc = acc * x + v
    return acc


def fit_interval(args):
    """Monomial coefficients (float64) for every u_n, w_n on [i, i+1); plus error report."""
    N, i = args
    _setup()
    d = DEG
    xs = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (d + 1)) for k in range(d + 1)]
    vals = [rys_exact(N, (i + (x + 1) / 2) / SUB) for x in xs]
    coefs = []          # [n][0=u,1=w][d+1] ascending powers, float64
    for n in range(N):
        both = []
        for which in range(2):
            f = [vals[k][which][n] for k in range(d + 1)]
            c = [2 * mp.fsum(f[k] * mp.cos(j * mp.pi * (k + mp.mpf(1) / 2) / (d + 1))
                             for k in range(d + 1)) / (d + 1) for j in range(d + 1)]
            c[0] /= 2
            both.append([float(v) for v in cheb_to_monomial(c)])
        coefs.append(both)
    # check at interior points, float64 Horner against the exact rule
    worst_u = worst_w = 0.0
    for x in (-0.987, -0.55, -0.11, 0.23, 0.71, 0.995):
        u, w = rys_exact(N, (i + (mp.mpf(x) + 1) / 2) / SUB)
        for n in range(N):
            eu = abs(horner64(coefs[n][0], x) - float(u[n])) / float(u[n])
            ew = abs(horner64(coefs[n][1], x) - float(w[n])) / float(w[n])
            worst_u = max(worst_u, eu)
            worst_w = max(worst_w, ew)
    return N, i, coefs, worst_u, worst_w


def cutoff_job(N):
    _setup()
    T, v, W = asym_cutoff(N)
    return N, T, [float(x) for x in v], [float(x / 2) for x in W]


def hexd(v: float) -> str:
    return float.hex(v)


def main(out_path):
    _setup()
    with mproc.get_context("spawn").Pool(os.cpu_count()) as pool:
        cut = sorted(pool.map(cutoff_job, range(1, NMAX + 1)))
        jobs = [(N, i) for N, T, _, _ in cut for i in range(T * SUB)]
        res = pool.map(fit_interval, jobs, chunksize=4)
    res.sort(key=lambda r: (r[0], r[1]))
    tmax = {N: T for N, T, _, _ in cut}
    # layout: for N, for interval i, for root n, [u coefs (DEG+1, descending)], [w coefs]
    offsets, flat = {}, []
    for N in range(1, NMAX + 1):
        offsets[N] = len(flat)
        for (NN, i, coefs, _, _) in res:
            if NN != N:
                continue
            for n in range(N):
                flat.extend(reversed(coefs[n][0]))
                flat.extend(reversed(coefs[n][1]))
    worst = {}
    for (N, i, _, eu, ew) in res:
        wu, ww = worst.get(N, (0.0, 0.0))
        worst[N] = (max(wu, eu), max(ww, ew))
    asym_u, asym_w, asym_off = [], [], {}
    for N, T, v, W in cut:
        asym_off[N] = len(asym_u)
        asym_u.extend(v)
        asym_w.extend(W)
    def arr(decl, vals):
        body = "\n".join("  " + ", ".join(hexd(v) for v in vals[k:k + 4]) + ","
                         for k in range(0, len(vals), 4))
        return "%s[%d] = {\n%s\n};\n" % (decl, len(vals), body)

    def ints(name, table):
        return "extern \"C\" const int %s[RYS_NMAX + 1] = {0, %s};\n" % (
            name, ", ".join(str(table[N]) for N in range(1, NMAX + 1)))

    head = ["// Generated by gen_rys_table.py -- do not edit.",
            "// Rys roots u_n = t_n^2 and weights w_n (sum_n w_n = F_0(T)) for N = 1..9 on intervals",
            "// [i/%d, (i+1)/%d) of T: degree-%d polynomials in x = 2 (%d T - i) - 1, highest power first," % (SUB, SUB, DEG, SUB),
            "// laid out [N][interval][root][u coefs, w coefs].  Above RYS_TCUT[N]:",
            "// u_n = RYS_ASYM_U[n] / T, w_n = RYS_ASYM_W[n] / sqrt(T).",
            "// Worst relative error seen at interior test points (float64 Horner):"]
    for N in range(1, NMAX + 1):
        head.append("//   N=%d  T_cut=%3d  u %.2e  w %.2e" % (N, tmax[N], worst[N][0], worst[N][1]))
    text = "\n".join(head) + "\n"
    text += '#include "rys_table.h"\n\n'
    text += "static_assert(RYS_DEG == %d && RYS_SUB == %d, \"rys_table.h does not match the table\");\n\n" % (DEG, SUB)
    text += ints("RYS_TCUT", tmax) + ints("RYS_COEF_OFFSET", offsets) + ints("RYS_ASYM_OFFSET", asym_off)
    text += "extern \"C\" const int RYS_NCOEF = %d;\n\n" % len(flat)
    text += arr("extern \"C\" const double RYS_COEF", flat)
    text += arr("extern \"C\" const double RYS_ASYM_U", asym_u)
    text += arr("extern \"C\" const double RYS_ASYM_W", asym_w)
    with open(out_path, "w") as f:
        f.write(text)
    for N in range(1, NMAX + 1):
        print("N=%d T_cut=%d worst rel err u %.2e w %.2e" % (N, tmax[N], worst[N][0], worst[N][1]))
    print("coefficients:", len(flat))


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "rys_table.cpp"))
