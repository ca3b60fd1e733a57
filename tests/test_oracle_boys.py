"""Pin the oracle's Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt.

The Boys function is the Rys quadrature's moment sequence (Eq. 1, Sec. 2) and
the base case of the oracle's Obara-Saika recursion.  Reference values come
from adaptive numerical quadrature at 30 digits (mpmath.quad), which shares
nothing with the oracle's series / recursion / erf evaluation.
"""

import math

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")

TS = [0.0, 1e-10, 1e-6, 1e-3, 0.05, 0.5, 1.0, 2.7, 6.0, 11.0, 17.5, 24.0, 30.0,
      34.9, 35.0, 35.1, 42.0, 60.0, 100.0, 300.0, 1000.0]


def boys_quad(m, T):
    """Adaptive Gauss-Legendre quadrature (mpmath.quad, 40 digits), with break points
    around the integrand's peak t* = sqrt(m/T) (width ~ 1/sqrt(T)) so it is resolved."""
    mp.mp.dps = 40
    T = mp.mpf(T)
    pts = {mp.mpf(0), mp.mpf(1), mp.mpf("0.5")}
    ts = mp.sqrt(mp.mpf(m) / T) if T > 0 else mp.mpf(1)
    ts = min(ts, mp.mpf(1))
    # divide by the integrand's peak value so quad's tolerance is relative to the result
    peak = ts ** (2 * m) * mp.exp(-T * ts * ts)
    f = lambda t: t ** (2 * m) * mp.exp(-T * t * t) / peak
    if T > 1:
        sig = 1 / mp.sqrt(T)
        top = min(mp.mpf(1), ts + 16 * sig)
        for k in range(1, 33):
            pts.add(top * k / 32)
    return mp.quad(f, sorted(pts), maxdegree=10) * peak


@pytest.mark.parametrize("T", TS)
def test_boys_against_quadrature(T):
    F = oracle.boys(16, T)
    for m in range(17):
        ref = float(boys_quad(m, T))
        assert abs(F[m] - ref) <= 1e-14 * abs(ref), (m, T, F[m], ref)


def test_boys_at_zero_and_closed_form():
    F = oracle.boys(16, 0.0)
    for m in range(17):
        assert F[m] == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)
    for T in (0.3, 7.0, 40.0):
        f0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        assert oracle.boys(0, T)[0] == pytest.approx(f0, rel=1e-14)


def test_boys_recursion_identity():
    # F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T) must hold for the returned table
    for T in (0.7, 12.0, 33.0, 36.0, 80.0):
        F = oracle.boys(12, T)
        for m in range(12):
            rhs = ((2 * m + 1) * F[m] - math.exp(-T)) / (2 * T)
            assert abs(F[m + 1] - rhs) <= 1e-12 * abs(F[m + 1]) + 1e-15 * F[m], (T, m)
