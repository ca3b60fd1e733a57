"""Pins of the oracle's operation counter (the numerator of the benchmark's roofline
fraction): hand counts for (ss|ss) and (ps|ss), the closed forms of the transfer and
digestion counts, linearity in the number of primitive quartets, and agreement of the
per-class counts with the counter on a real quartet."""

import itertools
import math

import numpy as np
import pytest

import oracle
from workloads import custom_molecule

# the synthetic quartet of oracle_class_ops: centres (bohr) and exponents
_XYZ = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.1], [0.9, 0.0, 0.0], [0.8, 1.2, 0.3]])
_EXP = [0.9, 0.6, 0.7, 0.5]


def _ncart(l):
    return (l + 1) * (l + 2) // 2


def _cart_below(l):
    return l * (l + 1) * (l + 2) // 6


def _boys_terms(T, mmax):
    """Length of the oracle's positive series for F_mmax(T) (T < 35): terms until the last
    one drops below 1e-18 of the sum (the series of the Boys function, Sec. 2's F_m)."""
    term = 1.0 / (2 * mmax + 1)
    s = term
    k = 1
    while True:
        term *= 2.0 * T / (2 * mmax + 2 * k + 1)
        s += term
        if term < 1e-18 * s:
            return k
        k += 1


def _synthetic_T():
    a, b, c, d = _EXP
    A, B, C, D = _XYZ
    zeta, eta = a + b, c + d
    P = (a * A + b * B) / zeta
    Q = (c * C + d * D) / eta
    return zeta * eta / (zeta + eta) * float(np.sum((P - Q) ** 2))


def test_ss_ss_hand_count():
    """(ss|ss), one primitive per shell, one density: set-up 5 + 3 axes x 28 + T + 16 for
    the prefactor; Boys exp + 1 + 5 per series term + F_0 = exp(-T) * sum; one VRR value
    (Theta F_0); contraction 3 coefficient products + 1 FMA pair; no transfer; digestion of
    8 ordered quartets x (J and K: 2 operations each) x 1 value."""
    pp, pq = oracle.class_ops(0, 0, 0, 0)
    assert pp["setup"] == 5 + 3 * 28 + 1 + 16
    assert pp["boys"] == 1 + 1 + 5 * _boys_terms(_synthetic_T(), 0) + 1
    assert pp["vrr"] == 1
    assert pp["contract"] == 3 + 2
    assert pq["hrr"] == 0
    assert pq["digest"] == 8 * 4


def test_ps_ss_vrr_steps():
    """(ps|ss): L = 1, so two base values Theta F_0, Theta F_1, then three bra steps
    [1_i|0]^(0) = PA_i [0|0]^(0) + WP_i [0|0]^(1) of 3 operations each."""
    pp, pq = oracle.class_ops(1, 0, 0, 0)
    assert pp["vrr"] == 2 + 3 * 3
    assert pp["contract"] == 3 + 2 * 3
    assert pq["digest"] == 8 * 4 * 3
    # the Boys function now runs to m = 1: one downward step of 4 operations more
    assert pp["boys"] == 1 + 1 + 5 * _boys_terms(_synthetic_T(), 1) + 1 + 4


def _vrr_closed_form(Le, Lf):
    """Operations of the OS vertical recursion written out per value: the base Theta F_m, a
    bra step [e+1_i|0] of 3 operations plus 7 when e_i > 0 (the [e-1_i|0] term), a ket step
    [e|f+1_i] of 3 plus 7 when f_i > 0 plus 4 when e_i > 0, each for every m it is needed at."""
    Lt = Le + Lf
    ops = Lt + 1

    def comps(l):
        for lx in range(l, -1, -1):
            for ly in range(l - lx, -1, -1):
                yield (lx, ly, l - lx - ly)

    for le in range(1, Le + 1):
        for e in comps(le):
            i = 0 if e[0] else (1 if e[1] else 2)
            n = e[i] - 1
            ops += (Lt - le + 1) * (3 + (7 if n > 0 else 0))
    for lf in range(1, Lf + 1):
        for f in comps(lf):
            i = 0 if f[0] else (1 if f[1] else 2)
            n = f[i] - 1
            for le in range(0, Le + 1):
                for e in comps(le):
                    if Lt - le - lf >= 0:
                        ops += (Lt - le - lf + 1) * (3 + (7 if n > 0 else 0) + (4 if e[i] > 0 else 0))
    return ops


def _hrr_closed_form(la, lb, lc, ld):
    """2 operations per transferred value: bra steps over the ket's f values, ket steps over
    the bra block."""
    nf = _cart_below(lc + ld + 1) - _cart_below(lc)
    ops = 0
    for k in range(1, lb + 1):
        ops += 2 * (_cart_below(la + lb - k + 1) - _cart_below(la)) * _ncart(k) * nf
    for k in range(1, ld + 1):
        ops += 2 * (_cart_below(lc + ld - k + 1) - _cart_below(lc)) * _ncart(k) * _ncart(la) * _ncart(lb)
    return ops


@pytest.mark.parametrize("cls", [(1, 1, 0, 0), (2, 1, 1, 0), (2, 2, 2, 1), (3, 1, 2, 2), (4, 4, 4, 4)])
def test_counts_match_closed_forms(cls):
    la, lb, lc, ld = cls
    pp, pq = oracle.class_ops(la, lb, lc, ld, nD=2)
    assert pp["vrr"] == _vrr_closed_form(la + lb, lc + ld)
    ne = _cart_below(la + lb + 1) - _cart_below(la)
    nf = _cart_below(lc + ld + 1) - _cart_below(lc)
    assert pp["contract"] == 3 + 2 * ne * nf
    assert pq["hrr"] == _hrr_closed_form(la, lb, lc, ld)
    nabcd = _ncart(la) * _ncart(lb) * _ncart(lc) * _ncart(ld)
    assert pq["digest"] == 8 * 4 * 2 * nabcd


def test_linear_in_primitive_quartets():
    """A contracted quartet with K-tuple (2, 1, 3, 1) costs 6 primitive quartets plus one
    contracted quartet: exactly for every phase but Boys (whose series length follows T)."""
    rng = np.random.default_rng(3)
    coords = rng.uniform(-1.0, 1.0, (4, 3))
    shells = [(0, 2, np.array([1.2, 0.4]), np.array([0.6, 0.5])), (1, 1, np.array([0.8]), np.array([1.0])),
              (2, 1, np.array([2.0, 0.9, 0.3]), np.array([0.2, 0.5, 0.6])), (3, 0, np.array([0.5]), np.array([1.0]))]
    m = custom_molecule(coords, shells)
    got = oracle.quartet_ops(m, 0, 1, 2, 3, nD=1)
    pp, pq = oracle.class_ops(2, 1, 1, 0, nD=1)
    for k in ("setup", "vrr", "contract", "hrr", "digest"):
        assert got[k] == 6 * pp[k] + pq[k], k
    assert 0.5 * 6 * pp["boys"] < got["boys"] < 2.0 * 6 * pp["boys"]


def test_stored_class_table_is_current():
    """The table the benchmark reads equals what the counter gives now."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    import make_oracle_class_ops as mk
    with open(os.path.join(here, "oracle_class_ops.json")) as f:
        stored = json.load(f)
    assert stored["classes"] == mk.table()["classes"]
