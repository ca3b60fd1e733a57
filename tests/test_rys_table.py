"""Pin the Rys root/weight table compiled into the library (no GPU).

The N-point Rys rule must reproduce the moments of its weight (Eq. 1, Sec. 2):
sum_n w_n u_n^k = F_k(T) for k = 0..2N-1, with u_n = t_n^2 in (0, 1) ascending
and w_n > 0.  The table is read from its generated C++ source and evaluated
here in float64 Horner arithmetic (the device evaluates the same polynomials);
the reference F_k(T) comes from mpmath's regularised incomplete gamma
function, F_k(T) = gamma(k + 1/2, T) / (2 T^(k + 1/2)), not from the
generator's series.
"""

import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2407_09700_gb300", "csrc", "rys_table.cpp")
HDR = os.path.join(os.path.dirname(SRC), "rys_table.h")
DEG = int(re.search(r"#define RYS_DEG (\d+)", open(HDR).read()).group(1))
SUB = int(re.search(r"#define RYS_SUB (\d+)", open(HDR).read()).group(1))


def _arr(text, name, conv):
    m = re.search(name + r"\[[^\]]*\]\s*=\s*\{([^}]*)\}", text)
    assert m, name
    return [conv(x) for x in m.group(1).replace("\n", " ").split(",") if x.strip()]


@pytest.fixture(scope="module")
def table():
    text = open(SRC).read()
    return {
        "tcut": _arr(text, "RYS_TCUT", int),
        "off": _arr(text, "RYS_COEF_OFFSET", int),
        "aoff": _arr(text, "RYS_ASYM_OFFSET", int),
        "coef": np.array(_arr(text, "RYS_COEF", float.fromhex)),
        "au": np.array(_arr(text, "RYS_ASYM_U", float.fromhex)),
        "aw": np.array(_arr(text, "RYS_ASYM_W", float.fromhex)),
    }


def rys_eval(tab, N, T):
    if T >= tab["tcut"][N]:
        a = tab["aoff"][N]
        return tab["au"][a:a + N] / T, tab["aw"][a:a + N] / np.sqrt(T)
    i = int(SUB * T)
    x = 2.0 * (SUB * T - i) - 1.0
    base = tab["off"][N] + i * N * 2 * (DEG + 1)
    u, w = np.zeros(N), np.zeros(N)
    for r in range(N):
        cu = tab["coef"][base + r * 2 * (DEG + 1): base + r * 2 * (DEG + 1) + DEG + 1]
        cw = tab["coef"][base + r * 2 * (DEG + 1) + DEG + 1: base + (r + 1) * 2 * (DEG + 1)]
        au = aw = 0.0
        for k in range(DEG + 1):
            au = au * x + cu[k]
            aw = aw * x + cw[k]
        u[r], w[r] = au, aw
    return u, w


def boys_ref(k, T):
    mp.mp.dps = 40
    if T == 0:
        return mp.mpf(1) / (2 * k + 1)
    T = mp.mpf(T)
    return mp.gammainc(k + mp.mpf(1) / 2, 0, T) / (2 * T ** (k + mp.mpf(1) / 2))


def _grid(tcut):
    ts = [0.0, 1e-12, 1e-7, 0.3, 0.999999, 1.0, 2.5, 7.3, 13.0, 19.9999, 26.5, 33.1]
    ts += [tcut - 1.5, tcut - 1e-9, float(tcut), tcut + 0.5, tcut * 1.7, 500.0, 3e4]
    return [t for t in ts if t >= 0]


@pytest.mark.parametrize("N", range(1, 10))
def test_moment_identity(table, N):
    for T in _grid(table["tcut"][N]):
        u, w = rys_eval(table, N, T)
        assert np.all(np.diff(u) > 0) and u[0] > 0 and u[-1] < 1, (N, T, u)
        assert np.all(w > 0), (N, T, w)
        for k in range(2 * N):
            ref = float(boys_ref(k, T))
            got = float(np.dot(w, u ** k))
            assert abs(got - ref) <= 2e-14 * ref, (N, T, k, got, ref, (got - ref) / ref)


def test_table_layout(table):
    # contiguous blocks: interval count of N is SUB times its cutoff, no gaps between N
    for N in range(1, 9):
        assert table["off"][N + 1] - table["off"][N] == SUB * table["tcut"][N] * N * 2 * (DEG + 1)
    assert len(table["coef"]) == table["off"][9] + SUB * table["tcut"][9] * 9 * 2 * (DEG + 1)
    assert len(table["au"]) == sum(range(1, 10))
