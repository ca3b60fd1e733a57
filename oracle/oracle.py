"""ctypes front end of the C oracle (test infrastructure only).

Builds ``oracle/_build/liboracle.so`` with gcc (plain -O2, IEEE arithmetic,
OpenMP) on first use.  Functions take a ``workloads.Molecule``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eri_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _OBasis(ctypes.Structure):
    _fields_ = [
        ("natm", ctypes.c_int), ("coords", _dp),
        ("nshell", ctypes.c_int), ("atom", _ip), ("l", _ip), ("nprim", _ip), ("off", _ip),
        ("exps", _dp), ("coefs", _dp),
    ]


def build_oracle(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        lib.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
        lib.oracle_normalise.argtypes = [ctypes.c_int, _ip, _ip, _ip, _dp, _dp, _dp]
        lib.oracle_shell_quartet.argtypes = [ctypes.POINTER(_OBasis)] + [ctypes.c_int] * 4 + [_dp]
        lib.oracle_schwarz.argtypes = [ctypes.POINTER(_OBasis), _dp]
        lib.oracle_jk.argtypes = [ctypes.POINTER(_OBasis), ctypes.c_int, _dp, _dp, _dp,
                                  ctypes.c_double, ctypes.c_int]
        lib.oracle_jk.restype = ctypes.c_longlong
        lib.oracle_jk_blocks.argtypes = [ctypes.POINTER(_OBasis), ctypes.c_int, _dp, ctypes.c_int,
                                         _ip, _dp, _dp, ctypes.c_double, ctypes.c_int]
        lib.oracle_jk_sample.argtypes = [ctypes.POINTER(_OBasis), ctypes.c_int, _dp, _dp, _dp,
                                         ctypes.c_double, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.c_longlong]
        lib.oracle_jk_sample.restype = ctypes.c_longlong
        lib.oracle_count_quartets.argtypes = [ctypes.POINTER(_OBasis), ctypes.c_int, _dp,
                                              ctypes.c_double, ctypes.c_int]
        lib.oracle_count_quartets.restype = ctypes.c_longlong
        lib.oracle_nbf.argtypes = [ctypes.POINTER(_OBasis)]
        lib.oracle_quartet_ops.argtypes = [ctypes.POINTER(_OBasis)] + [ctypes.c_int] * 5 + [_dp]
        lib.oracle_class_ops.argtypes = [ctypes.c_int] * 5 + [_dp, _dp]
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def boys(mmax: int, T: float) -> np.ndarray:
    """F_m(T) for m = 0..mmax from the oracle's own Boys routine."""
    out = np.zeros(mmax + 1)
    _get().oracle_boys(int(mmax), float(T), _d(out))
    return out


def normalise(mol) -> np.ndarray:
    """Normalised contraction coefficients (radial primitive norm, x^l unit self-overlap)."""
    out = np.zeros_like(mol.coefs)
    l = np.ascontiguousarray(mol.shell_l, dtype=np.int32)
    n = np.ascontiguousarray(mol.shell_nprim, dtype=np.int32)
    o = np.ascontiguousarray(mol.shell_off, dtype=np.int32)
    e = np.ascontiguousarray(mol.exps, dtype=np.float64)
    c = np.ascontiguousarray(mol.coefs, dtype=np.float64)
    _get().oracle_normalise(mol.nshell, _i(l), _i(n), _i(o), _d(e), _d(c), _d(out))
    return out


class OracleBasis:
    """Keeps the contiguous arrays alive while the C side holds pointers to them."""

    def __init__(self, mol, coefs=None):
        """coefs: final contraction coefficients (skips the normalisation) or None."""
        self.coords = np.ascontiguousarray(mol.coords, dtype=np.float64)
        self.atom = np.ascontiguousarray(mol.shell_atom, dtype=np.int32)
        self.l = np.ascontiguousarray(mol.shell_l, dtype=np.int32)
        self.nprim = np.ascontiguousarray(mol.shell_nprim, dtype=np.int32)
        self.off = np.ascontiguousarray(mol.shell_off, dtype=np.int32)
        self.exps = np.ascontiguousarray(mol.exps, dtype=np.float64)
        self.coefs = np.ascontiguousarray(normalise(mol) if coefs is None else coefs, dtype=np.float64)
        self.nshell = int(self.l.shape[0])
        self.nbf = int(sum((int(x) + 1) * (int(x) + 2) // 2 for x in self.l))
        self.D = getattr(mol, "D", None)
        self.tau = getattr(mol, "tau", 1e-12)
        self.s = _OBasis(self.coords.shape[0], _d(self.coords), self.nshell, _i(self.atom),
                         _i(self.l), _i(self.nprim), _i(self.off), _d(self.exps), _d(self.coefs))

    def ptr(self):
        return ctypes.byref(self.s)


def _basis(mol):
    return mol if isinstance(mol, OracleBasis) else OracleBasis(mol)


def _ncart(l):
    return (int(l) + 1) * (int(l) + 2) // 2


def shell_quartet(mol, i: int, j: int, k: int, l: int) -> np.ndarray:
    """Contracted (ij|kl) block, shape (n_i, n_j, n_k, n_l)."""
    b = _basis(mol)
    shp = tuple(_ncart(b.l[s]) for s in (i, j, k, l))
    out = np.zeros(shp)
    _get().oracle_shell_quartet(b.ptr(), int(i), int(j), int(k), int(l), _d(out))
    return out


def schwarz(mol) -> np.ndarray:
    """Q[I, J] = sqrt(max |(ab|ab)|) over a in I, b in J (Eq. 7)."""
    b = _basis(mol)
    Q = np.zeros((b.nshell, b.nshell))
    _get().oracle_schwarz(b.ptr(), _d(Q))
    return Q


def _dens(mol, D):
    if D is None:
        D = mol.D
    D = np.ascontiguousarray(D, dtype=np.float64)
    if D.ndim == 2:
        D = D[None]
    return D


def jk(mol, D=None, tau=None, screen: bool = True):
    """(J, K, n_unique_quartets) for every density; screen=False evaluates all quartets."""
    b = _basis(mol)
    D = _dens(mol, D)
    if tau is None:
        tau = getattr(mol, "tau", 1e-12)
    nD, nbf = D.shape[0], D.shape[1]
    assert nbf == b.nbf
    J = np.zeros_like(D)
    K = np.zeros_like(D)
    n = _get().oracle_jk(b.ptr(), nD, _d(D), _d(J), _d(K), float(tau), 1 if screen else 0)
    return J, K, int(n)


def jk_blocks(mol, pairs, D=None, tau=None, screen: bool = True):
    """Sampled J blocks J[I_s, J_s] and K blocks K[I_s, K_s] for shell pairs (I_s, X_s).

    Returns two lists of arrays shaped (nD, n_I, n_X)."""
    b = _basis(mol)
    D = _dens(mol, D)
    if tau is None:
        tau = getattr(mol, "tau", 1e-12)
    nD = D.shape[0]
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    ns = pairs.shape[0]
    mb = max(_ncart(x) for x in b.l)
    Jb = np.zeros((ns, nD, mb * mb))
    Kb = np.zeros((ns, nD, mb * mb))
    _get().oracle_jk_blocks(b.ptr(), nD, _d(D), ns, _i(pairs), _d(Jb), _d(Kb), float(tau),
                            1 if screen else 0)
    Jl, Kl = [], []
    for s in range(ns):
        ni, nx = _ncart(b.l[pairs[s, 0]]), _ncart(b.l[pairs[s, 1]])
        Jl.append(Jb[s, :, : ni * nx].reshape(nD, ni, nx))
        Kl.append(Kb[s, :, : ni * nx].reshape(nD, ni, nx))
    return Jl, Kl


def jk_sample(mol, qidx, D=None, tau=None, screen: bool = True):
    """Partial J/K over the listed unique-quartet indices (u = p(p+1)/2 + q, p >= q,
    p = I(I+1)/2 + J with I >= J).  Returns (J, K, n_evaluated)."""
    b = _basis(mol)
    D = _dens(mol, D)
    if tau is None:
        tau = getattr(mol, "tau", 1e-12)
    q = np.ascontiguousarray(np.asarray(qidx, dtype=np.int64))
    J = np.zeros_like(D)
    K = np.zeros_like(D)
    n = _get().oracle_jk_sample(b.ptr(), D.shape[0], _d(D), _d(J), _d(K), float(tau), 1 if screen else 0,
                                q.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), int(q.size))
    return J, K, int(n)


def count_quartets(mol, D=None, tau=None, screen: bool = True) -> int:
    b = _basis(mol)
    D = _dens(mol, D)
    if tau is None:
        tau = getattr(mol, "tau", 1e-12)
    return int(_get().oracle_count_quartets(b.ptr(), D.shape[0], _d(D), float(tau),
                                            1 if screen else 0))


def max_threads() -> int:
    return int(_get().oracle_max_threads())


OPS_PHASES = ("setup", "boys", "vrr", "contract", "hrr", "digest")


def quartet_ops(mol, i: int, j: int, k: int, l: int, nD: int = 1) -> dict:
    """Floating-point operations the oracle performs for the unique quartet (ij|kl) (all eight
    ordered quartets of its orbit taken as distinct) and its digestion of nD densities, by
    phase (add, subtract, multiply, divide and each exp / sqrt / erf / pow count 1)."""
    b = _basis(mol)
    out = np.zeros(len(OPS_PHASES))
    _get().oracle_quartet_ops(b.ptr(), int(i), int(j), int(k), int(l), int(nD), _d(out))
    return dict(zip(OPS_PHASES, out.tolist()))


def class_ops(la: int, lb: int, lc: int, ld: int, nD: int = 1):
    """(per_prim, per_quartet) operation counts of the oracle for class (la lb|lc ld): a quartet
    with P primitive quartets costs P * sum(per_prim) + sum(per_quartet) operations."""
    pp = np.zeros(len(OPS_PHASES))
    pq = np.zeros(len(OPS_PHASES))
    _get().oracle_class_ops(int(la), int(lb), int(lc), int(ld), int(nD), _d(pp), _d(pq))
    return dict(zip(OPS_PHASES, pp.tolist())), dict(zip(OPS_PHASES, pq.tolist()))
