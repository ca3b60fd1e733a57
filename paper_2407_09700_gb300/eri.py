"""Thin ctypes binding of liberi (include/eri.h): argument marshalling only.

Every step of the J/K build runs in the CUDA library; this module only passes
pointers and sizes.  If the library is missing it raises instead of falling
back to anything else.  Device buffers are torch tensors (torch provides the
device memory and the current stream).
"""

from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from .build import LIB, HERE

ERI_OK, ERI_ERR_ARG, ERI_ERR_BASIS, ERI_ERR_OOM, ERI_ERR_CUDA, ERI_ERR_NO_DEVICE, ERI_ERR_TIMEOUT, \
    ERI_ERR_UNSUPPORTED_L = range(8)
ERI_FP64, ERI_MIXED = 0, 1
ERI_WANT_J, ERI_WANT_K = 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class EriError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"liberi status {status}: {msg}")
        self.status = status


class eri_basis(ctypes.Structure):
    _fields_ = [("natm", ctypes.c_int), ("coords", _dp), ("nshell", ctypes.c_int),
                ("shell_atom", _ip), ("shell_l", _ip), ("shell_nprim", _ip), ("shell_off", _ip),
                ("exps", _dp), ("coefs", _dp), ("normalise", ctypes.c_int)]


class eri_opts(ctypes.Structure):
    _fields_ = [("screen_thresh", ctypes.c_double), ("precision", ctypes.c_int),
                ("mixed_thresh", ctypes.c_double), ("max_nd", ctypes.c_int), ("mixed_min_tasks", ctypes.c_int),
                ("check_symmetric", ctypes.c_int)]


class eri_stats(ctypes.Structure):
    _fields_ = [("quartets_candidate", ctypes.c_longlong), ("quartets_computed", ctypes.c_longlong),
                ("prim_quartets", ctypes.c_longlong), ("quartets_fp32", ctypes.c_longlong),
                ("model_flops", ctypes.c_double), ("npairs_total", ctypes.c_int),
                ("npairs_kept", ctypes.c_int), ("nclasses_launched", ctypes.c_int),
                ("model_flops_fp32", ctypes.c_double), ("device_status", ctypes.c_int)]


class eri_launch_record(ctypes.Structure):
    _fields_ = [("la", ctypes.c_int), ("lb", ctypes.c_int), ("lc", ctypes.c_int), ("ld", ctypes.c_int),
                ("team_size", ctypes.c_int), ("grid", ctypes.c_int), ("ms", ctypes.c_float),
                ("quartets", ctypes.c_longlong), ("prim_quartets", ctypes.c_longlong),
                ("model_flops", ctypes.c_double), ("model_flops_fp32", ctypes.c_double), ("fp32", ctypes.c_int),
                ("specialised", ctypes.c_int), ("shared_products", ctypes.c_int), ("compiled_class", ctypes.c_int),
                ("quartet_split", ctypes.c_int), ("listed", ctypes.c_int)]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "eri_plan_create": (ctypes.c_int, [ctypes.POINTER(eri_basis), ctypes.POINTER(eri_opts), ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "eri_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "eri_plan_nbf": (ctypes.c_int, [ctypes.c_void_p]),
    "eri_jk": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_int, ctypes.c_void_p]),
    "eri_jk_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "eri_jk_host": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_void_p]),
    "eri_jk_grad": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "eri_grad_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_longlong)]),
    "eri_shell_quartet": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 4 + [_dp]),
    "eri_check_density": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_int]),
    "eri_schwarz": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "eri_schwarz_transfer": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "eri_rys_roots": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]),
    "eri_flop_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(eri_stats)]),
    "eri_probe_fma_peak": (ctypes.c_int, [_dp, _dp]),
    "eri_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "eri_launch_records": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(eri_launch_record), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]),
    "eri_one_electron": (ctypes.c_int, [ctypes.POINTER(eri_basis), ctypes.c_int, _dp, _dp, _dp, _dp, _dp]),
    "eri_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p)]),
    "eri_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "eri_jk_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "eri_batch_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)]),
    "eri_check_class_tables": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "eri_last_error": (ctypes.c_char_p, []),
}


def header_symbols():
    """Function names declared in include/eri.h."""
    path = os.path.join(HERE, "..", "include", "eri.h")
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:eri_status|int|const char\*)\s+(eri_\w+)\s*\(", text, re.M)))


def load_library():
    """Load the in-tree liberi.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: run build() first (no fallback exists)")
        lib = ctypes.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(status):
    if status != ERI_OK:
        raise EriError(status, load_library().eri_last_error().decode())


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """An eri_plan built from a molecule-like object (coords, shell_* arrays, exps, coefs)."""

    def __init__(self, mol, tau=None, precision=ERI_FP64, mixed_thresh=1e-4, max_nd=8, normalise=True,
                 stream=None, check_symmetric=False, mixed_min_tasks=65536):
        lib = load_library()
        self._arrs = dict(
            coords=np.ascontiguousarray(mol.coords, dtype=np.float64),
            atom=np.ascontiguousarray(mol.shell_atom, dtype=np.int32),
            l=np.ascontiguousarray(mol.shell_l, dtype=np.int32),
            nprim=np.ascontiguousarray(mol.shell_nprim, dtype=np.int32),
            off=np.ascontiguousarray(mol.shell_off, dtype=np.int32),
            exps=np.ascontiguousarray(mol.exps, dtype=np.float64),
            coefs=np.ascontiguousarray(mol.coefs, dtype=np.float64),
        )
        A = self._arrs
        self.nshell = int(A["l"].shape[0])
        self.shell_l = A["l"]
        b = eri_basis(int(A["coords"].shape[0]), _d(A["coords"]), self.nshell, _i(A["atom"]), _i(A["l"]),
                      _i(A["nprim"]), _i(A["off"]), _d(A["exps"]), _d(A["coefs"]), 1 if normalise else 0)
        if tau is None:
            tau = getattr(mol, "tau", 1e-12)
        o = eri_opts(float(tau), int(precision), float(mixed_thresh), int(max_nd), int(mixed_min_tasks),
                     1 if check_symmetric else 0)
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(0) if stream is None else _stream_handle(stream)
        _check(lib.eri_plan_create(ctypes.byref(b), ctypes.byref(o), st, ctypes.byref(h)))
        self._h = h
        self.nbf = lib.eri_plan_nbf(h)
        self.max_nd = int(max_nd)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().eri_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- device path
    def jk(self, D, J=None, K=None, want=ERI_WANT_J | ERI_WANT_K, stream=None):
        """J, K for CUDA float64 tensors D [nD, nbf, nbf] (or [nbf, nbf]); asynchronous."""
        import torch
        squeeze = D.dim() == 2
        Dd = D.unsqueeze(0) if squeeze else D
        if Dd.dtype != torch.float64 or not Dd.is_cuda or not Dd.is_contiguous():
            raise ValueError("D must be a contiguous CUDA float64 tensor")
        nD = Dd.shape[0]
        if want & ERI_WANT_J and J is None:
            J = torch.empty_like(Dd)
        if want & ERI_WANT_K and K is None:
            K = torch.empty_like(Dd)
        _check(load_library().eri_jk(self._h, ctypes.c_void_p(Dd.data_ptr()), nD,
                                     ctypes.c_void_p(J.data_ptr() if J is not None else 0),
                                     ctypes.c_void_p(K.data_ptr() if K is not None else 0), want,
                                     _stream_handle(stream)))
        if squeeze:
            J = J[0] if J is not None else None
            K = K[0] if K is not None else None
        return J, K

    def jk_grad(self, D, gJ=None, gK=None, stream=None):
        """Gradients [natm, 3] of E_J = 1/2 sum (ab|cd) D_ab D_cd and E_K = -1/4 sum (ab|cd) D_ac D_bd
        with D (CUDA float64 [nbf, nbf], symmetric) held fixed; asynchronous."""
        import torch
        if D.dtype != torch.float64 or not D.is_cuda or not D.is_contiguous() or D.dim() != 2:
            raise ValueError("D must be a contiguous CUDA float64 [nbf, nbf] tensor")
        natm = int(self._arrs["coords"].shape[0])
        if gJ is None:
            gJ = torch.empty((natm, 3), dtype=torch.float64, device=D.device)
        if gK is None:
            gK = torch.empty((natm, 3), dtype=torch.float64, device=D.device)
        _check(load_library().eri_jk_grad(self._h, ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(gJ.data_ptr()),
                                          ctypes.c_void_p(gK.data_ptr()), _stream_handle(stream)))
        return gJ, gK

    def grad_stats(self):
        q, pq = ctypes.c_longlong(), ctypes.c_longlong()
        _check(load_library().eri_grad_stats(self._h, ctypes.byref(q), ctypes.byref(pq)))
        return {"quartets": q.value, "prim_quartets": pq.value}

    # -- host path (copies inside)
    def jk_host(self, D, want=ERI_WANT_J | ERI_WANT_K, stream=0):
        D = np.ascontiguousarray(D, dtype=np.float64)
        squeeze = D.ndim == 2
        if squeeze:
            D = D[None]
        J = np.zeros_like(D)
        K = np.zeros_like(D)
        st = ctypes.c_void_p(stream) if isinstance(stream, int) else _stream_handle(stream)
        _check(load_library().eri_jk_host(self._h, _d(D), D.shape[0], _d(J), _d(K), want, st))
        return (J[0], K[0]) if squeeze else (J, K)

    def shell_quartet(self, i, j, k, l):
        n = [(int(self.shell_l[s]) + 1) * (int(self.shell_l[s]) + 2) // 2 for s in (i, j, k, l)]
        out = np.zeros(n)
        _check(load_library().eri_shell_quartet(self._h, int(i), int(j), int(k), int(l), _d(out)))
        return out

    def schwarz(self):
        Q = np.zeros((self.nshell, self.nshell))
        _check(load_library().eri_schwarz(self._h, _d(Q)))
        return Q

    def schwarz_transfer(self):
        Qe = np.zeros((self.nshell, self.nshell))
        _check(load_library().eri_schwarz_transfer(self._h, _d(Qe)))
        return Qe

    def set_profiling(self, on=True):
        _check(load_library().eri_set_profiling(self._h, 1 if on else 0))

    def launch_records(self):
        """Per-launch records of the last jk call (class, team size, ms, counts, model FLOPs)."""
        arr = (eri_launch_record * 256)()
        n = ctypes.c_int()
        _check(load_library().eri_launch_records(self._h, arr, 256, ctypes.byref(n)))
        return [{k: getattr(arr[i], k) for k, _ in eri_launch_record._fields_} for i in range(n.value)]

    def stats(self):
        s = eri_stats()
        _check(load_library().eri_flop_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in eri_stats._fields_}


def check_density(D):
    """Raise EriError (ERI_ERR_ARG) unless every density of D [nD, nbf, nbf] (or [nbf, nbf],
    host array) is symmetric to 1e-12 of its largest element; needs no GPU."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    if D.ndim == 2:
        D = D[None]
    _check(load_library().eri_check_density(_d(D), int(D.shape[0]), int(D.shape[1])))


def rys_roots(N, T):
    """Device Rys roots u[len(T), N] and weights w[len(T), N]."""
    T = np.ascontiguousarray(np.atleast_1d(T), dtype=np.float64)
    u = np.zeros((T.size, N))
    w = np.zeros((T.size, N))
    _check(load_library().eri_rys_roots(int(N), int(T.size), _d(T), _d(u), _d(w)))
    return u, w


def check_class_tables():
    """(classes checked, violations) of the host self-check of the per-class tables."""
    n, bad = ctypes.c_int(), ctypes.c_int()
    _check(load_library().eri_check_class_tables(ctypes.byref(n), ctypes.byref(bad)))
    return n.value, bad.value


def probe_fma_peak():
    """(FP64, FP32) FMA throughput of the current device in TFLOP/s, measured."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load_library().eri_probe_fma_peak(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def one_electron(mol, charges=None, charge_xyz=None, normalise=True):
    """Host one-electron integrals (S, T, V) of a molecule-like object; V uses the
    molecule's nuclear charges at its atom positions unless charges are given."""
    lib = load_library()
    coords = np.ascontiguousarray(mol.coords, dtype=np.float64)
    arrs = [np.ascontiguousarray(x, dtype=np.int32) for x in (mol.shell_atom, mol.shell_l, mol.shell_nprim,
                                                             mol.shell_off)]
    exps = np.ascontiguousarray(mol.exps, dtype=np.float64)
    coefs = np.ascontiguousarray(mol.coefs, dtype=np.float64)
    b = eri_basis(coords.shape[0], _d(coords), int(arrs[1].shape[0]), _i(arrs[0]), _i(arrs[1]), _i(arrs[2]),
                  _i(arrs[3]), _d(exps), _d(coefs), 1 if normalise else 0)
    if charges is None:
        charges = mol.charges
        charge_xyz = coords
    q = np.ascontiguousarray(charges, dtype=np.float64)
    qx = np.ascontiguousarray(charge_xyz, dtype=np.float64).reshape(-1, 3)
    nbf = int(sum((int(l) + 1) * (int(l) + 2) // 2 for l in mol.shell_l))
    S = np.zeros((nbf, nbf))
    T = np.zeros((nbf, nbf))
    V = np.zeros((nbf, nbf))
    _check(lib.eri_one_electron(ctypes.byref(b), int(q.size), _d(qx), _d(q), _d(S), _d(T), _d(V)))
    return S, T, V


class Batch:
    """eri_jk_batch: one launch per class (and precision) across several jobs."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(load_library().eri_batch_create(ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().eri_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def jk(self, plans, Ds, Js=None, Ks=None, want=ERI_WANT_J | ERI_WANT_K, stream=None):
        """Ds: list of CUDA float64 tensors [nD, nbf, nbf] (one per plan).  Returns (Js, Ks)."""
        import torch
        n = len(plans)
        Ds = [D if D.dim() == 3 else D.unsqueeze(0) for D in Ds]
        if Js is None:
            Js = [torch.empty_like(D) for D in Ds]
        if Ks is None:
            Ks = [torch.empty_like(D) for D in Ds]
        P = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
        Dp = (ctypes.c_void_p * n)(*[D.data_ptr() for D in Ds])
        Jp = (ctypes.c_void_p * n)(*[J.data_ptr() for J in Js])
        Kp = (ctypes.c_void_p * n)(*[K.data_ptr() for K in Ks])
        nD = (ctypes.c_int * n)(*[D.shape[0] for D in Ds])
        fl = (ctypes.c_int * n)(*([want] * n))
        _check(load_library().eri_jk_batch(self._h, n, P, Dp, nD, Jp, Kp, fl, _stream_handle(stream)))
        return Js, Ks

    def stats(self):
        q, q32, nl = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
        _check(load_library().eri_batch_stats(self._h, ctypes.byref(q), ctypes.byref(q32), ctypes.byref(nl)))
        return {"quartets": q.value, "quartets_fp32": q32.value, "launches": nl.value}
