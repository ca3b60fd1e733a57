"""Restricted Hartree-Fock driver on the GPU (the workflow around the Fock build of Sec. 3).

Per iteration: density D = 2 C_occ C_occ^T, J and K from the CUDA J/K build
(eri_jk, FP64 or mixed precision), F = H + J - K/2, E = tr(D (H + F))/2 + E_nuc,
DIIS on the commutator FDS - SDF in the orthogonalised basis, and a new
eigen-decomposition.  Densities, Fock matrices, DIIS vectors and orbitals stay on
the device; the dense linear algebra (eigh, small solves, matrix products) goes to
cuSOLVER / cuBLAS through torch.  The one-electron integrals come from the
library's host routine (the paper also computes them on the CPU, Sec. 4).

Conventions (the paper does not print PySCF's): core-Hamiltonian guess,
canonical orthogonalisation dropping overlap eigenvalues below 1e-8, DIIS with 8
vectors from the second iteration.  Optionally the first damp_cycles new densities are
damped (D <- (1 - damp) D_new + damp D_old) and DIIS starts later (PySCF's `damp` and
`diis_start_cycle`): on the 8-atom lattice molecule of the SCF recipe that start
converges where plain DIIS stalls, on the 120-atom one it diverged, so plain DIIS is the
default.  With incremental = True (PySCF's direct-SCF
scheme, on which the paper's GPU4PySCF builds) every build after the first evaluates J
and K of the density change D_n - D_{n-1} and adds them to the previous J and K; the
screening of Eqs. 7-9 then uses max|D_n - D_{n-1}|, which shrinks as the SCF converges.
"""

from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .eri import ERI_FP64, Plan, one_electron


def nuclear_repulsion(coords, charges) -> float:
    c = np.asarray(coords, dtype=np.float64)
    q = np.asarray(charges, dtype=np.float64)
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=-1)
    iu = np.triu_indices(len(q), 1)
    return float(np.sum(q[iu[0]] * q[iu[1]] / d[iu]))


@dataclass
class SCFResult:
    energy: float
    energies: List[float]
    converged: bool
    iterations: int
    jk_seconds: List[float] = field(default_factory=list)
    total_seconds: float = 0.0
    D: Optional[object] = None
    mo_energy: Optional[object] = None


class RHF:
    def __init__(self, mol, charge: Optional[int] = None, precision: int = ERI_FP64, mixed_thresh: float = 1e-4,
                 tau: Optional[float] = None, lindep: float = 1e-8, plan: Optional[Plan] = None, stream=None,
                 device: str = "cuda", incremental: bool = False, damp: float = 0.0, damp_cycles: int = 0,
                 diis_start: int = 1):
        """device: where the matrices live ("cuda"; the step-wise start / update interface also
        runs on "cpu" with J and K supplied by the caller).  incremental: build J, K of the
        density change after the first iteration (see the module docstring)."""
        import torch
        self.torch = torch
        self.mol = mol
        self.incremental = bool(incremental)
        self.damp, self.damp_cycles, self.diis_start = float(damp), int(damp_cycles), int(diis_start)
        if charge is None:
            charge = int(getattr(mol, "net_charge", 0))
        nel = int(round(float(np.sum(mol.charges)))) - charge
        if nel % 2:
            raise ValueError(f"RHF needs an even electron count, got {nel}")
        self.nocc = nel // 2
        self.plan = plan if plan is not None else Plan(mol, tau=tau, precision=precision, mixed_thresh=mixed_thresh)
        self.stream = stream
        S, T, V = one_electron(mol)
        dev = torch.device(device)
        self.S = torch.from_numpy(S).to(dev)
        self.H = torch.from_numpy(T + V).to(dev)
        self.enuc = nuclear_repulsion(mol.coords, mol.charges)
        s, U = torch.linalg.eigh(self.S)
        keep = s > lindep
        self.X = U[:, keep] / torch.sqrt(s[keep])[None, :]
        if self.nocc > self.X.shape[1]:
            raise ValueError("more occupied orbitals than independent basis functions")

    def _density(self, F):
        torch = self.torch
        Fo = self.X.T @ F @ self.X
        e, Co = torch.linalg.eigh(Fo)
        C = self.X @ Co
        Cocc = C[:, : self.nocc]
        return 2.0 * Cocc @ Cocc.T, e

    # ---- step-wise interface (used by the serving loop): start(), then update(J, K) per build
    def start(self, diis_space: int = 8, D0=None):
        """Core-Hamiltonian guess (or D0); returns the first density [nbf, nbf] on the device."""
        self.diis_space = diis_space
        self.fs, self.es, self.energies = [], [], []
        self.e_old = None
        self.converged = False
        self.cycle = 0
        self.J_acc = self.K_acc = self.D_acc = None
        if D0 is None:
            self.D, self.mo_e = self._density(self.H)
        else:
            self.D, self.mo_e = D0, None
        return self.D

    def build_density(self):
        """The density whose J and K the next update() expects: D, or with incremental builds
        (after the first) the change D - D_prev since the last build."""
        if self.incremental and self.D_acc is not None:
            return self.D - self.D_acc
        return self.D

    def update(self, J, K, conv_tol: Optional[float] = 1e-8):
        """One SCF step from J, K of build_density(): Fock matrix, energy, DIIS, new density.
        Returns (energy, converged).  The energy is read back to the host once per step (the
        convergence test); DIIS runs on the device."""
        torch = self.torch
        D = self.D
        if self.incremental and self.D_acc is not None:
            J = self.J_acc + J
            K = self.K_acc + K
        if self.incremental:
            self.J_acc, self.K_acc, self.D_acc = J, K, D
        F = self.H + J - 0.5 * K
        e_dev = 0.5 * torch.sum(D * (self.H + F))
        err = self.X.T @ (F @ D @ self.S - self.S @ D @ F) @ self.X
        self.fs.append(F)
        self.es.append(err)
        if len(self.fs) > self.diis_space:
            self.fs.pop(0)
            self.es.pop(0)
        if self.cycle >= self.diis_start and len(self.fs) >= 2:
            # B_ij = <e_i, e_j> for all stored error vectors at once; the extrapolation is skipped
            # (coefficients of the newest Fock matrix) once the error is below 1e-13
            n = len(self.fs)
            E = torch.stack([e.reshape(-1) for e in self.es])
            B = torch.full((n + 1, n + 1), -1.0, dtype=torch.float64, device=F.device)
            B[:n, :n] = E @ E.T
            B[n, n] = 0.0
            rhs = torch.zeros(n + 1, dtype=torch.float64, device=F.device)
            rhs[n] = -1.0
            sol, info = torch.linalg.solve_ex(B, rhs)
            last = torch.zeros(n, dtype=torch.float64, device=F.device)
            last[n - 1] = 1.0
            use = (err.abs().max() > 1e-13) & (info == 0) & torch.isfinite(sol).all()
            c = torch.where(use, torch.nan_to_num(sol[:n]), last)
            F = torch.einsum("i,ijk->jk", c, torch.stack(self.fs))
        D_new, self.mo_e = self._density(F)
        if self.cycle < self.damp_cycles and self.damp > 0.0:
            D_new = (1.0 - self.damp) * D_new + self.damp * D
        self.D = D_new
        self.cycle += 1
        energy = float(e_dev) + self.enuc
        self.energies.append(energy)
        if conv_tol is not None and self.e_old is not None and abs(energy - self.e_old) < conv_tol:
            self.converged = True
        self.e_old = energy
        return energy, self.converged

    def kernel(self, max_iter: int = 50, conv_tol: float = 1e-8, fixed_iters: Optional[int] = None,
               diis_space: int = 8, D0=None) -> SCFResult:
        torch = self.torch
        t0 = time.perf_counter()
        self.start(diis_space, D0)
        nbf = self.H.shape[0]
        J = torch.empty((1, nbf, nbf), dtype=torch.float64, device=self.H.device)
        K = torch.empty_like(J)
        jk_t = []
        n_iter = fixed_iters if fixed_iters is not None else max_iter
        it = 0
        for it in range(1, n_iter + 1):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            self.plan.jk(self.build_density().unsqueeze(0).contiguous(), J, K, stream=self.stream)
            ev1.record()
            _, conv = self.update(J[0].clone() if self.incremental else J[0],
                                  K[0].clone() if self.incremental else K[0],
                                  conv_tol if fixed_iters is None else None)
            jk_t.append(ev0.elapsed_time(ev1) / 1e3)
            if conv:
                break
        torch.cuda.synchronize()
        return SCFResult(energy=self.energies[-1], energies=list(self.energies), converged=self.converged,
                         iterations=it, jk_seconds=jk_t, total_seconds=time.perf_counter() - t0, D=self.D,
                         mo_energy=self.mo_e)


def main():
    """RHF of the SCF recipe (jittered lattice, 30% heavy 3s2p1d / 70% light 2s1p):
    fixed iterations in FP64 and in mixed precision; prints one JSON line."""
    import argparse
    import json

    import torch

    from workloads import config_scf
    from . import ERI_MIXED, build

    ap = argparse.ArgumentParser()
    ap.add_argument("--natm", type=int, default=120)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--mixed-thresh", type=float, default=1e-4)
    args = ap.parse_args()
    build()
    mol = config_scf(seed=args.seed, natm=args.natm)
    out = {"workload": f"RHF, {args.natm}-atom jittered 1.8 A lattice, 30% 3s2p1d (Z=6) / 70% 2s1p (Z=1), "
                       f"6-31G(d)-like depths, {mol.nbf} Cartesian functions, charge {mol.net_charge}",
           "iterations": args.iters}
    for name, prec in (("fp64", ERI_FP64), ("mixed", ERI_MIXED)):
        t0 = time.perf_counter()
        scf = RHF(mol, precision=prec, mixed_thresh=args.mixed_thresh)
        setup = time.perf_counter() - t0
        r = scf.kernel(fixed_iters=args.iters)
        st = scf.plan.stats()
        out[name] = {"energy": r.energy, "energies": r.energies, "setup_s": setup, "scf_s": r.total_seconds,
                     "jk_s_total": float(sum(r.jk_seconds)), "jk_s_per_build": float(np.mean(r.jk_seconds)),
                     "quartets_per_build": st["quartets_computed"], "fp32_quartets": st["quartets_fp32"]}
        scf.plan.close()
        torch.cuda.empty_cache()
    out["abs_dE_mixed_vs_fp64"] = abs(out["fp64"]["energy"] - out["mixed"]["energy"])
    print(json.dumps(out))


if __name__ == "__main__":
    main()
