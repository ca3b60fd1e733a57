"""Plain RHF in numpy on top of the oracle's J/K and quadrature one-electron
integrals (test infrastructure only).

Textbook closed-shell SCF: D = 2 C_occ C_occ^T, F = H + J - K/2,
E = tr(D (H + F))/2 + E_nuc, core-Hamiltonian guess, canonical orthogonalisation
(overlap eigenvalues below 1e-8 dropped), DIIS on FDS - SDF with 8 vectors.  Optional
damping of the first new densities (D <- (1 - damp) D_new + damp D_old for damp_cycles
iterations) and DIIS from iteration diis_start on (PySCF's damp / diis_start_cycle);
the defaults (0, 0, 1) are plain DIIS from the second iteration.
"""

from __future__ import annotations

import numpy as np

from . import oracle as _orc
from .onee import nuclear_repulsion, one_electron


def rhf(mol, charge=0, max_iter=50, conv_tol=1e-10, fixed_iters=None, diis_space=8, onee=None, jk=None,
        damp=0.0, damp_cycles=0, diis_start=1):
    S, T, V = onee if onee is not None else one_electron(mol)
    H = T + V
    enuc = nuclear_repulsion(mol.coords, mol.charges)
    nel = int(round(float(np.sum(mol.charges)))) - charge
    nocc = nel // 2
    s, U = np.linalg.eigh(S)
    keep = s > 1e-8
    X = U[:, keep] / np.sqrt(s[keep])
    basis = _orc.OracleBasis(mol)

    def density(F):
        e, Co = np.linalg.eigh(X.T @ F @ X)
        C = X @ Co
        return 2.0 * C[:, :nocc] @ C[:, :nocc].T

    def jk_of(D):
        if jk is not None:
            return jk(D)
        J, K, _ = _orc.jk(basis, D=D[None], tau=getattr(mol, "tau", 1e-12), screen=True)
        return J[0], K[0]

    D = density(H)
    fs, es, energies = [], [], []
    e_old = None
    converged = False
    n_iter = fixed_iters if fixed_iters is not None else max_iter
    for it in range(1, n_iter + 1):
        J, K = jk_of(D)
        F = H + J - 0.5 * K
        E = 0.5 * np.sum(D * (H + F)) + enuc
        energies.append(float(E))
        err = X.T @ (F @ D @ S - S @ D @ F) @ X
        fs.append(F)
        es.append(err)
        if len(fs) > diis_space:
            fs.pop(0)
            es.pop(0)
        if it - 1 >= diis_start and len(fs) >= 2 and np.abs(err).max() > 1e-13:
            n = len(fs)
            B = -np.ones((n + 1, n + 1))
            B[n, n] = 0.0
            for i in range(n):
                for j in range(n):
                    B[i, j] = np.sum(es[i] * es[j])
            rhs = np.zeros(n + 1)
            rhs[n] = -1.0
            c = np.linalg.solve(B, rhs)
            F = sum(c[i] * fs[i] for i in range(n))
        D_new = density(F)
        D = (1.0 - damp) * D_new + damp * D if it - 1 < damp_cycles else D_new
        if fixed_iters is None and e_old is not None and abs(E - e_old) < conv_tol:
            converged = True
            break
        e_old = E
    return energies[-1], energies, converged
