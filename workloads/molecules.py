"""Seeded synthetic molecules, basis sets and densities.

Every generator draws from ``numpy.random.default_rng(seed)`` in a fixed order
(atom positions, then per shell: depth, smallest exponent, raw coefficients,
then the density factor), so a (config, seed) pair always gives the same arrays.

Units: the recipes below are stated in Angstrom and converted to Bohr here
(1 Angstrom = 1/0.529177210903 Bohr, CODATA 2018).  Everything returned is in
Bohr.  Exponents are even tempered, ``a * beta**k`` for ``k = 0..K-1`` inside one
shell.  Contraction coefficients are raw draws from U[0.1, 1]; normalising
them is the consumer's job.

These molecules stand in for the paper's polyglycine / RNA test set and the
(H2O)32 cc-pVTZ roofline workload (Sec. 5), whose geometries and basis files
are not available here.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.529177210903


def ncart(l: int) -> int:
    """Number of Cartesian components of a shell with angular momentum l."""
    return (l + 1) * (l + 2) // 2


@dataclasses.dataclass
class Molecule:
    name: str
    coords: np.ndarray          # (natm, 3) float64, Bohr
    charges: np.ndarray         # (natm,) float64 nuclear charges (0 where unused)
    shell_atom: np.ndarray      # (nshell,) int32
    shell_l: np.ndarray         # (nshell,) int32
    shell_nprim: np.ndarray     # (nshell,) int32
    shell_off: np.ndarray       # (nshell,) int32 offset into exps / coefs
    exps: np.ndarray            # (nprim_total,) float64
    coefs: np.ndarray           # (nprim_total,) float64, raw (un-normalised)
    D: Optional[np.ndarray] = None   # (nD, nbf, nbf) float64 symmetric PSD densities
    tau: float = 1e-12          # Schwarz / density screening threshold
    seed: int = 0
    net_charge: int = 0         # molecular charge (the SCF recipe sets +1 to make the electron count even)

    @property
    def natm(self) -> int:
        return int(self.coords.shape[0])

    @property
    def nshell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def nbf(self) -> int:
        return int(sum(ncart(int(l)) for l in self.shell_l))

    def shell_first_bf(self) -> np.ndarray:
        out = np.zeros(self.nshell, dtype=np.int64)
        acc = 0
        for i, l in enumerate(self.shell_l):
            out[i] = acc
            acc += ncart(int(l))
        return out

    def translated(self, shift_bohr: Sequence[float]) -> "Molecule":
        m = dataclasses.replace(self)
        m.coords = self.coords + np.asarray(shift_bohr, dtype=np.float64)[None, :]
        return m

    def nelectron(self, charge: Optional[int] = None) -> int:
        if charge is None:
            charge = self.net_charge
        return int(round(float(self.charges.sum()))) - charge


def _pack(name, coords_bohr, charges, shells, D=None, tau=1e-12, seed=0) -> Molecule:
    """shells: list of (atom, l, exps[K], coefs[K])."""
    shell_atom, shell_l, shell_nprim, shell_off = [], [], [], []
    exps, coefs = [], []
    for atom, l, e, c in shells:
        e = np.asarray(e, dtype=np.float64).ravel()
        c = np.asarray(c, dtype=np.float64).ravel()
        assert e.shape == c.shape and e.size >= 1
        shell_atom.append(int(atom))
        shell_l.append(int(l))
        shell_nprim.append(int(e.size))
        shell_off.append(len(exps))
        exps.extend(e.tolist())
        coefs.extend(c.tolist())
    return Molecule(
        name=name,
        coords=np.ascontiguousarray(np.asarray(coords_bohr, dtype=np.float64).reshape(-1, 3)),
        charges=np.asarray(charges, dtype=np.float64).ravel(),
        shell_atom=np.asarray(shell_atom, dtype=np.int32),
        shell_l=np.asarray(shell_l, dtype=np.int32),
        shell_nprim=np.asarray(shell_nprim, dtype=np.int32),
        shell_off=np.asarray(shell_off, dtype=np.int32),
        exps=np.asarray(exps, dtype=np.float64),
        coefs=np.asarray(coefs, dtype=np.float64),
        D=D,
        tau=tau,
        seed=seed,
    )


def custom_molecule(coords_bohr, shells, charges=None, name="custom", D=None, tau=1e-12) -> Molecule:
    """Build a Molecule from explicit shells [(atom, l, exps, coefs), ...] (Bohr)."""
    coords_bohr = np.asarray(coords_bohr, dtype=np.float64).reshape(-1, 3)
    if charges is None:
        charges = np.zeros(coords_bohr.shape[0])
    return _pack(name, coords_bohr, charges, shells, D=D, tau=tau)


# ---------------------------------------------------------------- geometry

def lattice_sites(n: int, spacing_ang: float, jitter_ang: float, rng) -> np.ndarray:
    """First n sites of the smallest m^3 cubic grid (lexicographic), plus U[-j, j] noise."""
    m = 1
    while m ** 3 < n:
        m += 1
    sites = np.array([(i, j, k) for i in range(m) for j in range(m) for k in range(m)][:n],
                     dtype=np.float64)
    coords = sites * spacing_ang + rng.uniform(-jitter_ang, jitter_ang, size=(n, 3))
    return coords * ANGSTROM_TO_BOHR


def random_box(n: int, box_ang: float, min_sep_ang: float, rng, max_tries=100000) -> np.ndarray:
    """n points uniform in a cube of side box_ang, rejection-sampled to a minimum separation."""
    pts: List[np.ndarray] = []
    tries = 0
    while len(pts) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_box: could not place atoms")
        p = rng.uniform(0.0, box_ang, size=3)
        if all(np.linalg.norm(p - q) >= min_sep_ang for q in pts):
            pts.append(p)
    return np.array(pts) * ANGSTROM_TO_BOHR


# ---------------------------------------------------------------- basis recipes

def _even_tempered_shells(atom: int, spec, beta: float, rng, a_range=None, a_fixed=None,
                          depth_choices=None, depth_fixed=None):
    """spec: list of l values for one atom.  Returns [(atom, l, exps, coefs)]."""
    out = []
    for l in spec:
        if depth_fixed is not None:
            K = int(depth_fixed)
        else:
            K = int(rng.integers(depth_choices[0], depth_choices[1] + 1))
        if a_fixed is not None:
            a = float(a_fixed)
        else:
            a = float(rng.uniform(a_range[0], a_range[1]))
        exps = a * beta ** np.arange(K, dtype=np.float64)
        coefs = rng.uniform(0.1, 1.0, size=K)
        out.append((atom, l, exps, coefs))
    return out


def random_psd_density(nbf: int, nocc: int, rng, nD: int = 1) -> np.ndarray:
    """D = C C^T with C ~ N(0,1)/sqrt(nbf), C of shape (nbf, nocc); stacked nD times."""
    Ds = []
    for _ in range(nD):
        C = rng.standard_normal((nbf, nocc)) / math.sqrt(nbf)
        Ds.append(C @ C.T)
    return np.ascontiguousarray(np.stack(Ds, axis=0))


# ---------------------------------------------------------------- the five workloads

def config_tiny(seed: int = 0, nD: int = 1) -> Molecule:
    """3 atoms in a 3 A box (min separation 0.9 A); per atom 2 s + 1 p shells of 3
    primitives, a ~ U[0.1, 0.3], beta = 3; D = C C^T with C of shape nbf x 5."""
    rng = np.random.default_rng(seed)
    coords = random_box(3, 3.0, 0.9, rng)
    shells = []
    for a in range(3):
        shells += _even_tempered_shells(a, [0, 0, 1], 3.0, rng, a_range=(0.1, 0.3), depth_fixed=3)
    m = _pack("tiny", coords, np.zeros(3), shells, tau=1e-12, seed=seed)
    m.D = random_psd_density(m.nbf, 5, rng, nD)
    return m


def config_medium(seed: int = 0, nD: int = 1, natm: int = 30) -> Molecule:
    """30 atoms on a jittered 1.8 A cubic lattice (+-0.2 A); per atom 3 s + 2 p + 1 d
    shells with depths U{1..6}, a ~ U[0.1, 0.3], beta = 2.5; D from 60 columns."""
    rng = np.random.default_rng(seed)
    coords = lattice_sites(natm, 1.8, 0.2, rng)
    shells = []
    for a in range(natm):
        shells += _even_tempered_shells(a, [0, 0, 0, 1, 1, 2], 2.5, rng, a_range=(0.1, 0.3),
                                        depth_choices=(1, 6))
    m = _pack("medium", coords, np.zeros(natm), shells, tau=1e-12, seed=seed)
    m.D = random_psd_density(m.nbf, 60, rng, nD)
    return m


def config_high_l(seed: int = 0, nD: int = 1, natm: int = 12, nocc: int = 40) -> Molecule:
    """12 atoms on the jittered 1.8 A lattice; per atom one s, p, d, f and g shell with
    depths U{1..3}, smallest exponent 0.15, beta = 2.2; D from 40 columns."""
    rng = np.random.default_rng(seed)
    coords = lattice_sites(natm, 1.8, 0.2, rng)
    shells = []
    for a in range(natm):
        shells += _even_tempered_shells(a, [0, 1, 2, 3, 4], 2.2, rng, a_fixed=0.15,
                                        depth_choices=(1, 3))
    m = _pack("high_l", coords, np.zeros(natm), shells, tau=1e-12, seed=seed)
    m.D = random_psd_density(m.nbf, min(nocc, m.nbf), rng, nD)
    return m


HEAVY_SHELLS = [0, 0, 0, 1, 1, 2]   # 3s2p1d, nuclear charge 6
LIGHT_SHELLS = [0, 0, 1]            # 2s1p,   nuclear charge 1
# contraction depths of the 6-31G(d)-like pattern: core s 6, valence s 3 + 1, p 3 + 1, d 1
HEAVY_DEPTHS = [6, 3, 1, 3, 1, 1]
LIGHT_DEPTHS = [3, 1, 1]


def config_scf(seed: int = 0, natm: int = 120, heavy_fraction: float = 0.3, depths: str = "631gd") -> Molecule:
    """Jittered 1.8 A lattice; a seeded 30% of atoms are heavy (3s2p1d, Z=6), the rest
    light (2s1p, Z=1); a ~ U[0.1, 0.3], beta = 2.5.  depths = "631gd" uses the fixed
    6-31G(d)-like contraction pattern above; depths = "random" draws U{1..6} per shell.
    The returned density is a random PSD placeholder; the SCF driver makes its own."""
    rng = np.random.default_rng(seed)
    coords = lattice_sites(natm, 1.8, 0.2, rng)
    heavy = rng.uniform(size=natm) < heavy_fraction
    shells, charges = [], np.zeros(natm)
    for a in range(natm):
        spec = HEAVY_SHELLS if heavy[a] else LIGHT_SHELLS
        charges[a] = 6.0 if heavy[a] else 1.0
        if depths == "631gd":
            dep = HEAVY_DEPTHS if heavy[a] else LIGHT_DEPTHS
            for l, K in zip(spec, dep):
                shells += _even_tempered_shells(a, [l], 2.5, rng, a_range=(0.1, 0.3), depth_fixed=K)
        else:
            shells += _even_tempered_shells(a, spec, 2.5, rng, a_range=(0.1, 0.3), depth_choices=(1, 6))
    m = _pack("scf", coords, charges, shells, tau=1e-12, seed=seed)
    if int(round(charges.sum())) % 2:
        m.net_charge = 1
    nel = m.nelectron(m.net_charge)
    nocc = (nel + (nel % 2)) // 2
    m.D = random_psd_density(m.nbf, min(nocc, m.nbf), rng, 1)
    return m


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    natm: int
    kind: str        # "jk" or "scf"
    seed: int


def config_served_requests(seed: int = 0, nreq: int = 512, mean_interarrival_s: float = 0.02,
                           natm_range=(5, 80), scf_fraction: float = 0.3) -> List[Request]:
    """512 requests, exponential inter-arrival (mean 20 ms), log-uniform atom counts on
    [5, 80], 30% full SCF and 70% single J/K builds; each carries its own molecule seed."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    lo, hi = math.log(natm_range[0]), math.log(natm_range[1])
    for i in range(nreq):
        t += float(rng.exponential(mean_interarrival_s))
        natm = int(round(math.exp(rng.uniform(lo, hi))))
        kind = "scf" if rng.uniform() < scf_fraction else "jk"
        reqs.append(Request(i, t, natm, kind, int(rng.integers(0, 2 ** 31 - 1))))
    return reqs
