"""Parity of the CUDA path (through the C-ABI) with the CPU oracle, on a GB300.

Tolerances: shell-quartet blocks 1e-12 relative to the block's largest value
(or 1e-13 absolute); J and K 1e-10 absolute (the FP64 path's bar).  Rys
roots / weights are checked by the moment identity against the oracle's
pinned Boys function.
"""

import itertools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2407_09700_gb300 as pkg  # noqa: E402
from workloads import config_high_l, config_medium, config_tiny, custom_molecule, random_psd_density  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    pkg.load_library()


def _mixed_molecule(seed=0, natm=3, lmax=4, kmax=2, spread=1.6):
    rng = np.random.default_rng(seed)
    coords = rng.uniform(-spread, spread, (natm, 3))
    shells = []
    for a in range(natm):
        for l in range(lmax + 1):
            K = int(rng.integers(1, kmax + 1))
            e = np.sort(rng.uniform(0.2, 3.0, K))[::-1]
            shells.append((a, l, e, rng.uniform(0.2, 1.0, K)))
    m = custom_molecule(coords, shells)
    m.D = random_psd_density(m.nbf, max(2, m.nbf // 4), rng, nD=2)
    return m


# ---------------------------------------------------------------- Rys quadrature on the device

@pytest.mark.parametrize("N", range(1, 10))
def test_device_rys_moment_identity(N):
    Ts = np.concatenate([[0.0, 1e-9, 0.5, 1.0, 3.3, 9.99, 17.0, 29.5], np.linspace(35, 120, 9), [400.0, 5e4]])
    u, w = pkg.rys_roots(N, Ts)
    for t, T in enumerate(Ts):
        F = oracle.boys(2 * N - 1, float(T))
        assert np.all(np.diff(u[t]) > 0) and np.all(w[t] > 0)
        for k in range(2 * N):
            got = float(np.dot(w[t], u[t] ** k))
            assert abs(got - F[k]) <= 3e-14 * F[k], (N, T, k, got, F[k])


# ---------------------------------------------------------------- single shell quartets

def test_shell_quartets_every_class_up_to_g():
    m = _mixed_molecule(seed=1, natm=2, lmax=4, kmax=2)
    ob = oracle.OracleBasis(m)
    plan = pkg.Plan(m, tau=0.0)
    ns = m.nshell
    # every (la, lb, lc, ld) combination appears; include non-canonical orders too
    seen = set()
    rng = np.random.default_rng(0)
    quartets = []
    for i, j, k, l in itertools.product(range(ns), repeat=4):
        key = (int(m.shell_l[i]), int(m.shell_l[j]), int(m.shell_l[k]), int(m.shell_l[l]))
        if key not in seen:
            seen.add(key)
            quartets.append((i, j, k, l))
    assert len(seen) == 5 ** 4
    worst = 0.0
    for (i, j, k, l) in quartets:
        g = plan.shell_quartet(i, j, k, l)
        r = oracle.shell_quartet(ob, i, j, k, l)
        err = np.abs(g - r).max()
        scale = np.abs(r).max()
        worst = max(worst, err / max(scale, 1e-300))
        assert err <= 1e-12 * scale + 1e-13, ((i, j, k, l), err, scale)


def test_schwarz_factors_match_oracle():
    m = _mixed_molecule(seed=2, natm=3, lmax=3, kmax=3)
    plan = pkg.Plan(m, tau=0.0)
    np.testing.assert_allclose(plan.schwarz(), oracle.schwarz(m), rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- J / K builds

def _jk_gpu(plan, D, want=3):
    Dd = torch.from_numpy(np.ascontiguousarray(D)).cuda()
    J, K = plan.jk(Dd, want=want)
    torch.cuda.synchronize()
    return (J.cpu().numpy() if J is not None else None), (K.cpu().numpy() if K is not None else None)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_jk_tiny(seed):
    m = config_tiny(seed=seed)
    plan = pkg.Plan(m)
    J, K = _jk_gpu(plan, m.D)
    Jr, Kr, n = oracle.jk(m)
    assert np.abs(J - Jr).max() <= 1e-10
    assert np.abs(K - Kr).max() <= 1e-10
    st = plan.stats()
    assert st["quartets_computed"] == n


def test_tiny_build_splits_deep_quartets():
    """A build too small to fill the GPU runs each quartet as several ranges of its primitive
    quartets (every range digests its partial sums) and screens in the kernel without a task
    list; J and K stay those of the oracle, and every quartet is counted once."""
    m = config_tiny(seed=5)
    plan = pkg.Plan(m)
    plan.set_profiling(True)
    J, K = _jk_gpu(plan, m.D)
    recs = plan.launch_records()
    assert any(r["quartet_split"] > 1 for r in recs)
    assert all(r["listed"] == 0 for r in recs)
    Jr, Kr, n = oracle.jk(m)
    assert np.abs(J - Jr).max() <= 1e-10 and np.abs(K - Kr).max() <= 1e-10
    assert sum(r["quartets"] for r in recs) == n
    assert plan.stats()["quartets_computed"] == n


def test_jk_mixed_l_two_densities():
    m = _mixed_molecule(seed=3, natm=3, lmax=4, kmax=2)
    plan = pkg.Plan(m)
    J, K = _jk_gpu(plan, m.D)
    Jr, Kr, _ = oracle.jk(m)
    assert np.abs(J - Jr).max() <= 1e-10, np.abs(J - Jr).max()
    assert np.abs(K - Kr).max() <= 1e-10, np.abs(K - Kr).max()
    assert np.abs(J - np.transpose(J, (0, 2, 1))).max() == 0.0


def test_jk_flags_and_host_path():
    m = _mixed_molecule(seed=4, natm=2, lmax=2, kmax=3)
    plan = pkg.Plan(m)
    Jr, Kr, _ = oracle.jk(m)
    J, _ = _jk_gpu(plan, m.D, want=pkg.ERI_WANT_J)
    _, K = _jk_gpu(plan, m.D, want=pkg.ERI_WANT_K)
    assert np.abs(J - Jr).max() <= 1e-10 and np.abs(K - Kr).max() <= 1e-10
    Jh, Kh = plan.jk_host(m.D)
    assert np.abs(Jh - Jr).max() <= 1e-10 and np.abs(Kh - Kr).max() <= 1e-10


def test_jk_everything_screened():
    m = config_tiny(seed=0)
    plan = pkg.Plan(m, tau=1e6)
    J, K = _jk_gpu(plan, m.D)
    assert np.all(J == 0) and np.all(K == 0)
    assert plan.stats()["npairs_kept"] == 0


def test_jk_medium_reduced():
    # the medium recipe (3s2p1d per atom, depths 1..6) on 4 atoms: several tiles and ragged tails
    m = config_medium(seed=5, natm=4)
    plan = pkg.Plan(m)
    J, K = _jk_gpu(plan, m.D)
    Jr, Kr, _ = oracle.jk(m)
    assert np.abs(J - Jr).max() <= 1e-10, np.abs(J - Jr).max()
    assert np.abs(K - Kr).max() <= 1e-10, np.abs(K - Kr).max()


def test_jk_high_l_reduced():
    m = config_high_l(seed=6, natm=2, nocc=20)
    plan = pkg.Plan(m)
    J, K = _jk_gpu(plan, m.D)
    Jr, Kr, _ = oracle.jk(m)
    assert np.abs(J - Jr).max() <= 1e-10, np.abs(J - Jr).max()
    assert np.abs(K - Kr).max() <= 1e-10, np.abs(K - Kr).max()


# ---------------------------------------------------------------- mixed precision (FP32 recurrences)

def _pair_type(l0, l1):
    a, b = max(l0, l1), min(l0, l1)
    return a * (a + 1) // 2 + b, (a, b)


def _fp32_classes(plan, D):
    """Classes (la, lb, lc, ld) that ran an FP32 launch in a profiled build of D."""
    plan.set_profiling(True)
    plan.jk(torch.from_numpy(np.ascontiguousarray(D)).cuda())
    recs = plan.launch_records()
    plan.set_profiling(False)
    return {(r["la"], r["lb"], r["lc"], r["ld"]) for r in recs if r["fp32"]}


def _expected_split(m, Q, Qe, tau, thr, fp32_classes=None):
    """Unique shell quartets passing the screen Q_ij * Q_kl * max|D| >= tau (six cross blocks),
    split by the mixed mode's bound Qe_ij * Qe_kl * max|D| > thr (FP64) or <= thr (FP32) in
    the classes that run an FP32 launch (every quartet of the others is FP64), evaluated in
    the kernel's order of operations."""
    f0 = m.shell_first_bf()
    ns = m.nshell
    nf = [(int(l) + 1) * (int(l) + 2) // 2 for l in m.shell_l]
    Dmax = np.zeros((ns, ns))
    for i in range(ns):
        for j in range(ns):
            Dmax[i, j] = np.abs(m.D[:, f0[i]:f0[i] + nf[i], f0[j]:f0[j] + nf[j]]).max()
    pairs = [(i, j) for i in range(ns) for j in range(i + 1) if Q[i, j] > tau]
    n64 = n32 = 0
    for a in range(len(pairs)):
        P, Qs = pairs[a]
        for b in range(a + 1):
            R, S = pairs[b]
            dm = max(max(Dmax[P, Qs], Dmax[R, S]), max(max(Dmax[P, R], Dmax[P, S]), max(Dmax[Qs, R], Dmax[Qs, S])))
            if Q[P, Qs] * Q[R, S] * dm >= tau:
                tx, cx = _pair_type(int(m.shell_l[P]), int(m.shell_l[Qs]))
                ty, cy = _pair_type(int(m.shell_l[R]), int(m.shell_l[S]))
                cls = cx + cy if tx >= ty else cy + cx
                split = fp32_classes is None or cls in fp32_classes
                if split and not (Qe[P, Qs] * Qe[R, S] * dm > thr):
                    n32 += 1
                else:
                    n64 += 1
    return n64, n32


MIXED_THRESH = 1e-4      # the split of the mixed mode: FP64 above a bound of 1e-4


@pytest.mark.parametrize("make,some_fp32", [(lambda: config_medium(seed=5, natm=4), True),
                                             (lambda: _mixed_molecule(seed=3, spread=4.0), True),
                                             (lambda: config_high_l(seed=6, natm=2, nocc=20), False)])
def test_jk_mixed_precision_within_1e6(make, some_fp32):
    m = make()
    plan = pkg.Plan(m, precision=pkg.ERI_MIXED, mixed_thresh=MIXED_THRESH, mixed_min_tasks=0)
    cls32 = _fp32_classes(plan, m.D)
    J, K = _jk_gpu(plan, m.D)
    Jr, Kr, n = oracle.jk(m)
    st = plan.stats()
    n64, n32 = _expected_split(m, plan.schwarz(), plan.schwarz_transfer(), m.tau, MIXED_THRESH, cls32)
    assert st["quartets_computed"] == n64 + n32
    assert st["quartets_fp32"] == n32
    assert n32 > 0 or not some_fp32
    dj, dk = np.abs(J - Jr).max(), np.abs(K - Kr).max()
    assert dj <= 1e-6 and dk <= 1e-6, (dj, dk)


def test_transfer_aware_factor_against_oracle():
    """Qe of every shell pair: at least Q; equal to Q (FP32 rounding up) when the pair's second
    shell is s; and sqrt(max_e [e0|e0]) (1 + max_x |A-B|_x)^lb with [e0|e0] from the oracle
    (a shell of l = |e| with the first shell's exponents and normalised coefficients on A and an
    s shell with the second shell's on B) for every pair with la + lb <= 4."""
    m = _mixed_molecule(seed=9, natm=3, lmax=2, kmax=3, spread=2.5)
    plan = pkg.Plan(m, tau=0.0)
    Q, Qe = plan.schwarz(), plan.schwarz_transfer()
    c = oracle.normalise(m)
    checked = 0
    for i in range(m.nshell):
        for j in range(i + 1):
            a, b = i, j
            if m.shell_l[b] > m.shell_l[a]:
                a, b = b, a
            la, lb = int(m.shell_l[a]), int(m.shell_l[b])
            assert Qe[i, j] >= Q[i, j] * (1 - 1e-12)
            if lb == 0:
                assert Qe[i, j] <= Q[i, j] * (1 + 3e-7) + 1e-300
            if la + lb > 4:
                continue
            sa = slice(m.shell_off[a], m.shell_off[a] + m.shell_nprim[a])
            sb = slice(m.shell_off[b], m.shell_off[b] + m.shell_nprim[b])
            A, B = m.coords[m.shell_atom[a]], m.coords[m.shell_atom[b]]
            emax = 0.0
            for L in range(la, la + lb + 1):
                mb = custom_molecule(np.stack([A, B]), [(0, L, m.exps[sa], c[sa]), (1, 0, m.exps[sb], c[sb])])
                blk = oracle.shell_quartet(oracle.OracleBasis(mb, coefs=mb.coefs), 0, 1, 0, 1)
                n = blk.shape[0]
                emax = max(emax, max(abs(blk[e, 0, e, 0]) for e in range(n)))
            h = (1.0 + np.abs(A - B).max()) ** lb
            ref = np.sqrt(emax) * h
            assert abs(Qe[i, j] - ref) <= 3e-7 * ref, (i, j, Qe[i, j], ref)
            checked += 1
    assert checked > 10


def test_mixed_threshold_extremes():
    m = config_tiny(seed=1)
    Jr, Kr, n = oracle.jk(m)
    # threshold 0: every kept quartet has bound > 0, so everything runs in FP64
    p0 = pkg.Plan(m, precision=pkg.ERI_MIXED, mixed_thresh=0.0)
    J, K = _jk_gpu(p0, m.D)
    assert p0.stats()["quartets_fp32"] == 0
    assert np.abs(J - Jr).max() <= 1e-10 and np.abs(K - Kr).max() <= 1e-10
    # threshold huge: everything runs in FP32; still close to the FP64 result
    p1 = pkg.Plan(m, precision=pkg.ERI_MIXED, mixed_thresh=1e30, mixed_min_tasks=0)
    J, K = _jk_gpu(p1, m.D)
    assert p1.stats()["quartets_fp32"] == n
    assert np.abs(J - Jr).max() <= 1e-5 and np.abs(K - Kr).max() <= 1e-5


# ---------------------------------------------------------------- batched launches across jobs

def test_batch_same_alone_and_in_the_mix():
    mols = [config_tiny(seed=3), _mixed_molecule(seed=5, natm=2, lmax=3), config_medium(seed=7, natm=3),
            config_high_l(seed=8, natm=2, nocc=20)]
    precs = [pkg.ERI_FP64, pkg.ERI_MIXED, pkg.ERI_FP64, pkg.ERI_MIXED]
    plans = [pkg.Plan(m, precision=p) for m, p in zip(mols, precs)]
    Ds = [torch.from_numpy(np.ascontiguousarray(m.D)).cuda() for m in mols]
    alone = []
    for p, D in zip(plans, Ds):
        J, K = p.jk(D)
        alone.append((J.clone(), K.clone()))
    batch = pkg.Batch()
    for rep in range(2):
        Js, Ks = batch.jk(plans, Ds)
        torch.cuda.synchronize()
        for (Ja, Ka), J, K, prec in zip(alone, Js, Ks, precs):
            tol = 1e-12 if prec == pkg.ERI_FP64 else 1e-9
            sj = float(Ja.abs().max())
            assert float((J - Ja).abs().max()) <= tol * sj
            assert float((K - Ka).abs().max()) <= tol * float(Ka.abs().max())
    st = batch.stats()
    total = sum(p.stats()["quartets_computed"] for p in plans)
    assert st["quartets"] == total


_OVERRIDE_CHILD = r"""
import sys, json
import numpy as np, torch
sys.path.insert(0, ".")
import paper_2407_09700_gb300 as pkg
from workloads import custom_molecule, random_psd_density
rng = np.random.default_rng(11)
coords = rng.uniform(-1.6, 1.6, (3, 3))
shells = []
for a in range(3):
    for l in range(3):
        K = int(rng.integers(1, 4))
        shells.append((a, l, np.sort(rng.uniform(0.2, 3.0, K))[::-1], rng.uniform(0.2, 1.0, K)))
m = custom_molecule(coords, shells)
D = random_psd_density(m.nbf, 6, rng)
np.save(sys.argv[1], D)
out = {}
for name, prec in (("fp64", pkg.ERI_FP64), ("mixed", pkg.ERI_MIXED)):
    plan = pkg.Plan(m, tau=0.0, precision=prec, mixed_thresh=1e-2, mixed_min_tasks=0)
    J, K = plan.jk(torch.from_numpy(D).cuda())
    torch.cuda.synchronize()
    assert plan.stats()["device_status"] == 0
    out[name] = [J.cpu().numpy().tolist(), K.cpu().numpy().tolist()]
    plan.close()
print(json.dumps(out))
"""


@pytest.mark.parametrize("cfg", [
    # every s/p/d team class forced to 2 or 4 lanes, shared products on where allowed
    "1 1 1 1 2 1;2 0 1 1 2 1;2 0 2 0 4 1;2 1 1 0 4 1;2 1 1 1 2 1;2 1 2 0 4 1;2 1 2 1 2 1;2 2 1 0 2 1;"
    "2 2 1 1 4 1;2 2 2 0 2 1;2 2 2 1 4 1;2 2 2 2 8 1",
    # the same classes at 8 and 32 lanes with lane programs only
    "1 1 1 1 32 0;2 0 1 1 8 0;2 0 2 0 32 0;2 1 1 0 8 0;2 1 1 1 32 0;2 1 2 0 8 0;2 1 2 1 32 0;2 2 1 0 8 0;"
    "2 2 1 1 8 0;2 2 2 0 32 0;2 2 2 1 32 0;2 2 2 2 32 0",
    # (dp|dp) with its pair records staged into shared memory by bulk copies, both assembly paths
    "2 1 2 1 8 1 1", "2 1 2 1 8 0 1",
])
def test_jk_team_size_overrides(tmp_path, cfg):
    """The tuning override changes team sizes and the assembly path, never the result:
    J and K against the oracle at 1e-10 (FP64) and 1e-6 (mixed), in a child process (the
    override is read once per process)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    dpath = str(tmp_path / "D.npy")
    res = subprocess.run([sys.executable, "-c", _OVERRIDE_CHILD, dpath], cwd=root, capture_output=True, text=True,
                         env=dict(os.environ, ERI_CLASS_CONFIG=cfg), timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    rng = np.random.default_rng(11)
    coords = rng.uniform(-1.6, 1.6, (3, 3))
    shells = []
    for a in range(3):
        for l in range(3):
            K = int(rng.integers(1, 4))
            shells.append((a, l, np.sort(rng.uniform(0.2, 3.0, K))[::-1], rng.uniform(0.2, 1.0, K)))
    m = custom_molecule(coords, shells)
    D = np.load(dpath)
    Jr, Kr, _ = oracle.jk(m, D=D, screen=False)
    for name, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        J, K = (np.array(x).reshape(Jr.shape) for x in out[name])
        assert np.abs(J - Jr).max() <= tol, (name, np.abs(J - Jr).max())
        assert np.abs(K - Kr).max() <= tol, (name, np.abs(K - Kr).max())


# ---------------------------------------------------------------- full-size workloads, sampled outputs

def _sample_pairs(m, n, seed):
    """Shell pairs (I, X) for sampled J / K blocks: n random ones plus, for every pair of
    angular momenta present, one pair with those momenta."""
    rng = np.random.default_rng(seed)
    ns = m.nshell
    pairs = [(int(rng.integers(ns)), int(rng.integers(ns))) for _ in range(n)]
    seen = set()
    for i in rng.permutation(ns):
        for x in rng.permutation(ns)[:8]:
            key = (int(m.shell_l[i]), int(m.shell_l[x]))
            if key not in seen:
                seen.add(key)
                pairs.append((int(i), int(x)))
    return pairs


_FULL = {}


def _full_case(name):
    """The benchmark's workloads at full size with oracle J / K blocks on sampled shell
    pairs (computed once per module)."""
    if name not in _FULL:
        m = config_medium(seed=0) if name == "medium" else config_high_l(seed=0)
        pairs = _sample_pairs(m, 4, seed=11)
        Jl, Kl = oracle.jk_blocks(m, pairs)
        _FULL[name] = (m, pairs, Jl, Kl)
    return _FULL[name]


def _check_blocks(m, pairs, Jl, Kl, J, K, tol):
    f0 = m.shell_first_bf()
    nf = [(int(l) + 1) * (int(l) + 2) // 2 for l in m.shell_l]
    worst = 0.0
    for (i, x), Jb, Kb in zip(pairs, Jl, Kl):
        gJ = J[:, f0[i]:f0[i] + nf[i], f0[x]:f0[x] + nf[x]]
        gK = K[:, f0[i]:f0[i] + nf[i], f0[x]:f0[x] + nf[x]]
        worst = max(worst, float(np.abs(gJ - Jb).max()), float(np.abs(gK - Kb).max()))
    assert worst <= tol, worst


@pytest.mark.parametrize("name,precision,tol,min_tasks", [("medium", pkg.ERI_FP64, 1e-10, None),
                                                          ("medium", pkg.ERI_MIXED, 1e-6, None),
                                                          ("high_l", pkg.ERI_FP64, 1e-10, None),
                                                          ("high_l", pkg.ERI_MIXED, 1e-6, None),
                                                          ("high_l", pkg.ERI_MIXED, 1e-6, 0)])
def test_jk_full_size_sampled_blocks(name, precision, tol, min_tasks):
    """The 30-atom medium build the benchmark times (and the 12-atom s..g build) through
    eri_jk in its launch configuration, against oracle J / K blocks on sampled shell pairs
    covering every pair of angular momenta; the mixed builds at the split 1e-4.  The s..g
    build's classes are below the default minimum size of an FP32 launch, so it also runs
    with no minimum: every class up to (gg|gg) then has FP32 quartets."""
    m, pairs, Jl, Kl = _full_case(name)
    kw = {} if min_tasks is None else {"mixed_min_tasks": min_tasks}
    plan = pkg.Plan(m, precision=precision, mixed_thresh=MIXED_THRESH, **kw)
    J, K = _jk_gpu(plan, m.D)
    _check_blocks(m, pairs, Jl, Kl, J, K, tol)
    st = plan.stats()
    assert st["quartets_computed"] > 0
    if min_tasks == 0:
        assert st["quartets_fp32"] > 0


def test_check_symmetric_option_rejects_asymmetric_density():
    """With check_symmetric the build verifies Sec. 3's precondition (symmetric D, needed by
    the 8-fold symmetry) on the device and on the host path, and returns ERI_ERR_ARG."""
    m = config_tiny(seed=4)
    plan = pkg.Plan(m, check_symmetric=True)
    D = torch.from_numpy(m.D).cuda()
    J, K = _jk_gpu(plan, m.D)
    Jr, Kr, _ = oracle.jk(m)
    assert np.abs(J - Jr).max() <= 1e-10
    bad = m.D.copy()
    bad[0, 2, 9] += 1e-6
    with pytest.raises(pkg.EriError) as ei:
        plan.jk(torch.from_numpy(bad).cuda())
    assert ei.value.status == pkg.eri.ERI_ERR_ARG and "not symmetric" in str(ei.value)
    with pytest.raises(pkg.EriError):
        plan.jk_host(bad)
    plain = pkg.Plan(m)             # without the option an asymmetric D is not checked
    plain.jk(torch.from_numpy(bad).cuda())
    torch.cuda.synchronize()


def test_mixed_min_tasks_and_fp32_classes():
    """A class gets its FP32 launch only when its task space reaches mixed_min_tasks; a
    large mixed_min_tasks gives the FP64 result and no FP32 quartet, 0 an FP32 launch for
    every class."""
    m = _mixed_molecule(seed=3, spread=4.0)
    big = pkg.Plan(m, precision=pkg.ERI_MIXED, mixed_thresh=1e30, mixed_min_tasks=1 << 30)
    J, K = _jk_gpu(big, m.D)
    Jr, Kr, _ = oracle.jk(m)
    assert big.stats()["quartets_fp32"] == 0
    assert np.abs(J - Jr).max() <= 1e-10 and np.abs(K - Kr).max() <= 1e-10
    allp = pkg.Plan(m, precision=pkg.ERI_MIXED, mixed_thresh=1e30, mixed_min_tasks=0)
    cls32 = _fp32_classes(allp, m.D)
    assert (1, 0, 0, 0) in cls32 and (1, 1, 1, 1) in cls32 and (4, 4, 4, 4) in cls32
    J, K = _jk_gpu(allp, m.D)        # every quartet FP32, up to (gg|gg): close, not 1e-6
    assert np.abs(J - Jr).max() <= 1e-3 * np.abs(Jr).max() and np.abs(K - Kr).max() <= 1e-3 * np.abs(Kr).max()
