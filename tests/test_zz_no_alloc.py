"""eri_jk_noalloc: the J/K build for callers that cannot allocate device memory during
the call (code running under an allocator or a memory budget that owns the device's
memory, or in a host callback, where a library's cudaMalloc / cudaFree is not allowed).
It must give the same J and K as eri_jk, call after call, while the device's free memory
stays unchanged; in the mixed mode its FP32 launches (which read no task list) must also
stay within the mixed mode's 1e-6 of the oracle.

Kept in its own file, collected last, so a run that stops at the first failure has
already run every other test.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_2407_09700_gb300 as pkg  # noqa: E402
from workloads import config_high_l, config_tiny, custom_molecule, random_psd_density  # noqa: E402

TOL = 1e-10   # the FP64 J/K tolerance of the parity tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    return pkg.load_library()


def _noalloc(lib, plan, D, J, K):
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.eri_jk_noalloc(plan._h, ctypes.c_void_p(D.data_ptr()), D.shape[0], ctypes.c_void_p(J.data_ptr()),
                            ctypes.c_void_p(K.data_ptr()), 3, ctypes.c_void_p(stream))
    assert rc == 0, lib.eri_last_error().decode()


def _mixed(seed):
    rng = np.random.default_rng(seed)
    shells = []
    for a in range(3):
        for l in range(5):
            K = int(rng.integers(1, 3))
            shells.append((a, l, np.sort(rng.uniform(0.2, 3.0, K))[::-1], rng.uniform(0.2, 1.0, K)))
    m = custom_molecule(rng.uniform(-1.6, 1.6, (3, 3)), shells)
    m.D = random_psd_density(m.nbf, m.nbf // 4, rng, nD=2)
    return m


@pytest.mark.parametrize("make,precision", [(lambda: config_tiny(seed=2), pkg.ERI_FP64),
                                            (lambda: _mixed(7), pkg.ERI_FP64),
                                            (lambda: config_high_l(seed=1, natm=2, nocc=20), pkg.ERI_FP64),
                                            (lambda: _mixed(7), pkg.ERI_MIXED),
                                            (lambda: config_high_l(seed=1, natm=3, nocc=20), pkg.ERI_MIXED)])
def test_noalloc_matches_eri_jk_twice(lib, make, precision):
    m = make()
    # mixed: split 1e-2 and no minimum class size, so FP32 launches (reading no task list) run
    plan = pkg.Plan(m, precision=precision, mixed_thresh=1e-2, mixed_min_tasks=0)
    D = torch.from_numpy(m.D).cuda()
    Jref, Kref = plan.jk(D)
    torch.cuda.synchronize()
    Jref, Kref = Jref.cpu().numpy(), Kref.cpu().numpy()
    for call in range(2):
        J = torch.full_like(D, float("nan"))
        K = torch.full_like(D, float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        _noalloc(lib, plan, D, J, K)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if call == 1:
            assert free_after == free_before, "eri_jk_noalloc changed the device's free memory"
        dj = float(np.abs(J.cpu().numpy() - Jref).max())
        dk = float(np.abs(K.cpu().numpy() - Kref).max())
        assert dj <= TOL and dk <= TOL, (call, dj, dk)
    if precision == pkg.ERI_MIXED:
        st = plan.stats()
        assert st["quartets_fp32"] > 0
        Jo, Ko, _ = oracle.jk(m)
        assert float(np.abs(J.cpu().numpy() - Jo).max()) <= 1e-6
        assert float(np.abs(K.cpu().numpy() - Ko).max()) <= 1e-6
    plan.close()


def test_noalloc_argument_errors(lib):
    m = config_tiny(seed=0)
    plan = pkg.Plan(m)
    D = torch.from_numpy(m.D).cuda()
    J = torch.empty_like(D)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.eri_jk_noalloc(plan._h, ctypes.c_void_p(D.data_ptr()), 0, ctypes.c_void_p(J.data_ptr()),
                            ctypes.c_void_p(J.data_ptr()), 3, stream)
    assert rc == pkg.eri.ERI_ERR_ARG
    rc = lib.eri_jk_noalloc(plan._h, ctypes.c_void_p(D.data_ptr()), 1, ctypes.c_void_p(J.data_ptr()),
                            ctypes.c_void_p(0), 3, stream)
    assert rc == pkg.eri.ERI_ERR_ARG and b"K requested" in lib.eri_last_error()
    plan.close()
