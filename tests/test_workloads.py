"""The seeded generators produce the stated shapes, sizes and structure."""

import numpy as np

from workloads import ANGSTROM_TO_BOHR, config_high_l, config_medium, config_scf, config_tiny, \
    config_served_requests


def test_tiny_recipe():
    m = config_tiny(seed=0)
    assert m.natm == 3 and m.nshell == 9 and m.nbf == 15
    assert list(m.shell_l) == [0, 0, 1] * 3
    assert np.all(m.shell_nprim == 3)
    d = np.linalg.norm(m.coords[:, None] - m.coords[None], axis=-1) / ANGSTROM_TO_BOHR
    assert d[np.triu_indices(3, 1)].min() >= 0.9
    assert np.all(m.coords / ANGSTROM_TO_BOHR >= 0) and np.all(m.coords / ANGSTROM_TO_BOHR <= 3.0)
    # even tempered, beta = 3, smallest exponent in [0.1, 0.3]
    for s in range(m.nshell):
        e = m.exps[m.shell_off[s]:m.shell_off[s] + 3]
        np.testing.assert_allclose(e[1:] / e[:-1], 3.0)
        assert 0.1 <= e[0] <= 0.3
    D = m.D[0]
    assert D.shape == (15, 15)
    np.testing.assert_allclose(D, D.T)
    assert np.linalg.eigvalsh(D).min() > -1e-12
    assert np.linalg.matrix_rank(D) == 5


def test_medium_and_high_l_sizes():
    m = config_medium(seed=0)
    assert m.natm == 30 and m.nshell == 180 and m.nbf == 450
    assert m.shell_nprim.min() >= 1 and m.shell_nprim.max() <= 6
    assert np.linalg.matrix_rank(m.D[0]) == 60
    h = config_high_l(seed=0)
    assert h.natm == 12 and h.nshell == 60 and h.nbf == 420
    assert int(h.shell_l.max()) == 4
    assert h.shell_nprim.max() <= 3
    assert np.isclose(h.exps.min(), 0.15)


def test_determinism():
    a, b = config_medium(seed=3), config_medium(seed=3)
    np.testing.assert_array_equal(a.coords, b.coords)
    np.testing.assert_array_equal(a.exps, b.exps)
    np.testing.assert_array_equal(a.D, b.D)
    c = config_medium(seed=4)
    assert not np.array_equal(a.coords, c.coords)


def test_scf_and_served():
    m = config_scf(seed=0)
    assert m.natm == 120
    assert set(np.unique(m.charges)) <= {1.0, 6.0}
    reqs = config_served_requests(seed=0)
    assert len(reqs) == 512
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert 0.01 < np.mean(np.diff(t)) < 0.03
    assert all(5 <= r.natm <= 80 for r in reqs)
