"""The seeded generators: determinism, symmetry, positive overlap, water geometry, gap."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.nolsm import csr_matrix, NolsmOracle
from synth import make_config, water_box
from synth.system import ANGLE_HOH, R_OH


def test_deterministic():
    a, b = water_box(3, seed=9), water_box(3, seed=9)
    for f in ("coords", "row_ptr", "col", "h", "s"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = water_box(3, seed=10)
    assert not np.array_equal(a.h, c.h)


def test_water_geometry():
    sysm = water_box(4, seed=2)
    x = sysm.coords.reshape(-1, 3, 3)
    d1 = np.linalg.norm(x[:, 1] - x[:, 0], axis=1)
    d2 = np.linalg.norm(x[:, 2] - x[:, 0], axis=1)
    np.testing.assert_allclose(d1, R_OH, atol=1e-12)
    np.testing.assert_allclose(d2, R_OH, atol=1e-12)
    cosang = np.sum((x[:, 1] - x[:, 0]) * (x[:, 2] - x[:, 0]), axis=1) / R_OH ** 2
    np.testing.assert_allclose(np.arccos(cosang), ANGLE_HOH, atol=1e-12)
    # minimum intermolecular distance (minimum image)
    a = sysm.coords
    d = a[:, None, :] - a[None, :, :]
    d -= sysm.box * np.round(d / sysm.box)
    r = np.linalg.norm(d, axis=2)
    mol = np.arange(a.shape[0]) // 3
    r[mol[:, None] == mol[None, :]] = np.inf
    assert r.min() >= 1.5


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_config1_matrices(seed):
    sysm = make_config(1, seed)
    n = sysm.n_basis
    assert n == 384 and sysm.n_atoms == 192 and sysm.n_electrons == 512
    h = csr_matrix(sysm.row_ptr, sysm.col, sysm.h, n).toarray()
    s = csr_matrix(sysm.row_ptr, sysm.col, sysm.s, n).toarray()
    np.testing.assert_array_equal(h, h.T)
    np.testing.assert_array_equal(s, s.T)
    np.testing.assert_array_equal(np.diag(s), 1.0)
    assert np.linalg.eigvalsh(s).min() >= 0.05
    e = sla.eigh(h, s, eigvals_only=True)
    assert e[256] - e[255] >= 0.02          # HOMO-LUMO gap of the whole system
    # CSR is well formed: ascending columns, full diagonal
    for r in range(0, n, 37):
        cols = sysm.col[sysm.row_ptr[r]:sysm.row_ptr[r + 1]]
        assert np.all(np.diff(cols) > 0) and r in cols


@pytest.mark.slow
def test_config2_sizes():
    sysm = make_config(2)
    assert sysm.n_basis == 24576 and sysm.n_blocks == 4096
    o = NolsmOracle.from_system(sysm)
    dims = np.array([len(o.index_set(b)) for b in range(0, 4096, 64)])
    assert 350 <= dims.min() and dims.max() <= 650
