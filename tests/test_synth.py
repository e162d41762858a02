"""The seeded generators: determinism, symmetry, positive overlap, water geometry, gap."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.nolsm import csr_matrix, NolsmOracle
from synth import make_config, water_box, water_clusters
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


@pytest.fixture(scope="module")
def small_globule():
    from synth import protein_globule
    return protein_globule(23, n_protein=600, n_water=300, box=34.0, radius=14.0)


def test_globule_geometry_and_blocks(small_globule):
    from scipy.spatial import cKDTree
    from synth.system import H
    s = small_globule
    n_p = 600
    chain, box = s.coords[:n_p], s.box
    centre = np.full(3, box / 2)
    assert np.linalg.norm(chain - centre, axis=1).max() <= 14.0 + 1e-9
    pairs = cKDTree(chain).query_pairs(1.2 - 1e-9, output_type="ndarray")
    assert np.all(np.abs(pairs[:, 0] - pairs[:, 1]) == 1)           # only chain neighbours that close
    o = s.coords[n_p::3]
    assert np.linalg.norm(o - centre, axis=1).min() > 14.0
    assert cKDTree(np.mod(o, box), boxsize=box).query_pairs(2.8 - 1e-9).__len__() == 0
    assert cKDTree(chain).query(o)[0].min() >= 2.5
    # blocks partition every basis function; at most 200 atoms each; waters kept whole
    assert np.array_equal(np.sort(s.blk_cols), np.arange(s.n_basis))
    atom_of = np.repeat(np.arange(s.n_atoms), np.diff(s.atom_bf_ptr))
    for b in range(s.n_blocks):
        atoms = np.unique(atom_of[s.block_cols(b)])
        assert atoms.size <= 200
        w = atoms[atoms >= n_p] - n_p
        assert np.all(np.bincount(w // 3, minlength=1)[np.unique(w // 3)] == 3)
    assert s.n_electrons == 2 * np.sum(s.element != H)


def test_globule_overlap_and_gap(small_globule):
    """Positive overlap, and a gap at N_e / 2 (2 electrons per heavy atom fill the heavy-atom s
    band; the valence count would fall inside the p band)."""
    s = small_globule
    n = s.n_basis
    h = csr_matrix(s.row_ptr, s.col, s.h, n).toarray()
    sm = csr_matrix(s.row_ptr, s.col, s.s, n).toarray()
    assert np.linalg.eigvalsh(sm)[0] >= 0.05
    w = sla.eigh(h, sm, eigvals_only=True)
    k = int(s.n_electrons // 2)
    assert w[k] - w[k - 1] >= 0.05


def test_displaced_geometry_keeps_onsite_energies_and_blocks():
    from synth import displaced
    s = water_box(4, seed=3, neighbourhood=8.0)
    d = displaced(s, 0.02, seed=5)
    assert d.n_basis == s.n_basis and np.array_equal(d.blk_cols, s.blk_cols)
    assert np.array_equal(d.extra_idx, s.extra_idx)
    move = d.coords - s.coords
    assert 0.005 < move.std() < 0.04
    hs, hd = (csr_matrix(x.row_ptr, x.col, x.h, x.n_basis).toarray() for x in (s, d))
    ss, sd = (csr_matrix(x.row_ptr, x.col, x.s, x.n_basis).toarray() for x in (s, d))
    np.testing.assert_array_equal(np.diag(hd), np.diag(hs))
    np.testing.assert_array_equal(hd, hd.T)
    np.testing.assert_array_equal(sd, sd.T)
    assert 0 < np.abs(hd - hs).max() < 0.05                  # a small step, not a new system
    assert np.linalg.eigvalsh(sd)[0] > 0.05


def test_device_generator_on_host_matches_numpy():
    """synth.device (pair search and CSR assembly in torch) against the numpy generator, torch on the
    host: same pattern, blocks and extra lists; values within the rounding of exp."""
    torch = pytest.importorskip("torch")
    from synth.device import water_clusters_device
    a = water_clusters(8, seed=31)
    b = water_clusters_device(8, seed=31, device="cpu")
    np.testing.assert_array_equal(a.row_ptr, b.row_ptr.numpy())
    np.testing.assert_array_equal(a.col, b.col.numpy())
    np.testing.assert_allclose(b.h.numpy(), a.h, rtol=0, atol=1e-15)
    np.testing.assert_allclose(b.s.numpy(), a.s, rtol=0, atol=1e-15)
    for k in ("blk_ptr", "blk_cols", "extra_ptr", "extra_idx"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert b.n_electrons == a.n_electrons and b.nnz == a.nnz
