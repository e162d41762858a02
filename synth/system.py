"""Seeded model systems: geometry, basis, sparse H0 / S in CSR, column blocks.

Units are Angstrom and Hartree.  The model Hamiltonian is a made-up tight-binding
form (exponential hopping and overlap times Slater-Koster direction cosines with a
hard atom-atom cutoff); its parameters are invented for these benchmarks and are
stated where they are defined.  Every random draw comes from one PCG64 stream per
system, in a fixed order, so a (config, seed) pair always gives the same arrays.
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np
from scipy.spatial import cKDTree

# element codes
O, H, C, N, S = 0, 1, 2, 3, 4
ELEMENT_NAMES = ("O", "H", "C", "N", "S")

# orbital kinds per element: ('s'|'p'|'d', axis) ; d orbitals couple like s times 0.5
_ORBITALS = {
    O: [("s", -1), ("p", 0), ("p", 1), ("p", 2)],
    H: [("s", -1)],
    C: [("s", -1), ("p", 0), ("p", 1), ("p", 2)],
    N: [("s", -1), ("p", 0), ("p", 1), ("p", 2)],
    S: [("s", -1), ("p", 0), ("p", 1), ("p", 2)] + [("d", -1)] * 5,
}
# on-site energies (Ha).  O and H as given for the water model; C, N, S invented.
_ONSITE = {
    O: {"s": -1.0, "p": -0.5},
    H: {"s": -0.4},
    C: {"s": -0.75, "p": -0.40},
    N: {"s": -0.90, "p": -0.45},
    S: {"s": -0.80, "p": -0.40, "d": -0.10},
}
# valence electrons per neutral atom (minimal-basis counting)
_VALENCE = {O: 6, H: 1, C: 4, N: 5, S: 6}

# h_ij = -0.3 exp(-r/1.0 A) * SK.  The water model as first stated decays over 1.5 A, which
# leaves a HOMO-LUMO gap of only 0.003-0.004 Ha in the 64-molecule box (a near-metal, where
# the zero-temperature sign function is ill-conditioned); 1.0 A opens it to ~0.04 Ha with the
# overlap unchanged (lambda_min(S) ~ 0.55).
H_PREF, H_DECAY = -0.3, 1.0
S_PREF, S_DECAY = 0.5, 1.2       # s_ij =  0.5 exp(-r/1.2 A) * SK
CUTOFF = 6.0                     # hard atom-atom cutoff (A)
ONSITE_NOISE = 0.01              # N(0, 0.01) Ha on every on-site energy

R_OH, ANGLE_HOH = 0.96, np.deg2rad(104.5)
LATTICE_SPACING = 3.1            # water lattice spacing (A): 12.4 A box for 4^3
JITTER = 0.25                    # uniform +-0.25 A per axis on O
MIN_INTER = 1.5                  # minimum intermolecular atom-atom distance (A)


@dataclass
class System:
    """A periodic model system with its sparse matrices and column blocks.

    row_ptr/col describe one CSR pattern shared by H and S (diagonal plus every
    basis pair of two different atoms closer than the cutoff).  Blocks are the
    column sets C_b (blk_ptr/blk_cols).  extra_ptr/extra_idx optionally list, per
    block, basis functions of geometric neighbours (the neighbourhood rule's
    geometric part); None when a config uses the plain pattern rule.
    """

    name: str
    box: float
    coords: np.ndarray
    element: np.ndarray
    atom_bf_ptr: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    h: np.ndarray
    s: np.ndarray
    n_electrons: float
    blk_ptr: np.ndarray
    blk_cols: np.ndarray
    extra_ptr: np.ndarray | None = None
    extra_idx: np.ndarray | None = None

    @property
    def n_atoms(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_basis(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def n_blocks(self) -> int:
        return int(self.blk_ptr.shape[0] - 1)

    def block_cols(self, b: int) -> np.ndarray:
        return self.blk_cols[self.blk_ptr[b]:self.blk_ptr[b + 1]]

    def block_extra(self, b: int) -> np.ndarray | None:
        if self.extra_ptr is None:
            return None
        return self.extra_idx[self.extra_ptr[b]:self.extra_ptr[b + 1]]

    def subset_blocks(self, blocks) -> "System":
        """Same matrices, only the listed blocks (a bounded sample of the work)."""
        blocks = np.asarray(blocks, dtype=np.int64)
        cols = [self.block_cols(int(b)) for b in blocks]
        ptr = np.zeros(len(blocks) + 1, np.int32)
        ptr[1:] = np.cumsum([len(c) for c in cols])
        ep = ei = None
        if self.extra_ptr is not None:
            ex = [self.block_extra(int(b)) for b in blocks]
            ep = np.zeros(len(blocks) + 1, np.int32)
            ep[1:] = np.cumsum([len(e) for e in ex])
            ei = np.concatenate(ex).astype(np.int32) if ex else np.zeros(0, np.int32)
        return System(self.name + f"[{len(blocks)} blocks]", self.box, self.coords, self.element,
                      self.atom_bf_ptr, self.row_ptr, self.col, self.h, self.s, self.n_electrons,
                      ptr, np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32),
                      ep, ei)


# --------------------------------------------------------------------------- geometry

def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from uniform unit quaternions (Shoemake 1992)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    q = np.stack([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
                  np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3),
                  np.sqrt(u1) * np.cos(2 * np.pi * u3)], axis=1)
    x, y, z, w = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _water_frame() -> np.ndarray:
    """H positions relative to O in the molecular frame (O at the origin)."""
    half = ANGLE_HOH / 2
    return np.array([[R_OH * np.sin(half), 0.0, R_OH * np.cos(half)],
                     [-R_OH * np.sin(half), 0.0, R_OH * np.cos(half)]])


def _place_waters(rng: np.random.Generator, o_pos: np.ndarray, box: float) -> np.ndarray:
    """Atoms (O,H,H per molecule) with random orientations; redraw clashing ones.

    An orientation is redrawn while any atom of the molecule is closer than 1.5 A
    to an atom of another molecule (the higher-indexed molecule of a clashing pair
    is redrawn, in rounds, until no clash is left).
    """
    n = o_pos.shape[0]
    frame = _water_frame()
    rot = _random_rotations(rng, n)
    for _ in range(10000):
        hpos = o_pos[:, None, :] + np.einsum("nij,kj->nki", rot, frame)
        atoms = np.concatenate([o_pos[:, None, :], hpos], axis=1).reshape(-1, 3)
        wrapped = np.mod(atoms, box)
        tree = cKDTree(wrapped, boxsize=box)
        pairs = tree.query_pairs(MIN_INTER, output_type="ndarray")
        if pairs.size:
            inter = (pairs[:, 0] // 3) != (pairs[:, 1] // 3)
            pairs = pairs[inter]
        if pairs.size == 0:
            return atoms
        bad = np.unique(np.maximum(pairs[:, 0] // 3, pairs[:, 1] // 3))
        rot[bad] = _random_rotations(rng, bad.size)
    raise RuntimeError("water placement did not converge")


# --------------------------------------------------------------------------- matrices

def _basis_layout(element: np.ndarray):
    nbf = np.array([len(_ORBITALS[int(e)]) for e in element], dtype=np.int64)
    ptr = np.zeros(element.size + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(nbf)
    return ptr


def _pair_factor(orb_a, orb_b, l):
    """Slater-Koster direction-cosine factor for orbital pair (a on atom A, b on atom B).

    l is the unit vector from A to B.  ss = 1; s_A p_B(beta) = l_beta;
    p_A(alpha) s_B = -l_alpha; p_A(alpha) p_B(beta) = l_alpha l_beta (sigma only);
    a d orbital couples like an s orbital times 0.5.
    """
    ka, aa = orb_a
    kb, ab = orb_b
    wa = 0.5 if ka == "d" else 1.0
    wb = 0.5 if kb == "d" else 1.0
    if ka != "p" and kb != "p":
        return np.full(l.shape[0], wa * wb)
    if ka != "p" and kb == "p":
        return wa * l[:, ab]
    if ka == "p" and kb != "p":
        return -l[:, aa] * wb
    return l[:, aa] * l[:, ab]


def build_matrices(coords: np.ndarray, element: np.ndarray, box: float, rng: np.random.Generator,
                   cutoff: float = CUTOFF):
    """CSR H0 and S on the shared pattern of atom pairs closer than the cutoff."""
    bf_ptr = _basis_layout(element)
    nbasis = int(bf_ptr[-1])
    wrapped = np.mod(coords, box)
    tree = cKDTree(wrapped, boxsize=box)
    pairs = tree.query_pairs(cutoff, output_type="ndarray")
    rows, cols, hv, sv = [], [], [], []
    if pairs.size:
        a, b = pairs[:, 0], pairs[:, 1]
        d = coords[b] - coords[a]
        d -= box * np.round(d / box)
        r = np.linalg.norm(d, axis=1)
        l = d / r[:, None]
        gh = H_PREF * np.exp(-r / H_DECAY)
        gs = S_PREF * np.exp(-r / S_DECAY)
        ea, eb = element[a], element[b]
        for ela in np.unique(ea):
            for elb in np.unique(eb):
                m = (ea == ela) & (eb == elb)
                if not m.any():
                    continue
                oa, ob = _ORBITALS[int(ela)], _ORBITALS[int(elb)]
                for i, orb_a in enumerate(oa):
                    for j, orb_b in enumerate(ob):
                        f = _pair_factor(orb_a, orb_b, l[m])
                        ri = bf_ptr[a[m]] + i
                        cj = bf_ptr[b[m]] + j
                        # both triangles: H and S are symmetric
                        rows += [ri, cj]
                        cols += [cj, ri]
                        hv += [gh[m] * f, gh[m] * f]
                        sv += [gs[m] * f, gs[m] * f]
    # on-site diagonal; off-diagonal on-site elements are zero and not stored
    onsite = np.empty(nbasis)
    for at in range(element.size):
        e = int(element[at])
        for k, (kind, _) in enumerate(_ORBITALS[e]):
            onsite[bf_ptr[at] + k] = _ONSITE[e][kind]
    onsite += rng.normal(0.0, ONSITE_NOISE, size=nbasis)
    diag = np.arange(nbasis, dtype=np.int64)
    rows.append(diag)
    cols.append(diag)
    hv.append(onsite)
    sv.append(np.ones(nbasis))
    rows = np.concatenate(rows).astype(np.int64)
    cols = np.concatenate(cols).astype(np.int64)
    hv = np.concatenate(hv)
    sv = np.concatenate(sv)
    order = np.lexsort((cols, rows))
    rows, cols, hv, sv = rows[order], cols[order], hv[order], sv[order]
    row_ptr = np.zeros(nbasis + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return bf_ptr, row_ptr, cols.astype(np.int32), hv, sv


# --------------------------------------------------------------------------- systems

def _lattice(m: int, spacing: float) -> np.ndarray:
    g = np.arange(m) * spacing + spacing / 2
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def _molecule_blocks(n_mol: int):
    ptr = (np.arange(n_mol + 1) * 6).astype(np.int32)
    return ptr, np.arange(6 * n_mol, dtype=np.int32)


def _neighbour_lists(centres: np.ndarray, box: float, radius: float, member_bf):
    """Per block, the basis functions of every molecule whose O lies within radius."""
    tree = cKDTree(np.mod(centres, box), boxsize=box)
    nbrs = tree.query_ball_point(np.mod(centres, box), r=radius)
    ptr = np.zeros(len(nbrs) + 1, dtype=np.int32)
    lists = []
    for i, nb in enumerate(nbrs):
        idx = np.sort(np.concatenate([member_bf(k) for k in nb]))
        lists.append(idx)
        ptr[i + 1] = ptr[i] + idx.size
    return ptr, np.concatenate(lists).astype(np.int32)


def water_box(n_side: int, seed: int, spacing: float = LATTICE_SPACING,
              neighbourhood: float | None = None, name: str | None = None) -> System:
    """n_side^3 water molecules on a jittered cubic lattice in a periodic box.

    One block per molecule (its 6 basis functions O 2s,2p, H 1s, H 1s).  With
    neighbourhood=r the geometric neighbour list holds every molecule whose O is
    within r (minimum image) of the block's O.  N_e = 8 per molecule.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    box = n_side * spacing
    o_pos = _lattice(n_side, spacing) + rng.uniform(-JITTER, JITTER, size=(n_side ** 3, 3))
    coords = _place_waters(rng, o_pos, box)
    n_mol = n_side ** 3
    element = np.tile(np.array([O, H, H]), n_mol)
    bf_ptr, row_ptr, col, h, s = build_matrices(coords, element, box, rng)
    blk_ptr, blk_cols = _molecule_blocks(n_mol)
    ep = ei = None
    if neighbourhood is not None:
        ep, ei = _neighbour_lists(o_pos, box, neighbourhood, lambda k: np.arange(6 * k, 6 * k + 6))
    return System(name or f"water{n_mol}", box, coords, element, bf_ptr, row_ptr, col, h, s,
                  8.0 * n_mol, blk_ptr, blk_cols, ep, ei)


def water_clusters(n_side: int, seed: int, cluster=(2, 4, 4), halo: float = 8.0,
                   spacing: float = LATTICE_SPACING, name: str | None = None) -> System:
    """The water box of `water_box` (same seed, same molecules) cut into column blocks of
    cluster[0] x cluster[1] x cluster[2] neighbouring lattice sites (32 molecules by default).

    A block's own columns are the basis functions of its molecules; its geometric list holds every
    molecule whose O lies within `halo` (minimum image) of any own O.  n_side must be a multiple of
    every cluster edge.
    """
    cx, cy, cz = cluster
    if n_side % cx or n_side % cy or n_side % cz:
        raise ValueError("n_side must be a multiple of every cluster edge")
    base = water_box(n_side, seed, spacing=spacing)
    o_pos = base.coords[0::3]
    box = base.box
    i, j, k = np.meshgrid(np.arange(n_side), np.arange(n_side), np.arange(n_side), indexing="ij")
    cid = ((i // cx) * (n_side // cy) + j // cy) * (n_side // cz) + k // cz
    members = np.argsort(cid.ravel(), kind="stable").reshape(-1, cx * cy * cz)
    n_blk = members.shape[0]
    blk_ptr = (np.arange(n_blk + 1) * 6 * cx * cy * cz).astype(np.int32)
    blk_cols = (6 * members[:, :, None] + np.arange(6)[None, None, :]).reshape(-1).astype(np.int32)
    tree = cKDTree(np.mod(o_pos, box), boxsize=box)
    ep = np.zeros(n_blk + 1, dtype=np.int32)
    lists = []
    for b in range(n_blk):
        near = tree.query_ball_point(np.mod(o_pos[members[b]], box), r=halo)
        mol = np.unique(np.concatenate([np.asarray(v, dtype=np.int64) for v in near]))
        idx = (6 * mol[:, None] + np.arange(6)[None, :]).reshape(-1)
        lists.append(idx)
        ep[b + 1] = ep[b] + idx.size
    return System(name or f"waterclusters{n_side ** 3}", box, base.coords, base.element, base.atom_bf_ptr,
                  base.row_ptr, base.col, base.h, base.s, base.n_electrons, blk_ptr, blk_cols, ep,
                  np.concatenate(lists).astype(np.int32))


def isolated_waters(n_mol: int, seed: int, spacing: float = 10.0) -> System:
    """Waters farther apart than the cutoff: H0 and S are block diagonal."""
    m = int(round(n_mol ** (1 / 3)))
    assert m ** 3 == n_mol
    return water_box(m, seed, spacing=spacing, name=f"isolated{n_mol}")


def dimer_system(a: float, b: float, s: float) -> System:
    """Two basis functions: H0 = [[a,b],[b,a]], S = [[1,s],[s,1]], one block per column."""
    row_ptr = np.array([0, 2, 4], dtype=np.int64)
    col = np.array([0, 1, 0, 1], dtype=np.int32)
    h = np.array([a, b, b, a], dtype=np.float64)
    sv = np.array([1.0, s, s, 1.0], dtype=np.float64)
    coords = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    return System("dimer", 100.0, coords, np.array([H, H]), np.array([0, 1, 2]), row_ptr, col, h, sv,
                  2.0, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32))


def dense_blocks(n: int, n_blocks: int, seed: int, noise: float = 0.1, n_unique: int | None = None) -> System:
    """n_blocks uncoupled dense blocks of dimension n (block-diagonal H0 and S, one column block
    per dense block, so every index set has exactly n entries): for timing the matrix products at
    a chosen n.

    S_k = I + E_k and H0_k = diag(d_k) + F_k, with E_k and F_k symmetric, entries N(0, (noise /
    sqrt(n))^2) (spectral norm about 2 * noise), and d_k = -1 or +0.5 Ha with equal probability, so
    the generalized spectrum lies in two clusters around -1 and +0.5 with a gap around -0.25 Ha.
    N_e counts the states below the gap twice.  With n_unique set, only that many blocks are
    drawn and block k repeats block k % n_unique (cheap large batches for timing).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sd = noise / np.sqrt(n)
    hv = np.empty((n_blocks, n, n))
    sv = np.empty((n_blocks, n, n))
    occ = 0
    n_unique = n_blocks if n_unique is None else max(1, min(n_unique, n_blocks))
    for k in range(n_blocks):
        if k >= n_unique:
            hv[k], sv[k] = hv[k % n_unique], sv[k % n_unique]
            occ += int((np.diag(hv[k]) < -0.25).sum())
            continue
        e = rng.normal(0.0, sd, size=(n, n))
        f = rng.normal(0.0, sd, size=(n, n))
        d = np.where(rng.random(n) < 0.5, -1.0, 0.5)
        occ += int((d < 0).sum())
        sv[k] = np.triu(e, 1) + np.triu(e, 1).T + np.eye(n)
        hv[k] = np.triu(f) + np.triu(f, 1).T + np.diag(d)
    nb = n * n_blocks
    row_ptr = (np.arange(nb + 1, dtype=np.int64) * n)
    col = ((np.arange(nb)[:, None] // n) * n + np.arange(n)[None, :]).reshape(-1).astype(np.int32)
    blk_ptr = (np.arange(n_blocks + 1) * n).astype(np.int32)
    coords = np.zeros((nb, 3))
    return System(f"dense{n}x{n_blocks}", 0.0, coords, np.full(nb, H), np.arange(nb + 1), row_ptr, col,
                  hv.reshape(-1), sv.reshape(-1), 2.0 * occ, blk_ptr, np.arange(nb, dtype=np.int32))


# --------------------------------------------------------------------------- named configs

CONFIGS = {
    1: dict(desc="64 waters, 12.4 A box, pattern rule, 1 block/molecule", seeds=(1, 2, 3, 4, 5)),
    2: dict(desc="4,096 waters, 49.6 A box, 8 A neighbourhood, 1 block/molecule", seeds=(11, 12, 13)),
    5: dict(desc="water, 32-molecule clusters with an 8 A halo (the 1,000,000-molecule system's block "
                 "shape), 13,824 molecules", seeds=(31,)),
}


def make_config(config: int, seed: int | None = None) -> System:
    """Named benchmark systems (seeded)."""
    if seed is None:
        seed = CONFIGS[config]["seeds"][0]
    if config == 1:
        return water_box(4, seed, name=f"water64-s{seed}")
    if config == 2:
        return water_box(16, seed, neighbourhood=8.0, name=f"water4096-s{seed}")
    if config == 5:
        return water_clusters(24, seed, name=f"waterclusters13824-s{seed}")
    raise ValueError(f"unknown config {config}")
