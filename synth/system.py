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


def _chain_walk(rng: np.random.Generator, n: int, centre: np.ndarray, radius: float, bond: float = 1.5,
                min_dist: float = 1.2, tries: int = 50) -> np.ndarray:
    """Self-avoiding random walk of n atoms, steps of `bond` A in uniform directions, kept inside a
    sphere and at least `min_dist` from every atom but its predecessor.  A step that fails `tries`
    times ends the chain and a new one starts at a free random point of the sphere."""
    pos = np.zeros((n, 3))
    cells: dict = {}

    def key(p):
        return tuple(np.floor(p / min_dist).astype(np.int64))

    def free(p, pred):
        if np.linalg.norm(p - centre) > radius:
            return False
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in cells.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        if j != pred and np.sum((pos[j] - p) ** 2) < min_dist * min_dist:
                            return False
        return True

    def restart():
        for _ in range(100000):
            v = rng.normal(size=3)
            p = centre + v / np.linalg.norm(v) * radius * rng.random() ** (1.0 / 3.0)
            if free(p, -1):
                return p
        raise RuntimeError("globule is full")

    pos[0] = centre
    cells.setdefault(key(pos[0]), []).append(0)
    for i in range(1, n):
        for _ in range(tries):
            v = rng.normal(size=3)
            p = pos[i - 1] + bond * v / np.linalg.norm(v)
            if free(p, i - 1):
                break
        else:
            p = restart()
        pos[i] = p
        cells.setdefault(key(p), []).append(i)
    return pos


def _kmeans_groups(rng: np.random.Generator, points: np.ndarray, k: int, weight: int, cap: int) -> list:
    """Groups of point indices: k-means (k-means++ seeding, seeded), then every group whose
    weight * size exceeds `cap` split in two along its longest extent until none does."""
    from scipy.cluster.vq import kmeans2
    _, label = kmeans2(points, k, minit="++", seed=rng, iter=20)
    out, todo = [], [np.flatnonzero(label == g) for g in range(k)]
    while todo:
        g = todo.pop()
        if g.size == 0:
            continue
        if g.size * weight <= cap:
            out.append(g)
            continue
        ext = points[g].max(0) - points[g].min(0)
        ax = int(np.argmax(ext))
        order = g[np.argsort(points[g, ax], kind="stable")]
        todo += [order[: g.size // 2], order[g.size // 2:]]
    return sorted(out, key=lambda g: int(g.min()))


def protein_globule(seed: int, n_protein: int = 12000, n_water: int = 6000, box: float = 100.0,
                    radius: float = 40.0, neighbourhood: float | None = 8.0, blocks: str = "clusters",
                    name: str | None = None) -> System:
    """A protein-like globule in water: a self-avoiding random-walk chain of n_protein C/N/O/H/S atoms
    (bond 1.5 A, non-bonded atoms >= 1.2 A apart, inside a sphere of `radius` at the box centre;
    element fractions H .49, C .31, N .09, O .10, S .01) and n_water waters outside it (O at least
    2.8 A from every other O -- at 2.5 A some molecules find no orientation free of clashes -- and
    2.5 A from every chain atom, random orientation) in a periodic box.

    Blocks (blocks="clusters"): the chain atoms k-means-clustered into groups of about 120 atoms,
    the waters (whole molecules) into groups of about 10, groups above 200 atoms split;
    blocks="atoms": one block per atom (the starting point of a submatrix combination).  Own
    columns are the blocks' basis functions; the index set of a block adds, to the pattern rule,
    every atom within `neighbourhood` of one of its atoms (minimum image).

    Electron count: the invented minimal-basis model has no gap at the valence count (the p and H
    levels form one band around -0.45 Ha), so N_e = 2 per heavy atom fills the band of heavy-atom s
    levels below the largest gap near it (about 0.1 Ha, near -0.6 Ha).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    centre = np.full(3, box / 2)
    chain = _chain_walk(rng, n_protein, centre, radius)
    chain_el = rng.choice(np.array([H, C, N, O, S]), size=n_protein, p=[0.49, 0.31, 0.09, 0.10, 0.01])
    # waters by random sequential addition outside the globule
    near_chain = cKDTree(chain)
    o_pos = np.zeros((n_water, 3))
    cells: dict = {}
    n_cell = int(box // 2.8)                 # periodic cell grid, cells at least 2.8 A wide
    got = 0
    while got < n_water:
        cand = rng.random((4096, 3)) * box
        ok = (np.linalg.norm(cand - centre, axis=1) > radius) & (near_chain.query(cand)[0] >= 2.5)
        for p in cand[ok]:
            k = tuple(np.floor(p / box * n_cell).astype(np.int64) % n_cell)
            clash = False
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        nk = ((k[0] + dx) % n_cell, (k[1] + dy) % n_cell, (k[2] + dz) % n_cell)
                        for j in cells.get(nk, ()):
                            d = o_pos[j] - p
                            d -= box * np.round(d / box)
                            if d @ d < 2.8 * 2.8:
                                clash = True
            if clash:
                continue
            o_pos[got] = p
            cells.setdefault(k, []).append(got)
            got += 1
            if got == n_water:
                break
    waters = _place_waters(rng, o_pos, box)
    coords = np.concatenate([chain, waters])
    element = np.concatenate([chain_el, np.tile(np.array([O, H, H]), n_water)])
    bf_ptr, row_ptr, col, h, s = build_matrices(coords, element, box, rng)
    groups = _kmeans_groups(rng, chain, max(1, round(n_protein / 120)), 1, 200)
    groups += [n_protein + 3 * g[:, None] + np.arange(3)[None, :]
               for g in _kmeans_groups(rng, o_pos, max(1, round(n_water / 10)), 3, 200)]
    if blocks == "atoms":
        groups = [np.array([a]) for a in range(coords.shape[0])]
    elif blocks != "clusters":
        raise ValueError(blocks)
    blk_ptr, blk_cols, ep, ei = _atom_group_blocks(coords, box, bf_ptr, groups, neighbourhood)
    n_e = 2.0 * float((element != H).sum())
    return System(name or f"globule{coords.shape[0]}", box, coords, element, bf_ptr, row_ptr, col, h, s, n_e,
                  blk_ptr, blk_cols, ep, ei)


def _atom_group_blocks(coords, box, bf_ptr, groups, neighbourhood):
    """Column blocks of atom groups: own columns = the group's basis functions; with a
    neighbourhood, the extra list = the basis functions of every atom within it of a group atom."""
    tree = cKDTree(np.mod(coords, box), boxsize=box)
    cols, ptr, extra, eptr = [], [0], [], [0]
    for g in groups:
        atoms = np.sort(np.asarray(g).reshape(-1))
        c = np.concatenate([np.arange(bf_ptr[a], bf_ptr[a + 1]) for a in atoms])
        cols.append(c)
        ptr.append(ptr[-1] + c.size)
        if neighbourhood is not None:
            near = tree.query_ball_point(np.mod(coords[atoms], box), r=neighbourhood)
            at = np.unique(np.concatenate([np.asarray(v, dtype=np.int64) for v in near]))
            e = np.concatenate([np.arange(bf_ptr[a], bf_ptr[a + 1]) for a in at])
            extra.append(e)
            eptr.append(eptr[-1] + e.size)
    ep = ei = None
    if neighbourhood is not None:
        ep, ei = np.array(eptr, np.int32), np.concatenate(extra).astype(np.int32)
    return np.array(ptr, np.int32), np.concatenate(cols).astype(np.int32), ep, ei


def atom_blocks(system: System, neighbourhood: float | None = 8.0) -> System:
    """The same matrices with one column block per atom (and its neighbourhood list): the starting
    point of a submatrix combination."""
    import dataclasses
    groups = [np.array([a]) for a in range(system.n_atoms)]
    blk_ptr, blk_cols, ep, ei = _atom_group_blocks(system.coords, system.box, system.atom_bf_ptr, groups,
                                                   neighbourhood)
    return dataclasses.replace(system, name=system.name + "-atoms", blk_ptr=blk_ptr, blk_cols=blk_cols,
                               extra_ptr=ep, extra_idx=ei)


def displaced(system: System, sigma: float, seed: int) -> System:
    """The next geometry of a short MD-like trajectory: every atom moved by N(0, sigma^2) per axis,
    H0 and S rebuilt on the new pattern with the same on-site energies (the diagonal of H0 is kept,
    its noise included), the same column blocks and extra lists."""
    import dataclasses
    rng = np.random.Generator(np.random.PCG64(seed))
    coords = system.coords + rng.normal(0.0, sigma, size=system.coords.shape)
    _, row_ptr, col, h, s = build_matrices(coords, system.element, system.box, rng)
    n = system.n_basis

    def diag_pos(rp, cl):
        rows = np.repeat(np.arange(n), np.diff(rp))
        return np.flatnonzero(rows == cl)

    h[diag_pos(row_ptr, col)] = system.h[diag_pos(system.row_ptr, system.col)]
    return dataclasses.replace(system, name=system.name + f"+d{seed}", coords=coords, row_ptr=row_ptr, col=col,
                               h=h, s=s)


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
    3: dict(desc="protein-like globule, 12,000 chain atoms in 6,000 waters (30,000 atoms), 100 A box, "
                 "10-200-atom blocks, pattern rule", seeds=(21, 22, 23)),
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
    if config == 3:
        return protein_globule(seed, name=f"globule30000-s{seed}")
    if config == 5:
        return water_clusters(24, seed, name=f"waterclusters13824-s{seed}")
    raise ValueError(f"unknown config {config}")
