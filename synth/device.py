"""The water model of `synth.system` built on the GPU, for systems too large for the numpy
generator (the 1,000,000-molecule configuration: 6,000,000 basis functions, about 1e9 stored
entries).

Same geometry, parameters and random draws as `water_box` / `water_clusters`: the lattice jitter,
the Haar-random orientations (redrawn for clashing molecules in the same rounds and order) and the
on-site noise come from the same PCG64 stream on the host; only the pair search, the matrix values
and the CSR assembly run on the device (torch).  The molecules sit on a jittered cubic lattice, so
the atom pairs within the cutoff are found among lattice neighbours: a molecule's atoms are within
0.96 A of its O and an O is within 0.25 A (per axis) of its site, so two molecules more than two
sites apart along an axis are more than 6 A apart.  Values equal the numpy generator's up to the
rounding of exp (the tests compare both on a small box).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .system import (CUTOFF, H_DECAY, H_PREF, JITTER, LATTICE_SPACING, MIN_INTER, ONSITE_NOISE, S_DECAY,
                     S_PREF, _lattice, _random_rotations, _water_frame)

O_ONSITE = (-1.0, -0.5, -0.5, -0.5)     # O 2s, 2p x3 (Ha)
H_ONSITE = -0.4                         # H 1s


@dataclass
class DeviceSystem:
    """A water system whose CSR (row_ptr int64, col int32, h, s float64) lives in device memory as
    torch tensors; blocks and extra lists are host arrays (as for `synth.System`)."""
    name: str
    box: float
    n_mol: int
    row_ptr: object
    col: object
    h: object
    s: object
    blk_ptr: np.ndarray
    blk_cols: np.ndarray
    extra_ptr: np.ndarray
    extra_idx: np.ndarray
    n_electrons: float
    on_device: bool = True

    @property
    def n_atoms(self) -> int:
        return 3 * self.n_mol

    @property
    def n_basis(self) -> int:
        return 6 * self.n_mol

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def n_blocks(self) -> int:
        return len(self.blk_ptr) - 1

    def block_cols(self, b: int) -> np.ndarray:
        return self.blk_cols[self.blk_ptr[b]:self.blk_ptr[b + 1]]

    def block_extra(self, b: int) -> np.ndarray:
        return self.extra_idx[self.extra_ptr[b]:self.extra_ptr[b + 1]]


def _offsets(r: int, dev):
    import torch
    g = torch.arange(-r, r + 1, device=dev)
    return torch.stack(torch.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


def _neighbour_molecules(mol, n_side: int, offs):
    """Linear indices (molecule = (i n + j) n + k) of the lattice sites mol + offs (periodic)."""
    i = mol // (n_side * n_side)
    j = (mol // n_side) % n_side
    k = mol % n_side
    ii = (i[:, None] + offs[None, :, 0]) % n_side
    jj = (j[:, None] + offs[None, :, 1]) % n_side
    kk = (k[:, None] + offs[None, :, 2]) % n_side
    return (ii * n_side + jj) * n_side + kk


def _min_image(d, box: float):
    import torch
    return d - box * torch.round(d / box)


def _clashing_molecules(atoms, n_side: int, box: float, dev, chunk: int = 1 << 16):
    """Sorted molecules that are the higher-indexed member of a pair of different molecules with
    two atoms at most MIN_INTER apart (the rule of `_place_waters`)."""
    import torch
    n_mol = n_side ** 3
    offs = _offsets(1, dev)
    bad = []
    at = atoms.view(n_mol, 3, 3)
    for m0 in range(0, n_mol, chunk):
        mol = torch.arange(m0, min(m0 + chunk, n_mol), device=dev)
        nb = _neighbour_molecules(mol, n_side, offs)                       # M x 27
        keep = nb > mol[:, None]                                           # each pair once, other molecule
        a = at[mol][:, None, :, None, :]                                   # M x 1 x 3 x 1 x 3
        b = at[nb][:, :, None, :, :]                                       # M x 27 x 1 x 3 x 3
        d = _min_image(b - a, box)
        r2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]
        hit = (r2 <= MIN_INTER * MIN_INTER).any(dim=(2, 3)) & keep
        if hit.any():
            bad.append(nb[hit])
    if not bad:
        return np.zeros(0, np.int64)
    return torch.unique(torch.cat(bad)).cpu().numpy()


def _place_waters_device(rng, o_pos: np.ndarray, box: float, n_side: int, dev):
    """`_place_waters` with the clash search on the device (same draws, same rounds)."""
    import torch
    n = o_pos.shape[0]
    frame = _water_frame()
    rot = _random_rotations(rng, n)
    o_t = torch.from_numpy(o_pos).to(dev)
    for _ in range(10000):
        hpos = o_pos[:, None, :] + np.einsum("nij,kj->nki", rot, frame)
        atoms = np.concatenate([o_pos[:, None, :], hpos], axis=1).reshape(-1, 3)
        bad = _clashing_molecules(torch.from_numpy(atoms).to(dev), n_side, box, dev)
        if bad.size == 0:
            del o_t
            return atoms
        rot[bad] = _random_rotations(rng, bad.size)
    raise RuntimeError("water placement did not converge")


def _matrices(atoms_t, n_side: int, box: float, onsite_t, dev, chunk: int = 1 << 15):
    """CSR (row_ptr, col, h, s) on the device: every basis pair of two different atoms at most
    CUTOFF apart (both triangles) and the diagonal; Slater-Koster sigma factors as in
    `synth.system._pair_factor`."""
    import torch
    n_mol = n_side ** 3
    N = 6 * n_mol
    offs = _offsets(2, dev)
    at = atoms_t.view(n_mol, 3, 3)
    # orbital tables of a molecule's 6 basis functions: atom (0 O, 1 H1, 2 H2), kind (-1 s, 0..2 p axis)
    bf_atom = torch.tensor([0, 0, 0, 0, 1, 2], device=dev)
    bf_axis = torch.tensor([-1, 0, 1, 2, -1, -1], device=dev)
    rp_parts, col_parts, h_parts, s_parts = [], [], [], []
    for m0 in range(0, n_mol, chunk):
        m1 = min(m0 + chunk, n_mol)
        mol = torch.arange(m0, m1, device=dev)
        M = m1 - m0
        nb = _neighbour_molecules(mol, n_side, offs)                          # M x 125
        a = at[mol][:, None, :, None, :]                                      # M x 1 x 3 x 1 x 3
        b = at[nb][:, :, None, :, :]                                          # M x 125 x 1 x 3 x 3
        d = _min_image(b - a, box)                                            # from atom a to atom b
        r = torch.sqrt(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2])
        same = (nb[:, :, None, None] == mol[:, None, None, None]) & \
            (torch.arange(3, device=dev)[None, None, :, None] == torch.arange(3, device=dev)[None, None, None, :])
        ok = (r <= CUTOFF) & ~same                                            # M x 125 x 3 x 3
        mi, oi, pa, pb = torch.nonzero(ok, as_tuple=True)                     # atom pairs (row atom pa)
        rr = r[mi, oi, pa, pb]
        dd = d[mi, oi, pa, pb]
        ll = dd / rr[:, None]
        gh = H_PREF * torch.exp(-rr / H_DECAY)
        gs = S_PREF * torch.exp(-rr / S_DECAY)
        ma = mol[mi]
        mb = nb[mi, oi]
        # expand to the 6 x 6 basis pairs of the two molecules, keep those of atoms pa (row), pb (col)
        ra = torch.arange(6, device=dev)
        sel_r = bf_atom[None, :] == pa[:, None]                               # E x 6
        sel_c = bf_atom[None, :] == pb[:, None]
        keep = sel_r[:, :, None] & sel_c[:, None, :]                          # E x 6 x 6
        e_i, r_i, c_i = torch.nonzero(keep, as_tuple=True)
        ax_r = bf_axis[r_i]
        ax_c = bf_axis[c_i]
        l_e = ll[e_i]
        lr = torch.where(ax_r >= 0, l_e.gather(1, ax_r.clamp(min=0)[:, None])[:, 0], torch.ones_like(l_e[:, 0]))
        lc = torch.where(ax_c >= 0, l_e.gather(1, ax_c.clamp(min=0)[:, None])[:, 0], torch.ones_like(l_e[:, 0]))
        # ss: 1; s_row p_col(beta): l_beta; p_row(alpha) s_col: -l_alpha; p p: l_alpha l_beta
        f = torch.where((ax_r < 0) & (ax_c < 0), torch.ones_like(lr),
                        torch.where(ax_r < 0, lc, torch.where(ax_c < 0, -lr, lr * lc)))
        rows = 6 * ma[e_i] + r_i
        cols = 6 * mb[e_i] + c_i
        hv = gh[e_i] * f
        sv = gs[e_i] * f
        del keep, e_i, r_i, c_i, ax_r, ax_c, l_e, lr, lc, f, sel_r, sel_c
        # the diagonal (on-site energies, S = 1)
        drow = torch.arange(6 * m0, 6 * m1, device=dev)
        rows = torch.cat([rows, drow])
        cols = torch.cat([cols, drow])
        hv = torch.cat([hv, onsite_t[6 * m0:6 * m1]])
        sv = torch.cat([sv, torch.ones(6 * M, dtype=torch.float64, device=dev)])
        key = (rows - 6 * m0) * N + cols
        key, order = torch.sort(key)
        counts = torch.bincount((key // N), minlength=6 * M)
        rp_parts.append(counts)
        col_parts.append((key % N).to(torch.int32))
        h_parts.append(hv[order])
        s_parts.append(sv[order])
        del key, order, rows, cols, hv, sv, d, r, ok, same, a, b, nb
    counts = torch.cat(rp_parts)
    row_ptr = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts, 0)
    col = torch.cat(col_parts)
    del col_parts
    h = torch.cat(h_parts)
    del h_parts
    s = torch.cat(s_parts)
    del s_parts
    return row_ptr, col, h, s


def _cluster_blocks(o_pos_t, n_side: int, box: float, cluster, halo: float, dev, chunk: int = 4096):
    """Blocks of cluster[0] x cluster[1] x cluster[2] lattice sites and, per block, the basis
    functions of every molecule whose O is within `halo` of one of the block's O (sorted)."""
    import torch
    cx, cy, cz = cluster
    n = n_side
    m = torch.arange(n ** 3, device=dev)
    i, j, k = m // (n * n), (m // n) % n, m % n
    cid = ((i // cx) * (n // cy) + j // cy) * (n // cz) + k // cz
    members = torch.argsort(cid, stable=True).view(-1, cx * cy * cz)          # ascending molecules
    n_blk = members.shape[0]
    blk_cols = (6 * members[:, :, None] + torch.arange(6, device=dev)).reshape(-1).to(torch.int32)
    # candidates: the block's sites widened by two sites per side (O-O > halo beyond that)
    r = int(np.ceil((halo + 2 * JITTER * np.sqrt(3.0)) / LATTICE_SPACING))
    gx = torch.arange(-r, cx + r, device=dev)
    gy = torch.arange(-r, cy + r, device=dev)
    gz = torch.arange(-r, cz + r, device=dev)
    win = torch.stack(torch.meshgrid(gx, gy, gz, indexing="ij"), -1).reshape(-1, 3)   # W x 3
    bi, bj, bk = torch.meshgrid(torch.arange(n // cx, device=dev), torch.arange(n // cy, device=dev),
                                torch.arange(n // cz, device=dev), indexing="ij")
    corner = torch.stack([bi.reshape(-1) * cx, bj.reshape(-1) * cy, bk.reshape(-1) * cz], -1)   # n_blk x 3
    keys = []
    for b0 in range(0, n_blk, chunk):
        b1 = min(b0 + chunk, n_blk)
        site = (corner[b0:b1, None, :] + win[None, :, :]) % n                   # B x W x 3
        cand = (site[..., 0] * n + site[..., 1]) * n + site[..., 2]              # B x W
        own = o_pos_t[members[b0:b1]]                                            # B x 32 x 3
        d = _min_image(o_pos_t[cand][:, :, None, :] - own[:, None, :, :], box)   # B x W x 32 x 3
        r2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]
        near = (r2 <= halo * halo).any(dim=2)                                    # B x W
        bidx, widx = torch.nonzero(near, as_tuple=True)
        keys.append((bidx + b0) * n ** 3 + cand[bidx, widx])
    key = torch.unique(torch.cat(keys))                                          # sorted: block, molecule
    blk = key // n ** 3
    mol = key % n ** 3
    per = torch.bincount(blk, minlength=n_blk) * 6
    extra_ptr = torch.zeros(n_blk + 1, dtype=torch.int64, device=dev)
    extra_ptr[1:] = torch.cumsum(per, 0)
    extra_idx = (6 * mol[:, None] + torch.arange(6, device=dev)).reshape(-1).to(torch.int32)
    blk_ptr = (np.arange(n_blk + 1) * 6 * cx * cy * cz).astype(np.int32)
    return blk_ptr, blk_cols.cpu().numpy(), extra_ptr.cpu().numpy().astype(np.int32), extra_idx.cpu().numpy()


def water_clusters_device(n_side: int, seed: int, cluster=(2, 4, 4), halo: float = 8.0, device="cuda",
                          name: str | None = None) -> DeviceSystem:
    """`synth.system.water_clusters` with its CSR built in device memory (n_side >= 5)."""
    import torch
    if n_side < 5:
        raise ValueError("n_side must be at least 5 (distinct lattice neighbours within two sites)")
    cx, cy, cz = cluster
    if n_side % cx or n_side % cy or n_side % cz:
        raise ValueError("n_side must be a multiple of every cluster edge")
    dev = torch.device(device)
    rng = np.random.Generator(np.random.PCG64(seed))
    box = n_side * LATTICE_SPACING
    n_mol = n_side ** 3
    o_pos = _lattice(n_side, LATTICE_SPACING) + rng.uniform(-JITTER, JITTER, size=(n_mol, 3))
    atoms = _place_waters_device(rng, o_pos, box, n_side, dev)
    onsite = np.tile(np.array(list(O_ONSITE) + [H_ONSITE, H_ONSITE]), n_mol)
    onsite += rng.normal(0.0, ONSITE_NOISE, size=6 * n_mol)
    atoms_t = torch.from_numpy(atoms).to(dev)
    row_ptr, col, h, s = _matrices(atoms_t, n_side, box, torch.from_numpy(onsite).to(dev), dev)
    del atoms_t
    bp, bc, ep, ei = _cluster_blocks(torch.from_numpy(o_pos).to(dev), n_side, box, cluster, halo, dev)
    return DeviceSystem(name or f"waterclusters{n_mol}-s{seed}", box, n_mol, row_ptr, col, h, s, bp, bc, ep, ei,
                        8.0 * n_mol)
