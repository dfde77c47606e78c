"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's matrices are B3LYP/6-31G** Fockians and density matrices of
water clusters at standard temperature and pressure, ordered along a
locality-preserving space-filling curve (Sec. 4; Fig. 1 shows the
exponential, clustered decay of magnitudes).  Those matrices are not
available, so this module builds stand-ins with the same structure:

* sites: three-site "molecules" (one centre plus two sites 1 Angstrom
  away in random directions) at random positions in a cube sized to one
  molecule per 30 cubic Angstrom, plus up to two single sites; the sites
  are ordered along a 3-D Morton curve (Z-order), the curve this library
  uses in place of the paper's Hilbert curve;
* `decaying_matrix`: a symmetric matrix with exponential decay in the
  inter-site distance, a_ij = u_ij exp(-r_ij / lambda), u_ij uniform in
  [0.5, 1] with a random sign, a_ii = 1 (the decay definition of Sec. 2);
* `tb_hamiltonian`: a gapped tight-binding Hamiltonian,
  h_ij = -exp(-r_ij / lambda) for i != j (set to zero below 1e-12),
  h_ii = -2 for sites with an even generation index, +2 for odd ones.

This module holds no SpAMM or SP2 arithmetic: it only draws inputs.  Both
the CUDA path and the CPU oracle consume the arrays it returns.  Every
draw comes from numpy's PCG64 generator seeded by the caller.
"""
from __future__ import annotations

import numpy as np

__all__ = ["water_sites", "morton3", "distances", "decaying_matrix",
           "tb_hamiltonian", "tb_hamiltonian_block", "tb_hamiltonian_torch", "batch_sizes"]

_MORTON_BITS = 21


def _spread3(x: np.ndarray) -> np.ndarray:
    """Insert two zero bits between each of the low 21 bits of x."""
    x = x.astype(np.uint64) & np.uint64(0x1FFFFF)
    x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
    return x


def morton3(pos: np.ndarray) -> np.ndarray:
    """63-bit Z-order keys of points, quantised to 21 bits per axis over their
    bounding box."""
    lo = pos.min(axis=0)
    ext = pos.max(axis=0) - lo
    ext[ext == 0] = 1.0
    q = np.floor((pos - lo) / ext * ((1 << _MORTON_BITS) - 1)).astype(np.uint64)
    return _spread3(q[:, 0]) | (_spread3(q[:, 1]) << np.uint64(1)) | (
        _spread3(q[:, 2]) << np.uint64(2))


def water_sites(n: int, rng: np.random.Generator):
    """Positions (n, 3) in Angstrom and generation indices (n,) of n sites,
    Morton ordered (stable sort, ties by generation index)."""
    if n <= 0:
        raise ValueError("n must be positive")
    nc = n // 3
    extra = n - 3 * nc
    side = (30.0 * (nc + (1 if extra > 0 else 0))) ** (1.0 / 3.0)
    centres = rng.uniform(0.0, side, size=(nc + extra, 3))
    dirs = rng.standard_normal(size=(nc, 2, 3))
    dirs /= np.linalg.norm(dirs, axis=2, keepdims=True)
    pos = np.empty((n, 3))
    pos[0:3 * nc:3] = centres[:nc]
    pos[1:3 * nc:3] = centres[:nc] + dirs[:, 0]
    pos[2:3 * nc:3] = centres[:nc] + dirs[:, 1]
    pos[3 * nc:] = centres[nc:]
    order = np.argsort(morton3(pos), kind="stable")
    return pos[order], order.astype(np.int64)


def distances(pos: np.ndarray, rows: slice | None = None) -> np.ndarray:
    """Euclidean distances between the points in `rows` and all points."""
    p = pos if rows is None else pos[rows]
    d = p[:, None, :] - pos[None, :, :]
    return np.sqrt(np.einsum("ijk,ijk->ij", d, d))


def decaying_matrix(n: int, seed: int, decay: float = 1.5) -> np.ndarray:
    """Symmetric n x n FP64 matrix a_ij = u_ij exp(-r_ij/decay), a_ii = 1,
    with u_ij uniform in [0.5, 1] times a random sign, drawn for i < j and
    mirrored."""
    rng = np.random.default_rng(seed)
    pos, _ = water_sites(n, rng)
    a = np.empty((n, n))
    step = 1024
    for r0 in range(0, n, step):
        a[r0:r0 + step] = np.exp(-distances(pos, slice(r0, r0 + step)) / decay)
    u = rng.uniform(0.5, 1.0, size=(n, n))
    u *= np.where(rng.random(size=(n, n)) < 0.5, -1.0, 1.0)
    iu = np.triu_indices(n, 1)
    a[iu] *= u[iu]
    a.T[iu] = a[iu]
    np.fill_diagonal(a, 1.0)
    return a


def tb_hamiltonian(n: int, seed: int, decay: float = 1.2, onsite: float = 2.0,
                   cut: float = 1e-12):
    """Tight-binding Hamiltonian h_ij = -exp(-r_ij/decay) (i != j), entries
    with |h_ij| < cut set to 0, h_ii = -onsite for even generation index and
    +onsite for odd.  Returns the matrix (n x n FP64)."""
    rng = np.random.default_rng(seed)
    pos, gen = water_sites(n, rng)
    h = np.empty((n, n))
    step = 1024
    for r0 in range(0, n, step):
        blk = -np.exp(-distances(pos, slice(r0, r0 + step)) / decay)
        blk[np.abs(blk) < cut] = 0.0
        h[r0:r0 + step] = blk
    np.fill_diagonal(h, np.where(gen % 2 == 0, -onsite, onsite))
    return h


def tb_hamiltonian_block(n: int, m: int, seed: int, decay: float = 1.2, onsite: float = 2.0,
                         cut: float = 1e-12) -> np.ndarray:
    """The leading m x m principal block of `tb_hamiltonian(n, seed, ...)`
    (the first m sites along the Morton curve), built without forming the
    n x n matrix."""
    if not 0 < m <= n:
        raise ValueError("need 0 < m <= n")
    rng = np.random.default_rng(seed)
    pos, gen = water_sites(n, rng)
    pos, gen = pos[:m], gen[:m]
    h = np.empty((m, m))
    step = 1024
    for r0 in range(0, m, step):
        blk = -np.exp(-distances(pos, slice(r0, r0 + step)) / decay)
        blk[np.abs(blk) < cut] = 0.0
        h[r0:r0 + step] = blk
    np.fill_diagonal(h, np.where(gen % 2 == 0, -onsite, onsite))
    return h


def tb_hamiltonian_torch(n: int, seed: int, decay: float = 1.2, onsite: float = 2.0,
                         cut: float = 1e-12, device="cuda", rows_per_block: int = 1024):
    """`tb_hamiltonian` built in a torch tensor on `device` (same sites, same
    formula; exp may differ from numpy's in the last bit), for sizes whose
    dense host copy would not fit in host memory."""
    import torch
    rng = np.random.default_rng(seed)
    pos, gen = water_sites(n, rng)
    p = torch.from_numpy(pos).to(device)
    h = torch.empty((n, n), dtype=torch.float64, device=device)
    for r0 in range(0, n, rows_per_block):
        d = p[r0:r0 + rows_per_block, None, :] - p[None, :, :]
        blk = -torch.exp(-torch.sqrt((d * d).sum(dim=2)) / decay)
        del d
        blk[blk.abs() < cut] = 0.0
        h[r0:r0 + rows_per_block] = blk
        del blk
    diag = torch.from_numpy(np.where(gen % 2 == 0, -onsite, onsite)).to(device)
    h.diagonal().copy_(diag)
    return h


def batch_sizes(count: int, seed: int, lo: int = 512, hi: int = 8192,
                quantum: int = 32):
    """Sizes drawn log-uniformly in [lo, hi] and rounded to `quantum`, with a
    decay length uniform in [1.0, 2.0] Angstrom for each."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))
    n = np.clip(np.round(n / quantum).astype(np.int64) * quantum, lo, hi)
    decay = rng.uniform(1.0, 2.0, size=count)
    return [int(x) for x in n], [float(x) for x in decay]
