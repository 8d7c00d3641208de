"""Independent numpy restatements used to pin the oracle (geometry by
brute-force distances, energies by full recomputation).  They import nothing
from the oracle or the CUDA binding."""
from __future__ import annotations

import itertools
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

SHELL_Z = {1: 8, 2: 6, 3: 12}
SHELL_D2 = {1: 3, 2: 4, 3: 8}  # squared distance in half-lattice units


def positions(nx, ny, nz):
    """Half-unit positions of all sites in canonical order (sub, z, y, x)."""
    sub, z, y, x = np.meshgrid(np.arange(2), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    p = np.stack([2 * x + sub, 2 * y + sub, 2 * z + sub], axis=-1).reshape(-1, 3)
    return p


def shell_vectors_bruteforce(shell):
    """All integer vectors of the BCC lattice (half units) at the shell's
    squared distance, found by enumeration."""
    out = []
    for v in itertools.product(range(-3, 4), repeat=3):
        if len({c % 2 for c in v}) == 1 and sum(c * c for c in v) == SHELL_D2[shell]:
            out.append(v)
    return sorted(out)


def neighbor_table(nx, ny, nz, shell):
    """[N, z_m] neighbour indices by periodic vector addition (with
    multiplicity in boxes small enough to alias)."""
    p = positions(nx, ny, nz)
    n = np.array([nx, ny, nz])
    vecs = np.array(shell_vectors_bruteforce(shell))
    q = p[:, None, :] + vecs[None, :, :]
    sub = q[..., 0] % 2
    cell = ((q - sub[..., None]) // 2) % n
    return ((sub * nz + cell[..., 2]) * ny + cell[..., 1]) * nx + cell[..., 0]


def pair_energy(occ, V, tables):
    """E = 1/2 sum_i sum_m sum_v V_m(s_i, s_{i+v}) for occ of shape [..., N]."""
    occ = np.asarray(occ).astype(np.int64)
    E = 0.0
    for m, nb in enumerate(tables):
        E = E + 0.5 * V[m][occ[..., :, None], occ[..., nb]].sum(axis=(-1, -2))
    return E


def read_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(t, 16) for t in line.split()]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows
