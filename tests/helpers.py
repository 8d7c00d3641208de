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


# ---------------------------------------------------------------------------
# MLP site energies: features and the error bound of the BF16 tensor-core path.
# ---------------------------------------------------------------------------
def site_neighbors(sites, dims):
    """[len(sites), 26] neighbour indices of the given sites (shell 1, then
    2, then 3, vectors in brute-force order) and the shell of each column."""
    nx, ny, nz = dims
    s = np.asarray(sites, dtype=np.int64).reshape(-1)
    x, y, z = s % nx, (s // nx) % ny, (s // (nx * ny)) % nz
    sub = s // (nx * ny * nz)
    p = np.stack([2 * x + sub, 2 * y + sub, 2 * z + sub], axis=-1)
    vecs, shell = [], []
    for m in (1, 2, 3):
        for v in shell_vectors_bruteforce(m):
            vecs.append(v)
            shell.append(m)
    q = p[:, None, :] + np.array(vecs)[None, :, :]
    qs = q[..., 0] % 2
    cell = ((q - qs[..., None]) // 2) % np.array([nx, ny, nz])
    idx = ((qs * nz + cell[..., 2]) * ny + cell[..., 1]) * nx + cell[..., 0]
    return idx, np.array(shell)


def mlp_features(occ, dims, sites, swap=None):
    """[len(sites), 20] MLP inputs [onehot(5) | shell-1, -2, -3 species
    counts]; with swap = (a, b) the species of a and b are exchanged first."""
    occ = np.asarray(occ).astype(np.int64)
    sites = np.asarray(sites, dtype=np.int64).reshape(-1)
    nb, shell = site_neighbors(sites, dims)

    def spec(idx):
        v = occ[idx]
        if swap is not None:
            a, b = swap
            v = np.where(idx == a, occ[b], np.where(idx == b, occ[a], v))
        return v

    X = np.zeros((sites.size, 20))
    X[np.arange(sites.size), spec(sites)] = 1.0
    sn = spec(nb)
    for m in (1, 2, 3):
        cols = sn[:, shell == m]
        for q in range(5):
            X[:, 5 * m + q] = (cols == q).sum(axis=1)
    return X


def omega(a, b, dims):
    """Sites whose MLP energy a swap of a and b changes: a, b and their
    neighbours within three shells (40 on BCC)."""
    nb, _ = site_neighbors([a, b], dims)
    return np.unique(np.concatenate([[a, b], nb.reshape(-1)]))


def _silu(z):
    return z / (1.0 + np.exp(-z))


TANH_APPROX_REL = 2.0 ** -10  # hardware tanh approximation: documented ~2^-11, with a factor-2 margin


def mlp_error_bound(X, w):
    """First-order bound on |f_GPU(x) - f(x)| per row of X, for the tensor-core
    evaluation: FP32 accumulation over K terms (error <= K 2^-22 of the sum of
    magnitudes, generous for truncating adders), SiLU as h + h tanh(h) with a
    relative tanh error TANH_APPROX_REL, layer-1 activations rounded to BF16
    (relative 2^-8), |silu'| <= 1.1.  w holds FP64 w1, b1, w2, b2, w3, b3.
    Returns (bound, f) with f the exact FP64 f(x)."""
    u_bf16 = 2.0 ** -8

    def gam(k):
        return k * 2.0 ** -22

    def e_silu(z):
        return np.abs(z) * (0.5 * TANH_APPROX_REL + 2.0 ** -22)

    w1, b1, w2, b2, w3, b3 = (w[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3"))
    z1 = X @ w1.T + b1
    dz1 = gam(32) * (np.abs(X) @ np.abs(w1).T + np.abs(b1))
    h1 = _silu(z1)
    e1 = 1.1 * dz1 + e_silu(z1)
    e1 = e1 + u_bf16 * (np.abs(h1) + e1)
    z2 = h1 @ w2.T + b2
    dz2 = e1 @ np.abs(w2).T + gam(64) * (np.abs(b2) + (np.abs(h1) + e1) @ np.abs(w2).T)
    h2 = _silu(z2)
    e2 = 1.1 * dz2 + e_silu(z2)
    f = h2 @ w3 + b3
    ef = e2 @ np.abs(w3) + gam(66) * (abs(b3) + (np.abs(h2) + e2) @ np.abs(w3))
    return ef, f


def bf16_round(v):
    """Round to the nearest BF16 value (ties to even) through FP32."""
    f = np.asarray(v, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_bf16_emulation(X, w):
    """The BF16 evaluation order in FP64: exact layer 1, SiLU, layer-1
    activations rounded to BF16, exact layer 2, SiLU, output.  Returns
    (f_emu, bound) where bound limits |f_GPU - f_emu| per row: FP32
    accumulation (K 2^-22 of the magnitudes), the tanh approximation
    (TANH_APPROX_REL) and, where an activation lies closer to a BF16 rounding
    boundary than its own error, one BF16 spacing for that activation."""
    def gam(k):
        return k * 2.0 ** -22

    def e_silu(z):
        return np.abs(z) * (0.5 * TANH_APPROX_REL + 2.0 ** -22)

    w1, b1, w2, b2, w3, b3 = (w[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3"))
    z1 = X @ w1.T + b1
    dz1 = gam(32) * (np.abs(X) @ np.abs(w1).T + np.abs(b1))
    s1 = _silu(z1)
    ds1 = 1.1 * dz1 + e_silu(z1) + 2.0 ** -23 * np.abs(s1)
    h1 = bf16_round(s1)
    mag = np.maximum(np.abs(s1), 1e-300)
    spacing = 2.0 ** (np.floor(np.log2(mag)) - 7)
    frac = np.abs(s1) / spacing
    dist = np.abs(frac - np.floor(frac) - 0.5) * spacing  # distance to the nearest rounding boundary
    dh1 = np.where(dist <= 2 * ds1, 2 * spacing, 0.0)
    z2 = h1 @ w2.T + b2
    dz2 = dh1 @ np.abs(w2).T + gam(64) * (np.abs(b2) + (np.abs(h1) + dh1) @ np.abs(w2).T)
    s2 = _silu(z2)
    ds2 = 1.1 * dz2 + e_silu(z2)
    f = s2 @ w3 + b3
    bound = ds2 @ np.abs(w3) + gam(66) * (abs(b3) + (np.abs(s2) + ds2) @ np.abs(w3))
    return f, bound


def mlp_grad_abs_terms(X, w):
    """Per MLP parameter (gradient layout: W1, b1, W2, b2, W3, b3), the sum
    over the rows of X of the magnitude of its gradient term in the
    absolute-value network (|W| everywhere, |silu| <= |z|, |silu'| <= 1.1), so
    that cancellations inside a term (the back-propagated d1 of a single
    site, say) cannot make the scale smaller than the rounding it carries."""
    w1, b1, w2, b2, w3 = (np.abs(w[k]) for k in ("w1", "b1", "w2", "b2", "w3"))
    X = np.abs(X)
    a1 = X @ w1.T + b1
    a2 = a1 @ w2.T + b2
    d2 = np.broadcast_to(1.1 * w3, a2.shape)
    d1 = 1.1 * (d2 @ w2)
    return np.concatenate([(d1.T @ X).reshape(-1), d1.sum(0), (d2.T @ a1).reshape(-1), d2.sum(0), a2.sum(0),
                           [float(X.shape[0])]])


def _bf16_spacing_near_boundary(a, da):
    """Two BF16 spacings where a value lies within 2 da of a BF16 rounding
    boundary (where the GPU's FP32 value may round the other way), else 0."""
    mag = np.maximum(np.abs(a), 1e-300)
    spacing = 2.0 ** (np.floor(np.log2(mag)) - 7)
    frac = np.abs(a) / spacing
    dist = np.abs(frac - np.floor(frac) - 0.5) * spacing
    return np.where(dist <= 2 * da, 2 * spacing, 0.0)


def mlpnet_bf16_emulation(X, w):
    """MLPNet's BF16 evaluation order in FP64: exact layer products, ReLU, the
    activations of the first two layers rounded to BF16 (the operands of the
    next products), FP32 output layer.  Returns (f_emu, bound) where bound
    limits |f_GPU - f_emu| per row: FP32 accumulation (K 2^-22 of the
    magnitudes), one BF16 step where an activation lies within its own error
    of a rounding boundary, and the error itself where ReLU's kink is that
    close."""
    def gam(k):
        return k * 2.0 ** -22

    def act(z, dz):
        a = np.maximum(z, 0.0)
        h = bf16_round(a)
        dh = _bf16_spacing_near_boundary(a, dz) + np.where(np.abs(z) <= dz, 2 * dz, 0.0)
        return h, dh

    w0, b0, w1, b1, w2, b2, w3, b3 = (w[k] for k in ("w0", "b0", "w1", "b1", "w2", "b2", "w3", "b3"))
    z0 = X @ w0.T + b0
    dz0 = gam(32) * (np.abs(X) @ np.abs(w0).T + np.abs(b0))
    h1, dh1 = act(z0, dz0)
    z1 = h1 @ w1.T + b1
    dz1 = dh1 @ np.abs(w1).T + gam(112) * (np.abs(b1) + (np.abs(h1) + dh1) @ np.abs(w1).T)
    h2, dh2 = act(z1, dz1)
    z2 = h2 @ w2.T + b2
    dz2 = dh2 @ np.abs(w2).T + gam(112) * (np.abs(b2) + (np.abs(h2) + dh2) @ np.abs(w2).T)
    h3 = np.maximum(z2, 0.0)
    f = h3 @ w3 + b3
    bound = (dz2 + 2.0 ** -23 * h3) @ np.abs(w3) + gam(98) * (abs(b3) + (h3 + dz2) @ np.abs(w3))
    return f, bound
