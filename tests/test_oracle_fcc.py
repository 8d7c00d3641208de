"""Pins of the oracle's FCC lattice (the paper's lattice, Sec. IV-C; link
cells of 4x4x4 cells, 256 mini-steps as in Sec. V-C), pair models, on CPU.

* Shells 1-3 equal the 12, 6 and 24 nearest sites by brute-force distance
  over the cubic box (positions in half cell units, minimum image).
* Link-cell independence: within every mini-step no trial writes a site
  another trial reads (all partner choices, 1-3 shells).
* Closed-form energies of the L1_2 (A3B) and L1_0 (AB layers) orderings.
* Every incremental dE equals the change of the total energy.
* A chain on 2x1x1 cells (8 sites, 70 states) samples the enumerated
  Boltzmann distribution.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs

BASIS = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [0, 1, 1]])


def positions(nx, ny, nz):
    """Half-unit positions of the sites in id order s = ((sub nz + z) ny + y) nx + x."""
    out = []
    for sub in range(4):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    out.append(2 * np.array([x, y, z]) + BASIS[sub])
    return np.array(out)


def brute_shells(dims):
    P = positions(*dims)
    box = 2 * np.array(dims)
    d = P[None, :, :] - P[:, None, :]
    d = d - box * np.round(d / box).astype(np.int64)
    d2 = (d ** 2).sum(-1)
    return {m: [set(np.flatnonzero(d2[i] == 2 * m)) for i in range(len(P))] for m in (1, 2, 3)}


def test_shells_by_brute_force_distance():
    dims = (4, 4, 4)
    lat = oracle.Lattice(*dims, 2)
    shells = brute_shells(dims)
    for m, n in ((1, 12), (2, 6), (3, 24)):
        vs = oracle.fcc_shell_vectors(m)
        assert len(vs) == n
        for i in range(oracle.fcc_nsites(lat)):
            got = {oracle.fcc_neighbor(lat, i, v) for v in vs}
            assert got == shells[m][i] and len(shells[m][i]) == n


@pytest.mark.parametrize("nsh", [1, 2, 3])
def test_link_cells_are_independent(nsh):
    dims = (8, 8, 8)
    lat = oracle.Lattice(*dims, 2)
    sh = brute_shells(dims)
    near = [set().union(*(sh[m][i] for m in range(1, nsh + 1))) for i in range(oracle.fcc_nsites(lat))]
    nA, L = oracle.fcc_schedule(lat)
    assert nA == 256 and L == (4, 4, 4)
    NL = [d // 4 for d in dims]
    for k in range(nA):
        dx, r = k % 4, k // 4
        dy, dz, sub = r % 4, (r // 4) % 4, r // 16
        writes, reads = [], []
        for cz in range(NL[2]):
            for cy in range(NL[1]):
                for cx in range(NL[0]):
                    a = (((sub * dims[2] + 4 * cz + dz) * dims[1] + 4 * cy + dy) * dims[0] + 4 * cx + dx)
                    w = {a} | sh[1][a]  # a and every partner it may pick
                    om = set(w)
                    for b in w:
                        om |= near[b]
                    rd = set(om)
                    for j in om:
                        rd |= near[j]
                    writes.append(w)
                    reads.append(rd)
        for t in range(len(writes)):
            for u in range(len(writes)):
                if t != u:
                    assert not (writes[t] & reads[u]), (k, t, u)


def _pair_model(seed, nsh, S=2):
    V = inputs.pair_int_coeffs(seed, nsh, S)
    return V, oracle.Model(oracle.PAIR_I32, nsh, V, unit_ev=1e-4)


def test_l12_ordering_energy():
    """Sublattice 0 species B (1), 1-3 species A (0): a B site has 12 A first
    neighbours, 6 B second, 24 A third; an A site 4 B + 8 A first, 6 A
    second, 8 B + 16 A third."""
    V, m = _pair_model(3, 3)
    lat = oracle.Lattice(4, 4, 4, 2)
    N = oracle.fcc_nsites(lat)
    occ = np.zeros(N, dtype=np.int8)
    occ[: N // 4] = 1
    A, B = 0, 1
    e_b = 12 * V[0, B, A] + 6 * V[1, B, B] + 24 * V[2, B, A]
    e_a = 4 * V[0, A, B] + 8 * V[0, A, A] + 6 * V[1, A, A] + 8 * V[2, A, B] + 16 * V[2, A, A]
    want2 = N // 4 * e_b + 3 * N // 4 * e_a
    assert want2 % 2 == 0
    assert oracle.fcc_total_energy_i64(lat, m, occ) == want2 // 2


def test_l10_ordering_energy():
    """Sublattices 0-1 species A, 2-3 species B (layers along z): every site
    has 4 like + 8 unlike first neighbours, 6 like second, 8 like + 16
    unlike third."""
    V, m = _pair_model(4, 3)
    lat = oracle.Lattice(4, 4, 4, 2)
    N = oracle.fcc_nsites(lat)
    occ = np.zeros(N, dtype=np.int8)
    occ[N // 2:] = 1
    tot2 = 0
    for s, o in ((0, 1), (1, 0)):
        tot2 += N // 2 * (4 * V[0, s, s] + 8 * V[0, s, o] + 6 * V[1, s, s] + 8 * V[2, s, s] + 16 * V[2, s, o])
    assert oracle.fcc_total_energy_i64(lat, m, occ) == tot2 // 2


@pytest.mark.parametrize("nsh,kind", [(1, "int"), (2, "int"), (3, "f32")])
def test_delta_e_is_the_change_of_the_total(nsh, kind):
    S = 3
    lat = oracle.Lattice(4, 5, 3, S)
    if kind == "int":
        V = inputs.pair_int_coeffs(nsh, nsh, S)
        m = oracle.Model(oracle.PAIR_I32, nsh, V, unit_ev=1e-4)
        tot = lambda o: oracle.fcc_total_energy_i64(lat, m, o)  # noqa: E731
    else:
        V = inputs.pair_f32_coeffs(nsh, nsh, S)
        m = oracle.Model(oracle.PAIR_F32, nsh, V)
        tot = lambda o: oracle.fcc_total_energy(lat, m, o)  # noqa: E731
    occ = oracle.fcc_init_lattice(lat, inputs.equiatomic_counts(oracle.fcc_nsites(lat), S), 2)
    rng = np.random.default_rng(nsh)
    for _ in range(30):
        a = int(rng.integers(oracle.fcc_nsites(lat)))
        b = oracle.fcc_neighbor(lat, a, oracle.fcc_shell_vectors(1)[rng.integers(12)])
        e0 = tot(occ)
        d = oracle.fcc_delta_e(lat, m, occ, a, b)
        occ[a], occ[b] = occ[b], occ[a]
        assert d == pytest.approx(tot(occ) - e0, abs=1e-9)


def test_chain_matches_enumeration_8_site():
    """2x1x1 cells, binary 4/4: <E> of the chain within 3 batch-means
    standard errors of the exact canonical average."""
    V = inputs.pair_int_coeffs(5, 2, 2, lo=-100, hi=100)
    m = oracle.Model(oracle.PAIR_I32, 2, V, unit_ev=1e-4)
    lat = oracle.Lattice(2, 1, 1, 2)
    kT = 0.02
    E = []
    for ones in itertools.combinations(range(8), 4):
        c = np.zeros(8, dtype=np.int8)
        c[list(ones)] = 1
        E.append(oracle.fcc_total_energy_i64(lat, m, c))
    E = np.array(E, dtype=np.float64) * 1e-4
    w = np.exp(-(E - E.min()) / kT)
    exact = (w * E).sum() / w.sum()
    assert E.std() > 0
    occ = np.array([0, 1] * 4, dtype=np.int8)  # any 4/4 start
    nsw = 30000
    Es = np.empty(nsw)
    for t in range(nsw):
        oracle.fcc_sweep(lat, m, occ, 3, t, 1, kT)
        Es[t] = oracle.fcc_total_energy_i64(lat, m, occ) * 1e-4
    nb = 50
    keep = (nsw - nsw // 10) // nb * nb
    bm = Es[nsw - keep:].reshape(nb, -1).mean(1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(bm.mean() - exact) < 3 * se, (bm.mean(), exact, se)


# ---- qSRO model on the FCC lattice (Eq. quadratic_local_SRO, shells 12/6/24) ----

Z_FCC = (12, 6, 24)


def _qsro(seed, nsh, S):
    V, W, C = inputs.qsro_coeffs(seed, nsh, S)
    return V, W, C, oracle.Model(oracle.QSRO, nsh, V, qsro_w=W, qsro_c=C)


@pytest.mark.parametrize("nsh", [1, 2, 3])
def test_qsro_without_w_is_a_pair_model(nsh):
    """W = 0: sum_i E_i = N C + sum_m (1/z_m) sum_i sum_{j in shell m} V_m(s_i, s_j),
    the pair energy of the coefficients 2 V_m / z_m (pinned by the closed forms
    above), plus N C."""
    S = 4
    V, W, C, _ = _qsro(nsh, nsh, S)
    m = oracle.Model(oracle.QSRO, nsh, V, qsro_w=np.zeros_like(W), qsro_c=C)
    Vp = np.stack([2.0 * V[k].astype(np.float64) / Z_FCC[k] for k in range(nsh)])
    pair = oracle.Model(oracle.PAIR_F32, nsh, Vp.astype(np.float32))
    lat = oracle.Lattice(4, 5, 3, S)
    N = oracle.fcc_nsites(lat)
    occ = oracle.fcc_init_lattice(lat, inputs.dirichlet_counts(N, S, 3), 4)
    want = oracle.fcc_total_energy(lat, pair, occ) + N * C
    # the pair model holds 2 V / z rounded to FP32: compare at that rounding
    assert oracle.fcc_total_energy(lat, m, occ) == pytest.approx(want, rel=1e-6)


def test_qsro_l12_closed_form():
    """L1_2 (B on sublattice 0): a B site sees 12 A, 6 B, 24 A in shells 1-3
    (pi^{BA} = 1, pi^{BB} = 1, pi^{BA} = 1); an A site 4 B + 8 A, 6 A, 8 B + 16 A
    (pi^{AB} = 1/3, pi^{AA} = 2/3; 1; 1/3, 2/3)."""
    S, A, B = 2, 0, 1
    V, W, C, m = _qsro(11, 3, S)
    V = V.astype(np.float64)
    W = W.astype(np.float64)
    lat = oracle.Lattice(4, 4, 4, S)
    N = oracle.fcc_nsites(lat)
    occ = np.zeros(N, dtype=np.int8)
    occ[: N // 4] = B
    e_b = C + V[0, B, A] + V[1, B, B] + W[1, B] + V[2, B, A]
    e_a = (C + V[0, A, B] / 3 + V[0, A, A] * 2 / 3 + W[0, A] * (2 / 3) ** 2 + V[1, A, A] + W[1, A]
           + V[2, A, B] / 3 + V[2, A, A] * 2 / 3 + W[2, A] * (2 / 3) ** 2)
    assert oracle.fcc_total_energy(lat, m, occ) == pytest.approx(N // 4 * e_b + 3 * N // 4 * e_a, rel=1e-12)


def test_qsro_l10_closed_form():
    """L1_0 (layers along z): every site has 4 like + 8 unlike first
    neighbours, 6 like second, 8 like + 16 unlike third."""
    S = 3
    V, W, C, m = _qsro(12, 3, S)
    V = V.astype(np.float64)
    W = W.astype(np.float64)
    lat = oracle.Lattice(4, 4, 4, S)
    N = oracle.fcc_nsites(lat)
    occ = np.full(N, 2, dtype=np.int8)  # species 2 on sublattices 0-1, 0 on 2-3
    occ[N // 2:] = 0
    tot = 0.0
    for s, o in ((2, 0), (0, 2)):
        hi, lo = max(s, o), min(s, o)
        e = (C + V[0, s, s] / 3 + V[0, hi, lo] * 2 / 3 + W[0, s] / 9 + V[1, s, s] + W[1, s]
             + V[2, s, s] / 3 + V[2, hi, lo] * 2 / 3 + W[2, s] / 9)
        tot += N // 2 * e
    assert oracle.fcc_total_energy(lat, m, occ) == pytest.approx(tot, rel=1e-12)


@pytest.mark.parametrize("nsh,dims", [(1, (4, 5, 3)), (2, (8, 8, 8)), (3, (4, 4, 6))])
def test_qsro_delta_e_is_the_change_of_the_total(nsh, dims):
    S = 5
    V, W, C, m = _qsro(20 + nsh, nsh, S)
    lat = oracle.Lattice(*dims, S)
    occ = oracle.fcc_init_lattice(lat, inputs.dirichlet_counts(oracle.fcc_nsites(lat), S, nsh), 9)
    rng = np.random.default_rng(nsh)
    for _ in range(20):
        a = int(rng.integers(oracle.fcc_nsites(lat)))
        b = oracle.fcc_neighbor(lat, a, oracle.fcc_shell_vectors(1)[rng.integers(12)])
        e0 = oracle.fcc_total_energy(lat, m, occ)
        d = oracle.fcc_delta_e(lat, m, occ, a, b)
        occ[a], occ[b] = occ[b], occ[a]
        assert d == pytest.approx(oracle.fcc_total_energy(lat, m, occ) - e0, abs=1e-10)


def test_qsro_chain_matches_enumeration_8_site():
    """2x1x1 cells, binary 4/4, 2 shells (aliased on this machine): <E> within 3
    batch-means standard errors of the exact canonical average."""
    V, W, C, m = _qsro(31, 2, 2)
    lat = oracle.Lattice(2, 1, 1, 2)
    kT = 0.08  # levels span 0.3 eV
    E = []
    for ones in itertools.combinations(range(8), 4):
        c = np.zeros(8, dtype=np.int8)
        c[list(ones)] = 1
        E.append(oracle.fcc_total_energy(lat, m, c))
    E = np.array(E)
    w = np.exp(-(E - E.min()) / kT)
    exact = (w * E).sum() / w.sum()
    assert E.std() > 0
    occ = np.array([0, 1] * 4, dtype=np.int8)
    nsw = 30000
    Es = np.empty(nsw)
    for t in range(nsw):
        oracle.fcc_sweep(lat, m, occ, 5, t, 1, kT)
        Es[t] = oracle.fcc_total_energy(lat, m, occ)
    nb = 50
    keep = (nsw - nsw // 10) // nb * nb
    bm = Es[nsw - keep:].reshape(nb, -1).mean(1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(bm.mean() - exact) < 3 * se, (bm.mean(), exact, se)
