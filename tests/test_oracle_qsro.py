"""Pins of the oracle's qSRO model (Sec. IV-B, Eq. quadratic_local_SRO) on CPU.

E_i = sum_{m, p'<=p} V_m^{pp'} pi_m^{pp'} + sum_{m,p} W_m^p (pi_m^{pp})^2 + C,
pi_m^{pp'} = n_m^{pp'} / z_m over the pairs (i, j), j in shell m of i.

* Without the quadratic term and C the model is the pair model with
  coefficients 2 V_m / z_m (a site's pairs counted from both ends against the
  pair model's 1/2 per site), whose oracle is pinned by enumeration and B2.
* Closed forms on three orderings: a pure element (pi^{ss} = 1 in every
  shell), B2 (shell 1 all unlike, shells 2 and 3 all like), and lamellae of
  one cell along x (pi^{ss} = 1/2, 2/3, 1/3 in shells 1, 2, 3), which weigh
  the quadratic term at fractional arguments.
* Every incremental dE equals the change of the total energy.
* A chain on the 16-site binary lattice samples the enumerated Boltzmann
  distribution of the model.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs
from tests import helpers

Z = (8, 6, 12)  # coordination numbers of shells 1-3 of BCC


def _exact_v(seed, nsh, S):
    """Symmetric V whose 2 V / z_m are exact in FP32 (V multiple of z_m/2 x 2^-12)."""
    rng = np.random.default_rng(seed)
    V = np.zeros((nsh, S, S), dtype=np.float32)
    for m in range(nsh):
        k = rng.integers(-40, 41, size=(S, S))
        k = np.triu(k) + np.triu(k, 1).T
        V[m] = (k * (Z[m] // 2) * 2.0 ** -12).astype(np.float32)
    return V


@pytest.mark.parametrize("nsh", [1, 2, 3])
def test_linear_part_is_the_pair_model(nsh):
    S = 4
    V = _exact_v(nsh, nsh, S)
    Vp = np.stack([2.0 * V[m] / Z[m] for m in range(nsh)]).astype(np.float32)
    assert np.array_equal(Vp.astype(np.float64) * np.array(Z[:nsh])[:, None, None] / 2, V.astype(np.float64))
    lat = oracle.Lattice(6, 4, 5, S)
    q = oracle.Model(oracle.QSRO, nsh, V, qsro_w=np.zeros((nsh, S), np.float32), qsro_c=0.0)
    p = oracle.Model(oracle.PAIR_F32, nsh, Vp)
    rng = np.random.default_rng(3)
    for seed in range(3):
        occ = oracle.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, S, seed), seed)
        eq, ep = oracle.total_energy(lat, q, occ), oracle.total_energy(lat, p, occ)
        assert eq == pytest.approx(ep, rel=1e-12, abs=1e-12)
        for _ in range(20):
            a = int(rng.integers(lat.nsites))
            v = oracle.shell_vectors(1)[rng.integers(8)]
            b = oracle.neighbor(lat, a, v)
            assert oracle.delta_e(lat, q, occ, a, b) == pytest.approx(oracle.delta_e(lat, p, occ, a, b),
                                                                      rel=1e-12, abs=1e-12)


def _model(nsh, S, seed=7):
    V, W, C = inputs.qsro_coeffs(seed, nsh, S)
    return V, W, C, oracle.Model(oracle.QSRO, nsh, V, qsro_w=W, qsro_c=C)


@pytest.mark.parametrize("nsh", [1, 2, 3])
def test_pure_element(nsh):
    S = 3
    V, W, C, m = _model(nsh, S)
    lat = oracle.Lattice(4, 4, 4, S)
    occ = np.zeros(lat.nsites, dtype=np.int8)
    want = lat.nsites * (sum(float(V[k, 0, 0]) + float(W[k, 0]) for k in range(nsh)) + C)
    assert oracle.total_energy(lat, m, occ) == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("nsh", [1, 2, 3])
def test_b2(nsh):
    """Sublattice 0 species 0, sublattice 1 species 1: a site's shell-1
    neighbours are all unlike, its shell-2 and shell-3 neighbours all like."""
    S = 2
    V, W, C, m = _model(nsh, S)
    lat = oracle.Lattice(4, 4, 4, S)
    N = lat.nsites
    occ = np.repeat(np.array([0, 1], dtype=np.int8), N // 2)
    per = {}
    for s in (0, 1):
        e = float(V[0, s, 1 - s]) + C
        for k in range(1, nsh):
            e += float(V[k, s, s]) + float(W[k, s])
        per[s] = e
    assert oracle.total_energy(lat, m, occ) == pytest.approx(N / 2 * (per[0] + per[1]), rel=1e-13)


@pytest.mark.parametrize("nsh", [1, 2, 3])
def test_lamellae_along_x(nsh):
    """Species = cell x mod 2 on both sublattices.  Shell 1 (+-1/2 along x):
    4 like, 4 unlike; shell 2: the 2 neighbours along x unlike, 4 like;
    shell 3 ((110) family): the 8 with an x component unlike, 4 like."""
    S = 2
    V, W, C, m = _model(nsh, S, seed=11)
    lat = oracle.Lattice(4, 4, 4, S)
    x = np.arange(lat.nsites) % lat.nx
    occ = (x % 2).astype(np.int8)
    like = (4 / 8, 4 / 6, 4 / 12)
    per = {}
    for s in (0, 1):
        o = 1 - s
        e = C
        for k in range(nsh):
            e += float(V[k, s, s]) * like[k] + float(V[k, s, o]) * (1 - like[k]) + float(W[k, s]) * like[k] ** 2
        per[s] = e
    want = lat.nsites / 2 * (per[0] + per[1])
    assert oracle.total_energy(lat, m, occ) == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("nsh", [1, 2, 3])
def test_delta_e_is_the_change_of_the_total(nsh):
    S = 5
    V, W, C, m = _model(nsh, S, seed=3)
    lat = oracle.Lattice(5, 4, 6, S)
    occ = oracle.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, S, 2), 2)
    rng = np.random.default_rng(nsh)
    for _ in range(40):
        a = int(rng.integers(lat.nsites))
        v = oracle.shell_vectors(1)[rng.integers(8)]
        b = oracle.neighbor(lat, a, v)
        e0 = oracle.total_energy(lat, m, occ)
        d = oracle.delta_e(lat, m, occ, a, b)
        occ[a], occ[b] = occ[b], occ[a]
        e1 = oracle.total_energy(lat, m, occ)
        assert d == pytest.approx(e1 - e0, abs=1e-10)


def test_chain_matches_enumeration_16_site():
    """<E> of the chain on the 2x2x2-cell binary lattice (8 + 8 sites) within
    3 batch-means standard errors of the exact canonical average."""
    S, nsh, kT = 2, 2, 0.05
    V, W, C = inputs.qsro_coeffs(21, nsh, S, sigma_v_ev=0.04, sigma_w_ev=0.04, c_ev=0.0)
    m = oracle.Model(oracle.QSRO, nsh, V, qsro_w=W, qsro_c=C)
    lat = oracle.Lattice(2, 2, 2, S)
    E = []
    for ones in itertools.combinations(range(16), 8):
        c = np.zeros(16, dtype=np.int8)
        c[list(ones)] = 1
        E.append(oracle.total_energy(lat, m, c))
    E = np.array(E)
    w = np.exp(-(E - E.min()) / kT)
    exact = (w * E).sum() / w.sum()
    occ = oracle.init_lattice(lat, [8, 8], 4)
    nsw = 20000
    Es = np.empty(nsw)
    for t in range(nsw):
        oracle.sweep(lat, m, occ, 9, t, 1, kT)
        Es[t] = oracle.total_energy(lat, m, occ)
    nb = 40
    keep = (nsw - nsw // 10) // nb * nb
    bm = Es[nsw - keep:].reshape(nb, -1).mean(1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(bm.mean() - exact) < 3 * se, (bm.mean(), exact, se)


def test_gradient_equals_finite_differences():
    """E is linear in every qSRO parameter, so central differences over the
    FP32-representable perturbation are exact up to rounding.  Layout:
    [V_m^{pq}, p <= q][W_m^p][C]."""
    S, nsh = 3, 3
    V, W, C = inputs.qsro_coeffs(5, nsh, S)
    lat = oracle.Lattice(4, 4, 5, S)
    occ = oracle.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, S, 1), 1)
    g = oracle.energy_grad(lat, oracle.Model(oracle.QSRO, nsh, V, qsro_w=W, qsro_c=C), occ)
    per = S * (S + 1) // 2
    assert g.size == nsh * per + nsh * S + 1

    def energy(V_, W_, C_):
        return oracle.total_energy(lat, oracle.Model(oracle.QSRO, nsh, V_, qsro_w=W_, qsro_c=C_), occ)

    h = np.float32(2.0 ** -6)
    i = 0
    for m in range(nsh):
        for p in range(S):
            for q in range(p, S):
                Vp, Vm = V.copy(), V.copy()
                Vp[m, p, q] = Vp[m, q, p] = V[m, p, q] + h
                Vm[m, p, q] = Vm[m, q, p] = V[m, p, q] - h
                fd = (energy(Vp, W, C) - energy(Vm, W, C)) / (float(Vp[m, p, q]) - float(Vm[m, p, q]))
                assert g[i] == pytest.approx(fd, rel=1e-9, abs=1e-9), (m, p, q)
                i += 1
    for m in range(nsh):
        for p in range(S):
            Wp, Wm = W.copy(), W.copy()
            Wp[m, p] += h
            Wm[m, p] -= h
            fd = (energy(V, Wp, C) - energy(V, Wm, C)) / (float(Wp[m, p]) - float(Wm[m, p]))
            assert g[i] == pytest.approx(fd, rel=1e-9, abs=1e-9), (m, p)
            i += 1
    assert g[i] == lat.nsites


@pytest.mark.parametrize("nsh,others", [(1, 14), (2, 20), (3, 38)])
def test_a_swap_changes_site_energies_only_in_its_zone(nsh, others):
    """Swapping a with a first-shell partner b changes the qSRO site energy
    of a, b and of sites that hold a or b within the model's shells, and of
    no other site.  Those sites number 14 / 20 / 38 besides a and b for 1 / 2
    / 3 shells, and none holds a and b in one shell (a and b lie on different
    sublattices, shells 1 and 2-3 join different and equal sublattices)."""
    dims, S = (8, 8, 8), 5
    lat = oracle.Lattice(*dims, S)
    V, W, C = inputs.qsro_coeffs(21 + nsh, nsh, S)
    model = oracle.Model(oracle.QSRO, nsh, V, qsro_w=W, qsro_c=C)
    tabs = [helpers.neighbor_table(*dims, m) for m in range(1, nsh + 1)]
    rng = np.random.default_rng(nsh)
    occ = rng.integers(0, S, size=lat.nsites).astype(np.int8)
    for a in (0, 517, lat.nsites - 1):
        for b in tabs[0][a]:
            b = int(b)
            shell_of = [{int(j): m for m, t in enumerate(tabs) for j in t[s]} for s in (a, b)]
            assert not any(shell_of[0][j] == shell_of[1][j] for j in set(shell_of[0]) & set(shell_of[1]))
            zone = (set(shell_of[0]) | set(shell_of[1])) - {a, b}
            assert len(zone) == others
            o = occ.copy()
            o[b] = (o[a] + 1) % S  # a and b differ
            before = np.array([oracle.site_energy(lat, model, o, i) for i in range(lat.nsites)])
            o[a], o[b] = o[b], o[a]
            after = np.array([oracle.site_energy(lat, model, o, i) for i in range(lat.nsites)])
            changed = set(np.nonzero(before != after)[0].tolist())
            assert changed <= zone | {a, b}
            assert {a, b} <= changed


def _strict_form_total(occ, V, W, C, tables):
    """Eq. quadratic_local_SRO as the paper prints it: the linear sum over
    p' < p, i.e. over the pairs (i, j) of unlike species only, each with
    weight V_m^{s_i s_j} / z_m; the quadratic term W_m^{s_i} (pi_m^{ss})^2
    with pi_m^{ss} the fraction of i's shell-m neighbours of i's own species;
    C per site.  Written from the equation with brute-force neighbour tables,
    independently of the oracle."""
    occ = np.asarray(occ).astype(np.int64)
    E = len(occ) * float(C)
    for m, nb in enumerate(tables):
        z = nb.shape[1]
        si, sj = occ[:, None], occ[nb]
        E += float((V[m].astype(np.float64)[si, sj] * (sj != si)).sum()) / z
        E += float((W[m].astype(np.float64)[occ] * ((sj == si).sum(1) / z) ** 2).sum())
    return E


def _fcc_tables(dims, nsh):
    from tests.test_oracle_fcc import brute_shells
    sh = brute_shells(dims)
    return [np.array([sorted(s) for s in sh[m]]) for m in range(1, nsh + 1)]


@pytest.mark.parametrize("lattice", ["bcc", "fcc"])
@pytest.mark.parametrize("nsh", [1, 2, 3])
@pytest.mark.parametrize("with_w", [False, True])
def test_linear_sum_is_the_strict_form_reparametrised(lattice, nsh, with_w):
    """The oracle sums the linear qSRO term over p' <= p with a full
    symmetric V.  The paper's sum runs over p' < p.  The two describe the same
    model: with V'^{pq} = V^{pq} - (V^{pp} + V^{qq}) / 2 (zero diagonal),
    E_oracle(V) = E_strict(V') + sum_m sum_p N_p V_m^{pp}, a constant at fixed
    composition, so every dE of the oracle is the strict form's dE with V'.
    Checked on totals and swaps, BCC and FCC, with and without the W term."""
    S = 4
    V, W, C = inputs.qsro_coeffs(40 + nsh, nsh, S)
    if not with_w:
        W = np.zeros_like(W)
    V64 = V.astype(np.float64)
    d = np.stack([np.diag(V64[m]) for m in range(nsh)])
    Vs = V64 - (d[:, :, None] + d[:, None, :]) / 2.0
    if lattice == "bcc":
        dims = (4, 4, 6)
        lat = oracle.Lattice(*dims, S)
        N = lat.nsites
        tables = [helpers.neighbor_table(*dims, m) for m in range(1, nsh + 1)]
        total, dE = oracle.total_energy, oracle.delta_e
        occ = oracle.init_lattice(lat, inputs.dirichlet_counts(N, S, nsh), nsh)
        first = tables[0]
    else:
        dims = (4, 4, 4)
        lat = oracle.Lattice(*dims, S)
        N = oracle.fcc_nsites(lat)
        tables = _fcc_tables(dims, nsh)
        total, dE = oracle.fcc_total_energy, oracle.fcc_delta_e
        occ = oracle.fcc_init_lattice(lat, inputs.dirichlet_counts(N, S, nsh), nsh)
        first = tables[0]
    model = oracle.Model(oracle.QSRO, nsh, V, qsro_w=W, qsro_c=C)
    Np = np.bincount(occ, minlength=S)
    const = float((d * Np[None, :]).sum())
    scale = float(np.abs(V64).max()) * N
    e_or = total(lat, model, occ)
    assert e_or == pytest.approx(_strict_form_total(occ, Vs, W, C, tables) + const, rel=1e-12, abs=1e-12 * scale)
    rng = np.random.default_rng(nsh + 10 * with_w)
    for _ in range(12):
        a = int(rng.integers(N))
        b = int(first[a][rng.integers(first.shape[1])])
        if occ[a] == occ[b]:
            continue
        d_or = dE(lat, model, occ, a, b)
        e0 = _strict_form_total(occ, Vs, W, C, tables)
        occ[a], occ[b] = occ[b], occ[a]
        e1 = _strict_form_total(occ, Vs, W, C, tables)
        assert d_or == pytest.approx(e1 - e0, rel=1e-10, abs=1e-12)
