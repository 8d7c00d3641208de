"""Pins of the oracle's Monte Carlo chain (CPU): Algorithm 1 as printed vs the
serial form, exact Boltzmann enumeration, infinite temperature, B2 ordering,
composition, resume, acceptance tables."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs
from tests import helpers


def _cfg1():
    lat = oracle.Lattice(8, 8, 8, 2)
    V = inputs.pair_int_coeffs(1, 2, 2)
    return lat, oracle.Model(oracle.PAIR_I32, 2, V, unit_ev=1e-4)


def test_accept_table_properties():
    unit, kT = 1e-4, 0.025
    T = oracle.accept_table(unit, kT)
    assert T[0] == 2 ** 29
    assert np.all(np.diff(T.astype(np.int64)) <= 0)
    # length: the first d with 2^29 exp(-d/250) < 1, i.e. d > 250 ln 2^29
    assert len(T) == math.floor(250 * 29 * math.log(2)) + 1
    for d in (1, 17, 250, 3000, len(T) - 1):
        assert T[d] == math.floor(2 ** 29 * math.exp(-d * unit / kT))


@pytest.mark.parametrize("kind", [oracle.PAIR_I32, oracle.PAIR_F32])
def test_serial_equals_algorithm1_literal(kind):
    """Algorithm 1 as printed (auxiliary lattice, local energies of every site
    before and after, reduction over Omega, masked copy) and the serial
    in-place oracle give identical trajectories."""
    if kind == oracle.PAIR_I32:
        lat, model = _cfg1()
        S, kT = 2, 0.025
    else:
        lat = oracle.Lattice(8, 8, 12, 5)
        model = oracle.Model(kind, 2, inputs.pair_f32_coeffs(2, 2, 5))
        S, kT = 5, 0.06
    occ0 = oracle.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), 5)
    a, b = occ0.copy(), occ0.copy()
    ea, na = oracle.sweep(lat, model, a, 1, 0, 3, kT, mode=0)
    eb, nb = oracle.sweep(lat, model, b, 1, 0, 3, kT, mode=1)
    assert np.array_equal(a, b) and na == nb
    assert ea == pytest.approx(eb, abs=1e-9)


def test_serial_equals_algorithm1_literal_mlp():
    lat = oracle.Lattice(8, 8, 8, 5)
    model = oracle.Model(oracle.MLP, mlp=inputs.mlp_weights(4))
    occ0 = oracle.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, 5, 4), 5)
    a = occ0.copy()
    b = occ0.copy()
    kT = inputs.K_B_EV * 800
    oracle.sweep(lat, model, a, 1, 0, 1, kT, mode=0)
    oracle.sweep(lat, model, b, 1, 0, 1, kT, mode=1)
    assert np.array_equal(a, b)


def test_composition_and_energy_bookkeeping():
    lat, model = _cfg1()
    occ = oracle.init_lattice(lat, [512, 512], 1)
    E0 = oracle.total_energy_i64(lat, model, occ)
    e, n = oracle.sweep(lat, model, occ, 1, 0, 20, 0.025)
    assert np.array_equal(np.bincount(occ, minlength=2), [512, 512])
    assert E0 + e == oracle.total_energy_i64(lat, model, occ)
    assert 0 < n < 20 * lat.nsites


def test_resume_is_exact():
    lat, model = _cfg1()
    a = oracle.init_lattice(lat, [512, 512], 1)
    b = a.copy()
    ea, na = oracle.sweep(lat, model, a, 1, 0, 40, 0.025)
    eb1, nb1 = oracle.sweep(lat, model, b, 1, 0, 20, 0.025)
    c = b.copy()  # checkpoint = occupancy + next sweep index
    eb2, nb2 = oracle.sweep(lat, model, c, 1, 20, 20, 0.025)
    assert np.array_equal(a, c) and na == nb1 + nb2 and ea == eb1 + eb2


def test_infinite_temperature_accepts_everything():
    lat = oracle.Lattice(8, 8, 8, 5)
    model = oracle.Model(oracle.PAIR_F32, 2, inputs.pair_f32_coeffs(2, 2, 5))
    occ = oracle.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, 5), 2)
    _, n = oracle.sweep(lat, model, occ, 1, 0, 4, math.inf)
    assert n == 4 * lat.nsites


def test_infinite_temperature_sro_closed_form():
    """At beta = 0 the chain samples uniform permutations with fixed counts;
    alpha_1 averaged over sweeps matches the canonical-random closed form."""
    lat = oracle.Lattice(4, 4, 4, 2)
    N = lat.nsites
    counts = [48, N - 48]
    model = oracle.Model(oracle.PAIR_F32, 2, np.zeros((2, 2, 2), np.float32))
    occ = oracle.init_lattice(lat, counts, 3)
    vals = []
    for t in range(4000):
        oracle.sweep(lat, model, occ, 7, t, 1, math.inf)
        vals.append(oracle.sro(lat, 1, occ)[0])
    vals = np.array(vals)
    nb = 40  # batch means
    bm = vals.reshape(nb, -1, 2, 2).mean(1)
    mean, se = bm.mean(0), bm.std(0, ddof=1) / math.sqrt(nb)
    want = np.array([[1 - N * (counts[0] - 1) / (counts[0] * (N - 1)), -1 / (N - 1)],
                     [-1 / (N - 1), 1 - N * (counts[1] - 1) / (counts[1] * (N - 1))]])
    assert np.all(np.abs(mean - want) < 3 * se + 1e-12)


def _enumerate_16(V):
    dims = (2, 2, 2)
    tabs = [helpers.neighbor_table(*dims, m) for m in (1, 2)]
    confs = []
    for ones in itertools.combinations(range(16), 8):
        c = np.zeros(16, dtype=np.int8)
        c[list(ones)] = 1
        confs.append(c)
    confs = np.array(confs)
    E = helpers.pair_energy(confs, V.astype(np.int64), tabs)
    n01 = ((confs[:, :, None] == 0) & (confs[:, tabs[0]] == 1)).sum((1, 2))
    alpha = 1.0 - n01 / (16 * 0.5 * 8 * 0.5)
    return confs, E, alpha


@pytest.mark.parametrize("kT", [0.010, 0.025, 0.100])
def test_boltzmann_enumeration_16_site(kT):
    """Exact averages over all C(16,8) states vs the MC chain: <E> and
    <alpha_1^{01}> within 3 batch-means standard errors.  Coefficients within
    +-10 meV keep the chain mixing at 10 meV (with +-50 meV it freezes into a
    local minimum on this time scale)."""
    V = inputs.pair_int_coeffs(1, 2, 2, lo=-100, hi=100)
    confs, E, alpha = _enumerate_16(V)
    w = np.exp(-(E - E.min()) * 1e-4 / kT)
    Z = w.sum()
    E_exact = (w * E).sum() / Z
    a_exact = (w * alpha).sum() / Z
    lat = oracle.Lattice(2, 2, 2, 2)
    model = oracle.Model(oracle.PAIR_I32, 2, V, unit_ev=1e-4)
    occ = oracle.init_lattice(lat, [8, 8], 11)
    Ecur = oracle.total_energy_i64(lat, model, occ)
    nsw = 25000
    Es = np.empty(nsw)
    As = np.empty(nsw)
    for t in range(nsw):
        e, _ = oracle.sweep(lat, model, occ, 5, t, 1, kT)
        Ecur += e
        Es[t] = Ecur
        As[t] = oracle.sro(lat, 1, occ)[0, 0, 1]
    assert Ecur == oracle.total_energy_i64(lat, model, occ)
    nb = 50
    for series, exact in ((Es, E_exact), (As, a_exact)):
        keep = (nsw - nsw // 10) // nb * nb
        bm = series[nsw - keep:].reshape(nb, -1).mean(1)
        se = bm.std(ddof=1) / math.sqrt(nb)
        assert abs(bm.mean() - exact) < 3 * se + 1e-9 * abs(exact), (bm.mean(), exact, se)


def test_b2_ordering_reached_by_annealing():
    """Binary ordering interactions: an anneal orders the lattice into B2
    (CsCl).  Swap dynamics can trap isolated antisite pairs (a B on the A
    sublattice and an A on the B sublattice) at low T; each isolated antisite
    turns 8 first-neighbour bonds like and 6 second-neighbour bonds unlike, so
    E = E_B2 + n_anti (8 (V1_AA - V1_AB) + 6 (V2_AB - V2_AA)) with
    E_B2 = N (4 V1_AB + 3/2 (V2_AA + V2_BB))."""
    V = inputs.ordering_coeffs_b2()
    model = oracle.Model(oracle.PAIR_I32, 2, V, unit_ev=1e-4)
    per_anti = 8 * (V[0, 0, 0] - V[0, 0, 1]) + 6 * (V[1, 0, 1] - V[1, 0, 0])
    lat = oracle.Lattice(4, 4, 4, 2)
    N = lat.nsites
    nb = np.concatenate([helpers.neighbor_table(4, 4, 4, m) for m in (1, 2)], axis=1)
    E_b2 = N * (4 * V[0, 0, 1] + 1.5 * (V[1, 0, 0] + V[1, 1, 1]))
    for seed in (1, 2, 3):
        occ = oracle.init_lattice(lat, [N // 2, N // 2], seed)
        nsw = 500
        oracle.sweep(lat, model, occ, seed, 0, nsw, np.geomspace(0.1, 0.004, nsw))
        major = int(round(occ[: N // 2].mean()))  # species that fills sublattice 0
        anti = np.nonzero(np.concatenate([occ[: N // 2] != major, occ[N // 2:] == major]))[0]
        assert len(anti) <= 4, len(anti)
        isolated = all(len(set(nb[a]) & set(anti)) == 0 for a in anti)
        if isolated:
            assert oracle.total_energy_i64(lat, model, occ) == E_b2 + len(anti) * per_anti


def test_init_lattice_properties():
    lat = oracle.Lattice(8, 4, 6, 3)
    counts = [150, 100, lat.nsites - 250]
    a = oracle.init_lattice(lat, counts, 42)
    assert np.array_equal(np.bincount(a, minlength=3), counts)
    assert np.array_equal(a, oracle.init_lattice(lat, counts, 42))
    assert not np.array_equal(a, oracle.init_lattice(lat, counts, 43))
    assert not np.array_equal(a, oracle.init_lattice(lat, counts, 42, replica=1))
    # every site is equally likely to hold each species
    freq = np.mean([oracle.init_lattice(lat, counts, s) == 0 for s in range(400)], axis=0)
    c0 = counts[0] / lat.nsites
    assert abs(freq.mean() - c0) < 1e-12
    assert np.abs(freq - c0).max() < 5 * math.sqrt(c0 * (1 - c0) / 400)
    with pytest.raises(ValueError):
        oracle.init_lattice(lat, [1, 2, 3], 1)
