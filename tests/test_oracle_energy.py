"""Pins of the oracle's energies, dE, pair counts, SRO, MLP and gradients (CPU)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs
from tests import helpers


def _tables(dims, nshells):
    return [helpers.neighbor_table(*dims, m) for m in range(1, nshells + 1)]


def test_total_energy_matches_recompute():
    dims = (8, 8, 8)
    lat = oracle.Lattice(*dims, 5)
    V = inputs.pair_f32_coeffs(7, 2, 5)
    m = oracle.Model(oracle.PAIR_F32, 2, V)
    occ = oracle.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, 5), 3)
    want = helpers.pair_energy(occ, V.astype(np.float64), _tables(dims, 2))
    assert oracle.total_energy(lat, m, occ) == pytest.approx(want, rel=1e-13, abs=1e-12)


def test_delta_e_exhaustive_16_site_binary():
    """Every equiatomic binary configuration of the 2x2x2-cell box (C(16,8) =
    12870), every site, every partner: the Omega-reduced dE equals the full
    recompute E(after) - E(before).  The box aliases shells 2 and 3, which is
    the hardest case for the local-zone bookkeeping."""
    dims = (2, 2, 2)
    lat = oracle.Lattice(*dims, 2)
    V = inputs.pair_int_coeffs(11, 2, 2)
    model = oracle.Model(oracle.PAIR_I32, 2, V, unit_ev=1e-4)
    tabs = _tables(dims, 2)
    s1 = helpers.neighbor_table(*dims, 1)
    confs = []
    for ones in itertools.combinations(range(16), 8):
        c = np.zeros(16, dtype=np.int8)
        c[list(ones)] = 1
        confs.append(c)
    confs = np.array(confs)
    E = helpers.pair_energy(confs, V.astype(np.int64), tabs)
    pairs = [(a, int(s1[a, d])) for a in range(16) for d in range(8)]
    want = np.empty((len(confs), len(pairs)), dtype=np.int64)
    for t, (a, b) in enumerate(pairs):
        sw = confs.copy()
        sw[:, [a, b]] = sw[:, [b, a]]
        want[:, t] = helpers.pair_energy(sw, V.astype(np.int64), tabs) - E
    de = oracle.lib().orc_delta_e
    lat_c, mod_c = oracle.C.byref(lat._c), oracle.C.byref(model._c)
    got = np.empty_like(want)
    for ci in range(len(confs)):
        occ = np.ascontiguousarray(confs[ci])
        p = oracle._ptr(occ, oracle.C.c_int8)
        for t, (a, b) in enumerate(pairs):
            got[ci, t] = de(lat_c, mod_c, p, a, b)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dims,kind", [((8, 8, 8), oracle.PAIR_I32), ((16, 16, 16), oracle.PAIR_I32),
                                       ((8, 8, 8), oracle.PAIR_F32), ((12, 8, 16), oracle.PAIR_F32)])
def test_delta_e_random_trials(dims, kind):
    S = 2 if kind == oracle.PAIR_I32 else 5
    lat = oracle.Lattice(*dims, S)
    if kind == oracle.PAIR_I32:
        V = inputs.pair_int_coeffs(5, 2, S)
        model = oracle.Model(kind, 2, V, unit_ev=1e-4)
        Vd = V.astype(np.int64)
    else:
        V = inputs.pair_f32_coeffs(5, 2, S)
        model = oracle.Model(kind, 2, V)
        Vd = V.astype(np.float64)
    tabs = _tables(dims, 2)
    s1 = helpers.neighbor_table(*dims, 1)
    occ = oracle.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), 9)
    E0 = helpers.pair_energy(occ, Vd, tabs)
    rng = np.random.default_rng(1)
    for _ in range(300):
        a = int(rng.integers(lat.nsites))
        b = int(s1[a, rng.integers(8)])
        sw = occ.copy()
        sw[[a, b]] = sw[[b, a]]
        want = helpers.pair_energy(sw, Vd, tabs) - E0
        got = oracle.delta_e(lat, model, occ, a, b)
        if kind == oracle.PAIR_I32:
            assert got == want
        else:
            assert got == pytest.approx(want, abs=1e-11)


def test_b2_ground_state_energy_closed_form():
    """Perfect B2 (sub 0 = A, sub 1 = B): every first neighbour is unlike and
    every second neighbour like, so E = N (4 V1_AB + 3/2 (V2_AA + V2_BB))."""
    lat = oracle.Lattice(8, 8, 8, 2)
    V = inputs.ordering_coeffs_b2()
    model = oracle.Model(oracle.PAIR_I32, 2, V, unit_ev=1e-4)
    occ = np.zeros(lat.nsites, dtype=np.int8)
    occ[lat.nsites // 2:] = 1
    want = lat.nsites * (4 * V[0, 0, 1] + 1.5 * (V[1, 0, 0] + V[1, 1, 1]))
    assert oracle.total_energy_i64(lat, model, occ) == want
    alpha = oracle.sro(lat, 2, occ)
    assert alpha[0, 0, 1] == -1.0 and alpha[0, 0, 0] == 1.0 and alpha[1, 0, 0] == -1.0


def test_pair_counts_and_sro_definitions():
    dims = (8, 12, 8)
    lat = oracle.Lattice(*dims, 3)
    occ = oracle.init_lattice(lat, [700, 500, lat.nsites - 1200], 4)
    cnt = oracle.pair_counts(lat, 3, occ)
    N = lat.nsites
    Np = np.bincount(occ, minlength=3)
    for m in (1, 2, 3):
        nb = helpers.neighbor_table(*dims, m)
        want = np.zeros((3, 3), dtype=np.int64)
        np.add.at(want, (occ[:, None].repeat(nb.shape[1], 1), occ[nb]), 1)
        assert np.array_equal(cnt[m - 1], want)
        # symmetric, and each row sums to z_m N_p
        assert np.array_equal(cnt[m - 1], cnt[m - 1].T)
        assert np.array_equal(cnt[m - 1].sum(1), helpers.SHELL_Z[m] * Np)
    alpha = oracle.sro(lat, 3, occ)
    c = Np / N
    for m in range(3):
        for p in range(3):
            # sum_q c_q alpha_m^{pq} = 0 (conditional probabilities sum to 1)
            assert abs((c * alpha[m, p]).sum()) < 1e-12


def test_canonical_random_sro_closed_form():
    """Averaged over random permutations with fixed counts,
    E[alpha^{pq}] = -1/(N-1) (p != q) and 1 - N(N_p - 1)/(N_p (N - 1)) (p = q)."""
    lat = oracle.Lattice(4, 4, 4, 2)
    N = lat.nsites
    counts = [40, N - 40]
    samples = np.array([oracle.sro(lat, 2, oracle.init_lattice(lat, counts, seed))[0]
                        for seed in range(3000)])
    mean = samples.mean(0)
    se = samples.std(0, ddof=1) / math.sqrt(len(samples))
    want = np.array([[1 - N * (counts[0] - 1) / (counts[0] * (N - 1)), -1 / (N - 1)],
                     [-1 / (N - 1), 1 - N * (counts[1] - 1) / (counts[1] * (N - 1))]])
    assert np.all(np.abs(mean - want) < 3.5 * se + 1e-12)


def _one_hot_mlp(pick_in, pick_hid1=3, pick_hid2=5, w=(0.5, 0.75, 2.0), b3=0.125):
    """An MLP whose output follows one path: input feature pick_in -> hidden
    unit pick_hid1 -> hidden unit pick_hid2 -> output."""
    w1 = np.zeros((64, 20))
    w2 = np.zeros((64, 64))
    w3 = np.zeros(64)
    w1[pick_hid1, pick_in] = w[0]
    w2[pick_hid2, pick_hid1] = w[1]
    w3[pick_hid2] = w[2]
    return {"w1": w1, "w2": w2, "w3": w3, "b1": np.zeros(64), "b2": np.zeros(64), "b3": b3}


def _silu(z):
    return z / (1 + math.exp(-z))


def test_mlp_wiring_closed_form():
    # with one path the network is b3 + w3 silu(w2 silu(w1 x_t)) + 62*w3*0 ...
    # every other hidden unit gets z = 0 and silu(0) = 0.
    for t in (0, 7, 19):
        model = oracle.Model(oracle.MLP, mlp=_one_hot_mlp(t))
        x = np.arange(20, dtype=np.float64) * 0.25
        want = 0.125 + 2.0 * _silu(0.75 * _silu(0.5 * x[t]))
        assert oracle.mlp_eval(model, x) == pytest.approx(want, rel=1e-15)


def test_mlp_features_on_b2():
    """On perfect B2, a sub-0 site (species 0) has 8 first neighbours of
    species 1, 6 second and 12 third neighbours of species 0.  Reading single
    features through a one-path MLP recovers them."""
    lat = oracle.Lattice(4, 4, 4, 2)
    occ = np.zeros(lat.nsites, dtype=np.int8)
    occ[lat.nsites // 2:] = 1
    want = np.zeros(20)
    want[0] = 1
    want[5 + 1] = 8
    want[10 + 0] = 6
    want[15 + 0] = 12
    for t in range(20):
        model = oracle.Model(oracle.MLP, mlp=_one_hot_mlp(t, w=(1.0, 1.0, 1.0), b3=0.0))
        got = oracle.site_energy(lat, model, occ, 0)
        assert got == pytest.approx(_silu(_silu(want[t])), rel=1e-14, abs=1e-300)


def test_pair_gradient_is_bond_count_and_exact_fd():
    dims = (8, 8, 8)
    lat = oracle.Lattice(*dims, 3)
    V = inputs.pair_f32_coeffs(3, 2, 3)
    model = oracle.Model(oracle.PAIR_F32, 2, V)
    occ = oracle.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, 3), 2)
    g = oracle.energy_grad(lat, model, occ)
    cnt = oracle.pair_counts(lat, 2, occ)
    t = 0
    tabs = _tables(dims, 2)
    for m in range(2):
        for p in range(3):
            for q in range(p, 3):
                want = cnt[m, p, q] if p != q else cnt[m, p, p] / 2
                assert g[t] == want
                # E is linear in V: a finite difference is exact up to rounding
                Vp = V.astype(np.float64).copy()
                Vp[m, p, q] += 1.0
                Vp[m, q, p] = Vp[m, p, q]
                fd = helpers.pair_energy(occ, Vp, tabs) - helpers.pair_energy(occ, V.astype(np.float64), tabs)
                assert fd == pytest.approx(want, abs=1e-8)
                t += 1


def test_mlp_gradient_matches_central_fd():
    lat = oracle.Lattice(4, 4, 4, 5)
    occ = oracle.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, 5), 6)
    base = inputs.mlp_weights(4, out_scale=1.0)
    mlp = {k: oracle._widen(base[k]) for k in ("w1", "w2", "w3", "b1", "b2")}
    mlp["b1"] = np.random.default_rng(0).normal(0, 0.3, 64)
    mlp["b2"] = np.random.default_rng(1).normal(0, 0.3, 64)
    mlp["b3"] = 0.2
    model = oracle.Model(oracle.MLP, mlp=mlp)
    g = oracle.energy_grad(lat, model, occ)
    assert g.size == oracle.MLP_NPARAM
    offsets = {"w1": 0, "b1": 1280, "w2": 1344, "b2": 5440, "w3": 5504}
    rng = np.random.default_rng(2)
    h = 1e-6
    for name, off in offsets.items():
        for idx in rng.choice(mlp[name].size, 6, replace=False):
            mp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in mlp.items()}
            mm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in mlp.items()}
            mp[name][idx] += h
            mm[name][idx] -= h
            fd = (oracle.total_energy(lat, oracle.Model(oracle.MLP, mlp=mp), occ)
                  - oracle.total_energy(lat, oracle.Model(oracle.MLP, mlp=mm), occ)) / (2 * h)
            assert g[off + idx] == pytest.approx(fd, rel=1e-6, abs=1e-7)
    assert g[-1] == lat.nsites  # dE/db3 = N


def test_mlp_delta_e_matches_recompute():
    lat = oracle.Lattice(8, 8, 8, 5)
    model = oracle.Model(oracle.MLP, mlp=inputs.mlp_weights(4))
    occ = oracle.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, 5, 4), 8)
    E0 = oracle.total_energy(lat, model, occ)
    rng = np.random.default_rng(3)
    s1 = oracle.shell_vectors(1)
    for _ in range(10):
        a = int(rng.integers(lat.nsites))
        b = oracle.neighbor(lat, a, s1[rng.integers(8)])
        sw = occ.copy()
        sw[[a, b]] = sw[[b, a]]
        want = oracle.total_energy(lat, model, sw) - E0
        assert oracle.delta_e(lat, model, occ, a, b) == pytest.approx(want, abs=1e-10)


def test_mlp_site_energies_match_numpy_restatement():
    """The oracle's MLP site energies equal an independent numpy evaluation
    (features from brute-force neighbour vectors, the network as matrix
    products) on a random quinary lattice, with biases switched on; a wrong
    feature column, shell or activation would show here."""
    dims, S = (8, 12, 8), 5
    lat = oracle.Lattice(*dims, S)
    rng = np.random.default_rng(7)
    occ = rng.integers(0, S, lat.nsites).astype(np.int8)
    mlp = inputs.mlp_weights(9, out_scale=1.0)
    mlp["b1"] = rng.normal(0, 0.3, 64).astype(np.float32)
    mlp["b2"] = rng.normal(0, 0.3, 64).astype(np.float32)
    mlp["b3"] = 0.25
    model = oracle.Model(oracle.MLP, mlp=mlp)
    w = {k: oracle._widen(mlp[k]).reshape(64, -1) if k in ("w1", "w2") else oracle._widen(mlp[k])
         for k in ("w1", "w2", "w3", "b1", "b2")}
    w["b3"] = 0.25
    sites = rng.choice(lat.nsites, 300, replace=False)
    _, f = helpers.mlp_error_bound(helpers.mlp_features(occ, dims, sites), w)
    got = np.array([oracle.site_energy(lat, model, occ, int(i)) for i in sites])
    assert np.allclose(got, f, rtol=1e-12, atol=1e-14)
    # Omega has 40 sites, and dE is the sum of the energy changes over it
    a = int(sites[0])
    b = oracle.neighbor(lat, a, oracle.shell_vectors(1)[3])
    om = helpers.omega(a, b, dims)
    assert om.size == 40
    _, f0 = helpers.mlp_error_bound(helpers.mlp_features(occ, dims, om), w)
    _, f1 = helpers.mlp_error_bound(helpers.mlp_features(occ, dims, om, swap=(a, b)), w)
    assert oracle.delta_e(lat, model, occ, a, b) == pytest.approx(f1.sum() - f0.sum(), rel=1e-10, abs=1e-13)
