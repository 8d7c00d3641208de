"""GPU parity of the FCC lattice (Sec. IV-C; 4x4x4 link cells, 256
mini-steps as in Sec. V-C) with pair models against the CPU oracle, through
the C ABI.

Integer models: the start state, trajectories, accepted counts, accepted
energy sums and total energies bit-exact.  FP32 models: every trial's dE
within DE_TOL_EV of the FP64 oracle and the same decision, mini-step by
mini-step (lock-step; after a decision flip the GPU continues from the oracle's state); the sweep
equals its traced mini-steps bit for bit; energies from exact pair counts in
FP64."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DE_TOL_EV = 1e-5  # FP32 dE vs FP64


@pytest.fixture(scope="module")
def smc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08250_gb300 import build, smc as s
    build.build()
    s.lib()
    return s


def dev():
    return torch.device("cuda:0")


def _state(smc, dims, S, seed, counts=None):
    lat = smc.Lattice(*dims, S)
    N = smc.fcc_nsites(lat)
    counts = inputs.equiatomic_counts(N, S) if counts is None else counts
    olat = oracle.Lattice(*dims, S)
    if min(dims[1:]) >= 2:
        occ = torch.empty(N, dtype=torch.int8, device=dev())
        smc.fcc_init_lattice(lat, counts, seed, occ)
        ref = oracle.fcc_init_lattice(olat, counts, seed)
    else:  # the start-state order needs ny, nz >= 2: a seeded permutation instead
        ref = np.random.default_rng(seed).permutation(np.repeat(np.arange(S), counts)).astype(np.int8)
        occ = torch.from_numpy(ref.copy()).to(dev())
    return lat, occ, olat, ref


@pytest.mark.parametrize("dims,S", [((8, 8, 8), 2), ((12, 8, 16), 5), ((3, 5, 2), 8)])
def test_init_matches_oracle(smc, dims, S):
    counts = inputs.dirichlet_counts(4 * dims[0] * dims[1] * dims[2], S, 4)
    lat, occ, olat, ref = _state(smc, dims, S, 6, counts)
    assert np.array_equal(occ.cpu().numpy(), ref)
    assert np.array_equal(np.bincount(ref, minlength=S), counts)


@pytest.mark.parametrize("dims,S,nsh,nsw", [((8, 8, 8), 2, 1, 3), ((12, 8, 16), 5, 2, 2), ((16, 16, 16), 8, 3, 1),
                                            ((8, 12, 8), 3, 3, 2), ((24, 24, 24), 5, 3, 1), ((28, 20, 24), 4, 2, 1)])
def test_int_trajectory_bit_exact(smc, dims, S, nsh, nsw):
    """Boxes of 2 link cells per axis run on the face path only; 24^3 and
    28 x 20 x 24 put most trials on the interior path."""
    V = inputs.pair_int_coeffs(nsh + S, nsh, S)
    lat, occ, olat, ref = _state(smc, dims, S, 2)
    model = smc.Model(smc.PAIR_I32, nsh, V, unit_ev=1e-4)
    omodel = oracle.Model(oracle.PAIR_I32, nsh, V, unit_ev=1e-4)
    kT = inputs.ladder_kT(nsw, 300.0, 1500.0) if nsw > 1 else [0.05]
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    e0 = oracle.fcc_total_energy_i64(olat, omodel, ref)
    smc.fcc_sweep(lat, model, occ, 7, 3, nsw, kT, e_acc=e_acc, n_acc=n_acc)
    oe, on = oracle.fcc_sweep(olat, omodel, ref, 7, 3, nsw, kT)
    smc.check()
    assert np.array_equal(occ.cpu().numpy(), ref)
    assert int(n_acc.item()) == on and on > 0
    assert float(e_acc.item()) == oe
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    e_int = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.fcc_energy(lat, model, occ, e=e, e_int=e_int)
    assert int(e_int.item()) == oracle.fcc_total_energy_i64(olat, omodel, ref) == e0 + int(oe)
    assert float(e.item()) == pytest.approx(int(e_int.item()) * 1e-4, rel=1e-15)


@pytest.mark.parametrize("dims", [(12, 8, 8), (1040, 8, 8), (1032, 8, 12)])
def test_int_trace_matches_oracle_per_trial(smc, dims):
    """dE, decision and the resulting state of single mini-steps, on boxes
    with 2, 260 and 258 link cells along x."""
    S, nsh = 4, 3
    V = inputs.pair_int_coeffs(21, nsh, S)
    lat, occ, olat, ref = _state(smc, dims, S, 5)
    model = smc.Model(smc.PAIR_I32, nsh, V, unit_ev=1e-4)
    omodel = oracle.Model(oracle.PAIR_I32, nsh, V, unit_ev=1e-4)
    nt = oracle.fcc_nsites(olat) // 256
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    for k in (0, 1, 63, 64, 130, 255):
        smc.fcc_ministep_trace(lat, model, occ, 11, 4, k, 0.04, dE=dE, acc=acc)
        odE, oacc, _, _ = oracle.fcc_ministep_trace(olat, omodel, ref, 11, 4, k, 0.04)
        assert np.array_equal(dE.cpu().numpy().astype(np.float64), odE)
        assert np.array_equal(acc.cpu().numpy().astype(bool), oacc)
        assert np.array_equal(occ.cpu().numpy(), ref)


@pytest.mark.parametrize("dims,kT", [((8, 8, 8), 0.05), ((12, 8, 16), 0.03)])
def test_f32_lockstep_against_oracle(smc, dims, kT):
    S, nsh = 5, 3
    V = inputs.pair_f32_coeffs(8, nsh, S)
    lat, occ, olat, ref = _state(smc, dims, S, 3)
    model = smc.Model(smc.PAIR_F32, nsh, V)
    omodel = oracle.Model(oracle.PAIR_F32, nsh, V)
    nt = oracle.fcc_nsites(olat) // 256
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    flips, worst = 0, 0.0
    for k in range(256):
        smc.fcc_ministep_trace(lat, model, occ, 9, 0, k, kT, dE=dE, acc=acc)
        odE, oacc, _, _ = oracle.fcc_ministep_trace(olat, omodel, ref, 9, 0, k, kT)
        g = dE.cpu().numpy().astype(np.float64)
        worst = max(worst, float(np.abs(g - odE).max()))
        assert np.all(np.abs(g - odE) <= DE_TOL_EV)
        ga = acc.cpu().numpy().astype(bool)
        if not np.array_equal(ga, oacc):  # the GPU continues from the oracle's state
            flips += int((ga != oacc).sum())
            occ.copy_(torch.from_numpy(ref.copy()).to(dev()))
        else:
            assert np.array_equal(occ.cpu().numpy(), ref)
    assert flips <= 1, flips
    assert worst < 1e-6


def test_f32_sweep_equals_trace_and_energy_closes(smc):
    dims, S, nsh = (8, 16, 12), 6, 2
    V = inputs.pair_f32_coeffs(4, nsh, S)
    lat, occ, olat, ref = _state(smc, dims, S, 8)
    model = smc.Model(smc.PAIR_F32, nsh, V)
    omodel = oracle.Model(oracle.PAIR_F32, nsh, V)
    occ2 = occ.clone()
    kT = [0.05, 0.08]
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.fcc_sweep(lat, model, occ, 4, 10, 2, kT, e_acc=e_acc, n_acc=n_acc)
    for t in range(2):
        for k in range(256):
            smc.fcc_ministep_trace(lat, model, occ2, 4, 10 + t, k, kT[t])
    smc.check()
    assert torch.equal(occ, occ2)
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.fcc_energy(lat, model, occ, e=e)
    # each accepted dE: 84 FP32 terms of |.| <= 2 max|V|; errors add like a random walk
    n = int(n_acc.item())
    tol = 6 * math.sqrt(max(n, 1)) * 84 * 2.0 ** -24 * 84 * 2 * float(np.abs(V).max())
    assert abs(float(e.item()) - (oracle.fcc_total_energy(olat, omodel, ref) + float(e_acc.item()))) <= tol


@pytest.mark.parametrize("dims,S,nsh,kind", [((4, 5, 3), 3, 3, "int"), ((2, 1, 1), 2, 2, "f32"),
                                             ((16, 8, 24), 8, 3, "f32"), ((1, 1, 1), 4, 1, "int")])
def test_energy_matches_oracle(smc, dims, S, nsh, kind):
    """Any box, including ones too small to sweep (shells alias)."""
    lat, occ, olat, ref = _state(smc, dims, S, 12, inputs.dirichlet_counts(4 * dims[0] * dims[1] * dims[2], S, 1))
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    if kind == "int":
        V = inputs.pair_int_coeffs(2, nsh, S)
        e_int = torch.zeros(1, dtype=torch.int64, device=dev())
        smc.fcc_energy(lat, smc.Model(smc.PAIR_I32, nsh, V, unit_ev=1e-4), occ, e=e, e_int=e_int)
        assert int(e_int.item()) == oracle.fcc_total_energy_i64(olat, oracle.Model(oracle.PAIR_I32, nsh, V,
                                                                                   unit_ev=1e-4), ref)
    else:
        V = inputs.pair_f32_coeffs(2, nsh, S)
        smc.fcc_energy(lat, smc.Model(smc.PAIR_F32, nsh, V), occ, e=e)
        want = oracle.fcc_total_energy(olat, oracle.Model(oracle.PAIR_F32, nsh, V), ref)
        assert float(e.item()) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_large_int_values_do_not_overflow(smc):
    """|V| at the 2^24 limit (a dE of 84 such terms can pass 2^31): the
    trajectory and the accepted sum stay exact."""
    dims, S, nsh = (8, 8, 8), 2, 3
    V = np.zeros((nsh, S, S), dtype=np.int32)
    V[:, 0, 1] = V[:, 1, 0] = -(1 << 24)
    V[:, 1, 1] = 1 << 24
    lat, occ, olat, ref = _state(smc, dims, S, 1)
    model = smc.Model(smc.PAIR_I32, nsh, V, unit_ev=1e-6)
    omodel = oracle.Model(oracle.PAIR_I32, nsh, V, unit_ev=1e-6)
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.fcc_sweep(lat, model, occ, 3, 0, 2, [0.05, 0.05], e_acc=e_acc, n_acc=n_acc)
    oe, on = oracle.fcc_sweep(olat, omodel, ref, 3, 0, 2, [0.05, 0.05])
    smc.check()
    assert np.array_equal(occ.cpu().numpy(), ref)
    assert int(n_acc.item()) == on and float(e_acc.item()) == oe


def test_unsupported_inputs_raise(smc):
    S = 2
    V = inputs.pair_int_coeffs(1, 2, S)
    model = smc.Model(smc.PAIR_I32, 2, V, unit_ev=1e-4)
    for dims in ((6, 8, 8), (8, 4, 8), (8, 8, 10)):
        lat = smc.Lattice(*dims, S)
        occ = torch.zeros(smc.fcc_nsites(lat), dtype=torch.int8, device=dev())
        with pytest.raises(smc.SMCError):
            smc.fcc_sweep(lat, model, occ, 1, 0, 1, [0.05])
    lat = smc.Lattice(8, 8, 8, S)
    occ = torch.zeros(smc.fcc_nsites(lat), dtype=torch.int8, device=dev())
    with pytest.raises(smc.SMCError):
        smc.fcc_ministep_trace(lat, model, occ, 1, 0, 256, 0.05,
                               dE=torch.zeros(8, dtype=torch.float32, device=dev()),
                               acc=torch.zeros(8, dtype=torch.uint8, device=dev()))
    with pytest.raises(smc.SMCError):
        smc.fcc_sweep(lat, model, occ, 1, 0, 1, [-1.0])
    mlp = smc.Model(smc.MLPNET_BF16, net=inputs.mlpnet_weights(1))  # neither pair nor qSRO
    with pytest.raises(smc.SMCError):
        smc.fcc_sweep(lat, mlp, occ, 1, 0, 1, [0.05])
    with pytest.raises(smc.SMCError):
        smc.fcc_init_lattice(lat, [10, 10], 1, occ)


def test_full_size_sampled_trials(smc):
    """256^3 cubic cells (67M sites), FP32 3-shell quinary at 800 K: the
    start state equals the oracle's everywhere; on it, mini-step 137 of
    sweep 1 (any state is a valid input to one mini-step) gives at 400
    sampled link cells (faces and interior) the oracle's dE of the same
    trial (a from the schedule, b from its Philox word) and decision, and
    the swap is applied where accepted."""
    n, S, seed, sweep, k = 256, 5, 1, 1, 137
    lat = smc.Lattice(n, n, n, S)
    N = smc.fcc_nsites(lat)
    V = inputs.pair_f32_coeffs(3, 3, S)
    model = smc.Model(smc.PAIR_F32, 3, V)
    kT = inputs.K_B_EV * 800.0
    occ = torch.empty(N, dtype=torch.int8, device=dev())
    smc.fcc_init_lattice(lat, inputs.equiatomic_counts(N, S), seed, occ)
    olat, omodel = oracle.Lattice(n, n, n, S), oracle.Model(oracle.PAIR_F32, 3, V)
    pre = oracle.fcc_init_lattice(olat, inputs.equiatomic_counts(N, S), seed)
    assert np.array_equal(occ.cpu().numpy(), pre)
    NL = n // 4
    dE = torch.zeros(NL ** 3, dtype=torch.float32, device=dev())
    acc = torch.zeros(NL ** 3, dtype=torch.uint8, device=dev())
    smc.fcc_ministep_trace(lat, model, occ, seed, sweep, k, kT, dE=dE, acc=acc)
    smc.check()
    post, g_dE, g_acc = occ.cpu().numpy(), dE.cpu().numpy(), acc.cpu().numpy()
    v1 = oracle.fcc_shell_vectors(1)
    rng = np.random.default_rng(5)
    cells = [(0, 0, 0), (NL - 1, NL - 1, NL - 1), (0, 5, 9), (NL - 1, 2, 30), (3, 0, 4), (7, NL - 1, 1)]
    cells += [tuple(int(v) for v in rng.integers(0, NL, 3)) for _ in range(394)]
    dx, dy, dz, sub = k % 4, (k // 4) % 4, (k // 16) % 4, k // 64
    for cx, cy, cz in cells:
        c = (cz * NL + cy) * NL + cx
        a = ((sub * n + 4 * cz + dz) * n + 4 * cy + dy) * n + 4 * cx + dx
        w = oracle.philox4x32_10([a & 0xFFFFFFFF, 0, sweep, 0], [seed, 0])
        b = oracle.fcc_neighbor(olat, a, v1[(int(w[1]) * 12) >> 32])
        ref = oracle.fcc_delta_e(olat, omodel, pre, a, b)
        assert abs(float(g_dE[c]) - ref) <= DE_TOL_EV, (c, float(g_dE[c]), ref)
        u = (float(int(w[0]) & ((1 << 29) - 1)) + 0.5) / 2.0 ** 29
        want = ref <= 0 or u < math.exp(-ref / kT)
        if abs(ref + kT * math.log(u)) > DE_TOL_EV:
            assert bool(g_acc[c]) == want, c
        if g_acc[c]:
            assert post[a] == pre[b] and post[b] == pre[a]
        else:
            assert post[a] == pre[a] and post[b] == pre[b]


# ---- qSRO on the FCC lattice (Eq. quadratic_local_SRO) ----

def _qsro_models(smc, seed, nsh, S):
    V, W, C = inputs.qsro_coeffs(seed, nsh, S)
    return (smc.Model(smc.QSRO_F32, nsh, V, qsro_w=W, qsro_c=C),
            oracle.Model(oracle.QSRO, nsh, V, qsro_w=W, qsro_c=C))


@pytest.mark.parametrize("dims,nsh,S", [((8, 8, 8), 3, 5), ((12, 8, 16), 2, 4), ((24, 24, 24), 3, 5),
                                        ((8, 12, 8), 2, 8), ((12, 8, 8), 1, 2)])
def test_qsro_lockstep_against_oracle(smc, dims, nsh, S):
    """Every trial of a sweep (24^3: 64 of the 256 mini-steps, mostly interior
    link cells): dE within 1e-5 eV of the FP64 oracle, the same decisions
    (after a flip the GPU continues from the oracle's state), 800 K."""
    model, omodel = _qsro_models(smc, 7 + nsh, nsh, S)
    lat, occ, olat, ref = _state(smc, dims, S, 4)
    kT = inputs.K_B_EV * 800.0
    nt = oracle.fcc_nsites(olat) // 256
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    flips, worst, nacc = 0, 0.0, 0
    ks = range(256) if dims[0] < 24 else range(0, 256, 4)
    for k in ks:
        smc.fcc_ministep_trace(lat, model, occ, 9, 1, k, kT, dE=dE, acc=acc)
        odE, oacc, _, _ = oracle.fcc_ministep_trace(olat, omodel, ref, 9, 1, k, kT)
        g = dE.cpu().numpy().astype(np.float64)
        worst = max(worst, float(np.abs(g - odE).max()))
        assert np.all(np.abs(g - odE) <= DE_TOL_EV), k
        ga = acc.cpu().numpy().astype(bool)
        nacc += int(ga.sum())
        if not np.array_equal(ga, oacc):  # the GPU continues from the oracle's state
            flips += int((ga != oacc).sum())
            occ.copy_(torch.from_numpy(ref.copy()).to(dev()))
        else:
            assert np.array_equal(occ.cpu().numpy(), ref)
    assert flips <= 1, flips
    assert worst < 2e-6
    assert nacc > 0


@pytest.mark.parametrize("dims,nsh", [((8, 16, 12), 3), ((24, 24, 24), 3), ((16, 8, 8), 1), ((12, 12, 8), 2)])
def test_qsro_sweep_equals_trace_and_energy_closes(smc, dims, nsh):
    """The sweep keeps the own-species count cache across its mini-steps;
    every traced mini-step rebuilds it from the occupancy: the trajectories
    must agree bit for bit.  E(after) - E_oracle(before) = e_acc within FP32
    rounding (the energy itself is pinned on oracle states elsewhere)."""
    S = 5
    model, omodel = _qsro_models(smc, 3 * nsh, nsh, S)
    lat, occ, olat, ref = _state(smc, dims, S, 8)
    occ2 = occ.clone()
    kT = [inputs.K_B_EV * 800.0, inputs.K_B_EV * 1200.0]
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.fcc_sweep(lat, model, occ, 4, 10, 2, kT, e_acc=e_acc, n_acc=n_acc)
    for t in range(2):
        for k in range(256):
            smc.fcc_ministep_trace(lat, model, occ2, 4, 10 + t, k, kT[t])
    smc.check()
    assert torch.equal(occ, occ2)
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.fcc_energy(lat, model, occ, e=e)
    after = occ.cpu().numpy()
    assert np.array_equal(np.bincount(after, minlength=S), np.bincount(ref, minlength=S))
    n = int(n_acc.item())
    assert n > 0
    # each accepted dE: about 130 FP32 terms of |.| <= 0.1 eV; errors add like a random walk
    tol = 6 * math.sqrt(n) * 130 * 2.0 ** -24 * 0.5
    assert abs(float(e.item()) - (oracle.fcc_total_energy(olat, omodel, ref) + float(e_acc.item()))) <= tol


@pytest.mark.parametrize("dims,nsh", [((4, 5, 3), 3), ((8, 8, 8), 2), ((16, 8, 24), 3), ((2, 1, 1), 1)])
def test_qsro_energy_matches_oracle(smc, dims, nsh):
    S = 4
    model, omodel = _qsro_models(smc, 40 + nsh, nsh, S)
    lat, occ, olat, ref = _state(smc, dims, S, 12, inputs.dirichlet_counts(4 * dims[0] * dims[1] * dims[2], S, 2))
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.fcc_energy(lat, model, occ, e=e)
    assert float(e.item()) == pytest.approx(oracle.fcc_total_energy(olat, omodel, ref), rel=1e-12)


def test_qsro_full_size_sampled_trials(smc):
    """256^3 cubic cells (67M sites), 3-shell quinary qSRO at 800 K on the
    oracle's start state: mini-step 77 of sweep 2 at 300 sampled link cells
    against the oracle's dE and decision, the swap applied where accepted."""
    n, S, seed, sweep, k = 256, 5, 1, 2, 77
    lat = smc.Lattice(n, n, n, S)
    N = smc.fcc_nsites(lat)
    model, omodel = _qsro_models(smc, 7, 3, S)
    kT = inputs.K_B_EV * 800.0
    occ = torch.empty(N, dtype=torch.int8, device=dev())
    smc.fcc_init_lattice(lat, inputs.equiatomic_counts(N, S), seed, occ)
    olat = oracle.Lattice(n, n, n, S)
    pre = oracle.fcc_init_lattice(olat, inputs.equiatomic_counts(N, S), seed)
    assert np.array_equal(occ.cpu().numpy(), pre)
    NL = n // 4
    dE = torch.zeros(NL ** 3, dtype=torch.float32, device=dev())
    acc = torch.zeros(NL ** 3, dtype=torch.uint8, device=dev())
    smc.fcc_ministep_trace(lat, model, occ, seed, sweep, k, kT, dE=dE, acc=acc)
    smc.check()
    post, g_dE, g_acc = occ.cpu().numpy(), dE.cpu().numpy(), acc.cpu().numpy()
    v1 = oracle.fcc_shell_vectors(1)
    rng = np.random.default_rng(6)
    cells = [(0, 0, 0), (NL - 1, NL - 1, NL - 1), (0, 5, 9), (NL - 1, 2, 30)]
    cells += [tuple(int(v) for v in rng.integers(0, NL, 3)) for _ in range(296)]
    dx, dy, dz, sub = k % 4, (k // 4) % 4, (k // 16) % 4, k // 64
    for cx, cy, cz in cells:
        c = (cz * NL + cy) * NL + cx
        a = ((sub * n + 4 * cz + dz) * n + 4 * cy + dy) * n + 4 * cx + dx
        w = oracle.philox4x32_10([a & 0xFFFFFFFF, 0, sweep, 0], [seed, 0])
        b = oracle.fcc_neighbor(olat, a, v1[(int(w[1]) * 12) >> 32])
        ref = oracle.fcc_delta_e(olat, omodel, pre, a, b)
        assert abs(float(g_dE[c]) - ref) <= DE_TOL_EV, (c, float(g_dE[c]), ref)
        u = (float(int(w[0]) & ((1 << 29) - 1)) + 0.5) / 2.0 ** 29
        want = ref <= 0 or u < math.exp(-ref / kT)
        if abs(ref + kT * math.log(u)) > DE_TOL_EV:
            assert bool(g_acc[c]) == want, c
        if g_acc[c]:
            assert post[a] == pre[b] and post[b] == pre[a]
        else:
            assert post[a] == pre[a] and post[b] == pre[b]


def test_degenerate_cases(smc):
    """One species (dE = 0 everywhere: all accepted, nothing moves) and, for
    FP32 pair and qSRO models, infinite temperature (every trial accepted
    whatever dE: trajectories equal the oracle's bit for bit)."""
    dims = (8, 8, 12)
    N = 4 * dims[0] * dims[1] * dims[2]
    lat1 = smc.Lattice(*dims, 1)
    occ1 = torch.zeros(N, dtype=torch.int8, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.fcc_sweep(lat1, smc.Model(smc.PAIR_I32, 3, np.zeros((3, 1, 1), dtype=np.int32), unit_ev=1e-4), occ1, 1, 0,
                  2, 0.05, e_acc=e_acc, n_acc=n_acc)
    smc.check()
    assert int(n_acc.item()) == 2 * N and float(e_acc.item()) == 0.0
    assert int(occ1.abs().sum().item()) == 0
    S = 5
    for kind in ("pair", "qsro"):
        lat, occ, olat, ref = _state(smc, dims, S, 9)
        if kind == "pair":
            V = inputs.pair_f32_coeffs(6, 2, S)
            gm, om = smc.Model(smc.PAIR_F32, 2, V), oracle.Model(oracle.PAIR_F32, 2, V)
        else:
            gm, om = _qsro_models(smc, 6, 2, S)
        smc.fcc_sweep(lat, gm, occ, 4, 0, 2, float("inf"))
        oracle.fcc_sweep(olat, om, ref, 4, 0, 2, float("inf"))
        smc.check()
        assert np.array_equal(occ.cpu().numpy(), ref), kind


def test_maximum_size_sampled_trials(smc):
    """Near the largest FCC lattice the API takes (N < 2^31): 1024 x 1024 x 508
    cubic cells, N = 2,130,706,432 sites, a seeded random quinary occupancy;
    one traced pair mini-step against the oracle's dE and decision at 200
    sampled trials, the swaps applied where accepted; the energy (64-bit site
    loop) changes by the sum of the accepted dE."""
    dims, S, seed, kT, k = (1024, 1024, 508), 5, 4, 0.07, 141
    N = 4 * dims[0] * dims[1] * dims[2]
    assert N < 2 ** 31
    pre = np.random.default_rng(seed).integers(0, S, N, dtype=np.int8)
    lat = smc.Lattice(*dims, S)
    V = inputs.pair_f32_coeffs(9, 2, S)
    model = smc.Model(smc.PAIR_F32, 2, V)
    occ = torch.from_numpy(pre).to(dev())
    e0 = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.fcc_energy(lat, model, occ, e=e0)
    NL = [d // 4 for d in dims]
    nt = NL[0] * NL[1] * NL[2]
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    smc.fcc_ministep_trace(lat, model, occ, seed, 2, k, kT, dE=dE, acc=acc)
    e1 = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.fcc_energy(lat, model, occ, e=e1)
    smc.check()
    g_dE, g_acc = dE.cpu().numpy(), acc.cpu().numpy().astype(bool)
    olat, omodel = oracle.Lattice(*dims, S), oracle.Model(oracle.PAIR_F32, 2, V)
    v1 = oracle.fcc_shell_vectors(1)
    dx, dy, dz, sub = k % 4, (k // 4) % 4, (k // 16) % 4, k // 64
    rng = np.random.default_rng(2)
    sites = []
    for c in np.concatenate([[0, nt - 1], rng.integers(0, nt, 198)]):
        cx, cy, cz = c % NL[0], (c // NL[0]) % NL[1], c // (NL[0] * NL[1])
        a = int(((sub * dims[2] + 4 * cz + dz) * dims[1] + 4 * cy + dy) * dims[0] + 4 * cx + dx)
        w = oracle.philox4x32_10([a & 0xFFFFFFFF, 0, 2, 0], [seed, 0])
        b = oracle.fcc_neighbor(olat, a, v1[(int(w[1]) * 12) >> 32])
        ref = oracle.fcc_delta_e(olat, omodel, pre, a, b)
        assert abs(float(g_dE[c]) - ref) <= DE_TOL_EV, (int(c), float(g_dE[c]), ref)
        u = (float(int(w[0]) & ((1 << 29) - 1)) + 0.5) / 2.0 ** 29
        if abs(ref + kT * math.log(u)) > DE_TOL_EV:
            assert bool(g_acc[c]) == (ref <= 0 or u < math.exp(-ref / kT)), int(c)
        sites.append((a, b, bool(g_acc[c])))
    got = occ[torch.tensor([p for t in sites for p in t[:2]], device=dev())].cpu().numpy().reshape(-1, 2)
    for (a, b, ac), (ga, gb) in zip(sites, got):
        assert (ga, gb) == ((pre[b], pre[a]) if ac else (pre[a], pre[b]))
    de_sum = float(g_dE[g_acc].astype(np.float64).sum())
    assert abs(float(e1.item()) - float(e0.item()) - de_sum) <= 6 * math.sqrt(max(int(g_acc.sum()), 1)) * DE_TOL_EV
