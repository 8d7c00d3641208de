"""GPU parity of the pair-model path against the CPU oracle (through the C ABI).

Integer models: bit-exact trajectories, energies, counts.  FP32 models: every
trial's dE within 1e-5 eV of the FP64 oracle and identical decisions, checked
mini-step by mini-step (lock-step; after a decision flip the GPU continues
from the oracle's state)."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs
from tests import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DE_TOL_EV = 1e-5


def acc_tol(n_acc, V, nx):
    """Bound on |sum of FP32 dE - exact sum| over n_acc accepted trials: each
    dE is a sum of 26 FP32 terms |D| <= 2 max|V|, so its rounding error is at
    most 26 * 2^-24 * 26 * 2 max|V|.  The sweep kernel sums each lane's
    accepted dE of a column (L = 4 ceil(nx / 128) trials at most) in FP32
    before widening to FP64: one more rounding of at most
    2^-24 * L * 26 * 2 max|V| per trial.  Errors of independent trials add
    like a random walk, and 6 sigma of that walk is the tolerance."""
    L = 4 * math.ceil(nx / 128)
    per_trial = (26 + L) * 2.0 ** -24 * 26 * 2 * float(np.abs(V).max())
    return 6 * math.sqrt(max(n_acc, 1)) * per_trial / math.sqrt(3)


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


def gpu_state(smc, dims, S, counts, seed, replica=0):
    lat = smc.Lattice(*dims, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device=dev())
    smc.init_lattice(lat, counts, seed, occ, replica=replica)
    return lat, occ


def int_model(S=2, nshells=2, seed=1):
    V = inputs.pair_int_coeffs(seed, nshells, S)
    return V


def test_philox_known_answers(smc):
    rows = helpers.read_kat()
    ctr = torch.tensor(np.array([r[0] for r in rows], dtype=np.uint32).view(np.int32), device=dev())
    key = torch.tensor(np.array([r[1] for r in rows], dtype=np.uint32).view(np.int32), device=dev())
    out = torch.zeros_like(ctr)
    smc.philox4x32_10(ctr.reshape(-1), key.reshape(-1), out.reshape(-1))
    got = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, np.array([r[2] for r in rows], dtype=np.uint32))
    # and random counters against the oracle's independent implementation
    rng = np.random.default_rng(0)
    c = rng.integers(0, 2 ** 32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
    k = rng.integers(0, 2 ** 32, size=(256, 2), dtype=np.uint64).astype(np.uint32)
    o = torch.zeros(256 * 4, dtype=torch.int32, device=dev())
    smc.philox4x32_10(torch.tensor(c.view(np.int32).reshape(-1), device=dev()),
                      torch.tensor(k.view(np.int32).reshape(-1), device=dev()), o)
    got = o.cpu().numpy().view(np.uint32).reshape(256, 4)
    for i in range(256):
        assert np.array_equal(got[i], oracle.philox4x32_10(c[i], k[i]))


@pytest.mark.parametrize("dims,counts", [((8, 8, 8), None), ((2, 2, 2), [8, 8]), ((6, 10, 4), [100, 0, 380]),
                                         ((16, 8, 12), None), ((4, 4, 4), [128]), ((8, 4, 6), [0, 0, 384]),
                                         ((12, 8, 8), [1, 2, 3, 4, 5, 6, 7, 1508])])
def test_init_matches_oracle(smc, dims, counts):
    N = 2 * dims[0] * dims[1] * dims[2]
    if counts is None:
        counts = inputs.equiatomic_counts(N, 5)
    S = len(counts)
    for seed, rep in ((1, 0), (12345678901, 3)):
        _, occ = gpu_state(smc, dims, S, counts, seed, rep)
        want = oracle.init_lattice(oracle.Lattice(*dims, S), counts, seed, replica=rep)
        assert np.array_equal(occ.cpu().numpy(), want)


def _run_int(smc, dims, S, nshells, nsweeps, kT, seed=1, vseed=1, chunks=1, sweep0=0):
    V = int_model(S, nshells, vseed)
    counts = inputs.equiatomic_counts(2 * dims[0] * dims[1] * dims[2], S)
    lat, occ = gpu_state(smc, dims, S, counts, seed)
    model = smc.Model(smc.PAIR_I32, nshells, V, unit_ev=1e-4)
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    olat = oracle.Lattice(*dims, S)
    omodel = oracle.Model(oracle.PAIR_I32, nshells, V, unit_ev=1e-4)
    ref = oracle.init_lattice(olat, counts, seed)
    oe = on = 0
    per = nsweeps // chunks
    for c in range(chunks):
        smc.sweep(lat, model, occ, seed, sweep0 + c * per, per, kT, e_acc=e_acc, n_acc=n_acc)
        e, n = oracle.sweep(olat, omodel, ref, seed, sweep0 + c * per, per, kT)
        oe += e
        on += n
        smc.check()
        assert np.array_equal(occ.cpu().numpy(), ref), f"occupancy differs after chunk {c}"
    assert int(n_acc.item()) == on
    assert float(e_acc.item()) == oe
    return lat, model, occ, olat, omodel, ref


def test_config1_trajectory_bit_exact(smc):
    """8^3 cells, binary, integer 2-shell coefficients, kT = 25 meV, 100 sweeps:
    occupancy after every 10 sweeps, accepted count and accumulated dE."""
    lat, model, occ, olat, omodel, ref = _run_int(smc, (8, 8, 8), 2, 2, 100, 0.025, chunks=10)
    e_int = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.energy(lat, model, occ, e_int=e_int)
    assert int(e_int.item()) == oracle.total_energy_i64(olat, omodel, ref)


@pytest.mark.parametrize("dims,S,nshells", [((2, 2, 2), 2, 2), ((6, 8, 12), 3, 2), ((8, 12, 16), 3, 3),
                                            ((16, 8, 8), 4, 1), ((4, 6, 2), 2, 3), ((12, 12, 12), 8, 2),
                                            ((10, 8, 16), 2, 2)])
def test_integer_trajectories_other_shapes(smc, dims, S, nshells):
    _run_int(smc, dims, S, nshells, 6, 0.03, seed=7, vseed=3, chunks=2, sweep0=5)


@pytest.mark.parametrize("streaming", [False, True])
@pytest.mark.parametrize("dims,S,nsw", [((128, 8, 8), 5, 3), ((256, 8, 8), 5, 3), ((512, 8, 8), 5, 3),
                                        ((132, 8, 8), 5, 3), ((128, 16, 16), 5, 3), ((512, 8, 8), 2, 2),
                                        ((260, 8, 12), 3, 2), ((1024, 8, 8), 5, 1)])
def test_integer_trajectories_full_row_lengths(smc, dims, S, nsw, streaming):
    """The pair sweeps on rows as long as the benchmark lattices' (128-1024
    cells: every lane owns one to eight link cells of a column, and the tile
    grid wraps), and on ragged rows (33 and 65 link cells), bit for bit
    against the oracle after every sweep: the default path (these lattices
    fit the resident kernel) and the streaming kernel that sweeps lattices
    too large for shared memory (rows of 128, 256 and 512 cells take its
    wide-row form: rows of nx + 128 bytes, random words in registers)."""
    smc.debug_set(smc.DBG_RESIDENT, 1 if streaming else 0)
    try:
        _run_int(smc, dims, S, 2, nsw, 0.03, seed=7, vseed=3, chunks=nsw, sweep0=2)
    finally:
        smc.debug_set(smc.DBG_RESIDENT, 0)


def test_tuning_does_not_change_results(smc):
    dims, S = (16, 16, 24), 3
    V = int_model(S, 2, 2)
    counts = inputs.equiatomic_counts(2 * 16 * 16 * 24, S)
    model = smc.Model(smc.PAIR_I32, 2, V, unit_ev=1e-4)
    outs = []
    for tu in [(0, 0, 0, 0), (1, 1, 32, 0), (2, 3, 64, 1), (4, 6, 128, 2), (3, 1, 96, 0)]:
        smc.set_tuning(*tu)
        lat, occ = gpu_state(smc, dims, S, counts, 5)
        n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
        smc.sweep(lat, model, occ, 5, 0, 3, 0.02, n_acc=n_acc)
        smc.check()
        outs.append((occ.cpu().numpy(), int(n_acc.item())))
    smc.set_tuning()
    for o, n in outs[1:]:
        assert np.array_equal(o, outs[0][0]) and n == outs[0][1]


def _f32_setup(smc, dims, S=5, seed=3, vseed=2):
    V = inputs.pair_f32_coeffs(vseed, 2, S)
    counts = inputs.equiatomic_counts(2 * dims[0] * dims[1] * dims[2], S)
    lat, occ = gpu_state(smc, dims, S, counts, seed)
    return V, counts, lat, occ, smc.Model(smc.PAIR_F32, 2, V), oracle.Lattice(*dims, S), oracle.Model(oracle.PAIR_F32, 2, V)


@pytest.mark.parametrize("dims,kT", [((8, 8, 8), 0.06), ((16, 12, 8), 0.03), ((12, 8, 6), 0.2)])
def test_f32_lockstep_against_oracle(smc, dims, kT):
    """Every trial of every mini-step of two sweeps: |dE_gpu - dE_oracle| <=
    1e-5 eV and the same decision (after a flip the GPU continues from the
    oracle's state)."""
    V, counts, lat, occ, model, olat, omodel = _f32_setup(smc, dims)
    ref = oracle.init_lattice(olat, counts, 3)  # the oracle's own start state (== the GPU's)
    assert np.array_equal(occ.cpu().numpy(), ref)
    nA, _ = oracle.schedule(olat)
    nt = olat.nsites // nA
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    flips = 0
    worst = 0.0
    for sw in range(2):
        for k in range(nA):
            smc.ministep_trace(lat, model, occ, 9, sw, k, kT, dE=dE, acc=acc)
            odE, oacc, _, _ = oracle.ministep_trace(olat, omodel, ref, 9, sw, k, kT)
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


@pytest.mark.parametrize("streaming", [False, True])
@pytest.mark.parametrize("dims", [(8, 8, 8), (16, 12, 8), (6, 8, 12), (2, 2, 2), (128, 16, 16), (512, 8, 8),
                                  (256, 8, 12)])
def test_f32_sweep_kernel_equals_trace_kernel(smc, dims, streaming):
    """The persistent sweeps (the resident kernel, and the streaming kernel
    with shared-memory windows) and the mini-step trace kernel (global reads)
    share the dE arithmetic: identical trajectories."""
    V, counts, lat, occ, model, olat, omodel = _f32_setup(smc, dims)
    occ2 = occ.clone()
    kT = [0.05, 0.08]
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.debug_set(smc.DBG_RESIDENT, 1 if streaming else 0)
    try:
        smc.sweep(lat, model, occ, 4, 10, 2, kT, e_acc=e_acc, n_acc=n_acc)
    finally:
        smc.debug_set(smc.DBG_RESIDENT, 0)
    nA, _ = oracle.schedule(olat)
    for t in range(2):
        for k in range(nA):
            smc.ministep_trace(lat, model, occ2, 4, 10 + t, k, kT[t])
    smc.check()
    assert torch.equal(occ, occ2)
    e = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.energy(lat, model, occ, e=e)
    e0 = oracle.total_energy(olat, omodel, oracle.init_lattice(olat, counts, 3))
    assert abs(float(e.item()) - (e0 + float(e_acc.item()))) <= acc_tol(int(n_acc.item()), V, dims[0])


def test_counts_sro_energy_grad_match_oracle(smc):
    for dims, S, nsh in (((8, 8, 8), 5, 3), ((6, 10, 4), 3, 2), ((2, 2, 2), 2, 3), ((16, 16, 16), 8, 3),
                         ((2, 6, 4), 3, 1), ((40, 8, 12), 5, 2), ((600, 2, 3), 4, 3), ((3, 5, 7), 2, 2),
                         ((1100, 4, 2), 8, 3),
                         # rows of a multiple of 16 cells take the 16-byte-load kernel
                         ((32, 8, 12), 5, 2), ((48, 2, 4), 3, 1), ((16, 6, 10), 2, 3), ((528, 4, 2), 4, 3),
                         ((1024, 2, 2), 7, 2), ((64, 4, 4), 6, 1),
                         # rows of a multiple of 32 cells (at most 84 pair counters) take the bit-plane kernel
                         ((64, 6, 10), 5, 3), ((96, 4, 6), 6, 2), ((32, 2, 2), 8, 1), ((256, 8, 8), 5, 2),
                         ((160, 6, 4), 2, 3), ((32, 3, 5), 4, 3), ((64, 4, 6), 8, 2), ((32, 4, 4), 7, 3)):
        N = 2 * dims[0] * dims[1] * dims[2]
        counts = inputs.equiatomic_counts(N, S)
        lat, occ = gpu_state(smc, dims, S, counts, 21)
        olat = oracle.Lattice(*dims, S)
        ref = oracle.init_lattice(olat, counts, 21)
        cnt = torch.zeros((nsh, S, S), dtype=torch.int64, device=dev())
        alpha = torch.zeros((nsh, S, S), dtype=torch.float64, device=dev())
        smc.sro(lat, nsh, occ, counts=cnt, alpha=alpha)
        assert np.array_equal(cnt.cpu().numpy(), oracle.pair_counts(olat, nsh, ref))
        assert np.array_equal(alpha.cpu().numpy(), oracle.sro(olat, nsh, ref))
        Vf = inputs.pair_f32_coeffs(8, nsh, S)
        m = smc.Model(smc.PAIR_F32, nsh, Vf)
        om = oracle.Model(oracle.PAIR_F32, nsh, Vf)
        e = torch.zeros(1, dtype=torch.float64, device=dev())
        smc.energy(lat, m, occ, e=e)
        assert float(e.item()) == pytest.approx(oracle.total_energy(olat, om, ref), rel=1e-12, abs=1e-12)
        g = torch.zeros(smc.grad_size(lat, m), dtype=torch.float32, device=dev())
        smc.energy_grad(lat, m, occ, g)
        assert np.array_equal(g.cpu().numpy().astype(np.float64), oracle.energy_grad(olat, om, ref))


@pytest.mark.parametrize("dims,S,nsh", [((512, 64, 64), 5, 2), ((128, 128, 128), 5, 3)])
def test_pair_counts_full_row_lengths(smc, dims, S, nsh):
    """The bit-plane count kernel on rows of 16 and 4 words (the lengths of
    the 512^3 and 128^3 lattices), bit-exact against the oracle."""
    N = 2 * dims[0] * dims[1] * dims[2]
    counts = inputs.equiatomic_counts(N, S)
    lat, occ = gpu_state(smc, dims, S, counts, 5)
    olat = oracle.Lattice(*dims, S)
    ref = oracle.init_lattice(olat, counts, 5)
    cnt = torch.zeros((nsh, S, S), dtype=torch.int64, device=dev())
    smc.sro(lat, nsh, occ, counts=cnt)
    assert np.array_equal(cnt.cpu().numpy(), oracle.pair_counts(olat, nsh, ref))


def test_batched_replicas_equal_single_runs(smc):
    edges = [8, 12, 16, 8, 20]
    S = 5
    V = inputs.pair_f32_coeffs(3, 2, S)
    model = smc.Model(smc.PAIR_F32, 2, V)
    kT = inputs.ladder_kT(len(edges))
    lats, occs, singles = [], [], []
    for r, e in enumerate(edges):
        counts = inputs.equiatomic_counts(2 * e ** 3, S)
        lat, occ = gpu_state(smc, (e, e, e), S, counts, 11, replica=r)
        lats.append(lat)
        occs.append(occ)
        singles.append(occ.clone())
    e_acc = torch.zeros(len(edges), dtype=torch.float64, device=dev())
    n_acc = torch.zeros(len(edges), dtype=torch.int64, device=dev())
    smc.sweep_batched(lats, model, occs, 11, 0, 3, np.repeat(kT[:, None], 3, 1), e_acc=e_acc, n_acc=n_acc)
    for r in range(len(edges)):
        n1 = torch.zeros(1, dtype=torch.int64, device=dev())
        smc.sweep(lats[r], model, singles[r], 11, 0, 3, kT[r], replica=r, n_acc=n1)
        smc.check()
        assert torch.equal(occs[r], singles[r])
        assert int(n1.item()) == int(n_acc[r].item())


@pytest.mark.parametrize("dims,streaming", [((16, 16, 16), False), ((16, 16, 16), True), ((128, 8, 8), True)])
def test_timeout_is_reported_and_gpu_stays_usable(smc, dims, streaming):
    """A tile that never publishes its progress: the waits of its neighbours
    give up after the time limit, the call reports SMC_ERR_TIMEOUT, and the
    next call runs normally -- the default path, the single-group streaming
    kernel and the paired one (rows of 128 cells)."""
    S = 2
    V = int_model(S, 2, 1)
    counts = inputs.equiatomic_counts(2 * dims[0] * dims[1] * dims[2], S)
    lat, occ = gpu_state(smc, dims, S, counts, 1)
    model = smc.Model(smc.PAIR_I32, 2, V, unit_ev=1e-4)
    smc.set_tuning(1, 1, 32, 0)
    smc.debug_set(smc.DBG_TIMEOUT_MS, 200)
    smc.debug_set(smc.DBG_SKIP_PUBLISH, 3)
    smc.debug_set(smc.DBG_RESIDENT, 1 if streaming else 0)
    try:
        smc.sweep(lat, model, occ, 1, 0, 2, 0.025)
        with pytest.raises(smc.SMCError) as ei:
            smc.check()
        assert ei.value.code == smc.SMC_ERR_TIMEOUT
    finally:
        smc.debug_set(smc.DBG_SKIP_PUBLISH, -1)
        smc.debug_set(smc.DBG_TIMEOUT_MS, 2000)
        smc.debug_set(smc.DBG_RESIDENT, 0)
        smc.set_tuning()
    # the context is intact: a normal run still matches the oracle
    _run_int(smc, (8, 8, 8), 2, 2, 3, 0.025)


def test_config2_full_size_sampled(smc):
    """128^3 cells, quinary, FP32 2-shell model: two sweeps of the anneal
    (composition conserved, accumulated dE equal to the recomputed E), then
    on the oracle's start state mini-step 0 of sweep 2 traced and compared
    trial by trial."""
    c = inputs.CONFIG2
    dims, S = c["cells"], c["nspecies"]
    V = inputs.pair_f32_coeffs(c["coeff_seed"], 2, S)
    counts = inputs.equiatomic_counts(2 * dims[0] * dims[1] * dims[2], S)
    lat, occ = gpu_state(smc, dims, S, counts, c["mc_seed"])
    model = smc.Model(smc.PAIR_F32, 2, V)
    kT = inputs.anneal_kT(c["nsweeps"])
    e0 = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.energy(lat, model, occ, e=e0)
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.sweep(lat, model, occ, c["mc_seed"], 0, 2, kT[:2], e_acc=e_acc, n_acc=n_acc)
    e1 = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.energy(lat, model, occ, e=e1)
    smc.check()
    err = abs(float(e1.item()) - (float(e0.item()) + float(e_acc.item())))
    assert err <= acc_tol(int(n_acc.item()), V, dims[0]), (err, int(n_acc.item()))
    assert np.array_equal(np.bincount(occ.cpu().numpy(), minlength=S), counts)
    # mini-step 0 of sweep 2 on the oracle's start state (a valid input to any mini-step)
    olat, omodel = oracle.Lattice(*dims, S), oracle.Model(oracle.PAIR_F32, 2, V)
    ref = oracle.init_lattice(olat, counts, c["mc_seed"])
    occ.copy_(torch.from_numpy(ref.copy()).to(dev()))
    nt = olat.nsites // 128
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    smc.ministep_trace(lat, model, occ, c["mc_seed"], 2, 0, kT[2], dE=dE, acc=acc)
    odE, oacc, _, _ = oracle.ministep_trace(olat, omodel, ref, c["mc_seed"], 2, 0, kT[2])
    g = dE.cpu().numpy().astype(np.float64)
    assert np.abs(g - odE).max() <= DE_TOL_EV
    assert (acc.cpu().numpy().astype(bool) != oacc).sum() <= 1


def test_degenerate_cases(smc):
    """One species: every trial swaps equal species (dE = 0, accepted, nothing
    moves); no sweeps: nothing changes; infinite temperature (FP models):
    every trial accepted whatever dE, so the FP32 trajectory equals the
    oracle's bit for bit."""
    dims = (8, 12, 8)
    N = 2 * dims[0] * dims[1] * dims[2]
    lat1 = smc.Lattice(*dims, 1)
    occ1 = torch.zeros(N, dtype=torch.int8, device=dev())
    m1 = smc.Model(smc.PAIR_I32, 2, np.zeros((2, 1, 1), dtype=np.int32), unit_ev=1e-4)
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.sweep(lat1, m1, occ1, 1, 0, 2, 0.05, e_acc=e_acc, n_acc=n_acc)
    smc.check()
    assert int(n_acc.item()) == 2 * N and float(e_acc.item()) == 0.0
    assert int(occ1.abs().sum().item()) == 0
    _, on = oracle.sweep(oracle.Lattice(*dims, 1), oracle.Model(oracle.PAIR_I32, 2, np.zeros((2, 1, 1), np.int32),
                                                                unit_ev=1e-4), np.zeros(N, np.int8), 1, 0, 2, 0.05)
    assert on == 2 * N
    # no sweeps
    S = 5
    V = inputs.pair_f32_coeffs(4, 2, S)
    counts = inputs.equiatomic_counts(N, S)
    lat, occ = gpu_state(smc, dims, S, counts, 2)
    before = occ.clone()
    smc.sweep(lat, smc.Model(smc.PAIR_F32, 2, V), occ, 1, 0, 0, [], e_acc=e_acc, n_acc=n_acc)
    smc.check()
    assert torch.equal(occ, before) and int(n_acc.item()) == 2 * N
    # infinite temperature
    ref = oracle.init_lattice(oracle.Lattice(*dims, S), counts, 2)
    smc.sweep(lat, smc.Model(smc.PAIR_F32, 2, V), occ, 3, 0, 2, float("inf"))
    oracle.sweep(oracle.Lattice(*dims, S), oracle.Model(oracle.PAIR_F32, 2, V), ref, 3, 0, 2, float("inf"))
    smc.check()
    assert np.array_equal(occ.cpu().numpy(), ref)


def test_maximum_size_sampled_trials(smc):
    """A lattice near the largest the API takes (N < 2^31): 1008 x 1024 x 1024
    cells, N = 2,113,929,216 sites, a seeded random quinary occupancy.  One
    traced mini-step (the trial index arithmetic near 2^31) against the
    oracle's dE and decision at 300 sampled trials, the swaps applied where
    accepted; the energy then changes by the sum of the accepted dE."""
    dims, S, seed, kT = (1008, 1024, 1024), 5, 3, 0.07
    N = 2 * dims[0] * dims[1] * dims[2]
    assert N < 2 ** 31
    pre = np.random.default_rng(seed).integers(0, S, N, dtype=np.int8)
    lat = smc.Lattice(*dims, S)
    V = inputs.pair_f32_coeffs(5, 2, S)
    model = smc.Model(smc.PAIR_F32, 2, V)
    occ = torch.from_numpy(pre).to(dev())
    e0 = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.energy(lat, model, occ, e=e0)
    k = 97  # sublattice 1, dx 1, dy 0, dz 2 on 4 x 4 x 4 link cells
    nt = N // 128
    dE = torch.zeros(nt, dtype=torch.float32, device=dev())
    acc = torch.zeros(nt, dtype=torch.uint8, device=dev())
    smc.ministep_trace(lat, model, occ, seed, 1, k, kT, dE=dE, acc=acc)
    e1 = torch.zeros(1, dtype=torch.float64, device=dev())
    smc.energy(lat, model, occ, e=e1)
    smc.check()
    g_dE, g_acc = dE.cpu().numpy(), acc.cpu().numpy().astype(bool)
    olat, omodel = oracle.Lattice(*dims, S), oracle.Model(oracle.PAIR_F32, 2, V)
    nv = oracle.shell_vectors(1)
    NLx, NLy, NLz = dims[0] // 4, dims[1] // 4, dims[2] // 4
    dx, dy, dz, sub = k % 4, (k // 4) % 4, (k // 16) % 4, k // 64
    rng = np.random.default_rng(8)
    cs = np.concatenate([[0, nt - 1], rng.integers(0, nt, 298)])
    post_a = []
    for c in cs:
        cx, cy, cz = c % NLx, (c // NLx) % NLy, c // (NLx * NLy)
        a = int(((sub * dims[2] + 4 * cz + dz) * dims[1] + 4 * cy + dy) * dims[0] + 4 * cx + dx)
        wd = oracle.philox4x32_10([a >> 2, 0, 1, 0], [seed, 0])[a & 3]
        b = oracle.neighbor(olat, a, nv[int(wd) >> 29])
        ref = oracle.delta_e(olat, omodel, pre, a, b)
        assert abs(float(g_dE[c]) - ref) <= DE_TOL_EV, (int(c), float(g_dE[c]), ref)
        u = (float(int(wd) & ((1 << 29) - 1)) + 0.5) / 2.0 ** 29
        if abs(ref + kT * math.log(u)) > DE_TOL_EV:
            assert bool(g_acc[c]) == (ref <= 0 or u < math.exp(-ref / kT)), int(c)
        post_a.append((a, b, bool(g_acc[c])))
    got = occ[torch.tensor([p for t in post_a for p in t[:2]], device=dev())].cpu().numpy().reshape(-1, 2)
    for (a, b, ac), (ga, gb) in zip(post_a, got):
        assert (ga, gb) == ((pre[b], pre[a]) if ac else (pre[a], pre[b]))
    # energy bookkeeping of the whole mini-step (FP32 dE per trial, FP64 energies)
    de_sum = float(g_dE[g_acc].astype(np.float64).sum())
    assert abs(float(e1.item()) - float(e0.item()) - de_sum) <= 6 * math.sqrt(max(int(g_acc.sum()), 1)) * DE_TOL_EV
