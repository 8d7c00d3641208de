"""GPU parity of the resident pair sweep (the lattice held in shared memory
for a whole call, rows exchanged between CTAs through a global copy) against
the oracle and against the streaming kernel.

Integer models: bit-exact trajectories, accepted counts and dE against the
oracle, for block shapes of 1 to 8 link-cell columns, two and three shells,
one and two species words.  FP32 models: the same occupancy, accepted count
and accumulated dE as the streaming kernel, bit for bit (the two run the
same arithmetic in the same schedule).  A stalled block is reported as a
timeout and the next call runs normally."""
import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08250_gb300 import build, smc as s
    build.build()
    s.lib()
    yield s
    s.set_tuning()
    s.debug_set(s.DBG_RESIDENT, 0)


def dev():
    return torch.device("cuda:0")


def _run_int(smc, dims, S, nshells, nsweeps, kT, tile=(0, 0), seed=7, vseed=3, chunks=1):
    V = inputs.pair_int_coeffs(vseed, nshells, S)
    counts = inputs.equiatomic_counts(2 * dims[0] * dims[1] * dims[2], S)
    lat = smc.Lattice(*dims, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device=dev())
    smc.init_lattice(lat, counts, seed, occ)
    model = smc.Model(smc.PAIR_I32, nshells, V, unit_ev=1e-4)
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    olat = oracle.Lattice(*dims, S)
    omodel = oracle.Model(oracle.PAIR_I32, nshells, V, unit_ev=1e-4)
    ref = oracle.init_lattice(olat, counts, seed)
    smc.set_tuning(tile[0], tile[1], 0, 0)
    oe = on = 0
    per = nsweeps // chunks
    try:
        for c in range(chunks):
            smc.sweep(lat, model, occ, seed, c * per, per, kT, e_acc=e_acc, n_acc=n_acc)
            e, n = oracle.sweep(olat, omodel, ref, seed, c * per, per, kT)
            oe += e
            on += n
            smc.check()
            assert np.array_equal(occ.cpu().numpy(), ref), f"occupancy differs after chunk {c}"
    finally:
        smc.set_tuning()
    assert int(n_acc.item()) == on
    assert float(e_acc.item()) == oe


@pytest.mark.parametrize("dims,S,nsh,tile", [((16, 12, 12), 5, 2, (0, 0)), ((32, 16, 16), 3, 3, (0, 0)),
                                             ((20, 12, 16), 5, 2, (0, 0)), ((36, 16, 12), 4, 3, (0, 0)),
                                             ((12, 16, 12), 5, 2, (0, 0)),
                                             ((32, 24, 48), 5, 2, (2, 4)), ((16, 24, 12), 8, 2, (2, 1)),
                                             ((48, 12, 36), 2, 3, (1, 3)), ((16, 28, 16), 5, 2, (2, 2))])
def test_resident_integer_trajectories(smc, dims, S, nsh, tile):
    _run_int(smc, dims, S, nsh, 4, 0.03, tile=tile, chunks=2)


def test_resident_full_size_integer_sweep_matches_oracle(smc):
    """The headline launch configuration (128^3, 2 x 4-column blocks, the
    compile-time-pitch kernel) with an integer quinary model: one full sweep
    bit-exact against the oracle (4.2 M trials; the oracle takes about 40 s)."""
    _run_int(smc, (128, 128, 128), 5, 2, 1, 0.03, seed=11, vseed=4)


def _f32_pair(smc, dims, nsweeps, kT, resident, seed=5):
    S = 5
    V = inputs.pair_f32_coeffs(inputs.CONFIG2["coeff_seed"], 2, S)
    lat = smc.Lattice(*dims, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device=dev())
    smc.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), seed, occ)
    e_acc = torch.zeros(1, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(1, dtype=torch.int64, device=dev())
    smc.debug_set(smc.DBG_RESIDENT, 0 if resident else 1)
    try:
        smc.sweep(lat, smc.Model(smc.PAIR_F32, 2, V), occ, seed, 0, nsweeps, kT, e_acc=e_acc, n_acc=n_acc)
        smc.check()
    finally:
        smc.debug_set(smc.DBG_RESIDENT, 0)
    return occ, float(e_acc.item()), int(n_acc.item())


@pytest.mark.parametrize("dims,nsweeps", [((128, 128, 128), 3), ((64, 64, 64), 4), ((32, 48, 40), 5),
                                          ((128, 128, 128), 40), ((64, 64, 64), 120)])
def test_resident_equals_streaming_fp32(smc, dims, nsweeps):
    """The anneal's model on the 128^3 box (2 x 4 blocks of columns) and on
    smaller boxes: per-sweep temperatures, identical results bit for bit.
    The long runs give the blocks' progress time to drift apart, so that
    every ordering of the exchange, release and compute warps occurs."""
    kT = inputs.anneal_kT(1000)[:nsweeps]
    a = _f32_pair(smc, dims, nsweeps, kT, True)
    b = _f32_pair(smc, dims, nsweeps, kT, False)
    assert torch.equal(a[0], b[0])
    assert a[1] == b[1] and a[2] == b[2]


def test_resident_timeout_is_reported_and_gpu_stays_usable(smc):
    dims, S = (16, 12, 12), 2
    V = inputs.pair_int_coeffs(1, 2, S)
    lat = smc.Lattice(*dims, S)
    occ = torch.empty(lat.nsites, dtype=torch.int8, device=dev())
    smc.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), 1, occ)
    model = smc.Model(smc.PAIR_I32, 2, V, unit_ev=1e-4)
    smc.debug_set(smc.DBG_TIMEOUT_MS, 200)
    smc.debug_set(smc.DBG_SKIP_PUBLISH, 4)
    try:
        smc.sweep(lat, model, occ, 1, 0, 2, 0.025)
        with pytest.raises(smc.SMCError) as ei:
            smc.check()
        assert ei.value.code == smc.SMC_ERR_TIMEOUT
    finally:
        smc.debug_set(smc.DBG_SKIP_PUBLISH, -1)
        smc.debug_set(smc.DBG_TIMEOUT_MS, 2000)
    _run_int(smc, dims, 2, 2, 2, 0.025)


def _batched(smc, edges, nsweeps, kT, is_int, resident):
    S = 5
    if is_int:
        model = smc.Model(smc.PAIR_I32, 2, inputs.pair_int_coeffs(3, 2, S), unit_ev=1e-4)
    else:
        model = smc.Model(smc.PAIR_F32, 2, inputs.pair_f32_coeffs(inputs.CONFIG2["coeff_seed"], 2, S))
    lats = [smc.Lattice(e, e + 4 * (i % 2), e, S) for i, e in enumerate(edges)]
    occs = []
    for r, lat in enumerate(lats):
        o = torch.empty(lat.nsites, dtype=torch.int8, device=dev())
        smc.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), 3, o, replica=r)
        occs.append(o)
    R = len(lats)
    e_acc = torch.zeros(R, dtype=torch.float64, device=dev())
    n_acc = torch.zeros(R, dtype=torch.int64, device=dev())
    kTr = np.repeat(np.asarray(kT, dtype=np.float64)[:, None], nsweeps, axis=1)
    smc.debug_set(smc.DBG_RESIDENT, 0 if resident else 1)
    try:
        smc.sweep_batched(lats, model, occs, 3, 0, nsweeps, kTr, e_acc=e_acc, n_acc=n_acc)
        smc.check()
    finally:
        smc.debug_set(smc.DBG_RESIDENT, 0)
    return lats, occs, e_acc, n_acc


@pytest.mark.parametrize("edges,is_int", [([16, 20, 24, 32, 16, 28], True), ([32] * 20 + [48] * 4, False),
                                          ([36, 44, 12, 52], True)])
def test_resident_replicas_equal_streaming_replicas(smc, edges, is_int):
    """Replicas of different sizes in waves of one launch each (the second
    case needs more than one wave): the same occupancies, accepted counts and
    energy sums as the streaming batched kernel, bit for bit."""
    kT = np.linspace(0.03, 0.09, len(edges))
    _, a, ea, na = _batched(smc, edges, 6, kT, is_int, True)
    _, b, eb, nb = _batched(smc, edges, 6, kT, is_int, False)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert torch.equal(na, nb) and torch.equal(ea, eb)


def test_resident_replicas_match_oracle(smc):
    edges, kT = [16, 20, 24], np.array([0.03, 0.05, 0.07])
    lats, occs, ea, na = _batched(smc, edges, 3, kT, True, True)
    S = 5
    V = inputs.pair_int_coeffs(3, 2, S)
    for r, lat in enumerate(lats):
        olat = oracle.Lattice(lat.nx, lat.ny, lat.nz, S)
        ref = oracle.init_lattice(olat, inputs.equiatomic_counts(lat.nsites, S), 3, replica=r)
        e, n = oracle.sweep(olat, oracle.Model(oracle.PAIR_I32, 2, V, unit_ev=1e-4), ref, 3, 0, 3, kT[r], replica=r)
        assert np.array_equal(occs[r].cpu().numpy(), ref)
        assert int(na[r].item()) == n
