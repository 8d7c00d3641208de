"""GPU tests of smc_sweep_noalloc, the entry point for callers that cannot
allocate device memory (for example code running while a CUDA graph is being
captured, where an allocation is an error, or an application that owns all
device memory through its own pool and must not see a library allocate).

The entry point is called through the C ABI (ctypes on libsmc.so) and
compared with smc_sweep on identical inputs, for two calls in a row: the same
occupancy, accepted count and accumulated dE, bit for bit (both run the same
kernel with the same plan and a fixed-order reduction).  Device memory in use
must not change across its calls, its status word must report a stalled
progress wait, and a NULL status is refused.  This file is named so that
pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

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
    return s


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _start_state(N, S, seed):
    """A seeded random configuration with equiatomic counts, made without the
    library (so that nothing has touched its workspace yet)."""
    counts = inputs.equiatomic_counts(N, S)
    occ = np.repeat(np.arange(S, dtype=np.int8), counts)
    np.random.default_rng(seed).shuffle(occ)
    return torch.from_numpy(occ).to("cuda:0")


def _noalloc(L, lat, model, occ, seed, sweep0, kt, e_acc, n_acc, status):
    kt = np.ascontiguousarray(kt, dtype=np.float64)
    return L.smc_sweep_noalloc(C.byref(lat._c), C.byref(model._c), C.c_void_p(occ.data_ptr()), C.c_uint64(seed),
                               C.c_uint32(0), C.c_uint64(sweep0), len(kt), kt.ctypes.data_as(C.POINTER(C.c_double)),
                               C.c_void_p(e_acc.data_ptr()) if e_acc is not None else None,
                               C.c_void_p(n_acc.data_ptr()) if n_acc is not None else None,
                               C.c_void_p(status.data_ptr()) if status is not None else None, _stream())


@pytest.mark.parametrize("dims", [(32, 16, 24), (6, 8, 12), (512, 8, 8)])
def test_noalloc_sweep_matches_smc_sweep(smc, dims):
    L = smc.lib()
    S = 5
    V = inputs.pair_f32_coeffs(2, 2, S)
    lat = smc.Lattice(*dims, S)
    model = smc.Model(smc.PAIR_F32, 2, V)
    a = _start_state(lat.nsites, S, 3)
    b = a.clone()
    dev = a.device
    ea = torch.zeros(1, dtype=torch.float64, device=dev)
    na = torch.zeros(1, dtype=torch.int64, device=dev)
    eb = torch.zeros(1, dtype=torch.float64, device=dev)
    nb = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.full((1,), -99, dtype=torch.int32, device=dev)
    kT = inputs.anneal_kT(8, 2500.0, 800.0)
    # a first call (on a scratch copy) loads the kernels; after it, two calls
    # in a row must leave device memory as it was
    warm = a.clone()
    assert _noalloc(L, lat, model, warm, 7, 0, kT[:4], None, None, status) == smc.SMC_OK, L.smc_last_error()
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    del warm
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for call in range(2):
        rc = _noalloc(L, lat, model, a, 7, 4 * call, kT[4 * call:4 * call + 4], ea, na, status)
        assert rc == smc.SMC_OK, L.smc_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
    assert int(status.item()) == 0
    for call in range(2):
        smc.sweep(lat, model, b, 7, 4 * call, 4, kT[4 * call:4 * call + 4], e_acc=eb, n_acc=nb)
    smc.check()
    assert torch.equal(a, b)
    assert int(na.item()) == int(nb.item())
    assert float(ea.item()) == float(eb.item())
    # composition is conserved
    assert np.array_equal(np.bincount(a.cpu().numpy(), minlength=S), inputs.equiatomic_counts(lat.nsites, S))


def test_noalloc_reports_a_stalled_wait_in_status(smc):
    """One tile never publishes its progress (test hook): the call's status
    word reports SMC_ERR_TIMEOUT within the wait limit, and the next call on
    the same array runs normally."""
    L = smc.lib()
    dims, S = (16, 16, 16), 5
    V = inputs.pair_f32_coeffs(2, 2, S)
    lat = smc.Lattice(*dims, S)
    model = smc.Model(smc.PAIR_F32, 2, V)
    occ = _start_state(lat.nsites, S, 4)
    status = torch.zeros(1, dtype=torch.int32, device=occ.device)
    smc.set_tuning(1, 1, 32, 0)
    smc.debug_set(smc.DBG_TIMEOUT_MS, 200)
    smc.debug_set(smc.DBG_SKIP_PUBLISH, 3)
    try:
        assert _noalloc(L, lat, model, occ, 1, 0, [0.05, 0.05], None, None, status) == smc.SMC_OK
        torch.cuda.synchronize()
        assert int(status.item()) == smc.SMC_ERR_TIMEOUT
    finally:
        smc.debug_set(smc.DBG_SKIP_PUBLISH, -1)
        smc.debug_set(smc.DBG_TIMEOUT_MS, 2000)
        smc.set_tuning()
    a = _start_state(lat.nsites, S, 5)
    b = a.clone()
    assert _noalloc(L, lat, model, a, 2, 0, [0.05, 0.05], None, None, status) == smc.SMC_OK
    smc.sweep(lat, model, b, 2, 0, 2, [0.05, 0.05])
    smc.check()
    assert int(status.item()) == 0
    assert torch.equal(a, b)


def test_noalloc_argument_errors(smc):
    L = smc.lib()
    lat = smc.Lattice(8, 8, 8, 2)
    occ = torch.zeros(lat.nsites, dtype=torch.int8, device="cuda:0")
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda:0")
    mi = smc.Model(smc.PAIR_I32, 2, inputs.pair_int_coeffs(1, 2, 2), unit_ev=1e-4)
    assert _noalloc(L, lat, mi, occ, 1, 0, [0.025], None, None, status) == smc.SMC_ERR_UNSUPPORTED
    mf = smc.Model(smc.PAIR_F32, 2, inputs.pair_f32_coeffs(1, 2, 2))
    assert _noalloc(L, lat, mf, occ, 1, 0, [0.025], None, None, None) == smc.SMC_ERR_ARG
    # no sweeps: nothing changes and the status word is cleared
    assert _noalloc(L, lat, mf, occ, 1, 0, [], None, None, status) == smc.SMC_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and int(occ.abs().sum().item()) == 0
