"""GPU test of smc_sweep_noalloc, the entry point for callers that cannot
allocate device memory (for example while a CUDA graph is being captured, or
inside an application that owns all device memory through its own pool).

It is called through the C ABI (ctypes on libsmc.so) and compared with
smc_sweep on identical inputs, for two calls in a row.  This file is named so
that pytest collects it last."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_2604_08250_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tol(n_acc, V):
    # same bound as the other GPU tests: FP32 dE rounding over n_acc trials
    per_trial = 26 * 2.0 ** -24 * 26 * 2 * float(np.abs(V).max())
    return 6 * math.sqrt(max(n_acc, 1)) * per_trial / math.sqrt(3)


@pytest.mark.parametrize("dims", [(32, 16, 24), (6, 8, 12)])
def test_noalloc_sweep_matches_smc_sweep(dims):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08250_gb300 import build, smc
    build.build()
    L = smc.lib()
    S = 5
    V = inputs.pair_f32_coeffs(2, 2, S)
    lat = smc.Lattice(*dims, S)
    model = smc.Model(smc.PAIR_F32, 2, V)
    counts = inputs.equiatomic_counts(lat.nsites, S)
    dev = torch.device("cuda:0")
    a = torch.empty(lat.nsites, dtype=torch.int8, device=dev)
    smc.init_lattice(lat, counts, 3, a)
    b = a.clone()
    ea = torch.zeros(1, dtype=torch.float64, device=dev)
    na = torch.zeros(1, dtype=torch.int64, device=dev)
    eb = torch.zeros(1, dtype=torch.float64, device=dev)
    nb = torch.zeros(1, dtype=torch.int64, device=dev)
    status = torch.full((1,), -99, dtype=torch.int32, device=dev)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    kT = inputs.anneal_kT(8, 2500.0, 800.0)
    for call in range(2):
        kt = np.ascontiguousarray(kT[4 * call:4 * call + 4])
        rc = L.smc_sweep_noalloc(C.byref(lat._c), C.byref(model._c), C.c_void_p(a.data_ptr()), C.c_uint64(7),
                                 C.c_uint32(0), C.c_uint64(4 * call), 4, kt.ctypes.data_as(C.POINTER(C.c_double)),
                                 C.c_void_p(ea.data_ptr()), C.c_void_p(na.data_ptr()), C.c_void_p(status.data_ptr()),
                                 stream)
        assert rc == smc.SMC_OK, L.smc_last_error()
        smc.sweep(lat, model, b, 7, 4 * call, 4, kt, e_acc=eb, n_acc=nb)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(a, b), f"occupancy differs after call {call}"
        assert int(na.item()) == int(nb.item())
        assert abs(float(ea.item()) - float(eb.item())) <= _tol(int(na.item()), V)
    smc.check()


def test_noalloc_rejects_unsupported_models():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_08250_gb300 import build, smc
    build.build()
    L = smc.lib()
    lat = smc.Lattice(8, 8, 8, 2)
    m = smc.Model(smc.PAIR_I32, 2, inputs.pair_int_coeffs(1, 2, 2), unit_ev=1e-4)
    kt = np.array([0.025])
    occ = torch.zeros(lat.nsites, dtype=torch.int8, device="cuda:0")
    rc = L.smc_sweep_noalloc(C.byref(lat._c), C.byref(m._c), C.c_void_p(occ.data_ptr()), 1, 0, 0, 1,
                             kt.ctypes.data_as(C.POINTER(C.c_double)), None, None, None,
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == smc.SMC_ERR_UNSUPPORTED
