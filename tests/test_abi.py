"""The C ABI library loads without a GPU and exports every symbol that
include/smc.h declares; argument errors are reported without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2604_08250_gb300 import build, inputs, smc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return smc.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "smc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(smc_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(smc.EXPORTS)


def test_argument_errors_need_no_gpu(L):
    bad = smc.Lattice(1, 8, 8, 2)
    counts = (ctypes.c_int64 * 2)(1, 1)
    rc = L.smc_init_lattice(ctypes.byref(bad._c), counts, 1, 0, None, None)
    assert rc == smc.SMC_ERR_ARG
    assert b"dimensions" in L.smc_last_error()
    lat = smc.Lattice(8, 8, 8, 2)
    m = smc.Model(smc.PAIR_I32, 2, [[[0, 1], [2, 0]], [[0, 0], [0, 0]]], unit_ev=1e-4)
    assert L.smc_energy(ctypes.byref(lat._c), ctypes.byref(m._c), ctypes.c_void_p(16), None, None, None) == \
        smc.SMC_ERR_ARG
    assert b"symmetric" in L.smc_last_error()
    assert L.smc_grad_size(ctypes.byref(lat._c), ctypes.byref(m._c)) == 6
    assert smc.grad_size(smc.Lattice(4, 4, 4, 5), smc.Model(smc.PAIR_F32_MLP_BF16, 2, [[[0.0] * 5] * 5] * 2,
                         mlp={"w1": [0] * 1280, "w2": [0] * 4096, "w3": [0] * 64, "b1": [0.0] * 64,
                              "b2": [0.0] * 64, "b3": 0.0})) == 30 + smc.MLP_NPARAM


def test_fcc_argument_errors_need_no_gpu(L):
    V = [[[0, 1], [1, 0]]]
    m = smc.Model(smc.PAIR_I32, 1, V, unit_ev=1e-4)
    kT = (ctypes.c_double * 1)(0.05)
    for dims in ((6, 8, 8), (8, 8, 4)):
        lat = smc.Lattice(*dims, 2)
        rc = L.smc_fcc_sweep(ctypes.byref(lat._c), ctypes.byref(m._c), ctypes.c_void_p(16), 1, 0, 0, 1, kT, None,
                             None, None)
        assert rc == smc.SMC_ERR_UNSUPPORTED
        assert b"multiple of 4" in L.smc_last_error()
    lat = smc.Lattice(8, 8, 8, 2)
    rc = L.smc_fcc_ministep_trace(ctypes.byref(lat._c), ctypes.byref(m._c), ctypes.c_void_p(16), 1, 0, 0, 256,
                                  0.05, ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert rc == smc.SMC_ERR_ARG and b"mini-step" in L.smc_last_error()
    q = smc.Model(smc.MLP_BF16, mlp=inputs.mlp_weights(1))
    rc = L.smc_fcc_energy(ctypes.byref(lat._c), ctypes.byref(q._c), ctypes.c_void_p(16), None, None, None)
    assert rc == smc.SMC_ERR_UNSUPPORTED and b"pair models" in L.smc_last_error()
