"""Serial CPU oracle for BCC swap Monte Carlo (SMC-X / SMC-AI, Algorithm 1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It wraps the
plain C oracle in ``smc_oracle.c`` (FP64 / int64, one trial at a time) with
ctypes over numpy arrays, and shares no code with the CUDA library.

Every function here is argument marshalling; the arithmetic is in C and each C
function cites the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "smc_oracle.c")

PAIR_I32, PAIR_F32, MLP, PAIR_F32_MLP, QSRO, MLPNET = 0, 1, 2, 3, 4, 5
MLP_IN, MLP_HID, NET_HID = 20, 64, 96
MLP_NPARAM = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID + 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain C, no FMA
    contraction so that x86 and Arm builds round identically)."""
    src_mtime = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "smc_oracle.h")))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= src_mtime:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Lat(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nspecies", C.c_int32)]


class _Model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nshells", C.c_int32),
                ("v_i32", C.POINTER(C.c_int32)), ("v_f32", C.POINTER(C.c_float)),
                ("unit_ev", C.c_double),
                ("w1", C.POINTER(C.c_double)), ("w2", C.POINTER(C.c_double)),
                ("w3", C.POINTER(C.c_double)),
                ("b1", C.POINTER(C.c_double)), ("b2", C.POINTER(C.c_double)),
                ("b3", C.c_double),
                ("qsro_w", C.POINTER(C.c_float)), ("qsro_c", C.c_double),
                ("net_w0", C.POINTER(C.c_double)), ("net_w1", C.POINTER(C.c_double)),
                ("net_w2", C.POINTER(C.c_double)), ("net_w3", C.POINTER(C.c_double)),
                ("net_b0", C.POINTER(C.c_double)), ("net_b1", C.POINTER(C.c_double)),
                ("net_b2", C.POINTER(C.c_double)), ("net_b3", C.c_double)]


_lib = None


def bind(L):
    """Declares the C signatures on a loaded oracle library (also used by the
    tests that load deliberately broken builds of the oracle)."""
    P = C.POINTER
    L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
    L.orc_nsites.argtypes = [P(_Lat)]
    L.orc_nsites.restype = C.c_int64
    L.orc_neighbor.argtypes = [P(_Lat), C.c_int64, C.c_int, C.c_int, C.c_int]
    L.orc_neighbor.restype = C.c_int64
    L.orc_shell_vectors.argtypes = [C.c_int, P(C.c_int)]
    L.orc_schedule.argtypes = [P(_Lat), P(C.c_int32)]
    L.orc_init_lattice.argtypes = [P(_Lat), P(C.c_int64), C.c_uint64, C.c_uint32, P(C.c_int8)]
    L.orc_site_energy.argtypes = [P(_Lat), P(_Model), P(C.c_int8), C.c_int64]
    L.orc_site_energy.restype = C.c_double
    L.orc_total_energy.argtypes = [P(_Lat), P(_Model), P(C.c_int8)]
    L.orc_total_energy.restype = C.c_double
    L.orc_total_energy_i64.argtypes = [P(_Lat), P(_Model), P(C.c_int8)]
    L.orc_total_energy_i64.restype = C.c_int64
    L.orc_delta_e.argtypes = [P(_Lat), P(_Model), P(C.c_int8), C.c_int64, C.c_int64]
    L.orc_delta_e.restype = C.c_double
    L.orc_pair_counts.argtypes = [P(_Lat), C.c_int, P(C.c_int8), P(C.c_int64)]
    L.orc_sro.argtypes = [P(_Lat), C.c_int, P(C.c_int8), P(C.c_double)]
    L.orc_accept_table.argtypes = [C.c_double, C.c_double, P(C.c_uint32), C.c_int64]
    L.orc_accept_table.restype = C.c_int64
    L.orc_sweep.argtypes = [P(_Lat), P(_Model), P(C.c_int8), C.c_uint64, C.c_uint32,
                            C.c_uint64, C.c_int32, P(C.c_double), P(C.c_double),
                            P(C.c_int64), C.c_int]
    L.orc_ministep_trace.argtypes = [P(_Lat), P(_Model), P(C.c_int8), C.c_uint64, C.c_uint32,
                                     C.c_uint64, C.c_int32, C.c_double, P(C.c_double),
                                     P(C.c_uint8), P(C.c_int64), P(C.c_int64)]
    L.orc_ministep_trace.restype = C.c_int64
    L.orc_slab_ghost_cells.argtypes = [P(_Model)]
    L.orc_slab_ministep.argtypes = [P(_Lat), P(_Model), P(C.c_int8), C.c_int32, C.c_int32, C.c_int32,
                                    C.c_uint64, C.c_uint32, C.c_uint64, C.c_int32, C.c_double,
                                    P(C.c_double), P(C.c_int64)]
    L.orc_slab_ministep.restype = C.c_int64
    L.orc_fcc_nsites.argtypes = [P(_Lat)]
    L.orc_fcc_nsites.restype = C.c_int64
    L.orc_fcc_neighbor.argtypes = [P(_Lat), C.c_int64, C.c_int, C.c_int, C.c_int]
    L.orc_fcc_neighbor.restype = C.c_int64
    L.orc_fcc_shell_vectors.argtypes = [C.c_int, P(C.c_int)]
    L.orc_fcc_schedule.argtypes = [P(_Lat), P(C.c_int32)]
    L.orc_fcc_total_energy.argtypes = [P(_Lat), P(_Model), P(C.c_int8)]
    L.orc_fcc_total_energy.restype = C.c_double
    L.orc_fcc_total_energy_i64.argtypes = [P(_Lat), P(_Model), P(C.c_int8)]
    L.orc_fcc_total_energy_i64.restype = C.c_int64
    L.orc_fcc_delta_e.argtypes = [P(_Lat), P(_Model), P(C.c_int8), C.c_int64, C.c_int64]
    L.orc_fcc_delta_e.restype = C.c_double
    L.orc_fcc_sweep.argtypes = [P(_Lat), P(_Model), P(C.c_int8), C.c_uint64, C.c_uint32, C.c_uint64, C.c_int32,
                                P(C.c_double), P(C.c_double), P(C.c_int64)]
    L.orc_fcc_ministep_trace.argtypes = [P(_Lat), P(_Model), P(C.c_int8), C.c_uint64, C.c_uint32, C.c_uint64,
                                         C.c_int32, C.c_double, P(C.c_double), P(C.c_uint8), P(C.c_int64),
                                         P(C.c_int64)]
    L.orc_fcc_ministep_trace.restype = C.c_int64
    L.orc_grad_size.argtypes = [P(_Lat), P(_Model)]
    L.orc_grad_size.restype = C.c_int64
    L.orc_energy_grad.argtypes = [P(_Lat), P(_Model), P(C.c_int8), P(C.c_double)]
    L.orc_mlp_eval.argtypes = [P(_Model), P(C.c_double)]
    L.orc_mlpnet_eval.argtypes = [P(_Model), P(C.c_double)]
    L.orc_mlpnet_eval.restype = C.c_double
    L.orc_mlp_eval.restype = C.c_double
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = bind(C.CDLL(_LIB_PATH))
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Lattice:
    """Box of nx x ny x nz BCC cells (N = 2 nx ny nz sites) with S species."""

    def __init__(self, nx: int, ny: int, nz: int, nspecies: int):
        self.nx, self.ny, self.nz, self.nspecies = int(nx), int(ny), int(nz), int(nspecies)
        self._c = _Lat(self.nx, self.ny, self.nz, self.nspecies)

    @property
    def nsites(self) -> int:
        return 2 * self.nx * self.ny * self.nz


def _widen(a) -> np.ndarray:
    """BF16 bit patterns (uint16) or floats -> float64, exactly."""
    a = np.asarray(a)
    if a.dtype == np.uint16:
        a = (a.astype(np.uint32) << 16).view(np.float32)
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


class Model:
    """Energy model.  ``v`` is [nshells][S][S] (int32 units or float32 eV);
    ``mlp`` is a dict with w1/w2/w3 (uint16 BF16 bit patterns, or float64
    values for finite-difference checks) and b1/b2 (float32/float64), b3.
    qSRO models take ``v`` = V_m^{pp'} (float32, symmetric), ``qsro_w`` =
    W_m^p [nshells][S] (float32) and ``qsro_c`` = C (a float32 value).
    BF16 and FP32 values are widened to FP64 exactly."""

    def __init__(self, kind: int, nshells: int = 0, v=None, unit_ev: float = 1e-4, mlp=None, qsro_w=None,
                 qsro_c: float = 0.0, net=None):
        self.kind, self.nshells, self.unit_ev = int(kind), int(nshells), float(unit_ev)
        self._keep = []
        c = _Model()
        c.kind, c.nshells, c.unit_ev = self.kind, self.nshells, self.unit_ev
        if kind == PAIR_I32:
            self.v = np.ascontiguousarray(v, dtype=np.int32)
            c.v_i32 = _ptr(self.v, C.c_int32)
        elif kind in (PAIR_F32, PAIR_F32_MLP, QSRO):
            self.v = np.ascontiguousarray(v, dtype=np.float32)
            c.v_f32 = _ptr(self.v, C.c_float)
        if kind == QSRO:
            self.qsro_w = np.ascontiguousarray(qsro_w, dtype=np.float32)
            c.qsro_w = _ptr(self.qsro_w, C.c_float)
            c.qsro_c = float(np.float32(qsro_c))
        if kind == MLPNET:  # net: w0..w3 (BF16 bit patterns or floats), b0..b2, b3
            self.net = {k: _widen(net[k]) for k in ("w0", "w1", "w2", "w3", "b0", "b1", "b2")}
            sizes = dict(w0=NET_HID * MLP_IN, w1=NET_HID * NET_HID, w2=NET_HID * NET_HID, w3=NET_HID,
                         b0=NET_HID, b1=NET_HID, b2=NET_HID)
            for k, n in sizes.items():
                assert self.net[k].size == n, k
                setattr(c, "net_" + k, _ptr(self.net[k], C.c_double))
            c.net_b3 = float(net["b3"])
        if kind in (MLP, PAIR_F32_MLP):
            self.mlp = {k: _widen(mlp[k]) for k in ("w1", "w2", "w3", "b1", "b2")}
            assert self.mlp["w1"].size == MLP_HID * MLP_IN
            assert self.mlp["w2"].size == MLP_HID * MLP_HID
            assert self.mlp["w3"].size == MLP_HID
            assert self.mlp["b1"].size == MLP_HID and self.mlp["b2"].size == MLP_HID
            for k in ("w1", "w2", "w3", "b1", "b2"):
                setattr(c, k, _ptr(self.mlp[k], C.c_double))
            c.b3 = float(mlp["b3"])
        self._c = c


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def shell_vectors(shell: int) -> np.ndarray:
    buf = np.zeros((12, 3), dtype=np.int32)
    n = lib().orc_shell_vectors(shell, _ptr(buf, C.c_int))
    return buf[:n].copy()


def neighbor(lat: Lattice, s: int, v) -> int:
    return int(lib().orc_neighbor(C.byref(lat._c), int(s), int(v[0]), int(v[1]), int(v[2])))


def schedule(lat: Lattice):
    L = np.zeros(3, dtype=np.int32)
    nA = lib().orc_schedule(C.byref(lat._c), _ptr(L, C.c_int32))
    return int(nA), tuple(int(x) for x in L)


def init_lattice(lat: Lattice, counts, seed: int, replica: int = 0) -> np.ndarray:
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    occ = np.zeros(lat.nsites, dtype=np.int8)
    rc = lib().orc_init_lattice(C.byref(lat._c), _ptr(cnt, C.c_int64), C.c_uint64(seed),
                                C.c_uint32(replica), _ptr(occ, C.c_int8))
    if rc != 0:
        raise ValueError("orc_init_lattice rejected its arguments")
    return occ


def _occ(occ: np.ndarray) -> np.ndarray:
    assert occ.dtype == np.int8 and occ.flags.c_contiguous
    return occ


def site_energy(lat, model, occ, i) -> float:
    return lib().orc_site_energy(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8), int(i))


def total_energy(lat, model, occ) -> float:
    return lib().orc_total_energy(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8))


def total_energy_i64(lat, model, occ) -> int:
    return int(lib().orc_total_energy_i64(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8)))


def delta_e(lat, model, occ, a, b) -> float:
    return lib().orc_delta_e(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8), int(a), int(b))


def pair_counts(lat, nshells, occ) -> np.ndarray:
    out = np.zeros((nshells, lat.nspecies, lat.nspecies), dtype=np.int64)
    lib().orc_pair_counts(C.byref(lat._c), int(nshells), _ptr(_occ(occ), C.c_int8), _ptr(out, C.c_int64))
    return out


def sro(lat, nshells, occ) -> np.ndarray:
    out = np.zeros((nshells, lat.nspecies, lat.nspecies), dtype=np.float64)
    lib().orc_sro(C.byref(lat._c), int(nshells), _ptr(_occ(occ), C.c_int8), _ptr(out, C.c_double))
    return out


def accept_table(unit_ev: float, kT: float) -> np.ndarray:
    n = lib().orc_accept_table(unit_ev, kT, None, 0)
    if n < 0:
        raise ValueError("acceptance table too long")
    t = np.zeros(max(n, 1), dtype=np.uint32)
    lib().orc_accept_table(unit_ev, kT, _ptr(t, C.c_uint32), n)
    return t[:n]


def sweep(lat, model, occ, seed, sweep0, nsweeps, kT, replica=0, mode=0):
    """Runs nsweeps sweeps in place; returns (sum of accepted dE, accepted count)."""
    kTa = np.ascontiguousarray(np.broadcast_to(np.asarray(kT, dtype=np.float64), (nsweeps,)))
    e = C.c_double(0.0)
    n = C.c_int64(0)
    rc = lib().orc_sweep(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8),
                         C.c_uint64(seed), C.c_uint32(replica), C.c_uint64(sweep0),
                         int(nsweeps), _ptr(kTa, C.c_double), C.byref(e), C.byref(n), int(mode))
    if rc != 0:
        raise ValueError("orc_sweep rejected its arguments")
    return e.value, n.value


def ministep_trace(lat, model, occ, seed, sweep_index, k, kT, replica=0):
    """Applies mini-step k; returns per-trial (dE, accepted, a, b) in link-cell order."""
    nA, _ = schedule(lat)
    nt = lat.nsites // nA
    dE = np.zeros(nt, dtype=np.float64)
    acc = np.zeros(nt, dtype=np.uint8)
    a = np.zeros(nt, dtype=np.int64)
    b = np.zeros(nt, dtype=np.int64)
    n = lib().orc_ministep_trace(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8),
                                 C.c_uint64(seed), C.c_uint32(replica), C.c_uint64(sweep_index),
                                 int(k), float(kT), _ptr(dE, C.c_double), _ptr(acc, C.c_uint8),
                                 _ptr(a, C.c_int64), _ptr(b, C.c_int64))
    if n < 0:
        raise ValueError("orc_ministep_trace rejected its arguments")
    return dE, acc.astype(bool), a, b


def slab_ghost_cells(model) -> int:
    return int(lib().orc_slab_ghost_cells(C.byref(model._c)))


def slab_ministep(lat, model, occ_loc, x0, w, g, seed, sweep_index, k, kT, replica=0):
    """Mini-step k on one x-slab: occ_loc holds cells [x0 - g, x0 + w + g) of
    the box `lat` as a [2][nz][ny][w + 2g] int8 array, updated in place.
    Returns (sum of accepted dE, accepted count, trials)."""
    e = C.c_double(0.0)
    n = C.c_int64(0)
    nt = lib().orc_slab_ministep(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ_loc), C.c_int8),
                                 int(x0), int(w), int(g), C.c_uint64(seed), C.c_uint32(replica),
                                 C.c_uint64(sweep_index), int(k), float(kT), C.byref(e), C.byref(n))
    if nt < 0:
        raise ValueError("orc_slab_ministep rejected its arguments")
    return e.value, n.value, int(nt)


# ---- FCC lattice (pair models): a Lattice(nx, ny, nz, S) read as nx x ny x nz
# cubic cells of 4 sites; N = 4 nx ny nz ----
def fcc_nsites(lat) -> int:
    return 4 * lat.nx * lat.ny * lat.nz


def fcc_shell_vectors(shell: int) -> np.ndarray:
    buf = np.zeros((24, 3), dtype=np.int32)
    n = lib().orc_fcc_shell_vectors(shell, _ptr(buf, C.c_int))
    return buf[:n].copy()


def fcc_neighbor(lat, s: int, v) -> int:
    return int(lib().orc_fcc_neighbor(C.byref(lat._c), int(s), int(v[0]), int(v[1]), int(v[2])))


def fcc_schedule(lat):
    L = np.zeros(3, dtype=np.int32)
    nA = lib().orc_fcc_schedule(C.byref(lat._c), _ptr(L, C.c_int32))
    return int(nA), tuple(int(x) for x in L)


def fcc_init_lattice(lat, counts, seed: int, replica: int = 0) -> np.ndarray:
    """The composition-conserving start state: the site order of the BCC init
    over the same N = 4 nx ny nz site ids."""
    return init_lattice(Lattice(2 * lat.nx, lat.ny, lat.nz, lat.nspecies), counts, seed, replica)


def fcc_total_energy(lat, model, occ) -> float:
    return lib().orc_fcc_total_energy(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8))


def fcc_total_energy_i64(lat, model, occ) -> int:
    return int(lib().orc_fcc_total_energy_i64(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8)))


def fcc_delta_e(lat, model, occ, a, b) -> float:
    return lib().orc_fcc_delta_e(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8), int(a), int(b))


def fcc_sweep(lat, model, occ, seed, sweep0, nsweeps, kT, replica=0):
    kTa = np.ascontiguousarray(np.broadcast_to(np.asarray(kT, dtype=np.float64), (nsweeps,)))
    e = C.c_double(0.0)
    n = C.c_int64(0)
    rc = lib().orc_fcc_sweep(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8), C.c_uint64(seed),
                             C.c_uint32(replica), C.c_uint64(sweep0), int(nsweeps), _ptr(kTa, C.c_double),
                             C.byref(e), C.byref(n))
    if rc != 0:
        raise ValueError("orc_fcc_sweep rejected its arguments")
    return e.value, n.value


def fcc_ministep_trace(lat, model, occ, seed, sweep_index, k, kT, replica=0):
    nA, _ = fcc_schedule(lat)
    nt = fcc_nsites(lat) // nA
    dE = np.zeros(nt, dtype=np.float64)
    acc = np.zeros(nt, dtype=np.uint8)
    a = np.zeros(nt, dtype=np.int64)
    b = np.zeros(nt, dtype=np.int64)
    n = lib().orc_fcc_ministep_trace(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8),
                                     C.c_uint64(seed), C.c_uint32(replica), C.c_uint64(sweep_index), int(k), float(kT),
                                     _ptr(dE, C.c_double), _ptr(acc, C.c_uint8), _ptr(a, C.c_int64),
                                     _ptr(b, C.c_int64))
    if n < 0:
        raise ValueError("orc_fcc_ministep_trace rejected its arguments")
    return dE, acc.astype(bool), a, b


def energy_grad(lat, model, occ) -> np.ndarray:
    n = lib().orc_grad_size(C.byref(lat._c), C.byref(model._c))
    g = np.zeros(n, dtype=np.float64)
    rc = lib().orc_energy_grad(C.byref(lat._c), C.byref(model._c), _ptr(_occ(occ), C.c_int8), _ptr(g, C.c_double))
    if rc != 0:
        raise ValueError("orc_energy_grad rejected its arguments")
    return g


def mlpnet_eval(model, x) -> float:
    xa = np.ascontiguousarray(x, dtype=np.float64)
    assert xa.size == MLP_IN
    return lib().orc_mlpnet_eval(C.byref(model._c), _ptr(xa, C.c_double))


def mlp_eval(model, x) -> float:
    xa = np.ascontiguousarray(x, dtype=np.float64)
    assert xa.size == MLP_IN
    return lib().orc_mlp_eval(C.byref(model._c), _ptr(xa, C.c_double))
