"""Python binding of libsmc.so (ctypes).  Argument marshalling only: every step
of the Monte Carlo path runs in the library's CUDA kernels.  Device buffers are
torch tensors; work is enqueued on torch's current CUDA stream.

The library must have been built (``paper_2604_08250_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsmc.so")

SMC_OK, SMC_ERR_ARG, SMC_ERR_UNSUPPORTED, SMC_ERR_CUDA, SMC_ERR_TIMEOUT, SMC_ERR_STATE = 0, -1, -2, -3, -4, -5
PAIR_I32, PAIR_F32, MLP_BF16, PAIR_F32_MLP_BF16, QSRO_F32, MLPNET_BF16 = 0, 1, 2, 3, 4, 5
DBG_TIMEOUT_MS, DBG_SKIP_PUBLISH, DBG_FAST_TEAM, DBG_FAST_BUFFERS, DBG_FAST_STAGING, DBG_RESIDENT = 1, 2, 3, 4, 5, 6
MLP_NPARAM = 64 * 20 + 64 + 64 * 64 + 64 + 64 + 1

# Every symbol declared in include/smc.h.
EXPORTS = ("smc_init_lattice", "smc_sweep", "smc_sweep_noalloc", "smc_sweep_batched", "smc_sro", "smc_energy", "smc_grad_size",
           "smc_energy_grad", "smc_ministep_trace", "smc_philox4x32_10", "smc_check", "smc_last_error",
           "smc_set_tuning", "smc_debug_set", "smc_fcc_init_lattice", "smc_fcc_sweep", "smc_fcc_ministep_trace",
           "smc_fcc_energy", "smc_slab_ministep")


class SMCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"smc error {code}: {msg}")
        self.code = code


class _Lat(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nspecies", C.c_int32)]


class _Model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nshells", C.c_int32),
                ("v_i32", C.POINTER(C.c_int32)), ("v_f32", C.POINTER(C.c_float)),
                ("unit_ev", C.c_double),
                ("mlp_w1", C.POINTER(C.c_uint16)), ("mlp_w2", C.POINTER(C.c_uint16)),
                ("mlp_w3", C.POINTER(C.c_uint16)),
                ("mlp_b1", C.POINTER(C.c_float)), ("mlp_b2", C.POINTER(C.c_float)),
                ("mlp_b3", C.c_float),
                ("qsro_w", C.POINTER(C.c_float)), ("qsro_c", C.c_float),
                ("net_w0", C.POINTER(C.c_uint16)), ("net_w1", C.POINTER(C.c_uint16)),
                ("net_w2", C.POINTER(C.c_uint16)), ("net_w3", C.POINTER(C.c_uint16)),
                ("net_b0", C.POINTER(C.c_float)), ("net_b1", C.POINTER(C.c_float)),
                ("net_b2", C.POINTER(C.c_float)), ("net_b3", C.c_float)]


class _Tuning(C.Structure):
    _fields_ = [("tile_y", C.c_int32), ("tile_z", C.c_int32), ("threads", C.c_int32),
                ("ctas_per_sm", C.c_int32)]


_lib = None


def lib():
    """Loads libsmc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsmc.so not found at {LIB_PATH}: build it with "
                              "paper_2604_08250_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P, vp = C.POINTER, C.c_void_p
        L.smc_last_error.restype = C.c_char_p
        L.smc_init_lattice.argtypes = [P(_Lat), P(C.c_int64), C.c_uint64, C.c_uint32, vp, vp]
        L.smc_sweep.argtypes = [P(_Lat), P(_Model), vp, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int32,
                                P(C.c_double), vp, vp, vp]
        L.smc_sweep_noalloc.argtypes = [P(_Lat), P(_Model), vp, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int32,
                                         P(C.c_double), vp, vp, vp, vp]
        L.smc_sweep_batched.argtypes = [C.c_int32, P(_Lat), P(_Model), P(vp), C.c_uint64, C.c_uint32,
                                        C.c_uint64, C.c_int32, P(C.c_double), vp, vp, vp]
        L.smc_sro.argtypes = [P(_Lat), C.c_int32, vp, vp, vp, vp]
        L.smc_energy.argtypes = [P(_Lat), P(_Model), vp, vp, vp, vp]
        L.smc_grad_size.argtypes = [P(_Lat), P(_Model)]
        L.smc_grad_size.restype = C.c_int64
        L.smc_energy_grad.argtypes = [P(_Lat), P(_Model), vp, vp, vp]
        L.smc_ministep_trace.argtypes = [P(_Lat), P(_Model), vp, C.c_uint64, C.c_uint32, C.c_uint64,
                                         C.c_int32, C.c_double, vp, vp, vp]
        L.smc_fcc_init_lattice.argtypes = [P(_Lat), P(C.c_int64), C.c_uint64, C.c_uint32, vp, vp]
        L.smc_fcc_sweep.argtypes = [P(_Lat), P(_Model), vp, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int32,
                                    P(C.c_double), vp, vp, vp]
        L.smc_fcc_ministep_trace.argtypes = [P(_Lat), P(_Model), vp, C.c_uint64, C.c_uint32, C.c_uint64,
                                             C.c_int32, C.c_double, vp, vp, vp]
        L.smc_fcc_energy.argtypes = [P(_Lat), P(_Model), vp, vp, vp, vp]
        L.smc_slab_ministep.argtypes = [P(_Lat), P(_Model), vp, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                                        C.c_uint32, C.c_uint64, C.c_int32, C.c_double, vp, vp, C.c_int32, vp]
        L.smc_philox4x32_10.argtypes = [vp, vp, vp, C.c_int64, vp]
        L.smc_check.argtypes = [vp]
        L.smc_set_tuning.argtypes = [P(_Tuning)]
        L.smc_debug_set.argtypes = [C.c_int32, C.c_int64]
        for name in ("smc_init_lattice", "smc_sweep", "smc_sweep_noalloc", "smc_sweep_batched", "smc_sro", "smc_energy",
                     "smc_energy_grad", "smc_ministep_trace", "smc_philox4x32_10", "smc_check",
                     "smc_set_tuning", "smc_debug_set", "smc_fcc_init_lattice", "smc_fcc_sweep",
                     "smc_fcc_ministep_trace", "smc_fcc_energy", "smc_slab_ministep"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _chk(code: int):
    if code != SMC_OK:
        raise SMCError(code, lib().smc_last_error().decode())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, dtype=None):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


class Lattice:
    """nx x ny x nz BCC cells (N = 2 nx ny nz sites), nspecies species."""

    def __init__(self, nx, ny, nz, nspecies):
        self.nx, self.ny, self.nz, self.nspecies = int(nx), int(ny), int(nz), int(nspecies)
        self._c = _Lat(self.nx, self.ny, self.nz, self.nspecies)

    @property
    def nsites(self):
        return 2 * self.nx * self.ny * self.nz


class Model:
    """Energy model: pair coefficients v [nshells][S][S] (int32 units of unit_ev,
    or float32 eV) and/or an MLP given as a dict of BF16 bit patterns
    (w1 [64,20], w2 [64,64], w3 [64], uint16) and FP32 biases (b1, b2, b3).
    qSRO: v = V_m^{pp'} (float32, symmetric), qsro_w = W_m^p [nshells][S]
    (float32), qsro_c = C."""

    def __init__(self, kind, nshells=0, v=None, unit_ev=1e-4, mlp=None, qsro_w=None, qsro_c=0.0, net=None):
        self.kind, self.nshells, self.unit_ev = int(kind), int(nshells), float(unit_ev)
        c = _Model()
        c.kind, c.nshells, c.unit_ev = self.kind, self.nshells, self.unit_ev
        if kind == PAIR_I32:
            self.v = np.ascontiguousarray(v, dtype=np.int32)
            c.v_i32 = self.v.ctypes.data_as(C.POINTER(C.c_int32))
        elif kind in (PAIR_F32, PAIR_F32_MLP_BF16, QSRO_F32):
            self.v = np.ascontiguousarray(v, dtype=np.float32)
            c.v_f32 = self.v.ctypes.data_as(C.POINTER(C.c_float))
        if kind == QSRO_F32:
            self.qsro_w = np.ascontiguousarray(qsro_w, dtype=np.float32)
            c.qsro_w = self.qsro_w.ctypes.data_as(C.POINTER(C.c_float))
            c.qsro_c = float(qsro_c)
        if kind == MLPNET_BF16:  # net: w0..w3 BF16 bit patterns, b0..b2 FP32, b3
            self.net = {k: np.ascontiguousarray(net[k], dtype=np.uint16).reshape(-1) for k in ("w0", "w1", "w2", "w3")}
            for k in ("b0", "b1", "b2"):
                self.net[k] = np.ascontiguousarray(net[k], dtype=np.float32).reshape(-1)
            for k in ("w0", "w1", "w2", "w3"):
                setattr(c, "net_" + k, self.net[k].ctypes.data_as(C.POINTER(C.c_uint16)))
            for k in ("b0", "b1", "b2"):
                setattr(c, "net_" + k, self.net[k].ctypes.data_as(C.POINTER(C.c_float)))
            c.net_b3 = float(net["b3"])
        if kind in (MLP_BF16, PAIR_F32_MLP_BF16):
            self.mlp = {k: np.ascontiguousarray(mlp[k], dtype=np.uint16).reshape(-1) for k in ("w1", "w2", "w3")}
            for k in ("b1", "b2"):
                self.mlp[k] = np.ascontiguousarray(mlp[k], dtype=np.float32).reshape(-1)
            for k in ("w1", "w2", "w3"):
                setattr(c, "mlp_" + k, self.mlp[k].ctypes.data_as(C.POINTER(C.c_uint16)))
            for k in ("b1", "b2"):
                setattr(c, "mlp_" + k, self.mlp[k].ctypes.data_as(C.POINTER(C.c_float)))
            c.mlp_b3 = float(mlp["b3"])
        self._c = c


def init_lattice(lat, counts, seed, occ, replica=0):
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    _chk(lib().smc_init_lattice(C.byref(lat._c), cnt.ctypes.data_as(C.POINTER(C.c_int64)), C.c_uint64(seed),
                                C.c_uint32(replica), _dptr(occ), _stream()))


def sweep(lat, model, occ, seed, sweep0, nsweeps, kT, replica=0, e_acc=None, n_acc=None):
    import torch
    kTa = np.ascontiguousarray(np.broadcast_to(np.asarray(kT, dtype=np.float64), (nsweeps,)))
    _chk(lib().smc_sweep(C.byref(lat._c), C.byref(model._c), _dptr(occ, torch.int8), C.c_uint64(seed),
                         C.c_uint32(replica), C.c_uint64(sweep0), int(nsweeps),
                         kTa.ctypes.data_as(C.POINTER(C.c_double)), _dptr(e_acc, torch.float64),
                         _dptr(n_acc, torch.int64), _stream()))


def sweep_batched(lats, model, occs, seed, sweep0, nsweeps, kT, replica0=0, e_acc=None, n_acc=None):
    import torch
    R = len(lats)
    larr = (_Lat * R)(*[l._c for l in lats])
    parr = (C.c_void_p * R)(*[_dptr(o, torch.int8).value for o in occs])
    kTa = np.ascontiguousarray(np.broadcast_to(np.asarray(kT, dtype=np.float64).reshape(R, -1), (R, nsweeps)))
    _chk(lib().smc_sweep_batched(R, larr, C.byref(model._c), parr, C.c_uint64(seed), C.c_uint32(replica0),
                                 C.c_uint64(sweep0), int(nsweeps), kTa.ctypes.data_as(C.POINTER(C.c_double)),
                                 _dptr(e_acc, torch.float64), _dptr(n_acc, torch.int64), _stream()))


def sro(lat, nshells, occ, counts=None, alpha=None):
    import torch
    _chk(lib().smc_sro(C.byref(lat._c), int(nshells), _dptr(occ, torch.int8), _dptr(counts, torch.int64),
                       _dptr(alpha, torch.float64), _stream()))


def energy(lat, model, occ, e=None, e_int=None):
    import torch
    _chk(lib().smc_energy(C.byref(lat._c), C.byref(model._c), _dptr(occ, torch.int8), _dptr(e, torch.float64),
                          _dptr(e_int, torch.int64), _stream()))


def grad_size(lat, model) -> int:
    return int(lib().smc_grad_size(C.byref(lat._c), C.byref(model._c)))


def energy_grad(lat, model, occ, grad):
    import torch
    _chk(lib().smc_energy_grad(C.byref(lat._c), C.byref(model._c), _dptr(occ, torch.int8),
                               _dptr(grad, torch.float32), _stream()))


def ministep_trace(lat, model, occ, seed, sweep_index, k, kT, dE=None, acc=None, replica=0):
    import torch
    _chk(lib().smc_ministep_trace(C.byref(lat._c), C.byref(model._c), _dptr(occ, torch.int8), C.c_uint64(seed),
                                  C.c_uint32(replica), C.c_uint64(sweep_index), int(k), float(kT),
                                  _dptr(dE, torch.float32), _dptr(acc, torch.uint8), _stream()))


def slab_ministep(lat, model, win, x0, w, g, seed, sweep_index, k, kT, part=0, e_acc=None, n_acc=None, replica=0):
    """Mini-step k on one x-slab: win (device int8 [2][nz][ny][w + 2g]) holds
    cells [x0 - g, x0 + w + g) of the box lat; part 0 all link cells, 1 the
    edge link cells, 2 the interior ones (smc_slab_ministep)."""
    import torch
    _chk(lib().smc_slab_ministep(C.byref(lat._c), C.byref(model._c), _dptr(win, torch.int8), int(x0), int(w), int(g),
                                 C.c_uint64(seed), C.c_uint32(replica), C.c_uint64(sweep_index), int(k), float(kT),
                                 _dptr(e_acc, torch.float64), _dptr(n_acc, torch.int64), int(part), _stream()))


def fcc_nsites(lat) -> int:
    """Sites of lat read as nx x ny x nz FCC cubic cells (4 per cell)."""
    return 4 * lat.nx * lat.ny * lat.nz


def fcc_init_lattice(lat, counts, seed, occ, replica=0):
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    _chk(lib().smc_fcc_init_lattice(C.byref(lat._c), cnt.ctypes.data_as(C.POINTER(C.c_int64)), C.c_uint64(seed),
                                    C.c_uint32(replica), _dptr(occ), _stream()))


def fcc_sweep(lat, model, occ, seed, sweep0, nsweeps, kT, replica=0, e_acc=None, n_acc=None):
    import torch
    kTa = np.ascontiguousarray(np.broadcast_to(np.asarray(kT, dtype=np.float64), (nsweeps,)))
    _chk(lib().smc_fcc_sweep(C.byref(lat._c), C.byref(model._c), _dptr(occ, torch.int8), C.c_uint64(seed),
                             C.c_uint32(replica), C.c_uint64(sweep0), int(nsweeps),
                             kTa.ctypes.data_as(C.POINTER(C.c_double)), _dptr(e_acc, torch.float64),
                             _dptr(n_acc, torch.int64), _stream()))


def fcc_ministep_trace(lat, model, occ, seed, sweep_index, k, kT, dE=None, acc=None, replica=0):
    import torch
    _chk(lib().smc_fcc_ministep_trace(C.byref(lat._c), C.byref(model._c), _dptr(occ, torch.int8),
                                      C.c_uint64(seed), C.c_uint32(replica), C.c_uint64(sweep_index), int(k),
                                      float(kT), _dptr(dE, torch.float32), _dptr(acc, torch.uint8), _stream()))


def fcc_energy(lat, model, occ, e=None, e_int=None):
    import torch
    _chk(lib().smc_fcc_energy(C.byref(lat._c), C.byref(model._c), _dptr(occ, torch.int8),
                              _dptr(e, torch.float64), _dptr(e_int, torch.int64), _stream()))


def philox4x32_10(ctr, key, out):
    import torch
    n = ctr.numel() // 4
    _chk(lib().smc_philox4x32_10(_dptr(ctr, torch.int32), _dptr(key, torch.int32), _dptr(out, torch.int32),
                                 n, _stream()))


def check():
    """Synchronises the current stream and raises on a latched device error."""
    _chk(lib().smc_check(_stream()))


def set_tuning(tile_y=0, tile_z=0, threads=0, ctas_per_sm=0):
    t = _Tuning(int(tile_y), int(tile_z), int(threads), int(ctas_per_sm))
    _chk(lib().smc_set_tuning(C.byref(t)))


def debug_set(what, value):
    _chk(lib().smc_debug_set(int(what), int(value)))


# ---------------------------------------------------------------------------
# Parameter vectors, autograd and observable gradients.
# ---------------------------------------------------------------------------
def _bf16_bits(a):
    """float -> BF16 bit patterns, round to nearest even (through FP32)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def n_pair_params(nshells, S):
    return nshells * S * (S + 1) // 2


def model_from_theta(kind, nshells, S, theta):
    """Model from a parameter vector in the smc_energy_grad layout: pair
    coefficients V_m(p, q), p <= q, row-major over (m, p, q) (FP32 eV), then
    the MLP parameters W1 [64][20], b1, W2 [64][64], b2, W3, b3 (weights are
    rounded to BF16, the precision the kernels use)."""
    th = np.asarray(theta, dtype=np.float64).reshape(-1)
    k = 0
    v = None
    if kind in (PAIR_F32, PAIR_F32_MLP_BF16):
        v = np.zeros((nshells, S, S), dtype=np.float32)
        for m in range(nshells):
            for p in range(S):
                for q in range(p, S):
                    v[m, p, q] = v[m, q, p] = th[k]
                    k += 1
    elif kind != MLP_BF16:
        raise ValueError("parameter vectors are defined for PAIR_F32, MLP_BF16 and PAIR_F32_MLP_BF16 models")
    mlp = None
    if kind in (MLP_BF16, PAIR_F32_MLP_BF16):
        sizes = (("w1", 64 * 20), ("b1", 64), ("w2", 64 * 64), ("b2", 64), ("w3", 64), ("b3", 1))
        mlp = {}
        for name, n in sizes:
            mlp[name] = th[k:k + n]
            k += n
        for name in ("w1", "w2", "w3"):
            mlp[name] = _bf16_bits(mlp[name])
        mlp["b3"] = float(mlp["b3"][0])
    if k != th.size:
        raise ValueError(f"theta has {th.size} entries, the model needs {k}")
    return Model(kind, nshells=nshells if v is not None else 0, v=v, mlp=mlp)


def _autograd_function():
    import torch

    class SMCEnergy(torch.autograd.Function):
        """E(theta) of the configuration occ.  theta is a 1-D tensor in the
        smc_energy_grad layout (see model_from_theta); forward runs
        smc_energy, backward grad_out * smc_energy_grad at the same theta."""

        @staticmethod
        def forward(ctx, theta, lat, occ, kind, nshells):
            th = theta.detach().cpu().numpy()
            model = model_from_theta(kind, nshells, lat.nspecies, th)
            e = torch.zeros(1, dtype=torch.float64, device=occ.device)
            energy(lat, model, occ, e)
            ctx.lat, ctx.occ, ctx.model = lat, occ, model
            return e.reshape(()).to(theta.dtype).to(theta.device)

        @staticmethod
        def backward(ctx, gout):
            g = torch.zeros(grad_size(ctx.lat, ctx.model), dtype=torch.float32, device=ctx.occ.device)
            energy_grad(ctx.lat, ctx.model, ctx.occ, g)
            return gout * g.to(gout.dtype).to(gout.device), None, None, None, None

    return SMCEnergy


_SMCEnergy = None


def smc_energy_fn(theta, lat, occ, kind, nshells=0):
    """Differentiable E(theta) (torch.autograd) of the configuration occ."""
    global _SMCEnergy
    if _SMCEnergy is None:
        _SMCEnergy = _autograd_function()
    return _SMCEnergy.apply(theta, lat, occ, kind, nshells)


def observable_gradient(A, G, beta):
    """Canonical-ensemble derivative of an observable's mean with respect to
    the energy parameters, d<A>/dtheta = -beta (<A dE/dtheta> - <A><dE/dtheta>),
    from equilibrium samples: A [n, ...] (e.g. SRO per sample), G [n, P]
    (dE/dtheta per sample).  Returns [..., P]."""
    import torch
    A = torch.as_tensor(A, dtype=torch.float64)
    G = torch.as_tensor(G, dtype=torch.float64, device=A.device)
    n = A.shape[0]
    Ac = A.reshape(n, -1) - A.reshape(n, -1).mean(0)
    Gc = G - G.mean(0)
    cov = Ac.T @ Gc / n
    return (-beta * cov).reshape(*A.shape[1:], G.shape[1])
