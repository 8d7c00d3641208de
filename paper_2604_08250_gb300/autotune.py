"""Launch tuning and CUDA-graph capture for batched replica sweeps.

A batched sweep (smc_sweep_batched) advances replicas of different sizes in
one persistent launch per call.  Its domain tiles (link-cell columns per
tile along y and z) and CTA size do not change any result, only the time:
`autotune_batched` times a few candidate tunings on copies of the replicas
(the chains themselves are not advanced) and leaves the fastest one set for
later calls on this thread.  `capture_batched` records one batched call of
many sweeps in a CUDA graph after an identical warm-up call has built the
launch plan and grown the library's workspace, so the captured call
allocates nothing; replaying the graph runs the whole call as one launch.
Only argument marshalling and timing live here; the sweeps run in libsmc.so.
"""
from __future__ import annotations

import numpy as np

from . import smc

# (tile_y, tile_z, threads, ctas_per_sm); 0 = the library's own choice
DEFAULT_CANDIDATES = [
    (0, 0, 0, 0),
    (1, 1, 128, 0),
    (1, 1, 256, 0),
    (1, 2, 256, 0),
    (2, 2, 256, 0),
    (2, 2, 128, 0),
]

_cache: dict = {}


def _key(lats, model):
    return (model.kind, model.nshells, tuple((l.nx, l.ny, l.nz, l.nspecies) for l in lats))


def autotune_batched(lats, model, occs, seed, kT, sweeps=2, candidates=None, replica0=0):
    """Times `sweeps` batched sweeps per candidate tuning on clones of `occs`
    and sets the fastest with smc.set_tuning.  kT: [R] or [R][sweeps] eV.
    Returns (best tuning tuple, {tuning: ms per sweep}).  Results are cached
    per (model kind, shells, replica shapes)."""
    import torch
    key = _key(lats, model)
    if key in _cache:
        best, times = _cache[key]
        smc.set_tuning(*best)
        return best, times
    R = len(lats)
    kTa = np.ascontiguousarray(np.broadcast_to(np.asarray(kT, dtype=np.float64).reshape(R, -1)[:, :1], (R, sweeps)))
    clones = [o.clone() for o in occs]
    stream = torch.cuda.current_stream()
    times = {}
    for cand in candidates or DEFAULT_CANDIDATES:
        smc.set_tuning(*cand)
        smc.sweep_batched(lats, model, clones, seed, 0, 1, kTa[:, :1], replica0=replica0)  # plan, workspace
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        smc.sweep_batched(lats, model, clones, seed, 1, sweeps, kTa, replica0=replica0)
        b.record(stream)
        b.synchronize()
        times[tuple(cand)] = a.elapsed_time(b) / sweeps
    smc.check()
    best = min(times, key=times.get)
    smc.set_tuning(*best)
    _cache[key] = (best, times)
    return best, times


def capture_batched(lats, model, occs, seed, sweep0, nsweeps, kT, replica0=0, e_acc=None, n_acc=None):
    """A CUDA graph of smc_sweep_batched(lats, model, occs, seed, sweep0,
    nsweeps, kT): each replay runs those sweeps on the current contents of
    `occs` (and adds to e_acc / n_acc).  Floating-point models only (an
    integer model's acceptance tables are copied from host memory per call).
    The warm-up call runs on clones, so `occs` is unchanged until a replay."""
    import torch
    if model.kind == smc.PAIR_I32:
        raise ValueError("graph capture takes floating-point models (integer tables are host copies)")
    R = len(lats)
    kTa = np.ascontiguousarray(np.broadcast_to(np.asarray(kT, dtype=np.float64).reshape(R, -1), (R, nsweeps)))
    clones = [o.clone() for o in occs]
    ea = None if e_acc is None else e_acc.clone()
    na = None if n_acc is None else n_acc.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # same shapes and arguments: plan cached, workspace grown
        smc.sweep_batched(lats, model, clones, seed, sweep0, nsweeps, kTa, replica0=replica0, e_acc=ea, n_acc=na)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    del clones
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        smc.sweep_batched(lats, model, occs, seed, sweep0, nsweeps, kTa, replica0=replica0, e_acc=e_acc,
                          n_acc=n_acc)
    return g
