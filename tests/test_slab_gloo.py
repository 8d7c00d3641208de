"""The slab-sharded schedule (1D slabs along x, ghost exchange after every
mini-step, Sec. III-B) run by CPU ranks of the oracle.

gloo ranks each hold one slab plus ghost cells and run the oracle's trials of
their link cells; the box they assemble must equal the single-rank oracle's
bit for bit, with the same accepted count and energy change.  Fault tests make
the failure on the host: a frame that is dropped or truncated before it is
sent, a rank that dies between mini-steps, a rank that arrives late.  The
surviving rank must raise SlabExchangeError within its receive timeout."""
import os
import re
import socket
import time

import numpy as np
import pytest

import oracle
from paper_2604_08250_gb300 import inputs, slab

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup(kind, dims, seed):
    """Oracle lattice, model, starting occupancy and temperature of one case."""
    if kind == "pair":
        S = 3
        lat = oracle.Lattice(*dims, S)
        model = oracle.Model(oracle.PAIR_I32, 2, inputs.pair_int_coeffs(3, 2, S), unit_ev=1e-4)
        occ = oracle.init_lattice(lat, inputs.equiatomic_counts(lat.nsites, S), seed)
        return lat, model, occ, 0.05
    S = 5
    lat = oracle.Lattice(*dims, S)
    model = oracle.Model(oracle.MLP, mlp=inputs.mlp_weights(4))
    occ = oracle.init_lattice(lat, inputs.dirichlet_counts(lat.nsites, S, 4), seed)
    return lat, model, occ, 0.07


def _ministep(lat, model, plan, rank, seed, kT):
    def f(local, s, k):
        e, n, _ = oracle.slab_ministep(lat, model, local, plan.x0(rank), plan.w, plan.ghost, seed, s, k, kT)
        return e, n
    return f


class _Faulty(slab.SlabExchange):
    """Drops or truncates one outgoing frame, on the host, before it is sent."""

    def __init__(self, *a, fault=None, at=None, **kw):
        super().__init__(*a, **kw)
        self.fault, self.at, self.now = fault, at, None

    def step(self, local, sweep, k):
        self.now = (sweep, k)
        return super().step(local, sweep, k)

    def _emit(self, frame, dst, tag):
        if self.now == self.at and tag == slab.LEFTWARD:
            if self.fault == "drop":
                return None
            if self.fault == "truncate":
                frame = frame.copy()
                hdr = frame[:slab.HEADER].view(np.int64)
                n = int(hdr[6])
                hdr[6] = max(n - 1, 0)
                frame[slab.HEADER + max(n - 1, 0) * self.plan.cell_bytes:] = 0
        return super()._emit(frame, dst, tag)


def _rank_main(rank, world, port, cfg, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    out = {"rank": rank}
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        if cfg.get("fault") == "late" and rank == 1:
            time.sleep(cfg["late_s"])
        lat, model, occ, kT = _setup(cfg["kind"], cfg["dims"], cfg["seed"])
        plan = slab.SlabPlan(lat.nx, lat.ny, lat.nz, world, oracle.slab_ghost_cells(model))
        if cfg.get("fault") in ("drop", "truncate") and rank == 1:
            ex = _Faulty(plan, rank, dist, timeout_s=cfg["timeout_s"], fault=cfg["fault"], at=cfg["at"])
        else:
            ex = slab.SlabExchange(plan, rank, dist, timeout_s=cfg["timeout_s"])
        local = plan.window_of(occ, rank)
        step = _ministep(lat, model, plan, rank, cfg["seed"], kT)
        if cfg.get("fault") == "crash" and rank == 1:
            inner = step

            def step(local, s, k):
                if (s, k) == cfg["at"]:
                    raise RuntimeError("rank 1 crashed")
                return inner(local, s, k)
        t0 = time.monotonic()
        try:
            if cfg.get("torch"):
                # the window as a tensor (CPU, gloo) exchanged by TorchSlabExchange
                win = torch.from_numpy(local)
                tex = slab.TorchSlabExchange(plan, rank, dist, timeout_s=cfg["timeout_s"])
                e, n, steps = 0.0, 0, 0
                for t in range(cfg["nsweeps"]):
                    for k in range(plan.nA):
                        de, dn = step(local, t, k)
                        e, n = e + de, n + dn
                        if cfg.get("fault") == "skip" and rank == 1 and (t, k) == cfg["at"]:
                            continue
                        tex.step(win, t, k)
                        steps += 1
                ex.frames_sent = 2 * steps
            else:
                e, n = slab.run_sweeps(ex, local, step, 0, cfg["nsweeps"])
        finally:
            out["elapsed"] = time.monotonic() - t0
        tot = torch.tensor([e, float(n)], dtype=torch.float64)
        dist.all_reduce(tot)
        box = slab.gather(plan, local, rank, dist)
        out.update(e=float(tot[0]), n=int(tot[1]), box=box, window=local.copy(), frames=ex.frames_sent)
    except Exception as exc:  # reported to the parent, which decides
        out.update(error=type(exc).__name__, msg=str(exc))
    q.put(out)
    q.close()
    q.join_thread()
    os._exit(0)


def _run(world, cfg, wait_s=300):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, cfg, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    try:
        deadline = time.monotonic() + wait_s
        while len(res) < world and time.monotonic() < deadline:
            try:
                r = q.get(timeout=max(deadline - time.monotonic(), 0.1))
            except Exception:
                break
            res[r["rank"]] = r
    finally:
        for p in procs:
            p.join(timeout=10)
            if p.is_alive():
                p.kill()
                p.join(timeout=10)
    return res


# -- plan, frames and one-process schedule ----------------------------------

@pytest.mark.parametrize("world,ghost", [(1, 2), (2, 2), (2, 3), (4, 3)])
def test_changed_ranges_are_disjoint_and_near_their_slab(world, ghost):
    P = slab.SlabPlan(16, 8, 8, world, ghost)
    for k in range(P.nA):
        owner = {}
        for r in range(world):
            lo, hi = P.modified(r, k)
            assert P.x0(r) - 1 <= lo and hi <= P.x0(r) + P.w + 1
            for x in range(lo, hi):
                assert owner.setdefault(x % P.nx, r) == r
    assert P.max_cells <= ghost + 1


@pytest.mark.parametrize("kind", ["pair", "mlp"])
def test_trials_change_only_the_planned_cells(kind):
    """Every cell an oracle slab mini-step changes lies in modified(rank, k)."""
    lat, model, occ, kT = _setup(kind, (16, 8, 8), 7)
    P = slab.SlabPlan(lat.nx, lat.ny, lat.nz, 4, oracle.slab_ghost_cells(model))
    rng = np.random.default_rng(1)
    ks = list(range(P.nA)) if kind == "pair" else sorted(rng.choice(P.nA, 12, replace=False))
    seen = 0
    for k in ks:
        for r in range(P.world):
            local = P.window_of(occ, r)
            before = local.copy()
            oracle.slab_ministep(lat, model, local, P.x0(r), P.w, P.ghost, 7, 0, int(k), kT)
            changed = np.nonzero((local != before).any(axis=(0, 1, 2)))[0]
            lo, hi = P.modified(r, int(k))
            for j in changed:
                assert lo <= P.x0(r) - P.ghost + j < hi
            seen += len(changed)
    assert seen > 0


def test_slab_rejects_bad_arguments():
    lat, model, occ, kT = _setup("pair", (16, 8, 8), 1)
    local = slab.SlabPlan(16, 8, 8, 2, 2).window_of(occ, 0)
    with pytest.raises(ValueError):  # ghost narrower than the read reach
        oracle.slab_ministep(lat, model, slab.SlabPlan(16, 8, 8, 2, 1).window_of(occ, 0), 0, 8, 1, 1, 0, 0, kT)
    with pytest.raises(ValueError):  # slab start not on a link-cell boundary
        oracle.slab_ministep(lat, model, local, 2, 8, 2, 1, 0, 0, kT)
    for args in [(12, 8, 8, 2, 2), (4, 8, 8, 1, 2), (16, 8, 8, 4, 4), (16, 8, 8, 0, 2)]:
        with pytest.raises(ValueError):
            slab.SlabPlan(*args)


def test_frames_detect_truncation_corruption_and_reordering():
    P = slab.SlabPlan(16, 8, 8, 2, 2)
    occ = np.arange(P.nx * P.ny * P.nz * 2, dtype=np.int64).astype(np.int8)
    local = P.window_of(occ, 1)
    k = 3 + 64  # dx = 3 on sublattice 1: three cells go right
    cells = P.outgoing(1, k, 1)
    assert cells[1] - cells[0] == 3
    f = P.encode(1, 4, k, slab.RIGHTWARD, cells, P.pack(local, 1, cells))
    assert P.decode(f, 1, 4, k, slab.RIGHTWARD, cells) == P.pack(local, 1, cells)
    bad = f.copy()
    bad[:slab.HEADER].view(np.int64)[6] = 2
    with pytest.raises(slab.SlabExchangeError, match="truncated"):
        P.decode(bad, 1, 4, k, slab.RIGHTWARD, cells)
    bad = f.copy()
    bad[slab.HEADER + 5] ^= 1
    with pytest.raises(slab.SlabExchangeError, match="checksum"):
        P.decode(bad, 1, 4, k, slab.RIGHTWARD, cells)
    with pytest.raises(slab.SlabExchangeError, match="header"):
        P.decode(f, 1, 4, k + 1, slab.RIGHTWARD, cells)
    with pytest.raises(slab.SlabExchangeError, match="magic"):
        P.decode(np.zeros_like(f), 1, 4, k, slab.RIGHTWARD, cells)


@pytest.mark.parametrize("kind", ["pair", "mlp"])
def test_one_rank_with_periodic_ghosts_matches_oracle(kind):
    """world = 1: the slab is the whole box and its ghosts are its own
    periodic images, refreshed through the same frames in memory."""
    lat, model, occ, kT = _setup(kind, (8, 8, 8), 11)
    ref = occ.copy()
    nsw = 2 if kind == "pair" else 1
    e_ref, n_ref = oracle.sweep(lat, model, ref, 11, 0, nsw, kT)
    P = slab.SlabPlan(lat.nx, lat.ny, lat.nz, 1, oracle.slab_ghost_cells(model))
    local = P.window_of(occ, 0)
    e, n = slab.run_sweeps(slab.SlabExchange(P, 0), local, _ministep(lat, model, P, 0, 11, kT), 0, nsw)
    assert np.array_equal(slab.gather(P, local, 0).reshape(-1), ref)
    assert np.array_equal(local, P.window_of(ref, 0))
    assert n == n_ref and n > 0
    assert e == e_ref if kind == "pair" else abs(e - e_ref) <= 1e-12 * max(1.0, abs(e_ref))


@pytest.mark.parametrize("world", [1, 2, 4])
def test_local_exchange_of_tensor_windows_matches_oracle(world):
    """LocalSlabExchange (all slabs in one process, windows as tensors; on a
    GPU the exchange is device-to-device copies), here with CPU tensors and
    the oracle's slab mini-step: the single-rank oracle's box bit for bit."""
    lat, model, occ, kT = _setup("pair", (16, 8, 8), 13)
    ref = occ.copy()
    e_ref, n_ref = oracle.sweep(lat, model, ref, 13, 0, 2, kT)
    P = slab.SlabPlan(lat.nx, lat.ny, lat.nz, world, oracle.slab_ghost_cells(model))
    wins = [torch.from_numpy(P.window_of(occ, r)) for r in range(world)]
    ex = slab.LocalSlabExchange(P)
    e, n = 0.0, 0
    for t in range(2):
        for k in range(P.nA):
            for r in range(world):
                de, dn, _ = oracle.slab_ministep(lat, model, wins[r].numpy(), P.x0(r), P.w, P.ghost, 13, t, k, kT)
                e, n = e + de, n + dn
            ex.step(wins, t, k)
    box = np.concatenate([P.owned(w.numpy()) for w in wins], axis=-1).reshape(-1)
    assert np.array_equal(box, ref)
    assert n == n_ref and n > 0 and e == e_ref


# -- gloo ranks -------------------------------------------------------------

@pytest.mark.parametrize("kind,world,nsweeps,tensors", [("pair", 2, 3, False), ("pair", 4, 3, False),
                                                        ("mlp", 2, 1, False), ("pair", 2, 2, True),
                                                        ("pair", 4, 2, True)])
def test_gloo_ranks_match_single_rank_oracle(kind, world, nsweeps, tensors):
    """Frames of SlabExchange (host arrays), or TorchSlabExchange (windows as
    tensors, the transport of the nccl path, here on CPU tensors)."""
    seed, dims = 5, (16, 8, 8)
    cfg = dict(kind=kind, dims=dims, seed=seed, nsweeps=nsweeps, timeout_s=60, torch=tensors)
    res = _run(world, cfg)
    lat, model, occ, kT = _setup(kind, dims, seed)
    e_ref, n_ref = oracle.sweep(lat, model, occ, seed, 0, nsweeps, kT)
    P = slab.SlabPlan(lat.nx, lat.ny, lat.nz, world, oracle.slab_ghost_cells(model))
    assert sorted(res) == list(range(world)), res
    for r, out in res.items():
        assert "error" not in out, out
        assert np.array_equal(out["box"].reshape(-1), occ)
        assert np.array_equal(out["window"], P.window_of(occ, r))  # ghosts up to date too
        assert out["n"] == n_ref and n_ref > 0
        assert out["frames"] == 2 * P.nA * nsweeps
        if kind == "pair":  # integer dE: sums are exact in any order
            assert out["e"] == e_ref
        else:
            assert abs(out["e"] - e_ref) <= 1e-12 * max(1.0, abs(e_ref))


def _failed(out):
    return out.get("error") == "SlabExchangeError"


@pytest.mark.parametrize("fault,match", [("drop", r"rank 1\b.*mini-step 5\b"),
                                         ("truncate", r"mini-step 5\b.*truncated")])
def test_lost_or_truncated_frame_raises(fault, match):
    """A dropped frame ends rank 0's receive either by its timeout or by the
    next frame arriving out of sequence (the header names mini-step 6)."""
    cfg = dict(kind="pair", dims=(16, 8, 8), seed=2, nsweeps=1, timeout_s=3, fault=fault, at=(0, 5))
    t0 = time.monotonic()
    res = _run(2, cfg, wait_s=120)
    assert 0 in res and _failed(res[0]), res
    assert re.search(match, res[0]["msg"]), res[0]["msg"]
    assert 1 in res and _failed(res[1]), res  # the peer learns at its next receive
    assert time.monotonic() - t0 < 90


def test_dead_rank_is_detected():
    cfg = dict(kind="pair", dims=(16, 8, 8), seed=2, nsweeps=1, timeout_s=5, fault="crash", at=(0, 3))
    res = _run(2, cfg, wait_s=120)
    assert res[1]["error"] == "RuntimeError" and "crashed" in res[1]["msg"]
    assert _failed(res[0]), res
    assert "mini-step 3" in res[0]["msg"] or "mini-step 2" in res[0]["msg"]
    assert res[0]["elapsed"] < 5 + 30


def test_tensor_exchange_skipped_by_a_rank_raises():
    """TorchSlabExchange: rank 1 skips its exchange after mini-step 5; rank 0
    raises SlabExchangeError (receive timeout or a header naming another
    mini-step), and so does rank 1 at its next exchange."""
    cfg = dict(kind="pair", dims=(16, 8, 8), seed=2, nsweeps=1, timeout_s=3, fault="skip", at=(0, 5), torch=True)
    res = _run(2, cfg, wait_s=120)
    assert 0 in res and _failed(res[0]), res
    assert "mini-step 5" in res[0]["msg"] or "mini-step 6" in res[0]["msg"], res[0]["msg"]
    assert 1 in res and _failed(res[1]), res


def test_late_rank_times_out_receive():
    """Rank 1 joins the group but reaches the exchange 8 s late; rank 0's
    first receive gives up after its 2 s limit."""
    cfg = dict(kind="pair", dims=(16, 8, 8), seed=2, nsweeps=1, timeout_s=2, fault="late", late_s=8)
    res = _run(2, cfg, wait_s=120)
    assert 0 in res and _failed(res[0]), res
    assert "mini-step 0" in res[0]["msg"]
