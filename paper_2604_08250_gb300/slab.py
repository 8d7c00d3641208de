"""1D slab decomposition along x with a per-mini-step ghost exchange (Sec. III-B).

The box of nx x ny x nz BCC cells is cut into `world` slabs of equal width w
(a multiple of the link-cell edge 4) along x; rank r owns cells
[r w, (r + 1) w).  Each rank keeps its slab plus g ghost cells on each side
(x modulo nx) as an int8 array [2][nz][ny][w + 2g], the layout of the box with
x restricted to the window.  g is the number of cells a trial reads past its
own along x (2 for pair models, 3 with the MLP site energies).

After each mini-step every rank tells its two x-neighbours which cells it
may have changed.  With trial sites at x = 4 cx + dx on sublattice `sub`,
a trial swaps its site with a first-shell partner one cell to the left
(sub = 0) or to the right (sub = 1) at most, so the cells a slab may change
in that mini-step are [x0 + d - 1, x0 + w + d - 3) with d = dx + sub.  These
ranges of different slabs are disjoint (the link-cell independence of
Sec. II-A), and each lies within one cell of its slab, so a rank is the only
writer of the cells it sends: the receiver overwrites every copy of them in
its window.  Per side and mini-step that is 0 to g + 1 cells of 2 ny nz bytes,
the message of the paper's size formula with k = 0..g + 1 layers.

Messages are framed: a 64-byte header (magic, sender, sweep, mini-step,
direction, first cell, cell count, Adler-32 of the payload) and a payload
padded to the plan's largest message, sent with torch.distributed
point-to-point calls.  A receive that times out, a peer that went away, or a
frame whose header disagrees with what the plan expects raises
SlabExchangeError naming the ranks, the sweep and the mini-step.

The trials of a mini-step on one slab are a callable supplied by the caller;
this module computes no energies and takes no acceptance decisions.
"""
from __future__ import annotations

import datetime
import zlib

import numpy as np

LC_EDGE = 4
HEADER = 64
MAGIC = 0x534C4142  # "SLAB"
LEFTWARD, RIGHTWARD = 0, 1


class SlabExchangeError(RuntimeError):
    """A ghost exchange failed: timeout, lost peer or malformed frame."""


def lc_edge(n: int) -> int:
    """Link-cell edge along an axis of n cells: 4, or the whole axis when it
    is shorter than 8 cells or not a multiple of 4 (Sec. II-A)."""
    return 4 if (n >= 8 and n % 4 == 0) else n


class SlabPlan:
    """Partition of an nx x ny x nz box into `world` x-slabs with `ghost`
    cells per side, and the cell ranges each mini-step exchanges."""

    def __init__(self, nx: int, ny: int, nz: int, world: int, ghost: int):
        self.nx, self.ny, self.nz, self.world, self.ghost = int(nx), int(ny), int(nz), int(world), int(ghost)
        if self.world < 1:
            raise ValueError("world must be >= 1")
        if self.nx < 8 or self.nx % LC_EDGE != 0:
            raise ValueError("slabs need nx >= 8 and a multiple of 4")
        if self.nx % (LC_EDGE * self.world) != 0:
            raise ValueError(f"nx = {nx} does not split into {world} slabs of a multiple of 4 cells")
        self.w = self.nx // self.world
        if not 1 <= self.ghost < self.w:
            raise ValueError(f"ghost cells must lie in [1, {self.w - 1}] for slabs of {self.w} cells")
        self.Ly, self.Lz = lc_edge(self.ny), lc_edge(self.nz)
        self.nA = 2 * LC_EDGE * self.Ly * self.Lz
        self.cell_bytes = 2 * self.ny * self.nz
        self.max_cells = max(self._width(self.outgoing(0, k, s)) for k in range(self.nA) for s in (-1, 1))
        self.frame_bytes = HEADER + max(self.max_cells, 1) * self.cell_bytes

    # geometry -----------------------------------------------------------
    def x0(self, rank: int) -> int:
        return rank * self.w

    @property
    def window(self) -> int:
        return self.w + 2 * self.ghost

    def local_shape(self):
        return (2, self.nz, self.ny, self.window)

    def neighbour(self, rank: int, side: int) -> int:
        return (rank + side) % self.world

    def d(self, k: int) -> int:
        """dx + sub of mini-step k = ((sub Lz + dz) Ly + dy) 4 + dx."""
        return k % LC_EDGE + k // (LC_EDGE * self.Ly * self.Lz)

    def modified(self, rank: int, k: int):
        """Half-open x range (unwrapped, may leave [0, nx)) of the cells rank
        `rank` may change in mini-step k."""
        x0, d = self.x0(rank), self.d(k)
        return x0 + d - 1, x0 + self.w + d - 3

    def outgoing(self, rank: int, k: int, side: int):
        """Cells rank sends to its neighbour on `side` (-1 left, +1 right)
        after mini-step k: its changed cells inside that neighbour's window."""
        lo, hi = self.modified(rank, k)
        x0, g = self.x0(rank), self.ghost
        if side < 0:
            hi = min(hi, x0 + g)
        else:
            lo = max(lo, x0 + self.w - g)
        return (lo, max(lo, hi))

    @staticmethod
    def _width(r):
        return r[1] - r[0]

    def local_index(self, rank: int, x_unwrapped: int) -> int:
        return x_unwrapped - self.x0(rank) + self.ghost

    def copies(self, rank: int, gx: int):
        """Window positions of rank `rank` holding global cell gx (mod nx)."""
        base = self.x0(rank) - self.ghost
        return [j for j in range(self.window) if (base + j) % self.nx == gx % self.nx]

    # data movement ------------------------------------------------------
    def window_of(self, occ_global: np.ndarray, rank: int) -> np.ndarray:
        """Rank's window cut from the whole box (occ as [2][nz][ny][nx] or flat)."""
        box = np.asarray(occ_global).reshape(2, self.nz, self.ny, self.nx)
        xs = (np.arange(self.window) + self.x0(rank) - self.ghost) % self.nx
        return np.ascontiguousarray(box[..., xs])

    def owned(self, local: np.ndarray) -> np.ndarray:
        g = self.ghost
        return local.reshape(self.local_shape())[..., g:g + self.w]

    def pack(self, local: np.ndarray, rank: int, cells) -> bytes:
        lo, hi = cells
        a, b = self.local_index(rank, lo), self.local_index(rank, hi)
        return np.ascontiguousarray(local.reshape(self.local_shape())[..., a:b]).tobytes()

    def unpack(self, local: np.ndarray, rank: int, first_cell: int, payload: bytes, ncells: int):
        v = local.reshape(self.local_shape())
        blk = np.frombuffer(payload, dtype=np.int8, count=ncells * self.cell_bytes)
        blk = blk.reshape(2, self.nz, self.ny, ncells)
        for j in range(ncells):
            for p in self.copies(rank, first_cell + j):
                v[..., p] = blk[..., j]

    # frames -------------------------------------------------------------
    def encode(self, sender: int, sweep: int, k: int, tag: int, cells, payload: bytes) -> np.ndarray:
        ncells = self._width(cells)
        frame = np.zeros(self.frame_bytes, dtype=np.uint8)
        hdr = np.array([MAGIC, sender, sweep, k, tag, cells[0] % self.nx, ncells, zlib.adler32(payload)],
                       dtype=np.int64)
        frame[:HEADER] = hdr.view(np.uint8)
        frame[HEADER:HEADER + len(payload)] = np.frombuffer(payload, dtype=np.uint8)
        return frame

    def decode(self, frame: np.ndarray, sender: int, sweep: int, k: int, tag: int, cells):
        """Payload of a frame after checking every header field against the
        plan; SlabExchangeError otherwise."""
        hdr = frame[:HEADER].view(np.int64)
        want_n = self._width(cells)
        where = f"frame from rank {sender}, sweep {sweep}, mini-step {k}"
        if int(hdr[0]) != MAGIC:
            raise SlabExchangeError(f"{where}: bad magic {int(hdr[0]):#x}")
        got = tuple(int(x) for x in hdr[1:5])
        if got != (sender, sweep, k, tag):
            raise SlabExchangeError(f"{where}: header names (rank, sweep, mini-step, direction) = {got}")
        if int(hdr[5]) != cells[0] % self.nx or int(hdr[6]) != want_n:
            raise SlabExchangeError(f"{where}: truncated or misplaced payload: cells {int(hdr[5])}+{int(hdr[6])}, "
                                    f"expected {cells[0] % self.nx}+{want_n}")
        payload = frame[HEADER:HEADER + want_n * self.cell_bytes].tobytes()
        if zlib.adler32(payload) != int(hdr[7]):
            raise SlabExchangeError(f"{where}: payload checksum mismatch")
        return payload


class SlabExchange:
    """Ghost exchange of one rank over a torch.distributed process group
    (gloo for CPU ranks).  With world = 1 the slab is its own neighbour and
    the frames are handed over in memory, through the same encode/decode."""

    def __init__(self, plan: SlabPlan, rank: int, dist=None, timeout_s: float = 30.0):
        self.plan, self.rank, self.dist = plan, int(rank), dist
        self.timeout = datetime.timedelta(seconds=float(timeout_s))
        if plan.world > 1 and dist is None:
            raise ValueError("world > 1 needs a torch.distributed module with an initialised group")
        self.bytes_sent = 0
        self.frames_sent = 0

    def _emit(self, frame: np.ndarray, dst: int, tag: int):
        """Starts sending one frame; returns the pending request (None in memory)."""
        import torch
        return self.dist.isend(torch.from_numpy(frame), dst=dst, tag=tag)

    def step(self, local: np.ndarray, sweep: int, k: int):
        """Exchange after mini-step k of sweep `sweep`: send this rank's
        changed boundary cells to both x-neighbours, receive theirs and
        write them into every copy in the local window."""
        P, r = self.plan, self.rank
        out = {}
        for side, tag in ((-1, LEFTWARD), (1, RIGHTWARD)):
            cells = P.outgoing(r, k, side)
            out[tag] = (P.neighbour(r, side), cells, P.encode(r, sweep, k, tag, cells, P.pack(local, r, cells)))
        incoming = [(P.neighbour(r, 1), LEFTWARD), (P.neighbour(r, -1), RIGHTWARD)]
        if P.world == 1:
            frames = {tag: out[tag][2] for _, tag in incoming}
        else:
            import torch
            bufs, reqs = {}, []
            for src, tag in incoming:
                bufs[tag] = torch.empty(P.frame_bytes, dtype=torch.uint8)
                reqs.append((src, tag, self.dist.irecv(bufs[tag], src=src, tag=tag)))
            sends = []
            for tag, (dst, _, frame) in out.items():
                req = self._emit(frame, dst, tag)
                if req is not None:
                    sends.append((dst, req))
                self.bytes_sent += P.frame_bytes
                self.frames_sent += 1
            for src, tag, req in reqs:
                self._wait(req, f"receive from rank {src}", sweep, k)
            for dst, req in sends:
                self._wait(req, f"send to rank {dst}", sweep, k)
            frames = {tag: bufs[tag].numpy() for tag in bufs}
        for src, tag in incoming:
            side = 1 if tag == RIGHTWARD else -1
            cells = P.outgoing(src, k, side)
            payload = P.decode(frames[tag], src, sweep, k, tag, cells)
            P.unpack(local, r, cells[0], payload, P._width(cells))

    def _wait(self, req, what, sweep, k):
        try:
            ok = req.wait(self.timeout)
        except Exception as e:  # gloo reports timeouts and closed peers as RuntimeError
            raise SlabExchangeError(f"rank {self.rank}: {what} failed at sweep {sweep}, mini-step {k}: {e}") from e
        if ok is False:
            raise SlabExchangeError(f"rank {self.rank}: {what} timed out at sweep {sweep}, mini-step {k}")


# ---- device windows (torch tensors) ------------------------------------------
# The same exchange for windows held as torch tensors [2][nz][ny][w + 2g]:
# CUDA tensors with the nccl backend (each GPU's own window, payloads sent
# device to device), CPU tensors with gloo.  A frame is a header tensor of 8
# int64 (magic, sender, sweep, mini-step, direction, first cell, cell count,
# 0) and a payload tensor [2][nz][ny][max_cells] (every frame of a plan the
# same size, so that a frame of another mini-step is received whole and
# rejected by its header); the header is checked on the host after the
# receive.  With the trials split into edge and interior link
# cells (smc_slab_ministep part 1 and 2), `start` after the edge trials and
# `finish` after the interior ones overlap the transfer with the interior
# trials (Sec. V-C).

def _cells_index(plan: SlabPlan, rank: int, first: int, ncells: int):
    """(window positions, payload columns) of every copy of the cells
    first .. first + ncells - 1 in rank's window."""
    pos, col = [], []
    for j in range(ncells):
        for p in plan.copies(rank, first + j):
            pos.append(p)
            col.append(j)
    return pos, col


class TorchSlabExchange:
    """Ghost exchange of one rank's torch window over a process group."""

    def __init__(self, plan: SlabPlan, rank: int, dist, timeout_s: float = 30.0):
        if plan.world < 2:
            raise ValueError("TorchSlabExchange needs world >= 2 (LocalSlabExchange runs slabs in one process)")
        self.plan, self.rank, self.dist = plan, int(rank), dist
        self.timeout = datetime.timedelta(seconds=float(timeout_s))
        self.bytes_sent = 0

    def _header(self, sweep, k, tag, cells, device):
        import torch
        P = self.plan
        return torch.tensor([MAGIC, self.rank, sweep, k, tag, cells[0] % P.nx, P._width(cells), 0],
                            dtype=torch.int64, device=device)

    def start(self, win, sweep: int, k: int):
        """Posts, as one batch of point-to-point operations (NCCL runs them
        as one group), the receives of the neighbours' frames and the sends
        of this rank's changed edge cells after mini-step k."""
        import torch
        P, r = self.plan, self.rank
        pend = {"sweep": sweep, "k": k, "recv": [], "send": []}
        ops = []
        for src, tag in ((P.neighbour(r, 1), LEFTWARD), (P.neighbour(r, -1), RIGHTWARD)):
            side = 1 if tag == RIGHTWARD else -1
            cells = P.outgoing(src, k, side)
            hdr = torch.empty(8, dtype=torch.int64, device=win.device)
            pay = torch.empty((2, P.nz, P.ny, max(P.max_cells, 1)), dtype=torch.int8, device=win.device)
            ops += [self.dist.P2POp(self.dist.irecv, hdr, src, tag=2 * tag),
                    self.dist.P2POp(self.dist.irecv, pay, src, tag=2 * tag + 1)]
            pend["recv"].append((src, tag, cells, hdr, pay))
        for side, tag in ((-1, LEFTWARD), (1, RIGHTWARD)):
            dst, cells = P.neighbour(r, side), P.outgoing(r, k, side)
            a, b = P.local_index(r, cells[0]), P.local_index(r, cells[1])
            pay = torch.zeros((2, P.nz, P.ny, max(P.max_cells, 1)), dtype=torch.int8, device=win.device)
            pay[..., :b - a] = win.reshape(P.local_shape())[..., a:b]
            hdr = self._header(sweep, k, tag, cells, win.device)
            ops += [self.dist.P2POp(self.dist.isend, hdr, dst, tag=2 * tag),
                    self.dist.P2POp(self.dist.isend, pay, dst, tag=2 * tag + 1)]
            pend["send"].append((dst, hdr, pay))
            self.bytes_sent += pay.numel() + 64
        pend["reqs"] = self.dist.batch_isend_irecv(ops)
        return pend

    def _wait(self, req, what, sweep, k):
        try:
            ok = req.wait(self.timeout)
        except Exception as e:  # gloo and nccl report timeouts and closed peers as RuntimeError
            raise SlabExchangeError(f"rank {self.rank}: {what} failed at sweep {sweep}, mini-step {k}: {e}") from e
        if ok is False:
            raise SlabExchangeError(f"rank {self.rank}: {what} timed out at sweep {sweep}, mini-step {k}")

    def finish(self, win, pend):
        """Waits for the pending exchange, checks the headers and writes the
        received cells into every copy in the window."""
        import torch
        P, sweep, k = self.plan, pend["sweep"], pend["k"]
        for req in pend["reqs"]:
            self._wait(req, "exchange with the neighbours", sweep, k)
        v = win.reshape(P.local_shape())
        for src, tag, cells, hdr, pay in pend["recv"]:
            h = [int(x) for x in hdr.cpu().tolist()]
            want = [MAGIC, src, sweep, k, tag, cells[0] % P.nx, P._width(cells)]
            if h[:7] != want:
                raise SlabExchangeError(f"rank {self.rank}: frame from rank {src}, sweep {sweep}, mini-step {k}: "
                                        f"header {h[:7]}, expected {want}")
            pos, col = _cells_index(P, self.rank, cells[0], P._width(cells))
            if pos:
                v[..., torch.tensor(pos, device=win.device)] = pay[..., torch.tensor(col, device=win.device)]

    def step(self, win, sweep: int, k: int):
        self.finish(win, self.start(win, sweep, k))


class LocalSlabExchange:
    """All slabs of a plan in one process (their windows as one list of
    tensors, e.g. on one GPU): the exchange after a mini-step copies every
    slab's changed edge cells into its neighbours' windows, device to device.
    All payloads are taken before any is written."""

    def __init__(self, plan: SlabPlan):
        self.plan = plan

    def step(self, wins, sweep: int, k: int):
        import torch
        P = self.plan
        moves = []
        for r in range(P.world):
            v = wins[r].reshape(P.local_shape())
            for side in (-1, 1):
                cells = P.outgoing(r, k, side)
                a, b = P.local_index(r, cells[0]), P.local_index(r, cells[1])
                if b > a:
                    moves.append((P.neighbour(r, side), cells, v[..., a:b].clone()))
        for dst, cells, pay in moves:
            pos, col = _cells_index(P, dst, cells[0], P._width(cells))
            if pos:
                d = wins[dst].reshape(P.local_shape())
                d[..., torch.tensor(pos, device=d.device)] = pay[..., torch.tensor(col, device=d.device)]


def run_sweeps(exchange: SlabExchange, local: np.ndarray, ministep, sweep0: int, nsweeps: int):
    """nsweeps sweeps of the slab schedule: for every mini-step, the callable
    ministep(local, sweep, k) -> (sum dE, accepted) runs this rank's trials,
    then the ghost exchange.  Returns this rank's (sum dE, accepted)."""
    e, n = 0.0, 0
    for t in range(nsweeps):
        s = sweep0 + t
        for k in range(exchange.plan.nA):
            de, dn = ministep(local, s, k)
            e += de
            n += dn
            exchange.step(local, s, k)
    return e, n


def gather(plan: SlabPlan, local: np.ndarray, rank: int, dist=None):
    """The whole box [2][nz][ny][nx] assembled from every rank's owned cells
    (all ranks receive it)."""
    own = np.ascontiguousarray(plan.owned(local))
    if plan.world == 1:
        return own.copy()
    import torch
    parts = [torch.empty(own.shape, dtype=torch.int8) for _ in range(plan.world)]
    dist.all_gather(parts, torch.from_numpy(own))
    return np.concatenate([p.numpy() for p in parts], axis=-1)
