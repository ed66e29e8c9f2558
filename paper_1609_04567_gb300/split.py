"""One grid over n devices: the 1:n deployment of Sec. 3.3 (Fig. 2).

The grid is cut into row blocks (3D: slabs of z-planes), one per device.  A
block keeps its own rows and H rows copied in from each neighbour (H = the
sweeps one exchange serves).  One pass of the loop:

  1. halo exchange: every block's first and last H own rows go to the
     neighbours' copied-in rows (on a torus the last block's neighbour is the
     first);
  2. kp <= H sweeps on every block (``slr_block_sweep``): the rows updated
     shrink by one on each side per sweep and end on the block's own rows,
     so after kp sweeps the own rows are exact;
  3. the blocks' per-sweep partial reduces are combined (maximum, integer
     sums, or: the whole grid's reduce, identical in any order);
  4. the convergence test of Sec. 3.1 reads each sweep's value in order; a
     test that passes inside a pass re-runs the pass from its saved input up
     to that sweep, so the state, the value and the iteration count are those
     of the unsplit loop, one sweep at a time.

The exchange and the combination go through an exchanger:
``ProcessGroupExchanger`` (one block per rank over torch.distributed: gloo for
host tensors, NCCL for device tensors) or ``LocalExchanger`` (every block in
this process, e.g. several blocks on one GPU, by copies).  The per-block
sweep goes through a sweeper: ``DeviceSweeper`` calls the library's C ABI;
the tests hand in the oracle's block sweep instead, to check the partition,
exchange and combination logic on the host.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass

from . import slr

ABS_MAX, MEAN_MASKED, LIVE = "max", "mean", "live"
REDUCE_OF = {slr.SLR_J2D5: ABS_MAX, slr.SLR_J3D7: ABS_MAX, slr.SLR_RESTORE8: MEAN_MASKED, slr.SLR_LIFE: LIVE}


def row_blocks(n_rows: int, parts: int) -> list[tuple[int, int]]:
    """[lo, hi) rows of each of `parts` contiguous blocks, sizes differing by
    at most one (the first n_rows % parts blocks get the extra row)."""
    if parts < 1 or n_rows < parts:
        raise ValueError(f"cannot cut {n_rows} rows into {parts} blocks")
    base, extra = divmod(n_rows, parts)
    out, lo = [], 0
    for i in range(parts):
        hi = lo + base + (1 if i < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


@dataclass
class Partial:
    """One sweep's reduce over some rows (a block's own rows, or all)."""
    maxbits: int = 0       # max |delta| as binary64 bits
    sum: int = 0           # sum of |delta| truncated to multiples of 2^-24
    count: int = 0         # live cells / masked pixels
    changed: int = 0       # any item changed

    @staticmethod
    def combine(parts) -> "Partial":
        parts = list(parts)
        return Partial(max(p.maxbits for p in parts), sum(p.sum for p in parts), sum(p.count for p in parts),
                       max(p.changed for p in parts))


def decide(reduce: str, p: Partial, tol: float) -> tuple[float, bool]:
    """The reduced value and the convergence test of Sec. 3.1 for one sweep,
    as the device loop takes it: max |delta| < tol; mean |delta| over the
    masked pixels < tol (0 without masked pixels); Life: no cell changed."""
    if reduce == LIVE:
        return float(p.count), p.changed == 0
    if reduce == MEAN_MASKED:
        value = (float(p.sum) * 2.0 ** -24) / float(p.count) if p.count else 0.0
        return value, value < tol
    value = struct.unpack("<d", struct.pack("<Q", p.maxbits))[0]
    return value, value < tol


# ---- exchangers ----------------------------------------------------------------

def _neighbours(i: int, n: int, wrap: bool):
    up = i - 1 if i > 0 else (n - 1 if wrap else None)
    down = i + 1 if i + 1 < n else (0 if wrap else None)
    return up, down


class LocalExchanger:
    """Every block of the grid in this process, in row order."""

    def swap(self, arrays, halo: int, wrap: bool) -> None:
        """Fill the copied-in rows of each block array (own rows in the
        middle, `halo` rows on each side) from its neighbours' own rows."""
        n = len(arrays)
        for i, a in enumerate(arrays):
            own = a.shape[0] - 2 * halo
            up, down = _neighbours(i, n, wrap)
            if up is not None:
                b = arrays[up]
                a[0:halo].copy_(b[b.shape[0] - 2 * halo:b.shape[0] - halo])
            if down is not None:
                a[own + halo:own + 2 * halo].copy_(arrays[down][halo:2 * halo])

    def combine(self, partials) -> list[Partial]:
        """partials[b][s]: sweep s of local block b; returns per sweep the
        combination over all blocks."""
        return [Partial.combine(col) for col in zip(*partials)]


class ProcessGroupExchanger:
    """One block per rank of a torch.distributed process group, rank order =
    row order.  Halo rows travel by point-to-point send/receive in two
    phases (first and last own rows up and down), each with at most one send
    and one receive per rank, so the pairing is unambiguous even when both
    neighbours are the same rank; partials are combined by two all-reduces."""

    def __init__(self, group=None, device="cpu"):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.device = torch.device(device)      # where the all-reduced partials live (CUDA for NCCL)
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def _peer(self, r):
        return None if r is None else self.dist.get_global_rank(self.group, r) if self.group is not None else r

    def _sendrecv(self, send, to, recv, frm, tag):
        if to is None and frm is None:
            return
        if to == self.rank and frm == self.rank:           # one block on a torus: its own rows
            recv.copy_(send)
            return
        reqs = []
        if to is not None:
            reqs.append(self.dist.isend(send.contiguous(), self._peer(to), group=self.group, tag=tag))
        if frm is not None:
            reqs.append(self.dist.irecv(recv, self._peer(frm), group=self.group, tag=tag))
        for r in reqs:
            r.wait()

    def swap(self, arrays, halo: int, wrap: bool) -> None:
        (a,) = arrays
        own = a.shape[0] - 2 * halo
        up, down = _neighbours(self.rank, self.world, wrap)
        # phase 1: the first own rows go up, the rows below come in
        self._sendrecv(a[halo:2 * halo], up, a[own + halo:own + 2 * halo], down, 1)
        # phase 2: the last own rows go down, the rows above come in
        self._sendrecv(a[own:own + halo], down, a[0:halo], up, 2)

    def combine(self, partials) -> list[Partial]:
        import torch
        (mine,) = partials
        mx = torch.tensor([[p.maxbits, p.changed] for p in mine], dtype=torch.int64, device=self.device)
        sm = torch.tensor([[p.sum, p.count] for p in mine], dtype=torch.int64, device=self.device)
        self.dist.all_reduce(mx, op=self.dist.ReduceOp.MAX, group=self.group)
        self.dist.all_reduce(sm, op=self.dist.ReduceOp.SUM, group=self.group)
        mx, sm = mx.cpu().tolist(), sm.cpu().tolist()
        return [Partial(a, c, d, b) for (a, b), (c, d) in zip(mx, sm)]


# ---- sweepers --------------------------------------------------------------------

class DeviceSweeper:
    """The library's block sweep (slr_block_sweep) on the current CUDA
    stream; the partial of each sweep goes to a device slot, read once per
    pass."""

    def __init__(self, desc: "slr.slr_desc"):
        self.desc = desc

    def slots(self, blocks: int, sweeps: int):
        import torch
        return torch.zeros((blocks, sweeps, 4), dtype=torch.int64, device="cuda")

    def sweep(self, geo: dict, src, dst, aux, slots, b: int, s: int) -> None:
        import torch
        blk = slr.slr_block(geo["rows"], geo["row0"], geo["lo"], geo["hi"], geo["own_lo"], geo["own_hi"])
        slr.slr_block_sweep(self.desc, blk, src.data_ptr(), dst.data_ptr(), 0 if aux is None else aux.data_ptr(),
                            slots[b, s].data_ptr(), torch.cuda.current_stream().cuda_stream)

    def read(self, slots, b: int, kp: int) -> list[Partial]:
        rows = slots[b, :kp].cpu().tolist()              # waits for the stream
        return [Partial(r[0] & (2 ** 64 - 1), r[1] & (2 ** 64 - 1), r[2] & (2 ** 64 - 1), r[3] & 0xFFFFFFFF)
                for r in rows]


# ---- the loop ----------------------------------------------------------------------

@dataclass
class SplitResult:
    iters: int
    value: float
    converged: bool
    count: int
    changed: bool
    passes: int


class SplitLoop:
    """The loop-of-stencil-reduce over row blocks of one grid.

    blocks: list of (u_rows, aux_rows or None, g_lo, g_hi) for the blocks held
    here (one per rank with ProcessGroupExchanger, all of them in row order
    with LocalExchanger); u_rows are the block's own rows (a tensor whose
    first dimension is rows, 3D: planes).  The loop keeps two state arrays per
    block with `halo` copied-in rows on each side; every block must own at
    least `halo` rows.  grid_rows: the grid's rows (3D: planes)."""

    def __init__(self, stencil: int, blocks, grid_rows: int, *, halo: int, exchanger, sweeper, tol: float,
                 wrap: bool):
        import torch
        if halo < 1:
            raise ValueError("halo must be >= 1")
        self.reduce = REDUCE_OF[stencil]
        self.halo, self.ex, self.sw, self.tol, self.wrap = halo, exchanger, sweeper, tol, wrap
        self.grid_rows = grid_rows
        self.blocks = []
        for u_rows, aux_rows, g_lo, g_hi in blocks:
            own = g_hi - g_lo
            if own < halo or u_rows.shape[0] != own:
                raise ValueError(f"block [{g_lo}, {g_hi}) must own at least {halo} rows")
            shape = (own + 2 * halo,) + tuple(u_rows.shape[1:])
            bufs = [torch.zeros(shape, dtype=u_rows.dtype, device=u_rows.device) for _ in range(2)]
            bufs[0][halo:halo + own].copy_(u_rows)
            aux = None
            if aux_rows is not None:
                aux = torch.zeros(shape, dtype=aux_rows.dtype, device=aux_rows.device)
                aux[halo:halo + own].copy_(aux_rows)
            self.blocks.append({"g_lo": g_lo, "g_hi": g_hi, "own": own, "buf": bufs, "aux": aux,
                                "save": torch.empty_like(bufs[0]) if halo > 1 else None})
        # f or the mask never changes: its copied-in rows are exchanged once
        if self.blocks[0]["aux"] is not None:
            self.ex.swap([b["aux"] for b in self.blocks], halo, wrap)
        self.slots = self.sw.slots(len(self.blocks), halo)
        self.cur = 0
        self.iters, self.value, self.converged, self.count, self.changed, self.passes = 0, 0.0, False, 0, False, 0

    def _geo(self, b, s: int, kp: int) -> dict:
        H = self.halo
        return {"rows": b["own"] + 2 * H, "row0": b["g_lo"] - H, "lo": H - (kp - s),
                "hi": H + b["own"] + (kp - s), "own_lo": H, "own_hi": H + b["own"]}

    def _pass(self, t: int, kp: int) -> None:
        for s in range(1, kp + 1):
            for i, b in enumerate(self.blocks):
                src, dst = b["buf"][t ^ ((s - 1) & 1)], b["buf"][t ^ (s & 1)]
                self.sw.sweep(self._geo(b, s, kp), src, dst, b["aux"], self.slots, i, s - 1)

    def run(self, max_iters: int) -> SplitResult:
        """Iterate until the test passes or the total iteration count reaches
        max_iters (a later call with a higher cap resumes)."""
        while not self.converged and self.iters < max_iters:
            kp = min(self.halo, max_iters - self.iters)
            t = self.cur
            self.ex.swap([b["buf"][t] for b in self.blocks], self.halo, self.wrap)
            if kp > 1:
                for b in self.blocks:
                    b["save"].copy_(b["buf"][t])
            self._pass(t, kp)
            parts = self.ex.combine([self.sw.read(self.slots, i, kp) for i in range(len(self.blocks))])
            stop = None
            for j, p in enumerate(parts):
                value, conv = decide(self.reduce, p, self.tol)
                if conv:
                    stop = j
                    break
            last = stop if stop is not None else kp - 1
            self.value, _ = decide(self.reduce, parts[last], self.tol)
            self.count, self.changed = parts[last].count, bool(parts[last].changed)
            self.iters += last + 1
            self.passes += 1
            if stop is not None and stop + 1 < kp:
                # the pass again from its input, up to the stopping sweep
                for b in self.blocks:
                    b["buf"][t].copy_(b["save"])
                self._pass(t, stop + 1)
            self.cur = t ^ ((last + 1) & 1)
            self.converged = stop is not None
        return self.result()

    def result(self) -> SplitResult:
        return SplitResult(self.iters, self.value, self.converged, self.count, self.changed, self.passes)

    def own_rows(self, i: int = 0):
        """The own rows of local block i (a view of its current state array)."""
        b = self.blocks[i]
        return b["buf"][self.cur][self.halo:self.halo + b["own"]]
