"""The row-block split of one grid (the 1:n deployment of Sec. 3.3) on the
host: the partition, the halo exchange, the combination of the partial
reduces and the convergence test of paper_1609_04567_gb300/split.py, driven
over the oracle's block sweep, must give bit for bit the unsplit oracle's
state, iteration count, reduced value and count.  Blocks in one process
(LocalExchanger) and one block per rank over gloo with world sizes 2 and 4
(ProcessGroupExchanger).  CPU only."""
import os
import socket

import numpy as np
import pytest
import torch

from paper_1609_04567_gb300 import inputs
from paper_1609_04567_gb300 import split as S
from paper_1609_04567_gb300 import slr

KIND = {slr.SLR_J2D5: "j2d5", slr.SLR_J3D7: "j3d7", slr.SLR_LIFE: "life", slr.SLR_RESTORE8: "restore8"}


class OracleSweeper:
    """The oracle's block sweep in place of the library's (host arrays)."""

    def __init__(self, orc, stencil, shape, **params):
        self.orc, self.kind, self.params = orc, KIND[stencil], params
        self.nx = shape[-1]
        self.ny = shape[-2] if len(shape) == 3 else shape[0]
        self.nz = shape[0] if len(shape) == 3 else 1

    def slots(self, blocks, sweeps):
        return [[None] * sweeps for _ in range(blocks)]

    def sweep(self, geo, src, dst, aux, slots, b, s):
        r = self.orc.block_sweep(self.kind, src.numpy(), dst.numpy(), None if aux is None else aux.numpy(),
                                 nx=self.nx, ny=self.ny, nz=self.nz, **geo, **self.params)
        slots[b][s] = S.Partial(r["maxbits"], r["sum"], r["count"], r["changed"])

    def read(self, slots, b, kp):
        return slots[b][:kp]


def case(stencil, seed=3):
    """(initial state, aux, oracle params, loop params, oracle solve) of a small seeded problem."""
    if stencil == "j2d5":
        f = inputs.helmholtz_rhs((37, 29), seed=seed)
        return np.zeros_like(f), f, dict(), dict(tol=1e-6, wrap=False), ("j2d5", dict(tol=1e-6))
    if stencil == "j2d5_bf16_wrap":
        f = torch.from_numpy(inputs.helmholtz_rhs((40, 24), seed=seed).astype(np.float32)).to(torch.bfloat16)
        f = f.float().numpy()
        return (np.zeros_like(f), f, dict(storage="bf16", wrap=True, ghost=0.0),
                dict(tol=1e-5, wrap=True), ("j2d5", dict(tol=1e-5, storage="bf16", wrap=True)))
    if stencil == "j2d5_ghost":
        f = inputs.helmholtz_rhs((33, 20), seed=seed)
        return (np.zeros_like(f), f, dict(ghost=0.5, sigma=2.0), dict(tol=1e-7, wrap=False),
                ("j2d5", dict(tol=1e-7, ghost=0.5, sigma=2.0)))
    if stencil == "j3d7":
        f = inputs.helmholtz_rhs((13, 9, 11), seed=seed)
        return np.zeros_like(f), f, dict(), dict(tol=1e-7, wrap=False), ("j3d7", dict(tol=1e-7))
    if stencil == "life_wrap":
        c = inputs.life_cells(34, 40, seed=seed)
        return c, None, dict(wrap=True), dict(tol=0.0, wrap=True), ("life", dict(wrap=True))
    if stencil == "life_dead":
        c = inputs.life_cells(30, 24, seed=seed)
        return c, None, dict(wrap=False), dict(tol=0.0, wrap=False), ("life", dict(wrap=False))
    frame, _ = inputs.noisy_frame(36, 48, seed=seed)
    return (frame.astype(np.float32), inputs.noise_mask(frame), dict(), dict(tol=1e-3, wrap=False),
            ("restore8", dict(tol=1e-3)))


STENCIL = {"j2d5": slr.SLR_J2D5, "j2d5_bf16_wrap": slr.SLR_J2D5, "j2d5_ghost": slr.SLR_J2D5,
           "j3d7": slr.SLR_J3D7, "life_wrap": slr.SLR_LIFE, "life_dead": slr.SLR_LIFE,
           "restore8": slr.SLR_RESTORE8}


def unsplit(orc, name, u0, aux, cap):
    fn, kw = case(name)[4]
    if fn == "life":
        return orc.life(u0, max_gens=cap, **kw)
    if fn == "restore8":
        return orc.restore8(u0, aux, max_iters=cap, **kw)
    return getattr(orc, fn)(u0, aux, max_iters=cap, **kw)


def blocks_of(u0, aux, parts, lo_hi=None):
    out = []
    for lo, hi in (lo_hi or S.row_blocks(u0.shape[0], parts)):
        out.append((torch.from_numpy(np.ascontiguousarray(u0[lo:hi])),
                    None if aux is None else torch.from_numpy(np.ascontiguousarray(aux[lo:hi])), lo, hi))
    return out


def test_row_blocks():
    assert S.row_blocks(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert S.row_blocks(8, 8) == [(i, i + 1) for i in range(8)]
    with pytest.raises(ValueError):
        S.row_blocks(3, 4)


def test_decide_matches_the_device_rule():
    import struct
    bits = struct.unpack("<Q", struct.pack("<d", 2.5e-7))[0]
    assert S.decide(S.ABS_MAX, S.Partial(maxbits=bits), 1e-6) == (2.5e-7, True)
    assert S.decide(S.MEAN_MASKED, S.Partial(sum=3 << 24, count=4), 1.0) == (0.75, True)
    assert S.decide(S.MEAN_MASKED, S.Partial(sum=0, count=0), 1e-3) == (0.0, True)
    assert S.decide(S.LIVE, S.Partial(count=7, changed=1), 0.0) == (7.0, False)


@pytest.mark.parametrize("name", list(STENCIL))
@pytest.mark.parametrize("parts,halo", [(1, 1), (2, 1), (3, 1), (2, 3), (3, 4), (4, 2)])
def test_local_split_matches_unsplit_oracle(orc, name, parts, halo):
    u0, aux, oparams, lparams, _ = case(name)
    cap = 150
    ref, rr = unsplit(orc, name, u0, aux, cap)
    stencil = STENCIL[name]
    loop = S.SplitLoop(stencil, blocks_of(u0, aux, parts), u0.shape[0], halo=halo, exchanger=S.LocalExchanger(),
                       sweeper=OracleSweeper(orc, stencil, u0.shape, **oparams), **lparams)
    r = loop.run(cap)
    got = np.concatenate([loop.own_rows(i).numpy() for i in range(parts)])
    assert np.array_equal(got.view(np.uint8), np.ascontiguousarray(ref).view(np.uint8))
    assert (r.iters, r.converged, r.value, r.count) == (rr.iters, rr.converged, rr.value, rr.count)


def test_local_split_resumes_and_uneven_blocks(orc):
    u0, aux, oparams, lparams, _ = case("restore8")
    ref, rr = unsplit(orc, "restore8", u0, aux, 5000)
    loop = S.SplitLoop(slr.SLR_RESTORE8, blocks_of(u0, aux, 0, [(0, 5), (5, 30), (30, 36)]), 36, halo=5,
                       exchanger=S.LocalExchanger(), sweeper=OracleSweeper(orc, slr.SLR_RESTORE8, u0.shape), **lparams)
    r1 = loop.run(7)
    assert r1.iters == 7
    r = loop.run(5000)
    got = np.concatenate([loop.own_rows(i).numpy() for i in range(3)])
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert (r.iters, r.value, r.count) == (rr.iters, rr.value, rr.count)


def test_blocks_must_own_the_halo(orc):
    u0, aux, oparams, lparams, _ = case("j2d5")
    with pytest.raises(ValueError):
        S.SplitLoop(slr.SLR_J2D5, blocks_of(u0, aux, 0, [(0, 2), (2, 37)]), 37, halo=3, exchanger=S.LocalExchanger(),
                    sweeper=OracleSweeper(orc, slr.SLR_J2D5, u0.shape), **lparams)


# ---- one block per rank over gloo --------------------------------------------------

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, name, halo, out):
    import torch.distributed as dist
    import oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        u0, aux, oparams, lparams, _ = case(name)
        stencil = STENCIL[name]
        lo, hi = S.row_blocks(u0.shape[0], world)[rank]
        loop = S.SplitLoop(stencil, blocks_of(u0, aux, 0, [(lo, hi)]), u0.shape[0], halo=halo,
                           exchanger=S.ProcessGroupExchanger(), sweeper=OracleSweeper(orc, stencil, u0.shape, **oparams),
                           **lparams)
        r = loop.run(150)
        ref, rr = unsplit(orc, name, u0, aux, 150)
        ok = np.array_equal(loop.own_rows().numpy().view(np.uint8), np.ascontiguousarray(ref[lo:hi]).view(np.uint8))
        ok = ok and (r.iters, r.converged, r.value, r.count) == (rr.iters, rr.converged, rr.value, rr.count)
        out.put((rank, bool(ok), (r.iters, r.value, r.count), (rr.iters, rr.value, rr.count)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("name,halo", [("j2d5", 1), ("life_wrap", 3), ("restore8", 2), ("j3d7", 2),
                                       ("j2d5_bf16_wrap", 4)])
def test_gloo_ranks_match_unsplit_oracle(orc, world, name, halo):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, halo, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _, _ in got), got
