"""The row-block split of one grid (the 1:n deployment of Sec. 3.3) with the
library's block sweep on the GPU: several blocks of one grid on one device,
exchanging their halo rows by copies (the same partition, exchange,
combination and test code that runs one block per rank over
torch.distributed), must equal the unsplit oracle bit for bit (state,
iteration count, reduced value, count)."""
import numpy as np
import pytest
import torch

from paper_1609_04567_gb300 import split as S

pytestmark = pytest.mark.gpu

from test_split_host import STENCIL, blocks_of, case, unsplit  # noqa: E402

TORCH_OF = {np.dtype(np.float64): torch.float64, np.dtype(np.float32): torch.float32, np.dtype(np.uint8): torch.uint8}


def device_blocks(u0, aux, parts, storage):
    out = []
    for u, a, lo, hi in blocks_of(u0, aux, parts):
        u = u.cuda() if storage is None else u.cuda().to(storage)
        if a is not None:
            a = a.cuda() if (storage is None or a.dtype == torch.uint8) else a.cuda().to(storage)
        out.append((u, a, lo, hi))
    return out


@pytest.mark.parametrize("name", list(STENCIL))
@pytest.mark.parametrize("parts,halo", [(1, 1), (2, 1), (3, 2), (2, 4), (4, 3)])
def test_blocks_on_one_device_match_unsplit_oracle(gpu, orc, name, parts, halo):
    u0, aux, oparams, lparams, _ = case(name)
    cap = 150
    ref, rr = unsplit(orc, name, u0, aux, cap)
    stencil = STENCIL[name]
    storage = torch.bfloat16 if oparams.get("storage") == "bf16" else None
    shape = u0.shape
    nz, ny, nx = (1,) * (3 - len(shape)) + tuple(shape)
    fields = {}
    if storage is not None:
        fields["storage"] = gpu.SLR_BF16
    if "ghost" in oparams:
        fields["ghost"] = oparams["ghost"]
    if "sigma" in oparams:
        fields["sigma"] = oparams["sigma"]
    if stencil == gpu.SLR_LIFE:
        fields["boundary"] = gpu.SLR_WRAP if oparams["wrap"] else gpu.SLR_DIRICHLET
    elif oparams.get("wrap"):
        fields["boundary"] = gpu.SLR_WRAP
    desc = gpu.slr_desc_init(stencil, nx, ny, nz, **fields)
    loop = S.SplitLoop(stencil, device_blocks(u0, aux, parts, storage), shape[0], halo=halo,
                       exchanger=S.LocalExchanger(), sweeper=S.DeviceSweeper(desc), **lparams)
    r = loop.run(cap)
    got = torch.cat([loop.own_rows(i) for i in range(parts)]).cpu()
    got = got.float().numpy() if storage is not None else got.numpy()
    assert np.array_equal(got.view(np.uint8), np.ascontiguousarray(ref).view(np.uint8))
    assert (r.iters, r.converged, r.value, r.count) == (rr.iters, rr.converged, rr.value, rr.count)


def test_block_sweep_refuses_inconsistent_ranges(gpu):
    d = gpu.slr_desc_init(gpu.SLR_J2D5, 16, 32, 1)
    a = torch.zeros((10, 16), dtype=torch.float64, device="cuda")
    b, f = torch.zeros_like(a), torch.zeros_like(a)
    p = torch.zeros(4, dtype=torch.int64, device="cuda")
    # row 0 of the block is global row 5: its row above (global 4) is not in the block
    bad = gpu.slr_block(10, 5, 0, 10, 0, 10)
    assert gpu.slr_block_sweep(d, bad, a.data_ptr(), b.data_ptr(), f.data_ptr(), p.data_ptr(), 0,
                               check=False) == gpu.SLR_ERR_INVALID_ARG
    assert "outside the block" in gpu.slr_last_error(None)
    for blk in (gpu.slr_block(10, 0, 3, 2, 3, 2), gpu.slr_block(10, 0, 0, 11, 0, 10), gpu.slr_block(10, 0, 1, 9, 0, 9)):
        assert gpu.slr_block_sweep(d, blk, a.data_ptr(), b.data_ptr(), f.data_ptr(), p.data_ptr(), 0,
                                   check=False) == gpu.SLR_ERR_INVALID_ARG
    # a block holding the whole grid: its first and last rows have the boundary beyond them
    whole = gpu.slr_desc_init(gpu.SLR_J2D5, 16, 10, 1)
    ok = gpu.slr_block(10, 0, 0, 10, 0, 10)
    assert gpu.slr_block_sweep(whole, ok, a.data_ptr(), b.data_ptr(), f.data_ptr(), p.data_ptr(), 0) == gpu.SLR_OK
    torch.cuda.synchronize()
