"""Batched persistent launch: many uneven instances (2D and 3D Helmholtz
Jacobi in several storage precisions, restoration frames) in one launch, each
with its own test and cap.  Every instance must match the oracle exactly as it
does when run alone, and instances added while others are running (the
continuous-batching use) must give the same results."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def jacobi_instance(shape, storage, seed, **kw):
    from paper_1609_04567_gb300 import inputs
    f64 = inputs.helmholtz_rhs(shape, seed=seed)
    if storage == "f64":
        ft, fo = torch.from_numpy(f64), f64
    else:
        ft = torch.from_numpy(f64.astype(np.float32)).to(TORCH[storage])
        fo = ft.float().numpy()
    u = torch.zeros(shape, dtype=TORCH[storage], device="cuda")
    return dict(kind="j", shape=shape, storage=storage, u=u, aux=ft.cuda(), f_oracle=fo, kw=kw)


def restore_instance(ny, nx, seed, **kw):
    from paper_1609_04567_gb300 import inputs
    frame, _ = inputs.noisy_frame(ny, nx, seed=seed)
    mask = inputs.noise_mask(frame)
    u = torch.from_numpy(frame.astype(np.float32)).cuda()
    return dict(kind="r", u=u, aux=torch.from_numpy(mask).cuda(), frame=frame, mask=mask, kw=kw)


def oracle_of(orc, inst, cap):
    kw = dict(inst["kw"])
    if kw.pop("defect_correction", 0):
        fn = orc.j3d7_dc if len(inst["shape"]) == 3 else orc.j2d5_dc
        k_in = kw.pop("inner_sweeps", 50)
        return fn(np.zeros(inst["shape"]), inst["f_oracle"], k_in=k_in, max_outer=cap, **kw)
    if inst["kind"] == "r":
        out, r = orc.restore8(inst["frame"].astype(np.float32), inst["mask"], tol=kw.get("tol", 1e-3), max_iters=cap)
        return out, r
    shape = inst["shape"]
    fn = orc.j3d7 if len(shape) == 3 else orc.j2d5
    wrap = kw.pop("boundary", 0) == 1
    out, r = fn(np.zeros(shape, dtype=inst["f_oracle"].dtype), inst["f_oracle"], wrap=wrap,
                storage=None if inst["storage"] == "f64" else inst["storage"], max_iters=cap, **kw)
    return out, r


def state(inst):
    u = inst["u"]
    return u.float().cpu().numpy() if u.dtype in (torch.bfloat16, torch.float16) else u.cpu().numpy()


def add(slr, batch, inst, cap):
    stencil = slr.SLR_RESTORE8 if inst["kind"] == "r" else (slr.SLR_J3D7 if len(inst["shape"]) == 3 else slr.SLR_J2D5)
    return batch.add(stencil, inst["u"], inst["aux"], cap, **inst["kw"])


def make_mix():
    insts = [
        (jacobi_instance((64, 64), "f64", 1, tol=1e-6), 5000),
        (jacobi_instance((33, 17), "f64", 2, tol=1e-9), 5000),
        (jacobi_instance((100, 130), "f64", 3, tol=1e-6, boundary=1), 5000),
        (jacobi_instance((48, 80), "f64", 4, tol=1e-8, ghost=0.5), 5000),
        (jacobi_instance((96, 80), "bf16", 5, tol=1e-6), 3000),
        (jacobi_instance((70, 70), "f16", 6, tol=1e-6), 3000),
        (jacobi_instance((40, 56), "f32", 7, tol=1e-7), 3000),
        (jacobi_instance((12, 20, 24), "f64", 8, tol=1e-6), 2000),
        (jacobi_instance((9, 10, 11), "bf16", 9, tol=1e-6), 2000),
        (jacobi_instance((256, 256), "f64", 10, tol=1e-6), 17),      # stopped by its cap
        (restore_instance(128, 200, 11), 5000),
        (restore_instance(37, 1, 12), 5000),
    ]
    return insts


def test_mixed_batch_matches_oracle_and_solo_runs(gpu, orc):
    b = gpu.Batch(64)
    mix = make_mix()
    slots = [add(gpu, b, inst, cap) for inst, cap in mix]
    b.run(100000)
    finished, running = b.poll()
    assert running == 0 and sorted(finished) == sorted(slots)
    for (inst, cap), s in zip(mix, slots):
        r = b.result(s)
        ref, rr = oracle_of(orc, inst, cap)
        got = state(inst)
        assert (r.iters, r.converged) == (rr.iters, rr.converged), (inst["kw"], r, rr)
        assert np.array_equal(got, ref.astype(got.dtype)), inst["kw"]
        assert r.value == rr.value
    b.close()


def test_instances_added_while_others_run(gpu, orc):
    # continuous batching: a run stops on its sweep budget with work still in
    # flight, new instances join, finished ones leave; every result is still
    # the one of the instance alone
    b = gpu.Batch(16)
    first = [(jacobi_instance((64, 64), "f64", 21, tol=1e-7), 5000),
             (restore_instance(64, 96, 22), 5000)]
    later = [(jacobi_instance((50, 40), "bf16", 23, tol=1e-6), 3000),
             (jacobi_instance((30, 30), "f64", 24, tol=1e-9), 5000)]
    slots = {add(gpu, b, inst, cap): (inst, cap) for inst, cap in first}
    b.run(7)
    done, running = b.poll()
    assert running >= 1
    for inst, cap in later:
        slots[add(gpu, b, inst, cap)] = (inst, cap)
    seen = set(done)
    for _ in range(2000):
        b.run(50)
        done, running = b.poll()
        seen.update(done)
        if running == 0:
            break
    assert seen == set(slots)
    for s, (inst, cap) in slots.items():
        r = b.result(s)
        ref, rr = oracle_of(orc, inst, cap)
        got = state(inst)
        assert (r.iters, r.converged) == (rr.iters, rr.converged)
        assert np.array_equal(got, ref.astype(got.dtype))
    # a freed slot is reused by a new instance
    s0 = next(iter(slots))
    b.remove(s0)
    inst, cap = jacobi_instance((20, 20), "f64", 25, tol=1e-9), 5000
    s_new = add(gpu, b, inst, cap)
    assert s_new == s0
    b.run(10000)
    done, running = b.poll()
    assert s_new in done and running == 0
    ref, rr = oracle_of(orc, inst, cap)
    assert np.array_equal(state(inst), ref) and b.result(s_new).iters == rr.iters
    b.close()


def test_batch_rejects_life_and_full_batches(gpu):
    b = gpu.Batch(1)
    u = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu.SlrError):
        b.add(gpu.SLR_LIFE, u, u, 10)
    inst = jacobi_instance((8, 8), "f64", 1)
    add(gpu, b, inst, 10)
    inst2 = jacobi_instance((8, 8), "f64", 2)
    with pytest.raises(gpu.SlrError) as e:
        add(gpu, b, inst2, 10)
    assert e.value.status == gpu.SLR_ERR_WORKSPACE
    b.close()


def dc_instances():
    return [
        (jacobi_instance((40, 36), "f64", 41, tol=1e-10, defect_correction=1, inner_sweeps=12), 5000),
        (jacobi_instance((7, 9, 11), "f64", 42, tol=1e-10, defect_correction=1, inner_sweeps=8), 5000),
        (jacobi_instance((96, 64), "f64", 43, tol=1e-10, defect_correction=1, inner_sweeps=25), 3),   # capped
        (jacobi_instance((1, 1), "f64", 44, tol=1e-12, defect_correction=1, inner_sweeps=3), 100),
        # on clusters of several CTAs (2048 cells a CTA at most): 3D z-slabs of
        # 3 planes, 3D with one plane a CTA (every plane below and above is
        # another CTA's), 2D row blocks
        (jacobi_instance((12, 20, 24), "f64", 47, tol=1e-10, defect_correction=1, inner_sweeps=10), 5000),
        (jacobi_instance((2, 30, 40), "f64", 48, tol=1e-10, defect_correction=1, inner_sweeps=6), 5000),
        (jacobi_instance((60, 50), "f64", 49, tol=1e-10, defect_correction=1, inner_sweeps=20), 5000),
    ]


def test_defect_correction_instances_in_a_mixed_batch(gpu, orc):
    # FP64 defect correction around binary32 inner sweeps, 2D and 3D, next to
    # plain Jacobi and restoration instances: each equals the oracle's defect
    # correction bit for bit (state, corrections, scaled defect) and its solo run
    b = gpu.Batch(64)
    dcs = dc_instances()
    mix = dcs + make_mix()[:4] + [(restore_instance(64, 80, 45), 5000)]
    slots = [add(gpu, b, inst, cap) for inst, cap in mix]
    b.run(100000)
    finished, running = b.poll()
    assert running == 0 and sorted(finished) == sorted(slots)
    for (inst, cap), s in zip(mix, slots):
        r = b.result(s)
        ref, rr = oracle_of(orc, inst, cap)
        got = state(inst)
        assert (r.iters, r.converged, r.value) == (rr.iters, rr.converged, rr.value), (inst["kw"], r, rr)
        assert np.array_equal(got.view(np.uint8), ref.astype(got.dtype).view(np.uint8)), inst["kw"]
    b.close()
    for inst, cap in dcs:
        solo = jacobi_instance(inst["shape"], "f64", 0, **inst["kw"])
        solo["aux"] = inst["aux"]
        stencil = gpu.SLR_J3D7 if len(inst["shape"]) == 3 else gpu.SLR_J2D5
        sv = gpu.Solver(stencil, solo["u"], solo["aux"], **inst["kw"])
        sv.run(cap)
        rs = sv.result(check=False)
        sv.close()
        assert torch.equal(solo["u"], inst["u"]) and rs.iters == oracle_of(orc, inst, cap)[1].iters


def test_defect_correction_in_short_runs_while_others_join(gpu, orc):
    # budgets that end between the phases of a correction: the phase count
    # carries over to the next run
    b = gpu.Batch(16)
    items = dc_instances()[:2]
    slots = {add(gpu, b, inst, cap): (inst, cap) for inst, cap in items}
    b.run(5)
    later = (jacobi_instance((30, 20), "f64", 46, tol=1e-10, defect_correction=1, inner_sweeps=7), 5000)
    slots[add(gpu, b, *later)] = later
    for _ in range(20000):
        b.run(3)
        _, running = b.poll()
        if running == 0:
            break
    for s, (inst, cap) in slots.items():
        r = b.result(s)
        ref, rr = oracle_of(orc, inst, cap)
        assert (r.iters, r.converged, r.value) == (rr.iters, rr.converged, rr.value)
        assert np.array_equal(state(inst).view(np.uint64), ref.view(np.uint64))
    b.close()


def test_cluster_sizes_and_partitions_match_the_oracle(gpu, orc):
    # Jacobi grids of at most 64K cells run on thread-block clusters of 1-16
    # CTAs (4096 cells a CTA at most), split into row blocks (2D) or z-slabs
    # (3D): clusters of 16, 8, 4, 2 and 1; fewer rows or planes than CTAs (some
    # CTAs hold nothing); a periodic 3D grid split across CTAs; and a single
    # row too long for one CTA's shared memory, which stays in the batch-wide loop
    mix = [
        (jacobi_instance((256, 256), "bf16", 31, tol=1e-6), 700),          # 16 CTAs, 16 rows each
        (jacobi_instance((200, 181), "f32", 32, tol=1e-7), 400),           # 16 CTAs, ragged last block
        (jacobi_instance((150, 150), "bf16", 38, tol=1e-6), 600),          # 8 CTAs
        (jacobi_instance((127, 129), "f16", 33, tol=1e-6), 900),           # 4 CTAs
        (jacobi_instance((3, 60, 64), "f32", 34, tol=1e-7), 2000),         # 4 CTAs, 3 planes
        (jacobi_instance((6, 40, 40), "f64", 35, tol=1e-9, boundary=1), 3000),   # 4 CTAs, periodic
        (jacobi_instance((2, 6000), "f32", 36, tol=1e-7), 2000),           # 4 CTAs, 2 rows
        (jacobi_instance((70, 100), "f32", 40, tol=1e-7), 2000),           # 2 CTAs
        (jacobi_instance((40, 100), "f32", 39, tol=1e-7), 2000),           # one CTA
        (jacobi_instance((1, 32768), "f32", 37, tol=1e-7), 50),            # no cluster
    ]
    b = gpu.Batch(len(mix))
    slots = [add(gpu, b, inst, cap) for inst, cap in mix]
    b.run(100000)
    b.poll()
    for (inst, cap), s in zip(mix, slots):
        r = b.result(s)
        ref, rr = oracle_of(orc, inst, cap)
        assert (r.iters, r.converged) == (rr.iters, rr.converged), (inst["shape"], r, rr)
        out = inst["u"].float().cpu().numpy() if inst["storage"] in ("bf16", "f16") else inst["u"].cpu().numpy()
        assert np.array_equal(out.view(np.uint64 if out.dtype == np.float64 else np.uint32),
                              ref.view(np.uint64 if ref.dtype == np.float64 else np.uint32)), inst["shape"]
        assert r.value == rr.value
    b.close()
