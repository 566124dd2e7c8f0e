"""Batched form and CUDA-graph mode: bit-identical to plain per-instance launches.

Batched workload: 64 independent jittered cube meshes, tet counts log-uniform in [2k, 50k],
each with its own 24-frame deactivate/reactivate stream (per-instance rate uniform in
[0.1%, 5%]); all instances are rebuilt or streamed with one launch sequence per frame.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sta():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_11673_gb300 as P
    P.load_library()
    return P


def _eq(a, b):
    import torch
    return a.shape == b.shape and bool(torch.equal(a.view(torch.int64), b.view(torch.int64)))


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_plain_every_frame(sta, orc, graph):
    import torch
    insts = W.batched_instances()
    batch = sta.BatchAssembler([(w.X, w.tets, w.E, w.nu) for w in insts])
    assert sta.sta_sizes(batch.h)["n_tets"] == sum(w.n_tets for w in insts)
    if graph:
        batch.graph_enable(max_edited=1 << 16)
    plains = [sta.Assembler(w.X, w.tets, w.E, w.nu) for w in insts]
    batch.full_rebuild([w.mask0 for w in insts])
    for p, w in zip(plains, insts):
        p.full_rebuild(w.mask0)
    for i, p in enumerate(plains):
        rb, cb, vb = batch.instance_csr(i)
        rp, cp, vp = p.csr()
        assert torch.equal(rb, rp) and torch.equal(cb, cp) and _eq(vb, vp)
    for f in range(len(insts[0].frames)):
        batch.apply_edits([w.frames[f] for w in insts])
        for p, w in zip(plains, insts):
            p.apply_edits(w.frames[f])
        for i, p in enumerate(plains):
            assert _eq(batch.instance_csr(i)[2], p.values()), (f, i)
    # the full rebuild of the batch at the last frame equals the streamed values
    v = batch.values().clone()
    batch.refold()
    assert _eq(batch.values(), v)
    # two instances against the oracle
    for i in (0, len(insts) - 1):
        w = insts[i]
        P = orc.Pattern(w.n_nodes, w.tets)
        Ke, _ = orc.element_all(w.X, w.tets, w.E, w.nu)
        ref = P.rebuild(Ke, w.masks()[-1])
        got = batch.instance_csr(i)[2].cpu().numpy()
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    for p in plains:
        p.close()
    batch.close()


def test_batch_rejects_out_of_instance_ids(sta):
    insts = W.batched_instances(count=3, tmin=200, tmax=2000, frames=1)
    batch = sta.BatchAssembler([(w.X, w.tets, w.E, w.nu) for w in insts])
    batch.full_rebuild([w.mask0 for w in insts])
    bad = [W.make_edits(off=[insts[0].n_tets]), W.make_edits(), W.make_edits()]
    with pytest.raises(sta.StaError):
        batch.apply_edits(bad)
    with pytest.raises(ValueError):  # one edit list per instance, checked in the binding
        batch.apply_edits([W.make_edits(), W.make_edits()])
    batch.close()


def test_graph_mode_matches_plain_launches(sta):
    for wl in (W.plain_small(seed=3), W.prefractured_block(N=12, sites=8, frames=6)):
        a = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
        b = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
        b.graph_enable(max_edited=4096)
        a.full_rebuild(wl.mask0)
        b.full_rebuild(wl.mask0)
        assert _eq(a.values(), b.values())
        for ed in wl.frames:
            a.apply_edits(ed)
            b.apply_edits(ed)
            assert _eq(a.values(), b.values())
            assert a.last_touched() == b.last_touched()
        b.refold()
        assert _eq(a.values(), b.values())
        with pytest.raises(sta.StaError):
            b.set_launch(64, 1)      # launch shape is frozen while graphs are captured
        b.graph_disable()
        b.set_launch(64, 1)
        b.refold()
        assert _eq(a.values(), b.values())
        a.close()
        b.close()


@pytest.mark.parametrize("threads", [64, 128, 256])
@pytest.mark.parametrize("per_sm", [0, 1, 3])
@pytest.mark.parametrize("form", [1, 2])  # STA_REBUILD_FUSED, STA_REBUILD_ZERO_FILL
@pytest.mark.parametrize("depth", [4, 6])  # operand loads in flight
def test_launch_shape_does_not_change_values(sta, threads, per_sm, form, depth):
    wl = W.prefractured_block(N=10, sites=6, frames=3)
    ref = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    got = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu, block_threads=threads, blocks_per_sm=per_sm)
    got.set_rebuild_form(form)
    got.set_fold_depth(depth)
    ref.full_rebuild(wl.mask0)
    got.full_rebuild(wl.mask0)
    assert _eq(ref.values(), got.values())
    for ed in wl.frames:
        ref.apply_edits(ed)
        got.apply_edits(ed)
        assert _eq(ref.values(), got.values())
        got.refold()
        assert _eq(ref.values(), got.values())
    ref.close()
    got.close()


def test_graph_staging_mixed_with_oversized_frames(sta):
    """Graph mode with a capacity below some frames: those take the copy path, the others the
    two host-mapped blocks in turn; values and touched counts match plain launches on every
    frame, and the last count survives sta_graph_disable."""
    wl = W.plain_small(seed=8, frames=24)
    sizes = [int(ed.shape[0] + (ed[:, 0] == 2).sum()) for ed in wl.frames]
    cap = sorted(sizes)[len(sizes) // 2]          # about half the frames exceed it
    a = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    b = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    a.full_rebuild(wl.mask0)
    b.full_rebuild(wl.mask0)
    b.graph_enable(max_edited=cap)
    assert any(m > cap for m in sizes) and any(m <= cap for m in sizes)
    for ed in wl.frames:
        a.apply_edits(ed)
        b.apply_edits(ed)
        assert _eq(a.values(), b.values())
        assert a.last_touched() == b.last_touched()
    last = b.last_touched()
    b.graph_disable()
    assert b.last_touched() == last
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["refold", "fixed", "proxy", "proxy_refold"])
def test_graph_counters_across_enable_disable_and_empty_frames(sta, case):
    """Graph mode keeps two counter sets; each frame's last kernel zeroes the other set for the
    next frame.  Values and touched counts match plain launches through empty frames, graph
    mode switched off and on mid-stream, a re-capture at another capacity and a frame past the
    capacity (the copy path), for both operators and both policies."""
    wl = W.plain_small(seed=11, frames=16)
    empty = np.zeros((0, 3), np.int32)
    sizes = [int(ed.shape[0] + (ed[:, 0] == 2).sum()) for ed in wl.frames]
    if case.startswith("proxy"):
        a, b = (sta.ProxyAssembler(wl.n_nodes, wl.tets, eps=1e-3) for _ in range(2))
    else:
        a, b = (sta.Assembler(wl.X, wl.tets, wl.E, wl.nu) for _ in range(2))
    policy = sta.STA_POLICY_FIXED if case in ("fixed", "proxy") else sta.STA_POLICY_REFOLD
    for x in (a, b):
        x.set_policy(policy)
        x.full_rebuild(wl.mask0)
    b.graph_enable(max_edited=max(sizes))
    for f, ed in enumerate(wl.frames):
        if f == 4:
            b.graph_disable()
        if f == 7:
            b.graph_enable(max_edited=max(sizes))
        if f == 11:  # a smaller capacity: the largest frames take the copy path
            b.graph_disable()
            b.graph_enable(max_edited=sorted(sizes)[len(sizes) // 2])
        for frame in ((ed, empty) if f % 3 == 0 else (ed,)):
            a.apply_edits(frame)
            b.apply_edits(frame)
            assert _eq(a.values(), b.values()), f"frame {f}"
            assert a.last_touched() == b.last_touched(), f"frame {f}"
    a.close()
    b.close()
