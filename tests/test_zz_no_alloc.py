"""The allocation-free streaming entry point (sta_apply_edits_noalloc) against the regular one.

sta_apply_edits_noalloc serves callers that cannot allocate: it keeps its scratch in a fixed
device array instead of growing buffers.  Here two contexts on the same mesh receive the same
frames, one through each entry point, and the values must agree bit for bit after each of two
calls in a row -- for the elasticity operator under both update policies (the canonical re-fold
and the exact fixed-point additive update) and for the graph-Laplacian proxy operator, each of
which writes its touched list into the shared array.  The fixed limit is checked from both
sides: exactly STA_NOALLOC_MAX_EDITED edited tetrahedra succeed, one more is rejected.  This
file is collected last so that, if it fails, every other test has already run; it passes alone
in a fresh process and after the rest of the suite.
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


def _vals(asm):
    return asm.values().cpu().numpy().copy().view(np.uint64)


def _pair(sta, wl, kind):
    """Two identical contexts of the given kind on the workload, rebuilt from its first mask."""
    out = []
    for _ in range(2):
        if kind == "proxy":
            a = sta.ProxyAssembler(wl.n_nodes, wl.tets, eps=1e-3)
        else:
            a = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
        a.full_rebuild(wl.mask0)
        if kind == "fixed":
            a.set_policy(sta.STA_POLICY_FIXED)
        out.append(a)
    return out


@pytest.mark.parametrize("kind", ["refold", "fixed", "proxy"])
def test_noalloc_matches_regular_entry_point(sta, kind):
    wl = W.plain_small(seed=11, frames=2)
    ref, got = _pair(sta, wl, kind)
    for f in range(2):  # two calls in a row
        sta.sta_apply_edits(ref.h, wl.frames[f])
        sta.sta_apply_edits_noalloc(got.h, wl.frames[f])
        assert np.array_equal(_vals(got), _vals(ref)), f"call {f}"
        assert got.last_touched() == ref.last_touched()
        assert np.array_equal(got.mask().cpu().numpy(), ref.mask().cpu().numpy())
    if kind == "proxy":
        for a, b in zip(got.state(), ref.state()):
            assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    ref.close()
    got.close()


@pytest.mark.parametrize("kind", ["refold", "fixed", "proxy"])
def test_noalloc_on_a_larger_frame(sta, kind):
    wl = W.prefractured_block(N=16, sites=12, frames=2)
    ref, got = _pair(sta, wl, kind)
    for f in range(2):
        sta.sta_apply_edits(ref.h, wl.frames[f])
        sta.sta_apply_edits_noalloc(got.h, wl.frames[f])
        assert np.array_equal(_vals(got), _vals(ref)), f"call {f}"
        assert got.last_touched() == ref.last_touched()
    ref.close()
    got.close()


def test_noalloc_limit_from_both_sides(sta):
    big = W.prefractured_block(N=24, sites=8, frames=1)
    lim = sta.STA_NOALLOC_MAX_EDITED
    assert big.n_tets > lim + 1
    ref = sta.Assembler(big.X, big.tets, big.E, big.nu)
    got = sta.Assembler(big.X, big.tets, big.E, big.nu)
    full = np.ones(big.n_tets, np.uint8)
    ref.full_rebuild(full)
    got.full_rebuild(full)
    # one more edited tetrahedron than the fixed scratch holds: rejected, nothing changes
    before = _vals(got)
    with pytest.raises(sta.StaError) as e:
        sta.sta_apply_edits_noalloc(got.h, W.make_edits(off=np.arange(lim + 1)))
    assert e.value.status == sta.STA_ERANGE
    assert np.array_equal(got.mask().cpu().numpy(), full)
    assert np.array_equal(_vals(got), before)
    # exactly the maximum (half of it as swaps: a swap edits two tetrahedra): accepted, and
    # equal to the regular entry point
    frames = [W.make_edits(off=np.arange(lim)),
              W.make_edits(swaps=[(lim + k, k) for k in range(lim // 2)])]
    for f, ed in enumerate(frames):
        sta.sta_apply_edits(ref.h, ed)
        sta.sta_apply_edits_noalloc(got.h, ed)
        assert np.array_equal(_vals(got), _vals(ref)), f"call {f}"
        assert got.last_touched() == ref.last_touched()
        assert np.array_equal(got.mask().cpu().numpy(), ref.mask().cpu().numpy())
    ref.close()
    got.close()
