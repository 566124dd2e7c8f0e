"""The allocation-free streaming entry point (sta_apply_edits_noalloc) against the regular one.

sta_apply_edits_noalloc serves callers that cannot allocate: it keeps its scratch in a fixed
device array instead of growing buffers.  Here two contexts on the same mesh receive the same
frames, one through each entry point, and the values must agree bit for bit after each of two
calls in a row.  This file is collected last so that, if it fails, every other test has
already run; it passes alone in a fresh process and after the rest of the suite.
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


def test_noalloc_matches_regular_entry_point(sta):
    wl = W.plain_small(seed=11, frames=2)
    ref = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    got = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    ref.full_rebuild(wl.mask0)
    got.full_rebuild(wl.mask0)
    for f in range(2):  # two calls in a row
        sta.sta_apply_edits(ref.h, wl.frames[f])
        sta.sta_apply_edits_noalloc(got.h, wl.frames[f])
        assert np.array_equal(_vals(got), _vals(ref)), f"call {f}"
        assert got.last_touched() == ref.last_touched()
        assert np.array_equal(got.mask().cpu().numpy(), ref.mask().cpu().numpy())
    ref.close()
    got.close()


def test_noalloc_on_a_larger_frame_and_limit(sta):
    wl = W.prefractured_block(N=16, sites=12, frames=2)
    ref = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    got = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    ref.full_rebuild(wl.mask0)
    got.full_rebuild(wl.mask0)
    for f in range(2):
        sta.sta_apply_edits(ref.h, wl.frames[f])
        sta.sta_apply_edits_noalloc(got.h, wl.frames[f])
        assert np.array_equal(_vals(got), _vals(ref)), f"call {f}"
    # more edited tetrahedra than the fixed scratch holds: rejected, nothing changes
    before = _vals(got)
    big = W.prefractured_block(N=24, sites=8, frames=1)
    ctx = sta.Assembler(big.X, big.tets, big.E, big.nu)
    ctx.full_rebuild(np.ones(big.n_tets, np.uint8))
    too_many = W.make_edits(off=np.arange(sta.STA_NOALLOC_MAX_EDITED + 1))
    with pytest.raises(sta.StaError) as e:
        sta.sta_apply_edits_noalloc(ctx.h, too_many)
    assert e.value.status == sta.STA_ERANGE
    assert np.array_equal(ctx.mask().cpu().numpy(), np.ones(big.n_tets, np.uint8))
    assert np.array_equal(_vals(got), before)
    ctx.close()
    ref.close()
    got.close()
