"""Fixed-point policy (STA_POLICY_FIXED, the paper's additive streaming_update made exact): the
CUDA path vs the oracle's fixed-point definition (orc_fx_*), bit for bit, on every frame; the
streamed values vs the GPU's own fixed-point rebuild; switching back to the canonical fold."""
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


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _assert_bitwise(got, ref, what):
    got = got.cpu().numpy() if hasattr(got, "cpu") else got
    gb, rb = _bits(got), _bits(ref)
    if not np.array_equal(gb, rb):
        bad = np.flatnonzero(gb != rb)
        raise AssertionError(f"{what}: {bad.size} entries differ, first {bad[0]}: "
                             f"{got[bad[0]]!r} vs {ref[bad[0]]!r}")


def _run_fixed(sta, orc, wl, eps=0.0, graph=False, noalloc=False, frames=None):
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    assert bad == 0
    e = P.fx_exponents(Ke)
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu, eps=eps)
    asm.full_rebuild(wl.mask0)
    asm.set_policy(sta.STA_POLICY_FIXED)
    mask = wl.mask0.copy()
    S, val = P.fx_rebuild(Ke, e, mask, eps)
    _assert_bitwise(asm.values(), val, "fixed-point rebuild vs oracle")
    fr = wl.frames if frames is None else wl.frames[:frames]
    if graph:
        asm.graph_enable(max(int(f.shape[0] + (f[:, 0] == 2).sum()) for f in fr) or 1)
    for f, ed in enumerate(fr):
        if noalloc:
            sta.sta_apply_edits_noalloc(asm.h, ed)
        else:
            asm.apply_edits(ed)
        P.fx_update(Ke, e, mask, ed, S, val, eps)
        _assert_bitwise(asm.values(), val, f"frame {f}: fixed-point streaming vs oracle")
        edited = np.concatenate([ed[:, 1], ed[ed[:, 0] == 2, 2]])
        expect = np.unique(P.scat[edited].reshape(-1)).size if edited.size else 0
        assert asm.last_touched() == expect
    v = asm.values().clone()
    asm.refold()
    _assert_bitwise(asm.values(), v.cpu().numpy(), "streamed vs GPU fixed-point rebuild")
    if graph:
        asm.graph_disable()
    asm.set_policy(sta.STA_POLICY_REFOLD)
    _assert_bitwise(asm.values(), P.rebuild(Ke, mask, eps), "back to the canonical fold")
    asm.close()


def test_fixed_point_small_workloads(sta, orc):
    _run_fixed(sta, orc, W.plain_small(seed=11))
    _run_fixed(sta, orc, W.plain_small(seed=12), eps=1e-3)
    _run_fixed(sta, orc, W.prefractured_block(N=10, sites=8, frames=8))
    _run_fixed(sta, orc, W.refinement_hierarchy(N=6, radius=0.3, frames=8))


def test_fixed_point_graph_mode_and_noalloc(sta, orc):
    _run_fixed(sta, orc, W.plain_small(seed=13), graph=True)
    _run_fixed(sta, orc, W.plain_small(seed=14), noalloc=True)


def test_fixed_point_long_contributor_lists(sta, orc):
    _run_fixed(sta, orc, W.edge_fan(seed=3, K=300))


def test_fixed_point_full_size_prefractured_block(sta, orc):
    _run_fixed(sta, orc, W.prefractured_block(), frames=6)


def test_fixed_point_policy_rejected_in_graph_mode(sta):
    wl = W.plain_small()
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    asm.full_rebuild(wl.mask0)
    asm.graph_enable(64)
    with pytest.raises(sta.StaError):
        asm.set_policy(sta.STA_POLICY_FIXED)
    with pytest.raises(sta.StaError):
        asm.set_policy(7)
    asm.close()


@pytest.mark.parametrize("seed", range(8))
def test_fixed_point_random_edit_streams(sta, orc, seed):
    """Random masks and frames mixing all three edit kinds on small supersets of the three
    shapes: the fixed-point frame ≡ the oracle's definition every frame (eps and graph mode
    alternating over the seeds)."""
    base = (W.plain_small(seed=seed, N=3, frames=1),
            W.prefractured_block(seed=seed, N=4, sites=4, frames=1),
            W.refinement_hierarchy(seed=seed, N=3, radius=0.4, frames=1))[seed % 3]
    _run_fixed(sta, orc, W.randomized(base, seed), eps=(0.0, 1e-3)[seed % 2],
               graph=bool(seed & 2))
