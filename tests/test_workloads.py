"""The full-size synthetic workloads match their stated recipes (sizes, active counts, edit
volume and structure), so the benchmark's configuration and the full-size parity cases cannot
drift silently, and every frame is a valid edit set under the oracle's rules (no GPU needed)."""
import numpy as np

import workloads as W


def _valid_stream(orc, wl):
    masks = wl.masks()
    for f, ed in enumerate(wl.frames):
        assert orc.validate_edits(wl.n_tets, masks[f], ed) == 0, f"frame {f}"
    return masks


def test_prefractured_block_recipe(orc):
    """40^3 x 6 Kuhn tets with a split copy of every tet on a cell boundary of 64 Voronoi
    cells; 24 frames of swaps (a tet traded for its split copy), so the active count stays."""
    wl = W.prefractured_block()
    assert (wl.n_tets, wl.n_nodes) == (579_239, 114_072)
    assert orc.Pattern(wl.n_nodes, wl.tets).nnz == 14_091_174
    assert len(wl.frames) == 24
    assert all((ed[:, 0] == 2).all() for ed in wl.frames)  # op 2 = swap
    swaps = [ed.shape[0] for ed in wl.frames]
    assert (min(swaps), max(swaps)) == (166, 6116)
    masks = _valid_stream(orc, wl)
    assert {int(m.sum()) for m in masks} == {40 ** 3 * 6}
    # a swap's new tet is a split copy: an id beyond the base mesh
    assert all((ed[:, 2] >= 40 ** 3 * 6).all() for ed in wl.frames)


def test_refinement_hierarchy_recipe(orc):
    """30^3 x 6 coarse tets, each with 8 preallocated children (ids 162,000 + 8p + k); at every
    frame each coarse tet is either active with no active child or inactive with all 8
    children active."""
    wl = W.refinement_hierarchy()
    nc = 30 ** 3 * 6
    assert (wl.n_tets, wl.n_nodes) == (9 * nc, 226_981)
    assert orc.Pattern(wl.n_nodes, wl.tets).nnz == 33_394_689
    masks = _valid_stream(orc, wl)
    for f, m in enumerate(masks):
        parent = m[:nc].astype(bool)
        kids = m[nc:].reshape(nc, 8).astype(int).sum(axis=1)
        assert np.all(kids[parent] == 0) and np.all(kids[~parent] == 8), f"frame {f}"
    active = np.mean([int(m.sum()) for m in masks[1:]])
    assert 170_000 < active < 186_000  # about 178k at radius 0.15


def test_batched_and_adjoint_recipes(orc):
    insts = W.batched_instances()
    T = [w.n_tets for w in insts]
    assert len(insts) == 64 and sum(T) == 1_081_044
    assert min(T) >= 2_000 and max(T) <= 50_000
    for w in insts[:4]:
        _valid_stream(orc, w)
    a = W.adjoint_block()
    assert (a.n_tets, a.n_nodes, len(a.frames)) == (20 ** 3 * 6, 21 ** 3, 24)
    _valid_stream(orc, a)


def test_random_edit_streams_are_valid_frames():
    """The randomized parity tests' input: every frame names each tetrahedron once, deactivates
    active ones, activates inactive ones and swaps an active one for an inactive one; some
    frames are empty and every edit kind occurs."""
    base = W.prefractured_block(seed=0, N=4, sites=4, frames=1)
    kinds, empty = set(), 0
    for seed in range(6):
        wl = W.randomized(base, seed)
        m = wl.mask0.copy()
        for ed in wl.frames:
            empty += ed.shape[0] == 0
            tets = np.concatenate([ed[:, 1], ed[ed[:, 0] == W.SWAP, 2]])
            assert np.unique(tets).size == tets.size
            for op, t, t2 in ed:
                kinds.add(int(op))
                assert m[t] == (op != W.ACTIVATE)
                if op == W.SWAP:
                    assert m[t2] == 0
            m = W.apply_edits_to_mask(m, ed)
    assert kinds == {W.DEACTIVATE, W.ACTIVATE, W.SWAP} and empty > 0
