"""CUDA path vs oracle, through the C-ABI (GPU only).

Bar: pattern, index arrays and touched counts bit-exact; element matrices and CSR values
bit-exact against the FP64 oracle (same fixed evaluation order, no implicit FMA on either
side), and streaming bit-exact against the GPU full rebuild on every frame.
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


def _bits(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.view(np.uint64)


def _vals(asm):
    return asm.values().cpu().numpy().copy()


def _check_pattern(asm, P):
    rp, col, _ = asm.csr()
    assert asm.nnz == P.nnz
    assert np.array_equal(rp.cpu().numpy(), P.row_ptr)
    assert np.array_equal(col.cpu().numpy(), P.col)
    assert np.array_equal(asm.scatter_map().cpu().numpy(), P.scat)


def _assert_bitwise(got, ref, what):
    gb, rb = _bits(got), _bits(ref)
    if not np.array_equal(gb, rb):
        bad = np.flatnonzero(gb != rb)
        k = bad[0]
        raise AssertionError(f"{what}: {bad.size} entries differ, first {k}: {got[k]!r} vs {ref[k]!r}")


def _run_stream(sta, orc, wl, eps=0.0, check_oracle_every=1, Ke=None, P=None):
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu, eps=eps)
    if P is None:
        P = orc.Pattern(wl.n_nodes, wl.tets)
    _check_pattern(asm, P)
    if Ke is None:
        Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
        assert bad == 0
    mask = wl.mask0.copy()
    asm.full_rebuild(mask)
    _assert_bitwise(_vals(asm), P.rebuild(Ke, mask, eps), "initial rebuild vs oracle")
    reb = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu, eps=eps)
    for f, ed in enumerate(wl.frames):
        asm.apply_edits(ed)
        mask = W.apply_edits_to_mask(mask, ed)
        got = _vals(asm)
        reb.full_rebuild(mask)
        _assert_bitwise(got, _vals(reb), f"frame {f}: streaming vs GPU rebuild")
        assert np.array_equal(asm.mask().cpu().numpy(), mask)
        edited = np.concatenate([ed[:, 1], ed[ed[:, 0] == 2, 2]])
        expect_touched = np.unique(P.scat[edited].reshape(-1)).size if edited.size else 0
        assert asm.last_touched() == expect_touched
        if f % check_oracle_every == 0 or f == len(wl.frames) - 1:
            _assert_bitwise(got, P.rebuild(Ke, mask, eps), f"frame {f}: GPU vs oracle")
    asm.close()
    reb.close()


def test_element_cache_bitwise(sta, orc):
    for wl in (W.plain_small(), W.adjoint_block(N=6)):
        asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
        Kg = asm.element_matrices(np.arange(wl.n_tets)).cpu().numpy().reshape(-1, 144)
        Ko, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
        assert bad == 0
        _assert_bitwise(Kg.reshape(-1), Ko.reshape(-1), "element matrices")
        asm.close()


def test_pattern_and_rebuild_small(sta, orc):
    rng = np.random.default_rng(3)
    wl = W.plain_small()
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, _ = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    _check_pattern(asm, P)
    # before any rebuild: empty active set, all +0.0
    assert np.all(_bits(_vals(asm)) == 0)
    for frac in (1.0, 0.5, 0.1, 0.0):
        mask = (rng.uniform(size=wl.n_tets) < frac).astype(np.uint8)
        asm.full_rebuild(mask)
        _assert_bitwise(_vals(asm), P.rebuild(Ke, mask), f"rebuild frac={frac}")
    asm.close()


def test_rebuild_device_mask_and_eps(sta, orc):
    import torch
    wl = W.plain_small(seed=2)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, _ = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu, eps=0.25)
    mask = wl.masks()[7]
    raw = mask * np.where(np.arange(mask.size) % 3 == 0, 3, 255).astype(np.uint8)  # any nonzero
    asm.full_rebuild(torch.as_tensor(raw, device="cuda"))
    _assert_bitwise(_vals(asm), P.rebuild(Ke, mask, 0.25), "device-mask rebuild with eps")
    assert np.array_equal(asm.mask().cpu().numpy(), mask), "kept mask is 0/1"
    # edits validated against the refreshed host mirror
    asm.apply_edits(wl.frames[7])
    _assert_bitwise(_vals(asm), P.rebuild(Ke, wl.masks()[8], 0.25), "stream after device mask")
    asm.close()


@pytest.mark.parametrize("depth", [4, 6])
@pytest.mark.parametrize("form", ["fused", "zero_fill"])
def test_rebuild_forms_bitwise(sta, orc, form, depth):
    """Both rebuild forms, with either fold depth (operand loads in flight), give the oracle's
    values bit for bit: on a mostly inactive superset (a small refinement hierarchy) and a
    mostly active one, with eps = 0 and eps != 0 (the zero-fill form still writes eps on the
    diagonal of units without an active contributor), after streaming, under the fixed-point
    policy, and captured in graph mode."""
    code = {"fused": sta.STA_REBUILD_FUSED, "zero_fill": sta.STA_REBUILD_ZERO_FILL}[form]
    for wl in (W.refinement_hierarchy(N=6, radius=0.3, frames=4),
               W.prefractured_block(N=8, sites=5, frames=4)):
        P = orc.Pattern(wl.n_nodes, wl.tets)
        Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
        assert bad == 0
        masks = wl.masks()
        for eps in (0.0, 0.5):
            asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu, eps=eps)
            asm.set_rebuild_form(code)
            asm.set_fold_depth(depth)
            asm.full_rebuild(masks[0])
            _assert_bitwise(_vals(asm), P.rebuild(Ke, masks[0], eps), f"{wl.name} {form} rebuild")
            for f, ed in enumerate(wl.frames):
                asm.apply_edits(ed)
                streamed = _vals(asm)
                asm.refold()
                ref = P.rebuild(Ke, masks[f + 1], eps)
                _assert_bitwise(streamed, ref, f"{wl.name} {form} frame {f}: stream")
                _assert_bitwise(_vals(asm), ref, f"{wl.name} {form} frame {f}: refold")
            asm.graph_enable(max(int(e.shape[0] + (e[:, 0] == 2).sum()) for e in wl.frames))
            asm.full_rebuild(masks[2])
            _assert_bitwise(_vals(asm), P.rebuild(Ke, masks[2], eps), f"{wl.name} {form} graph")
            asm.graph_disable()
            asm.set_policy(sta.STA_POLICY_FIXED)
            _, fv = P.fx_rebuild(Ke, P.fx_exponents(Ke), masks[2], eps)
            _assert_bitwise(_vals(asm), fv, f"{wl.name} {form} fixed-point rebuild")
            asm.refold()
            _assert_bitwise(_vals(asm), fv, f"{wl.name} {form} fixed-point refold")
            asm.close()


def test_rebuild_form_auto_follows_the_active_fraction(sta):
    """AUTO resolves to zero fill while fewer than 40% of the tetrahedra are active, else to the
    fused form, following the mask through rebuilds and streamed edits; an explicit form holds."""
    wl = W.plain_small(seed=4, frames=1)
    T = wl.n_tets
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    k = -(-2 * T // 5)  # the fewest active tetrahedra that are not below 40%
    mask = np.zeros(T, np.uint8)
    mask[:k] = 1
    asm.full_rebuild(mask)
    assert asm.rebuild_form() == sta.STA_REBUILD_FUSED
    asm.apply_edits(W.make_edits(off=[0]))  # one fewer: below 40%
    assert asm.rebuild_form() == sta.STA_REBUILD_ZERO_FILL
    asm.apply_edits(W.make_edits(on=[0]))
    assert asm.rebuild_form() == sta.STA_REBUILD_FUSED
    asm.full_rebuild(np.ones(T, np.uint8))
    assert asm.rebuild_form() == sta.STA_REBUILD_FUSED
    asm.set_rebuild_form(sta.STA_REBUILD_ZERO_FILL)
    assert asm.rebuild_form() == sta.STA_REBUILD_ZERO_FILL
    asm.set_rebuild_form(sta.STA_REBUILD_AUTO)
    asm.full_rebuild(np.zeros(T, np.uint8))
    assert asm.rebuild_form() == sta.STA_REBUILD_ZERO_FILL
    asm.close()


def test_rebuild_form_rejections(sta):
    wl = W.plain_small(seed=3, frames=1)
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    for call, bad in ((asm.set_rebuild_form, 3), (asm.set_fold_depth, 5), (asm.set_fold_depth, 0)):
        with pytest.raises(sta.StaError) as e:
            call(bad)
        assert e.value.status == sta.STA_EINVAL
    asm.graph_enable(64)
    for call, arg in ((asm.set_rebuild_form, sta.STA_REBUILD_FUSED), (asm.set_fold_depth, 6)):
        with pytest.raises(sta.StaError) as e:
            call(arg)
        assert e.value.status == sta.STA_ESTATE
    asm.graph_disable()
    asm.set_rebuild_form(sta.STA_REBUILD_AUTO)
    asm.set_fold_depth(6)
    asm.close()


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_streaming_plain_small_every_frame(sta, orc, seed):
    _run_stream(sta, orc, W.plain_small(seed=seed))


def test_streaming_eps_and_small_variants(sta, orc):
    _run_stream(sta, orc, W.plain_small(seed=7), eps=1e-3)
    _run_stream(sta, orc, W.prefractured_block(N=10, sites=8, frames=8))
    _run_stream(sta, orc, W.refinement_hierarchy(N=6, radius=0.3, frames=8))
    for wl in W.batched_instances(count=4, tmin=300, tmax=5000, frames=6):
        _run_stream(sta, orc, wl)


def test_long_contributor_lists(sta, orc):
    # one node pair and both its nodes shared by K tetrahedra (70% active at start): lists
    # longer than the folds' shared-memory staging (streamed units: 24 runs staged, longer
    # lists load their operands from global memory, lists beyond 64 active contributions of a
    # diagonal unit or 96 of a pair fold directly; rebuild tiles: 448 codes)
    for K, eps in ((40, 0.0), (80, 1e-3), (300, 0.0), (1000, 1e-2)):
        _run_stream(sta, orc, W.edge_fan(seed=K, K=K), eps=eps)


def test_edge_cases(sta, orc):
    # single tetrahedron with unused nodes around it
    X = np.random.default_rng(0).uniform(size=(7, 3))
    X[[5, 1, 3, 6]] = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    tets = np.array([[5, 1, 3, 6]], np.int32)
    E, nu = np.array([2.0]), np.array([0.25])
    asm = sta.Assembler(X, tets, E, nu)
    P = orc.Pattern(7, tets)
    _check_pattern(asm, P)
    Ke, _ = orc.element_all(X, tets, E, nu)
    asm.full_rebuild(np.ones(1, np.uint8))
    _assert_bitwise(_vals(asm), P.rebuild(Ke, np.ones(1, np.uint8)), "single tet")
    asm.apply_edits(W.make_edits(off=[0]))
    assert np.all(_bits(_vals(asm)) == 0)                 # back to exact +0.0
    asm.apply_edits(np.zeros((0, 3), np.int32))           # empty frame is a no-op
    assert asm.last_touched() == 0
    asm.apply_edits(W.make_edits(on=[0]))
    _assert_bitwise(_vals(asm), P.rebuild(Ke, np.ones(1, np.uint8)), "reactivated")
    asm.close()
    # empty mesh
    asm = sta.Assembler(np.zeros((3, 3)), np.zeros((0, 4), np.int32), np.zeros(0), np.zeros(0))
    assert asm.nnz == 0
    asm.full_rebuild(np.zeros(0, np.uint8))
    asm.apply_edits(np.zeros((0, 3), np.int32))
    asm.close()


def test_rejected_edits_change_nothing(sta, orc):
    wl = W.plain_small()
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    asm.full_rebuild(wl.mask0)
    asm.apply_edits(wl.frames[0])
    before, mask_before = _vals(asm), asm.mask().cpu().numpy().copy()
    m = W.apply_edits_to_mask(wl.mask0, wl.frames[0])
    inactive = int(np.flatnonzero(m == 0)[0])
    active = int(np.flatnonzero(m)[0])
    for bad in (W.make_edits(off=[inactive]), W.make_edits(on=[active]),
                W.make_edits(off=[active, active]), W.make_edits(off=[wl.n_tets]),
                W.make_edits(swaps=[(active, active)]), np.array([[7, 0, -1]], np.int32),
                np.concatenate([W.make_edits(off=[active]), W.make_edits(off=[inactive])])):
        with pytest.raises(sta.StaError):
            asm.apply_edits(bad)
        _assert_bitwise(_vals(asm), before, "values after a rejected call")
        assert np.array_equal(asm.mask().cpu().numpy(), mask_before)
    # the context still works
    asm.apply_edits(wl.frames[1])
    ref = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    ref.full_rebuild(W.apply_edits_to_mask(m, wl.frames[1]))
    _assert_bitwise(_vals(asm), _vals(ref), "after recovery")
    asm.close()
    ref.close()


def test_bad_meshes_rejected(sta):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    with pytest.raises(sta.StaError) as e:
        sta.Assembler(X, np.array([[0, 2, 1, 3]], np.int32), [1.0], [0.3])  # inverted
    assert e.value.status == sta.STA_EINVAL and "det <= 0" in str(e.value)
    with pytest.raises(sta.StaError):
        sta.Assembler(X, np.array([[0, 1, 2, 4]], np.int32), [1.0], [0.3])  # id out of range


def test_set_params_then_rebuild(sta, orc):
    wl = W.plain_small(seed=4)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    rng = np.random.default_rng(9)
    E2 = rng.uniform(5e4, 2e5, wl.n_tets)
    X2 = wl.X + rng.uniform(-0.01, 0.01, wl.X.shape)
    asm.set_params(X=X2, E=E2)
    mask = wl.masks()[3]
    asm.full_rebuild(mask)
    Ke, _ = orc.element_all(X2, wl.tets, E2, wl.nu)
    _assert_bitwise(_vals(asm), P.rebuild(Ke, mask), "after set_params")
    asm.recompute_elements(active_only=True)
    asm.full_rebuild(mask)
    _assert_bitwise(_vals(asm), P.rebuild(Ke, mask), "after active-only recompute")
    asm.close()


# ---------------------------------------------------------------- full-size workloads

def _full_size(sta, orc, wl, frames_to_oracle, form=None, depth=None, graph=False):
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    assert bad == 0
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    _check_pattern(asm, P)
    reb = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    for x in (asm, reb):  # the rebuild schedule under test (the values do not depend on it)
        if form is not None:
            x.set_rebuild_form(form)
        if depth is not None:
            x.set_fold_depth(depth)
    masks = wl.masks()
    if graph:
        asm.graph_enable(max(int(e.shape[0] + (e[:, 0] == 2).sum()) for e in wl.frames))
        reb.graph_enable(1)
    asm.full_rebuild(masks[0])
    for f, ed in enumerate(wl.frames):
        asm.apply_edits(ed)
        reb.full_rebuild(masks[f + 1])
        got = _vals(asm)
        _assert_bitwise(got, _vals(reb), f"{wl.name} frame {f}: stream vs rebuild")
        if f in frames_to_oracle:
            _assert_bitwise(got, P.rebuild(Ke, masks[f + 1]), f"{wl.name} frame {f}: vs oracle")
    asm.close()
    reb.close()


def test_full_size_prefractured_block(sta, orc):
    _full_size(sta, orc, W.prefractured_block(), {0, 11, 23})


def test_full_size_refinement(sta, orc):
    _full_size(sta, orc, W.refinement_hierarchy(), {0, 23})


def test_full_size_refinement_r040_tuned_schedule(sta, orc):
    """The "up to ~460k active" case with the schedule the autotuner picks for it on GB300 (zero
    fill, 6 operand loads in flight) and CUDA graphs: streamed ≡ rebuilt every frame, ≡ the
    oracle on three frames."""
    _full_size(sta, orc, W.refinement_hierarchy(radius=0.40), {0, 12, 23},
               form=sta.STA_REBUILD_ZERO_FILL, depth=6, graph=True)


@pytest.mark.parametrize("seed", range(24))
def test_random_edit_streams(sta, orc, seed):
    """Random masks and random frames mixing all three edit kinds, on small supersets of the
    three shapes (plain, pre-fractured, refinement), each seed with its own schedule (rebuild
    form, fold depth, eps, graph mode with a capacity some frames exceed): streamed values ≡
    the oracle's rebuild every frame, the touched count and the mask exact, a refold every third
    frame ≡ the same values."""
    base = (W.plain_small(seed=seed, N=3, frames=1),
            W.prefractured_block(seed=seed, N=4, sites=4, frames=1),
            W.refinement_hierarchy(seed=seed, N=3, radius=0.4, frames=1))[seed % 3]
    wl = W.randomized(base, seed)
    rng = np.random.default_rng(7000 + seed)  # the schedule
    eps = (0.0, 1e-3)[seed % 2]
    form = (sta.STA_REBUILD_AUTO, sta.STA_REBUILD_FUSED, sta.STA_REBUILD_ZERO_FILL)[(seed // 3) % 3]
    depth = (4, 6)[int(rng.integers(2))]
    graph = bool(rng.integers(2))
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    assert bad == 0
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu, eps=eps)
    asm.set_rebuild_form(form)
    asm.set_fold_depth(depth)
    mask = wl.mask0.copy()
    asm.full_rebuild(mask)
    _assert_bitwise(_vals(asm), P.rebuild(Ke, mask, eps), f"seed {seed}: initial rebuild")
    if graph:
        asm.graph_enable(max_edited=12)  # frames of more edited tets take the copy path
    for f, ed in enumerate(wl.frames):
        asm.apply_edits(ed)
        mask = W.apply_edits_to_mask(mask, ed)
        ref = P.rebuild(Ke, mask, eps)
        what = f"seed {seed} frame {f} ({ed.shape[0]} edits, form {form}, depth {depth}, graph {graph})"
        _assert_bitwise(_vals(asm), ref, what)
        assert np.array_equal(asm.mask().cpu().numpy(), mask), what
        edited = np.concatenate([ed[:, 1], ed[ed[:, 0] == 2, 2]]) if ed.shape[0] else ed[:, 1]
        expect = np.unique(P.scat[edited].reshape(-1)).size if edited.size else 0
        assert asm.last_touched() == expect, what
        if f % 3 == 2:
            asm.refold()
            _assert_bitwise(_vals(asm), ref, what + ", refold")
    asm.close()
