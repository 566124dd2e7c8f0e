"""Graph-Laplacian proxy operator (Eqs. 1-7, Algorithm 1): the CUDA path vs the oracle's
orc_proxy_* through the C-ABI (GPU only).

Bar: everything is integer arithmetic plus one IEEE addition of eps on the diagonal, so the
pattern, the multiplicities, the degrees, the values and the visited-entry counts are
bit-exact against the oracle on every frame, and the streamed state equals the GPU rebuild.
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
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _assert_bitwise(got, ref, what):
    gb, rb = _bits(got), _bits(ref)
    if not np.array_equal(gb, rb):
        bad = np.flatnonzero(gb != rb)
        raise AssertionError(f"{what}: {bad.size} entries differ, first {bad[0]}: "
                             f"{got[bad[0]]!r} vs {ref[bad[0]]!r}")


class _Ref:
    """The oracle's proxy state for one workload, and the GPU's upper-block view of it."""

    def __init__(self, orc, wl, eps):
        self.P = orc.Pattern(wl.n_nodes, wl.tets)
        self.ptr, self.col = self.P.proxy_pattern()
        rows = np.repeat(np.arange(wl.n_nodes), np.diff(self.ptr))
        self.upper = self.col > rows
        self.eps = eps

    def check(self, px, mult, deg, val, what):
        _, _, v = (a.cpu().numpy() for a in px.csr())
        gm, gd = (a.cpu().numpy() for a in px.state())
        _assert_bitwise(v, val, f"{what}: values")
        assert np.array_equal(gm[self.upper], mult[self.upper]), f"{what}: multiplicities"
        assert not np.any(gm[~self.upper]), f"{what}: multiplicity outside upper blocks"
        assert np.array_equal(gd, deg), f"{what}: degrees"


def _run(sta, orc, wl, eps=0.0, graph=False, noalloc=False, frames=None, policy=None):
    R = _Ref(orc, wl, eps)
    px = sta.ProxyAssembler(wl.n_nodes, wl.tets, eps=eps)
    if policy is not None:  # REFOLD: local recompute of the touched entries
        px.set_policy(policy)
    rp, col, _ = px.csr()
    assert px.nnz == R.col.size
    assert np.array_equal(rp.cpu().numpy(), R.ptr)
    assert np.array_equal(col.cpu().numpy(), R.col)
    # created all inactive: A = eps I on the mesh's nodes
    R.check(px, *R.P.proxy_rebuild(np.zeros(wl.n_tets, np.uint8), eps), "create")
    mask = wl.mask0.copy()
    px.full_rebuild(mask)
    mult, deg, val = R.P.proxy_rebuild(mask, eps)
    R.check(px, mult, deg, val, "full rebuild")
    fr = wl.frames if frames is None else wl.frames[:frames]
    if graph:
        px.graph_enable(max(int(f.shape[0] + (f[:, 0] == 2).sum()) for f in fr) or 1)
    for f, ed in enumerate(fr):
        if noalloc:
            sta.sta_apply_edits_noalloc(px.h, ed)
        else:
            px.apply_edits(ed)
        visited = R.P.proxy_update(mask, ed, mult, deg, val, eps)
        R.check(px, mult, deg, val, f"frame {f}")
        assert px.last_touched() == visited, f"frame {f}: visited entries"
        assert np.array_equal(px.mask().cpu().numpy(), mask), f"frame {f}: mask"
    v = px.values().cpu().numpy().copy()
    px.refold()  # the proxy's rebuild from the current mask
    _assert_bitwise(px.values().cpu().numpy(), v, "streamed vs GPU rebuild")
    if graph:
        px.graph_disable()
    px.close()


def test_proxy_small_workloads(sta, orc):
    _run(sta, orc, W.plain_small(seed=11))
    _run(sta, orc, W.plain_small(seed=12), eps=1e-3)
    _run(sta, orc, W.prefractured_block(N=10, sites=8, frames=8), eps=0.5)
    _run(sta, orc, W.refinement_hierarchy(N=6, radius=0.3, frames=8))
    _run(sta, orc, W.edge_fan(seed=3, K=300))


def test_proxy_local_recompute_policy(sta, orc):
    for wl, eps in ((W.plain_small(seed=21), 0.0), (W.prefractured_block(N=10, sites=8, frames=8), 0.5),
                    (W.refinement_hierarchy(N=6, radius=0.3, frames=8), 1e-3),
                    (W.edge_fan(seed=5, K=300), 0.0)):
        _run(sta, orc, wl, eps=eps, policy=sta.STA_POLICY_REFOLD)
    _run(sta, orc, W.plain_small(seed=22), graph=True, policy=sta.STA_POLICY_REFOLD)
    _run(sta, orc, W.plain_small(seed=23), noalloc=True, policy=sta.STA_POLICY_REFOLD)


def test_proxy_graph_mode_and_noalloc(sta, orc):
    _run(sta, orc, W.plain_small(seed=13), graph=True)
    _run(sta, orc, W.prefractured_block(N=10, sites=8, frames=8), graph=True)
    _run(sta, orc, W.plain_small(seed=14), noalloc=True)


def test_proxy_full_size_prefractured_block(sta, orc):
    _run(sta, orc, W.prefractured_block(), eps=1e-2, frames=6)


def test_proxy_full_size_refinement_hierarchy(sta, orc):
    _run(sta, orc, W.refinement_hierarchy(), frames=4)


def test_proxy_edge_cases(sta, orc):
    # a node of no tetrahedron (empty row), an empty frame, all tets toggled at once
    X = np.random.default_rng(2).uniform(size=(7, 3))
    tets = np.array([[5, 1, 3, 6], [5, 1, 3, 0]], np.int32)
    px = sta.ProxyAssembler(7, tets, eps=0.25)
    P = orc.Pattern(7, tets)
    mask = np.zeros(2, np.uint8)
    for ed in (np.zeros((0, 3), np.int32), W.make_edits(on=[0, 1]), W.make_edits(off=[1]),
               np.zeros((0, 3), np.int32), W.make_edits(swaps=[(0, 1)]), W.make_edits(off=[1])):
        px.apply_edits(ed)
        mask = W.apply_edits_to_mask(mask, ed)
        _, _, ref = P.proxy_rebuild(mask, 0.25)
        _assert_bitwise(px.values().cpu().numpy(), ref, "edge case frame")
    assert px.csr()[0].cpu().numpy()[3] == px.csr()[0].cpu().numpy()[2]  # node 2: empty row
    px.close()
    # no tetrahedra at all
    px = sta.ProxyAssembler(3, np.zeros((0, 4), np.int32), eps=1.0)
    px.full_rebuild(np.zeros(0, np.uint8))
    px.apply_edits(np.zeros((0, 3), np.int32))
    assert px.nnz == 0
    px.close()


def test_proxy_spmv_and_rejections(sta, orc):
    import scipy.sparse as sp
    import torch
    wl = W.plain_small(seed=4)
    px = sta.ProxyAssembler(wl.n_nodes, wl.tets, eps=0.5)
    px.full_rebuild(wl.masks()[6])
    rp, col, val = (a.cpu().numpy() for a in px.csr())
    A = sp.csr_matrix((val, col, rp), shape=(wl.n_nodes, wl.n_nodes))
    x = np.random.default_rng(0).standard_normal(wl.n_nodes)
    y = sta.sta_spmv(px.h, torch.as_tensor(x, device="cuda"))
    assert np.allclose(y.cpu().numpy(), A @ x, rtol=1e-14, atol=1e-14)
    for call in (lambda: px.set_params(E=wl.E),
                 lambda: px.element_matrices(np.array([0], np.int32)),
                 lambda: px.scatter_map(),
                 lambda: px.recompute_elements()):
        with pytest.raises(sta.StaError) as ei:
            call()
        assert ei.value.status == sta.STA_ESTATE
    px.close()
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    with pytest.raises(sta.StaError) as ei:
        sta.sta_proxy_state(asm.h)
    assert ei.value.status == sta.STA_ESTATE
    asm.close()


def test_proxy_solve_vs_direct(sta, orc):
    """sta_solve on the proxy system A = L + eps I (the paper's per-frame solve, Algorithm 1)
    against scipy's sparse direct solve, on the mesh's nodes."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    wl = W.prefractured_block(N=10, sites=8, frames=4)
    eps = 1e-2
    px = sta.ProxyAssembler(wl.n_nodes, wl.tets, eps=eps)
    mask = wl.masks()[3]
    px.full_rebuild(mask)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    ptr, col = P.proxy_pattern()
    _, _, val = P.proxy_rebuild(mask, eps)
    A = sp.csr_matrix((val, col, ptr), shape=(wl.n_nodes, wl.n_nodes))
    free = np.diff(ptr) > 0
    b = np.random.default_rng(4).standard_normal(wl.n_nodes)
    idx = np.flatnonzero(free)
    ref = np.zeros(wl.n_nodes)
    ref[idx] = spla.spsolve(A[idx][:, idx].tocsc(), b[idx])
    x, it, rel = sta.sta_solve(px.h, torch.as_tensor(b, device="cuda"),
                               torch.as_tensor(free, device="cuda"), tol=1e-12)
    xn = x.cpu().numpy()
    assert rel <= 1e-12 and it > 0
    assert np.linalg.norm(xn - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.all(xn[~free] == 0.0)
    px.close()


def test_proxy_full_size_local_recompute_and_solve(sta, orc):
    """The full-size prefractured block under the local-recompute policy (bit-exact against the
    oracle on each frame), and the per-frame solve's residual under the oracle's matrix."""
    import scipy.sparse as sp
    import torch
    wl = W.prefractured_block()
    _run(sta, orc, wl, eps=1e-2, frames=4, policy=sta.STA_POLICY_REFOLD)
    px = sta.ProxyAssembler(wl.n_nodes, wl.tets, eps=1e-2)
    mask = wl.masks()[4]
    px.full_rebuild(mask)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    ptr, col = P.proxy_pattern()
    _, _, val = P.proxy_rebuild(mask, 1e-2)
    A = sp.csr_matrix((val, col, ptr), shape=(wl.n_nodes, wl.n_nodes))
    free = np.diff(ptr) > 0
    b = np.where(free, np.random.default_rng(9).standard_normal(wl.n_nodes), 0.0)
    x, it, rel = sta.sta_solve(px.h, torch.as_tensor(b, device="cuda"),
                               torch.as_tensor(free, device="cuda"), tol=1e-10)
    xn = x.cpu().numpy()
    assert rel <= 1e-10 and it > 0
    assert np.linalg.norm((A @ xn - b)[free]) <= 10 * 1e-10 * np.linalg.norm(b)
    px.close()


@pytest.mark.parametrize("seed", range(8))
def test_proxy_random_edit_streams(sta, orc, seed):
    """Random masks and frames mixing all three edit kinds: values, multiplicities, degrees and
    visited counts ≡ the oracle every frame, both policies and graph mode over the seeds."""
    base = (W.plain_small(seed=seed, N=3, frames=1),
            W.prefractured_block(seed=seed, N=4, sites=4, frames=1),
            W.refinement_hierarchy(seed=seed, N=3, radius=0.4, frames=1))[seed % 3]
    _run(sta, orc, W.randomized(base, seed), eps=(0.0, 1e-3)[seed % 2], graph=bool(seed & 2),
         policy=sta.STA_POLICY_REFOLD if seed & 4 else None)
