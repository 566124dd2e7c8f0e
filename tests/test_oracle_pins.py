"""Pins of the oracle against what the mathematics and the paper fix (no GPU needed).

Each test checks the oracle against something other than itself: hand-derived closed
forms, rigid-body invariants, a literal B^T D B product, dense brute force, the linear
patch test, finite differences, complex step, and the exactness invariant of Sec. 3.3.
"""
from pathlib import Path

import numpy as np
import pytest

import workloads as W

GOLD = Path(__file__).resolve().parent / "golden"


def _random_tet(rng, quality=0.3):
    while True:
        x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
        x = x + rng.uniform(-quality, quality, size=(4, 3))
        x = x * rng.uniform(0.1, 10.0) + rng.uniform(-5, 5, size=3)
        d = x[1:] - x[0]
        if np.linalg.det(d.T) > 1e-6:
            return x


def _load_golden():
    cases, cur = {}, None
    for line in (GOLD / "reference_tet.txt").read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        if line.startswith("case"):
            parts = dict(p.split("=") for p in line.split()[2:])
            num, den = parts["scale"].split("/")
            cur = (float(parts["E"]), float(parts["nu"]), float(num) / float(den))
            cases[cur] = []
        else:
            cases[cur].append([int(v) for v in line.split()])
    return {k: np.array(v, float) for k, v in cases.items()}


# ---------------------------------------------------------------- element matrix


def test_element_reference_tet_closed_form(orc):
    """Hand-derived values on the unit right tetrahedron (tests/golden/reference_tet.txt)."""
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    for (E, nu, scale), M in _load_golden().items():
        assert M.shape == (12, 12)
        K = orc.element(x, E, nu)
        np.testing.assert_allclose(K, scale * M, rtol=0, atol=4e-16)


def test_element_symmetric_exactly_and_rigid_modes(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = _random_tet(rng)
        E, nu = rng.uniform(1e3, 1e6), rng.uniform(0.0, 0.45)
        K = orc.element(x, E, nu)
        assert np.array_equal(K, K.T)
        w = np.linalg.eigvalsh(K)
        lmax = w[-1]
        assert np.sum(np.abs(w) <= 1e-12 * lmax) == 6, w
        assert np.sum(w >= 1e-6 * lmax) == 6, w
        assert w[0] >= -1e-12 * lmax
        # 3 translations and 3 infinitesimal rotations u(x) = omega x x
        modes = []
        for ax in range(3):
            u = np.zeros((4, 3))
            u[:, ax] = 1.0
            modes.append(u.reshape(12))
        for ax in range(3):
            om = np.zeros(3)
            om[ax] = 1.0
            modes.append(np.cross(om, x).reshape(12))
        nK = np.linalg.norm(K, 2)
        for r in modes:
            assert np.linalg.norm(K @ r) <= 1e-12 * nK * np.linalg.norm(r)


def test_element_matches_literal_btdb(orc):
    """The fixed-order closed form equals V B^T D B formed literally (different rounding)."""
    rng = np.random.default_rng(2)
    for _ in range(100):
        x = _random_tet(rng)
        E, nu = rng.uniform(1e3, 1e6), rng.uniform(0.0, 0.45)
        K = orc.element(x, E, nu)
        K2 = orc.element_btdb(x, E, nu)
        assert np.max(np.abs(K - K2)) <= 1e-14 * np.max(np.abs(K2)) * 10


def test_element_scaling_and_rotation(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = _random_tet(rng)
        E, nu = rng.uniform(1e3, 1e6), rng.uniform(0.0, 0.45)
        K = orc.element(x, E, nu)
        # linear in E, exactly for a factor 2 (all steps scale by a power of two)
        assert np.array_equal(orc.element(x, 2 * E, nu), 2 * K)
        # K scales like length^1 (V ~ s^3, g ~ 1/s)
        s = 3.7
        np.testing.assert_allclose(orc.element(s * x, E, nu), s * K, rtol=1e-12,
                                   atol=1e-13 * np.abs(K).max())
        # rotation covariance: K(Rx) = R_blk K R_blk^T
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        Rb = np.kron(np.eye(4), q)
        Kr = orc.element(x @ q.T, E, nu)
        np.testing.assert_allclose(Kr, Rb @ K @ Rb.T, rtol=0, atol=1e-12 * np.abs(K).max())


def test_element_rejects_inverted(orc):
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    with pytest.raises(ValueError):
        orc.element(x[[0, 2, 1, 3]], 1.0, 0.3)
    with pytest.raises(ValueError):
        orc.element(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 0, 1.0]]), 1.0, 0.3)


# ---------------------------------------------------------------- pattern + rebuild


def _dense_bruteforce(n, tets, Ke, mask):
    """Dense 3n x 3n assembly, tetrahedra in ascending order, P_tau as DOF indexing."""
    D = np.zeros((3 * n, 3 * n))
    for t in range(tets.shape[0]):
        if not mask[t]:
            continue
        dofs = (3 * tets[t][:, None] + np.arange(3)[None, :]).reshape(12)
        for p in range(12):
            for q in range(12):
                D[dofs[p], dofs[q]] += Ke[t].reshape(12, 12)[p, q]
    return D


def _tiny_meshes():
    rng = np.random.default_rng(7)
    out = []
    X, tets, _ = W.kuhn_cube(1, 0.1, rng, nx=2)      # 2 hexes -> 12 tets
    out.append((X, tets))
    X, tets, _ = W.kuhn_cube(1, 0.2, rng)            # 1 hex -> 6 tets
    out.append((X, tets))
    # a single tet with unused node ids around it (empty rows), shuffled node numbering
    X = rng.uniform(0, 1, size=(7, 3))
    X[[5, 1, 3, 6]] = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    out.append((X, np.array([[5, 1, 3, 6]], np.int32)))
    return out


def test_pattern_and_rebuild_vs_dense_bruteforce(orc):
    rng = np.random.default_rng(8)
    for X, tets in _tiny_meshes():
        n, T = X.shape[0], tets.shape[0]
        E = rng.uniform(1e4, 1e5, T)
        nu = rng.uniform(0.1, 0.4, T)
        Ke, bad = orc.element_all(X, tets, E, nu)
        assert bad == 0
        P = orc.Pattern(n, tets)
        # pattern = all (node, node) pairs sharing a tetrahedron, full 3x3 blocks
        pairs = {(int(a), int(b)) for t in tets for a in t for b in t}
        expect_nnz = 9 * len(pairs)
        assert P.nnz == expect_nnz
        rows = np.repeat(np.arange(P.nrows), np.diff(P.row_ptr))
        got = {(int(r // 3), int(c // 3)) for r, c in zip(rows, P.col)}
        assert got == pairs
        for r in range(P.nrows):  # ascending columns
            assert np.all(np.diff(P.col[P.row_ptr[r]:P.row_ptr[r + 1]]) > 0)
        for mask in (np.ones(T, np.uint8), (rng.uniform(size=T) < 0.5).astype(np.uint8),
                     np.zeros(T, np.uint8)):
            val = P.rebuild(Ke, mask)
            D = _dense_bruteforce(n, tets, Ke, mask)
            S = P.csr(val).toarray()
            assert np.array_equal(S, D)                # bitwise, same order of additions
            assert np.array_equal(S, S.T)              # exactly symmetric
            assert not np.any(np.signbit(val) & (val == 0))  # no -0.0
        # eps on the diagonal only, added last
        val = P.rebuild(Ke, np.ones(T, np.uint8), eps=0.5)
        D = _dense_bruteforce(n, tets, Ke, np.ones(T, np.uint8))
        D[np.diag_indices(3 * n)] += np.where(np.isin(np.arange(3 * n) // 3, tets), 0.5, 0.0)
        assert np.array_equal(P.csr(val).toarray(), D)


def test_rebuild_row_sums_and_patch_test(orc):
    wl = W.plain_small()
    n, T = wl.n_nodes, wl.n_tets
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    assert bad == 0
    P = orc.Pattern(n, wl.tets)
    K = P.csr(P.rebuild(Ke, np.ones(T, np.uint8)))
    scale = np.abs(K).max()
    for ax in range(3):                      # constant displacement -> zero force
        u = np.zeros((n, 3))
        u[:, ax] = 1.0
        assert np.abs(K @ u.reshape(-1)).max() <= 1e-12 * scale
    # linear patch test: u = A x + b gives zero force at interior nodes
    rng = np.random.default_rng(0)
    A = rng.standard_normal((3, 3))
    u = wl.X @ A.T + rng.standard_normal(3)
    f = (K @ u.reshape(-1)).reshape(n, 3)
    gi = wl.meta["grid_index"]
    N = wl.meta["N"]
    interior = np.all((gi > 0) & (gi < N), axis=1)
    assert interior.sum() > 0
    assert np.abs(f[interior]).max() <= 1e-10 * scale * np.abs(u).max()
    assert np.abs(f[~interior]).max() > 1e-3 * scale * np.abs(u).max()  # boundary loads
    # energy >= 0; SPD once the bottom layer is clamped
    w = np.linalg.eigvalsh(K.toarray())
    assert w[0] >= -1e-10 * w[-1]
    free = np.repeat(gi[:, 2] > 0, 3)
    Kff = K.toarray()[np.ix_(free, free)]
    np.linalg.cholesky(Kff)


def test_rebuild_vs_scipy_coo_sum(orc):
    """Library cross-check at a size beyond brute force: scipy's COO duplicate sum."""
    import scipy.sparse as sp
    wl = W.prefractured_block(N=8, sites=6, frames=2)
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    assert bad == 0
    P = orc.Pattern(wl.n_nodes, wl.tets)
    mask = wl.masks()[-1]
    val = P.rebuild(Ke, mask)
    act = np.flatnonzero(mask)
    dofs = (3 * wl.tets[act][:, :, None] + np.arange(3)).reshape(-1, 12)
    rr = np.repeat(dofs, 12, axis=1).reshape(-1)
    cc = np.tile(dofs, (1, 12)).reshape(-1)
    ref = sp.coo_matrix((Ke[act].reshape(-1), (rr, cc)),
                        shape=(P.nrows, P.nrows)).tocsr().toarray()
    got = P.csr(val).toarray()
    absum = sp.coo_matrix((np.abs(Ke[act]).reshape(-1), (rr, cc)),
                          shape=(P.nrows, P.nrows)).tocsr().toarray()
    assert np.all(np.abs(got - ref) <= 1e-13 * absum)
    # every entry with no active contributor is exactly +0.0
    assert np.all(got[absum == 0] == 0)


def test_entry_matches_rebuild(orc):
    wl = W.plain_small()
    Ke, _ = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    mask = wl.masks()[5]
    val = P.rebuild(Ke, mask, eps=1e-3)
    rng = np.random.default_rng(4)
    rows = np.repeat(np.arange(P.nrows), np.diff(P.row_ptr))
    for k in rng.choice(P.nnz, 300, replace=False):
        v = P.entry(wl.X, wl.E, wl.nu, mask, rows[k], P.col[k], eps=1e-3)
        assert v == val[k] or (np.isnan(v) and np.isnan(val[k]))


# ---------------------------------------------------------------- streaming


def _stream_check(orc, wl, eps=0.0, check_additive=True):
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    assert bad == 0
    P = orc.Pattern(wl.n_nodes, wl.tets)
    mask = wl.mask0.copy()
    val = P.rebuild(Ke, mask, eps)
    mask_a = mask.copy()
    val_a = val.copy()
    act0 = np.flatnonzero(mask)
    hist = np.zeros(P.nnz)       # sum of |contribution| ever added to or removed from an entry
    np.add.at(hist, P.scat[act0].reshape(-1), np.abs(Ke[act0]).reshape(-1))
    worst = 0.0
    for f, ed in enumerate(wl.frames):
        touched = P.local_recompute(Ke, mask, ed, val, eps)
        ref_mask = W.apply_edits_to_mask(mask_a, ed)
        ref = P.rebuild(Ke, ref_mask, eps)
        assert np.array_equal(mask, ref_mask)
        assert np.array_equal(val.view(np.uint64), ref.view(np.uint64)), f"frame {f}"
        edited = np.concatenate([ed[:, 1], ed[ed[:, 0] == 2, 2]])
        uniq = np.unique(P.scat[edited].reshape(-1))
        assert touched == uniq.size
        if check_additive:
            P.additive_update(Ke, mask_a, ed, val_a)
            np.add.at(hist, P.scat[edited].reshape(-1), np.abs(Ke[edited]).reshape(-1))
            err = np.abs(val_a - ref)
            scale = np.where(hist > 0, hist, 1.0)
            worst = max(worst, float(np.max(err / scale)))
        else:
            mask_a = ref_mask
    return worst


def test_local_recompute_equals_rebuild_every_frame(orc):
    """Sec. 3.3 invariant, bitwise, for the rescan policy over whole edit streams."""
    for seed in range(3):
        worst = _stream_check(orc, W.plain_small(seed=seed))
        # additive (paper streaming_update) only up to rounding (cf. 8.3e-17 in Sec. 6.1)
        assert worst <= 1e-13
    _stream_check(orc, W.plain_small(seed=9), eps=1e-2)
    _stream_check(orc, W.prefractured_block(N=8, sites=6, frames=6))
    _stream_check(orc, W.refinement_hierarchy(N=5, radius=0.3, frames=6))
    for wl in W.batched_instances(count=3, tmin=200, tmax=2000, frames=4):
        _stream_check(orc, wl)


def test_edit_validation(orc):
    T = 10
    mask = np.array([1, 1, 1, 1, 1, 0, 0, 0, 0, 0], np.uint8)
    ok = W.make_edits(off=[0, 1], on=[5], swaps=[(2, 6)])
    assert orc.validate_edits(T, mask, ok) == 0
    bad_cases = [
        W.make_edits(off=[5]),                 # deactivate inactive
        W.make_edits(on=[0]),                  # activate active
        W.make_edits(off=[0, 0]),              # twice
        W.make_edits(off=[0], swaps=[(1, 1)]),  # swap onto itself
        W.make_edits(off=[10]),                # out of range
        W.make_edits(swaps=[(5, 6)]),          # swap off an inactive
        np.array([[3, 0, -1]], np.int32),      # bad op
    ]
    for ed in bad_cases:
        assert orc.validate_edits(T, mask, ed) > 0
    # a rejected call changes nothing
    X, tets, _ = W.kuhn_cube(1, 0.1, np.random.default_rng(0))
    Ke, _ = orc.element_all(X, tets, np.full(6, 1e5), np.full(6, 0.3))
    P = orc.Pattern(X.shape[0], tets)
    m = np.ones(6, np.uint8)
    v = P.rebuild(Ke, m)
    v0, m0 = v.copy(), m.copy()
    with pytest.raises(ValueError):
        P.local_recompute(Ke, m, W.make_edits(off=[1, 1]), v)
    assert np.array_equal(v, v0) and np.array_equal(m, m0)


# ---------------------------------------------------------------- gradients


def test_element_param_grad_vs_fd_and_linearity(orc):
    rng = np.random.default_rng(11)
    for _ in range(20):
        x = _random_tet(rng)
        E, nu = rng.uniform(1e3, 1e6), rng.uniform(0.05, 0.45)
        G = rng.standard_normal((12, 12))
        dE, dnu = orc.element_param_grad(x, E, nu, G)
        K = orc.element(x, E, nu)
        # K is linear in E: dL/dE = (G : K) / E
        ref = np.sum(G * K) / E
        assert abs(dE - ref) <= 1e-12 * np.sum(np.abs(G * K)) / E
        h = 1e-6 * nu
        fd = (np.sum(G * orc.element(x, E, nu + h)) - np.sum(G * orc.element(x, E, nu - h))) / (2 * h)
        assert abs(dnu - fd) <= 1e-6 * np.sum(np.abs(G * K)) / nu


def test_element_x_grad_complex_step_vs_fd(orc):
    rng = np.random.default_rng(12)
    for _ in range(20):
        x = _random_tet(rng)
        E, nu = rng.uniform(1e3, 1e6), rng.uniform(0.05, 0.45)
        G = rng.standard_normal((12, 12))
        dx = orc.element_x_grad_cs(x, E, nu, G)
        # translation invariance: gradients sum to zero over the four nodes
        assert np.abs(dx.sum(0)).max() <= 1e-10 * np.abs(dx).max()
        # rotation invariance of the contraction with a rotated G is not assumed; use FD
        L = np.abs(x).max()
        for m in range(12):
            h = 1e-6 * L
            xp, xm = x.copy().reshape(12), x.copy().reshape(12)
            xp[m] += h
            xm[m] -= h
            fd = (np.sum(G * orc.element(xp.reshape(4, 3), E, nu)) -
                  np.sum(G * orc.element(xm.reshape(4, 3), E, nu))) / (2 * h)
            scale = np.sum(np.abs(G * orc.element(x, E, nu))) / L
            assert abs(dx.reshape(12)[m] - fd) <= 1e-6 * scale


def test_compliance_gradient_vs_central_fd(orc):
    """Whole chain: assembly -> direct solve -> L = f^T u, gradients by the adjoint rule
    dL/dK_ij = -u_i u_j gathered per element, against central differences of L."""
    wl = W.adjoint_block(N=3, frames=4)
    mask = wl.masks()[2]
    f = wl.meta["load"]
    free = W.free_dofs(wl.tets, mask, wl.meta["clamped_nodes"])
    P = orc.Pattern(wl.n_nodes, wl.tets)

    def loss(X, E, nu):
        Ke, bad = orc.element_all(X, wl.tets, E, nu)
        assert bad == 0
        K = P.csr(P.rebuild(Ke, mask))
        u = orc.solve_free(K, f, free)
        return float(f @ u), u

    L0, u = loss(wl.X, wl.E, wl.nu)
    gv = orc.compliance_grad_val(P, u, free)
    dE, dnu, dX = P.grad_all(wl.X, wl.E, wl.nu, mask, gv)
    assert np.all(dE[mask == 0] == 0)
    rng = np.random.default_rng(5)
    act = np.flatnonzero(mask)
    # per-element E and nu
    for e in rng.choice(act, 5, replace=False):
        h = 1e-6 * wl.E[e]
        Ep, Em = wl.E.copy(), wl.E.copy()
        Ep[e] += h
        Em[e] -= h
        fd = (loss(wl.X, Ep, wl.nu)[0] - loss(wl.X, Em, wl.nu)[0]) / (2 * h)
        assert abs(dE[e] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(L0) / wl.E[e]
        h = 1e-6 * wl.nu[e]
        np_, nm = wl.nu.copy(), wl.nu.copy()
        np_[e] += h
        nm[e] -= h
        fd = (loss(wl.X, wl.E, np_)[0] - loss(wl.X, wl.E, nm)[0]) / (2 * h)
        assert abs(dnu[e] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(L0)
    # directional derivative in X
    Dx = rng.standard_normal(wl.X.shape)
    h = 1e-6
    fd = (loss(wl.X + h * Dx, wl.E, wl.nu)[0] - loss(wl.X - h * Dx, wl.E, wl.nu)[0]) / (2 * h)
    assert abs(np.sum(dX * Dx) - fd) <= 1e-6 * abs(fd)


# -------------------------------------------------------------------------------------------
# Exact additive streaming in fixed point (orc_fx_*): the paper's streaming_update (Sec. 3.4,
# Sec. 3.5) with integer sums, so that adding and subtracting element contributions in any
# order equals a rebuild bit for bit.
# -------------------------------------------------------------------------------------------

def _fx_stream(orc, wl, eps=0.0):
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    assert bad == 0
    e = P.fx_exponents(Ke)
    mask = wl.mask0.copy()
    S, val = P.fx_rebuild(Ke, e, mask, eps)
    for ed in wl.frames:
        P.fx_update(Ke, e, mask, ed, S, val, eps)
        S_r, val_r = P.fx_rebuild(Ke, e, mask, eps)
        assert np.array_equal(S, S_r)
        assert np.array_equal(val.view(np.uint64), val_r.view(np.uint64))
    return P, Ke, e, mask, S, val


def test_fx_additive_stream_equals_fx_rebuild_every_frame(orc):
    _fx_stream(orc, W.plain_small(seed=2))
    _fx_stream(orc, W.plain_small(seed=3), eps=1e-3)
    _fx_stream(orc, W.prefractured_block(N=8, sites=6, frames=6))
    _fx_stream(orc, W.refinement_hierarchy(N=5, radius=0.3, frames=6))


def test_fx_within_its_error_bound_of_the_fp64_fold(orc):
    # |val_fx - val_fold| <= kappa_k 2^(e_k - 1) + 2 ulp(val), and <= 1e-13 sum_k |c|
    P, Ke, e, mask, S, val = _fx_stream(orc, W.prefractured_block(N=8, sites=6, frames=4))
    fold = P.rebuild(Ke, mask)
    absum = P.rebuild(np.abs(Ke), mask)
    kappa = np.bincount(P.scat.reshape(-1), minlength=P.nnz)
    err = np.abs(val - fold)
    bound = kappa * np.ldexp(1.0, e - 1) + 2 * np.spacing(np.abs(fold)) + 2 * np.spacing(absum)
    assert np.all(err <= bound)
    assert np.all(err <= 1e-13 * absum + 1e-300)
    assert np.all(np.abs(S) < 2 ** 62)


def test_fx_exact_when_contributions_are_small_integers(orc):
    # integer element contributions (|c| <= 2^10, at most 2^6 per entry): the fold is exact in
    # FP64 and so must the fixed-point value be
    wl = W.plain_small(seed=4)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    rng = np.random.default_rng(5)
    A = rng.integers(-1024, 1025, size=(wl.n_tets, 12, 12)).astype(np.float64)
    Ke = (A + np.transpose(A, (0, 2, 1))).reshape(wl.n_tets, 144)
    e = P.fx_exponents(Ke)
    mask = wl.mask0.copy()
    S, val = P.fx_rebuild(Ke, e, mask)
    assert np.array_equal(val.view(np.uint64), P.rebuild(Ke, mask).view(np.uint64))
    for ed in wl.frames[:6]:
        P.fx_update(Ke, e, mask, ed, S, val)
    assert np.array_equal(val.view(np.uint64), P.rebuild(Ke, mask).view(np.uint64))


def test_fx_order_of_edits_does_not_matter(orc):
    wl = W.plain_small(seed=6)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, _ = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    e = P.fx_exponents(Ke)
    m1, m2 = wl.mask0.copy(), wl.mask0.copy()
    S1, v1 = P.fx_rebuild(Ke, e, m1)
    S2, v2 = S1.copy(), v1.copy()
    rng = np.random.default_rng(7)
    for ed in wl.frames[:8]:
        P.fx_update(Ke, e, m1, ed, S1, v1)
        for i in rng.permutation(ed.shape[0]):  # one edit per call, shuffled
            P.fx_update(Ke, e, m2, ed[i:i + 1], S2, v2)
    assert np.array_equal(S1, S2)
    assert np.array_equal(v1.view(np.uint64), v2.view(np.uint64))


# ---------------------------------------------------------------- graph-Laplacian proxy


def _proxy_dense(P, val):
    import scipy.sparse as sp
    ptr, col = P.proxy_pattern()
    return sp.csr_matrix((val, col, ptr), shape=(P.n, P.n)).toarray()


def _active_edges(tets, mask):
    """{(u, v): count} over the six edges of every active tetrahedron, both orientations."""
    cnt = {}
    for t in np.flatnonzero(mask):
        q = [int(v) for v in tets[t]]
        for a in range(4):
            for b in range(a + 1, 4):
                for e in ((q[a], q[b]), (q[b], q[a])):
                    cnt[e] = cnt.get(e, 0) + 1
    return cnt


def test_proxy_rebuild_vs_textbook_laplacian(orc):
    """Eqs. 1-4 against scipy's graph Laplacian of the active edge set (dense, small meshes),
    the multiplicities against a count by brute force, the pattern against the node pairs."""
    from scipy.sparse.csgraph import laplacian
    rng = np.random.default_rng(21)
    meshes = [(X.shape[0], tets) for X, tets in _tiny_meshes()]
    wl = W.plain_small(seed=3, N=3)
    meshes.append((wl.n_nodes, wl.tets))
    for n, tets in meshes:
        T = tets.shape[0]
        P = orc.Pattern(n, tets)
        ptr, col = P.proxy_pattern()
        pairs = {(int(a), int(b)) for t in tets for a in t for b in t}
        rows = np.repeat(np.arange(n), np.diff(ptr))
        assert {(int(r), int(c)) for r, c in zip(rows, col)} == pairs
        for mask in (np.ones(T, np.uint8), (rng.uniform(size=T) < 0.5).astype(np.uint8),
                     np.zeros(T, np.uint8)):
            for eps in (0.0, 1e-3, 0.75):
                mult, deg, val = P.proxy_rebuild(mask, eps)
                cnt = _active_edges(tets, mask)
                assert [cnt.get((int(r), int(c)), 0) if r != c else 0
                        for r, c in zip(rows, col)] == mult.tolist()
                adj = np.zeros((n, n))
                for (u, v) in cnt:
                    adj[u, v] = 1.0
                in_mesh = np.isin(np.arange(n), tets)   # a node of no tetrahedron: empty row
                ref = laplacian(adj) + np.diag(np.where(in_mesh, eps, 0.0))
                got = _proxy_dense(P, val)
                assert np.array_equal(got, ref)                       # bitwise
                assert np.array_equal(deg, adj.sum(axis=1).astype(np.int32))
                assert not np.any(np.signbit(val) & (val == 0))       # no -0.0


def test_proxy_invariants_rows_symmetry_components(orc):
    """L 1 = 0 exactly (row sums = eps), symmetry, and the multiplicity of eigenvalue eps
    equals the number of connected components of the active graph (isolated nodes too)."""
    from scipy.sparse.csgraph import connected_components
    import scipy.sparse as sp
    for seed in range(3):
        wl = W.plain_small(seed=seed, N=4, frames=6)
        P = orc.Pattern(wl.n_nodes, wl.tets)
        for mask in wl.masks()[::2]:
            _, _, val = P.proxy_rebuild(mask, 0.25)
            A = _proxy_dense(P, val)
            assert np.array_equal(A, A.T)
            assert np.all(A.sum(axis=1) == 0.25)
            off = (A != 0) & ~np.eye(wl.n_nodes, dtype=bool)
            ncomp, _ = connected_components(sp.csr_matrix(off.astype(float)), directed=False)
            w = np.linalg.eigvalsh(A - 0.25 * np.eye(wl.n_nodes))
            assert np.sum(np.abs(w) < 1e-9) == ncomp
            assert w[0] > -1e-9


def _proxy_stream(orc, wl, eps=0.0):
    P = orc.Pattern(wl.n_nodes, wl.tets)
    ptr, col = P.proxy_pattern()
    mask = wl.mask0.copy()
    mult, deg, val = P.proxy_rebuild(mask, eps)
    for f, ed in enumerate(wl.frames):
        visited = P.proxy_update(mask, ed, mult, deg, val, eps)
        ref_mask = W.apply_edits_to_mask(wl.masks()[f], ed)
        assert np.array_equal(mask, ref_mask)
        rm, rd, rv = P.proxy_rebuild(mask, eps)
        assert np.array_equal(mult, rm) and np.array_equal(deg, rd), f"frame {f}"
        assert np.array_equal(val.view(np.uint64), rv.view(np.uint64)), f"frame {f}"
        # visited entries: both entries of every edge and the diagonal of every node of an
        # edited tetrahedron, counted by a set
        edited = np.concatenate([ed[:, 1], ed[ed[:, 0] == 2, 2]])
        ents = {(int(a), int(b)) for t in edited for a in wl.tets[t] for b in wl.tets[t]}
        assert visited == len(ents)


def test_proxy_stream_equals_rebuild_every_frame(orc):
    """Sec. 3.3 invariant for the proxy's streaming rule (Sec. 3.2), bitwise, every frame."""
    for seed in range(3):
        _proxy_stream(orc, W.plain_small(seed=seed))
    _proxy_stream(orc, W.plain_small(seed=5), eps=1e-3)
    _proxy_stream(orc, W.prefractured_block(N=8, sites=6, frames=6), eps=0.5)
    _proxy_stream(orc, W.refinement_hierarchy(N=5, radius=0.3, frames=6))
    _proxy_stream(orc, W.edge_fan(seed=1, K=40, frames=6))


def test_slab_cycles_workload_is_a_valid_repeated_edit_stream(orc):
    """Sec. 6.5 workload: the same slab deleted and reinserted, the mask back at mask0 every
    two frames, the slab growing with its half-width."""
    sizes = []
    for hw in (0.01, 0.02, 0.04, 0.08):
        wl = W.slab_cycles(N=8, half_width=hw, frames=6)
        masks = wl.masks()
        for f, ed in enumerate(wl.frames):
            assert orc.validate_edits(wl.n_tets, masks[f], ed) == 0
        for f in range(0, len(masks), 2):
            assert (masks[f] == wl.mask0).all()
        assert set(wl.frames[0][:, 1]) == set(wl.frames[1][:, 1])
        sizes.append(wl.meta["slab_tets"])
    assert sizes == sorted(sizes) and sizes[0] > 0


# ---------------------------------------------------------------- implicit-Euler loop (Eq. 9)


def test_lumped_mass_vs_volumes(orc):
    """m_v = sum of rho V / 4 over the active tets at v: total = rho * active volume (numpy
    determinants, computed independently), node by node, the unit right tet exactly, and +0.0
    for nodes without an active tet."""
    rng = np.random.default_rng(31)
    wl = W.plain_small(seed=2, N=4, frames=4)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    for mask in wl.masks()[::2] + [np.zeros(wl.n_tets, np.uint8)]:
        rho = float(rng.uniform(1.0, 2000.0))
        m = P.lumped_mass(wl.X, rho, mask)
        act = np.flatnonzero(mask)
        x = wl.X[wl.tets[act]]
        vol = np.linalg.det(x[:, 1:] - x[:, :1]) / 6.0
        ref = np.zeros(wl.n_nodes)
        np.add.at(ref, wl.tets[act].reshape(-1), np.repeat(rho * vol / 4.0, 4))
        assert np.allclose(m, ref, rtol=1e-13, atol=0.0)
        assert abs(m.sum() - rho * vol.sum()) <= 1e-12 * max(1.0, rho * vol.sum())
        untouched = ~np.isin(np.arange(wl.n_nodes), wl.tets[act])
        assert np.all(m[untouched] == 0.0) and not np.any(np.signbit(m))
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [5, 5, 5]], float)
    P1 = orc.Pattern(5, np.array([[0, 1, 2, 3]], np.int32))
    assert P1.lumped_mass(X, 24.0, np.ones(1, np.uint8)).tolist() == [1.0, 1.0, 1.0, 1.0, 0.0]


def test_implicit_euler_step_closed_forms(orc):
    """Eq. 9 step: with K = 0 it is u + h v + h^2 f / m; for large h it tends to the static
    solve K_ff u = f_f; a single free node against numpy's dense solve; clamped DOFs stay 0
    and massless ones keep their displacement with zero velocity."""
    import scipy.sparse as sp
    wl = W.adjoint_block(N=4)
    n = wl.n_nodes
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    P = orc.Pattern(n, wl.tets)
    mask = wl.mask0.copy()
    K = P.csr(P.rebuild(Ke, mask))
    mass = P.lumped_mass(wl.X, 1000.0, mask)
    clamped = wl.meta["clamped_nodes"]
    rng = np.random.default_rng(5)
    u, v, f = (rng.standard_normal(3 * n) for _ in range(3))
    h = 1e-2
    free = orc.dyn_free(mass, clamped)
    u1, v1 = orc.implicit_euler_step(sp.csr_matrix(K.shape), mass, u, v, f, h, clamped)
    m3 = np.repeat(mass, 3)
    ref = u + h * v + h * h * f / np.where(m3 > 0, m3, 1.0)
    assert np.allclose(u1[free], ref[free], rtol=1e-13, atol=1e-15)
    assert np.all(u1[np.repeat(clamped, 3)] == 0.0) and np.all(v1[~free] == 0.0)
    assert np.allclose(v1[free], (u1[free] - u[free]) / h, rtol=1e-15)
    # static limit: (M / h^2 + K) u1 = M (u + h v) / h^2 + f -> K u = f as h grows
    f0 = wl.meta["load"]
    us = orc.solve_free(K, f0, free)
    ul, _ = orc.implicit_euler_step(K, mass, np.zeros(3 * n), np.zeros(3 * n), f0, 1e6, clamped)
    assert np.linalg.norm(ul - us) <= 1e-6 * np.linalg.norm(us)
    # at rest with no load it stays at rest
    z, zv = orc.implicit_euler_step(K, mass, np.zeros(3 * n), np.zeros(3 * n), np.zeros(3 * n),
                                    h, clamped)
    assert not np.any(z) and not np.any(zv)
    # one tet, three nodes clamped: a 3x3 system for the free node
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.2, 0.3, 1.1], [4, 4, 4]], float)
    tets = np.array([[0, 1, 2, 3]], np.int32)
    K1, _ = orc.element_all(X, tets, np.array([3e4]), np.array([0.3]))
    P1 = orc.Pattern(5, tets)
    Kc = P1.csr(P1.rebuild(K1, np.ones(1, np.uint8)))
    m1 = P1.lumped_mass(X, 500.0, np.ones(1, np.uint8))
    cl = np.array([1, 1, 1, 0, 0], bool)
    u0, v0, f1 = (rng.standard_normal(15) for _ in range(3))
    got, _ = orc.implicit_euler_step(Kc, m1, u0, v0, f1, 0.05, cl)
    A = m1[3] * np.eye(3) + 0.05 ** 2 * K1[0].reshape(12, 12)[9:, 9:]
    want = np.linalg.solve(A, m1[3] * (u0[9:12] + 0.05 * v0[9:12]) + 0.05 ** 2 * f1[9:12])
    assert np.allclose(got[9:12], want, rtol=1e-12)
    assert np.all(got[:9] == 0.0) and np.array_equal(got[12:], u0[12:])   # node 4: no mass


def test_slab_sequence_workloads_are_valid(orc):
    """Fracture deletes disjoint slabs one per frame; merge starts from all of them deleted
    and reinserts them; every frame is a valid edit list."""
    for merge in (False, True):
        wl = W.slab_sequence(N=8, half_width=0.02, frames=4, merge=merge)
        masks = wl.masks()
        for f, ed in enumerate(wl.frames):
            assert orc.validate_edits(wl.n_tets, masks[f], ed) == 0
            assert ed.shape[0] > 0 and np.all(ed[:, 0] == (1 if merge else 0))
        ids = np.concatenate([ed[:, 1] for ed in wl.frames])
        assert np.unique(ids).size == ids.size               # the slabs are disjoint
        assert np.all(masks[-1] == (1 if merge else np.isin(np.arange(wl.n_tets), ids, invert=True)))
