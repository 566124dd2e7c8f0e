"""Adjoint form: the CUDA adjoint kernel and the autograd chain against the oracle's reference
gradients (analytic dE/dnu, complex-step dX) entry by entry, each against its own element's
magnitude, and against central finite differences (directional, and on single elements and
nodes).

Workload for the chain: 20^3 hexes x 6 = 48,000 tets, lognormal E, bottom layer clamped,
uniform downward traction on the top face, gradient of the compliance f^T u after frame 12
of a 2%-per-frame deactivation stream; DOFs not rigidly anchored are pinned.
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


def element_scales(orc, X, tets, E, nu, mask, gv, P):
    """Per-entry magnitudes for the adjoint comparisons, from the oracle's element matrices.
    With G the upstream gradient gathered on an element (G_pq = gv at the element's CSR entry
    (p, q)) and K = lambda A + mu B its matrix split into the lambda and mu parts:
      dE_e  = sum G K / E           scale sum |G| |K| / E
      dnu_e = sum G (lambda' A + mu' B)   scale sum |G| (|lambda'| |A| + |mu'| |B|)
      dX_v  = sum over the active elements at v of sum G dK/dx_v   scale sum |G| |K| / h_e
    (h_e = V_e^(1/3): dK/dx is K over a length).  A rounding error of the adjoint's arithmetic
    is a small multiple of these, whatever the cancellation inside an element; 0 on an
    inactive element."""
    Ke, bad = orc.element_all(X, tets, E, nu)
    assert bad == 0
    G = np.abs(gv[P.scat])                                   # (T, 144)
    act = mask.astype(bool)
    sK = (G * np.abs(Ke)).sum(1) * act
    B = orc.element_all(X, tets, np.full(len(E), 2.0), np.zeros(len(E)))[0]   # lambda 0, mu 1
    K1 = orc.element_all(X, tets, np.ones(len(E)), np.full(len(E), 0.25))[0]  # lambda = mu = 0.4
    A = (K1 - 0.4 * B) / 0.4
    dlam = E * (1 + 2 * nu ** 2) / ((1 + nu) ** 2 * (1 - 2 * nu) ** 2)
    dmu = -E / (2 * (1 + nu) ** 2)
    s_nu = (G * (np.abs(dlam)[:, None] * np.abs(A) + np.abs(dmu)[:, None] * np.abs(B))).sum(1) * act
    d = X[tets[:, 1:]] - X[tets[:, :1]]
    h = (np.abs(np.linalg.det(d)) / 6.0) ** (1.0 / 3.0)
    s_X = np.zeros(len(X))
    for a in range(4):
        np.add.at(s_X, tets[:, a], sK / h)
    return sK / E, s_nu, s_X


def assert_per_entry(got, ref, scale, tol, what):
    """|got - ref| <= tol (|ref| + scale) entry by entry (scale broadcast over columns)."""
    got, ref = np.asarray(got), np.asarray(ref)
    sc = scale if np.ndim(scale) == np.ndim(ref) else scale[:, None]
    lim = tol * (np.abs(ref) + sc)
    bad = np.argwhere(np.abs(got - ref) > lim)
    if bad.size:
        k = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} entries beyond {tol} x (|ref| + scale); first "
                             f"{k}: {got[k]!r} vs {ref[k]!r} (scale {np.broadcast_to(sc, ref.shape)[k]!r})")


def test_adjoint_kernel_vs_oracle(sta, orc):
    """The adjoint kernel against the oracle's gradients -- analytic dE and dnu, complex-step dX
    (an independent derivative, exact to rounding) -- entry by entry, each within 1e-12 of its
    own element's magnitude."""
    import torch
    wl = W.plain_small(seed=5)
    rng = np.random.default_rng(0)
    E = rng.uniform(5e4, 2e5, wl.n_tets)
    nu = rng.uniform(0.1, 0.45, wl.n_tets)
    mask = (rng.uniform(size=wl.n_tets) < 0.8).astype(np.uint8)
    asm = sta.Assembler(wl.X, wl.tets, E, nu)
    asm.full_rebuild(mask)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    # an upstream gradient spanning six orders of magnitude over the pattern
    gv = rng.standard_normal(P.nnz) * 10.0 ** rng.uniform(-3, 3, P.nnz)
    dE, dnu, dX = (a.cpu().numpy() for a in sta.sta_adjoint(asm.h, torch.as_tensor(gv, device="cuda")))
    oE, onu, oX = P.grad_all(wl.X, E, nu, mask, gv)
    sE, snu, sX = element_scales(orc, wl.X, wl.tets, E, nu, mask, gv, P)
    assert np.all(dE[mask == 0] == 0) and np.all(dnu[mask == 0] == 0)
    assert_per_entry(dE, oE, sE, 1e-12, "dE")
    assert_per_entry(dnu, onu, snu, 1e-12, "dnu")
    assert_per_entry(dX, oX, sX, 1e-12, "dX vs complex step")
    asm.close()


def test_spmv_vs_scipy(sta, orc):
    import torch
    wl = W.plain_small(seed=1)
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    asm.full_rebuild(wl.mask0)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, _ = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    K = P.csr(P.rebuild(Ke, wl.mask0))
    x = np.random.default_rng(2).standard_normal(P.nrows)
    y = sta.sta_spmv(asm.h, torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref = K @ x
    assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(K) @ np.abs(x))
    asm.close()


@pytest.fixture(scope="module")
def chain(sta, orc):
    """The adjoint workload at frame 12 on the GPU (autograd) and in the oracle."""
    import torch
    from paper_2605_11673_gb300.autograd import Assemble, Solve
    wl = W.adjoint_block()
    mask = wl.masks()[12]
    f_np = wl.meta["load"]
    free_np = W.free_dofs(wl.tets, mask, wl.meta["clamped_nodes"])
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    asm.full_rebuild(mask)
    dev = "cuda"
    f = torch.as_tensor(f_np, device=dev)
    free = torch.as_tensor(free_np, device=dev)

    def loss(E, nu, X, tol=1e-12):
        val = Assemble.apply(E, nu, X, asm)
        u = Solve.apply(val, f, asm, free, tol)
        return torch.dot(f, u)

    E = torch.as_tensor(wl.E, device=dev).requires_grad_()
    nu = torch.as_tensor(wl.nu, device=dev).requires_grad_()
    X = torch.as_tensor(wl.X, device=dev).requires_grad_()
    L = loss(E, nu, X)
    L.backward()
    g = {"E": E.grad.cpu().numpy(), "nu": nu.grad.cpu().numpy(), "X": X.grad.cpu().numpy()}
    # the same chain with the solves to 1e-14, for the per-entry checks
    E14, nu14, X14 = (t.detach().clone().requires_grad_() for t in (E, nu, X))
    loss(E14, nu14, X14, tol=1e-14).backward()
    g14 = {"E": E14.grad.cpu().numpy(), "nu": nu14.grad.cpu().numpy(), "X": X14.grad.cpu().numpy()}
    # oracle: element matrices, rebuild, sparse direct solve, adjoint rule, reference grads
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    assert bad == 0
    K = P.csr(P.rebuild(Ke, mask))
    u_o = orc.solve_free(K, f_np, free_np)
    gv = orc.compliance_grad_val(P, u_o, free_np)
    oE, onu, oX = P.grad_all(wl.X, wl.E, wl.nu, mask, gv)
    yield {"wl": wl, "mask": mask, "loss": loss, "L": float(L.detach()), "g": g, "g14": g14,
           "L_o": float(f_np @ u_o), "o": {"E": oE, "nu": onu, "X": oX}, "asm": asm, "gv_o": gv,
           "P": P}
    asm.close()


def test_chain_matches_oracle_gradient(chain, orc):
    """The whole GPU chain (assembly, CG to 1e-14, adjoint CG, adjoint kernel) against the
    oracle's (assembly, sparse direct solve, adjoint rule, reference gradients), entry by entry
    within 1e-7 of each element's own magnitude (the solves' difference, about 1e-9 relative to
    u, enters each element's gradient through its u values)."""
    assert abs(chain["L"] - chain["L_o"]) <= 1e-9 * abs(chain["L_o"])
    wl, mask = chain["wl"], chain["mask"]
    g = chain["g14"]
    sE, snu, sX = element_scales(orc, wl.X, wl.tets, wl.E, wl.nu, mask, chain["gv_o"], chain["P"])
    assert_per_entry(g["E"], chain["o"]["E"], sE, 1e-7, "dL/dE")
    assert_per_entry(g["nu"], chain["o"]["nu"], snu, 1e-7, "dL/dnu")
    assert_per_entry(g["X"], chain["o"]["X"], sX, 1e-7, "dL/dX")
    assert np.all(chain["g"]["E"][mask == 0] == 0)


def test_chain_per_element_central_differences(chain):
    """Central finite differences of the GPU chain's loss on single parameters: the 8 elements
    with the largest |dL/dE| and, for the 4 nodes with the largest |dL/dX|, their largest
    component; each within 1e-6 of the adjoint gradient.  Step: 1e-4 relative (a single element
    changes the compliance by about its share of the strain energy, so a smaller step would
    leave the difference at the solves' rounding; the truncation error at this step is about
    1e-8 relative)."""
    import torch
    wl, loss, g = chain["wl"], chain["loss"], chain["g14"]
    dev = "cuda"
    base = {"E": wl.E, "nu": wl.nu, "X": wl.X}
    picks = [("E", int(e), 1e-4 * wl.E[int(e)]) for e in np.argsort(-np.abs(g["E"]))[:8]]
    for v in np.argsort(-np.abs(g["X"]).max(1))[:4]:
        k = int(np.argmax(np.abs(g["X"][v])))
        picks.append(("X", (int(v), k), 1e-4 / wl.meta["N"]))
    for name, idx, h in picks:
        Lpm = []
        for sgn in (1.0, -1.0):
            args = {k2: torch.as_tensor(v2.copy(), device=dev) for k2, v2 in base.items()}
            args[name][idx] += sgn * h
            with torch.no_grad():
                Lpm.append(float(loss(args["E"], args["nu"], args["X"], tol=1e-14)))
        fd = (Lpm[0] - Lpm[1]) / (2 * h)
        an = float(g[name][idx])
        assert abs(an - fd) <= 1e-6 * abs(fd), (name, idx, an, fd)


def test_chain_vs_central_differences(chain):
    import torch
    wl = chain["wl"]
    loss = chain["loss"]
    rng = np.random.default_rng(7)
    dev = "cuda"
    base = {"E": wl.E, "nu": wl.nu, "X": wl.X}
    for name in ("E", "nu", "X"):
        d = rng.standard_normal(base[name].shape) * (np.abs(base[name]) if name != "X" else 1.0)
        if name == "X":
            d *= 1.0 / wl.meta["N"]
        h = 1e-6
        args_p = {k: torch.as_tensor(v, device=dev) for k, v in base.items()}
        args_m = {k: torch.as_tensor(v, device=dev) for k, v in base.items()}
        args_p[name] = torch.as_tensor(base[name] + h * d, device=dev)
        args_m[name] = torch.as_tensor(base[name] - h * d, device=dev)
        with torch.no_grad():
            Lp = float(loss(args_p["E"], args_p["nu"], args_p["X"], tol=1e-14))
            Lm = float(loss(args_m["E"], args_m["nu"], args_m["X"], tol=1e-14))
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(chain["g"][name] * d))
        assert abs(an - fd) <= 1e-6 * abs(fd), (name, an, fd)


def test_solve_and_outer_grad_vs_oracle(sta, orc):
    """sta_solve (the CG consumer) against the oracle's sparse direct solve on the free DOFs;
    sta_outer_grad against the adjoint rule written out in numpy."""
    import torch
    wl = W.adjoint_block(N=8)
    mask = wl.masks()[6]
    free_np = W.free_dofs(wl.tets, mask, wl.meta["clamped_nodes"])
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, _ = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    K = P.csr(P.rebuild(Ke, mask))
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    asm.full_rebuild(mask)
    f = torch.as_tensor(wl.meta["load"], device="cuda")
    free = torch.as_tensor(free_np, device="cuda")
    x, it, rel = sta.sta_solve(asm.h, f, free, tol=1e-12)
    ref = orc.solve_free(K, wl.meta["load"], free_np)
    xn = x.cpu().numpy()
    assert rel <= 1e-12 and it > 0
    assert np.linalg.norm(xn - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.all(xn[~free_np] == 0.0)
    # the same solve from a warm start takes fewer iterations; a zero right-hand side is 0
    _, it2, _ = sta.sta_solve(asm.h, f, free, tol=1e-12, x0=x)
    assert it2 < it
    z, it0, rel0 = sta.sta_solve(asm.h, torch.zeros_like(f), free)
    assert it0 == 0 and rel0 == 0.0 and not z.any()
    lam = torch.as_tensor(np.random.default_rng(2).standard_normal(3 * wl.n_nodes), device="cuda")
    g = sta.sta_outer_grad(asm.h, lam, x, free).cpu().numpy()
    rows = np.repeat(np.arange(P.nrows), np.diff(P.row_ptr))
    both = free_np[rows] & free_np[P.col]
    want = np.where(both, -lam.cpu().numpy()[rows] * xn[P.col], 0.0)
    assert np.array_equal(g, want)
    asm.close()


def test_binding_checks_array_sizes_before_the_library(sta, orc):
    """The library takes raw pointers; the binding rejects arrays of the wrong length or dtype
    before any call, and the context is unchanged afterwards."""
    import torch
    wl = W.plain_small(seed=6)
    asm = sta.Assembler(wl.X, wl.tets, wl.E, wl.nu)
    mask = wl.masks()[2]
    asm.full_rebuild(mask)
    n3, nnz = asm.n_rows, asm.nnz
    dev = lambda n, dt=torch.float64: torch.zeros(n, dtype=dt, device="cuda")  # noqa: E731
    free = torch.ones(n3, dtype=torch.bool, device="cuda")
    for call, err in (
            (lambda: sta.sta_spmv(asm.h, dev(n3 - 1)), ValueError),
            (lambda: sta.sta_spmv(asm.h, dev(n3, torch.float32)), TypeError),
            (lambda: sta.sta_spmv(asm.h, dev(n3).cpu()), TypeError),
            (lambda: sta.sta_spmv(asm.h, dev(n3), val=dev(nnz - 9)), ValueError),
            (lambda: sta.sta_solve(asm.h, dev(n3), free[:-3]), ValueError),
            (lambda: sta.sta_solve(asm.h, dev(n3), free, x0=dev(n3 + 3)), ValueError),
            (lambda: sta.sta_outer_grad(asm.h, dev(n3), dev(n3 - 3), free), ValueError),
            (lambda: sta.sta_adjoint(asm.h, dev(nnz + 1)), ValueError),
            (lambda: asm.full_rebuild(mask[:-1]), ValueError),
            (lambda: asm.full_rebuild(torch.as_tensor(mask[:-1], device="cuda")), ValueError),
            (lambda: asm.full_rebuild(torch.as_tensor(mask, device="cuda").float()), TypeError),
            (lambda: asm.set_params(E=wl.E[:-1]), ValueError),
            (lambda: asm.set_params(X=wl.X[:-1]), ValueError),
            (lambda: asm.dyn_setup(1.0, 1e-2, np.zeros(n3 - 3)), ValueError),
            (lambda: asm.dyn_setup(1.0, 1e-2, None, np.zeros(wl.n_nodes + 1)), ValueError)):
        with pytest.raises(err):
            call()
    # nothing reached the library: the values are still those of the mask
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, _ = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    ref = P.rebuild(Ke, mask)
    assert np.array_equal(asm.values().cpu().numpy().view(np.uint64), ref.view(np.uint64))
    asm.dyn_setup(1.0, 1e-2)
    with pytest.raises(ValueError):
        asm.dyn_apply(dev(n3 - 1))
    with pytest.raises(ValueError):
        asm.dyn_set_state(u=np.zeros(n3 + 3))
    asm.close()
