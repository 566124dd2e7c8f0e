"""Adjoint form: the CUDA adjoint kernel and the autograd chain against the oracle's reference
gradients (analytic dE/dnu, complex-step dX) and against central finite differences.

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


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_adjoint_kernel_vs_oracle(sta, orc):
    import torch
    wl = W.plain_small(seed=5)
    rng = np.random.default_rng(0)
    E = rng.uniform(5e4, 2e5, wl.n_tets)
    nu = rng.uniform(0.1, 0.45, wl.n_tets)
    mask = (rng.uniform(size=wl.n_tets) < 0.8).astype(np.uint8)
    asm = sta.Assembler(wl.X, wl.tets, E, nu)
    asm.full_rebuild(mask)
    P = orc.Pattern(wl.n_nodes, wl.tets)
    gv = rng.standard_normal(P.nnz)
    dE, dnu, dX = sta.sta_adjoint(asm.h, torch.as_tensor(gv, device="cuda"))
    oE, onu, oX = P.grad_all(wl.X, E, nu, mask, gv)
    assert np.all(dE.cpu().numpy()[mask == 0] == 0)
    assert _rel(dE.cpu().numpy(), oE) < 1e-11
    assert _rel(dnu.cpu().numpy(), onu) < 1e-11
    assert _rel(dX.cpu().numpy(), oX) < 1e-11
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
    # oracle: element matrices, rebuild, sparse direct solve, adjoint rule, reference grads
    P = orc.Pattern(wl.n_nodes, wl.tets)
    Ke, bad = orc.element_all(wl.X, wl.tets, wl.E, wl.nu)
    assert bad == 0
    K = P.csr(P.rebuild(Ke, mask))
    u_o = orc.solve_free(K, f_np, free_np)
    gv = orc.compliance_grad_val(P, u_o, free_np)
    oE, onu, oX = P.grad_all(wl.X, wl.E, wl.nu, mask, gv)
    yield {"wl": wl, "mask": mask, "loss": loss, "L": float(L.detach()), "g": g, "L_o": float(f_np @ u_o),
           "o": {"E": oE, "nu": onu, "X": oX}, "asm": asm}
    asm.close()


def test_chain_matches_oracle_gradient(chain):
    assert abs(chain["L"] - chain["L_o"]) <= 1e-9 * abs(chain["L_o"])
    for k in ("E", "nu", "X"):
        assert _rel(chain["g"][k], chain["o"][k]) < 1e-7, k
    assert np.all(chain["g"]["E"][chain["mask"] == 0] == 0)


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
