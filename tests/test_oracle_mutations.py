"""Mistakes planted in copies of the oracle must fail a pin.

Each mutation is a plausible slip -- a transposed operand, a dropped term, a wrong sign or
index, an ignored mask -- compiled on the CPU from a modified copy of the source; the oracle
wrapper is re-bound to it and the relevant pins of test_oracle_pins run and must fail."""
import subprocess
from pathlib import Path

import pytest

import oracle
import tests.test_oracle_pins as pins

ROOT = Path(__file__).resolve().parent.parent
SRC = ROOT / "oracle" / "sta_oracle.c"

MUTATIONS = {
    "transposed_operand": ("v = fma(P[a][i], g[b][j], Q[a][j] * g[b][i]);",
                           "v = fma(P[a][i], g[b][j], Q[a][i] * g[b][j]);",
                           [pins.test_element_reference_tet_closed_form,
                            pins.test_element_matches_literal_btdb]),
    "dropped_dot_term": ("v = fma(P[a][i], g[b][i], fma(Q[a][i], g[b][i], D[a][b]));",
                         "v = fma(P[a][i], g[b][i], Q[a][i] * g[b][i]);",
                         [pins.test_element_reference_tet_closed_form,
                          pins.test_element_symmetric_exactly_and_rigid_modes]),
    "g0_sign": ("for (int m = 0; m < 3; ++m) g[0][m] = -((g[1][m] + g[2][m]) + g[3][m]);",
                "for (int m = 0; m < 3; ++m) g[0][m] = ((g[1][m] + g[2][m]) + g[3][m]);",
                [pins.test_element_symmetric_exactly_and_rigid_modes]),
    "lame_lambda": ("double lam = (E * nu) / (onu * (1.0 - (nu + nu)));",
                    "double lam = (E * nu) / (onu * (1.0 - nu));",
                    [pins.test_element_reference_tet_closed_form,
                     pins.test_element_matches_literal_btdb]),
    "rebuild_ignores_mask": ("        if (!mask[t]) continue;\n        for (int pq = 0; pq < 144; ++pq) val[p->scat",
                             "        for (int pq = 0; pq < 144; ++pq) val[p->scat",
                             [pins.test_pattern_and_rebuild_vs_dense_bruteforce]),
    "recompute_wrong_local_index": ("            acc += Ke[144 * t + 12 * (3 * la + i) + 3 * lb + j];\n        }\n        if (r == c) acc += eps;\n        val[k] = acc;",
                                    "            acc += Ke[144 * t + 12 * (3 * lb + i) + 3 * la + j];\n        }\n        if (r == c) acc += eps;\n        val[k] = acc;",
                                    [pins.test_local_recompute_equals_rebuild_every_frame]),
    "dnu_sign": ("- sb * E / (2.0 * onu * onu));", "+ sb * E / (2.0 * onu * onu));",
                 [pins.test_element_param_grad_vs_fd_and_linearity]),
    "fx_removal_truncates": ("                S[k] += side == 0 ? -q : q;",
                             "                S[k] += side == 0 ? -(int64_t)trunc(ldexp(Ke[144 * (int64_t)t + pq], -e[k])) : q;",
                             [pins.test_fx_additive_stream_equals_fx_rebuild_every_frame]),
    "fx_exponent_too_coarse": ("        int ek = mk[k] + 1 + L - 62;", "        int ek = mk[k] + 1 + L - 40;",
                               [pins.test_fx_within_its_error_bound_of_the_fp64_fold,
                                pins.test_fx_exact_when_contributions_are_small_integers]),
    "proxy_threshold_dropped": ("            val[k] = a ? -1.0 : 0.0;",
                                "            val[k] = -(double)mult[k];",
                                [pins.test_proxy_rebuild_vs_textbook_laplacian]),
    "proxy_degree_counts_multiplicity": ("            deg[u] += a;", "            deg[u] += mult[k];",
                                         [pins.test_proxy_rebuild_vs_textbook_laplacian,
                                          pins.test_proxy_invariants_rows_symmetry_components]),
    "proxy_update_misses_removal": ("                    if ((before == 0) != (after == 0)) {",
                                    "                    if (before == 0 && after > 0) {",
                                    [pins.test_proxy_stream_equals_rebuild_every_frame]),
    "proxy_update_wrong_mirror": ("                        val[kvu] = val[kuv];",
                                  "                        val[kvu] = -1.0;",
                                  [pins.test_proxy_stream_equals_rebuild_every_frame]),
    "mass_half_not_quarter": ("            m += (rho * tet_volume(X, p->tets + 4 * t)) * 0.25;",
                              "            m += (rho * tet_volume(X, p->tets + 4 * t)) * 0.5;",
                              [pins.test_lumped_mass_vs_volumes]),
    "mass_volume_cross_sign": ("    double c1 = fma(d[1][2], d[2][0], -(d[1][0] * d[2][2]));",
                               "    double c1 = fma(d[1][0], d[2][2], -(d[1][2] * d[2][0]));",
                               [pins.test_lumped_mass_vs_volumes]),
    "proxy_step_sign": ("            int32_t step = side == 0 ? -1 : 1;",
                        "            int32_t step = side == 0 ? 1 : -1;",
                        [pins.test_proxy_stream_equals_rebuild_every_frame]),
    "proxy_eps_dropped": ("        if (kd >= 0) val[kd] = (double)deg[u] + eps;  /* a node of no tetrahedron has no row */",
                          "        if (kd >= 0) val[kd] = (double)deg[u];",
                          [pins.test_proxy_rebuild_vs_textbook_laplacian]),
    "mass_ignores_mask": ("            if (!mask[t]) continue;\n            m += (rho * tet_volume",
                          "            m += (rho * tet_volume",
                          [pins.test_lumped_mass_vs_volumes]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_oracle_mistake_fails_a_pin(name, tmp_path):
    old, new, checks = MUTATIONS[name]
    src = SRC.read_text()
    assert src.count(old) == 1, name
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(mut), "-lm"])
    try:
        oracle.use_library(so)
        failed = 0
        for check in checks:
            try:
                if "tmp_path" in check.__code__.co_varnames[:check.__code__.co_argcount]:
                    check(oracle, tmp_path)
                else:
                    check(oracle)
            except AssertionError:
                failed += 1
        assert failed > 0, f"mutation {name} passed every pin"
    finally:
        oracle.use_library(None)


# Mistakes planted in the oracle's Python steps: the function's source is edited, executed in
# the oracle module's namespace and swapped in for the duration of the pins.
PY_MUTATIONS = {
    "euler_drops_velocity": ("implicit_euler_step", "b = m3 * (u + h * v) + (h * h) * f",
                             "b = m3 * u + (h * h) * f",
                             [pins.test_implicit_euler_step_closed_forms]),
    "euler_h_not_h_squared": ("implicit_euler_step", "A = (sp.diags(m3) + (h * h) * K.tocsr())",
                              "A = (sp.diags(m3) + h * K.tocsr())",
                              [pins.test_implicit_euler_step_closed_forms]),
    "euler_velocity_sign": ("implicit_euler_step", "v1[idx] = (u1[idx] - u[idx]) / h",
                            "v1[idx] = (u[idx] - u1[idx]) / h",
                            [pins.test_implicit_euler_step_closed_forms]),
    "euler_clamped_keep_u": ("implicit_euler_step",
                             "u1 = np.where(np.repeat(np.asarray(clamped, bool), 3), 0.0, u)",
                             "u1 = np.asarray(u)",
                             [pins.test_implicit_euler_step_closed_forms]),
    "dyn_free_ignores_mass": ("dyn_free", "& (np.asarray(mass) > 0)", "",
                              [pins.test_implicit_euler_step_closed_forms]),
    "adjoint_rule_sign": ("compliance_grad_val", "g = -u[rows] * u[cols]", "g = u[rows] * u[cols]",
                          [pins.test_compliance_gradient_vs_central_fd]),
}


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_planted_python_oracle_mistake_fails_a_pin(name, monkeypatch):
    import inspect
    import textwrap
    fname, old, new, checks = PY_MUTATIONS[name]
    src = textwrap.dedent(inspect.getsource(getattr(oracle, fname)))
    assert src.count(old) == 1, name
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), ns)
    monkeypatch.setattr(oracle, fname, ns[fname])
    import warnings
    failed = 0
    for check in checks:
        try:
            with warnings.catch_warnings():  # a mutant may make the solve singular
                warnings.simplefilter("ignore")
                check(oracle)
        except (AssertionError, ValueError, RuntimeError):
            failed += 1
    assert failed > 0, f"mutation {name} passed every pin"
