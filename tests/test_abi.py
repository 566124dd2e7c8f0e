"""The C-ABI library builds, loads and exports every symbol include/sta.h declares; host-side
validation runs before any device work (no GPU needed)."""
import re
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(sta_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2605_11673_gb300 import build
    build.build()
    import paper_2605_11673_gb300 as P
    return P


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert "sta_create" in declared and "sta_apply_edits" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", str(lib.LIB_PATH)], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sta_[a-z0-9_]+)", out))
    assert declared <= exported, declared - exported
    assert set(lib.EXPORTED) == declared
    L = lib.load_library()
    for name in declared:
        assert hasattr(L, name)


def test_host_validation_before_device(lib):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    cases = [np.array([[0, 1, 2, 2]]), np.array([[0, 1, 2, 4]]), np.array([[-1, 1, 2, 3]])]
    for tets in cases:
        with pytest.raises(lib.StaError) as e:
            lib.sta_create(X, tets, [1.0], [0.3])
        assert e.value.status == lib.STA_EINVAL
    with pytest.raises(ValueError):
        lib.sta_create(X, np.array([[0, 1, 2, 3]]), [1.0, 2.0], [0.3])
    o = lib.sta_default_options()
    o.block_threads = 48
    with pytest.raises(lib.StaError) as e:
        lib.sta_create(X, np.array([[0, 1, 2, 3]]), [1.0], [0.3], o)
    assert e.value.status == lib.STA_EINVAL


def test_status_strings(lib):
    L = lib.load_library()
    for code in (0, -1, -2, -3, -4, -5):
        assert L.sta_status_string(code)


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2605_11673_gb300 as P
    saved = P._lib
    try:
        P._lib = None
        with pytest.raises(ImportError):
            P.load_library(tmp_path / "missing.so")
    finally:
        P._lib = saved


def test_oracle_and_product_share_no_code():
    """The CUDA sources never include or name the oracle, and the oracle never names the
    library; the only shared Python module is the input generator package."""
    csrc = ROOT / "paper_2605_11673_gb300"
    for f in list(csrc.rglob("*.cu")) + list(csrc.rglob("*.cuh")):
        assert "oracle" not in f.read_text().lower(), f
    for f in csrc.rglob("*.py"):
        text = f.read_text()
        assert "import oracle" not in text and "from oracle" not in text, f
    for f in (ROOT / "oracle").glob("*"):
        if f.is_file() and f.suffix in (".c", ".py", ".h"):
            text = f.read_text()
            assert "paper_2605_11673_gb300" not in text and "libsta" not in text


def test_entry_points_reject_null_context_and_bad_meshes_on_the_host(lib):
    """Every entry point checks its handle (and the proxy create its mesh) before any device
    work: these calls fail with STA_EINVAL on a machine without a GPU."""
    import ctypes as C
    L = lib.load_library()
    i32, f64 = C.c_int32(), C.c_double()
    p = C.c_void_p()
    calls = [
        L.sta_set_policy(None, 0, None), L.sta_set_params(None, None, None, None, 0, None),
        L.sta_proxy_state(None, C.byref(p), C.byref(p)),
        L.sta_dyn_setup(None, 1.0, 1.0, None, None, None),
        L.sta_dyn_step(None, 1e-8, 10, C.byref(i32), C.byref(f64), None),
        L.sta_dyn_apply(None, None, None, None), L.sta_dyn_state(None, C.byref(p), None, None),
        L.sta_dyn_set_state(None, None, None, 0, None),
        L.sta_solve(None, None, None, None, 1e-8, 10, None, None, None, None),
        L.sta_outer_grad(None, None, None, None, None, None),
        L.sta_apply_edits(None, None, 0, None), L.sta_full_rebuild(None, None, 0, None),
        L.sta_refold(None, None), L.sta_graph_enable(None, 1, None),
        L.sta_set_rebuild_form(None, 0), L.sta_get_rebuild_form(None, C.byref(i32)),
        L.sta_set_launch(None, 128, 0), L.sta_set_fold_depth(None, 4),
        L.sta_last_touched(None, None, None),
    ]
    assert all(r == lib.STA_EINVAL for r in calls), calls
    for tets in (np.array([[0, 1, 2, 2]]), np.array([[0, 1, 2, 9]]), np.array([[-1, 1, 2, 3]])):
        with pytest.raises(lib.StaError) as e:
            lib.sta_proxy_create(4, tets)
        assert e.value.status == lib.STA_EINVAL


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "sta.h"

int main(void) {
    sta_options o;
    sta_ctx *ctx = NULL;
    const double X[12] = {0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1};
    const int32_t bad[4] = {0, 1, 2, 2};
    const double E = 1.0, nu = 0.3;
    sta_default_options(&o);
    if (o.eps != 0.0 || o.block_threads != 0 || o.blocks_per_sm != 0) return 1;
    if (sta_create(X, 4, bad, 1, &E, &nu, &o, NULL, &ctx) != STA_EINVAL || ctx != NULL) return 2;
    if (strstr(sta_last_error(), "repeated node") == NULL) return 3;
    if (strcmp(sta_status_string(STA_OK), "ok") != 0) return 4;
    if (sta_destroy(NULL) != STA_OK) return 5;
    if (sta_apply_edits(NULL, NULL, 0, NULL) != STA_EINVAL) return 6;
    if (sta_set_rebuild_form(NULL, STA_REBUILD_ZERO_FILL) != STA_EINVAL) return 7;
    if (sta_set_fold_depth(NULL, 6) != STA_EINVAL) return 8;
    puts("ok");
    return 0;
}
"""


@pytest.mark.parametrize("compiler, std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_header_is_a_plain_c_boundary(lib, tmp_path, compiler, std):
    """include/sta.h compiles as strict C99 (and as C++ through its extern "C" guard), and a
    client with no Python and no torch links against libsta and calls it: host-side calls
    only, so no GPU is needed."""
    import shutil
    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not installed")
    src = tmp_path / ("client.c" if compiler == "gcc" else "client.cpp")
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = lib.LIB_PATH.parent
    subprocess.run([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror",
                    f"-I{ROOT / 'include'}", str(src), str(lib.LIB_PATH),
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


def test_binding_array_checks(lib):
    """The binding's checks of what it hands the library (raw pointers, no lengths): host arrays
    of the wrong length and tensors that are not CUDA tensors of the expected dtype and length
    are rejected before any call (no GPU needed)."""
    import torch
    with pytest.raises(ValueError):
        lib._host_n(np.zeros(5), np.float64, 6, "f")
    assert lib._host_n(np.zeros((2, 3)), np.float64, 6, "f").shape == (6,)
    with pytest.raises(TypeError):
        lib._dev(torch.zeros(6, dtype=torch.float64), 6, "x")  # a host tensor
    with pytest.raises(TypeError):
        lib._dev(np.zeros(6), 6, "x")
    with pytest.raises(TypeError):
        lib._dev_flags([1, 0, 1], 3, "free")


def test_size_limits_rejected_on_the_host(lib):
    """Sizes whose indices would overflow the int32 pattern or the 31-bit element-cache offsets
    are rejected with STA_ERANGE before any array is read or any device work (no GPU needed)."""
    import ctypes as C
    L = lib.load_library()
    x = np.zeros(12)
    t = np.array([0, 1, 2, 3], np.int32)
    one = np.ones(1)
    h = C.c_void_p()
    P = lambda a: a.ctypes.data  # noqa: E731
    # n_tets >= 2^27 (the arrays are never read: the size check comes first)
    assert L.sta_create(P(x), 4, P(t), 1 << 27, P(one), P(one), None, None,
                        C.byref(h)) == lib.STA_ERANGE
    assert h.value is None
    # element-cache offsets are 31-bit: 84 doubles per tetrahedron, so at most 25,565,281 tets
    assert L.sta_create(P(x), 4, P(t), 25_565_282, P(one), P(one), None, None,
                        C.byref(h)) == lib.STA_ERANGE
    # 3 n_nodes + 1 beyond int32 (no tetrahedra, so nothing is read)
    assert L.sta_create(P(x), (1 << 31) // 3 + 1, None, 0, None, None, None, None,
                        C.byref(h)) == lib.STA_ERANGE
    assert L.sta_proxy_create(1 << 27, P(t), 1 << 27, 0.0, None, C.byref(h)) == lib.STA_ERANGE
    assert L.sta_proxy_create((1 << 31) - 1, None, 0, 0.0, None, C.byref(h)) == lib.STA_ERANGE
    assert b"n_nodes" in L.sta_last_error()
    # negative sizes
    assert L.sta_create(P(x), -1, None, 0, None, None, None, None, C.byref(h)) == lib.STA_EINVAL
    assert L.sta_graph_enable(None, 0, None) == lib.STA_EINVAL
