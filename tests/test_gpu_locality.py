"""Repeated edits of one slab (Sec. 6.4, 6.5 workloads): every policy and both operators
against the oracle, bit for bit on every frame, at the smallest and largest half-width."""
import pytest

import workloads as W
from tests.test_gpu_fixed import _run_fixed
from tests.test_gpu_parity import _run_stream
from tests.test_gpu_proxy import _run as _run_proxy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sta():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_11673_gb300 as P
    P.load_library()
    return P


@pytest.mark.parametrize("hw", [0.01, 0.08])
def test_slab_cycles_all_policies(sta, orc, hw):
    wl = W.slab_cycles(N=12, half_width=hw, frames=8)
    _run_stream(sta, orc, wl)
    _run_fixed(sta, orc, wl)
    _run_proxy(sta, orc, wl, eps=1e-3, graph=True)
