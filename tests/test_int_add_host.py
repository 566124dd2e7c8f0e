"""The fold's integer-pipe IEEE addition (csrc/softfloat.cuh), compiled for the host, gives
the same bits as the CPU's binary64 addition on random, near-cancelling, exact-tie, edge and
special operands (no GPU needed)."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_int_add_matches_host_ieee_addition(tmp_path):
    exe = tmp_path / "int_add_check"
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17",
                           f"-I{ROOT / 'paper_2605_11673_gb300' / 'csrc'}",
                           str(ROOT / "tests" / "native" / "int_add_check.cpp"), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
    cases, bad = map(int, r.stdout.split()[-2:])
    assert cases > 10_000_000 and bad == 0
