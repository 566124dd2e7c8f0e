"""Host logic of the autotuner: selection and cache round trip (no GPU)."""
from paper_2605_11673_gb300 import autotune as A


def test_pick_best_and_ties():
    t = {(A.FUSED, 128, 0, 4): 1.0, (A.FUSED, 64, 2, 6): 0.5, (A.ZERO_FILL, 64, 1, 4): 0.5,
         (A.FUSED, 256, 2, 6): 0.5}
    assert A.pick_best(t) == (A.FUSED, 64, 2, 6)  # first in SHAPES order among equal times
    assert A.pick_best({}) is None
    assert {f for f, _, _, _ in A.SHAPES} == {A.FUSED, A.ZERO_FILL}
    assert {d for _, _, _, d in A.SHAPES} == {4, 6}
    assert len(set(A.SHAPES)) == len(A.SHAPES)


def test_cache_roundtrip(tmp_path):
    p = tmp_path / "c.json"
    assert A.load_cache(p) == {}
    k = A.key_for("GPU", {"n_tets": 1, "n_blocks": 2, "nnz": 18}, 3)
    assert k != A.key_for("GPU", {"n_tets": 1, "n_blocks": 2, "nnz": 18}, 9)
    A.save_cache({k: {"shape": [2, 64, 3, 6]}}, p)
    assert A.load_cache(p)[k]["shape"] == [2, 64, 3, 6]
    p.write_text("not json")
    assert A.load_cache(p) == {}
