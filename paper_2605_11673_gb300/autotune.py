"""Launch autotuner for the full rebuild.

Sweeps the rebuild form (fused, or zero fill + fold of the flagged tiles; sta_set_rebuild_form),
the fold's CTA size (64, 128, 256 threads), CTAs per SM (0 = occupancy maximum, or a fixed
count) and the operand loads each lane keeps in flight (4 at 32 resident warps per SM, or 6 at
24; sta_set_fold_depth) on a given context, timing the full refold with CUDA events after an L2
flush, and keeps the fastest choice in a JSON cache keyed by GPU name, the context's sizes and
its active fraction (in tenths: the best form depends on how much of the superset is active).
The choice changes only the schedule: values are identical for every form and shape.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

CACHE = Path(os.environ.get("STA_AUTOTUNE_CACHE",
                            Path(__file__).resolve().parent / "_build" / "autotune.json"))
FUSED, ZERO_FILL = 1, 2  # sta.h STA_REBUILD_FUSED, STA_REBUILD_ZERO_FILL
# (rebuild form, threads per CTA, CTAs per SM, operand loads in flight)
SHAPES = [(f, t, b, d) for f in (FUSED, ZERO_FILL) for d in (4, 6) for t in (64, 128, 256)
          for b in (0, 1, 2, 3, 4, 6, 8)]


def key_for(gpu_name: str, sizes: dict, active_tenths: int = 10) -> str:
    return (f"{gpu_name}|T={sizes['n_tets']}|blocks={sizes['n_blocks']}|nnz={sizes['nnz']}"
            f"|active={active_tenths}/10")


def load_cache(path: Path = CACHE) -> dict:
    try:
        return json.loads(Path(path).read_text())
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: Path = CACHE) -> None:
    path = Path(path)
    path.parent.mkdir(parents=True, exist_ok=True)
    tmp = path.with_suffix(f".{os.getpid()}.tmp")
    tmp.write_text(json.dumps(cache, indent=1, sort_keys=True))
    os.replace(tmp, path)


def pick_best(timings: dict) -> tuple:
    """Shape with the smallest median time; ties go to the earlier shape in SHAPES order."""
    best = None
    for shape in SHAPES:
        if shape in timings and (best is None or timings[shape] < timings[best]):
            best = shape
    return best


def apply(asm, choice) -> None:
    form, threads, per_sm, depth = choice
    asm.set_rebuild_form(form)
    asm.set_launch(threads, per_sm)
    asm.set_fold_depth(depth)


def measure(asm, shape, repeats: int = 11, flush_bytes: int = 256 << 20) -> float:
    import torch
    apply(asm, shape)
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    times = []
    asm.refold()
    for _ in range(repeats):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        asm.refold()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def tune(asm, repeats: int = 11, use_cache: bool = True, path: Path = CACHE,
         shapes=None) -> tuple:
    """Best (form, block_threads, blocks_per_sm, operands in flight) for this context at its
    current mask; applied to it and cached."""
    import torch
    sizes = asm.sizes()
    tenths = int(10 * int(asm.mask().sum().item()) // max(1, sizes["n_tets"]))
    key = key_for(torch.cuda.get_device_name(), sizes, tenths)
    cache = load_cache(path) if use_cache else {}
    if use_cache and key in cache and len(cache[key].get("shape", ())) == len(SHAPES[0]):
        shape = tuple(cache[key]["shape"])
    else:
        timings = {s: measure(asm, s, repeats) for s in (shapes or SHAPES)}
        shape = pick_best(timings)
        cache[key] = {"shape": list(shape), "ms": timings[shape],
                      "all": {f"{f}:{t}x{b}:d{d}": ms for (f, t, b, d), ms in timings.items()}}
        save_cache(cache, path)
    apply(asm, shape)
    return shape
