"""Launch-shape autotuner for the fold kernels.

Sweeps the fold's CTA size (64, 128, 256 threads) and CTAs per SM (0 = occupancy maximum, or a
fixed count) on a given context, timing the full refold with CUDA events after an L2 flush,
and keeps the fastest shape in a JSON cache keyed by GPU name and the context's sizes.  The
shape changes only the schedule: values are identical for every shape.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

CACHE = Path(os.environ.get("STA_AUTOTUNE_CACHE",
                            Path(__file__).resolve().parent / "_build" / "autotune.json"))
SHAPES = [(t, b) for t in (64, 128, 256) for b in (0, 1, 2, 3, 4, 6, 8)]


def key_for(gpu_name: str, sizes: dict) -> str:
    return f"{gpu_name}|T={sizes['n_tets']}|blocks={sizes['n_blocks']}|nnz={sizes['nnz']}"


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


def measure(asm, shape, repeats: int = 11, flush_bytes: int = 256 << 20) -> float:
    import torch
    asm.set_launch(*shape)
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
    """Best (block_threads, blocks_per_sm) for this context; applied to it and cached."""
    import torch
    key = key_for(torch.cuda.get_device_name(), asm.sizes())
    cache = load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        shape = tuple(cache[key]["shape"])
    else:
        timings = {s: measure(asm, s, repeats) for s in (shapes or SHAPES)}
        shape = pick_best(timings)
        cache[key] = {"shape": list(shape), "ms": timings[shape],
                      "all": {f"{t}x{b}": ms for (t, b), ms in timings.items()}}
        save_cache(cache, path)
    asm.set_launch(*shape)
    return shape
