"""Autotuner for the table kernel's launch shape.

Times candidate (threads per CTA, blocks per thread) pairs with CUDA events on
the launching stream and keeps the fastest.  Results are cached in a JSON file
keyed by (GPU name, key size, direction, size bucket) so a process pays the
search once per GPU model.  The tuner only chooses among shapes the kernels
were compiled for; it never changes what is computed (every shape is checked
bit-exact by the tests).
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np

from . import KERNEL_TABLE, BatchPlan, Key, ecb_ex, load, set_tuning

ECB_CANDIDATES = [(1024, 1), (1024, 2), (1024, 4), (768, 2), (768, 4), (512, 2), (512, 4)]
BATCH_CANDIDATES = [(1024, 2), (1024, 4), (1024, 1), (768, 2), (512, 4), (512, 8)]
_lock = threading.Lock()


def cache_path() -> str:
    base = os.environ.get("GBAES_TUNE_CACHE")
    if base:
        return base
    from . import _build

    return os.path.join(_build.OUT_DIR, "tune_cache.json")


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(c: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def size_bucket(nbytes: int) -> int:
    """log4 bucket of a buffer size (4 KiB -> 6, 1 MiB -> 10, 1 GiB -> 15)."""
    return int(np.floor(np.log(max(nbytes, 16)) / np.log(4)))


def _time(fn, reps: int, stream) -> float:
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_ecb(bits: int, decrypt: bool, nbytes: int = 256 << 20, reps: int = 10, force: bool = False,
             apply: bool = True) -> dict:
    """Best (threads, blocks_per_thread) of the table kernel for one key size and
    direction on a buffer of nbytes; installs it as the default launch shape."""
    import torch

    load()
    name = torch.cuda.get_device_name()
    key = f"ecb|{name}|{bits}|{int(bool(decrypt))}|{size_bucket(nbytes)}"
    with _lock:
        cache = _load_cache()
        hit = cache.get(key)
    if hit is None or force:
        k = Key(np.random.default_rng(bits).integers(0, 256, bits // 8, dtype=np.uint8).tobytes())
        x = torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device="cuda")
        y = torch.empty_like(x)
        stream = torch.cuda.current_stream()
        times = {}
        for threads, bpt in ECB_CANDIDATES:
            ms = _time(lambda: ecb_ex(k, x, y, decrypt=decrypt, kernel=KERNEL_TABLE, threads=threads,
                                      blocks_per_thread=bpt, stream=stream), reps, stream)
            times[f"{threads}x{bpt}"] = ms
        best = min(times, key=times.get)
        threads, bpt = (int(v) for v in best.split("x"))
        hit = {"threads": threads, "blocks_per_thread": bpt, "ms": times[best], "nbytes": nbytes,
               "gbs": nbytes / (times[best] / 1e3) / 1e9, "candidates_ms": times}
        with _lock:
            cache = _load_cache()
            cache[key] = hit
            _save_cache(cache)
    if apply:
        set_tuning(bits, decrypt, hit["threads"], hit["blocks_per_thread"])
    return hit


def tune_all_ecb(nbytes: int = 256 << 20, force: bool = False) -> dict:
    return {f"aes{b}_{'dec' if d else 'enc'}": tune_ecb(b, d, nbytes, force=force) for b in (128, 192, 256)
            for d in (False, True)}


def tune_batch(descs, keys, inp, out, reps: int = 3):
    """Builds a plan per candidate shape, times it, returns (best_plan, report)."""
    import torch

    stream = torch.cuda.current_stream()
    times, plans = {}, {}
    for threads, bpt in BATCH_CANDIDATES:
        p = BatchPlan(descs, keys, threads, bpt)
        times[f"{threads}x{bpt}"] = _time(lambda: p.launch(inp, out, stream=stream), reps, stream)
        plans[f"{threads}x{bpt}"] = p
    best = min(times, key=times.get)
    for k in list(plans):
        if k != best:
            del plans[k]
    return plans[best], {"best": best, "candidates_ms": times}
