"""Autotuner for the DWT / iDWT tile shapes.

For a plan, every tile-shape variant the library offers for its bandwidth and
mode (soft_plan_num_variants) is timed with the plan's own CUDA-event phase
timers on random data, and the fastest is selected (soft_plan_set_variant).
Results are cached in a JSON file keyed by (GPU name, B, mode): the path is
$SOFT_TUNE_CACHE, or ~/.cache/soft_gb300/tiles.json.
"""
from __future__ import annotations

import json
import os

import torch

from . import capi

KERNELS = {0: "dwt", 1: "idwt"}


def cache_path() -> str:
    return os.environ.get("SOFT_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "soft_gb300", "tiles.json"))


def _key(plan) -> str:
    return f"{torch.cuda.get_device_name(plan.device)}|B={plan.B}|{plan.dtype}"


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(cache: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_kernel(plan, kernel: int, reps: int) -> float:
    """Mean milliseconds of one DWT (kernel 0) or iDWT (kernel 1) launch."""
    gen = torch.Generator(device=plan.device).manual_seed(1808)
    if kernel == 0:
        x = torch.randn(plan.n ** 3, dtype=torch.complex128, device=plan.device, generator=gen).reshape((plan.n,) * 3)
        run = lambda: plan.forward(x)  # noqa: E731
    else:
        x = torch.randn(plan.ncoef, dtype=torch.complex128, device=plan.device, generator=gen)
        run = lambda: plan.inverse(x)  # noqa: E731
    run()
    plan.sync()
    capi.soft_plan_read_timing(plan.handle)
    capi.soft_plan_enable_timing(plan.handle, True)
    try:
        for _ in range(reps):
            run()
        ms, cnt = capi.soft_plan_read_timing(plan.handle)
    finally:
        capi.soft_plan_enable_timing(plan.handle, False)
    idx = 1 if kernel == 0 else 2
    return ms[idx] / max(1, cnt[idx])


def tune(plan, reps: int = 3, use_cache: bool = True, write_cache: bool = True) -> dict:
    """Select the fastest tile shape of each kernel for `plan`; returns
    {"dwt": variant, "idwt": variant, "ms": {...}}."""
    lib = capi.load()
    key = _key(plan)
    cache = _load_cache() if use_cache else {}
    if use_cache and key in cache:
        choice = cache[key]
        for k, name in KERNELS.items():
            capi.check(lib.soft_plan_set_variant(plan.handle, k, int(choice[name])), "soft_plan_set_variant")
        return choice
    choice = {"ms": {}}
    for k, name in KERNELS.items():
        nv = lib.soft_plan_num_variants(plan.handle, k)
        best, best_ms = 0, None
        for v in range(max(1, nv)):
            capi.check(lib.soft_plan_set_variant(plan.handle, k, v), "soft_plan_set_variant")
            t = _time_kernel(plan, k, reps)
            choice["ms"][f"{name}{v}"] = t
            if best_ms is None or t < best_ms:
                best, best_ms = v, t
        capi.check(lib.soft_plan_set_variant(plan.handle, k, best), "soft_plan_set_variant")
        choice[name] = best
    if write_cache:
        cache = _load_cache()
        cache[key] = choice
        _save_cache(cache)
    return choice
