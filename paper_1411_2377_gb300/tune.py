"""Autotuned SpMV launch configurations, cached on disk.

The configuration of a matrix's products (threads per block; the variant:
register staging of the row loop, word or radix-2^29 column products; the
shared-memory carve-out) changes the time of y = A x, never its
value.  `autotune` times every configuration once per (GPU, precision,
mode, row-length histogram) through mp_csr_tune and stores the winner in a
JSON file, so that later matrices of the same shape class reuse it with
mp_csr_set_config instead of timing again.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import CSR

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "mpkrylov", "tune.json")


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def signature(A: CSR, mode: str) -> str:
    """Cache key of a matrix: GPU, precision, mode and row-length histogram
    (counts rounded to two significant digits)."""
    hist = [float(f"{c:.2g}") for c in A.row_hist]
    raw = json.dumps([_gpu_name(), A.prec, mode, hist])
    return hashlib.sha1(raw.encode()).hexdigest()[:16]


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune(A: CSR, modes=("ordered", "exact"), reps: int = 5, cache: str | None = DEFAULT_CACHE,
             retune: bool = False) -> dict:
    """Sets the fastest launch configuration of A for each mode.  Returns
    {mode: {"threads_per_block", "variant", "carveout", "ms" (None when cached),
    "cached"}}."""
    if A.prec > 1024:  # one fixed warp-per-row form at 2048-8192 bits: nothing to tune
        return {mode: {"threads_per_block": 128, "variant": -1, "carveout": -1, "ms": None,
                       "cached": False, "fixed": True} for mode in modes}
    store = _load(cache) if cache else {}
    out = {}
    for mode in modes:
        key = signature(A, mode)
        hit = store.get(key)
        if hit is not None and not retune:
            A.set_config(mode, hit["threads_per_block"], hit["variant"], hit.get("carveout", -1))
            out[mode] = dict(hit, ms=None, cached=True)
            continue
        res = A.tune(mode, reps)
        store[key] = {k: res[k] for k in ("threads_per_block", "variant", "carveout")}
        out[mode] = dict(res, cached=False)
    if cache:
        os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
        tmp = f"{cache}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return out
