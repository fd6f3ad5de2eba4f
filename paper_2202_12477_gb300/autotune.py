"""Persistent choice of the element-kernel variant per GPU, degree and precision.

The library's hb_autotune times every variant on a given mesh (C ABI). This
module keeps the winners in a JSON cache keyed by GPU name, SM count, degree
N and precision, so later meshes of the same kind reuse the choice without
re-timing. The cache file is HB_AUTOTUNE_CACHE if set, else
~/.cache/hipbone_gb300/autotune.json.
"""
from __future__ import annotations

import json
import os
import threading

from . import hb

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("HB_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "hipbone_gb300", "autotune.json")


def device_key(name: str, sms: int) -> str:
    return f"{name.strip()}|{sms}SM"


_PREC_NAME = {hb.HB_F64: "f64", hb.HB_F32: "f32", hb.HB_F64X: "f64x"}


def entry_key(N: int, prec: int, exclude: int = 0) -> str:
    return f"N{N}|{_PREC_NAME[prec]}" + (f"|x{exclude}" if exclude else "")


def load(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(cache: dict, dev: str, N: int, prec: int, exclude: int = 0):
    e = cache.get(dev, {}).get(entry_key(N, prec, exclude))
    valid = hb.VARIANTS_F64X if prec == hb.HB_F64X else (
        hb.VARIANTS + hb.VARIANTS_TC if prec == hb.HB_F64 and N == 7 else hb.VARIANTS)
    if isinstance(e, dict) and e.get("variant") in valid and not (e["variant"] & exclude):
        return e["variant"]
    return None


def record(cache: dict, dev: str, N: int, prec: int, variant: int, timings: dict, exclude: int = 0) -> dict:
    cache.setdefault(dev, {})[entry_key(N, prec, exclude)] = {
        "variant": int(variant), "ms": {str(k): float(v) for k, v in timings.items()}}
    return cache


def best_allowed(timings: dict, exclude: int) -> int | None:
    """Fastest timed variant with none of the `exclude` flag bits."""
    allowed = {v: ms for v, ms in timings.items() if not (int(v) & exclude)}
    return min(allowed, key=allowed.get) if allowed else None


def current_device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return device_key(p.name, p.multi_processor_count)


def tune_mesh(mesh, precs=(hb.HB_F64, hb.HB_F32), screen=hb.HB_SCREEN_IDENTITY, lam=0.1, reps=5,
              path: str | None = None, force: bool = False, exclude: int = 0) -> dict:
    """Sets the best variant on `mesh` for each precision, from the cache when
    present (unless force), else by timing and then recording it. `exclude`
    leaves out every variant with one of those flag bits, e.g.
    hb.HB_VARIANT_GRID for a choice that holds on any mesh (the lattice
    gather relies on the box's structure)."""
    dev = current_device_key()
    chosen = {}
    with _lock:
        cache = load(path)
        changed = False
        for prec in precs:
            if prec == hb.HB_F32 and not mesh.info.geo32:
                continue
            v = None if force else lookup(cache, dev, mesh.N, prec, exclude)
            if v is None:
                v, timings = hb.hb_autotune(mesh.handle, prec, screen, lam, reps)
                if exclude and v & exclude:
                    v = best_allowed(timings, exclude)
                    hb.hb_set_kernel_variant(mesh.handle, prec, v)
                record(cache, dev, mesh.N, prec, v, timings, exclude)
                changed = True
            else:
                hb.hb_set_kernel_variant(mesh.handle, prec, v)
            chosen[prec] = v
        if changed:
            store(cache, path)
    return chosen
