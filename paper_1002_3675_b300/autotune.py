"""Autotuner front end: launch shapes per level and size class, cached as JSON.

``tune(geom, levels, cache_path)`` looks every level of a geometry up in the cache by
its size class (volume and imager sizes); misses are measured on the device with
``cbct_autotune`` (CUDA events over a few launches of each candidate shape) and
stored.  Hits are applied with ``cbct_set_tuning``.  Launch shapes change no result
bit, so a cache made on one run can be used by any other.
"""
from __future__ import annotations

import json
import os

from . import cbct


def size_class(geom: cbct.Geometry, level: int) -> str:
    nx, ny, nz, nu, nv = cbct.cbct_level_dims(geom, level)
    return f"vol{nx}x{ny}x{nz}_det{len(geom.angles)}x{nv}x{nu}"


def load(path: str) -> dict:
    if path and os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def save(path: str, table: dict):
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(geom: cbct.Geometry, levels: int, cache_path: str | None = None, force: bool = False) -> dict:
    """Tune (or apply cached shapes for) levels 0..levels-1; returns {size_class: shape}."""
    table = load(cache_path) if cache_path else {}
    used, changed = {}, False
    for level in range(levels):
        key = size_class(geom, level)
        if key in table and not force:
            cbct.cbct_set_tuning(geom, level, table[key])
        else:
            table[key] = cbct.cbct_autotune(geom, level)
            changed = True
        used[key] = table[key]
    if cache_path and changed:
        save(cache_path, table)
    return used
