"""Cached force-kernel tuning (JSON).

``tuned(sim, cache_path)`` applies the tile shape recorded for this GPU, N,
precision and mass type, or runs ``Simulation.autotune`` and records it.
The cache is a JSON object keyed by "<gpu name>|N=<N>|prec=<p>|eqmass=<0/1>".
"""
import json
import os

import numpy as np


def key(gpu_name, N, prec, equal_masses):
    return f"{gpu_name}|N={int(N)}|prec={int(prec)}|eqmass={int(bool(equal_masses))}"


def load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(path, cache):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned(sim, cache_path, masses, gpu_name, reps=3):
    """Apply (or measure and record) the fastest FP32 force shape for sim.
    Returns the record {"shape": s, "ms": [...]}."""
    m = np.asarray(masses, dtype=np.float32)
    k = key(gpu_name, sim.N, sim.prec, bool(m.size and np.all(m == m.flat[0])))
    cache = load(cache_path) if cache_path else {}
    if k in cache:
        sim.set_tuning(cache[k]["shape"])
        return cache[k]
    shape, ms = sim.autotune(reps)
    rec = {"shape": shape, "ms": ms}
    if cache_path:
        cache[k] = rec
        save(cache_path, cache)
    return rec
