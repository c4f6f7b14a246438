"""Schedule cache for the batched-patch executor.

``wc_patches_autotune`` (native) times every candidate schedule on the bound
state and keeps the fastest.  This module remembers the winner per GPU and
workload so later runs skip the search: the key is the GPU name plus a hash
of the patch-size histogram, phase count, flux, precision and the number of
schedule kinds the library tries.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

DEFAULT_PATH = os.path.join(os.path.expanduser("~"), ".cache", "wenoc_b300", "autotune.json")


def key(patches, precision, flux, nphase):
    hist = {}
    for e in patches.edges:
        hist[e] = hist.get(e, 0) + 1
    # "kinds": the schedule kinds the library tries (a cache written when it
    # tried fewer is not reused)
    blob = json.dumps({"hist": sorted(hist.items()), "precision": precision, "flux": flux,
                       "nphase": nphase, "kinds": 3}, sort_keys=True)
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return gpu + ":" + hashlib.sha256(blob.encode()).hexdigest()[:16]


def load(path=DEFAULT_PATH):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned_schedule(patches, cfl, precision, flux, nphase, steps=2, path=DEFAULT_PATH,
                   stream=None):
    """Applies the cached schedule for this GPU and workload, or autotunes
    (on a copy of the bound state) and caches the result."""
    k = key(patches, precision, flux, nphase)
    cache = load(path)
    if k in cache:
        s = cache[k]
        patches.set_schedule(s["block"], s["ctas_per_sm"], s["dynamic"])
        return dict(s, cached=True)
    best = patches.autotune(cfl, steps=steps, stream=stream)
    cache[k] = best
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return dict(best, cached=False)
