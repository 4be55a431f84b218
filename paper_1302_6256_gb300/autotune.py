"""Cached autotuning of the solve's work split, task queue, heuristic extent
and graph replay.

``tuned(g, key)`` returns the options ``mc_autotune`` found fastest for a
workload, keeping results in a JSON file (``_build/autotune.json``) keyed by
the GPU's name and the workload key, so later runs skip the trials.
"""
from __future__ import annotations

import json
import os

from . import _build, mc_autotune

CACHE = os.path.join(_build.BUILD, "autotune.json")


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


# Version of the tuner's coordinate list: cached results from an older list
# are tuned again, so a coordinate added later is never hidden by the cache.
COORDS = "v3:warp_max,split,layout,no_bitmap,heuristic,graph"


def tuned(g, key: str, repeats: int = 2, cache: str = CACHE, **base):
    ck = "%s|%s|%s" % (COORDS, _gpu_name(), key)
    data = {}
    if os.path.exists(cache):
        try:
            data = json.load(open(cache))
        except Exception:
            data = {}
    if ck in data:
        return data[ck]["options"], data[ck]["ms"], True
    opts, ms = mc_autotune(g, repeats=repeats, **base)
    data[ck] = {"options": opts, "ms": ms}
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    with open(cache, "w") as f:
        json.dump(data, f, indent=1)
    return opts, ms, False
