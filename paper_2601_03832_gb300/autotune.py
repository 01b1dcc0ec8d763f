"""Project-written autotuner for the batched persistent launch.

The batched kernel runs one instance per thread block; the block size sets
how many lane groups share each factorisation and how many blocks fit on an
SM (shared memory and 2048 threads per SM).  `tune_batch` times the actual
batch on a short slice of its iterations (k_i capped) for each candidate
block size through the C ABI and keeps the fastest; results are cached in a
JSON file keyed by (GPU name and SM count, library build, dtype, contraction
mode, largest expanded bond, batch size), so later runs on the same device
and build reuse them.  Within a block, the lanes per task of each Householder
step are chosen on the device by a cost model of the step's rows and columns
(`pick_g` in the kernels), not here.
"""
from __future__ import annotations

import copy
import json
import os
import time

from . import binding

CACHE = os.environ.get("GMPS_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json"))
CANDIDATES = (64, 128, 256)


def _device_tag():
    """The GPU (name and SM count) and the library build the timings belong to."""
    import torch
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    try:
        st = os.stat(binding.LIB_PATH)
        build = f"{st.st_size}-{int(st.st_mtime)}"
    except (OSError, AttributeError):
        build = "unknown"
    return f"{props.name}|sm{props.multi_processor_count}|{build}"


def _key(insts, dtype, apply):
    xcap = 0
    for i in insts:
        chi = min(i.chi_max, i.M + 3)
        x = {"fused": chi + i.M + 1, "split": chi + i.M}.get(apply, (i.M + 1) * chi)
        xcap = max(xcap, x)
    return f"{_device_tag()}|{dtype}|{apply}|x{xcap}|b{len(insts)}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_batch(insts, dtype="c64", apply="fused", kslice=10, candidates=CANDIDATES, stream=None,
               use_cache=True):
    """Best block size for this batch (and the per-candidate seconds measured)."""
    key = _key(insts, dtype, apply)
    cache = _load()
    if use_cache and key in cache:
        return cache[key]["threads"], cache[key]
    sliced = []
    for i in insts:
        j = copy.copy(i)
        j.k = min(i.k, kslice)
        sliced.append(j)
    b = binding.GroverBatch(sliced, dtype=dtype, apply=apply, stream=stream)
    times = {}
    for t in candidates:
        b.set_threads(t)
        b.run(use_graph=False)          # warm-up (attributes, caches)
        b.result()
        t0 = time.perf_counter()
        b.run(use_graph=False)
        b.result()
        times[str(t)] = time.perf_counter() - t0
    b.close()
    best = int(min(times, key=times.get))
    rec = {"threads": best, "seconds": times, "kslice": kslice}
    cache[key] = rec
    try:
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return best, rec
