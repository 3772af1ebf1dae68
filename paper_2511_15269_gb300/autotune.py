"""Leaf-size autotuner for batches of charge sets.

For a list of point sets, builds the batch (one tree per set, merged) for
every candidate leaf size N_max and times one evaluation (CUDA events, best of
`reps` after a warm-up); returns the fastest.  The leaf size also fixes the
near-field tile shape (targets per lane).  Results are cached per GPU
architecture, order, precision, theta and batch shape in
autotune_cache.json next to this file.
"""
import json
import os

import numpy as np
import torch

from . import fmm

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def _key(sets, p, s, theta, precision):
    cap = torch.cuda.get_device_capability()
    sizes = sorted(len(pos) for pos in sets)
    return "sm_%d%d|p%d|s%d|theta%g|prec%d|sets%d|n%d|nmax%d" % (
        cap[0], cap[1], p, s, theta, precision, len(sets), sum(sizes), sizes[-1])


def build_batch(sets, p, leaf, s, theta, precision):
    trees = [fmm.fmm_build_tree(torch.from_numpy(pos).cuda(), p, leaf, s, theta, precision) for pos in sets]
    batch = fmm.fmm_tree_merge(trees)
    for t in trees:
        t.free()
    return batch


def time_eval(tree, q, reps=3):
    u = torch.empty_like(q)
    fmm.fmm_eval_potential(tree, q, out=u)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fmm.fmm_eval_potential(tree, q, out=u)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_leaf_size(sets, charges, p, s=2, theta=0.6, precision=fmm.FMM_FP32C,
                   candidates=(32, 64, 128, 256), reps=3, use_cache=True):
    """sets: list of (n_i x 3) float64 arrays; charges: concatenated float64.
    Returns (best leaf size, {leaf: ms})."""
    key = _key(sets, p, s, theta, precision)
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            cache = json.load(open(_CACHE))
        except ValueError:
            cache = {}
    if use_cache and key in cache:
        e = cache[key]
        return int(e["best"]), {int(k): v for k, v in e["ms"].items()}
    q = torch.from_numpy(np.ascontiguousarray(charges, dtype=np.float64)).cuda()
    ms = {}
    for leaf in candidates:
        if leaf < (1 << s):
            continue
        batch = build_batch(sets, p, leaf, s, theta, precision)
        ms[leaf] = time_eval(batch, q, reps)
        batch.free()
    best = min(ms, key=ms.get)
    if use_cache:
        cache[key] = {"best": best, "ms": ms}
        tmp = _CACHE + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, _CACHE)
    return best, ms
