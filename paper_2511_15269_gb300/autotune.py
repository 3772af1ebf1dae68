"""Autotuner for batches of charge sets: leaf size and launch shapes.

For a list of point sets, builds the batch (one tree per set, merged) for
every candidate leaf size N_max (which also fixes the near-field tile shape,
targets per lane) and, on each, times one evaluation (CUDA events, best of
`reps` after a warm-up) for every combination of the launch options
(fmm_tree_set_option): stage order, M2M in one launch or per round,
symmetric or one-sided near field, cap on M2L blocks per SM.  Returns the
fastest.  Results are cached per GPU architecture, order, precision, theta
and batch shape in autotune_cache.json next to this file.
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


def build_batch(sets, p, leaf, s, theta, precision, workers=8):
    """One tree per set, built by `workers` host threads on their own CUDA
    streams (the builds overlap on the device), then merged into a batch."""
    import concurrent.futures as cf
    dev = torch.cuda.current_device()
    streams = [torch.cuda.Stream() for _ in range(workers)]
    torch.cuda.synchronize()

    def one(k):
        with torch.cuda.device(dev), torch.cuda.stream(streams[k % workers]):
            pos = torch.from_numpy(np.ascontiguousarray(sets[k], dtype=np.float64)).cuda(non_blocking=False)
            return fmm.fmm_build_tree(pos, p, leaf, s, theta, precision)

    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        trees = list(ex.map(one, range(len(sets))))
    torch.cuda.synchronize()
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


OPTION_GRID = {
    fmm.FMM_OPT_SCHEDULE: (1, 0, 3),
    fmm.FMM_OPT_M2M_ONE_LAUNCH: (1, 0),
    fmm.FMM_OPT_NEAR_SYMMETRIC: (1, 0),
    fmm.FMM_OPT_M2L_BLOCKS_PER_SM: (0, 2),
}


def option_combos():
    import itertools
    keys = list(OPTION_GRID)
    for vals in itertools.product(*(OPTION_GRID[k] for k in keys)):
        yield dict(zip(keys, vals))


def apply_options(tree, opts):
    for k, v in opts.items():
        fmm.fmm_tree_set_option(tree, k, v)


def tune(sets, charges, p, s=2, theta=0.6, precision=fmm.FMM_FP32C, candidates=(32, 64, 128, 256), reps=3,
         use_cache=True):
    """Leaf size and launch options of the fastest batched evaluation.
    Returns (leaf, {option: value}, {"leaf/opts": ms})."""
    key = "full|" + _key(sets, p, s, theta, precision)
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            cache = json.load(open(_CACHE))
        except ValueError:
            cache = {}
    if use_cache and key in cache:
        e = cache[key]
        return int(e["leaf"]), {int(k): int(v) for k, v in e["opts"].items()}, e["ms"]
    q = torch.from_numpy(np.ascontiguousarray(charges, dtype=np.float64)).cuda()
    table, best = {}, None
    for leaf in candidates:
        if leaf < (1 << s):
            continue
        batch = build_batch(sets, p, leaf, s, theta, precision)
        for opts in option_combos():
            apply_options(batch, opts)
            ms = time_eval(batch, q, reps)
            label = "%d/%s" % (leaf, ",".join("%d=%d" % kv for kv in sorted(opts.items())))
            table[label] = ms
            if best is None or ms < best[0]:
                best = (ms, leaf, dict(opts))
        fmm.fmm_tree_status(batch)
        batch.free()
    _, leaf, opts = best
    if use_cache:
        cache[key] = {"leaf": leaf, "opts": {str(k): v for k, v in opts.items()}, "ms": table}
        tmp = _CACHE + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, _CACHE)
    return leaf, opts, table


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
