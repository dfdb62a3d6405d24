"""Autotuner for the launch shape of the persistent Newton kernel.

The Newton kernel runs one Gauss point per thread; its launch shape is the CTA
size (points per CTA) and the number of resident CTAs per SM.  Handles with
several trees (mixed depths) are tuned on their own batch and cached under a
key of their own.  The FP64 form is
bound by the FP64 pipe once each SM holds a few warps, the FP32 form hides
latency with more resident warps, and both trade occupancy against registers.
`tune` times every candidate shape on a caller-provided batch through the C ABI
(per-kernel CUDA events of the Newton kernel) and returns the fastest;
`tune_stage` does the same for the first stage's kernel, which has a launch
shape of its own.  Results are cached per (GPU, SM count, depth, shape
functions, phases, precision) in `_build/autotune.json` next to this file.
"""
from __future__ import annotations

import json
import os

from . import dmn

CANDIDATES = ((128, 2), (128, 3), (128, 4), (64, 4), (64, 6), (64, 8), (96, 4), (32, 12), (32, 16))
STAGE_CANDIDATES = (2, 3, 4, 6, 8)   # resident CTAs of 128 threads per SM of the first stage's kernel
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(tree, precision, device):
    """Cache key: GPU, SM count, and per tree its depth, shape functions and phase kinds (a handle
    with several trees, e.g. a batch of mixed depths, has a key of its own)."""
    import torch
    p = torch.cuda.get_device_properties(device)
    trees = list(tree) if isinstance(tree, (list, tuple)) else [tree]
    parts = ["K%d|M%d|ph%s" % (t.K, t.M, "".join(str(int(ph.kind)) for ph in t.phases)) for t in trees]
    return "%s|sm%d|%s|%s" % (p.name, p.multi_processor_count, "+".join(parts), precision)


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cached(tree, precision, device=None):
    """(block, ctas_per_sm) from the cache, or None."""
    import torch
    device = device or torch.device("cuda", torch.cuda.current_device())
    e = _load().get(_key(tree, precision, device))
    return (int(e["block"]), int(e["ctas_per_sm"])) if e else None


def tune(tree, precision, lam, Q, E_n, dE, state_in, reps=2, candidates=CANDIDATES, save=True, tree_id=None,
         first_stage=None):
    """Time the Newton kernel of every candidate shape on this batch; returns
    dict(block, ctas_per_sm, newton_ms, table).  tree may be a list of trees (one handle with
    several trees, as dmn.DMN takes it), with tree_id [n] (int32, device) selecting each
    point's tree.  first_stage as in dmn.DMN; with the first stage the time is that of the stage
    and the Newton kernel together (the stage keeps its own launch shape)."""
    import torch
    dev = lam.device
    n = lam.shape[0]
    table = []
    for block, cps in candidates:
        m = dmn.DMN(tree, precision=precision, block=block, ctas_per_sm=cps, first_stage=first_stage,
                    warp_per_point=-1)
        out = m.alloc_outputs(n, dev)
        m.update(lam, Q, E_n, dE, state_in, out=out, tree_id=tree_id)
        torch.cuda.synchronize()
        m.profile(True)
        for _ in range(reps):
            m.update(lam, Q, E_n, dE, state_in, out=out, tree_id=tree_id)
        kms, cnt = m.profile_read()
        m.profile(False)
        m.close()
        del out
        table.append((block, cps, kms["newton"] / cnt))
    torch.cuda.empty_cache()
    block, cps, ms = min(table, key=lambda r: r[2])
    res = dict(block=block, ctas_per_sm=cps, newton_ms=ms, points=n,
               table=[dict(block=b, ctas_per_sm=c, newton_ms=t) for b, c, t in table])
    if save:
        data = _load()
        data[_key(tree, precision, dev) + ("" if first_stage is None else "|stage%d" % int(bool(first_stage)))] = res
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, CACHE)
    return res


def tune_stage(tree, precision, lam, Q, E_n, dE, state_in, reps=1, candidates=STAGE_CANDIDATES, save=True,
               tree_id=None, block=0, ctas_per_sm=0):
    """Time the first stage's kernel at every candidate number of resident CTAs per SM on this batch
    (the Newton kernel at the given shape); returns dict(stage_ctas_per_sm, stage_ms, table).  The
    stage computes every point in one thread whatever the shape, so the results do not depend on it."""
    import torch
    dev = lam.device
    n = lam.shape[0]
    table = []
    for cps in candidates:
        m = dmn.DMN(tree, precision=precision, block=block, ctas_per_sm=ctas_per_sm, first_stage=True,
                    stage_ctas_per_sm=cps)
        out = m.alloc_outputs(n, dev)
        m.update(lam, Q, E_n, dE, state_in, out=out, tree_id=tree_id)
        torch.cuda.synchronize()
        m.profile(True)
        for _ in range(reps):
            m.update(lam, Q, E_n, dE, state_in, out=out, tree_id=tree_id)
        kms, _, cnt = m.profile_read_stages()
        m.profile(False)
        m.close()
        del out
        table.append((cps, kms["stage"] / cnt))
    torch.cuda.empty_cache()
    cps, ms = min(table, key=lambda r: r[1])
    res = dict(stage_ctas_per_sm=cps, stage_ms=ms, points=n,
               table=[dict(stage_ctas_per_sm=c, stage_ms=t) for c, t in table])
    if save:
        data = _load()
        data[_key(tree, precision, dev) + "|stage_shape"] = res
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, CACHE)
    return res
