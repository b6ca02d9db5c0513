"""Autotuner: tile shapes of batched evaluation, split counts of products.

``tune`` (batched): a batch of uneven problems can be tiled several ways:
128 x 128 tensor-core tiles, SIMT tiles of 64 x 64 or 32 x 32 for every
problem, or the per-problem padded-work rule.  Which is fastest depends on
the size mix, so the candidates are timed on the caller's own batch (CUDA
events, a few repetitions after a warm-up) and the fastest plan is kept.

``tune_plan`` (one expression): the K split count of its products (the CTAs
that share an output tile; ARMA_PLAN_SPLITS) is timed on the caller's own
operands over the library's model and 1, 2, 4, 8 and 15 splits, distinct
effective counts only, and the fastest plan is kept.

Results are cached by a signature (batched: element type, count and a
histogram of the problem sizes; one expression: its nodes, tier and flags),
so a family is tuned once per process; the table persists across processes
as JSON (``save`` / ``load``; with the environment variable
ARMA_AUTOTUNE_CACHE set to a file path, ``tune`` and ``tune_plan`` load it
before the first lookup and write it after every new result).
"""
from __future__ import annotations

import json
import math
import os

from . import PLAN_NO_TENSOR, PLAN_SPLITS, PLAN_TILE32, PLAN_TILE64, ArmaError, BatchedPlan, Plan

CANDIDATES = (("auto", 0), ("simt_rule", PLAN_NO_TENSOR), ("simt64", PLAN_NO_TENSOR | PLAN_TILE64),
              ("simt32", PLAN_NO_TENSOR | PLAN_TILE32))
SPLIT_CANDIDATES = tuple((f"splits{k}", k) for k in (0, 1, 2, 4, 8, 15))   # 0: the library's model

_cache: dict = {}
_loaded_from: set = set()


def _key(sig) -> str:
    return json.dumps(sig)


def save(path: str) -> None:
    """Write the tuning table (signature -> winning candidate) as JSON."""
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump({_key(k): v for k, v in _cache.items()}, f)
    os.replace(tmp, path)


def load(path: str) -> int:
    """Merge a saved tuning table; returns the number of entries read."""
    with open(path) as f:
        d = json.load(f)
    names = {n for n, _ in CANDIDATES} | {n for n, _ in SPLIT_CANDIDATES}
    for k, v in d.items():
        if v in names:
            _cache[_freeze(json.loads(k))] = v
    return len(d)


def _freeze(x):
    return tuple(_freeze(v) for v in x) if isinstance(x, list) else x


def _env_path():
    return os.environ.get("ARMA_AUTOTUNE_CACHE") or None


def signature(instances) -> tuple:
    """Element type, count and a log2 histogram of m, n, k: batches with the
    same signature share a tuning result."""
    hist = {}
    dtype = None
    for nodes, _ in instances:
        ins = [d for d in nodes if d["op"] == "input"]
        dtype = dtype or ins[0].get("dtype", "f64")
        a, b = ins[0], ins[1]
        key = (int(math.log2(max(1, a["cols"]))), int(math.log2(max(1, b["cols"]))),
               int(math.log2(max(1, a["rows"]))))
        hist[key] = hist.get(key, 0) + 1
    return (dtype, len(instances), tuple(sorted(hist.items())))


def _time(plan, reps, torch, call=None):
    call = call or plan
    s = torch.cuda.current_stream()
    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        call()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _load_env():
    path = _env_path()
    if path and path not in _loaded_from and os.path.exists(path):
        load(path)
        _loaded_from.add(path)
    return path


def plan_signature(nodes, outs, tier="native", flags=0) -> tuple:
    """One expression's tuning key: its nodes (shapes, types, leading
    dimensions), outputs, tier and flags."""
    return ("plan", json.dumps([nodes, outs], sort_keys=True), str(tier), int(flags))


def tune_plan(nodes, outs, inputs, outputs=None, device="cuda", reps=5, tier="native", flags=0):
    """Time the distinct split counts of the expression's products on these
    operands; returns (best Plan, {name: ms}).  ``flags`` must not already
    hold a split count."""
    import torch
    path = _load_env()
    sig = plan_signature(nodes, outs, tier, flags)
    known = sig in _cache
    results = {}
    best = None
    seen = set()
    for name, k in SPLIT_CANDIDATES:
        if known and name != _cache[sig]:
            continue
        try:
            p = Plan(nodes, outs, tier=tier, flags=flags | PLAN_SPLITS(k))
        except ArmaError:
            continue
        key = tuple(st.get("splits", 0) for st in p.info["steps"])
        if key in seen:
            continue
        seen.add(key)
        out = outputs if outputs is not None else p.alloc_outputs(torch.device(device))
        ms = _time(p, reps, torch, call=lambda: p(*inputs, outputs=out))
        results[name] = ms
        if best is None or ms < best[0]:
            best = (ms, name, p)
        p._ws.clear()
    _cache[sig] = best[1]
    if path and not known:
        save(path)
    return best[2], results


def tune(instances, inputs, outputs, device="cuda", reps=5, tier="native"):
    """Time every distinct candidate plan on this batch; returns
    (best BatchedPlan bound to inputs/outputs, {name: ms})."""
    import torch
    path = _load_env()
    sig = signature(instances)
    known = sig in _cache
    results = {}
    best = None
    seen = set()
    for name, flags in CANDIDATES:
        if sig in _cache and name != _cache[sig]:
            continue
        try:
            p = BatchedPlan(instances, tier=tier, flags=flags)
        except ArmaError:
            continue
        key = (p.info["steps"][0]["kernel"], p.info["tile"], p.info["tiles"])
        if key in seen:
            continue
        seen.add(key)
        p.bind(inputs, outputs, device)
        ms = _time(p, reps, torch)
        results[name] = ms
        if best is None or ms < best[0]:
            best = (ms, name, p)
    _cache[sig] = best[1]
    if path and not known:
        save(path)
    return best[2], results
