"""Autotuner for batched evaluation.

A batch of uneven problems can be tiled several ways: 128 x 128 tensor-core
tiles (BF16 operands), SIMT tiles of 64 x 64 or 32 x 32 for every problem, or
the per-problem padded-work rule.  Which is fastest depends on the size mix,
so the candidates are timed on the caller's own batch (CUDA events, a few
repetitions after a warm-up) and the fastest plan is kept.  Results are
cached by a signature of the batch (element type, count and a histogram of
the problem sizes), so a batch family is tuned once per process; the table
persists across processes as JSON (``save`` / ``load``; with the environment
variable ARMA_AUTOTUNE_CACHE set to a file path, ``tune`` loads it before the
first lookup and writes it after every new result).
"""
from __future__ import annotations

import json
import math
import os

from . import PLAN_NO_TENSOR, PLAN_TILE32, PLAN_TILE64, ArmaError, BatchedPlan

CANDIDATES = (("auto", 0), ("simt_rule", PLAN_NO_TENSOR), ("simt64", PLAN_NO_TENSOR | PLAN_TILE64),
              ("simt32", PLAN_NO_TENSOR | PLAN_TILE32))

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
    names = {n for n, _ in CANDIDATES}
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


def _time(plan, reps, torch):
    s = torch.cuda.current_stream()
    plan()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        plan()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(instances, inputs, outputs, device="cuda", reps=5, tier="native"):
    """Time every distinct candidate plan on this batch; returns
    (best BatchedPlan bound to inputs/outputs, {name: ms})."""
    import torch
    path = _env_path()
    if path and path not in _loaded_from and os.path.exists(path):
        load(path)
        _loaded_from.add(path)
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
