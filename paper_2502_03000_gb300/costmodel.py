"""Learned ranking of candidate plans.

For an expression the planner can produce several candidate plans (exact
chain order, the paper's greedy chain rule, written order, no elementwise
fusion, the literal one-kernel-per-operator plan).  This module records
their run times, trains the library's cost network on the GPU (forward,
gradient and Adam kernels of libarma_gpu.so) to predict log run time from
the plan features, and ranks candidates with it.  The FLOP/byte roofline
estimate (arma_gpu_plan_heuristic_cost) is the fallback and the yardstick.
"""
from __future__ import annotations

import ctypes
import json
import math

import numpy as np

from . import (PLAN_CHAIN_GREEDY, PLAN_CHAIN_LEFT, PLAN_LITERAL, PLAN_NO_FUSE, N_FEATURES, ArmaError, Plan,
               _check, lib)

CANDIDATES = (("dp", 0), ("paper_greedy", PLAN_CHAIN_GREEDY), ("written_order", PLAN_CHAIN_LEFT),
              ("unfused", PLAN_NO_FUSE), ("literal", PLAN_LITERAL))
HIDDEN = 64


def candidate_plans(nodes, outputs, tier="native"):
    """Distinct candidate plans (duplicates by kernel sequence removed; the
    literal plan is always kept as the reference point)."""
    out, seen = [], set()
    for name, flags in CANDIDATES:
        p = Plan(nodes, outputs, tier=tier, flags=flags)
        key = json.dumps([(s["kernel"], s["note"]) for s in p.info["steps"]])
        if key in seen and name != "literal":
            continue
        seen.add(key)
        out.append((name, p))
    return out


def time_plan(plan, inputs, reps=3, device="cuda"):
    import torch
    outs = plan.alloc_outputs(device)
    plan(*inputs, outputs=outs)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        plan(*inputs, outputs=outs)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps * 1e-3


def collect(dags, device="cuda", reps=3, gen_seed=7):
    """Time every distinct candidate of every DAG.  dags: list of
    (nodes, outputs, dtype).  Returns a list of records."""
    import torch
    from synth.dags import input_shapes
    g = torch.Generator(device=device)
    g.manual_seed(gen_seed)
    recs = []
    for di, (nodes, outs, dt) in enumerate(dags):
        td = torch.float32 if dt == "f32" else torch.bfloat16
        ins = [(torch.rand((c, r), device=device, generator=g) * 2 - 1).to(td).t() for r, c in input_shapes(nodes)]
        for ci, (name, p) in enumerate(candidate_plans(nodes, outs)):
            t = time_plan(p, ins, reps, device)
            recs.append({"dag": di, "cand": name, "features": p.features(), "time": t,
                         "heuristic": p.heuristic_cost(), "kernels": len(p.info["steps"])})
            p._ws.clear()
        del ins
    return recs


class CostNet:
    """The cost network on the GPU; inputs are standardised features."""

    def __init__(self, features=N_FEATURES, hidden=HIDDEN, seed=0, device="cuda"):
        import torch
        self.F, self.H, self.device = features, hidden, device
        self.P = int(lib().arma_gpu_mlp_param_count(features, hidden))
        rng = np.random.default_rng(seed)
        w = []
        # He-style initialisation for ReLU layers
        w.append(rng.normal(0, math.sqrt(2.0 / features), hidden * features))
        w.append(np.zeros(hidden))
        w.append(rng.normal(0, math.sqrt(2.0 / hidden), hidden * hidden))
        w.append(np.zeros(hidden))
        w.append(rng.normal(0, math.sqrt(1.0 / hidden), hidden))
        w.append(np.zeros(1))
        self.params = torch.tensor(np.concatenate(w), dtype=torch.float32, device=device)
        self.mu = np.zeros(features)
        self.sd = np.ones(features)

    def _x(self, X):
        import torch
        Z = (np.asarray(X, dtype=np.float64) - self.mu) / self.sd
        return torch.tensor(Z, dtype=torch.float32, device=self.device).contiguous()

    def predict(self, X):
        import torch
        x = self._x(X)
        y = torch.empty(x.shape[0], dtype=torch.float32, device=self.device)
        st = torch.cuda.current_stream().cuda_stream
        _check(lib().arma_gpu_mlp_forward(ctypes.c_void_p(self.params.data_ptr()), self.F, self.H,
                                          ctypes.c_void_p(x.data_ptr()), x.shape[0], ctypes.c_void_p(y.data_ptr()),
                                          ctypes.c_void_p(st)), "arma_gpu_mlp_forward")
        return y.double().cpu().numpy()

    def fit(self, X, T, steps=2000, lr=3e-3):
        """Full-batch Adam on the mean squared error of log time."""
        import torch
        X = np.asarray(X, dtype=np.float64)
        self.mu = X.mean(axis=0)
        self.sd = X.std(axis=0) + 1e-6
        x = self._x(X)
        t = torch.tensor(np.asarray(T), dtype=torch.float32, device=self.device)
        n = x.shape[0]
        g = torch.zeros(self.P, dtype=torch.float32, device=self.device)
        m = torch.zeros_like(g)
        v = torch.zeros_like(g)
        y = torch.empty(n, dtype=torch.float32, device=self.device)
        ws = torch.empty(int(lib().arma_gpu_mlp_workspace(self.F, self.H, n)), dtype=torch.uint8, device=self.device)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        L = lib()
        losses = []
        for k in range(1, steps + 1):
            _check(L.arma_gpu_mlp_grad(ctypes.c_void_p(self.params.data_ptr()), self.F, self.H,
                                       ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()), n,
                                       ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(ws.data_ptr()), ws.numel(), st), "arma_gpu_mlp_grad")
            _check(L.arma_gpu_mlp_adam(ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                       ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()), self.P, k,
                                       lr, 0.9, 0.999, 1e-8, st), "arma_gpu_mlp_adam")
            if k % 200 == 0 or k == steps:
                losses.append(float(((y - t) ** 2).mean().item()))
        return losses


def choose(recs_by_dag, scores):
    """For each DAG the candidate with the smallest score."""
    return {d: min(rs, key=lambda r: scores[id(r)]) for d, rs in recs_by_dag.items()}


def evaluate(recs, net=None):
    """Geometric-mean time over DAGs of the network's pick, the heuristic's
    pick, the literal plan and the best candidate (regret = pick / best)."""
    by = {}
    for r in recs:
        by.setdefault(r["dag"], []).append(r)
    heur = choose(by, {id(r): r["heuristic"] for r in recs})
    res = {"dags": len(by)}
    picks = {"heuristic": heur,
             "literal": {d: next(r for r in rs if r["cand"] == "literal") for d, rs in by.items()},
             "best": {d: min(rs, key=lambda r: r["time"]) for d, rs in by.items()}}
    if net is not None:
        pred = net.predict([r["features"] for r in recs])
        picks["mlp"] = choose(by, {id(r): p for r, p in zip(recs, pred)})
    for name, pk in picks.items():
        lt = [math.log(pk[d]["time"]) for d in by]
        res[name + "_geomean_s"] = math.exp(sum(lt) / len(lt))
        res[name + "_regret"] = math.exp(sum(math.log(pk[d]["time"] / picks["best"][d]["time"]) for d in by) / len(by))
    return res


def make_dags(seed, count, lo=16, hi=8192, cap_flops=2e11, max_inputs_bytes=2e9, start=0):
    """`count` valid random DAGs (synth.dags), skipping those whose literal
    plan exceeds cap_flops or whose inputs exceed max_inputs_bytes; a DAG
    whose BF16 variant does not conform is drawn again in FP32."""
    from synth.dags import input_shapes, random_dag
    out, i = [], start
    while len(out) < count:
        nodes, outs, dt = random_dag(seed, i, lo, hi)
        i += 1
        try:
            p = Plan(nodes, outs, flags=PLAN_LITERAL)
        except ArmaError as e:
            if e.status != "dtype":
                continue
            nodes, outs, dt = random_dag(seed, i - 1, lo, hi, dtype="f32")
            try:
                p = Plan(nodes, outs, flags=PLAN_LITERAL)
            except ArmaError:
                continue
        es = 4 if dt == "f32" else 2
        if p.info["flops"] > cap_flops:
            continue
        if sum(r * c for r, c in input_shapes(nodes)) * es > max_inputs_bytes:
            continue
        out.append((nodes, outs, dt))
    return out


def split_train_test(recs, frac=0.8):
    dags = sorted({r["dag"] for r in recs})
    cut = dags[int(len(dags) * frac)] if dags else 0
    return [r for r in recs if r["dag"] < cut], [r for r in recs if r["dag"] >= cut]
