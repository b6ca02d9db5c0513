"""Learned ranking of candidate plans.

For one expression the library plans several candidates
(arma_gpu_plan_candidates: chain order, elementwise fusion, split-K and,
with ARMA_PLAN_TIER_CHOICE, every precision tier at least as accurate as the
one asked for).  This module records their run times on the GPU, trains the
library's cost network with the library's own forward, gradient and Adam
kernels, and hands the trained network to the library, whose planner then
ranks the candidates itself (ARMA_PLAN_COST_MLP).

The network predicts a correction to the FLOP/byte roofline estimate
(arma_gpu_plan_heuristic_cost): predicted seconds = estimate *
exp(network(standardised features)).  The estimate is also one of the
features, so an untrained network (output 0) ranks exactly like the
estimate.  The estimate remains the fallback (no model loaded) and the check
on the network's picks (the guard factor of arma_gpu_cost_model_load).

Weights, feature scaling and the timing records persist as JSON
(``CostNet.save`` / ``CostNet.load``, ``save_records`` / ``load_records``).
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np

from . import (PLAN_LITERAL, PLAN_TIER_CHOICE, PLAN_COST_MLP, N_FEATURES, ArmaError, Plan, _check, candidates,
               lib, load_cost_model)

HIDDEN = 64
HEURISTIC_FEATURE = 16      # ln(FLOP/byte estimate) among the plan features
# the network trained on GB300 timings (train_costnet.py), if present
DEFAULT_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "costnet_gb300.json")


def candidate_plans(nodes, outputs, tier="native", flags=PLAN_TIER_CHOICE):
    """The library's distinct candidates for an expression, as (index, Plan)
    in its enumeration order, and the literal plan last with index -1."""
    out = [(i, p) for i, p in enumerate(candidates(nodes, outputs, tier=tier, flags=flags))]
    out.append((-1, Plan(nodes, outputs, tier=tier, flags=PLAN_LITERAL)))
    return out


def time_plan(plan, inputs, device="cuda", target_s=1e-3, max_reps=50, outputs=None, slow_above=None):
    """Mean seconds per evaluation (CUDA events): one warm-up, one timed
    evaluation to size the repetition count, then enough repetitions for
    about target_s of GPU time (at least 3).  A candidate whose single timed
    evaluation exceeds `slow_above` seconds is clearly not the fastest: its
    single time is returned without repetitions."""
    import torch
    outs = outputs if outputs is not None else plan.alloc_outputs(device)
    plan(*inputs, outputs=outs)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    plan(*inputs, outputs=outs)
    e1.record(s)
    torch.cuda.synchronize()
    t1 = max(e0.elapsed_time(e1) * 1e-3, 1e-7)
    if slow_above is not None and t1 > slow_above:
        return t1
    reps = int(min(max_reps, max(3, target_s / t1)))
    e0.record(s)
    for _ in range(reps):
        plan(*inputs, outputs=outs)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps * 1e-3


def dag_inputs(nodes, dtype, g, device="cuda"):
    import torch
    from synth.dags import input_shapes
    td = torch.float32 if dtype == "f32" else torch.bfloat16
    return [(torch.rand((c, r), device=device, generator=g) * 2 - 1).to(td).t() for r, c in input_shapes(nodes)]


def collect(dags, device="cuda", gen_seed=7, flags=PLAN_TIER_CHOICE, target_s=1e-3, slow_factor=4.0):
    """Time every candidate (and the literal plan) of every DAG.  dags: list
    of (nodes, outputs, dtype).  All candidates of a DAG share its inputs and
    outputs; a candidate more than slow_factor times slower than the fastest
    one so far is timed once.  Returns a list of records."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(gen_seed)
    recs = []
    for di, (nodes, outs, dt) in enumerate(dags):
        ins = dag_inputs(nodes, dt, g, device)
        cands = candidate_plans(nodes, outs, flags=flags)
        out_bufs = cands[0][1].alloc_outputs(device)
        best = None
        for ci, p in cands:
            t = time_plan(p, ins, device, target_s=target_s, outputs=out_bufs,
                          slow_above=None if best is None else slow_factor * best)
            if ci >= 0:
                best = t if best is None else min(best, t)
            recs.append({"dag": di, "cand": ci, "features": p.features(), "time": t,
                         "heuristic": p.heuristic_cost(), "kernels": len(p.info["steps"])})
            p._ws.clear()
        del ins, out_bufs
    return recs


def save_records(recs, path):
    with open(path, "w") as f:
        json.dump(recs, f)


def load_records(path):
    with open(path) as f:
        return json.load(f)


class CostNet:
    """The cost network on the GPU; inputs are standardised features, the
    output a log-seconds correction to the FLOP/byte estimate."""

    def __init__(self, features=N_FEATURES, hidden=HIDDEN, seed=0, device="cuda"):
        import torch
        self.F, self.H, self.device = features, hidden, device
        self.P = int(lib().arma_gpu_mlp_param_count(features, hidden))
        rng = np.random.default_rng(seed)
        w = []
        # He-style initialisation for the ReLU layers; the output layer
        # starts at zero, so the untrained network reproduces the estimate
        w.append(rng.normal(0, math.sqrt(2.0 / features), hidden * features))
        w.append(np.zeros(hidden))
        w.append(rng.normal(0, math.sqrt(2.0 / hidden), hidden * hidden))
        w.append(np.zeros(hidden))
        w.append(np.zeros(hidden))
        w.append(np.zeros(1))
        self.params = torch.tensor(np.concatenate(w), dtype=torch.float32, device=device)
        self.mu = np.zeros(features)
        self.sd = np.ones(features)

    def _x(self, X):
        """Standardised features, in FP32 exactly as the library's planner
        forms them: (f - mean) / scale with FP32 operands."""
        import torch
        Z = (np.asarray(X, dtype=np.float32) - self.mu.astype(np.float32)) / self.sd.astype(np.float32)
        return torch.tensor(Z.astype(np.float32), dtype=torch.float32, device=self.device).contiguous()

    def correction(self, X):
        """network(standardised X): the predicted ln(time / estimate)."""
        import torch
        x = self._x(X)
        y = torch.empty(x.shape[0], dtype=torch.float32, device=self.device)
        st = torch.cuda.current_stream().cuda_stream
        _check(lib().arma_gpu_mlp_forward(ctypes.c_void_p(self.params.data_ptr()), self.F, self.H,
                                          ctypes.c_void_p(x.data_ptr()), x.shape[0], ctypes.c_void_p(y.data_ptr()),
                                          ctypes.c_void_p(st)), "arma_gpu_mlp_forward")
        return y.double().cpu().numpy()

    def predict_log_seconds(self, X):
        X = np.asarray(X, dtype=np.float64)
        return X[:, HEURISTIC_FEATURE] + self.correction(X)

    def fit(self, X, log_t, steps=2000, lr=3e-3, groups=None):
        """Full-batch Adam on the mean squared error of ln(time / estimate).
        With `groups` (the expression each record belongs to), the target is
        centred per expression: only differences between the candidates of
        one expression decide a pick, so an expression-wide offset is not
        learned."""
        import torch
        X = np.asarray(X, dtype=np.float64)
        target = np.asarray(log_t, dtype=np.float64) - X[:, HEURISTIC_FEATURE]
        if groups is not None:
            groups = np.asarray(groups)
            for gid in np.unique(groups):
                sel = groups == gid
                target[sel] -= target[sel].mean()
        self.mu = X.mean(axis=0)
        self.sd = X.std(axis=0)
        self.sd[self.sd < 1e-6] = 1.0
        x = self._x(X)
        t = torch.tensor(target, dtype=torch.float32, device=self.device)
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
            if k == 1:
                losses.append(float(((y - t) ** 2).mean().item()))
            _check(L.arma_gpu_mlp_adam(ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                       ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()), self.P, k,
                                       lr, 0.9, 0.999, 1e-8, st), "arma_gpu_mlp_adam")
            if k % 200 == 0 or k == steps:
                losses.append(float(((y - t) ** 2).mean().item()))
        return losses

    def host_params(self):
        return self.params.detach().float().cpu().numpy()

    def to_library(self, guard=0.0, margin=0.0):
        """Load this network into the library's planner (ARMA_PLAN_COST_MLP)."""
        load_cost_model(self.host_params(), self.mu, self.sd, self.H, guard, margin)

    def save(self, path):
        with open(path, "w") as f:
            json.dump({"features": self.F, "hidden": self.H, "params": self.host_params().tolist(),
                       "mean": [float(x) for x in self.mu], "scale": [float(x) for x in self.sd]}, f)

    @classmethod
    def load(cls, path, device="cuda"):
        import torch
        with open(path) as f:
            d = json.load(f)
        net = cls(d["features"], d["hidden"], device=device)
        net.params = torch.tensor(np.asarray(d["params"], dtype=np.float32), device=device)
        net.mu = np.asarray(d["mean"], dtype=np.float64)
        net.sd = np.asarray(d["scale"], dtype=np.float64)
        return net


def load_default(guard=4.0, margin=0.0, device="cuda"):
    """Load the shipped GB300 cost network into the library's planner
    (ARMA_PLAN_COST_MLP); returns it, or None when the file is absent."""
    if not os.path.exists(DEFAULT_MODEL):
        return None
    net = CostNet.load(DEFAULT_MODEL, device=device)
    net.to_library(guard=guard, margin=margin)
    return net


def by_dag(recs):
    by = {}
    for r in recs:
        by.setdefault(r["dag"], []).append(r)
    return by


def picks(recs, net=None, guard=0.0, margin=0.0):
    """Per DAG, the candidate the estimate picks and (with a network) the one
    the library's rule picks: the network's fastest candidate replaces the
    estimate's pick when the network predicts it at least `margin` faster and
    the estimate rates it at most `guard` times slower than its own pick.
    Only the library's candidates are eligible."""
    by = by_dag(recs)
    heur, mlp, guarded = {}, {}, 0
    pred = {}
    if net is not None:
        cand = [r for r in recs if r["cand"] >= 0]
        lp = net.predict_log_seconds([r["features"] for r in cand])
        pred = {id(r): v for r, v in zip(cand, lp)}
    for d, rs in by.items():
        cs = [r for r in rs if r["cand"] >= 0]
        h = min(cs, key=lambda r: (r["heuristic"], r["cand"]))
        heur[d] = h
        if net is not None:
            m = min(cs, key=lambda r: (pred[id(r)], r["cand"]))
            pick = h
            if m is not h and pred[id(m)] < math.log(1.0 - margin) + pred[id(h)]:
                if guard > 0 and m["heuristic"] > guard * h["heuristic"]:
                    guarded += 1
                else:
                    pick = m
            mlp[d] = pick
    return heur, mlp, guarded


def evaluate(recs, net=None, guard=0.0, margin=0.0):
    """Geometric-mean time over DAGs of the network's pick, the estimate's
    pick, the literal plan and the best candidate (regret = pick / best)."""
    by = by_dag(recs)
    heur, mlp, guarded = picks(recs, net, guard, margin)
    best = {d: min((r for r in rs if r["cand"] >= 0), key=lambda r: r["time"]) for d, rs in by.items()}
    sel = {"heuristic": heur, "best": best,
           "literal": {d: next(r for r in rs if r["cand"] == -1) for d, rs in by.items()}}
    if net is not None:
        sel["mlp"] = mlp
    res = {"dags": len(by)}
    for name, pk in sel.items():
        lt = [math.log(pk[d]["time"]) for d in by]
        res[name + "_geomean_s"] = math.exp(sum(lt) / len(lt))
        res[name + "_regret"] = math.exp(sum(math.log(pk[d]["time"] / best[d]["time"]) for d in by) / len(by))
    if net is not None:
        res["mlp_beats_heuristic_dags"] = sum(1 for d in by if mlp[d]["time"] < heur[d]["time"])
        res["heuristic_beats_mlp_dags"] = sum(1 for d in by if heur[d]["time"] < mlp[d]["time"])
        res["overrides"] = sum(1 for d in by if mlp[d] is not heur[d])
        res["guarded"] = guarded
    return res


def library_pick(nodes, outputs, flags=PLAN_TIER_CHOICE):
    """The candidate index the library's planner picks with ARMA_PLAN_COST_MLP
    (the loaded network, or the estimate when none is loaded)."""
    p = Plan(nodes, outputs, flags=flags | PLAN_COST_MLP)
    ch = p.info["choice"]
    return ch["picked"], ch["scorer"]


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
