"""Seeded random expression DAGs for the cost-model workload.

Expressions of depth <= 5 over +, -, % (Schur), scalar *, trans, * (matrix
product), diagmat and trace, with dimensions drawn log-uniform in
[lo, hi].  Shapes are chosen first and operands generated to conform, so
every expression conforms in shape; element types may not (see the end
of ``random_dag``).  Uniforms come from the counter-based generator
in ``synth`` (stream 1000 + index), so DAG i is the same on every machine.
"""
from __future__ import annotations

import math

import numpy as np

from synth import raw_u64


class Draw:
    """Sequential uniforms from one counter stream."""

    def __init__(self, seed: int, stream: int, chunk: int = 256):
        self.seed, self.stream, self.pos, self.buf, self.chunk = seed, stream, 0, None, chunk
        self.i = chunk

    def u(self) -> float:
        if self.i >= self.chunk:
            z = raw_u64(self.seed, self.stream, self.pos, self.chunk)
            self.buf = (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
            self.pos += self.chunk
            self.i = 0
        v = float(self.buf[self.i])
        self.i += 1
        return v

    def logu(self, lo: int, hi: int) -> int:
        return int(min(hi, max(lo, round(math.exp(math.log(lo) + self.u() * (math.log(hi) - math.log(lo)))))))


def random_dag(seed: int, index: int, lo: int = 16, hi: int = 8192, max_depth: int = 5,
               dtype: str | None = None):
    """(nodes, outputs, dtype) of DAG `index`."""
    d = Draw(seed, 1000 + index)
    dt = dtype or ("f32" if d.u() < 0.5 else "bf16")
    nodes = []
    slots = [0]

    def add(nd):
        nodes.append(nd)
        return len(nodes) - 1

    def leaf(r, c):
        s = slots[0]
        slots[0] += 1
        return add({"op": "input", "slot": s, "rows": r, "cols": c, "dtype": dt, "ld": max(1, r)})

    def gen(r, c, depth):
        if depth == 0 or d.u() < 0.25:
            return leaf(r, c)
        x = d.u()
        if x < 0.30:
            op = ("add", "sub", "schur")[min(2, int(d.u() * 3))]
            a = gen(r, c, depth - 1)
            b = gen(r, c, depth - 1)
            return add({"op": op, "a": a, "b": b})
        if x < 0.40:
            a = gen(r, c, depth - 1)
            return add({"op": "scale", "a": a, "s": 0.5 + d.u()})
        if x < 0.55:
            a = gen(c, r, depth - 1)
            return add({"op": "trans", "a": a})
        if x < 0.85 or r != c:
            k = d.logu(lo, hi)
            a = gen(r, k, depth - 1)
            b = gen(k, c, depth - 1)
            return add({"op": "matmul", "a": a, "b": b})
        v = gen(r, 1, depth - 1)
        dm = add({"op": "diagmat", "a": v})
        b = gen(r, c, depth - 1)
        return add({"op": "matmul", "a": dm, "b": b})

    r = d.logu(lo, hi)
    c = r if d.u() < 0.3 else d.logu(lo, hi)
    e = gen(r, c, max_depth)
    if nodes[e]["op"] == "input":          # a bare input is not an expression
        e = add({"op": "scale", "a": e, "s": 2.0})
    if r == c and d.u() < 0.3:
        e = add({"op": "trace", "a": e})
    # products of BF16 operands return FP32, so an elementwise op that mixes
    # a product with a BF16 leaf does not conform: the caller draws such a
    # DAG again with dtype="f32"
    return nodes, [e], dt


def input_shapes(nodes):
    shapes = {}
    for nd in nodes:
        if nd["op"] == "input":
            shapes[nd["slot"]] = (nd["rows"], nd["cols"])
    return [shapes[s] for s in sorted(shapes)]
