"""Build expression descriptors with Armadillo-like operators.

    g = Graph()
    A = g.input(0, m, n); B = g.input(1, m, n)
    Z = 0.4 * A + 0.6 * B              # elementwise (Sec. II example)
    k = trace(A * B.t())                 # '*' (or '@') is the matrix product, '%' Schur
    nodes, outputs = g.build(Z, k)

The result is the plain node-dict list that ``Plan`` (and the tests'
oracle) consume.  Nothing is evaluated here: this is the delayed-evaluation
tree of Sec. II written down as data.
"""
from __future__ import annotations


class Graph:
    def __init__(self):
        self.nodes: list[dict] = []

    def _add(self, d: dict) -> "X":
        self.nodes.append(d)
        return X(self, len(self.nodes) - 1)

    def input(self, slot: int, rows: int, cols: int, dtype: str = "f64", ld: int | None = None) -> "X":
        return self._add({"op": "input", "slot": slot, "rows": rows, "cols": cols, "dtype": dtype,
                          "ld": ld if ld is not None else max(1, rows)})

    def build(self, *outs: "X"):
        return [dict(d) for d in self.nodes], [o.i for o in outs]

    def shape(self, i: int) -> tuple[int, int]:
        """(rows, cols) of node i."""
        d = self.nodes[i]
        op = d["op"]
        if op in ("input", "submat"):
            return d["rows"], d["cols"]
        if op == "trans":
            r, c = self.shape(d["a"])
            return c, r
        if op in ("matmul", "solve"):
            return self.shape(d["a"])[0], self.shape(d["b"])[1]
        if op == "diagmat":
            r, c = self.shape(d["a"])
            return (r * c, r * c) if r == 1 or c == 1 else (r, c)
        if op in ("trace", "accu", "norm_fro"):
            return 1, 1
        return self.shape(d["a"])


class X:
    __array_priority__ = 1000

    def __init__(self, g: Graph, i: int):
        self.g, self.i = g, i

    def _bin(self, op, other):
        return self.g._add({"op": op, "a": self.i, "b": other.i})

    def __add__(self, o):
        if isinstance(o, X):
            return self._bin("add", o)
        return self.g._add({"op": "add_scalar", "a": self.i, "s": float(o)})

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, X):
            return self._bin("sub", o)
        return self.g._add({"op": "add_scalar", "a": self.i, "s": -float(o)})

    def __rsub__(self, s):
        # s - X = (-X) + s
        return (-self) + float(s)

    def __neg__(self):
        return self.g._add({"op": "neg", "a": self.i})

    def __mul__(self, o):
        if isinstance(o, X):
            return self._bin("matmul", o)   # Armadillo: '*' between matrices is the product
        return self.g._add({"op": "scale", "a": self.i, "s": float(o)})

    def __rmul__(self, s):
        return self.g._add({"op": "scale", "a": self.i, "s": float(s)})

    def __matmul__(self, o):
        return self._bin("matmul", o)

    def sub(self, r0: int, c0: int, rows: int, cols: int):
        """Submatrix view: rows r0 .. r0+rows-1, columns c0 .. c0+cols-1."""
        return self.g._add({"op": "submat", "a": self.i, "slot": int(r0), "ld": int(c0),
                            "rows": int(rows), "cols": int(cols)})

    def col(self, j: int):
        """Column j as an m x 1 view (Armadillo's A.col(j) / A(:, j))."""
        m, _ = self.g.shape(self.i)
        return self.sub(0, j, m, 1)

    def row(self, i: int):
        """Row i as a 1 x n view (Armadillo's A.row(i) / A(i, :))."""
        _, n = self.g.shape(self.i)
        return self.sub(i, 0, 1, n)

    def __mod__(self, o):
        return self._bin("schur", o)

    def __truediv__(self, o):
        if isinstance(o, X):
            return self._bin("div", o)
        return self.g._add({"op": "div_scalar", "a": self.i, "s": float(o)})

    def t(self):
        return self.g._add({"op": "trans", "a": self.i})


def trans(x: X) -> X:
    return x.t()


def diagmat(x: X) -> X:
    return x.g._add({"op": "diagmat", "a": x.i})


def trace(x: X) -> X:
    return x.g._add({"op": "trace", "a": x.i})


def accu(x: X) -> X:
    return x.g._add({"op": "accu", "a": x.i})


def norm_fro(x: X) -> X:
    return x.g._add({"op": "norm_fro", "a": x.i})


def inv(x: X) -> X:
    return x.g._add({"op": "inv", "a": x.i})


def solve(a: X, b: X) -> X:
    """X with a X = b (Armadillo's solve(A, B))."""
    return a.g._add({"op": "solve", "a": a.i, "b": b.i})


# ---- the benchmark expressions (seeded shapes; names follow the paper) ----

def config_plain(n: int = 256, dtype: str = "f64"):
    """The six expressions over A, B, C, D (n x n) and v (n): C+A-2*D+B%D,
    trans(A)*B, 2*A*B+C, trace(A*B), diagmat(v)*B, accu(A%B).  Slots:
    A=0, B=1, C=2, D=3, v=4."""
    out = {}
    for name in ("ew", "transAB", "2AB+C", "traceAB", "diagvB", "accuAoB"):
        g = Graph()
        A, B, C, D = (g.input(s, n, n, dtype) for s in range(4))
        v = g.input(4, n, 1, dtype)
        e = {"ew": lambda: C + A - 2 * D + B % D,
             "transAB": lambda: A.t() * B,
             "2AB+C": lambda: 2 * A * B + C,
             "traceAB": lambda: trace(A * B),
             "diagvB": lambda: diagmat(v) * B,
             "accuAoB": lambda: accu(A % B)}[name]()
        out[name] = g.build(e)
    return out


def config_next(n: int = 256, dtype: str = "f64"):
    """The rewrites ranked next after the hot path: diagmat(A*B) (Sec. III
    (4)), trans(v)*diagmat(B)*w (Sec. III (7)), A(:,1) + B(2,:)^T read as
    views (Sec. III (2)) and the symmetric product A*A^T (Sec. III (8)).
    Slots: A=0, B=1 (n x n), v=2, w=3 (n x 1)."""
    out = {}
    for name in ("diagmatAB", "vdiagBw", "colrow", "AAt"):
        g = Graph()
        A, B = g.input(0, n, n, dtype), g.input(1, n, n, dtype)
        v, w = g.input(2, n, 1, dtype), g.input(3, n, 1, dtype)
        e = {"diagmatAB": lambda: diagmat(A * B),
             "vdiagBw": lambda: v.t() * diagmat(B) * w,
             "colrow": lambda: A.col(1) + B.row(2).t(),
             "AAt": lambda: A * A.t()}[name]()
        out[name] = g.build(e)
    return out


def config_fused(n: int = 8192, dtype: str = "f32"):
    """out = A%B + 3*C - D/2 with accu(out) and norm(out,'fro'); slots A..D = 0..3."""
    g = Graph()
    A, B, C, D = (g.input(s, n, n, dtype) for s in range(4))
    out = A % B + 3 * C - D / 2
    return g.build(out, accu(out), norm_fro(out))


def config_products(n: int = 8192, dtype: str = "f64"):
    """2*trans(A)*B + C (slots A=0, B=1, C=2)."""
    g = Graph()
    A, B, C = (g.input(s, n, n, dtype) for s in range(3))
    return g.build(2 * A.t() * B + C)


def config_chain(dims=(4096, 8192, 512, 4096, 1), dtype: str = "f64"):
    """A*B*C*v with A dims[0]xdims[1], ... (slots 0..3)."""
    g = Graph()
    Ms = [g.input(s, dims[s], dims[s + 1], dtype) for s in range(len(dims) - 1)]
    e = Ms[0]
    for M in Ms[1:]:
        e = e * M
    return g.build(e)


def config_solve(n: int = 4096, nrhs: int = 64, dtype: str = "f64"):
    """inv(A)*B (slots A=0, B=1)."""
    g = Graph()
    A = g.input(0, n, n, dtype)
    B = g.input(1, n, nrhs, dtype)
    return g.build(inv(A) * B)


def config_batched_instance(m: int, n: int, k: int, dtype: str = "f32"):
    """One instance of the batched family: 2*trans(A)*B + C and
    trace(trans(A)*B), A k x m, B k x n (dtype), C m x n FP32; slots A=0,
    B=1, C=2.  The trace is read as trace(A^T B) = sum over i < min(m, n)
    of (A^T B)_ii, the conforming form of trace(A*B) for these shapes."""
    g = Graph()
    A = g.input(0, k, m, dtype)
    B = g.input(1, k, n, dtype)
    C = g.input(2, m, n, "f32")
    return g.build(2 * A.t() * B + C, trace(A.t() * B))
