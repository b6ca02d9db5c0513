"""Python binding of libarma_gpu.so, a GB300 evaluator for compound
linear-algebra expressions (delayed evaluation, elementwise fusion, product
rewrites and chain reordering as in Sanderson & Curtin, ICCAE 2025).

This module only marshals arguments: every step of an evaluation runs in
the library's CUDA kernels.  PyTorch supplies device memory and streams.
There is no fallback: if the library is missing, importing ``lib()`` raises.

Expressions are lists of node dicts in topological order (the same plain
format the tests use), e.g.::

    nodes = [{"op": "input", "slot": 0, "rows": m, "cols": n, "dtype": "f64"},
             {"op": "input", "slot": 1, "rows": m, "cols": n, "dtype": "f64"},
             {"op": "scale", "a": 0, "s": 0.4},
             {"op": "scale", "a": 1, "s": 0.6},
             {"op": "add", "a": 2, "b": 3}]
    plan = Plan(nodes, outputs=[4])
    (Z,) = plan(X, Y)          # X, Y column-major CUDA tensors

Matrices are column-major: a tensor ``t`` of shape (rows, cols) with
``t.stride(0) == 1`` (see ``colmajor``).
"""
from __future__ import annotations

import ctypes
import json
import os
from functools import lru_cache

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libarma_gpu.so")

# ---- enums (include/arma_gpu.h) ----
F64, F32, BF16 = 0, 1, 2
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16}
OPS = {"input": 0, "add": 1, "sub": 2, "schur": 3, "div": 4, "scale": 5, "div_scalar": 6,
       "add_scalar": 7, "neg": 8, "trans": 9, "matmul": 10, "diagmat": 11, "trace": 12,
       "accu": 13, "norm_fro": 14, "inv": 15, "submat": 16, "solve": 17}
TIERS = {"native": 0, "f64": 1, "split_bf16": 2, "bf16": 3, "lu32_ir64": 4, "f64_sliced": 5}
PLAN_LITERAL, PLAN_CHAIN_LEFT, PLAN_CHAIN_GREEDY, PLAN_COST_MLP, PLAN_NO_FUSE, PLAN_NO_TENSOR = 1, 2, 4, 8, 16, 32
PLAN_TILE64, PLAN_TILE32, PLAN_NO_SYRK, PLAN_NO_SOLVE_ANALYSIS = 64, 128, 256, 512
PLAN_COST_HEURISTIC, PLAN_TIER_CHOICE, PLAN_NO_SPLITK, PLAN_DFMA_RESIDUAL = 0x400, 0x800, 0x1000, 0x2000
PLAN_NO_LOOKAHEAD = 0x4000
STATUS = {0: "ok", 1: "invalid", 2: "shape", 3: "dtype", 4: "align", 5: "workspace",
          6: "singular", 7: "noconverge", 8: "cuda", 9: "unsupported", 10: "timeout"}
PLAN_REFINE_SHIFT, PLAN_REFINE_MASK = 16, 0xF0000


def PLAN_REFINE_STEPS(k: int) -> int:
    """Plan flag: stop FP64 iterative refinement after k (1..15) steps."""
    return (int(k) & 0xF) << PLAN_REFINE_SHIFT


def PLAN_SPLITS(k: int) -> int:
    """Flag bits asking every product for k K splits (1..15); 0 keeps the
    library's per-SM model (ARMA_PLAN_SPLITS)."""
    if not 0 <= int(k) <= 15:
        raise ValueError("split count must be in 0..15")
    return (int(k) & 0xF) << 20


class ArmaError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        self.status = STATUS.get(code, str(code))
        self.detail = detail
        super().__init__(f"{where}: {self.status} ({code})" + (f": {detail}" if detail else ""))


class Node(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("scalar", ctypes.c_double)]


class Expr(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_outputs", ctypes.c_int32),
                ("nodes", ctypes.POINTER(Node)), ("outputs", ctypes.POINTER(ctypes.c_int32)),
                ("tier", ctypes.c_int32), ("flags", ctypes.c_uint32)]


EXPORTS = ["arma_gpu_plan", "arma_gpu_plan_workspace", "arma_gpu_output_info", "arma_gpu_eval",
           "arma_gpu_eval_status", "arma_gpu_eval_solve_path", "arma_gpu_plan_info", "arma_gpu_plan_free",
           "arma_gpu_status_string", "arma_gpu_last_cuda_error", "arma_gpu_set_wait_limit_ns",
           "arma_gpu_chain_order",
           "arma_gpu_eval_fused_static",
           "arma_gpu_plan_batched", "arma_gpu_batched_table_bytes", "arma_gpu_batched_table_fill",
           "arma_gpu_eval_batched", "arma_gpu_plan_features", "arma_gpu_plan_heuristic_cost",
           "arma_gpu_mlp_param_count", "arma_gpu_mlp_workspace", "arma_gpu_mlp_forward", "arma_gpu_mlp_grad",
           "arma_gpu_mlp_adam", "arma_gpu_plan_candidates", "arma_gpu_cost_model_load",
           "arma_gpu_cost_model_clear", "arma_gpu_cost_model_predict", "arma_gpu_device_address"]
N_FEATURES = 32
STATIC_SCRATCH_BYTES = 131072


@lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.arma_gpu_plan.argtypes = [ctypes.POINTER(Expr), ctypes.POINTER(vp)]
    L.arma_gpu_plan_workspace.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.arma_gpu_output_info.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)]
    L.arma_gpu_eval.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp, ctypes.c_size_t, vp]
    L.arma_gpu_eval_status.argtypes = [vp, vp, vp, ctypes.POINTER(i64)]
    L.arma_gpu_eval_solve_path.argtypes = [vp, vp, vp] + [ctypes.POINTER(i32)] * 4
    L.arma_gpu_plan_info.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.arma_gpu_plan_free.argtypes = [vp]
    L.arma_gpu_plan_free.restype = None
    L.arma_gpu_status_string.argtypes = [ctypes.c_int]
    L.arma_gpu_status_string.restype = ctypes.c_char_p
    L.arma_gpu_last_cuda_error.argtypes = []
    L.arma_gpu_last_cuda_error.restype = ctypes.c_char_p
    L.arma_gpu_set_wait_limit_ns.argtypes = [ctypes.c_uint64]
    L.arma_gpu_set_wait_limit_ns.restype = ctypes.c_uint64
    L.arma_gpu_device_address.argtypes = [vp, ctypes.POINTER(vp)]
    L.arma_gpu_chain_order.argtypes = [i32, ctypes.POINTER(i64), i32, ctypes.POINTER(i32),
                                       ctypes.POINTER(ctypes.c_uint64)]
    L.arma_gpu_eval_fused_static.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.arma_gpu_plan_batched.argtypes = [ctypes.POINTER(Expr), i32, ctypes.POINTER(vp)]
    L.arma_gpu_batched_table_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.arma_gpu_batched_table_fill.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.arma_gpu_eval_batched.argtypes = [vp, vp, vp, ctypes.c_size_t, vp]
    L.arma_gpu_plan_features.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i32]
    L.arma_gpu_plan_heuristic_cost.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.arma_gpu_plan_candidates.argtypes = [ctypes.POINTER(Expr), ctypes.POINTER(vp), i32, ctypes.POINTER(i32)]
    L.arma_gpu_cost_model_load.argtypes = [vp, i32, i32, vp, vp, ctypes.c_double, ctypes.c_double]
    L.arma_gpu_cost_model_clear.argtypes = []
    L.arma_gpu_cost_model_clear.restype = None
    L.arma_gpu_cost_model_predict.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.arma_gpu_mlp_param_count.argtypes = [i32, i32]
    L.arma_gpu_mlp_param_count.restype = i64
    L.arma_gpu_mlp_workspace.argtypes = [i32, i32, i32]
    L.arma_gpu_mlp_workspace.restype = ctypes.c_size_t
    L.arma_gpu_mlp_forward.argtypes = [vp, i32, i32, vp, i32, vp, vp]
    L.arma_gpu_mlp_grad.argtypes = [vp, i32, i32, vp, vp, i32, vp, vp, vp, ctypes.c_size_t, vp]
    L.arma_gpu_mlp_adam.argtypes = [vp, vp, vp, vp, i64, i32, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, vp]
    return L


def _check(code: int, where: str):
    if code != 0:
        detail = ""
        if STATUS.get(code) == "cuda":
            detail = (lib().arma_gpu_last_cuda_error() or b"").decode(errors="replace")
        raise ArmaError(code, where, detail)


def set_wait_limit_ns(ns: int) -> int:
    """Limit of each bounded device wait of the solve kernels (ns, process
    wide); 0 gives up at the first unset poll.  Returns the previous limit."""
    return int(lib().arma_gpu_set_wait_limit_ns(int(ns)))


def device_address(ptr: int) -> int:
    """The address at which the library's kernels reach memory at ``ptr``
    (device memory: ``ptr``; pinned host memory the GPU maps: its mapped
    address).  Raises ArmaError for memory the device cannot address."""
    out = ctypes.c_void_p()
    _check(lib().arma_gpu_device_address(ctypes.c_void_p(ptr), ctypes.byref(out)), "arma_gpu_device_address")
    return int(out.value)


def torch_dtype(dt: int):
    import torch
    return {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}[dt]


def colmajor(t):
    """Column-major copy (or view) of a 2-D tensor: stride (1, rows)."""
    if t.dim() == 1:
        t = t.reshape(-1, 1)
    if t.stride(0) == 1 and (t.shape[1] <= 1 or t.stride(1) >= max(1, t.shape[0])):
        return t
    return t.t().contiguous().t()


def empty_colmajor(rows: int, cols: int, dtype, device):
    import torch
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def ld_of(t) -> int:
    rows = t.shape[0]
    if t.shape[1] <= 1:
        return max(1, rows)
    return int(t.stride(1))


def _mk_nodes(nodes):
    arr = (Node * len(nodes))()
    for i, d in enumerate(nodes):
        n = arr[i]
        n.op = OPS[d["op"]]
        n.a = d.get("a", -1)
        n.b = d.get("b", -1)
        n.slot = d.get("slot", 0)
        dt = d.get("dtype", "f64")
        n.dtype = DTYPES[dt] if isinstance(dt, str) else int(dt)
        n.rows = d.get("rows", 0)
        n.cols = d.get("cols", 0)
        n.ld = d.get("ld", max(1, d.get("rows", 0)))
        n.scalar = float(d.get("s", 0.0))
    return arr


def _mk_expr(nodes, outputs, tier, flags):
    arr = _mk_nodes(nodes)
    outs = (ctypes.c_int32 * len(outputs))(*outputs)
    e = Expr(len(nodes), len(outputs), arr, outs, TIERS[tier] if isinstance(tier, str) else int(tier), int(flags))
    return e, arr, outs


def candidates(nodes, outputs, tier="native", flags=0, capacity=128):
    """Every distinct candidate plan the library considers for an expression
    (arma_gpu_plan_candidates), in its enumeration order: the index of the
    candidate a COST-flag plan picked (``info["choice"]["picked"]``)."""
    L = lib()
    e, arr, outs = _mk_expr(nodes, outputs, tier, flags)
    hs = (ctypes.c_void_p * capacity)()
    n = ctypes.c_int32()
    _check(L.arma_gpu_plan_candidates(ctypes.byref(e), hs, capacity, ctypes.byref(n)), "arma_gpu_plan_candidates")
    return [Plan(nodes, outputs, _handle=ctypes.c_void_p(hs[i])) for i in range(min(n.value, capacity))]


def load_cost_model(params, mean, scale, hidden, guard=0.0, margin=0.0):
    """Give the library a trained cost network (host arrays; see
    arma_gpu_cost_model_load).  ARMA_PLAN_COST_MLP plans consult it."""
    import numpy as np
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    mu = np.ascontiguousarray(np.asarray(mean, dtype=np.float32))
    sd = np.ascontiguousarray(np.asarray(scale, dtype=np.float32))
    _check(lib().arma_gpu_cost_model_load(p.ctypes.data, len(mu), int(hidden), mu.ctypes.data, sd.ctypes.data,
                                          float(guard), float(margin)), "arma_gpu_cost_model_load")


def clear_cost_model():
    lib().arma_gpu_cost_model_clear()


class Plan:
    """A planned expression.  Planning runs on the host only; ``__call__``
    enqueues the plan's kernels on the current CUDA stream."""

    def __init__(self, nodes, outputs, tier="native", flags=0, _handle=None):
        self.nodes = [dict(d) for d in nodes]
        self.outputs = list(outputs)
        L = lib()
        if _handle is None:
            e, self._arr, self._outs = _mk_expr(self.nodes, self.outputs, tier, flags)
            h = ctypes.c_void_p()
            _check(L.arma_gpu_plan(ctypes.byref(e), ctypes.byref(h)), "arma_gpu_plan")
        else:
            h = _handle
        self._h = h
        ws = ctypes.c_size_t()
        _check(L.arma_gpu_plan_workspace(h, ctypes.byref(ws)), "arma_gpu_plan_workspace")
        self.workspace_bytes = int(ws.value)
        self.out_info = []
        for i in range(len(self.outputs)):
            r, c, dt = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
            _check(L.arma_gpu_output_info(h, i, ctypes.byref(r), ctypes.byref(c), ctypes.byref(dt)),
                   "arma_gpu_output_info")
            scalar = self.nodes[self.outputs[i]]["op"] in ("trace", "accu", "norm_fro")
            self.out_info.append((int(r.value), int(c.value), int(dt.value), scalar))
        self.n_slots = 1 + max((d.get("slot", 0) for d in self.nodes if d["op"] == "input"), default=-1)
        self._ws = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().arma_gpu_plan_free(h)
            except Exception:
                pass

    @property
    def info(self) -> dict:
        L = lib()
        need = ctypes.c_size_t()
        L.arma_gpu_plan_info(self._h, None, 0, ctypes.byref(need))
        buf = ctypes.create_string_buffer(need.value)
        _check(L.arma_gpu_plan_info(self._h, buf, need.value, None), "arma_gpu_plan_info")
        return json.loads(buf.value.decode())

    def features(self):
        f = (ctypes.c_float * N_FEATURES)()
        _check(lib().arma_gpu_plan_features(self._h, f, N_FEATURES), "arma_gpu_plan_features")
        return list(f)

    def predicted_cost(self) -> float:
        """Seconds the loaded cost network predicts (host forward pass)."""
        c = ctypes.c_double()
        _check(lib().arma_gpu_cost_model_predict(self._h, ctypes.byref(c)), "arma_gpu_cost_model_predict")
        return float(c.value)

    def heuristic_cost(self) -> float:
        c = ctypes.c_double()
        _check(lib().arma_gpu_plan_heuristic_cost(self._h, ctypes.byref(c)), "arma_gpu_plan_heuristic_cost")
        return float(c.value)

    def workspace(self, device):
        import torch
        key = str(device)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < self.workspace_bytes:
            ws = torch.empty(max(256, self.workspace_bytes), dtype=torch.uint8, device=device)
            self._ws[key] = ws
        return ws

    def alloc_outputs(self, device):
        import torch
        outs = []
        for (r, c, dt, scalar) in self.out_info:
            if scalar:
                outs.append(torch.empty(1, dtype=torch.float64, device=device))
            else:
                outs.append(empty_colmajor(r, c, torch_dtype(dt), device))
        return outs

    def pointers(self, inputs, outputs):
        ins = (ctypes.c_void_p * max(1, self.n_slots))()
        for k, t in enumerate(inputs):
            ins[k] = t.data_ptr() if t is not None else None
        outs = (ctypes.c_void_p * len(outputs))(*[o.data_ptr() for o in outputs])
        return ins, outs

    def __call__(self, *inputs, outputs=None, workspace=None, stream=None):
        import torch
        dev = inputs[0].device if inputs else torch.device("cuda")
        if outputs is None:
            outputs = self.alloc_outputs(dev)
        if workspace is None:
            workspace = self.workspace(dev)
        ins, outs = self.pointers(inputs, outputs)
        st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        _check(lib().arma_gpu_eval(self._h, ins, outs, ctypes.c_void_p(workspace.data_ptr()),
                                   workspace.numel(), ctypes.c_void_p(st)), "arma_gpu_eval")
        return outputs

    def call_static(self, *inputs, outputs=None, stream=None):
        """Evaluate with the library's own static scratch instead of a
        workspace (fused elementwise plans only; see arma_gpu_eval_fused_static)."""
        import torch
        dev = inputs[0].device if inputs else torch.device("cuda")
        if outputs is None:
            outputs = self.alloc_outputs(dev)
        ins, outs = self.pointers(inputs, outputs)
        st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        _check(lib().arma_gpu_eval_fused_static(self._h, ins, outs, ctypes.c_void_p(st)),
               "arma_gpu_eval_fused_static")
        return outputs

    def _last_workspace(self, workspace):
        if workspace is not None:
            return workspace
        if not self._ws:
            raise ValueError("no evaluation to report on: evaluate the plan first or pass its workspace")
        return next(iter(self._ws.values()))

    def status(self, workspace=None, stream=None):
        """Device-side status of the last evaluation (synchronises)."""
        import torch
        ws = self._last_workspace(workspace)
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        info = ctypes.c_int64()
        code = lib().arma_gpu_eval_status(self._h, ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(st),
                                          ctypes.byref(info))
        return STATUS.get(code, str(code)), int(info.value)


SOLVE_PATHS = {0: "none", 1: "general", 2: "diagonal", 3: "band", 4: "upper", 5: "lower", 6: "cholesky"}


def _solve_path(self, workspace=None, stream=None):
    """The solver the last evaluation's analysed solve took and what the
    analysis of its matrix found (synchronises): (path, kl, ku, symmetric)."""
    import torch
    ws = self._last_workspace(workspace)
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().arma_gpu_eval_solve_path(self._h, ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(st),
                                          *[ctypes.byref(x) for x in v]), "arma_gpu_eval_solve_path")
    return SOLVE_PATHS.get(v[0].value, str(v[0].value)), v[1].value, v[2].value, bool(v[3].value)


Plan.solve_path = _solve_path


class BatchedPlan:
    """Many instances of one expression family evaluated by one grouped launch.

    ``instances`` is a list of (nodes, outputs) with the same structure.
    ``bind(inputs, outputs)`` builds the device problem table for lists of
    per-instance tensors; ``__call__`` then runs the whole batch."""

    def __init__(self, instances, tier="native", flags=0):
        L = lib()
        self.count = len(instances)
        self._keep = []
        exprs = (Expr * self.count)()
        for i, (nodes, outs) in enumerate(instances):
            arr = _mk_nodes(nodes)
            o = (ctypes.c_int32 * len(outs))(*outs)
            self._keep += [arr, o]
            exprs[i] = Expr(len(nodes), len(outs), arr, o, TIERS[tier] if isinstance(tier, str) else int(tier),
                            int(flags))
        h = ctypes.c_void_p()
        _check(L.arma_gpu_plan_batched(exprs, self.count, ctypes.byref(h)), "arma_gpu_plan_batched")
        self._h = h
        self.n_slots = 1 + max(d.get("slot", 0) for d in instances[0][0] if d["op"] == "input")
        self.n_outs = len(instances[0][1])
        tb = ctypes.c_size_t()
        _check(L.arma_gpu_batched_table_bytes(h, ctypes.byref(tb)), "arma_gpu_batched_table_bytes")
        self.table_bytes = int(tb.value)
        ws = ctypes.c_size_t()
        _check(L.arma_gpu_plan_workspace(h, ctypes.byref(ws)), "arma_gpu_plan_workspace")
        self.workspace_bytes = int(ws.value)
        self.table = None
        self.ws = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().arma_gpu_plan_free(h)
            except Exception:
                pass

    @property
    def info(self) -> dict:
        L = lib()
        need = ctypes.c_size_t()
        L.arma_gpu_plan_info(self._h, None, 0, ctypes.byref(need))
        buf = ctypes.create_string_buffer(need.value)
        _check(L.arma_gpu_plan_info(self._h, buf, need.value, None), "arma_gpu_plan_info")
        return json.loads(buf.value.decode())

    def bind(self, inputs, outputs, device):
        """inputs[i][s], outputs[i][o]: tensors of instance i."""
        import numpy as np
        import torch
        ins = (ctypes.c_void_p * (self.count * self.n_slots))()
        outs = (ctypes.c_void_p * (self.count * self.n_outs))()
        for i in range(self.count):
            for s_, t in enumerate(inputs[i]):
                ins[i * self.n_slots + s_] = t.data_ptr()
            for o, t in enumerate(outputs[i]):
                outs[i * self.n_outs + o] = t.data_ptr()
        host = np.zeros(self.table_bytes, dtype=np.uint8)
        _check(lib().arma_gpu_batched_table_fill(self._h, ins, outs, host.ctypes.data_as(ctypes.c_void_p)),
               "arma_gpu_batched_table_fill")
        self.table = torch.from_numpy(host).to(device)
        self.ws = torch.empty(max(256, self.workspace_bytes), dtype=torch.uint8, device=device)

    def status(self, stream=None):
        """Device-side status of the last batched evaluation (synchronises)."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        info = ctypes.c_int64()
        code = lib().arma_gpu_eval_status(self._h, ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_void_p(st),
                                          ctypes.byref(info))
        return STATUS.get(code, str(code)), int(info.value)

    def __call__(self, stream=None):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(lib().arma_gpu_eval_batched(self._h, ctypes.c_void_p(self.table.data_ptr()),
                                           ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                           ctypes.c_void_p(st)), "arma_gpu_eval_batched")


def chain_order(dims, method: int = 0):
    """(splits in preorder, cost) of the planner's chain order: 0 exact DP,
    1 the paper's greedy rule, 2 left to right."""
    n = len(dims) - 1
    d = (ctypes.c_int64 * len(dims))(*dims)
    sp = (ctypes.c_int32 * max(1, n - 1))()
    cost = ctypes.c_uint64()
    _check(lib().arma_gpu_chain_order(n, d, method, sp, ctypes.byref(cost)), "arma_gpu_chain_order")
    return [int(sp[i]) for i in range(n - 1)], int(cost.value)


def tree_from_splits(splits, lo: int, hi: int):
    """Rebuild a (split, left, right) tree from a preorder split list."""
    it = iter(splits)

    def rec(i, j):
        if i == j:
            return i
        k = next(it)
        return (k, rec(i, k), rec(k + 1, j))
    return rec(lo, hi)
