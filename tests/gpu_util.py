"""Helpers for the GPU parity tests: move seeded host arrays to the device in
column-major layout, bring results back, and compare with the oracle."""
import numpy as np
import pytest

import oracle
import synth

# tolerances on the relative Frobenius error against the FP64 oracle
TOL = {"f64": 1e-12, "split_bf16": 1e-6, "f32": 1e-5, "bf16": 2e-2}


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_03000_gb300 import build
    build.build()
    import paper_2502_03000_gb300 as ag
    ag.lib.cache_clear()
    ag.lib()
    return torch


def to_dev(a, dtype="f64", pad=0, offset=0):
    """Column-major device tensor holding the host array ``a``; ``pad`` extra
    rows in the leading dimension, ``offset`` elements of misalignment."""
    import torch
    a = np.asarray(a)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    m, n = a.shape
    td = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    ld = max(1, m + pad)
    buf = torch.zeros(offset + ld * max(n, 1) + 8, dtype=torch.float64 if dtype == "f64" else torch.float32)
    host = np.zeros((max(n, 1), ld), dtype=np.float64)
    host[:n, :m] = a.T
    flat = torch.from_numpy(host.reshape(-1).astype(np.float64))
    buf[offset:offset + flat.numel()] = flat.to(buf.dtype)
    dev = buf.to(td).cuda()
    t = dev[offset:offset + ld * max(n, 1)].view(max(n, 1), ld).t()[:m, :n]
    return t


def to_host(t) -> np.ndarray:
    if t.numel() == 1 and t.dim() == 1:
        return float(t.double().item())
    return np.asfortranarray(t.double().cpu().numpy())


def inputs(seed, shapes, dtype):
    """Seeded host arrays of the given shapes in the storage dtype."""
    return [synth.matrix(seed, s + 1, r, c, dtype) for s, (r, c) in enumerate(shapes)]


def check(got, ref, tol, what=""):
    for i, (g, r) in enumerate(zip(got, ref)):
        g = to_host(g)
        err = oracle.rel_err(g, r)
        assert err <= tol, f"{what} output {i}: rel err {err:.3e} > {tol:.1e}"
