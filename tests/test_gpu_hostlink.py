"""Inputs and outputs in pinned host memory: arma_gpu_device_address gives
the address the kernels use, and the fused pass reading the inputs over the
host link (no staging copy) gives the result of the same plan on device
copies, bit for bit; plain pageable host memory is refused."""
import ctypes

import numpy as np
import pytest

import paper_2502_03000_gb300 as ag
from paper_2502_03000_gb300 import expr as E
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def test_device_address_of_device_and_pageable_memory(torch):
    d = torch.empty(1024, device="cuda")
    assert ag.device_address(d.data_ptr()) == d.data_ptr()
    a = np.zeros(1024)
    with pytest.raises(ag.ArmaError):
        ag.device_address(a.ctypes.data)
    out = ctypes.c_void_p(1)
    assert ag.lib().arma_gpu_device_address(None, ctypes.byref(out)) != 0
    assert out.value is None


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_fused_pass_reads_pinned_host_inputs(torch, dtype):
    n = 777   # several blocks and a ragged tail
    td = torch.float32 if dtype == "f32" else torch.float64
    nodes, outs = E.config_fused(n, dtype)
    plan = ag.Plan(nodes, outs)
    g = torch.Generator().manual_seed(11)
    host = [(torch.rand((n, n), generator=g, dtype=torch.float64) * 2 - 1).to(td).pin_memory() for _ in range(4)]
    dev = [h.to("cuda") for h in host]
    ref = plan(*[d.t() for d in dev])
    ws = plan.workspace(torch.device("cuda"))
    got = plan.alloc_outputs(torch.device("cuda"))
    ins = (ctypes.c_void_p * max(1, plan.n_slots))()
    for k, h in enumerate(host):
        ins[k] = ag.device_address(h.data_ptr())
    # the output matrix in pinned host memory too
    hout = torch.empty_like(host[0]).pin_memory()
    outp = [ag.device_address(hout.data_ptr())] + [o.data_ptr() for o in got[1:]]
    outs_c = (ctypes.c_void_p * len(outp))(*outp)
    st = torch.cuda.current_stream().cuda_stream
    assert ag.lib().arma_gpu_eval(plan._h, ins, outs_c, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                  ctypes.c_void_p(st)) == 0
    torch.cuda.synchronize()
    assert torch.equal(hout.t(), ref[0].cpu())
    for a, b in zip(got[1:], ref[1:]):
        assert torch.equal(a, b)
