"""The workspace-free entry point, arma_gpu_eval_fused_static, for callers
that cannot allocate device memory (plug-ins handed only raw pointers, code
inside another framework's memory pool, loops that cannot afford
cudaMalloc's implicit synchronisation).  Its results must match the
ordinary arma_gpu_eval on the same inputs, call after call, because every
call reuses the same library-owned scratch array.

Kept in its own file that sorts last, so a run that stops at the first
failure has already run every other test."""
import ctypes

import pytest

import paper_2502_03000_gb300 as ag
from paper_2502_03000_gb300 import expr as E
from tests.gpu_util import TOL, check, inputs, need_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


@pytest.mark.parametrize("dtype,shape", [("f64", (257, 263)), ("f32", (1031, 517)), ("f64", (1, 1))])
def test_static_scratch_matches_workspace_eval(torch, dtype, shape):
    m, n = shape
    g = E.Graph()
    A, B, C, D = (g.input(s, m, n, dtype) for s in range(4))
    out = A % B + 3 * C - D / 2
    nodes, outs = g.build(out, E.accu(out), E.norm_fro(out), E.trace(A % B))
    plan = ag.Plan(nodes, outs)
    assert plan.workspace_bytes <= ag.STATIC_SCRATCH_BYTES
    host = inputs(123, [shape] * 4, dtype)
    ins = [to_dev(h, dtype) for h in host]
    ref = plan(*ins)                      # ordinary entry point, caller workspace
    torch.cuda.synchronize()
    ref = [to_host(r) for r in ref]
    for _ in range(2):                    # two calls in a row share the static array
        L = ag.lib()
        outs_t = plan.alloc_outputs(ins[0].device)
        pin, pout = plan.pointers(ins, outs_t)
        st = torch.cuda.current_stream().cuda_stream
        code = L.arma_gpu_eval_fused_static(plan._h, pin, pout, ctypes.c_void_p(st))
        assert code == 0, ag.STATUS.get(code)
        torch.cuda.synchronize()
        check(outs_t, ref, TOL[dtype], "static scratch vs workspace")


def test_static_scratch_rejects_what_it_cannot_run(torch):
    # a product plan is not a fused elementwise plan
    p = ag.Plan(*E.config_products(64))
    A = [to_dev(h) for h in inputs(5, [(64, 64)] * 3, "f64")]
    with pytest.raises(ag.ArmaError) as ei:
        p.call_static(*A)
    assert ei.value.status == "unsupported"
    # a literal plan whose temporaries exceed the static array
    big = ag.Plan(*E.config_fused(256, "f64"), flags=ag.PLAN_LITERAL)
    assert big.workspace_bytes > ag.STATIC_SCRATCH_BYTES
    X = [to_dev(h) for h in inputs(6, [(256, 256)] * 4, "f64")]
    with pytest.raises(ag.ArmaError) as ei:
        big.call_static(*X)
    assert ei.value.status == "workspace"
