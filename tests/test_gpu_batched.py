"""Batched evaluation: many independent 2*trans(A_i)*B_i + C_i and
trace(A_i^T B_i) of uneven sizes in one grouped launch, against the oracle
instance by instance; CUDA-graph replay; the full 10,000-instance batch on
sampled instances."""
import numpy as np
import pytest

import oracle
import paper_2502_03000_gb300 as ag
import synth
from paper_2502_03000_gb300 import expr as E
from tests.gpu_util import TOL, need_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def sizes(seed, count, lo=8, hi=512):
    m = synth.log_uniform_ints(seed, 1, count, lo, hi)
    n = synth.log_uniform_ints(seed, 2, count, lo, hi)
    k = synth.log_uniform_ints(seed, 3, count, lo, hi)
    return m, n, k


def build_batch(torch, seed, count, dtype, lo=8, hi=512):
    m, n, k = sizes(seed, count, lo, hi)
    inst, host, ins, outs = [], [], [], []
    for i in range(count):
        nodes, o = E.config_batched_instance(int(m[i]), int(n[i]), int(k[i]), dtype)
        inst.append((nodes, o))
        A = synth.matrix(seed + i, 1, int(k[i]), int(m[i]), dtype)
        B = synth.matrix(seed + i, 2, int(k[i]), int(n[i]), dtype)
        C = synth.matrix(seed + i, 3, int(m[i]), int(n[i]), "f32")
        host.append([A, B, C])
        ins.append([to_dev(A, dtype), to_dev(B, dtype), to_dev(C, "f32")])
        outs.append([ag.empty_colmajor(int(m[i]), int(n[i]), torch.float32, "cuda"),
                     torch.zeros(1, dtype=torch.float64, device="cuda")])
    return inst, host, ins, outs


def check_instance(nodes, o, host, out, dtype):
    ref = oracle.evaluate(nodes, o, host)
    D = to_host(out[0])
    assert oracle.rel_err(D, ref[0]) <= TOL[dtype if dtype == "bf16" else "f32"]
    # trace: compare against the size of its terms (a random trace can be near 0)
    At = np.asarray(host[0], dtype=np.float64)
    Bv = np.asarray(host[1], dtype=np.float64)
    d = min(At.shape[1], Bv.shape[1])
    terms = np.abs(At[:, :d] * Bv[:, :d]).sum()
    t = to_host(out[1])
    assert abs(t - ref[1]) <= 1e-6 * max(terms, 1e-300)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batched_matches_oracle(torch, dtype):
    inst, host, ins, outs = build_batch(torch, 101, 60, dtype)
    bp = ag.BatchedPlan(inst)
    assert bp.info["mode"] == "batched"
    bp.bind(ins, outs, "cuda")
    bp()
    torch.cuda.synchronize()
    for i in range(len(inst)):
        check_instance(*inst[i], host[i], outs[i], dtype)


def test_batched_tiny_and_degenerate(torch):
    inst, host, ins, outs = build_batch(torch, 7, 30, "f32", lo=1, hi=40)
    bp = ag.BatchedPlan(inst)
    bp.bind(ins, outs, "cuda")
    bp()
    torch.cuda.synchronize()
    for i in range(len(inst)):
        check_instance(*inst[i], host[i], outs[i], "f32")


def test_batched_graph_replay(torch):
    inst, host, ins, outs = build_batch(torch, 55, 40, "f32")
    bp = ag.BatchedPlan(inst)
    bp.bind(ins, outs, "cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bp(stream=s.cuda_stream)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    first = [o[0].clone() for o in outs]
    for o in outs:
        o[0].zero_()
        o[1].zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bp(stream=torch.cuda.current_stream().cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    for a, o in zip(first, outs):
        assert torch.equal(a, o[0])
    for i in range(len(inst)):
        check_instance(*inst[i], host[i], outs[i], "f32")


def test_batched_rejects_other_families(torch):
    g = E.Graph()
    A, B = g.input(0, 16, 16, "f32"), g.input(1, 16, 16, "f32")
    with pytest.raises(ag.ArmaError) as ei:
        ag.BatchedPlan([g.build(A % B + A)])
    assert ei.value.status == "unsupported"


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batched_benchmark_size_sampled(torch, dtype):
    """10,000 instances (m, n, k log-uniform in [8, 512]) in one launch;
    sampled instances against the oracle"""
    count = 10000
    m, n, k = sizes(20250203 + 4, count)
    inst, ins, outs = [], [], []
    rng = np.random.default_rng(4)
    sample = set(rng.choice(count, 24, replace=False).tolist())
    gen = torch.Generator(device="cuda")
    gen.manual_seed(20250203 + 4)

    td = torch.float32 if dtype == "f32" else torch.bfloat16

    def uni(r, c, t=torch.float32):
        return (torch.rand((c, r), device="cuda", generator=gen) * 2 - 1).to(t).t()

    for i in range(count):
        nodes, o = E.config_batched_instance(int(m[i]), int(n[i]), int(k[i]), dtype)
        inst.append((nodes, o))
        ins.append([uni(int(k[i]), int(m[i]), td), uni(int(k[i]), int(n[i]), td), uni(int(m[i]), int(n[i]))])
        outs.append([ag.empty_colmajor(int(m[i]), int(n[i]), torch.float32, "cuda"),
                     torch.zeros(1, dtype=torch.float64, device="cuda")])
    bp = ag.BatchedPlan(inst)
    bp.bind(ins, outs, "cuda")
    bp()
    torch.cuda.synchronize()
    assert bp.info["tensor_cores"] is True
    for i in sorted(sample):
        h = [to_host(t) for t in ins[i]]
        check_instance(*inst[i], h, outs[i], dtype)


def batch_of(torch, shapes, dtype, seed):
    inst, host, ins, outs = [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        nodes, o = E.config_batched_instance(m, n, k, dtype)
        inst.append((nodes, o))
        A = synth.matrix(seed + i, 1, k, m, dtype)
        B = synth.matrix(seed + i, 2, k, n, dtype)
        C = synth.matrix(seed + i, 3, m, n, "f32")
        host.append([A, B, C])
        ins.append([to_dev(A, dtype), to_dev(B, dtype), to_dev(C, "f32")])
        outs.append([ag.empty_colmajor(m, n, torch.float32, "cuda"),
                     torch.zeros(1, dtype=torch.float64, device="cuda")])
    return inst, host, ins, outs


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batched_tensor_core_tiles(torch, dtype):
    """128 x 128 tcgen05 tiles (BF16 operands as they are, FP32 operands as
    three exact BF16 slices): exact tile, ragged edges in m, n and K, several
    K blocks, K longer than the 512 of the benchmark, one element, more tiles
    than CTAs"""
    shapes = [(128, 128, 64), (129, 127, 65), (300, 257, 1000), (1, 1, 1), (8, 300, 3), (256, 5, 130),
              (640, 384, 16), (1100, 1030, 70)]
    inst, host, ins, outs = batch_of(torch, shapes, dtype, 900)
    bp = ag.BatchedPlan(inst)
    assert bp.info["tensor_cores"] is True
    assert bp.info["steps"][0]["kernel"] == "grouped_tc"
    bp.bind(ins, outs, "cuda")
    bp()
    torch.cuda.synchronize()
    assert bp.status()[0] == "ok"
    for i in range(len(inst)):
        check_instance(*inst[i], host[i], outs[i], dtype)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batched_tensor_and_simt_paths_agree(torch, dtype):
    """the SIMT tiles (PLAN_NO_TENSOR) and the tensor-core tiles meet the
    same oracle on the same batch"""
    inst, host, ins, outs = build_batch(torch, 303, 40, dtype)
    for flags in (0, ag.PLAN_NO_TENSOR):
        bp = ag.BatchedPlan(inst, flags=flags)
        assert bp.info["tensor_cores"] is (flags == 0)
        bp.bind(ins, outs, "cuda")
        for o in outs:
            o[0].fill_(float("nan"))
            o[1].zero_()
        bp()
        torch.cuda.synchronize()
        for i in range(len(inst)):
            check_instance(*inst[i], host[i], outs[i], dtype)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batched_autotune(torch, dtype):
    """the autotuner times the distinct tilings of the batch, keeps the
    fastest, and that plan meets the oracle; a second call with the same
    batch family reuses the choice"""
    from paper_2502_03000_gb300 import autotune
    inst, host, ins, outs = build_batch(torch, 404, 50, dtype)
    bp, times = autotune.tune(inst, ins, outs, "cuda", reps=2)
    assert len(times) >= 2 and all(t > 0 for t in times.values())
    bp()
    torch.cuda.synchronize()
    for i in range(len(inst)):
        check_instance(*inst[i], host[i], outs[i], dtype)
    bp2, times2 = autotune.tune(inst, ins, outs, "cuda", reps=2)
    assert len(times2) == 1 and list(times2)[0] == min(times, key=times.get)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batched_strided_unaligned_operands(torch, dtype):
    """operands as views with leading dimensions larger than K (even and
    odd) and bases one element off alignment: the tensor-core path packs
    them whatever their strides, and meets the oracle"""
    shapes = [(37, 45, 70), (130, 20, 129), (5, 200, 64), (64, 64, 1), (200, 150, 300), (17, 130, 66)]
    inst, host, ins, outs = [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        pa, pb = (1, 3, 8, 0, 5, 2)[i], (2, 0, 1, 7, 4, 9)[i]
        g = E.Graph()
        A = g.input(0, k, m, dtype, ld=k + pa)
        B = g.input(1, k, n, dtype, ld=k + pb)
        C = g.input(2, m, n, "f32")
        nodes, o = g.build(2 * A.t() * B + C, E.trace(A.t() * B))
        inst.append((nodes, o))
        Ah = synth.matrix(1200 + i, 1, k, m, dtype)
        Bh = synth.matrix(1200 + i, 2, k, n, dtype)
        Ch = synth.matrix(1200 + i, 3, m, n, "f32")
        host.append([Ah, Bh, Ch])
        ins.append([to_dev(Ah, dtype, pad=pa, offset=1), to_dev(Bh, dtype, pad=pb, offset=i % 2),
                    to_dev(Ch, "f32")])
        outs.append([ag.empty_colmajor(m, n, torch.float32, "cuda"),
                     torch.zeros(1, dtype=torch.float64, device="cuda")])
    bp = ag.BatchedPlan(inst)
    assert bp.info["tensor_cores"] is True
    bp.bind(ins, outs, "cuda")
    bp()
    torch.cuda.synchronize()
    assert bp.status()[0] == "ok"
    for i in range(len(inst)):
        check_instance(*inst[i], host[i], outs[i], dtype)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("form", ["no_c", "alpha_beta"])
def test_batched_box_heights_and_forms(torch, dtype, form):
    """m and n on both sides of every operand box height (16, 32, 64, 128)
    and of the tile edge, one-element K and several K blocks; the family
    without C (alpha*op(A)*op(B)) and with other alpha and beta"""
    shapes = [(16, 17, 64), (17, 16, 65), (32, 33, 1), (33, 32, 127), (64, 65, 128), (65, 64, 129),
              (128, 129, 200), (129, 128, 8), (255, 257, 2), (1, 300, 70)]
    inst, host, ins, outs = [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        g = E.Graph()
        A = g.input(0, k, m, dtype)
        B = g.input(1, k, n, dtype)
        Ah = synth.matrix(1500 + i, 1, k, m, dtype)
        Bh = synth.matrix(1500 + i, 2, k, n, dtype)
        if form == "no_c":
            nodes, o = g.build(A.t() * B, E.trace(A.t() * B))
            host.append([Ah, Bh])
            ins.append([to_dev(Ah, dtype), to_dev(Bh, dtype)])
        else:
            C = g.input(2, m, n, "f32")
            nodes, o = g.build(0.5 * A.t() * B - 1.5 * C, E.trace(A.t() * B))
            Ch = synth.matrix(1500 + i, 3, m, n, "f32")
            host.append([Ah, Bh, Ch])
            ins.append([to_dev(Ah, dtype), to_dev(Bh, dtype), to_dev(Ch, "f32")])
        inst.append((nodes, o))
        outs.append([ag.empty_colmajor(m, n, torch.float32, "cuda"),
                     torch.zeros(1, dtype=torch.float64, device="cuda")])
    bp = ag.BatchedPlan(inst)
    assert bp.info["tensor_cores"] is True
    bp.bind(ins, outs, "cuda")
    for o in outs:
        o[0].fill_(float("nan"))
    bp()
    torch.cuda.synchronize()
    assert bp.status()[0] == "ok"
    for i in range(len(inst)):
        check_instance(*inst[i], host[i], outs[i], dtype)
