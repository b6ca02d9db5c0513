"""Host logic of the batched tensor-core path, no GPU: the device table that
arma_gpu_batched_table_fill writes.  The pack kernel's work items must
cover every packed row of every operand exactly once, in source order; the
packed row offsets must be prefix sums of R * ceil(K / 64); every tile
record must carry the rows and box heights its problem's shape gives."""
import ctypes

import numpy as np
import pytest

import paper_2502_03000_gb300 as ag
import synth
from paper_2502_03000_gb300 import expr as E

PROB_BYTES = 128   # GroupedProblem
REC_BYTES = 64     # GroupedTile


def up256(x):
    return (x + 255) // 256 * 256


def filled_table(shapes, dtype):
    inst = [E.config_batched_instance(m, n, k, dtype) for m, n, k in shapes]
    bp = ag.BatchedPlan(inst)
    assert bp.info["tensor_cores"] is True
    count = len(shapes)
    # stand-in addresses: the fill only records them
    ins = (ctypes.c_void_p * (count * bp.n_slots))(*[0x10000 * (i + 1) for i in range(count * bp.n_slots)])
    outs = (ctypes.c_void_p * (count * bp.n_outs))(*[0x90000000 + 0x10000 * i for i in range(count * bp.n_outs)])
    host = np.zeros(bp.table_bytes, dtype=np.uint8)
    assert ag.lib().arma_gpu_batched_table_fill(bp._h, ins, outs, host.ctypes.data_as(ctypes.c_void_p)) == 0
    return bp, host


def parse(bp, host, shapes):
    count = len(shapes)
    tiles = bp.info["tiles"]
    off = 0
    probs = host[off:off + count * PROB_BYTES].view(np.int64).reshape(count, PROB_BYTES // 8)
    off = up256(off + count * PROB_BYTES)
    off = up256(off + tiles * 4)   # tile -> problem
    off = up256(off + tiles * 4)   # tile codes
    off = up256(off + tiles * 4)   # processing order
    recs = host[off:off + tiles * REC_BYTES]
    off = up256(off + tiles * REC_BYTES)
    items = host[off:].view(np.int32)
    items = items[:len(items) // 3 * 3].reshape(-1, 3)
    items = items[items[:, 2] > 0]   # the table's zero padding ends the list
    return probs, recs, items


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_pack_items_cover_every_row_once(dtype):
    shapes = [(int(m), int(n), int(k)) for m, n, k in zip(synth.log_uniform_ints(3, 1, 60, 1, 700),
                                                           synth.log_uniform_ints(3, 2, 60, 1, 700),
                                                           synth.log_uniform_ints(3, 3, 60, 1, 900))]
    shapes += [(1, 1, 1), (128, 128, 64), (129, 257, 65), (64, 64, 4096)]
    bp, host = filled_table(shapes, dtype)
    probs, recs, items = parse(bp, host, shapes)
    # packed row offsets (int64 fields 14 and 15 of a problem record: pa, pb)
    pa = pb = 0
    for i, (m, n, k) in enumerate(shapes):
        nkb = (k + 63) // 64
        assert probs[i, 0] == m and probs[i, 1] == n and probs[i, 2] == k
        assert probs[i, 14] == pa and probs[i, 15] == pb
        pa += m * nkb
        pb += n * nkb
    # every row of every operand exactly once, in order, runs of about 64 packed rows
    seen = {}
    for code, r0, nr in items:
        i, op = int(code) >> 1, int(code) & 1
        m, n, k = shapes[i]
        R, nkb = (n if op else m), (k + 63) // 64
        assert nr == min(max(1, 64 // nkb), R - r0)
        seen.setdefault((i, op), []).append((int(r0), int(nr)))
    for i, (m, n, k) in enumerate(shapes):
        for op, R in ((0, m), (1, n)):
            runs = seen[(i, op)]
            pos = 0
            for r0, nr in runs:
                assert r0 == pos
                pos += nr
            assert pos == R


def test_tile_records_rows_and_boxes():
    shapes = [(16, 17, 64), (17, 16, 65), (33, 300, 1), (200, 129, 130), (640, 64, 8)]
    bp, host = filled_table(shapes, "bf16")
    probs, recs, _ = parse(bp, host, shapes)
    r = recs.reshape(-1, REC_BYTES)

    def i32(row, off):
        return int(row[off:off + 4].view(np.int32)[0])

    def u16(row, off):
        return int(row[off:off + 2].view(np.uint16)[0])

    def box(rows):
        return 16 if rows <= 16 else 32 if rows <= 32 else 64 if rows <= 64 else 128

    # record: C, D (0, 8), ya, yb (16, 20), sa, sb (24, 28), m, n, k, ldc
    # (32 .. 44), tm, tn (48, 50), t (52), ha, hb (56, 58)
    counted = 0
    for row in r:
        m, n, k = i32(row, 32), i32(row, 36), i32(row, 40)
        i = shapes.index((m, n, k))
        tm, tn = u16(row, 48), u16(row, 50)
        assert i32(row, 24) == m and i32(row, 28) == n       # packed rows per K block
        assert i32(row, 16) == probs[i, 14] + 128 * tm        # ya
        assert i32(row, 20) == probs[i, 15] + 128 * tn        # yb
        assert u16(row, 56) == box(m - 128 * tm)              # ha
        assert u16(row, 58) == box(n - 128 * tn)              # hb
        counted += 1
    assert counted == sum(((m + 127) // 128) * ((n + 127) // 128) for m, n, _ in shapes)


def test_batched_planning_checks():
    """arma_gpu_plan_batched: the conformance check per instance, one
    expression family per batch (same nodes and scalars, sizes free), FP32 or
    BF16 operands; operands that are not K-contiguous take the SIMT kernel."""
    import copy

    def status(inst):
        try:
            bp = ag.BatchedPlan(inst)
        except ag.ArmaError as e:
            return e.status
        return "tc" if bp.info["tensor_cores"] else "simt"

    n, o = E.config_batched_instance(20, 30, 40, "f32")
    assert status([(n, o), E.config_batched_instance(64, 8, 512, "f32")]) == "tc"
    assert status([E.config_batched_instance(20, 30, 40, "bf16")]) == "tc"
    bad = copy.deepcopy(n)
    bad[1]["rows"] = bad[1]["ld"] = 41                      # B's K differs from A's
    assert status([(bad, o)]) == "shape"
    assert status([]) == "invalid"
    assert status([E.config_batched_instance(20, 30, 40, "f64")]) == "dtype"
    assert status([E.config_fused(16, "f32")]) == "unsupported"
    assert status([(n, o), E.config_fused(16, "f32")]) == "unsupported"
    other = copy.deepcopy(n)
    other[4]["s"] = 3.0                                     # another alpha: another family
    assert status([(n, o), (other, o)]) == "unsupported"
    # A stored m x k (op(A) = A, K along its rows): planned, on the SIMT kernel
    nt = copy.deepcopy(n)
    nt[0] = {"op": "input", "slot": 0, "rows": 20, "cols": 40, "dtype": "f32", "ld": 20}
    nt[3] = {"op": "scale", "a": 0, "s": 1.0}
    nt[7] = {"op": "scale", "a": 0, "s": 1.0}
    assert status([(nt, o)]) == "simt"
