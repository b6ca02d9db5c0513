#include <cstdio>
// C-ABI entry points (include/arma_gpu.h) and the executor that enqueues a
// plan's steps on the caller's stream.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "grouped.h"
#include "internal.h"

namespace arma {
arma_status plan_expression(const arma_expr* e, arma_plan* p, std::string* msg);
arma_status plan_batched(const arma_expr* exprs, int32_t count, arma_plan* p);
arma_status plan_features(const arma_plan* p, float* out, int32_t n);
arma_status plan_heuristic(const arma_plan* p, double* seconds);
arma_status chain_order_api(int32_t n, const int64_t* dims, int32_t method, int32_t* splits,
                            uint64_t* cost);
arma_status plan_candidates_api(const arma_expr* e, arma_plan** plans, int32_t capacity, int32_t* count);
arma_status cost_model_load(const float* params, int32_t F, int32_t H, const float* mean, const float* scale,
                            double guard, double margin);
void cost_model_clear();
arma_status cost_model_predict(const arma_plan* p, double* seconds);
}  // namespace arma

using namespace arma;

namespace {
std::atomic<uint64_t>& wait_ns_setting();
}

uint64_t arma::wait_limit_ns() { return wait_ns_setting().load(std::memory_order_relaxed); }

namespace {

struct Bind {
  const void* const* in;
  void* const* out;
  char* ws;
  int32_t n_slots;
  int32_t n_out;
};

const void* cptr(const Bind& b, const Ref& r) {
  switch (r.kind) {
    case REF_INPUT: return static_cast<const char*>(b.in[r.idx]) + r.boff;
    case REF_OUTPUT: return static_cast<const char*>(b.out[r.idx]) + r.boff;
    case REF_WS: return b.ws + r.idx + r.boff;
    default: return nullptr;
  }
}
void* mptr(const Bind& b, const Ref& r) { return const_cast<void*>(cptr(b, r)); }

thread_local char g_last_cuda[160] = "";

std::atomic<uint64_t>& wait_ns_setting() {
  static std::atomic<uint64_t> v{2000000000ull};
  return v;
}

// records the CUDA error for arma_gpu_last_cuda_error() and maps it
arma_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ARMA_OK;
  snprintf(g_last_cuda, sizeof g_last_cuda, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return ARMA_ERR_CUDA;
}

arma_status run_step(const Step& st, const Bind& b, cudaStream_t s, int* launches) {
  unsigned int* tickets = reinterpret_cast<unsigned int*>(b.ws + 64);
  switch (st.kind) {
    case ST_EW: {
      const EwStep& e = st.ew;
      EwArgs a;
      std::memset(&a, 0, sizeof a);
      a.m = e.m; a.n = e.n;
      a.mode = e.mode; a.nin = e.nin; a.nops = e.nops; a.red = e.red;
      a.compute_f64 = e.compute_f64; a.out_dtype = e.out_dtype;
      for (int k = 0; k < e.nin; ++k) {
        a.in[k] = static_cast<const char*>(cptr(b, e.in[k].ref)) + e.in[k].off * (int64_t)dtype_size(e.in[k].dtype);
        a.rs[k] = e.in[k].rs; a.cs[k] = e.in[k].cs;
        a.in_dtype[k] = e.in[k].dtype; a.in_flags[k] = e.in[k].flags;
      }
      for (int i = 0; i < e.nops; ++i) {
        a.ops[i] = e.ops[i];
        a.ops[i].sf = static_cast<float>(e.ops[i].s);
        a.ops[i].sl = static_cast<float>(e.ops[i].s - static_cast<double>(a.ops[i].sf));
      }
      a.out = e.out.valid() ? mptr(b, e.out) : nullptr;
      a.out_ld = e.out_ld;
      a.partials = e.partials.valid() ? reinterpret_cast<double*>(mptr(b, e.partials)) : nullptr;
      a.ticket = tickets + e.ticket;
      a.sum_out = e.sum_out.valid() ? reinterpret_cast<double*>(mptr(b, e.sum_out)) : nullptr;
      a.norm_out = e.norm_out.valid() ? reinterpret_cast<double*>(mptr(b, e.norm_out)) : nullptr;
      return cuda_status(launch_ew(a, s, launches));
    }
    case ST_GEMM: {
      const GemmStep& g = st.gemm;
      GemmArgs a;
      std::memset(&a, 0, sizeof a);
      a.m = g.m; a.n = g.n; a.k = g.k;
      a.A = cptr(b, g.A.ref); a.lda = g.A.ld; a.ta = g.A.trans; a.adt = g.A.dtype;
      a.B = cptr(b, g.B.ref); a.ldb = g.B.ld; a.tb = g.B.trans; a.bdt = g.B.dtype;
      a.C = g.C.ref.valid() ? cptr(b, g.C.ref) : nullptr; a.ldc = g.C.ld; a.cdt = g.C.dtype;
      a.D = mptr(b, g.D.ref); a.ldd = g.D.ld; a.ddt = g.D.dtype;
      a.alpha = g.alpha; a.beta = g.beta;
      a.rs = g.rowscale.ref.valid() ? cptr(b, g.rowscale.ref) : nullptr;
      a.rs_inc = g.rowscale.inc; a.rsdt = g.rowscale.dtype;
      a.cs = g.colscale.ref.valid() ? cptr(b, g.colscale.ref) : nullptr;
      a.cs_inc = g.colscale.inc; a.csdt = g.colscale.dtype;
      a.tier = g.tier;
      a.scratch = g.scratch.valid() ? mptr(b, g.scratch) : nullptr;
      a.scratch_bytes = g.scratch_bytes;
      a.status = reinterpret_cast<int32_t*>(b.ws);
      // the run-time half of the symmetric-product check: two slots bound
      // to the same memory (launch_gemm re-checks every condition)
      a.sym = g.sym == 1 || (g.sym == 2 && a.A == a.B) ? 1 : 0;
      a.nosplit = g.nosplit;
      a.split_req = g.split_req;
      return cuda_status(launch_gemm(a, s, launches));
    }
    case ST_DOT: {
      const DotStep& d = st.dot;
      DotArgs a;
      std::memset(&a, 0, sizeof a);
      a.m = d.m; a.n = d.n; a.k = d.k;
      a.A = cptr(b, d.A.ref); a.lda = d.A.ld; a.ta = d.A.trans; a.adt = d.A.dtype;
      a.B = cptr(b, d.B.ref); a.ldb = d.B.ld; a.tb = d.B.trans; a.bdt = d.B.dtype;
      a.alpha = d.alpha;
      a.out = reinterpret_cast<double*>(mptr(b, d.out));
      a.partials = reinterpret_cast<double*>(mptr(b, d.partials));
      a.ticket = tickets + d.ticket;
      a.per_diag = d.per_diag;
      return cuda_status(launch_diagdot(a, s, launches));
    }
    case ST_TRANSPOSE:
    case ST_DIAGBUILD: {
      CopyArgs a;
      std::memset(&a, 0, sizeof a);
      a.m = st.cm; a.n = st.cn;
      a.src = cptr(b, st.csrc.ref); a.lds = st.csrc.ld; a.inc = st.cinc; a.sdt = st.csrc.dtype;
      a.dst = mptr(b, st.cdst.ref); a.ldd = st.cdst.ld; a.ddt = st.cdst.dtype;
      return cuda_status(st.kind == ST_TRANSPOSE ? launch_transpose(a, s, launches)
                                                 : launch_diag_build(a, s, launches));
    }
    case ST_SOLVE: {
      const SolveStep& v = st.solve;
      SolveArgs a;
      std::memset(&a, 0, sizeof a);
      a.n = v.n; a.nrhs = v.nrhs;
      a.A = cptr(b, v.A.ref); a.lda = v.A.ld; a.adt = v.A.dtype;
      a.B = v.B.ref.valid() ? cptr(b, v.B.ref) : nullptr; a.ldb = v.B.ld; a.bdt = v.B.dtype;
      a.X = mptr(b, v.X.ref); a.ldx = v.X.ld; a.xdt = v.X.dtype;
      a.tier = v.tier;
      a.scratch = mptr(b, v.scratch); a.scratch_bytes = v.scratch_bytes;
      a.status_code = reinterpret_cast<int32_t*>(b.ws);
      a.status_info = reinterpret_cast<int64_t*>(b.ws + 8);
      a.analyse = v.analyse;
      a.props = reinterpret_cast<int32_t*>(b.ws + kSolveRecordOffset);
      a.max_ir = v.max_ir;
      a.dfma_residual = v.dfma_residual;
      a.no_lookahead = v.no_lookahead;
      return cuda_status(launch_solve(a, s, launches));
    }
  }
  return ARMA_ERR_INVALID;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" {

// ARMA_PLAN_LOG set to anything but "" or "0": every arma_gpu_plan call
// writes one line to stderr, the plan's decision log or the status it failed
// with (read once per process).
static bool plan_log_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("ARMA_PLAN_LOG");
    return v != nullptr && *v != 0 && std::strcmp(v, "0") != 0;
  }();
  return on;
}

arma_status arma_gpu_plan(const arma_expr* expr, arma_plan** plan) {
  if (!plan) return ARMA_ERR_INVALID;
  *plan = nullptr;
  if (!expr) return ARMA_ERR_INVALID;
  arma_plan* p = new (std::nothrow) arma_plan();
  if (!p) return ARMA_ERR_INVALID;
  arma_status s;
  try {
    s = plan_expression(expr, p, nullptr);
  } catch (...) {
    s = ARMA_ERR_INVALID;
  }
  if (plan_log_enabled()) {
    if (s == ARMA_OK) std::fprintf(stderr, "arma_gpu_plan: %s\n", p->log.c_str());
    else std::fprintf(stderr, "arma_gpu_plan: failed: %s\n", arma_gpu_status_string(s));
  }
  if (s != ARMA_OK) {
    delete p;
    return s;
  }
  *plan = p;
  return ARMA_OK;
}

arma_status arma_gpu_plan_workspace(const arma_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return ARMA_ERR_INVALID;
  *bytes = plan->ws_bytes;
  return ARMA_OK;
}

arma_status arma_gpu_output_info(const arma_plan* plan, int32_t i, int64_t* rows, int64_t* cols,
                                 int32_t* dtype) {
  if (!plan || i < 0 || i >= (int32_t)plan->outs.size()) return ARMA_ERR_INVALID;
  if (rows) *rows = plan->outs[i].rows;
  if (cols) *cols = plan->outs[i].cols;
  if (dtype) *dtype = plan->outs[i].dtype;
  return ARMA_OK;
}

arma_status arma_gpu_eval(const arma_plan* plan, const void* const* in_ptrs, void* const* out_ptrs,
                          void* workspace, size_t workspace_bytes, void* stream) {
  if (!plan || !out_ptrs || (plan->n_slots > 0 && !in_ptrs)) return ARMA_ERR_INVALID;
  if (!workspace || workspace_bytes < plan->ws_bytes) return ARMA_ERR_WORKSPACE;
  if (!aligned(workspace, 256)) return ARMA_ERR_ALIGN;
  for (size_t o = 0; o < plan->outs.size(); ++o) {
    bool empty = !plan->outs[o].scalar && (plan->outs[o].rows == 0 || plan->outs[o].cols == 0);
    if (!out_ptrs[o] && !empty) return ARMA_ERR_INVALID;
    size_t es = plan->outs[o].scalar ? 8 : dtype_size(plan->outs[o].dtype);
    if (!aligned(out_ptrs[o], es)) return ARMA_ERR_ALIGN;
  }
  for (int32_t k = 0; k < plan->n_slots; ++k)
    if (in_ptrs[k] && !aligned(in_ptrs[k], 2)) return ARMA_ERR_ALIGN;
  Bind b{in_ptrs, out_ptrs, static_cast<char*>(workspace), plan->n_slots,
         (int32_t)plan->outs.size()};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaError_t e = cudaMemsetAsync(workspace, 0, kHeaderBytes, s)) return cuda_status(e);
  // NVTX ranges name the evaluation and each of its steps on a profiler's
  // timeline (the GPU-side counterpart of the plan's decision log); with no
  // profiler attached the calls return at once
  static const char* const kStepRange[] = {"arma:ew", "arma:gemm", "arma:diagdot",
                                           "arma:transpose", "arma:diagbuild", "arma:solve"};
  nvtxRangePushA("arma_gpu_eval");
  int launches = 0;
  arma_status r = ARMA_OK;
  for (const Step& st : plan->steps) {
    const int k = (int)st.kind;
    nvtxRangePushA(k >= 0 && k <= ST_SOLVE ? kStepRange[k] : "arma:step");
    r = run_step(st, b, s, &launches);
    nvtxRangePop();
    if (r != ARMA_OK) break;
  }
  nvtxRangePop();
  return r;
}

arma_status arma_gpu_eval_status(const arma_plan* plan, const void* workspace, void* stream,
                                 int64_t* info) {
  if (!plan || !workspace) return ARMA_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t hdr[2] = {0, 0};
  if (cudaError_t e = cudaStreamSynchronize(s)) return cuda_status(e);
  if (cudaError_t e = cudaMemcpy(hdr, workspace, sizeof hdr, cudaMemcpyDeviceToHost)) return cuda_status(e);
  int32_t code = static_cast<int32_t>(hdr[0] & 0xffffffff);
  if (info) *info = hdr[1];
  if (code == 0) return ARMA_OK;
  return static_cast<arma_status>(code);
}

arma_status arma_gpu_eval_solve_path(const arma_plan* plan, const void* workspace, void* stream,
                                     int32_t* path, int32_t* kl, int32_t* ku, int32_t* symmetric) {
  if (!plan || !workspace) return ARMA_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t rec[SP_WORDS] = {};
  if (cudaError_t e = cudaStreamSynchronize(s)) return cuda_status(e);
  if (cudaError_t e = cudaMemcpy(rec, static_cast<const char*>(workspace) + kSolveRecordOffset, sizeof rec,
                                 cudaMemcpyDeviceToHost))
    return cuda_status(e);
  if (path) *path = rec[SP_PATH];
  if (kl) *kl = rec[SP_KL];
  if (ku) *ku = rec[SP_KU];
  if (symmetric) *symmetric = rec[SP_PATH] != ARMA_SOLVE_NONE && rec[SP_ASYM] == 0 ? 1 : 0;
  return ARMA_OK;
}

arma_status arma_gpu_plan_info(const arma_plan* plan, char* buf, size_t len, size_t* needed) {
  if (!plan) return ARMA_ERR_INVALID;
  if (needed) *needed = plan->log.size() + 1;
  if (buf && len > 0) {
    size_t n = plan->log.size() < len - 1 ? plan->log.size() : len - 1;
    std::memcpy(buf, plan->log.data(), n);
    buf[n] = 0;
  }
  return ARMA_OK;
}

void arma_gpu_plan_free(arma_plan* plan) { delete plan; }

const char* arma_gpu_last_cuda_error(void) { return g_last_cuda; }

uint64_t arma_gpu_set_wait_limit_ns(uint64_t ns) { return wait_ns_setting().exchange(ns); }

arma_status arma_gpu_device_address(const void* p, void** dptr) {
  if (!dptr) return ARMA_ERR_INVALID;
  *dptr = nullptr;
  if (!p) return ARMA_ERR_INVALID;
  cudaPointerAttributes at;
  std::memset(&at, 0, sizeof at);
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return ARMA_ERR_INVALID;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    *dptr = const_cast<void*>(p);
    return ARMA_OK;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *dptr = at.devicePointer;
    return ARMA_OK;
  }
  return ARMA_ERR_INVALID;
}

const char* arma_gpu_status_string(arma_status s) {
  switch (s) {
    case ARMA_OK: return "ok";
    case ARMA_ERR_INVALID: return "invalid argument or malformed expression";
    case ARMA_ERR_SHAPE: return "non-conforming operand sizes";
    case ARMA_ERR_DTYPE: return "element types do not match";
    case ARMA_ERR_ALIGN: return "device pointer misaligned";
    case ARMA_ERR_WORKSPACE: return "workspace missing or too small";
    case ARMA_ERR_SINGULAR: return "matrix is singular (zero pivot)";
    case ARMA_ERR_NOCONVERGE: return "iterative refinement did not converge";
    case ARMA_ERR_CUDA: return "CUDA runtime error";
    case ARMA_ERR_UNSUPPORTED: return "expression not supported";
    case ARMA_ERR_TIMEOUT: return "a bounded device-side wait ran out";
  }
  return "unknown status";
}

arma_status arma_gpu_chain_order(int32_t n, const int64_t* dims, int32_t method, int32_t* splits,
                                 uint64_t* cost) {
  return chain_order_api(n, dims, method, splits, cost);
}

arma_status arma_gpu_plan_features(const arma_plan* plan, float* features, int32_t n) {
  return plan_features(plan, features, n);
}

arma_status arma_gpu_plan_heuristic_cost(const arma_plan* plan, double* seconds) {
  return plan_heuristic(plan, seconds);
}

arma_status arma_gpu_plan_candidates(const arma_expr* expr, arma_plan** plans, int32_t capacity,
                                     int32_t* count) {
  try {
    return plan_candidates_api(expr, plans, capacity, count);
  } catch (...) {
    return ARMA_ERR_INVALID;
  }
}

arma_status arma_gpu_cost_model_load(const float* params, int32_t features, int32_t hidden, const float* mean,
                                     const float* scale, double guard, double margin) {
  try {
    return cost_model_load(params, features, hidden, mean, scale, guard, margin);
  } catch (...) {
    return ARMA_ERR_INVALID;
  }
}

void arma_gpu_cost_model_clear(void) { cost_model_clear(); }

arma_status arma_gpu_cost_model_predict(const arma_plan* plan, double* seconds) {
  return cost_model_predict(plan, seconds);
}

arma_status arma_gpu_plan_batched(const arma_expr* exprs, int32_t count, arma_plan** plan) {
  if (!plan) return ARMA_ERR_INVALID;
  *plan = nullptr;
  arma_plan* p = new (std::nothrow) arma_plan();
  if (!p) return ARMA_ERR_INVALID;
  arma_status s;
  try {
    s = plan_batched(exprs, count, p);
  } catch (...) {
    s = ARMA_ERR_INVALID;
  }
  if (s != ARMA_OK) {
    delete p;
    return s;
  }
  *plan = p;
  return ARMA_OK;
}

static size_t table_layout(const BatchedInfo& b, size_t* probs_off, size_t* prob_off, size_t* code_off,
                           size_t* order_off, size_t* rec_off = nullptr, size_t* item_off = nullptr) {
  size_t off = 0;
  *probs_off = off;
  off += (size_t)b.count * sizeof(GroupedProblem);
  off = (off + 255) / 256 * 256;
  *prob_off = off;
  off += (size_t)b.tiles * sizeof(int32_t);
  off = (off + 255) / 256 * 256;
  *code_off = off;
  off += (size_t)b.tiles * sizeof(uint32_t);
  off = (off + 255) / 256 * 256;
  *order_off = off;
  off += (size_t)b.tiles * sizeof(int32_t);
  off = (off + 255) / 256 * 256;
  if (rec_off) *rec_off = off;
  if (b.tc) off += (size_t)b.tiles * sizeof(GroupedTile);
  off = (off + 255) / 256 * 256;
  if (item_off) *item_off = off;
  if (b.tc) off += b.pack_items.size() * sizeof(int32_t);
  return (off + 255) / 256 * 256;
}

arma_status arma_gpu_batched_table_bytes(const arma_plan* plan, size_t* bytes) {
  if (!plan || !bytes || !plan->batched) return ARMA_ERR_INVALID;
  size_t a, b, c, d;
  *bytes = table_layout(plan->bi, &a, &b, &c, &d);
  return ARMA_OK;
}

arma_status arma_gpu_batched_table_fill(const arma_plan* plan, const void* const* in_ptrs,
                                        void* const* out_ptrs, void* host_table) {
  if (!plan || !plan->batched || !in_ptrs || !out_ptrs || !host_table) return ARMA_ERR_INVALID;
  const BatchedInfo& b = plan->bi;
  size_t po, pr, pc, pd, pt, pi;
  table_layout(b, &po, &pr, &pc, &pd, &pt, &pi);
  char* base = static_cast<char*>(host_table);
  GroupedProblem* probs = reinterpret_cast<GroupedProblem*>(base + po);
  for (int32_t i = 0; i < b.count; ++i) {
    const void* const* in = in_ptrs + (size_t)i * b.n_slots;
    void* const* out = out_ptrs + (size_t)i * b.n_outs;
    GroupedProblem& g = probs[i];
    g.m = b.m[i]; g.n = b.n[i]; g.k = b.k[i];
    g.A = in[b.slot_a]; g.lda = b.lda[i];
    g.B = in[b.slot_b]; g.ldb = b.ldb[i];
    g.C = b.slot_c >= 0 ? in[b.slot_c] : nullptr; g.ldc = b.ldc[i];
    g.D = out[b.out_d]; g.ldd = g.m > 0 ? g.m : 1;
    g.trace = b.out_t >= 0 ? static_cast<double*>(out[b.out_t]) : nullptr;
    g.first_tile = b.first_tile[i];
    g.tile = b.tile[i];
    g.pad = 0;
    g.pa = b.tc ? b.pa[i] : 0;
    g.pb = b.tc ? b.pb[i] : 0;
    if ((!g.A || !g.B || !g.D) && g.m * g.n > 0) return ARMA_ERR_INVALID;
  }
  std::memcpy(base + pr, b.tile_prob.data(), b.tile_prob.size() * sizeof(int32_t));
  std::memcpy(base + pc, b.tile_code.data(), b.tile_code.size() * sizeof(uint32_t));
  std::memcpy(base + pd, b.tile_order.data(), b.tile_order.size() * sizeof(int32_t));
  if (b.tc) {
    GroupedTile* recs = reinterpret_cast<GroupedTile*>(base + pt);
    for (int64_t pos = 0; pos < b.tiles; ++pos) {
      const int32_t t = b.tile_order[(size_t)pos];
      const GroupedProblem& g = probs[b.tile_prob[(size_t)t]];
      if (g.m > INT32_MAX || g.n > INT32_MAX || g.k > INT32_MAX || g.ldc > INT32_MAX)
        return ARMA_ERR_UNSUPPORTED;
      GroupedTile& r = recs[pos];
      std::memset(&r, 0, sizeof r);
      r.C = g.C; r.D = g.D;
      r.m = (int32_t)g.m; r.n = (int32_t)g.n; r.k = (int32_t)g.k;
      r.ldc = (int32_t)g.ldc;
      r.tm = (uint16_t)(b.tile_code[(size_t)t] >> 16);
      r.tn = (uint16_t)(b.tile_code[(size_t)t] & 0xFFFFu);
      r.t = t;
      // the tile's rows in the packed arrays, and the smallest box that
      // covers the rows it has (rows past them only feed outputs that are
      // never stored)
      r.ya = (int32_t)(g.pa + 128 * (int64_t)r.tm);
      r.yb = (int32_t)(g.pb + 128 * (int64_t)r.tn);
      r.sa = r.m;
      r.sb = r.n;
      auto box = [](int64_t rows) -> uint16_t { return rows <= 16 ? 16 : rows <= 32 ? 32 : rows <= 64 ? 64 : 128; };
      r.ha = box(g.m - 128 * (int64_t)r.tm);
      r.hb = box(g.n - 128 * (int64_t)r.tn);
    }
    std::memcpy(base + pi, b.pack_items.data(), b.pack_items.size() * sizeof(int32_t));
  }
  return ARMA_OK;
}

arma_status arma_gpu_eval_batched(const arma_plan* plan, const void* device_table, void* workspace,
                                  size_t workspace_bytes, void* stream) {
  if (!plan || !plan->batched || !device_table) return ARMA_ERR_INVALID;
  if (!workspace || workspace_bytes < plan->ws_bytes) return ARMA_ERR_WORKSPACE;
  const BatchedInfo& b = plan->bi;
  size_t po, pr, pc, pd, pt, pi;
  table_layout(b, &po, &pr, &pc, &pd, &pt, &pi);
  const char* base = static_cast<const char*>(device_table);
  GroupedArgs g;
  std::memset(&g, 0, sizeof g);
  g.count = b.count; g.tiles = b.tiles;
  g.probs = reinterpret_cast<const GroupedProblem*>(base + po);
  g.tile_prob = reinterpret_cast<const int32_t*>(base + pr);
  g.tile_code = reinterpret_cast<const uint32_t*>(base + pc);
  g.tile_order = reinterpret_cast<const int32_t*>(base + pd);
  g.recs = b.tc ? reinterpret_cast<const GroupedTile*>(base + pt) : nullptr;
  g.next_tile = reinterpret_cast<unsigned int*>(static_cast<char*>(workspace) + 16);
  g.ta = b.ta; g.tb = b.tb; g.abdt = b.abdt; g.cdt = b.cdt; g.ddt = b.ddt;
  g.alpha = b.alpha; g.beta = b.beta;
  g.alpha_f = (float)b.alpha; g.beta_f = (float)b.beta;
  g.trace_partials = b.out_t >= 0 ? reinterpret_cast<double*>(static_cast<char*>(workspace) + kHeaderBytes) : nullptr;
  g.tc = b.tc;
  g.status = static_cast<int32_t*>(workspace);
  if (b.tc) {
    g.pack_a = static_cast<char*>(workspace) + b.pack_off;
    g.pack_b = static_cast<char*>(workspace) + b.pack_off + (size_t)b.slices * (size_t)b.rows_a * 128;
    g.rows_a = b.rows_a;
    g.rows_b = b.rows_b;
    g.slices = b.slices;
    g.pack_items = reinterpret_cast<const int32_t*>(base + pi);
    g.n_items = (int64_t)(b.pack_items.size() / 3);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // status, info and the tile counter start at zero
  if (cudaError_t e = cudaMemsetAsync(workspace, 0, 32, s)) return cuda_status(e);
  int launches = 0;
  return cuda_status(launch_grouped(g, s, &launches));
}

}  // extern "C"
