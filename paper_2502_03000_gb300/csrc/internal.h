// Internal structures shared by the planner (host) and the kernel launchers.
// Not part of the public ABI (include/arma_gpu.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/arma_gpu.h"

namespace arma {

constexpr int kMaxIn = 8;       // distinct operands of one fused elementwise pass
constexpr int kMaxOps = 48;     // instructions of one fused elementwise program
constexpr int kMaxStack = 4;    // spill slots of the elementwise accumulator machine
constexpr int kMaxRedBlocks = 2048;  // partial-sum slots of a reduction
constexpr size_t kHeaderBytes = 4096;  // workspace header: status + tickets
constexpr int kMaxTickets = 960;

// --------------------------------------------------------------------------
// References to buffers, resolved at eval time
// --------------------------------------------------------------------------
enum RefKind : int32_t { REF_NONE = 0, REF_INPUT = 1, REF_OUTPUT = 2, REF_WS = 3 };

struct Ref {
  int32_t kind = REF_NONE;
  int32_t pad = 0;
  int64_t idx = 0;   // input slot, output index, or workspace byte offset
  int64_t boff = 0;  // bytes from the buffer's start: a submatrix view read in place
  bool valid() const { return kind != REF_NONE; }
  bool same(const Ref& o) const { return kind == o.kind && idx == o.idx && boff == o.boff; }
};

inline Ref ref_input(int64_t slot) { Ref r; r.kind = REF_INPUT; r.idx = slot; return r; }
inline Ref ref_output(int64_t i) { Ref r; r.kind = REF_OUTPUT; r.idx = i; return r; }
inline Ref ref_ws(int64_t off) { Ref r; r.kind = REF_WS; r.idx = off; return r; }

// limit of one bounded device wait on another CTA's progress, in ns
// (arma_gpu_set_wait_limit_ns; 0: give up at the first unset poll)
uint64_t wait_limit_ns();

inline size_t dtype_size(int dt) { return dt == ARMA_F64 ? 8 : dt == ARMA_F32 ? 4 : 2; }

// --------------------------------------------------------------------------
// K1: fused elementwise + reduction pass (an accumulator machine)
// --------------------------------------------------------------------------
// acc is a per-element register; X_k is operand k at the element; S_j a
// spill slot.  Every instruction updates acc.
enum EwOpcode : int32_t {
  EW_LD = 0,     // acc = X_k
  EW_ADD,        // acc = acc + X_k
  EW_SUB,        // acc = acc - X_k
  EW_RSUB,       // acc = X_k - acc
  EW_MUL,        // acc = acc * X_k
  EW_DIV,        // acc = acc / X_k
  EW_RDIV,       // acc = X_k / acc
  EW_AXPY,       // acc = acc + s * X_k
  EW_SCAL,       // acc = s * acc
  EW_DIVS,       // acc = acc / s
  EW_ADDS,       // acc = acc + s
  EW_NEG,        // acc = -acc
  EW_PUSH,       // S_j = acc
  EW_POPADD,     // acc = S_j + acc
  EW_POPSUB,     // acc = S_j - acc
  EW_POPMUL,     // acc = S_j * acc
  EW_POPDIV,     // acc = S_j / acc
  EW_FMA,        // acc = X_k * X_k2 + acc      (k2 = arg2)
  EW_FNMA,       // acc = -(X_k * X_k2) + acc
  EW_LDP2,       // acc = s * X_k, s = +-2^arg2: exact; FP64 passes scale the exponent field
  EW_NOPS
};

struct EwIns {
  int32_t op;
  int32_t arg;   // operand index k or slot j
  double s;
  float sf = 0.f;  // s as a float pair sf + sl (filled at eval time):
  float sl = 0.f;  //   sf alone is the FP32 scalar of FP32 passes
  int32_t arg2 = 0;  // second operand (EW_FMA, EW_FNMA) or exponent (EW_LDP2)
};

enum EwMode : int32_t { EW_FLAT = 0, EW_GRID = 1, EW_DIAG = 2 };

// operand flags
enum : int32_t { EWF_DIAGMASK = 1 };  // value is zero off the main diagonal

struct EwOperand {
  Ref ref;
  int64_t off = 0;          // element offset of the view from the buffer's base
  int64_t rs = 1, cs = 0;   // element (i, j) at base[off + i*rs + j*cs]
  int32_t dtype = ARMA_F64;
  int32_t flags = 0;
};

struct EwStep {
  int64_t m = 0, n = 0;
  int32_t mode = EW_FLAT;
  int32_t nin = 0, nops = 0;
  EwOperand in[kMaxIn];
  EwIns ops[kMaxOps];
  Ref out;                    // optional matrix store
  int64_t out_ld = 0;
  int32_t out_dtype = ARMA_F64;
  int32_t compute_f64 = 1;    // 1: FP64 arithmetic, 0: FP32
  int32_t red = 0;            // bit0: sum, bit1: sum of squares
  Ref sum_out, norm_out;      // FP64 scalars (norm = sqrt(sum of squares))
  Ref partials;               // 2*kMaxRedBlocks doubles
  int32_t ticket = 0;         // index of the ticket counter in the header
};

// Device-side argument block of K1 (passed by value).
struct EwArgs {
  int64_t m, n;
  int32_t mode, nin, nops, red;
  int32_t compute_f64, out_dtype;
  const void* in[kMaxIn];
  int64_t rs[kMaxIn], cs[kMaxIn];
  int32_t in_dtype[kMaxIn], in_flags[kMaxIn];
  EwIns ops[kMaxOps];
  void* out;
  int64_t out_ld;
  double* partials;
  unsigned int* ticket;
  double* sum_out;
  double* norm_out;
};

cudaError_t launch_ew(const EwArgs& a, cudaStream_t s, int* launches);

// --------------------------------------------------------------------------
// Products
// --------------------------------------------------------------------------
struct MatOperand {
  Ref ref;
  int64_t ld = 0;
  int32_t dtype = ARMA_F64;
  int32_t trans = 0;
};

struct VecOperand {
  Ref ref;
  int64_t inc = 1;
  int32_t dtype = ARMA_F64;
};

// D = alpha * diag(r) * op(A) * op(B) * diag(c) + beta * C
struct GemmStep {
  int64_t m = 0, n = 0, k = 0;
  MatOperand A, B, C, D;    // C optional (beta term); D output (trans ignored)
  double alpha = 1.0, beta = 0.0;
  VecOperand rowscale, colscale;  // optional
  int32_t tier = ARMA_TIER_F64;
  // symmetric product op(A) op(B) = X X^T or X^T X (the paper's run-time
  // analysis that maps A*A^T to xSYRK, Sec. II): 1 when both operands are the
  // same value, one of them transposed (known when planning); 2 when they are
  // two input slots of the same shape and layout, decided at evaluation by
  // comparing the bound pointers
  int32_t sym = 0;
  int32_t nosplit = 0;      // 1: no split-K over CTAs (ARMA_PLAN_NO_SPLITK)
  int32_t split_req = 0;    // K splits asked for (ARMA_PLAN_SPLITS), 0: the library's model
  Ref scratch;              // workspace for operand conversion / split-K partials
  int64_t scratch_bytes = 0;
};

struct GemmArgs {
  int64_t m, n, k;
  const void* A; int64_t lda; int32_t ta, adt;
  const void* B; int64_t ldb; int32_t tb, bdt;
  const void* C; int64_t ldc; int32_t cdt;
  void* D; int64_t ldd; int32_t ddt;
  double alpha, beta;
  const void* rs; int64_t rs_inc; int32_t rsdt;
  const void* cs; int64_t cs_inc; int32_t csdt;
  int32_t tier;
  void* scratch; int64_t scratch_bytes;
  int32_t* status;   // workspace status word (device-side failures)
  const int* skip;   // optional: the kernels return at once when *skip != 0
  int32_t sym;       // 1: A == B, lda == ldb, ta != tb, no C or scalings: only the
                     // lower-triangle tiles are computed, the rest is mirrored
  int32_t nosplit;   // 1: one CTA per output tile over the whole of K (no split-K)
  int32_t split_req; // K splits asked for, 0: the library's model (nosplit wins)
  int32_t reuse_a;   // F64_SLICED: op(A)'s slices are already in scratch (an earlier call
                     // with the same A and scratch)
  int32_t max_ctas;  // tensor-core products: at most this many CTAs (0: one per SM), leaving
                     // SMs to a kernel that runs beside the product
  int32_t no_gemv;   // 1: one-row or one-column products take the product kernels too
};

cudaError_t launch_gemm(const GemmArgs& a, cudaStream_t s, int* launches);
int64_t gemm_scratch_bytes(const GemmStep& g);
int64_t gemm_tc_scratch_bytes(int64_t m, int64_t n, int64_t k, int32_t tier, int32_t split_req = 0);
int gemm_tc_splits(int64_t m, int64_t n, int64_t k, int32_t tier, bool sym, bool nosplit, int32_t split_req = 0);
void gemm_step_shape(const GemmStep& g, int* splits, double* tiles);
int64_t gemm_simt_scratch_bytes(int64_t m, int64_t n, int64_t k, int32_t split_req = 0);
// FP64-accurate products from exact BF16 slices (tier ARMA_TIER_F64_SLICED)
int64_t gemm_ozaki_scratch_bytes(int64_t m, int64_t n, int64_t k);
bool gemm_ozaki_supported(const GemmArgs& a);
cudaError_t launch_gemm_ozaki(const GemmArgs& a, cudaStream_t s, int* launches);

// trace(op(A) * op(B)) -> FP64 scalar.  op(A) is m x k, op(B) is k x n;
// the sum runs over i < min(m, n), l < k.
struct DotStep {
  int64_t m = 0, n = 0, k = 0;
  MatOperand A, B;
  double alpha = 1.0;
  Ref out;
  Ref partials;
  int32_t ticket = 0;
  int32_t per_diag = 0;     // 1: out[i] = alpha * (op(A) op(B))_ii for i < min(m, n) (FP64 vector)
};

struct DotArgs {
  int64_t m, n, k;
  const void* A; int64_t lda; int32_t ta, adt;
  const void* B; int64_t ldb; int32_t tb, bdt;
  double alpha;
  double* out;
  double* partials;
  unsigned int* ticket;
  int32_t per_diag;
};

cudaError_t launch_diagdot(const DotArgs& a, cudaStream_t s, int* launches);
constexpr int DIAGVEC_MAX_CHUNKS = 16;   // K chunks of the per-diagonal product (partials rows)

// --------------------------------------------------------------------------
// Literal-plan helpers and the solve
// --------------------------------------------------------------------------
struct CopyArgs {  // transpose / diagonal build
  int64_t m, n;
  const void* src; int64_t lds; int64_t inc; int32_t sdt;
  void* dst; int64_t ldd; int32_t ddt;
};
cudaError_t launch_transpose(const CopyArgs& a, cudaStream_t s, int* launches);
// D(i, j) = D(j, i) for i < j: the strictly upper triangle of an n x n matrix
// from its lower triangle (the second half of a symmetric product)
cudaError_t launch_mirror_lower(void* D, int64_t n, int64_t ldd, int32_t ddt, cudaStream_t s, int* launches);
cudaError_t launch_diag_build(const CopyArgs& a, cudaStream_t s, int* launches);

// X = inv(A) * B  (n x n, n x nrhs) by blocked LU with partial pivoting
struct SolveStep {
  int64_t n = 0, nrhs = 0;
  MatOperand A, B, X;      // B may be absent: X = inv(A)
  int32_t tier = ARMA_TIER_LU32_IR64;
  int32_t explicit_inverse = 0;  // literal plan: form inv(A) then multiply
  int32_t analyse = 0;     // run-time analysis of A picks the solver (Sec. III (10))
  int32_t max_ir = 10;     // refinement step limit (ARMA_PLAN_REFINE_STEPS)
  int32_t dfma_residual = 0;   // 1: the refinement residual by the DFMA product always
  int32_t no_lookahead = 0;    // 1: the LU factorisation on one stream
  Ref scratch;
  int64_t scratch_bytes = 0;
};

// The solve record in the workspace header (int32 words at byte 16): the
// solver taken and what the analysis of A found.
enum SolveProp : int32_t { SP_PATH = 0, SP_KL = 1, SP_KU = 2, SP_ASYM = 3, SP_ZDIAG = 4, SP_FALLBACK = 5,
                           SP_NONPOS = 6, SP_WORDS = 7 };
constexpr size_t kSolveRecordOffset = 16;

// band solver limits: kl <= 31 keeps the pivot candidates within one warp
constexpr int32_t kBandMaxKl = 31, kBandMaxKu = 32;

struct SolveArgs {
  int64_t n, nrhs;
  const void* A; int64_t lda; int32_t adt;
  const void* B; int64_t ldb; int32_t bdt;   // null: identity
  void* X; int64_t ldx; int32_t xdt;
  int32_t tier;
  void* scratch; int64_t scratch_bytes;
  int32_t* status_code;   // workspace header
  int64_t* status_info;
  int32_t analyse;        // 1: analyse A first and dispatch
  int32_t* props;         // the solve record (SP_WORDS int32)
  int32_t max_ir;         // refinement step limit (1 .. 15)
  int32_t dfma_residual;  // 1: the refinement residual by the DFMA product always
  int32_t no_lookahead;   // 1: the LU factorisation on one stream
};
int64_t solve_scratch_bytes(int64_t n, int64_t nrhs, int32_t tier, int32_t analyse = 0,
                            int32_t dfma_residual = 0);
cudaError_t launch_solve(const SolveArgs& a, cudaStream_t s, int* launches);

struct BandArgs {
  int64_t n, nrhs;
  int32_t kl, ku;
  const void* A; int64_t lda; int32_t adt;
  const void* B; int64_t ldb; int32_t bdt;   // null: identity
  void* X; int64_t ldx; int32_t xdt;
  void* work;             // band_work_bytes() when the band does not fit shared memory
  int32_t in_smem;
  int32_t* status; int64_t* info;
  int32_t refine;         // FP64 data: FP32 factors + FP64 refinement (tridiagonal)
  int32_t* fallback;      // set when that refinement gives up
  const int32_t* gate;    // the kernel runs only when *gate != 0 (null: always)
};
int64_t band_work_bytes(int64_t n, int64_t nrhs, int32_t kl, int32_t ku, int32_t es);
cudaError_t launch_analyse(const void* A, int64_t lda, int32_t adt, int64_t n, int32_t* props, cudaStream_t s,
                           int* launches);
cudaError_t launch_set_props(int32_t* props, int32_t path, int32_t* status, int64_t* info, int64_t singular_at,
                             cudaStream_t s, int* launches);
cudaError_t launch_diag_solve(const SolveArgs& a, bool f64, cudaStream_t s, int* launches);
cudaError_t launch_band_solve(BandArgs a, bool f64, cudaStream_t s, int* launches);

// --------------------------------------------------------------------------
// Plan
// --------------------------------------------------------------------------
enum StepKind : int32_t { ST_EW = 0, ST_GEMM, ST_DOT, ST_TRANSPOSE, ST_DIAGBUILD, ST_SOLVE };

struct Step {
  StepKind kind = ST_EW;
  EwStep ew;
  GemmStep gemm;
  DotStep dot;
  SolveStep solve;
  // ST_TRANSPOSE / ST_DIAGBUILD
  int64_t cm = 0, cn = 0;
  MatOperand csrc, cdst;
  int64_t cinc = 1;
  std::string note;         // decision-log text
  double flops = 0, bytes = 0;  // algorithmic work of the step
};

struct OutInfo {
  int64_t rows, cols;
  int32_t dtype;
  int32_t scalar;
};

// A batch of instances that all reduce to one product with folded scalars
// (and optionally the trace of that product), evaluated by the grouped kernel.
struct BatchedInfo {
  int32_t count = 0;
  int32_t slot_a = 0, slot_b = 0, slot_c = -1, out_d = 0, out_t = -1;
  int32_t n_slots = 0, n_outs = 0;
  int32_t ta = 0, tb = 0, abdt = ARMA_F32, cdt = ARMA_F32, ddt = ARMA_F32;
  int32_t tc = 0;           // 128 x 128 tiles on the tensor cores
  double alpha = 1.0, beta = 0.0;
  std::vector<int64_t> m, n, k, lda, ldb, ldc;
  std::vector<int32_t> tile;
  std::vector<int64_t> first_tile;
  std::vector<int32_t> tile_prob;
  std::vector<uint32_t> tile_code;
  std::vector<int32_t> tile_order;   // tiles by decreasing work (longest first)
  int64_t tiles = 0;
  // tensor cores: packed operand rows (K-block-major, 64 BF16 per row)
  std::vector<int64_t> pa, pb;       // per problem: first packed row of op(A), op(B)^T
  int64_t rows_a = 0, rows_b = 0;    // packed rows per slice
  int32_t slices = 1;                // 1 (BF16) or 3 (FP32 as exact BF16 slices)
  std::vector<int32_t> pack_items;   // pack work: (2 problem + operand, first row, rows) triplets
  size_t pack_off = 0, pack_bytes = 0;   // the packed arrays in the workspace
};

}  // namespace arma

struct arma_plan {
  std::vector<arma::Step> steps;
  std::vector<arma::OutInfo> outs;
  std::vector<int64_t> in_align_need;  // per slot: required byte alignment (0 = none)
  int32_t n_slots = 0;
  size_t ws_bytes = arma::kHeaderBytes;
  int32_t tickets = 0;
  uint32_t flags = 0;
  int32_t tier = 0;
  std::string log;          // JSON decision log
  double flops = 0, bytes = 0;
  bool batched = false;
  arma::BatchedInfo bi;
};
