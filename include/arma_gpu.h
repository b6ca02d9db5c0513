/*
 * arma_gpu.h -- C ABI of a GB300 (sm_103a) evaluator for compound
 * linear-algebra expressions.
 *
 * The method follows Sanderson & Curtin, "Armadillo: An Efficient Framework
 * for Numerical Linear Algebra" (ICCAE 2025):
 *   - delayed evaluation: an expression is first described as a tree of
 *     operations and only evaluated as a whole (Sec. II);
 *   - elementwise fusion: chains of elementwise operations run as one pass
 *     with no temporaries (Sec. II, the Z = 0.4*X + 0.6*Y example);
 *   - products map onto a small set of kernels with transposes and scalar
 *     factors folded in (Sec. II, the paragraph on xGEMM/xGEMV; Fig. 3);
 *   - pattern rewrites: inv(A)*B becomes a solve (Sec. I; Sec. II, the
 *     Glue<Op<Mat,op_inv>,Vec,glue_times> paragraph; Sec. III (9)),
 *     diagmat(v)*B a row scaling (Sec. III (3)), trace(A*B) a diagonal-only
 *     product (Sec. III (5)), and matrix chains are re-parenthesised
 *     (Sec. II, chain paragraph; Sec. III (6)).
 *
 * Usage: build an expression descriptor (arma_expr), call arma_gpu_plan()
 * once (host only, no GPU work), then arma_gpu_eval() any number of times on
 * device buffers.  The library allocates no device memory during eval: the
 * caller supplies a workspace of at least arma_gpu_plan_workspace() bytes.
 *
 * Storage conventions (all calls):
 *   - matrices are column-major, element (i, j) at base[i + j*ld], with ld
 *     in elements and ld >= rows (BLAS/LAPACK convention, which the paper's
 *     library maps onto);
 *   - a vector is an n x 1 (or 1 x n) matrix;
 *   - matrix outputs are written contiguous (ld = rows) in the node's result
 *     element type (arma_gpu_output_info);
 *   - scalar outputs (trace, accu, norm_fro) are one FP64 value.
 *
 * Ownership: the caller owns every device buffer (inputs, outputs,
 * workspace).  A plan is owned by the library until arma_gpu_plan_free().
 * Plans are immutable after creation and may be evaluated concurrently on
 * different streams provided each evaluation has its own workspace.
 *
 * Errors: every call returns an arma_status.  Shape and dtype errors are
 * reported by arma_gpu_plan (the paper's conformance check, Sec. II);
 * pointer alignment and workspace size by arma_gpu_eval.  Numerical
 * failures detected on the device (exact zero pivot, iterative refinement
 * not converging) are recorded in the workspace and read back with
 * arma_gpu_eval_status() after the stream has been synchronised; they are
 * never raised as device traps.
 */
#ifndef ARMA_GPU_H
#define ARMA_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element types.  BF16 products accumulate and return FP32. */
typedef enum { ARMA_F64 = 0, ARMA_F32 = 1, ARMA_BF16 = 2 } arma_dtype;

typedef enum {
  ARMA_OK = 0,
  ARMA_ERR_INVALID = 1,     /* null pointer, bad node index, malformed descriptor */
  ARMA_ERR_SHAPE = 2,       /* non-conforming operand sizes (Sec. II conformance check) */
  ARMA_ERR_DTYPE = 3,       /* mixed element types where the operation needs equal ones */
  ARMA_ERR_ALIGN = 4,       /* device pointer misaligned for the kernel the plan chose */
  ARMA_ERR_WORKSPACE = 5,   /* workspace null or smaller than arma_gpu_plan_workspace() */
  ARMA_ERR_SINGULAR = 6,    /* LU met an exact zero pivot (LAPACK info > 0) */
  ARMA_ERR_NOCONVERGE = 7,  /* iterative refinement did not reach its tolerance */
  ARMA_ERR_CUDA = 8,        /* a CUDA runtime call failed */
  ARMA_ERR_UNSUPPORTED = 9, /* a valid expression this library does not evaluate */
  ARMA_ERR_TIMEOUT = 10     /* a bounded device-side wait ran out (arma_gpu_set_wait_limit_ns);
                               the kernels concerned returned early and the outputs are
                               not valid */
} arma_status;

/* Operations of the expression tree.  Operands are earlier node indices. */
typedef enum {
  ARMA_OP_INPUT = 0,       /* operand in_ptrs[slot]: rows, cols, ld, dtype from the node */
  ARMA_OP_ADD = 1,         /* a + b (elementwise) */
  ARMA_OP_SUB = 2,         /* a - b */
  ARMA_OP_SCHUR = 3,       /* a % b, elementwise (Schur) product */
  ARMA_OP_DIV = 4,         /* a / b, elementwise */
  ARMA_OP_SCALE = 5,       /* scalar * a */
  ARMA_OP_DIV_SCALAR = 6,  /* a / scalar */
  ARMA_OP_ADD_SCALAR = 7,  /* a + scalar */
  ARMA_OP_NEG = 8,         /* -a */
  ARMA_OP_TRANS = 9,       /* a^T */
  ARMA_OP_MATMUL = 10,     /* a * b, matrix product */
  ARMA_OP_DIAGMAT = 11,    /* vector -> diagonal matrix; matrix -> off-diagonals zero */
  ARMA_OP_TRACE = 12,      /* sum of the main diagonal -> FP64 scalar */
  ARMA_OP_ACCU = 13,       /* sum of all elements -> FP64 scalar */
  ARMA_OP_NORM_FRO = 14,   /* sqrt(sum of squares) -> FP64 scalar */
  ARMA_OP_INV = 15,        /* matrix inverse (square a) */
  ARMA_OP_SUBMAT = 16,     /* view of a: rows [slot, slot + rows), columns [ld, ld + cols)
                              (node fields: slot = first row, ld = first column, rows x
                              cols = size; Sec. III (2)).  Read in place: by the fused
                              elementwise pass always, and by products, trace, solves and
                              reductions when no transpose lies between the view and its
                              matrix; the literal plan copies it */
  ARMA_OP_SOLVE = 17       /* solve(a, b): X with a X = b, a square (Sec. III (10)).  The
                              optimised plan analyses a when evaluated and picks the solver
                              (arma_solve_path); the literal plan always factors a densely. */
} arma_op;

/* The solver an analysed solve took (Sec. III (10); the band, triangular and
 * symmetry checks of the solve trace, Fig. 3), in the order they are tried.
 * Diagonal, band and triangular solves compute in the data's precision;
 * the general solve follows the plan's tier. */
typedef enum {
  ARMA_SOLVE_NONE = 0,      /* no analysed solve ran (literal plan, or the stream was
                               being captured into a graph: then the general solve) */
  ARMA_SOLVE_GENERAL = 1,   /* dense LU with partial pivoting (+ refinement per tier) */
  ARMA_SOLVE_DIAGONAL = 2,  /* X = B ./ diag(A) */
  ARMA_SOLVE_BAND = 3,      /* band LU with partial pivoting: kl <= 31 subdiagonals,
                               ku <= 32 superdiagonals, 4 (2 kl + ku + 1) <= n
                               (tridiagonal systems included) */
  ARMA_SOLVE_UPPER = 4,     /* upper triangular: back substitution */
  ARMA_SOLVE_LOWER = 5,     /* lower triangular: forward substitution */
  ARMA_SOLVE_CHOLESKY = 6   /* symmetric with a positive diagonal: Cholesky, no pivoting
                               (+ refinement per tier); a matrix that turns out not to be
                               positive definite is solved by the general LU (path 1) */
} arma_solve_path;

/* Precision tier for products and solves (elementwise work always runs in
 * the operands' own type, FP32 arithmetic for BF16 data). */
typedef enum {
  ARMA_TIER_NATIVE = 0,      /* by element type: FP64 -> F64, FP32 -> SPLIT_BF16, BF16 -> BF16;
                                solves: FP64 -> LU32_IR64, FP32 -> SPLIT_BF16 */
  ARMA_TIER_F64 = 1,         /* FP64 arithmetic throughout */
  ARMA_TIER_SPLIT_BF16 = 2,  /* operands split into 3 BF16 terms, 6 tensor-core products
                                with FP32 accumulation (about FP32 accuracy) */
  ARMA_TIER_BF16 = 3,        /* operands rounded to BF16, one tensor-core product, FP32 accumulate */
  ARMA_TIER_LU32_IR64 = 4,   /* solves: FP32-accurate LU on tensor cores, FP64 iterative refinement */
  ARMA_TIER_F64_SLICED = 5   /* products: FP64-accurate from exact BF16 slices on the tensor cores
                                (FP64 operands scaled per row / column, cut into 8 integer
                                slices of 7 bits, the 36 slice products of weight >= 2^-63
                                accumulated exactly in K chunks of 1024 and combined in FP64;
                                the error-free splitting of Ozaki et al. 2012).  Needs finite
                                FP64 operands whose row and column maxima multiply within FP64
                                range; other operands take the FP64 (DFMA) product.  Solves:
                                as LU32_IR64 */
} arma_tier;

/* Plan flags. */
#define ARMA_PLAN_LITERAL      0x1u  /* one kernel per operator with temporaries: the naive
                                        evaluation the paper compares against (Sec. III) */
#define ARMA_PLAN_CHAIN_LEFT   0x2u  /* keep the written left-to-right order of product chains */
#define ARMA_PLAN_CHAIN_GREEDY 0x4u  /* the paper's chain rule (smallest adjacent result first)
                                        instead of the exact minimum-cost order */
#define ARMA_PLAN_COST_MLP     0x8u  /* choose among candidate plans (arma_gpu_plan_candidates)
                                        with the learned cost model loaded by
                                        arma_gpu_cost_model_load: the network's fastest
                                        candidate replaces the FLOP/byte estimate's pick when
                                        the network predicts it faster by the model's margin
                                        and the estimate does not rate it slower than its own
                                        pick by more than the model's guard factor; with no
                                        model loaded, the estimate's pick */
#define ARMA_PLAN_NO_FUSE      0x10u /* optimised rewrites but no elementwise fusion */
#define ARMA_PLAN_NO_TENSOR    0x20u /* batched plans: SIMT tiles instead of tensor-core tiles */
#define ARMA_PLAN_TILE64       0x40u /* batched SIMT tiles: 64 x 64 for every problem */
#define ARMA_PLAN_TILE32       0x80u /* batched SIMT tiles: 32 x 32 for every problem */
#define ARMA_PLAN_NO_SYRK      0x100u /* products X*X^T and X^T*X as general products (the
                                         paper's semi-optimised mapping to xGEMM, Sec. III (8));
                                         by default only their lower triangle is computed and
                                         then mirrored (xSYRK, Sec. II run-time analysis) */
#define ARMA_PLAN_NO_SOLVE_ANALYSIS 0x200u /* solves skip the run-time analysis of their
                                         matrix: always the general LU, and the evaluation
                                         never waits on its stream */
#define ARMA_PLAN_COST_HEURISTIC 0x400u /* choose among candidate plans the one with the
                                         smallest FLOP/byte estimate
                                         (arma_gpu_plan_heuristic_cost) */
#define ARMA_PLAN_TIER_CHOICE  0x800u /* with a COST flag: candidates also take every
                                         precision tier at least as accurate as the requested
                                         one (BF16 < SPLIT_BF16 < LU32_IR64 < F64 = F64_SLICED;
                                         NATIVE may move to F64 or F64_SLICED, and to
                                         SPLIT_BF16 when all inputs are BF16) */
#define ARMA_PLAN_NO_SPLITK    0x1000u /* products without split-K: one CTA per output tile
                                         over the whole reduction dimension */
#define ARMA_PLAN_DFMA_RESIDUAL 0x2000u /* iterative refinement forms r = B - A X with the
                                         FP64 (DFMA) product; by default systems of n >= 1024
                                         with >= 8 right-hand sides use the sliced FP64
                                         product of tier ARMA_TIER_F64_SLICED, A sliced once
                                         per solve */
#define ARMA_PLAN_NO_LOOKAHEAD 0x4000u /* the FP32 LU factorisation on one stream.  By default
                                         systems of 192 <= n <= 4096 overlap the trailing
                                         update of each panel with the factorisation of the
                                         next (look-ahead) on a high-priority stream of the
                                         calling host thread (created on first use and kept);
                                         the results are the same bit for bit */
/* Step limit of the FP64 iterative refinement of mixed-precision solves
 * (tiers LU32_IR64 and BF16; Sec. I and Sec. III (9): inv(A)*b as a
 * solve).  ARMA_PLAN_REFINE_STEPS(k), 1 <= k <= 15, stops after k steps; 0
 * (the default) means 10.  A solve that has not reached its stopping rule
 * (normwise backward error <= 1e-14) within the limit reports
 * ARMA_ERR_NOCONVERGE with info = the steps taken. */
#define ARMA_PLAN_REFINE_SHIFT 16
#define ARMA_PLAN_REFINE_MASK  0xF0000u
#define ARMA_PLAN_REFINE_STEPS(k) ((((uint32_t)(k)) & 0xFu) << ARMA_PLAN_REFINE_SHIFT)
/* K splits of every product (the CTAs that share one output tile, their
 * partial sums added by a combine pass): ARMA_PLAN_SPLITS(k), 1 <= k <= 15,
 * asks for k (fewer when K has fewer blocks of the kernel's K step, or when
 * the partial sums would pass 256 MB in the DFMA kernel); 0 (the default)
 * keeps the library's per-SM work model.  ARMA_PLAN_NO_SPLITK is k = 1.  The
 * products on the FP64-accurate sliced tier and matrix-vector products keep
 * their own rule.  This is what an autotuner varies to time split counts on
 * the caller's own operands. */
#define ARMA_PLAN_SPLITS_SHIFT 20
#define ARMA_PLAN_SPLITS_MASK  0xF00000u
#define ARMA_PLAN_SPLITS(k)    ((((uint32_t)(k)) & 0xFu) << ARMA_PLAN_SPLITS_SHIFT)

typedef struct arma_node {
  int32_t op;        /* arma_op */
  int32_t a;         /* first operand node index (< this node's index), -1 if none */
  int32_t b;         /* second operand node index, -1 if none */
  int32_t slot;      /* ARMA_OP_INPUT: index into in_ptrs */
  int32_t dtype;     /* ARMA_OP_INPUT: arma_dtype */
  int32_t reserved;  /* must be 0 */
  int64_t rows;      /* ARMA_OP_INPUT: number of rows */
  int64_t cols;      /* ARMA_OP_INPUT: number of columns */
  int64_t ld;        /* ARMA_OP_INPUT: leading dimension in elements (>= rows) */
  double scalar;     /* SCALE, DIV_SCALAR, ADD_SCALAR: the scalar */
} arma_node;

typedef struct arma_expr {
  int32_t n_nodes;          /* 1 .. 256 */
  int32_t n_outputs;        /* 1 .. 32 */
  const arma_node* nodes;   /* topological order: operands before users */
  const int32_t* outputs;   /* node indices; out_ptrs[i] receives node outputs[i] */
  int32_t tier;             /* arma_tier */
  uint32_t flags;           /* ARMA_PLAN_* */
} arma_expr;

typedef struct arma_plan arma_plan;

/* Validate and plan an expression (host only; no CUDA call).  This is the
 * point where the delayed expression of Sec. II is looked at as a whole and
 * mapped onto kernels: the conformance checks, the rewrites of Sec. III
 * (1)-(10), the chain order and, with ARMA_PLAN_COST_*, the choice among
 * candidate plans.  expr and the arrays it points to are read only during
 * the call.  Errors: ARMA_ERR_INVALID (null pointers, counts out of range,
 * an operand index not below its node's, one input slot described twice
 * differently), ARMA_ERR_SHAPE (non-conforming sizes, negative sizes,
 * ld < max(1, rows)), ARMA_ERR_DTYPE (an unknown element type, or mixed
 * element types where the operation needs equal ones), ARMA_ERR_UNSUPPORTED
 * (a valid expression outside what this library evaluates).  On success
 * *plan is a new plan, owned by the caller until arma_gpu_plan_free(); on
 * error *plan is set to NULL.  With the environment variable ARMA_PLAN_LOG
 * set (to anything but "" or "0") every call also writes one line to stderr:
 * the decision log of arma_gpu_plan_info, or the status it failed with. */
arma_status arma_gpu_plan(const arma_expr* expr, arma_plan** plan);

/* Workspace bytes arma_gpu_eval needs for this plan (the buffer itself must
 * be 256-byte aligned).  ARMA_ERR_INVALID for a null argument. */
arma_status arma_gpu_plan_workspace(const arma_plan* plan, size_t* bytes);

/* Shape and element type of output i (scalars: 1 x 1, ARMA_F64), so that
 * the caller can allocate out_ptrs[i].  ARMA_ERR_INVALID for a null plan or
 * an i outside 0 .. n_outputs - 1; null output pointers are skipped. */
arma_status arma_gpu_output_info(const arma_plan* plan, int32_t i, int64_t* rows,
                                 int64_t* cols, int32_t* dtype);

/* Enqueue the plan on `stream` (a cudaStream_t; NULL = legacy default).
 * in_ptrs[slot] are device pointers to the operands described by the INPUT
 * nodes; out_ptrs[i] device pointers for the outputs; workspace a device
 * buffer of workspace_bytes >= arma_gpu_plan_workspace(), 256-byte aligned.
 * Asynchronous: returns after launching; it does not synchronise, with one
 * exception: a plan with an analysed solve (ARMA_OP_SOLVE, or inv(A)*B in an
 * optimised plan) waits on `stream` for the analysis of its matrix before it
 * launches the solver (and once more when a Cholesky attempt fails).  While
 * `stream` is being captured into a CUDA graph no analysis runs and the
 * general solver is recorded instead; ARMA_PLAN_NO_SOLVE_ANALYSIS gives the
 * same behaviour always. */
arma_status arma_gpu_eval(const arma_plan* plan, const void* const* in_ptrs,
                          void* const* out_ptrs, void* workspace, size_t workspace_bytes,
                          void* stream);

/* After the stream of an arma_gpu_eval has been synchronised: read the
 * device-side status the evaluation left in `workspace`.  Returns ARMA_OK
 * (info = refinement steps a mixed-precision solve took, else 0),
 * ARMA_ERR_SINGULAR (info = 1-based column of the zero pivot) or
 * ARMA_ERR_NOCONVERGE (info = refinement steps taken).  Synchronises `stream`. */
arma_status arma_gpu_eval_status(const arma_plan* plan, const void* workspace, void* stream,
                                 int64_t* info);

/* After the stream of an arma_gpu_eval has been synchronised: the solver
 * the plan's (last) analysed solve took and what the analysis of its matrix
 * found: lower and upper bandwidth (largest i - j and j - i over non-zero
 * elements) and whether it equals its transpose exactly.  An optimised solve
 * waits on its stream for this analysis before it launches the solver; the
 * record lives in `workspace`.  Any output pointer may be NULL.
 * Synchronises `stream`. */
arma_status arma_gpu_eval_solve_path(const arma_plan* plan, const void* workspace, void* stream,
                                     int32_t* path, int32_t* kl, int32_t* ku, int32_t* symmetric);

/* Human- and machine-readable decision log of the plan (JSON text): the
 * rewrites taken, chain order, precision tier, kernels, predicted work.
 * The counterpart of the paper's internal call trace (Fig. 3).  Writes at
 * most len bytes including the terminating NUL; *needed (if non-NULL)
 * receives the full length + 1. */
arma_status arma_gpu_plan_info(const arma_plan* plan, char* buf, size_t len, size_t* needed);

/* Release a plan (NULL is ignored).  No evaluation of it may still be
 * running on a stream; the caller's buffers are not touched. */
void arma_gpu_plan_free(arma_plan* plan);

/* A static, NUL-terminated name for a status code ("unknown status" for
 * values outside arma_status). */
const char* arma_gpu_status_string(arma_status status);

/* Time limit of each bounded device-side wait that the solve kernels make
 * on one another's progress (the flag waits of the cooperative blocked
 * substitution and the grid barrier of the cooperative panel), in
 * nanoseconds; 2e9 (2 s) by default.  A wait that runs out records
 * ARMA_ERR_TIMEOUT in the evaluation's status word, every other wait of the
 * launch then gives up, and all kernels return.  0 means: give up at the
 * first poll that finds the awaited flag unset.  The setting is process-wide
 * and read when a kernel is launched; it exists so that callers (and this
 * library's tests) can exercise failure detection without a hung GPU.
 * Returns the previous limit. */
uint64_t arma_gpu_set_wait_limit_ns(uint64_t ns);

/* The address at which this library's kernels reach the memory at p (the
 * paper has no counterpart: it runs on the host).  Device and managed
 * memory: p itself.  Pinned host memory that the current device maps
 * (cudaHostAlloc, cudaHostRegister; with unified addressing the same
 * pointer): the mapped address, so arma_gpu_eval can take inputs and
 * outputs in host memory and its kernels read and write them over the host
 * link, with no staging copy.  Memory the device cannot address (plain
 * pageable host memory included) gives ARMA_ERR_INVALID and *dptr = NULL.
 * Host-only; it allocates nothing. */
arma_status arma_gpu_device_address(const void* p, void** dptr);

/* Name and text of the last CUDA runtime error behind an ARMA_ERR_CUDA
 * returned to the calling thread ("" if none).  The string is owned by the
 * library and stays valid until the thread's next failing call. */
const char* arma_gpu_last_cuda_error(void);

/* ---- Cost model.  The paper chooses an evaluation by fixed rules
 * (compile-time patterns, Sec. II; the greedy chain rule, Sec. II chain
 * paragraph).  Here arma_gpu_plan itself can choose among candidate plans of
 * one expression (ARMA_PLAN_COST_HEURISTIC, ARMA_PLAN_COST_MLP): chain
 * order, fusion, split-K and precision tier, ranked either by a FLOP/byte
 * roofline estimate or by a small learned network trained on timings that
 * this library records with its own GPU kernels.  The plan's decision log
 * (arma_gpu_plan_info) lists the candidates, their scores and the pick. ---- */

#define ARMA_PLAN_FEATURES 32

/* Host only: the plan's feature vector; n >= ARMA_PLAN_FEATURES floats.
 *   0 log2(1 + flops)            1 log2(1 + bytes)         2 steps
 *   3 elementwise steps          4 product steps           5 matrix-vector steps
 *   6 diagonal-dot steps         7 copy steps              8 solve steps
 *   9 log2(1 + largest step flops)  10 log2(1 + largest step bytes)
 *  11 log2(1 + workspace bytes)  12 tensor-core share of flops
 *  13 literal plan               14 split-BF16 share of flops
 *  15 log2(1 + flops / bytes)    16 ln(FLOP/byte estimate, seconds)
 *  17 kernel launches            18 FP64 DFMA share of flops
 *  19 share of the estimate spent in elementwise passes
 *  20 share of the estimate spent in products
 *  21 log2(1 + smallest dimension of the largest product)
 *  22 products without split-K   23 log2(1 + largest output elements)
 *  24 products whose K is split over CTAs (a combine launch each)
 *  25 log2(1 + elements read with a stride by fused passes)
 *  26 share of the estimate in FP64 (DFMA) products
 *  27 useful / padded output of the tensor-core products (1 if none)
 *  28 log2(1 + work items of the largest product / 152 SMs)
 *  29 operand preparation passes of the tensor-core products
 *  30 log2(1 + K of the largest product)
 *  31 share of the estimate in kernel launches */
arma_status arma_gpu_plan_features(const arma_plan* plan, float* features, int32_t n);

/* Host only: estimated seconds, summing per step a launch plus the larger
 * of its compute time and its memory time on GB300. */
arma_status arma_gpu_plan_heuristic_cost(const arma_plan* plan, double* seconds);

/* Host only: plan every distinct candidate evaluation of an expression: the
 * chain orders (exact DP, the paper's greedy rule, written order), with and
 * without elementwise fusion, with and without split-K, and, with
 * ARMA_PLAN_TIER_CHOICE, every admissible precision tier.  Candidates whose
 * step lists coincide are planned once.  plans[i] (i < *count) receive new
 * plans, owned by the caller (arma_gpu_plan_free); at most capacity are
 * written and *count receives the number of distinct candidates.  The
 * expression's own COST flags are ignored; ARMA_PLAN_LITERAL gives the
 * literal plan alone. */
arma_status arma_gpu_plan_candidates(const arma_expr* expr, arma_plan** plans, int32_t capacity,
                                     int32_t* count);

/* Load the learned cost model that ARMA_PLAN_COST_MLP consults (host
 * memory, copied; process-wide, replaces any earlier model).  The network
 * (layout as arma_gpu_mlp_forward) maps the standardised feature vector
 * z_i = (f_i - mean[i]) / scale[i] of a plan to a correction of the
 * FLOP/byte estimate: predicted seconds = estimate * exp(network(z)).
 * features must be ARMA_PLAN_FEATURES; hidden <= 128.  The network's
 * fastest candidate replaces the estimate's pick only when the network
 * predicts it at least a fraction `margin` (0 <= margin < 1) faster than the
 * estimate's pick, and only when the estimate rates it at most `guard`
 * times slower than its own pick (guard >= 1; 0: no such check). */
arma_status arma_gpu_cost_model_load(const float* params, int32_t features, int32_t hidden, const float* mean,
                                     const float* scale, double guard, double margin);

/* Forget the loaded cost model (ARMA_PLAN_COST_MLP then uses the estimate). */
void arma_gpu_cost_model_clear(void);

/* Host only: seconds the loaded cost model predicts for a plan (the same
 * arithmetic as arma_gpu_mlp_forward, in FP32 on the host).  Returns
 * ARMA_ERR_UNSUPPORTED when no model is loaded. */
arma_status arma_gpu_cost_model_predict(const arma_plan* plan, double* seconds);

/* Cost network (this library's learned plan choice; the paper has none):
 * y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, FP32, with 1 <= features <= 64
 * inputs and 1 <= hidden <= 128 units; parameters packed as W1 (hidden x
 * features, row-major), b1, W2 (hidden x hidden), b2, W3, b3.  Samples are
 * rows of x (n x features, row-major).  All pointers are device pointers
 * owned by the caller; calls are asynchronous on stream.  Sizes out of range
 * or null pointers give ARMA_ERR_INVALID, a failed launch ARMA_ERR_CUDA. */
int64_t arma_gpu_mlp_param_count(int32_t features, int32_t hidden);

/* Workspace bytes for arma_gpu_mlp_grad with n samples (per-sample
 * activations and deltas, plus 1 KiB). */
size_t arma_gpu_mlp_workspace(int32_t features, int32_t hidden, int32_t n);

/* y[i] = network(x[i * features ...]) for i < n (n = 0: nothing). */
arma_status arma_gpu_mlp_forward(const float* params, int32_t features, int32_t hidden, const float* x,
                                 int32_t n, float* y, void* stream);

/* grad = d/dparams of (1/n) sum_i (network(x_i) - target_i)^2; y_out (may be
 * null) receives the predictions.  Deterministic: every gradient entry is
 * summed over the samples in sample order. */
arma_status arma_gpu_mlp_grad(const float* params, int32_t features, int32_t hidden, const float* x,
                              const float* target, int32_t n, float* grad, float* y_out, void* workspace,
                              size_t workspace_bytes, void* stream);

/* One Adam step (Kingma and Ba, 2015) over count parameters, in place on
 * params and the moment vectors m and v, with bias correction for step >= 1
 * (ARMA_ERR_INVALID for step < 1, count < 1 or a null pointer). */
arma_status arma_gpu_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t count,
                              int32_t step, float lr, float beta1, float beta2, float eps, void* stream);

/* ---- Batched evaluation: many independent instances of one expression
 * family (same nodes and outputs, per-instance sizes) in one grouped
 * launch.  Each instance must reduce to a single product with folded
 * transposes and scalars plus an optional added matrix,
 *     D_i = alpha * op(A_i) * op(B_i) + beta * C_i,
 * optionally with trace(op(A_i) * op(B_i)) as a further output: the folded
 * product and diagonal-only trace of Sec. II / Sec. III (5), batched.
 * A, B are FP32 or BF16, D FP32, traces FP64; accumulation is FP32.
 * Otherwise arma_gpu_plan_batched returns ARMA_ERR_UNSUPPORTED. ---- */

/* Plan count >= 1 instances (exprs[i] describes instance i; read only
 * during the call).  All instances share one family: the same nodes, scalars
 * and outputs, with their own sizes.  Errors: ARMA_ERR_INVALID (count < 1,
 * null pointers), ARMA_ERR_SHAPE (an instance does not conform),
 * ARMA_ERR_DTYPE (operands that are not FP32 or BF16), ARMA_ERR_UNSUPPORTED
 * (another form, or instances of different families).  Operands that are
 * K-contiguous (op(A) = trans of a k x m matrix, B k x n) run on the tensor
 * cores; others on the SIMT grouped kernel (the plan log's "tensor_cores").
 * On success *plan is owned by the caller until arma_gpu_plan_free(). */
arma_status arma_gpu_plan_batched(const arma_expr* exprs, int32_t count, arma_plan** plan);

/* Bytes of the problem table that describes one batch of pointers. */
arma_status arma_gpu_batched_table_bytes(const arma_plan* plan, size_t* bytes);

/* Fill a host buffer of arma_gpu_batched_table_bytes() bytes with the
 * problem table: in_ptrs[i * n_slots + s] and out_ptrs[i * n_outputs + o]
 * are device pointers of instance i (n_slots, n_outputs as in exprs[0]).
 * The caller copies the table to device memory (once, if the pointers do
 * not change). */
arma_status arma_gpu_batched_table_fill(const arma_plan* plan, const void* const* in_ptrs,
                                        void* const* out_ptrs, void* host_table);

/* Evaluate every instance of the batch.  On the tensor cores (both
 * operands K-contiguous, BF16 or FP32; the plan log's "tensor_cores") a pack
 * kernel first copies every instance's op(A) and op(B)^T into packed
 * K-block-major BF16 arrays in the workspace (FP32 as three exact BF16
 * slices), then one persistent tcgen05 kernel reads them with TMA; the
 * workspace (arma_gpu_plan_workspace) therefore holds about
 * slices * 128 bytes per row of 64 of K of every operand.  Otherwise one
 * persistent SIMT grouped kernel runs.  A small kernel adds the traces.
 * device_table is the filled table in device memory.  Asynchronous on
 * stream; capturable in a CUDA graph. */
arma_status arma_gpu_eval_batched(const arma_plan* plan, const void* device_table, void* workspace,
                                  size_t workspace_bytes, void* stream);

/* Size of the library-owned scratch array used by arma_gpu_eval_fused_static. */
#define ARMA_STATIC_SCRATCH_BYTES 131072

/* Evaluate a plan without any caller workspace, for callers that cannot
 * allocate device memory (a plug-in that receives only raw input and
 * output pointers, code inside another framework's memory pool, loops that
 * cannot afford cudaMalloc's implicit synchronisation).  The paper has no
 * counterpart to this call.
 *
 * Only plans made entirely of fused elementwise passes (elementwise
 * expressions, with accu / norm_fro / trace of them) are accepted, and only
 * if arma_gpu_plan_workspace() <= ARMA_STATIC_SCRATCH_BYTES; otherwise the
 * call returns ARMA_ERR_UNSUPPORTED or ARMA_ERR_WORKSPACE and launches
 * nothing.  The scratch lives in one file-scope device array of
 * ARMA_STATIC_SCRATCH_BYTES per GPU, held until the process exits.  Every
 * call outside stream capture looks up that array's device address (with
 * the device current); a call under capture reuses the address found by the
 * last call outside capture, so make the first call on a device before any
 * stream capture.  The
 * call allocates nothing.  Every call shares the array: calls whose kernels
 * overlap on the GPU (different streams, or other threads) race on it.
 * in_ptrs, out_ptrs and stream mean the same as in arma_gpu_eval. */
arma_status arma_gpu_eval_fused_static(const arma_plan* plan, const void* const* in_ptrs,
                                       void* const* out_ptrs, void* stream);

/* Matrix-chain ordering used by the planner (Sec. II, chain paragraph;
 * Sec. III (6)).  dims[0..n] give factor t as dims[t] x dims[t+1].
 * method 0: exact minimum number of scalar multiply-adds (dynamic
 * programming; among equal costs the lexicographically smallest preorder
 * sequence of split points); 1: the paper's greedy rule (multiply first the
 * adjacent pair with the smallest result, left-most on ties); 2: left to
 * right.  splits receives the n-1 split points in preorder (split k joins
 * factors [i..k] and [k+1..j]); cost the total multiply-adds. */
arma_status arma_gpu_chain_order(int32_t n, const int64_t* dims, int32_t method, int32_t* splits,
                                 uint64_t* cost);

#ifdef __cplusplus
}
#endif
#endif /* ARMA_GPU_H */
