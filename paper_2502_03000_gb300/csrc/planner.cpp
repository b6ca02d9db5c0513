// Expression planner: validation (Sec. II conformance checks), the rewrites
// of Sec. II-III onto a small kernel set, matrix-chain ordering, and the
// literal one-kernel-per-operator plan the paper compares against.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "grouped.h"
#include "internal.h"

namespace arma {

// ---------------------------------------------------------------------------
// Matrix-chain ordering (Sec. II chain paragraph; Sec. III expression (6))
// ---------------------------------------------------------------------------
typedef unsigned __int128 u128;

static uint64_t sat64(u128 v) { return v > (u128)UINT64_MAX ? UINT64_MAX : (uint64_t)v; }

// Exact minimum of the number of scalar multiply-adds by dynamic
// programming over sub-chains [i..j].  Among equal costs the smallest split
// point wins at every sub-chain, which yields the tree with the
// lexicographically smallest preorder split sequence.
static void chain_dp(int n, const int64_t* p, std::vector<int>& split, std::vector<u128>& cost) {
  split.assign(n * n, -1);
  cost.assign(n * n, 0);
  for (int len = 2; len <= n; ++len)
    for (int i = 0; i + len - 1 < n; ++i) {
      int j = i + len - 1;
      u128 best = 0;
      int bk = -1;
      for (int k = i; k < j; ++k) {
        u128 c = cost[i * n + k] + cost[(k + 1) * n + j] +
                 (u128)(uint64_t)p[i] * (u128)(uint64_t)p[k + 1] * (u128)(uint64_t)p[j + 1];
        if (bk < 0 || c < best) { best = c; bk = k; }
      }
      cost[i * n + j] = best;
      split[i * n + j] = bk;
    }
}

struct ChainTree {  // node t: leaf if lo == hi
  int lo, hi, k;
  int left, right;
};

static int build_tree_from_split(int i, int j, int n, const std::vector<int>& split,
                                 std::vector<ChainTree>& t) {
  int id = (int)t.size();
  t.push_back({i, j, -1, -1, -1});
  if (i == j) return id;
  int k = split[i * n + j];
  t[id].k = k;
  int l = build_tree_from_split(i, k, n, split, t);
  int r = build_tree_from_split(k + 1, j, n, split, t);
  t[id].left = l;
  t[id].right = r;
  return id;
}

// The paper's rule: repeatedly multiply the adjacent pair whose result has
// the fewest elements (left-most on ties).
static void chain_greedy(int n, const int64_t* p, std::vector<ChainTree>& t, int& root) {
  struct Part { int lo, hi, node; };
  std::vector<Part> parts;
  t.clear();
  for (int i = 0; i < n; ++i) {
    t.push_back({i, i, -1, -1, -1});
    parts.push_back({i, i, i});
  }
  while (parts.size() > 1) {
    size_t bq = 0;
    u128 best = 0;
    for (size_t q = 0; q + 1 < parts.size(); ++q) {
      u128 sz = (u128)(uint64_t)p[parts[q].lo] * (u128)(uint64_t)p[parts[q + 1].hi + 1];
      if (q == 0 || sz < best) { best = sz; bq = q; }
    }
    Part a = parts[bq], b = parts[bq + 1];
    int id = (int)t.size();
    t.push_back({a.lo, b.hi, a.hi, a.node, b.node});
    parts[bq] = {a.lo, b.hi, id};
    parts.erase(parts.begin() + bq + 1);
  }
  root = parts[0].node;
}

static void chain_left(int n, std::vector<ChainTree>& t, int& root) {
  t.clear();
  for (int i = 0; i < n; ++i) t.push_back({i, i, -1, -1, -1});
  root = 0;
  for (int i = 1; i < n; ++i) {
    int id = (int)t.size();
    t.push_back({0, i, i - 1, root, i});
    root = id;
  }
}

static u128 tree_cost(const std::vector<ChainTree>& t, int node, const int64_t* p) {
  const ChainTree& c = t[node];
  if (c.lo == c.hi) return 0;
  return tree_cost(t, c.left, p) + tree_cost(t, c.right, p) +
         (u128)(uint64_t)p[c.lo] * (u128)(uint64_t)p[c.k + 1] * (u128)(uint64_t)p[c.hi + 1];
}

static void tree_preorder(const std::vector<ChainTree>& t, int node, std::vector<int>& out) {
  const ChainTree& c = t[node];
  if (c.lo == c.hi) return;
  out.push_back(c.k);
  tree_preorder(t, c.left, out);
  tree_preorder(t, c.right, out);
}

// method: 0 = exact DP, 1 = paper greedy, 2 = left to right
static void chain_order(int n, const int64_t* p, int method, std::vector<ChainTree>& t, int& root) {
  t.clear();
  if (method == 1) { chain_greedy(n, p, t, root); return; }
  if (method == 2) { chain_left(n, t, root); return; }
  std::vector<int> split;
  std::vector<u128> cost;
  chain_dp(n, p, split, cost);
  root = build_tree_from_split(0, n - 1, n, split, t);
}

// ---------------------------------------------------------------------------
// Planner
// ---------------------------------------------------------------------------
namespace {

struct NInfo {
  int64_t rows = 0, cols = 0;
  int32_t dtype = ARMA_F64;
  bool scalar = false;
};

bool is_ew_op(int op) {
  return op == ARMA_OP_ADD || op == ARMA_OP_SUB || op == ARMA_OP_SCHUR || op == ARMA_OP_DIV ||
         op == ARMA_OP_SCALE || op == ARMA_OP_DIV_SCALAR || op == ARMA_OP_ADD_SCALAR ||
         op == ARMA_OP_NEG;
}
bool is_binary(int op) {
  return op == ARMA_OP_ADD || op == ARMA_OP_SUB || op == ARMA_OP_SCHUR || op == ARMA_OP_DIV ||
         op == ARMA_OP_MATMUL || op == ARMA_OP_SOLVE;
}
const char* op_name(int op) {
  static const char* names[] = {"input", "add", "sub", "schur", "div", "scale", "div_scalar",
                                "add_scalar", "neg", "trans", "matmul", "diagmat", "trace",
                                "accu", "norm_fro", "inv", "submat", "solve"};
  return (op >= 0 && op <= ARMA_OP_SOLVE) ? names[op] : "?";
}
const char* tier_name(int t) {
  if (t == ARMA_TIER_F64_SLICED) return "f64_sliced";
  static const char* names[] = {"native", "f64", "split_bf16", "bf16", "lu32_ir64"};
  return (t >= 0 && t <= 4) ? names[t] : "?";
}

struct Factor {
  enum Kind { DENSE, DIAG, INV } kind = DENSE;
  MatOperand m;       // DENSE: operand (trans flag = op); INV: the matrix to invert
  VecOperand v;       // DIAG: the diagonal
  int64_t rows = 0, cols = 0;   // shape of op(factor)
  int32_t dtype = ARMA_F64;
};

class Planner {
 public:
  Planner(const arma_expr& e, arma_plan& p) : e_(e), p_(p) {}
  arma_status run();

 private:
  const arma_expr& e_;
  arma_plan& p_;
  std::vector<arma_node> nd_;
  std::vector<NInfo> info_;
  std::vector<int> uses_;
  std::vector<int> out_of_;      // node -> output index or -1
  std::vector<MatOperand> loc_;  // materialised location
  std::vector<char> scalar_done_;
  bool literal_ = false, fuse_ = true;
  int chain_method_ = 0;
  arma_status err_ = ARMA_OK;
  std::string err_msg_;

  arma_status validate();
  arma_status fail(arma_status s, const std::string& m) {
    if (err_ == ARMA_OK) { err_ = s; err_msg_ = m; }
    return s;
  }

  // workspace
  int64_t alloc_ws(int64_t bytes) {
    int64_t off = (int64_t)p_.ws_bytes;
    p_.ws_bytes += (size_t)((bytes + 255) / 256 * 256);
    return off;
  }
  int32_t alloc_ticket() {
    if (p_.tickets >= kMaxTickets) { fail(ARMA_ERR_UNSUPPORTED, "too many reductions"); return 0; }
    return p_.tickets++;
  }
  MatOperand temp_mat(int64_t r, int64_t c, int32_t dt) {
    MatOperand m;
    m.ref = ref_ws(alloc_ws(std::max<int64_t>(1, r * c) * (int64_t)dtype_size(dt)));
    m.ld = std::max<int64_t>(1, r);
    m.dtype = dt;
    return m;
  }
  MatOperand dest_for(int x) {
    if (out_of_[x] >= 0 && !info_[x].scalar) {
      MatOperand m;
      m.ref = ref_output(out_of_[x]);
      m.ld = std::max<int64_t>(1, info_[x].rows);
      m.dtype = info_[x].dtype;
      return m;
    }
    return temp_mat(info_[x].rows, info_[x].cols, info_[x].dtype);
  }
  int32_t product_tier(int32_t dt) const {
    int t = e_.tier;
    if (t == ARMA_TIER_NATIVE || t == ARMA_TIER_LU32_IR64)
      return dt == ARMA_F64 ? ARMA_TIER_F64 : dt == ARMA_F32 ? ARMA_TIER_SPLIT_BF16 : ARMA_TIER_BF16;
    // the sliced product takes FP64 operands; FP64 accuracy on others is DFMA
    if (t == ARMA_TIER_F64_SLICED && dt != ARMA_F64) return ARMA_TIER_F64;
    return t;
  }
  int32_t solve_tier(int32_t dt) const {
    int t = e_.tier;
    if (t == ARMA_TIER_NATIVE)
      return dt == ARMA_F64 ? ARMA_TIER_LU32_IR64 : dt == ARMA_F32 ? ARMA_TIER_SPLIT_BF16 : ARMA_TIER_BF16;
    if (t == ARMA_TIER_F64_SLICED) return ARMA_TIER_LU32_IR64;
    return t;
  }

  // steps
  void push_step(Step&& s) { p_.steps.push_back(std::move(s)); }
  MatOperand materialize(int x);
  void plan_ew_root(int x, const MatOperand* dest, bool diag_mode, Ref sum_out, Ref norm_out,
                    bool attach_reductions);
  void plan_product(int x, MatOperand dest, double alpha_extra, const MatOperand* C, double beta);
  void plan_scalar(int r);
  void emit_reduce(const MatOperand& src, int64_t m, int64_t n, bool diag, Ref sum_out,
                   Ref norm_out, const char* why);
  void emit_gemm(int64_t m, int64_t n, int64_t k, const MatOperand& A, const MatOperand& B,
                 const MatOperand& D, double alpha, const MatOperand* C, double beta,
                 const VecOperand* rs, const VecOperand* cs, const char* why);
  void emit_solve(const MatOperand& A, int64_t n, const MatOperand* B, int64_t nrhs,
                  const MatOperand& X, int32_t dt, bool explicit_inverse, const char* why);
  void flatten_product(int x, double& alpha, std::vector<Factor>& f);
  MatOperand eval_chain(std::vector<Factor>& dense, int64_t lo, int64_t hi,
                        const std::vector<ChainTree>& t, int node, const MatOperand* dest,
                        double alpha, const MatOperand* C, double beta, const VecOperand* rs,
                        const VecOperand* cs);
  void literal();
  // elementwise compilation
  struct EwBuild {
    EwStep st;
    std::vector<int> leaf_node;   // operand k -> node
    bool overflow = false;
  };
  bool ew_is_leaf(int y, int root) const;
  int ew_operand(EwBuild& b, int y);
  void ew_emit(EwBuild& b, int op, int arg, double s, int arg2 = 0) {
    if (b.st.nops >= kMaxOps) { b.overflow = true; return; }
    EwIns& in = b.st.ops[b.st.nops++];
    in = EwIns{op, arg, s};
    in.arg2 = arg2;
  }
  void ew_compile(EwBuild& b, int y, int depth, int root);
  // a sum of signed terms: leaves (times a scalar), elementwise products of
  // two leaves, and at most one other subtree
  struct SumTerm {
    int kind;    // 0 leaf, 1 product of two leaves, 2 other subtree
    int a, b;
    double c;    // coefficient (+-1 for kinds 1 and 2)
  };
  bool sum_terms(int y, double sign, int root, bool top, std::vector<SumTerm>& t) const;
  bool ew_sum(EwBuild& b, int y, int depth, int root);
  bool ew_leafable_view(int y) const;
  void linearize(int x, double c, std::vector<std::pair<int, double>>& terms, bool top);
};

arma_status Planner::validate() {
  if (e_.n_nodes < 1 || e_.n_nodes > 256 || !e_.nodes)
    return fail(ARMA_ERR_INVALID, "n_nodes must be 1..256 with a node array");
  if (e_.n_outputs < 1 || e_.n_outputs > 32 || !e_.outputs)
    return fail(ARMA_ERR_INVALID, "n_outputs must be 1..32 with an output array");
  if (e_.tier < 0 || e_.tier > ARMA_TIER_F64_SLICED) return fail(ARMA_ERR_INVALID, "bad tier");
  int n = e_.n_nodes;
  nd_.assign(e_.nodes, e_.nodes + n);
  info_.assign(n, NInfo());
  uses_.assign(n, 0);
  out_of_.assign(n, -1);
  std::vector<arma_node> slot_seen(256);
  std::vector<char> slot_used(256, 0);
  for (int i = 0; i < n; ++i) {
    const arma_node& d = nd_[i];
    NInfo& I = info_[i];
    char buf[160];
    if (d.op < 0 || d.op > ARMA_OP_SOLVE) {
      snprintf(buf, sizeof buf, "node %d: unknown op %d", i, d.op);
      return fail(ARMA_ERR_INVALID, buf);
    }
    if (d.op == ARMA_OP_INPUT) {
      if (d.slot < 0 || d.slot >= 256) return fail(ARMA_ERR_INVALID, "input slot out of range");
      if (d.dtype < ARMA_F64 || d.dtype > ARMA_BF16) return fail(ARMA_ERR_DTYPE, "bad input dtype");
      if (d.rows < 0 || d.cols < 0 || d.ld < std::max<int64_t>(1, d.rows))
        return fail(ARMA_ERR_SHAPE, "input needs rows, cols >= 0 and ld >= max(1, rows)");
      if (slot_used[d.slot]) {
        const arma_node& o = slot_seen[d.slot];
        if (o.rows != d.rows || o.cols != d.cols || o.ld != d.ld || o.dtype != d.dtype)
          return fail(ARMA_ERR_INVALID, "one slot described twice with different shapes");
      }
      slot_used[d.slot] = 1;
      slot_seen[d.slot] = d;
      p_.n_slots = std::max(p_.n_slots, d.slot + 1);
      I.rows = d.rows; I.cols = d.cols; I.dtype = d.dtype;
      continue;
    }
    bool bin = is_binary(d.op);
    if (d.a < 0 || d.a >= i || (bin && (d.b < 0 || d.b >= i))) {
      snprintf(buf, sizeof buf, "node %d (%s): operand index must refer to an earlier node", i,
               op_name(d.op));
      return fail(ARMA_ERR_INVALID, buf);
    }
    const NInfo& A = info_[d.a];
    if (A.scalar || (bin && info_[d.b].scalar))
      return fail(ARMA_ERR_UNSUPPORTED, "scalar results (trace/accu/norm) can only be outputs");
    uses_[d.a]++;
    if (bin) uses_[d.b]++;
    switch (d.op) {
      case ARMA_OP_ADD: case ARMA_OP_SUB: case ARMA_OP_SCHUR: case ARMA_OP_DIV: {
        const NInfo& B = info_[d.b];
        if (A.rows != B.rows || A.cols != B.cols) {
          snprintf(buf, sizeof buf, "node %d (%s): %lldx%lld and %lldx%lld do not conform", i,
                   op_name(d.op), (long long)A.rows, (long long)A.cols, (long long)B.rows,
                   (long long)B.cols);
          return fail(ARMA_ERR_SHAPE, buf);
        }
        if (A.dtype != B.dtype) return fail(ARMA_ERR_DTYPE, "elementwise operands differ in dtype");
        I.rows = A.rows; I.cols = A.cols; I.dtype = A.dtype;
        break;
      }
      case ARMA_OP_SCALE: case ARMA_OP_DIV_SCALAR: case ARMA_OP_ADD_SCALAR: case ARMA_OP_NEG:
        if (!std::isfinite(d.scalar) && d.op != ARMA_OP_NEG)
          return fail(ARMA_ERR_INVALID, "scalar must be finite");
        I.rows = A.rows; I.cols = A.cols; I.dtype = A.dtype;
        break;
      case ARMA_OP_TRANS:
        I.rows = A.cols; I.cols = A.rows; I.dtype = A.dtype;
        break;
      case ARMA_OP_MATMUL: {
        const NInfo& B = info_[d.b];
        if (A.cols != B.rows) {
          snprintf(buf, sizeof buf, "node %d (matmul): %lldx%lld * %lldx%lld do not conform", i,
                   (long long)A.rows, (long long)A.cols, (long long)B.rows, (long long)B.cols);
          return fail(ARMA_ERR_SHAPE, buf);
        }
        if (A.dtype != B.dtype) return fail(ARMA_ERR_DTYPE, "product operands differ in dtype");
        I.rows = A.rows; I.cols = B.cols;
        I.dtype = A.dtype == ARMA_F64 ? ARMA_F64 : ARMA_F32;
        break;
      }
      case ARMA_OP_DIAGMAT:
        if (A.rows == 1 || A.cols == 1) {
          I.rows = I.cols = A.rows * A.cols;
        } else {
          I.rows = A.rows; I.cols = A.cols;
        }
        I.dtype = A.dtype;
        break;
      case ARMA_OP_TRACE: case ARMA_OP_ACCU: case ARMA_OP_NORM_FRO:
        I.rows = I.cols = 1; I.dtype = ARMA_F64; I.scalar = true;
        break;
      case ARMA_OP_SUBMAT: {
        const int64_t r0 = d.slot, c0 = d.ld;
        if (r0 < 0 || c0 < 0 || d.rows < 0 || d.cols < 0 || r0 + d.rows > A.rows || c0 + d.cols > A.cols) {
          snprintf(buf, sizeof buf, "node %d (submat): rows [%lld, %lld) x cols [%lld, %lld) outside %lldx%lld", i,
                   (long long)r0, (long long)(r0 + d.rows), (long long)c0, (long long)(c0 + d.cols),
                   (long long)A.rows, (long long)A.cols);
          return fail(ARMA_ERR_SHAPE, buf);
        }
        I.rows = d.rows; I.cols = d.cols; I.dtype = A.dtype;
        break;
      }
      case ARMA_OP_SOLVE: {
        const NInfo& B = info_[d.b];
        if (A.rows != A.cols) return fail(ARMA_ERR_SHAPE, "solve needs a square matrix");
        if (B.rows != A.rows) {
          snprintf(buf, sizeof buf, "node %d (solve): %lldx%lld matrix, %lldx%lld right-hand side", i,
                   (long long)A.rows, (long long)A.cols, (long long)B.rows, (long long)B.cols);
          return fail(ARMA_ERR_SHAPE, buf);
        }
        if (A.dtype == ARMA_BF16 || B.dtype == ARMA_BF16)
          return fail(ARMA_ERR_DTYPE, "solve with BF16 operands is not supported");
        if (A.dtype != B.dtype) return fail(ARMA_ERR_DTYPE, "solve operands differ in dtype");
        I.rows = A.rows; I.cols = B.cols; I.dtype = A.dtype;
        break;
      }
      case ARMA_OP_INV:
        if (A.rows != A.cols) return fail(ARMA_ERR_SHAPE, "inv needs a square matrix");
        if (A.dtype == ARMA_BF16) return fail(ARMA_ERR_DTYPE, "inv of a BF16 matrix is not supported");
        I.rows = A.rows; I.cols = A.cols; I.dtype = A.dtype;
        break;
      default:
        return fail(ARMA_ERR_INVALID, "unknown op");
    }
  }
  for (int o = 0; o < e_.n_outputs; ++o) {
    int x = e_.outputs[o];
    if (x < 0 || x >= n) return fail(ARMA_ERR_INVALID, "output index out of range");
    if (out_of_[x] >= 0) return fail(ARMA_ERR_INVALID, "a node is listed twice as an output");
    if (nd_[x].op == ARMA_OP_INPUT) return fail(ARMA_ERR_UNSUPPORTED, "an input cannot be an output");
    out_of_[x] = o;
    uses_[x]++;
    OutInfo oi;
    oi.rows = info_[x].rows; oi.cols = info_[x].cols; oi.dtype = info_[x].dtype;
    oi.scalar = info_[x].scalar ? 1 : 0;
    p_.outs.push_back(oi);
  }
  return ARMA_OK;
}

// ---------------------------------------------------------------------------
// elementwise compilation
// ---------------------------------------------------------------------------
// A view that the elementwise kernel can read directly without a pass of
// its own: an input or materialised matrix, its transpose, or a diagonal.
// y read in place: an input or a materialised node, seen through a chain of
// transposes and submatrix views (and at most one diagmat, outermost)
bool Planner::ew_leafable_view(int y) const {
  const arma_node& d = nd_[y];
  if (d.op == ARMA_OP_INPUT || loc_[y].ref.valid()) return true;
  int z = y;
  if (d.op == ARMA_OP_DIAGMAT) z = d.a;
  while (!loc_[z].ref.valid() && (nd_[z].op == ARMA_OP_TRANS || nd_[z].op == ARMA_OP_SUBMAT)) z = nd_[z].a;
  if (z == y) return false;
  return nd_[z].op == ARMA_OP_INPUT || loc_[z].ref.valid() ||
         (nd_[y].op == ARMA_OP_DIAGMAT && z == d.a);   // diagmat(x): x materialised first
}

bool Planner::ew_is_leaf(int y, int root) const {
  if (y == root) return false;
  if (ew_leafable_view(y)) return true;
  if (!is_ew_op(nd_[y].op)) return true;            // products etc.: materialised first
  if (uses_[y] > 1 || out_of_[y] >= 0) return true;  // shared: materialised once
  return false;
}

int Planner::ew_operand(EwBuild& b, int y) {
  for (size_t k = 0; k < b.leaf_node.size(); ++k)
    if (b.leaf_node[k] == y) return (int)k;
  if (b.st.nin >= kMaxIn) { b.overflow = true; return 0; }
  EwOperand op;
  const arma_node& d = nd_[y];
  bool dg = false;
  int top = y;
  if (!loc_[y].ref.valid() && d.op == ARMA_OP_DIAGMAT) { top = d.a; dg = true; }
  // the chain of transposes and submatrix views from top down to its base
  std::vector<int> chain;
  int base = top;
  while (!loc_[base].ref.valid() && (nd_[base].op == ARMA_OP_TRANS || nd_[base].op == ARMA_OP_SUBMAT)) {
    chain.push_back(base);
    base = nd_[base].a;
  }
  MatOperand src = materialize(base);
  op.ref = src.ref;
  op.dtype = src.dtype;
  // element (i, j) of the view at base[off + i*rs + j*cs], composed from the base up
  int64_t off = 0, rs = 1, cs = src.ld;
  for (auto it = chain.rbegin(); it != chain.rend(); ++it) {
    const arma_node& v = nd_[*it];
    if (v.op == ARMA_OP_TRANS) std::swap(rs, cs);
    else off += (int64_t)v.slot * rs + v.ld * cs;   // SUBMAT: first row, first column
  }
  op.off = off;
  const NInfo& ti = info_[top];
  if (dg) {
    op.flags = EWF_DIAGMASK;
    if (ti.rows == 1 || ti.cols == 1) {   // vector v -> value v_i on (i, i)
      op.rs = (ti.rows == 1) ? cs : rs;
      op.cs = 0;
    } else {
      op.rs = rs; op.cs = cs;
    }
  } else {
    op.rs = rs; op.cs = cs;
  }
  int k = b.st.nin++;
  b.st.in[k] = op;
  b.leaf_node.push_back(y);
  return k;
}

bool Planner::sum_terms(int y, double sign, int root, bool top, std::vector<SumTerm>& t) const {
  if (t.size() > 16) return false;
  if (!top && ew_is_leaf(y, root)) { t.push_back({0, y, -1, sign}); return true; }
  const arma_node& d = nd_[y];
  switch (d.op) {
    case ARMA_OP_ADD:
      return sum_terms(d.a, sign, root, false, t) && sum_terms(d.b, sign, root, false, t);
    case ARMA_OP_SUB:
      return sum_terms(d.a, sign, root, false, t) && sum_terms(d.b, -sign, root, false, t);
    case ARMA_OP_NEG:
      return sum_terms(d.a, -sign, root, false, t);
    case ARMA_OP_SCALE:
      if (ew_is_leaf(d.a, root)) { t.push_back({0, d.a, -1, sign * d.scalar}); return true; }
      break;
    case ARMA_OP_DIV_SCALAR:
      if (ew_is_leaf(d.a, root)) { t.push_back({0, d.a, -1, sign / d.scalar}); return true; }
      break;
    case ARMA_OP_SCHUR:
      if (ew_is_leaf(d.a, root) && ew_is_leaf(d.b, root)) { t.push_back({1, d.a, d.b, sign}); return true; }
      break;
    default:
      break;
  }
  t.push_back({2, y, -1, sign});
  return true;
}

// A sum containing elementwise products of two leaves is evaluated as: the
// one general subtree (or a scaled leaf) first, then the other scaled leaves
// (fused multiply-adds), then each product as acc = +-x*y + acc (one fused
// multiply-add each).  A leading leaf whose coefficient is +-2^e is loaded
// with EW_LDP2, which FP64 passes apply to the exponent field exactly.  This
// is a reordering of the sum (rounding differs from left to right by a few
// units of the last place).
bool Planner::ew_sum(EwBuild& b, int y, int depth, int root) {
  std::vector<SumTerm> t;
  if (!sum_terms(y, 1.0, root, true, t)) return false;
  int nprod = 0, ngen = 0;
  for (const SumTerm& u : t) {
    nprod += u.kind == 1;
    ngen += u.kind == 2;
  }
  if (nprod == 0 || ngen > 1 || t.size() < 2) return false;
  auto pow2 = [](double c, int& e) {
    int ex = 0;
    const double m = std::frexp(std::fabs(c), &ex);
    e = ex - 1;
    return c != 0.0 && m == 0.5 && e >= -1000 && e <= 1000;
  };
  std::vector<char> done(t.size(), 0);
  // the first term: the general subtree, else a leaf (power-of-two
  // coefficient preferred), else the first product
  int first = -1;
  for (size_t i = 0; i < t.size() && first < 0; ++i)
    if (t[i].kind == 2) first = (int)i;
  int e2 = 0;
  for (size_t i = 0; i < t.size() && first < 0; ++i)
    if (t[i].kind == 0 && pow2(t[i].c, e2)) first = (int)i;
  for (size_t i = 0; i < t.size() && first < 0; ++i)
    if (t[i].kind == 0) first = (int)i;
  if (first < 0) first = 0;
  const SumTerm& f = t[first];
  done[first] = 1;
  if (f.kind == 2) {
    ew_compile(b, f.a, depth, root);
    if (f.c < 0) ew_emit(b, EW_NEG, 0, 0);
  } else if (f.kind == 0) {
    int e = 0;
    if (pow2(f.c, e)) ew_emit(b, EW_LDP2, ew_operand(b, f.a), f.c, e);
    else {
      ew_emit(b, EW_LD, ew_operand(b, f.a), 0);
      ew_emit(b, EW_SCAL, 0, f.c);
    }
  } else {
    ew_emit(b, EW_LD, ew_operand(b, f.a), 0);
    ew_emit(b, EW_MUL, ew_operand(b, f.b), 0);
    if (f.c < 0) ew_emit(b, EW_NEG, 0, 0);
  }
  for (size_t i = 0; i < t.size(); ++i) {
    if (done[i] || t[i].kind != 0) continue;
    const int k = ew_operand(b, t[i].a);
    if (t[i].c == 1.0) ew_emit(b, EW_ADD, k, 0);
    else if (t[i].c == -1.0) ew_emit(b, EW_SUB, k, 0);
    else ew_emit(b, EW_AXPY, k, t[i].c);
  }
  for (size_t i = 0; i < t.size(); ++i) {
    if (done[i] || t[i].kind != 1) continue;
    const int ka = ew_operand(b, t[i].a), kb = ew_operand(b, t[i].b);
    ew_emit(b, t[i].c > 0 ? EW_FMA : EW_FNMA, ka, 0, kb);
  }
  return true;
}

void Planner::ew_compile(EwBuild& b, int y, int depth, int root) {
  if (b.overflow) return;
  if (ew_is_leaf(y, root)) { ew_emit(b, EW_LD, ew_operand(b, y), 0); return; }
  const arma_node& d = nd_[y];
  switch (d.op) {
    case ARMA_OP_SCALE: ew_compile(b, d.a, depth, root); ew_emit(b, EW_SCAL, 0, d.scalar); return;
    case ARMA_OP_DIV_SCALAR: ew_compile(b, d.a, depth, root); ew_emit(b, EW_DIVS, 0, d.scalar); return;
    case ARMA_OP_ADD_SCALAR: ew_compile(b, d.a, depth, root); ew_emit(b, EW_ADDS, 0, d.scalar); return;
    case ARMA_OP_NEG: ew_compile(b, d.a, depth, root); ew_emit(b, EW_NEG, 0, 0); return;
    default: break;
  }
  if ((d.op == ARMA_OP_ADD || d.op == ARMA_OP_SUB) && !literal_ && ew_sum(b, y, depth, root))
    return;
  int A = d.a, B = d.b, op = d.op;
  static const int in_op[] = {0, EW_ADD, EW_SUB, EW_MUL, EW_DIV};
  static const int rev_op[] = {0, EW_ADD, EW_RSUB, EW_MUL, EW_RDIV};
  static const int pop_op[] = {0, EW_POPADD, EW_POPSUB, EW_POPMUL, EW_POPDIV};
  if (ew_is_leaf(B, root)) {
    ew_compile(b, A, depth, root);
    ew_emit(b, in_op[op], ew_operand(b, B), 0);
    return;
  }
  // a + s*z, a - s*z, a - z/s, a + (-z): one fused multiply-add
  if ((op == ARMA_OP_ADD || op == ARMA_OP_SUB) && !ew_is_leaf(B, root)) {
    const arma_node& bn = nd_[B];
    if ((bn.op == ARMA_OP_SCALE || bn.op == ARMA_OP_DIV_SCALAR || bn.op == ARMA_OP_NEG) &&
        ew_is_leaf(bn.a, root)) {
      double s = bn.op == ARMA_OP_SCALE ? bn.scalar : bn.op == ARMA_OP_NEG ? -1.0 : 1.0 / bn.scalar;
      if (op == ARMA_OP_SUB) s = -s;
      ew_compile(b, A, depth, root);
      ew_emit(b, EW_AXPY, ew_operand(b, bn.a), s);
      return;
    }
  }
  if (ew_is_leaf(A, root)) {
    ew_compile(b, B, depth, root);
    ew_emit(b, rev_op[op], ew_operand(b, A), 0);
    return;
  }
  if (depth >= kMaxStack) { b.overflow = true; return; }
  ew_compile(b, A, depth, root);
  ew_emit(b, EW_PUSH, depth, 0);
  ew_compile(b, B, depth + 1, root);
  ew_emit(b, pop_op[op], depth, 0);
}

// the instruction list of a fused pass, e.g. " ldp2 x2 -0.5; axpy x1 3; fma x0 x3"
static std::string ew_program_text(const EwStep& s) {
  static const char* names[] = {"ld", "add", "sub", "rsub", "mul", "div", "rdiv", "axpy", "scal", "divs",
                                "adds", "neg", "push", "popadd", "popsub", "popmul", "popdiv", "fma", "fnma",
                                "ldp2"};
  static_assert(sizeof(names) / sizeof(names[0]) == EW_NOPS, "one name per opcode");
  std::ostringstream os;
  os.precision(17);
  for (int i = 0; i < s.nops; ++i) {
    const EwIns& in = s.ops[i];
    os << (i ? "; " : " ") << names[in.op];
    switch (in.op) {
      case EW_LD: case EW_ADD: case EW_SUB: case EW_RSUB: case EW_MUL: case EW_DIV: case EW_RDIV:
        os << " x" << in.arg; break;
      case EW_AXPY: case EW_LDP2: os << " x" << in.arg << " " << in.s; break;
      case EW_SCAL: case EW_DIVS: case EW_ADDS: os << " " << in.s; break;
      case EW_FMA: case EW_FNMA: os << " x" << in.arg << " x" << in.arg2; break;
      case EW_PUSH: case EW_POPADD: case EW_POPSUB: case EW_POPMUL: case EW_POPDIV: os << " s" << in.arg; break;
      default: break;
    }
  }
  return os.str();
}

static double ew_bytes(const EwStep& s) {
  double b = 0;
  double elems = s.mode == EW_DIAG ? (double)std::min(s.m, s.n) : (double)s.m * (double)s.n;
  for (int k = 0; k < s.nin; ++k) {
    double e = elems;
    if (s.in[k].flags & EWF_DIAGMASK) e = (double)std::min(s.m, s.n);
    else if (s.in[k].cs == 0) e = (double)s.m;
    else if (s.in[k].rs == 0) e = (double)s.n;
    b += e * (double)dtype_size(s.in[k].dtype);
  }
  if (s.out.valid()) b += elems * (double)dtype_size(s.out_dtype);
  return b;
}

static bool ew_is_flat(const EwStep& s) {
  if (s.mode != EW_FLAT) return false;
  for (int k = 0; k < s.nin; ++k)
    if (s.in[k].flags || s.in[k].rs != 1 || (s.n > 1 && s.in[k].cs != s.m)) return false;
  if (s.out.valid() && s.n > 1 && s.out_ld != s.m) return false;
  return true;
}

// Plan the elementwise tree rooted at x as one fused pass.  If `dest` is
// given the result is stored there; if attach_reductions, accu/norm outputs
// of x are computed in the same pass.
void Planner::plan_ew_root(int x, const MatOperand* dest, bool diag_mode, Ref sum_out,
                           Ref norm_out, bool attach_reductions) {
  for (int attempt = 0; attempt < 64; ++attempt) {
    EwBuild b;
    ew_compile(b, x, 0, x);
    if (b.overflow) {
      // too large for one pass: materialise the right operand subtree of the
      // deepest binary chain and try again
      int y = x;
      while (is_ew_op(nd_[y].op) && !is_binary(nd_[y].op)) y = nd_[y].a;
      if (!is_binary(nd_[y].op) || ew_is_leaf(nd_[y].b, x)) {
        fail(ARMA_ERR_UNSUPPORTED, "elementwise expression too large to fuse");
        return;
      }
      int z = nd_[y].b;
      loc_[z] = dest_for(z);
      plan_ew_root(z, &loc_[z], false, Ref(), Ref(), false);
      continue;
    }
    EwStep& s = b.st;
    s.m = info_[x].rows;
    s.n = info_[x].cols;
    s.mode = diag_mode ? EW_DIAG : EW_FLAT;
    s.compute_f64 = info_[x].dtype == ARMA_F64 ? 1 : 0;
    if (dest) {
      s.out = dest->ref;
      s.out_ld = dest->ld;
      s.out_dtype = dest->dtype;
    }
    if (sum_out.valid()) { s.red |= 1; s.sum_out = sum_out; }
    if (norm_out.valid()) { s.red |= 2; s.norm_out = norm_out; }
    if (attach_reductions && !diag_mode) {
      for (int r = 0; r < (int)nd_.size(); ++r) {
        if (scalar_done_[r] || out_of_[r] < 0 || nd_[r].a != x) continue;
        if (nd_[r].op == ARMA_OP_ACCU && !(s.red & 1)) {
          s.red |= 1; s.sum_out = ref_output(out_of_[r]); scalar_done_[r] = 1;
        } else if (nd_[r].op == ARMA_OP_NORM_FRO && !(s.red & 2)) {
          s.red |= 2; s.norm_out = ref_output(out_of_[r]); scalar_done_[r] = 1;
        }
      }
    }
    if (!ew_is_flat(s) && s.mode == EW_FLAT) s.mode = EW_GRID;
    if (s.red) {
      s.partials = ref_ws(alloc_ws(2 * kMaxRedBlocks * sizeof(double)));
      s.ticket = alloc_ticket();
    }
    Step st;
    st.kind = ST_EW;
    st.ew = s;
    double elems = diag_mode ? (double)std::min(s.m, s.n) : (double)s.m * (double)s.n;
    st.flops = elems * (s.nops + ((s.red & 1) ? 1 : 0) + ((s.red & 2) ? 2 : 0));
    st.bytes = ew_bytes(s);
    std::ostringstream os;
    os << "fused elementwise pass (" << (s.mode == EW_FLAT ? "flat" : s.mode == EW_GRID ? "strided" : "diagonal")
       << ", " << s.nin << " operands, " << s.nops << " instructions"
       << (dest ? ", stored" : ", not stored") << ((s.red & 1) ? ", +sum" : "")
       << ((s.red & 2) ? ", +sumsq" : "") << ") for node " << x << "; program:" << ew_program_text(s);
    st.note = os.str();
    push_step(std::move(st));
    return;
  }
  fail(ARMA_ERR_UNSUPPORTED, "elementwise expression could not be split");
}

void Planner::emit_reduce(const MatOperand& src, int64_t m, int64_t n, bool diag, Ref sum_out,
                          Ref norm_out, const char* why) {
  EwStep s;
  s.m = m; s.n = n;
  s.mode = diag ? EW_DIAG : EW_FLAT;
  s.nin = 1;
  s.in[0].ref = src.ref;
  s.in[0].rs = 1;
  s.in[0].cs = src.ld;
  s.in[0].dtype = src.dtype;
  s.nops = 1;
  s.ops[0] = {EW_LD, 0, 0};
  s.compute_f64 = src.dtype == ARMA_F64 ? 1 : 0;
  if (sum_out.valid()) { s.red |= 1; s.sum_out = sum_out; }
  if (norm_out.valid()) { s.red |= 2; s.norm_out = norm_out; }
  if (!ew_is_flat(s) && s.mode == EW_FLAT) s.mode = EW_GRID;
  s.partials = ref_ws(alloc_ws(2 * kMaxRedBlocks * sizeof(double)));
  s.ticket = alloc_ticket();
  Step st;
  st.kind = ST_EW;
  st.ew = s;
  double elems = diag ? (double)std::min(m, n) : (double)m * (double)n;
  st.flops = elems * 2;
  st.bytes = ew_bytes(s);
  st.note = why;
  push_step(std::move(st));
}

void Planner::emit_gemm(int64_t m, int64_t n, int64_t k, const MatOperand& A, const MatOperand& B,
                        const MatOperand& D, double alpha, const MatOperand* C, double beta,
                        const VecOperand* rs, const VecOperand* cs, const char* why) {
  GemmStep g;
  g.m = m; g.n = n; g.k = k;
  g.A = A; g.B = B; g.D = D;
  g.alpha = alpha;
  if (C && beta != 0.0) { g.C = *C; g.beta = beta; }
  if (rs) g.rowscale = *rs;
  if (cs) g.colscale = *cs;
  int32_t dt = (A.dtype == ARMA_F64 && B.dtype == ARMA_F64) ? ARMA_F64
               : (A.dtype == ARMA_BF16 && B.dtype == ARMA_BF16) ? ARMA_BF16 : ARMA_F32;
  g.tier = product_tier(dt);
  // Symmetric products (Sec. II run-time analysis, Sec. III (8)): the same
  // value on both sides, one side transposed, no beta*C and no diagonal
  // scalings.  The same node is known now; two input slots of the same shape
  // and layout are compared by pointer at evaluation.
  if (!literal_ && !(e_.flags & ARMA_PLAN_NO_SYRK) && m == n && m > 1 && A.trans != B.trans &&
      A.dtype == B.dtype && A.ld == B.ld && !g.C.ref.valid() && !rs && !cs && A.ref.kind == B.ref.kind) {
    if (A.ref.same(B.ref)) g.sym = 1;
    else if (A.ref.kind == REF_INPUT) g.sym = 2;
  }
  g.nosplit = (e_.flags & ARMA_PLAN_NO_SPLITK) ? 1 : 0;
  g.split_req = (int32_t)((e_.flags & ARMA_PLAN_SPLITS_MASK) >> ARMA_PLAN_SPLITS_SHIFT);
  g.scratch_bytes = gemm_scratch_bytes(g);
  if (g.scratch_bytes > 0) g.scratch = ref_ws(alloc_ws(g.scratch_bytes));
  Step st;
  st.kind = ST_GEMM;
  st.gemm = g;
  // a symmetric product computes n (n + 1) / 2 of the n^2 dot products
  st.flops = g.sym == 1 ? (double)m * (double)(m + 1) * (double)k : 2.0 * (double)m * (double)n * (double)k;
  st.bytes = (double)(m * k) * dtype_size(A.dtype) + (double)(k * n) * dtype_size(B.dtype) +
             (double)(m * n) * dtype_size(D.dtype) * (g.C.ref.valid() ? 2.0 : 1.0);
  std::ostringstream os;
  os << (n == 1 || m == 1 ? "gemv" : g.sym == 1 ? "syrk" : "gemm") << " " << m << "x" << n << "x" << k
     << (g.sym == 2 ? " (symmetric if both slots hold the same matrix)" : "") << " op(A)="
     << (A.trans ? "T" : "N") << " op(B)=" << (B.trans ? "T" : "N") << " alpha=" << alpha
     << " beta=" << g.beta << (rs ? " rowscale" : "") << (cs ? " colscale" : "") << " tier="
     << tier_name(g.tier) << (g.nosplit ? " nosplit" : "")
     << (g.split_req > 0 && !g.nosplit ? " splits=" + std::to_string(g.split_req) : std::string()) << " (" << why << ")";
  st.note = os.str();
  push_step(std::move(st));
}

void Planner::emit_solve(const MatOperand& A, int64_t n, const MatOperand* B, int64_t nrhs,
                         const MatOperand& X, int32_t dt, bool explicit_inverse, const char* why) {
  SolveStep s;
  s.n = n; s.nrhs = B ? nrhs : n;
  s.A = A;
  if (B) s.B = *B;
  s.X = X;
  s.tier = solve_tier(dt);
  // an explicit inverse has no right-hand side to refine against: FP64 data
  // is factored in FP64 (the paper's naive GETRF + GETRI in the data's type)
  if (explicit_inverse && dt == ARMA_F64 &&
      (e_.tier == ARMA_TIER_NATIVE || e_.tier == ARMA_TIER_LU32_IR64 || e_.tier == ARMA_TIER_F64_SLICED))
    s.tier = ARMA_TIER_F64;
  s.explicit_inverse = explicit_inverse ? 1 : 0;
  // the run-time analysis that picks a diagonal, band or triangular solver
  // (Sec. III (10)); the literal plan and explicit inverses factor densely
  s.analyse = (!literal_ && !explicit_inverse && !(e_.flags & ARMA_PLAN_NO_SOLVE_ANALYSIS)) ? 1 : 0;
  const uint32_t ir = (e_.flags & ARMA_PLAN_REFINE_MASK) >> ARMA_PLAN_REFINE_SHIFT;
  s.max_ir = ir ? (int32_t)ir : 10;
  s.dfma_residual = (e_.flags & ARMA_PLAN_DFMA_RESIDUAL) ? 1 : 0;
  s.no_lookahead = (e_.flags & ARMA_PLAN_NO_LOOKAHEAD) ? 1 : 0;
  s.scratch_bytes = solve_scratch_bytes(n, s.nrhs, s.tier, s.analyse, s.dfma_residual);
  s.scratch = ref_ws(alloc_ws(s.scratch_bytes));
  Step st;
  st.kind = ST_SOLVE;
  st.solve = s;
  double dn = (double)n;
  st.flops = 2.0 / 3.0 * dn * dn * dn + 2.0 * dn * dn * (double)s.nrhs;
  st.bytes = dn * dn * dtype_size(A.dtype) + 2.0 * dn * (double)s.nrhs * dtype_size(X.dtype);
  std::ostringstream os;
  os << (s.analyse ? "analysed solve (diagonal / band / triangular / LU) n=" : "LU solve n=") << n
     << " nrhs=" << s.nrhs << " tier=" << tier_name(s.tier) << " (" << why << ")";
  st.note = os.str();
  push_step(std::move(st));
}

// Collect the factors of a product tree, folding scalars into alpha and
// transposes into operand flags (Sec. II: glue_times carries the scalar
// and transpose flags into one xGEMM call, Fig. 3).
void Planner::flatten_product(int x, double& alpha, std::vector<Factor>& f) {
  const arma_node& d = nd_[x];
  bool inner = !loc_[x].ref.valid() && uses_[x] <= 1 && out_of_[x] < 0;
  if (inner) {
    if (d.op == ARMA_OP_MATMUL) {
      flatten_product(d.a, alpha, f);
      flatten_product(d.b, alpha, f);
      return;
    }
    if (d.op == ARMA_OP_SCALE) { alpha *= d.scalar; flatten_product(d.a, alpha, f); return; }
    if (d.op == ARMA_OP_NEG) { alpha = -alpha; flatten_product(d.a, alpha, f); return; }
    if (d.op == ARMA_OP_DIV_SCALAR) { alpha /= d.scalar; flatten_product(d.a, alpha, f); return; }
  }
  Factor fc;
  fc.rows = info_[x].rows;
  fc.cols = info_[x].cols;
  fc.dtype = info_[x].dtype;
  if (!loc_[x].ref.valid() && d.op == ARMA_OP_TRANS) {
    fc.m = materialize(d.a);
    fc.m.trans = 1;
    f.push_back(fc);
    return;
  }
  if (!loc_[x].ref.valid() && d.op == ARMA_OP_DIAGMAT) {
    const NInfo& v = info_[d.a];
    MatOperand src = materialize(d.a);
    fc.kind = Factor::DIAG;
    fc.v.ref = src.ref;
    fc.v.dtype = src.dtype;
    if (v.rows == 1 || v.cols == 1) {
      fc.v.inc = (v.rows == 1) ? src.ld : 1;
      f.push_back(fc);
      return;
    }
    if (v.rows == v.cols) {   // diagmat of a square matrix: its diagonal, stride ld+1
      fc.v.inc = src.ld + 1;
      f.push_back(fc);
      return;
    }
    fc.kind = Factor::DENSE;
    fc.m = materialize(x);
    f.push_back(fc);
    return;
  }
  if (!loc_[x].ref.valid() && d.op == ARMA_OP_INV) {
    fc.kind = Factor::INV;
    fc.m = materialize(d.a);
    f.push_back(fc);
    return;
  }
  fc.m = materialize(x);
  f.push_back(fc);
}

static int64_t op_rows(const Factor& f) { return f.rows; }
static int64_t op_cols(const Factor& f) { return f.cols; }

MatOperand Planner::eval_chain(std::vector<Factor>& dense, int64_t lo, int64_t hi,
                               const std::vector<ChainTree>& t, int node, const MatOperand* dest,
                               double alpha, const MatOperand* C, double beta,
                               const VecOperand* rs, const VecOperand* cs) {
  const ChainTree& c = t[node];
  if (c.lo == c.hi) return dense[c.lo].m;
  MatOperand L = eval_chain(dense, lo, hi, t, c.left, nullptr, 1.0, nullptr, 0.0, nullptr, nullptr);
  MatOperand R = eval_chain(dense, lo, hi, t, c.right, nullptr, 1.0, nullptr, 0.0, nullptr, nullptr);
  int64_t m = op_rows(dense[c.lo]);
  int64_t k = op_cols(dense[c.k]);
  int64_t n = op_cols(dense[c.hi]);
  int32_t dt = (L.dtype == ARMA_F64 && R.dtype == ARMA_F64) ? ARMA_F64 : ARMA_F32;
  MatOperand D = dest ? *dest : temp_mat(m, n, dt);
  D.trans = 0;
  emit_gemm(m, n, k, L, R, D, alpha, C, beta, rs, cs,
            dest ? "product root" : "chain intermediate");
  return D;
}

void Planner::plan_product(int x, MatOperand dest, double alpha_extra, const MatOperand* C,
                           double beta) {
  double alpha = alpha_extra;
  std::vector<Factor> f;
  // flatten the top node even if it is an output: its own factors are inner
  const arma_node& d = nd_[x];
  if (d.op == ARMA_OP_MATMUL) {
    flatten_product(d.a, alpha, f);
    flatten_product(d.b, alpha, f);
  } else {
    flatten_product(x, alpha, f);
  }
  if (err_ != ARMA_OK) return;
  // inv(A) * rest -> solve (Sec. I; Sec. II inv pattern; Sec. III (9))
  for (size_t i = 0; i < f.size(); ++i) {
    if (f[i].kind != Factor::INV) continue;
    if (i == 0 && f.size() > 1) {
      // right-hand side: product of the remaining factors
      std::vector<Factor> rest(f.begin() + 1, f.end());
      int64_t n = f[0].rows;
      int64_t nrhs = rest.back().cols;
      MatOperand rhs;
      bool rhs_plain = rest.size() == 1 && rest[0].kind == Factor::DENSE && !rest[0].m.trans;
      if (rhs_plain) {
        rhs = rest[0].m;
      } else {
        // materialise the right-hand side as its own chain
        bool all_dense = true;
        for (auto& r : rest) all_dense &= r.kind == Factor::DENSE;
        if (!all_dense) { fail(ARMA_ERR_UNSUPPORTED, "inv(A) followed by diagonal factors"); return; }
        std::vector<int64_t> dims;
        dims.push_back(rest[0].rows);
        for (auto& r : rest) dims.push_back(r.cols);
        rhs = temp_mat(n, nrhs, rest[0].dtype == ARMA_F64 ? ARMA_F64 : ARMA_F32);
        if (rest.size() == 1) {
          // inv(A) * trans(B): the right-hand side needs an explicit transpose
          Step st;
          st.kind = ST_TRANSPOSE;
          st.cm = rest[0].cols; st.cn = rest[0].rows;
          st.csrc = rest[0].m; st.csrc.trans = 0;
          st.cdst = rhs;
          st.bytes = 2.0 * (double)(st.cm * st.cn) * dtype_size(rhs.dtype);
          st.note = "transposed right-hand side of a solve";
          push_step(std::move(st));
        } else {
        std::vector<ChainTree> t;
        int root;
        chain_order((int)rest.size(), dims.data(), chain_method_, t, root);
        eval_chain(rest, 0, (int64_t)rest.size() - 1, t, root, &rhs, 1.0, nullptr, 0, nullptr, nullptr);
        }
      }
      bool direct = f.size() == 2 && alpha == 1.0 && !C;
      MatOperand X = direct ? dest : temp_mat(n, nrhs, f[0].dtype);
      emit_solve(f[0].m, n, &rhs, nrhs, X, f[0].dtype, false, "inv(A)*B rewritten as a solve");
      if (direct) { loc_[x] = dest; return; }
      Factor fx;
      fx.kind = Factor::DENSE;
      fx.m = X;
      fx.rows = n; fx.cols = nrhs; fx.dtype = X.dtype;
      f.erase(f.begin() + 1, f.end());
      f[0] = fx;
      break;
    }
    // elsewhere: explicit inverse
    int64_t n = f[i].rows;
    MatOperand X = temp_mat(n, n, f[i].dtype);
    emit_solve(f[i].m, n, nullptr, n, X, f[i].dtype, true, "inv(A) not leading a product: explicit inverse");
    f[i].kind = Factor::DENSE;
    f[i].m = X;
  }
  // a^T diagmat(X) c (a, c vectors): sum_i a_i X_ii c_i in one strided
  // elementwise pass with a reduction (Sec. III (7)), no dense diagonal
  if (!literal_ && f.size() == 3 && f[0].kind == Factor::DENSE && f[0].rows == 1 && f[1].kind == Factor::DIAG &&
      f[2].kind == Factor::DENSE && f[2].cols == 1 && info_[x].rows == 1 && info_[x].cols == 1) {
    const int64_t len = f[1].rows;
    EwStep s;
    s.m = len;
    s.n = 1;
    s.mode = EW_FLAT;
    s.compute_f64 = dest.dtype == ARMA_F64 ? 1 : 0;
    // element i of a 1 x len factor / len x 1 factor, as a stride from its base
    auto stride_of = [](const MatOperand& m, bool row_vec) -> int64_t {
      return row_vec ? (m.trans ? 1 : m.ld) : (m.trans ? m.ld : 1);
    };
    s.in[0].ref = f[0].m.ref; s.in[0].dtype = f[0].m.dtype; s.in[0].rs = stride_of(f[0].m, true); s.in[0].cs = 0;
    s.in[1].ref = f[1].v.ref; s.in[1].dtype = f[1].v.dtype; s.in[1].rs = f[1].v.inc; s.in[1].cs = 0;
    s.in[2].ref = f[2].m.ref; s.in[2].dtype = f[2].m.dtype; s.in[2].rs = stride_of(f[2].m, false); s.in[2].cs = 0;
    s.nin = 3;
    s.ops[s.nops++] = {EW_LD, 0, 0};
    s.ops[s.nops++] = {EW_MUL, 1, 0};
    s.ops[s.nops++] = {EW_MUL, 2, 0};
    if (alpha != 1.0) s.ops[s.nops++] = {EW_SCAL, 0, alpha};
    const bool direct = dest.dtype == ARMA_F64;
    MatOperand acc = direct ? dest : temp_mat(1, 1, ARMA_F64);
    s.red = 1;
    s.sum_out = acc.ref;
    s.partials = ref_ws(alloc_ws(2 * kMaxRedBlocks * sizeof(double)));
    s.ticket = alloc_ticket();
    if (!ew_is_flat(s)) s.mode = EW_GRID;
    Step st;
    st.kind = ST_EW;
    st.ew = s;
    st.flops = 3.0 * (double)len;
    st.bytes = ew_bytes(s);
    st.note = "a'*diagmat(X)*c as one diagonal reduction pass (no dense diagonal, no product)";
    push_step(std::move(st));
    if (!direct) {   // the FP64 sum stored in the product's element type
      EwStep c;
      c.m = 1; c.n = 1;
      c.mode = EW_GRID;
      c.in[0].ref = acc.ref; c.in[0].dtype = ARMA_F64; c.in[0].rs = 1; c.in[0].cs = 1;
      c.nin = 1;
      c.ops[c.nops++] = {EW_LD, 0, 0};
      c.out = dest.ref; c.out_ld = dest.ld; c.out_dtype = dest.dtype;
      Step sc;
      sc.kind = ST_EW;
      sc.ew = c;
      sc.bytes = 8.0 + dtype_size(dest.dtype);
      sc.note = "sum stored in the result's element type";
      push_step(std::move(sc));
    }
    loc_[x] = dest;
    return;
  }
  // leading / trailing diagonal factors become row / column scalings
  VecOperand rs, cs;
  bool has_rs = false, has_cs = false;
  size_t b0 = 0, e0 = f.size();
  if (f.size() >= 2 && f[0].kind == Factor::DIAG) { rs = f[0].v; has_rs = true; b0 = 1; }
  if (e0 - b0 >= 2 && f[e0 - 1].kind == Factor::DIAG) { cs = f[e0 - 1].v; has_cs = true; e0--; }
  std::vector<Factor> dense(f.begin() + b0, f.begin() + e0);
  for (auto& q : dense) {
    if (q.kind == Factor::DIAG) {   // interior diagonal: build it densely
      MatOperand M = temp_mat(q.rows, q.cols, q.dtype);
      Step st;
      st.kind = ST_DIAGBUILD;
      st.cm = q.rows; st.cn = q.cols;
      st.csrc.ref = q.v.ref; st.csrc.dtype = q.v.dtype;
      st.cinc = q.v.inc;
      st.cdst = M;
      st.bytes = (double)(q.rows * q.cols) * dtype_size(q.dtype);
      st.note = "interior diagmat built densely";
      push_step(std::move(st));
      q.kind = Factor::DENSE;
      q.m = M;
    }
  }
  if (dense.empty()) { fail(ARMA_ERR_UNSUPPORTED, "product of diagonal matrices only"); return; }
  if (dense.size() == 1) {
    // alpha * diag(r) * op(F) * diag(c) (+ beta C): one elementwise pass
    EwStep s;
    s.m = info_[x].rows;
    s.n = info_[x].cols;
    s.mode = EW_FLAT;
    s.compute_f64 = dest.dtype == ARMA_F64 ? 1 : 0;
    const MatOperand& F = dense[0].m;
    s.in[0].ref = F.ref;
    s.in[0].dtype = F.dtype;
    if (F.trans) { s.in[0].rs = F.ld; s.in[0].cs = 1; } else { s.in[0].rs = 1; s.in[0].cs = F.ld; }
    s.nin = 1;
    s.ops[s.nops++] = {EW_LD, 0, 0};
    if (has_rs) {
      s.in[s.nin] = EwOperand();
      s.in[s.nin].ref = rs.ref; s.in[s.nin].rs = rs.inc; s.in[s.nin].cs = 0; s.in[s.nin].dtype = rs.dtype;
      s.ops[s.nops++] = {EW_MUL, s.nin, 0};
      s.nin++;
    }
    if (has_cs) {
      s.in[s.nin] = EwOperand();
      s.in[s.nin].ref = cs.ref; s.in[s.nin].rs = 0; s.in[s.nin].cs = cs.inc; s.in[s.nin].dtype = cs.dtype;
      s.ops[s.nops++] = {EW_MUL, s.nin, 0};
      s.nin++;
    }
    if (alpha != 1.0) s.ops[s.nops++] = {EW_SCAL, 0, alpha};
    if (C && beta != 0.0) {
      s.in[s.nin] = EwOperand();
      s.in[s.nin].ref = C->ref; s.in[s.nin].rs = 1; s.in[s.nin].cs = C->ld; s.in[s.nin].dtype = C->dtype;
      s.ops[s.nops++] = {EW_AXPY, s.nin, beta};
      s.nin++;
    }
    s.out = dest.ref;
    s.out_ld = dest.ld;
    s.out_dtype = dest.dtype;
    if (!ew_is_flat(s)) s.mode = EW_GRID;
    Step st;
    st.kind = ST_EW;
    st.ew = s;
    st.flops = (double)s.m * s.n * s.nops;
    st.bytes = ew_bytes(s);
    st.note = has_rs || has_cs ? "diagmat(v)*B as a row/column scaling pass (no dense diagonal, no product)"
                               : "scaled single factor as an elementwise pass";
    push_step(std::move(st));
    loc_[x] = dest;
    return;
  }
  std::vector<int64_t> dims;
  dims.push_back(dense[0].rows);
  for (auto& q : dense) dims.push_back(q.cols);
  std::vector<ChainTree> t;
  int root;
  chain_order((int)dense.size(), dims.data(), chain_method_, t, root);
  eval_chain(dense, 0, (int64_t)dense.size() - 1, t, root, &dest, alpha, C, beta,
             has_rs ? &rs : nullptr, has_cs ? &cs : nullptr);
  loc_[x] = dest;
}

// x = sum_t c_t * term_t through +, -, scalar *, /scalar, unary minus
void Planner::linearize(int x, double c, std::vector<std::pair<int, double>>& terms, bool top) {
  const arma_node& d = nd_[x];
  bool inner = top || (!loc_[x].ref.valid() && uses_[x] <= 1 && out_of_[x] < 0);
  if (inner) {
    switch (d.op) {
      case ARMA_OP_ADD: linearize(d.a, c, terms, false); linearize(d.b, c, terms, false); return;
      case ARMA_OP_SUB: linearize(d.a, c, terms, false); linearize(d.b, -c, terms, false); return;
      case ARMA_OP_SCALE: linearize(d.a, c * d.scalar, terms, false); return;
      case ARMA_OP_NEG: linearize(d.a, -c, terms, false); return;
      case ARMA_OP_DIV_SCALAR: linearize(d.a, c / d.scalar, terms, false); return;
      default: break;
    }
  }
  terms.push_back({x, c});
}

MatOperand Planner::materialize(int x) {
  if (loc_[x].ref.valid()) return loc_[x];
  const arma_node& d = nd_[x];
  if (d.op == ARMA_OP_INPUT) {
    MatOperand m;
    m.ref = ref_input(d.slot);
    m.ld = d.ld;
    m.dtype = d.dtype;
    loc_[x] = m;
    return m;
  }
  if (err_ != ARMA_OK) return MatOperand();
  // a submatrix of a matrix (no transpose on the way) is that matrix's
  // buffer at an offset with the same leading dimension: read in place by
  // every kernel, no copy (Sec. III (2)); an output still gets its copy
  if (d.op == ARMA_OP_SUBMAT && out_of_[x] < 0 && !literal_) {
    int z = d.a;
    while (!loc_[z].ref.valid() && nd_[z].op == ARMA_OP_SUBMAT) z = nd_[z].a;
    if (loc_[z].ref.valid() || nd_[z].op != ARMA_OP_TRANS) {
      MatOperand base = materialize(d.a);
      if (err_ != ARMA_OK) return MatOperand();
      if (!base.trans) {
        MatOperand v = base;
        v.ref.boff += ((int64_t)d.slot + (int64_t)d.ld * base.ld) * (int64_t)dtype_size(base.dtype);
        loc_[x] = v;
        return v;
      }
    }
  }
  MatOperand dest = dest_for(x);
  switch (d.op) {
    case ARMA_OP_MATMUL:
      plan_product(x, dest, 1.0, nullptr, 0.0);
      break;
    case ARMA_OP_TRANS: {
      MatOperand src = materialize(d.a);
      Step st;
      st.kind = ST_TRANSPOSE;
      st.cm = info_[d.a].rows; st.cn = info_[d.a].cols;
      st.csrc = src; st.cdst = dest;
      st.bytes = 2.0 * (double)(st.cm * st.cn) * dtype_size(src.dtype);
      st.note = "explicit transpose (result needed as a matrix)";
      push_step(std::move(st));
      break;
    }
    case ARMA_OP_DIAGMAT: {
      const NInfo& v = info_[d.a];
      const arma_node& ad = nd_[d.a];
      const bool a_inner = !loc_[d.a].ref.valid() && uses_[d.a] <= 1 && out_of_[d.a] < 0;
      const bool scaled = ad.op == ARMA_OP_SCALE || ad.op == ARMA_OP_NEG || ad.op == ARMA_OP_DIV_SCALAR;
      if (!literal_ && a_inner && (ad.op == ARMA_OP_MATMUL || scaled) && v.rows > 1 && v.cols > 1) {
        // diagmat(s*A*B): only the diagonal of the product (Sec. III (4)),
        // then the diagonal placed into the zero matrix
        double alpha = 1.0;
        std::vector<Factor> f;
        flatten_product(d.a, alpha, f);
        bool two_dense = f.size() == 2 && f[0].kind == Factor::DENSE && f[1].kind == Factor::DENSE;
        if (two_dense) {
          const int64_t dn = std::min(v.rows, v.cols);
          MatOperand dv = temp_mat(dn, 1, ARMA_F64);
          DotStep ds;
          ds.m = f[0].rows; ds.k = f[0].cols; ds.n = f[1].cols;
          ds.A = f[0].m; ds.B = f[1].m;
          ds.alpha = alpha;
          ds.out = dv.ref;
          ds.per_diag = 1;
          ds.partials = ref_ws(alloc_ws((int64_t)DIAGVEC_MAX_CHUNKS * dn * (int64_t)sizeof(double)));
          Step st;
          st.kind = ST_DOT;
          st.dot = ds;
          st.flops = 2.0 * (double)dn * (double)ds.k;
          st.bytes = (double)dn * (double)ds.k * (dtype_size(ds.A.dtype) + dtype_size(ds.B.dtype));
          st.note = "diagmat(A*B) as a diagonal-only product: d_i = sum_l A_il B_li";
          push_step(std::move(st));
          Step sb;
          sb.kind = ST_DIAGBUILD;
          sb.cm = info_[x].rows; sb.cn = info_[x].cols;
          sb.csrc = dv;
          sb.cinc = 1;
          sb.cdst = dest;
          sb.bytes = (double)(sb.cm * sb.cn) * dtype_size(dest.dtype);
          sb.note = "the product's diagonal placed into the result";
          push_step(std::move(sb));
          break;
        }
      }
      if (v.rows == 1 || v.cols == 1) {
        MatOperand src = materialize(d.a);
        Step st;
        st.kind = ST_DIAGBUILD;
        st.cm = info_[x].rows; st.cn = info_[x].cols;
        st.csrc = src;
        st.cinc = v.rows == 1 ? src.ld : 1;
        st.cdst = dest;
        st.bytes = (double)(st.cm * st.cn) * dtype_size(dest.dtype);
        st.note = "diagmat(v) built densely (result needed as a matrix)";
        push_step(std::move(st));
      } else {
        // diagmat(X) of any other matrix: X (materialised), its off-diagonal
        // zeroed in one pass
        MatOperand src = materialize(d.a);
        if (err_ != ARMA_OK) break;
        EwStep s;
        s.m = info_[x].rows; s.n = info_[x].cols;
        s.mode = EW_GRID;
        s.compute_f64 = info_[x].dtype == ARMA_F64 ? 1 : 0;
        s.in[0].ref = src.ref; s.in[0].rs = 1; s.in[0].cs = src.ld;
        s.in[0].dtype = src.dtype; s.in[0].flags = EWF_DIAGMASK;
        s.nin = 1;
        s.ops[s.nops++] = {EW_LD, 0, 0};
        s.out = dest.ref; s.out_ld = dest.ld; s.out_dtype = dest.dtype;
        Step st;
        st.kind = ST_EW;
        st.ew = s;
        st.bytes = ew_bytes(s);
        st.note = "diagmat of a materialised matrix (off-diagonal zeroed)";
        push_step(std::move(st));
      }
      break;
    }
    case ARMA_OP_INV: {
      MatOperand A = materialize(d.a);
      emit_solve(A, info_[x].rows, nullptr, info_[x].rows, dest, info_[x].dtype, true,
                 "inv(A) needed as a matrix");
      break;
    }
    case ARMA_OP_SOLVE: {
      MatOperand A = materialize(d.a), B = materialize(d.b);
      emit_solve(A, info_[x].rows, &B, info_[x].cols, dest, info_[x].dtype, false, "solve(A, B)");
      break;
    }
    case ARMA_OP_SUBMAT: {
      // a view needed as a matrix of its own: one copy pass reading it in place
      EwBuild b;
      const int k = ew_operand(b, x);
      if (b.overflow || err_ != ARMA_OK) { if (err_ == ARMA_OK) fail(ARMA_ERR_UNSUPPORTED, "submat view"); break; }
      EwStep& s = b.st;
      s.ops[s.nops++] = {EW_LD, k, 0};
      s.m = info_[x].rows; s.n = info_[x].cols;
      s.mode = EW_FLAT;
      s.compute_f64 = info_[x].dtype == ARMA_F64 ? 1 : 0;
      s.out = dest.ref; s.out_ld = dest.ld; s.out_dtype = dest.dtype;
      if (!ew_is_flat(s)) s.mode = EW_GRID;
      Step st;
      st.kind = ST_EW;
      st.ew = s;
      st.bytes = ew_bytes(s);
      st.note = "submatrix view copied (result needed as a matrix)";
      push_step(std::move(st));
      break;
    }
    default: {
      if (!is_ew_op(d.op)) { fail(ARMA_ERR_UNSUPPORTED, "cannot materialise node"); break; }
      // 2*A*B + C and friends: one product term plus an elementwise rest
      std::vector<std::pair<int, double>> terms;
      linearize(x, 1.0, terms, true);
      int prod = -1, nprod = 0;
      for (size_t t = 0; t < terms.size(); ++t) {
        int y = terms[t].first;
        if (nd_[y].op == ARMA_OP_MATMUL && !loc_[y].ref.valid() && uses_[y] <= 1 && out_of_[y] < 0) {
          nprod++;
          prod = (int)t;
        }
      }
      if (fuse_ && nprod == 1 && terms.size() >= 1) {
        int P = terms[prod].first;
        double cP = terms[prod].second;
        std::vector<std::pair<int, double>> rest;
        for (size_t t = 0; t < terms.size(); ++t)
          if ((int)t != prod) rest.push_back(terms[t]);
        if (rest.empty()) {
          plan_product(P, dest, cP, nullptr, 0.0);
        } else if (rest.size() == 1 && ew_leafable_view(rest[0].first) &&
                   nd_[rest[0].first].op != ARMA_OP_TRANS && nd_[rest[0].first].op != ARMA_OP_DIAGMAT) {
          MatOperand Cm = materialize(rest[0].first);
          plan_product(P, dest, cP, &Cm, rest[0].second);
        } else {
          // evaluate the elementwise rest into dest, then accumulate the product
          // build a synthetic linear combination by compiling the rest terms
          EwBuild b;
          bool first = true;
          for (auto& tc : rest) {
            int y = tc.first;
            if (ew_is_leaf(y, -1)) {
              int k = ew_operand(b, y);
              if (first) { ew_emit(b, EW_LD, k, 0); if (tc.second != 1.0) ew_emit(b, EW_SCAL, 0, tc.second); }
              else ew_emit(b, EW_AXPY, k, tc.second);
            } else {
              if (!first) ew_emit(b, EW_PUSH, 0, 0);
              ew_compile(b, y, first ? 0 : 1, y);
              if (tc.second != 1.0) ew_emit(b, EW_SCAL, 0, tc.second);
              if (!first) ew_emit(b, EW_POPADD, 0, 0);
            }
            first = false;
          }
          if (b.overflow) { fail(ARMA_ERR_UNSUPPORTED, "elementwise rest too large"); break; }
          EwStep& s = b.st;
          s.m = info_[x].rows; s.n = info_[x].cols;
          s.mode = EW_FLAT;
          s.compute_f64 = info_[x].dtype == ARMA_F64 ? 1 : 0;
          s.out = dest.ref; s.out_ld = dest.ld; s.out_dtype = dest.dtype;
          if (!ew_is_flat(s)) s.mode = EW_GRID;
          Step st;
          st.kind = ST_EW;
          st.ew = s;
          st.flops = (double)s.m * s.n * s.nops;
          st.bytes = ew_bytes(s);
          st.note = "elementwise addend evaluated into the product's output";
          push_step(std::move(st));
          plan_product(P, dest, cP, &dest, 1.0);
        }
        loc_[x] = dest;
        break;
      }
      if (!fuse_) {
        // one kernel per elementwise operator, but with the other rewrites
        const arma_node& n2 = nd_[x];
        EwBuild b;
        MatOperand A = materialize(n2.a);
        (void)A;
        int ka = ew_operand(b, n2.a);
        ew_emit(b, EW_LD, ka, 0);
        if (is_binary(n2.op)) {
          materialize(n2.b);
          int kb = ew_operand(b, n2.b);
          static const int in_op[] = {0, EW_ADD, EW_SUB, EW_MUL, EW_DIV};
          ew_emit(b, in_op[n2.op], kb, 0);
        } else {
          int o = n2.op == ARMA_OP_SCALE ? EW_SCAL : n2.op == ARMA_OP_DIV_SCALAR ? EW_DIVS
                  : n2.op == ARMA_OP_ADD_SCALAR ? EW_ADDS : EW_NEG;
          ew_emit(b, o, 0, n2.scalar);
        }
        EwStep& s = b.st;
        s.m = info_[x].rows; s.n = info_[x].cols;
        s.mode = EW_FLAT;
        s.compute_f64 = info_[x].dtype == ARMA_F64 ? 1 : 0;
        s.out = dest.ref; s.out_ld = dest.ld; s.out_dtype = dest.dtype;
        if (!ew_is_flat(s)) s.mode = EW_GRID;
        Step st;
        st.kind = ST_EW;
        st.ew = s;
        st.flops = (double)s.m * s.n;
        st.bytes = ew_bytes(s);
        st.note = std::string("unfused elementwise ") + op_name(n2.op);
        push_step(std::move(st));
        loc_[x] = dest;
        return dest;
      }
      plan_ew_root(x, &dest, false, Ref(), Ref(), true);
      break;
    }
  }
  loc_[x] = dest;
  return dest;
}

void Planner::plan_scalar(int r) {
  if (scalar_done_[r]) return;
  scalar_done_[r] = 1;
  const arma_node& d = nd_[r];
  int x = d.a;
  // trace(X^T) = trace(X) (the same diagonal elements, summed in the same
  // order); accu and the Frobenius norm sum every element, so they too are
  // those of X up to the order of the sum.  A transpose that only this
  // reduction uses is looked through, so the rewrites below see X itself and
  // no transpose is materialised.
  while (nd_[x].op == ARMA_OP_TRANS && !loc_[x].ref.valid() && uses_[x] <= 1 && out_of_[x] < 0) x = nd_[x].a;
  Ref out = ref_output(out_of_[r]);
  const arma_node& xd = nd_[x];
  bool x_inner = !loc_[x].ref.valid() && uses_[x] <= 1 && out_of_[x] < 0;
  if (d.op == ARMA_OP_TRACE) {
    if (x_inner && xd.op == ARMA_OP_MATMUL) {
      // trace(A*B): only the diagonal of the product (Sec. III (5))
      double alpha = 1.0;
      std::vector<Factor> f;
      flatten_product(xd.a, alpha, f);
      flatten_product(xd.b, alpha, f);
      bool all_dense = true;
      for (auto& q : f) all_dense &= q.kind == Factor::DENSE;
      if (all_dense && f.size() >= 2) {
        if (f.size() > 2) {
          // trace(F1 ... Fn) = trace((F1 ... Fn-1) Fn): materialise the left part
          std::vector<Factor> left(f.begin(), f.end() - 1);
          std::vector<int64_t> dims;
          dims.push_back(left[0].rows);
          for (auto& q : left) dims.push_back(q.cols);
          std::vector<ChainTree> t;
          int root;
          chain_order((int)left.size(), dims.data(), chain_method_, t, root);
          MatOperand L = temp_mat(left[0].rows, left.back().cols,
                                  left[0].dtype == ARMA_F64 ? ARMA_F64 : ARMA_F32);
          eval_chain(left, 0, (int64_t)left.size() - 1, t, root, &L, 1.0, nullptr, 0, nullptr, nullptr);
          Factor fl;
          fl.m = L; fl.rows = left[0].rows; fl.cols = left.back().cols; fl.dtype = L.dtype;
          Factor last = f.back();
          f.clear();
          f.push_back(fl);
          f.push_back(last);
        }
        DotStep s;
        s.m = f[0].rows; s.k = f[0].cols; s.n = f[1].cols;
        s.A = f[0].m; s.B = f[1].m;
        s.alpha = alpha;
        s.out = out;
        s.partials = ref_ws(alloc_ws(2 * kMaxRedBlocks * sizeof(double)));
        s.ticket = alloc_ticket();
        Step st;
        st.kind = ST_DOT;
        st.dot = s;
        double dm = (double)std::min(s.m, s.n);
        st.flops = 2.0 * dm * (double)s.k;
        st.bytes = dm * (double)s.k * (dtype_size(s.A.dtype) + dtype_size(s.B.dtype));
        st.note = "trace(A*B) as a diagonal-only product: sum_i sum_l A_il B_li";
        push_step(std::move(st));
        return;
      }
    }
    if (x_inner && is_ew_op(xd.op)) {
      plan_ew_root(x, nullptr, true, out, Ref(), false);
      return;
    }
    MatOperand m = materialize(x);
    emit_reduce(m, info_[x].rows, info_[x].cols, true, out, Ref(), "trace of a materialised matrix");
    return;
  }
  // accu / norm
  Ref sum_out = d.op == ARMA_OP_ACCU ? out : Ref();
  Ref norm_out = d.op == ARMA_OP_NORM_FRO ? out : Ref();
  if (x_inner && is_ew_op(xd.op) && fuse_) {
    // not needed as a matrix: one pass with no store, sharing with sibling reductions
    for (int r2 = 0; r2 < (int)nd_.size(); ++r2) {
      if (r2 == r || scalar_done_[r2] || out_of_[r2] < 0 || nd_[r2].a != x) continue;
      if (nd_[r2].op == ARMA_OP_ACCU && !sum_out.valid()) { sum_out = ref_output(out_of_[r2]); scalar_done_[r2] = 1; }
      if (nd_[r2].op == ARMA_OP_NORM_FRO && !norm_out.valid()) { norm_out = ref_output(out_of_[r2]); scalar_done_[r2] = 1; }
    }
    plan_ew_root(x, nullptr, false, sum_out, norm_out, false);
    return;
  }
  MatOperand m = materialize(x);
  if (fuse_) {
    for (int r2 = 0; r2 < (int)nd_.size(); ++r2) {
      if (r2 == r || scalar_done_[r2] || out_of_[r2] < 0 || nd_[r2].a != x) continue;
      if (nd_[r2].op == ARMA_OP_ACCU && !sum_out.valid()) { sum_out = ref_output(out_of_[r2]); scalar_done_[r2] = 1; }
      if (nd_[r2].op == ARMA_OP_NORM_FRO && !norm_out.valid()) { norm_out = ref_output(out_of_[r2]); scalar_done_[r2] = 1; }
    }
  }
  emit_reduce(m, info_[x].rows, info_[x].cols, false, sum_out, norm_out, "reduction of a materialised matrix");
}

// The paper's naive evaluation: every operator on its own, one temporary
// each, explicit transposes, dense diagonals, explicit inverse (Sec. III).
void Planner::literal() {
  std::vector<char> need(nd_.size(), 0);
  for (int o = 0; o < e_.n_outputs; ++o) need[e_.outputs[o]] = 1;
  for (int x = (int)nd_.size() - 1; x >= 0; --x)
    if (need[x] && nd_[x].op != ARMA_OP_INPUT) {
      need[nd_[x].a] = 1;
      if (is_binary(nd_[x].op)) need[nd_[x].b] = 1;
    }
  for (int x = 0; x < (int)nd_.size() && err_ == ARMA_OK; ++x) {
    if (!need[x]) continue;
    const arma_node& d = nd_[x];
    if (d.op == ARMA_OP_INPUT) { materialize(x); continue; }
    if (info_[x].scalar) {
      MatOperand src = loc_[d.a];
      Ref out = ref_output(out_of_[x]);
      if (d.op == ARMA_OP_TRACE) emit_reduce(src, info_[d.a].rows, info_[d.a].cols, true, out, Ref(), "literal trace");
      else if (d.op == ARMA_OP_ACCU) emit_reduce(src, info_[d.a].rows, info_[d.a].cols, false, out, Ref(), "literal accu");
      else emit_reduce(src, info_[d.a].rows, info_[d.a].cols, false, Ref(), out, "literal norm");
      continue;
    }
    MatOperand dest = dest_for(x);
    if (is_ew_op(d.op)) {
      EwStep s;
      s.m = info_[x].rows; s.n = info_[x].cols;
      s.mode = EW_FLAT;
      s.compute_f64 = info_[x].dtype == ARMA_F64 ? 1 : 0;
      const MatOperand& A = loc_[d.a];
      s.in[0].ref = A.ref; s.in[0].rs = 1; s.in[0].cs = A.ld; s.in[0].dtype = A.dtype;
      s.nin = 1;
      s.ops[s.nops++] = {EW_LD, 0, 0};
      if (is_binary(d.op)) {
        const MatOperand& B = loc_[d.b];
        s.in[1].ref = B.ref; s.in[1].rs = 1; s.in[1].cs = B.ld; s.in[1].dtype = B.dtype;
        s.nin = 2;
        static const int in_op[] = {0, EW_ADD, EW_SUB, EW_MUL, EW_DIV};
        s.ops[s.nops++] = {in_op[d.op], 1, 0};
      } else {
        int o = d.op == ARMA_OP_SCALE ? EW_SCAL : d.op == ARMA_OP_DIV_SCALAR ? EW_DIVS
                : d.op == ARMA_OP_ADD_SCALAR ? EW_ADDS : EW_NEG;
        s.ops[s.nops++] = {o, 0, d.scalar};
      }
      s.out = dest.ref; s.out_ld = dest.ld; s.out_dtype = dest.dtype;
      if (!ew_is_flat(s)) s.mode = EW_GRID;
      Step st;
      st.kind = ST_EW;
      st.ew = s;
      st.flops = (double)s.m * s.n;
      st.bytes = ew_bytes(s);
      st.note = std::string("literal ") + op_name(d.op) + " into a temporary";
      push_step(std::move(st));
    } else if (d.op == ARMA_OP_TRANS) {
      Step st;
      st.kind = ST_TRANSPOSE;
      st.cm = info_[d.a].rows; st.cn = info_[d.a].cols;
      st.csrc = loc_[d.a]; st.cdst = dest;
      st.bytes = 2.0 * (double)(st.cm * st.cn) * dtype_size(dest.dtype);
      st.note = "literal explicit transpose";
      push_step(std::move(st));
    } else if (d.op == ARMA_OP_MATMUL) {
      MatOperand A = loc_[d.a], B = loc_[d.b];
      emit_gemm(info_[d.a].rows, info_[d.b].cols, info_[d.a].cols, A, B, dest, 1.0, nullptr, 0.0,
                nullptr, nullptr, "literal product");
    } else if (d.op == ARMA_OP_DIAGMAT) {
      const NInfo& v = info_[d.a];
      if (v.rows == 1 || v.cols == 1) {
        Step st;
        st.kind = ST_DIAGBUILD;
        st.cm = info_[x].rows; st.cn = info_[x].cols;
        st.csrc = loc_[d.a];
        st.cinc = v.rows == 1 ? loc_[d.a].ld : 1;
        st.cdst = dest;
        st.bytes = (double)(st.cm * st.cn) * dtype_size(dest.dtype);
        st.note = "literal dense diagmat";
        push_step(std::move(st));
      } else {
        EwStep s;
        s.m = v.rows; s.n = v.cols;
        s.mode = EW_GRID;
        s.compute_f64 = v.dtype == ARMA_F64 ? 1 : 0;
        s.in[0].ref = loc_[d.a].ref; s.in[0].rs = 1; s.in[0].cs = loc_[d.a].ld;
        s.in[0].dtype = loc_[d.a].dtype; s.in[0].flags = EWF_DIAGMASK;
        s.nin = 1;
        s.ops[s.nops++] = {EW_LD, 0, 0};
        s.out = dest.ref; s.out_ld = dest.ld; s.out_dtype = dest.dtype;
        Step st;
        st.kind = ST_EW;
        st.ew = s;
        st.bytes = ew_bytes(s);
        st.note = "literal diagmat of a matrix";
        push_step(std::move(st));
      }
    } else if (d.op == ARMA_OP_INV) {
      emit_solve(loc_[d.a], info_[x].rows, nullptr, info_[x].rows, dest, info_[x].dtype, true,
                 "literal explicit inverse");
    } else if (d.op == ARMA_OP_SOLVE) {
      emit_solve(loc_[d.a], info_[x].rows, &loc_[d.b], info_[x].cols, dest, info_[x].dtype, false,
                 "literal solve: dense LU, the matrix's structure not examined");
    } else if (d.op == ARMA_OP_SUBMAT) {
      EwStep s;
      s.m = info_[x].rows; s.n = info_[x].cols;
      s.mode = EW_GRID;
      s.compute_f64 = info_[x].dtype == ARMA_F64 ? 1 : 0;
      s.in[0].ref = loc_[d.a].ref; s.in[0].rs = 1; s.in[0].cs = loc_[d.a].ld;
      s.in[0].off = (int64_t)d.slot + d.ld * loc_[d.a].ld;
      s.in[0].dtype = loc_[d.a].dtype;
      s.nin = 1;
      s.ops[s.nops++] = {EW_LD, 0, 0};
      s.out = dest.ref; s.out_ld = dest.ld; s.out_dtype = dest.dtype;
      Step st;
      st.kind = ST_EW;
      st.ew = s;
      st.bytes = ew_bytes(s);
      st.note = "literal submatrix copy";
      push_step(std::move(st));
    }
    loc_[x] = dest;
  }
}

arma_status Planner::run() {
  if (validate() != ARMA_OK) return err_;
  literal_ = (e_.flags & ARMA_PLAN_LITERAL) != 0;
  fuse_ = (e_.flags & ARMA_PLAN_NO_FUSE) == 0;
  chain_method_ = (e_.flags & ARMA_PLAN_CHAIN_GREEDY) ? 1 : (e_.flags & ARMA_PLAN_CHAIN_LEFT) ? 2 : 0;
  loc_.assign(nd_.size(), MatOperand());
  scalar_done_.assign(nd_.size(), 0);
  p_.flags = e_.flags;
  p_.tier = e_.tier;
  if (literal_) {
    literal();
  } else {
    // matrix outputs first (their passes may also produce sibling reductions)
    for (int o = 0; o < e_.n_outputs && err_ == ARMA_OK; ++o) {
      int x = e_.outputs[o];
      if (!info_[x].scalar) materialize(x);
    }
    for (int o = 0; o < e_.n_outputs && err_ == ARMA_OK; ++o) {
      int x = e_.outputs[o];
      if (info_[x].scalar) plan_scalar(x);
    }
  }
  if (err_ != ARMA_OK) return err_;
  // decision log (JSON)
  std::ostringstream os;
  os.precision(17);
  os << "{\"mode\": \"" << (literal_ ? "literal" : fuse_ ? "optimised" : "optimised_unfused")
     << "\", \"tier\": \"" << tier_name(e_.tier) << "\", \"chain\": \""
     << (chain_method_ == 0 ? "dp" : chain_method_ == 1 ? "paper_greedy" : "left_to_right")
     << "\", \"workspace\": " << p_.ws_bytes << ", \"steps\": [";
  static const char* kn[] = {"ew", "gemm", "diagdot", "transpose", "diagbuild", "solve"};
  for (size_t i = 0; i < p_.steps.size(); ++i) {
    const Step& s = p_.steps[i];
    p_.flops += s.flops;
    p_.bytes += s.bytes;
    std::string note = s.note;
    for (auto& ch : note) if (ch == '"') ch = '\'';
    const char* kname = (s.kind == ST_GEMM && s.gemm.sym == 1 && s.gemm.m > 1) ? "syrk" : kn[s.kind];
    os << (i ? ", " : "") << "{\"kernel\": \"" << kname << "\", \"flops\": " << s.flops
       << ", \"bytes\": " << s.bytes << ", \"note\": \"" << note << "\"";
    if (s.kind == ST_GEMM) {   // the K splits the product kernels will use
      int sp = 1;
      double tiles = 0;
      gemm_step_shape(s.gemm, &sp, &tiles);
      os << ", \"splits\": " << sp;
    }
    os << "}";
  }
  os << "], \"flops\": " << p_.flops << ", \"bytes\": " << p_.bytes << "}";
  p_.log = os.str();
  return ARMA_OK;
}

}  // namespace

arma_status plan_single(const arma_expr* e, arma_plan* p) {
  Planner pl(*e, *p);
  return pl.run();
}

arma_status plan_ranked(const arma_expr* e, arma_plan* p);

arma_status plan_expression(const arma_expr* e, arma_plan* p, std::string* msg) {
  (void)msg;
  if ((e->flags & (ARMA_PLAN_COST_MLP | ARMA_PLAN_COST_HEURISTIC)) && !(e->flags & ARMA_PLAN_LITERAL))
    return plan_ranked(e, p);
  return plan_single(e, p);
}

// Plan `count` instances of one expression family for the grouped kernel.
arma_status plan_batched(const arma_expr* exprs, int32_t count, arma_plan* p) {
  if (!exprs || count < 1) return ARMA_ERR_INVALID;
  BatchedInfo& b = p->bi;
  b.count = count;
  for (int32_t i = 0; i < count; ++i) {
    arma_plan one;
    Planner pl(exprs[i], one);
    arma_status st = pl.run();
    if (st != ARMA_OK) return st;
    const size_t ns = one.steps.size();
    if (ns < 1 || ns > 2 || one.steps[0].kind != ST_GEMM) return ARMA_ERR_UNSUPPORTED;
    const GemmStep& g = one.steps[0].gemm;
    if (g.A.ref.kind != REF_INPUT || g.B.ref.kind != REF_INPUT || g.D.ref.kind != REF_OUTPUT)
      return ARMA_ERR_UNSUPPORTED;
    if (g.C.ref.valid() && g.C.ref.kind != REF_INPUT) return ARMA_ERR_UNSUPPORTED;
    if (g.rowscale.ref.valid() || g.colscale.ref.valid()) return ARMA_ERR_UNSUPPORTED;
    if (g.A.dtype != g.B.dtype || g.A.dtype == ARMA_F64 || g.D.dtype != ARMA_F32) return ARMA_ERR_UNSUPPORTED;
    int32_t out_t = -1;
    if (ns == 2) {
      const Step& st2 = one.steps[1];
      if (st2.kind != ST_DOT) return ARMA_ERR_UNSUPPORTED;
      const DotStep& d = st2.dot;
      if (d.A.ref.kind != REF_INPUT || d.B.ref.kind != REF_INPUT || d.A.ref.boff || d.B.ref.boff ||
          d.A.ref.idx != g.A.ref.idx ||
          d.B.ref.idx != g.B.ref.idx || d.A.trans != g.A.trans || d.B.trans != g.B.trans || d.alpha != 1.0 ||
          d.out.kind != REF_OUTPUT)
        return ARMA_ERR_UNSUPPORTED;
      out_t = (int32_t)d.out.idx;
    }
    const int32_t sc = g.C.ref.valid() ? (int32_t)g.C.ref.idx : -1;
    if (i == 0) {
      b.slot_a = (int32_t)g.A.ref.idx; b.slot_b = (int32_t)g.B.ref.idx; b.slot_c = sc;
      b.out_d = (int32_t)g.D.ref.idx; b.out_t = out_t;
      b.n_slots = one.n_slots; b.n_outs = (int32_t)one.outs.size();
      b.ta = g.A.trans; b.tb = g.B.trans; b.abdt = g.A.dtype;
      b.cdt = g.C.ref.valid() ? g.C.dtype : ARMA_F32; b.ddt = g.D.dtype;
      b.alpha = g.alpha; b.beta = g.beta;
      p->outs = one.outs;
      p->n_slots = one.n_slots;
    } else if (b.slot_a != g.A.ref.idx || b.slot_b != g.B.ref.idx || b.slot_c != sc || b.out_d != g.D.ref.idx ||
               b.out_t != out_t || b.ta != g.A.trans || b.tb != g.B.trans || b.abdt != g.A.dtype ||
               b.alpha != g.alpha || b.beta != g.beta || b.n_slots != one.n_slots ||
               b.n_outs != (int32_t)one.outs.size()) {
      return ARMA_ERR_UNSUPPORTED;   // instances must share one structure
    }
    b.m.push_back(g.m); b.n.push_back(g.n); b.k.push_back(g.k);
    b.lda.push_back(g.A.ld); b.ldb.push_back(g.B.ld); b.ldc.push_back(g.C.ref.valid() ? g.C.ld : 0);
    // tile shape per problem: 128 x 128 on the tensor cores when both
    // operands are K-contiguous (op(A) = A^T, op(B) = B): BF16 operands as
    // they are, FP32 operands as three exact BF16 slices (six products).
    // SIMT tiles otherwise: 32 x 32 runs at about half the efficiency of
    // 64 x 64 per output and wins only when 64-tiles would pad more than 2x
    // (ARMA_PLAN_TILE64 / ARMA_PLAN_TILE32 force one shape; the Python
    // autotuner times these candidates).  ARMA_PLAN_NO_TENSOR keeps every
    // batch on the SIMT tiles.
    if (i == 0)
      b.tc = (g.A.trans == 1 && g.B.trans == 0 && (g.A.dtype == ARMA_BF16 || g.A.dtype == ARMA_F32) &&
              !(exprs[0].flags & ARMA_PLAN_NO_TENSOR))
                 ? 1 : 0;
    const int64_t t32 = ((g.m + 31) / 32) * ((g.n + 31) / 32);
    const int64_t t64 = ((g.m + 63) / 64) * ((g.n + 63) / 64);
    const uint32_t fl = exprs[0].flags;
    const int32_t T = b.tc ? 128 : (fl & ARMA_PLAN_TILE64) ? 64 : (fl & ARMA_PLAN_TILE32) ? 32 : (t32 < 2 * t64) ? 32 : 64;
    b.tile.push_back(T);
    b.first_tile.push_back(b.tiles);
    if (b.tc) {   // packed rows: K blocks of 64, each holding the problem's op(A) / op(B)^T rows
      const int64_t nkb = (g.k + 63) / 64;
      b.pa.push_back(b.rows_a);
      b.pb.push_back(b.rows_b);
      b.rows_a += g.m * nkb;
      b.rows_b += g.n * nkb;
      // the pack kernel's work: runs of whole rows of one operand (all their
      // K blocks, about kPackRun packed rows a run), in source order
      for (int op = 0; op < 2; ++op) {
        const int64_t R = op ? g.n : g.m;
        if (R * nkb > INT32_MAX) return ARMA_ERR_UNSUPPORTED;
        const int64_t run = std::max<int64_t>(1, kPackRun / std::max<int64_t>(nkb, 1));
        for (int64_t r = 0; r < R && nkb > 0; r += run) {
          b.pack_items.push_back(2 * i + op);
          b.pack_items.push_back((int32_t)r);
          b.pack_items.push_back((int32_t)std::min<int64_t>(run, R - r));
        }
      }
    }
    const int64_t ntm = (g.m + T - 1) / T, ntn = (g.n + T - 1) / T;
    if (ntm > 65535 || ntn > 65535) return ARMA_ERR_UNSUPPORTED;
    for (int64_t tm = 0; tm < ntm; ++tm)
      for (int64_t tn = 0; tn < ntn; ++tn) {
        b.tile_prob.push_back(i);
        b.tile_code.push_back((uint32_t)((tm << 16) | tn));
      }
    b.tiles += ntm * ntn;
    p->flops += 2.0 * (double)g.m * (double)g.n * (double)g.k;
  }
  // CTAs take tiles from a shared counter, longest first (the longest-
  // processing-time rule): a tile's work is its area times the problem's K
  {
    std::vector<double> work((size_t)b.tiles);
    for (int64_t t = 0; t < b.tiles; ++t) {
      const int32_t i = b.tile_prob[(size_t)t];
      const double T = (double)b.tile[(size_t)i];
      work[(size_t)t] = T * T * (double)std::max<int64_t>(b.k[(size_t)i], 1);
    }
    b.tile_order.resize((size_t)b.tiles);
    for (int64_t t = 0; t < b.tiles; ++t) b.tile_order[(size_t)t] = (int32_t)t;
    std::stable_sort(b.tile_order.begin(), b.tile_order.end(),
                     [&](int32_t x, int32_t y) { return work[(size_t)x] > work[(size_t)y]; });
  }
  if (b.tiles > INT32_MAX) return ARMA_ERR_UNSUPPORTED;
  p->batched = true;
  p->ws_bytes = kHeaderBytes + (size_t)((b.tiles * 8 * 8 + 255) / 256 * 256);   // 8 trace partials per tile
  if (b.tc) {
    // the packed operands (TMA reads them with 32-bit row coordinates)
    b.slices = b.abdt == ARMA_BF16 ? 1 : 3;
    if ((int64_t)b.slices * std::max(b.rows_a, b.rows_b) + 128 > INT32_MAX) return ARMA_ERR_UNSUPPORTED;
    b.pack_off = (p->ws_bytes + 1023) / 1024 * 1024;
    b.pack_bytes = (size_t)b.slices * (size_t)(b.rows_a + b.rows_b) * 128;
    p->ws_bytes = b.pack_off + b.pack_bytes;
  }
  std::ostringstream os;
  os.precision(17);
  os << "{\"mode\": \"batched\", \"count\": " << count << ", \"tiles\": " << b.tiles
     << ", \"trace\": " << (b.out_t >= 0 ? "true" : "false") << ", \"flops\": " << p->flops
     << ", \"workspace\": " << p->ws_bytes << ", \"tensor_cores\": " << (b.tc ? "true" : "false")
     << ", \"tile\": " << (b.tc ? 128 : (exprs[0].flags & ARMA_PLAN_TILE64) ? 64 : (exprs[0].flags & ARMA_PLAN_TILE32) ? 32 : 0)
     << ", \"steps\": [{\"kernel\": \"" << (b.tc ? "grouped_tc" : "grouped")
     << "\"}]}";
  p->log = os.str();
  return ARMA_OK;
}

// ---------------------------------------------------------------------------
// Plan features and the FLOP/byte heuristic (cost model inputs)
// ---------------------------------------------------------------------------
static double l2(double x) { return std::log2(1.0 + (x > 0 ? x : 0)); }

// Roofline estimate in the paper's spirit (fewer operations and fewer
// passes over memory are faster): every step costs a launch plus the larger
// of its compute time and its memory time on GB300.  `ew` and `prod`
// receive the parts spent in elementwise passes and in products.
static double heuristic_parts(const arma_plan* p, double* ew, double* prod) {
  const double hbm = 6.5e12, launch = 4e-6, dp = 0.3e12, simt = 40e12, bf16 = 1.2e15;
  double t = 0, te = 0, tp = 0;
  for (const Step& st : p->steps) {
    double c = 0;
    switch (st.kind) {
      case ST_EW:
        c = st.ew.compute_f64 ? st.flops / dp : 0;
        break;
      case ST_GEMM:
        if (st.gemm.m == 1 || st.gemm.n == 1) c = 0;
        else if (st.gemm.tier == ARMA_TIER_SPLIT_BF16) c = 6 * st.flops / bf16 + 2e-6;
        else if (st.gemm.tier == ARMA_TIER_BF16) c = st.flops / bf16 + 2e-6;
        else if (st.gemm.tier == ARMA_TIER_F64) c = st.flops / dp;
        else if (st.gemm.tier == ARMA_TIER_F64_SLICED) c = 36 * st.flops / bf16 + 8e-6 + st.bytes * 3 / hbm;
        else c = st.flops / simt;
        break;
      case ST_SOLVE:
        c = st.flops / (st.solve.tier == ARMA_TIER_F64 ? dp : 0.3e15) + (double)st.solve.n * 3e-6;
        break;
      default:
        break;
    }
    const double ts = launch + std::max(c, st.bytes / hbm);
    t += ts;
    if (st.kind == ST_EW) te += ts;
    if (st.kind == ST_GEMM) tp += ts;
  }
  if (ew) *ew = te;
  if (prod) *prod = tp;
  return t;
}

// kernel launches a step makes (approximately: the products' split-K
// combine and the solve's refinement depend on run-time data)
static double step_launches(const Step& st) {
  switch (st.kind) {
    case ST_GEMM: {
      const GemmStep& g = st.gemm;
      if (g.m == 1 || g.n == 1) return g.nosplit ? 1 : 2;
      const bool tc = g.tier == ARMA_TIER_SPLIT_BF16 || g.tier == ARMA_TIER_BF16;
      return (tc ? (g.sym ? 2 : 3) : 1) + (g.nosplit ? 0 : 1) + (g.sym ? 1 : 0);
    }
    case ST_DOT: return 2;
    case ST_SOLVE: return 8 + 4.0 * (double)((st.solve.n + 63) / 64);
    default: return 1;
  }
}

arma_status plan_heuristic(const arma_plan* p, double* seconds) {
  if (!p || !seconds) return ARMA_ERR_INVALID;
  *seconds = heuristic_parts(p, nullptr, nullptr);
  return ARMA_OK;
}

arma_status plan_features(const arma_plan* p, float* out, int32_t n) {
  if (!p || !out || n < ARMA_PLAN_FEATURES) return ARMA_ERR_INVALID;
  double f[ARMA_PLAN_FEATURES] = {0};
  double maxf = 0, maxb = 0, tc_flops = 0, split_flops = 0, dp_flops = 0, launches = 0, nosplit = 0;
  double big_flops = -1, big_min_dim = 0, max_out = 0;
  for (const Step& st : p->steps) {
    f[2] += 1;
    launches += step_launches(st);
    switch (st.kind) {
      case ST_EW:
        f[3] += 1;
        max_out = std::max(max_out, (double)st.ew.m * (double)st.ew.n);
        break;
      case ST_GEMM: {
        const GemmStep& g = st.gemm;
        if (g.m == 1 || g.n == 1) f[5] += 1;
        else f[4] += 1;
        if (g.tier == ARMA_TIER_SPLIT_BF16 || g.tier == ARMA_TIER_BF16) tc_flops += st.flops;
        if (g.tier == ARMA_TIER_SPLIT_BF16) split_flops += st.flops;
        if (g.tier == ARMA_TIER_F64) dp_flops += st.flops;
        if (g.nosplit) nosplit += 1;
        if (st.flops > big_flops) {
          big_flops = st.flops;
          big_min_dim = (double)std::min(g.m, std::min(g.n, g.k));
        }
        max_out = std::max(max_out, (double)g.m * (double)g.n);
        break;
      }
      case ST_DOT: f[6] += 1; break;
      case ST_TRANSPOSE: case ST_DIAGBUILD: f[7] += 1; break;
      case ST_SOLVE:
        f[8] += 1;
        if (st.solve.tier == ARMA_TIER_F64) dp_flops += st.flops;
        break;
    }
    maxf = std::max(maxf, st.flops);
    maxb = std::max(maxb, st.bytes);
  }
  // what the estimate leaves out: split-K combine launches, strided reads
  // in fused passes, FP64 (DFMA) product time, tile padding and parallelism
  // of the tensor-core products, operand preparation passes
  double combines = 0, strided = 0, dp_time = 0, tc_useful = 0, tc_padded = 0, big_tiles = 0, big_k = 0,
         preps = 0, big_f = -1;
  for (const Step& st : p->steps) {
    if (st.kind == ST_EW) {
      for (int k = 0; k < st.ew.nin; ++k)
        if (st.ew.in[k].rs != 1 || st.ew.in[k].flags) strided += (double)st.ew.m * (double)st.ew.n;
    } else if (st.kind == ST_GEMM) {
      const GemmStep& g = st.gemm;
      int splits = 1;
      double tiles = 0;
      gemm_step_shape(g, &splits, &tiles);
      if (splits > 1) combines += 1;
      const bool tc = g.tier == ARMA_TIER_SPLIT_BF16 || g.tier == ARMA_TIER_BF16;
      if (g.tier == ARMA_TIER_F64 && g.m > 1 && g.n > 1) dp_time += st.flops / 0.3e12;
      if (tc && g.m > 1 && g.n > 1) {
        tc_useful += (double)g.m * (double)g.n;
        tc_padded += (double)((g.m + 127) / 128 * 128) * (double)((g.n + 255) / 256 * 256);
        preps += (g.A.dtype == ARMA_BF16 && g.A.trans ? 0 : 1) + (g.B.dtype == ARMA_BF16 && !g.B.trans ? 0 : 1);
      }
      if (st.flops > big_f) {
        big_f = st.flops;
        big_tiles = tiles * splits;
        big_k = (double)g.k;
      }
    }
  }
  double te = 0, tp = 0;
  const double h = heuristic_parts(p, &te, &tp);
  f[0] = l2(p->flops);
  f[1] = l2(p->bytes);
  f[9] = l2(maxf);
  f[10] = l2(maxb);
  f[11] = l2((double)p->ws_bytes);
  f[12] = p->flops > 0 ? tc_flops / p->flops : 0;
  f[13] = (p->flags & ARMA_PLAN_LITERAL) ? 1 : 0;
  f[14] = p->flops > 0 ? split_flops / p->flops : 0;
  f[15] = l2(p->bytes > 0 ? p->flops / p->bytes : 0);
  f[16] = std::log(h > 0 ? h : 1e-9);
  f[17] = launches;
  f[18] = p->flops > 0 ? dp_flops / p->flops : 0;
  f[19] = h > 0 ? te / h : 0;
  f[20] = h > 0 ? tp / h : 0;
  f[21] = l2(big_min_dim);
  f[22] = nosplit;
  f[23] = l2(max_out);
  f[24] = combines;
  f[25] = l2(strided);
  f[26] = h > 0 ? dp_time / h : 0;
  f[27] = tc_padded > 0 ? tc_useful / tc_padded : 1;
  f[28] = l2(big_tiles / 152.0);
  f[29] = preps;
  f[30] = l2(big_k);
  f[31] = h > 0 ? launches * 4e-6 / h : 0;
  for (int i = 0; i < ARMA_PLAN_FEATURES; ++i) out[i] = (float)f[i];
  for (int i = ARMA_PLAN_FEATURES; i < n; ++i) out[i] = 0.f;
  return ARMA_OK;
}

// ---------------------------------------------------------------------------
// The learned cost model on the host, and the choice among candidate plans
// ---------------------------------------------------------------------------
namespace {

struct CostModel {
  int F = 0, H = 0;
  std::vector<float> params, mean, scale;
  double guard = 0;    // the estimate overrules picks it rates > guard x its own pick
  double margin = 0;   // the network must predict its pick this much faster than the estimate's
};

std::mutex g_model_mu;
std::shared_ptr<const CostModel> g_model;

std::shared_ptr<const CostModel> loaded_model() {
  std::lock_guard<std::mutex> lock(g_model_mu);
  return g_model;
}

// y = W3 relu(W2 relu(W1 z + b1) + b2) + b3 with the packing and the
// operation order of the GPU forward kernel (fused multiply-adds in FP32,
// inputs in index order), so the two agree bit for bit
float model_forward(const CostModel& M, const float* feat) {
  const int F = M.F, H = M.H;
  const float* P = M.params.data();
  const int64_t W1 = 0, b1 = W1 + (int64_t)H * F, W2 = b1 + H, b2 = W2 + (int64_t)H * H, W3 = b2 + H,
                b3 = W3 + H;
  std::vector<float> z(F), h1(H);
  for (int f = 0; f < F; ++f) z[f] = (feat[f] - M.mean[f]) / M.scale[f];
  for (int i = 0; i < H; ++i) {
    float a = P[b1 + i];
    for (int f = 0; f < F; ++f) a = std::fmaf(P[W1 + (int64_t)i * F + f], z[f], a);
    h1[i] = a > 0.f ? a : 0.f;
  }
  float y = P[b3];
  for (int i = 0; i < H; ++i) {
    float a = P[b2 + i];
    for (int j = 0; j < H; ++j) a = std::fmaf(P[W2 + (int64_t)i * H + j], h1[j], a);
    y = std::fmaf(P[W3 + i], a > 0.f ? a : 0.f, y);
  }
  return y;
}

double model_seconds(const CostModel& M, const arma_plan* p) {
  float feat[ARMA_PLAN_FEATURES];
  plan_features(p, feat, ARMA_PLAN_FEATURES);
  const double h = heuristic_parts(p, nullptr, nullptr);
  return h * std::exp((double)model_forward(M, feat));
}

constexpr uint32_t kChoiceFlags = ARMA_PLAN_COST_MLP | ARMA_PLAN_COST_HEURISTIC | ARMA_PLAN_TIER_CHOICE;
constexpr uint32_t kVariantFlags = ARMA_PLAN_CHAIN_LEFT | ARMA_PLAN_CHAIN_GREEDY | ARMA_PLAN_NO_FUSE |
                                   ARMA_PLAN_NO_SPLITK;

struct Variant {
  uint32_t flags;
  int32_t tier;
};

bool all_inputs(const arma_expr& e, int32_t dt) {
  bool any = false;
  for (int i = 0; i < e.n_nodes; ++i)
    if (e.nodes[i].op == ARMA_OP_INPUT) {
      any = true;
      if (e.nodes[i].dtype != dt) return false;
    }
  return any;
}

// Precision tiers at least as accurate as the requested one
// (BF16 < SPLIT_BF16 < LU32_IR64 < F64; NATIVE resolves by element type).
std::vector<int32_t> admissible_tiers(const arma_expr& e) {
  const int32_t t = e.tier;
  std::vector<int32_t> v{t};
  if (!(e.flags & ARMA_PLAN_TIER_CHOICE)) return v;
  switch (t) {
    case ARMA_TIER_BF16:
      v.push_back(ARMA_TIER_SPLIT_BF16); v.push_back(ARMA_TIER_F64); v.push_back(ARMA_TIER_F64_SLICED);
      break;
    case ARMA_TIER_SPLIT_BF16: case ARMA_TIER_LU32_IR64:
      v.push_back(ARMA_TIER_F64); v.push_back(ARMA_TIER_F64_SLICED);
      break;
    case ARMA_TIER_F64: v.push_back(ARMA_TIER_F64_SLICED); break;
    case ARMA_TIER_NATIVE:
      if (all_inputs(e, ARMA_BF16)) v.push_back(ARMA_TIER_SPLIT_BF16);
      v.push_back(ARMA_TIER_F64);
      v.push_back(ARMA_TIER_F64_SLICED);
      break;
    default: break;
  }
  return v;
}

std::vector<Variant> variants(const arma_expr& e) {
  const uint32_t base = e.flags & ~(kChoiceFlags | kVariantFlags);
  if (e.flags & ARMA_PLAN_LITERAL) return {Variant{base, e.tier}};
  std::vector<Variant> v;
  const uint32_t chains[3] = {0u, ARMA_PLAN_CHAIN_GREEDY, ARMA_PLAN_CHAIN_LEFT};
  for (int32_t t : admissible_tiers(e))
    for (uint32_t c : chains)
      for (uint32_t fuse : {0u, (uint32_t)ARMA_PLAN_NO_FUSE})
        for (uint32_t split : {0u, (uint32_t)ARMA_PLAN_NO_SPLITK}) v.push_back(Variant{base | c | fuse | split, t});
  return v;
}

// the step list of a plan's decision log: plans with equal step lists
// launch the same kernels with the same arguments
std::string step_signature(const arma_plan& p) {
  const size_t a = p.log.find("\"steps\": [");
  const size_t b = p.log.rfind("], \"flops\"");
  std::string sig = (a != std::string::npos && b != std::string::npos && b > a) ? p.log.substr(a, b - a) : p.log;
  for (const Step& st : p.steps) {
    if (st.kind == ST_SOLVE) sig += " solve:" + std::to_string(st.solve.tier);
    if (st.kind == ST_GEMM) sig += " gemm:" + std::to_string(st.gemm.nosplit);
  }
  return sig;
}

const char* variant_name(uint32_t f) {
  const bool greedy = f & ARMA_PLAN_CHAIN_GREEDY, left = f & ARMA_PLAN_CHAIN_LEFT;
  const bool nofuse = f & ARMA_PLAN_NO_FUSE, nosplit = f & ARMA_PLAN_NO_SPLITK;
  static const char* names[3][4] = {{"dp", "dp+nosplit", "dp+unfused", "dp+unfused+nosplit"},
                                    {"greedy", "greedy+nosplit", "greedy+unfused", "greedy+unfused+nosplit"},
                                    {"written", "written+nosplit", "written+unfused", "written+unfused+nosplit"}};
  return names[left ? 2 : greedy ? 1 : 0][(nofuse ? 2 : 0) + (nosplit ? 1 : 0)];
}

}  // namespace

arma_status plan_single(const arma_expr* e, arma_plan* p);

// Every distinct candidate plan of an expression, in enumeration order.
static arma_status plan_candidates(const arma_expr* e, std::vector<std::unique_ptr<arma_plan>>& out,
                                   std::vector<Variant>* used) {
  out.clear();
  std::vector<std::string> sigs;
  arma_status first_err = ARMA_OK;
  for (const Variant& v : variants(*e)) {
    arma_expr x = *e;
    x.flags = v.flags;
    x.tier = v.tier;
    std::unique_ptr<arma_plan> p(new arma_plan());
    arma_status s = plan_single(&x, p.get());
    if (s != ARMA_OK) {
      if (first_err == ARMA_OK) first_err = s;
      continue;
    }
    const std::string sig = step_signature(*p);
    if (std::find(sigs.begin(), sigs.end(), sig) != sigs.end()) continue;
    sigs.push_back(sig);
    out.push_back(std::move(p));
    if (used) used->push_back(v);
  }
  return out.empty() ? (first_err != ARMA_OK ? first_err : ARMA_ERR_INVALID) : ARMA_OK;
}

// Plan the candidates and keep the one the scorer ranks fastest; the
// decision log records every candidate with its scores.
arma_status plan_ranked(const arma_expr* e, arma_plan* p) {
  std::vector<std::unique_ptr<arma_plan>> cands;
  std::vector<Variant> used;
  arma_status s = plan_candidates(e, cands, &used);
  if (s != ARMA_OK) return s;
  std::shared_ptr<const CostModel> model = (e->flags & ARMA_PLAN_COST_MLP) ? loaded_model() : nullptr;
  const size_t n = cands.size();
  std::vector<double> h(n), m(n, 0.0);
  size_t hb = 0, mb = 0;
  for (size_t i = 0; i < n; ++i) {
    h[i] = heuristic_parts(cands[i].get(), nullptr, nullptr);
    if (h[i] < h[hb]) hb = i;
    if (model) {
      m[i] = model_seconds(*model, cands[i].get());
      if (m[i] < m[mb]) mb = i;
    }
  }
  // the network's pick replaces the estimate's only when the network
  // predicts it at least `margin` faster, and the estimate does not rate it
  // more than `guard` times slower than its own pick
  size_t pick = hb;
  bool guarded = false;
  if (model && mb != hb && m[mb] < (1.0 - model->margin) * m[hb]) {
    if (model->guard > 0 && h[mb] > model->guard * h[hb]) guarded = true;
    else pick = mb;
  }
  std::ostringstream os;
  os.precision(6);
  os << ", \"choice\": {\"scorer\": \"" << (model ? "mlp" : "heuristic") << "\", \"picked\": " << pick
     << ", \"heuristic_pick\": " << hb << ", \"guarded\": " << (guarded ? "true" : "false")
     << ", \"candidates\": [";
  for (size_t i = 0; i < n; ++i) {
    os << (i ? ", " : "") << "{\"variant\": \"" << variant_name(used[i].flags) << "\", \"tier\": \""
       << tier_name(used[i].tier) << "\", \"heuristic_s\": " << h[i];
    if (model) os << ", \"predicted_s\": " << m[i];
    os << "}";
  }
  os << "]}";
  arma_plan& best = *cands[pick];
  if (!best.log.empty() && best.log.back() == '}') best.log.insert(best.log.size() - 1, os.str());
  *p = std::move(best);
  return ARMA_OK;
}

arma_status plan_candidates_api(const arma_expr* e, arma_plan** plans, int32_t capacity, int32_t* count) {
  if (!e || !count || capacity < 0 || (capacity > 0 && !plans)) return ARMA_ERR_INVALID;
  std::vector<std::unique_ptr<arma_plan>> cands;
  arma_status s = plan_candidates(e, cands, nullptr);
  if (s != ARMA_OK) return s;
  *count = (int32_t)cands.size();
  for (int32_t i = 0; i < capacity; ++i) plans[i] = i < (int32_t)cands.size() ? cands[i].release() : nullptr;
  return ARMA_OK;
}

arma_status cost_model_load(const float* params, int32_t F, int32_t H, const float* mean, const float* scale,
                            double guard, double margin) {
  if (!params || !mean || !scale || F != ARMA_PLAN_FEATURES || H < 1 || H > 128 || guard < 0 ||
      !std::isfinite(guard) || !(margin >= 0 && margin < 1))
    return ARMA_ERR_INVALID;
  auto M = std::make_shared<CostModel>();
  M->F = F;
  M->H = H;
  const int64_t np = (int64_t)H * F + H + (int64_t)H * H + H + H + 1;
  M->params.assign(params, params + np);
  M->mean.assign(mean, mean + F);
  M->scale.assign(scale, scale + F);
  for (float x : M->params)
    if (!std::isfinite(x)) return ARMA_ERR_INVALID;
  for (int i = 0; i < F; ++i)
    if (!std::isfinite(M->mean[i]) || !std::isfinite(M->scale[i]) || M->scale[i] == 0.f) return ARMA_ERR_INVALID;
  M->guard = guard;
  M->margin = margin;
  std::lock_guard<std::mutex> lock(g_model_mu);
  g_model = std::move(M);
  return ARMA_OK;
}

void cost_model_clear() {
  std::lock_guard<std::mutex> lock(g_model_mu);
  g_model.reset();
}

arma_status cost_model_predict(const arma_plan* p, double* seconds) {
  if (!p || !seconds || p->batched) return ARMA_ERR_INVALID;
  std::shared_ptr<const CostModel> M = loaded_model();
  if (!M) return ARMA_ERR_UNSUPPORTED;
  *seconds = model_seconds(*M, p);
  return ARMA_OK;
}

arma_status chain_order_api(int32_t n, const int64_t* dims, int32_t method, int32_t* splits,
                            uint64_t* cost) {
  if (n < 1 || n > 4096 || !dims || method < 0 || method > 2) return ARMA_ERR_INVALID;
  for (int i = 0; i <= n; ++i)
    if (dims[i] < 0) return ARMA_ERR_SHAPE;
  if (n == 1) {
    if (cost) *cost = 0;
    return ARMA_OK;
  }
  std::vector<ChainTree> t;
  int root;
  chain_order(n, dims, method, t, root);
  std::vector<int> pre;
  tree_preorder(t, root, pre);
  if (splits)
    for (int i = 0; i < (int)pre.size(); ++i) splits[i] = pre[i];
  if (cost) *cost = sat64(tree_cost(t, root, dims));
  return ARMA_OK;
}

}  // namespace arma
