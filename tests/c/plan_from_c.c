/* The C ABI used from plain C99, host calls only (no GPU needed): plan the
 * fused benchmark expression out = A%B + 3*C - D/2 with accu(out) and
 * norm(out, "fro") (Sec. II's single-pass evaluation), read its decision
 * log, check a conformance error (Sec. II), and order the benchmark chain
 * A*B*C*v (Sec. II, chain paragraph).  Prints one line per check; exits 0
 * when all hold. */
#include <stdio.h>
#include <string.h>

#include "arma_gpu.h"

static arma_node input(int slot, int64_t rows, int64_t cols) {
  arma_node n;
  memset(&n, 0, sizeof n);
  n.op = ARMA_OP_INPUT; n.a = -1; n.b = -1; n.slot = slot; n.dtype = ARMA_F64;
  n.rows = rows; n.cols = cols; n.ld = rows;
  return n;
}

static arma_node op(int code, int a, int b, double s) {
  arma_node n;
  memset(&n, 0, sizeof n);
  n.op = code; n.a = a; n.b = b; n.scalar = s;
  return n;
}

int main(void) {
  int fails = 0;
  arma_node nodes[11];
  nodes[0] = input(0, 64, 48);
  nodes[1] = input(1, 64, 48);
  nodes[2] = input(2, 64, 48);
  nodes[3] = input(3, 64, 48);
  nodes[4] = op(ARMA_OP_SCHUR, 0, 1, 0.0);        /* A % B */
  nodes[5] = op(ARMA_OP_SCALE, 2, -1, 3.0);       /* 3 * C */
  nodes[6] = op(ARMA_OP_ADD, 4, 5, 0.0);
  nodes[7] = op(ARMA_OP_DIV_SCALAR, 3, -1, 2.0);  /* D / 2 */
  nodes[8] = op(ARMA_OP_SUB, 6, 7, 0.0);          /* out */
  nodes[9] = op(ARMA_OP_ACCU, 8, -1, 0.0);
  nodes[10] = op(ARMA_OP_NORM_FRO, 8, -1, 0.0);
  int32_t outs[3] = {8, 9, 10};
  arma_expr e;
  memset(&e, 0, sizeof e);
  e.n_nodes = 11; e.n_outputs = 3; e.nodes = nodes; e.outputs = outs; e.tier = ARMA_TIER_NATIVE;

  arma_plan* plan = NULL;
  arma_status s = arma_gpu_plan(&e, &plan);
  printf("plan %s\n", arma_gpu_status_string(s));
  if (s != ARMA_OK || !plan) return 1;

  size_t ws = 0;
  s = arma_gpu_plan_workspace(plan, &ws);
  printf("workspace %zu\n", ws);
  fails += s != ARMA_OK || ws == 0;

  int64_t r = 0, c = 0;
  int32_t dt = -1;
  s = arma_gpu_output_info(plan, 1, &r, &c, &dt);
  printf("accu output %lld x %lld dtype %d\n", (long long)r, (long long)c, (int)dt);
  fails += s != ARMA_OK || r != 1 || c != 1 || dt != ARMA_F64;
  fails += arma_gpu_output_info(plan, 3, &r, &c, &dt) != ARMA_ERR_INVALID;

  char log[8192];
  size_t need = 0;
  s = arma_gpu_plan_info(plan, log, sizeof log, &need);
  /* one fused pass: a single "ew" step that also forms both reductions */
  int steps = 0;
  for (const char* q = strstr(log, "\"kernel\""); q; q = strstr(q + 1, "\"kernel\"")) ++steps;
  printf("steps %d fused %d\n", steps, strstr(log, "+sumsq") != NULL);
  fails += s != ARMA_OK || need > sizeof log || steps != 1 || !strstr(log, "+sum") || !strstr(log, "+sumsq");
  arma_gpu_plan_free(plan);

  /* A % B with B 64 x 47: the paper's conformance check rejects it at plan time */
  nodes[1] = input(1, 64, 47);
  plan = (arma_plan*)&e;   /* must be reset to NULL on error */
  s = arma_gpu_plan(&e, &plan);
  printf("non-conforming %s\n", arma_gpu_status_string(s));
  fails += s != ARMA_ERR_SHAPE || plan != NULL;

  /* the benchmark chain: A 4096x8192, B 8192x512, C 512x4096, v 4096x1 */
  int64_t dims[5] = {4096, 8192, 512, 4096, 1};
  int32_t splits[3];
  uint64_t cost = 0;
  s = arma_gpu_chain_order(4, dims, 0, splits, &cost);
  printf("chain cost %llu\n", (unsigned long long)cost);
  fails += s != ARMA_OK || cost != 39845888ull;

  printf("%s\n", fails ? "FAIL" : "OK");
  return fails != 0;
}
