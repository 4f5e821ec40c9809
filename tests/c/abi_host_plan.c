/* Plain-C user of the C ABI (no Python, no CUDA headers): plans a small circuit
 * on the host only and checks the plan's figures and the error paths.  Built and
 * run by tests/test_c_abi.py; needs no GPU (host_only plans touch no device). */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "tn_gb300.h"

static void set_1q(tn_gate* g, int q, double a) {   /* exp(-i a Y) */
  memset(g, 0, sizeof(*g));
  g->arity = 1;
  g->q0 = q;
  g->re[0] = cos(a); g->re[1] = -sin(a);
  g->re[2] = sin(a); g->re[3] = cos(a);
}

static void set_cz(tn_gate* g, int q0, int q1) {
  memset(g, 0, sizeof(*g));
  g->arity = 2;
  g->q0 = q0;
  g->q1 = q1;
  g->re[0] = 1; g->re[5] = 1; g->re[10] = 1; g->re[15] = -1;
}

int main(void) {
  enum { N = 4 };
  tn_gate gates[16];
  int ng = 0;
  for (int layer = 0; layer < 2; ++layer) {
    for (int q = 0; q < N; ++q) set_1q(&gates[ng++], q, 0.3 + 0.1 * q + layer);
    for (int q = layer; q + 1 < N; q += 2) set_cz(&gates[ng++], q, q + 1);
  }
  tn_circuit circ = {N, ng, gates};
  int open_q[2] = {2, 3};
  uint64_t tails[2] = {0u, 1u};
  tn_open_spec spec = {open_q, 2, tails, 2};
  tn_edge edges[1] = {{N, 0, TN_EDGE_SLICE, 0}};   /* the wire entering the first CZ on its q0 */
  tn_plan_opts opts;
  memset(&opts, 0, sizeof(opts));
  opts.host_only = 1;
  tn_plan_t* plan = NULL;
  int rc = tn_plan(&circ, &spec, edges, 1, NULL, 0, &opts, &plan);
  if (rc != TN_OK || !plan) {
    printf("tn_plan failed: %d %s\n", rc, tn_last_error());
    return 1;
  }
  tn_plan_stats st;
  if (tn_plan_get_stats(plan, &st) != TN_OK) return 2;
  if (st.n_qubits != N || st.n_open != 2 || st.n_tails != 2 || st.n_sliced != 1) return 3;
  const char* d = tn_plan_describe(plan, 0);
  if (!d || !strstr(d, "\"n_sliced\":1")) return 4;
  int64_t np = 0;
  if (tn_plan_order(plan, NULL, 0, &np) != TN_OK || np < 1) return 5;
  /* per-step tile variants: every step has at least one; choosing the last
     and then the first again is accepted, one past the last is not */
  for (int64_t i = 0; i + 1 < st.n_launches; ++i) {
    int nv = 0, chosen = -1;
    if (tn_plan_step_variants(plan, i, &nv, &chosen) != TN_OK || nv < 1 || chosen != 0) return 9;
    if (tn_plan_set_step_variant(plan, i, nv - 1) != TN_OK) return 10;
    if (tn_plan_step_variants(plan, i, &nv, &chosen) != TN_OK || chosen != nv - 1) return 11;
    if (tn_plan_set_step_variant(plan, i, 0) != TN_OK) return 12;
    if (tn_plan_set_step_variant(plan, i, nv) != TN_ERR_INVALID) return 13;
  }
  /* the tuner needs the device: a host-only plan is refused */
  if (tn_plan_tune_steps(plan, 1, NULL, NULL, NULL) != TN_ERR_INVALID) return 14;
  tn_plan_free(plan);
  /* errors come back as codes with a message, never as an abort */
  spec.n_tails = 0;
  plan = NULL;
  if (tn_plan(&circ, &spec, edges, 1, NULL, 0, &opts, &plan) != TN_ERR_INVALID || plan) return 6;
  if (strlen(tn_last_error()) == 0) return 7;
  spec.n_tails = 2;
  edges[0].gate = 999;
  if (tn_plan(&circ, &spec, edges, 1, NULL, 0, &opts, &plan) != TN_ERR_INVALID) return 8;
  printf("c abi ok: %s, %d leaves, %d launches per slice\n", tn_version(), st.n_leaves, st.n_launches);
  return 0;
}
