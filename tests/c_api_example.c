/* A C99 caller of libdfl: two triangles joined by one edge, static Louvain,
 * then one batch (the bridge deleted, an edge inserted inside the first
 * triangle's community) and a DF update, then a second batch (the bridge
 * back, an edge of the second triangle deleted) as one dfl_step call.  The
 * test suite compiles and links it on any machine; run on a GPU it prints
 * the memberships and modularities and exits 0 when every call succeeded
 * and the two triangles were separate communities after the first update. */
#include <stdio.h>
#include <stdlib.h>

#include "dfl.h"

#define CHECK(h, call)                                                                  \
  do {                                                                                  \
    int rc_ = (call);                                                                   \
    if (rc_ != DFL_OK) {                                                                \
      fprintf(stderr, "%s: %d (%s)\n", #call, rc_, (h) ? dfl_last_error(h) : "no handle"); \
      dfl_destroy(h);                                                                   \
      return 1;                                                                         \
    }                                                                                   \
  } while (0)

int main(void) {
  /* edges 0-1, 0-2, 1-2, 3-4, 3-5, 4-5, 2-3 as a symmetric CSR with sorted rows */
  static const uint64_t offsets[7] = {0, 2, 4, 7, 10, 12, 14};
  static const uint32_t indices[14] = {1, 2, 0, 2, 0, 1, 3, 2, 4, 5, 3, 5, 3, 4};
  static const uint32_t weights[14] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
  const dfl_edge dels[1] = {{2, 3, 0}};  /* w = 0: the whole edge */
  const dfl_edge ins[1] = {{0, 1, 2}};   /* adds weight 2 to edge 0-1 */
  const dfl_edge dels2[1] = {{4, 5, 0}};
  const dfl_edge ins2[1] = {{2, 3, 1}};
  dfl_handle* h = NULL;
  uint32_t C[6], C2[6];
  double q = 0.0;
  int64_t parts[4];
  dfl_options opt;
  dfl_stats_t st;
  int v;

  dfl_default_options(&opt);
  CHECK(h, dfl_create(&h, 6, offsets, indices, weights, 14, DFL_MEM_HOST, &opt, NULL));
  CHECK(h, dfl_static(h));
  CHECK(h, dfl_membership(h, C, DFL_MEM_HOST));
  printf("static:");
  for (v = 0; v < 6; ++v) printf(" %u", (unsigned)C[v]);
  printf("\n");
  CHECK(h, dfl_apply_batch(h, dels, 1, ins, 1, DFL_MEM_HOST));
  CHECK(h, dfl_update(h, DFL_DF));
  CHECK(h, dfl_membership(h, C, DFL_MEM_HOST));
  CHECK(h, dfl_modularity(h, &q, parts));
  CHECK(h, dfl_stats(h, &st));
  printf("after DF:");
  for (v = 0; v < 6; ++v) printf(" %u", (unsigned)C[v]);
  printf("  Q = %.6f  passes = %u  affected = %llu\n", q, (unsigned)st.passes,
         (unsigned long long)st.affected_initial);
  CHECK(h, dfl_step(h, dels2, 1, ins2, 1, DFL_MEM_HOST, DFL_DF));
  CHECK(h, dfl_membership(h, C2, DFL_MEM_HOST));
  CHECK(h, dfl_modularity(h, &q, parts));
  printf("after step:");
  for (v = 0; v < 6; ++v) printf(" %u", (unsigned)C2[v]);
  printf("  Q = %.12f\n", q);
  dfl_destroy(h);
  return (C[0] == C[1] && C[1] == C[2] && C[3] == C[4] && C[4] == C[5] && C[0] != C[3]) ? 0 : 2;
}
