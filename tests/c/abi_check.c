/* The C ABI used from plain C99 (no C++, no CUDA headers, no torch): the
 * header must compile on its own and the library must link and answer its
 * host-only entries.  Prints one line per check; the pytest wrapper
 * compares them.  No device work is requested. */
#include <stdio.h>
#include <string.h>

#include "fastalign.h"

int main(void) {
  fa_params p;
  fa_params_default(&p);
  printf("params %d %d %.2f %.2f\n", p.k_rwr, p.k_prop, p.eps, p.alpha);

  int32_t plan[8];
  fa_status s = fa_sweep_plan(50000, 50048, FA_BF16, plan);
  printf("plan %d %d %d %d %d %d %d\n", (int)s, plan[0], plan[1], plan[2], plan[3], plan[4],
         plan[5]);

  /* a triangle with a duplicate, a reversed pair and a self-loop */
  const int32_t src[6] = {0, 1, 2, 1, 0, 2};
  const int32_t dst[6] = {1, 2, 0, 0, 1, 2};
  int64_t nnz = -1;
  s = fa_graph_csr_host(4, 6, src, dst, &nnz, NULL, NULL, NULL, NULL, 0);
  int32_t rp[5], col[6];
  float vr[6], vc[6];
  memset(rp, 0, sizeof rp);
  s = fa_graph_csr_host(4, 6, src, dst, &nnz, rp, col, vr, vc, 6);
  printf("csr %d %lld %d %d %d %d %d %d %.2f\n", (int)s, (long long)nnz, rp[0], rp[1], rp[2],
         rp[3], rp[4], col[0], vr[0]);

  fa_graph* g = NULL;
  s = fa_build_graph(3, 1, src, NULL, &g);
  printf("error %d %d\n", (int)s, g == NULL);
  printf("message %s\n", fa_last_error_string());
  return 0;
}
