/* A plain C99 user of the C ABI (tests/test_c_abi.py compiles and links it
 * against libifmm.so): takes the address of every entry point the header
 * declares (the generated abi_table.h lists them), then runs the host-side part
 * of the path that needs no GPU -- the octree of Sec. 2.1 and the Algorithm 3
 * coloring -- and the error protocol. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "ifmm.h"

typedef void (*any_fn)(void);
#define X(name) (any_fn) name,
static const any_fn table[] = {IFMM_ABI_TABLE};
#undef X

static int fails = 0;
#define CHECK(cond, what)               \
  do {                                  \
    if (!(cond)) {                      \
      printf("FAIL: %s\n", what);       \
      ++fails;                          \
    }                                   \
  } while (0)

int main(void) {
  const size_t nfn = sizeof(table) / sizeof(table[0]);
  for (size_t i = 0; i < nfn; ++i) CHECK(table[i] != NULL, "entry point resolved");

  /* points on the unit sphere (golden-angle spiral), row-major x y z */
  const int64_t n = 3000;
  double* xyz = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n, r = sqrt(1.0 - z * z);
    const double phi = 2.399963229728653 * (double)i;
    xyz[3 * i] = r * cos(phi);
    xyz[3 * i + 1] = r * sin(phi);
    xyz[3 * i + 2] = z;
  }
  ifmm_tree* t = NULL;
  CHECK(ifmm_build_tree(xyz, n, 4, &t) == IFMM_OK && t != NULL, "ifmm_build_tree");
  int32_t ncol[5] = {0, 0, 0, 0, 0};
  CHECK(ifmm_color(t, 3, ncol) == IFMM_OK, "ifmm_color");
  for (int l = 2; l <= 4; ++l) CHECK(ncol[l] > 0, "colors at every level from 2");

  /* the permutation: a bijection of 0..n-1 */
  int64_t cnt = 0;
  CHECK(ifmm_tree_query(t, 0, "perm", NULL, 0, &cnt) == IFMM_OK && cnt == n, "perm count");
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  char* seen = (char*)calloc((size_t)n, 1);
  CHECK(ifmm_tree_query(t, 0, "perm", perm, n, &cnt) == IFMM_OK, "perm");
  for (int64_t i = 0; i < n; ++i) {
    const int32_t p = perm[i];
    CHECK(p >= 0 && p < n && !seen[p], "perm is a bijection");
    if (p >= 0 && p < n) seen[p] = 1;
  }
  /* every leaf-level node has a color below the level's count */
  CHECK(ifmm_tree_query(t, 4, "color", NULL, 0, &cnt) == IFMM_OK && cnt > 0, "color count");
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)cnt);
  CHECK(ifmm_tree_query(t, 4, "color", col, cnt, &cnt) == IFMM_OK, "color");
  for (int64_t i = 0; i < cnt; ++i) CHECK(col[i] >= 0 && col[i] < ncol[4], "color in range");

  /* the error protocol: a bad argument gives IFMM_EINVAL, a NULL handle and a message */
  ifmm_tree* bad = (ifmm_tree*)1;
  CHECK(ifmm_build_tree(xyz, n, 1, &bad) == IFMM_EINVAL, "depth below 2 is refused");
  CHECK(bad == NULL, "the output handle is cleared on error");
  CHECK(ifmm_last_error() != NULL && strlen(ifmm_last_error()) > 0, "the error is described");
  CHECK(ifmm_color(t, 2, NULL) == IFMM_EINVAL, "sigma below 3 is refused");

  ifmm_tree_free(t);
  free(col);
  free(seen);
  free(perm);
  free(xyz);
  if (fails == 0) printf("c_abi ok (%zu entry points)\n", nfn);
  return fails ? 1 : 0;
}
