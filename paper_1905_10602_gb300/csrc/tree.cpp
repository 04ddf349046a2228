// Host side of the hierarchy: uniform octree with neighbour and interaction
// lists (Sec. 2.1) and the greedy coloring of Algorithm 3 (Sec. 3.4).
//
// Integer work on O(N) data; the paper builds it once before the factorization
// and reports < 0.1 s for the coloring at 116k nodes.  Compiled with
// -ffp-contract=off so the cell of every point is decided by the same IEEE
// operations on every machine.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include <cuda_runtime.h>

#include "common.h"

namespace ifmm {

int LevelLists::find(int64_t ix, int64_t iy, int64_t iz) const {
  if (ix < 0 || iy < 0 || iz < 0 || ix >= m || iy >= m || iz >= m) return -1;
  int64_t key = (iz * m + iy) * m + ix;
  auto it = std::lower_bound(lin.begin(), lin.end(), key);
  if (it == lin.end() || *it != key) return -1;
  return (int)(it - lin.begin());
}

static void build_level_from_cells(LevelLists& L, int kappa, std::vector<int64_t> lins) {
  L.kappa = kappa;
  L.m = 1 << kappa;
  std::sort(lins.begin(), lins.end());
  lins.erase(std::unique(lins.begin(), lins.end()), lins.end());
  L.lin = std::move(lins);
  L.n = (int)L.lin.size();
  L.cells.resize(3 * (size_t)L.n);
  const int64_t m = L.m;
  for (int i = 0; i < L.n; ++i) {
    int64_t v = L.lin[i];
    L.cells[3 * i + 0] = (int32_t)(v % m);
    L.cells[3 * i + 1] = (int32_t)((v / m) % m);
    L.cells[3 * i + 2] = (int32_t)(v / (m * m));
  }
}

// Algorithm 3.  The scan of a row visits its occupied cells only: a miss moves
// i by one cell, so jumping to the next occupied cell at or after i is the
// same walk.
static void greedy_coloring(LevelLists& L, int sigma) {
  const int m = L.m;
  // rows keyed by (k, j): sorted (ix, node)
  std::unordered_map<int64_t, std::vector<std::pair<int, int>>> rows;
  rows.reserve(L.n);
  for (int v = 0; v < L.n; ++v) {
    int64_t key = (int64_t)L.cells[3 * v + 2] * m + L.cells[3 * v + 1];
    rows[key].push_back({L.cells[3 * v + 0], v});
  }
  for (auto& kv : rows) std::sort(kv.second.begin(), kv.second.end());
  std::vector<int32_t> color(L.n, -1);
  std::vector<int32_t> gptr{0}, glist;
  glist.reserve(L.n);
  int g = 0;
  auto scan_row = [&](int j, int k, int i, int gcol) {
    auto it = rows.find((int64_t)k * m + j);
    if (it == rows.end()) return false;
    bool hit = false;
    for (auto& e : it->second) {
      if (e.first < i || color[e.second] >= 0) continue;
      color[e.second] = gcol;
      glist.push_back(e.second);
      hit = true;
      i = e.first + sigma;
    }
    return hit;
  };
  // nodes are in (k, j, i) lexicographic order already: the outer triple loop
  // of Algorithm 3 visits them in node order.
  for (int u = 0; u < L.n; ++u) {
    if (color[u] >= 0) continue;
    const int i0 = L.cells[3 * u], j0 = L.cells[3 * u + 1], k0 = L.cells[3 * u + 2];
    color[u] = g;
    glist.push_back(u);
    bool j_stride = true, k_stride = true;
    int k = k0;
    while (k < m) {
      int j = (k == k0) ? j0 : 0;
      while (j < m) {
        int i = (j == j0 && k == k0) ? i0 + sigma : 0;
        if (scan_row(j, k, i, g)) {
          j_stride = true;
          k_stride = true;
        }
        j = j_stride ? j + sigma : j + 1;
        j_stride = false;
      }
      k = k_stride ? k + sigma : k + 1;
      k_stride = false;
    }
    gptr.push_back((int32_t)glist.size());
    ++g;
  }
  L.color = std::move(color);
  L.group_ptr = std::move(gptr);
  L.group = std::move(glist);
}

}  // namespace ifmm

using namespace ifmm;

static ifmm_tree* build_tree(const double* xyz, int64_t n, int depth) {
  IFMM_REQUIRE(xyz != nullptr, IFMM_EINVAL, "xyz is NULL");
  IFMM_REQUIRE(n >= 1 && n < (int64_t)1 << 31, IFMM_EINVAL, "n out of range");
  IFMM_REQUIRE(depth >= 2 && depth <= 10, IFMM_EINVAL, "depth must be in [2, 10]");
  auto* t = new ifmm_tree();
  t->N = n;
  t->depth = depth;
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) lo[d] = hi[d] = xyz[d];
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      double v = xyz[3 * i + d];
      IFMM_REQUIRE(std::isfinite(v), IFMM_EINVAL, "non-finite coordinate");
      lo[d] = std::min(lo[d], v);
      hi[d] = std::max(hi[d], v);
    }
  double center[3], ext = 0;
  for (int d = 0; d < 3; ++d) {
    center[d] = 0.5 * (lo[d] + hi[d]);
    ext = std::max(ext, hi[d] - lo[d]);
  }
  t->side = ext * (1.0 + 1e-12);
  if (t->side == 0.0) t->side = 1.0;
  for (int d = 0; d < 3; ++d) t->origin[d] = center[d] - 0.5 * t->side;
  const int64_t m = (int64_t)1 << depth;
  const double h = t->side / (double)m;
  std::vector<int64_t> leaf_lin(n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t g[3];
    for (int d = 0; d < 3; ++d) {
      double q = std::floor((xyz[3 * i + d] - t->origin[d]) / h);
      int64_t v = (int64_t)q;
      g[d] = std::min<int64_t>(std::max<int64_t>(v, 0), m - 1);
    }
    leaf_lin[i] = (g[2] * m + g[1]) * m + g[0];
  }
  std::vector<int32_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return leaf_lin[a] < leaf_lin[b]; });
  t->perm = perm;
  t->pts.resize(3 * (size_t)n);
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) t->pts[3 * i + d] = xyz[3 * (int64_t)perm[i] + d];
  t->lv.resize(depth + 1);
  build_level_from_cells(t->lv[depth], depth, leaf_lin);
  for (int kappa = depth - 1; kappa >= 0; --kappa) {
    const LevelLists& C = t->lv[kappa + 1];
    std::vector<int64_t> lins(C.n);
    const int64_t mp = (int64_t)1 << kappa;
    for (int c = 0; c < C.n; ++c) {
      int64_t ix = C.cells[3 * c] / 2, iy = C.cells[3 * c + 1] / 2, iz = C.cells[3 * c + 2] / 2;
      lins[c] = (iz * mp + iy) * mp + ix;
    }
    build_level_from_cells(t->lv[kappa], kappa, lins);
  }
  // leaf point CSR
  {
    LevelLists& Lf = t->lv[depth];
    t->leaf_ptr.assign(Lf.n + 1, 0);
    int node = 0;
    for (int64_t i = 0; i < n; ++i) {
      int64_t v = leaf_lin[perm[i]];
      while (Lf.lin[node] != v) ++node;
      t->leaf_ptr[node + 1] = (int32_t)(i + 1);
    }
    for (int k = 1; k <= Lf.n; ++k) t->leaf_ptr[k] = std::max(t->leaf_ptr[k], t->leaf_ptr[k - 1]);
  }
  // parents / children
  for (int kappa = depth; kappa >= 1; --kappa) {
    LevelLists& L = t->lv[kappa];
    LevelLists& P = t->lv[kappa - 1];
    L.parent.resize(L.n);
    std::vector<int32_t> cnt(P.n + 1, 0);
    for (int c = 0; c < L.n; ++c) {
      int p = P.find(L.cells[3 * c] / 2, L.cells[3 * c + 1] / 2, L.cells[3 * c + 2] / 2);
      L.parent[c] = p;
      cnt[p + 1]++;
    }
    for (int k = 0; k < P.n; ++k) cnt[k + 1] += cnt[k];
    P.child_ptr = cnt;
    P.child.resize(L.n);
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (int c = 0; c < L.n; ++c) P.child[fill[L.parent[c]]++] = c;  // ascending
  }
  // neighbour lists: offsets walked with dz slowest, dx fastest = ascending node id
  for (int kappa = 0; kappa <= depth; ++kappa) {
    LevelLists& L = t->lv[kappa];
    L.nbr_ptr.assign(1, 0);
    for (int v = 0; v < L.n; ++v) {
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (!dx && !dy && !dz) continue;
            int k = L.find(L.cells[3 * v] + dx, L.cells[3 * v + 1] + dy, L.cells[3 * v + 2] + dz);
            if (k >= 0) L.nbr.push_back(k);
          }
      L.nbr_ptr.push_back((int32_t)L.nbr.size());
    }
  }
  // interaction lists: children of the parent's neighbours that are not adjacent
  for (int kappa = 0; kappa <= depth; ++kappa) {
    LevelLists& L = t->lv[kappa];
    L.il_ptr.assign(1, 0);
    for (int v = 0; v < L.n; ++v) {
      if (kappa >= 2) {
        const LevelLists& P = t->lv[kappa - 1];
        int p = L.parent[v];
        size_t start = L.il.size();
        for (int a = P.nbr_ptr[p]; a < P.nbr_ptr[p + 1]; ++a) {
          int pn = P.nbr[a];
          for (int b = P.child_ptr[pn]; b < P.child_ptr[pn + 1]; ++b) {
            int c = P.child[b];
            int d = std::max({std::abs(L.cells[3 * v] - L.cells[3 * c]), std::abs(L.cells[3 * v + 1] - L.cells[3 * c + 1]),
                              std::abs(L.cells[3 * v + 2] - L.cells[3 * c + 2])});
            if (d >= 2) L.il.push_back(c);
          }
        }
        std::sort(L.il.begin() + start, L.il.end());
      }
      L.il_ptr.push_back((int32_t)L.il.size());
    }
  }
  return t;
}

static const std::vector<int32_t>* pick(const LevelLists& L, const std::string& w) {
  if (w == "cells") return &L.cells;
  if (w == "parent") return &L.parent;
  if (w == "nbr_ptr") return &L.nbr_ptr;
  if (w == "nbr") return &L.nbr;
  if (w == "il_ptr") return &L.il_ptr;
  if (w == "il") return &L.il;
  if (w == "color") return &L.color;
  if (w == "group_ptr") return &L.group_ptr;
  if (w == "group") return &L.group;
  if (w == "child_ptr") return &L.child_ptr;
  if (w == "child") return &L.child;
  return nullptr;
}

extern "C" {

ifmm_status ifmm_build_tree(const double* xyz, int64_t n, int depth, ifmm_tree** out) {
  if (out) *out = nullptr;
  try {
    IFMM_REQUIRE(out != nullptr, IFMM_EINVAL, "out is NULL");
    IFMM_REQUIRE(xyz != nullptr, IFMM_EINVAL, "xyz is NULL");
    IFMM_REQUIRE(n >= 1 && n <= ((int64_t)1 << 31) - 1, IFMM_EINVAL, "n out of range");
    // device points are copied to the host: the octree and lists are built there
    cudaPointerAttributes a;
    const bool on_dev = cudaPointerGetAttributes(&a, xyz) == cudaSuccess &&
                        (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (on_dev) {
      std::vector<double> h(3 * (size_t)n);
      const cudaError_t e = cudaMemcpy(h.data(), xyz, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost);
      IFMM_REQUIRE(e == cudaSuccess, IFMM_ECUDA, std::string("copying device points: ") + cudaGetErrorString(e));
      *out = build_tree(h.data(), n, depth);
    } else {
      *out = build_tree(xyz, n, depth);
    }
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return IFMM_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return IFMM_EINVAL;
  }
}

// Levels below tau: one node per color, in node (scan) order -- the nodes are
// eliminated one after the other, each with the whole GPU (matrix-parallel).
static void sequential_coloring(LevelLists& L) {
  L.color.resize(L.n);
  L.group_ptr.resize(L.n + 1);
  L.group.resize(L.n);
  for (int i = 0; i < L.n; ++i) {
    L.color[i] = i;
    L.group_ptr[i] = i;
    L.group[i] = i;
  }
  L.group_ptr[L.n] = L.n;
}

ifmm_status ifmm_color(ifmm_tree* t, int sigma, int32_t* ncolors) { return ifmm_color_levels(t, sigma, 2, ncolors); }

ifmm_status ifmm_color_levels(ifmm_tree* t, int sigma, int tau, int32_t* ncolors) {
  try {
    IFMM_REQUIRE(t != nullptr, IFMM_EINVAL, "tree is NULL");
    IFMM_REQUIRE(sigma >= 3 && sigma <= 64, IFMM_EINVAL, "sigma must be in [3, 64] (sigma >= 3 keeps neighbour sets of a color disjoint)");
    IFMM_REQUIRE(tau >= 2 && tau <= t->depth, IFMM_EINVAL, "tau must be in [2, depth]");
    for (int kappa = 0; kappa <= t->depth; ++kappa) {
      LevelLists& L = t->lv[kappa];
      if (kappa >= tau) {
        greedy_coloring(L, sigma);
      } else if (kappa >= 2) {
        sequential_coloring(L);
      } else {
        L.color.assign(L.n, -1);
        L.group_ptr.assign(1, 0);
        L.group.clear();
      }
      if (ncolors) ncolors[kappa] = kappa >= 2 ? (int32_t)(L.group_ptr.size() - 1) : 0;
    }
    t->sigma = sigma;
    t->tau = tau;
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return IFMM_ENOMEM;
  }
}

ifmm_status ifmm_tree_query(const ifmm_tree* t, int level, const char* what, int32_t* buf, int64_t cap,
                            int64_t* count) {
  try {
    IFMM_REQUIRE(t && what && count, IFMM_EINVAL, "NULL argument");
    std::string w(what);
    const std::vector<int32_t>* v = nullptr;
    if (w == "perm") {
      v = &t->perm;
    } else if (w == "matvec_block") {
      v = &t->matvec_block_v;
    } else if (w == "leaf_ptr") {
      v = &t->leaf_ptr;
    } else {
      IFMM_REQUIRE(level >= 0 && level <= t->depth, IFMM_EINVAL, "level out of range");
      v = pick(t->lv[level], w);
      IFMM_REQUIRE(v != nullptr, IFMM_EINVAL, "unknown query " + w);
    }
    *count = (int64_t)v->size();
    if (buf && cap > 0) std::memcpy(buf, v->data(), sizeof(int32_t) * (size_t)std::min<int64_t>(cap, *count));
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

}  // extern "C"
