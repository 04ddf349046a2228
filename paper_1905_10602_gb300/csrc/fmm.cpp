// The FMM matvec y = A~ x (Sec. 2.2, Eq. (1); the paper's FMBEM applies its A
// through an FMM, Algorithm 4): the device structure of one tree at one
// Chebyshev order and kernel -- the leaves' interpolation matrices, the M2M
// table of the 8 octants, the M2L table of every level, the lists -- built once
// and cached on the tree, and its application (kernels in runtime.cu).
#include <cmath>
#include <mutex>

#include "fact.h"
#include "ifmm_kernels.h"

namespace ifmm {

struct FmmPlan {
  int order = 0, rc = 0;
  double scale = 0, diag = 0;
  int device = -1;
  DeviceArena mem;
  double* S = nullptr;
  long* soff = nullptr;
  int* leaf_ptr = nullptr;
  int* nbr_ptr = nullptr;
  int* nbr = nullptr;
  double* m2m = nullptr;
  struct Lev {
    int n = 0;
    int *il_ptr = nullptr, *il = nullptr, *cells = nullptr, *parent = nullptr, *child_ptr = nullptr, *child = nullptr;
    double *tab = nullptr, *M = nullptr, *L = nullptr;
  };
  std::vector<Lev> lv;
};

void fmm_free(FmmPlan* p) { delete p; }

static std::mutex g_fmm_mutex;

template <class T>
static T* up(DeviceArena& mem, const std::vector<T>& v, cudaStream_t s) {
  T* d = (T*)mem.alloc_bytes(sizeof(T) * std::max<size_t>(1, v.size()));
  if (!v.empty()) CK(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
  return d;
}

FmmPlan* fmm_plan(ifmm_tree& T, int order, double scale, double diag, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_fmm_mutex);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (T.fmm && T.fmm->order == order && T.fmm->scale == scale && T.fmm->diag == diag && T.fmm->device == dev)
    return T.fmm;
  IFMM_REQUIRE(order >= 2 && order <= 6, IFMM_EINVAL, "FMM order must be in [2, 6]");
  T.ensure_device();
  auto P = new FmmPlan();
  try {
    P->order = order;
    P->rc = order * order * order;
    P->scale = scale;
    P->diag = diag;
    P->device = dev;
    const int ell = T.depth, rc = P->rc;
    const LevelLists& LL = T.lv[ell];
    DescStage st;
    st.stream = s;
    // leaf interpolation matrices S (rc x n, ld rc), leaf after leaf
    std::vector<long> soff(LL.n + 1, 0);
    for (int i = 0; i < LL.n; ++i) soff[i + 1] = soff[i] + (long)rc * (T.leaf_ptr[i + 1] - T.leaf_ptr[i]);
    P->S = P->mem.alloc(std::max<long>(1, soff[LL.n]));
    std::vector<InterpDesc> ip;
    const double h = 0.5 * T.side / (double)((int64_t)1 << ell);
    for (int i = 0; i < LL.n; ++i) {
      InterpDesc d;
      d.dst = P->S + soff[i];
      d.cx = T.origin[0] + (LL.cells[3 * i] + 0.5) * 2 * h;
      d.cy = T.origin[1] + (LL.cells[3 * i + 1] + 0.5) * 2 * h;
      d.cz = T.origin[2] + (LL.cells[3 * i + 2] + 0.5) * 2 * h;
      d.h = h;
      d.p0 = T.leaf_ptr[i];
      d.n = T.leaf_ptr[i + 1] - T.leaf_ptr[i];
      d.ld = rc;
      d.pad = 0;
      if (d.n) ip.push_back(d);
    }
    launch_interp(st, ip, T.d_pts, (int)T.N, order, 1);
    P->soff = up(P->mem, soff, s);
    P->leaf_ptr = up(P->mem, T.leaf_ptr, s);
    P->nbr_ptr = up(P->mem, LL.nbr_ptr, s);
    P->nbr = up(P->mem, LL.nbr, s);
    P->m2m = P->mem.alloc((size_t)8 * rc * rc);
    launch_m2m_table(s, P->m2m, order, 1);
    P->lv.assign(ell + 1, FmmPlan::Lev());
    for (int kappa = 2; kappa <= ell; ++kappa) {
      const LevelLists& L = T.lv[kappa];
      FmmPlan::Lev& V = P->lv[kappa];
      V.n = L.n;
      V.il_ptr = up(P->mem, L.il_ptr, s);
      V.il = up(P->mem, L.il, s);
      V.cells = up(P->mem, L.cells, s);
      V.parent = up(P->mem, L.parent, s);
      V.child_ptr = up(P->mem, L.child_ptr, s);
      V.child = up(P->mem, L.child, s);
      V.tab = P->mem.alloc((size_t)343 * rc * rc);
      ifmm_kernel kk{};
      kk.scale = scale;
      kk.diag = diag;
      launch_m2l_table(s, V.tab, order, 0.5 * T.side / (double)((int64_t)1 << kappa), kk);
      V.M = P->mem.alloc((size_t)std::max(1, L.n) * rc);
      V.L = P->mem.alloc((size_t)std::max(1, L.n) * rc);
    }
    CK(cudaStreamSynchronize(s));
  } catch (...) {
    delete P;
    throw;
  }
  fmm_free(T.fmm);
  T.fmm = P;
  return P;
}

// x, y: tree-ordered device vectors of length N
void fmm_apply(const ifmm_tree& T, FmmPlan& P, const double* x, double* y, cudaStream_t s) {
  const int ell = T.depth, rc = P.rc;
  auto& lv = P.lv;
  launch_fmm_p2m(s, P.S, P.soff, P.leaf_ptr, x, lv[ell].M, lv[ell].n, rc);
  for (int kappa = ell; kappa >= 3; --kappa)
    launch_fmm_m2m(s, lv[kappa - 1].child_ptr, lv[kappa - 1].child, lv[kappa].cells, P.m2m, lv[kappa].M,
                   lv[kappa - 1].M, lv[kappa - 1].n, rc);
  for (int kappa = 2; kappa <= ell; ++kappa)
    launch_fmm_m2l(s, lv[kappa].il_ptr, lv[kappa].il, lv[kappa].cells, lv[kappa].tab, lv[kappa].M, lv[kappa].L,
                   lv[kappa].n, rc);
  for (int kappa = 3; kappa <= ell; ++kappa)
    launch_fmm_l2l(s, lv[kappa].parent, lv[kappa].cells, P.m2m, lv[kappa - 1].L, lv[kappa].L, lv[kappa].n, rc);
  launch_fmm_l2p(s, P.S, P.soff, P.leaf_ptr, P.nbr_ptr, P.nbr, lv[ell].L, T.d_pts, (int)T.N, x, y, lv[ell].n, rc,
                 P.scale, P.diag);
  check_launch("fmm matvec", 3L * ell);
}

}  // namespace ifmm
