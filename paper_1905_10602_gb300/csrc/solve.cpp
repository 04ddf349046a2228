// IFMM solve (Algorithm 2 on the extended system), direct-summation matvec and
// GMRES(m) with right preconditioning (Algorithms 4 and 5).
//
// The solve's launches are fixed once the factor exists: the plan is built
// once, uploaded once and captured into a CUDA graph; applying the
// preconditioner is one graph launch.  Vectors of all levels live in one
// buffer laid out so that a node's R-row vector (its y in the backward pass) is
// the matching slice of its parent's x vector: aggregation (Algorithm 2,
// "aggregate x of the children") and splitting cost nothing.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "fact.h"
#include "ifmm_kernels.h"

namespace ifmm {

// A GEMV over many rows becomes several descriptors of at most 64 rows (one
// CTA each), so a large pivot block is spread over several SMs.
static void push_gemv_rows(std::vector<GemvDesc>& out, const GemvDesc& g) {
  const int chunk = 64;
  if (g.trans || g.m <= chunk) {
    out.push_back(g);
    return;
  }
  for (int r = 0; r < g.m; r += chunk) {
    GemvDesc c = g;
    c.A = g.A + r;
    c.y = g.y + r;
    c.m = std::min(chunk, g.m - r);
    out.push_back(c);
  }
}

void build_solve_plan(ifmm_fact& F, cudaStream_t s) {
  const ifmm_tree& T = *F.t;
  const int ell = T.depth;
  SolvePlan& P = F.plan;
  // offsets of every node's x segment per level, and of the top vector
  std::vector<std::vector<int64_t>> xoff(ell + 1);
  std::vector<int64_t> base(ell + 1, 0);
  int64_t total = 0;
  base[1] = 0;
  total = F.ntop;
  for (int kappa = 2; kappa <= ell; ++kappa) {
    const LevelFactor& LF = F.lv[kappa];
    base[kappa] = total;
    xoff[kappa].resize(LF.nn + 1);
    int64_t o = 0;
    for (int i = 0; i < LF.nn; ++i) {
      xoff[kappa][i] = o;
      o += LF.n[i];
    }
    xoff[kappa][LF.nn] = o;
    total += o;
  }
  // R-vector location (absolute index into X) of node i at level kappa
  auto rloc = [&](int kappa, int i) -> int64_t {
    if (kappa == 2) return base[1] + F.top_off[i];
    const LevelLists& PL = T.lv[kappa - 1];
    const int par = T.lv[kappa].parent[i];
    int64_t off = 0;
    for (int c = PL.child_ptr[par]; c < PL.child_ptr[par + 1]; ++c) {
      const int ch = PL.child[c];
      if (ch == i) break;
      off += F.lv[kappa].r[ch];
    }
    return base[kappa - 1] + xoff[kappa - 1][par] + off;
  };
  int64_t tlen = std::max<int64_t>(F.ntop, 1);
  for (int kappa = 2; kappa <= ell; ++kappa) {
    int64_t t = 0;
    for (int i = 0; i < F.lv[kappa].nn; ++i) t += F.lv[kappa].n[i] + F.lv[kappa].r[i];
    tlen = std::max(tlen, t);
  }
  P.xlen = total;
  P.X = P.mem.alloc((size_t)std::max<int64_t>(total, 1));
  P.tvec = P.mem.alloc((size_t)tlen);
  double* X = P.X;
  std::vector<CopyDesc> all_copy;
  std::vector<GemvDesc> all_gemv;
  std::vector<GemvSumDesc> all_sum;
  std::vector<GemvTerm> all_terms;
  struct L {
    int kind;
    size_t first, count;
  };
  std::vector<L> prog;
  auto emit_gemv = [&](std::vector<GemvDesc>& v) {
    if (v.empty()) return;
    prog.push_back({1, all_gemv.size(), v.size()});
    all_gemv.insert(all_gemv.end(), v.begin(), v.end());
    v.clear();
  };
  auto emit_copy = [&](std::vector<CopyDesc>& v) {
    if (v.empty()) return;
    prog.push_back({0, all_copy.size(), v.size()});
    all_copy.insert(all_copy.end(), v.begin(), v.end());
    v.clear();
  };
  auto emit_sum = [&](std::vector<GemvSumDesc>& v) {
    if (v.empty()) return;
    prog.push_back({2, all_sum.size(), v.size()});
    all_sum.insert(all_sum.end(), v.begin(), v.end());
    v.clear();
  };
  // per-node t/s scratch offsets (re-used across levels)
  std::vector<std::vector<int64_t>> toff(ell + 1);
  for (int kappa = 2; kappa <= ell; ++kappa) {
    const LevelFactor& LF = F.lv[kappa];
    toff[kappa].resize(LF.nn);
    int64_t o = 0;
    for (int i = 0; i < LF.nn; ++i) {
      toff[kappa][i] = o;
      o += LF.n[i] + LF.r[i];
    }
  }
  // ---- forward substitution (upward), colors ascending
  for (int kappa = ell; kappa >= 2; --kappa) {
    const LevelFactor& LF = F.lv[kappa];
    double* Xk = X + base[kappa];
    for (const auto& grp : LF.order) {
      std::vector<GemvDesc> g1, g2;
      std::vector<CopyDesc> c2;
      for (int i : grp) {
        const NodeFactor& nf = LF.nf[i];
        const int n = nf.n, r = nf.r, m = n + r;
        double* t = P.tvec + toff[kappa][i];
        if (m == 0) continue;
        if (n) push_gemv_rows(g1, gmv(nf.piinv, m, m, n, 0, Xk + xoff[kappa][i], t, 1.0, 0.0));
        else c2.push_back(cpy(nullptr, 0, t, m, m, 1));
        for (size_t a = 0; a < nf.nb.size(); ++a) {
          const int q = nf.nb[a];
          const int mq = nf.lcol_rows[a];
          if (!mq || !n) continue;
          double* y = nf.was_elim[a] ? X + rloc(kappa, q) : Xk + xoff[kappa][q];
          push_gemv_rows(g2, gmv(nf.lcol[a], nf.lcol_ld[a], mq, n, 0, t, y, -1.0, 1.0));
        }
        if (r) c2.push_back(cpy(t + n, m, X + rloc(kappa, i), r, r, 1));
      }
      emit_gemv(g1);
      emit_copy(c2);
      emit_gemv(g2);
    }
  }
  // ---- top: y2 = D^{-1} rhs
  if (F.ntop) {
    std::vector<GemvDesc> g;
    std::vector<CopyDesc> c;
    push_gemv_rows(g, gmv(F.top_inv, F.ntop, F.ntop, F.ntop, 0, X + base[1], P.tvec, 1.0, 0.0));
    c.push_back(cpy(P.tvec, F.ntop, X + base[1], F.ntop, F.ntop, 1));
    emit_gemv(g);
    emit_copy(c);
  }
  // ---- backward substitution (downward), colors descending
  for (int kappa = 2; kappa <= ell; ++kappa) {
    const LevelFactor& LF = F.lv[kappa];
    double* Xk = X + base[kappa];
    for (auto it = LF.order.rbegin(); it != LF.order.rend(); ++it) {
      std::vector<CopyDesc> c1;
      std::vector<GemvSumDesc> s1;
      std::vector<GemvDesc> g2;
      for (int i : *it) {
        const NodeFactor& nf = LF.nf[i];
        const int n = nf.n, r = nf.r, m = n + r;
        if (!n) continue;
        double* sv = P.tvec + toff[kappa][i];
        c1.push_back(cpy(Xk + xoff[kappa][i], n, sv, m, n, 1));
        if (r) c1.push_back(cpy(X + rloc(kappa, i), r, sv + n, m, r, 1));
        GemvSumDesc sd;
        sd.y = sv;
        sd.m = n;
        sd.row0 = 0;
        sd.first = (int)all_terms.size();
        sd.count = 0;
        sd.alpha = -1.0;
        sd.beta = 1.0;
        for (size_t a = 0; a < nf.nb.size(); ++a) {
          const int q = nf.nb[a];
          const int mq = nf.urow_cols[a];
          if (!mq) continue;
          const double* val = nf.was_elim[a] ? X + rloc(kappa, q) : Xk + xoff[kappa][q];
          all_terms.push_back(GemvTerm{nf.urow[a], val, n, mq});
          sd.count++;
        }
        if (sd.count)
          for (int r0 = 0; r0 < n; r0 += 32) {
            GemvSumDesc c = sd;
            c.m = std::min(32, n - r0);
            c.y = sd.y + r0;
            c.row0 = r0;
            s1.push_back(c);
          }
        push_gemv_rows(g2, gmv(nf.piinv, m, n, m, 0, sv, Xk + xoff[kappa][i], 1.0, 0.0));
      }
      emit_copy(c1);
      emit_sum(s1);
      emit_gemv(g2);
    }
  }
  // upload
  CopyDesc* dc = (CopyDesc*)P.mem.alloc_bytes(std::max<size_t>(1, all_copy.size()) * sizeof(CopyDesc));
  GemvDesc* dg = (GemvDesc*)P.mem.alloc_bytes(std::max<size_t>(1, all_gemv.size()) * sizeof(GemvDesc));
  GemvSumDesc* ds = (GemvSumDesc*)P.mem.alloc_bytes(std::max<size_t>(1, all_sum.size()) * sizeof(GemvSumDesc));
  GemvTerm* dt = (GemvTerm*)P.mem.alloc_bytes(std::max<size_t>(1, all_terms.size()) * sizeof(GemvTerm));
  if (!all_copy.empty()) CK(cudaMemcpy(dc, all_copy.data(), all_copy.size() * sizeof(CopyDesc), cudaMemcpyHostToDevice));
  if (!all_gemv.empty()) CK(cudaMemcpy(dg, all_gemv.data(), all_gemv.size() * sizeof(GemvDesc), cudaMemcpyHostToDevice));
  if (!all_sum.empty())
    CK(cudaMemcpy(ds, all_sum.data(), all_sum.size() * sizeof(GemvSumDesc), cudaMemcpyHostToDevice));
  if (!all_terms.empty())
    CK(cudaMemcpy(dt, all_terms.data(), all_terms.size() * sizeof(GemvTerm), cudaMemcpyHostToDevice));
  P.prog.clear();
  for (auto& l : prog) {
    SolveLaunch sl;
    sl.kind = l.kind;
    sl.count = (int)l.count;
    sl.terms = dt;
    if (l.kind == 0) sl.desc = dc + l.first;
    else if (l.kind == 1) sl.desc = dg + l.first;
    else sl.desc = ds + l.first;
    P.prog.push_back(sl);
  }
  P.stage_in = X + base[ell];
  // capture the program into a graph on a private stream
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  for (auto& l : P.prog) {
    if (l.kind == 0) launch_copy_dev(cs, (const CopyDesc*)l.desc, l.count);
    else if (l.kind == 1) launch_gemv_dev(cs, (const GemvDesc*)l.desc, l.count);
    else launch_gemv_sum_dev(cs, (const GemvSumDesc*)l.desc, (const GemvTerm*)l.terms, l.count);
  }
  cudaGraph_t g;
  CK(cudaStreamEndCapture(cs, &g));
  CK(cudaGraphInstantiate(&P.graph, g, 0));
  P.graph_def = g;
  CK(cudaStreamDestroy(cs));
  F.stat("solve_launches", (double)P.prog.size());
  F.stat("solve_vector_len", (double)total);
  (void)s;
}

// in/out: tree-ordered device vectors of length N (may alias)
void run_solve_tree(const ifmm_fact& F, const double* in, double* out, cudaStream_t s) {
  const SolvePlan& P = F.plan;
  const int64_t N = F.t->N;
  CK(cudaMemcpyAsync(P.stage_in, in, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  static const bool direct = [] {
    const char* e = getenv("IFMM_SOLVE_NOGRAPH");
    return e && e[0] == '1';
  }();
  if (direct) {  // the same program as individual launches, each timed when profiling
    for (auto& l : P.prog) {
      const int kind = l.kind == 0 ? KK_COPY : (l.kind == 1 ? KK_GEMV : KK_GEMV_SUM);
      prof_batch_tag() = l.count;
      cudaEvent_t pe = profiler().begin(kind, s);
      if (l.kind == 0) launch_copy_dev(s, (const CopyDesc*)l.desc, l.count);
      else if (l.kind == 1) launch_gemv_dev(s, (const GemvDesc*)l.desc, l.count);
      else launch_gemv_sum_dev(s, (const GemvSumDesc*)l.desc, (const GemvTerm*)l.terms, l.count);
      profiler().end(kind, s, pe);
    }
  } else {
    cudaEvent_t pe = profiler().begin(KK_SOLVE_GRAPH, s, (long)P.prog.size());
    CK(cudaGraphLaunch(P.graph, s));
    profiler().end(KK_SOLVE_GRAPH, s, pe);
    profiler().count(KK_ALL, (long)P.prog.size());
  }
  CK(cudaMemcpyAsync(out, P.stage_in, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
}

static std::mutex g_tune_mutex;

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace ifmm

using namespace ifmm;

void ifmm_tree::ensure_device() {
  if (d_pts) return;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    throw Error(IFMM_ECUDA, "no CUDA device");
  }
  CK(cudaGetDevice(&device));
  std::vector<double> soa(3 * (size_t)N);
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) soa[(size_t)d * N + i] = pts[3 * i + d];
  CK(cudaMalloc(&d_pts, sizeof(double) * 3 * N));
  CK(cudaMemcpy(d_pts, soa.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
  CK(cudaMalloc(&d_perm, sizeof(int32_t) * N));
  CK(cudaMemcpy(d_perm, perm.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice));
  std::vector<float> dfp(6 * (size_t)N);
  for (int64_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) {
      const double v = pts[3 * i + d];
      const float h = (float)v;
      dfp[(size_t)(2 * d) * N + i] = h;
      dfp[(size_t)(2 * d + 1) * N + i] = (float)(v - (double)h);
    }
  CK(cudaMalloc(&d_pts_df, sizeof(float) * 6 * N));
  CK(cudaMemcpy(d_pts_df, dfp.data(), sizeof(float) * 6 * N, cudaMemcpyHostToDevice));
  registry().add(d_pts, sizeof(double) * 3 * N);
  registry().add(d_perm, sizeof(int32_t) * N);
  registry().add(d_pts_df, sizeof(float) * 6 * N);
}

ifmm_tree::~ifmm_tree() {
  if (d_pts) {
    registry().remove_range(d_pts, sizeof(double) * 3 * N);
    cudaFree(d_pts);
  }
  if (d_perm) {
    registry().remove_range(d_perm, sizeof(int32_t) * N);
    cudaFree(d_perm);
  }
  if (d_pts_df) {
    registry().remove_range(d_pts_df, sizeof(float) * 6 * N);
    cudaFree(d_pts_df);
  }
}

// device buffers for the GMRES / solve wrappers
struct Vecs {
  std::vector<std::pair<double*, size_t>> p;
  ~Vecs() {
    for (auto x : p) {
      registry().remove_range(x.first, x.second);
      cudaFree(x.first);
    }
  }
  double* get(size_t n) {
    double* x = nullptr;
    const size_t bytes = sizeof(double) * std::max<size_t>(n, 1);
    CK(cudaMalloc(&x, bytes));
    registry().add(x, bytes);
    p.push_back({x, bytes});
    return x;
  }
};

// dot products / norms on the device through the GEMV kernel, read on the host
struct Blas1 {
  cudaStream_t s;
  DescStage st;
  double* d_out;
  double* h_out;
  explicit Blas1(cudaStream_t s_) : s(s_) {
    st.stream = s;
    CK(cudaMalloc(&d_out, sizeof(double) * 64));
    registry().add(d_out, sizeof(double) * 64);
    CK(cudaMallocHost(&h_out, sizeof(double) * 64));
  }
  ~Blas1() {
    registry().remove_range(d_out, sizeof(double) * 64);
    cudaFree(d_out);
    cudaFreeHost(h_out);
  }
};

extern "C" {

void ifmm_tree_free(ifmm_tree* t) { delete t; }

ifmm_status ifmm_solve(const ifmm_fact* f, const double* r, double* v, int nrhs, void* stream) {
  try {
    IFMM_REQUIRE(f && r && v && nrhs >= 1, IFMM_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = f->t->N;
    const bool dev = is_device_ptr(r);
    IFMM_REQUIRE(dev == is_device_ptr(v), IFMM_EINVAL, "r and v must both be host or both device");
    Vecs V;
    double* a = V.get(N);
    double* b = V.get(N);
    for (int c = 0; c < nrhs; ++c) {
      const double* rc = r + (int64_t)c * N;
      double* vc = v + (int64_t)c * N;
      const double* src = rc;
      if (!dev) {
        CK(cudaMemcpyAsync(b, rc, sizeof(double) * N, cudaMemcpyHostToDevice, s));
        src = b;
      }
      launch_gather_perm(s, src, f->t->d_perm, a, (int)N);
      run_solve_tree(*f, a, a, s);
      if (dev) {
        launch_scatter_perm(s, a, f->t->d_perm, vc, (int)N);
      } else {
        launch_scatter_perm(s, a, f->t->d_perm, b, (int)N);
        CK(cudaMemcpyAsync(vc, b, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
      }
    }
    CK(cudaStreamSynchronize(s));
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return IFMM_ECUDA;
  }
}

ifmm_status bem_matvec(const ifmm_tree* t, const ifmm_kernel* k, const double* x, double* y, void* stream) {
  try {
    IFMM_REQUIRE(t && k && x && y, IFMM_EINVAL, "bad argument");
    const_cast<ifmm_tree*>(t)->ensure_device();
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = t->N;
    const bool dev = is_device_ptr(x);
    IFMM_REQUIRE(dev == is_device_ptr(y), IFMM_EINVAL, "x and y must both be host or both device");
    Vecs V;
    double* a = V.get(N);
    double* b = V.get(N);
    double* c = V.get(N);
    const double* src = x;
    if (!dev) {
      CK(cudaMemcpyAsync(c, x, sizeof(double) * N, cudaMemcpyHostToDevice, s));
      src = c;
    }
    launch_gather_perm(s, src, t->d_perm, a, (int)N);
    if (k->arith == IFMM_ARITH_DF) {
      float* q = (float*)V.get(N);
      launch_split_df(s, a, q, q + N, (int)N);
      ifmm_tree* tm = const_cast<ifmm_tree*>(t);
      if (!tm->matvec_block) {
        tm->matvec_block = autotune_matvec_df(s, t->d_pts_df, q, q + N, a, b, (int)N, k->scale, k->diag);
        tm->matvec_block_v[0] = tm->matvec_block;
      }
      launch_matvec_df(s, t->d_pts_df, q, q + N, a, b, (int)N, k->scale, k->diag, tm->matvec_block);
    } else {
      launch_matvec(s, t->d_pts, (int)N, a, b, k->scale, k->diag);
    }
    if (dev) {
      launch_scatter_perm(s, b, t->d_perm, y, (int)N);
    } else {
      launch_scatter_perm(s, b, t->d_perm, c, (int)N);
      CK(cudaMemcpyAsync(y, c, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return IFMM_ECUDA;
  }
}

ifmm_status bem_gmres(const ifmm_tree* t, const ifmm_kernel* k, const ifmm_fact* pre, const double* b, double* x,
                      int restart, double tol, int maxit, int* iters, double* relres, void* stream) {
  try {
    IFMM_REQUIRE(t && k && b && x, IFMM_EINVAL, "bad argument");
    IFMM_REQUIRE(restart >= 1 && restart <= 1000 && maxit >= 1 && tol > 0, IFMM_EINVAL, "bad GMRES parameters");
    IFMM_REQUIRE(!pre || pre->t == t, IFMM_EINVAL, "preconditioner built on another tree");
    const_cast<ifmm_tree*>(t)->ensure_device();
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = t->N;
    const int m = restart;
    const bool dev = is_device_ptr(b);
    IFMM_REQUIRE(dev == is_device_ptr(x), IFMM_EINVAL, "b and x must both be host or both device");
    Vecs Vm;
    double* bt = Vm.get(N);   // b in tree order
    double* xt = Vm.get(N);   // x in tree order
    double* rt = Vm.get(N);
    double* wt = Vm.get(N);
    double* zt = Vm.get(N);
    double* Vb = Vm.get((size_t)N * (m + 1));
    double* hv = Vm.get((size_t)2 * (m + 2));
    double* tmp = Vm.get(N);
    Blas1 B(s);
    const double* src = b;
    if (!dev) {
      CK(cudaMemcpyAsync(tmp, b, sizeof(double) * N, cudaMemcpyHostToDevice, s));
      src = tmp;
    }
    launch_gather_perm(s, src, t->d_perm, bt, (int)N);
    auto dot = [&](const double* u, const double* v) -> double {
      std::vector<GemvDesc> g{gmv(u, (int)N, (int)N, 1, 1, v, B.d_out, 1.0, 0.0)};
      launch_gemv(B.st, g);
      CK(cudaMemcpyAsync(B.h_out, B.d_out, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      B.st.reset();
      return B.h_out[0];
    };
    auto axpby = [&](double alpha, const double* u, double beta, double* v) {
      std::vector<CopyDesc> c{cpy(u, (int)N, v, (int)N, (int)N, 1, alpha, beta)};
      launch_copy(B.st, c);
    };
    auto precond = [&](const double* in, double* out) {
      if (pre) run_solve_tree(*pre, in, out, s);
      else CK(cudaMemcpyAsync(out, in, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    };
    const bool df_mv = k->arith == IFMM_ARITH_DF;
    float* qdf = df_mv ? (float*)Vm.get(N) : nullptr;
    auto Amul = [&](const double* in, double* out) {
      if (df_mv) {
        launch_split_df(s, in, qdf, qdf + N, (int)N);
        ifmm_tree* tm = const_cast<ifmm_tree*>(t);
        if (!tm->matvec_block) {
          std::lock_guard<std::mutex> lock(g_tune_mutex);
          if (!tm->matvec_block) {
            tm->matvec_block = autotune_matvec_df(s, t->d_pts_df, qdf, qdf + N, in, out, (int)N, k->scale, k->diag);
            tm->matvec_block_v[0] = tm->matvec_block;
          }
        }
        launch_matvec_df(s, t->d_pts_df, qdf, qdf + N, in, out, (int)N, k->scale, k->diag, tm->matvec_block);
      } else {
        launch_matvec(s, t->d_pts, (int)N, in, out, k->scale, k->diag);
      }
    };
    CK(cudaMemsetAsync(xt, 0, sizeof(double) * N, s));
    CK(cudaMemcpyAsync(rt, bt, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    const double bnorm = std::sqrt(dot(bt, bt));
    IFMM_REQUIRE(bnorm > 0, IFMM_EINVAL, "b is zero");
    int its = 0;
    double rel = 1.0;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1);
    while (its < maxit) {
      const double beta = std::sqrt(dot(rt, rt));
      rel = beta / bnorm;
      if (rel <= tol) break;
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      axpby(1.0 / beta, rt, 0.0, Vb);
      int kdone = 0;
      for (int j = 0; j < m; ++j) {
        double* vj = Vb + (size_t)j * N;
        precond(vj, zt);
        Amul(zt, wt);
        ++its;
        // classical Gram-Schmidt, twice
        std::vector<double> h(j + 1, 0.0);
        for (int pass = 0; pass < 2; ++pass) {
          std::vector<GemvDesc> gg{gmv(Vb, (int)N, (int)N, j + 1, 1, wt, hv, 1.0, 0.0)};
          launch_gemv(B.st, gg);
          CK(cudaMemcpyAsync(B.h_out, hv, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
          std::vector<GemvDesc> g2{gmv(Vb, (int)N, (int)N, j + 1, 0, hv, wt, -1.0, 1.0)};
          launch_gemv(B.st, g2);
          CK(cudaStreamSynchronize(s));
          B.st.reset();
          for (int i = 0; i <= j; ++i) h[i] += B.h_out[i];
        }
        const double hn = std::sqrt(dot(wt, wt));
        for (int i = 0; i <= j; ++i) H[i + (size_t)j * (m + 1)] = h[i];
        H[j + 1 + (size_t)j * (m + 1)] = hn;
        if (hn > 0) axpby(1.0 / hn, wt, 0.0, Vb + (size_t)(j + 1) * N);
        for (int i = 0; i < j; ++i) {
          double& a = H[i + (size_t)j * (m + 1)];
          double& c = H[i + 1 + (size_t)j * (m + 1)];
          const double tt = cs[i] * a + sn[i] * c;
          c = -sn[i] * a + cs[i] * c;
          a = tt;
        }
        double& hjj = H[j + (size_t)j * (m + 1)];
        double& hj1 = H[j + 1 + (size_t)j * (m + 1)];
        const double den = std::hypot(hjj, hj1);
        cs[j] = hjj / den;
        sn[j] = hj1 / den;
        hjj = den;
        hj1 = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        kdone = j + 1;
        if (std::fabs(g[j + 1]) / bnorm <= tol || its >= maxit || hn == 0) break;
      }
      // y = H^{-1} g (upper triangular), u = V y, x += M u
      std::vector<double> y(kdone);
      for (int i = kdone - 1; i >= 0; --i) {
        double sacc = g[i];
        for (int jj = i + 1; jj < kdone; ++jj) sacc -= H[i + (size_t)jj * (m + 1)] * y[jj];
        y[i] = sacc / H[i + (size_t)i * (m + 1)];
      }
      CK(cudaMemcpyAsync(hv, y.data(), sizeof(double) * kdone, cudaMemcpyHostToDevice, s));
      std::vector<GemvDesc> gu{gmv(Vb, (int)N, (int)N, kdone, 0, hv, wt, 1.0, 0.0)};
      launch_gemv(B.st, gu);
      precond(wt, zt);
      axpby(1.0, zt, 1.0, xt);
      Amul(xt, rt);
      axpby(1.0, bt, -1.0, rt);
      CK(cudaStreamSynchronize(s));
      B.st.reset();
    }
    {
      const double rn = std::sqrt(dot(rt, rt));
      rel = rn / bnorm;
    }
    if (dev) {
      launch_scatter_perm(s, xt, t->d_perm, x, (int)N);
    } else {
      launch_scatter_perm(s, xt, t->d_perm, tmp, (int)N);
      CK(cudaMemcpyAsync(x, tmp, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    if (iters) *iters = its;
    if (relres) *relres = rel;
    if (rel > tol) {
      set_last_error("GMRES did not reach tol within maxit");
      return IFMM_ENOCONV;
    }
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return IFMM_ECUDA;
  }
}

}  // extern "C"
