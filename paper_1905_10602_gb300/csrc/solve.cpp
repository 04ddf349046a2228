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
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "fact.h"
#include "ifmm_kernels.h"

namespace ifmm {

// lanes sharing one row of ncols coefficients, v per 16-byte vector: enough
// lanes that each takes about two vectors, at most a warp
int solve_row_lanes(int ncols, int v) {
  int g = 1;
  while (g < 32 && g * v * 2 < ncols) g *= 2;
  return g;
}
static int pad4(int x) { return (x + 3) & ~3; }

// Uploads the launches of a solve program (op lists, with gather / scatter
// index lists given as offsets into idx_all, -1 for none) and captures them
// into the plan's CUDA graph.
void capture_solve_plan(SolvePlan& P, const std::vector<std::vector<SolveOp>>& launches,
                        const std::vector<std::vector<int64_t>>& xoff, const std::vector<std::vector<int64_t>>& ooff,
                        const std::vector<int32_t>& idx_all) {
  int32_t* dx = (int32_t*)P.mem.alloc_bytes(sizeof(int32_t) * std::max<size_t>(1, idx_all.size()));
  if (!idx_all.empty()) CK(cudaMemcpy(dx, idx_all.data(), sizeof(int32_t) * idx_all.size(), cudaMemcpyHostToDevice));
  std::vector<SolveOp> ops_all;
  std::vector<int> wp_all;
  std::vector<std::array<size_t, 3>> where;  // op offset, warp_ptr offset, warps
  for (size_t li = 0; li < launches.size(); ++li) {
    const size_t o0 = ops_all.size(), w0 = wp_all.size();
    int warps = 0;
    wp_all.push_back(0);
    for (size_t k = 0; k < launches[li].size(); ++k) {
      SolveOp o = launches[li][k];
      if (xoff[li][k] >= 0) o.xidx = dx + xoff[li][k];
      if (ooff[li][k] >= 0) o.oidx = dx + ooff[li][k];
      warps += (o.rows + 32 / o.lanes - 1) / (32 / o.lanes);
      ops_all.push_back(o);
      wp_all.push_back(warps);
    }
    where.push_back({o0, w0, (size_t)warps});
  }
  SolveOp* dops = (SolveOp*)P.mem.alloc_bytes(sizeof(SolveOp) * std::max<size_t>(1, ops_all.size()));
  int* dwp = (int*)P.mem.alloc_bytes(sizeof(int) * std::max<size_t>(1, wp_all.size()));
  if (!ops_all.empty()) CK(cudaMemcpy(dops, ops_all.data(), sizeof(SolveOp) * ops_all.size(), cudaMemcpyHostToDevice));
  if (!wp_all.empty()) CK(cudaMemcpy(dwp, wp_all.data(), sizeof(int) * wp_all.size(), cudaMemcpyHostToDevice));
  P.prog.clear();
  for (size_t li = 0; li < launches.size(); ++li)
    P.prog.push_back(SolveLaunch{dops + where[li][0], dwp + where[li][1], (int)launches[li].size(), (int)where[li][2]});
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  for (auto& l : P.prog) launch_solve_ops(cs, l.ops, l.warp_ptr, l.nops, l.nwarps, P.pairs);
  cudaGraph_t g;
  CK(cudaStreamEndCapture(cs, &g));
  CK(cudaGraphInstantiate(&P.graph, g, 0));
  P.graph_def = g;
  CK(cudaStreamDestroy(cs));
}

void build_solve_plan(ifmm_fact& F, cudaStream_t s) {
  const ifmm_tree& T = *F.t;
  const int ell = T.depth;
  SolvePlan& P = F.plan;
  P.pairs = F.o.precision != IFMM_PREC_FP64;
  const int esz = P.pairs ? 4 : 8;  // bytes of one packed coefficient
  const int vw = 16 / esz;          // coefficients per 16-byte vector
  // offsets (in elements of V) of every node's x segment per level, of the top
  // vector (level 1), and of the per-node scratch
  std::vector<std::vector<int64_t>> xoff(ell + 1);
  std::vector<int64_t> base(ell + 1, 0);
  int64_t total = F.ntop;
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
  // V index of node i's R-row vector (its y): the matching slice of its
  // parent's x, or of the top vector at level 2
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
  std::vector<std::vector<int64_t>> toff(ell + 1);
  int64_t tlen = std::max<int64_t>(F.ntop, 1);
  for (int kappa = 2; kappa <= ell; ++kappa) {
    const LevelFactor& LF = F.lv[kappa];
    toff[kappa].resize(LF.nn);
    int64_t o = 0;
    for (int i = 0; i < LF.nn; ++i) {
      toff[kappa][i] = o;
      o += LF.n[i] + LF.r[i];
    }
    tlen = std::max(tlen, o);
  }
  P.xlen = total;
  P.vlen = total + tlen;
  IFMM_REQUIRE(P.vlen < ((int64_t)1 << 31), IFMM_EINVAL, "solve vectors exceed 2^31 elements");
  P.V = P.mem.alloc_bytes(8 * (size_t)P.vlen);
  const int64_t TB = total;  // scratch starts here
  char* V = (char*)P.V;
  auto vp = [&](int64_t idx) { return (void*)(V + 8 * idx); };
  // packed row-major copies of every block the solve reads
  std::vector<PackDesc> pk;
  auto packed = [&](const double* src, int lds, int rows, int cols, int& ldm) -> void* {
    ldm = pad4(std::max(cols, 1));
    void* dst = P.mem.alloc_bytes((size_t)esz * std::max(rows, 1) * ldm);
    if (rows && cols) pk.push_back(PackDesc{src, dst, lds, ldm, rows, cols});
    return dst;
  };
  std::vector<int32_t> xidx_all;  // gather indices, uploaded once
  std::vector<std::vector<SolveOp>> launches;
  auto op = [&](const void* M, int ldm, int rows, int ncols, const void* x, void* out, const void* base_, double alpha,
                double beta) {
    SolveOp o;
    o.M = M;
    o.x = x;
    o.xidx = nullptr;
    o.oidx = nullptr;
    o.out = out;
    o.base = base_;
    o.alpha = alpha;
    o.beta = beta;
    o.rows = rows;
    o.ncols = ncols;
    o.ldm = ldm;
    o.lanes = solve_row_lanes(ncols, vw);
    return o;
  };
  std::vector<std::vector<int64_t>> launch_xidx;  // per launch: xidx offset per op (-1: none)
  // each pivot inverse is packed once (all m x m), read by both passes
  std::vector<std::vector<std::pair<const char*, int>>> pip(ell + 1);
  for (int kappa = 2; kappa <= ell; ++kappa) pip[kappa].assign(F.lv[kappa].nn, {nullptr, 0});
  auto pivot = [&](int kappa, int i) -> std::pair<const char*, int> {
    auto& e = pip[kappa][i];
    if (!e.first) {
      const NodeFactor& nf = F.lv[kappa].nf[i];
      const int m = nf.n + nf.r;
      e.first = (const char*)packed(nf.piinv, m, m, m, e.second);
    }
    return e;
  };
  auto emit = [&](std::vector<SolveOp>& v, std::vector<int64_t>& xo) {
    if (v.empty()) return;
    launches.push_back(std::move(v));
    launch_xidx.push_back(std::move(xo));
    v.clear();
    xo.clear();
  };
  // ---- forward substitution (upward), colors ascending
  for (int kappa = ell; kappa >= 2; --kappa) {
    const LevelFactor& LF = F.lv[kappa];
    for (const auto& grp : LF.order) {
      std::vector<SolveOp> l1, l2;
      std::vector<int64_t> x1, x2;
      for (int i : grp) {
        const NodeFactor& nf = LF.nf[i];
        const int n = nf.n, r = nf.r, m = n + r;
        if (m == 0) continue;
        const auto [Pi, ldp] = pivot(kappa, i);
        const int64_t ti = TB + toff[kappa][i];
        const int64_t xi = base[kappa] + xoff[kappa][i];
        // t = Pi^-1 [x_i; 0]: rows [0, n) to scratch, rows [n, m) to the R-row slot
        if (n) {
          l1.push_back(op(Pi, ldp, n, n, vp(xi), vp(ti), nullptr, 1.0, 0.0));
          x1.push_back(-1);
        }
        if (r) {
          l1.push_back(op(Pi + (size_t)esz * n * ldp, ldp, r, n, vp(xi), vp(rloc(kappa, i)), nullptr, 1.0, 0.0));
          x1.push_back(-1);
        }
        if (!n) continue;
        // neighbours: their current row variable -= L_q t[:n]
        for (size_t a = 0; a < nf.nb.size(); ++a) {
          const int q = nf.nb[a];
          const int mq = nf.lcol_rows[a];
          if (!mq) continue;
          int ldl = 0;
          const void* Lq = packed(nf.lcol[a], nf.lcol_ld[a], mq, n, ldl);
          const int64_t yq = nf.was_elim[a] ? rloc(kappa, q) : base[kappa] + xoff[kappa][q];
          l2.push_back(op(Lq, ldl, mq, n, vp(ti), vp(yq), vp(yq), -1.0, 1.0));
          x2.push_back(-1);
        }
      }
      emit(l1, x1);
      emit(l2, x2);
    }
  }
  // ---- top: y2 = D^-1 rhs (through the scratch, then back)
  if (F.ntop) {
    std::vector<SolveOp> l1, l2;
    std::vector<int64_t> x1, x2;
    int ldt = 0;
    const void* Dm = packed(F.top_inv, F.ntop, F.ntop, F.ntop, ldt);
    l1.push_back(op(Dm, ldt, F.ntop, F.ntop, vp(base[1]), vp(TB), nullptr, 1.0, 0.0));
    x1.push_back(-1);
    l2.push_back(op(nullptr, 4, F.ntop, 0, nullptr, vp(base[1]), vp(TB), 1.0, 1.0));
    x2.push_back(-1);
    emit(l1, x1);
    emit(l2, x2);
  }
  // ---- backward substitution (downward), colors descending
  for (int kappa = 2; kappa <= ell; ++kappa) {
    const LevelFactor& LF = F.lv[kappa];
    for (auto it = LF.order.rbegin(); it != LF.order.rend(); ++it) {
      std::vector<SolveOp> l1, l2;
      std::vector<int64_t> x1, x2;
      for (int i : *it) {
        const NodeFactor& nf = LF.nf[i];
        const int n = nf.n, r = nf.r, m = n + r;
        if (!n) continue;
        const int64_t ti = TB + toff[kappa][i];
        const int64_t xi = base[kappa] + xoff[kappa][i];
        // s = x_i - sum_q U_q v_q over the neighbours' current column variables
        int cols = 0;
        for (size_t a = 0; a < nf.nb.size(); ++a) cols += nf.urow_cols[a];
        const int ldu = pad4(std::max(cols, 1));
        void* U = P.mem.alloc_bytes((size_t)esz * n * ldu);
        const int64_t xo = (int64_t)xidx_all.size();
        int c0 = 0;
        for (size_t a = 0; a < nf.nb.size(); ++a) {
          const int q = nf.nb[a];
          const int mq = nf.urow_cols[a];
          if (!mq) continue;
          pk.push_back(PackDesc{nf.urow[a], (char*)U + (size_t)esz * c0, n, ldu, n, mq});
          const int64_t vq = nf.was_elim[a] ? rloc(kappa, q) : base[kappa] + xoff[kappa][q];
          for (int j = 0; j < mq; ++j) xidx_all.push_back((int32_t)(vq + j));
          c0 += mq;
        }
        l1.push_back(op(U, ldu, n, cols, P.V, vp(ti), vp(xi), -1.0, 1.0));
        x1.push_back(cols ? xo : -1);
        // x_i = Pi^-1[:n, :] [s; y_i]
        const auto [Pi, ldp] = pivot(kappa, i);
        const int64_t xo2 = (int64_t)xidx_all.size();
        for (int j = 0; j < n; ++j) xidx_all.push_back((int32_t)(ti + j));
        const int64_t yi = r ? rloc(kappa, i) : 0;
        for (int j = 0; j < r; ++j) xidx_all.push_back((int32_t)(yi + j));
        l2.push_back(op(Pi, ldp, n, m, P.V, vp(xi), nullptr, 1.0, 0.0));
        x2.push_back(xo2);
      }
      emit(l1, x1);
      emit(l2, x2);
    }
  }
  // ---- pack, upload, capture
  {
    DescStage st;
    st.stream = s;
    launch_pack(st, pk, P.pairs);
    CK(cudaStreamSynchronize(s));
  }
  std::vector<std::vector<int64_t>> no_oidx(launches.size());
  for (size_t li = 0; li < launches.size(); ++li) no_oidx[li].assign(launches[li].size(), -1);
  capture_solve_plan(P, launches, launch_xidx, no_oidx, xidx_all);
  P.stage_in = vp(base[ell]);
  std::vector<SolveOp> ops_all;
  for (auto& l : launches) ops_all.insert(ops_all.end(), l.begin(), l.end());
  F.stat("solve_launches", (double)P.prog.size());
  F.stat("solve_vector_len", (double)total);
  F.stat("bytes_solve", (double)P.mem.high);
  double mbytes = 0;  // coefficient bytes one application streams
  for (auto& o : ops_all) mbytes += (double)esz * o.rows * o.ncols;
  F.stat("solve_matrix_bytes", mbytes);
}

// in/out: tree-ordered device vectors of length N (may alias)
void run_solve_tree(const ifmm_fact& F, const double* in, double* out, cudaStream_t s) {
  const SolvePlan& P = F.plan;
  const int64_t N = F.t->N * kernel_dof(F.k);  // doubles per vector
  if (P.pairs)
    launch_pair_split(s, in, P.stage_in, N);
  else
    CK(cudaMemcpyAsync(P.stage_in, in, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  static const bool direct = [] {
    const char* e = getenv("IFMM_SOLVE_NOGRAPH");
    return e && e[0] == '1';
  }();
  if (direct) {  // the same program as individual launches, each timed when profiling
    for (auto& l : P.prog) {
      prof_batch_tag() = l.nops;
      cudaEvent_t pe = profiler().begin(KK_GEMV, s);
      launch_solve_ops(s, l.ops, l.warp_ptr, l.nops, l.nwarps, P.pairs);
      profiler().end(KK_GEMV, s, pe);
    }
    check_launch("k_solve_rows", (long)P.prog.size());
  } else {
    cudaEvent_t pe = profiler().begin(KK_SOLVE_GRAPH, s, (long)P.prog.size());
    CK(cudaGraphLaunch(P.graph, s));
    profiler().end(KK_SOLVE_GRAPH, s, pe);
    profiler().count(KK_ALL, (long)P.prog.size());
  }
  const void* res = P.stage_out ? P.stage_out : P.stage_in;
  if (P.pairs)
    launch_pair_join(s, res, out, N);
  else
    CK(cudaMemcpyAsync(out, res, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
}

static std::mutex g_tune_mutex;

// The float-pair matvec's tile for a tree: the autotuner's choice, remembered
// per device and point count for the life of the process, so that trees of a
// size already seen (a new tree per problem, as in a time loop) skip the
// timing runs (fifteen launches of the full product).
static int matvec_tile(ifmm_tree* tm, cudaStream_t s, const float* q, const double* in, double* out, int64_t N,
                       const ifmm_kernel* k, float2* part) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  if (tm->matvec_block) return tm->matvec_block;
  // IFMM_MATVEC_TILE (read when a tree first needs its tile) forces a kernel:
  // "sym", or "<threads>x<targets per thread>" (128x1, 256x1, 512x1, 128x2,
  // 256x2); for tests and experiments
  if (const char* e = getenv("IFMM_MATVEC_TILE")) {
    int code = 0, bs = 0, tpt = 0;
    if (std::string(e) == "sym" && part)
      code = 128 | 3 << 16;
    else if (sscanf(e, "%dx%d", &bs, &tpt) == 2 && (tpt == 1 || tpt == 2) &&
             (bs == 128 || bs == 256 || (bs == 512 && tpt == 1)))
      code = bs | tpt << 16;
    IFMM_REQUIRE(code, IFMM_EINVAL, std::string("IFMM_MATVEC_TILE not understood or not available: ") + e);
    tm->matvec_block = code;
    tm->matvec_block_v = {code & 0xffff, code >> 16};
    return code;
  }
  static std::map<std::pair<int, int64_t>, int> seen;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  auto it = seen.find({dev, N});
  const int code = it != seen.end()
                       ? it->second
                       : autotune_matvec_df(s, tm->d_pts_df, q, q + N, in, out, (int)N, k->scale, k->diag, part);
  seen[{dev, N}] = code;
  tm->matvec_block = code;
  tm->matvec_block_v = {code & 0xffff, code >> 16};
  return code;
}

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
  noalloc_prepare_device(device);
}

ifmm_tree::~ifmm_tree() {
  fmm_free(fmm);
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

// partial-sum buffer of the symmetric float-pair matvec, when it is at most
// 8 GiB (N up to about 300,000 points); NULL otherwise
static float2* sym_part(Vecs& V, int64_t N) {
  const size_t floats = matvec_sym_part_floats((int)N);
  if (floats * sizeof(float) > ((size_t)8 << 30)) return nullptr;
  return (float2*)V.get(floats / 2);
}

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
    const int dof = kernel_dof(f->k);
    const int64_t NP = f->t->N, N = NP * dof;  // points, doubles per vector
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
      launch_gather_perm(s, src, f->t->d_perm, a, (int)NP, dof);
      run_solve_tree(*f, a, a, s);
      if (dev) {
        launch_scatter_perm(s, a, f->t->d_perm, vc, (int)NP, dof);
      } else {
        launch_scatter_perm(s, a, f->t->d_perm, b, (int)NP, dof);
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
    IFMM_REQUIRE(k->wavenumber == 0.0 || k->arith == IFMM_ARITH_FP64, IFMM_EINVAL,
                 "the Helmholtz kernel takes the FP64 direct sum (arith IFMM_ARITH_FP64)");
    const_cast<ifmm_tree*>(t)->ensure_device();
    cudaStream_t s = (cudaStream_t)stream;
    const int dof = kernel_dof(*k);
    const int64_t NP = t->N, N = NP * dof;
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
    launch_gather_perm(s, src, t->d_perm, a, (int)NP, dof);
    if (k->arith == IFMM_ARITH_FMM) {
      FmmPlan* P = fmm_plan(*const_cast<ifmm_tree*>(t), k->order ? k->order : 4, k->scale, k->diag, s);
      fmm_apply(*t, *P, a, b, s);
    } else if (k->arith == IFMM_ARITH_DF) {
      float* q = (float*)V.get(N);
      launch_split_df(s, a, q, q + N, (int)N);
      ifmm_tree* tm = const_cast<ifmm_tree*>(t);
      float2* part = (!tm->matvec_block || (tm->matvec_block >> 16) == 3) ? sym_part(V, N) : nullptr;
      const int tile = tm->matvec_block ? tm->matvec_block : matvec_tile(tm, s, q, a, b, N, k, part);
      launch_matvec_df(s, t->d_pts_df, q, q + N, a, b, (int)N, k->scale, k->diag, tile, part);
    } else {
      launch_matvec(s, t->d_pts, (int)NP, a, b, *k);
    }
    if (dev) {
      launch_scatter_perm(s, b, t->d_perm, y, (int)NP, dof);
    } else {
      launch_scatter_perm(s, b, t->d_perm, c, (int)NP, dof);
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
    IFMM_REQUIRE(k->wavenumber == 0.0 || k->arith == IFMM_ARITH_FP64, IFMM_EINVAL,
                 "the Helmholtz kernel takes the FP64 direct sum (arith IFMM_ARITH_FP64)");
    IFMM_REQUIRE(!pre || kernel_dof(pre->k) == kernel_dof(*k), IFMM_EINVAL,
                 "preconditioner built for a real (complex) kernel used with a complex (real) one");
    const_cast<ifmm_tree*>(t)->ensure_device();
    cudaStream_t s = (cudaStream_t)stream;
    const int dof = kernel_dof(*k);
    const int64_t NP = t->N, N = NP * dof;  // points; doubles per vector (real form)
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
    launch_gather_perm(s, src, t->d_perm, bt, (int)NP, dof);
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
    // the symmetric matvec's partial sums, unless this tree took another kernel
    float2* sympart = nullptr;
    if (df_mv && (!t->matvec_block || (t->matvec_block >> 16) == 3)) sympart = sym_part(Vm, N);
    FmmPlan* fmm = k->arith == IFMM_ARITH_FMM
                       ? fmm_plan(*const_cast<ifmm_tree*>(t), k->order ? k->order : 4, k->scale, k->diag, s)
                       : nullptr;
    auto Amul = [&](const double* in, double* out) {
      if (fmm) {
        fmm_apply(*t, *fmm, in, out, s);
      } else if (df_mv) {
        launch_split_df(s, in, qdf, qdf + N, (int)N);
        ifmm_tree* tm = const_cast<ifmm_tree*>(t);
        const int tile = tm->matvec_block ? tm->matvec_block : matvec_tile(tm, s, qdf, in, out, N, k, sympart);
        launch_matvec_df(s, t->d_pts_df, qdf, qdf + N, in, out, (int)N, k->scale, k->diag, tile, sympart);
      } else {
        launch_matvec(s, t->d_pts, (int)NP, in, out, *k);
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
      launch_scatter_perm(s, xt, t->d_perm, x, (int)NP, dof);
    } else {
      launch_scatter_perm(s, xt, t->d_perm, tmp, (int)NP, dof);
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
