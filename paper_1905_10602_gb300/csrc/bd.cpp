// Block-diagonal preconditioner BD / BDbot l_BD (Sec. 4.3, applied as in
// Algorithm 5): for every non-empty cell of level l_BD, the self block of A over
// the cell's points, inverted (FP64 Gauss-Jordan with partial pivoting, the
// kernels of the IFMM pivots); applying it solves every block independently.
// The paper's BD takes the leaf level of the FMM tree; BDbot l_BD a coarser
// level, whose wider blocks approximate A^-1 better at a higher set-up cost.
//
// The result is an ifmm_fact whose solve program is the block-diagonal
// application (one launch of the solve's row operations gathering each cell's
// entries, one scattering them back), so ifmm_solve and bem_gmres take it as
// they take an IFMM factor.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "fact.h"
#include "ifmm_kernels.h"

namespace ifmm {

static void build_bd(ifmm_fact& F, int level, cudaStream_t s) {
  const ifmm_tree& T = *F.t;
  const int ell = T.depth;
  const LevelLists& L = T.lv[level];
  const int nc = L.n;
  // the leaves under every cell of the level, in leaf order
  std::vector<std::vector<int>> leaves(nc);
  for (int i = 0; i < T.lv[ell].n; ++i) {  // walk every leaf up to the level
    int a = i;
    for (int kappa = ell; kappa > level; --kappa) a = T.lv[kappa].parent[a];
    leaves[a].push_back(i);
  }
  std::vector<int> off(nc + 1, 0);
  for (int c = 0; c < nc; ++c) {
    int n = 0;
    for (int l : leaves[c]) n += T.leaf_ptr[l + 1] - T.leaf_ptr[l];
    off[c + 1] = off[c] + n;
  }
  const int64_t N = T.N;
  IFMM_REQUIRE(off[nc] == N, IFMM_EINVAL, "internal: cells do not cover the points");
  // every cell's points (tree order) and its self block (column-major, ld n)
  std::vector<int32_t> idx;
  for (int c = 0; c < nc; ++c)
    for (int l : leaves[c])
      for (int p = T.leaf_ptr[l]; p < T.leaf_ptr[l + 1]; ++p) idx.push_back(p);
  DeviceArena blocks;
  DescStage st;
  st.stream = s;
  std::vector<double*> blk(nc, nullptr);
  std::vector<BdBlockDesc> fill;
  std::vector<InvDesc> inv;
  int* d_info = (int*)blocks.alloc_bytes(sizeof(int) * std::max(nc, 1));
  int* d_idx = (int*)blocks.alloc_bytes(sizeof(int) * std::max<size_t>(1, idx.size()));
  CK(cudaMemsetAsync(d_info, 0, sizeof(int) * std::max(nc, 1), s));
  CK(cudaMemcpyAsync(d_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
  double flops = 0;
  for (int c = 0; c < nc; ++c) {
    const int n = off[c + 1] - off[c];
    blk[c] = blocks.alloc((size_t)std::max(1, n) * std::max(1, n));
    if (!n) continue;
    fill.push_back(BdBlockDesc{blk[c], d_idx + off[c], n, 0});
    inv.push_back(InvDesc{blk[c], n, n, d_info + c, 0});
    flops += 2.0 * std::pow((double)n, 3);
  }
  launch_bd_fill(st, fill, T.d_pts, (int)N, F.k.scale, F.k.diag);
  launch_inv(st, inv);
  std::vector<int> info(std::max(nc, 1));
  CK(cudaMemcpyAsync(info.data(), d_info, sizeof(int) * std::max(nc, 1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  st.reset();
  for (int c = 0; c < nc; ++c)
    IFMM_REQUIRE(info[c] == 0, IFMM_ESINGULAR, "singular diagonal block at level " + std::to_string(level));
  // the program: V = [input (tree order) | output (tree order)]
  SolvePlan& P = F.plan;
  P.pairs = false;
  P.xlen = N;
  P.vlen = 2 * N;
  P.V = P.mem.alloc_bytes(8 * (size_t)P.vlen);
  double* V = (double*)P.V;
  std::vector<PackDesc> pk;
  std::vector<std::vector<SolveOp>> launches(1);
  std::vector<std::vector<int64_t>> xo(1), oo(1);
  for (int c = 0; c < nc; ++c) {
    const int n = off[c + 1] - off[c];
    if (!n) continue;
    const int ldm = (n + 3) & ~3;
    double* M = P.mem.alloc((size_t)n * ldm);
    pk.push_back(PackDesc{blk[c], M, n, ldm, n, n});
    const int64_t first = off[c];
    SolveOp o;
    o.M = M;
    o.x = V;
    o.xidx = nullptr;
    o.oidx = nullptr;
    o.out = V + N;
    o.base = nullptr;
    o.alpha = 1.0;
    o.beta = 0.0;
    o.rows = n;
    o.ncols = n;
    o.ldm = ldm;
    o.lanes = solve_row_lanes(n, 2);
    launches[0].push_back(o);
    xo[0].push_back(first);  // v_c = A_cc^-1 r_c, gathered from and scattered to the
    oo[0].push_back(first);  // cell's points in tree order
  }
  launch_pack(st, pk, false);
  CK(cudaStreamSynchronize(s));
  st.reset();
  blocks.release();
  capture_solve_plan(P, launches, xo, oo, idx);
  P.stage_in = V;
  P.stage_out = V + N;
  double mbytes = 0;
  for (auto& o : launches[0]) mbytes += 8.0 * o.rows * o.ncols;
  F.stat("bd_level", level);
  F.stat("bd_blocks", nc);
  F.stat("bd_max_block", [&] {
    int m = 0;
    for (int c = 0; c < nc; ++c) m = std::max(m, off[c + 1] - off[c]);
    return (double)m;
  }());
  F.stat("flops_inv", flops);
  F.stat("solve_launches", (double)P.prog.size());
  F.stat("bytes_solve", (double)P.mem.high);
  F.stat("solve_matrix_bytes", mbytes);
}

}  // namespace ifmm

using namespace ifmm;

extern "C" ifmm_status ifmm_bd_factor(const ifmm_tree* t, const ifmm_kernel* k, int level, void* stream,
                                      ifmm_fact** out) {
  if (out) *out = nullptr;
  ifmm_fact* F = nullptr;
  try {
    IFMM_REQUIRE(t && k && out, IFMM_EINVAL, "NULL argument");
    IFMM_REQUIRE(level >= 0 && level <= t->depth, IFMM_EINVAL, "level must be in [0, depth]");
    IFMM_REQUIRE(k->wavenumber == 0.0, IFMM_EINVAL, "the block-diagonal preconditioner is Laplace only");
    const_cast<ifmm_tree*>(t)->ensure_device();
    F = new ifmm_fact();
    F->t = t;
    F->k = *k;
    F->o = ifmm_opts{};
    F->o.precision = IFMM_PREC_FP64;
    const auto t0 = std::chrono::steady_clock::now();
    build_bd(*F, level, (cudaStream_t)stream);
    F->stat("time_factor", std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    *out = F;
    return IFMM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    delete F;
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    delete F;
    return IFMM_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    delete F;
    return IFMM_ECUDA;
  }
}
