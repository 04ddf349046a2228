// The factor handle: device block pool plus the host-side plan of the solve.
#pragma once

#include <array>
#include <string>
#include <vector>

#include "common.h"
#include "runtime.h"

namespace ifmm {

// What the solve needs of one eliminated node (Algorithm 2 on the extended system).
struct NodeFactor {
  const double* piinv = nullptr;  // (n + r) x (n + r), ld n + r
  int n = 0, r = 0;
  std::vector<int> nb;         // neighbours at elimination time
  std::vector<char> was_elim;  // neighbour eliminated earlier (its variable is y, not x)
  std::vector<const double*> lcol;  // row-var(q) x x_i   (rows m_q, ld lcol_ld)
  std::vector<int> lcol_ld, lcol_rows;
  std::vector<const double*> urow;  // E_x,i x col-var(q) (cols m_q, ld n)
  std::vector<int> urow_cols;
};

struct LevelFactor {
  int kappa = 0, nn = 0;
  std::vector<int> n, r;                // x dimension, final rank
  std::vector<std::vector<int>> order;  // colors in elimination order
  std::vector<NodeFactor> nf;
};

// The solve as a fixed program of SolveOp launches over one vector buffer V:
// the top vector, every node vector of levels 2..ell, then per-node scratch.
// Elements are FP64, or float pairs in the reduced-precision modes (8 bytes
// either way).  The blocks the solve reads are packed row-major in `mem`.
struct SolveLaunch {
  const SolveOp* ops;
  const int* warp_ptr;  // prefix sums of the warps of each op
  int nops, nwarps;
};

struct SolvePlan {
  void* V = nullptr;
  int64_t xlen = 0, vlen = 0;
  void* stage_in = nullptr;   // tree-ordered input vector (level ell's segment of V)
  void* stage_out = nullptr;  // tree-ordered output vector (nullptr: stage_in)
  bool pairs = false;
  std::vector<SolveLaunch> prog;
  cudaGraphExec_t graph = nullptr;
  cudaGraph_t graph_def = nullptr;
  DeviceArena mem;
};

}  // namespace ifmm

struct ifmm_fact {
  const ifmm_tree* t = nullptr;
  ifmm_kernel k{};
  ifmm_opts o{};
  int p = 0, rc = 0;
  std::vector<ifmm::LevelFactor> lv;
  ifmm::DeviceArena persist;
  double* top_inv = nullptr;
  int ntop = 0;
  std::vector<int> top_off;
  ifmm::SolvePlan plan;
  std::vector<std::array<int, 4>> rank_log;
  std::vector<float> event_feat;  // rank-predictor inputs of every event, in rank_log order
  std::vector<std::pair<std::string, double>> stats;
  void stat(const std::string& name, double v) {
    for (auto& s : stats)
      if (s.first == name) {
        s.second = v;
        return;
      }
    stats.push_back({name, v});
  }
  void stat_add(const std::string& name, double v) {
    for (auto& s : stats)
      if (s.first == name) {
        s.second += v;
        return;
      }
    stats.push_back({name, v});
  }
  ~ifmm_fact();
};

namespace ifmm {
void build_solve_plan(ifmm_fact& F, cudaStream_t s);
void capture_solve_plan(SolvePlan& P, const std::vector<std::vector<SolveOp>>& launches,
                        const std::vector<std::vector<int64_t>>& xoff, const std::vector<std::vector<int64_t>>& ooff,
                        const std::vector<int32_t>& idx_all);
int solve_row_lanes(int ncols, int v);
FmmPlan* fmm_plan(ifmm_tree& T, int order, double scale, double diag, cudaStream_t s);
void fmm_apply(const ifmm_tree& T, FmmPlan& P, const double* x, double* y, cudaStream_t s);
void run_solve(const ifmm_fact& F, cudaStream_t s);
}  // namespace ifmm
