// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ifmm.h"

namespace ifmm {

// Thrown inside the library; converted to a status at the ABI boundary.
struct Error : std::runtime_error {
  ifmm_status code;
  Error(ifmm_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);
// loads the allocation-free matvec's module on device `dev` (noalloc.cu)
void noalloc_prepare_device(int dev);
struct FmmPlan;  // the FMM matvec's device structure of a tree (fmm.cpp)
void fmm_free(FmmPlan* p);

#define IFMM_REQUIRE(cond, code, msg)                 \
  do {                                                \
    if (!(cond)) throw ::ifmm::Error((code), (msg));  \
  } while (0)

// One level of the uniform octree (non-empty cells only), Sec. 2.1.
struct LevelLists {
  int kappa = 0, m = 0, n = 0;
  std::vector<int32_t> cells;  // 3 per node: ix iy iz
  std::vector<int64_t> lin;    // (iz*m + iy)*m + ix, ascending = node order
  std::vector<int32_t> parent;
  std::vector<int32_t> child_ptr, child;
  std::vector<int32_t> nbr_ptr, nbr;
  std::vector<int32_t> il_ptr, il;
  std::vector<int32_t> color, group_ptr, group;  // Algorithm 3 output
  int find(int64_t ix, int64_t iy, int64_t iz) const;
};

}  // namespace ifmm

struct ifmm_tree {
  int64_t N = 0;
  int depth = 0;
  double origin[3] = {0, 0, 0};
  double side = 0;
  std::vector<double> pts;       // tree order, N x 3 row-major
  std::vector<int32_t> perm;     // tree order -> caller index
  std::vector<int32_t> leaf_ptr; // points of leaf i: [leaf_ptr[i], leaf_ptr[i+1])
  std::vector<ifmm::LevelLists> lv;
  int sigma = 0;
  int tau = 2;  // levels below tau are colored one node per color
  // device copies
  double* d_pts = nullptr;    // SoA: x[N], y[N], z[N] in tree order
  int32_t* d_perm = nullptr;  // tree order -> caller index
  float* d_pts_df = nullptr;  // points as float pairs: xh xl yh yl zh zl [N] each
  int matvec_block = 0;       // autotuned tile of the float-pair matvec, BS | TPT << 16 (0: not yet)
  std::vector<int32_t> matvec_block_v{0, 0};
  int device = -1;
  ifmm::FmmPlan* fmm = nullptr;  // cached by the first FMM matvec
  void ensure_device();
  ~ifmm_tree();
};
