// Host-callable launchers of the IFMM-specific kernels (defined in runtime.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "descs.h"
#include "runtime.h"

namespace ifmm {

// Near-field block between point ranges [i0, i0+ni) and [j0, j0+nj) (tree order).
struct P2pDesc {
  double* dst;
  int i0, ni, j0, nj, ld, same;
};

// Leaf interpolation matrix of points [p0, p0+n) in a cell (centre, half-width).
struct InterpDesc {
  double* dst;
  double cx, cy, cz, h;
  int p0, n, ld, pad;
};

// entries per point: 2 (real and imaginary part) for the Helmholtz kernel, else 1
inline int kernel_dof(const ifmm_kernel& k) { return k.wavenumber != 0.0 ? 2 : 1; }
void launch_p2p(DescStage& st, const std::vector<P2pDesc>& v, const double* pts, int N, const ifmm_kernel& k);
// Self block of A over the points idx[0..n) (tree order), column-major with ld n.
struct BdBlockDesc {
  double* dst;
  const int* idx;
  int n, pad;
};
void launch_bd_fill(DescStage& st, const std::vector<BdBlockDesc>& v, const double* pts, int N, double scale,
                    double diag);
void launch_interp(DescStage& st, const std::vector<InterpDesc>& v, const double* pts, int N, int p, int dof);
void launch_m2l_table(cudaStream_t s, double* out, int p, double h, const ifmm_kernel& k);
void launch_m2m_table(cudaStream_t s, double* out, int p, int dof);
void launch_matvec(cudaStream_t s, const double* pts, int N, const double* x, double* y, const ifmm_kernel& k);
void launch_split_df(cudaStream_t s, const double* in, float* hi, float* lo, int n);
// part: the symmetric kernel's partial sums (matvec_sym_part_floats(N) floats,
// as float2), or NULL where none was allocated (the symmetric candidate is then
// not taken)
void launch_matvec_df(cudaStream_t s, const float* pts_df, const float* qh, const float* ql, const double* x, double* y,
                      int N, double scale, double diag, int bs, float2* part);
int autotune_matvec_df(cudaStream_t s, const float* pts_df, const float* qh, const float* ql, const double* x,
                       double* y, int N, double scale, double diag, float2* part);
size_t matvec_sym_part_floats(int n);
void launch_gram_sum(DescStage& st, const std::vector<double*>& dst, const std::vector<const double*>& terms,
                     const std::vector<int>& first, int r);
void launch_chol(DescStage& st, const std::vector<double*>& mats, int r, double delta);
void launch_gather_perm(cudaStream_t s, const double* src, const int* perm, double* dst, int n, int dof = 1);
void launch_scatter_perm(cudaStream_t s, const double* src, const int* perm, double* dst, int n, int dof = 1);
void big_inverse(cudaStream_t s, double* A, int ld, int n, int* d_work_int, double* d_work, int* d_info);
// phase-B basis changes of the touched IL entries `list` (every rank <= md <= 64)
void launch_il_transform(DescStage& st, const std::vector<int>& list, const IlTables& t, int md, int prec);
// level-start M2L blocks T'_a K T_b of the entries grouped by offset (rc <= 64)
void launch_m2l_init(DescStage& st, const std::vector<M2lChunk>& chunks, const M2lTables& t, int prec);
// recompression weight stacks gathered on the device from the IL tables
void launch_zgather(DescStage& st, const std::vector<ZGatherDesc>& v, const ZTables& t);
// Schur-complement blocks of the eliminated nodes added into their near blocks
void launch_schur_scatter(DescStage& st, const std::vector<ScatterDesc>& v, const ScatterTables& t, int maxdeg);
void launch_copy_dev(cudaStream_t s, const CopyDesc* d, int n);
// the solve's row operations (pairs: float-pair vectors and FP32 matrices)
void launch_solve_ops(cudaStream_t s, const SolveOp* ops, const int* warp_ptr, int nops, int nwarps, bool pairs);
// column-major FP64 blocks -> row-major FP64 / FP32 copies
void launch_pack(DescStage& st, const std::vector<PackDesc>& v, bool fp32);
// FP64 <-> float pairs (hi = nearest float, lo = nearest float of the rest)
void launch_pair_split(cudaStream_t s, const double* in, void* out, int64_t n);
void launch_pair_join(cudaStream_t s, const void* in, double* out, int64_t n);
// FMM matvec stages (runtime.cu)
void launch_fmm_p2m(cudaStream_t s, const double* S, const long* soff, const int* leaf_ptr, const double* x, double* M,
                    int nleaf, int rc);
void launch_fmm_m2m(cudaStream_t s, const int* child_ptr, const int* child, const int* ccells, const double* m2m,
                    const double* Mc, double* Mp, int nparent, int rc);
void launch_fmm_m2l(cudaStream_t s, const int* il_ptr, const int* il, const int* cells, const double* tab,
                    const double* M, double* L, int n, int rc);
void launch_fmm_l2l(cudaStream_t s, const int* parent, const int* cells, const double* m2m, const double* Lp,
                    double* Lc, int n, int rc);
void launch_fmm_l2p(cudaStream_t s, const double* S, const long* soff, const int* leaf_ptr, const int* nbr_ptr,
                    const int* nbr, const double* L, const double* pts, int N, const double* x, double* y, int nleaf,
                    int rc, double scale, double diag);
const char* last_error();

}  // namespace ifmm
