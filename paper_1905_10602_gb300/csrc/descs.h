// Launch descriptors of the batched dense kernels (plain structs shared by
// host and device code).
#pragma once

namespace ifmm {

// dst = alpha * op(src) + beta * dst ; src == nullptr means op(src) = 0.
// beta == 0 never reads dst.
struct CopyDesc {
  const double* src;
  double* dst;
  int lds, ldd, rows, cols;  // rows x cols of dst
  double alpha, beta;
  int trans;  // op(src) = src^T (src is cols x rows)
  int pad;
};

// C = alpha * op(A) * op(B) + beta * C, C is m x n, inner dimension k.
struct GemmDesc {
  const double* A;
  const double* B;
  double* C;
  int lda, ldb, ldc, m, n, k;
  int ta, tb;
  double alpha, beta;
};

// In-place inverse of the n x n matrix A; info[0] = 0 on success, k+1 if the
// k-th pivot was zero.
struct InvDesc {
  double* A;
  int ld, n;
  int* info;
  int pad;
};

// Householder QR of the m x n matrix A in place; on exit the upper triangle of
// the leading min(m,n) x n block holds R and everything below it is zero.
struct QrDesc {
  double* A;
  int ld, m, n;
};

// y = alpha * op(A) x + beta * y ; A is m x n (op(A) is n x m when trans).
struct GemvDesc {
  const double* A;
  const double* x;
  double* y;
  int lda, m, n, trans;
  double alpha, beta;
};

// One operation of the IFMM solve (Algorithm 2): for r in [0, rows)
//   out[o(r)] = beta * base[o(r)] + alpha * sum_{c < ncols} M[r * ldm + c] * v(c),
// v(c) = x[c] (xidx == nullptr) or x[xidx[c]], o(r) = r (oidx == nullptr) or
// oidx[r].  M is row-major with ldm a
// multiple of 4 and 16-byte aligned rows: FP64, or FP32 in the reduced-precision
// modes.  The vectors are FP64, or float pairs (hi, lo) in the reduced-precision
// modes, where alpha is +-1 and beta 0 or 1.  lanes (a power of two <= 32) lanes
// share one row.
struct SolveOp {
  const void* M;
  const void* x;
  const int* xidx;
  const int* oidx;
  void* out;
  const void* base;
  double alpha, beta;
  int rows, ncols, ldm, lanes;
};

// dst (row-major, ldd) = src (rows x cols, column-major, lds), as FP64 or FP32.
struct PackDesc {
  const double* src;
  void* dst;
  int lds, ldd, rows, cols;
};

// Householder QR with column pivoting of the m x n matrix A, stopped at the
// first step whose largest remaining column norm is <= tau_rel times the
// largest initial column norm.  On exit the leading kout rows of A hold R (in
// pivoted column order, zero below the diagonal), jpvt[pos] is the original
// index of pivoted column pos, and *kout the number of steps taken.
struct QrcpDesc {
  double* A;
  int ld, m, n;
  double tau_rel;
  int* jpvt;
  int* kout;
  int kcap;      // > 0: also stop after kcap steps (predicted rank + margin)
  int pad;
  double* tail;  // out (may be NULL): largest remaining column norm / largest
                 // initial column norm when stopped by kcap, else 0
  int rb, rs;    // rb > 0: row i of the logical matrix is row (i / rb) * rs + i % rb
                 // of A (stacked rb-row blocks rs rows apart); rb = 0: row i
};

// Right singular vectors of Y from its truncated pivoted QR (Y P ~ Q R_k):
// one-sided Jacobi on B = P R_k^T (n x k); the rotated, normalised columns of B
// are the right singular vectors, their norms the singular values.  V (n x n,
// ldv): first k columns valid, the rest zero; sig (n) likewise, descending.
// work: n x n doubles used when B does not fit in shared memory.
struct SvdRtDesc {
  const double* A;
  int ld, n;
  const int* jpvt;
  const int* kin;
  double* V;
  int ldv, pad;
  double* sig;
  double* work;
};

// Interaction-list blocks of one level on the device, and the basis changes of
// one color (the interaction-list updates of Algorithm 1 that Sec. 3.3 serializes
// for sigma = 3, done as one pass after the color's eliminations).  IL entry e is the
// block M2L_ab, a = il_row[e], b = il[e], stored at far[e] with ld capr[a];
// rbefore[x] is node x's rank before the color, newk[x] its new rank (-1: not
// re-based), T[x] (rbefore x newk, ld rbefore) and Tp[x] (newk x rbefore, ld
// newk) its transforms when re-based.
struct IlTables {
  const int* il_row;
  const int* il;
  double* const* far;
  const int* capr;
  const int* rbefore;
  const int* newk;
  const double* const* T;
  const double* const* Tp;
};

// Level start (every node re-based before its level's eliminations, Sec. 2.3):
// every interaction-list block of the level in the
// new bases, M2L_ab = T'_a K(c_a - c_b) T_b, with K the translation table
// (343 offsets of rc x rc, column-major).  The entries (positions in the IL
// CSR) are grouped by offset; chunk c covers ent[first, first + count), all
// with offset `off`.  k[x]: new rank of node x; T[x] (rc x k[x], ld rc) and
// Tp[x] (k[x] x rc, ld k[x]) its transforms.
struct M2lChunk {
  int off, first, count, pad;
};
struct M2lTables {
  const int* ent;
  const int* il_row;
  const int* il;
  double* const* far;
  const int* capr;
  const int* k;
  const double* const* T;
  const double* const* Tp;
  const double* tab;
  int rc, pad;
};

// Weight stack Z of one side of a recompression event of node q (the far-field
// operators the basis must keep representing, Sec. 2.3, Algorithm 1): for l in IL_q with a nonzero rank, in IL order, the block M2L_lq
// (side 0) or M2L_ql^T (side 1), r_l rows each; then, when the level has a
// parent (tail != 0), M2M_q (side 0) or L2L_q^T (side 1), rc rows.  Z has ld ldz.
struct ZGatherDesc {
  double* Z;
  int ldz, q, side, pad;
};
struct ZTables {
  const int* il_ptr;
  const int* il;
  const int* il_T;
  double* const* far;
  const int* capr;
  const int* r;
  double* const* M2M;
  double* const* L2L;
  int rc, tail;
};

// Schur-complement scatter of one eliminated node i (Algorithm 1's updates of
// the neighbours' P2P / M2P / P2L / M2L blocks): F (M x M, ld M) holds -L Pi^-1 U over i's neighbours in CSR
// order, each neighbour q owning dim(q) rows and columns (dim = r if q is
// eliminated, else n); every block (q, q2) with q2 = q or q2 a neighbour of q
// is added to the current near block of stage elim[q] + elim[q2] (ld n[q]).
struct ScatterDesc {
  const double* F;
  int M, i;
};
struct ScatterTables {
  const int* nbr_ptr;
  const int* nbr;
  const int* slot_ptr;
  const int* n;
  const int* r;
  const unsigned char* elim;
  double* const* nb0;
  double* const* nb1;
  double* const* nb2;
};

// Random sketch matrix (m x s, ld m) of +-1 entries from a counter stream.
struct SketchDesc {
  double* omega;
  int m, s;
  unsigned long long seed;
};

// out[0] = Frobenius norm of an m x n block.
struct FrobDesc {
  const double* A;
  int ld, m, n;
  double* out;
};

}  // namespace ifmm
