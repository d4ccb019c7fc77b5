// Dense kernels of the per-mode update: Gram products, the r x r SPD factorisation
// (Cholesky, pseudo-inverse fallback), leverage scores of factor rows with the
// fixed-point sampling weights, and the row-wise normal-equation solve.
#pragma once

#include "cpa_internal.cuh"

namespace cpa {

// Result of factoring an r x r symmetric positive semidefinite matrix G.
// kind 0: F holds the inverse of the lower Cholesky factor of P^T (S G S) P
//         (row-major, lower triangular), its leading rank x rank block only when
//         pivoting found G singular; P is the permutation perm, S = diag(scale).
// kind 1: F holds the pseudo-inverse of S G S.
// kind 2: F holds the inverse of S G S.
// With normalize = 1, scale_c = 1/sqrt(G_cc) (0 for a zero column) and lambda_c =
// sqrt(G_cc); otherwise scale = 1, lambda = sqrt(G_cc).
struct SmallFactor {
  double F[kMaxRank * kMaxRank];
  double scale[kMaxRank];
  double lambda[kMaxRank];
  int perm[kMaxRank];
  int kind;
  int rank;
  int pad[2];
};

// Per-mode fixed-point distribution summary (device).
struct DistInfo {
  uint64_t T;     // sum of q
  uint64_t maxq;  // largest q
  int64_t nnzq;   // number of q > 0
  int64_t pad;
};

// G = A^T A for a row-major n x r matrix of FT (float or double): FP64 products of
// FP64 rows; FP32 rows summed per 64-row tile in float-pair arithmetic (2^-44
// relative); tiles added in FP64.  The blocks' partial sums are added in block order
// (S: a workspace of block_sums_bytes(max_blocks, r (r + 1) / 2) bytes with its
// ticket zeroed), so the result is reproducible bit for bit.
// lda: row stride of A in elements (0: r).
// status (device, may be null): a run's status word; with it, FP32 factors of many rows
// take the tensor-core kernel (lev_tc.cu), which records a timed-out wait there.
template <class FT>
int gram_rows(const FT* A, int64_t n, int r, double* G, const BlockSums& S, cudaStream_t st, int lda = 0,
              int* status = nullptr);
// Width of the block sums of gram_rows for rank r.
inline int gram_sums_width(int r) { return r * (r + 1) / 2; }

// Factor G (see SmallFactor).  rel_tol: a Cholesky pivot must exceed rel_tol times
// the largest diagonal entry.  pivot = 0: plain Cholesky; if a pivot fails, the
// pseudo-inverse (eigenvalues above rel_tol * largest) is used.  pivot = 1:
// diagonal pivoting (largest remaining diagonal first) stops at the numerical rank,
// which is exact for leverage scores of rank-deficient matrices.  Either way a
// singular G OR-s `warn_bit` into *warn.
// zero_info (may be null) has its maxq/nnzq cleared for the lev_rows that follows.
int factor_spd(const double* G, int r, int normalize, int pivot, double rel_tol,
               SmallFactor* out, int* warn, int warn_bit, cudaStream_t st,
               DistInfo* zero_info = nullptr);

// For every row a_i of A a sampling score s_i (sum over rows r):
//   dist = CPA_DIST_LEVERAGE: s_i = || L^{-1} S a_i ||^2 (kind 0) or a_i^T S F S a_i
//     (kind 1), the leverage score;
//   dist = CPA_DIST_UNIFORM: s_i = r / n;
//   dist = CPA_DIST_LENGTH_SQUARED: s_i = r ||b_i||^2 / ||B||_F^2 with B = A with its
//     columns divided by lambda (zero columns dropped) if A_out is non-null (the
//     factor the next Khatri-Rao product uses), else B = A;
// q_i = round-half-even(2^62 s_i / r) written to q (if non-null), s_i to lev (if
// non-null), DistInfo maxq/nnzq accumulated (zeroed by the caller); rows divided by
// lambda (columns with lambda = 0 untouched) and written to A_out if non-null (may be A).
// lda: row stride of A in elements (0: r; A_out always has stride r, and may be A
// only when lda = r).
template <class FT>
int lev_rows(const FT* A, int64_t n, int r, const SmallFactor* f, double* lev,
             uint64_t* q, DistInfo* info, FT* A_out, cudaStream_t st, int dist = CPA_DIST_LEVERAGE,
             int lda = 0, int* status = nullptr);

// The fast leverage kernels for FP32 factors, on by default for the mixed-precision
// refresh of factors with >= 65,536 rows (about FP32 accuracy): the Gram on the FP32
// pipe with bulk-copy streaming (gram_stream.cu, r <= kGramStreamMaxRank) and the row
// forms as tcgen05 kind::tf32 products with the hi/lo split (lev_tc.cu).
// CPA_LEV_FLOAT_PAIR=1 selects the float-pair kernels (2^-44, the FP64 path's) instead;
// CPA_GRAM_TC=1 takes the tensor-core Gram of lev_tc.cu.
bool lev_tensor_cores();
bool gram_tensor_cores();
constexpr int kGramStreamMaxRank = 32;
int gram_rows_stream(const float* A, int64_t n, int r, int lda, double* G, const BlockSums& S, int* status,
                     cudaStream_t st);
// The FP64 refresh's Gram of many rows, in float pairs on the FP32 pipe with the same
// streaming (about 2^-44 relative), r <= kGramStreamFP64MaxRank; CPA_GRAM_STREAM_FP64=0
// takes the one-pair-per-thread float-pair kernel instead.
bool gram_stream_fp64();
constexpr int kGramStreamFP64MaxRank = 28;
int gram_rows_stream(const double* A, int64_t n, int r, int lda, double* G, const BlockSums& S, int* status,
                     cudaStream_t st);


// The rows can be streamed by the bulk copies of the tensor-core kernels: a 16-byte
// aligned base (row strides lda >= r; lda 0 means r).
bool tc_rows_ok(const float* A, int r, int lda);
int gram_rows_tc(const float* A, int64_t n, int r, int lda, double* G, const BlockSums& S, int* status,
                 cudaStream_t st);
int lev_rows_tc(const float* A, int64_t n, int r, int lda, const SmallFactor* f, double* lev, uint64_t* q,
                DistInfo* info, float* A_out, int* status, cudaStream_t st);

// The relative pivot cut of the leverage factorisation (factor_spd's rel_tol) for the
// Gram that gram_rows computes for these arguments: 1e-12 for the FP64 and float-pair
// Grams (2^-44 relative or better); 2^-20 for the fast FP32 kernels, whose Gram carries
// FP32 rounding (products summed in FP32 over 128 rows): a pivot below that is noise,
// and keeping it would put spurious leverage on the rows along its direction.
constexpr double kLevPivotTolFP32 = 1.0 / (1 << 20);
constexpr int64_t kManyRows = 1 << 16;  // from here on the per-row kernels take one thread per row
template <class FT>
double lev_pivot_tol(const FT* A, int64_t n, int r, int lda, const int* status) {
  if constexpr (sizeof(FT) == 4) {
    if (n >= kManyRows && status && lev_tensor_cores() && tc_rows_ok(reinterpret_cast<const float*>(A), r, lda))
      return kLevPivotTolFP32;
  }
  return 1e-12;
}

// A = M G^{-1} row by row with the factor of G (kind 0: two triangular solves;
// kind 1: A = M F).
// zero_gram (may be null): an r x r FP64 matrix cleared for the Gram that follows.
template <class FT>
int solve_rows(const FT* M, int64_t n, int r, const SmallFactor* f, FT* A, cudaStream_t st,
               double* zero_gram = nullptr);

// A(:, c) /= lambda_c for lambda_c > 0.
template <class FT>
int scale_columns(FT* A, int64_t n, int r, const double* lambda, cudaStream_t st);

// C = inclusive prefix sum of q (in place allowed); info->T = total; if p is
// non-null, p[i] = q_i / T (IEEE division), the per-row sampling probabilities.
int cdf_from_q(uint64_t* q, uint64_t* C, int64_t n, DistInfo* info, double* p, void* scan_scratch,
               cudaStream_t st);

inline unsigned grid_cap(int64_t blocks, int per_sm = 8) {
  const int64_t cap = (int64_t)num_sms() * per_sm;
  if (blocks < 1) blocks = 1;
  return (unsigned)(blocks < cap ? blocks : cap);
}

}  // namespace cpa
