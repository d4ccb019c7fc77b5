// Exact fit of Eq. 5.1 and the estimated fit of Section 5.4 on the GPU.
#pragma once

#include "mttkrp.cuh"

namespace cpa {

size_t fit_buffers_bytes(int D, int r);
// Enqueue the fit of [[lambda; A_1..A_D]] against X; result in *fit_dev (device).
// scratch: fit_buffers_bytes(D, r) bytes of device memory; S: block-ordered sums of
// width >= gram_sums_width(r) (the Grams and the inner product <X, M>, so the fit is
// the same bit for bit at every run).
template <class FT>
// terms (device, may be null): ||X||^2, <X, M>, ||M||^2 (Eq. 5.1) beside the fit.
int fit_enqueue(const cpa_index* X, const FactorPtrs& F, const double* lambda, int r, double* scratch,
                const BlockSums& S, double* fit_dev, cudaStream_t st, double* terms = nullptr);

// Stratified element sample of the estimated fit (Section 5.4), drawn once and kept
// on the device: coords (D rows of int32, row m at coords + m * stride), xs (values, the
// s_nz nonzero samples first, zeros after), phi = (nnz / s_nz, (prod n - nnz) / s_z).
struct FitSample {
  int32_t* coords = nullptr;
  double* xs = nullptr;
  double* partial = nullptr;  // per-block partial sums of the estimate
  int64_t s_fit = 0, s_nz = 0, s_z = 0, attempts = 0;
  int64_t stride = 0;  // row stride of coords
  double phi[2] = {0.0, 0.0};
  double alpha = 0.0;
  uint64_t seed = 0;
  int reject_cap = 0;
  void release();
  ~FitSample() { release(); }
};

// Draws the sample into *S (allocating its buffers):
//  - nonzero slot j < s_nz = ceil(alpha s_fit): word 0 of Philox counter
//    (j, 0, kDomainFit, 0), key (seed, 0), scaled to a position p = floor(u nnz / 2^64)
//    in mode 0's fibre index, whose order is ascending linear index of Eq. 2.2 (the
//    index is sorted by (packed key of modes 1.., i_0));
//  - zero slot j < s_z = s_fit - s_nz (0 if the tensor has no zero cell), attempt a:
//    i_m = floor(u_m n_m / 2^64), u_m word m % 4 of counter (j, a, kDomainFit | 1 |
//    (m / 4) << 16, 0); rejected while (i_0..i_{D-1}) is a nonzero (probe of mode 0's
//    index, then a bisection of i_0 in the fibre); CPA_ERR_REJECT_LIMIT past reject_cap.
// Synchronises the stream (the counts and the status are read back).
int fit_sample_draw(const cpa_index* X, int64_t s_fit, double alpha, uint64_t seed, int reject_cap,
                    FitSample* S, cudaStream_t st);

// Reorders the sample within each stratum by the coordinate of the largest mode, so
// that the evaluation reads that factor's rows in ascending order (the estimate is a
// sum: its value does not depend on the order).  Synchronises the stream.
int fit_sample_sort(const cpa_index* X, FitSample* S, cudaStream_t st);

// Enqueues F_hat = sum_j phi_j (m_j - x_j)^2 over the sample and *fit_dev =
// 1 - sqrt(F_hat) / ||X|| (fit_dev[1] = F_hat).  Deterministic for a given grid.
// fold_scratch (FP64, may be null): min_m n_m x r doubles the FP64 kernel may use for
// the factor with lambda folded into its rows.
template <class FT>
int fit_estimate_enqueue(const cpa_index* X, const FitSample& S, const FactorPtrs& F, const double* lambda,
                         int r, double* fit_dev, cudaStream_t st, double* fold_scratch = nullptr);

}  // namespace cpa
