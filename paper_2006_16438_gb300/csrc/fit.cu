// Fit of Eq. 5.1: fit = 1 - ||X - M|| / ||X|| with
// ||X - M||^2 = ||X||^2 - 2 <X, M> + ||M||^2,  M = [[lambda; A_1, ..., A_D]].
//
// <X, M> is one pass over the fibre index of the mode with the fewest fibres: a
// warp takes a fibre, forms z = lambda * prod_t A_{m_t}(i_t, :) once, and for each
// nonzero of the fibre accumulates x * A_k(i_k, :) per lane; the fibre contributes
// z . acc.  ||M||^2 = lambda^T (Hadamard product of the Grams A_m^T A_m) lambda.
#include "fit.cuh"

namespace cpa {

namespace {

constexpr int kThreads = 256;

template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_fit_inner(FibreIndex<VT> X, KeyLayout L, FactorPtrs F,
                                                        int kf, const double* __restrict__ lambda,
                                                        int r, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const FT* Ak = static_cast<const FT*>(F.A[kf]);
  double part = 0.0;
  for (int64_t f = gw; f < X.nfib; f += nwarps) {
    const uint64_t key = X.keys[f];
    FT z[CPL], acc[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int c = lane + 32 * q;
      FT v = FT(0);
      if (c < r) {
        v = (FT)lambda[c];
        for (int t = 0; t < L.d; ++t)
          v *= static_cast<const FT*>(F.A[L.mode[t]])[(int64_t)L.get(key, t) * r + c];
      }
      z[q] = v;
      acc[q] = FT(0);
    }
    const uint64_t b = X.off[f], e = X.off[f + 1];
    for (uint64_t p0 = b; p0 < e; p0 += 32) {
      int32_t ik_l = 0;
      FT v_l = FT(0);
      if (p0 + lane < e) {
        ik_l = X.ik[p0 + lane];
        v_l = (FT)X.val[p0 + lane];
      }
      const int nb = (int)(e - p0 < 32 ? e - p0 : 32);
      for (int q2 = 0; q2 < nb; ++q2) {
        const int32_t ik = __shfl_sync(0xffffffffu, ik_l, q2);
        const FT v = __shfl_sync(0xffffffffu, v_l, q2);
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
          const int c = lane + 32 * q;
          if (c < r) acc[q] = fma(v, Ak[(int64_t)ik * r + c], acc[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) part += (double)(z[q] * acc[q]);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0 && part != 0.0) atomicAdd(out, part);
}

__global__ void k_fit_final(const double* __restrict__ grams, int D, const double* __restrict__ lambda,
                            int r, const double* __restrict__ inner, double norm_x2,
                            double* __restrict__ fit_out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) {
    const int a = i / r, b = i % r;
    double h = lambda[a] * lambda[b];
    for (int m = 0; m < D; ++m) h *= grams[(int64_t)m * r * r + i];
    s += h;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double nm2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) nm2 += red[w];
    double F2 = norm_x2 - 2.0 * (*inner) + nm2;
    if (F2 < 0.0) F2 = 0.0;
    *fit_out = norm_x2 > 0.0 ? 1.0 - sqrt(F2) / sqrt(norm_x2) : 0.0;
  }
}

}  // namespace

size_t fit_buffers_bytes(int D, int r) { return sizeof(double) * ((size_t)D * r * r + 8) + 512; }

template <class FT>
int fit_enqueue(const cpa_index* X, const FactorPtrs& F, const double* lambda, int r, double* scratch,
                double* fit_dev, cudaStream_t st) {
  const int D = X->order;
  double* grams = scratch;
  double* inner = scratch + (size_t)D * r * r;
  CPA_CUDA_TRY(cudaMemsetAsync(scratch, 0, sizeof(double) * ((size_t)D * r * r + 1), st));
  for (int m = 0; m < D; ++m)
    CPA_TRY(gram_rows<FT>(static_cast<const FT*>(F.A[m]), X->dims[m], r, grams + (size_t)m * r * r, st));
  int kf = 0;
  for (int m = 1; m < D; ++m)
    if (X->mode[m].nfib < X->mode[kf].nfib) kf = m;
  const int sms = num_sms();
  const int64_t want = ceil_div(X->mode[kf].nfib, kThreads / 32);
  const unsigned grid = (unsigned)(want < sms * 8 ? (want > 0 ? want : 1) : sms * 8);
  if (X->val_dtype == CPA_F32) {
    const FibreIndex<float> fx = fibre_view<float>(X, kf);
    if (r <= 32) k_fit_inner<FT, float, 1><<<grid, kThreads, 0, st>>>(fx, X->mode[kf].L, F, kf, lambda, r, inner);
    else k_fit_inner<FT, float, 2><<<grid, kThreads, 0, st>>>(fx, X->mode[kf].L, F, kf, lambda, r, inner);
  } else {
    const FibreIndex<double> fx = fibre_view<double>(X, kf);
    if (r <= 32) k_fit_inner<FT, double, 1><<<grid, kThreads, 0, st>>>(fx, X->mode[kf].L, F, kf, lambda, r, inner);
    else k_fit_inner<FT, double, 2><<<grid, kThreads, 0, st>>>(fx, X->mode[kf].L, F, kf, lambda, r, inner);
  }
  k_fit_final<<<1, 256, 0, st>>>(grams, D, lambda, r, inner, X->norm_x2, fit_dev);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}
template int fit_enqueue<double>(const cpa_index*, const FactorPtrs&, const double*, int, double*, double*,
                                 cudaStream_t);
template int fit_enqueue<float>(const cpa_index*, const FactorPtrs&, const double*, int, double*, double*,
                                cudaStream_t);

}  // namespace cpa
