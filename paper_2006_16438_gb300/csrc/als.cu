// Full CP-ALS on the GPU (Sec. 2, the exact least-squares update that Alg. 3
// randomizes): for each mode k,
//   M = X_(k) (A_D ⊙ ... ⊙ A_{k+1} ⊙ A_{k-1} ⊙ ... ⊙ A_1)   (exact MTTKRP),
//   G = ⊛_{m≠k} A_m^T A_m                                    (Hadamard of Grams),
//   A_k = M G^{-1}, then columns normalised into λ,
// with the same factorisation, solve and fit kernels as the randomized path.
//
// The exact MTTKRP walks the mode-k fibre index: a warp takes a fibre (a distinct
// multi-index of the other modes), forms z = ∏_t A_{m_t}(i_t, :) once (lane c holds
// column c) and adds x * z into row i_k of M for every nonzero of the fibre.
#include "fit.cuh"

namespace cpa {
namespace {

constexpr int kThreads = 256;

template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_exact_mttkrp(FibreIndex<VT> X, KeyLayout L, FactorPtrs F,
                                                           int r, FT* __restrict__ M) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t f = gw; f < X.nfib; f += nwarps) {
    const uint64_t key = X.keys[f];
    FT z[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int c = lane + 32 * q;
      FT v = FT(0);
      if (c < r) {
        v = FT(1);
        for (int t = 0; t < L.d; ++t) v *= static_cast<const FT*>(F.A[L.mode[t]])[(int64_t)L.get(key, t) * r + c];
      }
      z[q] = v;
    }
    const uint64_t b = X.off[f], e = X.off[f + 1];
    for (uint64_t p0 = b; p0 < e; p0 += 32) {
      int32_t ik_l = 0;
      FT v_l = FT(0);
      if (p0 + lane < e) {
        ik_l = X.ik[p0 + lane];
        v_l = (FT)X.value(p0 + lane);
      }
      const int nb = (int)(e - p0 < 32 ? e - p0 : 32);
      for (int q2 = 0; q2 < nb; ++q2) {
        const int32_t ik = __shfl_sync(0xffffffffu, ik_l, q2);
        const FT x = __shfl_sync(0xffffffffu, v_l, q2);
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
          const int c = lane + 32 * q;
          if (c < r) atomicAdd(&M[(int64_t)ik * r + c], x * z[q]);
        }
      }
    }
  }
}

// G = ⊛_{m≠k} grams[m] (r x r each, FP64)
__global__ void k_hadamard_grams(const double* __restrict__ grams, int D, int k, int r, double* __restrict__ G) {
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < D; ++m)
      if (m != k) v *= grams[(int64_t)m * r * r + i];
    G[i] = v;
  }
}

// After A_k's Gram g (r x r) is known: lambda_c = sqrt(g_cc), and g becomes the Gram
// of the normalised A_k (g_ab / (lambda_a lambda_b), zero columns untouched).
__global__ void k_lambda_from_gram(double* __restrict__ g, int r, double* __restrict__ lambda) {
  __shared__ double inv[kMaxRank];
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    const double d = g[c * r + c];
    const double l = d > 0.0 ? sqrt(d) : 0.0;
    lambda[c] = l;
    inv[c] = l > 0.0 ? 1.0 / l : 1.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) g[i] *= inv[i / r] * inv[i % r];
}

template <class FT>
__global__ void k_scale_cols(FT* A, int64_t n, int r, const double* __restrict__ lambda) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * r;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double l = lambda[i % r];
    if (l > 0.0) A[i] = (FT)((double)A[i] / l);
  }
}

template <class FT, class TI>
__global__ void k_conv(const TI* __restrict__ in, int64_t n, FT* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (FT)in[i];
}

unsigned grid_of(int64_t n) {
  const int64_t b = ceil_div(n > 0 ? n : 1, kThreads);
  const int64_t cap = (int64_t)num_sms() * 8;
  return (unsigned)(b < cap ? b : cap);
}

template <class FT>
int exact_mttkrp(const cpa_index* X, int k, const FactorPtrs& F, int r, FT* M, cudaStream_t st) {
  CPA_CUDA_TRY(cudaMemsetAsync(M, 0, sizeof(FT) * X->dims[k] * r, st));
  const auto& mode = X->mode[k];
  if (mode.nfib <= 0) return CPA_OK;
  const unsigned grid = grid_of(mode.nfib * 32);
  with_value_type(X, [&](auto tag) {
    using VT = decltype(tag);
    const FibreIndex<VT> fx = fibre_view<VT>(X, k);
    if (r <= 32) k_exact_mttkrp<FT, VT, 1><<<grid, kThreads, 0, st>>>(fx, mode.L, F, r, M);
    else k_exact_mttkrp<FT, VT, 2><<<grid, kThreads, 0, st>>>(fx, mode.L, F, r, M);
    return 0;
  });
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

// Workspace and the iterations of CP-ALS in element type FT.
template <class FT>
int run_als(const cpa_index* X, const cpa_options* opt, double* lambda, double* const* factors,
            int32_t io_on_device, double* fit, cpa_stats* stats) {
  const int D = X->order, r = opt->rank;
  cudaStream_t st = (cudaStream_t)opt->stream;
  int64_t nmax = 1;
  for (int m = 0; m < D; ++m) nmax = X->dims[m] > nmax ? X->dims[m] : nmax;
  Arena a;
  FT* Fm[kMaxOrder] = {};
  double *stage = nullptr, *grams = nullptr, *G = nullptr, *lam = nullptr, *fitd = nullptr, *fit_ws = nullptr;
  FT* M = nullptr;
  SmallFactor* fs = nullptr;
  int* warn = nullptr;
  BlockSums sums;
  for (int pass = 0; pass < 2; ++pass) {
    a.used = 0;
    for (int m = 0; m < D; ++m) Fm[m] = a.take<FT>((size_t)X->dims[m] * r);
    stage = a.take<double>((size_t)nmax * r);
    M = a.take<FT>((size_t)nmax * r);
    grams = a.take<double>((size_t)D * r * r);
    G = a.take<double>((size_t)r * r);
    lam = a.take<double>(kMaxRank);
    fitd = a.take<double>(4);
    fit_ws = a.take<double>(fit_buffers_bytes(D, r) / sizeof(double) + 1);
    fs = a.take<SmallFactor>(1);
    warn = a.take<int>(4);
    sums = a.take_sums(kSumMaxBlocks, gram_sums_width(r));
    if (pass == 0 && cudaMalloc((void**)&a.base, a.used) != cudaSuccess) return CPA_ERR_OOM;
  }
  struct Free {
    char* p;
    ~Free() {
      if (p) {
        cudaDeviceSynchronize();
        cudaFree(p);
      }
    }
  } guard{a.base};
  const cudaMemcpyKind kin = io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CPA_CUDA_TRY(cudaMemsetAsync(warn, 0, sizeof(int) * 4, st));
  CPA_CUDA_TRY(cudaMemsetAsync(sums.ticket, 0, sizeof(unsigned), st));
  for (int m = 0; m < D; ++m) {
    const int64_t cnt = X->dims[m] * r;
    CPA_CUDA_TRY(cudaMemcpyAsync(stage, factors[m], sizeof(double) * cnt, kin, st));
    k_conv<FT, double><<<grid_of(cnt), kThreads, 0, st>>>(stage, cnt, Fm[m]);
    CPA_LAUNCH_CHECK();
    CPA_TRY(gram_rows<FT>(Fm[m], X->dims[m], r, grams + (size_t)m * r * r, sums, st));
  }
  FactorPtrs F;
  for (int m = 0; m < D; ++m) F.A[m] = Fm[m];
  {
    std::vector<double> ones(kMaxRank, 1.0);
    CPA_CUDA_TRY(cudaMemcpyAsync(lam, ones.data(), sizeof(double) * kMaxRank, cudaMemcpyHostToDevice, st));
    CPA_CUDA_TRY(cudaStreamSynchronize(st));
  }
  for (int it = 0; it < opt->iters; ++it) {
    for (int k = 0; k < D; ++k) {
      const int64_t nk = X->dims[k];
      double* gk = grams + (size_t)k * r * r;
      k_hadamard_grams<<<1, 256, 0, st>>>(grams, D, k, r, G);
      CPA_LAUNCH_CHECK();
      CPA_TRY(exact_mttkrp<FT>(X, k, F, r, M, st));
      CPA_TRY(factor_spd(G, r, 0, 0, 1e-13, fs, warn, CPA_WARN_SINGULAR_GRAM, st));
      CPA_TRY(solve_rows<FT>(M, nk, r, fs, Fm[k], st, gk));  // also clears gk
      CPA_TRY(gram_rows<FT>(Fm[k], nk, r, gk, sums, st));
      k_lambda_from_gram<<<1, 256, 0, st>>>(gk, r, lam);
      CPA_LAUNCH_CHECK();
      k_scale_cols<FT><<<grid_of(nk * r), kThreads, 0, st>>>(Fm[k], nk, r, lam);
      CPA_LAUNCH_CHECK();
    }
  }
  double fv = NAN;
  if (opt->fit_mode == CPA_FIT_EXACT) {
    CPA_TRY(fit_enqueue<FT>(X, F, lam, r, fit_ws, sums, fitd, st));
    CPA_CUDA_TRY(cudaMemcpyAsync(&fv, fitd, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  const cudaMemcpyKind kout = io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int m = 0; m < D; ++m) {
    const int64_t cnt = X->dims[m] * r;
    k_conv<double, FT><<<grid_of(cnt), kThreads, 0, st>>>(Fm[m], cnt, stage);
    CPA_LAUNCH_CHECK();
    CPA_CUDA_TRY(cudaMemcpyAsync(factors[m], stage, sizeof(double) * cnt, kout, st));
    CPA_CUDA_TRY(cudaStreamSynchronize(st));  // stage is reused by the next mode
  }
  CPA_CUDA_TRY(cudaMemcpyAsync(lambda, lam, sizeof(double) * r, kout, st));
  int hwarn = 0;
  CPA_CUDA_TRY(cudaMemcpyAsync(&hwarn, warn, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (fit) {
    if (io_on_device) CPA_CUDA_TRY(cudaMemcpy(fit, &fv, sizeof(double), cudaMemcpyHostToDevice));
    else *fit = fv;
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iters_done = opt->iters;
    stats->mode_updates = opt->iters * D;
    stats->warnings = hwarn;
    stats->kernel_launches = -1;
  }
  return hwarn;
}

}  // namespace
}  // namespace cpa

extern "C" int cp_als(const cpa_index* X, const cpa_options* opt, double* lambda, double* const* factors,
                      int32_t io_on_device, double* fit, cpa_stats* stats) {
  if (!X || !opt || !lambda || !factors) return CPA_ERR_ARG;
  if (opt->rank < 1 || opt->rank > cpa::kMaxRank || opt->iters < 0) return CPA_ERR_ARG;
  if (opt->precision != CPA_FP64 && opt->precision != CPA_MIXED) return CPA_ERR_ARG;
  if (opt->fit_mode != CPA_FIT_EXACT && opt->fit_mode != CPA_FIT_NONE) return CPA_ERR_ARG;
  for (int m = 0; m < X->order; ++m)
    if (!factors[m]) return CPA_ERR_ARG;
  return opt->precision == CPA_MIXED ? cpa::run_als<float>(X, opt, lambda, factors, io_on_device, fit, stats)
                                     : cpa::run_als<double>(X, opt, lambda, factors, io_on_device, fit, stats);
}
