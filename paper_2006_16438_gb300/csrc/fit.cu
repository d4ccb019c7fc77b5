// Exact fit (Eq. 5.1) and estimated fit (Section 5.4).
//
// Exact: fit = 1 - ||X - M|| / ||X|| with
// ||X - M||^2 = ||X||^2 - 2 <X, M> + ||M||^2,  M = [[lambda; A_1, ..., A_D]].
//
// <X, M> is one pass over the fibre index of the mode with the fewest fibres: a
// warp takes a fibre, forms z = lambda * prod_t A_{m_t}(i_t, :) once, and for each
// nonzero of the fibre accumulates x * A_k(i_k, :) per lane; the fibre contributes
// z . acc.  ||M||^2 = lambda^T (Hadamard product of the Grams A_m^T A_m) lambda.
//
// Estimated: a stratified sample of elements drawn once (nonzeros uniformly, zero
// cells uniformly by rejection) and F_hat = sum_j phi_j (m_j - x_j)^2 per evaluation,
// O(s_fit D r) work instead of O(nnz D r).
#include <algorithm>

#include "fit.cuh"

namespace cpa {

namespace {

constexpr int kThreads = 256;

template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_fit_inner(FibreIndex<VT> X, KeyLayout L, FactorPtrs F,
                                                        int kf, const double* __restrict__ lambda,
                                                        int r, double* __restrict__ out, BlockSums S) {
  __shared__ double wsum[kThreads / 32];
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
        v_l = (FT)X.value(p0 + lane);
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
  // warps in order, then blocks in order (the last block to finish adds them)
  if (lane == 0) wsum[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) b += wsum[w];
    S.part[blockIdx.x] = b;
  }
  if (!last_block_to_arrive(S.ticket)) return;
  if (threadIdx.x == 0) *out = ordered_block_sum(S.part, gridDim.x, 1, 0);
  rearm_ticket(S.ticket);
}

// terms (may be null): receives ||X||^2, <X, M> and ||M||^2, the three terms of Eq. 5.1.
__global__ void k_fit_final(const double* __restrict__ grams, int D, const double* __restrict__ lambda,
                            int r, const double* __restrict__ inner, double norm_x2,
                            double* __restrict__ fit_out, double* __restrict__ terms) {
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
    if (terms) {
      terms[0] = norm_x2;
      terms[1] = *inner;
      terms[2] = nm2;
    }
  }
}

}  // namespace

size_t fit_buffers_bytes(int D, int r) { return sizeof(double) * ((size_t)D * r * r + 8) + 512; }

template <class FT>
int fit_enqueue(const cpa_index* X, const FactorPtrs& F, const double* lambda, int r, double* scratch,
                const BlockSums& S, double* fit_dev, cudaStream_t st, double* terms) {
  const int D = X->order;
  double* grams = scratch;
  double* inner = scratch + (size_t)D * r * r;
  CPA_CUDA_TRY(cudaMemsetAsync(inner, 0, sizeof(double), st));  // an empty tensor launches no inner kernel
  for (int m = 0; m < D; ++m)
    CPA_TRY(gram_rows<FT>(static_cast<const FT*>(F.A[m]), X->dims[m], r, grams + (size_t)m * r * r, S, st));
  int kf = 0;
  for (int m = 1; m < D; ++m)
    if (X->mode[m].nfib < X->mode[kf].nfib) kf = m;
  // grid from the size only: the block-ordered sum is then the same at every run
  const int64_t want = ceil_div(X->mode[kf].nfib, kThreads / 32);
  const int64_t cap = S.max_blocks < kSumMaxBlocks ? S.max_blocks : kSumMaxBlocks;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  if (X->mode[kf].nfib > 0)
    with_value_type(X, [&](auto tag) {
      using VT = decltype(tag);
      const FibreIndex<VT> fx = fibre_view<VT>(X, kf);
      if (r <= 32) k_fit_inner<FT, VT, 1><<<grid, kThreads, 0, st>>>(fx, X->mode[kf].L, F, kf, lambda, r, inner, S);
      else k_fit_inner<FT, VT, 2><<<grid, kThreads, 0, st>>>(fx, X->mode[kf].L, F, kf, lambda, r, inner, S);
      return 0;
    });
  k_fit_final<<<1, 256, 0, st>>>(grams, D, lambda, r, inner, X->norm_x2, fit_dev, terms);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}
template int fit_enqueue<double>(const cpa_index*, const FactorPtrs&, const double*, int, double*,
                                 const BlockSums&, double*, cudaStream_t, double*);
template int fit_enqueue<float>(const cpa_index*, const FactorPtrs&, const double*, int, double*,
                                const BlockSums&, double*, cudaStream_t, double*);


// ---------------------------------------------------------------------------
// Estimated fit (Section 5.4)
// ---------------------------------------------------------------------------
namespace {

constexpr int kEstThreads = 256;
constexpr int kEstLanes = 8;  // lanes per sample in the evaluation
constexpr int kDrawThreads = 256;

__device__ __forceinline__ int64_t scale_u64(uint64_t u, int64_t n) {
  return (int64_t)__umul64hi(u, (uint64_t)n);
}

// Nonzero slot j: the nonzero at position floor(u nnz / 2^64) of mode 0's index.
template <class VT>
__global__ void __launch_bounds__(kDrawThreads) k_fit_draw_nz(FibreIndex<VT> X0, KeyLayout L0, int64_t nnz,
                                                              int64_t s_nz, uint64_t seed, int32_t* __restrict__ coords,
                                                              int64_t S, double* __restrict__ xs) {
  const int64_t j = (int64_t)blockIdx.x * kDrawThreads + threadIdx.x;
  if (j >= s_nz) return;
  uint64_t w0 = (uint64_t)j, w1 = 0, w2 = kDomainFit, w3 = 0;
  Philox4x64::block(w0, w1, w2, w3, seed, 0ull);
  const uint64_t p = (uint64_t)scale_u64(w0, nnz);
  // fibre f with off[f] <= p < off[f + 1]
  int64_t a = 0, z = X0.nfib;  // first offset greater than p is off[a + 1]
  while (a < z) {
    const int64_t mid = a + ((z - a) >> 1);
    if (X0.off[mid + 1] <= p) a = mid + 1; else z = mid;
  }
  const uint64_t key = X0.keys[a];
  coords[j] = X0.ik[p];
  for (int t = 0; t < L0.d; ++t) coords[(int64_t)L0.mode[t] * S + j] = (int32_t)L0.get(key, t);
  xs[j] = (double)X0.value(p);
}

// Zero slot j: uniform cells until one is not a nonzero.
template <class VT>
__global__ void __launch_bounds__(kDrawThreads) k_fit_draw_zero(FibreIndex<VT> X0, KeyLayout L0, int D, int64_t n0,
                                                                int64_t s_nz, int64_t s_z, uint64_t seed,
                                                                int reject_cap, int32_t* __restrict__ coords,
                                                                int64_t S, double* __restrict__ xs,
                                                                int* __restrict__ status,
                                                                unsigned long long* __restrict__ attempts) {
  const int64_t j = (int64_t)blockIdx.x * kDrawThreads + threadIdx.x;
  unsigned long long tried = 0;
  if (j < s_z) {
    bool done = false;
    for (int a = 0; a < reject_cap && !done; ++a) {
      int32_t c[kMaxOrder];
      uint64_t w[4];
      for (int m = 0; m < D; ++m) {
        if ((m & 3) == 0) {
          w[0] = (uint64_t)j;
          w[1] = (uint64_t)a;
          w[2] = kDomainFit | 1ull | ((uint64_t)(m >> 2) << 16);
          w[3] = 0;
          Philox4x64::block(w[0], w[1], w[2], w[3], seed, 0ull);
        }
        const int64_t nm = m == 0 ? n0 : L0.n[m - 1];
        c[m] = (int32_t)scale_u64(w[m & 3], nm);
      }
      ++tried;
      uint64_t key = 0;
      for (int t = 0; t < L0.d; ++t) key |= (uint64_t)(uint32_t)c[L0.mode[t]] << L0.off[t];
      uint64_t lo, hi;
      X0.probe(key, &lo, &hi);
      uint64_t a0 = lo, b0 = hi;  // first position in the fibre with i_0 >= c_0 (ascending)
      while (a0 < b0) {
        const uint64_t mid = a0 + ((b0 - a0) >> 1);
        if (X0.ik[mid] < c[0]) a0 = mid + 1; else b0 = mid;
      }
      const bool is_nz = a0 < hi && X0.ik[a0] == c[0];
      if (!is_nz) {
        for (int m = 0; m < D; ++m) coords[(int64_t)m * S + s_nz + j] = c[m];
        xs[s_nz + j] = 0.0;
        done = true;
      }
    }
    if (!done) set_status(status, CPA_ERR_REJECT_LIMIT);
  }
  for (int o = 16; o > 0; o >>= 1) tried += __shfl_xor_sync(0xffffffffu, tried, o);
  if ((threadIdx.x & 31) == 0 && tried) atomicAdd(attempts, tried);
}

// Per block: sum over its samples of phi_j (m_j - x_j)^2, eight lanes per sample
// (lane g of a group takes columns g, g + 8, ...), model value accumulated in FT.
// MD >= D bounds the unrolled per-mode loops (registers for 2 MD coordinates).
template <class FT, int CPL, int MD>
__global__ void __launch_bounds__(kEstThreads) k_fit_est(const int32_t* __restrict__ coords, int64_t stride,
                                                         const double* __restrict__ xs, int64_t S, int64_t s_nz,
                                                         double phi_nz, double phi_z, FactorPtrs F,
                                                         const double* __restrict__ lambda, int r, int D,
                                                         double* __restrict__ partial) {
  __shared__ double red[kEstThreads / 32];
  const int lane = threadIdx.x & 31;
  const int g = lane & (kEstLanes - 1);
  // the four groups of a warp take samples base + 0..3; every lane of the warp runs
  // the same number of iterations (full-mask shuffles)
  const int64_t base0 = (((int64_t)blockIdx.x * kEstThreads + threadIdx.x) >> 5) * (32 / kEstLanes);
  const int64_t ngroups = ((int64_t)gridDim.x * kEstThreads) / kEstLanes;
  const int sub = lane / kEstLanes;
  FT lam[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) {
    const int c = g + kEstLanes * q;
    lam[q] = c < r ? (FT)lambda[c] : FT(0);
  }
  double acc = 0.0;
  // two samples per group and iteration (j and j + ngroups), all coordinate loads
  // issued before the row loads; each lane still adds its samples in ascending j
  for (int64_t base = base0; base < S; base += 2 * ngroups) {
    const int64_t jj[2] = {base + sub, base + ngroups + sub};
    const bool lv[2] = {jj[0] < S, jj[1] < S};
    int32_t ci[2][MD];
#pragma unroll
    for (int m = 0; m < MD; ++m) {
      if (m < D) {
#pragma unroll
        for (int h = 0; h < 2; ++h) ci[h][m] = lv[h] ? __ldg(coords + (int64_t)m * stride + jj[h]) : 0;
      }
    }
    double xv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) xv[h] = (lv[h] && g == 0) ? xs[jj[h]] : 0.0;
    FT v[2][CPL];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < CPL; ++q) v[h][q] = lam[q];
#pragma unroll
    for (int m = 0; m < MD; ++m) {
      if (m < D) {
        const FT* Am = static_cast<const FT*>(F.A[m]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const FT* A = Am + (int64_t)ci[h][m] * r;  // row 0 for a sample past the end (result unused)
#pragma unroll
          for (int q = 0; q < CPL; ++q) {
            const int c = g + kEstLanes * q;
            if (c < r) v[h][q] *= A[c];
          }
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      FT mv = FT(0);
#pragma unroll
      for (int q = 0; q < CPL; ++q) mv += v[h][q];
      for (int o = kEstLanes / 2; o > 0; o >>= 1) mv += __shfl_xor_sync(0xffffffffu, mv, o);
      if (lv[h] && g == 0) {
        const double res = (double)mv - xv[h];
        acc += (jj[h] < s_nz ? phi_nz : phi_z) * res * res;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kEstThreads / 32; ++w) b += red[w];
    partial[blockIdx.x] = b;
  }
}

// FP64 estimate with the FP64 work at its floor (two multiplies and one multiply-add
// per coordinate and sample; GB300's FP64 pipe is the bound): per round a warp takes 16
// samples, copies their factor rows into shared memory (cp.async, one row per copy
// instruction, coalesced), and two lanes evaluate each sample's model value from there
// (lane h takes the coordinates c = h mod 2, in two chains), so no lane idles on padding
// and the only cross-lane step is one pair sum.  The copies of the next round are issued
// before this round is evaluated (two buffers per warp); the coordinates are loaded two
// rounds ahead.  Per block: the sum over its samples of phi_j (m_j - x_j)^2.
constexpr int kErWarps = 4;
constexpr int kErSamples = 16;  // samples per warp and round
constexpr int kErMaxRank = 32;

// lambda null: lambda is folded into the rows of one factor of F (one multiply fewer
// per coordinate).
template <int MD>
__global__ void __launch_bounds__(32 * kErWarps, 2) k_fit_est_rows(const int32_t* __restrict__ coords, int64_t stride,
                                                                   const double* __restrict__ xs, int64_t S,
                                                                   int64_t s_nz, double phi_nz, double phi_z,
                                                                   FactorPtrs F, const double* __restrict__ lambda,
                                                                   int r, int D, double* __restrict__ partial) {
  extern __shared__ __align__(16) double er_smem[];
  __shared__ double red[kErWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rs = r | 1;                      // odd row stride: the two lanes' reads spread over the banks
  const int bufd = MD * kErSamples * rs;     // doubles of one buffer
  double* lam = er_smem;                     // kErMaxRank
  double* rows = er_smem + kErMaxRank + (size_t)warp * 2 * bufd;
  for (int c = threadIdx.x; c < r; c += blockDim.x) lam[c] = lambda ? lambda[c] : 1.0;
  const bool folded = lambda == nullptr;
  __syncthreads();
  const int64_t gw = (int64_t)blockIdx.x * kErWarps + warp, nw = (int64_t)gridDim.x * kErWarps;
  const int64_t nrounds = S > gw * kErSamples ? (S - 1 - gw * kErSamples) / (nw * kErSamples) + 1 : 0;
  // lane l holds the coordinates of sample l & 15 for the modes m = (l >> 4) + 2 u
  constexpr int MH = (MD + 1) / 2;
  auto load_coords = [&](int64_t k, int32_t (&cv)[MH]) {
    const int64_t j = (gw + k * nw) * kErSamples + (lane & 15);
#pragma unroll
    for (int u = 0; u < MH; ++u) {
      const int m = (lane >> 4) + 2 * u;
      cv[u] = (k < nrounds && j < S && m < D) ? __ldg(coords + (int64_t)m * stride + j) : 0;
    }
  };
  auto load_x = [&](int64_t k) {
    const int64_t j = (gw + k * nw) * kErSamples + (lane & 15);
    return (k < nrounds && j < S && lane < 16) ? xs[j] : 0.0;
  };
  auto issue = [&](int b, const int32_t (&cv)[MH]) {
    double* dst = rows + (size_t)b * bufd;
#pragma unroll
    for (int m = 0; m < MD; ++m) {
      if (m >= D) break;
      const double* Am = static_cast<const double*>(F.A[m]);
#pragma unroll
      for (int sm = 0; sm < kErSamples; ++sm) {
        const int row = __shfl_sync(0xffffffffu, cv[m >> 1], sm + 16 * (m & 1));
        if (lane < r) cp_async8(dst + (m * kErSamples + sm) * rs + lane, Am + (int64_t)row * r + lane);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int32_t cnext[MH];
  double acc = 0.0;
  if (nrounds > 0) {
    load_coords(0, cnext);
    issue(0, cnext);
    load_coords(1, cnext);
  }
  double xcur = load_x(0);
  const int sm = lane >> 1, h = lane & 1;
  for (int64_t k = 0; k < nrounds; ++k) {
    if (k + 1 < nrounds) issue((int)((k + 1) & 1), cnext);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");  // an empty group keeps the count
    load_coords(k + 2, cnext);
    const double xnext = load_x(k + 1);
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this round's rows have landed
    __syncwarp();
    const double* R = rows + (size_t)(k & 1) * bufd + sm * rs;
    double m0 = 0.0, m1 = 0.0;
    for (int c = h; c < r; c += 4) {
      double t = folded ? R[c] : lam[c] * R[c];
#pragma unroll
      for (int m = 1; m < MD - 1; ++m)
        if (m < D - 1) t *= R[m * kErSamples * rs + c];
      m0 = fma(t, R[(D - 1) * kErSamples * rs + c], m0);
      const int c2 = c + 2;
      if (c2 < r) {
        double t2 = folded ? R[c2] : lam[c2] * R[c2];
#pragma unroll
        for (int m = 1; m < MD - 1; ++m)
          if (m < D - 1) t2 *= R[m * kErSamples * rs + c2];
        m1 = fma(t2, R[(D - 1) * kErSamples * rs + c2], m1);
      }
    }
    double mv = m0 + m1;
    mv += __shfl_xor_sync(0xffffffffu, mv, 1);
    const double xv = __shfl_sync(0xffffffffu, xcur, sm);
    const int64_t j = (gw + k * nw) * kErSamples + sm;
    if (h == 0 && j < S) {
      const double res = mv - xv;
      acc += (j < s_nz ? phi_nz : phi_z) * res * res;
    }
    xcur = xnext;
    __syncwarp();  // the buffer is refilled two rounds on
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kErWarps; ++w) b += red[w];
    partial[blockIdx.x] = b;
  }
}

// out = A diag(lambda) for an n x r row-major factor (lambda folded into its rows).
__global__ void k_scale_cols(const double* __restrict__ A, int64_t n, int r, const double* __restrict__ lambda,
                             double* __restrict__ out) {
  const int64_t total = n * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = A[e] * lambda[e % r];
}

size_t fit_est_rows_smem(int r, int md) {
  return sizeof(double) * ((size_t)kErMaxRank + (size_t)kErWarps * 2 * md * kErSamples * (r | 1));
}

// F_hat = the partials summed in a fixed order; fit = 1 - sqrt(F_hat) / ||X||.
__global__ void k_fit_est_final(const double* __restrict__ partial, int nb, double norm_x2,
                                double* __restrict__ fit_out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) F += red[w];
    fit_out[0] = norm_x2 > 0.0 ? 1.0 - sqrt(F) / sqrt(norm_x2) : 0.0;
    fit_out[1] = F;
  }
}

// Blocks of the estimate: from the sample size only (8 per SM of a GB300 at most),
// so the fixed-order sum of the block partials is the same whatever the SM budget.
constexpr int kEstMaxBlocks = 1216;
int est_blocks(int64_t S) {
  const int64_t per_block = kEstThreads / kEstLanes;
  const int64_t want = ceil_div(S > 0 ? S : 1, per_block);
  return (int)(want < kEstMaxBlocks ? want : kEstMaxBlocks);
}

}  // namespace

void FitSample::release() {
  if (coords) cudaFree(coords);
  if (xs) cudaFree(xs);
  if (partial) cudaFree(partial);
  coords = nullptr;
  xs = nullptr;
  partial = nullptr;
  s_fit = s_nz = s_z = attempts = 0;
}

int fit_sample_draw(const cpa_index* X, int64_t s_fit, double alpha, uint64_t seed, int reject_cap,
                    FitSample* S, cudaStream_t st) {
  if (s_fit < 1 || !(alpha > 0.0 && alpha <= 1.0) || X->nnz < 1 || reject_cap < 1) return CPA_ERR_ARG;
  const int D = X->order;
  double cells = 1.0;
  for (int m = 0; m < D; ++m) cells *= (double)X->dims[m];
  const bool has_zeros = cells > (double)X->nnz;
  int64_t s_nz = (int64_t)ceil(alpha * (double)s_fit);
  if (s_nz > s_fit) s_nz = s_fit;
  const int64_t s_z = has_zeros ? s_fit - s_nz : 0;
  S->release();
  CPA_CUDA_TRY(cudaMalloc((void**)&S->coords, sizeof(int32_t) * (size_t)D * s_fit));
  CPA_CUDA_TRY(cudaMalloc((void**)&S->xs, sizeof(double) * (size_t)s_fit));
  CPA_CUDA_TRY(cudaMalloc((void**)&S->partial, sizeof(double) * ((size_t)kEstMaxBlocks + 8)));
  int* d_status = nullptr;
  CPA_CUDA_TRY(cudaMallocAsync((void**)&d_status, sizeof(int) * 2 + sizeof(unsigned long long), st));
  unsigned long long* d_att = reinterpret_cast<unsigned long long*>(d_status + 2);
  CPA_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int) * 2 + sizeof(unsigned long long), st));
  const KeyLayout& L0 = X->mode[0].L;
  auto draw = [&](auto tag) -> int {
    using VT = decltype(tag);
    const FibreIndex<VT> x0 = fibre_view<VT>(X, 0);
    if (s_nz > 0)
      k_fit_draw_nz<VT><<<(unsigned)ceil_div(s_nz, kDrawThreads), kDrawThreads, 0, st>>>(
          x0, L0, X->nnz, s_nz, seed, S->coords, s_fit, S->xs);
    CPA_LAUNCH_CHECK();
    if (s_z > 0)
      k_fit_draw_zero<VT><<<(unsigned)ceil_div(s_z, kDrawThreads), kDrawThreads, 0, st>>>(
          x0, L0, D, X->dims[0], s_nz, s_z, seed, reject_cap, S->coords, s_fit, S->xs, d_status, d_att);
    CPA_LAUNCH_CHECK();
    return CPA_OK;
  };
  int rc = with_value_type(X, draw);
  int h_status = 0;
  unsigned long long h_att = 0;
  if (rc == CPA_OK) {
    if (cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&h_att, d_att, sizeof(h_att), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = CPA_ERR_CUDA;
  }
  cudaFreeAsync(d_status, st);
  if (rc == CPA_OK && h_status < 0) rc = h_status;
  if (rc < 0) {
    S->release();
    return rc;
  }
  S->s_fit = s_fit;
  S->stride = s_fit;
  S->s_nz = s_nz;
  S->s_z = s_z;
  S->attempts = (int64_t)h_att;
  S->phi[0] = s_nz > 0 ? (double)X->nnz / (double)s_nz : 0.0;
  S->phi[1] = s_z > 0 ? (cells - (double)X->nnz) / (double)s_z : 0.0;
  S->alpha = alpha;
  S->seed = seed;
  S->reject_cap = reject_cap;
  return CPA_OK;
}

namespace {

// Sort key of sample j: its stratum above the coordinate of the largest mode.
__global__ void k_fit_sort_keys(const int32_t* __restrict__ coords_m, int64_t n, int64_t s_nz,
                                uint64_t* __restrict__ keys, uint32_t* __restrict__ pos) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    keys[j] = ((uint64_t)(j >= s_nz) << 32) | (uint32_t)coords_m[j];
    pos[j] = (uint32_t)j;
  }
}

__global__ void k_fit_gather(const int32_t* __restrict__ coords, const double* __restrict__ xs, int64_t stride,
                             int D, int64_t n, const uint32_t* __restrict__ pos, int32_t* __restrict__ coords_out,
                             double* __restrict__ xs_out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = pos[j];
    for (int m = 0; m < D; ++m) coords_out[(int64_t)m * stride + j] = coords[(int64_t)m * stride + src];
    xs_out[j] = xs[src];
  }
}

}  // namespace

int fit_sample_sort(const cpa_index* X, FitSample* S, cudaStream_t st) {
  const int64_t n = S->s_nz + S->s_z;
  if (n < 2 || n >= (1ll << 32)) return CPA_OK;
  const int D = X->order;
  int mbig = 0;
  for (int m = 1; m < D; ++m)
    if (X->dims[m] > X->dims[mbig]) mbig = m;
  const int bits = 33;  // stratum bit + a 32-bit coordinate
  const size_t ws = sort_workspace(n);
  char* buf = nullptr;
  const size_t need = sizeof(uint64_t) * 2 * n + sizeof(uint32_t) * 2 * n + ws + 1024;
  CPA_CUDA_TRY(cudaMallocAsync((void**)&buf, need, st));
  uint64_t* k0 = reinterpret_cast<uint64_t*>(buf);
  uint64_t* k1 = k0 + n;
  uint32_t* p0 = reinterpret_cast<uint32_t*>(k1 + n);
  uint32_t* p1 = p0 + n;
  char* scratch = reinterpret_cast<char*>(((uintptr_t)(p1 + n) + 255) & ~(uintptr_t)255);
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8);
  k_fit_sort_keys<<<grid, 256, 0, st>>>(S->coords + (size_t)mbig * S->stride, n, S->s_nz, k0, p0);
  CPA_LAUNCH_CHECK();
  int in_alt = 0;
  int rc = radix_sort<uint32_t>(k0, k1, p0, p1, DevCount{nullptr, n}, 0, bits, scratch, st, &in_alt);
  int32_t* coords2 = nullptr;
  double* xs2 = nullptr;
  if (rc == CPA_OK && (cudaMalloc((void**)&coords2, sizeof(int32_t) * (size_t)D * S->stride) != cudaSuccess ||
                       cudaMalloc((void**)&xs2, sizeof(double) * (size_t)S->stride) != cudaSuccess))
    rc = CPA_ERR_OOM;
  if (rc == CPA_OK) {
    k_fit_gather<<<grid, 256, 0, st>>>(S->coords, S->xs, S->stride, D, n, in_alt ? p1 : p0, coords2, xs2);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = CPA_ERR_CUDA;
  }
  cudaFreeAsync(buf, st);
  if (rc < 0) {
    if (coords2) cudaFree(coords2);
    if (xs2) cudaFree(xs2);
    return rc;
  }
  cudaFree(S->coords);
  cudaFree(S->xs);
  S->coords = coords2;
  S->xs = xs2;
  return CPA_OK;
}

// CPA_FIT_EST_ROWS=0 keeps the eight-lanes-per-sample FP64 estimate (for comparison).
static bool rows_est_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("CPA_FIT_EST_ROWS");
    on = (e && atoi(e) == 0) ? 0 : 1;
  }
  return on == 1;
}

template <class FT>
int fit_estimate_enqueue(const cpa_index* X, const FitSample& S, const FactorPtrs& F, const double* lambda,
                         int r, double* fit_dev, cudaStream_t st, double* fold_scratch) {
  const int64_t n = S.s_nz + S.s_z;
  const int nb = est_blocks(n);
  const int D = X->order;
  auto launch = [&](auto cpl_tag) {
    constexpr int CPL = decltype(cpl_tag)::value;
    if (D <= 3)
      k_fit_est<FT, CPL, 3><<<nb, kEstThreads, 0, st>>>(S.coords, S.stride, S.xs, n, S.s_nz, S.phi[0], S.phi[1], F,
                                                        lambda, r, D, S.partial);
    else if (D == 4)
      k_fit_est<FT, CPL, 4><<<nb, kEstThreads, 0, st>>>(S.coords, S.stride, S.xs, n, S.s_nz, S.phi[0], S.phi[1], F,
                                                        lambda, r, D, S.partial);
    else
      k_fit_est<FT, CPL, kMaxOrder><<<nb, kEstThreads, 0, st>>>(S.coords, S.stride, S.xs, n, S.s_nz, S.phi[0],
                                                                S.phi[1], F, lambda, r, D, S.partial);
  };
  if (sizeof(FT) == 8 && r <= kErMaxRank && D <= 4 && rows_est_enabled()) {
    const size_t smem = fit_est_rows_smem(r, D <= 3 ? 3 : 4);
    static std::atomic<unsigned long long> attr{0};
    CPA_CUDA_TRY(set_attr_once(attr, [] {
      cudaError_t e = cudaFuncSetAttribute(k_fit_est_rows<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)fit_est_rows_smem(kErMaxRank, 3));
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(k_fit_est_rows<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fit_est_rows_smem(kErMaxRank, 4));
    }));
    // lambda folded into the rows of the mode with the fewest rows (any mode will do:
    // the kernel multiplies the D rows of a sample and drops its lambda multiply)
    FactorPtrs G = F;
    const double* lam = lambda;
    if (fold_scratch) {
      int mf = 0;
      for (int m = 1; m < D; ++m)
        if (X->dims[m] < X->dims[mf]) mf = m;
      const int64_t cnt = X->dims[mf] * r;
      k_scale_cols<<<(unsigned)std::min<int64_t>(ceil_div(cnt, 256), 4096), 256, 0, st>>>(
          static_cast<const double*>(F.A[mf]), X->dims[mf], r, lambda, fold_scratch);
      G.A[mf] = fold_scratch;
      lam = nullptr;
    }
    if (D <= 3)
      k_fit_est_rows<3><<<nb, 32 * kErWarps, smem, st>>>(S.coords, S.stride, S.xs, n, S.s_nz, S.phi[0], S.phi[1], G,
                                                          lam, r, D, S.partial);
    else
      k_fit_est_rows<4><<<nb, 32 * kErWarps, smem, st>>>(S.coords, S.stride, S.xs, n, S.s_nz, S.phi[0], S.phi[1], G,
                                                          lam, r, D, S.partial);
  } else if (r <= 8) launch(std::integral_constant<int, 1>());
  else if (r <= 16) launch(std::integral_constant<int, 2>());
  else if (r <= 32) launch(std::integral_constant<int, 4>());
  else launch(std::integral_constant<int, 8>());
  CPA_LAUNCH_CHECK();
  k_fit_est_final<<<1, 256, 0, st>>>(S.partial, nb, X->norm_x2, fit_dev);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}
template int fit_estimate_enqueue<double>(const cpa_index*, const FitSample&, const FactorPtrs&, const double*,
                                          int, double*, cudaStream_t, double*);
template int fit_estimate_enqueue<float>(const cpa_index*, const FitSample&, const FactorPtrs&, const double*,
                                         int, double*, cudaStream_t, double*);

}  // namespace cpa
