// KrpSamp + TnsrSamp + sampled normal equations (Section 5.2, Section 5.3).
//
// 1. probe:    one thread per sample finds its fibre [lo, lo + len) in the mode-k
//              stream through the bucket directory and a short binary search (the
//              same kernel clears M and G).
// 2. krp_gram: samples in tiles of 32: y_j = wgt_j * prod_t A_{m_t}(i_t, :) is formed
//              (row gathers of the other factors), stored for step 4, and
//              G += y_j y_j^T is accumulated per thread over upper-triangle pairs.
// 3. scan:     pos = exclusive prefix of len (nnz of the sampled right-hand side).
// 4. mttkrp:   the flattened list of sampled nonzeros is cut into groups of 32, one
//              per warp at a time (so a heavy fibre is spread over many warps and a
//              run of short fibres is resolved 32 at a time); lane c accumulates
//              M(i_k, c) += wgt_j * x * y_j(c) with atomics, into shared memory when
//              M fits, else straight to global memory.
#include "mttkrp.cuh"

namespace cpa {

namespace {

constexpr int kTileRows = 32;
constexpr int kThreads = 256;

__device__ __forceinline__ void pair_of(int p, int r, int* a, int* b) {
  int row = 0, start = 0;
  while (p >= start + (r - row)) {
    start += r - row;
    ++row;
  }
  *a = row;
  *b = row + (p - start);
}

// also clears M (mz elements) and G (r*r) for the kernels that accumulate into them
template <class VT, class FT>
__global__ void k_probe(FibreIndex<VT> X, const uint64_t* __restrict__ idx, DevCount sbar,
                        uint64_t* __restrict__ lo, uint32_t* __restrict__ len, FT* __restrict__ M,
                        int64_t mz, double* __restrict__ G, int gz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mz;
       i += (int64_t)gridDim.x * blockDim.x)
    M[i] = FT(0);
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < gz; i += blockDim.x) G[i] = 0.0;
  const int64_t n = sbar.get();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    uint64_t a, b;
    X.probe(idx[j], &a, &b);
    lo[j] = a;
    len[j] = (uint32_t)(b - a);
  }
}

template <class FT, int PMAX>
__global__ void __launch_bounds__(kThreads) k_krp_gram(FactorPtrs F, KeyLayout L, int r,
                                                       const uint64_t* __restrict__ idx,
                                                       const double* __restrict__ wgt,
                                                       DevCount sbar, FT* __restrict__ Y,
                                                       double* __restrict__ G) {
  extern __shared__ __align__(16) unsigned char krp_smem[];
  FT* tile = reinterpret_cast<FT*>(krp_smem);  // kTileRows * r
  __shared__ uint32_t rows[kTileRows][kMaxOrder];
  __shared__ FT wsh[kTileRows];
  const int np = r * (r + 1) / 2;
  int pa[PMAX], pb[PMAX];
  double acc[PMAX];
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * kThreads;
    if (p < np) pair_of(p, r, &pa[q], &pb[q]); else pa[q] = pb[q] = 0;
    acc[q] = 0.0;
  }
  const int64_t n = sbar.get();
  for (int64_t t0 = (int64_t)blockIdx.x * kTileRows; t0 < n; t0 += (int64_t)gridDim.x * kTileRows) {
    const int cnt = (int)((n - t0) < kTileRows ? (n - t0) : kTileRows);
    __syncthreads();
    if (threadIdx.x < cnt) {
      const uint64_t key = idx[t0 + threadIdx.x];
      for (int t = 0; t < L.d; ++t) rows[threadIdx.x][t] = L.get(key, t);
      wsh[threadIdx.x] = (FT)wgt[t0 + threadIdx.x];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTileRows * r; i += kThreads) {
      const int sl = i / r, c = i - sl * r;
      FT v = FT(0);
      if (sl < cnt) {
        v = wsh[sl];
        for (int t = 0; t < L.d; ++t)
          v *= static_cast<const FT*>(F.A[L.mode[t]])[(int64_t)rows[sl][t] * r + c];
        Y[(t0 + sl) * r + c] = v;
      }
      tile[i] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
      const int p = threadIdx.x + q * kThreads;
      if (p < np) {
        FT s = FT(0);
        for (int i = 0; i < cnt; ++i) s = fma(tile[i * r + pa[q]], tile[i * r + pb[q]], s);
        acc[q] += (double)s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * kThreads;
    if (p < np && acc[q] != 0.0) {
      atomicAdd(&G[pa[q] * r + pb[q]], acc[q]);
      if (pa[q] != pb[q]) atomicAdd(&G[pb[q] * r + pa[q]], acc[q]);
    }
  }
}

// last j in [0, n) with pos[j] <= e (pos ascending, pos[0] = 0 <= e)
__device__ __forceinline__ int64_t sample_of(const uint64_t* __restrict__ pos, int64_t n, uint64_t e) {
  int64_t a = 0, b = n - 1;
  while (a < b) {
    const int64_t mid = (a + b + 1) >> 1;
    if (pos[mid] <= e) a = mid; else b = mid - 1;
  }
  return a;
}

// Lane-parallel gather: a warp takes 32 consecutive sampled nonzeros; each lane
// resolves its own (sample, fibre offset, i_k, wgt_j * x) with independent loads, then
// the warp walks the 32 nonzeros and lane c adds coef * y_j(c) into row i_k of M.
template <class FT, class VT, int CPL, bool kShared>
__global__ void __launch_bounds__(kThreads) k_mttkrp(FibreIndex<VT> X, const FT* __restrict__ Y,
                                                     const double* __restrict__ wgt,
                                                     const uint64_t* __restrict__ lo,
                                                     const uint64_t* __restrict__ pos, DevCount sbar,
                                                     const uint64_t* __restrict__ d_total, int r,
                                                     int64_t nk, FT* __restrict__ M) {
  extern __shared__ __align__(16) unsigned char mk_smem[];
  FT* Ms = reinterpret_cast<FT*>(mk_smem);
  if (kShared) {
    for (int64_t i = threadIdx.x; i < nk * r; i += kThreads) Ms[i] = FT(0);
    __syncthreads();
  }
  const int64_t n = sbar.get();
  const uint64_t total = *d_total;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  for (uint64_t base = (uint64_t)gw * 32; base < total; base += (uint64_t)nwarps * 32) {
    const uint64_t e = base + lane;
    int64_t j = 0;
    int32_t ik = 0;
    FT coef = FT(0);
    if (e < total) {
      j = sample_of(pos, n, e);
      const uint64_t off = lo[j] + (e - pos[j]);
      ik = X.ik[off];
      coef = (FT)wgt[j] * (FT)X.val[off];
    }
    const int nb = total - base < 32 ? (int)(total - base) : 32;
    for (int q = 0; q < nb; ++q) {
      const int64_t jq = __shfl_sync(0xffffffffu, j, q);
      const int32_t iq = __shfl_sync(0xffffffffu, ik, q);
      const FT cq = __shfl_sync(0xffffffffu, coef, q);
#pragma unroll
      for (int u = 0; u < CPL; ++u) {
        const int c = lane + 32 * u;
        if (c < r) {
          const FT v = cq * Y[jq * r + c];
          if (kShared) atomicAdd(&Ms[(int64_t)iq * r + c], v);
          else atomicAdd(&M[(int64_t)iq * r + c], v);
        }
      }
    }
  }
  if (kShared) {
    __syncthreads();
    for (int64_t i = threadIdx.x; i < nk * r; i += kThreads)
      if (Ms[i] != FT(0)) atomicAdd(&M[i], Ms[i]);
  }
}

template <class FT, class VT>
int run(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx, const double* wgt,
        DevCount sbar, FT* M, double* G, MttkrpBuffers& B, cudaStream_t st, cudaEvent_t* ev) {
  const auto& mode = X->mode[k];
  const FibreIndex<VT> fx = fibre_view<VT>(X, k);
  const int64_t s = sbar.max;
  const int sms = num_sms();
  FT* Y = static_cast<FT*>(B.Y);
  int64_t pb = ceil_div(s, kThreads);
  k_probe<VT, FT><<<(unsigned)(pb < sms * 16 ? pb : sms * 16), kThreads, 0, st>>>(
      fx, idx, sbar, B.lo, B.len, M, X->dims[k] * r, G, r * r);
  if (ev && ev[0]) CPA_CUDA_TRY(record_event(ev[0], st));
  const int np = r * (r + 1) / 2;
  int64_t tb = ceil_div(s, kTileRows);
  const unsigned tgrid = (unsigned)(tb < sms * 2 ? tb : sms * 2);
  const size_t tsm = sizeof(FT) * kTileRows * r;
  if (np <= kThreads)
    k_krp_gram<FT, 1><<<tgrid, kThreads, tsm, st>>>(F, mode.L, r, idx, wgt, sbar, Y, G);
  else if (np <= 4 * kThreads)
    k_krp_gram<FT, 4><<<tgrid, kThreads, tsm, st>>>(F, mode.L, r, idx, wgt, sbar, Y, G);
  else
    k_krp_gram<FT, 9><<<tgrid, kThreads, tsm, st>>>(F, mode.L, r, idx, wgt, sbar, Y, G);
  CPA_LAUNCH_CHECK();
  if (ev && ev[1]) CPA_CUDA_TRY(record_event(ev[1], st));
  ScanExtras ex;
  ex.end = true;  // pos[sbar] = nnz of the sampled right-hand side
  CPA_TRY(scan_u64<uint32_t>(B.len, B.pos, sbar, false, B.total, B.scratch, st, ex));
  if (ev && ev[2]) CPA_CUDA_TRY(record_event(ev[2], st));
  const int64_t nk = X->dims[k];
  const bool shared = nk * r * sizeof(FT) <= 48 * 1024;
  const size_t msm = shared ? sizeof(FT) * nk * r : 0;
  const unsigned mgrid = (unsigned)(shared ? sms : sms * 4);
  if (r <= 32) {
    if (shared)
      k_mttkrp<FT, VT, 1, true><<<mgrid, kThreads, msm, st>>>(fx, Y, wgt, B.lo, B.pos, sbar, B.total, r, nk, M);
    else
      k_mttkrp<FT, VT, 1, false><<<mgrid, kThreads, 0, st>>>(fx, Y, wgt, B.lo, B.pos, sbar, B.total, r, nk, M);
  } else {
    if (shared)
      k_mttkrp<FT, VT, 2, true><<<mgrid, kThreads, msm, st>>>(fx, Y, wgt, B.lo, B.pos, sbar, B.total, r, nk, M);
    else
      k_mttkrp<FT, VT, 2, false><<<mgrid, kThreads, 0, st>>>(fx, Y, wgt, B.lo, B.pos, sbar, B.total, r, nk, M);
  }
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

}  // namespace

size_t mttkrp_buffers_bytes(int64_t s, int r, int ft_bytes) {
  Arena a;
  MttkrpBuffers B;
  mttkrp_buffers_carve(a, s, r, ft_bytes, &B);
  return a.used + 256;
}

void mttkrp_buffers_carve(Arena& a, int64_t s, int r, int ft_bytes, MttkrpBuffers* B) {
  B->Y = a.take<char>((size_t)s * r * ft_bytes);
  B->lo = a.take<uint64_t>(s);
  B->len = a.take<uint32_t>(s);
  B->pos = a.take<uint64_t>(s + 1);
  B->total = a.take<uint64_t>(1);
  B->scratch = a.take<char>(scan_workspace(s));
}

template <class FT>
int sampled_mttkrp(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx_packed,
                   const double* wgt, DevCount sbar, FT* M, double* G, MttkrpBuffers& B,
                   cudaStream_t st, cudaEvent_t* ev) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (sbar.max <= 0) return CPA_OK;
  if (X->val_dtype == CPA_F32)
    return run<FT, float>(X, k, F, r, idx_packed, wgt, sbar, M, G, B, st, ev);
  return run<FT, double>(X, k, F, r, idx_packed, wgt, sbar, M, G, B, st, ev);
}
template int sampled_mttkrp<double>(const cpa_index*, int, const FactorPtrs&, int, const uint64_t*,
                                    const double*, DevCount, double*, double*, MttkrpBuffers&,
                                    cudaStream_t, cudaEvent_t*);
template int sampled_mttkrp<float>(const cpa_index*, int, const FactorPtrs&, int, const uint64_t*,
                                   const double*, DevCount, float*, double*, MttkrpBuffers&,
                                   cudaStream_t, cudaEvent_t*);

}  // namespace cpa
