// KrpSamp, TnsrSamp and the sampled normal-equation products (Section 5.2, 5.3).
//
// Two kernels per update, independent of each other (both read only the samples and
// the factors), so the update runs them as two branches of its graph:
//
// 1. k_krp_gram (KrpSamp + sampled Gram): samples in tiles of 64;
//    y_j = wgt_j * prod_t A_{m_t}(i_t, :) is formed in shared memory (row gathers of
//    the other factors) and G += y_j y_j^T is accumulated per thread over the
//    upper-triangle pairs (tile partials in FT, added across tiles in FP64).
// 2. k_tnsr_mttkrp (KrpSamp + TnsrSamp + sampled MTTKRP, fused): a warp takes 32
//    consecutive samples; lane l probes the fibre of sample l through the bucket
//    directory of the mode-k index; then for each sample with a nonempty fibre the
//    warp forms u_j = wgt_j^2 * prod_t A_{m_t}(i_t, :) (lane c holds column c) and,
//    for every nonzero (i_k, x) of the fibre, adds x * u_j into row i_k of M.  Chunks
//    are taken from a counter; fibres longer than kHeavy are listed and spread over
//    the warps of one block each by k_tnsr_heavy.  The KRP rows are never written.
//
// Optionally (CPA_MTTKRP_SLAB_BYTES = bytes per slab; off by default, since one pass
// with the piece list measured faster on the 1.75e9-nonzero tensor), M's rows are
// split into P slabs.  k_slab_prep probes every sample's fibre once, stores u_j and,
// since the nonzeros of a fibre are sorted by i_k, where each slab's rows start in the
// fibre; then for p = 0..P-1, k_slab_light and k_slab_heavy add the nonzeros of slab p
// only.  Every nonzero is read once; the additions of one pass hit one slab of M,
// small enough to stay in L2, instead of scattering over the whole of it in DRAM.
#include <stdlib.h>

#include "mttkrp.cuh"

namespace cpa {

namespace {

constexpr int kTileRows = 64;        // samples per k_krp_gram tile
constexpr int kThreads = 256;
constexpr int kGramMaxThreads = 1024;

__device__ __forceinline__ void pair_of(int p, int r, int* a, int* b) {
  int row = 0, start = 0;
  while (p >= start + (r - row)) {
    start += r - row;
    ++row;
  }
  *a = row;
  *b = row + (p - start);
}

// blockDim.x threads, each owning up to PMAX upper-triangle pairs (a, b) of G; the
// block size is chosen so that the pairs split evenly (one pair per thread at r = 25).
template <class FT, int PMAX>
__global__ void __launch_bounds__(kGramMaxThreads) k_krp_gram(FactorPtrs F, KeyLayout L, int r,
                                                              const uint64_t* __restrict__ idx,
                                                              const double* __restrict__ wgt,
                                                              DevCount sbar, double* __restrict__ G) {
  extern __shared__ __align__(16) unsigned char krp_smem[];
  FT* tile = reinterpret_cast<FT*>(krp_smem);  // kTileRows * r
  __shared__ uint32_t rows[kTileRows][kMaxOrder];
  __shared__ FT wsh[kTileRows];
  const int np = r * (r + 1) / 2;
  const int nt = blockDim.x;
  int pa[PMAX], pb[PMAX];
  double acc[PMAX];
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * nt;
    if (p < np) pair_of(p, r, &pa[q], &pb[q]); else pa[q] = pb[q] = 0;
    acc[q] = 0.0;
  }
  const int64_t n = sbar.get();
  for (int64_t t0 = (int64_t)blockIdx.x * kTileRows; t0 < n; t0 += (int64_t)gridDim.x * kTileRows) {
    const int cnt = (int)((n - t0) < kTileRows ? (n - t0) : kTileRows);
    __syncthreads();
    for (int sl = threadIdx.x; sl < cnt; sl += nt) {  // nt may be below the tile size
      const uint64_t key = idx[t0 + sl];
      for (int t = 0; t < L.d; ++t) rows[sl][t] = L.get(key, t);
      wsh[sl] = (FT)wgt[t0 + sl];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTileRows * r; i += nt) {
      const int sl = i / r, c = i - sl * r;
      FT v = FT(0);
      if (sl < cnt) {
        v = wsh[sl];
        for (int t = 0; t < L.d; ++t)
          v *= static_cast<const FT*>(F.A[L.mode[t]])[(int64_t)rows[sl][t] * r + c];
      }
      tile[i] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
      const int p = threadIdx.x + q * nt;
      if (p < np) {
        FT s0 = FT(0), s1 = FT(0);  // two chains for the FMA latency
        int i = 0;
        for (; i + 1 < cnt; i += 2) {
          s0 = fma(tile[i * r + pa[q]], tile[i * r + pb[q]], s0);
          s1 = fma(tile[(i + 1) * r + pa[q]], tile[(i + 1) * r + pb[q]], s1);
        }
        if (i < cnt) s0 = fma(tile[i * r + pa[q]], tile[i * r + pb[q]], s0);
        acc[q] += (double)s0 + (double)s1;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * nt;
    if (p < np && acc[q] != 0.0) {
      atomicAdd(&G[pa[q] * r + pb[q]], acc[q]);
      if (pa[q] != pb[q]) atomicAdd(&G[pb[q] * r + pa[q]], acc[q]);
    }
  }
}

constexpr int kHeavy = 64;          // fibres longer than this go to the heavy list
constexpr int kPiece = 4096;        // heavy fibres are listed in pieces of at most this length
constexpr int kHeavyPerSample = 4;  // heavy-list entries per sample of the buffer

// Light pass: warps take chunks of 32 consecutive samples from a counter.  Lane l
// probes sample l; a fibre longer than kHeavy is appended to the heavy list
// (processed by k_tnsr_heavy); the others are walked one sample at a time (lane c
// holds column c of u_j) with the nonzeros loaded 32 at a time.  kPriv: every warp
// accumulates into its own copy of M in shared memory with plain adds (lanes of a
// warp touch distinct columns of one row), summed into M at the end; otherwise
// atomics into M.  ctr[0] += sampled nonzeros, ctr[1] = chunk counter, ctr[2] =
// heavy-list length.
template <class FT, class VT, int CPL, bool kPriv>
__global__ void __launch_bounds__(kThreads, 4) k_tnsr_mttkrp(FibreIndex<VT> X, FactorPtrs F, KeyLayout L,
                                                          int r, const uint64_t* __restrict__ idx,
                                                          const double* __restrict__ wgt, DevCount sbar,
                                                          int64_t nk, FT* __restrict__ M,
                                                          unsigned long long* __restrict__ ctr,
                                                          uint4* __restrict__ heavy, int64_t heavy_cap) {
  extern __shared__ __align__(16) unsigned char mk_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t mz = nk * r;
  FT* Mw = kPriv ? reinterpret_cast<FT*>(mk_smem) + warp * mz : M;
  if (kPriv) {
    for (int64_t i = lane; i < mz; i += 32) Mw[i] = FT(0);
    __syncwarp();
  }
  const int64_t n = sbar.get();
  const int64_t nchunks = (n + 31) >> 5;
  uint64_t my_nnz = 0;
  for (;;) {
    unsigned long long cidx = 0;
    if (lane == 0) cidx = atomicAdd(&ctr[1], 1ull);
    cidx = __shfl_sync(0xffffffffu, cidx, 0);
    if ((int64_t)cidx >= nchunks) break;
    const int64_t base = (int64_t)cidx * 32;
    const int64_t j = base + lane;
    uint64_t key = 0, lo = 0, hi = 0;
    FT w = FT(0);
    if (j < n) {
      key = idx[j];
      X.probe(key, &lo, &hi);
      w = (FT)wgt[j];
    }
    uint32_t len = (uint32_t)(hi - lo);
    my_nnz += len;
    if (len > kHeavy) {  // listed in pieces, each taken whole by one block of k_tnsr_heavy
      const uint32_t np = (len + kPiece - 1) / kPiece;
      const unsigned long long h = atomicAdd(&ctr[2], (unsigned long long)np);
      if (h + np <= (unsigned long long)heavy_cap) {
        for (uint32_t q = 0; q < np; ++q) {
          const uint64_t ps = lo + (uint64_t)q * kPiece;
          const uint32_t pl = len - q * kPiece < (uint32_t)kPiece ? len - q * kPiece : kPiece;
          heavy[h + q] = make_uint4((unsigned)j, (unsigned)(ps & 0xffffffffu), (unsigned)(ps >> 32), pl);
        }
        len = 0;
      } else {  // list full: empty the slots reserved below the capacity, walk the fibre here
        for (unsigned long long q = h; q < h + np && q < (unsigned long long)heavy_cap; ++q)
          heavy[q] = make_uint4((unsigned)j, 0u, 0u, 0u);
      }
    }
    unsigned todo = __ballot_sync(0xffffffffu, len > 0);
    while (todo) {
      const int q = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t lq = __shfl_sync(0xffffffffu, len, q);
      const uint64_t kq = __shfl_sync(0xffffffffu, key, q);
      const uint64_t oq = __shfl_sync(0xffffffffu, lo, q);
      const FT wq = __shfl_sync(0xffffffffu, w, q);
      FT u[CPL];
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int c = lane + 32 * v;
        FT z = FT(0);
        if (c < r) {
          z = wq * wq;
          for (int t = 0; t < L.d; ++t)
            z *= static_cast<const FT*>(F.A[L.mode[t]])[(int64_t)L.get(kq, t) * r + c];
        }
        u[v] = z;
      }
      for (uint32_t g = 0; g < lq; g += 32) {  // nonzeros 32 at a time
        const int nb = lq - g < 32 ? (int)(lq - g) : 32;
        int32_t ikl = 0;
        FT xl = FT(0);
        if (lane < nb) {
          ikl = X.ik[oq + g + lane];
          xl = (FT)X.val[oq + g + lane];
        }
        for (int q2 = 0; q2 < nb; ++q2) {
          const int32_t ik = __shfl_sync(0xffffffffu, ikl, q2);
          const FT x = __shfl_sync(0xffffffffu, xl, q2);
#pragma unroll
          for (int v = 0; v < CPL; ++v) {
            const int c = lane + 32 * v;
            if (c < r) {
              if (kPriv) Mw[(int64_t)ik * r + c] += x * u[v];
              else atomicAdd(&Mw[(int64_t)ik * r + c], x * u[v]);
            }
          }
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) my_nnz += __shfl_xor_sync(0xffffffffu, my_nnz, o);
  if (lane == 0 && my_nnz) atomicAdd(&ctr[0], (unsigned long long)my_nnz);
  if (kPriv) {
    __syncthreads();
    const FT* Mb = reinterpret_cast<const FT*>(mk_smem);
    const int nw = kThreads / 32;
    for (int64_t i = threadIdx.x; i < mz; i += kThreads) {
      FT t = FT(0);
      for (int ww = 0; ww < nw; ++ww) t += Mb[ww * mz + i];
      if (t != FT(0)) atomicAdd(&M[i], t);
    }
  }
}

// Heavy pass: blocks take listed pieces from a counter (ctr[3]); each forms u_j of its
// sample and its warps take the piece's nonzeros in groups of 32 (w, w + 8, ...), the
// next group's loads issued before the current group is added.
template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_tnsr_heavy(FibreIndex<VT> X, FactorPtrs F, KeyLayout L,
                                                         int r, const uint64_t* __restrict__ idx,
                                                         const double* __restrict__ wgt, FT* __restrict__ M,
                                                         unsigned long long* __restrict__ ctr,
                                                         const uint4* __restrict__ heavy, int64_t heavy_cap) {
  __shared__ long long item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long nh = (long long)(ctr[2] < (unsigned long long)heavy_cap ? ctr[2] : heavy_cap);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) item = (long long)atomicAdd(&ctr[3], 1ull);
    __syncthreads();
    const long long h = item;
    if (h >= nh) break;
    const uint4 e = heavy[h];
    const int64_t j = e.x;
    const uint64_t lo = (uint64_t)e.y | ((uint64_t)e.z << 32);
    const uint32_t len = e.w;
    if (len == 0) continue;
    const uint64_t key = idx[j];
    const FT wq = (FT)wgt[j];
    FT u[CPL];
#pragma unroll
    for (int v = 0; v < CPL; ++v) {
      const int c = lane + 32 * v;
      FT z = FT(0);
      if (c < r) {
        z = wq * wq;
        for (int t = 0; t < L.d; ++t)
          z *= static_cast<const FT*>(F.A[L.mode[t]])[(int64_t)L.get(key, t) * r + c];
      }
      u[v] = z;
    }
    uint64_t g = (uint64_t)warp * 32;
    int32_t ikl = 0;
    FT xl = FT(0);
    if (g + lane < len) {
      ikl = X.ik[lo + g + lane];
      xl = (FT)X.val[lo + g + lane];
    }
    for (; g < len; g += kThreads) {
      const int nb = len - g < 32 ? (int)(len - g) : 32;
      const uint64_t gn = g + kThreads;
      int32_t ikn = 0;
      FT xn = FT(0);
      if (gn + lane < len) {
        ikn = X.ik[lo + gn + lane];
        xn = (FT)X.val[lo + gn + lane];
      }
      for (int q2 = 0; q2 < nb; ++q2) {
        const int32_t ik = __shfl_sync(0xffffffffu, ikl, q2);
        const FT x = __shfl_sync(0xffffffffu, xl, q2);
#pragma unroll
        for (int v = 0; v < CPL; ++v) {
          const int c = lane + 32 * v;
          if (c < r) atomicAdd(&M[(int64_t)ik * r + c], x * u[v]);
        }
      }
      ikl = ikn;
      xl = xn;
    }
  }
}

// ---- row-slab path ----------------------------------------------------------
constexpr int kSlabHeavy = 256;    // slab ranges longer than this go to the pass's heavy list
constexpr int kSlabPiece = kPiece;  // heavy slab ranges are listed in pieces of this length

// Per sample (a warp takes 32 consecutive samples): probe the fibre, store u_j and the
// start of each slab's rows in the fibre (ballots over the loaded i_k for fibres of at
// most 32 nonzeros, one bisection per slab boundary otherwise).
template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_slab_prep(FibreIndex<VT> X, FactorPtrs F, KeyLayout L, int r,
                                                        const uint64_t* __restrict__ idx,
                                                        const double* __restrict__ wgt, DevCount sbar,
                                                        int64_t slab_rows, int P, FT* __restrict__ U,
                                                        uint64_t* __restrict__ los, uint32_t* __restrict__ bnd,
                                                        unsigned long long* __restrict__ ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t n = sbar.get();
  const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
  uint64_t my_nnz = 0;
  for (int64_t base = gw * 32; base < n; base += nw * 32) {
    const int64_t j = base + lane;
    uint64_t key = 0, lo = 0, hi = 0;
    FT w = FT(0);
    if (j < n) {
      key = idx[j];
      X.probe(key, &lo, &hi);
      w = (FT)wgt[j];
      los[j] = lo;
    }
    const uint32_t len = (uint32_t)(hi - lo);
    my_nnz += len;
    const int cnt = (int)(n - base < 32 ? n - base : 32);
    for (int q = 0; q < cnt; ++q) {
      const int64_t jq = base + q;
      const uint32_t lq = __shfl_sync(0xffffffffu, len, q);
      const uint64_t kq = __shfl_sync(0xffffffffu, key, q);
      const uint64_t oq = __shfl_sync(0xffffffffu, lo, q);
      const FT wq = __shfl_sync(0xffffffffu, w, q);
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int c = lane + 32 * v;
        if (c < r) {
          FT z = wq * wq;
          for (int t = 0; t < L.d; ++t)
            z *= static_cast<const FT*>(F.A[L.mode[t]])[(int64_t)L.get(kq, t) * r + c];
          U[jq * r + c] = z;
        }
      }
      uint32_t b = 0;
      if (lq <= 32) {
        const int32_t ik = lane < (int)lq ? X.ik[oq + lane] : INT32_MAX;
        for (int p2 = 1; p2 < P; ++p2) {
          const uint32_t below = __popc(__ballot_sync(0xffffffffu, (int64_t)ik < (int64_t)p2 * slab_rows));
          if (lane == p2) b = below;
        }
      } else if (lane > 0 && lane < P) {
        const int64_t target = (int64_t)lane * slab_rows;
        uint64_t a = 0, z = lq;
        while (a < z) {
          const uint64_t mid = a + ((z - a) >> 1);
          if ((int64_t)X.ik[oq + mid] < target) a = mid + 1; else z = mid;
        }
        b = (uint32_t)a;
      }
      if (lane == P) b = lq;
      if (lane <= P) bnd[jq * 32 + lane] = b;
    }
  }
  for (int o = 16; o > 0; o >>= 1) my_nnz += __shfl_xor_sync(0xffffffffu, my_nnz, o);
  if (lane == 0 && my_nnz) atomicAdd(&ctr[0], (unsigned long long)my_nnz);
}

// Pass p, light part: warps take chunks of 32 samples; a sample's range of slab p
// longer than kSlabHeavy is listed for k_slab_heavy, the others are walked as in
// k_tnsr_mttkrp with u_j read back (the nonzero stream is read once: streaming loads).
template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_slab_light(FibreIndex<VT> X, int r, DevCount sbar, int p,
                                                         const FT* __restrict__ U,
                                                         const uint64_t* __restrict__ los,
                                                         const uint32_t* __restrict__ bnd, FT* __restrict__ M,
                                                         unsigned long long* __restrict__ pctr,
                                                         uint4* __restrict__ heavy, int64_t heavy_cap) {
  const int lane = threadIdx.x & 31;
  const int64_t n = sbar.get();
  const int64_t nchunks = (n + 31) >> 5;
  for (;;) {
    unsigned long long cidx = 0;
    if (lane == 0) cidx = atomicAdd(&pctr[0], 1ull);
    cidx = __shfl_sync(0xffffffffu, cidx, 0);
    if ((int64_t)cidx >= nchunks) break;
    const int64_t j = (int64_t)cidx * 32 + lane;
    uint64_t start = 0;
    uint32_t len = 0;
    if (j < n) {
      const uint32_t a = bnd[j * 32 + p], b = bnd[j * 32 + p + 1];
      len = b - a;
      start = los[j] + a;
    }
    if (len > kSlabHeavy) {  // listed in pieces, each taken whole by one block
      const uint32_t np = (len + kSlabPiece - 1) / kSlabPiece;
      const unsigned long long h = atomicAdd(&pctr[1], (unsigned long long)np);
      if (h + np <= (unsigned long long)heavy_cap) {
        for (uint32_t q = 0; q < np; ++q) {
          const uint64_t ps = start + (uint64_t)q * kSlabPiece;
          const uint32_t pl = len - q * kSlabPiece < (uint32_t)kSlabPiece ? len - q * kSlabPiece : kSlabPiece;
          heavy[h + q] = make_uint4((unsigned)j, (unsigned)(ps & 0xffffffffu), (unsigned)(ps >> 32), pl);
        }
        len = 0;
      } else {  // list full: empty the slots reserved below the capacity, walk the range here
        for (unsigned long long q = h; q < h + np && q < (unsigned long long)heavy_cap; ++q)
          heavy[q] = make_uint4((unsigned)j, 0u, 0u, 0u);
      }
    }
    unsigned todo = __ballot_sync(0xffffffffu, len > 0);
    while (todo) {
      const int q = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t lq = __shfl_sync(0xffffffffu, len, q);
      const uint64_t sq = __shfl_sync(0xffffffffu, start, q);
      const int64_t jq = (int64_t)cidx * 32 + q;
      FT u[CPL];
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int c = lane + 32 * v;
        u[v] = c < r ? U[jq * r + c] : FT(0);
      }
      for (uint32_t g = 0; g < lq; g += 32) {
        const int nb = lq - g < 32 ? (int)(lq - g) : 32;
        int32_t ikl = 0;
        FT xl = FT(0);
        if (lane < nb) {
          ikl = __ldcs(X.ik + sq + g + lane);
          xl = (FT)__ldcs(X.val + sq + g + lane);
        }
        for (int q2 = 0; q2 < nb; ++q2) {
          const int32_t ik = __shfl_sync(0xffffffffu, ikl, q2);
          const FT x = __shfl_sync(0xffffffffu, xl, q2);
#pragma unroll
          for (int v = 0; v < CPL; ++v) {
            const int c = lane + 32 * v;
            if (c < r) atomicAdd(&M[(int64_t)ik * r + c], x * u[v]);
          }
        }
      }
    }
  }
}

// Pass p, heavy part: blocks take listed pieces from a counter (pctr[2]); the warps of
// a block take the piece's nonzeros in groups of 32 (w, w + 8, ...), the next group's
// loads issued before the current group is added.
template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_slab_heavy(FibreIndex<VT> X, int r, const FT* __restrict__ U,
                                                         FT* __restrict__ M, unsigned long long* __restrict__ pctr,
                                                         const uint4* __restrict__ heavy, int64_t heavy_cap) {
  __shared__ long long item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long nh = (long long)(pctr[1] < (unsigned long long)heavy_cap ? pctr[1] : heavy_cap);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) item = (long long)atomicAdd(&pctr[2], 1ull);
    __syncthreads();
    const long long h = item;
    if (h >= nh) break;
    const uint4 e = heavy[h];
    const int64_t j = e.x;
    const uint64_t start = (uint64_t)e.y | ((uint64_t)e.z << 32);
    const uint32_t len = e.w;
    FT u[CPL];
#pragma unroll
    for (int v = 0; v < CPL; ++v) {
      const int c = lane + 32 * v;
      u[v] = c < r ? U[j * r + c] : FT(0);
    }
    uint64_t g = (uint64_t)warp * 32;
    int32_t ikl = 0;
    FT xl = FT(0);
    if (g + lane < len) {
      ikl = __ldcs(X.ik + start + g + lane);
      xl = (FT)__ldcs(X.val + start + g + lane);
    }
    for (; g < len; g += kThreads) {
      const int nb = len - g < 32 ? (int)(len - g) : 32;
      const uint64_t gn = g + kThreads;  // prefetch of this warp's next group
      int32_t ikn = 0;
      FT xn = FT(0);
      if (gn + lane < len) {
        ikn = __ldcs(X.ik + start + gn + lane);
        xn = (FT)__ldcs(X.val + start + gn + lane);
      }
      for (int q2 = 0; q2 < nb; ++q2) {
        const int32_t ik = __shfl_sync(0xffffffffu, ikl, q2);
        const FT x = __shfl_sync(0xffffffffu, xl, q2);
#pragma unroll
        for (int v = 0; v < CPL; ++v) {
          const int c = lane + 32 * v;
          if (c < r) atomicAdd(&M[(int64_t)ik * r + c], x * u[v]);
        }
      }
      ikl = ikn;
      xl = xn;
    }
  }
}

template <class FT, class VT>
int launch_mttkrp_slabs(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx,
                        const double* wgt, DevCount sbar, FT* M, MttkrpBuffers& B, int P, cudaStream_t st) {
  const FibreIndex<VT> fx = fibre_view<VT>(X, k);
  const KeyLayout& L = X->mode[k].L;
  const int sms = num_sms();
  const int64_t nk = X->dims[k];
  const int64_t slab_rows = ceil_div(nk, P);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(B.ctr);
  uint4* heavy = reinterpret_cast<uint4*>(B.heavy);
  FT* U = static_cast<FT*>(B.U);
  const int64_t want = ceil_div(sbar.max, (int64_t)kThreads);
  const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? (want > 0 ? want : 1) : (int64_t)sms * 8);
  if (r <= 32)
    k_slab_prep<FT, VT, 1><<<grid, kThreads, 0, st>>>(fx, F, L, r, idx, wgt, sbar, slab_rows, P, U, B.los, B.bnd, ctr);
  else
    k_slab_prep<FT, VT, 2><<<grid, kThreads, 0, st>>>(fx, F, L, r, idx, wgt, sbar, slab_rows, P, U, B.los, B.bnd, ctr);
  CPA_LAUNCH_CHECK();
  const int64_t cap = (int64_t)kHeavyPerSample * (sbar.max > 0 ? sbar.max : 1);
  for (int p = 0; p < P; ++p) {
    unsigned long long* pctr = ctr + 4 + 3 * p;
    if (r <= 32) {
      k_slab_light<FT, VT, 1><<<grid, kThreads, 0, st>>>(fx, r, sbar, p, U, B.los, B.bnd, M, pctr, heavy, cap);
      k_slab_heavy<FT, VT, 1><<<(unsigned)sms * 2, kThreads, 0, st>>>(fx, r, U, M, pctr, heavy, cap);
    } else {
      k_slab_light<FT, VT, 2><<<grid, kThreads, 0, st>>>(fx, r, sbar, p, U, B.los, B.bnd, M, pctr, heavy, cap);
      k_slab_heavy<FT, VT, 2><<<(unsigned)sms * 2, kThreads, 0, st>>>(fx, r, U, M, pctr, heavy, cap);
    }
    CPA_LAUNCH_CHECK();
  }
  return CPA_OK;
}

template <class FT>
int launch_gram(const FactorPtrs& F, const KeyLayout& L, int r, const uint64_t* idx, const double* wgt,
                DevCount sbar, double* G, cudaStream_t st) {
  const int sms = num_sms();
  const int np = r * (r + 1) / 2;
  // threads: the pair count rounded up to whole warps, at most 1024 (r > 44: 2-3 pairs each)
  const int nt = np <= kGramMaxThreads ? ((np + 31) / 32) * 32 : kGramMaxThreads;
  const int per = (np + nt - 1) / nt;
  const int64_t tb = ceil_div(sbar.max, (int64_t)kTileRows);
  const int64_t cap = (int64_t)sms * (nt <= 512 ? 2 : 1);
  const unsigned tgrid = (unsigned)(tb < cap ? tb : cap);
  const size_t tsm = sizeof(FT) * kTileRows * r;
  if (per <= 1)
    k_krp_gram<FT, 1><<<tgrid, nt, tsm, st>>>(F, L, r, idx, wgt, sbar, G);
  else
    k_krp_gram<FT, 3><<<tgrid, nt, tsm, st>>>(F, L, r, idx, wgt, sbar, G);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

template <class FT, class VT>
int launch_mttkrp(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx,
                  const double* wgt, DevCount sbar, FT* M, MttkrpBuffers& B, cudaStream_t st) {
  const FibreIndex<VT> fx = fibre_view<VT>(X, k);
  const KeyLayout& L = X->mode[k].L;
  const int sms = num_sms();
  const int64_t nk = X->dims[k];
  const size_t priv = sizeof(FT) * (size_t)nk * r * (kThreads / 32);  // warp-private copies of M
  const bool use_priv = priv <= 160 * 1024;
  const int64_t want = ceil_div(sbar.max, (int64_t)kThreads);  // one warp per 32 samples
  const int64_t cap = (int64_t)sms * (use_priv ? 1 : 8);
  const unsigned grid = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(B.ctr);
  uint4* heavy = reinterpret_cast<uint4*>(B.heavy);
  const int64_t hcap = (int64_t)kHeavyPerSample * (sbar.max > 0 ? sbar.max : 1);
#define CPA_MK(CPL, PRIV)                                                                         \
  do {                                                                                            \
    if (PRIV) {                                                                                   \
      static bool attr = false;                                                                   \
      if (!attr) {                                                                                \
        CPA_CUDA_TRY(cudaFuncSetAttribute(k_tnsr_mttkrp<FT, VT, CPL, PRIV>,                       \
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024)); \
        attr = true;                                                                              \
      }                                                                                           \
    }                                                                                             \
    k_tnsr_mttkrp<FT, VT, CPL, PRIV><<<grid, kThreads, PRIV ? priv : 0, st>>>(                    \
        fx, F, L, r, idx, wgt, sbar, nk, M, ctr, heavy, hcap);                                    \
  } while (0)
  if (r <= 32) {
    if (use_priv) CPA_MK(1, true); else CPA_MK(1, false);
  } else {
    if (use_priv) CPA_MK(2, true); else CPA_MK(2, false);
  }
#undef CPA_MK
  CPA_LAUNCH_CHECK();
  const unsigned hgrid = (unsigned)sms * 2;
  if (r <= 32)
    k_tnsr_heavy<FT, VT, 1><<<hgrid, kThreads, 0, st>>>(fx, F, L, r, idx, wgt, M, ctr, heavy, hcap);
  else
    k_tnsr_heavy<FT, VT, 2><<<hgrid, kThreads, 0, st>>>(fx, F, L, r, idx, wgt, M, ctr, heavy, hcap);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

}  // namespace

size_t mttkrp_slab_bytes() {
  const char* e = getenv("CPA_MTTKRP_SLAB_BYTES");
  if (e) {
    const long long v = atoll(e);
    if (v > 0) return (size_t)v;
  }
  return 0;  // off: at 1.75e9 nonzeros one pass with the piece list is faster (1.30 vs 1.66 ms per update)
}

int mttkrp_slabs(int64_t nk, int r, int ftb) {
  const size_t bytes = (size_t)nk * r * ftb;
  const size_t slab = mttkrp_slab_bytes();
  if (slab == 0 || bytes <= slab || nk < 2) return 1;
  int64_t P = (int64_t)((bytes + slab - 1) / slab);
  if (P > kSlabMax) P = kSlabMax;
  if (P > nk) P = nk;
  return (int)P;
}

void mttkrp_buffers_carve(Arena& a, int64_t s, int r, int ftb, bool slabs, MttkrpBuffers* B) {
  const size_t ss = (size_t)(s > 0 ? s : 1);
  B->ctr = a.take<uint64_t>(kMttkrpCounters);
  B->total = B->ctr;
  B->heavy = a.take<uint32_t>(4 * ss * kHeavyPerSample);
  if (slabs) {
    B->U = a.take<char>(ss * r * ftb);
    B->los = a.take<uint64_t>(ss);
    B->bnd = a.take<uint32_t>(32 * ss);
  } else {
    B->U = nullptr;
    B->los = nullptr;
    B->bnd = nullptr;
  }
}

template <class FT>
int sampled_mttkrp(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx_packed,
                   const double* wgt, DevCount sbar, FT* M, double* G, MttkrpBuffers& B,
                   cudaStream_t st, cudaEvent_t* ev, const Fork* fork) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  CPA_CUDA_TRY(cudaMemsetAsync(M, 0, sizeof(FT) * X->dims[k] * r, st));
  CPA_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double) * r * r, st));
  CPA_CUDA_TRY(cudaMemsetAsync(B.ctr, 0, kMttkrpCounters * sizeof(uint64_t), st));
  if (sbar.max <= 0) return CPA_OK;
  const KeyLayout& L = X->mode[k].L;
  const int P = B.U ? mttkrp_slabs(X->dims[k], r, (int)sizeof(FT)) : 1;
  auto mttkrp = [&](cudaStream_t s2) {
    if (P > 1)
      return X->val_dtype == CPA_F32
                 ? launch_mttkrp_slabs<FT, float>(X, k, F, r, idx_packed, wgt, sbar, M, B, P, s2)
                 : launch_mttkrp_slabs<FT, double>(X, k, F, r, idx_packed, wgt, sbar, M, B, P, s2);
    return X->val_dtype == CPA_F32
               ? launch_mttkrp<FT, float>(X, k, F, r, idx_packed, wgt, sbar, M, B, s2)
               : launch_mttkrp<FT, double>(X, k, F, r, idx_packed, wgt, sbar, M, B, s2);
  };
  const bool timed = ev && ev[0];
  if (fork && fork->aux && !timed) {
    // the Gram on the side stream, the MTTKRP on st, joined before returning
    CPA_CUDA_TRY(cudaEventRecord(fork->ev_fork, st));
    CPA_CUDA_TRY(cudaStreamWaitEvent(fork->aux, fork->ev_fork, 0));
    CPA_TRY(launch_gram<FT>(F, L, r, idx_packed, wgt, sbar, G, fork->aux));
    CPA_CUDA_TRY(cudaEventRecord(fork->ev_join, fork->aux));
    CPA_TRY(mttkrp(st));
    CPA_CUDA_TRY(cudaStreamWaitEvent(st, fork->ev_join, 0));
    return CPA_OK;
  }
  if (timed) CPA_CUDA_TRY(record_event(ev[0], st));
  CPA_TRY(launch_gram<FT>(F, L, r, idx_packed, wgt, sbar, G, st));
  if (timed && ev[1]) CPA_CUDA_TRY(record_event(ev[1], st));
  CPA_TRY(mttkrp(st));
  return CPA_OK;
}
template int sampled_mttkrp<double>(const cpa_index*, int, const FactorPtrs&, int, const uint64_t*,
                                    const double*, DevCount, double*, double*, MttkrpBuffers&,
                                    cudaStream_t, cudaEvent_t*, const Fork*);
template int sampled_mttkrp<float>(const cpa_index*, int, const FactorPtrs&, int, const uint64_t*,
                                   const double*, DevCount, float*, double*, MttkrpBuffers&,
                                   cudaStream_t, cudaEvent_t*, const Fork*);

}  // namespace cpa
