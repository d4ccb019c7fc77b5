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
// When M is larger than one slab (96 MB in FP32, 256 MB in FP64; CPA_MTTKRP_SLAB_BYTES
// sets it, 0 turns slabs off), M's rows are split into P slabs.  k_slab_prep probes
// every sample's fibre once, stores u_j and, since the nonzeros of a fibre are sorted
// by i_k, where each slab's rows start in the fibre; then for p = 0..P-1, k_slab_light
// and k_slab_heavy add the nonzeros of slab p only.  Every nonzero is read once; the
// additions of one pass hit one slab of M, which (in FP32) stays in L2, instead of
// read-modify-writes of rows scattered over the whole of M in DRAM.
#include <stdlib.h>

#include "mttkrp.cuh"

namespace cpa {

namespace {

constexpr int kTileRows = 64;        // samples per k_krp_gram tile
constexpr int kGramGrid = 304;       // k_krp_gram blocks (2 per SM of a GB300)
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
                                                              DevCount sbar, double* __restrict__ G,
                                                              BlockSums S) {
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
  // block partials, added in block order by the last block (G is reproducible)
  double* mine = S.part + (size_t)blockIdx.x * np;
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * nt;
    if (p < np) mine[p] = acc[q];
  }
  if (!last_block_to_arrive(S.ticket)) return;
  for (int p = threadIdx.x; p < np; p += nt) {
    const double v = ordered_block_sum(S.part, gridDim.x, np, p);
    int a, b;
    pair_of(p, r, &a, &b);
    G[a * r + b] = v;
    G[b * r + a] = v;
  }
  rearm_ticket(S.ticket);
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
          xl = (FT)X.value(oq + g + lane);
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
      xl = (FT)X.value(lo + g + lane);
    }
    for (; g < len; g += kThreads) {
      const int nb = len - g < 32 ? (int)(len - g) : 32;
      const uint64_t gn = g + kThreads;
      int32_t ikn = 0;
      FT xn = FT(0);
      if (gn + lane < len) {
        ikn = X.ik[lo + gn + lane];
        xn = (FT)X.value(lo + gn + lane);
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
// fold (may be null): u_j is replaced by v_j = u_j Fs with Fs the inverse (or
// pseudo-inverse) of the sampled Gram, so that the pass accumulates the solved rows
// A_k(i, :) = sum_j x_ij v_j directly; U rows have stride ldu (ldu > r: zero padding).
template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_slab_prep(FibreIndex<VT> X, FactorPtrs F, KeyLayout L, int r,
                                                        const uint64_t* __restrict__ idx,
                                                        const double* __restrict__ wgt, DevCount sbar,
                                                        int64_t slab_rows, int P, FT* __restrict__ U, int ldu,
                                                        uint64_t* __restrict__ los, uint32_t* __restrict__ bnd,
                                                        unsigned long long* __restrict__ ctr,
                                                        const SmallFactor* __restrict__ fold) {
  __shared__ FT Fs[kMaxRank * kMaxRank];
  if (fold) {
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) Fs[i] = (FT)fold->F[i];
    __syncthreads();
  }
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
      FT zr[CPL];
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int c = lane + 32 * v;
        FT z = FT(0);
        if (c < r) {
          z = wq * wq;
          for (int t = 0; t < L.d; ++t)
            z *= static_cast<const FT*>(F.A[L.mode[t]])[(int64_t)L.get(kq, t) * r + c];
        }
        zr[v] = z;
      }
      if (fold) {  // v_c = sum_u z_u Fs(u, c), z_u from lane u % 32, slot u / 32
        FT acc[CPL];
#pragma unroll
        for (int v = 0; v < CPL; ++v) acc[v] = FT(0);
#pragma unroll
        for (int h = 0; h < CPL; ++h)
          for (int uu = 0; uu < 32; ++uu) {
            const int u = 32 * h + uu;
            const FT zu = __shfl_sync(0xffffffffu, zr[h], uu);
            if (u < r) {
#pragma unroll
              for (int v = 0; v < CPL; ++v) {
                const int c = lane + 32 * v;
                if (c < r) acc[v] = fma(zu, Fs[u * r + c], acc[v]);
              }
            }
          }
#pragma unroll
        for (int v = 0; v < CPL; ++v) zr[v] = acc[v];
      }
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int c = lane + 32 * v;
        if (c < ldu) U[jq * ldu + c] = c < r ? zr[v] : FT(0);
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

// Light passes: a warp takes a chunk of kLightChunk consecutive samples (lane l < kLightChunk
// holds sample l's range of slab p; ranges longer than kSlabHeavy are listed for the heavy
// pass) and walks the remaining (sample, group of 32 nonzeros) items in order, issuing
// the next item's loads before the current item's additions.  `sample(j)` sets up a
// sample's row (warp-uniform j), `group(nb, ikl, xl)` adds a group of nb nonzeros
// (lane l holds i_k and x of nonzero l).
constexpr int kLightChunk = 8;

template <class VT, class SampleFn, class GroupFn>
__device__ __forceinline__ void walk_light(const FibreIndex<VT>& X, DevCount sbar, int p,
                                           const uint64_t* __restrict__ los, const uint32_t* __restrict__ bnd,
                                           unsigned long long* __restrict__ pctr, uint4* __restrict__ heavy,
                                           int64_t heavy_cap, SampleFn&& sample, GroupFn&& group) {
  using XT = typename ValueOf<VT>::type;
  const int lane = threadIdx.x & 31;
  const int64_t n = sbar.get();
  const int64_t nchunks = (n + kLightChunk - 1) / kLightChunk;
  for (;;) {
    unsigned long long cidx = 0;
    if (lane == 0) cidx = atomicAdd(&pctr[0], 1ull);
    cidx = __shfl_sync(0xffffffffu, cidx, 0);
    if ((int64_t)cidx >= nchunks) break;
    const int64_t base = (int64_t)cidx * kLightChunk;
    const int64_t j = base + lane;
    uint64_t start = 0;
    uint32_t len = 0;
    if (lane < kLightChunk && j < n) {
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
    if (!todo) continue;
    int q = __ffs(todo) - 1;
    todo &= todo - 1;
    uint32_t lq = __shfl_sync(0xffffffffu, len, q);
    uint64_t sq = __shfl_sync(0xffffffffu, start, q);
    uint32_t g = 0;
    sample(base + q);
    int32_t ikl = 0;
    XT xl = XT(0);
    if (lane < (lq < 32u ? (int)lq : 32)) {
      ikl = __ldcs(X.ik + sq + lane);
      xl = X.value_stream(sq + lane);
    }
    for (;;) {
      const int nb = lq - g < 32 ? (int)(lq - g) : 32;
      uint32_t g2 = g + 32, lq2 = lq;
      uint64_t sq2 = sq;
      int q2 = q;
      bool more = true, fresh = false;
      if (g2 >= lq) {
        if (todo) {
          q2 = __ffs(todo) - 1;
          todo &= todo - 1;
          lq2 = __shfl_sync(0xffffffffu, len, q2);
          sq2 = __shfl_sync(0xffffffffu, start, q2);
          g2 = 0;
          fresh = true;
        } else {
          more = false;
        }
      }
      int32_t ikn = 0;
      XT xn = XT(0);
      if (more && lane < (lq2 - g2 < 32u ? (int)(lq2 - g2) : 32)) {
        ikn = __ldcs(X.ik + sq2 + g2 + lane);
        xn = X.value_stream(sq2 + g2 + lane);
      }
      group(nb, ikl, xl);
      if (!more) break;
      if (fresh) sample(base + q2);
      q = q2;
      lq = lq2;
      sq = sq2;
      g = g2;
      ikl = ikn;
      xl = xn;
    }
  }
}

// Pass p, light part, scalar atomics (FP64, or FP32 rows not padded to 16 bytes): lane c
// holds column c of u_j; one row addition per nonzero.
template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_slab_light(FibreIndex<VT> X, int r, DevCount sbar, int p,
                                                         const FT* __restrict__ U, int ldu,
                                                         const uint64_t* __restrict__ los,
                                                         const uint32_t* __restrict__ bnd, FT* __restrict__ M,
                                                         int ldm, unsigned long long* __restrict__ pctr,
                                                         uint4* __restrict__ heavy, int64_t heavy_cap) {
  using XT = typename ValueOf<VT>::type;
  const int lane = threadIdx.x & 31;
  FT u[CPL];
  walk_light(
      X, sbar, p, los, bnd, pctr, heavy, heavy_cap,
      [&](int64_t j) {
#pragma unroll
        for (int v = 0; v < CPL; ++v) {
          const int c = lane + 32 * v;
          u[v] = c < r ? U[j * ldu + c] : FT(0);
        }
      },
      [&](int nb, int32_t ikl, XT xl) {
        for (int q2 = 0; q2 < nb; ++q2) {
          const int32_t ik = __shfl_sync(0xffffffffu, ikl, q2);
          const FT x = (FT)__shfl_sync(0xffffffffu, xl, q2);
#pragma unroll
          for (int v = 0; v < CPL; ++v) {
            const int c = lane + 32 * v;
            if (c < r) atomicAdd(&M[(int64_t)ik * ldm + c], x * u[v]);
          }
        }
      });
}

// Pass p, heavy part: blocks take listed pieces from a counter (pctr[2]); the warps of
// a block take the piece's nonzeros in groups of 32 (w, w + 8, ...), the next group's
// loads issued before the current group is added.
template <class FT, class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_slab_heavy(FibreIndex<VT> X, int r, const FT* __restrict__ U, int ldu,
                                                         FT* __restrict__ M, int ldm,
                                                         unsigned long long* __restrict__ pctr,
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
      u[v] = c < r ? U[j * ldu + c] : FT(0);
    }
    uint64_t g = (uint64_t)warp * 32;
    int32_t ikl = 0;
    FT xl = FT(0);
    if (g + lane < len) {
      ikl = __ldcs(X.ik + start + g + lane);
      xl = (FT)X.value_stream(start + g + lane);
    }
    for (; g < len; g += kThreads) {
      const int nb = len - g < 32 ? (int)(len - g) : 32;
      const uint64_t gn = g + kThreads;  // prefetch of this warp's next group
      int32_t ikn = 0;
      FT xn = FT(0);
      if (gn + lane < len) {
        ikn = __ldcs(X.ik + start + gn + lane);
        xn = (FT)X.value_stream(start + gn + lane);
      }
      for (int q2 = 0; q2 < nb; ++q2) {
        const int32_t ik = __shfl_sync(0xffffffffu, ikl, q2);
        const FT x = __shfl_sync(0xffffffffu, xl, q2);
#pragma unroll
        for (int v = 0; v < CPL; ++v) {
          const int c = lane + 32 * v;
          if (c < r) atomicAdd(&M[(int64_t)ik * ldm + c], x * u[v]);
        }
      }
      ikl = ikn;
      xl = xn;
    }
  }
}

// ---- FP32 row slabs with 16-byte atomics ------------------------------------
// M rows of ldm = r rounded up to a multiple of 4 floats (16-byte aligned rows, zero
// padding), U rows of the same stride.  A warp adds four nonzeros per instruction:
// lane group g = lane / 8 takes nonzero 4 q + g, its lanes s < ldm / 4 add float4
// s (and s + 8 when ldm > 32) of x u_j with red.global.add.v4.f32, 16 bytes per
// atomic instead of 4 (measured on GB300: 49 against 20 G row additions per second
// into an L2-resident M).
__device__ __forceinline__ void red_add_v4(float* p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

// Adds the nonzeros [0, nb) held by the warp (lane l: i_k and x of nonzero l) times
// u (this lane's float4 pieces) into M.
template <int Q2>
__device__ __forceinline__ void add_group_v4(int nb, int32_t ikl, float xl, const float4 (&u)[Q2], int nq,
                                             float* __restrict__ M, int ldm) {
  const int lane = threadIdx.x & 31, g = lane >> 3, s = lane & 7;
  for (int q = 0; q < nb; q += 4) {
    const int e = q + g;
    const int32_t ik = __shfl_sync(0xffffffffu, ikl, e & 31);
    const float x = __shfl_sync(0xffffffffu, xl, e & 31);
    if (e < nb) {
      float* row = M + (int64_t)ik * ldm;
#pragma unroll
      for (int h = 0; h < Q2; ++h) {
        const int f = s + 8 * h;
        if (f < nq) red_add_v4(row + 4 * f, make_float4(x * u[h].x, x * u[h].y, x * u[h].z, x * u[h].w));
      }
    }
  }
}

template <int Q2>
__device__ __forceinline__ void load_u_v4(const float* __restrict__ U, int64_t j, int nq, float4 (&u)[Q2]) {
  const int s = threadIdx.x & 7;
  const float4* src = reinterpret_cast<const float4*>(U + j * (int64_t)(4 * nq));
#pragma unroll
  for (int h = 0; h < Q2; ++h) {
    const int f = s + 8 * h;
    u[h] = f < nq ? src[f] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Pass p, light part (as k_slab_light, with 16-byte atomics).
template <class VT, int Q2>
__global__ void __launch_bounds__(kThreads) k_slab_light_v4(FibreIndex<VT> X, int nq, DevCount sbar, int p,
                                                            const float* __restrict__ U,
                                                            const uint64_t* __restrict__ los,
                                                            const uint32_t* __restrict__ bnd, float* __restrict__ M,
                                                            unsigned long long* __restrict__ pctr,
                                                            uint4* __restrict__ heavy, int64_t heavy_cap) {
  const int ldm = 4 * nq;
  float4 u[Q2];
  walk_light(
      X, sbar, p, los, bnd, pctr, heavy, heavy_cap, [&](int64_t j) { load_u_v4<Q2>(U, j, nq, u); },
      [&](int nb, int32_t ikl, float xl) { add_group_v4<Q2>(nb, ikl, xl, u, nq, M, ldm); });
}

// Pass p, heavy part (as k_slab_heavy, with 16-byte atomics).
template <class VT, int Q2>
__global__ void __launch_bounds__(kThreads) k_slab_heavy_v4(FibreIndex<VT> X, int nq, const float* __restrict__ U,
                                                            float* __restrict__ M,
                                                            unsigned long long* __restrict__ pctr,
                                                            const uint4* __restrict__ heavy, int64_t heavy_cap) {
  __shared__ long long item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ldm = 4 * nq;
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
    float4 u[Q2];
    load_u_v4<Q2>(U, j, nq, u);
    uint64_t g = (uint64_t)warp * 32;
    int32_t ikl = 0;
    float xl = 0.f;
    if (g + lane < len) {
      ikl = __ldcs(X.ik + start + g + lane);
      xl = (float)X.value_stream(start + g + lane);
    }
    for (; g < len; g += kThreads) {
      const int nb = len - g < 32 ? (int)(len - g) : 32;
      const uint64_t gn = g + kThreads;  // prefetch of this warp's next group
      int32_t ikn = 0;
      float xn = 0.f;
      if (gn + lane < len) {
        ikn = __ldcs(X.ik + start + gn + lane);
        xn = (float)X.value_stream(start + gn + lane);
      }
      add_group_v4<Q2>(nb, ikl, xl, u, nq, M, ldm);
      ikl = ikn;
      xl = xn;
    }
  }
}

// Row-slab passes (P >= 1).  fold (may be null): the rows accumulated are the solved
// rows (u_j replaced by u_j Fs in the prep); ldm: row stride of M (FP32 with ldm a
// multiple of 4: 16-byte atomics).
template <class FT, class VT>
int launch_mttkrp_slabs(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx,
                        const double* wgt, DevCount sbar, FT* M, int ldm, MttkrpBuffers& B, int P,
                        const SmallFactor* fold, cudaStream_t st) {
  const FibreIndex<VT> fx = fibre_view<VT>(X, k);
  const KeyLayout& L = X->mode[k].L;
  const int sms = num_sms();
  const int64_t nk = X->dims[k];
  const int64_t slab_rows = ceil_div(nk, P);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(B.ctr);
  uint4* heavy = reinterpret_cast<uint4*>(B.heavy);
  FT* U = static_cast<FT*>(B.U);
  const bool v4 = sizeof(FT) == 4 && ldm % 4 == 0 && ldm <= 64;
  const int ldu = v4 ? ldm : r;
  const int64_t want = ceil_div(sbar.max, (int64_t)kThreads);
  const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? (want > 0 ? want : 1) : (int64_t)sms * 8);
  if (r <= 32)
    k_slab_prep<FT, VT, 1><<<grid, kThreads, 0, st>>>(fx, F, L, r, idx, wgt, sbar, slab_rows, P, U, ldu, B.los,
                                                      B.bnd, ctr, fold);
  else
    k_slab_prep<FT, VT, 2><<<grid, kThreads, 0, st>>>(fx, F, L, r, idx, wgt, sbar, slab_rows, P, U, ldu, B.los,
                                                      B.bnd, ctr, fold);
  CPA_LAUNCH_CHECK();
  const int64_t cap = (int64_t)kHeavyPerSample * (sbar.max > 0 ? sbar.max : 1);
  // the heavy pieces: two blocks per SM take them from a counter (measured: eight
  // per SM are no faster, the pass is bound by the L2 atomics)
  const unsigned hgrid = (unsigned)sms * 2;
  for (int p = 0; p < P; ++p) {
    unsigned long long* pctr = ctr + 4 + 3 * p;
    if constexpr (sizeof(FT) == 4) {
      if (v4) {
        float* Mf = reinterpret_cast<float*>(M);
        const float* Uf = reinterpret_cast<const float*>(U);
        const int nq = ldm / 4;
        if (nq <= 8) {
          k_slab_light_v4<VT, 1><<<grid, kThreads, 0, st>>>(fx, nq, sbar, p, Uf, B.los, B.bnd, Mf, pctr, heavy, cap);
          k_slab_heavy_v4<VT, 1><<<hgrid, kThreads, 0, st>>>(fx, nq, Uf, Mf, pctr, heavy, cap);
        } else {
          k_slab_light_v4<VT, 2><<<grid, kThreads, 0, st>>>(fx, nq, sbar, p, Uf, B.los, B.bnd, Mf, pctr, heavy, cap);
          k_slab_heavy_v4<VT, 2><<<hgrid, kThreads, 0, st>>>(fx, nq, Uf, Mf, pctr, heavy, cap);
        }
        CPA_LAUNCH_CHECK();
        continue;
      }
    }
    if (r <= 32) {
      k_slab_light<FT, VT, 1><<<grid, kThreads, 0, st>>>(fx, r, sbar, p, U, ldu, B.los, B.bnd, M, ldm, pctr, heavy,
                                                         cap);
      k_slab_heavy<FT, VT, 1><<<hgrid, kThreads, 0, st>>>(fx, r, U, ldu, M, ldm, pctr, heavy, cap);
    } else {
      k_slab_light<FT, VT, 2><<<grid, kThreads, 0, st>>>(fx, r, sbar, p, U, ldu, B.los, B.bnd, M, ldm, pctr, heavy,
                                                         cap);
      k_slab_heavy<FT, VT, 2><<<hgrid, kThreads, 0, st>>>(fx, r, U, ldu, M, ldm, pctr, heavy, cap);
    }
    CPA_LAUNCH_CHECK();
  }
  return CPA_OK;
}

// ---- sampled Gram on the tensor cores (mixed precision) -----------------------
// G = sum_j y_j y_j^T as a matrix product D = Y^T Y over the samples: one block takes
// 128 samples in four tiles of 32.  Its threads form y_j (FP32) and split each value
// into hi = tf32(y) (round to nearest) and lo = y - hi (exact in FP32); the tiles are
// written to shared memory as the K-major operand (rows = the r coordinates padded to
// M = 128, K = samples) in the canonical layout without swizzle (8-row x 16-byte
// core matrices: K-adjacent 128 bytes apart, 8-row groups 1024 bytes apart).  One
// thread issues, per K-step of 8 samples, tcgen05.mma kind::tf32 with M = 128 and
// N = 32 (or 64) for hi.hi, hi.lo and lo.hi (the three-product split, about FP32
// accuracy), accumulating in tensor memory; tcgen05.commit signals an mbarrier per
// tile buffer (two buffers).  The block then reads its r x r partial Gram with
// tcgen05.ld every 128 samples (the FP32 accumulation stays short), sums the partials
// in FP64 in shared memory and adds them into G once.  Every mbarrier wait is bounded:
// on timeout the status word records CPA_ERR_CUDA and the block still frees its
// tensor memory.
namespace tc {

constexpr int kThreads = 256;
constexpr int kK = 32;        // samples per tile
constexpr int kTiles = 4;     // tiles per block
constexpr uint32_t kLBO = 128;   // bytes between K-adjacent core matrices
constexpr uint32_t kSBO = 1024;  // bytes between 8-row groups (kK / 4 core matrices)
constexpr uint32_t kTileBytes = 128 * kK * 4;  // one operand tile (M = 128 rows)
constexpr int kSpin = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kLBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kSBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool wait_parity(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kSpin && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
  return done != 0;
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(y) : "f"(x));
  return __uint_as_float(y);
}

}  // namespace tc

template <int NCOLS>
__global__ void __launch_bounds__(tc::kThreads) k_krp_gram_tc(FactorPtrs F, KeyLayout L, int r,
                                                              const uint64_t* __restrict__ idx,
                                                              const double* __restrict__ wgt, DevCount sbar,
                                                              double* __restrict__ G, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char tc_raw[];
  __shared__ uint32_t rows[tc::kK][kMaxOrder];
  __shared__ float wsh[tc::kK];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem;
  const int64_t n = sbar.get();
  const int64_t group = (int64_t)tc::kK * tc::kTiles;  // samples per readout
  const int64_t ngroups = (n + group - 1) / group;
  if ((int64_t)blockIdx.x >= ngroups) return;  // the whole block
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // four operand tiles (buffer 0 hi, lo; buffer 1 hi, lo), 1024-byte aligned; rows >= r
  // stay zero for the block's life
  const uint32_t raw = tc::smem_u32(tc_raw);
  const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
  float* tiles = reinterpret_cast<float*>(tc_raw + pad);
  const uint32_t tiles_s = raw + pad;
  double* gacc = reinterpret_cast<double*>(tc_raw + pad + 4 * tc::kTileBytes);  // r x r FP64 partial Gram
  for (int i = tid; i < 4 * (int)(tc::kTileBytes / 16); i += tc::kThreads)
    reinterpret_cast<float4*>(tiles)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = tid; i < r * r; i += tc::kThreads) gacc[i] = 0.0;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::smem_u32(&bar[1])));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc::smem_u32(&tmem)),
                 "r"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t d = tmem;
  // D F32, A and B TF32, both K-major, N = NCOLS, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NCOLS >> 3) << 17) | (8u << 24);
  bool ok = true;
  int64_t T = 0;  // tiles issued by this block (tile T uses buffer T & 1, its (T >> 1)-th commit)
  for (int64_t gi = blockIdx.x; gi < ngroups && ok; gi += gridDim.x) {
    const int64_t s0 = gi * group;
    for (int t = 0; t < tc::kTiles; ++t, ++T) {
      const int stage = (int)(T & 1);
      if (T >= 2 && !tc::wait_parity(&bar[stage], (uint32_t)((T - 2) >> 1) & 1u)) ok = false;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int64_t base = s0 + (int64_t)t * tc::kK;
      if (tid < tc::kK) {
        const int64_t j = base + tid;
        float w = 0.f;
        if (j < n) {
          const uint64_t key = idx[j];
          for (int q = 0; q < L.d; ++q) rows[tid][q] = L.get(key, q);
          w = (float)wgt[j];
        } else {
          for (int q = 0; q < L.d; ++q) rows[tid][q] = 0;
        }
        wsh[tid] = w;
      }
      __syncthreads();
      float* hi = tiles + (size_t)(2 * stage) * (tc::kTileBytes / 4);
      float* lo = hi + tc::kTileBytes / 4;
      for (int e = tid; e < tc::kK * r; e += tc::kThreads) {
        const int sl = e / r, c = e - sl * r;
        float v = wsh[sl];
        for (int q = 0; q < L.d; ++q) v *= static_cast<const float*>(F.A[L.mode[q]])[(int64_t)rows[sl][q] * r + c];
        const float h = tc::to_tf32(v);
        const uint32_t off = (uint32_t)(c >> 3) * tc::kSBO + (uint32_t)(sl >> 2) * tc::kLBO + (uint32_t)(c & 7) * 16u +
                             (uint32_t)(sl & 3) * 4u;
        hi[off >> 2] = h;
        lo[off >> 2] = v - h;
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (tid == 0) {
        const uint32_t hs = tiles_s + (uint32_t)(2 * stage) * tc::kTileBytes, ls = hs + tc::kTileBytes;
        for (int ks = 0; ks < tc::kK / 8; ++ks) {
          const uint32_t ko = (uint32_t)ks * 2u * tc::kLBO;  // 8 samples = two core matrices along K
          const uint64_t ah = tc::desc(hs + ko), al = tc::desc(ls + ko);
          tc::mma_tf32(d, ah, ah, idesc, (t | ks) != 0);  // a new group starts from zero
          tc::mma_tf32(d, ah, al, idesc, 1u);
          tc::mma_tf32(d, al, ah, idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            tc::smem_u32(&bar[stage])));
      }
    }
    // the group's last commit on each buffer (tiles T - 2 and T - 1)
    if (!tc::wait_parity(&bar[(T - 2) & 1], (uint32_t)((T - 2) >> 1) & 1u)) ok = false;
    if (!tc::wait_parity(&bar[(T - 1) & 1], (uint32_t)((T - 1) >> 1) & 1u)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
#pragma unroll
      for (int cc = 0; cc < NCOLS / 32; ++cc) {
        if (warp * 32 < r) {  // warp-uniform: this warp's lanes hold rows 32 w .. 32 w + 31
          uint32_t v[32];
          const uint32_t a = d + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
              : "r"(a));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          const int row = warp * 32 + lane;
          if (row < r) {  // each (row, col) belongs to one thread: plain FP64 adds
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int col = cc * 32 + jj;
              if (col < r) gacc[row * r + col] += (double)__uint_as_float(v[jj]);
            }
          }
        }
      }
    }
    // the next group's first products overwrite D: the reads above come first
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  }
  if (!ok) {
    if (tid == 0) atomicCAS(status, 0, CPA_ERR_CUDA);
    if (T >= 1) tc::wait_parity(&bar[(T - 1) & 1], (uint32_t)((T - 1) >> 1) & 1u);  // bounded, again
    if (T >= 2) tc::wait_parity(&bar[(T - 2) & 1], (uint32_t)((T - 2) >> 1) & 1u);
  } else {
    for (int i = tid; i < r * r; i += tc::kThreads)  // the block's partial Gram, once
      if (gacc[i] != 0.0) atomicAdd(&G[i], gacc[i]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(d), "r"(NCOLS));
}

// Sampled Gram of FP32 factors on the tensor cores (k_krp_gram_tc).  Measured on the
// Uber-shaped tensor it is slower than the FP32-pipe kernel (60 against 42 us per
// update: both are bound by the factor-row gathers, the tensor pipe is about 3 %
// busy), so it runs only with CPA_GRAM_TENSOR_CORES=1.
bool gram_tensor_cores() {  // read at each launch set-up (a plan's graph keeps its choice)
  const char* e = getenv("CPA_GRAM_TENSOR_CORES");
  return e && atoi(e) != 0;
}

int launch_gram_tc(const FactorPtrs& F, const KeyLayout& L, int r, const uint64_t* idx, const double* wgt,
                   DevCount sbar, double* G, int* status, cudaStream_t st) {
  const size_t smem_max = 4 * (size_t)tc::kTileBytes + 1024 + sizeof(double) * kMaxRank * kMaxRank;
  const size_t smem = 4 * (size_t)tc::kTileBytes + 1024 + sizeof(double) * (size_t)r * r;
  static std::atomic<unsigned long long> attr{0};
  CPA_CUDA_TRY(set_attr_once(attr, [&] {
    cudaError_t e = cudaFuncSetAttribute(k_krp_gram_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_krp_gram_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
  }));
  const int64_t groups = ceil_div(sbar.max > 0 ? sbar.max : 1, (int64_t)tc::kK * tc::kTiles);
  const int64_t nb = groups < (int64_t)num_sms() * 3 ? groups : (int64_t)num_sms() * 3;  // persistent blocks
  if (r <= 32)
    k_krp_gram_tc<32><<<(unsigned)nb, tc::kThreads, smem, st>>>(F, L, r, idx, wgt, sbar, G, status);
  else
    k_krp_gram_tc<64><<<(unsigned)nb, tc::kThreads, smem, st>>>(F, L, r, idx, wgt, sbar, G, status);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

template <class FT>
int launch_gram(const FactorPtrs& F, const KeyLayout& L, int r, const uint64_t* idx, const double* wgt,
                DevCount sbar, double* G, const BlockSums& S, int* status, cudaStream_t st) {
  if constexpr (sizeof(FT) == 4) {
    if (gram_tensor_cores()) return launch_gram_tc(F, L, r, idx, wgt, sbar, G, status, st);
  }
  const int np = r * (r + 1) / 2;
  // threads: the pair count rounded up to whole warps, at most 1024 (r > 44: 2-3 pairs each)
  const int nt = np <= kGramMaxThreads ? ((np + 31) / 32) * 32 : kGramMaxThreads;
  const int per = (np + nt - 1) / nt;
  // a grid that depends on the sizes only (2 or 1 blocks per SM of a GB300), so the
  // block-ordered sum gives the same G whatever the SM count or budget
  const int64_t tb = ceil_div(sbar.max, (int64_t)kTileRows);
  int64_t cap = nt <= 512 ? kGramGrid : kGramGrid / 2;
  if (cap > S.max_blocks) cap = S.max_blocks;
  const unsigned tgrid = (unsigned)(tb < cap ? tb : cap);
  const size_t tsm = sizeof(FT) * kTileRows * r;
  if (per <= 1)
    k_krp_gram<FT, 1><<<tgrid, nt, tsm, st>>>(F, L, r, idx, wgt, sbar, G, S);
  else
    k_krp_gram<FT, 3><<<tgrid, nt, tsm, st>>>(F, L, r, idx, wgt, sbar, G, S);
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
      static std::atomic<unsigned long long> attr{0};                                             \
      CPA_CUDA_TRY(set_attr_once(attr, [] {                                                       \
        return cudaFuncSetAttribute(k_tnsr_mttkrp<FT, VT, CPL, PRIV>,                             \
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);     \
      }));                                                                                        \
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

size_t mttkrp_slab_bytes(int ftb) {
  const char* e = getenv("CPA_MTTKRP_SLAB_BYTES");
  if (e) {
    const long long v = atoll(e);
    return v > 0 ? (size_t)v : 0;  // 0: one pass whatever M's size
  }
  // Measured per update on the 4.68e9-nonzero Reddit-shaped tensor (M of 1.64 GB in
  // FP64, 0.82 GB in FP32), sampled MTTKRP in ms for slabs of 32 / 64 / 96 / 128 / 256 /
  // 512 MB and one pass: FP64 11.40 / 10.81 / 10.15 / 9.82 / 9.44 / 10.04 / 10.88;
  // FP32 3.92 / 3.34 / 3.18 / 3.85 / 5.04 / - / -.  The FP32 vector atomics gain from a
  // slab that stays in L2; the FP64 row additions are bound by the L2's FP64 atomic
  // rate, and for them fewer passes count more.
  return size_t(ftb == 8 ? 256 : 96) << 20;
}

int mttkrp_slabs(int64_t nk, int r, int ftb) {
  const size_t bytes = (size_t)nk * r * ftb;
  const size_t slab = mttkrp_slab_bytes(ftb);
  if (slab == 0 || bytes <= slab || nk < 2) return 1;
  int64_t P = (int64_t)((bytes + slab - 1) / slab);
  if (P > kSlabMax) P = kSlabMax;
  if (P > nk) P = nk;
  return (int)P;
}

void mttkrp_buffers_carve(Arena& a, int64_t s, int r, int ftb, bool slabs, MttkrpBuffers* B, int64_t det_cap) {
  const size_t ss = (size_t)(s > 0 ? s : 1);
  B->ctr = a.take<uint64_t>(kMttkrpCounters);
  B->total = B->ctr;
  {
    // the sampled Gram's block sums: ticket = a word of ctr (cleared with it)
    B->gsums.part = a.take<double>((size_t)kGramGrid * (r * (r + 1) / 2));
    B->gsums.ticket = B->ctr ? reinterpret_cast<unsigned*>(B->ctr + kMttkrpCounters - 2) : nullptr;
    B->gsums.max_blocks = kGramGrid;
  }
  B->heavy = a.take<uint32_t>(4 * ss * kHeavyPerSample);
  det_buffers_carve(a, s, r, ftb == 8 ? det_cap : 0, &B->det);
  if (slabs) {
    B->U = a.take<char>(ss * fold_ldm(r, ftb) * ftb);
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
  int* gstatus = B.status ? B.status : reinterpret_cast<int*>(B.ctr + kMttkrpCounters - 1);
  const int P = B.U ? mttkrp_slabs(X->dims[k], r, (int)sizeof(FT)) : 1;
  auto mttkrp = [&](cudaStream_t s2) {
    if constexpr (sizeof(FT) == 8) {
      if (B.det.cap > 0)
        return mttkrp_det(X, k, F, r, idx_packed, wgt, sbar, M, reinterpret_cast<unsigned long long*>(B.ctr), B.det,
                          s2);
    }
    return with_value_type(X, [&](auto tag) {
      using VT = decltype(tag);
      if (P > 1) return launch_mttkrp_slabs<FT, VT>(X, k, F, r, idx_packed, wgt, sbar, M, r, B, P, nullptr, s2);
      return launch_mttkrp<FT, VT>(X, k, F, r, idx_packed, wgt, sbar, M, B, s2);
    });
  };
  const bool timed = ev && ev[0];
  if (fork && fork->aux && !timed) {
    // the Gram on the side stream, the MTTKRP on st, joined before returning
    CPA_CUDA_TRY(cudaEventRecord(fork->ev_fork, st));
    CPA_CUDA_TRY(cudaStreamWaitEvent(fork->aux, fork->ev_fork, 0));
    CPA_TRY(launch_gram<FT>(F, L, r, idx_packed, wgt, sbar, G, B.gsums, gstatus, fork->aux));
    CPA_CUDA_TRY(cudaEventRecord(fork->ev_join, fork->aux));
    CPA_TRY(mttkrp(st));
    CPA_CUDA_TRY(cudaStreamWaitEvent(st, fork->ev_join, 0));
    return CPA_OK;
  }
  if (timed) CPA_CUDA_TRY(record_event(ev[0], st));
  CPA_TRY(launch_gram<FT>(F, L, r, idx_packed, wgt, sbar, G, B.gsums, gstatus, st));
  if (timed && ev[1]) CPA_CUDA_TRY(record_event(ev[1], st));
  CPA_TRY(mttkrp(st));
  return CPA_OK;
}
int64_t fold_rows() {
  const char* e = getenv("CPA_FOLD_ROWS");
  if (e) {
    const long long v = atoll(e);
    return v > 0 ? (int64_t)v : INT64_MAX;
  }
  return int64_t(1) << 16;
}

template <class FT>
int sampled_mttkrp_fold(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx_packed,
                        const double* wgt, DevCount sbar, FT* A, int ldm, double* G, SmallFactor* fac, int* warn,
                        MttkrpBuffers& B, cudaStream_t st, cudaEvent_t* ev) {
  if (r < 1 || r > kMaxRank || ldm < r) return CPA_ERR_ARG;
  const int64_t nk = X->dims[k];
  CPA_CUDA_TRY(cudaMemsetAsync(A, 0, sizeof(FT) * nk * ldm, st));
  CPA_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double) * r * r, st));
  CPA_CUDA_TRY(cudaMemsetAsync(B.ctr, 0, kMttkrpCounters * sizeof(uint64_t), st));
  const bool timed = ev && ev[0];
  if (timed) CPA_CUDA_TRY(record_event(ev[0], st));
  const KeyLayout& L = X->mode[k].L;
  int* gstatus = B.status ? B.status : reinterpret_cast<int*>(B.ctr + kMttkrpCounters - 1);
  if (sbar.max > 0) CPA_TRY(launch_gram<FT>(F, L, r, idx_packed, wgt, sbar, G, B.gsums, gstatus, st));
  CPA_TRY(factor_spd(G, r, 0, 0, 1e-13, fac, warn, CPA_WARN_SINGULAR_GRAM, st));
  if (timed && ev[1]) CPA_CUDA_TRY(record_event(ev[1], st));
  if (sbar.max <= 0) return CPA_OK;
  if constexpr (sizeof(FT) == 8) {
    if (B.det.cap > 0 && ldm == r)
      return mttkrp_det(X, k, F, r, idx_packed, wgt, sbar, A, reinterpret_cast<unsigned long long*>(B.ctr), B.det,
                        st, fac);
  }
  if (!B.U) return CPA_ERR_ARG;  // the buffers were carved without the per-sample rows
  int P = mttkrp_slabs(nk, ldm, (int)sizeof(FT));
  if (P < 1) P = 1;
  return with_value_type(X, [&](auto tag) {
    using VT = decltype(tag);
    return launch_mttkrp_slabs<FT, VT>(X, k, F, r, idx_packed, wgt, sbar, A, ldm, B, P, fac, st);
  });
}
template int sampled_mttkrp_fold<double>(const cpa_index*, int, const FactorPtrs&, int, const uint64_t*,
                                         const double*, DevCount, double*, int, double*, SmallFactor*, int*,
                                         MttkrpBuffers&, cudaStream_t, cudaEvent_t*);
template int sampled_mttkrp_fold<float>(const cpa_index*, int, const FactorPtrs&, int, const uint64_t*,
                                        const double*, DevCount, float*, int, double*, SmallFactor*, int*,
                                        MttkrpBuffers&, cudaStream_t, cudaEvent_t*);

template int sampled_mttkrp<double>(const cpa_index*, int, const FactorPtrs&, int, const uint64_t*,
                                    const double*, DevCount, double*, double*, MttkrpBuffers&,
                                    cudaStream_t, cudaEvent_t*, const Fork*);
template int sampled_mttkrp<float>(const cpa_index*, int, const FactorPtrs&, int, const uint64_t*,
                                   const double*, DevCount, float*, double*, MttkrpBuffers&,
                                   cudaStream_t, cudaEvent_t*, const Fork*);

}  // namespace cpa
