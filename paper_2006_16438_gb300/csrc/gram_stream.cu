// Factor Gram G = A^T A of an FP32 factor with many rows (the mixed-precision refresh of
// Alg. 3: the Gram whose Cholesky factor gives the leverage scores of Definition 3.4)
// on the FP32 pipe.
//
// The pass is bound by HBM: r (r + 1) / 2 multiply-adds per row of 4 r bytes, about 6.5
// flop per byte at r = 25, where the FP32 pipe alone reaches 12 flop per byte of this
// part's bandwidth.  (A tensor-core Gram has to pad the r coordinates to the MMA's
// M = 128 and wastes 80 % of its products.)  So the kernel is organised for streaming:
// every warp owns a ring of shared-memory slots of 32 rows, which its lane 0 fills with
// bulk asynchronous copies (cp.async.bulk, completion counted in bytes on an mbarrier
// per slot), several tiles ahead; the warps run independently (no block barrier in the
// loop).  Lane L owns 4 x 4 blocks of the upper triangle of G (padded to a multiple of
// 4) and adds the products of every row of the tile into FP32 registers; after every
// 128 rows those are folded into float-pair accumulators (two_sum), so the result is a
// sum of exact FP32 products with FP32 rounding over 128 rows only.  The warps'
// partials are added in warp order, the blocks' partials in block order (a fixed grid):
// the result is reproducible bit for bit.  Every wait is bounded: on a timeout the
// status word records CPA_ERR_CUDA and the warp drains its copies (bounded again).
//
// The second kernel of this file, k_gram_rows_ffs, streams the rows of an FP64 factor
// the same way for the FP64 refresh and forms G in float-pair arithmetic (about 2^-44
// relative), which is instruction bound rather than HBM bound on this part.
#include "dense.cuh"
#include "ffloat.cuh"
#include "tc.cuh"

namespace cpa {

namespace {

constexpr int kGsWarps = 8;
constexpr int kGsThreads = 32 * kGsWarps;
constexpr int kGsRows = 32;      // rows per warp tile
constexpr int kGsSlotsMax = 8;   // ring slots per warp
constexpr int kGsFold = 4;       // tiles summed in FP32 before the float-pair fold
constexpr int kGsGrid = 304;     // persistent blocks (two per SM of a GB300; fixed: block-ordered sums)

__device__ __forceinline__ int tri_idx(int a, int b, int r) { return a * r - a * (a - 1) / 2 + (b - a); }

// Coordinates c0 .. c0 + 3 of a row.  Past r they hold whatever follows in shared
// memory (the next row, or the space after the ring): those products only reach Gram
// entries past r, which are never written out.
__device__ __forceinline__ void load4(const float* x, int c0, bool vec, float (&v)[4]) {
  if (vec) {  // 16-byte aligned rows
    const float4 t = *reinterpret_cast<const float4*>(x + c0);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = x[c0 + i];
  }
}

// BPL: 4 x 4 blocks per lane (1 for r <= 28, 2 for r <= 32).
template <int BPL>
__global__ void __launch_bounds__(kGsThreads, 2) k_gram_rows_stream(const float* __restrict__ A, int64_t n, int r,
                                                                    int lda, int slots, double* __restrict__ G,
                                                                    BlockSums S, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char gs_smem[];
  __shared__ __align__(8) uint64_t bars[kGsWarps][kGsSlotsMax];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = r * (r + 1) / 2;
  const int tile_f = kGsRows * lda;
  float* ring = reinterpret_cast<float*>(gs_smem) + (size_t)warp * slots * tile_f;
  double* wpart = reinterpret_cast<double*>(gs_smem + (size_t)kGsWarps * slots * tile_f * 4);  // warps x np
  uint64_t* bar = bars[warp];
  // this lane's blocks (bi <= bj) of the upper triangle
  const int nq = (r + 3) >> 2, nb = nq * (nq + 1) / 2;
  int bi[BPL], bj[BPL];
  bool bv[BPL];
#pragma unroll
  for (int j = 0; j < BPL; ++j) {
    int b = lane + 32 * j, i = 0;
    bv[j] = b < nb;
    if (!bv[j]) b = 0;
    while (b >= nq - i) {
      b -= nq - i;
      ++i;
    }
    bi[j] = 4 * i;
    bj[j] = 4 * (i + b);
  }
  float acc[BPL][16], hi[BPL][16], lo[BPL][16];
#pragma unroll
  for (int j = 0; j < BPL; ++j)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[j][e] = hi[j][e] = lo[j][e] = 0.f;
  if (lane == 0) {
    for (int s = 0; s < slots; ++s) tc::mbar_init(&bar[s]);
    tc::fence_mbar_init();
  }
  __syncwarp();
  const int64_t ntiles = (n + kGsRows - 1) / kGsRows;
  const int64_t gw = (int64_t)blockIdx.x * kGsWarps + warp, nw = (int64_t)gridDim.x * kGsWarps;
  const int64_t mine = gw < ntiles ? (ntiles - 1 - gw) / nw + 1 : 0;
  const uint32_t tile_bytes = (uint32_t)tile_f * 4u;
  uint32_t pending = 0, parity = 0;  // lane 0: slots with a copy in flight, parity of each slot's next phase
  if (lane == 0)
    for (int s = 0; s < slots && s < mine; ++s) {
      const int64_t ti = gw + s * nw;
      if ((ti + 1) * kGsRows <= n) {
        tc::mbar_expect_tx(&bar[s], tile_bytes);
        tc::bulk_g2s(ring + (size_t)s * tile_f, A + ti * kGsRows * lda, tile_bytes, &bar[s]);
        pending |= 1u << s;
      }
    }
  const bool vec = (lda & 3) == 0;
  bool ok = true;
  for (int64_t k = 0; k < mine; ++k) {
    const int64_t ti = gw + k * nw;
    const int s = (int)(k % slots);
    float* rw = ring + (size_t)s * tile_f;
    if ((ti + 1) * kGsRows <= n) {
      int got = 1;
      if (lane == 0) {
        got = tc::wait_parity(&bar[s], (parity >> s) & 1u) ? 1 : 0;
        if (got) {
          parity ^= 1u << s;
          pending &= ~(1u << s);
        }
      }
      if (!__shfl_sync(0xffffffffu, got, 0)) {
        ok = false;
        break;
      }
    } else {  // the partial last tile: plain loads, zeros past n
      const int live = (int)(n - ti * kGsRows) * lda;
      const float* src = A + ti * kGsRows * lda;
      for (int e = lane; e < tile_f; e += 32) rw[e] = e < live ? src[e] : 0.f;
    }
    __syncwarp();
#pragma unroll 4
    for (int row = 0; row < kGsRows; ++row) {
      const float* x = rw + row * lda;
#pragma unroll
      for (int j = 0; j < BPL; ++j) {  // lanes without a block compute block (0, 0) and drop it
        float a[4], b[4];
        load4(x, bi[j], vec, a);
        load4(x, bj[j], vec, b);
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[j][4 * p + q] = fmaf(a[p], b[q], acc[j][4 * p + q]);
      }
    }
    __syncwarp();  // the tile has been read: lane 0 refills its slot
    if (lane == 0) {
      const int64_t kn = k + slots;
      if (kn < mine) {
        const int64_t tn = gw + kn * nw;
        if ((tn + 1) * kGsRows <= n) {
          tc::fence_async_smem();
          tc::mbar_expect_tx(&bar[s], tile_bytes);
          tc::bulk_g2s(rw, A + tn * kGsRows * lda, tile_bytes, &bar[s]);
          pending |= 1u << s;
        }
      }
    }
    if (k % kGsFold == kGsFold - 1) {
#pragma unroll
      for (int j = 0; j < BPL; ++j)
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          float sh, se;
          two_sum(hi[j][e], acc[j][e], sh, se);
          hi[j][e] = sh;
          lo[j][e] += se;
          acc[j][e] = 0.f;
        }
    }
  }
  if (!ok && lane == 0) {
    atomicCAS(status, 0, CPA_ERR_CUDA);
    for (int s = 0; s < slots; ++s)  // bounded waits for the copies still in flight
      if (pending & (1u << s)) tc::wait_parity(&bar[s], (parity >> s) & 1u);
  }
  // this warp's partial (the upper triangle), then the block's in warp order
#pragma unroll
  for (int j = 0; j < BPL; ++j) {
    if (!bv[j]) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = bi[j] + p, b = bj[j] + q;
        if (a <= b && b < r) {
          float sh, se;
          two_sum(hi[j][4 * p + q], acc[j][4 * p + q], sh, se);
          wpart[warp * np + tri_idx(a, b, r)] = (double)sh + ((double)lo[j][4 * p + q] + (double)se);
        }
      }
  }
  __syncthreads();
  double* mine_part = S.part + (size_t)blockIdx.x * np;
  for (int i = tid; i < np; i += kGsThreads) {
    double v = wpart[i];
    for (int w = 1; w < kGsWarps; ++w) v += wpart[w * np + i];
    mine_part[i] = v;
  }
  if (!last_block_to_arrive(S.ticket)) return;
  for (int i = tid; i < r * r; i += kGsThreads) {
    const int a = i / r, b = i - a * r;
    if (b < a) continue;
    const double v = ordered_block_sum(S.part, gridDim.x, np, tri_idx(a, b, r));
    G[a * r + b] = v;
    G[b * r + a] = v;
  }
  rearm_ticket(S.ticket);
}

// ---- FP64 rows in float-pair arithmetic ------------------------------------
// The same streaming layout for an FP64 factor (the FP64 refresh: G to about 2^-44
// relative, as the FP64 path's leverage scores need).  GB300 issues one FP64 warp
// instruction per 64 cycles per SM sub-partition, so the products run on the FP32
// pipe: once a tile of kGdRows rows has landed, the warp rewrites it in place as float
// pairs (split_ff: the value's top 24 significand bits and the rest, 8 bytes like the
// double they replace).  G's upper triangle, padded to nq = ceil(r / B) blocks of B x B,
// has nb = nq (nq + 1) / 2 blocks; lane L owns block L mod nb of the rows congruent to
// L / nb modulo R (R: the largest power of two with R nb <= 32, at most kGdRows), and
// adds each product in float-pair arithmetic (ff_fma: twelve FP32 instructions).  After
// every 64 rows of a lane each pair is renormalised (TwoSum), its high part added to the
// warp's FP64 partial in shared memory (the FP64 value built by integer operations; the
// R row groups one after another) and its low part to an FP32 remainder (in shared
// memory, lane-major: registers hold the B^2 pairs), added once at the end.  Warps in
// order, blocks in order: the result is reproducible bit for bit.
// B = 5 serves r = 21..25 with two rows per pass (375 products per row pair against
// 448 per row for B = 4).  Up to r = kGramStreamFP64MaxRank = 28: from 29 on one block
// per lane pads to 35 coordinates (700 products per row for 528), and an 8.2M x 32
// factor measured no faster than with the one-pair-per-thread kernel.
constexpr int kGdRows = 16;         // FP64 rows per warp tile (16 lda doubles: a multiple of 16 bytes)
constexpr int kGdRun = 4;           // tiles per float-pair run and row group (64 products per pair)
constexpr int kGdGrid = 304;        // blocks (two per SM of a GB300; fixed: block-ordered sums)
constexpr int kGdRingBytes = 6400;  // ring bytes per warp (two 25-column tiles)
constexpr int kGdRemMax = 25;       // FP32 remainders per lane (B^2 for B <= 5)

__device__ __forceinline__ void gd_fold(float& hi, float& lo, float* rem, double* dst, bool valid) {
  float s, e;
  two_sum(hi, lo, s, e);
  if (valid) *dst += f2d_exact(s);
  *rem = __fadd_rn(*rem, e);
  hi = 0.f;
  lo = 0.f;
}

// Blocks of G and rows per pass of the FP64 streaming Gram for block size b.
inline int gd_blocks(int r, int b) {
  const int nq = (r + b - 1) / b;
  return nq * (nq + 1) / 2;
}
inline int gd_rows_per_pass(int nb) {
  int R = 1;
  while (2 * R * nb <= 32 && 2 * R <= kGdRows) R *= 2;
  return R;
}

template <int B>
__device__ __forceinline__ void gd_fold_all(float (&hi)[B * B], float (&lo)[B * B], float* rem, double* wp,
                                            int bi, int bj, int r, bool bv, int ro, int R, bool last) {
  for (int g = 0; g < R; ++g) {  // row groups in turn: their lanes share the block's entries
    if (ro == g) {
#pragma unroll
      for (int p = 0; p < B; ++p)
#pragma unroll
        for (int q = 0; q < B; ++q) {
          const int a = bi + p, b = bj + q;
          const bool valid = bv && a <= b && b < r;
          double* dst = wp + (valid ? tri_idx(a, b, r) : 0);
          gd_fold(hi[B * p + q], lo[B * p + q], rem + 32 * (B * p + q), dst, valid);
          if (last && valid) *dst += f2d_exact(rem[32 * (B * p + q)]);
        }
    }
    __syncwarp();
  }
}

template <int B>
__global__ void __launch_bounds__(kGsThreads, 2)
    k_gram_rows_ffs(const double* __restrict__ A, int64_t n, int r, int lda, int slots, double* __restrict__ G,
                    BlockSums S, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char gd_smem[];
  __shared__ __align__(8) uint64_t bars[kGsWarps][kGsSlotsMax];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = r * (r + 1) / 2;
  const int tile_d = kGdRows * lda;
  double* ring = reinterpret_cast<double*>(gd_smem) + (size_t)warp * slots * tile_d;
  double* wpart = reinterpret_cast<double*>(gd_smem) + (size_t)kGsWarps * slots * tile_d;  // warps x np
  double* wp = wpart + warp * np;
  float* rem = reinterpret_cast<float*>(wpart + kGsWarps * np) + (warp * kGdRemMax) * 32 + lane;  // stride 32
  uint64_t* bar = bars[warp];
  const int nq = (r + B - 1) / B, nb = nq * (nq + 1) / 2;
  int R = 1;
  while (2 * R * nb <= 32 && 2 * R <= kGdRows) R *= 2;
  // this lane's row group and block (bi <= bj); lanes past R nb take block 0 of group 0
  // and drop it
  const bool bv = lane < R * nb;
  const int ro = bv ? lane / nb : 0;
  int bi, bj;
  {
    int b = bv ? lane - ro * nb : 0, i = 0;
    while (b >= nq - i) {
      b -= nq - i;
      ++i;
    }
    bi = B * i;
    bj = B * (i + b);
  }
  float hi[B * B], lo[B * B];
#pragma unroll
  for (int e = 0; e < B * B; ++e) {
    hi[e] = lo[e] = 0.f;
    rem[32 * e] = 0.f;
  }
  for (int i = lane; i < np; i += 32) wp[i] = 0.0;
  if (lane == 0) {
    for (int s = 0; s < slots; ++s) tc::mbar_init(&bar[s]);
    tc::fence_mbar_init();
  }
  __syncwarp();
  const int64_t ntiles = (n + kGdRows - 1) / kGdRows;
  const int64_t gw = (int64_t)blockIdx.x * kGsWarps + warp, nw = (int64_t)gridDim.x * kGsWarps;
  const int64_t mine = gw < ntiles ? (ntiles - 1 - gw) / nw + 1 : 0;
  const uint32_t tile_bytes = (uint32_t)tile_d * 8u;
  const int run = kGdRun * R;  // tiles between folds
  uint32_t pending = 0, parity = 0;  // lane 0: slots with a copy in flight, parity of each slot's next phase
  if (lane == 0)
    for (int s = 0; s < slots && s < mine; ++s) {
      const int64_t ti = gw + s * nw;
      if ((ti + 1) * kGdRows <= n) {
        tc::mbar_expect_tx(&bar[s], tile_bytes);
        tc::bulk_g2s(ring + (size_t)s * tile_d, A + ti * kGdRows * lda, tile_bytes, &bar[s]);
        pending |= 1u << s;
      }
    }
  bool ok = true;
  for (int64_t k = 0; k < mine; ++k) {
    const int64_t ti = gw + k * nw;
    const int s = (int)(k % slots);
    double* rw = ring + (size_t)s * tile_d;
    float2* tw = reinterpret_cast<float2*>(rw);  // the same bytes, as float pairs
    if ((ti + 1) * kGdRows <= n) {
      int got = 1;
      if (lane == 0) {
        got = tc::wait_parity(&bar[s], (parity >> s) & 1u) ? 1 : 0;
        if (got) {
          parity ^= 1u << s;
          pending &= ~(1u << s);
        }
      }
      if (!__shfl_sync(0xffffffffu, got, 0)) {
        ok = false;
        break;
      }
      for (int e = lane; e < tile_d; e += 32) tw[e] = split_ff(rw[e]);  // each lane its own entries
    } else {  // the partial last tile: plain loads, zeros past n
      const int live = (int)(n - ti * kGdRows) * lda;
      const double* src = A + ti * kGdRows * lda;
      for (int e = lane; e < tile_d; e += 32) tw[e] = e < live ? split_ff(src[e]) : make_float2(0.f, 0.f);
    }
    __syncwarp();
#pragma unroll(B == 5 ? 1 : 2)
    for (int row = ro; row < kGdRows; row += R) {
      // coordinates past r read the next row or the space after the ring: those
      // products only reach entries past r, which are never written out
      const float2* x = tw + row * lda;
      float2 a[B], b[B];
#pragma unroll
      for (int i = 0; i < B; ++i) {
        a[i] = x[bi + i];
        b[i] = x[bj + i];
      }
#pragma unroll
      for (int p = 0; p < B; ++p)
#pragma unroll
        for (int q = 0; q < B; ++q) ff_fma(a[p].x, a[p].y, b[q].x, b[q].y, hi[B * p + q], lo[B * p + q]);
    }
    __syncwarp();  // the tile has been read: lane 0 refills its slot
    if (lane == 0) {
      const int64_t kn = k + slots;
      if (kn < mine) {
        const int64_t tn = gw + kn * nw;
        if ((tn + 1) * kGdRows <= n) {
          tc::fence_async_smem();
          tc::mbar_expect_tx(&bar[s], tile_bytes);
          tc::bulk_g2s(rw, A + tn * kGdRows * lda, tile_bytes, &bar[s]);
          pending |= 1u << s;
        }
      }
    }
    if (k % run == run - 1) gd_fold_all<B>(hi, lo, rem, wp, bi, bj, r, bv, ro, R, false);
  }
  if (!ok && lane == 0) {
    atomicCAS(status, 0, CPA_ERR_CUDA);
    for (int s = 0; s < slots; ++s)  // bounded waits for the copies still in flight
      if (pending & (1u << s)) tc::wait_parity(&bar[s], (parity >> s) & 1u);
  }
  gd_fold_all<B>(hi, lo, rem, wp, bi, bj, r, bv, ro, R, true);
  __syncthreads();
  double* mine_part = S.part + (size_t)blockIdx.x * np;
  for (int i = tid; i < np; i += kGsThreads) {
    double v = wpart[i];
    for (int w = 1; w < kGsWarps; ++w) v += wpart[w * np + i];
    mine_part[i] = v;
  }
  if (!last_block_to_arrive(S.ticket)) return;
  for (int i = tid; i < r * r; i += kGsThreads) {
    const int a = i / r, b = i - a * r;
    if (b < a) continue;
    const double v = ordered_block_sum(S.part, gridDim.x, np, tri_idx(a, b, r));
    G[a * r + b] = v;
    G[b * r + a] = v;
  }
  rearm_ticket(S.ticket);
}

int gram_ffs_slots(int lda) {
  const int s = kGdRingBytes / (kGdRows * lda * 8);
  return s < 2 ? 2 : (s > kGsSlotsMax ? kGsSlotsMax : s);
}
// ring, the warps' partials, their FP32 remainders, 32 bytes read past them (four
// float pairs at most)
size_t gram_ffs_smem(int r, int lda) {
  return (size_t)kGsWarps * gram_ffs_slots(lda) * kGdRows * lda * 8 +
         (size_t)kGsWarps * (r * (r + 1) / 2) * sizeof(double) + (size_t)kGsWarps * kGdRemMax * 32 * 4 + 32;
}

int gram_stream_slots(int lda) {
  const int s = 12288 / (kGsRows * lda * 4);
  return s < 2 ? 2 : (s > kGsSlotsMax ? kGsSlotsMax : s);
}
size_t gram_stream_smem(int r, int lda) {
  return (size_t)kGsWarps * gram_stream_slots(lda) * kGsRows * lda * 4 +
         (size_t)kGsWarps * (r * (r + 1) / 2) * sizeof(double) + 16;
}

}  // namespace

int gram_rows_stream(const float* A, int64_t n, int r, int lda, double* G, const BlockSums& S, int* status,
                     cudaStream_t st) {
  if (lda == 0) lda = r;
  if (n < 1 || r < 1 || r > kGramStreamMaxRank || lda < r || lda > kMaxRank || !status || ((uintptr_t)A & 15u))
    return CPA_ERR_ARG;
  static std::atomic<unsigned long long> attr{0};
  CPA_CUDA_TRY(set_attr_once(attr, [&] {
    // bound over r <= lda <= kMaxRank: ring <= 16 KB per warp (two slots of 64 floats at
    // least), partials of r <= 32, 16 bytes read past the ring
    const int smax = (int)(kGsWarps * 16384 + kGsWarps * (32 * 33 / 2) * sizeof(double) + 16);
    cudaError_t e = cudaFuncSetAttribute(k_gram_rows_stream<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gram_rows_stream<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  }));
  int64_t grid = kGsGrid;
  const int64_t need = ceil_div(ceil_div(n, (int64_t)kGsRows), (int64_t)kGsWarps);
  if (grid > need) grid = need;
  if (grid > S.max_blocks) grid = S.max_blocks;  // partials of gram_sums_width(r) each
  if (grid < 1) return CPA_ERR_ARG;
  const int slots = gram_stream_slots(lda);
  const size_t smem = gram_stream_smem(r, lda);
  const int nq = (r + 3) / 4;
  if (nq * (nq + 1) / 2 <= 32)
    k_gram_rows_stream<1><<<(unsigned)grid, kGsThreads, smem, st>>>(A, n, r, lda, slots, G, S, status);
  else
    k_gram_rows_stream<2><<<(unsigned)grid, kGsThreads, smem, st>>>(A, n, r, lda, slots, G, S, status);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

bool gram_stream_fp64() {
  const char* e = getenv("CPA_GRAM_STREAM_FP64");  // 0: the one-pair-per-thread kernel
  return !(e && atoi(e) == 0);
}

int gram_rows_stream(const double* A, int64_t n, int r, int lda, double* G, const BlockSums& S, int* status,
                     cudaStream_t st) {
  if (lda == 0) lda = r;
  if (n < 1 || r < 1 || r > kGramStreamFP64MaxRank || lda < r || lda > kMaxRank || !status ||
      ((uintptr_t)A & 15u))
    return CPA_ERR_ARG;
  static std::atomic<unsigned long long> attr{0};
  CPA_CUDA_TRY(set_attr_once(attr, [&] {
    // bound over r <= 32, r <= lda <= kMaxRank: two slots of kMaxRank columns at most
    const int smax = (int)(kGsWarps * 2 * kGdRows * kMaxRank * 8 + kGsWarps * (32 * 33 / 2) * sizeof(double) +
                           kGsWarps * kGdRemMax * 32 * 4 + 32);
    cudaError_t e = cudaFuncSetAttribute(k_gram_rows_ffs<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gram_rows_ffs<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  }));
  // the block size with fewer FP32 instructions per row: B^2 float-pair products
  // (twelve instructions) and 2 B loads per pass of R rows
  auto per_row = [&](int b) {
    const int nb = gd_blocks(r, b);
    if (nb > 32) return 1e30;
    return (double)(12 * b * b + 2 * b) / gd_rows_per_pass(nb);
  };
  const bool five = per_row(5) < per_row(4);
  int64_t grid = kGdGrid;
  const int64_t need = ceil_div(ceil_div(n, (int64_t)kGdRows), (int64_t)kGsWarps);
  if (grid > need) grid = need;
  if (grid > S.max_blocks) grid = S.max_blocks;  // partials of gram_sums_width(r) each
  if (grid < 1) return CPA_ERR_ARG;
  const int slots = gram_ffs_slots(lda);
  const size_t smem = gram_ffs_smem(r, lda);
  if (five)
    k_gram_rows_ffs<5><<<(unsigned)grid, kGsThreads, smem, st>>>(A, n, r, lda, slots, G, S, status);
  else
    k_gram_rows_ffs<4><<<(unsigned)grid, kGsThreads, smem, st>>>(A, n, r, lda, slots, G, S, status);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

}  // namespace cpa
