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

}  // namespace cpa
