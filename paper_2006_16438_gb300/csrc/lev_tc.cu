// Leverage distribution of FP32 factors with many rows (the mixed-precision refresh of
// Alg. 3) on the tensor cores: the factor Gram G = A^T A and the row forms
// y_i = L^{-1} P^T S a_i (Definition 3.4: l_i = ||y_i||^2) as tcgen05 kind::tf32 matrix
// products with the three-product hi/lo split (hi = tf32(x), lo = x - hi; hi.hi + hi.lo
// + lo.hi, about FP32 accuracy), FP32 accumulation in tensor memory.
//
// Both kernels are persistent and stream the factor through shared memory with bulk
// asynchronous copies (cp.async.bulk, completion counted in bytes on an mbarrier per
// ring slot): thread 0 keeps several row tiles in flight per block, the threads turn
// each landed tile into the K-major hi/lo operands, thread 0 issues the MMAs, and the
// copies of later tiles overlap the conversion and the MMAs.  A partial last tile is
// read with plain loads.  Thread 0 does every mbarrier wait (the block barrier that
// follows hands the data to the other threads); every wait is bounded, and on a timeout
// the status word records CPA_ERR_CUDA, the block drains what it issued (bounded
// again), frees its tensor memory and writes nothing more.
//
// k_gram_rows_tc: tiles of 32 rows; each is staged as the operand Y^T (M = the r
// coordinates padded to 128, K = 32 rows); D += Y^T Y (N = 32 or 64) accumulates four
// tiles (128 rows) in FP32, then the r x r partial is read out of tensor memory into a
// float-pair sum in shared memory; the blocks' partials are added in block order.
//
// k_lev_rows_tc: tiles of 128 rows (M = 128, K = N = r padded to 32 or 64);
// F' = L^{-1} P^T S (the pivoted inverse factor with the column scales folded in, so
// the rows need no permutation) is staged once as the B operand; per tile the rows are
// converted (and written out divided by lambda), D = A_tile F'^T lands in tensor memory,
// and in the next round the four warps read D (lane = row) and sum its squares.
#include "dense.cuh"
#include "ffloat.cuh"
#include "tc.cuh"

namespace cpa {

namespace {

// p > 0 ? min(p, 1) : 0 (NaN -> 0), by integer compares of the bit pattern
__device__ __forceinline__ double clamp01_tc(double p) {
  const long long b = __double_as_longlong(p);
  if (b <= 0 || b > 0x7ff0000000000000ll) return 0.0;
  return b < 0x3ff0000000000000ll ? p : 1.0;
}

// The fixed-point sampling weight q = round(2^62 min(l / r, 1)) of an FP32 leverage
// score: f = l (2^62 / r) in FP32 (qscale = 2^62 / r), clamped, converted by integer
// operations (an FP32 value >= 2^23 is an integer: its significand shifted into place).
__device__ __forceinline__ uint64_t q_from_f32(float l, float qscale) {
  const float f = l * qscale;
  if (!(f > 0.f)) return 0;  // zero, negative or NaN
  if (f >= 4611686018427387904.f) return 1ull << 62;
  const uint32_t b = __float_as_uint(f);
  const int e = (int)(b >> 23) - 127;
  if (e < 23) return (uint64_t)__float2uint_rn(f);
  return (uint64_t)((b & 0x7fffffu) | 0x800000u) << (e - 23);
}

// Index of the upper-triangle entry (a, b), a <= b, of an r x r matrix, row-major.
__device__ __forceinline__ int tri_index(int a, int b, int r) { return a * r - a * (a - 1) / 2 + (b - a); }

// Thread 0's record of one ring of bulk copies: which slots have a copy in flight and
// the parity of each slot's next phase.
struct RingState {
  uint32_t pending = 0;
  uint32_t parity = 0;
  __device__ void issued(int s) { pending |= 1u << s; }
  // wait for slot s's copy; false on timeout
  __device__ bool wait(uint64_t* bars, int s) {
    if (!tc::wait_parity(&bars[s], (parity >> s) & 1u)) return false;
    parity ^= 1u << s;
    pending &= ~(1u << s);
    return true;
  }
  // bounded waits for every copy still in flight (after a failure)
  __device__ void drain(uint64_t* bars) {
    for (int s = 0; s < 32; ++s)
      if (pending & (1u << s)) wait(bars, s);
  }
};

// Thread 0's record of the MMA commits (tile u commits on bars[u & 1] as that barrier's
// (u >> 1)-th phase; at most two tiles are outstanding).
struct MmaState {
  int64_t issued = -1;  // last tile whose MMAs were committed
  int64_t done = -1;    // last tile known complete (commits complete in order)
  __device__ bool wait(uint64_t* bars, int64_t u) {
    if (u <= done || u > issued) return true;
    if (!tc::wait_parity(&bars[u & 1], (uint32_t)((u >> 1) & 1))) return false;
    done = u;
    return true;
  }
};

// Rows [row0, row0 + rows) of A (row stride lda floats) into a shared tile of
// `cap` rows with plain loads, zeros past n.
__device__ __forceinline__ void load_partial(float* dst, const float* A, int64_t row0, int64_t n, int lda, int cap,
                                             int tid, int nt) {
  const int64_t have = n - row0;
  const int valid = have <= 0 ? 0 : (have < cap ? (int)have : cap);
  const int total = cap * lda, live = valid * lda;
  const float* src = A + (row0 > 0 ? row0 : 0) * (int64_t)lda;
  for (int e = tid; e < total; e += nt) dst[e] = e < live ? src[e] : 0.f;
}

constexpr int kGramThreads = 256;
constexpr int kGramK = 32;      // rows per tile
constexpr int kGramTiles = 4;   // tiles per readout group (FP32 accumulation over 128 rows)
constexpr int kGramRawMax = 16; // ring slots
constexpr uint32_t kGramSBO = (kGramK / 4) * tc::kLBO;
constexpr uint32_t kGramTileBytes = 128 * kGramK * 4;
constexpr int kGramGrid = 304;  // persistent blocks (two per SM of a GB300; fixed: block-ordered sums)

template <int NC>
__global__ void __launch_bounds__(kGramThreads, 2) k_gram_rows_tc(const float* __restrict__ A, int64_t n, int r,
                                                                  int lda, int nraw, double* __restrict__ G,
                                                                  BlockSums S, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char gtc_raw[];
  __shared__ __align__(8) uint64_t rbar[kGramRawMax];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem;
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw_s = tc::smem_u32(gtc_raw);
  const uint32_t pad = ((raw_s + 1023u) & ~1023u) - raw_s;
  float* op = reinterpret_cast<float*>(gtc_raw + pad);  // [stage][hi, lo] 128 x 32 operand tiles
  const uint32_t op_s = raw_s + pad;
  const int tile_f = kGramK * lda;                            // floats of one row tile
  float* ring = op + 4 * (kGramTileBytes / 4);                // nraw row tiles
  float* gh = ring + (size_t)nraw * tile_f;                   // r x r float-pair partial: hi
  float* gl = gh + r * r;                                     // lo
  const int64_t ngroups = (n + kGramK * kGramTiles - 1) / (kGramK * kGramTiles);
  const int64_t T = blockIdx.x < ngroups ? kGramTiles * ((ngroups - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  auto row0_of = [&](int64_t t) {
    return ((int64_t)blockIdx.x + (t / kGramTiles) * gridDim.x) * (kGramK * kGramTiles) + (t % kGramTiles) * kGramK;
  };
  for (int i = tid; i < (int)(4 * kGramTileBytes / 16); i += kGramThreads)
    reinterpret_cast<float4*>(op)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = tid; i < r * r; i += kGramThreads) gh[i] = gl[i] = 0.f;
  if (tid == 0) {
    for (int s = 0; s < nraw; ++s) tc::mbar_init(&rbar[s]);
    tc::mbar_init(&mbar[0]);
    tc::mbar_init(&mbar[1]);
    tc::fence_mbar_init();
    s_bad = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem, NC);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t d = tmem;
  const uint32_t idesc = tc::idesc_tf32(NC);
  const uint32_t tile_bytes = (uint32_t)tile_f * 4u;
  RingState ring_st;
  MmaState mma_st;
  if (tid == 0)
    for (int s = 0; s < nraw && s < T; ++s) {
      const int64_t r0 = row0_of(s);
      if (r0 + kGramK <= n) {
        tc::mbar_expect_tx(&rbar[s], tile_bytes);
        tc::bulk_g2s(ring + (size_t)s * tile_f, A + r0 * lda, tile_bytes, &rbar[s]);
        ring_st.issued(s);
      }
    }
  int bad = 0;
  for (int64_t t = 0; t <= T; ++t) {
    const bool have = t < T;
    const int s = (int)(t % nraw);
    float* rw = ring + (size_t)s * tile_f;
    const int64_t r0 = have ? row0_of(t) : 0;
    const bool full = have && r0 + kGramK <= n;
    const bool readout = (t % kGramTiles == 0 && t >= kGramTiles) || (t == T && T > 0);
    // phase 1: the tile's copy has landed, its operand stage is free (MMA t - 2), and
    // before a readout the previous group's MMAs are complete
    if (tid == 0 && !bad) {
      bool ok = true;
      if (full) ok = ring_st.wait(rbar, s);
      if (ok && t >= 2) ok = mma_st.wait(mbar, t - 2);
      if (ok && readout) ok = mma_st.wait(mbar, t - 1);
      if (!ok) s_bad = 1;
    }
    if (have && !full && !bad) load_partial(rw, A, r0, n, lda, kGramK, tid, kGramThreads);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    bad = s_bad;
    // phase 2: read out the finished group; stage the tile as Y^T (hi, lo)
    if (!bad) {
      if (readout) {
        const int qw = warp & 3, half = warp >> 2;  // lanes 32 qw ..: coordinates; half: columns
        if (32 * qw < r && 32 * qw < NC) {
#pragma unroll
          for (int cc = 0; cc < NC / 32; ++cc) {
            uint32_t v[16];
            tc::tmem_ld16(d + ((uint32_t)(32 * qw) << 16) + (uint32_t)(cc * 32 + half * 16), v);
            const int row = 32 * qw + lane;
            if (row < r) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const int col = cc * 32 + half * 16 + jj;
                if (col < r) {
                  float sh, se;
                  two_sum(gh[row * r + col], __uint_as_float(v[jj]), sh, se);
                  gh[row * r + col] = sh;
                  gl[row * r + col] += se;
                }
              }
            }
          }
        }
      }
      if (have) {
        float* hi = op + (size_t)(2 * (t & 1)) * (kGramTileBytes / 4);
        float* lo = hi + kGramTileBytes / 4;
        // unit (coordinate c, rows 4 rq .. 4 rq + 3): one 16-byte store per half
        for (int u = tid; u < NC * (kGramK / 4); u += kGramThreads) {
          const int c8 = u & 7, rq = (u >> 3) & (kGramK / 4 - 1), cg = u / (8 * (kGramK / 4));
          const int c = cg * 8 + c8;
          float x[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) x[i] = c < r ? rw[(4 * rq + i) * lda + c] : 0.f;
          float4 h4, l4;
          h4.x = tc::to_tf32(x[0]);
          h4.y = tc::to_tf32(x[1]);
          h4.z = tc::to_tf32(x[2]);
          h4.w = tc::to_tf32(x[3]);
          l4 = make_float4(x[0] - h4.x, x[1] - h4.y, x[2] - h4.z, x[3] - h4.w);
          const uint32_t off = tc::kmajor_off(c, 4 * rq, kGramSBO);
          *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(hi) + off) = h4;
          *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(lo) + off) = l4;
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    // phase 3: the tile's MMAs; the copy of the tile nraw places ahead into this slot
    if (tid == 0 && have && !bad) {
      const uint32_t hs = op_s + (uint32_t)(2 * (t & 1)) * kGramTileBytes, ls = hs + kGramTileBytes;
#pragma unroll
      for (int ks = 0; ks < kGramK / 8; ++ks) {
        const uint32_t ko = (uint32_t)ks * 2u * tc::kLBO;  // 8 rows = two core matrices along K
        const uint64_t ah = tc::desc(hs + ko, kGramSBO), al = tc::desc(ls + ko, kGramSBO);
        tc::mma_tf32(d, ah, ah, idesc, ((t % kGramTiles) | ks) != 0);  // a new group starts from zero
        tc::mma_tf32(d, ah, al, idesc, 1u);
        tc::mma_tf32(d, al, ah, idesc, 1u);
      }
      tc::commit(&mbar[t & 1]);
      mma_st.issued = t;
      const int64_t tn = t + nraw;
      if (tn < T) {
        const int64_t rn = row0_of(tn);
        if (rn + kGramK <= n) {
          tc::fence_async_smem();
          tc::mbar_expect_tx(&rbar[s], tile_bytes);
          tc::bulk_g2s(rw, A + rn * lda, tile_bytes, &rbar[s]);
          ring_st.issued(s);
        }
      }
    }
  }
  if (tid == 0 && bad) {
    atomicCAS(status, 0, CPA_ERR_CUDA);
    ring_st.drain(rbar);
    mma_st.wait(mbar, mma_st.issued);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(d, NC);
  // the block's upper triangle (after a failure too: the ticket protocol stays whole), then the blocks' partials in block order (G symmetric)
  const int np = r * (r + 1) / 2;
  double* mine = S.part + (size_t)blockIdx.x * np;
  for (int i = tid; i < r * r; i += kGramThreads) {
    const int a = i / r, b = i - a * r;
    if (b >= a) mine[tri_index(a, b, r)] = (double)gh[i] + (double)gl[i];
  }
  if (!last_block_to_arrive(S.ticket)) return;
  for (int i = tid; i < r * r; i += kGramThreads) {
    const int a = i / r, b = i - a * r;
    if (b < a) continue;
    const double v = ordered_block_sum(S.part, gridDim.x, np, tri_index(a, b, r));
    G[a * r + b] = v;
    G[b * r + a] = v;
  }
  rearm_ticket(S.ticket);
}

constexpr int kLevThreads = 128;  // four warps: thread = row of a 128-row tile
constexpr int kLevRawMax = 6;     // ring slots

// NC: N = K = r padded to 32 or 64.
template <int NC>
__global__ void __launch_bounds__(kLevThreads) k_lev_rows_tc(const float* __restrict__ A, int64_t n, int r, int lda,
                                                             int nraw, const SmallFactor* __restrict__ f,
                                                             double* __restrict__ lev, uint64_t* __restrict__ q,
                                                             DistInfo* info, float* A_out, float qscale,
                                                             int* __restrict__ status) {
  constexpr uint32_t kSBO_A = (NC / 4) * tc::kLBO;  // 8-row groups of a 128 x NC tile
  constexpr uint32_t kTileA = 128 * NC * 4;
  constexpr uint32_t kTileB = NC * NC * 4;
  extern __shared__ __align__(16) unsigned char ltc_raw[];
  __shared__ __align__(8) uint64_t rbar[kLevRawMax];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem;
  __shared__ int s_bad;
  __shared__ float ilam[kMaxRank];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (f->kind != 0) {  // a pseudo-inverse factor (not produced by the pivoted refresh): FP64 loop
    const double* F = f->F;
    for (int64_t row = (int64_t)blockIdx.x * kLevThreads + tid; row < n; row += (int64_t)gridDim.x * kLevThreads) {
      double l = 0.0;
      for (int c = 0; c < r; ++c) {
        double tsum = 0.0;
        for (int u = 0; u < r; ++u) tsum += F[c * r + u] * f->scale[u] * (double)A[row * lda + u];
        l += f->scale[c] * (double)A[row * lda + c] * tsum;
      }
      if (lev) lev[row] = l;
      if (q) {
        const uint64_t qi = __double2ull_rn(clamp01_tc(l / (double)r) * 4611686018427387904.0);
        q[row] = qi;
        atomicMax((unsigned long long*)&info->maxq, (unsigned long long)qi);
        if (qi) atomicAdd((unsigned long long*)&info->nnzq, 1ull);
      }
      if (A_out) {
        float x[kMaxRank];
        for (int c = 0; c < r; ++c) x[c] = A[row * lda + c];
        for (int c = 0; c < r; ++c) {
          const double lm = f->lambda[c];
          A_out[row * r + c] = x[c] * (pos_finite(lm) ? (float)(1.0 / lm) : 1.f);
        }
      }
    }
    return;
  }
  const uint32_t raw_s = tc::smem_u32(ltc_raw);
  const uint32_t pad = ((raw_s + 1023u) & ~1023u) - raw_s;
  unsigned char* base = ltc_raw + pad;
  const uint32_t base_s = raw_s + pad;
  // [hi, lo] 128 x NC operand tiles at base, then
  float* tB = reinterpret_cast<float*>(base + 2 * kTileA);  // [hi, lo] NC x NC
  float* ring = reinterpret_cast<float*>(base + 2 * kTileA + 2 * kTileB);  // nraw tiles of 128 rows
  const uint32_t tA_s = base_s, tB_s = base_s + 2 * kTileA;
  const int tile_f = 128 * lda;
  for (int i = tid; i < (int)((2 * kTileA + 2 * kTileB) / 16); i += kLevThreads)
    reinterpret_cast<float4*>(base)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  // F'(c, perm[u]) = F(c, u) scale(perm[u]): rows c >= rank are zero in F
  for (int i = tid; i < r * r; i += kLevThreads) {
    const int c = i / r, u = i - c * r;
    const int v = f->perm[u];
    const float x = (float)(f->F[i] * f->scale[v]);
    const float h = tc::to_tf32(x);
    const uint32_t off = tc::kmajor_off(c, v, kSBO_A);  // N x K tile: the same strides as A
    tB[off >> 2] = h;
    tB[(kTileB + off) >> 2] = x - h;
  }
  for (int i = tid; i < r; i += kLevThreads) {
    const double l = f->lambda[i];
    ilam[i] = pos_finite(l) ? (float)(1.0 / l) : 1.f;
  }
  if (tid == 0) {
    for (int s = 0; s < nraw; ++s) tc::mbar_init(&rbar[s]);
    tc::mbar_init(&mbar[0]);
    tc::mbar_init(&mbar[1]);
    tc::fence_mbar_init();
    s_bad = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem, NC);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t d = tmem;
  const uint32_t idesc = tc::idesc_tf32(NC);
  const uint32_t tile_bytes = (uint32_t)tile_f * 4u;
  const int64_t ntiles = (n + 127) / 128;
  const int64_t T = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto row0_of = [&](int64_t t) { return ((int64_t)blockIdx.x + t * gridDim.x) * 128; };
  RingState ring_st;
  MmaState mma_st;
  if (tid == 0)
    for (int s = 0; s < nraw && s < T; ++s) {
      const int64_t r0 = row0_of(s);
      if (r0 + 128 <= n) {
        tc::mbar_expect_tx(&rbar[s], tile_bytes);
        tc::bulk_g2s(ring + (size_t)s * tile_f, A + r0 * lda, tile_bytes, &rbar[s]);
        ring_st.issued(s);
      }
    }
  uint64_t my_max = 0;
  uint32_t my_nz = 0;
  const bool vec = (lda & 3) == 0;  // rows start on 16 bytes in the ring
  int bad = 0;
  for (int64_t t = 0; t <= T; ++t) {
    const bool have = t < T;
    const int s = (int)(t % nraw);
    float* rw = ring + (size_t)s * tile_f;
    const int64_t r0 = have ? row0_of(t) : 0;
    const bool full = have && r0 + 128 <= n;
    // phase 1: the tile's copy has landed and the previous tile's MMAs are complete
    // (its result is read below, and the operand tile is rewritten)
    if (tid == 0 && !bad) {
      bool ok = true;
      if (full) ok = ring_st.wait(rbar, s);
      if (ok && t >= 1) ok = mma_st.wait(mbar, t - 1);
      if (!ok) s_bad = 1;
    }
    if (have && !full && !bad) load_partial(rw, A, r0, n, lda, 128, tid, kLevThreads);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    bad = s_bad;
    // phase 2: l of the previous tile's rows; this tile's rows into the operand
    if (!bad) {
      if (t >= 1) {
        float l = 0.f;
#pragma unroll
        for (int cc = 0; cc < NC / 32; ++cc) {
          uint32_t v[32];
          tc::tmem_ld32(d + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const float y = __uint_as_float(v[jj]);
            l = fmaf(y, y, l);
          }
        }
        const int64_t row = row0_of(t - 1) + tid;
        if (row < n) {
          if (lev) lev[row] = (double)l;
          if (q) {
            const uint64_t qi = q_from_f32(l, qscale);
            q[row] = qi;
            my_max = qi > my_max ? qi : my_max;
            my_nz += qi > 0;
          }
        }
      }
      if (have) {
        const float* src = rw + tid * lda;  // this thread's row
#pragma unroll
        for (int c0 = 0; c0 < NC; c0 += 4) {
          float x[4];
          if (vec && c0 < lda) {
            const float4 v4 = *reinterpret_cast<const float4*>(src + c0);
            x[0] = v4.x;
            x[1] = v4.y;
            x[2] = v4.z;
            x[3] = v4.w;
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (c0 + i >= r) x[i] = 0.f;
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = c0 + i < r ? src[c0 + i] : 0.f;
          }
          float4 h4, l4;
          h4.x = tc::to_tf32(x[0]);
          h4.y = tc::to_tf32(x[1]);
          h4.z = tc::to_tf32(x[2]);
          h4.w = tc::to_tf32(x[3]);
          l4 = make_float4(x[0] - h4.x, x[1] - h4.y, x[2] - h4.z, x[3] - h4.w);
          const uint32_t off = tc::kmajor_off(tid, c0, kSBO_A);
          *reinterpret_cast<float4*>(base + off) = h4;
          *reinterpret_cast<float4*>(base + kTileA + off) = l4;
        }
        if (A_out) {  // the rows divided by lambda, coalesced: element e = rr r + c
          const int64_t left = n - r0;
          const int rows = left < 128 ? (int)left : 128;
          float* dst = A_out + r0 * r;
          const int step_r = kLevThreads / r, step_c = kLevThreads - step_r * r;
          int rr = tid / r, c = tid - rr * r;
          for (int e = tid; e < rows * r; e += kLevThreads) {
            dst[e] = rw[rr * lda + c] * ilam[c];
            rr += step_r;
            c += step_c;
            if (c >= r) {
              c -= r;
              ++rr;
            }
          }
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    // phase 3: the tile's MMAs; the copy of the tile nraw places ahead into this slot
    if (tid == 0 && have && !bad) {
      const uint32_t hs = tA_s, ls = tA_s + kTileA;
      const uint32_t bh = tB_s, bl = tB_s + kTileB;
#pragma unroll
      for (int ks = 0; ks < NC / 8; ++ks) {
        const uint32_t ko = (uint32_t)ks * 2u * tc::kLBO;
        const uint64_t ah = tc::desc(hs + ko, kSBO_A), al = tc::desc(ls + ko, kSBO_A);
        const uint64_t bhd = tc::desc(bh + ko, kSBO_A), bld = tc::desc(bl + ko, kSBO_A);
        tc::mma_tf32(d, ah, bhd, idesc, ks != 0);
        tc::mma_tf32(d, ah, bld, idesc, 1u);
        tc::mma_tf32(d, al, bhd, idesc, 1u);
      }
      tc::commit(&mbar[t & 1]);
      mma_st.issued = t;
      const int64_t tn = t + nraw;
      if (tn < T) {
        const int64_t rn = row0_of(tn);
        if (rn + 128 <= n) {
          tc::fence_async_smem();
          tc::mbar_expect_tx(&rbar[s], tile_bytes);
          tc::bulk_g2s(rw, A + rn * lda, tile_bytes, &rbar[s]);
          ring_st.issued(s);
        }
      }
    }
  }
  if (tid == 0 && bad) {
    atomicCAS(status, 0, CPA_ERR_CUDA);
    ring_st.drain(rbar);
    mma_st.wait(mbar, mma_st.issued);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(d, NC);
  if (q && info && !bad) {
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t om = __shfl_xor_sync(0xffffffffu, my_max, o);
      my_max = om > my_max ? om : my_max;
      my_nz += __shfl_xor_sync(0xffffffffu, my_nz, o);
    }
    if (lane == 0) {
      atomicMax((unsigned long long*)&info->maxq, (unsigned long long)my_max);
      atomicAdd((unsigned long long*)&info->nnzq, (unsigned long long)my_nz);
    }
  }
}

// Ring slots of the Gram kernel for a row stride of lda floats: about 36 KB of row
// tiles in flight per block, two blocks per SM.
int gram_ring_slots(int lda) {
  const int s = 36864 / (kGramK * lda * 4);
  return s < 2 ? 2 : (s > kGramRawMax ? kGramRawMax : s);
}
size_t gram_smem_bytes(int r, int lda) {
  return 1024 + 4 * (size_t)kGramTileBytes + (size_t)gram_ring_slots(lda) * kGramK * lda * 4 +
         2 * sizeof(float) * (size_t)r * r;
}
// Ring slots of the leverage kernel: about 64 KB of row tiles in flight per block.
int lev_ring_slots(int lda) {
  const int s = 65536 / (128 * lda * 4);
  return s < 2 ? 2 : (s > kLevRawMax ? kLevRawMax : s);
}
size_t lev_smem_bytes(int nc, int lda) {
  return 1024 + 2 * (size_t)128 * nc * 4 + 2 * (size_t)nc * nc * 4 + (size_t)lev_ring_slots(lda) * 128 * lda * 4;
}

}  // namespace

bool lev_tensor_cores() {
  const char* e = getenv("CPA_LEV_FLOAT_PAIR");  // 1: the float-pair kernels instead
  return !(e && atoi(e) != 0);
}

bool gram_tensor_cores() {
  const char* e = getenv("CPA_GRAM_TC");
  return e && atoi(e) != 0;
}

bool tc_rows_ok(const float* A, int r, int lda) {
  return r >= 1 && r <= kMaxRank && (lda == 0 || lda >= r) && ((uintptr_t)A & 15u) == 0;
}

int gram_rows_tc(const float* A, int64_t n, int r, int lda, double* G, const BlockSums& S, int* status,
                 cudaStream_t st) {
  if (lda == 0) lda = r;
  if (n < 1 || !tc_rows_ok(A, r, lda) || lda > kMaxRank || !status) return CPA_ERR_ARG;
  static std::atomic<unsigned long long> attr{0};
  CPA_CUDA_TRY(set_attr_once(attr, [&] {
    // bound over all r <= lda <= kMaxRank: ring <= 36 KB, float-pair partial <= 2 kMaxRank^2 floats
    const int smax = (int)(1024 + 4 * (size_t)kGramTileBytes + 36864 + 2 * sizeof(float) * kMaxRank * kMaxRank);
    cudaError_t e = cudaFuncSetAttribute(k_gram_rows_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gram_rows_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  }));
  const int64_t groups = ceil_div(n, (int64_t)kGramK * kGramTiles);
  int64_t grid = groups < kGramGrid ? groups : kGramGrid;
  if (grid > S.max_blocks) grid = S.max_blocks;  // partials of gram_sums_width(r) each
  if (grid < 1) return CPA_ERR_ARG;
  const int nraw = gram_ring_slots(lda);
  const size_t smem = gram_smem_bytes(r, lda);
  if (r <= 32)
    k_gram_rows_tc<32><<<(unsigned)grid, kGramThreads, smem, st>>>(A, n, r, lda, nraw, G, S, status);
  else
    k_gram_rows_tc<64><<<(unsigned)grid, kGramThreads, smem, st>>>(A, n, r, lda, nraw, G, S, status);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

int lev_rows_tc(const float* A, int64_t n, int r, int lda, const SmallFactor* f, double* lev, uint64_t* q,
                DistInfo* info, float* A_out, int* status, cudaStream_t st) {
  if (lda == 0) lda = r;
  if (n < 1 || !tc_rows_ok(A, r, lda) || lda > kMaxRank || !status) return CPA_ERR_ARG;
  static std::atomic<unsigned long long> attr{0};
  CPA_CUDA_TRY(set_attr_once(attr, [&] {
    cudaError_t e = cudaFuncSetAttribute(k_lev_rows_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)lev_smem_bytes(32, 32));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_lev_rows_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)lev_smem_bytes(64, kMaxRank));
  }));
  const int64_t ntiles = ceil_div(n, (int64_t)128);
  const int64_t cap = (int64_t)num_sms() * 2;
  const unsigned grid = (unsigned)(ntiles < cap ? ntiles : cap);
  const int nraw = lev_ring_slots(lda);
  const float qscale = (float)(4611686018427387904.0 / r);
  if (r <= 32)
    k_lev_rows_tc<32><<<grid, kLevThreads, lev_smem_bytes(32, lda), st>>>(A, n, r, lda, nraw, f, lev, q, info,
                                                                          A_out, qscale, status);
  else
    k_lev_rows_tc<64><<<grid, kLevThreads, lev_smem_bytes(64, lda), st>>>(A, n, r, lda, nraw, f, lev, q, info,
                                                                          A_out, qscale, status);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

}  // namespace cpa
