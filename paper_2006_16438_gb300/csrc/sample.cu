// SkrpLev (Alg. 1) on the GPU.
//
// Readings shared with the oracle (they fix every bit of the output):
//  * mode t row i has probability p_t(i) = q_i / T_t, q from the fixed-point CDF;
//  * p of a multi-index = p_0(i_0) * p_1(i_1) * ... in ascending mode order;
//  * deterministic iff p > tau; a random draw is accepted iff p <= tau;
//  * slot j, attempt a draws Philox4x64-10 with counter
//    (j, a, mode_k | (t/4) << 16 | 1 << 32, iter) and key (seed, 0); other mode t
//    takes word t % 4 as u and the row min{i : C_i > floor(u T / 2^64)};
//  * p_det is the correctly rounded sum of the deterministic p (order free);
//  * combined weight sqrt(c (1 - p_det) / (p s_rnd)) (Eq. 4.4 with s_rnd, Alg. 2);
//  * output: deterministic keys ascending, then distinct random keys ascending.
// All FP64 steps use explicit round-to-nearest intrinsics so that no contraction
// can change them.
#include "sample.cuh"

namespace cpa {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double mode_prob_from_cdf(const uint64_t* __restrict__ C, uint64_t T,
                                                     int64_t i) {
  const uint64_t q = C[i] - (i > 0 ? C[i - 1] : 0ull);
  return __ddiv_rn(__ull2double_rn(q), __ull2double_rn(T));
}

__global__ void k_phat(const uint64_t* __restrict__ C, int64_t n, const DistInfo* __restrict__ info,
                       double* __restrict__ p) {
  const uint64_t T = info->T;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = mode_prob_from_cdf(C, T, i);
}

// smallest i with C[i] > t (C inclusive, C[n-1] = T > t)
__device__ __forceinline__ int64_t cdf_search(const uint64_t* __restrict__ C, int64_t n, uint64_t t) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (C[mid] > t) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// probability of a packed multi-index
__device__ __forceinline__ double key_prob(const SampleParams& P, uint64_t packed) {
  double p = 0.0;
  for (int t = 0; t < P.L.d; ++t) {
    const double pt = P.D.P[t][P.L.get(packed, t)];
    p = t == 0 ? pt : __dmul_rn(p, pt);
  }
  return p;
}

// ---- exact sum of positive doubles --------------------------------------
// Each term m * 2^(e) is added as 32-bit chunks into integer bins whose unit is
// 2^-1074; the bins are later carried and rounded once (ties to even).
__device__ __forceinline__ void xs_add(uint64_t* bins, double v) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const int bexp = (int)((bits >> 52) & 0x7ff);
  uint64_t mant = bits & ((1ull << 52) - 1ull);
  int shift = 0;
  if (bexp != 0) {
    mant |= 1ull << 52;
    shift = bexp - 1;
  }
  const int limb = shift >> 5, off = shift & 31;
  const uint64_t lo = mant << off;
  const uint64_t hi = off ? (mant >> (64 - off)) : 0ull;
  atomicAdd((unsigned long long*)&bins[limb], (unsigned long long)(lo & 0xffffffffull));
  atomicAdd((unsigned long long*)&bins[limb + 1], (unsigned long long)(lo >> 32));
  if (hi) atomicAdd((unsigned long long*)&bins[limb + 2], (unsigned long long)hi);
}

// The three 32-bit chunks of v (as in xs_add) and the limb of the first one.
__device__ __forceinline__ int xs_parts(double v, uint64_t* c0, uint64_t* c1, uint64_t* c2) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const int bexp = (int)((bits >> 52) & 0x7ff);
  uint64_t mant = bits & ((1ull << 52) - 1ull);
  int shift = 0;
  if (bexp != 0) {
    mant |= 1ull << 52;
    shift = bexp - 1;
  }
  const int off = shift & 31;
  const uint64_t lo = mant << off;
  *c0 = lo & 0xffffffffull;
  *c1 = lo >> 32;
  *c2 = off ? (mant >> (64 - off)) : 0ull;
  return shift >> 5;
}

// Per-thread accumulation of exact-sum chunks in a three-limb window at the limb of
// the thread's first term (terms elsewhere go straight to the bins), merged across
// the warp before touching the shared bins: lanes with the same window reduce each
// chunk sum in 16-bit pieces (exact), and one lane adds the result.
struct XsWindow {
  int base = -1;
  uint64_t w0 = 0, w1 = 0, w2 = 0;
  __device__ __forceinline__ void add(uint64_t* bins, double v) {
    uint64_t c0, c1, c2;
    const int limb = xs_parts(v, &c0, &c1, &c2);
    if (base < 0) base = limb;
    if (limb == base) {
      w0 += c0;
      w1 += c1;
      w2 += c2;
    } else {
      atomicAdd((unsigned long long*)&bins[limb], (unsigned long long)c0);
      atomicAdd((unsigned long long*)&bins[limb + 1], (unsigned long long)c1);
      if (c2) atomicAdd((unsigned long long*)&bins[limb + 2], (unsigned long long)c2);
    }
  }
  // all 32 lanes call this
  __device__ __forceinline__ void flush(uint64_t* bins) {
    const unsigned grp = __match_any_sync(0xffffffffu, base);
    const int lane = threadIdx.x & 31;
    const uint64_t wv[3] = {w0, w1, w2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint64_t tot = 0;
#pragma unroll
      for (int piece = 0; piece < 4; ++piece) {
        const unsigned part = (unsigned)((wv[k] >> (16 * piece)) & 0xffffu);
        tot += (uint64_t)__reduce_add_sync(grp, part) << (16 * piece);
      }
      if (base >= 0 && lane == __ffs(grp) - 1 && tot)
        atomicAdd((unsigned long long*)&bins[base + k], (unsigned long long)tot);
    }
  }
};

// bits [pos, pos + 64) of the little-endian limb array (missing bits read 0)
__device__ __forceinline__ uint64_t bits64(const uint32_t* w, int nlimbs, int pos) {
  uint64_t v = 0;
  for (int k = 0; k < 3; ++k) {  // the window touches at most three limbs
    const int lb = pos >= 0 ? (pos >> 5) + k : -((-pos + 31) >> 5) + k;
    if (lb < 0 || lb >= nlimbs) continue;
    const int shift = lb * 32 - pos;  // position of limb lb inside the window
    const uint64_t limb = w[lb];
    if (shift >= 64 || shift <= -32) continue;
    v |= shift >= 0 ? (limb << shift) : (limb >> -shift);
  }
  return v;
}

// any bit set below position pos
__device__ __forceinline__ bool any_below(const uint32_t* w, int pos) {
  if (pos <= 0) return false;
  const int full = pos >> 5, rem = pos & 31;
  for (int i = 0; i < full; ++i)
    if (w[i]) return true;
  return rem ? (w[full] & ((1u << rem) - 1u)) != 0 : false;
}

// bins_in: kXsRep replicas of kXsLimbs bins, added limb by limb (integer, exact)
__device__ double xs_round(const uint64_t* bins_in) {
  constexpr int kL = kXsLimbs + 2;
  uint32_t w[kL];
  uint64_t carry = 0;
  for (int i = 0; i < kXsLimbs; ++i) {
    uint64_t v = carry;
    for (int rr = 0; rr < kXsRep; ++rr) v += bins_in[rr * kXsLimbs + i];
    w[i] = (uint32_t)v;
    carry = v >> 32;
  }
  w[kXsLimbs] = (uint32_t)carry;
  w[kXsLimbs + 1] = (uint32_t)(carry >> 32);
  int top = -1;
  for (int i = kL - 1; i >= 0; --i)
    if (w[i]) {
      top = i * 32 + 31 - __clz(w[i]);
      break;
    }
  if (top < 0) return 0.0;
  if (top < 53) {  // below 2^-1021: the integer itself is the IEEE bit pattern
    return __longlong_as_double((long long)bits64(w, kL, 0));
  }
  // 64-bit window whose top bit is `top`: 53 kept bits, the round bit, 10 more
  const uint64_t win = bits64(w, kL, top - 63);
  uint64_t m = win >> 11;
  const bool round_bit = (win >> 10) & 1ull;
  const bool sticky = (win & 0x3ffull) != 0 || any_below(w, top - 63);
  if (round_bit && (sticky || (m & 1ull))) ++m;
  uint64_t bexp = (uint64_t)(top - 51);
  if (m == (1ull << 53)) {
    m >>= 1;
    ++bexp;
  }
  return __longlong_as_double((long long)((bexp << 52) | (m & ((1ull << 52) - 1ull))));
}

// ---- combine table -------------------------------------------------------
// CombineRepeats counts the repeats of each drawn key in an open-addressing table
// (linear probing, 2^hbits >= 2 s slots); deterministic keys go in with their flag
// bit clear, random ones with it set, so the two never merge.
constexpr uint64_t kEmptyKey = ~0ull;

__device__ __forceinline__ uint64_t slot_of(uint64_t key, int hbits) {
  return (key * 0x9E3779B97F4A7C15ull) >> (64 - hbits);
}

__device__ __forceinline__ bool table_add(uint64_t* __restrict__ keys, uint32_t* __restrict__ cnt,
                                          int hbits, uint64_t key) {
  const uint64_t mask = (1ull << hbits) - 1ull;
  uint64_t h = slot_of(key, hbits);
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const unsigned long long prev =
        atomicCAS((unsigned long long*)&keys[h], (unsigned long long)kEmptyKey, (unsigned long long)key);
    if (prev == kEmptyKey || prev == key) {
      atomicAdd(&cnt[h], 1u);
      return true;
    }
    h = (h + 1) & mask;
  }
  return false;
}

__device__ __forceinline__ uint32_t table_count(const uint64_t* __restrict__ keys,
                                                const uint32_t* __restrict__ cnt, int hbits,
                                                uint64_t key) {
  const uint64_t mask = (1ull << hbits) - 1ull;
  uint64_t h = slot_of(key, hbits);
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const uint64_t k = keys[h];
    if (k == key) return cnt[h];
    if (k == kEmptyKey) return 0;
    h = (h + 1) & mask;
  }
  return 0;
}

// weight of a combined row (Eq. 4.4 with s_rnd) or 1 for a deterministic row
__device__ __forceinline__ double row_weight(const SampleParams& P, uint64_t packed, bool det, uint64_t c,
                                             double one_minus_pdet, int64_t srnd) {
  if (det) return 1.0;
  const double p = key_prob(P, packed);
  return __dsqrt_rn(__ddiv_rn(__dmul_rn(__ull2double_rn(c), one_minus_pdet),
                              __dmul_rn(p, __ll2double_rn(srnd))));
}

// ---- kernels ----------------------------------------------------------
// One warp: scalars cleared, alpha_t = max_i p_t(i) for every other mode t (lane t),
// alpha_* = their product in mode order, candidate thresholds
// thr_t = (tau alpha_t / alpha_*) (1 - 2^-40).
__global__ void k_prepare(SampleParams P, SampleState* S) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int t = threadIdx.x;
  for (int i = t; i < kXsRep * kXsLimbs; i += 32) S->xs[i] = 0;
  if (t < kMaxOrder) S->ncand[t] = 0;
  double alpha = 1.0;
  if (t < P.L.d) {
    const DistInfo* I = P.D.info[t];
    alpha = __ddiv_rn(__ull2double_rn(I->maxq), __ull2double_rn(I->T));
    // a distribution without mass (all-zero factor) cannot be drawn from: fail now
    // rather than after reject_cap attempts of every slot
    if (I->T == 0) set_status(&S->status, CPA_ERR_REJECT_LIMIT);
  }
  double astar = 0.0;
  for (int u = 0; u < P.L.d; ++u) {
    const double au = __shfl_sync(0xffffffffu, alpha, u);
    astar = u == 0 ? au : __dmul_rn(astar, au);
  }
  const double slack = 1.0 - 0x1p-40;
  if (t < P.L.d) S->thr[t] = __dmul_rn(__ddiv_rn(__dmul_rn(P.tau, alpha), astar), slack);
  if (t == 0) {
    // S->status is sticky across passes: the caller zeroes it once
    S->need_topk = 0;
    S->cand_total = 0;
    S->det_count = 0;
    S->sdet = 0;
    S->srnd = 0;
    S->nsort = 0;
    S->sbar = 0;
    S->nuniq = 0;
    S->attempts = 0;
    S->slot_ctr = 0;
    S->pdet = 0.0;
    S->alpha_star = astar;
    S->no_det = !(pos_finite(astar) && nonneg_gt(astar, P.tau));
  }
}

// candidates of every other mode: p_t(i) >= thr_t (unordered)
__global__ void k_det_filter(SampleParams P, SampleState* S, uint32_t* __restrict__ cand,
                             int64_t off1, int64_t off2, int64_t off3, int64_t off4, int64_t off5,
                             int64_t off6, int64_t total) {
  if (S->no_det) return;
  const int64_t offs[kMaxOrder] = {0, off1, off2, off3, off4, off5, off6, total};
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int t = 0;
    while (t + 1 < P.L.d && g >= offs[t + 1]) ++t;
    const int64_t i = g - offs[t];
    const double p = P.D.P[t][i];
    if (!nonneg_gt(S->thr[t], p)) {  // p >= thr
      const unsigned long long at = atomicAdd((unsigned long long*)&S->ncand[t], 1ull);
      cand[offs[t] + (int64_t)at] = (uint32_t)i;
    }
  }
}

// enumerate the candidate product; keep p > tau
__global__ void k_det_enum(SampleParams P, SampleState* S, const uint32_t* __restrict__ cand,
                           int64_t off1, int64_t off2, int64_t off3, int64_t off4, int64_t off5,
                           int64_t off6, uint64_t* __restrict__ det_keys, double* __restrict__ det_p) {
  __shared__ uint64_t bins[kXsLimbs];
  __shared__ int any;
  if (S->no_det) return;
  // size of the candidate product (every block computes it; block 0 records it)
  int64_t nc[kMaxOrder];
  double prod = 1.0;
  uint64_t total = 1;
  for (int t = 0; t < P.L.d; ++t) {
    nc[t] = S->ncand[t];
    prod *= (double)nc[t];
    total *= (uint64_t)nc[t];
  }
  if (prod > (double)P.det_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(&S->status, CPA_ERR_DET_CAP);
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) S->cand_total = total;
  for (int i = threadIdx.x; i < kXsLimbs; i += blockDim.x) bins[i] = 0;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int64_t offs[kMaxOrder] = {0, off1, off2, off3, off4, off5, off6, 0};
  const bool narrow = total < (1ull << 32);  // 32-bit division (64-bit is emulated)
  XsWindow win;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t rest = e, packed = 0;
    uint32_t rest32 = (uint32_t)e;
    double p = 0.0;
    for (int t = 0; t < P.L.d; ++t) {
      uint64_t pos;
      if (narrow) {
        const uint32_t q = rest32 / (uint32_t)nc[t];
        pos = rest32 - q * (uint32_t)nc[t];
        rest32 = q;
      } else {
        pos = rest % (uint64_t)nc[t];
        rest /= (uint64_t)nc[t];
      }
      const uint32_t i = cand[offs[t] + (int64_t)pos];
      const double pt = P.D.P[t][i];
      p = t == 0 ? pt : __dmul_rn(p, pt);
      packed |= (uint64_t)i << P.L.off[t];
    }
    if (nonneg_gt(p, P.tau)) {  // p > tau
      const unsigned long long at = atomicAdd((unsigned long long*)&S->det_count, 1ull);
      if ((int64_t)at < P.det_buf) {
        det_keys[at] = packed;
        det_p[at] = p;
      }
      win.add(bins, p);
      any = 1;
    }
  }
  win.flush(bins);
  __syncthreads();
  if (any) {
    uint64_t* rep = S->xs + (blockIdx.x % kXsRep) * kXsLimbs;
    for (int i = threadIdx.x; i < kXsLimbs; i += blockDim.x)
      if (bins[i]) atomicAdd((unsigned long long*)&rep[i], (unsigned long long)bins[i]);
  }
}

// s_det, s_rnd and p_det once the deterministic enumeration is done
struct DetSummary {
  int64_t sdet, srnd;
  double pdet;
  int topk, bad;
};

// with_pdet = false skips the exact-sum rounding (pdet left 0).
__device__ DetSummary det_summary(const SampleParams& P, const SampleState* S, bool with_pdet = true) {
  DetSummary r;
  r.topk = 0;
  r.bad = 0;
  r.pdet = 0.0;
  int64_t sdet = (int64_t)S->det_count;
  if (sdet > P.det_buf) {
    // only reachable when tau * s >= 1 by rounding at the threshold: refuse
    r.bad = 1;
    sdet = 0;
  } else if (sdet > P.s) {
    r.topk = 1;  // the host runs the top-s selection
    sdet = P.s;
  } else if (with_pdet) {
    r.pdet = xs_round(S->xs);
  }
  r.sdet = sdet;
  // all rows of nonzero probability already deterministic: nothing left to draw
  double support = 1.0;
  for (int t = 0; t < P.L.d; ++t) support *= (double)P.D.info[t]->nnzq;
  r.srnd = (double)sdet >= support ? 0 : P.s - sdet;
  return r;
}

__device__ void det_store(SampleState* S, const DetSummary& d) {
  if (d.bad) set_status(&S->status, CPA_ERR_DET_CAP);
  S->need_topk = d.topk;
  S->sdet = d.sdet;
  S->srnd = d.srnd;
  if (!d.topk) S->pdet = d.pdet;
  S->nsort = d.sdet + d.srnd;
}

__global__ void k_det_finish(SampleParams P, SampleState* S) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  det_store(S, det_summary(P, S));
}

constexpr size_t kRndSmemMax = 96 * 1024;  // CDFs + probabilities staged up to this size
constexpr int kGuideBits = 9;              // guide-table buckets per staged CDF
constexpr int kGuide = 1 << kGuideBits;

// Alg. 2 with one Philox counter per (slot, attempt)
// finish = 1: the deterministic summary is computed here (thread 0 of each block,
// block 0 stores it); finish = 0: k_det_finish (and the host top-s step) did it.
// Slot j < s_rnd draws its random row, stored in rkeys[j]; k_table_insert then
// enters the deterministic and random rows into the combine table.
// staged = 1: the CDFs and row probabilities of the d other modes are first copied
// to shared memory (C_0, P_0, C_1, P_1, ...), so the searches run there.
__global__ void __launch_bounds__(kThreads) k_rnd(SampleParams P, SampleState* S,
                                                  uint64_t* __restrict__ rkeys, int finish,
                                                  uint64_t* __restrict__ raw_key,
                                                  double* __restrict__ raw_w, int staged,
                                                  int64_t nsum_smem) {
  extern __shared__ __align__(16) uint64_t rnd_smem[];
  __shared__ int64_t sh_sdet, sh_srnd;
  __shared__ double sh_pdet;
  __shared__ int sh_topk, sh_failed;
  // guide[t][b] (b <= kGuide) = first index i with C_t[i] > mulhi(b << (64 - kGuideBits), T_t),
  // kGuide buckets by the top bits of the draw u; the answer for u lies in
  // [guide[b], guide[b + 1]] with b = u >> (64 - kGuideBits).
  uint32_t* guide = reinterpret_cast<uint32_t*>(rnd_smem + 2 * (staged ? nsum_smem : 0));
  __shared__ int sh_span;  // widest guide bucket over the staged CDFs
  if (threadIdx.x == 0) sh_span = 1;
  if (staged) {
    uint64_t* o = rnd_smem;
    for (int t = 0; t < P.L.d; ++t) {  // all copies in flight at once
      const int64_t n = P.L.n[t];
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        cp_async8(o + i, P.D.C[t] + i);
        cp_async8(o + n + i, P.D.P[t] + i);
      }
      o += 2 * n;
    }
    cp_async_wait_all();
    if (P.L.d <= 4) {
      __syncthreads();
      const uint64_t* c = rnd_smem;
      for (int t = 0; t < P.L.d; ++t) {
        const int64_t n = P.L.n[t];
        const uint64_t T = P.D.info[t]->T;
        for (int b = threadIdx.x; b <= kGuide; b += blockDim.x) {
          uint32_t g = (uint32_t)(n - 1);
          if (b < kGuide) g = (uint32_t)cdf_search(c, n, __umul64hi((uint64_t)b << (64 - kGuideBits), T));
          guide[t * (kGuide + 1) + b] = g;
        }
        c += 2 * n;
      }
      __syncthreads();
      int span = 1;
      for (int t = 0; t < P.L.d; ++t)
        for (int b = threadIdx.x; b < kGuide; b += blockDim.x) {
          const int w = (int)(guide[t * (kGuide + 1) + b + 1] - guide[t * (kGuide + 1) + b]) + 1;
          span = w > span ? w : span;
        }
      span = (int)__reduce_max_sync(0xffffffffu, (unsigned)span);
      if ((threadIdx.x & 31) == 0) atomicMax(&sh_span, span);
    }
  }
  if (threadIdx.x == 0) {
    sh_failed = *(volatile int*)&S->status < 0;
    if (finish) {
      // only block 0 (which stores it) and the optional raw weights need p_det
      const DetSummary d = det_summary(P, S, blockIdx.x == 0 || raw_w != nullptr);
      if (blockIdx.x == 0) det_store(S, d);
      sh_sdet = d.sdet;
      sh_srnd = d.srnd;
      sh_pdet = d.pdet;
      sh_topk = d.topk;
    } else {
      sh_sdet = S->sdet;
      sh_srnd = S->srnd;
      sh_pdet = S->pdet;
      sh_topk = S->need_topk;
    }
  }
  __syncthreads();
  const int64_t srnd = sh_srnd;
  const double pdet = sh_pdet;
  const uint64_t iter = P.iter_ptr ? *P.iter_ptr : P.iter;
  uint64_t tries = 0;
  if (sh_failed) return;  // an earlier step failed (e.g. no mass); block-uniform
  // Random slots come from a queue: a lane whose slot is accepted (or gives up)
  // takes the next unclaimed slot, so the lanes of a warp stay busy whatever the
  // number of attempts of each slot.  Attempt a of slot j always uses the Philox
  // counter (j, a, ...), so the draws do not depend on the schedule.
  const int lane = threadIdx.x & 31;
  const bool narrow = P.L.d <= 4;
  const uint64_t* Cb[4];
  const double* Pb[4];
  const uint32_t* Gb[4];
  uint64_t Tb[4];
  int steps = 0;  // bisection steps that always suffice (whole CDF, or one guide bucket)
  if (narrow) {
    const uint64_t* o = rnd_smem;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const bool on = t < P.L.d;
      const int64_t n = on ? P.L.n[t] : 1;
      Cb[t] = on ? (staged ? o : P.D.C[t]) : nullptr;
      Pb[t] = on ? (staged ? reinterpret_cast<const double*>(o + n) : P.D.P[t]) : nullptr;
      Gb[t] = staged ? guide + t * (kGuide + 1) : nullptr;
      Tb[t] = on ? P.D.info[t]->T : 0;
      if (on) o += 2 * n;
      const int64_t span = staged ? (int64_t)sh_span : n;
      int lg = 0;
      while ((1ll << lg) < span) ++lg;
      steps = lg > steps ? lg : steps;
    }
  }
  int64_t jj = -1;  // current slot (-1: take one; >= srnd: done)
  int a = 0;
  for (;;) {
    const unsigned want = __ballot_sync(0xffffffffu, jj < 0);
    if (want) {
      unsigned long long base = 0;
      if (lane == __ffs(want) - 1)
        base = atomicAdd((unsigned long long*)&S->slot_ctr, (unsigned long long)__popc(want));
      base = __shfl_sync(0xffffffffu, base, __ffs(want) - 1);
      if (jj < 0) {
        jj = (int64_t)base + __popc(want & ((1u << lane) - 1u));
        a = 0;
      }
    }
    const bool active = jj < srnd;
    if (!__any_sync(0xffffffffu, active)) break;
    if (!active) continue;
    uint64_t packed = 0;
    double p = 0.0;
    if (narrow) {
      uint64_t w[4] = {(uint64_t)jj, (uint64_t)a, (uint64_t)(uint32_t)P.mode_k | kDomainSample, iter};
      Philox4x64::block(w[0], w[1], w[2], w[3], P.seed, 0ull);
      uint32_t lo[4], hi[4];
      uint64_t tg[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        tg[t] = __umul64hi(w[t], Tb[t]);
        if (staged) {
          const uint32_t b = (uint32_t)(w[t] >> (64 - kGuideBits));
          lo[t] = t < P.L.d ? Gb[t][b] : 0u;
          hi[t] = t < P.L.d ? Gb[t][b + 1] : 0u;
        } else {
          lo[t] = 0;
          hi[t] = t < P.L.d ? (uint32_t)(P.L.n[t] - 1) : 0u;
        }
      }
      for (int it = 0; it < steps; ++it) {  // first index with C > target, as cdf_search
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (lo[t] < hi[t]) {
            const uint32_t mid = lo[t] + ((hi[t] - lo[t]) >> 1);
            if (Cb[t][mid] > tg[t]) hi[t] = mid; else lo[t] = mid + 1;
          }
        }
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t < P.L.d) {
          const double pt = Pb[t][lo[t]];
          p = t == 0 ? pt : __dmul_rn(p, pt);
          packed |= (uint64_t)lo[t] << P.L.off[t];
        }
      }
    } else {
      uint64_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
      const uint64_t* o = rnd_smem;
      for (int t = 0; t < P.L.d; ++t) {
        const int64_t n = P.L.n[t];
        const uint64_t* Ct = staged ? o : P.D.C[t];
        const double* Pt = staged ? reinterpret_cast<const double*>(o + n) : P.D.P[t];
        o += 2 * n;
        if ((t & 3) == 0) {
          w0 = (uint64_t)jj;
          w1 = (uint64_t)a;
          w2 = (uint64_t)(uint32_t)P.mode_k | ((uint64_t)(t >> 2) << 16) | kDomainSample;
          w3 = iter;
          Philox4x64::block(w0, w1, w2, w3, P.seed, 0ull);
        }
        const uint64_t u = (t & 3) == 0 ? w0 : (t & 3) == 1 ? w1 : (t & 3) == 2 ? w2 : w3;
        const uint64_t T = P.D.info[t]->T;
        const int64_t i = cdf_search(Ct, n, __umul64hi(u, T));
        const double pt = Pt[i];
        p = t == 0 ? pt : __dmul_rn(p, pt);
        packed |= (uint64_t)i << P.L.off[t];
      }
    }
    ++tries;
    ++a;
    const bool ok = !nonneg_gt(p, P.tau);  // p <= tau
    if (ok || a >= P.reject_cap) {
      if (!ok) set_status(&S->status, CPA_ERR_REJECT_LIMIT);
      rkeys[jj] = packed;  // entered into the combine table by k_table_insert
      if (raw_key) raw_key[jj] = P.L.linear(packed);
      if (raw_w)
        raw_w[jj] = __dsqrt_rn(__ddiv_rn(__dsub_rn(1.0, pdet), __dmul_rn(p, __ll2double_rn(srnd))));
      jj = -1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) tries += __shfl_xor_sync(0xffffffffu, tries, o);
  if ((threadIdx.x & 31) == 0 && tries)
    atomicAdd((unsigned long long*)&S->attempts, (unsigned long long)tries);
}

// CombineRepeats input: the s_det deterministic keys (unless the top-s path entered
// them) and the s_rnd random keys, the latter with the flag bit, into the table.
__global__ void k_table_insert(SampleParams P, SampleState* S, uint64_t* __restrict__ hkeys,
                               uint32_t* __restrict__ hcnt, int hbits,
                               const uint64_t* __restrict__ det_keys,
                               const uint64_t* __restrict__ rkeys) {
  const int64_t sdet = S->need_topk ? 0 : S->sdet, srnd = S->srnd;
  const uint64_t flag = 1ull << P.L.total_bits;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < sdet + srnd;
       g += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = g < sdet ? det_keys[g] : (flag | rkeys[g - sdet]);
    if (!table_add(hkeys, hcnt, hbits, key)) set_status(&S->status, CPA_ERR_UNSUPPORTED);
  }
}

// occupied table slots -> output rows, unordered; each block takes kCompactPer
// consecutive slots per thread and claims its output range with one atomic
constexpr int kCompactPer = 4;
__global__ void __launch_bounds__(kThreads) k_table_compact(SampleParams P, SampleState* S,
                                                            uint64_t* __restrict__ hkeys,
                                                            uint32_t* __restrict__ hcnt, int hbits,
                                                            uint64_t* __restrict__ idx_packed,
                                                            uint32_t* __restrict__ cnt,
                                                            double* __restrict__ wgt) {
  __shared__ unsigned wsum[kThreads / 32];
  __shared__ unsigned long long bbase;
  const int64_t H = 1ll << hbits;
  const int64_t srnd = S->srnd;
  const double one_minus_pdet = __dsub_rn(1.0, S->pdet);
  const uint64_t flag_bit = 1ull << P.L.total_bits;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t span = (int64_t)kThreads * kCompactPer;
  for (int64_t b0 = blockIdx.x * span; b0 < H; b0 += (int64_t)gridDim.x * span) {
    uint64_t v[kCompactPer];
    unsigned mine = 0;
#pragma unroll
    for (int u = 0; u < kCompactPer; ++u) {
      const int64_t h = b0 + (int64_t)u * kThreads + threadIdx.x;
      v[u] = h < H ? hkeys[h] : kEmptyKey;
      mine += v[u] != kEmptyKey;
    }
    // block-exclusive prefix of the per-thread counts
    unsigned incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned tot = 0;
      for (int w = 0; w < kThreads / 32; ++w) {
        const unsigned c = wsum[w];
        wsum[w] = tot;
        tot += c;
      }
      bbase = tot ? atomicAdd((unsigned long long*)&S->sbar, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    int64_t u_out = (int64_t)bbase + wsum[warp] + (incl - mine);
#pragma unroll
    for (int u = 0; u < kCompactPer; ++u) {
      if (v[u] == kEmptyKey) continue;
      const int64_t h = b0 + (int64_t)u * kThreads + threadIdx.x;
      const uint64_t packed = v[u] & (flag_bit - 1ull);
      const bool det = !(v[u] & flag_bit);
      const uint32_t c = det ? 1u : hcnt[h];
      idx_packed[u_out] = packed;
      cnt[u_out] = c;
      wgt[u_out] = row_weight(P, packed, det, c, one_minus_pdet, srnd);
      hkeys[h] = kEmptyKey;  // leave the table empty for the next pass
      hcnt[h] = 0;
      ++u_out;
    }
    __syncthreads();  // wsum and bbase are reused by the next span
  }
}

__global__ void k_table_collect(SampleState* S, const uint64_t* __restrict__ hkeys, int hbits,
                                uint64_t* __restrict__ out) {
  const int64_t H = 1ll << hbits;
  const int lane = threadIdx.x & 31;
  for (int64_t h0 = blockIdx.x * (int64_t)blockDim.x; h0 < H; h0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t h = h0 + threadIdx.x;
    const uint64_t v = h < H ? hkeys[h] : kEmptyKey;
    const bool occ = v != kEmptyKey;
    const unsigned bal = __ballot_sync(0xffffffffu, occ);
    unsigned long long base = 0;
    if (lane == 0 && bal) base = atomicAdd((unsigned long long*)&S->sbar, (unsigned long long)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (occ) out[(int64_t)base + __popc(bal & ((1u << lane) - 1u))] = v;
  }
}

// sorted flagged keys (deterministic first, each block ascending) -> output rows
__global__ void k_table_emit(SampleParams P, const SampleState* S, const uint64_t* __restrict__ sorted,
                             const uint64_t* __restrict__ hkeys, const uint32_t* __restrict__ hcnt,
                             int hbits, uint64_t* __restrict__ idx_packed, uint32_t* __restrict__ cnt,
                             double* __restrict__ wgt, uint64_t* __restrict__ idx_linear) {
  const int64_t nu = S->sbar;
  const int64_t srnd = S->srnd;
  const double one_minus_pdet = __dsub_rn(1.0, S->pdet);
  const uint64_t flag_bit = 1ull << P.L.total_bits;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
       u += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t v = sorted[u];
    const uint64_t packed = v & (flag_bit - 1ull);
    const bool det = !(v & flag_bit);
    const uint32_t c = det ? 1u : table_count(hkeys, hcnt, hbits, v);
    idx_packed[u] = packed;
    if (idx_linear) idx_linear[u] = P.L.linear(packed);
    cnt[u] = c;
    wgt[u] = row_weight(P, packed, det, c, one_minus_pdet, srnd);
  }
}

// top-s path (tau * s < 1 only): rank keys by p descending, ties by key ascending
__global__ void k_topk_keys(const SampleState* S, const double* __restrict__ det_p,
                            uint64_t* __restrict__ rank_key, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    rank_key[j] = ~(uint64_t)__double_as_longlong(det_p[j]);  // p > 0: bits increase with p
}

__global__ void k_topk_take(SampleParams P, SampleState* S, const uint64_t* __restrict__ keys_by_p,
                            uint64_t* __restrict__ hkeys, uint32_t* __restrict__ hcnt, int hbits) {
  __shared__ uint64_t bins[kXsLimbs];
  for (int i = threadIdx.x; i < kXsLimbs; i += blockDim.x) bins[i] = 0;
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.s;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t packed = keys_by_p[j];
    if (!table_add(hkeys, hcnt, hbits, packed)) set_status(&S->status, CPA_ERR_UNSUPPORTED);
    xs_add(bins, key_prob(P, packed));
  }
  __syncthreads();
  uint64_t* rep = S->xs + (blockIdx.x % kXsRep) * kXsLimbs;
  for (int i = threadIdx.x; i < kXsLimbs; i += blockDim.x)
    if (bins[i]) atomicAdd((unsigned long long*)&rep[i], (unsigned long long)bins[i]);
}

__global__ void k_topk_finish(SampleState* S) {
  if (threadIdx.x == 0 && blockIdx.x == 0) S->pdet = xs_round(S->xs);
}

__global__ void k_zero_bins(SampleState* S) {
  for (int i = threadIdx.x; i < kXsRep * kXsLimbs; i += blockDim.x) S->xs[i] = 0;
}

inline unsigned blocks_for(int64_t n);

}  // namespace

int phat_from_cdf(const uint64_t* C, int64_t n, const DistInfo* info, double* p, cudaStream_t st) {
  if (n <= 0) return CPA_OK;
  int64_t b = ceil_div(n, kThreads);
  const int64_t cap = (int64_t)num_sms() * 8;
  k_phat<<<(unsigned)(b < cap ? b : cap), kThreads, 0, st>>>(C, n, info, p);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

namespace {

inline unsigned blocks_for(int64_t n) {
  int64_t b = ceil_div(n > 0 ? n : 1, kThreads);
  const int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(b < cap ? b : cap);
}

}  // namespace

int64_t det_buffer_capacity(int64_t s, double tau, int64_t det_cap) {
  if (!(tau < 1.0)) return 1;
  if (tau * (double)s >= 1.0) return s < det_cap ? s : det_cap;
  return det_cap;
}

size_t sample_buffers_bytes(const KeyLayout& L, int64_t s, int64_t det_buf) {
  Arena a;
  SampleBuffers B;
  sample_buffers_carve(a, L, s, det_buf, &B);
  return a.used + 256;
}

void sample_buffers_carve(Arena& a, const KeyLayout& L, int64_t s, int64_t det_cap,
                          SampleBuffers* B) {
  int64_t ncand = 0;
  for (int t = 0; t < L.d; ++t) {
    B->cand_off[t] = ncand;
    ncand += L.n[t];
  }
  for (int t = L.d; t < kMaxOrder; ++t) B->cand_off[t] = ncand;
  B->state = a.take<SampleState>(1);
  B->cand = a.take<uint32_t>(ncand);
  B->det_keys = a.take<uint64_t>(det_cap);
  B->det_p = a.take<double>(det_cap);
  B->sortA = a.take<uint64_t>(s);
  B->sortB = a.take<uint64_t>(s);
  int hb = 10;
  while ((1ll << hb) < 2 * s) ++hb;
  B->hbits = hb;
  B->hkeys = a.take<uint64_t>(1ull << hb);
  B->hcnt = a.take<uint32_t>(1ull << hb);
  const size_t ws_s = sort_workspace(s), ws_c = scan_workspace(s);
  const int64_t big = det_cap > s ? det_cap : s;
  const size_t ws_t = sort_workspace(big);
  size_t ws = ws_s > ws_c ? ws_s : ws_c;
  ws = ws > ws_t ? ws : ws_t;
  B->scratch = a.take<char>(ws);
  B->idx_packed = a.take<uint64_t>(s);
  B->cnt = a.take<uint32_t>(s);
  B->wgt = a.take<double>(s);
  B->idx_linear = nullptr;
  B->raw_key = nullptr;
  B->raw_w = nullptr;
}

int skrp_lev(const SampleParams& P, SampleBuffers& B, cudaStream_t st, bool sorted_output) {
  SampleState* S = B.state;
  const int64_t* co = B.cand_off;
  int64_t total_cand = 0;
  for (int t = 0; t < P.L.d; ++t) total_cand += P.L.n[t];
  if (sorted_output) {  // the compacting path leaves the table empty itself
    CPA_CUDA_TRY(cudaMemsetAsync(B.hkeys, 0xff, sizeof(uint64_t) << B.hbits, st));
    CPA_CUDA_TRY(cudaMemsetAsync(B.hcnt, 0, sizeof(uint32_t) << B.hbits, st));
  }
  k_prepare<<<1, 32, 0, st>>>(P, S);
  const bool may_det = P.tau < 1.0;
  if (may_det) {
    k_det_filter<<<blocks_for(total_cand), kThreads, 0, st>>>(
        P, S, B.cand, co[1], co[2], co[3], co[4], co[5], co[6], total_cand);
    k_det_enum<<<(unsigned)num_sms() * 4, kThreads, 0, st>>>(P, S, B.cand, co[1], co[2], co[3],
                                                              co[4], co[5], co[6], B.det_keys,
                                                              B.det_p);
  }
  const bool host_topk = may_det && P.tau * (double)P.s < 1.0;
  if (host_topk) k_det_finish<<<1, 32, 0, st>>>(P, S);
  CPA_LAUNCH_CHECK();
  if (host_topk) {
    // the deterministic set may hold more than s rows: keep the s most probable
    SampleState h;
    CPA_CUDA_TRY(cudaMemcpyAsync(&h, S, sizeof(SampleState), cudaMemcpyDeviceToHost, st));
    CPA_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.need_topk) {
      const int64_t n = (int64_t)h.det_count;
      // det buffers: sort (key) by p descending with ties by key ascending:
      // first order by key, then stable by ~bits(p)
      uint64_t* k1 = B.det_keys;
      double* p1 = B.det_p;
      // work arrays: reuse the candidate-free tail of scratch via a temporary allocation
      uint64_t *ka = nullptr, *kb = nullptr, *va = nullptr, *vb = nullptr;
      void* ws = nullptr;
      CPA_CUDA_TRY(cudaMallocAsync((void**)&ka, sizeof(uint64_t) * n * 4 + sort_workspace(n) + 1024, st));
      kb = ka + n;
      va = kb + n;
      vb = va + n;
      ws = vb + n;
      int alt = 0;
      // sort p values by key: payload = p bits
      CPA_CUDA_TRY(cudaMemcpyAsync(ka, k1, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
      CPA_CUDA_TRY(cudaMemcpyAsync(va, p1, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
      CPA_TRY(radix_sort<uint64_t>(ka, kb, va, vb, DevCount{nullptr, n}, 0, P.L.total_bits, ws, st,
                                   &alt));
      uint64_t* keys_sorted = alt ? kb : ka;
      uint64_t* p_sorted = alt ? vb : va;
      uint64_t* spare_k = alt ? ka : kb;
      uint64_t* spare_v = alt ? va : vb;
      // rank key = ~bits(p); payload = packed key
      k_topk_keys<<<blocks_for(n), kThreads, 0, st>>>(S, reinterpret_cast<const double*>(p_sorted),
                                                       spare_k, n);
      CPA_CUDA_TRY(cudaMemcpyAsync(spare_v, keys_sorted, sizeof(uint64_t) * n,
                                   cudaMemcpyDeviceToDevice, st));
      CPA_TRY(radix_sort<uint64_t>(spare_k, keys_sorted, spare_v, p_sorted, DevCount{nullptr, n}, 0,
                                   64, ws, st, &alt));
      uint64_t* by_p = alt ? p_sorted : spare_v;
      k_zero_bins<<<1, 64, 0, st>>>(S);
      k_topk_take<<<blocks_for(P.s), kThreads, 0, st>>>(P, S, by_p, B.hkeys, B.hcnt, B.hbits);
      k_topk_finish<<<1, 32, 0, st>>>(S);
      CPA_LAUNCH_CHECK();
      CPA_CUDA_TRY(cudaFreeAsync(ka, st));
    }
  }
  int64_t nsum = 0;
  for (int t = 0; t < P.L.d; ++t) nsum += P.L.n[t];
  const size_t rsm = sizeof(uint64_t) * 2 * (size_t)nsum + sizeof(uint32_t) * 4 * (kGuide + 1);
  const int staged = rsm <= kRndSmemMax && nsum < (1ll << 31) ? 1 : 0;
  {
    static std::atomic<unsigned long long> attr{0};
    CPA_CUDA_TRY(set_attr_once(attr, [] {
      return cudaFuncSetAttribute(k_rnd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRndSmemMax);
    }));
  }
  // a few warps per SM: the random slots come from a queue, and a warp's last slots
  // (one sequence of attempts each) set its length
  const int64_t rblocks = ceil_div(P.s, kThreads);
  const int64_t rcap = (int64_t)num_sms() * 2;
  k_rnd<<<(unsigned)(rblocks < rcap ? rblocks : rcap), kThreads, staged ? rsm : 0, st>>>(
      P, S, B.sortA, host_topk ? 0 : 1, B.raw_key, B.raw_w, staged, nsum);
  CPA_LAUNCH_CHECK();
  k_table_insert<<<blocks_for(2 * P.s), kThreads, 0, st>>>(P, S, B.hkeys, B.hcnt, B.hbits, B.det_keys, B.sortA);
  CPA_LAUNCH_CHECK();
  const int64_t H = 1ll << B.hbits;
  if (!sorted_output) {
    k_table_compact<<<blocks_for(ceil_div(H, kCompactPer)), kThreads, 0, st>>>(P, S, B.hkeys, B.hcnt, B.hbits,
                                                                              B.idx_packed, B.cnt, B.wgt);
    CPA_LAUNCH_CHECK();
    return CPA_OK;
  }
  // ascending output: deterministic keys (flag bit clear) first, then random ones
  k_table_collect<<<blocks_for(H), kThreads, 0, st>>>(S, B.hkeys, B.hbits, B.sortA);
  int alt = 0;
  CPA_TRY(radix_sort<uint64_t>(B.sortA, B.sortB, (uint64_t*)nullptr, (uint64_t*)nullptr,
                               DevCount{&S->sbar, P.s}, 0, P.L.total_bits + 1, B.scratch, st, &alt));
  const uint64_t* sorted = alt ? B.sortB : B.sortA;
  k_table_emit<<<blocks_for(P.s), kThreads, 0, st>>>(P, S, sorted, B.hkeys, B.hcnt, B.hbits, B.idx_packed,
                                                     B.cnt, B.wgt, B.idx_linear);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

}  // namespace cpa
