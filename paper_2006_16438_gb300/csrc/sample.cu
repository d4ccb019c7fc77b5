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

__device__ __forceinline__ double mode_prob(const uint64_t* __restrict__ C, uint64_t T, int64_t i) {
  const uint64_t q = C[i] - (i > 0 ? C[i - 1] : 0ull);
  return __ddiv_rn(__ull2double_rn(q), __ull2double_rn(T));
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
    const double pt = mode_prob(P.D.C[t], P.D.info[t]->T, P.L.get(packed, t));
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

__device__ double xs_round(const uint64_t* bins_in) {
  uint32_t w[kXsLimbs + 2];
  uint64_t carry = 0;
  for (int i = 0; i < kXsLimbs; ++i) {
    const uint64_t v = bins_in[i] + carry;
    w[i] = (uint32_t)v;
    carry = v >> 32;
  }
  w[kXsLimbs] = (uint32_t)carry;
  w[kXsLimbs + 1] = (uint32_t)(carry >> 32);
  int top = -1;
  for (int i = kXsLimbs + 1; i >= 0; --i)
    if (w[i]) {
      top = i * 32 + 31 - __clz(w[i]);
      break;
    }
  if (top < 0) return 0.0;
  auto bit = [&](int pos) -> uint32_t { return pos < 0 ? 0u : (w[pos >> 5] >> (pos & 31)) & 1u; };
  if (top < 53) {  // below 2^-1021: the integer itself is the IEEE bit pattern
    uint64_t m = 0;
    for (int b = top; b >= 0; --b) m = (m << 1) | bit(b);
    return __longlong_as_double((long long)m);
  }
  uint64_t m = 0;
  for (int b = top; b > top - 53; --b) m = (m << 1) | bit(b);
  const uint32_t round_bit = bit(top - 54 + 1);
  uint32_t sticky = 0;
  for (int b = top - 54; b >= 0 && !sticky; --b) sticky |= bit(b);
  if (round_bit && (sticky || (m & 1ull))) ++m;
  uint64_t bexp = (uint64_t)(top - 51);
  if (m == (1ull << 53)) {
    m >>= 1;
    ++bexp;
  }
  return __longlong_as_double((long long)((bexp << 52) | (m & ((1ull << 52) - 1ull))));
}

// ---- kernels ----------------------------------------------------------
__global__ void k_prepare(SampleParams P, SampleState* S) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
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
  S->pdet = 0.0;
  for (int i = 0; i < kXsLimbs; ++i) S->xs[i] = 0;
  double astar = 0.0;
  double alpha[kMaxOrder];
  for (int t = 0; t < P.L.d; ++t) {
    S->ncand[t] = 0;
    const DistInfo* I = P.D.info[t];
    alpha[t] = __ddiv_rn(__ull2double_rn(I->maxq), __ull2double_rn(I->T));
    astar = t == 0 ? alpha[t] : __dmul_rn(astar, alpha[t]);
  }
  S->alpha_star = astar;
  S->no_det = !(astar > P.tau);
  const double slack = 1.0 - 0x1p-40;
  for (int t = 0; t < P.L.d; ++t)
    S->thr[t] = __dmul_rn(__ddiv_rn(__dmul_rn(P.tau, alpha[t]), astar), slack);
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
    const double p = mode_prob(P.D.C[t], P.D.info[t]->T, i);
    if (p >= S->thr[t]) {
      const unsigned long long at = atomicAdd((unsigned long long*)&S->ncand[t], 1ull);
      cand[offs[t] + (int64_t)at] = (uint32_t)i;
    }
  }
}

__global__ void k_det_count(SampleParams P, SampleState* S) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || S->no_det) return;
  double prod = 1.0;
  for (int t = 0; t < P.L.d; ++t) prod *= (double)S->ncand[t];
  if (prod > (double)P.det_cap) {
    set_status(&S->status, CPA_ERR_DET_CAP);
    S->no_det = 1;
    return;
  }
  uint64_t total = 1;
  for (int t = 0; t < P.L.d; ++t) total *= (uint64_t)S->ncand[t];
  S->cand_total = total;
}

// enumerate the candidate product; keep p > tau
__global__ void k_det_enum(SampleParams P, SampleState* S, const uint32_t* __restrict__ cand,
                           int64_t off1, int64_t off2, int64_t off3, int64_t off4, int64_t off5,
                           int64_t off6, uint64_t* __restrict__ det_keys, double* __restrict__ det_p) {
  __shared__ uint64_t bins[kXsLimbs];
  __shared__ int any;
  if (S->no_det) return;
  for (int i = threadIdx.x; i < kXsLimbs; i += blockDim.x) bins[i] = 0;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int64_t offs[kMaxOrder] = {0, off1, off2, off3, off4, off5, off6, 0};
  const uint64_t total = S->cand_total;
  int64_t nc[kMaxOrder];
  for (int t = 0; t < P.L.d; ++t) nc[t] = S->ncand[t];
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
       e += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t rest = e, packed = 0;
    double p = 0.0;
    for (int t = 0; t < P.L.d; ++t) {
      const uint64_t pos = rest % (uint64_t)nc[t];
      rest /= (uint64_t)nc[t];
      const uint32_t i = cand[offs[t] + (int64_t)pos];
      const double pt = mode_prob(P.D.C[t], P.D.info[t]->T, i);
      p = t == 0 ? pt : __dmul_rn(p, pt);
      packed |= (uint64_t)i << P.L.off[t];
    }
    if (p > P.tau) {
      const unsigned long long at = atomicAdd((unsigned long long*)&S->det_count, 1ull);
      if ((int64_t)at < P.det_cap) {
        det_keys[at] = packed;
        det_p[at] = p;
      }
      xs_add(bins, p);
      any = 1;
    }
  }
  __syncthreads();
  if (any)
    for (int i = threadIdx.x; i < kXsLimbs; i += blockDim.x)
      if (bins[i]) atomicAdd((unsigned long long*)&S->xs[i], (unsigned long long)bins[i]);
}

__global__ void k_det_finish(SampleParams P, SampleState* S) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t sdet = (int64_t)S->det_count;
  if (sdet > P.s) {
    S->need_topk = 1;  // the host runs the top-s selection
    sdet = P.s;
  } else {
    S->pdet = xs_round(S->xs);
  }
  S->sdet = sdet;
  // all rows of nonzero probability already deterministic: nothing left to draw
  double support = 1.0;
  for (int t = 0; t < P.L.d; ++t) support *= (double)P.D.info[t]->nnzq;
  int64_t srnd = P.s - sdet;
  if ((double)sdet >= support) srnd = 0;
  S->srnd = srnd;
  S->nsort = sdet + srnd;
}

__global__ void k_copy_det(SampleState* S, const uint64_t* __restrict__ det_keys,
                           uint64_t* __restrict__ sortbuf) {
  const int64_t sdet = S->sdet;
  if (S->need_topk) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < sdet;
       j += (int64_t)gridDim.x * blockDim.x)
    sortbuf[j] = det_keys[j];
}

// Alg. 2 with one Philox counter per (slot, attempt)
__global__ void __launch_bounds__(kThreads) k_rnd(SampleParams P, SampleState* S,
                                                  uint64_t* __restrict__ sortbuf,
                                                  uint64_t* __restrict__ raw_key,
                                                  double* __restrict__ raw_w) {
  const int64_t srnd = S->srnd, sdet = S->sdet;
  const double pdet = S->pdet;
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  uint64_t tries = 0;
  if (j < srnd) {
    uint64_t packed = 0;
    double p = 0.0;
    bool ok = false;
    for (int a = 0; a < P.reject_cap; ++a) {
      uint64_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
      packed = 0;
      for (int t = 0; t < P.L.d; ++t) {
        if ((t & 3) == 0) {
          w0 = (uint64_t)j;
          w1 = (uint64_t)a;
          w2 = (uint64_t)(uint32_t)P.mode_k | ((uint64_t)(t >> 2) << 16) | kDomainSample;
          w3 = P.iter;
          Philox4x64::block(w0, w1, w2, w3, P.seed, 0ull);
        }
        const uint64_t u = (t & 3) == 0 ? w0 : (t & 3) == 1 ? w1 : (t & 3) == 2 ? w2 : w3;
        const uint64_t T = P.D.info[t]->T;
        const int64_t i = cdf_search(P.D.C[t], P.L.n[t], __umul64hi(u, T));
        const double pt = mode_prob(P.D.C[t], T, i);
        p = t == 0 ? pt : __dmul_rn(p, pt);
        packed |= (uint64_t)i << P.L.off[t];
      }
      ++tries;
      if (p <= P.tau) {
        ok = true;
        break;
      }
    }
    if (!ok) set_status(&S->status, CPA_ERR_REJECT_LIMIT);
    sortbuf[sdet + j] = (1ull << P.L.total_bits) | packed;
    if (raw_key) raw_key[j] = P.L.linear(packed);
    if (raw_w)
      raw_w[j] = __dsqrt_rn(__ddiv_rn(__dsub_rn(1.0, pdet), __dmul_rn(p, __ll2double_rn(srnd))));
  }
  for (int o = 16; o > 0; o >>= 1) tries += __shfl_xor_sync(0xffffffffu, tries, o);
  if ((threadIdx.x & 31) == 0 && tries)
    atomicAdd((unsigned long long*)&S->attempts, (unsigned long long)tries);
}

__global__ void k_run_flags(const SampleState* S, const uint64_t* __restrict__ sorted,
                            uint32_t* __restrict__ flag) {
  const int64_t n = S->nsort;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    flag[j] = (j == 0 || sorted[j] != sorted[j - 1]) ? 1u : 0u;
}

__global__ void k_run_starts(SampleState* S, const uint32_t* __restrict__ flag,
                             const uint64_t* __restrict__ uid, uint64_t* __restrict__ run_start) {
  const int64_t n = S->nsort;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    if (flag[j]) run_start[uid[j]] = (uint64_t)j;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t nu = n > 0 ? (int64_t)(uid[n - 1] + flag[n - 1]) : 0;
    S->nuniq = nu;
    S->sbar = nu;
    run_start[nu] = (uint64_t)n;
  }
}

// run u of the sorted buffer -> output row u
__global__ void k_combine(SampleParams P, const SampleState* S, const uint64_t* __restrict__ sorted,
                          const uint64_t* __restrict__ run_start, uint64_t* __restrict__ idx_packed,
                          uint32_t* __restrict__ cnt, double* __restrict__ wgt,
                          uint64_t* __restrict__ idx_linear) {
  const int64_t nu = S->nuniq;
  const int64_t srnd = S->srnd;
  const double one_minus_pdet = __dsub_rn(1.0, S->pdet);
  const uint64_t flag_bit = 1ull << P.L.total_bits;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
       u += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t b = run_start[u];
    const uint64_t c = run_start[u + 1] - b;
    const uint64_t v = sorted[b];
    const uint64_t packed = v & (flag_bit - 1ull);
    idx_packed[u] = packed;
    if (idx_linear) idx_linear[u] = P.L.linear(packed);
    if (!(v & flag_bit)) {  // deterministic row
      cnt[u] = 1;
      wgt[u] = 1.0;
    } else {
      const double p = key_prob(P, packed);
      cnt[u] = (uint32_t)c;
      wgt[u] = __dsqrt_rn(__ddiv_rn(__dmul_rn(__ull2double_rn(c), one_minus_pdet),
                                    __dmul_rn(p, __ll2double_rn(srnd))));
    }
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
                            uint64_t* __restrict__ sortbuf) {
  __shared__ uint64_t bins[kXsLimbs];
  for (int i = threadIdx.x; i < kXsLimbs; i += blockDim.x) bins[i] = 0;
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < P.s;
       j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t packed = keys_by_p[j];
    sortbuf[j] = packed;
    xs_add(bins, key_prob(P, packed));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kXsLimbs; i += blockDim.x)
    if (bins[i]) atomicAdd((unsigned long long*)&S->xs[i], (unsigned long long)bins[i]);
}

__global__ void k_topk_finish(SampleState* S) {
  if (threadIdx.x == 0 && blockIdx.x == 0) S->pdet = xs_round(S->xs);
}

__global__ void k_zero_bins(SampleState* S) {
  if (threadIdx.x < kXsLimbs) S->xs[threadIdx.x] = 0;
}

inline unsigned blocks_for(int64_t n) {
  int64_t b = ceil_div(n > 0 ? n : 1, kThreads);
  const int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(b < cap ? b : cap);
}

}  // namespace

size_t sample_buffers_bytes(const KeyLayout& L, int64_t s, int64_t det_cap) {
  Arena a;
  SampleBuffers B;
  sample_buffers_carve(a, L, s, det_cap, &B);
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
  B->flag = a.take<uint32_t>(s);
  B->uid = a.take<uint64_t>(s);
  B->run_start = a.take<uint64_t>(s + 1);
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

int skrp_lev(const SampleParams& P, SampleBuffers& B, cudaStream_t st) {
  SampleState* S = B.state;
  const int64_t* co = B.cand_off;
  int64_t total_cand = 0;
  for (int t = 0; t < P.L.d; ++t) total_cand += P.L.n[t];
  k_prepare<<<1, 32, 0, st>>>(P, S);
  const bool may_det = P.tau < 1.0;
  if (may_det) {
    k_det_filter<<<blocks_for(total_cand), kThreads, 0, st>>>(
        P, S, B.cand, co[1], co[2], co[3], co[4], co[5], co[6], total_cand);
    k_det_count<<<1, 32, 0, st>>>(P, S);
    k_det_enum<<<(unsigned)num_sms() * 4, kThreads, 0, st>>>(P, S, B.cand, co[1], co[2], co[3],
                                                              co[4], co[5], co[6], B.det_keys,
                                                              B.det_p);
  }
  k_det_finish<<<1, 32, 0, st>>>(P, S);
  CPA_LAUNCH_CHECK();
  if (may_det && P.tau * (double)P.s < 1.0) {
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
      k_topk_take<<<blocks_for(P.s), kThreads, 0, st>>>(P, S, by_p, B.sortA);
      k_topk_finish<<<1, 32, 0, st>>>(S);
      CPA_LAUNCH_CHECK();
      CPA_CUDA_TRY(cudaFreeAsync(ka, st));
    }
  }
  k_copy_det<<<blocks_for(P.s), kThreads, 0, st>>>(S, B.det_keys, B.sortA);
  k_rnd<<<(unsigned)ceil_div(P.s, kThreads), kThreads, 0, st>>>(P, S, B.sortA, B.raw_key, B.raw_w);
  CPA_LAUNCH_CHECK();
  // combine: sort (flag bit keeps deterministic rows first), run-length encode
  int alt = 0;
  const DevCount n_sort{&S->nsort, P.s};
  CPA_TRY(radix_sort<uint64_t>(B.sortA, B.sortB, (uint64_t*)nullptr, (uint64_t*)nullptr, n_sort, 0,
                               P.L.total_bits + 1, B.scratch, st, &alt));
  const uint64_t* sorted = alt ? B.sortB : B.sortA;
  k_run_flags<<<blocks_for(P.s), kThreads, 0, st>>>(S, sorted, B.flag);
  CPA_TRY(scan_u64<uint32_t>(B.flag, B.uid, n_sort, false, nullptr, B.scratch, st));
  k_run_starts<<<blocks_for(P.s), kThreads, 0, st>>>(S, B.flag, B.uid, B.run_start);
  k_combine<<<blocks_for(P.s), kThreads, 0, st>>>(P, S, sorted, B.run_start, B.idx_packed, B.cnt,
                                                  B.wgt, B.idx_linear);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

}  // namespace cpa
