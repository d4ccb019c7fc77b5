// C ABI of the CP-ARLS-LEV library (include/cpa.h) and the Alg. 3 driver.
//
// The driver keeps everything on the device: per mode the factor matrix, its
// fixed-point CDF and distribution summary; per update one SkrpLev pass, the fused
// sampled MTTKRP, the FP64 solve, the Gram + leverage refresh of the solved mode.
// The host enqueues all of it and reads status, statistics and the fit once at the
// end (and once per epoch when the fit-based stopping rule is on).
#include <math.h>

#include <algorithm>

#include "fit.cuh"
#include "sample.cuh"

using namespace cpa;

namespace {

struct DevStats {
  int64_t sdet_last, sbar_last, nnz_last, attempts_last;
  double pdet_last;
  int64_t nnz_total, sbar_total;
  int warnings;
  int pad;
};

__global__ void k_stats(DevStats* ds, const SampleState* S, const uint64_t* nnz, const int* warn) {
  ds->sdet_last = S->sdet;
  ds->sbar_last = S->sbar;
  ds->nnz_last = (int64_t)*nnz;
  ds->attempts_last = (int64_t)S->attempts;
  ds->pdet_last = S->pdet;
  ds->nnz_total += (int64_t)*nnz;
  ds->sbar_total += S->sbar;
  ds->warnings = *warn;
}

__global__ void k_copy_lambda(const SmallFactor* f, int r, double* lambda) {
  if (threadIdx.x < r) lambda[threadIdx.x] = f->lambda[threadIdx.x];
}

__global__ void k_q_from_lev(const double* __restrict__ lev, int64_t n, int r, uint64_t* __restrict__ q,
                             DistInfo* info) {
  uint64_t mx = 0;
  uint32_t nz = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double p = __ddiv_rn(lev[i], (double)r);
    p = p > 0.0 ? (p < 1.0 ? p : 1.0) : 0.0;
    const uint64_t qi = __double2ull_rn(__dmul_rn(p, 4611686018427387904.0));
    q[i] = qi;
    mx = qi > mx ? qi : mx;
    nz += qi > 0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t om = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = om > mx ? om : mx;
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax((unsigned long long*)&info->maxq, (unsigned long long)mx);
    atomicAdd((unsigned long long*)&info->nnzq, (unsigned long long)nz);
  }
}

// linear key (Eq. 2.2) -> packed key
__global__ void k_linear_to_packed(KeyLayout L, const uint64_t* __restrict__ lin, int64_t n,
                                   uint64_t* __restrict__ packed) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = lin[j], out = 0;
    for (int t = 0; t < L.d; ++t) {
      const uint64_t i = key % (uint64_t)L.n[t];
      key /= (uint64_t)L.n[t];
      out |= i << L.off[t];
    }
    packed[j] = out;
  }
}

__global__ void k_philox(const uint64_t* __restrict__ ctr, uint64_t k0, uint64_t k1, int64_t n,
                         uint64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t w0 = ctr[4 * i], w1 = ctr[4 * i + 1], w2 = ctr[4 * i + 2], w3 = ctr[4 * i + 3];
    Philox4x64::block(w0, w1, w2, w3, k0, k1);
    out[4 * i] = w0;
    out[4 * i + 1] = w1;
    out[4 * i + 2] = w2;
    out[4 * i + 3] = w3;
  }
}

inline unsigned blocks(int64_t n, int threads = 256) {
  int64_t b = ceil_div(n > 0 ? n : 1, threads);
  const int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)(b < cap ? b : cap);
}

// RAII device allocation on a stream
struct DevBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~DevBuf() {
    if (p) {
      cudaFreeAsync(p, st);
      cudaStreamSynchronize(st);
    }
  }
  int alloc(size_t bytes, cudaStream_t s) {
    st = s;
    if (cudaMallocAsync(&p, bytes ? bytes : 1, s) != cudaSuccess) {
      p = nullptr;
      return CPA_ERR_OOM;
    }
    return CPA_OK;
  }
};

// Leverage distribution of one factor: lev (optional), CDF C, info; A normalised in
// place when `normalize_out` (the update path), untouched otherwise.
int refresh_distribution(double* A, int64_t n, int r, uint64_t* C, DistInfo* info, double* GA,
                         SmallFactor* fac, int* warn, void* scan_scratch, bool normalize_out,
                         double* lev_out, cudaStream_t st) {
  CPA_CUDA_TRY(cudaMemsetAsync(GA, 0, sizeof(double) * r * r, st));
  CPA_TRY(gram_rows(A, n, r, GA, st));
  CPA_TRY(factor_spd(GA, r, 1, 1, 1e-12, fac, warn, CPA_WARN_RANK_DEFICIENT_LEV, st));
  CPA_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(DistInfo), st));
  CPA_TRY(lev_rows(A, n, r, fac, lev_out, C, info, normalize_out ? A : nullptr, st));
  CPA_TRY(cdf_from_q(C, C, n, info, scan_scratch, st));
  return CPA_OK;
}

// Optional stage timing: events recorded at stage boundaries on the work stream.
struct Profiler {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> stage_of;  // stage of the interval ending at event i (-1: none)
  cudaEvent_t make() {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    ev.push_back(e);
    stage_of.push_back(-1);
    return e;
  }
  // mark the end of an interval of `stage` that began at the previous mark
  int mark(int stage) {
    if (!on) return CPA_OK;
    cudaEvent_t e = make();
    stage_of.back() = stage;
    CPA_CUDA_TRY(cudaEventRecord(e, st));
    return CPA_OK;
  }
  // an event for the caller to record later (it ends an interval of `stage`)
  cudaEvent_t pending(int stage) {
    if (!on) return nullptr;
    cudaEvent_t e = make();
    stage_of.back() = stage;
    return e;
  }
  void collect(cpa_stats* s) {
    if (!on || !s) return;
    for (size_t i = 1; i < ev.size(); ++i) {
      if (stage_of[i] < 0) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i - 1], ev[i]) == cudaSuccess) {
        s->stage_ms[stage_of[i]] += ms;
        s->stage_launches[stage_of[i]] += 1;
      }
    }
    if (ev.size() >= 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev.front(), ev.back()) == cudaSuccess) s->stage_ms[6] = ms;
      s->stage_launches[6] = 1;
    }
  }
  ~Profiler() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

int check_options(const cpa_options* o) {
  if (!o) return CPA_ERR_ARG;
  if (o->rank < 1 || o->rank > kMaxRank) return CPA_ERR_ARG;
  if (o->samples < 1 || o->samples >= (1ll << 31)) return CPA_ERR_ARG;
  if (!(o->tau >= 0.0 && o->tau <= 1.0)) return CPA_ERR_ARG;
  if (o->iters < 0 || o->reject_cap < 1 || o->det_cap < 1) return CPA_ERR_ARG;
  if (o->precision != CPA_FP64) return CPA_ERR_UNSUPPORTED;
  if (o->fit_mode != CPA_FIT_EXACT && o->fit_mode != CPA_FIT_NONE) return CPA_ERR_ARG;
  if (o->tol < 0.0) return CPA_ERR_ARG;
  return CPA_OK;
}

}  // namespace

extern "C" {

void cpa_options_default(cpa_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->rank = 10;
  opt->samples = 1 << 17;
  opt->tau = 1.0 / (double)(1 << 17);
  opt->iters = 10;
  opt->epoch_len = 5;
  opt->patience = 3;
  opt->tol = 0.0;
  opt->seed = 0;
  opt->iter_offset = 0;
  opt->precision = CPA_FP64;
  opt->fit_mode = CPA_FIT_EXACT;
  opt->det_cap = 1 << 24;
  opt->reject_cap = 4096;
  opt->stream = nullptr;
}

const char* cpa_strerror(int code) {
  switch (code) {
    case CPA_OK: return "ok";
    case CPA_ERR_ARG: return "invalid argument";
    case CPA_ERR_COO_RANGE: return "COO index out of range";
    case CPA_ERR_COO_DUP: return "duplicate COO coordinate";
    case CPA_ERR_OOM: return "out of device memory";
    case CPA_ERR_REJECT_LIMIT: return "rejection limit reached in random sampling";
    case CPA_ERR_DET_CAP: return "deterministic candidate product exceeds det_cap";
    case CPA_ERR_CUDA: return "CUDA error";
    case CPA_ERR_UNSUPPORTED: return "unsupported shape or option";
    default:
      if (code > 0) return "success with warnings";
      return "unknown error";
  }
}

int cpa_index_build(const cpa_coo* coo, void* stream, cpa_index** out) {
  return index_build(coo, (cudaStream_t)stream, out);
}

int cpa_index_free(cpa_index* index) {
  index_free(index);
  return CPA_OK;
}

int cpa_index_info(const cpa_index* X, int32_t mode, int32_t* order, int64_t* dims, int64_t* nnz,
                   int64_t* nfib) {
  if (!X) return CPA_ERR_ARG;
  if (order) *order = X->order;
  if (dims)
    for (int m = 0; m < X->order; ++m) dims[m] = X->dims[m];
  if (nnz) *nnz = X->nnz;
  if (nfib) {
    if (mode < 0 || mode >= X->order) return CPA_ERR_ARG;
    *nfib = X->mode[mode].nfib;
  }
  return CPA_OK;
}

int cpa_index_export(const cpa_index* X, int32_t mode, uint64_t* keys, uint64_t* off, int32_t* ik,
                     void* val, void* stream) {
  return index_export(X, mode, keys, off, ik, val, (cudaStream_t)stream);
}

int cpa_philox4x64(const uint64_t* ctr, const uint64_t* key, int64_t n, uint64_t* out, void* stream) {
  if (!key || n < 0 || (n > 0 && (!ctr || !out))) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (n > 0) k_philox<<<blocks(n), 256, 0, st>>>(ctr, key[0], key[1], n, out);
  CPA_LAUNCH_CHECK();
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  return CPA_OK;
}

int cpa_leverage(const double* A, int64_t n, int32_t r, double* lev, void* stream) {
  if (!A || !lev || n < 1 || r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf buf;
  Arena a;
  for (int pass = 0; pass < 2; ++pass) {
    a.used = 0;
    double* G = a.take<double>(r * r);
    SmallFactor* f = a.take<SmallFactor>(1);
    int* warn = a.take<int>(1);
    if (pass == 0) {
      CPA_TRY(buf.alloc(a.used, st));
      a.base = (char*)buf.p;
      continue;
    }
    CPA_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double) * r * r, st));
    CPA_CUDA_TRY(cudaMemsetAsync(warn, 0, sizeof(int), st));
    CPA_TRY(gram_rows(A, n, r, G, st));
    CPA_TRY(factor_spd(G, r, 1, 1, 1e-12, f, warn, CPA_WARN_RANK_DEFICIENT_LEV, st));
    CPA_TRY(lev_rows(A, n, r, f, lev, nullptr, nullptr, nullptr, st));
    int hwarn = 0;
    CPA_CUDA_TRY(cudaMemcpyAsync(&hwarn, warn, sizeof(int), cudaMemcpyDeviceToHost, st));
    CPA_CUDA_TRY(cudaStreamSynchronize(st));
    return hwarn;
  }
  return CPA_OK;
}

int cpa_cdf(const double* lev, int64_t n, int32_t r, uint64_t* C, uint64_t* info_out, void* stream) {
  if (!lev || !C || n < 1 || r < 1) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf buf;
  CPA_TRY(buf.alloc(sizeof(DistInfo) + 256 + scan_workspace(n), st));
  DistInfo* info = (DistInfo*)buf.p;
  void* scratch = (char*)buf.p + 256;
  CPA_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(DistInfo), st));
  k_q_from_lev<<<blocks(n), 256, 0, st>>>(lev, n, r, C, info);
  CPA_LAUNCH_CHECK();
  CPA_TRY(cdf_from_q(C, C, n, info, scratch, st));
  DistInfo h;
  CPA_CUDA_TRY(cudaMemcpyAsync(&h, info, sizeof(h), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (info_out) {
    info_out[0] = h.T;
    info_out[1] = h.maxq;
    info_out[2] = (uint64_t)h.nnzq;
  }
  return CPA_OK;
}

int cpa_skrp_lev(int32_t d, const int64_t* dims, const double* const* lev, int32_t r,
                 const cpa_options* opt, int32_t mode_k, uint64_t iter, uint64_t* idx, uint32_t* cnt,
                 double* wgt, int64_t* counts, double* pdet) {
  if (d < 1 || d > kMaxOrder - 1 || !dims || !lev || !opt || !idx || !cnt || !wgt) return CPA_ERR_ARG;
  if (r < 1 || opt->samples < 1 || !(opt->tau >= 0.0 && opt->tau <= 1.0) || opt->reject_cap < 1 ||
      opt->det_cap < 1)
    return CPA_ERR_ARG;
  for (int t = 0; t < d; ++t)
    if (dims[t] < 1 || dims[t] > 0x7fffffffll || !lev[t]) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)opt->stream;
  KeyLayout L;
  if (!make_layout(d, dims, -1, &L)) return CPA_ERR_UNSUPPORTED;
  const int64_t s = opt->samples;
  const int64_t det_cap = opt->tau < 1.0 ? opt->det_cap : 1;
  int64_t nmax = 1;
  for (int t = 0; t < d; ++t) nmax = std::max<int64_t>(nmax, dims[t]);
  DevBuf buf;
  Arena a;
  SampleBuffers B;
  uint64_t* Cs[kMaxOrder];
  DistInfo* info = nullptr;
  char* scan_ws = nullptr;
  for (int pass = 0; pass < 2; ++pass) {
    a.used = 0;
    for (int t = 0; t < d; ++t) Cs[t] = a.take<uint64_t>(dims[t]);
    info = a.take<DistInfo>(kMaxOrder);
    scan_ws = a.take<char>(scan_workspace(nmax));
    sample_buffers_carve(a, L, s, det_cap, &B);
    B.idx_linear = idx;
    if (pass == 0) {
      CPA_TRY(buf.alloc(a.used, st));
      a.base = (char*)buf.p;
    }
  }
  B.idx_linear = idx;
  CPA_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(DistInfo) * kMaxOrder, st));
  CPA_CUDA_TRY(cudaMemsetAsync(B.state, 0, sizeof(SampleState), st));
  for (int t = 0; t < d; ++t) {
    k_q_from_lev<<<blocks(dims[t]), 256, 0, st>>>(lev[t], dims[t], r, Cs[t], info + t);
    CPA_LAUNCH_CHECK();
    CPA_TRY(cdf_from_q(Cs[t], Cs[t], dims[t], info + t, scan_ws, st));
  }
  SampleParams P;
  memset(&P, 0, sizeof(P));
  P.L = L;
  for (int t = 0; t < d; ++t) {
    P.D.C[t] = Cs[t];
    P.D.info[t] = info + t;
  }
  P.s = s;
  P.tau = opt->tau;
  P.seed = opt->seed;
  P.iter = iter;
  P.mode_k = mode_k;
  P.reject_cap = opt->reject_cap;
  P.det_cap = det_cap;
  CPA_TRY(skrp_lev(P, B, st));
  SampleState h;
  CPA_CUDA_TRY(cudaMemcpyAsync(&h, B.state, sizeof(h), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (h.status < 0) return h.status;
  CPA_CUDA_TRY(cudaMemcpyAsync(cnt, B.cnt, sizeof(uint32_t) * h.sbar, cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(wgt, B.wgt, sizeof(double) * h.sbar, cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (counts) {
    counts[0] = h.sbar;
    counts[1] = h.sdet;
    counts[2] = (int64_t)h.attempts;
  }
  if (pdet) *pdet = h.pdet;
  return CPA_OK;
}

int cpa_sampled_mttkrp(const cpa_index* X, int32_t mode_k, const double* const* factors, int32_t r,
                       const uint64_t* idx, const double* wgt, int64_t sbar, double* M, double* G,
                       int64_t* nnz_sampled, void* stream) {
  if (!X || mode_k < 0 || mode_k >= X->order || !factors || r < 1 || r > kMaxRank || sbar < 0 || !M ||
      !G || (sbar > 0 && (!idx || !wgt)))
    return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const auto& mode = X->mode[mode_k];
  FactorPtrs F;
  for (int m = 0; m < X->order; ++m) {
    F.A[m] = factors[m];
    if (m != mode_k && !factors[m]) return CPA_ERR_ARG;
  }
  CPA_CUDA_TRY(cudaMemsetAsync(M, 0, sizeof(double) * X->dims[mode_k] * r, st));
  CPA_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double) * r * r, st));
  if (sbar == 0) {
    if (nnz_sampled) *nnz_sampled = 0;
    CPA_CUDA_TRY(cudaStreamSynchronize(st));
    return CPA_OK;
  }
  DevBuf buf;
  Arena a;
  MttkrpBuffers B;
  uint64_t* packed = nullptr;
  for (int pass = 0; pass < 2; ++pass) {
    a.used = 0;
    packed = a.take<uint64_t>(sbar);
    mttkrp_buffers_carve(a, sbar, r, &B);
    if (pass == 0) {
      CPA_TRY(buf.alloc(a.used, st));
      a.base = (char*)buf.p;
    }
  }
  k_linear_to_packed<<<blocks(sbar), 256, 0, st>>>(mode.L, idx, sbar, packed);
  CPA_LAUNCH_CHECK();
  CPA_TRY(sampled_mttkrp(X, mode_k, F, r, packed, wgt, DevCount{nullptr, sbar}, M, G, B, st));
  uint64_t tot = 0;
  CPA_CUDA_TRY(cudaMemcpyAsync(&tot, B.total, sizeof(tot), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (nnz_sampled) *nnz_sampled = (int64_t)tot;
  return CPA_OK;
}

int cpa_solve(const double* G, const double* M, int64_t n, int32_t r, double* A, double* lambda,
              void* stream) {
  if (!G || !M || !A || !lambda || n < 1 || r < 1 || r > kMaxRank || A == M) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf buf;
  CPA_TRY(buf.alloc(sizeof(SmallFactor) * 2 + sizeof(double) * r * r + 1024, st));
  SmallFactor* fs = (SmallFactor*)buf.p;
  SmallFactor* fl = fs + 1;
  double* GA = (double*)(fl + 1);
  int* warn = (int*)(GA + r * r);
  CPA_CUDA_TRY(cudaMemsetAsync(warn, 0, sizeof(int), st));
  CPA_TRY(factor_spd(G, r, 0, 0, 1e-13, fs, warn, CPA_WARN_SINGULAR_GRAM, st));
  CPA_TRY(solve_rows(M, n, r, fs, A, st));
  CPA_CUDA_TRY(cudaMemsetAsync(GA, 0, sizeof(double) * r * r, st));
  CPA_TRY(gram_rows(A, n, r, GA, st));
  int dummy_warn_bit = 0;
  CPA_TRY(factor_spd(GA, r, 1, 1, 1e-12, fl, warn, dummy_warn_bit, st));
  k_copy_lambda<<<1, 64, 0, st>>>(fl, r, lambda);
  CPA_TRY(scale_columns(A, n, r, lambda, st));
  int hwarn = 0;
  CPA_CUDA_TRY(cudaMemcpyAsync(&hwarn, warn, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  return hwarn;
}

int cpa_fit(const cpa_index* X, const double* const* factors, const double* lambda, int32_t r,
            double* fit, void* stream) {
  if (!X || !factors || !lambda || !fit || r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FactorPtrs F;
  for (int m = 0; m < X->order; ++m) {
    if (!factors[m]) return CPA_ERR_ARG;
    F.A[m] = factors[m];
  }
  DevBuf buf;
  CPA_TRY(buf.alloc(fit_buffers_bytes(X->order, r) + 256, st));
  double* fit_dev = (double*)buf.p;
  double* scratch = fit_dev + 32;
  CPA_TRY(fit_enqueue(X, F, lambda, r, scratch, fit_dev, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(fit, fit_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  return CPA_OK;
}

int cp_arls_lev(const cpa_index* X, const cpa_options* opt, double* lambda, double* const* factors,
                int32_t io_on_device, double* fit, cpa_stats* stats) {
  if (!X || !lambda || !factors) return CPA_ERR_ARG;
  CPA_TRY(check_options(opt));
  const int D = X->order;
  const int r = opt->rank;
  const int64_t s = opt->samples;
  const double tau = opt->tau;
  const int64_t det_cap = tau < 1.0 ? opt->det_cap : 1;
  cudaStream_t st = (cudaStream_t)opt->stream;
  for (int m = 0; m < D; ++m)
    if (!factors[m]) return CPA_ERR_ARG;
  KeyLayout Lmax;  // candidate buffer must hold the largest sum of other-mode sizes
  int64_t nmax = 1, nsum = 0;
  for (int m = 0; m < D; ++m) {
    nmax = std::max<int64_t>(nmax, X->dims[m]);
    nsum += X->dims[m];
  }
  memset(&Lmax, 0, sizeof(Lmax));
  Lmax.d = 1;
  Lmax.n[0] = nsum;
  // ---- workspace ----
  DevBuf buf;
  Arena a;
  double* Fm[kMaxOrder];
  uint64_t* Cm[kMaxOrder];
  DistInfo* info = nullptr;
  double *M = nullptr, *Gs = nullptr, *GA = nullptr, *lam = nullptr, *fitd = nullptr, *fit_ws = nullptr;
  SmallFactor *fsolve = nullptr, *flev = nullptr;
  int* warn = nullptr;
  DevStats* dstats = nullptr;
  char* scan_ws = nullptr;
  SampleBuffers SB;
  MttkrpBuffers MB;
  for (int pass = 0; pass < 2; ++pass) {
    a.used = 0;
    for (int m = 0; m < D; ++m) {
      Fm[m] = a.take<double>((size_t)X->dims[m] * r);
      Cm[m] = a.take<uint64_t>(X->dims[m]);
    }
    info = a.take<DistInfo>(kMaxOrder);
    M = a.take<double>((size_t)nmax * r);
    Gs = a.take<double>(r * r);
    GA = a.take<double>(r * r);
    lam = a.take<double>(kMaxRank);
    fitd = a.take<double>(4);
    fit_ws = a.take<double>(fit_buffers_bytes(D, r) / sizeof(double) + 1);
    fsolve = a.take<SmallFactor>(1);
    flev = a.take<SmallFactor>(1);
    warn = a.take<int>(4);
    dstats = a.take<DevStats>(1);
    scan_ws = a.take<char>(scan_workspace(nmax));
    sample_buffers_carve(a, Lmax, s, det_cap, &SB);
    mttkrp_buffers_carve(a, s, r, &MB);
    if (pass == 0) {
      CPA_TRY(buf.alloc(a.used, st));
      a.base = (char*)buf.p;
    }
  }
  // SB.cand_off was computed for the single merged "mode"; per update it is reset below.
  CPA_CUDA_TRY(cudaMemsetAsync(SB.state, 0, sizeof(SampleState), st));
  CPA_CUDA_TRY(cudaMemsetAsync(warn, 0, sizeof(int) * 4, st));
  CPA_CUDA_TRY(cudaMemsetAsync(dstats, 0, sizeof(DevStats), st));
  CPA_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(DistInfo) * kMaxOrder, st));
  const cudaMemcpyKind kin = io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int m = 0; m < D; ++m)
    CPA_CUDA_TRY(cudaMemcpyAsync(Fm[m], factors[m], sizeof(double) * X->dims[m] * r, kin, st));
  // initial leverage distributions (Alg. 3: p_k <- l(A_k)/r for the initial guess)
  for (int m = 0; m < D; ++m)
    CPA_TRY(refresh_distribution(Fm[m], X->dims[m], r, Cm[m], info + m, GA, flev, warn, scan_ws,
                                 false, nullptr, st));
  {
    // lambda = 1 until the first solve; fit = NaN unless computed
    std::vector<double> ones(kMaxRank, 1.0);
    const double nan4[4] = {NAN, NAN, NAN, NAN};
    CPA_CUDA_TRY(cudaMemcpyAsync(lam, ones.data(), sizeof(double) * kMaxRank, cudaMemcpyHostToDevice, st));
    CPA_CUDA_TRY(cudaMemcpyAsync(fitd, nan4, sizeof(nan4), cudaMemcpyHostToDevice, st));
    CPA_CUDA_TRY(cudaStreamSynchronize(st));
  }
  FactorPtrs F;
  for (int m = 0; m < D; ++m) F.A[m] = Fm[m];
  Profiler prof;
  prof.on = opt->profile != 0;
  prof.st = st;
  CPA_TRY(prof.mark(-1));
  int iters_done = 0, epochs = 0, bad = 0;
  double best = -INFINITY, fit_val = NAN;
  const int eta = opt->epoch_len > 0 ? opt->epoch_len : 1;
  int it = 0;
  while (it < opt->iters) {
    for (int l = 0; l < eta && it < opt->iters; ++l, ++it) {
      for (int k = 0; k < D; ++k) {
        const auto& mode = X->mode[k];
        SampleParams P;
        memset(&P, 0, sizeof(P));
        P.L = mode.L;
        for (int t = 0; t < mode.L.d; ++t) {
          P.D.C[t] = Cm[mode.L.mode[t]];
          P.D.info[t] = info + mode.L.mode[t];
          SB.cand_off[t] = 0;
        }
        {
          int64_t off = 0;
          for (int t = 0; t < mode.L.d; ++t) {
            SB.cand_off[t] = off;
            off += mode.L.n[t];
          }
          for (int t = mode.L.d; t < kMaxOrder; ++t) SB.cand_off[t] = off;
        }
        P.s = s;
        P.tau = tau;
        P.seed = opt->seed;
        P.iter = opt->iter_offset + (uint64_t)it;
        P.mode_k = k;
        P.reject_cap = opt->reject_cap;
        P.det_cap = det_cap;
        CPA_TRY(prof.mark(-1));
        CPA_TRY(skrp_lev(P, SB, st));
        CPA_TRY(prof.mark(0));
        const int64_t nk = X->dims[k];
        CPA_CUDA_TRY(cudaMemsetAsync(M, 0, sizeof(double) * nk * r, st));
        CPA_CUDA_TRY(cudaMemsetAsync(Gs, 0, sizeof(double) * r * r, st));
        cudaEvent_t mid = prof.pending(1);
        CPA_TRY(sampled_mttkrp(X, k, F, r, SB.idx_packed, SB.wgt, DevCount{&SB.state->sbar, s}, M, Gs,
                               MB, st, mid));
        CPA_TRY(prof.mark(2));
        CPA_TRY(factor_spd(Gs, r, 0, 0, 1e-13, fsolve, warn, CPA_WARN_SINGULAR_GRAM, st));
        CPA_TRY(solve_rows(M, nk, r, fsolve, Fm[k], st));
        CPA_TRY(prof.mark(3));
        CPA_TRY(refresh_distribution(Fm[k], nk, r, Cm[k], info + k, GA, flev, warn, scan_ws, true,
                                     nullptr, st));
        k_copy_lambda<<<1, 64, 0, st>>>(flev, r, lam);
        k_stats<<<1, 1, 0, st>>>(dstats, SB.state, MB.total, warn);
        CPA_LAUNCH_CHECK();
        CPA_TRY(prof.mark(4));
      }
    }
    iters_done = it;
    if (opt->tol > 0.0 && opt->fit_mode == CPA_FIT_EXACT) {
      CPA_TRY(prof.mark(-1));
      CPA_TRY(fit_enqueue(X, F, lam, r, fit_ws, fitd, st));
      CPA_TRY(prof.mark(5));
      double f = 0.0;
      int status = 0;
      CPA_CUDA_TRY(cudaMemcpyAsync(&f, fitd, sizeof(double), cudaMemcpyDeviceToHost, st));
      CPA_CUDA_TRY(cudaMemcpyAsync(&status, &SB.state->status, sizeof(int), cudaMemcpyDeviceToHost, st));
      CPA_CUDA_TRY(cudaStreamSynchronize(st));
      if (status < 0) return status;
      ++epochs;
      fit_val = f;
      if (f > best + opt->tol) {
        best = f;
        bad = 0;
      } else if (++bad >= opt->patience) {
        break;
      }
    }
  }
  if (!(opt->tol > 0.0) && opt->fit_mode == CPA_FIT_EXACT) {
    CPA_TRY(prof.mark(-1));
    CPA_TRY(fit_enqueue(X, F, lam, r, fit_ws, fitd, st));
    CPA_TRY(prof.mark(5));
    CPA_CUDA_TRY(cudaMemcpyAsync(&fit_val, fitd, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  int status = 0;
  DevStats hs;
  CPA_CUDA_TRY(cudaMemcpyAsync(&status, &SB.state->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(&hs, dstats, sizeof(hs), cudaMemcpyDeviceToHost, st));
  int hwarn = 0;
  CPA_CUDA_TRY(cudaMemcpyAsync(&hwarn, warn, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (status < 0) return status;
  const cudaMemcpyKind kout = io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int m = 0; m < D; ++m)
    CPA_CUDA_TRY(cudaMemcpyAsync(factors[m], Fm[m], sizeof(double) * X->dims[m] * r, kout, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(lambda, lam, sizeof(double) * r, kout, st));
  if (fit && io_on_device)
    CPA_CUDA_TRY(cudaMemcpyAsync(fit, fitd, sizeof(double), cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (fit && !io_on_device) *fit = opt->fit_mode == CPA_FIT_EXACT ? fit_val : NAN;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iters_done = iters_done;
    stats->mode_updates = iters_done * D;
    stats->warnings = hwarn;
    stats->epochs = epochs;
    stats->sdet_last = hs.sdet_last;
    stats->sbar_last = hs.sbar_last;
    stats->nnz_sampled_last = hs.nnz_last;
    stats->attempts_last = hs.attempts_last;
    stats->pdet_last = hs.pdet_last;
    stats->nnz_sampled_total = hs.nnz_total;
    stats->sbar_total = hs.sbar_total;
    prof.collect(stats);
  }
  return hwarn;
}

int cp_arls_lev_coo(const cpa_coo* coo, const cpa_options* opt, double* lambda, double* const* factors,
                    int32_t io_on_device, double* fit, cpa_stats* stats) {
  CPA_TRY(check_options(opt));
  cpa_index* X = nullptr;
  CPA_TRY(cpa_index_build(coo, opt->stream, &X));
  const int rc = cp_arls_lev(X, opt, lambda, factors, io_on_device, fit, stats);
  cpa_index_free(X);
  return rc;
}

}  // extern "C"
