// C ABI of the CP-ARLS-LEV library (include/cpa.h) and the Alg. 3 driver.
//
// The driver keeps everything on the device: per mode the factor matrix, its
// fixed-point CDF and distribution summary; per update one SkrpLev pass, the fused
// sampled MTTKRP, the FP64 solve, the Gram + leverage refresh of the solved mode.
// The host enqueues all of it and reads status, statistics and the fit once at the
// end (and once per epoch when the fit-based stopping rule is on).
#include <math.h>

#include <algorithm>
#include <memory>
#include <mutex>
#include <vector>

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

__global__ void k_copy_lambda(const SmallFactor* f, int r, double* lambda) {
  if (threadIdx.x < r) lambda[threadIdx.x] = f->lambda[threadIdx.x];
}

// end of one mode update: lambda of the solved mode and the statistics
__global__ void k_finish_update(const SmallFactor* f, int r, double* lambda, DevStats* ds,
                                const SampleState* S, const uint64_t* nnz, const int* warn) {
  if (threadIdx.x < r) lambda[threadIdx.x] = f->lambda[threadIdx.x];
  if (threadIdx.x == 0) {
    ds->sdet_last = S->sdet;
    ds->sbar_last = S->sbar;
    ds->nnz_last = (int64_t)*nnz;
    ds->attempts_last = (int64_t)S->attempts;
    ds->pdet_last = S->pdet;
    ds->nnz_total += (int64_t)*nnz;
    ds->sbar_total += S->sbar;
    ds->warnings = *warn;
  }
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

template <class TO, class TI>
__global__ void k_convert(const TI* __restrict__ in, int64_t n, TO* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
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
// place when `normalize_out` (the update path), untouched otherwise.  GA receives the
// factor's Gram (block-ordered sums in S).
// dist: the row distribution (leverage, or uniform / length-squared for comparison);
// the Gram and its factor are formed in every case (lambda, normalisation).
// src (optional, row stride lda): the rows are read from src and the normalised
// rows written to A (the update with the solve folded into the sampled MTTKRP, whose
// output src holds the unnormalised new factor).
template <class FT>
int refresh_distribution(FT* A, int64_t n, int r, uint64_t* C, DistInfo* info, double* Pm,
                         double* GA, const BlockSums& S, SmallFactor* fac, int* warn, void* scan_scratch,
                         bool normalize_out, double* lev_out, cudaStream_t st, int dist = CPA_DIST_LEVERAGE,
                         const FT* src = nullptr, int lda = 0, int* status = nullptr) {
  const FT* in = src ? src : A;
  CPA_TRY(gram_rows<FT>(in, n, r, GA, S, st, src ? lda : r, status));
  // a rank-deficient factor matters only to leverage scores (warning bit 0: no warning);
  // the pivots are cut where the Gram's own rounding would reach them
  const double tol = lev_pivot_tol<FT>(in, n, r, src ? lda : r, status);
  CPA_TRY(factor_spd(GA, r, 1, 1, tol, fac, warn, dist == CPA_DIST_LEVERAGE ? CPA_WARN_RANK_DEFICIENT_LEV : 0,
                     st, info));
  CPA_TRY(lev_rows<FT>(in, n, r, fac, lev_out, C, info, normalize_out || src ? A : nullptr, st, dist,
                       src ? lda : r, status));
  CPA_TRY(cdf_from_q(C, C, n, info, Pm, scan_scratch, st));
  return CPA_OK;
}

// Optional stage timing: events recorded at stage boundaries on the work stream.
struct Profiler {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> stage_of;  // stage of the interval ending at event i (-1: none)
  std::vector<cudaEvent_t> pool;  // created ahead of a stream capture
  void reserve(int n) {
    for (int i = 0; i < n; ++i) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) == cudaSuccess) pool.push_back(e);
    }
  }
  cudaEvent_t make() {
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    ev.push_back(e);
    stage_of.push_back(-1);
    return e;
  }
  // mark the end of an interval of `stage` that began at the previous mark
  int mark(int stage) {
    if (!on) return CPA_OK;
    cudaEvent_t e = make();
    stage_of.back() = stage;
    CPA_CUDA_TRY(record_event(e, st));
    return CPA_OK;
  }
  // an event for the caller to record later (it ends an interval of `stage`)
  cudaEvent_t pending(int stage) {
    if (!on) return nullptr;
    cudaEvent_t e = make();
    stage_of.back() = stage;
    return e;
  }
  // add the intervals between consecutive marks to s->stage_ms
  void collect_add(cpa_stats* s) {
    if (!on || !s) return;
    for (size_t i = 1; i < ev.size(); ++i) {
      if (stage_of[i] < 0) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i - 1], ev[i]) == cudaSuccess) {
        s->stage_ms[stage_of[i]] += ms;
        s->stage_launches[stage_of[i]] += 1;
      }
    }
  }
  ~Profiler() {
    for (auto e : ev) cudaEventDestroy(e);
    for (auto e : pool) cudaEventDestroy(e);
  }
};

int check_options(const cpa_options* o) {
  if (!o) return CPA_ERR_ARG;
  if (o->rank < 1 || o->rank > kMaxRank) return CPA_ERR_ARG;
  if (o->samples < 1 || o->samples >= (1ll << 31)) return CPA_ERR_ARG;
  if (!(o->tau >= 0.0 && o->tau <= 1.0)) return CPA_ERR_ARG;
  if (o->iters < 0 || o->reject_cap < 1 || o->det_cap < 1) return CPA_ERR_ARG;
  if (o->precision != CPA_FP64 && o->precision != CPA_MIXED) return CPA_ERR_ARG;
  if (o->distribution != CPA_DIST_LEVERAGE && o->distribution != CPA_DIST_UNIFORM &&
      o->distribution != CPA_DIST_LENGTH_SQUARED)
    return CPA_ERR_ARG;
  if (o->fit_mode != CPA_FIT_EXACT && o->fit_mode != CPA_FIT_NONE && o->fit_mode != CPA_FIT_ESTIMATED)
    return CPA_ERR_ARG;
  if (o->fit_mode == CPA_FIT_ESTIMATED && (o->fit_samples < 1 || !(o->fit_alpha > 0.0 && o->fit_alpha <= 1.0)))
    return CPA_ERR_ARG;
  if (o->tol < 0.0) return CPA_ERR_ARG;
  return CPA_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Plan: the workspace of cp_arls_lev for one (index, rank, s, tau, ...) and the
// instantiated CUDA graph of one outer iteration (every mode updated once).  The
// Philox iteration lives in device memory and the graph advances it, so the graph
// is replayed unchanged for every iteration and every later call.
// ---------------------------------------------------------------------------
namespace cpa {

__global__ void k_advance_iter(uint64_t* it) { *it += 1; }

// Per-call state: lambda = 1, fit = NaN, iteration counter = the caller's offset.
__global__ void k_run_init(double* lam, double* fitd, uint64_t* it, uint64_t it0) {
  for (int i = threadIdx.x; i < kMaxRank; i += blockDim.x) lam[i] = 1.0;
  if (threadIdx.x < 4) fitd[threadIdx.x] = NAN;
  if (threadIdx.x == 0) *it = it0;
}

// As k_run_init with the iteration offset read from, and advanced in, device memory
// (a captured call continues where the previous replay stopped).
__global__ void k_run_init_dev(double* lam, double* fitd, uint64_t* it, uint64_t* it0, uint64_t advance) {
  for (int i = threadIdx.x; i < kMaxRank; i += blockDim.x) lam[i] = 1.0;
  if (threadIdx.x < 4) fitd[threadIdx.x] = NAN;
  __syncthreads();
  if (threadIdx.x == 0) {
    *it = *it0;
    *it0 += advance;
  }
}

// Status of a captured call: the sticky status word, the warnings and the counters.
struct CallOut {
  int status;
  int warnings;
  int64_t nnz_total;
  int64_t sbar_total;
  int64_t sdet_last, sbar_last, nnz_last, attempts_last;
  double pdet_last;
};
__global__ void k_call_out(const int* status, const int* warn, const DevStats* ds, CallOut* out) {
  out->status = *status;
  out->warnings = *warn;
  out->nnz_total = ds->nnz_total;
  out->sbar_total = ds->sbar_total;
  out->sdet_last = ds->sdet_last;
  out->sbar_last = ds->sbar_last;
  out->nnz_last = ds->nnz_last;
  out->attempts_last = ds->attempts_last;
  out->pdet_last = ds->pdet_last;
}

constexpr int kEpochGraphMax = 256;  // longest fixed-length call run as one graph

struct Plan {
  // key
  int r = 0, D = 0, reject_cap = 0, profile = 0, prec = CPA_FP64, ftb = 8, dist = CPA_DIST_LEVERAGE;
  int64_t s = 0, det_cap = 0, det_buf = 0;
  int64_t fold_min = 0;  // modes of at least this many rows take the folded update
  double tau = 0.0;
  uint64_t seed = 0;
  // workspace
  char* base = nullptr;
  void* Fm[kMaxOrder] = {};   // factors in the run's element type (ftb bytes)
  uint64_t* Cm[kMaxOrder] = {};
  double* Pm[kMaxOrder] = {};
  double* stage64 = nullptr;  // FP64 staging of one factor (mixed precision in/out)
  DistInfo* info = nullptr;
  void* M = nullptr;
  double *Gs = nullptr, *GA = nullptr, *lam = nullptr, *fitd = nullptr, *fit_ws = nullptr;
  SmallFactor *fsolve = nullptr, *flev = nullptr;
  BlockSums sums_lev;   // block-ordered sums of the factor Grams and the fit (main stream)
  BlockSums sums_gram;  // of the sampled Gram (its own branch)
  int* warn = nullptr;
  DevStats* dstats = nullptr;
  char* scan_ws = nullptr;
  uint64_t* iter_dev = nullptr;
  SampleBuffers SB[kMaxOrder];
  MttkrpBuffers MB;
  Fork fork;  // side stream of the Gram branch
  // graph of one outer iteration
  bool use_graph = false;
  cudaGraphExec_t exec = nullptr;       // one outer iteration
  cudaGraphExec_t init_exec = nullptr;  // initial leverage distributions
  cudaGraphExec_t fit_exec = nullptr;   // exact fit
  int64_t k_iter = 0, k_init = 0, k_fit = 0;  // kernel nodes of each graph
  cudaGraph_t g_iter = nullptr, g_init = nullptr, g_fit = nullptr;  // kept to compose the epoch
  cudaGraphExec_t epoch_exec = nullptr;  // init + epoch_iters iterations + fit, one launch
  int epoch_iters = -1;
  int epoch_fit = CPA_FIT_NONE;
  // estimated fit (Section 5.4): the element sample and the graph that evaluates it
  FitSample est;
  cudaGraphExec_t est_exec = nullptr;
  cudaGraph_t g_est = nullptr;
  int64_t k_est = 0;
  int64_t k_epoch = 0;
  cudaStream_t cap_stream = nullptr;
  Profiler gprof;  // event nodes captured into the graph (profile = 1)

  bool matches(const cpa_options* o) const {
    return o->rank == r && o->samples == s && o->tau == tau && o->seed == seed &&
           o->reject_cap == reject_cap && o->det_cap == det_cap && (o->profile != 0) == (profile != 0) &&
           o->precision == prec && o->distribution == dist;
  }

  int init(const cpa_index* X, const cpa_options* o, cudaStream_t st) {
    r = o->rank;
    D = X->order;
    s = o->samples;
    tau = o->tau;
    seed = o->seed;
    reject_cap = o->reject_cap;
    det_cap = o->det_cap;
    profile = o->profile != 0;
    prec = o->precision;
    dist = o->distribution;
    ftb = prec == CPA_MIXED ? 4 : 8;
    det_buf = det_buffer_capacity(s, tau, det_cap);
    use_graph = !(tau < 1.0 && tau * (double)s < 1.0);  // no top-s host sync possible
    int64_t nmax = 1, nsum = 0;
    bool slabs = false;  // some mode's M is accumulated slab by slab, or its update folded
    fold_min = fold_rows();
    for (int m = 0; m < D; ++m) {
      nmax = std::max<int64_t>(nmax, X->dims[m]);
      nsum += X->dims[m];
      slabs = slabs || mttkrp_slabs(X->dims[m], r, ftb) > 1 || X->dims[m] >= fold_min;
    }
    KeyLayout Lsum;
    memset(&Lsum, 0, sizeof(Lsum));
    Lsum.d = 1;
    Lsum.n[0] = nsum;
    Arena a;
    for (int pass = 0; pass < 2; ++pass) {
      a.used = 0;
      for (int m = 0; m < D; ++m) {
        Fm[m] = a.take<char>((size_t)X->dims[m] * r * ftb);
        Cm[m] = a.take<uint64_t>(X->dims[m]);
        Pm[m] = a.take<double>(X->dims[m]);
      }
      stage64 = prec == CPA_MIXED ? a.take<double>((size_t)nmax * r) : nullptr;
      info = a.take<DistInfo>(kMaxOrder);
      M = a.take<char>((size_t)nmax * fold_ldm(r, ftb) * ftb);
      Gs = a.take<double>(r * r);
      GA = a.take<double>(r * r);
      lam = a.take<double>(kMaxRank);
      fitd = a.take<double>(4);
      fit_ws = a.take<double>(fit_buffers_bytes(D, r) / sizeof(double) + 1);
      fsolve = a.take<SmallFactor>(1);
      flev = a.take<SmallFactor>(1);
      sums_lev = a.take_sums(kSumMaxBlocks, gram_sums_width(r));
      sums_gram = a.take_sums(kSumMaxBlocks, gram_sums_width(r));
      warn = a.take<int>(4);
      dstats = a.take<DevStats>(1);
      scan_ws = a.take<char>(scan_workspace(nmax));
      iter_dev = a.take<uint64_t>(1);
      sample_buffers_carve(a, Lsum, s, det_buf, &SB[0]);
      mttkrp_buffers_carve(a, s, r, ftb, slabs, &MB, det_capacity(X, prec));
      if (pass == 0) {
        if (cudaMalloc((void**)&a.base, a.used) != cudaSuccess) return CPA_ERR_OOM;
        base = a.base;
      }
    }
    if (cudaStreamCreateWithFlags(&fork.aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork.ev_join, cudaEventDisableTiming) != cudaSuccess)
      return CPA_ERR_CUDA;
    MB.status = &SB[0].state->status;  // the tensor-core Gram reports a timed-out wait here
    // per-mode copies of the sample buffers differ only in the candidate offsets
    for (int k = 0; k < D; ++k) {
      SB[k] = SB[0];
      const KeyLayout& L = X->mode[k].L;
      int64_t off = 0;
      for (int t = 0; t < L.d; ++t) {
        SB[k].cand_off[t] = off;
        off += L.n[t];
      }
      for (int t = L.d; t < kMaxOrder; ++t) SB[k].cand_off[t] = off;
    }
    CPA_CUDA_TRY(cudaMemsetAsync(SB[0].state, 0, sizeof(SampleState), st));
    CPA_CUDA_TRY(cudaMemsetAsync(sums_lev.ticket, 0, sizeof(unsigned), st));
    CPA_CUDA_TRY(cudaMemsetAsync(sums_gram.ticket, 0, sizeof(unsigned), st));
    // the combine table starts empty; each pass's compaction empties it again
    CPA_CUDA_TRY(cudaMemsetAsync(SB[0].hkeys, 0xff, sizeof(uint64_t) << SB[0].hbits, st));
    CPA_CUDA_TRY(cudaMemsetAsync(SB[0].hcnt, 0, sizeof(uint32_t) << SB[0].hbits, st));
    return CPA_OK;
  }

  // Enqueue one outer iteration: every mode updated once (Alg. 3 inner loop).
  int enqueue_iteration(const cpa_index* X, Profiler& prof, cudaStream_t st) {
    return prec == CPA_MIXED ? enqueue_iteration_t<float>(X, prof, st)
                             : enqueue_iteration_t<double>(X, prof, st);
  }

  template <class FT>
  int enqueue_iteration_t(const cpa_index* X, Profiler& prof, cudaStream_t st) {
    FactorPtrs F;
    for (int m = 0; m < D; ++m) F.A[m] = Fm[m];
    for (int k = 0; k < D; ++k) {
      const auto& mode = X->mode[k];
      SampleParams Ps;
      memset(&Ps, 0, sizeof(Ps));
      Ps.L = mode.L;
      for (int t = 0; t < mode.L.d; ++t) {
        Ps.D.C[t] = Cm[mode.L.mode[t]];
        Ps.D.info[t] = info + mode.L.mode[t];
        Ps.D.P[t] = Pm[mode.L.mode[t]];
      }
      Ps.s = s;
      Ps.tau = tau;
      Ps.seed = seed;
      Ps.iter_ptr = iter_dev;
      Ps.mode_k = k;
      Ps.reject_cap = reject_cap;
      Ps.det_cap = tau < 1.0 ? det_cap : 1;
      Ps.det_buf = det_buf;
      CPA_TRY(prof.mark(-1));
      // FP64: the sampled rows in ascending key order, so that every later sum over
      // them (Gram, MTTKRP) runs in one order and the run is reproducible
      CPA_TRY(skrp_lev(Ps, SB[k], st, prec == CPA_FP64));
      CPA_TRY(prof.mark(0));
      const int64_t nk = X->dims[k];
      FT* Mt = static_cast<FT*>(M);
      FT* Fk = static_cast<FT*>(Fm[k]);
      cudaEvent_t evs[2] = {prof.pending(-1), prof.pending(1)};
      if (nk >= fold_min) {
        // the solve folded into the sampled MTTKRP: Mt holds the unnormalised new
        // factor, which the leverage refresh normalises into Fk
        const int ldm = fold_ldm(r, ftb);
        CPA_TRY(sampled_mttkrp_fold<FT>(X, k, F, r, SB[k].idx_packed, SB[k].wgt, DevCount{&SB[k].state->sbar, s},
                                        Mt, ldm, Gs, fsolve, warn, MB, st, prof.on ? evs : nullptr));
        CPA_TRY(prof.mark(2));
        CPA_TRY(prof.mark(3));
        CPA_TRY(refresh_distribution<FT>(Fk, nk, r, Cm[k], info + k, Pm[k], GA, sums_lev, flev, warn, scan_ws,
                                         true, nullptr, st, dist, Mt, ldm, MB.status));
      } else {
        CPA_TRY(sampled_mttkrp<FT>(X, k, F, r, SB[k].idx_packed, SB[k].wgt, DevCount{&SB[k].state->sbar, s},
                                   Mt, Gs, MB, st, prof.on ? evs : nullptr, &fork));
        CPA_TRY(prof.mark(2));
        CPA_TRY(factor_spd(Gs, r, 0, 0, 1e-13, fsolve, warn, CPA_WARN_SINGULAR_GRAM, st));
        CPA_TRY(solve_rows<FT>(Mt, nk, r, fsolve, Fk, st, GA));
        CPA_TRY(prof.mark(3));
        CPA_TRY(refresh_distribution<FT>(Fk, nk, r, Cm[k], info + k, Pm[k], GA, sums_lev, flev, warn, scan_ws,
                                         true, nullptr, st, dist, nullptr, 0, MB.status));
      }
      k_finish_update<<<1, 64, 0, st>>>(flev, r, lam, dstats, SB[k].state, MB.total, warn);
      CPA_LAUNCH_CHECK();
      CPA_TRY(prof.mark(4));
    }
    k_advance_iter<<<1, 1, 0, st>>>(iter_dev);
    CPA_LAUNCH_CHECK();
    return CPA_OK;
  }

  // Graphs are captured on a private stream (the legacy default stream cannot be
  // captured) and launched on the caller's stream.  *nk receives the number of
  // kernel nodes of the graph.
  template <class Fn>
  int capture_graph(Fn&& fn, cudaGraphExec_t* out, int64_t* nk, cudaGraph_t* keep = nullptr) {
    cudaGraph_t g = nullptr;
    if (!cap_stream) CPA_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    CPA_CUDA_TRY(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = fn(cap_stream);
    const cudaError_t ec = cudaStreamEndCapture(cap_stream, &g);
    if (rc < 0 || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc < 0 ? rc : CPA_ERR_CUDA;
    }
    size_t n = 0;
    int64_t kernels = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) == cudaSuccess && n > 0) {
      std::vector<cudaGraphNode_t> nodes(n);
      if (cudaGraphGetNodes(g, nodes.data(), &n) == cudaSuccess)
        for (size_t i = 0; i < n; ++i) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
        }
    }
    *nk = kernels;
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    if (keep) *keep = g; else cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      *out = nullptr;
      return CPA_ERR_CUDA;
    }
    return CPA_OK;
  }

  // One outer iteration (all D updates), replayed per iteration.
  int capture(const cpa_index* X) {
    gprof.on = profile != 0;
    gprof.st = nullptr;
    if (gprof.on) gprof.reserve(7 * D);
    return capture_graph(
        [&](cudaStream_t cs) {
          gprof.st = cs;
          return enqueue_iteration(X, gprof, cs);
        },
        &exec, &k_iter, &g_iter);
  }

  // Leverage distributions of the initial factors (Alg. 3 starts from l(A_k)/r).
  int enqueue_init(const cpa_index* X, cudaStream_t st) {
    for (int m = 0; m < D; ++m) {
      if (prec == CPA_MIXED)
        CPA_TRY(refresh_distribution<float>(static_cast<float*>(Fm[m]), X->dims[m], r, Cm[m], info + m,
                                            Pm[m], GA, sums_lev, flev, warn, scan_ws, false, nullptr, st, dist,
                                            nullptr, 0, MB.status));
      else
        CPA_TRY(refresh_distribution<double>(static_cast<double*>(Fm[m]), X->dims[m], r, Cm[m], info + m,
                                             Pm[m], GA, sums_lev, flev, warn, scan_ws, false, nullptr, st, dist,
                                             nullptr, 0, MB.status));
    }
    return CPA_OK;
  }

  // The fit of the current factors into fitd: exact (Eq. 5.1) or estimated from the
  // drawn element sample (Section 5.4).
  int enqueue_fit(const cpa_index* X, int kind, cudaStream_t st) {
    FactorPtrs F;
    for (int m = 0; m < D; ++m) F.A[m] = Fm[m];
    if (kind == CPA_FIT_ESTIMATED)
      return prec == CPA_MIXED ? fit_estimate_enqueue<float>(X, est, F, lam, r, fitd, st)
                               : fit_estimate_enqueue<double>(X, est, F, lam, r, fitd, st, static_cast<double*>(M));
    return prec == CPA_MIXED ? fit_enqueue<float>(X, F, lam, r, fit_ws, sums_lev, fitd, st)
                             : fit_enqueue<double>(X, F, lam, r, fit_ws, sums_lev, fitd, st);
  }

  // Draws the element sample of the estimated fit unless the one held matches the
  // options; a new sample invalidates the graphs that read the old one.
  int ensure_est(const cpa_index* X, const cpa_options* o, cudaStream_t st, int64_t* kernels = nullptr) {
    if (est.coords && est.s_fit == o->fit_samples && est.alpha == o->fit_alpha && est.seed == o->seed &&
        est.reject_cap == o->reject_cap)
      return CPA_OK;
    if (est_exec) {
      cudaGraphExecDestroy(est_exec);
      est_exec = nullptr;
    }
    if (g_est) {
      cudaGraphDestroy(g_est);
      g_est = nullptr;
    }
    if (epoch_exec && epoch_fit == CPA_FIT_ESTIMATED) {
      cudaGraphExecDestroy(epoch_exec);
      epoch_exec = nullptr;
    }
    CPA_TRY(fit_sample_draw(X, o->fit_samples, o->fit_alpha, o->seed, o->reject_cap, &est, st));
    CPA_TRY(fit_sample_sort(X, &est, st));
    (void)kernels;  // one-time work, not counted (see cpa_stats.kernel_launches)
    return CPA_OK;
  }

  int run(const cpa_index* X, const cpa_options* opt, double* lambda, double* const* factors,
          int32_t io_on_device, double* fit, cpa_stats* stats, cudaStream_t st);

  // One update of mode k (the driver's steps), rows exported in ascending order.
  template <class FT>
  int update_once(const cpa_index* X, int k, uint64_t iter, uint64_t* idx_linear, cudaStream_t st) {
    FactorPtrs F;
    for (int m = 0; m < D; ++m) F.A[m] = Fm[m];
    const auto& mode = X->mode[k];
    SampleParams Ps;
    memset(&Ps, 0, sizeof(Ps));
    Ps.L = mode.L;
    for (int t = 0; t < mode.L.d; ++t) {
      Ps.D.C[t] = Cm[mode.L.mode[t]];
      Ps.D.info[t] = info + mode.L.mode[t];
      Ps.D.P[t] = Pm[mode.L.mode[t]];
    }
    Ps.s = s;
    Ps.tau = tau;
    Ps.seed = seed;
    Ps.iter = iter;
    Ps.mode_k = k;
    Ps.reject_cap = reject_cap;
    Ps.det_cap = tau < 1.0 ? det_cap : 1;
    Ps.det_buf = det_buf;
    SampleBuffers B = SB[k];
    B.idx_linear = idx_linear;
    CPA_TRY(skrp_lev(Ps, B, st, true));
    const int64_t nk = X->dims[k];
    FT* Mt = static_cast<FT*>(M);
    FT* Fk = static_cast<FT*>(Fm[k]);
    if (nk >= fold_min) {
      const int ldm = fold_ldm(r, ftb);
      CPA_TRY(sampled_mttkrp_fold<FT>(X, k, F, r, B.idx_packed, B.wgt, DevCount{&B.state->sbar, s}, Mt, ldm, Gs,
                                      fsolve, warn, MB, st));
      CPA_TRY(refresh_distribution<FT>(Fk, nk, r, Cm[k], info + k, Pm[k], GA, sums_lev, flev, warn, scan_ws, true,
                                       nullptr, st, dist, Mt, ldm, MB.status));
    } else {
      CPA_TRY(sampled_mttkrp<FT>(X, k, F, r, B.idx_packed, B.wgt, DevCount{&B.state->sbar, s}, Mt, Gs, MB,
                                 st));
      CPA_TRY(factor_spd(Gs, r, 0, 0, 1e-13, fsolve, warn, CPA_WARN_SINGULAR_GRAM, st));
      CPA_TRY(solve_rows<FT>(Mt, nk, r, fsolve, Fk, st));
      CPA_TRY(refresh_distribution<FT>(Fk, nk, r, Cm[k], info + k, Pm[k], GA, sums_lev, flev, warn, scan_ws, true,
                                       nullptr, st, dist, nullptr, 0, MB.status));
    }
    k_copy_lambda<<<1, 64, 0, st>>>(flev, r, lam);
    CPA_LAUNCH_CHECK();
    return CPA_OK;
  }

  // A whole fixed-length call on device buffers as one graph (batched entry point):
  // state reset, copy-in, initial leverage, `iters` outer iterations, fit, copy-out
  // and the call's status into *out.  The iteration offset lives in *it0_dev and is
  // advanced by `iters` per replay.  Grid sizes follow num_sms() at capture time.
  int capture_call(const cpa_index* X, int iters, int fit_kind, double* lambda, double* const* factors,
                   double* fit_dev, uint64_t* it0_dev, CallOut* out, cudaGraph_t* g_out) {
    if (!cap_stream) CPA_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = cap_stream;
    Profiler off;
    cudaGraph_t g = nullptr;
    CPA_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    auto body = [&]() -> int {
      CPA_CUDA_TRY(cudaMemsetAsync(warn, 0, sizeof(int) * 4, cs));
      CPA_CUDA_TRY(cudaMemsetAsync(dstats, 0, sizeof(DevStats), cs));
      CPA_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(DistInfo) * kMaxOrder, cs));
      CPA_CUDA_TRY(cudaMemsetAsync(&SB[0].state->status, 0, sizeof(int), cs));
      for (int m = 0; m < D; ++m) {
        const int64_t cnt = X->dims[m] * r;
        if (prec == CPA_MIXED) {
          CPA_CUDA_TRY(cudaMemcpyAsync(stage64, factors[m], sizeof(double) * cnt, cudaMemcpyDeviceToDevice, cs));
          k_convert<float, double><<<blocks(cnt), 256, 0, cs>>>(stage64, cnt, static_cast<float*>(Fm[m]));
          CPA_LAUNCH_CHECK();
        } else {
          CPA_CUDA_TRY(cudaMemcpyAsync(Fm[m], factors[m], sizeof(double) * cnt, cudaMemcpyDeviceToDevice, cs));
        }
      }
      k_run_init_dev<<<1, 64, 0, cs>>>(lam, fitd, iter_dev, it0_dev, (uint64_t)iters);
      CPA_LAUNCH_CHECK();
      CPA_TRY(enqueue_init(X, cs));
      for (int i = 0; i < iters; ++i) CPA_TRY(enqueue_iteration(X, off, cs));
      if (fit_kind != CPA_FIT_NONE) CPA_TRY(enqueue_fit(X, fit_kind, cs));
      for (int m = 0; m < D; ++m) {
        const int64_t cnt = X->dims[m] * r;
        if (prec == CPA_MIXED) {
          k_convert<double, float><<<blocks(cnt), 256, 0, cs>>>(static_cast<const float*>(Fm[m]), cnt, stage64);
          CPA_LAUNCH_CHECK();
          CPA_CUDA_TRY(cudaMemcpyAsync(factors[m], stage64, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, cs));
        } else {
          CPA_CUDA_TRY(cudaMemcpyAsync(factors[m], Fm[m], sizeof(double) * cnt, cudaMemcpyDeviceToDevice, cs));
        }
      }
      CPA_CUDA_TRY(cudaMemcpyAsync(lambda, lam, sizeof(double) * r, cudaMemcpyDeviceToDevice, cs));
      if (fit_dev) CPA_CUDA_TRY(cudaMemcpyAsync(fit_dev, fitd, sizeof(double), cudaMemcpyDeviceToDevice, cs));
      k_call_out<<<1, 1, 0, cs>>>(&SB[0].state->status, warn, dstats, out);
      CPA_LAUNCH_CHECK();
      return CPA_OK;
    };
    const int rc = body();
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (rc < 0 || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc < 0 ? rc : CPA_ERR_CUDA;
    }
    *g_out = g;
    return CPA_OK;
  }

  // One graph for a whole fixed-length call: the initial leverage, `iters` replays of
  // the outer iteration and the fit, as child graphs in a chain.  A single launch
  // per call leaves the GPU queue full whatever the host does meanwhile.
  int build_epoch(int iters, int fit_kind) {
    if (epoch_exec && epoch_iters == iters && epoch_fit == fit_kind) return CPA_OK;
    if (epoch_exec) {
      cudaGraphExecDestroy(epoch_exec);
      epoch_exec = nullptr;
    }
    cudaGraph_t eg = nullptr;
    CPA_CUDA_TRY(cudaGraphCreate(&eg, 0));
    cudaGraphNode_t prev = nullptr, node = nullptr;
    int rc = CPA_OK;
    auto add = [&](cudaGraph_t child) {
      if (rc < 0) return;
      if (cudaGraphAddChildGraphNode(&node, eg, prev ? &prev : nullptr, prev ? 1 : 0, child) != cudaSuccess)
        rc = CPA_ERR_CUDA;
      prev = node;
    };
    add(g_init);
    for (int i = 0; i < iters; ++i) add(g_iter);
    if (fit_kind == CPA_FIT_EXACT) add(g_fit);
    if (fit_kind == CPA_FIT_ESTIMATED) add(g_est);
    if (rc == CPA_OK && cudaGraphInstantiate(&epoch_exec, eg, 0) != cudaSuccess) {
      epoch_exec = nullptr;
      rc = CPA_ERR_CUDA;
    }
    cudaGraphDestroy(eg);
    if (rc < 0) return rc;
    epoch_iters = iters;
    epoch_fit = fit_kind;
    k_epoch = k_init + (int64_t)iters * k_iter + (fit_kind == CPA_FIT_EXACT ? k_fit : 0) +
              (fit_kind == CPA_FIT_ESTIMATED ? k_est : 0);
    return CPA_OK;
  }

  ~Plan() {
    if (epoch_exec) cudaGraphExecDestroy(epoch_exec);
    if (g_iter) cudaGraphDestroy(g_iter);
    if (g_init) cudaGraphDestroy(g_init);
    if (g_fit) cudaGraphDestroy(g_fit);
    if (g_est) cudaGraphDestroy(g_est);
    if (est_exec) cudaGraphExecDestroy(est_exec);
    if (exec) cudaGraphExecDestroy(exec);
    if (init_exec) cudaGraphExecDestroy(init_exec);
    if (fit_exec) cudaGraphExecDestroy(fit_exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (fork.aux) cudaStreamDestroy(fork.aux);
    if (fork.ev_fork) cudaEventDestroy(fork.ev_fork);
    if (fork.ev_join) cudaEventDestroy(fork.ev_join);
    if (base) {
      cudaDeviceSynchronize();
      cudaFree(base);
    }
  }
};

void plan_free(Plan* p) { delete p; }

int Plan::run(const cpa_index* X, const cpa_options* opt, double* lambda, double* const* factors,
              int32_t io_on_device, double* fit, cpa_stats* stats, cudaStream_t st) {
  int64_t kernels = 0;  // launched by this call
  if (opt->fit_mode == CPA_FIT_ESTIMATED) CPA_TRY(ensure_est(X, opt, st, &kernels));
  CPA_CUDA_TRY(cudaMemsetAsync(warn, 0, sizeof(int) * 4, st));
  CPA_CUDA_TRY(cudaMemsetAsync(dstats, 0, sizeof(DevStats), st));
  CPA_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(DistInfo) * kMaxOrder, st));
  CPA_CUDA_TRY(cudaMemsetAsync(&SB[0].state->status, 0, sizeof(int), st));
  const cudaMemcpyKind kin = io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int m = 0; m < D; ++m) {
    const int64_t cnt = X->dims[m] * r;
    if (prec == CPA_MIXED) {
      CPA_CUDA_TRY(cudaMemcpyAsync(stage64, factors[m], sizeof(double) * cnt, kin, st));
      k_convert<float, double><<<blocks(cnt), 256, 0, st>>>(stage64, cnt, static_cast<float*>(Fm[m]));
      CPA_LAUNCH_CHECK();
      ++kernels;
    } else {
      CPA_CUDA_TRY(cudaMemcpyAsync(Fm[m], factors[m], sizeof(double) * cnt, kin, st));
    }
  }
  k_run_init<<<1, 64, 0, st>>>(lam, fitd, iter_dev, opt->iter_offset);
  CPA_LAUNCH_CHECK();
  ++kernels;
  cudaEvent_t call0 = nullptr, call1 = nullptr;
  if (profile) {
    cudaEventCreate(&call0);
    cudaEventCreate(&call1);
    cudaEventRecord(call0, st);
  }
  // fixed-length call without stage events: the whole call is one graph launch
  const bool one_graph = use_graph && !profile && !(opt->tol > 0.0) && opt->iters <= kEpochGraphMax;
  const int fit_kind = opt->fit_mode;
  if (use_graph) {
    if (!init_exec)
      CPA_TRY(capture_graph([&](cudaStream_t cs) { return enqueue_init(X, cs); }, &init_exec, &k_init, &g_init));
    if (!exec) CPA_TRY(capture(X));
    if (!fit_exec)
      CPA_TRY(capture_graph([&](cudaStream_t cs) { return enqueue_fit(X, CPA_FIT_EXACT, cs); }, &fit_exec, &k_fit,
                            &g_fit));
    if (fit_kind == CPA_FIT_ESTIMATED && !est_exec)
      CPA_TRY(capture_graph([&](cudaStream_t cs) { return enqueue_fit(X, CPA_FIT_ESTIMATED, cs); }, &est_exec,
                            &k_est, &g_est));
    if (one_graph) {
      CPA_TRY(build_epoch(opt->iters, fit_kind));
      CPA_CUDA_TRY(cudaGraphLaunch(epoch_exec, st));
      kernels += k_epoch;
    } else {
      CPA_CUDA_TRY(cudaGraphLaunch(init_exec, st));
      kernels += k_init;
    }
  } else {
    CPA_TRY(enqueue_init(X, st));
    kernels = -1;
  }
  // the fit, as a graph where the updates run as one
  auto fit_now = [&](Profiler& pr) -> int {
    CPA_TRY(pr.mark(-1));
    if (use_graph) {
      CPA_CUDA_TRY(cudaGraphLaunch(fit_kind == CPA_FIT_ESTIMATED ? est_exec : fit_exec, st));
      if (kernels >= 0) kernels += fit_kind == CPA_FIT_ESTIMATED ? k_est : k_fit;
    } else {
      CPA_TRY(enqueue_fit(X, fit_kind, st));
    }
    return pr.mark(5);
  };
  Profiler eprof;  // eager path
  eprof.on = profile != 0;
  eprof.st = st;
  CPA_TRY(eprof.mark(-1));
  cpa_stats acc;
  memset(&acc, 0, sizeof(acc));
  int iters_done = 0, epochs = 0, bad = 0;
  double best = -INFINITY, fit_val = NAN;
  const int eta = opt->epoch_len > 0 ? opt->epoch_len : 1;
  int it = 0;
  if (one_graph) it = opt->iters;  // done by the graph launched above
  iters_done = it;
  while (it < opt->iters) {
    for (int l = 0; l < eta && it < opt->iters; ++l, ++it) {
      if (use_graph) {
        CPA_CUDA_TRY(cudaGraphLaunch(exec, st));
        kernels += k_iter;
        if (profile) {  // the captured events hold this replay's timestamps
          CPA_CUDA_TRY(cudaStreamSynchronize(st));
          gprof.collect_add(&acc);
        }
      } else {
        CPA_TRY(enqueue_iteration(X, eprof, st));
      }
    }
    iters_done = it;
    if (opt->tol > 0.0 && fit_kind != CPA_FIT_NONE) {
      CPA_TRY(fit_now(eprof));
      double f = 0.0;
      int status = 0;
      CPA_CUDA_TRY(cudaMemcpyAsync(&f, fitd, sizeof(double), cudaMemcpyDeviceToHost, st));
      CPA_CUDA_TRY(cudaMemcpyAsync(&status, &SB[0].state->status, sizeof(int), cudaMemcpyDeviceToHost, st));
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
  if (!(opt->tol > 0.0) && fit_kind != CPA_FIT_NONE) {
    if (!one_graph) CPA_TRY(fit_now(eprof));
    CPA_CUDA_TRY(cudaMemcpyAsync(&fit_val, fitd, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  if (profile) cudaEventRecord(call1, st);
  int status = 0;
  DevStats hs;
  int hwarn = 0;
  CPA_CUDA_TRY(cudaMemcpyAsync(&status, &SB[0].state->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(&hs, dstats, sizeof(hs), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(&hwarn, warn, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (status < 0) return status;
  const cudaMemcpyKind kout = io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int m = 0; m < D; ++m) {
    const int64_t cnt = X->dims[m] * r;
    if (prec == CPA_MIXED) {
      k_convert<double, float><<<blocks(cnt), 256, 0, st>>>(static_cast<const float*>(Fm[m]), cnt, stage64);
      CPA_LAUNCH_CHECK();
      if (kernels >= 0) ++kernels;
      CPA_CUDA_TRY(cudaMemcpyAsync(factors[m], stage64, sizeof(double) * cnt, kout, st));
      CPA_CUDA_TRY(cudaStreamSynchronize(st));  // stage64 is reused by the next mode
    } else {
      CPA_CUDA_TRY(cudaMemcpyAsync(factors[m], Fm[m], sizeof(double) * cnt, kout, st));
    }
  }
  CPA_CUDA_TRY(cudaMemcpyAsync(lambda, lam, sizeof(double) * r, kout, st));
  if (fit && io_on_device) CPA_CUDA_TRY(cudaMemcpyAsync(fit, fitd, sizeof(double), cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (fit && !io_on_device) *fit = fit_kind != CPA_FIT_NONE ? fit_val : NAN;
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
    stats->kernel_launches = kernels;
    if (profile) {
      eprof.collect_add(stats);
      for (int i = 0; i < 6; ++i) {
        stats->stage_ms[i] += acc.stage_ms[i];
        stats->stage_launches[i] += acc.stage_launches[i];
      }
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, call0, call1) == cudaSuccess) stats->stage_ms[8] = ms;
      stats->stage_launches[8] = 1;
    }
  }
  if (call0) cudaEventDestroy(call0);
  if (call1) cudaEventDestroy(call1);
  return hwarn;
}

}  // namespace cpa


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
  opt->fit_samples = 1ll << 27;
  opt->fit_alpha = 0.5;
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

int cpa_index_device_bytes(const cpa_index* X, int64_t* bytes) {
  if (!X || !bytes) return CPA_ERR_ARG;
  *bytes = (int64_t)X->device_bytes;
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
    int* warn = a.take<int>(2);  // warning bits, then the status word of the streaming Gram
    BlockSums sums = a.take_sums(kSumMaxBlocks, gram_sums_width(r));
    if (pass == 0) {
      CPA_TRY(buf.alloc(a.used, st));
      a.base = (char*)buf.p;
      continue;
    }
    CPA_CUDA_TRY(cudaMemsetAsync(warn, 0, 2 * sizeof(int), st));
    CPA_CUDA_TRY(cudaMemsetAsync(sums.ticket, 0, sizeof(unsigned), st));
    CPA_TRY(gram_rows<double>(A, n, r, G, sums, st, r, warn + 1));
    CPA_TRY(factor_spd(G, r, 1, 1, 1e-12, f, warn, CPA_WARN_RANK_DEFICIENT_LEV, st));
    CPA_TRY(lev_rows<double>(A, n, r, f, lev, nullptr, nullptr, (double*)nullptr, st));
    int hwarn[2] = {0, 0};
    CPA_CUDA_TRY(cudaMemcpyAsync(hwarn, warn, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CPA_CUDA_TRY(cudaStreamSynchronize(st));
    return hwarn[1] ? hwarn[1] : hwarn[0];
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
  CPA_TRY(cdf_from_q(C, C, n, info, nullptr, scratch, st));
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
  const int64_t det_buf = det_buffer_capacity(s, opt->tau, opt->det_cap);
  int64_t nmax = 1;
  for (int t = 0; t < d; ++t) nmax = std::max<int64_t>(nmax, dims[t]);
  DevBuf buf;
  Arena a;
  SampleBuffers B;
  uint64_t* Cs[kMaxOrder];
  double* Ps[kMaxOrder];
  DistInfo* info = nullptr;
  char* scan_ws = nullptr;
  for (int pass = 0; pass < 2; ++pass) {
    a.used = 0;
    for (int t = 0; t < d; ++t) {
      Cs[t] = a.take<uint64_t>(dims[t]);
      Ps[t] = a.take<double>(dims[t]);
    }
    info = a.take<DistInfo>(kMaxOrder);
    scan_ws = a.take<char>(scan_workspace(nmax));
    sample_buffers_carve(a, L, s, det_buf, &B);
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
    CPA_TRY(cdf_from_q(Cs[t], Cs[t], dims[t], info + t, Ps[t], scan_ws, st));
  }
  SampleParams P;
  memset(&P, 0, sizeof(P));
  P.L = L;
  for (int t = 0; t < d; ++t) {
    P.D.C[t] = Cs[t];
    P.D.info[t] = info + t;
    P.D.P[t] = Ps[t];
  }
  P.s = s;
  P.tau = opt->tau;
  P.seed = opt->seed;
  P.iter = iter;
  P.mode_k = mode_k;
  P.reject_cap = opt->reject_cap;
  P.det_cap = det_cap;
  P.det_buf = det_buf;
  P.iter_ptr = nullptr;
  CPA_TRY(skrp_lev(P, B, st, true));
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
  if (sbar == 0) {
    CPA_CUDA_TRY(cudaMemsetAsync(M, 0, sizeof(double) * X->dims[mode_k] * r, st));
    CPA_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double) * r * r, st));
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
    mttkrp_buffers_carve(a, sbar, r, (int)sizeof(double), mttkrp_slabs(X->dims[mode_k], r, 8) > 1, &B,
                         det_capacity(X, CPA_FP64));
    if (pass == 0) {
      CPA_TRY(buf.alloc(a.used, st));
      a.base = (char*)buf.p;
    }
  }
  k_linear_to_packed<<<blocks(sbar), 256, 0, st>>>(mode.L, idx, sbar, packed);
  CPA_LAUNCH_CHECK();
  CPA_TRY(sampled_mttkrp<double>(X, mode_k, F, r, packed, wgt, DevCount{nullptr, sbar}, M, G, B, st));
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
  const size_t sums_bytes = block_sums_bytes(kSumMaxBlocks, gram_sums_width(r));
  CPA_TRY(buf.alloc(sizeof(SmallFactor) * 2 + sizeof(double) * r * r + 1024 + sums_bytes, st));
  SmallFactor* fs = (SmallFactor*)buf.p;
  SmallFactor* fl = fs + 1;
  double* GA = (double*)(fl + 1);
  int* warn = (int*)(GA + r * r);
  BlockSums sums = block_sums_at((char*)buf.p + sizeof(SmallFactor) * 2 + sizeof(double) * r * r + 1024, kSumMaxBlocks);
  CPA_CUDA_TRY(cudaMemsetAsync(warn, 0, sizeof(int), st));
  CPA_CUDA_TRY(cudaMemsetAsync(sums.ticket, 0, sizeof(unsigned), st));
  CPA_TRY(factor_spd(G, r, 0, 0, 1e-13, fs, warn, CPA_WARN_SINGULAR_GRAM, st));
  CPA_TRY(solve_rows<double>(M, n, r, fs, A, st));
  CPA_TRY(gram_rows<double>(A, n, r, GA, sums, st));
  int dummy_warn_bit = 0;
  CPA_TRY(factor_spd(GA, r, 1, 1, 1e-12, fl, warn, dummy_warn_bit, st));
  k_copy_lambda<<<1, 64, 0, st>>>(fl, r, lambda);
  CPA_TRY(scale_columns<double>(A, n, r, lambda, st));
  int hwarn = 0;
  CPA_CUDA_TRY(cudaMemcpyAsync(&hwarn, warn, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  return hwarn;
}

int cpa_rrf_init(const cpa_index* X, int32_t mode, int64_t s_init, uint64_t seed, const double* omega, int32_t r,
                 double* A, void* stream) {
  if (!X) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CPA_TRY(rrf_enqueue(X, mode, s_init, seed, omega, r, A, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  return CPA_OK;
}

int cpa_fit_sample(const cpa_index* X, int64_t fit_samples, double fit_alpha, uint64_t seed, int32_t reject_cap,
                   int32_t* coords, double* xs, int64_t* counts, double* phi, void* stream) {
  if (!X || !coords || !xs || !counts || !phi) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FitSample S;
  CPA_TRY(fit_sample_draw(X, fit_samples, fit_alpha, seed, reject_cap, &S, st));
  const int64_t n = S.s_nz + S.s_z;
  for (int m = 0; m < X->order; ++m)
    CPA_CUDA_TRY(cudaMemcpyAsync(coords + (size_t)m * fit_samples, S.coords + (size_t)m * S.s_fit,
                                 sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(xs, S.xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  counts[0] = S.s_nz;
  counts[1] = S.s_z;
  counts[2] = S.attempts;
  phi[0] = S.phi[0];
  phi[1] = S.phi[1];
  return CPA_OK;
}

int cpa_fit_estimate(const cpa_index* X, const int32_t* coords, const double* xs, const int64_t* counts,
                     const double* phi, int64_t stride, const double* lambda, const double* const* factors,
                     int32_t r, int32_t precision, double* fit, double* F_hat, void* stream) {
  if (!X || !coords || !xs || !counts || !phi || !lambda || !factors || !fit || r < 1 || r > kMaxRank)
    return CPA_ERR_ARG;
  if (precision != CPA_FP64 && precision != CPA_MIXED) return CPA_ERR_ARG;
  if (counts[0] < 0 || counts[1] < 0 || counts[0] + counts[1] > stride) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int D = X->order;
  int64_t conv = 0;
  for (int m = 0; m < D; ++m) {
    if (!factors[m]) return CPA_ERR_ARG;
    conv += X->dims[m] * r;
  }
  DevBuf buf;
  const size_t partial_bytes = sizeof(double) * ((size_t)device_sms() * 8 + 8);
  CPA_TRY(buf.alloc(partial_bytes + 64 + (precision == CPA_MIXED ? sizeof(float) * conv + 256 : 0), st));
  double* fit_dev = (double*)buf.p;
  FitSample S;  // a view of the caller's sample: released as a view below
  S.coords = const_cast<int32_t*>(coords);
  S.xs = const_cast<double*>(xs);
  S.partial = fit_dev + 8;
  S.stride = stride;
  S.s_nz = counts[0];
  S.s_z = counts[1];
  S.phi[0] = phi[0];
  S.phi[1] = phi[1];
  FactorPtrs F;
  int rc = CPA_OK;
  if (precision == CPA_MIXED) {
    float* f32 = reinterpret_cast<float*>((char*)buf.p + partial_bytes + 64);
    for (int m = 0; m < D; ++m) {
      const int64_t cnt = X->dims[m] * r;
      k_convert<float, double><<<blocks(cnt), 256, 0, st>>>(factors[m], cnt, f32);
      F.A[m] = f32;
      f32 += cnt;
    }
    if (cudaGetLastError() != cudaSuccess) rc = CPA_ERR_CUDA;
    if (rc == CPA_OK) rc = fit_estimate_enqueue<float>(X, S, F, lambda, r, fit_dev, st);
  } else {
    for (int m = 0; m < D; ++m) F.A[m] = factors[m];
    rc = fit_estimate_enqueue<double>(X, S, F, lambda, r, fit_dev, st);
  }
  double h[2] = {NAN, NAN};
  if (rc == CPA_OK) {
    if (cudaMemcpyAsync(h, fit_dev, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = CPA_ERR_CUDA;
  }
  S.coords = nullptr;
  S.xs = nullptr;
  S.partial = nullptr;
  if (rc < 0) return rc;
  *fit = h[0];
  if (F_hat) *F_hat = h[1];
  return CPA_OK;
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
  const size_t fb = (fit_buffers_bytes(X->order, r) + 256 + 255) & ~size_t(255);
  CPA_TRY(buf.alloc(fb + block_sums_bytes(kSumMaxBlocks, gram_sums_width(r)), st));
  double* fit_dev = (double*)buf.p;
  double* scratch = fit_dev + 32;
  BlockSums sums = block_sums_at((char*)buf.p + fb, kSumMaxBlocks);
  CPA_CUDA_TRY(cudaMemsetAsync(sums.ticket, 0, sizeof(unsigned), st));
  CPA_TRY(fit_enqueue<double>(X, F, lambda, r, scratch, sums, fit_dev, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(fit, fit_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  return CPA_OK;
}

int cpa_fit_terms(const cpa_index* X, const double* const* factors, const double* lambda, int32_t r,
                  double* terms, void* stream) {
  if (!X || !factors || !lambda || !terms || r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FactorPtrs F;
  for (int m = 0; m < X->order; ++m) {
    if (!factors[m]) return CPA_ERR_ARG;
    F.A[m] = factors[m];
  }
  DevBuf buf;
  const size_t fb = (fit_buffers_bytes(X->order, r) + 256 + 255) & ~size_t(255);
  CPA_TRY(buf.alloc(fb + block_sums_bytes(kSumMaxBlocks, gram_sums_width(r)), st));
  double* fit_dev = (double*)buf.p;  // fit_dev[0]: fit, [1..3]: the terms
  double* scratch = fit_dev + 32;
  BlockSums sums = block_sums_at((char*)buf.p + fb, kSumMaxBlocks);
  CPA_CUDA_TRY(cudaMemsetAsync(sums.ticket, 0, sizeof(unsigned), st));
  CPA_TRY(fit_enqueue<double>(X, F, lambda, r, scratch, sums, fit_dev, st, fit_dev + 1));
  CPA_CUDA_TRY(cudaMemcpyAsync(terms, fit_dev + 1, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  return CPA_OK;
}

int cp_arls_lev(const cpa_index* Xc, const cpa_options* opt, double* lambda, double* const* factors,
                int32_t io_on_device, double* fit, cpa_stats* stats) {
  if (!Xc || !lambda || !factors) return CPA_ERR_ARG;
  CPA_TRY(check_options(opt));
  cpa_index* X = const_cast<cpa_index*>(Xc);  // only the plan cache is modified
  const int D = X->order;
  for (int m = 0; m < D; ++m)
    if (!factors[m]) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)opt->stream;
  // a cached plan per index; a concurrent call on the same index gets its own
  std::unique_lock<std::mutex> lock(X->plan_mu, std::try_to_lock);
  Plan* own = nullptr;
  Plan* P = nullptr;
  if (lock.owns_lock()) {
    if (X->plan && !X->plan->matches(opt)) {
      plan_free(X->plan);
      X->plan = nullptr;
    }
    if (!X->plan) {
      X->plan = new (std::nothrow) Plan();
      if (!X->plan) return CPA_ERR_OOM;
      const int rc = X->plan->init(X, opt, st);
      if (rc < 0) {
        plan_free(X->plan);
        X->plan = nullptr;
        return rc;
      }
    }
    P = X->plan;
  } else {
    own = new (std::nothrow) Plan();
    if (!own) return CPA_ERR_OOM;
    const int rc = own->init(X, opt, st);
    if (rc < 0) {
      plan_free(own);
      return rc;
    }
    P = own;
  }
  const int rc = P->run(X, opt, lambda, factors, io_on_device, fit, stats, st);
  if (own) plan_free(own);
  return rc;
}

int cpa_mode_update(const cpa_index* X, const cpa_options* opt, int32_t mode_k, uint64_t iter,
                    double* const* factors, double* lambda, uint64_t* idx, uint32_t* cnt, double* wgt,
                    int64_t* counts, double* pdet) {
  if (!X || !factors || !lambda || !idx || !cnt || !wgt || mode_k < 0 || mode_k >= X->order)
    return CPA_ERR_ARG;
  CPA_TRY(check_options(opt));
  for (int m = 0; m < X->order; ++m)
    if (!factors[m]) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)opt->stream;
  Plan* P = new (std::nothrow) Plan();
  if (!P) return CPA_ERR_OOM;
  struct Guard {
    Plan* p;
    ~Guard() { plan_free(p); }
  } guard{P};
  CPA_TRY(P->init(X, opt, st));
  const int D = X->order, r = P->r;
  CPA_CUDA_TRY(cudaMemsetAsync(P->warn, 0, sizeof(int) * 4, st));
  CPA_CUDA_TRY(cudaMemsetAsync(P->info, 0, sizeof(DistInfo) * kMaxOrder, st));
  for (int m = 0; m < D; ++m) {
    const int64_t c = X->dims[m] * r;
    if (P->prec == CPA_MIXED) {
      k_convert<float, double><<<blocks(c), 256, 0, st>>>(factors[m], c, static_cast<float*>(P->Fm[m]));
      CPA_LAUNCH_CHECK();
      CPA_TRY(refresh_distribution<float>(static_cast<float*>(P->Fm[m]), X->dims[m], r, P->Cm[m], P->info + m,
                                          P->Pm[m], P->GA, P->sums_lev, P->flev, P->warn, P->scan_ws, false, nullptr,
                                          st, P->dist));
    } else {
      CPA_CUDA_TRY(cudaMemcpyAsync(P->Fm[m], factors[m], sizeof(double) * c, cudaMemcpyDeviceToDevice, st));
      CPA_TRY(refresh_distribution<double>(static_cast<double*>(P->Fm[m]), X->dims[m], r, P->Cm[m],
                                           P->info + m, P->Pm[m], P->GA, P->sums_lev, P->flev, P->warn, P->scan_ws,
                                           false, nullptr, st, P->dist));
    }
  }
  if (P->prec == CPA_MIXED) CPA_TRY(P->update_once<float>(X, mode_k, iter, idx, st));
  else CPA_TRY(P->update_once<double>(X, mode_k, iter, idx, st));
  SampleState h;
  int hwarn = 0;
  CPA_CUDA_TRY(cudaMemcpyAsync(&h, P->SB[mode_k].state, sizeof(h), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(&hwarn, P->warn, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (h.status < 0) return h.status;
  const int64_t c = X->dims[mode_k] * r;
  if (P->prec == CPA_MIXED)
    k_convert<double, float><<<blocks(c), 256, 0, st>>>(static_cast<const float*>(P->Fm[mode_k]), c,
                                                        factors[mode_k]);
  else
    CPA_CUDA_TRY(cudaMemcpyAsync(factors[mode_k], P->Fm[mode_k], sizeof(double) * c, cudaMemcpyDeviceToDevice,
                                 st));
  CPA_CUDA_TRY(cudaMemcpyAsync(lambda, P->lam, sizeof(double) * r, cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(cnt, P->SB[mode_k].cnt, sizeof(uint32_t) * h.sbar, cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(wgt, P->SB[mode_k].wgt, sizeof(double) * h.sbar, cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (counts) {
    counts[0] = h.sbar;
    counts[1] = h.sdet;
    counts[2] = (int64_t)h.attempts;
  }
  if (pdet) *pdet = h.pdet;
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

// ---------------------------------------------------------------------------
// Batched decompositions: many independent fixed-length cp_arls_lev calls as the
// branches of one CUDA graph (one launch), with the SM budget their kernels are sized
// for chosen by timing the candidate graphs.
// ---------------------------------------------------------------------------
struct cpa_batch {
  int n = 0;
  std::vector<cpa::Plan*> plans;
  std::vector<const cpa_index*> idx;
  std::vector<cpa_options> opts;
  std::vector<double*> lambdas, fits;
  std::vector<std::vector<double*>> factors;
  char* dev = nullptr;
  cpa::CallOut* outs = nullptr;
  uint64_t* it0 = nullptr;
  cudaGraphExec_t exec = nullptr;
  int budget = 0;
  int64_t kernels = 0;
  double tune_ms[4] = {0, 0, 0, 0};
  int tune_budget[4] = {0, 0, 0, 0};

  ~cpa_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto* p : plans) cpa::plan_free(p);
    if (dev) {
      cudaDeviceSynchronize();
      cudaFree(dev);
    }
  }

  // capture every problem's call with grids sized for `sms` SMs and compose them
  int build(int sms) {
    using namespace cpa;
    if (exec) {
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
    // element samples of estimated fits are drawn before any capture
    for (int i = 0; i < n; ++i)
      if (opts[i].fit_mode == CPA_FIT_ESTIMATED) CPA_TRY(plans[i]->ensure_est(idx[i], &opts[i], nullptr));
    cudaGraph_t bg = nullptr;
    CPA_CUDA_TRY(cudaGraphCreate(&bg, 0));
    int rc = CPA_OK;
    int64_t kern = 0;
    sm_budget_override() = sms;
    for (int i = 0; i < n && rc == CPA_OK; ++i) {
      cudaGraph_t g = nullptr;
      rc = plans[i]->capture_call(idx[i], opts[i].iters, opts[i].fit_mode, lambdas[i],
                                  factors[i].data(), fits[i], it0 + i, outs + i, &g);
      if (rc < 0) break;
      size_t nn = 0;
      if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
          for (size_t q = 0; q < nn; ++q) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[q], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
          }
      }
      cudaGraphNode_t node = nullptr;
      if (cudaGraphAddChildGraphNode(&node, bg, nullptr, 0, g) != cudaSuccess) rc = CPA_ERR_CUDA;
      cudaGraphDestroy(g);
    }
    sm_budget_override() = 0;
    if (rc == CPA_OK && cudaGraphInstantiate(&exec, bg, 0) != cudaSuccess) {
      exec = nullptr;
      rc = CPA_ERR_CUDA;
    }
    cudaGraphDestroy(bg);
    if (rc < 0) return rc;
    budget = sms;
    kernels = kern;
    return CPA_OK;
  }
};

extern "C" {

int cpa_batch_create(int32_t nprob, const cpa_index* const* indices, const cpa_options* opts,
                     double* const* lambdas, double* const* const* factors, double* const* fits,
                     int32_t autotune, void* stream, cpa_batch** out) {
  using namespace cpa;
  if (!out || nprob < 1 || !indices || !opts || !lambdas || !factors) return CPA_ERR_ARG;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < nprob; ++i) {
    const cpa_options& o = opts[i];
    CPA_TRY(check_options(&o));
    if (!indices[i] || !lambdas[i] || !factors[i]) return CPA_ERR_ARG;
    for (int m = 0; m < indices[i]->order; ++m)
      if (!factors[i][m]) return CPA_ERR_ARG;
    // fixed-length calls only, replayable as a graph
    if (o.tol > 0.0 || o.profile || o.iters > kEpochGraphMax) return CPA_ERR_UNSUPPORTED;
    if (o.tau < 1.0 && o.tau * (double)o.samples < 1.0) return CPA_ERR_UNSUPPORTED;
  }
  std::unique_ptr<cpa_batch> b(new (std::nothrow) cpa_batch());
  if (!b) return CPA_ERR_OOM;
  b->n = nprob;
  for (int i = 0; i < nprob; ++i) {
    b->idx.push_back(indices[i]);
    b->opts.push_back(opts[i]);
    b->lambdas.push_back(lambdas[i]);
    b->fits.push_back(fits ? fits[i] : nullptr);
    b->factors.emplace_back(factors[i], factors[i] + indices[i]->order);
    Plan* p = new (std::nothrow) Plan();
    if (!p) return CPA_ERR_OOM;
    b->plans.push_back(p);
    CPA_TRY(p->init(indices[i], &opts[i], st));
  }
  const size_t outs_bytes = ((sizeof(CallOut) * nprob + 255) / 256) * 256;
  if (cudaMalloc((void**)&b->dev, outs_bytes + sizeof(uint64_t) * nprob) != cudaSuccess) return CPA_ERR_OOM;
  b->outs = reinterpret_cast<CallOut*>(b->dev);
  b->it0 = reinterpret_cast<uint64_t*>(b->dev + outs_bytes);
  std::vector<uint64_t> it0h(nprob);
  for (int i = 0; i < nprob; ++i) it0h[i] = opts[i].iter_offset;
  CPA_CUDA_TRY(cudaMemcpy(b->it0, it0h.data(), sizeof(uint64_t) * nprob, cudaMemcpyHostToDevice));
  const int sms = num_sms();
  if (!autotune) {
    CPA_TRY(b->build(sms));
    *out = b.release();
    return CPA_OK;
  }
  // autotune: run each candidate once untimed and once timed from the same starting
  // factors and iteration offsets, restoring both afterwards
  std::vector<std::pair<double*, size_t>> snap;
  DevBuf sbuf;
  size_t total = 0;
  for (int i = 0; i < nprob; ++i)
    for (int m = 0; m < indices[i]->order; ++m) total += sizeof(double) * indices[i]->dims[m] * opts[i].rank;
  CPA_TRY(sbuf.alloc(total, st));
  auto copy_all = [&](bool save) -> int {
    char* q = (char*)sbuf.p;
    for (int i = 0; i < nprob; ++i)
      for (int m = 0; m < indices[i]->order; ++m) {
        const size_t nb = sizeof(double) * indices[i]->dims[m] * opts[i].rank;
        CPA_CUDA_TRY(cudaMemcpyAsync(save ? (void*)q : (void*)factors[i][m], save ? (void*)factors[i][m] : (void*)q,
                                     nb, cudaMemcpyDeviceToDevice, st));
        q += nb;
      }
    CPA_CUDA_TRY(cudaMemcpyAsync(b->it0, it0h.data(), sizeof(uint64_t) * nprob, cudaMemcpyHostToDevice, st));
    CPA_CUDA_TRY(cudaStreamSynchronize(st));
    return CPA_OK;
  };
  CPA_TRY(copy_all(true));
  const int cand[4] = {sms, (sms + 1) / 2, (sms + 3) / 4, (sms + 7) / 8};
  cudaEvent_t e0, e1;
  CPA_CUDA_TRY(cudaEventCreate(&e0));
  CPA_CUDA_TRY(cudaEventCreate(&e1));
  int best = -1;
  double best_ms = 0.0;
  int rc = CPA_OK;
  for (int c = 0; c < 4 && rc == CPA_OK; ++c) {
    rc = b->build(cand[c]);
    if (rc < 0) break;
    for (int rep = 0; rep < 2 && rc == CPA_OK; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess || cudaGraphLaunch(b->exec, st) != cudaSuccess ||
          cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        rc = CPA_ERR_CUDA;
    }
    float ms = 0.f;
    if (rc == CPA_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = CPA_ERR_CUDA;
    if (rc == CPA_OK) rc = copy_all(false);
    b->tune_budget[c] = cand[c];
    b->tune_ms[c] = ms;
    if (rc == CPA_OK && (best < 0 || ms < best_ms)) {
      best = c;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc < 0) return rc;
  if (b->budget != cand[best]) CPA_TRY(b->build(cand[best]));
  *out = b.release();
  return CPA_OK;
}

int cpa_batch_run(cpa_batch* b, void* stream, cpa_stats* stats) {
  using namespace cpa;
  if (!b || !b->exec) return CPA_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CPA_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  std::vector<CallOut> h(b->n);
  CPA_CUDA_TRY(cudaMemcpyAsync(h.data(), b->outs, sizeof(CallOut) * b->n, cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  int warn = 0;
  for (int i = 0; i < b->n; ++i) {
    if (h[i].status < 0) return h[i].status;
    warn |= h[i].warnings;
    if (stats) {
      cpa_stats& s = stats[i];
      memset(&s, 0, sizeof(s));
      s.iters_done = b->opts[i].iters;
      s.mode_updates = b->opts[i].iters * b->idx[i]->order;
      s.warnings = h[i].warnings;
      s.nnz_sampled_total = h[i].nnz_total;
      s.sbar_total = h[i].sbar_total;
      s.sdet_last = h[i].sdet_last;
      s.sbar_last = h[i].sbar_last;
      s.nnz_sampled_last = h[i].nnz_last;
      s.attempts_last = h[i].attempts_last;
      s.pdet_last = h[i].pdet_last;
      s.kernel_launches = i == 0 ? b->kernels : 0;  // the whole batch is counted once
    }
  }
  return warn;
}

int cpa_batch_info(const cpa_batch* b, int32_t* sm_budget, int32_t* cand_budgets, double* cand_ms,
                   int64_t* kernels) {
  if (!b) return CPA_ERR_ARG;
  if (sm_budget) *sm_budget = b->budget;
  for (int c = 0; c < 4; ++c) {
    if (cand_budgets) cand_budgets[c] = b->tune_budget[c];
    if (cand_ms) cand_ms[c] = b->tune_ms[c];
  }
  if (kernels) *kernels = b->kernels;
  return CPA_OK;
}

int cpa_batch_free(cpa_batch* b) {
  delete b;
  return CPA_OK;
}

}  // extern "C"
