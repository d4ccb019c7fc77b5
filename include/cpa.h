/*
 * cpa.h -- C ABI of the GB300 CP-ARLS-LEV library (libcpa.so).
 *
 * CP-ARLS-LEV (Larsen & Kolda, "Practical Leverage-Based Sampling for Low-Rank
 * Tensor Decomposition", Alg. 3) computes a rank-r CP decomposition of a sparse
 * (d+1)-way tensor by alternating least squares in which every least-squares
 * problem  min_B || Z B^T - X_(k)^T ||  (Eq. 1.1), Z the Khatri-Rao product of the
 * other factor matrices, is replaced by a sketch that keeps a few rows of Z chosen
 * by the product of the factors' leverage scores (Lemma 5.3), part of them
 * deterministically (Section 4.2, Section 5.3) and repeats merged (Section 4.1).
 *
 * Every step runs on one CUDA GPU (sm_103a kernels); the host only marshals
 * arguments.  All functions are synchronous with respect to the host: they enqueue
 * their work on the caller's stream and wait for it before returning.  Work of
 * different calls may overlap only if they use different streams and different
 * output buffers; one cpa_index may be shared by concurrent calls (read only).
 *
 * Conventions
 *  - Indices are 0-based (the paper is 1-based).
 *  - Factor matrices are row-major n_k x r.  The "other" modes of an update of
 *    mode k are the modes m != k in ascending order m_0 < ... < m_{d-1}; a
 *    multi-index (i_0, ..., i_{d-1}) over them has the linear index
 *      key = sum_t i_t * prod_{u<t} n_{m_u}     (Eq. 2.2, first mode fastest).
 *  - A pointer documented as "device" must be CUDA device (or managed) memory;
 *    "host" must be host memory.  The caller owns every buffer it passes; the
 *    library never frees caller memory.  cpa_index owns the device memory it
 *    allocates and releases it in cpa_index_free.
 *  - Return value: 0 = success, negative = error (CPA_ERR_*; outputs undefined),
 *    positive = success with warning bits (CPA_WARN_*).
 *  - stream: a cudaStream_t passed as void*; NULL means the legacy default stream.
 */
#ifndef CPA_H
#define CPA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define CPA_OK 0
#define CPA_ERR_ARG (-1)          /* invalid argument (rank <= 0, s < 1, tau outside [0,1], ...) */
#define CPA_ERR_COO_RANGE (-2)    /* a COO index is outside [0, dim) */
#define CPA_ERR_COO_DUP (-3)      /* the same coordinate appears twice */
#define CPA_ERR_OOM (-4)          /* device allocation failed */
#define CPA_ERR_REJECT_LIMIT (-5) /* a random slot was rejected reject_cap times in a row */
#define CPA_ERR_DET_CAP (-6)      /* deterministic candidate product exceeds det_cap */
#define CPA_ERR_CUDA (-7)         /* a CUDA runtime call or kernel failed */
#define CPA_ERR_UNSUPPORTED (-8)  /* shape outside the supported range (see each call) */
#define CPA_WARN_SINGULAR_GRAM 1      /* a sampled Gram matrix was singular: pinv used */
#define CPA_WARN_RANK_DEFICIENT_LEV 2 /* a factor matrix was rank deficient: pinv used */

/* ---- enumerations -------------------------------------------------------- */
#define CPA_F32 1 /* float values */
#define CPA_F64 2 /* double values */
#define CPA_FP64 0      /* every product and solve in FP64 */
#define CPA_MIXED 1     /* factors, Grams, sampled products and row solves in FP32 (FP64
                           accumulation across tiles); r x r factorisations, sampling
                           probabilities and lambda in FP64 */
#define CPA_DIST_LEVERAGE 0       /* row sampling by leverage scores (Lemma 5.3) */
#define CPA_DIST_UNIFORM 1        /* uniform rows of every factor (App. B comparison) */
#define CPA_DIST_LENGTH_SQUARED 2 /* squared row norms of every factor (App. B comparison) */
#define CPA_FIT_NONE 0  /* no fit computed (fit output set to NaN) */
#define CPA_FIT_EXACT 1 /* exact fit of Eq. 5.1 after the run (and per epoch if tol > 0) */
#define CPA_FIT_ESTIMATED 2 /* estimated fit of Section 5.4 from a stratified sample of
                               fit_samples elements (fraction fit_alpha nonzeros) */

/* Sparse tensor in coordinate format (Section 5.3: (d+2) nnz storage).
 *   order      number of modes D = d + 1, 2 <= D <= 8
 *   dims       host array of D mode sizes, each in [1, 2^31 - 1]
 *   nnz        number of stored nonzeros, 0 <= nnz < 2^35
 *   idx        host array of D pointers; idx[m][e] (int32) is the mode-m index of
 *              nonzero e.  The pointed-to arrays are device memory if on_device,
 *              host memory otherwise.
 *   vals       nnz values of type val_dtype (same memory space as idx[m])
 *   val_dtype  CPA_F32 or CPA_F64
 *   on_device  1 if idx[m] and vals are device pointers, 0 if host
 * Coordinates must be distinct (CPA_ERR_COO_DUP otherwise).  The packed
 * other-mode coordinates of every mode must fit in 64 bits:
 * sum_{m != k} ceil(log2 n_m) <= 63 for every k (CPA_ERR_UNSUPPORTED otherwise). */
typedef struct {
  int32_t order;
  const int64_t* dims;
  int64_t nnz;
  const int32_t* const* idx;
  const void* vals;
  int32_t val_dtype;
  int32_t on_device;
} cpa_coo;

/* Options of Alg. 3 (the defaults of cpa_options_default are the paper's Section 6
 * settings for the hybrid method with the fixed iteration count used here):
 *   rank        r >= 1 (r <= 64)
 *   samples     s >= 1 rows per least-squares problem (s < 2^31)
 *   tau         deterministic threshold in [0, 1]; 1 = random only, 1/s = hybrid
 *   iters       maximum number of outer iterations (each updates every mode once)
 *   epoch_len   eta, outer iterations per epoch (5)
 *   patience    pi, epochs without improvement before stopping (3)
 *   tol         fit improvement tolerance; 0 = run exactly `iters` iterations
 *   seed        Philox key of the random draws
 *   iter_offset added to the outer iteration number in the Philox counter, so a run
 *               can be resumed with the same stream of draws
 *   precision   CPA_FP64 or CPA_MIXED
 *   distribution  per-factor row distribution whose product is sampled:
 *               CPA_DIST_LEVERAGE (the method), or for comparison (App. B)
 *               CPA_DIST_UNIFORM (p_m(i) = 1/n_m) or CPA_DIST_LENGTH_SQUARED
 *               (p_m(i) = ||A_m(i,:)||^2 / ||A_m||_F^2 of the factor as the next
 *               Khatri-Rao product uses it: column-normalised after an update, as
 *               given at the start); the threshold, weights and combining are the
 *               same for all three
 *   fit_mode    CPA_FIT_EXACT, CPA_FIT_ESTIMATED or CPA_FIT_NONE
 *   fit_samples s_fit, elements in the sample of the estimated fit (>= 1; default
 *               2^27, the paper's Section 6 setting); used with CPA_FIT_ESTIMATED
 *   fit_alpha   fraction alpha in (0, 1] of the sample taken from the nonzeros
 *               (0.5); the sample is drawn once per (index, seed, fit_samples,
 *               fit_alpha, reject_cap) and reused by later calls
 *   det_cap     largest candidate product the deterministic search may enumerate
 *   reject_cap  largest number of draws of one random slot
 *   profile     1: time the stages of every update with CUDA events on `stream`
 *               (results in cpa_stats.stage_ms); 0: no timing
 *   stream      cudaStream_t (void*) for all work */
typedef struct {
  int32_t rank;
  int64_t samples;
  double tau;
  int32_t iters;
  int32_t epoch_len;
  int32_t patience;
  double tol;
  uint64_t seed;
  uint64_t iter_offset;
  int32_t precision;
  int32_t distribution;
  int32_t fit_mode;
  int64_t fit_samples;
  double fit_alpha;
  int64_t det_cap;
  int32_t reject_cap;
  int32_t profile;
  void* stream;
} cpa_options;

/* Statistics of a run (totals over all mode updates, plus the last update). */
typedef struct {
  int32_t iters_done;      /* outer iterations performed */
  int32_t mode_updates;    /* least-squares solves performed */
  int32_t warnings;        /* OR of CPA_WARN_* */
  int32_t epochs;          /* fits computed by the stopping rule */
  int64_t sdet_last;       /* s_det of the last update */
  int64_t sbar_last;       /* rows kept after combining, last update */
  int64_t nnz_sampled_last;/* nonzeros of the sampled right-hand side, last update */
  int64_t attempts_last;   /* random draws made (accepted + rejected), last update */
  double pdet_last;        /* p_det of the last update */
  int64_t nnz_sampled_total; /* sum over updates */
  int64_t sbar_total;      /* sum over updates */
  /* with cpa_options.profile = 1: milliseconds summed over all updates of
   * [0] SkrpLev (sampling, combine), [1] sampled KRP rows + sampled Gram (one
   * kernel), [2] fibre probe + sampled KRP rows + sampled MTTKRP (one kernel),
   * [3] the r x r solve, [4] the leverage refresh of the solved mode, [5] the
   * fit(s); and [8] the whole call.  stage_launches[i] counts the timed intervals.
   * Profiling runs [1] and [2] one after the other; otherwise they run concurrently. */
  double stage_ms[12];
  int64_t stage_launches[12];
  /* kernels this call launched on the GPU (each kernel node of a replayed CUDA
   * graph counted once per replay); -1 where the updates ran outside a graph
   * (the top-s path with tau * samples < 1), where the count is not kept.  The
   * one-time drawing and ordering of the estimated fit's element sample (first
   * call with new fit options) is not counted. */
  int64_t kernel_launches;
} cpa_stats;

typedef struct cpa_index cpa_index; /* opaque; owns device memory */

/* Fills *opt with: rank 10, samples 2^17, tau 2^-17, iters 10, epoch_len 5,
 * patience 3, tol 0, seed 0, iter_offset 0, CPA_FP64, CPA_DIST_LEVERAGE, CPA_FIT_EXACT, fit_samples
 * 2^27, fit_alpha 0.5, det_cap 2^24, reject_cap 4096, stream NULL. */
void cpa_options_default(cpa_options* opt);

/* Human-readable text of a status code (static string). */
const char* cpa_strerror(int code);

/* Builds the per-mode fibre index of Section 5.3 (every mode's linear indices
 * computed once and kept, D extra words per nonzero) on the GPU:
 * for every mode k the nonzeros are sorted by (other-mode multi-index, i_k), so the
 * fibre X(:, key) of every key is one contiguous run that a sampled key finds by
 * one probe.  Values are stored in the COO's dtype, fibre offsets as 32-bit words
 * (with the few fibres where the offsets pass a multiple of 2^32 kept aside).  The
 * build works in segments of at most 2^29 nonzeros by default (ranges of the
 * other mode of highest number; CPA_INDEX_SEGMENT_NNZ in the environment sets the
 * size), so its scratch is about 44 bytes per nonzero of a segment on top of the
 * index itself (about 8 bytes per nonzero and 12 per fibre, per mode).
 *   coo    input tensor (host or device, see cpa_coo)
 *   stream cudaStream_t
 *   out    receives the new index (host pointer to an opaque handle)
 * Errors: CPA_ERR_ARG, CPA_ERR_COO_RANGE, CPA_ERR_COO_DUP, CPA_ERR_UNSUPPORTED,
 * CPA_ERR_OOM, CPA_ERR_CUDA; *out is untouched on error. */
int cpa_index_build(const cpa_coo* coo, void* stream, cpa_index** out);

/* Releases an index (NULL is allowed). */
int cpa_index_free(cpa_index* index);

/* Shape of an index: order, mode sizes (host array of >= order entries, may be
 * NULL), nnz, and the number of distinct fibres F_k of mode `mode` (may be NULL). */
int cpa_index_info(const cpa_index* index, int32_t mode, int32_t* order, int64_t* dims,
                   int64_t* nnz, int64_t* nfib);

/* Device memory held by an index, in bytes (all modes: permuted streams, fibre
 * tables, directories, hash tables). */
int cpa_index_device_bytes(const cpa_index* index, int64_t* bytes);

/* Copies the fibre index of one mode to DEVICE buffers: keys[F_k] (linear keys of
 * Eq. 2.2, ascending), off[F_k + 1] (start of each fibre), ik[nnz] (mode index of
 * each nonzero in index order) and val[nnz] (values, index dtype).  Any output may
 * be NULL. */
int cpa_index_export(const cpa_index* index, int32_t mode, uint64_t* keys, uint64_t* off,
                     int32_t* ik, void* val, void* stream);

/* CP-ARLS-LEV, Alg. 3: runs opt->iters outer iterations (or stops earlier by the
 * epoch/patience rule when opt->tol > 0).
 *   index     tensor index from cpa_index_build
 *   opt       options (see cpa_options)
 *   lambda    r doubles, out: weights of the normalised model (column norms of the
 *             last factor solved)
 *   factors   array (host) of `order` pointers to n_k x r row-major doubles; in:
 *             initial guess, out: factors with unit-norm columns
 *   io_on_device  1 if lambda, fit and factors[k] are device pointers, 0 if host
 *   fit       out: fit of Eq. 5.1, or its estimate (Section 5.4) with
 *             CPA_FIT_ESTIMATED (the element sample of cpa_fit_sample with the
 *             run's seed, drawn at the first call and reused while the options
 *             keep it); NaN if fit_mode is CPA_FIT_NONE; may be NULL
 *   stats     out: statistics; may be NULL
 * Errors: CPA_ERR_ARG, CPA_ERR_REJECT_LIMIT, CPA_ERR_DET_CAP, CPA_ERR_OOM,
 * CPA_ERR_CUDA.  Warnings: CPA_WARN_SINGULAR_GRAM, CPA_WARN_RANK_DEFICIENT_LEV. */
int cp_arls_lev(const cpa_index* index, const cpa_options* opt, double* lambda,
                double* const* factors, int32_t io_on_device, double* fit, cpa_stats* stats);

/* Full CP-ALS (Sec. 2, Eq. 2.3: the exact least-squares update that Alg. 3
 * randomizes), for comparison and for the tau = 0 reduction at scale: per mode,
 * M = X_(k) times the Khatri-Rao product of the other factors (exact MTTKRP over the
 * mode-k fibre index), G = Hadamard product of the other factors' Grams, A_k =
 * M G^{-1} (FP64 factorisation, pseudo-inverse fallback), columns normalised into
 * lambda.  Runs exactly opt->iters outer iterations; uses opt->rank, iters,
 * precision (CPA_FP64 or CPA_MIXED: FP32 factors and MTTKRP), fit_mode
 * (CPA_FIT_NONE or CPA_FIT_EXACT; CPA_FIT_ESTIMATED is CPA_ERR_ARG), stream;
 * samples, tau, seed and the epoch rule are ignored.  Arguments, ownership and
 * errors as cp_arls_lev (stats: iters_done, mode_updates, warnings only). */
int cp_als(const cpa_index* index, const cpa_options* opt, double* lambda, double* const* factors,
           int32_t io_on_device, double* fit, cpa_stats* stats);

/* Batched decompositions (no counterpart in the paper; the serving pattern of many
 * independent CP-ARLS-LEV runs, e.g. random restarts or ranks, sharing the GPU).
 * A batch holds nprob fixed-length cp_arls_lev calls on DEVICE buffers; each run
 * replays all of them as the independent branches of one CUDA graph (one launch),
 * each call continuing its decomposition where the previous run stopped (the
 * Philox iteration offset advances by opts[i].iters per run).
 *   indices   nprob tensor indices (may repeat)
 *   opts      nprob options: tol must be 0, profile 0, iters <= 256, and the draws
 *             graph-replayable (not tau < 1 with tau * samples < 1), else
 *             CPA_ERR_UNSUPPORTED
 *   lambdas   nprob device pointers to r_i doubles (out)
 *   factors   nprob host arrays of order_i device pointers (in/out, as cp_arls_lev)
 *   fits      nprob device pointers to one double (out), or NULL
 *   autotune  1: time the batch graph with its kernels sized for all, 1/2, 1/4 and
 *             1/8 of the SMs (two runs each from the same factors, which are then
 *             restored) and keep the fastest; 0: all SMs
 * The buffers must stay valid for the batch's lifetime; cpa_batch_free releases it.
 * Errors as cp_arls_lev; CPA_ERR_UNSUPPORTED as above. */
typedef struct cpa_batch cpa_batch;
int cpa_batch_create(int32_t nprob, const cpa_index* const* indices, const cpa_options* opts,
                     double* const* lambdas, double* const* const* factors, double* const* fits,
                     int32_t autotune, void* stream, cpa_batch** out);
/* Runs every call of the batch once (one graph launch, then one synchronisation).
 * stats (nprob entries, may be NULL): iters_done, mode_updates, warnings, the
 * sampled-row totals and the last update's counters (sdet, sbar, nnz_sampled,
 * attempts, pdet); kernel_launches of the whole launch in stats[0]. Returns the first
 * negative status of a call, else the OR of the warnings. */
int cpa_batch_run(cpa_batch* batch, void* stream, cpa_stats* stats);
/* The SM budget chosen, the four candidate budgets and their timed milliseconds
 * (zeros without autotuning) and the kernel nodes of one run; outputs may be NULL. */
int cpa_batch_info(const cpa_batch* batch, int32_t* sm_budget, int32_t* cand_budgets, double* cand_ms,
                   int64_t* kernels);
int cpa_batch_free(cpa_batch* batch);

/* The same from a COO tensor: builds the index, runs cp_arls_lev and frees the
 * index.  Arguments as for cpa_index_build and cp_arls_lev. */
int cp_arls_lev_coo(const cpa_coo* coo, const cpa_options* opt, double* lambda,
                    double* const* factors, int32_t io_on_device, double* fit, cpa_stats* stats);

/* One update of mode `mode_k` (the inner step of Alg. 3): leverage scores of every
 * factor, SkrpLev over the other modes, the sampled MTTKRP and Gram, the solve, the
 * normalisation -- the same kernels and precision as cp_arls_lev (opt->precision).
 *   factors   host array of `order` DEVICE pointers to n_m x r doubles; factor
 *             mode_k is overwritten with the new (column-normalised) factor
 *   lambda    device, r doubles out
 *   iter      global outer iteration of the Philox counters
 *   idx, cnt, wgt  device outputs (opt->samples entries): the rows used, in the
 *             order of cpa_skrp_lev (linear keys, counts, weights)
 *   counts    host out: {sbar, s_det, attempts}; pdet: host out
 * Errors as cp_arls_lev. */
int cpa_mode_update(const cpa_index* index, const cpa_options* opt, int32_t mode_k, uint64_t iter,
                    double* const* factors, double* lambda, uint64_t* idx, uint32_t* cnt, double* wgt,
                    int64_t* counts, double* pdet);

/* ---- randomized range finder initialisation (App. F) ----------------------------- */

/* Initial factor of mode `mode` as a random linear combination of the tensor's
 * mode-k fibres (the columns of the unfolding X_(k)): A = X_(k)(:, S) Omega, S =
 * s_init fibres drawn uniformly with replacement from the F_k nonzero fibres.  Draw j
 * takes the fibre at position floor(u F_k / 2^64) in ascending order of the fibre's
 * linear key (Eq. 2.2), u = word 0 of Philox4x64-10(counter (j, 0, 3<<32 | mode, 0),
 * key (seed, 0)).
 *   omega   device, s_init x r row-major doubles: the Gaussian combination weights,
 *           drawn by the caller
 *   A       device, n_mode x r row-major doubles out (overwritten)
 * The sums are FP64 atomic additions (order not fixed).  Errors: CPA_ERR_ARG (mode
 * out of range, s_init < 1, r outside [1, 64], empty tensor), CPA_ERR_CUDA. */
int cpa_rrf_init(const cpa_index* index, int32_t mode, int64_t s_init, uint64_t seed, const double* omega,
                 int32_t r, double* A, void* stream);

/* ---- estimated fit (Section 5.4) ------------------------------------------------ */

/* Draws the stratified element sample of the estimated fit: s_nz = ceil(alpha *
 * fit_samples) nonzeros and s_z = fit_samples - s_nz zero cells (the paper's
 * floor((1 - alpha) s_fit) in exact arithmetic; 0 if the tensor has no zero cell),
 * each uniform over its stratum, with replacement.
 *   nonzero slot j: u = word 0 of Philox4x64-10(counter (j, 0, 2<<32, 0), key
 *     (seed, 0)); the nonzero at position floor(u nnz / 2^64) in ascending order of
 *     the linear index of Eq. 2.2 over all modes (mode 0 fastest)
 *   zero slot j, attempt a: i_m = floor(u_m n_m / 2^64) with u_m word m % 4 of
 *     Philox(counter (j, a, 2<<32 | 1 | (m/4)<<16, 0), key (seed, 0)); the attempt
 *     is rejected if the cell is a nonzero
 *   coords  device, order x fit_samples int32 (row m at coords + m * fit_samples)
 *   xs      device, fit_samples doubles: the values (nonzero samples first, then
 *           zeros with value 0)
 *   counts  host out: {s_nz, s_z, zero-cell attempts}
 *   phi     host out: {nnz / s_nz, (prod n - nnz) / s_z} (0 for an empty stratum)
 * Errors: CPA_ERR_ARG (fit_samples < 1, alpha outside (0, 1], nnz = 0,
 * reject_cap < 1), CPA_ERR_REJECT_LIMIT (a zero slot drew reject_cap nonzeros in a
 * row), CPA_ERR_OOM, CPA_ERR_CUDA. */
int cpa_fit_sample(const cpa_index* index, int64_t fit_samples, double fit_alpha, uint64_t seed,
                   int32_t reject_cap, int32_t* coords, double* xs, int64_t* counts, double* phi,
                   void* stream);

/* Estimated fit of a model [[lambda; A_0..A_{D-1}]] on a sample from cpa_fit_sample:
 * F_hat = sum_j phi_j (m_j - x_j)^2, m_j = sum_c lambda_c prod_m A_m(i_m, c), and
 * *fit = 1 - sqrt(F_hat) / ||X||.
 *   coords, xs  device, as cpa_fit_sample wrote them (row stride `stride`)
 *   counts, phi host, as cpa_fit_sample returned them
 *   lambda      device, r doubles; factors: host array of order device pointers to
 *               n_m x r row-major doubles
 *   precision   CPA_FP64 (every product in FP64) or CPA_MIXED (the factors rounded
 *               to FP32 and each model value formed in FP32; residuals in FP64)
 *   fit, F_hat  host out (F_hat may be NULL)
 * Errors: CPA_ERR_ARG, CPA_ERR_OOM, CPA_ERR_CUDA. */
int cpa_fit_estimate(const cpa_index* index, const int32_t* coords, const double* xs, const int64_t* counts,
                     const double* phi, int64_t stride, const double* lambda, const double* const* factors,
                     int32_t r, int32_t precision, double* fit, double* F_hat, void* stream);

/* ---- stage entry points (each one step of the per-mode update) --------------- */

/* Philox4x64-10 block function (Salmon et al., SC'11) on the GPU: for each i < n,
 * out[4i..4i+3] = Philox(ctr[4i..4i+3], key[0..1]).  ctr/out: device, key: host. */
int cpa_philox4x64(const uint64_t* ctr, const uint64_t* key, int64_t n, uint64_t* out,
                   void* stream);

/* Leverage scores of a factor matrix (Definition 3.4): lev_i = a_i^T (A^T A)^+ a_i,
 * the squared row norms of any orthonormal basis of range(A).  A^T A is formed in
 * FP64 (from 65,536 rows on in float-pair arithmetic, about 2^-44 relative) and
 * factored by Cholesky; if that fails the pseudo-inverse from a Jacobi
 * eigendecomposition is used and CPA_WARN_RANK_DEFICIENT_LEV is returned.
 *   A (device) n x r row-major doubles; lev (device) n doubles; 1 <= r <= 64.
 * Errors: CPA_ERR_ARG, CPA_ERR_OOM, CPA_ERR_CUDA (also when a bulk copy of the
 * streaming Gram did not complete within its bounded wait). */
int cpa_leverage(const double* A, int64_t n, int32_t r, double* lev, void* stream);

/* The leverage scores of cpa_leverage, computed without allocating any memory.
 * This entry point has no counterpart in the paper.  It is for callers that may not
 * allocate device memory while running (for example a process that reserves the
 * GPU's memory for its own pool at start-up, or a latency-critical loop where
 * cudaMalloc/cudaFree would synchronise the device): they pass only A and lev.
 *   A (device) n x r row-major doubles; lev (device) n doubles out;
 *   1 <= r <= 64 (r > 64 returns CPA_ERR_UNSUPPORTED: the scratch holds r <= 64).
 * Its scratch (the r x r Gram with its per-block partial sums, its factorisation, a
 * warning word) is a 1 MiB device array in the library, present on every GPU that
 * loads the library until the process exits.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  All calls share the array: calls whose work overlaps on a
 * GPU race on it.  Same warnings and errors as cpa_leverage; the same scores up to
 * rounding (the Gram may be summed over fewer blocks; reproducible call to call). */
int cpa_leverage_noalloc(const double* A, int64_t n, int32_t r, double* lev, void* stream);

/* Fixed-point sampling distribution of one mode (Lemma 5.3 draws
 * i ~ Multinomial(l/r)): q_i = round-half-even(2^62 * (lev_i / r)) and the inclusive
 * prefix sums C_i = q_0 + ... + q_i (device, n words).  info (host, 3 words) gets
 * T = C_{n-1}, max q and the number of nonzero q.  Precondition: sum lev <= r
 * (1 + 2^-20), so that T < 2^63. */
int cpa_cdf(const double* lev, int64_t n, int32_t r, uint64_t* C, uint64_t* info,
            void* stream);

/* SkrpLev (Alg. 1): hybrid deterministic + random Khatri-Rao row sample over the d
 * other modes of an update of mode `mode_k`.
 *   d, dims     number of other modes (1..7) and their sizes (host)
 *   lev         host array of d device pointers, leverage scores of each other mode
 *   r           rank (the leverage scores are divided by r)
 *   opt         samples, tau, seed, det_cap, reject_cap and stream are used
 *   mode_k, iter  select the Philox counters (iter is the global outer iteration)
 *   idx, cnt, wgt  device outputs of opt->samples entries: linear keys (Eq. 2.2),
 *               repeat counts c_j and weights; rows 0..s_det-1 are the deterministic
 *               rows (ascending keys, weight 1, count 1), then the combined random rows
 *               (ascending keys, weight sqrt(c (1 - p_det) / (p_i s_rnd)), Eq. 4.4)
 *   counts      host out: {sbar, s_det, attempts}
 *   pdet        host out: p_det, the correctly rounded sum of p_i over the
 *               deterministic rows
 * Sampling details: p_m(i) = q_i / T_m from cpa_cdf; p_i is the product of the
 * p_m(i_t) in ascending mode order; a row is deterministic iff p_i > tau; slot j of
 * the random block draws with Philox counter (j, attempt, mode_k | 1<<32 |
 * (t/4)<<16, iter) and key (seed, 0), word t%4 for other mode t, the index being
 * min{i : C_i > floor(u T / 2^64)}; a draw is accepted iff p_i <= tau.
 * Errors: CPA_ERR_DET_CAP, CPA_ERR_REJECT_LIMIT, CPA_ERR_ARG. */
int cpa_skrp_lev(int32_t d, const int64_t* dims, const double* const* lev, int32_t r,
                 const cpa_options* opt, int32_t mode_k, uint64_t iter, uint64_t* idx,
                 uint32_t* cnt, double* wgt, int64_t* counts, double* pdet);

/* KrpSamp + TnsrSamp + the sampled normal equations (Section 5.2, Section 5.3):
 * with z_j = prod_t A_{m_t}(i_t(j), :) (Eq. 2.1),
 *   M = sum_j wgt_j^2 x(:, idx_j) z_j^T   (n_k x r, the sampled MTTKRP)
 *   G = sum_j wgt_j^2 z_j z_j^T           (r x r; rows with empty fibres count too)
 *   factors   host array of `order` device pointers (factors[mode_k] unused)
 *   idx, wgt  device, sbar linear keys and weights (as from cpa_skrp_lev)
 *   M, G      device outputs (doubles, row-major)
 *   nnz_sampled  host out (may be NULL): nonzeros of the sampled right-hand side */
int cpa_sampled_mttkrp(const cpa_index* index, int32_t mode_k, const double* const* factors,
                       int32_t r, const uint64_t* idx, const double* wgt, int64_t sbar,
                       double* M, double* G, int64_t* nnz_sampled, void* stream);

/* Solve of the sampled normal equations, A G = M (Alg. 3, argmin step), by FP64
 * Cholesky of G (pseudo-inverse from a Jacobi eigendecomposition if a pivot is not
 * above 1e-13 of the largest diagonal entry, returning CPA_WARN_SINGULAR_GRAM), then
 * column normalisation: lambda_c = ||A(:, c)||, A(:, c) /= lambda_c (zero columns
 * stay zero).  G, M, A, lambda: device; A may not alias M. */
int cpa_solve(const double* G, const double* M, int64_t n, int32_t r, double* A,
              double* lambda, void* stream);

/* Fit of Eq. 5.1: 1 - sqrt(max(0, ||X||^2 - 2 <X, M> + ||M||^2)) / ||X|| for the
 * model M = [[lambda; A_1, ..., A_D]].  factors: host array of device pointers;
 * lambda: device; fit: host out. */
int cpa_fit(const cpa_index* index, const double* const* factors, const double* lambda,
            int32_t r, double* fit, void* stream);

/* The three terms of the fit of Eq. 5.1 for the nonzeros of `index`:
 * terms[0] = ||X||^2, terms[1] = <X, M>, terms[2] = ||M||^2 (host out, FP64), with
 * M = [[lambda; A_1, ..., A_D]] (factors: host array of device pointers; lambda:
 * device).  The first two are sums over the nonzeros, so the terms of tensors that
 * hold disjoint parts of one tensor's nonzeros (the shards of a sharded run) add up
 * to the whole tensor's; the third depends on the factors only.  Errors as cpa_fit. */
int cpa_fit_terms(const cpa_index* index, const double* const* factors, const double* lambda,
                  int32_t r, double* terms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CPA_H */
