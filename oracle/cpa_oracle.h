/*
 * Plain FP64 CPU oracle for the CP-ARLS-LEV sampled least-squares step
 * (Larsen & Kolda, "Practical Leverage-Based Sampling for Low-Rank Tensor
 * Decomposition").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code; it
 * exists so that tests, the smoke check and the CPU-baseline leg of the benchmark
 * can check the CUDA path against an independent, slow, obviously-correct
 * implementation.  It shares no code, header, table or constant with the CUDA
 * library.
 *
 * Conventions: indices are 0-based (the paper is 1-based); factor matrices are
 * row-major n x r float64; the "other" modes of an update of mode k are taken in
 * ascending order m_0 < m_1 < ... < m_{d-1}; a multi-index (i_0..i_{d-1}) over them
 * has linear index  key = sum_t i_t * prod_{u<t} n_{m_u}  (Eq. 2.2, first mode
 * fastest).
 *
 * Return codes: 0 ok, negative errors, positive warning bits (listed below).
 */
#ifndef CPA_ORACLE_H
#define CPA_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_COO_RANGE (-2)
#define ORC_ERR_COO_DUP (-3)
#define ORC_ERR_OOM (-4)
#define ORC_ERR_REJECT_LIMIT (-5)
#define ORC_ERR_DET_CAP (-6)
#define ORC_WARN_SINGULAR_GRAM 1
#define ORC_WARN_RANK_DEFICIENT_LEV 2
/* per-factor row distributions (leverage: the method; uniform and length-squared:
 * the comparison of App. B) */
#define ORC_DIST_LEVERAGE 0
#define ORC_DIST_UNIFORM 1
#define ORC_DIST_LENGTH_SQUARED 2

/* Philox4x64-10 block function. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Leverage scores l_i = ||Q(i,:)||^2 of A (n x r) by column-pivoted Householder QR
 * (Definition 3.4); rank from |R_jj| > 1e-12 |R_00|.  Returns rank via *rank. */
int orc_leverage(const double* A, int64_t n, int r, double* lev, int* rank);

/* Fixed-point sampling distribution of one mode: q_i = rint(2^62 * (l_i / r)),
 * C = inclusive prefix sum of q.  Returns T = C[n-1]; *maxq = max q, *nnzq = #q>0. */
uint64_t orc_cdf(const double* lev, int64_t n, int r, uint64_t* q, uint64_t* C,
                 uint64_t* maxq, int64_t* nnzq);

/* One multinomial draw by inverse CDF: i = min{ i : C_i > floor(u*T/2^64) }. */
int64_t orc_draw(const uint64_t* C, int64_t n, uint64_t T, uint64_t u);

/* Correctly rounded sum of doubles (exact accumulation, one rounding). */
double orc_exact_sum(const double* x, int64_t n);

/* Parameters of one sampling problem: the d other modes of an update. */
typedef struct {
  int d;                      /* number of other modes */
  const int64_t* n;           /* n[t]: size of other mode t */
  const uint64_t* const* C;   /* C[t]: inclusive fixed-point CDF, n[t] entries */
  const uint64_t* T;          /* T[t] = C[t][n[t]-1] */
  const uint64_t* maxq;       /* maxq[t] */
  const int64_t* nnzq;        /* nnzq[t] */
} orc_sampler;

/* DetSkrp (Section 5.3, Alg. 1): every multi-index with p_i > tau, ascending key.
 * idet/pvals need room for min(cap, s) entries... callers pass cap-sized buffers.
 * If more than s pass the test, the s most probable (ties: smaller key) are kept. */
int orc_det_skrp(const orc_sampler* S, double tau, int64_t s, int64_t cap,
                 uint64_t* idet, double* pvals, int64_t* sdet, double* pdet);

/* RndSkrp (Alg. 2) with one Philox counter per (slot, attempt). */
int orc_rnd_skrp(const orc_sampler* S, int64_t srnd, double tau, double pdet,
                 uint64_t seed, uint64_t iter, int mode_k, int reject_cap,
                 uint64_t* irnd, double* wrnd, int64_t* attempts);

/* SkrpLev (Alg. 1): det block (weight 1, count 1), then combined random block.
 * idx/cnt/wgt need s entries (det_cap for the det scratch is internal). */
int orc_skrp_lev(const orc_sampler* S, int64_t s, double tau, uint64_t seed, uint64_t iter,
                 int mode_k, int64_t det_cap, int reject_cap,
                 uint64_t* idx, uint32_t* cnt, double* wgt, int64_t* sbar,
                 int64_t* sdet, double* pdet, int64_t* attempts);

/* Per-mode fibre index (Section 5.3): nonzeros sorted by (key_k, i_k). */
typedef struct {
  int order;
  int64_t dims[16];
  int64_t nnz;
  int64_t nfib[16];      /* F_k */
  uint64_t* keys[16];    /* F_k sorted fibre keys */
  int64_t* off[16];      /* F_k + 1 offsets into ik/val */
  int32_t* ik[16];       /* nnz, mode-k index of each nonzero in sorted order */
  double* val[16];       /* nnz */
  int64_t* perm[16];     /* nnz, original position of each sorted nonzero */
  const int32_t* coo_idx[16];
  const double* coo_val;
} orc_index;

int orc_index_build(int order, const int64_t* dims, int64_t nnz, const int32_t* const* idx,
                    const double* vals, orc_index** out);
void orc_index_free(orc_index* X);
int64_t orc_index_nfib(const orc_index* X, int k);
void orc_index_export(const orc_index* X, int k, uint64_t* keys, int64_t* off, int32_t* ik,
                      double* val);

/* KrpSamp + TnsrSamp + sampled products: M = Xs^T diag(w^2) Zs (n_k x r) and
 * G = Zs^T diag(w^2) Zs (r x r).  factors[k] is ignored. *nnz_sampled = nnz(Xs). */
int orc_sampled_mttkrp(const orc_index* X, int k, const double* const* factors, int r,
                       const uint64_t* idx, const double* wgt, int64_t sbar,
                       double* M, double* G, int64_t* nnz_sampled);

/* Exact MTTKRP (CP-ALS): M = X_(k) Z, G = Hadamard product of A_m^T A_m. */
int orc_exact_mttkrp(const orc_index* X, int k, const double* const* factors, int r,
                     double* M, double* G);

/* Solve A G = M for A (n x r) by Cholesky (pinv by Jacobi eigen on failure). */
int orc_solve(const double* G, const double* M, int64_t n, int r, double* A);

/* Column norms -> lambda, columns scaled to unit norm (zero columns stay zero). */
void orc_normalize(double* A, int64_t n, int r, double* lambda);

/* fit = 1 - sqrt(max(0, ||X||^2 - 2<X,M> + ||M||^2)) / ||X|| (Eq. 5.1). */
double orc_fit(const orc_index* X, const double* const* factors, const double* lambda, int r);

/* One randomized mode update: sample, solve, normalise, refresh leverage of mode k.
 * lev[m] (n_m) and the fixed-point CDF state of every mode are kept by the caller
 * in an orc_state. */
typedef struct {
  int order, r;
  int dist;               /* ORC_DIST_* */
  int64_t dims[16];
  double* lev[16];
  uint64_t* q[16];
  uint64_t* C[16];
  uint64_t T[16], maxq[16];
  int64_t nnzq[16];
  int warnings;
  /* statistics of the most recent update */
  int64_t sdet, sbar, nnz_sampled, attempts;
  double pdet;
} orc_state;

int orc_state_init(orc_state* st, int order, const int64_t* dims, int r,
                   double* const* factors, int dist);

/* Row scores of a factor summing to r (p_i = score_i / r): leverage scores
 * (orc_leverage), r / n (uniform) or r ||a_i||^2 / ||A||_F^2 (length-squared). */
int orc_scores(const double* A, int64_t n, int r, int dist, double* s, int* rank);
void orc_state_free(orc_state* st);
int orc_mode_update(const orc_index* X, orc_state* st, int k, double* const* factors,
                    double* lambda, int64_t s, double tau, uint64_t seed, uint64_t iter,
                    int64_t det_cap, int reject_cap,
                    uint64_t* idx_out, uint32_t* cnt_out, double* wgt_out);

/* Alg. 3 with a fixed number of outer iterations (tol = 0) or the epoch/patience
 * stopping rule (tol > 0).  factors: in = init, out = result. */
int orc_cp_arls_lev(const orc_index* X, int r, int64_t s, double tau, int iters, int epoch_len,
                    int patience, double tol, uint64_t seed, uint64_t iter_offset,
                    int64_t det_cap, int reject_cap, double* const* factors, double* lambda,
                    double* fit, int* iters_done, int dist);

/* One mode update from the given factors (leverage of all modes recomputed first).
 * stats = {sbar, sdet, nnz_sampled, attempts}. */
int orc_mode_update_once(const orc_index* X, int r, int k, double* const* factors,
                         double* lambda, int64_t s, double tau, uint64_t seed, uint64_t iter,
                         int64_t det_cap, int reject_cap, uint64_t* idx, uint32_t* cnt,
                         double* wgt, int64_t* stats, double* pdet, int dist);

/* Estimated fit (Section 5.4).  orc_fit_sample draws the stratified sample once:
 * s_nz = ceil(alpha * s_fit) nonzeros and s_z = s_fit - s_nz zero elements (the
 * paper's floor((1 - alpha) s_fit) in exact arithmetic), each uniform over its
 * stratum, with replacement; s_z = 0 when the tensor has no zero element.
 *   nonzero slot j: u = word 0 of Philox(ctr = (j, 0, 2<<32, 0), key = (seed, 0));
 *     the element is the nonzero at position floor(u nnz / 2^64) in ascending order
 *     of the linear index of Eq. 2.2 over all modes (mode 0 fastest);
 *   zero slot j, attempt a: i_m = floor(u_m n_m / 2^64), u_m = word m%4 of
 *     Philox(ctr = (j, a, 2<<32 | 1 | (m/4)<<16, 0), key = (seed, 0)); the attempt is
 *     rejected if (i_0..i_{D-1}) is a nonzero; more than reject_cap attempts is
 *     ORC_ERR_REJECT_LIMIT.
 * Outputs: coords (order x s_fit int32, row m at coords + m*s_fit), xs (s_fit values,
 * 0 for zero samples; nonzero samples first), counts = {s_nz, s_z, zero attempts},
 * phi = {nnz / s_nz, (prod n - nnz) / s_z} (0 for an empty stratum).
 * 0 < alpha <= 1, s_fit >= 1 and nnz >= 1, else ORC_ERR_ARG. */
int orc_fit_sample(const orc_index* X, int64_t s_fit, double alpha, uint64_t seed, int reject_cap,
                   int32_t* coords, double* xs, int64_t* counts, double* phi);

/* F_hat = sum_j phi_j (m_j - x_j)^2 over the sample (m_j the model's entry,
 * sum_c lambda_c prod_m A_m(i_m, c)); returns 1 - sqrt(F_hat) / ||X||.  *F_hat_out
 * (may be NULL) receives F_hat. */
double orc_fit_estimate(const orc_index* X, const int32_t* coords, const double* xs,
                        const int64_t* counts, const double* phi, int64_t stride,
                        const double* const* factors, const double* lambda, int r, double* F_hat_out);

/* Randomized range finder initialisation of factor k (App. F):
 * A = X_(k)(:, S) * Omega, S = s_init fibres drawn uniformly with replacement from the
 * F_k nonzero mode-k fibres: draw j takes the fibre at position
 * floor(u F_k / 2^64) in ascending order of the fibre's linear key (Eq. 2.2),
 * u = word 0 of Philox(counter (j, 0, 3<<32 | k, 0), key (seed, 0)).  omega: s_init x r
 * (the Gaussian draws, supplied by the caller), A: n_k x r out. */
int orc_rrf_init(const orc_index* X, int k, int64_t s_init, uint64_t seed, const double* omega, int r,
                 double* A);

/* Standard CP-ALS (exact MTTKRP) with a fixed iteration count. */
int orc_cp_als(const orc_index* X, int r, int iters, double* const* factors, double* lambda,
               double* fit);

#endif
