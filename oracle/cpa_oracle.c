/*
 * Plain FP64 CPU oracle for the CP-ARLS-LEV sampled least-squares step.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's
 * CPU-baseline leg.  It is written for a reader checking it against the paper, not
 * for speed: plain loops, FP64, one thread, no blocking or fusion.  It shares no code
 * with the CUDA library.  Each function names the passage of the paper it follows.
 *
 * Readings of points the paper leaves open (all also listed in the design notes):
 *  - random draws: Philox4x64-10, counter (slot, attempt, mode | 1<<32, iteration),
 *    key (seed, 0); the multinomial of Lemma 5.3 is drawn per mode by inverse CDF on
 *    a fixed-point CDF q_i = rint(2^62 l_i / r), so both implementations agree bit
 *    for bit; the sampling probability of row i of mode m is p_m(i) = q_i / T_m;
 *  - p_i of a multi-index is the product of its p_m in ascending mode order;
 *  - deterministic set: p_i > tau (strict); a random draw is accepted iff p_i <= tau;
 *  - random weight uses s_rnd = s - s_det (Alg. 2), combined weight
 *    sqrt(c (1 - p_det) / (p_i s_rnd)) (Eq. 4.4 with s_rnd);
 *  - p_det is the correctly rounded sum over the deterministic set;
 *  - if the deterministic set holds every row of nonzero probability, no random
 *    samples are drawn;
 *  - the solve uses the normal equations with Cholesky (pinv on failure);
 *  - after each solve the columns are normalised and lambda keeps the norms.
 */
#include "cpa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Each round multiplies words 0 and 2 by fixed   */
/* odd constants, mixes the 128-bit products with words 1 and 3 and the      */
/* round key, and permutes; the key is bumped by two Weyl increments.        */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL
#define PHILOX_W1 0xBB67AE8584CAA73BULL

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
    unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Leverage scores (Definition 3.4): l_i = ||Q(i,:)||^2 for an orthonormal   */
/* basis Q of range(A).  Q from column-pivoted Householder QR (Businger and  */
/* Golub), truncated at the numerical rank.                                  */
/* ------------------------------------------------------------------------ */
int orc_leverage(const double* A, int64_t n, int r, double* lev, int* rank_out) {
  if (n <= 0 || r <= 0) return ORC_ERR_ARG;
  int kmax = (int)(n < r ? n : r);
  double* W = (double*)malloc(sizeof(double) * (size_t)n * r);  /* column-major copy */
  double* beta = (double*)calloc((size_t)kmax, sizeof(double));
  if (!W || !beta) { free(W); free(beta); return ORC_ERR_OOM; }
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < r; ++c) W[(size_t)c * n + i] = A[(size_t)i * r + c];
  double r00 = 0.0;
  int rank = 0;
  for (int k = 0; k < kmax; ++k) {
    /* pivot: column with the largest remaining norm */
    int piv = k;
    double best = -1.0;
    for (int c = k; c < r; ++c) {
      double s2 = 0.0;
      for (int64_t i = k; i < n; ++i) s2 += W[(size_t)c * n + i] * W[(size_t)c * n + i];
      if (s2 > best) { best = s2; piv = c; }
    }
    if (piv != k)
      for (int64_t i = 0; i < n; ++i) {
        double t = W[(size_t)k * n + i];
        W[(size_t)k * n + i] = W[(size_t)piv * n + i];
        W[(size_t)piv * n + i] = t;
      }
    double* x = W + (size_t)k * n;
    double normx = sqrt(best > 0 ? best : 0.0);
    if (k == 0) r00 = normx;
    if (!(normx > 1e-12 * r00) || normx == 0.0) break;
    rank = k + 1;
    /* Householder vector v = x + sign(x_k) ||x|| e_k, stored in place of x[k:] */
    double alpha = x[k] >= 0 ? -normx : normx;
    double v0 = x[k] - alpha;
    x[k] = v0;
    double vnorm2 = v0 * v0;
    for (int64_t i = k + 1; i < n; ++i) vnorm2 += x[i] * x[i];
    beta[k] = vnorm2 > 0 ? 2.0 / vnorm2 : 0.0;
    for (int c = k + 1; c < r; ++c) {
      double* y = W + (size_t)c * n;
      double dot = 0.0;
      for (int64_t i = k; i < n; ++i) dot += x[i] * y[i];
      dot *= beta[k];
      for (int64_t i = k; i < n; ++i) y[i] -= dot * x[i];
    }
  }
  /* Q(:, 0:rank) = H_0 H_1 ... H_{rank-1} [I; 0]; apply reflectors in reverse */
  double* Q = (double*)calloc((size_t)n * (rank > 0 ? rank : 1), sizeof(double));
  if (!Q) { free(W); free(beta); return ORC_ERR_OOM; }
  for (int c = 0; c < rank; ++c) Q[(size_t)c * n + c] = 1.0;
  for (int k = rank - 1; k >= 0; --k) {
    const double* v = W + (size_t)k * n;
    for (int c = 0; c < rank; ++c) {
      double* y = Q + (size_t)c * n;
      double dot = 0.0;
      for (int64_t i = k; i < n; ++i) dot += v[i] * y[i];
      dot *= beta[k];
      for (int64_t i = k; i < n; ++i) y[i] -= dot * v[i];
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    double s2 = 0.0;
    for (int c = 0; c < rank; ++c) s2 += Q[(size_t)c * n + i] * Q[(size_t)c * n + i];
    lev[i] = s2;
  }
  if (rank_out) *rank_out = rank;
  free(Q); free(W); free(beta);
  return rank < r ? ORC_WARN_RANK_DEFICIENT_LEV : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Fixed-point CDF of p = l / r (Lemma 5.3 draws i_k ~ Multinomial(l(A_k)/r)) */
/* ------------------------------------------------------------------------ */
uint64_t orc_cdf(const double* lev, int64_t n, int r, uint64_t* q, uint64_t* C,
                 uint64_t* maxq, int64_t* nnzq) {
  const double two62 = 4611686018427387904.0; /* 2^62 */
  uint64_t run = 0, mx = 0;
  int64_t nz = 0;
  for (int64_t i = 0; i < n; ++i) {
    double p = lev[i] / (double)r;
    if (!(p > 0.0)) p = 0.0;
    if (p > 1.0) p = 1.0;
    uint64_t qi = (uint64_t)rint(p * two62); /* round half to even */
    if (q) q[i] = qi;
    run += qi;
    C[i] = run;
    if (qi > mx) mx = qi;
    if (qi > 0) ++nz;
  }
  if (maxq) *maxq = mx;
  if (nnzq) *nnzq = nz;
  return run;
}

int64_t orc_draw(const uint64_t* C, int64_t n, uint64_t T, uint64_t u) {
  uint64_t t = (uint64_t)(((unsigned __int128)u * T) >> 64); /* t in [0, T) */
  int64_t lo = 0, hi = n - 1;                               /* C[n-1] = T > t */
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (C[mid] > t) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/* ------------------------------------------------------------------------ */
/* Exact sum of nonnegative doubles: every term is added into one long        */
/* fixed-point integer whose unit is 2^-1074 (the smallest subnormal), then   */
/* the integer is rounded once to the nearest double (ties to even).          */
/* ------------------------------------------------------------------------ */
#define XS_LIMBS 72 /* 72 x 32 bits > 1074 + 1024 + 64 */
double orc_exact_sum(const double* x, int64_t n) {
  uint64_t acc[XS_LIMBS];
  memset(acc, 0, sizeof(acc));
  for (int64_t i = 0; i < n; ++i) {
    double v = x[i];
    if (v == 0.0) continue;
    int ex;
    double f = frexp(v, &ex);                 /* v = f 2^ex, f in [0.5, 1) */
    uint64_t mant = (uint64_t)ldexp(f, 53);   /* exact: v = mant 2^(ex-53) */
    int shift = ex - 53 + 1074;               /* v = mant 2^(shift-1074) */
    while (shift < 0) { mant >>= 1; ++shift; } /* only zero bits drop (subnormals) */
    int limb = shift / 32, off = shift % 32;
    unsigned __int128 w = (unsigned __int128)mant << off;
    acc[limb] += (uint32_t)w;
    acc[limb + 1] += (uint32_t)(w >> 32);
    acc[limb + 2] += (uint32_t)(w >> 64);
  }
  for (int l = 0; l + 1 < XS_LIMBS; ++l) {
    acc[l + 1] += acc[l] >> 32;
    acc[l] &= 0xffffffffULL;
  }
  int top = -1;
  for (int l = XS_LIMBS - 1; l >= 0 && top < 0; --l)
    if (acc[l]) for (int b = 31; b >= 0; --b) if ((acc[l] >> b) & 1) { top = l * 32 + b; break; }
  if (top < 0) return 0.0;
#define XS_BIT(pos) ((pos) < 0 ? 0u : (unsigned)((acc[(pos) / 32] >> ((pos) % 32)) & 1))
  if (top < 53) { /* fits in 53 bits: exact */
    uint64_t m = 0;
    for (int b = top; b >= 0; --b) m = (m << 1) | XS_BIT(b);
    return ldexp((double)m, -1074);
  }
  uint64_t m = 0;
  for (int b = top; b > top - 53; --b) m = (m << 1) | XS_BIT(b);
  unsigned rbit = XS_BIT(top - 53);
  unsigned sticky = 0;
  for (int b = top - 54; b >= 0 && !sticky; --b) sticky |= XS_BIT(b);
  if (rbit && (sticky || (m & 1))) ++m;
  int e = top - 52 - 1074;
  if (m == (1ULL << 53)) { m >>= 1; ++e; }
#undef XS_BIT
  return ldexp((double)m, e);
}

/* ------------------------------------------------------------------------ */
/* Multi-index <-> linear index (Eq. 2.2, 0-based, first mode fastest)       */
/* ------------------------------------------------------------------------ */
static void key_decode(uint64_t key, int d, const int64_t* n, int64_t* it) {
  for (int t = 0; t < d; ++t) {
    it[t] = (int64_t)(key % (uint64_t)n[t]);
    key /= (uint64_t)n[t];
  }
}

static uint64_t key_encode(int d, const int64_t* n, const int64_t* it) {
  uint64_t key = 0, stride = 1;
  for (int t = 0; t < d; ++t) {
    key += (uint64_t)it[t] * stride;
    stride *= (uint64_t)n[t];
  }
  return key;
}

/* p_m(i) = q_i / T_m recovered from the inclusive CDF */
static double mode_prob(const orc_sampler* S, int t, int64_t i) {
  uint64_t qi = S->C[t][i] - (i > 0 ? S->C[t][i - 1] : 0);
  return (double)qi / (double)S->T[t];
}

/* p_i = prod_t p_{m_t}(i_t), multiplied in ascending mode order (Section 5.3) */
static double multi_prob(const orc_sampler* S, const int64_t* it) {
  double p = mode_prob(S, 0, it[0]);
  for (int t = 1; t < S->d; ++t) p = p * mode_prob(S, t, it[t]);
  return p;
}

/* ------------------------------------------------------------------------ */
/* DetSkrp (Section 5.3 and Alg. 1): D = { i : p_i > tau }.                  */
/* alpha_m = max p_m, alpha_* = prod alpha_m; only rows with                  */
/* p_m(i) > tau alpha_m / alpha_* can take part, so the candidates are the    */
/* product of those per-mode sets (kept with a relative slack of 2^-40 so      */
/* that rounding never drops a member); each candidate is tested exactly.     */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; double p; } kp_t;

static int cmp_key_asc(const void* a, const void* b) {
  uint64_t x = ((const kp_t*)a)->key, y = ((const kp_t*)b)->key;
  return x < y ? -1 : x > y;
}
static int cmp_p_desc_key_asc(const void* a, const void* b) {
  const kp_t* x = (const kp_t*)a;
  const kp_t* y = (const kp_t*)b;
  if (x->p > y->p) return -1;
  if (x->p < y->p) return 1;
  return x->key < y->key ? -1 : x->key > y->key;
}

int orc_det_skrp(const orc_sampler* S, double tau, int64_t s, int64_t cap,
                 uint64_t* idet, double* pvals, int64_t* sdet, double* pdet) {
  int d = S->d;
  *sdet = 0;
  *pdet = 0.0;
  double alpha[16], astar = 1.0;
  for (int t = 0; t < d; ++t) {
    alpha[t] = (double)S->maxq[t] / (double)S->T[t];
    astar = (t == 0) ? alpha[t] : astar * alpha[t];
  }
  if (!(astar > tau)) return ORC_OK; /* every p_i <= alpha_* <= tau */
  int64_t* cand[16];
  int64_t ncand[16];
  double total = 1.0;
  for (int t = 0; t < d; ++t) {
    double thr = (tau * alpha[t] / astar) * (1.0 - 0x1p-40);
    cand[t] = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S->n[t] > 0 ? S->n[t] : 1));
    ncand[t] = 0;
    for (int64_t i = 0; i < S->n[t]; ++i)
      if (mode_prob(S, t, i) >= thr) cand[t][ncand[t]++] = i;
    total *= (double)ncand[t];
  }
  if (total > (double)cap) {
    for (int t = 0; t < d; ++t) free(cand[t]);
    return ORC_ERR_DET_CAP;
  }
  int64_t ntot = (int64_t)total;
  kp_t* found = (kp_t*)malloc(sizeof(kp_t) * (size_t)(ntot > 0 ? ntot : 1));
  int64_t nf = 0;
  int64_t pos[16], it[16];
  for (int t = 0; t < d; ++t) pos[t] = 0;
  for (int64_t e = 0; e < ntot; ++e) {
    for (int t = 0; t < d; ++t) it[t] = cand[t][pos[t]];
    double p = multi_prob(S, it);
    if (p > tau) { found[nf].key = key_encode(d, S->n, it); found[nf].p = p; ++nf; }
    for (int t = 0; t < d; ++t) { /* odometer, first mode fastest */
      if (++pos[t] < ncand[t]) break;
      pos[t] = 0;
    }
  }
  if (nf > s) { /* more than s rows pass: keep the s most probable (Alg. 1 notes) */
    qsort(found, (size_t)nf, sizeof(kp_t), cmp_p_desc_key_asc);
    nf = s;
  }
  qsort(found, (size_t)nf, sizeof(kp_t), cmp_key_asc);
  double* pv = (double*)malloc(sizeof(double) * (size_t)(nf > 0 ? nf : 1));
  for (int64_t j = 0; j < nf; ++j) {
    idet[j] = found[j].key;
    if (pvals) pvals[j] = found[j].p;
    pv[j] = found[j].p;
  }
  *sdet = nf;
  *pdet = orc_exact_sum(pv, nf);
  free(pv);
  free(found);
  for (int t = 0; t < d; ++t) free(cand[t]);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* RndSkrp (Alg. 2).  Slot j keeps drawing (attempt a = 0, 1, ...) until the  */
/* draw has p_i <= tau (rejection of the deterministic set, Section 5.3).     */
/* ------------------------------------------------------------------------ */
static void draw_multi(const orc_sampler* S, uint64_t seed, uint64_t iter, int mode_k,
                       uint64_t j, uint64_t a, int64_t* it) {
  const uint64_t key[2] = {seed, 0};
  uint64_t out[4];
  for (int t = 0; t < S->d; ++t) {
    if (t % 4 == 0) {
      uint64_t ctr[4] = {j, a, (uint64_t)(uint32_t)mode_k | ((uint64_t)(t / 4) << 16) | (1ULL << 32),
                         iter};
      orc_philox4x64_10(ctr, key, out);
    }
    it[t] = orc_draw(S->C[t], S->n[t], S->T[t], out[t % 4]);
  }
}

int orc_rnd_skrp(const orc_sampler* S, int64_t srnd, double tau, double pdet,
                 uint64_t seed, uint64_t iter, int mode_k, int reject_cap,
                 uint64_t* irnd, double* wrnd, int64_t* attempts) {
  int64_t it[16];
  int64_t tries = 0;
  for (int64_t j = 0; j < srnd; ++j) {
    int accepted = 0;
    for (int a = 0; a < reject_cap; ++a) {
      draw_multi(S, seed, iter, mode_k, (uint64_t)j, (uint64_t)a, it);
      ++tries;
      double p = multi_prob(S, it);
      if (p <= tau) {
        irnd[j] = key_encode(S->d, S->n, it);
        if (wrnd) wrnd[j] = sqrt((1.0 - pdet) / (p * (double)srnd));
        accepted = 1;
        break;
      }
    }
    if (!accepted) {
      if (attempts) *attempts = tries;
      return ORC_ERR_REJECT_LIMIT;
    }
  }
  if (attempts) *attempts = tries;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SkrpLev (Alg. 1) with CombineRepeats (Section 4.1, Eq. 4.4)               */
/* ------------------------------------------------------------------------ */
static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : x > y;
}

int orc_skrp_lev(const orc_sampler* S, int64_t s, double tau, uint64_t seed, uint64_t iter,
                 int mode_k, int64_t det_cap, int reject_cap,
                 uint64_t* idx, uint32_t* cnt, double* wgt, int64_t* sbar,
                 int64_t* sdet_out, double* pdet_out, int64_t* attempts) {
  int64_t detbuf = det_cap < 1 ? 1 : det_cap;
  uint64_t* idet = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)detbuf);
  if (!idet) return ORC_ERR_OOM;
  int64_t sdet = 0;
  double pdet = 0.0;
  int rc = orc_det_skrp(S, tau, s, det_cap, idet, NULL, &sdet, &pdet);
  if (rc < 0) { free(idet); return rc; }
  int64_t srnd = s - sdet;
  /* every row with nonzero probability is already deterministic */
  double support = 1.0;
  for (int t = 0; t < S->d; ++t) support *= (double)S->nnzq[t];
  if ((double)sdet >= support) srnd = 0;
  uint64_t* irnd = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(srnd > 0 ? srnd : 1));
  int64_t tries = 0;
  rc = orc_rnd_skrp(S, srnd, tau, pdet, seed, iter, mode_k, reject_cap, irnd, NULL, &tries);
  if (attempts) *attempts = tries;
  if (rc < 0) { free(idet); free(irnd); return rc; }
  for (int64_t j = 0; j < sdet; ++j) { idx[j] = idet[j]; cnt[j] = 1; wgt[j] = 1.0; }
  qsort(irnd, (size_t)srnd, sizeof(uint64_t), cmp_u64);
  int64_t u = sdet, it[16];
  for (int64_t j = 0; j < srnd;) {
    int64_t e = j;
    while (e < srnd && irnd[e] == irnd[j]) ++e;
    uint64_t c = (uint64_t)(e - j);
    key_decode(irnd[j], S->d, S->n, it);
    double p = multi_prob(S, it);
    idx[u] = irnd[j];
    cnt[u] = (uint32_t)c;
    wgt[u] = sqrt(((double)c * (1.0 - pdet)) / (p * (double)srnd));
    ++u;
    j = e;
  }
  *sbar = u;
  if (sdet_out) *sdet_out = sdet;
  if (pdet_out) *pdet_out = pdet;
  free(idet);
  free(irnd);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Fibre index (Section 5.3): for mode k every nonzero gets the linear index  */
/* of its other-mode multi-index; nonzeros are sorted by (key, i_k) so each   */
/* fibre X(:, key) is one contiguous run.                                    */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; int32_t ik; int64_t e; } fib_t;

static int cmp_fib(const void* a, const void* b) {
  const fib_t* x = (const fib_t*)a;
  const fib_t* y = (const fib_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->ik != y->ik) return x->ik < y->ik ? -1 : 1;
  return x->e < y->e ? -1 : x->e > y->e;
}

int orc_index_build(int order, const int64_t* dims, int64_t nnz, const int32_t* const* idx,
                    const double* vals, orc_index** out) {
  if (order < 2 || order > 16 || nnz < 0) return ORC_ERR_ARG;
  for (int m = 0; m < order; ++m) if (dims[m] <= 0) return ORC_ERR_ARG;
  for (int m = 0; m < order; ++m)
    for (int64_t e = 0; e < nnz; ++e)
      if (idx[m][e] < 0 || idx[m][e] >= dims[m]) return ORC_ERR_COO_RANGE;
  orc_index* X = (orc_index*)calloc(1, sizeof(orc_index));
  X->order = order;
  X->nnz = nnz;
  for (int m = 0; m < order; ++m) { X->dims[m] = dims[m]; X->coo_idx[m] = idx[m]; }
  X->coo_val = vals;
  fib_t* tmp = (fib_t*)malloc(sizeof(fib_t) * (size_t)(nnz > 0 ? nnz : 1));
  for (int k = 0; k < order; ++k) {
    int64_t n_o[16];
    int d = 0;
    for (int m = 0; m < order; ++m) if (m != k) n_o[d++] = dims[m];
    for (int64_t e = 0; e < nnz; ++e) {
      int64_t it[16];
      int t = 0;
      for (int m = 0; m < order; ++m) if (m != k) it[t++] = idx[m][e];
      tmp[e].key = key_encode(d, n_o, it);
      tmp[e].ik = idx[k][e];
      tmp[e].e = e;
    }
    qsort(tmp, (size_t)nnz, sizeof(fib_t), cmp_fib);
    for (int64_t e = 1; e < nnz; ++e)
      if (tmp[e].key == tmp[e - 1].key && tmp[e].ik == tmp[e - 1].ik) {
        free(tmp);
        orc_index_free(X);
        return ORC_ERR_COO_DUP;
      }
    int64_t F = 0;
    for (int64_t e = 0; e < nnz; ++e) if (e == 0 || tmp[e].key != tmp[e - 1].key) ++F;
    X->nfib[k] = F;
    X->keys[k] = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(F > 0 ? F : 1));
    X->off[k] = (int64_t*)malloc(sizeof(int64_t) * (size_t)(F + 1));
    X->ik[k] = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    X->val[k] = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    X->perm[k] = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t f = 0;
    for (int64_t e = 0; e < nnz; ++e) {
      if (e == 0 || tmp[e].key != tmp[e - 1].key) {
        X->keys[k][f] = tmp[e].key;
        X->off[k][f] = e;
        ++f;
      }
      X->ik[k][e] = tmp[e].ik;
      X->val[k][e] = vals[tmp[e].e];
      X->perm[k][e] = tmp[e].e;
    }
    X->off[k][F] = nnz;
  }
  free(tmp);
  *out = X;
  return ORC_OK;
}

void orc_index_free(orc_index* X) {
  if (!X) return;
  for (int k = 0; k < X->order; ++k) {
    free(X->keys[k]); free(X->off[k]); free(X->ik[k]); free(X->val[k]); free(X->perm[k]);
  }
  free(X);
}

int64_t orc_index_nfib(const orc_index* X, int k) { return X->nfib[k]; }

void orc_index_export(const orc_index* X, int k, uint64_t* keys, int64_t* off, int32_t* ik,
                      double* val) {
  int64_t F = X->nfib[k];
  if (keys) memcpy(keys, X->keys[k], sizeof(uint64_t) * (size_t)F);
  if (off) memcpy(off, X->off[k], sizeof(int64_t) * (size_t)(F + 1));
  if (ik) memcpy(ik, X->ik[k], sizeof(int32_t) * (size_t)X->nnz);
  if (val) memcpy(val, X->val[k], sizeof(double) * (size_t)X->nnz);
}

/* ------------------------------------------------------------------------ */
/* KrpSamp, TnsrSamp and the sampled normal equations (Section 5.2-5.3):     */
/* z_j = w_j * (A_{m_0}(i_0,:) * ... * A_{m_{d-1}}(i_{d-1},:)) (Eq. 2.1),     */
/* Xs(j, i) = w_j x(idx_j, i); M = Xs^T Zs, G = Zs^T Zs.                      */
/* ------------------------------------------------------------------------ */
static int64_t find_fibre(const orc_index* X, int k, uint64_t key) {
  int64_t lo = 0, hi = X->nfib[k];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (X->keys[k][mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < X->nfib[k] && X->keys[k][lo] == key) ? lo : -1;
}

int orc_sampled_mttkrp(const orc_index* X, int k, const double* const* factors, int r,
                       const uint64_t* idx, const double* wgt, int64_t sbar,
                       double* M, double* G, int64_t* nnz_sampled) {
  int order = X->order, d = order - 1;
  int64_t n_o[16];
  int mo[16];
  for (int m = 0, t = 0; m < order; ++m) if (m != k) { n_o[t] = X->dims[m]; mo[t] = m; ++t; }
  memset(M, 0, sizeof(double) * (size_t)X->dims[k] * r);
  memset(G, 0, sizeof(double) * (size_t)r * r);
  double* z = (double*)malloc(sizeof(double) * (size_t)r);
  int64_t it[16], nzs = 0;
  for (int64_t j = 0; j < sbar; ++j) {
    key_decode(idx[j], d, n_o, it);
    for (int c = 0; c < r; ++c) {
      double v = factors[mo[0]][(size_t)it[0] * r + c];
      for (int t = 1; t < d; ++t) v *= factors[mo[t]][(size_t)it[t] * r + c];
      z[c] = v;
    }
    double w2 = wgt[j] * wgt[j];
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) G[a * r + b] += w2 * z[a] * z[b];
    int64_t f = find_fibre(X, k, idx[j]);
    if (f < 0) continue; /* empty fibre: a zero row of Xs */
    for (int64_t e = X->off[k][f]; e < X->off[k][f + 1]; ++e) {
      double xv = w2 * X->val[k][e];
      double* Mi = M + (size_t)X->ik[k][e] * r;
      for (int c = 0; c < r; ++c) Mi[c] += xv * z[c];
      ++nzs;
    }
  }
  if (nnz_sampled) *nnz_sampled = nzs;
  free(z);
  return ORC_OK;
}

int orc_exact_mttkrp(const orc_index* X, int k, const double* const* factors, int r,
                     double* M, double* G) {
  int order = X->order;
  memset(M, 0, sizeof(double) * (size_t)X->dims[k] * r);
  for (int a = 0; a < r; ++a) for (int b = 0; b < r; ++b) G[a * r + b] = 1.0;
  for (int m = 0; m < order; ++m) {
    if (m == k) continue;
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) {
        double s2 = 0.0;
        for (int64_t i = 0; i < X->dims[m]; ++i)
          s2 += factors[m][(size_t)i * r + a] * factors[m][(size_t)i * r + b];
        G[a * r + b] *= s2;
      }
  }
  for (int64_t e = 0; e < X->nnz; ++e) {
    double* Mi = M + (size_t)X->coo_idx[k][e] * r;
    for (int c = 0; c < r; ++c) {
      double v = X->coo_val[e];
      for (int m = 0; m < order; ++m)
        if (m != k) v *= factors[m][(size_t)X->coo_idx[m][e] * r + c];
      Mi[c] += v;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Normal-equation solve of min ||Zs B^T - Xs^T|| (Alg. 3, solve step):       */
/* A G = M with G = L L^T; if a Cholesky pivot is not positive (relative to   */
/* the largest diagonal entry), fall back to the pseudo-inverse from a cyclic */
/* Jacobi eigendecomposition.                                                 */
/* ------------------------------------------------------------------------ */
static int cholesky(const double* G, int r, double* L) {
  double dmax = 0.0;
  for (int i = 0; i < r; ++i) if (G[i * r + i] > dmax) dmax = G[i * r + i];
  memset(L, 0, sizeof(double) * (size_t)r * r);
  for (int j = 0; j < r; ++j) {
    double s2 = G[j * r + j];
    for (int c = 0; c < j; ++c) s2 -= L[j * r + c] * L[j * r + c];
    if (!(s2 > 1e-13 * dmax)) return -1;
    double ljj = sqrt(s2);
    L[j * r + j] = ljj;
    for (int i = j + 1; i < r; ++i) {
      double t = G[i * r + j];
      for (int c = 0; c < j; ++c) t -= L[i * r + c] * L[j * r + c];
      L[i * r + j] = t / ljj;
    }
  }
  return 0;
}

static void jacobi_pinv(const double* G, int r, double* P) {
  double* a = (double*)malloc(sizeof(double) * (size_t)r * r);
  double* v = (double*)calloc((size_t)r * r, sizeof(double));
  memcpy(a, G, sizeof(double) * (size_t)r * r);
  for (int i = 0; i < r; ++i) v[i * r + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) {
        tot += a[i * r + j] * a[i * r + j];
        if (i != j) off += a[i * r + j] * a[i * r + j];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < r; ++p)
      for (int q = p + 1; q < r; ++q) {
        double apq = a[p * r + q];
        if (apq == 0.0) continue;
        double theta = (a[q * r + q] - a[p * r + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < r; ++k) { /* rotate columns p, q */
          double akp = a[k * r + p], akq = a[k * r + q];
          a[k * r + p] = c * akp - s * akq;
          a[k * r + q] = s * akp + c * akq;
        }
        for (int k = 0; k < r; ++k) { /* rotate rows p, q */
          double apk = a[p * r + k], aqk = a[q * r + k];
          a[p * r + k] = c * apk - s * aqk;
          a[q * r + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < r; ++k) {
          double vkp = v[k * r + p], vkq = v[k * r + q];
          v[k * r + p] = c * vkp - s * vkq;
          v[k * r + q] = s * vkp + c * vkq;
        }
      }
  }
  double emax = 0.0;
  for (int i = 0; i < r; ++i) if (fabs(a[i * r + i]) > emax) emax = fabs(a[i * r + i]);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) {
      double s2 = 0.0;
      for (int k = 0; k < r; ++k) {
        double ev = a[k * r + k];
        if (ev > 1e-13 * emax) s2 += v[i * r + k] * v[j * r + k] / ev;
      }
      P[i * r + j] = s2;
    }
  free(a);
  free(v);
}

int orc_solve(const double* G, const double* M, int64_t n, int r, double* A) {
  double* L = (double*)malloc(sizeof(double) * (size_t)r * r);
  double* y = (double*)malloc(sizeof(double) * (size_t)r);
  int rc = ORC_OK;
  if (cholesky(G, r, L) == 0) {
    for (int64_t i = 0; i < n; ++i) {
      const double* m = M + (size_t)i * r;
      for (int a = 0; a < r; ++a) { /* L y = m */
        double t = m[a];
        for (int c = 0; c < a; ++c) t -= L[a * r + c] * y[c];
        y[a] = t / L[a * r + a];
      }
      double* x = A + (size_t)i * r;
      for (int a = r - 1; a >= 0; --a) { /* L^T x = y */
        double t = y[a];
        for (int c = a + 1; c < r; ++c) t -= L[c * r + a] * x[c];
        x[a] = t / L[a * r + a];
      }
    }
  } else {
    double* P = (double*)malloc(sizeof(double) * (size_t)r * r);
    jacobi_pinv(G, r, P);
    for (int64_t i = 0; i < n; ++i)
      for (int b = 0; b < r; ++b) {
        double t = 0.0;
        for (int a = 0; a < r; ++a) t += M[(size_t)i * r + a] * P[a * r + b];
        A[(size_t)i * r + b] = t;
      }
    free(P);
    rc = ORC_WARN_SINGULAR_GRAM;
  }
  free(L);
  free(y);
  return rc;
}

void orc_normalize(double* A, int64_t n, int r, double* lambda) {
  for (int c = 0; c < r; ++c) {
    double s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) s2 += A[(size_t)i * r + c] * A[(size_t)i * r + c];
    double nrm = sqrt(s2);
    lambda[c] = nrm;
    if (nrm > 0.0)
      for (int64_t i = 0; i < n; ++i) A[(size_t)i * r + c] /= nrm;
  }
}

/* Eq. 5.1 with ||X - M||^2 = ||X||^2 - 2 <X, M> + ||M||^2 */
double orc_fit(const orc_index* X, const double* const* factors, const double* lambda, int r) {
  int order = X->order;
  double nx2 = 0.0, inner = 0.0;
  for (int64_t e = 0; e < X->nnz; ++e) {
    double x = X->coo_val[e];
    nx2 += x * x;
    double mval = 0.0;
    for (int c = 0; c < r; ++c) {
      double v = lambda[c];
      for (int m = 0; m < order; ++m) v *= factors[m][(size_t)X->coo_idx[m][e] * r + c];
      mval += v;
    }
    inner += x * mval;
  }
  double nm2 = 0.0;
  for (int a = 0; a < r; ++a)
    for (int b = 0; b < r; ++b) {
      double h = lambda[a] * lambda[b];
      for (int m = 0; m < order; ++m) {
        double s2 = 0.0;
        for (int64_t i = 0; i < X->dims[m]; ++i)
          s2 += factors[m][(size_t)i * r + a] * factors[m][(size_t)i * r + b];
        h *= s2;
      }
      nm2 += h;
    }
  double F = nx2 - 2.0 * inner + nm2;
  if (F < 0.0) F = 0.0;
  return nx2 > 0.0 ? 1.0 - sqrt(F) / sqrt(nx2) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Estimated fit (Section 5.4): a stratified sample of tensor elements,      */
/* ceil(alpha s_fit) nonzeros and the rest zeros, each uniform over its      */
/* stratum; the zeros by rejection of uniform coordinates.  The squared      */
/* residual of each sampled element is weighted by the stratum's size over   */
/* its sample count.                                                        */
/* ------------------------------------------------------------------------ */
static const orc_index* g_lin_X; /* comparator context (the oracle is single-threaded) */

/* compare two coordinates by the linear index of Eq. 2.2 over all modes (mode 0
 * fastest): the last mode is the most significant digit */
static int cmp_coord(const int32_t* a, const int32_t* b, int order) {
  for (int m = order - 1; m >= 0; --m)
    if (a[m] != b[m]) return a[m] < b[m] ? -1 : 1;
  return 0;
}

static int cmp_nz_linear(const void* pa, const void* pb) {
  const int64_t ea = *(const int64_t*)pa, eb = *(const int64_t*)pb;
  int32_t a[16], b[16];
  for (int m = 0; m < g_lin_X->order; ++m) {
    a[m] = g_lin_X->coo_idx[m][ea];
    b[m] = g_lin_X->coo_idx[m][eb];
  }
  return cmp_coord(a, b, g_lin_X->order);
}

/* floor(u * n / 2^64) */
static int64_t scale_u64(uint64_t u, int64_t n) {
  return (int64_t)(((unsigned __int128)u * (uint64_t)n) >> 64);
}

int orc_fit_sample(const orc_index* X, int64_t s_fit, double alpha, uint64_t seed, int reject_cap,
                   int32_t* coords, double* xs, int64_t* counts, double* phi) {
  const int order = X->order;
  const int64_t nnz = X->nnz;
  if (s_fit < 1 || !(alpha > 0.0 && alpha <= 1.0) || nnz < 1) return ORC_ERR_ARG;
  /* number of elements, prod n (rounded in FP64 when above 2^53) */
  double cells = 1.0;
  for (int m = 0; m < order; ++m) cells *= (double)X->dims[m];
  const int has_zeros = cells > (double)nnz;
  int64_t s_nz = (int64_t)ceil(alpha * (double)s_fit);
  if (s_nz > s_fit) s_nz = s_fit;
  const int64_t s_z = has_zeros ? s_fit - s_nz : 0;
  /* the nonzeros in ascending linear-index order */
  int64_t* order_e = (int64_t*)malloc(sizeof(int64_t) * (size_t)nnz);
  if (!order_e) return ORC_ERR_OOM;
  for (int64_t e = 0; e < nnz; ++e) order_e[e] = e;
  g_lin_X = X;
  qsort(order_e, (size_t)nnz, sizeof(int64_t), cmp_nz_linear);
  const uint64_t key[2] = {seed, 0};
  for (int64_t j = 0; j < s_nz; ++j) {
    const uint64_t ctr[4] = {(uint64_t)j, 0, 2ull << 32, 0};
    uint64_t out[4];
    orc_philox4x64_10(ctr, key, out);
    const int64_t e = order_e[scale_u64(out[0], nnz)];
    for (int m = 0; m < order; ++m) coords[(size_t)m * s_fit + j] = X->coo_idx[m][e];
    xs[j] = X->coo_val[e];
  }
  int64_t attempts = 0;
  for (int64_t j = 0; j < s_z; ++j) {
    int accepted = 0;
    for (int a = 0; a < reject_cap && !accepted; ++a) {
      int32_t c[16];
      for (int m = 0; m < order; ++m) {
        const uint64_t ctr[4] = {(uint64_t)j, (uint64_t)a, (2ull << 32) | 1ull | ((uint64_t)(m / 4) << 16), 0};
        uint64_t out[4];
        orc_philox4x64_10(ctr, key, out);
        c[m] = (int32_t)scale_u64(out[m % 4], X->dims[m]);
      }
      ++attempts;
      /* is c a nonzero?  bisection over the sorted nonzeros */
      int64_t lo = 0, hi = nnz;
      int hit = 0;
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        int32_t b[16];
        for (int m = 0; m < order; ++m) b[m] = X->coo_idx[m][order_e[mid]];
        const int cmp = cmp_coord(b, c, order);
        if (cmp == 0) { hit = 1; break; }
        if (cmp < 0) lo = mid + 1; else hi = mid;
      }
      if (!hit) {
        for (int m = 0; m < order; ++m) coords[(size_t)m * s_fit + s_nz + j] = c[m];
        xs[s_nz + j] = 0.0;
        accepted = 1;
      }
    }
    if (!accepted) {
      free(order_e);
      return ORC_ERR_REJECT_LIMIT;
    }
  }
  free(order_e);
  counts[0] = s_nz;
  counts[1] = s_z;
  counts[2] = attempts;
  phi[0] = s_nz > 0 ? (double)nnz / (double)s_nz : 0.0;
  phi[1] = s_z > 0 ? (cells - (double)nnz) / (double)s_z : 0.0;
  return ORC_OK;
}

double orc_fit_estimate(const orc_index* X, const int32_t* coords, const double* xs,
                        const int64_t* counts, const double* phi, int64_t stride,
                        const double* const* factors, const double* lambda, int r, double* F_hat_out) {
  const int order = X->order;
  double nx2 = 0.0;
  for (int64_t e = 0; e < X->nnz; ++e) nx2 += X->coo_val[e] * X->coo_val[e];
  const int64_t S = counts[0] + counts[1];
  double F = 0.0;
  for (int64_t j = 0; j < S; ++j) {
    double mval = 0.0;
    for (int c = 0; c < r; ++c) {
      double v = lambda[c];
      for (int m = 0; m < order; ++m) v *= factors[m][(size_t)coords[(size_t)m * stride + j] * r + c];
      mval += v;
    }
    const double res = mval - xs[j];
    F += (j < counts[0] ? phi[0] : phi[1]) * res * res;
  }
  if (F_hat_out) *F_hat_out = F;
  return nx2 > 0.0 ? 1.0 - sqrt(F) / sqrt(nx2) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Randomized range finder initialisation (App. F): a random linear         */
/* combination of s_init mode-k fibres (columns of the unfolding X_(k))     */
/* drawn uniformly, with replacement, from the nonzero fibres.              */
/* ------------------------------------------------------------------------ */
int orc_rrf_init(const orc_index* X, int k, int64_t s_init, uint64_t seed, const double* omega, int r,
                 double* A) {
  if (k < 0 || k >= X->order || s_init < 1 || r < 1 || X->nnz < 1) return ORC_ERR_ARG;
  const int64_t F = X->nfib[k];
  memset(A, 0, sizeof(double) * (size_t)X->dims[k] * r);
  const uint64_t key[2] = {seed, 0};
  for (int64_t j = 0; j < s_init; ++j) {
    const uint64_t ctr[4] = {(uint64_t)j, 0, (3ull << 32) | (uint64_t)k, 0};
    uint64_t out[4];
    orc_philox4x64_10(ctr, key, out);
    /* the f-th nonzero fibre in ascending order of its linear key (Eq. 2.2) */
    const int64_t f = scale_u64(out[0], F);
    for (int64_t e = X->off[k][f]; e < X->off[k][f + 1]; ++e) {
      const double x = X->val[k][e];
      double* row = A + (size_t)X->ik[k][e] * r;
      for (int c = 0; c < r; ++c) row[c] += x * omega[(size_t)j * r + c];
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3                                                                   */
/* ------------------------------------------------------------------------ */
/* Row scores of one factor, summing to r, whose ratio to r is the factor's sampling
 * distribution: leverage scores (Alg. 3), or for the comparison of App. B the
 * uniform score r / n or the length-squared score r ||a_i||^2 / ||A||_F^2 (of the
 * factor as given: column-normalised after an update, the caller's initial guess at
 * the start). */
int orc_scores(const double* A, int64_t n, int r, int dist, double* s, int* rank) {
  if (dist == ORC_DIST_LEVERAGE) return orc_leverage(A, n, r, s, rank);
  *rank = r;
  if (dist == ORC_DIST_UNIFORM) {
    for (int64_t i = 0; i < n; ++i) s[i] = (double)r / (double)n;
    return ORC_OK;
  }
  if (dist != ORC_DIST_LENGTH_SQUARED) return ORC_ERR_ARG;
  double fro = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < r; ++c) fro += A[(size_t)i * r + c] * A[(size_t)i * r + c];
  for (int64_t i = 0; i < n; ++i) {
    double row = 0.0;
    for (int c = 0; c < r; ++c) row += A[(size_t)i * r + c] * A[(size_t)i * r + c];
    s[i] = fro > 0.0 ? (double)r * row / fro : 0.0;
  }
  return ORC_OK;
}

static int refresh_mode(orc_state* st, int m, const double* A) {
  int rank = 0;
  int rc = orc_scores(A, st->dims[m], st->r, st->dist, st->lev[m], &rank);
  if (rc < 0) return rc;
  if (rc & ORC_WARN_RANK_DEFICIENT_LEV) st->warnings |= ORC_WARN_RANK_DEFICIENT_LEV;
  st->T[m] = orc_cdf(st->lev[m], st->dims[m], st->r, st->q[m], st->C[m], &st->maxq[m],
                     &st->nnzq[m]);
  return ORC_OK;
}

int orc_state_init(orc_state* st, int order, const int64_t* dims, int r,
                   double* const* factors, int dist) {
  memset(st, 0, sizeof(*st));
  st->order = order;
  st->r = r;
  st->dist = dist;
  for (int m = 0; m < order; ++m) {
    st->dims[m] = dims[m];
    st->lev[m] = (double*)malloc(sizeof(double) * (size_t)dims[m]);
    st->q[m] = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)dims[m]);
    st->C[m] = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)dims[m]);
    int rc = refresh_mode(st, m, factors[m]);
    if (rc < 0) return rc;
  }
  return ORC_OK;
}

void orc_state_free(orc_state* st) {
  for (int m = 0; m < st->order; ++m) { free(st->lev[m]); free(st->q[m]); free(st->C[m]); }
}

int orc_mode_update(const orc_index* X, orc_state* st, int k, double* const* factors,
                    double* lambda, int64_t s, double tau, uint64_t seed, uint64_t iter,
                    int64_t det_cap, int reject_cap,
                    uint64_t* idx_out, uint32_t* cnt_out, double* wgt_out) {
  int order = X->order, r = st->r;
  int64_t n_o[16], nnzq_o[16];
  const uint64_t* C_o[16];
  uint64_t T_o[16], maxq_o[16];
  int d = 0;
  for (int m = 0; m < order; ++m) {
    if (m == k) continue;
    n_o[d] = st->dims[m]; C_o[d] = st->C[m]; T_o[d] = st->T[m];
    maxq_o[d] = st->maxq[m]; nnzq_o[d] = st->nnzq[m];
    ++d;
  }
  orc_sampler S = {d, n_o, C_o, T_o, maxq_o, nnzq_o};
  uint64_t* idx = idx_out ? idx_out : (uint64_t*)malloc(sizeof(uint64_t) * (size_t)s);
  uint32_t* cnt = cnt_out ? cnt_out : (uint32_t*)malloc(sizeof(uint32_t) * (size_t)s);
  double* wgt = wgt_out ? wgt_out : (double*)malloc(sizeof(double) * (size_t)s);
  int64_t sbar = 0;
  int rc = orc_skrp_lev(&S, s, tau, seed, iter, k, det_cap, reject_cap, idx, cnt, wgt, &sbar,
                        &st->sdet, &st->pdet, &st->attempts);
  if (rc >= 0) {
    st->sbar = sbar;
    int64_t nk = st->dims[k];
    double* M = (double*)malloc(sizeof(double) * (size_t)nk * r);
    double* G = (double*)malloc(sizeof(double) * (size_t)r * r);
    orc_sampled_mttkrp(X, k, (const double* const*)factors, r, idx, wgt, sbar, M, G,
                       &st->nnz_sampled);
    int src = orc_solve(G, M, nk, r, factors[k]);
    if (src > 0) st->warnings |= src;
    orc_normalize(factors[k], nk, r, lambda);
    rc = refresh_mode(st, k, factors[k]);
    free(M);
    free(G);
  }
  if (!idx_out) free(idx);
  if (!cnt_out) free(cnt);
  if (!wgt_out) free(wgt);
  return rc;
}

int orc_cp_arls_lev(const orc_index* X, int r, int64_t s, double tau, int iters, int epoch_len,
                    int patience, double tol, uint64_t seed, uint64_t iter_offset,
                    int64_t det_cap, int reject_cap, double* const* factors, double* lambda,
                    double* fit, int* iters_done, int dist) {
  int order = X->order;
  orc_state st;
  int rc = orc_state_init(&st, order, X->dims, r, factors, dist);
  if (rc < 0) { orc_state_free(&st); return rc; }
  for (int c = 0; c < r; ++c) lambda[c] = 1.0;
  int it = 0, bad = 0;
  double best = -INFINITY, f = 0.0;
  if (epoch_len < 1) epoch_len = 1;
  while (it < iters) {
    for (int l = 0; l < epoch_len && it < iters; ++l, ++it)
      for (int k = 0; k < order; ++k) {
        rc = orc_mode_update(X, &st, k, factors, lambda, s, tau, seed, iter_offset + (uint64_t)it,
                             det_cap, reject_cap, NULL, NULL, NULL);
        if (rc < 0) { orc_state_free(&st); return rc; }
      }
    if (tol > 0.0) {
      f = orc_fit(X, (const double* const*)factors, lambda, r);
      if (f > best + tol) { best = f; bad = 0; } else if (++bad >= patience) break;
    }
  }
  if (!(tol > 0.0)) f = orc_fit(X, (const double* const*)factors, lambda, r);
  if (fit) *fit = f;
  if (iters_done) *iters_done = it;
  int warn = st.warnings;
  orc_state_free(&st);
  return warn;
}

int orc_cp_als(const orc_index* X, int r, int iters, double* const* factors, double* lambda,
               double* fit) {
  int order = X->order;
  int warn = 0;
  for (int c = 0; c < r; ++c) lambda[c] = 1.0;
  for (int it = 0; it < iters; ++it)
    for (int k = 0; k < order; ++k) {
      int64_t nk = X->dims[k];
      double* M = (double*)malloc(sizeof(double) * (size_t)nk * r);
      double* G = (double*)malloc(sizeof(double) * (size_t)r * r);
      orc_exact_mttkrp(X, k, (const double* const*)factors, r, M, G);
      int src = orc_solve(G, M, nk, r, factors[k]);
      if (src > 0) warn |= src;
      orc_normalize(factors[k], nk, r, lambda);
      free(M);
      free(G);
    }
  if (fit) *fit = orc_fit(X, (const double* const*)factors, lambda, r);
  return warn;
}

/* One mode update from scratch: leverage of every mode from the given factors,
 * then orc_mode_update.  Outputs the sampled rows and the statistics. */
int orc_mode_update_once(const orc_index* X, int r, int k, double* const* factors,
                         double* lambda, int64_t s, double tau, uint64_t seed, uint64_t iter,
                         int64_t det_cap, int reject_cap, uint64_t* idx, uint32_t* cnt,
                         double* wgt, int64_t* stats /* sbar, sdet, nnz_sampled, attempts */,
                         double* pdet, int dist) {
  orc_state st;
  int rc = orc_state_init(&st, X->order, X->dims, r, factors, dist);
  if (rc >= 0)
    rc = orc_mode_update(X, &st, k, factors, lambda, s, tau, seed, iter, det_cap, reject_cap,
                         idx, cnt, wgt);
  if (rc >= 0) {
    stats[0] = st.sbar; stats[1] = st.sdet; stats[2] = st.nnz_sampled; stats[3] = st.attempts;
    *pdet = st.pdet;
    rc = st.warnings;
  }
  orc_state_free(&st);
  return rc;
}
