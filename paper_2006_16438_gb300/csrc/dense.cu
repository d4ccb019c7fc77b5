// Dense kernels of the per-mode update (see dense.cuh).
//
// The factor-matrix Gram A^T A and the solve are FP64 on CUDA cores: r is at most
// 64, so they are skinny (n x r times r x n) and bound by FP64 issue on this part.
// The r x r factorisation runs in one thread block.
#include "dense.cuh"
#include "ffloat.cuh"

namespace cpa {

namespace {

constexpr int kGramRows = 32;   // rows staged per tile
constexpr int kGramThreads = 256;      // threads when a thread owns several pairs
constexpr int kGramMaxThreads = 1024;  // one pair per thread up to this many pairs

// Upper-triangle pair p -> (a, b), a <= b, row-major over a.
__device__ __forceinline__ void pair_of(int p, int r, int* a, int* b) {
  int row = 0, start = 0;
  while (p >= start + (r - row)) {
    start += r - row;
    ++row;
  }
  *a = row;
  *b = row + (p - start);
}

// The block's pair sums go to its partials; the last block to finish adds all
// blocks' partials in block order and writes the symmetric G (so G is the same bit
// for bit at every run with the same grid).
template <int PMAX>
__device__ __forceinline__ void gram_block_finish(const double* acc, int np, int r, double* G, const BlockSums& S) {
  double* mine = S.part + (size_t)blockIdx.x * np;
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * (int)blockDim.x;
    if (p < np) mine[p] = acc[q];
  }
  if (!last_block_to_arrive(S.ticket)) return;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double v = ordered_block_sum(S.part, gridDim.x, np, p);
    int a, b;
    pair_of(p, r, &a, &b);
    G[a * r + b] = v;
    G[b * r + a] = v;
  }
  rearm_ticket(S.ticket);
}

// Factor rows of storage type FT are multiplied and summed in FP64 (the Gram feeds
// leverage scores and the fit).  The tile is converted to FP64 once when staged: on
// GB300 a conversion issues on the FP64 pipe like a multiply-add.
template <class FT, int PMAX>
__global__ void __launch_bounds__(kGramMaxThreads) k_gram_rows(const FT* __restrict__ A,
                                                            int64_t n, int r, int lda,
                                                            double* __restrict__ G, BlockSums S) {
  const int nt = blockDim.x;
  extern __shared__ __align__(16) unsigned char gram_smem[];
  double* tile = reinterpret_cast<double*>(gram_smem);  // kGramRows * r
  const int np = r * (r + 1) / 2;
  int pa[PMAX], pb[PMAX];
  double acc[PMAX];
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * nt;
    if (p < np) pair_of(p, r, &pa[q], &pb[q]); else pa[q] = pb[q] = 0;
    acc[q] = 0.0;
  }
  for (int64_t row0 = (int64_t)blockIdx.x * kGramRows; row0 < n;
       row0 += (int64_t)gridDim.x * kGramRows) {
    const int rows = (int)((n - row0) < kGramRows ? (n - row0) : kGramRows);
    __syncthreads();
    const FT* src = A + row0 * lda;
    for (int i = threadIdx.x; i < kGramRows * r; i += nt) {
      const int rr = i / r, c = i - rr * r;
      tile[i] = rr < rows ? (double)src[(int64_t)rr * lda + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
      const int p = threadIdx.x + q * nt;
      if (p < np) {
        double s = 0.0;
        for (int i = 0; i < rows; ++i) s = fma(tile[i * r + pa[q]], tile[i * r + pb[q]], s);
        acc[q] += s;
      }
    }
  }
  gram_block_finish<PMAX>(acc, np, r, G, S);
}

// FP32 factors: the same Gram on the FP32 pipe.  Each float product is split
// exactly into its rounded value p and error e = fma(a, b, -p); p is added to a
// float pair (hi, lo) by TwoSum (Knuth) and e into lo, so a 64-row tile is summed to
// about 2^-44 relative before the tile is added in FP64.  The _rn intrinsics keep the
// compiler from fusing the error-free steps.
constexpr int kGramRowsFF = 64;

template <int PMAX>
__global__ void __launch_bounds__(kGramMaxThreads) k_gram_rows_ff(const float* __restrict__ A, int64_t n, int r,
                                                               int lda, double* __restrict__ G, BlockSums S) {
  const int nt = blockDim.x;
  extern __shared__ __align__(16) unsigned char gram_smem[];
  float* tile = reinterpret_cast<float*>(gram_smem);  // kGramRowsFF * r
  const int np = r * (r + 1) / 2;
  int pa[PMAX], pb[PMAX];
  double acc[PMAX];
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * nt;
    if (p < np) pair_of(p, r, &pa[q], &pb[q]); else pa[q] = pb[q] = 0;
    acc[q] = 0.0;
  }
  for (int64_t row0 = (int64_t)blockIdx.x * kGramRowsFF; row0 < n; row0 += (int64_t)gridDim.x * kGramRowsFF) {
    const int rows = (int)((n - row0) < kGramRowsFF ? (n - row0) : kGramRowsFF);
    __syncthreads();
    const float* src = A + row0 * lda;
    for (int i = threadIdx.x; i < kGramRowsFF * r; i += nt) {
      const int rr = i / r, c = i - rr * r;
      tile[i] = rr < rows ? src[(int64_t)rr * lda + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
      const int p = threadIdx.x + q * nt;
      if (p < np) {
        float hi = 0.f, lo = 0.f;
        for (int i = 0; i < rows; ++i) {
          const float a = tile[i * r + pa[q]], b = tile[i * r + pb[q]];
          const float pr = __fmul_rn(a, b);
          const float e = __fmaf_rn(a, b, -pr);
          const float t = __fadd_rn(hi, pr);
          const float z = __fsub_rn(t, hi);
          const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(pr, z));
          hi = t;
          lo = __fadd_rn(lo, __fadd_rn(err, e));
        }
        acc[q] += (double)hi + (double)lo;
      }
    }
  }
  gram_block_finish<PMAX>(acc, np, r, G, S);
}

// ---- r x r factorisation in one block -------------------------------------
constexpr int kFactorThreads = 256;

// Cyclic Jacobi eigendecomposition of the symmetric matrix in `a` (r x r in shared
// memory, overwritten by its eigenvalues on the diagonal), eigenvectors in the
// columns of `v`, by all threads of the block (every thread must call it).  Each
// round applies r/2 disjoint rotations (round-robin pairing: index m - 1 fixed, the
// others rotating; m = r rounded up to even, pairs with the padding index skipped):
// the angles from the round's a_pp, a_qq, a_pq (Rutishauser's formulas), then the
// column phase a <- a J, v <- v J and the row phase a <- J^T a, exact because the
// rotations of a round touch disjoint index pairs.  A sweep is m - 1 rounds; sweeps
// stop when the off-diagonal mass falls below 1e-30 of the total (at most 60).
__device__ __noinline__ void jacobi_eigen_block(double* a, double* v, int r, int tid, int nt) {
  __shared__ double rc[kMaxRank / 2], rs[kMaxRank / 2];
  __shared__ int rp[kMaxRank / 2], rq[kMaxRank / 2];
  __shared__ double red[kFactorThreads / 32];
  __shared__ int done;
  const int m = (r + 1) & ~1;
  const int half = m / 2;
  for (int i = tid; i < r * r; i += nt) v[i] = (i / r == i % r) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    // convergence: off = 2 sum_{i<j} a_ij^2 against diag = sum a_ii^2
    double off = 0.0, diag = 0.0;
    for (int i = tid; i < r * r; i += nt) {
      const int row = i / r, col = i - row * r;
      const double x = a[i];
      if (row == col) diag += x * x; else off += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      diag += __shfl_xor_sync(0xffffffffu, diag, o);
    }
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      double o_sum = 0.0;
      for (int w = 0; w < (nt >> 5); ++w) o_sum += red[w];
      red[0] = o_sum;
    }
    __syncthreads();
    const double off_all = red[0];
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = diag;
    __syncthreads();
    if (tid == 0) {
      double d_sum = 0.0;
      for (int w = 0; w < (nt >> 5); ++w) d_sum += red[w];
      done = (off_all == 0.0 || off_all <= 1e-30 * (off_all + d_sum)) ? 1 : 0;
    }
    __syncthreads();
    if (done) break;
    for (int round = 0; round < m - 1; ++round) {
      if (tid < half) {
        int p, q;
        if (tid == 0) {
          p = m - 1;
          q = round;
        } else {
          p = (round + tid) % (m - 1);
          q = (round - tid + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int t2 = p;
          p = q;
          q = t2;
        }
        double c = 1.0, sn = 0.0;
        if (q < r) {
          const double apq = a[p * r + q];
          if (apq != 0.0) {
            const double zeta = (a[q * r + q] - a[p * r + p]) / (2.0 * apq);
            const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = rsqrt(1.0 + t * t);
            sn = t * c;
          }
        } else {
          p = q = -1;  // pairs with the padding index do nothing
        }
        rc[tid] = c;
        rs[tid] = sn;
        rp[tid] = p;
        rq[tid] = q;
      }
      __syncthreads();
      for (int w = tid; w < half * r; w += nt) {  // a <- a J, v <- v J (columns p, q)
        const int k = w / r, i = w - k * r;
        const int p = rp[k], q = rq[k];
        if (p < 0) continue;
        const double c = rc[k], sn = rs[k];
        const double aip = a[i * r + p], aiq = a[i * r + q];
        a[i * r + p] = c * aip - sn * aiq;
        a[i * r + q] = sn * aip + c * aiq;
        const double vip = v[i * r + p], viq = v[i * r + q];
        v[i * r + p] = c * vip - sn * viq;
        v[i * r + q] = sn * vip + c * viq;
      }
      __syncthreads();
      for (int w = tid; w < half * r; w += nt) {  // a <- J^T a (rows p, q)
        const int k = w / r, j = w - k * r;
        const int p = rp[k], q = rq[k];
        if (p < 0) continue;
        const double c = rc[k], sn = rs[k];
        const double apj = a[p * r + j], aqj = a[q * r + j];
        a[p * r + j] = c * apj - sn * aqj;
        a[q * r + j] = sn * apj + c * aqj;
      }
      __syncthreads();
    }
  }
}

// 1/sqrt(d) for d > 0 in FP64, without a branch (so the compiler can overlap it with
// the pivot search): d = m 4^k with m in [1, 4) by integer operations, an FP32 seed
// y0 = rsqrt(f) from m's exponent and upper 20 significand bits, e = 1 - m y0^2
// (|e| < 2^-18), y0 (1 + e/2 + 3 e^2 / 8) (the binomial series of (1 - e)^(-1/2) to
// second order: relative error about 5 e^3 / 16 < 2^-55 before rounding), then the
// exponent lowered by k.  The power-of-4 scaling is exact, so the result is the one the
// same steps give on d itself.  GB300 FP64 division and square root cost hundreds of
// cycles each (every FP64 warp instruction issues over 64 cycles), so the
// factorisation keeps them off its chain.  d must be a positive normal number
// (anything else gives 0).
__device__ __forceinline__ double rsqrt_newton(double d) {
  const unsigned long long ub = (unsigned long long)__double_as_longlong(d);
  const int E = (int)((ub >> 52) & 0x7ffu);
  const int ex = E - 1023, k = ex >> 1, em = ex - 2 * k;  // d = m 4^k, m = 1.f 2^em, em in {0, 1}
  const double m = __longlong_as_double((long long)((ub & 0x000fffffffffffffull) | ((unsigned long long)(1023 + em) << 52)));
  const float f = __int_as_float(((em + 127) << 23) | (int)((ub >> 29) & 0x7ffff8u));
  const int yb = __float_as_int(rsqrtf(f));
  const int ye = ((yb >> 23) & 0xff) - 127;
  const double y0 = __hiloint2double(((ye + 1023) << 20) | ((yb & 0x7fffff) >> 3), (yb & 7) << 29);
  const double e = fma(-m, y0 * y0, 1.0);
  const double y = fma(y0, e * fma(e, 0.375, 0.5), y0);  // 1 / sqrt(m), in (0.5, 1]
  const long long r = __double_as_longlong(y) - (long long)k * (1ll << 52);
  return E >= 1 && E <= 2046 && !(ub >> 63) ? __longlong_as_double(r) : 0.0;
}

// 1/d for d > 0 in FP64 (0 for d <= 0, not finite, subnormal or from 2^1022 on),
// without a branch: d = m 2^ex with m in [1, 2) by integer operations, an FP32 seed
// from m's upper 20 significand bits, x = its approximate FP32 reciprocal, e = 1 - m x
// (|e| < 2^-19), x (1 + e + e^2) (the truncated series of 1/(1 - e): relative error
// about e^3 < 2^-56 before rounding), then the exponent lowered by ex.  The
// power-of-2 scaling is exact, so the result is the one the same steps give on d.
__device__ __forceinline__ double rcp_newton(double d) {
  const unsigned long long ub = (unsigned long long)__double_as_longlong(d);
  const int E = (int)((ub >> 52) & 0xfffu);  // with the sign bit: negative d gives E > 2047
  const double m = __longlong_as_double((long long)((ub & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
  const float f = __int_as_float((127 << 23) | (int)((ub >> 29) & 0x7ffff8u));
  float xf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(xf) : "f"(f));  // the seed needs no correct rounding
  const int xb = __float_as_int(xf);
  const int xe = ((xb >> 23) & 0xff) - 127;
  const double x = __hiloint2double(((xe + 1023) << 20) | ((xb & 0x7fffff) >> 3), (xb & 7) << 29);
  const double e = fma(-m, x, 1.0);
  const double y = fma(x, fma(e, e, e), x);  // 1 / m, in (0.5, 1]
  const long long r = __double_as_longlong(y) - (long long)(E - 1023) * (1ll << 52);
  return E >= 1 && E <= 2044 ? __longlong_as_double(r) : 0.0;
}

// Order-preserving 32-bit key of a double for the pivot search: the upper word of a
// positive double orders like its value (ties within 2^-20 relative); values <= 0 map
// to 0.  Integer operations only (FP64 conversions use the slow FP64 pipe).
__device__ __forceinline__ unsigned pivot_key(double v) {
  const long long b = __double_as_longlong(v);
  return b > 0 ? (unsigned)((unsigned long long)b >> 32) : 0u;
}

// Factor one r x r PSD matrix in one block of kFactorThreads threads (see SmallFactor).
//
// Square-root-free Cholesky S = P L D L^T P^T of S = diag(scale) G diag(scale), L unit
// lower triangular, with diagonal pivoting (pivot = 1: the largest remaining diagonal
// entry first, stopping at the numerical rank) or without (pivot = 0).  The unit
// lower inverse X = L^{-1} is accumulated in the same sweep: by the recurrence
// X(j, :) = e_j - sum_{u<j} L(j, u) X(u, :), row j of X is final when j is pivoted,
// and its contribution L(i, j) X(j, :) is added at once to every remaining row i
// (kept as B = -sum L X).  Pivoting is by index: entries stay in place (S is kept
// symmetric, by original index) and ord[] maps pivot positions to original indices.
//
// One block barrier per step.  The Schur complement lives in two buffers (step j
// reads one and writes the other).  Step j's pivot p, D_j, 1 / D_j and its staged row
// sp = S(p, :), sh = sp / D_j are ready when the step starts.  In the step, warp 0 runs
// the serial chain: the remaining diagonal, the next pivot, its reciprocal (seeded by
// integer operations) and the next pivot row, each entry with the same arithmetic as
// the pair update below, so the next step needs no staging phase.  Meanwhile the warps
// on the other three SM sub-partitions update every remaining off-diagonal entry and
// every entry of B(i, 0..j), one FMA of staged values each, packed over their threads
// (a GB300 FP64 warp instruction costs the same with any number of active lanes).
// Outputs:
//  * pivot = 1: F = D^{-1/2} X (the inverse of the Cholesky factor L D^{1/2}),
//    perm = the pivot order, rank = the number of pivots (kind 0);
//  * pivot = 0: F = X^T D^{-1} X = S^{-1} (kind 2);
//  * pivot = 0 and a pivot <= rel_tol * max diag: F = pinv(S) by Jacobi (kind 1).
__global__ void __launch_bounds__(kFactorThreads) k_factor_spd(const double* __restrict__ G,
                                                               int r, int normalize, int pivot,
                                                               double rel_tol,
                                                               SmallFactor* __restrict__ out,
                                                               int* warn, int warn_bit,
                                                               DistInfo* zero_info) {
  extern __shared__ double sm[];
  double* Sb0 = sm;            // r x r Schur complements (two buffers), by original index
  double* Sb1 = sm + r * r;
  double* B = sm + 2 * r * r;  // r x r: B(i, c) = -sum_u L(i, u) X(u, c), c in pivot order
  double* spb = B + r * r;     // 2 x r: S(p, c) of the pivot of step j (buffer j & 1)
  double* shb = spb + 2 * r;   // 2 x r: S(p, c) / D_j
  double* dinv = shb + 2 * r;  // r: 1 / D_j
  double* Dv = dinv + r;       // r: D_j
  double* scale = Dv + r;      // r
  __shared__ int ordb[2][kMaxRank];  // pivot position -> original index (after step j's swap: [(j + 1) & 1])
  __shared__ unsigned short tri[kMaxRank * (kMaxRank - 1) / 2];  // q -> (a, b), a > b
  __shared__ int perm[kMaxRank];
  __shared__ int s_fail;
  __shared__ double s_dmax;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  if (zero_info && tid == 0) {
    zero_info->maxq = 0;
    zero_info->nnzq = 0;
  }
  // every load of G issued up front (r <= 32: four entries per thread)
  constexpr int kGPer = (32 * 32 + kFactorThreads - 1) / kFactorThreads;
  const bool small = r <= 32;
  double gv[kGPer];
#pragma unroll
  for (int u = 0; u < kGPer; ++u) {
    const int i = tid + u * kFactorThreads;
    gv[u] = small && i < r * r ? G[i] : 0.0;
  }
  const double gd = tid < r ? G[tid * (r + 1)] : 0.0;
  for (int c = tid; c < r; c += nt) ordb[0][c] = c;
  for (int a = 1 + tid; a < r; a += nt)
    for (int b = 0; b < a; ++b) tri[a * (a - 1) / 2 + b] = (unsigned short)((a << 8) | b);
  if (normalize) {  // the column scales 1 / sqrt(G_cc) first: S = diag(scale) G diag(scale)
    if (tid < r) {
      const bool pos = pos_finite(gd);
      const double y = pos ? rsqrt_newton(gd) : 0.0;
      scale[tid] = y;
      out->scale[tid] = y;
      out->lambda[tid] = pos ? gd * y : 0.0;
    }
    __syncthreads();
  } else if (tid < r) {
    scale[tid] = 1.0;
    out->scale[tid] = 1.0;
  }
  if (small) {
#pragma unroll
    for (int u = 0; u < kGPer; ++u) {
      const int i = tid + u * kFactorThreads;
      if (i < r * r) {
        const int a = i / r, b = i - a * r;
        Sb0[i] = normalize ? gv[u] * (scale[a] * scale[b]) : gv[u];
        B[i] = 0.0;
      }
    }
  } else {
    for (int i = tid; i < r * r; i += nt) {
      const int a = i / r, b = i - a * r;
      Sb0[i] = normalize ? G[i] * (scale[a] * scale[b]) : G[i];
      B[i] = 0.0;
    }
  }
  __syncthreads();
  if (!normalize && warp == 4) {  // lambda_c = sqrt(G_cc), beside warp 0's first pivot
    for (int c = lane; c < r; c += 32) {
      const double g = Sb0[c * (r + 1)];
      out->lambda[c] = pos_finite(g) ? g * rsqrt_newton(g) : 0.0;
    }
  }
  // First pivot (warp 0): the diagonal's maximum, key argmax, reciprocal and row.
  if (warp == 0) {
    const int x0 = lane, x1 = lane + 32;
    const double v0 = x0 < r ? Sb0[x0 * (r + 1)] : 0.0, v1 = x1 < r ? Sb0[x1 * (r + 1)] : 0.0;
    // largest diagonal entry (negative entries count as 0) by integer max of bits
    long long mb = max(max(__double_as_longlong(v0), __double_as_longlong(v1)), 0ll);
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    int pp = 0;
    if (pivot) {
      const unsigned k0 = x0 < r ? pivot_key(v0) : 0u, k1 = x1 < r ? pivot_key(v1) : 0u;
      const unsigned km = __reduce_max_sync(0xffffffffu, k0 > k1 ? k0 : k1);
      const unsigned b0 = __ballot_sync(0xffffffffu, x0 < r && k0 == km);
      const unsigned b1 = __ballot_sync(0xffffffffu, x1 < r && k1 == km);
      pp = b0 ? __ffs(b0) - 1 : 32 + __ffs(b1) - 1;
    }
    const double dp = __shfl_sync(0xffffffffu, pp < 32 ? v0 : v1, pp & 31);
    const double di = pos_finite(dp) ? rcp_newton(dp) : 0.0;
    for (int c = lane; c < r; c += 32) {
      const double v = Sb0[pp * r + c];
      spb[c] = v;
      shb[c] = v * di;
      ordb[1][c] = c == 0 ? pp : (c == pp ? 0 : c);
    }
    if (lane == 0) {
      s_dmax = __longlong_as_double(mb);
      s_fail = 0;
      perm[0] = pp;
      Dv[0] = dp;
      dinv[0] = di;
    }
  }
  __syncthreads();
  const double cut = rel_tol * s_dmax;
  // the workers: the warps off warp 0's SM sub-partition (warp % 4 != 0)
  const int nwarps = nt >> 5;
  const int nworkers = (nwarps - (nwarps + 3) / 4) * 32;
  const int wt = (warp - 1 - (warp >> 2)) * 32 + lane;
  int k = r;
  for (int j = 0; j < r; ++j) {
    const double d = Dv[j];
    if (!(pos_finite(d) && nonneg_gt(d, cut))) {  // d > cut; same decision in every thread
      if (pivot) k = j; else if (tid == 0) s_fail = 1;
      break;
    }
    const int p = perm[j];
    const double* sp = spb + (j & 1) * r;
    const double* sh = shb + (j & 1) * r;
    const int* ordn = ordb[(j + 1) & 1];
    const int m = r - j - 1;        // remaining pivot positions j + 1 .. r - 1
    const int* rem = ordn + j + 1;  // their original indices
    const double* Sc = (j & 1) ? Sb1 : Sb0;
    double* Sn = (j & 1) ? Sb0 : Sb1;
    if (warp == 0) {
      if (m > 0) {
        const bool two = m > 32;  // warp-uniform: a second position per lane
        double v0 = 0.0, v1 = 0.0;  // the remaining diagonal
        if (lane < m) {
          const int i = rem[lane];
          v0 = fma(-sh[i], sp[i], Sc[i * (r + 1)]);
          Sn[i * (r + 1)] = v0;
        }
        if (two && lane + 32 < m) {
          const int i = rem[lane + 32];
          v1 = fma(-sh[i], sp[i], Sc[i * (r + 1)]);
          Sn[i * (r + 1)] = v1;
        }
        // the reciprocals of the whole remaining diagonal, overlapping the pivot search
        const double w0 = rcp_newton(v0);
        const double w1 = two ? rcp_newton(v1) : 0.0;
        int pq = 0;  // offset of the next pivot among the remaining positions
        if (pivot) {
          const unsigned k0 = lane < m ? pivot_key(v0) : 0u;
          const unsigned k1 = two && lane + 32 < m ? pivot_key(v1) : 0u;
          const unsigned km = __reduce_max_sync(0xffffffffu, k0 > k1 ? k0 : k1);
          const unsigned b0 = __ballot_sync(0xffffffffu, lane < m && k0 == km);
          const unsigned b1 = two ? __ballot_sync(0xffffffffu, lane + 32 < m && k1 == km) : 0u;
          pq = b0 ? __ffs(b0) - 1 : 32 + __ffs(b1) - 1;
        }
        const double dn = __shfl_sync(0xffffffffu, pq >= 32 ? v1 : v0, pq & 31);
        const double din = __shfl_sync(0xffffffffu, pq >= 32 ? w1 : w0, pq & 31);
        const int pn = rem[pq];
        double* spn = spb + ((j + 1) & 1) * r;
        double* shn = shb + ((j + 1) & 1) * r;
        // the next pivot row: the pair update's value for (pn, x), the row at the higher
        // position taking the role of i (at x = pn: the diagonal update's value, dn)
        for (int l = lane; l < m; l += 32) {
          const int x = rem[l];
          const bool up = l > pq;
          const double v = fma(-sh[up ? x : pn], sp[up ? pn : x], Sc[up ? x * r + pn : pn * r + x]);
          spn[x] = v;
          shn[x] = v * din;
        }
        int* ordnn = ordb[j & 1];  // the ordering after step j + 1's swap
        for (int c = lane; c < r; c += 32)
          ordnn[c] = c == j + 1 ? pn : (c == j + 1 + pq ? ordn[j + 1] : ordn[c]);
        if (lane == 0) {
          perm[j + 1] = pn;
          Dv[j + 1] = dn;
          dinv[j + 1] = din;
        }
      }
    } else if (warp & 3) {
      const int np = m * (m - 1) / 2;
      for (int q = wt; q < np; q += nworkers) {  // off-diagonal Schur complement
        const int ab = tri[q];
        const int i = rem[ab >> 8], c = rem[ab & 255];
        const double v = fma(-sh[i], sp[c], Sc[i * r + c]);
        Sn[i * r + c] = v;
        Sn[c * r + i] = v;
      }
      const int w = j + 1;
      const float inv_w = 1.0f / (float)w;
      for (int q = wt; q < m * w; q += nworkers) {  // B(i, :) -= L(i, j) X(j, :)
        const int row = __float2int_rz(((float)q + 0.5f) * inv_w);
        const int c = q - row * w;
        const int i = rem[row];
        const double xjc = c == j ? 1.0 : B[p * r + c];
        B[i * r + c] = fma(-sh[i], xjc, B[i * r + c]);
      }
    }
    __syncthreads();
  }
  __syncthreads();  // s_fail, and the step that ended the loop early
  double* S = Sb0;  // scratch from here on
  if (s_fail) {  // plain Cholesky failed: pseudo-inverse from the eigendecomposition
    double* X = B;
    double* y = shb;
    for (int i = tid; i < r * r; i += nt) {
      const int a = i / r, b = i - a * r;
      S[i] = G[i] * scale[a] * scale[b];
    }
    __syncthreads();
    jacobi_eigen_block(S, X, r, tid, nt);
    if (tid == 0) {
      double emax = 0.0;
      for (int c = 0; c < r; ++c) emax = fmax(emax, fabs(S[c * r + c]));
      for (int c = 0; c < r; ++c) {
        const double ev = S[c * r + c];
        y[c] = ev > rel_tol * emax ? 1.0 / ev : 0.0;
      }
      out->kind = 1;
      out->rank = r;
      atomicOr(warn, warn_bit);
    }
    __syncthreads();
    for (int i = tid; i < r * r; i += nt) {
      const int a = i / r, b = i - a * r;
      double s2 = 0.0;
      for (int c = 0; c < r; ++c) s2 += X[a * r + c] * y[c] * X[b * r + c];
      out->F[i] = s2;
    }
    for (int c = tid; c < r; c += nt) out->perm[c] = c;
    return;
  }
  // X(j, c) = [c == j] + B(perm_j, c) for c <= j < k
  if (pivot) {
    double* rs = shb;
    for (int j = tid; j < k; j += nt) rs[j] = rsqrt_newton(Dv[j]);
    __syncthreads();
    for (int i = tid; i < r * r; i += nt) {
      const int j = i / r, c = i - j * r;
      double v = 0.0;
      if (j < k && c <= j) v = (c == j ? 1.0 : B[perm[j] * r + c]) * rs[j];  // B(perm_j, j) = 0
      out->F[i] = v;
    }
    const int* ordk = ordb[k & 1];
    for (int c = tid; c < r; c += nt) out->perm[c] = c < k ? perm[c] : ordk[c];
    if (tid == 0) {
      out->kind = 0;
      out->rank = k;
      if (k < r) atomicOr(warn, warn_bit);
    }
    return;
  }
  // S^{-1} = X^T D^{-1} X (no pivoting: pivot order = original order): X to S, then
  // Y = D^{-1} X to B; F(a, b) = sum_{u >= a} X(u, a) Y(u, b) for b <= a, one pair per
  // thread (pairs by ascending a, so a warp's dot products have equal lengths), each in
  // four interleaved chains
  for (int i = tid; i < r * r; i += nt) {
    const int j = i / r, c = i - j * r;
    const double x = c == j ? 1.0 : (c < j ? B[j * r + c] : 0.0);  // B(j, j) = 0
    S[i] = x;
  }
  __syncthreads();
  for (int i = tid; i < r * r; i += nt) B[i] = S[i] * dinv[i / r];
  __syncthreads();
  const int npairs = r * (r + 1) / 2;
  for (int q = tid; q < npairs; q += nt) {
    int a = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= q) ++a;
    while (a * (a + 1) / 2 > q) --a;
    const int b = q - a * (a + 1) / 2;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int u = a;
    for (; u + 3 < r; u += 4) {
      s0 = fma(S[u * r + a], B[u * r + b], s0);
      s1 = fma(S[(u + 1) * r + a], B[(u + 1) * r + b], s1);
      s2 = fma(S[(u + 2) * r + a], B[(u + 2) * r + b], s2);
      s3 = fma(S[(u + 3) * r + a], B[(u + 3) * r + b], s3);
    }
    for (; u < r; ++u) s0 = fma(S[u * r + a], B[u * r + b], s0);
    const double v = (s0 + s1) + (s2 + s3);
    out->F[a * r + b] = v;
    out->F[b * r + a] = v;
  }
  for (int c = tid; c < r; c += nt) out->perm[c] = c;
  if (tid == 0) {
    out->kind = 2;
    out->rank = r;
  }
}

// ---- per-row kernels -------------------------------------------------------
// p > 0 ? min(p, 1) : 0 (NaN -> 0), by integer compares of the bit pattern
__device__ __forceinline__ double clamp01(double p) {
  const long long b = __double_as_longlong(p);
  if (b <= 0 || b > 0x7ff0000000000000ll) return 0.0;
  return b < 0x3ff0000000000000ll ? p : 1.0;
}

constexpr int kRowThreads = 256;

// Leverage of row a_i (one warp per row, lane c owns coordinate c and c + 32), in
// FP64 whatever the storage type FT of the factor:
// kind 0: y = X P^T (S a), l = ||y||^2 over the rank's coordinates;
// kind 1: l = (S a)^T F (S a).
// Denominator of the length-squared score: ||B||_F^2 with B the column-normalised
// factor (the number of nonzero columns) or the factor itself (sum of lambda_c^2).
__device__ __forceinline__ double lensq_den(const SmallFactor* f, int r, bool normalised) {
  double den = 0.0;
  for (int c = 0; c < r; ++c) {
    const double l = f->lambda[c];
    den += normalised ? (pos_finite(l) ? 1.0 : 0.0) : l * l;
  }
  return den;
}

template <class FT>
__global__ void __launch_bounds__(kRowThreads) k_lev_rows(const FT* A, int64_t n, int r, int lda,
                                                          const SmallFactor* __restrict__ f,
                                                          double* __restrict__ lev,
                                                          uint64_t* __restrict__ q,
                                                          DistInfo* info, FT* A_out, int dist) {
  extern __shared__ __align__(16) unsigned char lev_smem[];
  double* F = reinterpret_cast<double*>(lev_smem);  // r * r
  double* sc = F + r * r;                           // r
  FT* lam = reinterpret_cast<FT*>(sc + r);          // r
  __shared__ int perm[kMaxRank];
  __shared__ double brow[kRowThreads / 32][kMaxRank];  // each warp's row, scaled, FP64
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) F[i] = f->F[i];
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    sc[i] = f->scale[i];
    const double l = f->lambda[i];
    lam[i] = pos_finite(l) ? (FT)(1.0 / l) : FT(1);  // 1 / lambda_c, or 1 for a zero column
    perm[i] = f->perm[i];
  }
  __syncthreads();
  const int kind = f->kind;
  const int k = kind == 0 ? f->rank : r;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kRowThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kRowThreads) >> 5;
  const bool normalised = A_out != nullptr;
  const double den = dist == CPA_DIST_LENGTH_SQUARED ? lensq_den(f, r, normalised) : 1.0;
  uint64_t my_max = 0;
  uint32_t my_nz = 0;
  double* b = brow[threadIdx.x >> 5];
  for (int64_t row = gw; row < n; row += nwarps) {
    const FT* a = A + row * lda;
    double part = 0.0;
    if (dist == CPA_DIST_LEVERAGE) {
      // S a_i converted and scaled once (one FP64-pipe operation each), not per use
      __syncwarp();
      for (int c = lane; c < r; c += 32) b[c] = (double)a[c] * sc[c];
      __syncwarp();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        if (c < k) {
          double t = 0.0;
          if (kind == 0) {
            for (int u = 0; u <= c; ++u) t = fma(F[c * r + u], b[perm[u]], t);
            part = fma(t, t, part);
          } else {
            for (int u = 0; u < r; ++u) t = fma(F[c * r + u], b[u], t);
            part = fma(b[c], t, part);
          }
        }
      }
    } else if (dist == CPA_DIST_LENGTH_SQUARED) {
      for (int c = lane; c < r; c += 32) {
        const double b = normalised ? (double)a[c] * (double)lam[c] : (double)a[c];
        part = fma(b, b, part);
      }
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (dist == CPA_DIST_UNIFORM) part = (double)r / (double)n;
    else if (dist == CPA_DIST_LENGTH_SQUARED) part = den > 0.0 ? (double)r * part / den : 0.0;
    if (lane == 0) {
      if (lev) lev[row] = part;
      if (q) {
        double p = part / (double)r;
        p = clamp01(p);
        const uint64_t qi = __double2ull_rn(p * 4611686018427387904.0);  // 2^62
        q[row] = qi;
        my_max = qi > my_max ? qi : my_max;
        my_nz += qi > 0;
      }
    }
    if (A_out) {
      __syncwarp();
      for (int c = lane; c < r; c += 32) A_out[row * r + c] = a[c] * lam[c];
    }
  }
  if (q && info) {
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

// FP32 rows (mixed precision, many rows): one thread per row.  The rows of a tile are
// staged through shared memory (coalesced loads and stores), each thread holds its
// row and its r sums in registers and reads F four columns per shared-memory load
// (every thread the same address: a broadcast).  Each sum takes the products in the
// order u = 0..r-1 with fused multiply-adds, as k_solve_rows does, so the results are
// the same bit for bit.
template <int RB>
__global__ void __launch_bounds__(kRowThreads) k_solve_rows_f32(const float* __restrict__ M, int64_t n, int r,
                                                                const SmallFactor* __restrict__ f,
                                                                float* __restrict__ A, double* zero_gram) {
  extern __shared__ __align__(16) unsigned char solve_smem[];
  const int rp = (r + 3) & ~3;
  const int ld = r | 1;
  float* F = reinterpret_cast<float*>(solve_smem);  // r x rp, zero padded
  float* T = F + r * rp;                            // kRowThreads x ld tile of rows
  if (zero_gram && blockIdx.x == 0)
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) zero_gram[i] = 0.0;
  for (int i = threadIdx.x; i < r * rp; i += blockDim.x) {
    const int u = i / rp, c = i - u * rp;
    F[i] = c < r ? (float)f->F[u * r + c] : 0.f;
  }
  for (int64_t row0 = (int64_t)blockIdx.x * kRowThreads; row0 < n; row0 += (int64_t)gridDim.x * kRowThreads) {
    const int rows = (int)(n - row0 < kRowThreads ? n - row0 : kRowThreads);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
      const int rr = i / r, c = i - rr * r;
      T[rr * ld + c] = M[row0 * r + i];
    }
    __syncthreads();
    if (threadIdx.x < rows) {
      float x[RB], t[RB];
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        x[u] = u < r ? T[threadIdx.x * ld + u] : 0.f;
        t[u] = 0.f;
      }
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        if (u < r) {
          const float4* Fu = reinterpret_cast<const float4*>(F + u * rp);
#pragma unroll
          for (int c4 = 0; c4 < RB / 4; ++c4) {
            if (4 * c4 < r) {
              const float4 w = Fu[c4];
              t[4 * c4 + 0] = fmaf(x[u], w.x, t[4 * c4 + 0]);
              t[4 * c4 + 1] = fmaf(x[u], w.y, t[4 * c4 + 1]);
              t[4 * c4 + 2] = fmaf(x[u], w.z, t[4 * c4 + 2]);
              t[4 * c4 + 3] = fmaf(x[u], w.w, t[4 * c4 + 3]);
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < RB; ++c)  // the thread's own row of the tile
        if (c < r) T[threadIdx.x * ld + c] = t[c];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
      const int rr = i / r, c = i - rr * r;
      A[row0 * r + i] = T[rr * ld + c];
    }
  }
}

// A = M F with F the explicit inverse (kind 2) or pseudo-inverse (kind 1) of G:
// one thread per output element.
template <class FT>
__global__ void __launch_bounds__(kRowThreads) k_solve_rows(const FT* __restrict__ M,
                                                            int64_t n, int r,
                                                            const SmallFactor* __restrict__ f,
                                                            FT* __restrict__ A, double* zero_gram) {
  extern __shared__ __align__(16) unsigned char solve_smem[];
  FT* F = reinterpret_cast<FT*>(solve_smem);  // r * r
  if (zero_gram && blockIdx.x == 0)
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) zero_gram[i] = 0.0;
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) F[i] = (FT)f->F[i];
  __syncthreads();
  const int64_t total = n * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / r;
    const int c = (int)(e - row * r);
    const FT* m = M + row * r;
    FT t = FT(0);
    for (int u = 0; u < r; ++u) t = fma(m[u], F[u * r + c], t);
    A[e] = t;
  }
}

template <class FT>
__global__ void k_scale_columns(FT* A, int64_t n, int r, const double* __restrict__ lambda) {
  const int64_t total = n * r;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double l = lambda[i % r];
    if (l > 0.0) A[i] = (FT)((double)A[i] / l);
  }
}

// Leverage for many rows: one thread per row, rows staged through shared memory
// (coalesced), runtime loops over r (FP32 factors of large modes).
template <class FT>
__global__ void __launch_bounds__(kRowThreads) k_lev_rows_tpr(const FT* A, int64_t n, int r, int lda,
                                                              const SmallFactor* __restrict__ f,
                                                              double* __restrict__ lev,
                                                              uint64_t* __restrict__ q,
                                                              DistInfo* info, FT* A_out, int dist) {
  extern __shared__ __align__(16) unsigned char tpr_smem[];
  double* F = reinterpret_cast<double*>(tpr_smem);  // r * r
  double* sc = F + r * r;                           // r
  FT* lam = reinterpret_cast<FT*>(sc + r);          // r
  // rows staged as S a_i in FP64 (converted and scaled once each); an odd row stride
  // in doubles keeps a half-warp's reads of one column in distinct banks
  double* xs = reinterpret_cast<double*>(lam + ((r + 1) & ~1));  // kRowThreads * ld
  __shared__ int perm[kMaxRank];
  const int ld = r | 1;
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) F[i] = f->F[i];
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    sc[i] = f->scale[i];
    const double l = f->lambda[i];
    lam[i] = pos_finite(l) ? (FT)(1.0 / l) : FT(1);  // 1 / lambda_c, or 1 for a zero column
    perm[i] = f->perm[i];
  }
  const int kind = f->kind;
  const int k = kind == 0 ? f->rank : r;
  const bool normalised = A_out != nullptr;
  const double den = dist == CPA_DIST_LENGTH_SQUARED ? lensq_den(f, r, normalised) : 1.0;
  uint64_t my_max = 0;
  uint32_t my_nz = 0;
  for (int64_t row0 = (int64_t)blockIdx.x * kRowThreads; row0 < n; row0 += (int64_t)gridDim.x * kRowThreads) {
    const int rows = (int)(n - row0 < kRowThreads ? n - row0 : kRowThreads);
    __syncthreads();
    if (dist == CPA_DIST_LEVERAGE)
      for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
        const int rr = i / r, c = i - rr * r;
        xs[rr * ld + c] = (double)A[(row0 + rr) * lda + c] * sc[c];
      }
    __syncthreads();
    if (threadIdx.x < rows) {
      const double* x = xs + threadIdx.x * ld;
      const int64_t row = row0 + threadIdx.x;
      double l = 0.0;
      if (dist == CPA_DIST_LEVERAGE) {
        for (int c = 0; c < k; ++c) {
          double t = 0.0;
          if (kind == 0) {
            for (int u = 0; u <= c; ++u) t = fma(F[c * r + u], x[perm[u]], t);
            l = fma(t, t, l);
          } else {
            for (int u = 0; u < r; ++u) t = fma(F[c * r + u], x[u], t);
            l = fma(x[c], t, l);
          }
        }
      } else if (dist == CPA_DIST_UNIFORM) {
        l = (double)r / (double)n;
      } else {  // comparison distribution: read the row directly
        const FT* a = A + row * lda;
        for (int c = 0; c < r; ++c) {
          const double b = normalised ? (double)a[c] * (double)lam[c] : (double)a[c];
          l = fma(b, b, l);
        }
        l = den > 0.0 ? (double)r * l / den : 0.0;
      }
      if (lev) lev[row] = l;
      if (q) {
        double p = l / (double)r;
        p = clamp01(p);
        const uint64_t qi = __double2ull_rn(p * 4611686018427387904.0);  // 2^62
        q[row] = qi;
        my_max = qi > my_max ? qi : my_max;
        my_nz += qi > 0;
      }
    }
    if (A_out) {
      for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
        const int rr = i / r, c = i - rr * r;
        A_out[row0 * r + i] = A[(row0 + rr) * lda + c] * lam[c];
      }
    }
  }
  if (q && info) {
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t om = __shfl_xor_sync(0xffffffffu, my_max, o);
      my_max = om > my_max ? om : my_max;
      my_nz += __shfl_xor_sync(0xffffffffu, my_nz, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax((unsigned long long*)&info->maxq, (unsigned long long)my_max);
      atomicAdd((unsigned long long*)&info->nnzq, (unsigned long long)my_nz);
    }
  }
}

// ---- leverage of many FP32 rows on the FP32 pipe (float pairs: ffloat.cuh) ----
// ---- FP64 rows of many-row factors on the FP32 pipe --------------------------
// GB300's FP64 pipe runs at 1/64 of the FP32 rate, so the Gram and the leverage
// quadratic forms of FP64 factors with >= kManyRows rows take float-pair arithmetic:
// each FP64 value is split once into floats hi + lo (hi = the value with its low 29
// mantissa bits cleared, exact; lo = the rest rounded, 2^-48 relative), products and
// sums as in the FP32-row kernels (about 2^-44 relative), tiles added in FP64.
template <int PMAX>
__global__ void __launch_bounds__(kGramMaxThreads) k_gram_rows_ffd(const double* __restrict__ A, int64_t n, int r,
                                                                int lda, double* __restrict__ G, BlockSums S) {
  const int nt = blockDim.x;
  extern __shared__ __align__(16) unsigned char gram_smem2[];
  float2* tile = reinterpret_cast<float2*>(gram_smem2);  // kGramRowsFF * r
  const int np = r * (r + 1) / 2;
  int pa[PMAX], pb[PMAX];
  double acc[PMAX];
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * nt;
    if (p < np) pair_of(p, r, &pa[q], &pb[q]); else pa[q] = pb[q] = 0;
    acc[q] = 0.0;
  }
  for (int64_t row0 = (int64_t)blockIdx.x * kGramRowsFF; row0 < n; row0 += (int64_t)gridDim.x * kGramRowsFF) {
    const int rows = (int)((n - row0) < kGramRowsFF ? (n - row0) : kGramRowsFF);
    __syncthreads();
    const double* src = A + row0 * lda;
    for (int i = threadIdx.x; i < kGramRowsFF * r; i += nt) {
      const int rr = i / r, c = i - rr * r;
      tile[i] = rr < rows ? split_ff(src[(int64_t)rr * lda + c]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
      const int p = threadIdx.x + q * nt;
      if (p < np) {
        float hi = 0.f, lo = 0.f;
        for (int i = 0; i < rows; ++i) {
          const float2 a = tile[i * r + pa[q]], b = tile[i * r + pb[q]];
          ff_fma(a.x, a.y, b.x, b.y, hi, lo);
        }
        acc[q] += (double)hi + (double)lo;
      }
    }
  }
  gram_block_finish<PMAX>(acc, np, r, G, S);
}

// Leverage scores (kind 0 factors: l = ||L^{-1} P^T (S a)||^2) of FP32 rows, one
// thread per row, in float-pair arithmetic (about 2^-44 relative): F and the column
// scales are split into float pairs once per block, S a is formed as a float pair
// when the row is staged.  A kind 1 (pseudo-inverse) factor takes the FP64 loop.
// Outputs as k_lev_rows_tpr.
__global__ void __launch_bounds__(kRowThreads) k_lev_rows_ff(const float* A, int64_t n, int r, int lda,
                                                             const SmallFactor* __restrict__ f,
                                                             double* __restrict__ lev, uint64_t* __restrict__ q,
                                                             DistInfo* info, float* A_out) {
  extern __shared__ __align__(16) unsigned char ff_smem[];
  float* Fh = reinterpret_cast<float*>(ff_smem);  // r * r
  float* Fl = Fh + r * r;                         // r * r
  float* sch = Fl + r * r;                        // r
  float* scl = sch + r;                           // r
  float* lam = scl + r;                           // r
  float2* xs = reinterpret_cast<float2*>(lam + ((r + 1) & ~1));  // kRowThreads * ld (S a as float pairs)
  __shared__ int perm[kMaxRank];
  const int ld = r | 1;
  const int kind = f->kind;
  const int k = kind == 0 ? f->rank : r;
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) {
    const double v = f->F[i];
    const float h = (float)v;
    Fh[i] = h;
    Fl[i] = (float)(v - (double)h);
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double sc = f->scale[i];
    const float h = (float)sc;
    sch[i] = h;
    scl[i] = (float)(sc - (double)h);
    const double l = f->lambda[i];
    lam[i] = pos_finite(l) ? (float)(1.0 / l) : 1.f;
    perm[i] = f->perm[i];
  }
  uint64_t my_max = 0;
  uint32_t my_nz = 0;
  for (int64_t row0 = (int64_t)blockIdx.x * kRowThreads; row0 < n; row0 += (int64_t)gridDim.x * kRowThreads) {
    const int rows = (int)(n - row0 < kRowThreads ? n - row0 : kRowThreads);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
      const int rr = i / r, c = i - rr * r;
      const float x = A[(row0 + rr) * lda + c];
      const float p = __fmul_rn(x, sch[c]);
      const float rest = __fmaf_rn(x, scl[c], __fmaf_rn(x, sch[c], -p));
      const float h = __fadd_rn(p, rest);
      xs[rr * ld + c] = make_float2(h, __fsub_rn(rest, __fsub_rn(h, p)));
    }
    __syncthreads();
    if (threadIdx.x < rows) {
      const float2* b = xs + threadIdx.x * ld;
      const int64_t row = row0 + threadIdx.x;
      double l = 0.0;
      if (kind == 0) {
        float lh = 0.f, ll = 0.f;
        for (int c = 0; c < k; ++c) {
          float th = 0.f, tl = 0.f;
          for (int u = 0; u <= c; ++u) {
            const float2 bu = b[perm[u]];
            ff_fma(Fh[c * r + u], Fl[c * r + u], bu.x, bu.y, th, tl);
          }
          float s, e;
          two_sum(th, tl, s, e);
          ff_fma(s, e, s, e, lh, ll);
        }
        l = (double)lh + (double)ll;
      } else {
        for (int c = 0; c < r; ++c) {
          double t = 0.0;
          for (int u = 0; u < r; ++u)
            t = fma((double)Fh[c * r + u] + (double)Fl[c * r + u], (double)b[u].x + (double)b[u].y, t);
          l = fma((double)b[c].x + (double)b[c].y, t, l);
        }
      }
      if (lev) lev[row] = l;
      if (q) {
        double pr = l / (double)r;
        pr = clamp01(pr);
        const uint64_t qi = __double2ull_rn(pr * 4611686018427387904.0);  // 2^62
        q[row] = qi;
        my_max = qi > my_max ? qi : my_max;
        my_nz += qi > 0;
      }
    }
    if (A_out) {
      for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
        const int rr = i / r, c = i - rr * r;
        A_out[row0 * r + i] = A[(row0 + rr) * lda + c] * lam[c];
      }
    }
  }
  if (q && info) {
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t om = __shfl_xor_sync(0xffffffffu, my_max, o);
      my_max = om > my_max ? om : my_max;
      my_nz += __shfl_xor_sync(0xffffffffu, my_nz, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax((unsigned long long*)&info->maxq, (unsigned long long)my_max);
      atomicAdd((unsigned long long*)&info->nnzq, (unsigned long long)my_nz);
    }
  }
}

constexpr int kLevBatch = 5;  // row elements a thread loads before it stages them

// Leverage scores of FP64 rows (kind 0 factors), one thread per row, in float-pair
// arithmetic as k_lev_rows_ff; the rows are written out divided by lambda in FP64.
// F is staged as float pairs with each row padded by zeros to r4 (a multiple of 4)
// entries, and the block's rows S a as float pairs in pivot order with a stride ld
// = r4 + 2 (16-byte rows, and eight consecutive rows on distinct 16-byte bank groups),
// so the inner loop takes four products per two 16-byte loads of F (the same address
// in every thread) and two of the row; the zeros of F past the diagonal make the
// products past u = c vanish.  The normalised row is written while the row is staged.
__global__ void __launch_bounds__(kRowThreads) k_lev_rows_ffd(const double* A, int64_t n, int r, int lda,
                                                              const SmallFactor* __restrict__ f,
                                                              double* __restrict__ lev, uint64_t* __restrict__ q,
                                                              DistInfo* info, double* A_out) {
  extern __shared__ __align__(16) unsigned char ffd_smem[];
  const int r4 = (r + 3) & ~3, ld = r4 + 2;
  float2* Ff = reinterpret_cast<float2*>(ffd_smem);  // r x r4: F as float pairs
  float2* xs = Ff + r * r4;                           // kRowThreads x ld: S a in pivot order
  double* ilam = reinterpret_cast<double*>(xs + kRowThreads * ld);  // r: 1 / lambda_c (1 for a zero column)
  float* sch = reinterpret_cast<float*>(ilam + r);                  // r
  float* scl = sch + r;                                             // r
  __shared__ int ipos[kMaxRank];  // kind 0: position of column c in the pivot order
  const int kind = f->kind;
  const int k = kind == 0 ? f->rank : r;
  const double inv_r = 1.0 / (double)r;
  for (int i = threadIdx.x; i < r * r4; i += blockDim.x) {
    const int c = i / r4, u = i - c * r4;
    const double v = u < r ? f->F[c * r + u] : 0.0;
    const float h = (float)v;
    Ff[i] = make_float2(h, (float)(v - (double)h));
  }
  for (int i = threadIdx.x; i < kRowThreads * (r4 - r); i += blockDim.x) {  // zero padding of the rows
    const int t = i / (r4 - r);
    xs[t * ld + r + (i - t * (r4 - r))] = make_float2(0.f, 0.f);
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double sc = f->scale[i];
    const float h = (float)sc;
    sch[i] = h;
    scl[i] = (float)(sc - (double)h);
    const double l = f->lambda[i];
    ilam[i] = pos_finite(l) ? 1.0 / l : 1.0;
    ipos[i] = i;
  }
  __syncthreads();
  if (kind == 0)
    for (int i = threadIdx.x; i < r; i += blockDim.x) ipos[f->perm[i]] = i;
  // the staging walk: element i = threadIdx.x + t kRowThreads of the block's rows, its
  // (row, column) advanced by (step_r, step_c) with a carry instead of a division
  const int step_r = kRowThreads / r, step_c = kRowThreads - step_r * r;
  const int rr0 = threadIdx.x / r, c0 = threadIdx.x - rr0 * r;
  uint64_t my_max = 0;
  uint32_t my_nz = 0;
  for (int64_t row0 = (int64_t)blockIdx.x * kRowThreads; row0 < n; row0 += (int64_t)gridDim.x * kRowThreads) {
    const int rows = (int)(n - row0 < kRowThreads ? n - row0 : kRowThreads);
    __syncthreads();
    // kLevBatch loads issued ahead of their stores (A_out may be A, so the compiler
    // keeps each load behind the previous store otherwise)
    int rr = rr0, c = c0;
    const int total = rows * r;
    for (int i0 = threadIdx.x; i0 < total; i0 += kLevBatch * kRowThreads) {
      double v[kLevBatch];
      int rb[kLevBatch], cb[kLevBatch];
#pragma unroll
      for (int j = 0; j < kLevBatch; ++j) {
        rb[j] = rr;
        cb[j] = c;
        v[j] = i0 + j * kRowThreads < total ? A[(row0 + rr) * lda + c] : 0.0;
        rr += step_r;
        c += step_c;
        if (c >= r) {
          c -= r;
          ++rr;
        }
      }
#pragma unroll
      for (int j = 0; j < kLevBatch; ++j) {
        const int i = i0 + j * kRowThreads;
        if (i >= total) break;
        const int cc = cb[j];
        if (A_out) A_out[row0 * r + i] = v[j] * ilam[cc];  // same element when A_out = A (lda = r)
        const float2 x = split_ff(v[j]);
        const float p = __fmul_rn(x.x, sch[cc]);
        const float rest = __fmaf_rn(x.x, scl[cc], __fmaf_rn(x.y, sch[cc], __fmaf_rn(x.x, sch[cc], -p)));
        const float h = __fadd_rn(p, rest);
        xs[rb[j] * ld + ipos[cc]] = make_float2(h, __fsub_rn(rest, __fsub_rn(h, p)));
      }
    }
    __syncthreads();
    if (threadIdx.x < rows) {
      const float2* b = xs + threadIdx.x * ld;
      const int64_t row = row0 + threadIdx.x;
      double l = 0.0;
      if (kind == 0) {
        const float4* b4 = reinterpret_cast<const float4*>(b);
        float lh = 0.f, ll = 0.f;
        for (int c2 = 0; c2 < k; ++c2) {
          const float4* f4 = reinterpret_cast<const float4*>(Ff + c2 * r4);
          float th = 0.f, tl = 0.f;
          for (int u = 0; u <= c2; u += 4) {  // F(c2, u') = 0 for u' > c2
            const float4 f0 = f4[u >> 1], f1 = f4[(u >> 1) + 1];
            const float4 x0 = b4[u >> 1], x1 = b4[(u >> 1) + 1];
            ff_fma(f0.x, f0.y, x0.x, x0.y, th, tl);
            ff_fma(f0.z, f0.w, x0.z, x0.w, th, tl);
            ff_fma(f1.x, f1.y, x1.x, x1.y, th, tl);
            ff_fma(f1.z, f1.w, x1.z, x1.w, th, tl);
          }
          float s2, e2;
          two_sum(th, tl, s2, e2);
          ff_fma(s2, e2, s2, e2, lh, ll);
        }
        l = f2d_exact(lh) + f2d_exact(ll);
      } else {
        for (int c2 = 0; c2 < r; ++c2) {
          double t = 0.0;
          for (int u = 0; u < r; ++u) {
            const float2 fu = Ff[c2 * r4 + u];
            t = fma((double)fu.x + (double)fu.y, (double)b[u].x + (double)b[u].y, t);
          }
          l = fma((double)b[c2].x + (double)b[c2].y, t, l);
        }
      }
      if (lev) lev[row] = l;
      if (q) {
        double pr = l * inv_r;
        pr = clamp01(pr);
        const uint64_t qi = __double2ull_rn(pr * 4611686018427387904.0);  // 2^62
        q[row] = qi;
        my_max = qi > my_max ? qi : my_max;
        my_nz += qi > 0;
      }
    }
  }
  if (q && info) {
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t om = __shfl_xor_sync(0xffffffffu, my_max, o);
      my_max = om > my_max ? om : my_max;
      my_nz += __shfl_xor_sync(0xffffffffu, my_nz, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax((unsigned long long*)&info->maxq, (unsigned long long)my_max);
      atomicAdd((unsigned long long*)&info->nnzq, (unsigned long long)my_nz);
    }
  }
}

}  // namespace

template <class FT>
int gram_rows(const FT* A, int64_t n, int r, double* G, const BlockSums& S, cudaStream_t st, int lda, int* status) {
  if (lda <= 0) lda = r;
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (!S.ticket || S.max_blocks < 1) return CPA_ERR_ARG;
  const int np = r * (r + 1) / 2;
  const unsigned one_pair = (unsigned)((np + 31) / 32 * 32);  // threads of the one-pair-per-thread layout
  if (n <= 0) {
    CPA_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double) * r * r, st));
    return CPA_OK;
  }
  // grid from the sizes only (not the SM count): the block-ordered sum then gives the
  // same G on every run
  auto grid_for = [&](int64_t rows_per_block) {
    int64_t g = ceil_div(n, rows_per_block);
    const int64_t cap = S.max_blocks < kSumMaxBlocks ? S.max_blocks : kSumMaxBlocks;
    return (unsigned)(g < cap ? g : cap);
  };
  if constexpr (sizeof(FT) == 4) {
    if (n >= kManyRows && status && lev_tensor_cores() && tc_rows_ok(reinterpret_cast<const float*>(A), r, lda)) {
      if (r <= kGramStreamMaxRank && !gram_tensor_cores())
        return gram_rows_stream(reinterpret_cast<const float*>(A), n, r, lda, G, S, status, st);
      return gram_rows_tc(reinterpret_cast<const float*>(A), n, r, lda, G, S, status, st);
    }
    const unsigned grid = grid_for(kGramRowsFF);
    const size_t smem = sizeof(float) * kGramRowsFF * r;
    if (np <= kGramMaxThreads)
      k_gram_rows_ff<1><<<grid, one_pair, smem, st>>>(A, n, r, lda, G, S);
    else if (np <= 4 * kGramThreads)
      k_gram_rows_ff<4><<<grid, kGramThreads, smem, st>>>(A, n, r, lda, G, S);
    else
      k_gram_rows_ff<9><<<grid, kGramThreads, smem, st>>>(A, n, r, lda, G, S);
    CPA_LAUNCH_CHECK();
    return CPA_OK;
  }
  if (n >= kManyRows) {  // FP64 rows of a many-row factor: float pairs on the FP32 pipe
    if (status && r <= kGramStreamFP64MaxRank && ((uintptr_t)A & 15u) == 0 && gram_stream_fp64())
      return gram_rows_stream(reinterpret_cast<const double*>(A), n, r, lda, G, S, status, st);
    const unsigned grid = grid_for(kGramRowsFF);
    const size_t smem = sizeof(float2) * kGramRowsFF * r;
    if (np <= kGramMaxThreads)
      k_gram_rows_ffd<1><<<grid, one_pair, smem, st>>>(reinterpret_cast<const double*>(A), n, r, lda, G, S);
    else if (np <= 4 * kGramThreads)
      k_gram_rows_ffd<4><<<grid, kGramThreads, smem, st>>>(reinterpret_cast<const double*>(A), n, r, lda, G, S);
    else
      k_gram_rows_ffd<9><<<grid, kGramThreads, smem, st>>>(reinterpret_cast<const double*>(A), n, r, lda, G, S);
    CPA_LAUNCH_CHECK();
    return CPA_OK;
  }
  const unsigned grid = grid_for(kGramRows);
  const size_t smem = sizeof(double) * kGramRows * r;
  if (np <= kGramMaxThreads)
    k_gram_rows<FT, 1><<<grid, one_pair, smem, st>>>(A, n, r, lda, G, S);
  else if (np <= 4 * kGramThreads)
    k_gram_rows<FT, 4><<<grid, kGramThreads, smem, st>>>(A, n, r, lda, G, S);
  else
    k_gram_rows<FT, 9><<<grid, kGramThreads, smem, st>>>(A, n, r, lda, G, S);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}
template int gram_rows<double>(const double*, int64_t, int, double*, const BlockSums&, cudaStream_t, int, int*);
template int gram_rows<float>(const float*, int64_t, int, double*, const BlockSums&, cudaStream_t, int, int*);

int factor_spd(const double* G, int r, int normalize, int pivot, double rel_tol, SmallFactor* out,
               int* warn, int warn_bit, cudaStream_t st, DistInfo* zero_info) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  const size_t smem = sizeof(double) * (3 * r * r + 7 * r);
  static std::atomic<unsigned long long> attr{0};
  CPA_CUDA_TRY(set_attr_once(attr, [] {
    return cudaFuncSetAttribute(k_factor_spd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * (3 * kMaxRank * kMaxRank + 7 * kMaxRank)));
  }));
  k_factor_spd<<<1, kFactorThreads, smem, st>>>(G, r, normalize, pivot, rel_tol, out, warn, warn_bit,
                                                zero_info);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

template <class FT>
int lev_rows(const FT* A, int64_t n, int r, const SmallFactor* f, double* lev, uint64_t* q,
             DistInfo* info, FT* A_out, cudaStream_t st, int dist, int lda, int* status) {
  if (lda <= 0) lda = r;
  if (lda != r && A_out == A) return CPA_ERR_ARG;  // in place only at stride r
  if (dist != CPA_DIST_LEVERAGE && dist != CPA_DIST_UNIFORM && dist != CPA_DIST_LENGTH_SQUARED)
    return CPA_ERR_ARG;
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (n <= 0) return CPA_OK;
  if constexpr (sizeof(FT) == 4) {
    if (n >= kManyRows && dist == CPA_DIST_LEVERAGE && status && lev_tensor_cores() &&
        tc_rows_ok(reinterpret_cast<const float*>(A), r, lda))
      return lev_rows_tc(reinterpret_cast<const float*>(A), n, r, lda, f, lev, q, info,
                         reinterpret_cast<float*>(A_out), status, st);
  }
  if (n >= kManyRows && dist == CPA_DIST_LEVERAGE) {  // float pairs on the FP32 pipe
    if constexpr (sizeof(FT) == 4) {
      auto bytes = [](int rr) {
        return sizeof(float) * ((size_t)2 * rr * rr + 3 * rr + 1) + sizeof(float2) * (size_t)kRowThreads * (rr | 1) +
               16;
      };
      static std::atomic<unsigned long long> attr{0};
      CPA_CUDA_TRY(set_attr_once(attr, [&] {
        return cudaFuncSetAttribute(k_lev_rows_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes(kMaxRank));
      }));
      const unsigned grid = grid_cap(ceil_div(n, kRowThreads), 8);
      k_lev_rows_ff<<<grid, kRowThreads, bytes(r), st>>>(reinterpret_cast<const float*>(A), n, r, lda, f, lev, q,
                                                         info, reinterpret_cast<float*>(A_out));
    } else {
      auto bytes = [](int rr) {  // F (r x r4 pairs), rows (kRowThreads x (r4 + 2) pairs), 1 / lambda, scales
        const size_t r4 = (size_t)((rr + 3) & ~3);
        return sizeof(float2) * ((size_t)rr * r4 + (size_t)kRowThreads * (r4 + 2)) + sizeof(double) * rr +
               sizeof(float) * 2 * rr;
      };
      static std::atomic<unsigned long long> attr{0};
      CPA_CUDA_TRY(set_attr_once(attr, [&] {
        return cudaFuncSetAttribute(k_lev_rows_ffd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bytes(kMaxRank));
      }));
      const unsigned grid = grid_cap(ceil_div(n, kRowThreads), 8);
      k_lev_rows_ffd<<<grid, kRowThreads, bytes(r), st>>>(reinterpret_cast<const double*>(A), n, r, lda, f, lev, q,
                                                          info, reinterpret_cast<double*>(A_out));
    }
    CPA_LAUNCH_CHECK();
    return CPA_OK;
  }
  if (n >= kManyRows) {
    auto bytes = [](int rr) {
      return sizeof(double) * ((size_t)rr * rr + rr) + sizeof(FT) * (size_t)((rr + 1) & ~1) +
             sizeof(double) * (size_t)kRowThreads * (rr | 1);
    };
    const size_t smem = bytes(r);
    static std::atomic<unsigned long long> attr{0};
    CPA_CUDA_TRY(set_attr_once(attr, [&] {
      return cudaFuncSetAttribute(k_lev_rows_tpr<FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)bytes(kMaxRank));
    }));
    const unsigned grid = grid_cap(ceil_div(n, kRowThreads), 8);
    k_lev_rows_tpr<FT><<<grid, kRowThreads, smem, st>>>(A, n, r, lda, f, lev, q, info, A_out, dist);
  } else {
    const size_t smem = sizeof(double) * ((size_t)r * r + r) + sizeof(FT) * r;
    const unsigned grid = grid_cap(ceil_div(n, kRowThreads / 32), 16);
    k_lev_rows<FT><<<grid, kRowThreads, smem, st>>>(A, n, r, lda, f, lev, q, info, A_out, dist);
  }
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}
template int lev_rows<double>(const double*, int64_t, int, const SmallFactor*, double*, uint64_t*,
                              DistInfo*, double*, cudaStream_t, int, int, int*);
template int lev_rows<float>(const float*, int64_t, int, const SmallFactor*, double*, uint64_t*,
                             DistInfo*, float*, cudaStream_t, int, int, int*);

template <class FT>
int solve_rows(const FT* M, int64_t n, int r, const SmallFactor* f, FT* A, cudaStream_t st,
               double* zero_gram) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (n <= 0) return CPA_OK;
  if constexpr (sizeof(FT) == 4) {
    if (n >= kManyRows) {
      auto bytes = [](int rr) {
        return sizeof(float) * ((size_t)rr * ((rr + 3) & ~3) + (size_t)kRowThreads * (rr | 1));
      };
      static std::atomic<unsigned long long> attr{0};
      CPA_CUDA_TRY(set_attr_once(attr, [&] {
        cudaError_t e = cudaFuncSetAttribute(k_solve_rows_f32<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes(kMaxRank));
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_solve_rows_f32<kMaxRank>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bytes(kMaxRank));
      }));
      const unsigned grid = grid_cap(ceil_div(n, kRowThreads), 8);
      if (r <= 32)
        k_solve_rows_f32<32><<<grid, kRowThreads, bytes(r), st>>>(M, n, r, f, A, zero_gram);
      else
        k_solve_rows_f32<kMaxRank><<<grid, kRowThreads, bytes(r), st>>>(M, n, r, f, A, zero_gram);
      CPA_LAUNCH_CHECK();
      return CPA_OK;
    }
  }
  const size_t smem = sizeof(FT) * (size_t)r * r;
  const unsigned grid = grid_cap(ceil_div(n * r, kRowThreads), 16);
  k_solve_rows<FT><<<grid, kRowThreads, smem, st>>>(M, n, r, f, A, zero_gram);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}
template int solve_rows<double>(const double*, int64_t, int, const SmallFactor*, double*, cudaStream_t,
                                double*);
template int solve_rows<float>(const float*, int64_t, int, const SmallFactor*, float*, cudaStream_t,
                               double*);

template <class FT>
int scale_columns(FT* A, int64_t n, int r, const double* lambda, cudaStream_t st) {
  if (n <= 0) return CPA_OK;
  k_scale_columns<FT><<<grid_cap(ceil_div(n * r, 256), 8), 256, 0, st>>>(A, n, r, lambda);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}
template int scale_columns<double>(double*, int64_t, int, const double*, cudaStream_t);
template int scale_columns<float>(float*, int64_t, int, const double*, cudaStream_t);

int cdf_from_q(uint64_t* q, uint64_t* C, int64_t n, DistInfo* info, double* p, void* scan_scratch,
               cudaStream_t st) {
  ScanExtras ex;
  ex.ratio = p;
  CPA_TRY(scan_u64<uint64_t>(q, C, DevCount{nullptr, n}, true, &info->T, scan_scratch, st, ex));
  return CPA_OK;
}

}  // namespace cpa
