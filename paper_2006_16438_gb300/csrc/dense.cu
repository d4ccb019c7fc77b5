// Dense kernels of the per-mode update (see dense.cuh).
//
// The factor-matrix Gram A^T A and the solve are FP64 on CUDA cores: r is at most
// 64, so they are skinny (n x r times r x n) and bound by FP64 issue on this part.
// The r x r factorisation runs in one thread block.
#include "dense.cuh"

namespace cpa {

namespace {

constexpr int kGramRows = 32;   // rows staged per tile
constexpr int kGramThreads = 256;

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

// Per-thread partial sums over a tile are in FT; tile partials are added in FP64.
template <class FT, int PMAX>
__global__ void __launch_bounds__(kGramThreads) k_gram_rows(const FT* __restrict__ A,
                                                            int64_t n, int r,
                                                            double* __restrict__ G) {
  extern __shared__ __align__(16) unsigned char gram_smem[];
  FT* tile = reinterpret_cast<FT*>(gram_smem);  // kGramRows * r
  const int np = r * (r + 1) / 2;
  int pa[PMAX], pb[PMAX];
  double acc[PMAX];
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * kGramThreads;
    if (p < np) pair_of(p, r, &pa[q], &pb[q]); else pa[q] = pb[q] = 0;
    acc[q] = 0.0;
  }
  for (int64_t row0 = (int64_t)blockIdx.x * kGramRows; row0 < n;
       row0 += (int64_t)gridDim.x * kGramRows) {
    const int rows = (int)((n - row0) < kGramRows ? (n - row0) : kGramRows);
    __syncthreads();
    const FT* src = A + row0 * r;
    for (int i = threadIdx.x; i < kGramRows * r; i += kGramThreads)
      tile[i] = i < rows * r ? src[i] : FT(0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
      const int p = threadIdx.x + q * kGramThreads;
      if (p < np) {
        FT s = FT(0);
        for (int i = 0; i < rows; ++i) s = fma(tile[i * r + pa[q]], tile[i * r + pb[q]], s);
        acc[q] += (double)s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < PMAX; ++q) {
    const int p = threadIdx.x + q * kGramThreads;
    if (p < np) {
      atomicAdd(&G[pa[q] * r + pb[q]], acc[q]);
      if (pa[q] != pb[q]) atomicAdd(&G[pb[q] * r + pa[q]], acc[q]);
    }
  }
}

// ---- r x r factorisation in one block -------------------------------------
constexpr int kFactorThreads = 256;

// Cyclic Jacobi eigendecomposition of the symmetric matrix in `a` (r x r,
// overwritten by its eigenvalues on the diagonal), eigenvectors in the columns of
// `v`.  Serial: run by one thread (it is the rare fallback path).
__device__ void jacobi_eigen_serial(double* a, double* v, int r) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) v[i * r + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < r; ++i) {
      diag += a[i * r + i] * a[i * r + i];
      for (int j = i + 1; j < r; ++j) off += 2.0 * a[i * r + j] * a[i * r + j];
    }
    if (off == 0.0 || off <= 1e-30 * (off + diag)) break;
    for (int p = 0; p < r - 1; ++p) {
      for (int q = p + 1; q < r; ++q) {
        const double apq = a[p * r + q];
        if (apq == 0.0) continue;
        const double app = a[p * r + p], aqq = a[q * r + q];
        // rotation angle that zeroes a_pq (Rutishauser's formulas)
        const double zeta = (aqq - app) / (2.0 * apq);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = rsqrt(1.0 + t * t);
        const double s = t * c;
        for (int k = 0; k < r; ++k) {
          const double akp = a[k * r + p], akq = a[k * r + q];
          a[k * r + p] = c * akp - s * akq;
          a[k * r + q] = s * akp + c * akq;
        }
        for (int k = 0; k < r; ++k) {
          const double apk = a[p * r + k], aqk = a[q * r + k];
          a[p * r + k] = c * apk - s * aqk;
          a[q * r + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < r; ++k) {
          const double vkp = v[k * r + p], vkq = v[k * r + q];
          v[k * r + p] = c * vkp - s * vkq;
          v[k * r + q] = s * vkp + c * vkq;
        }
      }
    }
  }
}

// 1/sqrt(d) for d > 0 in FP64: FP32 seed, then two Newton steps
// y <- y (3 - d y^2) / 2 in FP64 (about 24 -> 48 -> 96 correct bits).  GB300 FP64
// division and square root cost hundreds of cycles each, so the factorisation keeps
// them off its serial chain.
__device__ __forceinline__ double rsqrt_newton(double d) {
  double y = (double)rsqrtf((float)d);
  if (!(y > 0.0) || isinf(y)) y = rsqrt(d);  // outside float range: library rsqrt
  y = y * (1.5 - 0.5 * d * y * y);
  y = y * (1.5 - 0.5 * d * y * y);
  return y;
}

// Factor one r x r PSD matrix in one block (see SmallFactor):
//  * right-looking Cholesky of S = diag(scale) G diag(scale), with diagonal pivoting
//    (pivot = 1, stops at the numerical rank) or without (pivot = 0);
//  * the inverse X = L^{-1} of the rank x rank factor by right-looking substitution;
//  * pivot = 1: F = X (kind 0); pivot = 0: F = X^T X = S^{-1} (kind 2);
//  * pivot = 0 and a pivot <= rel_tol * max diag: F = pinv(S) by Jacobi (kind 1).
__global__ void __launch_bounds__(kFactorThreads) k_factor_spd(const double* __restrict__ G,
                                                               int r, int normalize, int pivot,
                                                               double rel_tol,
                                                               SmallFactor* __restrict__ out,
                                                               int* warn, int warn_bit,
                                                               DistInfo* zero_info) {
  extern __shared__ double sm[];
  double* S = sm;              // r x r working matrix (L in its lower triangle)
  double* X = sm + r * r;      // r x r inverse / eigenvectors
  double* scale = X + r * r;   // r
  double* y = scale + r;       // r: 1 / L_jj
  __shared__ int ok, rank, piv;
  __shared__ int perm[kMaxRank];
  __shared__ double dmax, dcur;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (zero_info && tid == 0) {
    zero_info->maxq = 0;
    zero_info->nnzq = 0;
  }
  for (int c = tid; c < r; c += nt) {
    const double g = G[c * r + c];
    const double lam = g > 0.0 ? sqrt(g) : 0.0;
    out->lambda[c] = lam;
    scale[c] = normalize ? (lam > 0.0 ? 1.0 / lam : 0.0) : 1.0;
    out->scale[c] = scale[c];
    perm[c] = c;
  }
  __syncthreads();
  for (int i = tid; i < r * r; i += nt) {
    const int a = i / r, b = i - a * r;
    const double v = G[i] * scale[a] * scale[b];
    S[i] = v;
    out->gram[i] = v;
    X[i] = 0.0;
  }
  __syncthreads();
  if (tid < 32) {  // largest diagonal entry
    double m = 0.0;
    for (int c = tid; c < r; c += 32) m = fmax(m, S[c * r + c]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (tid == 0) {
      dmax = m;
      ok = 1;
      rank = r;
    }
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (tid < 32) {  // pivot choice and 1/sqrt of the pivot
      int p = j;
      if (pivot) {
        double best = -1.0;
        for (int i = j + tid; i < r; i += 32) {
          const double d = S[i * r + i];
          if (d > best) {
            best = d;
            p = i;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int op = __shfl_xor_sync(0xffffffffu, p, o);
          if (ob > best || (ob == best && op < p)) {
            best = ob;
            p = op;
          }
        }
      }
      const double d = S[p * r + p];
      if (tid == 0) {
        piv = p;
        dcur = d;
        if (!(d > rel_tol * dmax)) {
          if (pivot) rank = j; else ok = 0;
        } else {
          y[j] = rsqrt_newton(d);
        }
      }
    }
    __syncthreads();
    if (rank == j || !ok) break;
    const int p = piv;
    if (p != j) {  // symmetric swap of rows/columns j and p (includes computed L entries)
      for (int c = tid; c < r; c += nt) {
        const double t = S[j * r + c];
        S[j * r + c] = S[p * r + c];
        S[p * r + c] = t;
      }
      if (tid == 0) {
        const int t = perm[j];
        perm[j] = perm[p];
        perm[p] = t;
      }
      __syncthreads();
      for (int c = tid; c < r; c += nt) {
        const double t = S[c * r + j];
        S[c * r + j] = S[c * r + p];
        S[c * r + p] = t;
      }
      __syncthreads();
    }
    const double yj = y[j];
    for (int i = j + 1 + tid; i < r; i += nt) S[i * r + j] *= yj;  // column j of L
    if (tid == 0) S[j * r + j] = dcur * yj;                        // L_jj = sqrt(d)
    __syncthreads();
    // trailing update of the lower triangle: S_ic -= L_ij L_cj for j < c <= i
    const int m = r - j - 1;
    const int npairs = m * (m + 1) / 2;
    for (int q = tid; q < npairs; q += nt) {
      // q -> (i, c) with c <= i, both offset by j + 1
      int ii = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
      while (ii * (ii + 1) / 2 > q) --ii;
      const int cc = q - ii * (ii + 1) / 2;
      const int i = ii + j + 1, c = cc + j + 1;
      const double v = S[i * r + c] - S[i * r + j] * S[c * r + j];
      S[i * r + c] = v;
      if (c != i) S[c * r + i] = v;  // keep the trailing block symmetric for swaps
    }
    __syncthreads();
  }
  if (!ok) {  // plain Cholesky failed: pseudo-inverse from the eigendecomposition
    for (int i = tid; i < r * r; i += nt) {
      const int a = i / r, b = i - a * r;
      S[i] = G[i] * scale[a] * scale[b];
    }
    __syncthreads();
    if (tid == 0) {
      jacobi_eigen_serial(S, X, r);
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
  const int k = rank;
  // X = L^{-1} (k x k), right-looking: row i of X is final once the rows above are
  // folded in; y holds 1/L_ii.  X starts at zero and accumulates -sum L_iu X_uc.
  for (int i = 0; i < k; ++i) {
    const double yi = y[i];
    for (int c = tid; c <= i; c += nt) X[i * r + c] = ((i == c ? 1.0 : 0.0) - X[i * r + c]) * yi;
    __syncthreads();
    const int rows = k - i - 1, cols = i + 1;
    for (int q = tid; q < rows * cols; q += nt) {
      const int i2 = i + 1 + q / cols, c = q % cols;
      X[i2 * r + c] += S[i2 * r + i] * X[i * r + c];
    }
    __syncthreads();
  }
  if (pivot) {
    for (int i = tid; i < r * r; i += nt) out->F[i] = X[i];
    for (int c = tid; c < r; c += nt) out->perm[c] = perm[c];
    if (tid == 0) {
      out->kind = 0;
      out->rank = k;
      if (k < r) atomicOr(warn, warn_bit);
    }
    return;
  }
  // F = X^T X = (L L^T)^{-1}
  for (int i = tid; i < r * r; i += nt) {
    const int a = i / r, b = i - a * r;
    const int u0 = a > b ? a : b;
    double s2 = 0.0;
    for (int u = u0; u < r; ++u) s2 = fma(X[u * r + a], X[u * r + b], s2);
    out->F[i] = s2;
  }
  for (int c = tid; c < r; c += nt) out->perm[c] = c;
  if (tid == 0) {
    out->kind = 2;
    out->rank = r;
  }
}

// ---- per-row kernels -------------------------------------------------------
constexpr int kRowThreads = 256;
constexpr int64_t kManyRows = 1 << 16;  // from here on one thread per row

// Leverage of row a_i (one warp per row, lane c owns coordinate c and c + 32):
// kind 0: y = X P^T (S a), l = ||y||^2 over the rank's coordinates;
// kind 1: l = (S a)^T F (S a).
template <class FT>
__global__ void __launch_bounds__(kRowThreads) k_lev_rows(const FT* A, int64_t n, int r,
                                                          const SmallFactor* __restrict__ f,
                                                          double* __restrict__ lev,
                                                          uint64_t* __restrict__ q,
                                                          DistInfo* info, FT* A_out) {
  extern __shared__ __align__(16) unsigned char lev_smem[];
  FT* F = reinterpret_cast<FT*>(lev_smem);  // r * r
  FT* sc = F + r * r;                       // r
  FT* lam = sc + r;                         // r
  __shared__ int perm[kMaxRank];
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) F[i] = (FT)f->F[i];
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    sc[i] = (FT)f->scale[i];
    lam[i] = (FT)f->lambda[i];
    perm[i] = f->perm[i];
  }
  __syncthreads();
  const int kind = f->kind;
  const int k = kind == 0 ? f->rank : r;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kRowThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kRowThreads) >> 5;
  uint64_t my_max = 0;
  uint32_t my_nz = 0;
  for (int64_t row = gw; row < n; row += nwarps) {
    const FT* a = A + row * r;
    FT part = FT(0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      if (c < k) {
        FT t = FT(0);
        if (kind == 0) {
          for (int u = 0; u <= c; ++u) {
            const int pu = perm[u];
            t = fma(F[c * r + u], a[pu] * sc[pu], t);
          }
          part = fma(t, t, part);
        } else {
          for (int u = 0; u < r; ++u) t = fma(F[c * r + u], a[u] * sc[u], t);
          part = fma(a[c] * sc[c], t, part);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) {
      if (lev) lev[row] = (double)part;
      if (q) {
        double p = (double)part / (double)r;
        p = p > 0.0 ? (p < 1.0 ? p : 1.0) : 0.0;
        const uint64_t qi = __double2ull_rn(p * 4611686018427387904.0);  // 2^62
        q[row] = qi;
        my_max = qi > my_max ? qi : my_max;
        my_nz += qi > 0;
      }
    }
    if (A_out) {
      __syncwarp();
      for (int c = lane; c < r; c += 32) {
        const FT v = a[c];
        A_out[row * r + c] = lam[c] > FT(0) ? v / lam[c] : v;
      }
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
__global__ void __launch_bounds__(kRowThreads) k_lev_rows_tpr(const FT* A, int64_t n, int r,
                                                              const SmallFactor* __restrict__ f,
                                                              double* __restrict__ lev,
                                                              uint64_t* __restrict__ q,
                                                              DistInfo* info, FT* A_out) {
  extern __shared__ __align__(16) unsigned char tpr_smem[];
  FT* F = reinterpret_cast<FT*>(tpr_smem);  // r * r
  FT* sc = F + r * r;                       // r
  FT* lam = sc + r;                         // r
  FT* xs = lam + r;                         // kRowThreads * (r + 1)
  __shared__ int perm[kMaxRank];
  const int ld = r + 1;
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) F[i] = (FT)f->F[i];
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    sc[i] = (FT)f->scale[i];
    lam[i] = (FT)f->lambda[i];
    perm[i] = f->perm[i];
  }
  const int kind = f->kind;
  const int k = kind == 0 ? f->rank : r;
  uint64_t my_max = 0;
  uint32_t my_nz = 0;
  for (int64_t row0 = (int64_t)blockIdx.x * kRowThreads; row0 < n; row0 += (int64_t)gridDim.x * kRowThreads) {
    const int rows = (int)(n - row0 < kRowThreads ? n - row0 : kRowThreads);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
      const int rr = i / r, c = i - rr * r;
      xs[rr * ld + c] = A[row0 * r + i] * sc[c];
    }
    __syncthreads();
    if (threadIdx.x < rows) {
      const FT* x = xs + threadIdx.x * ld;
      FT l = FT(0);
      for (int c = 0; c < k; ++c) {
        FT t = FT(0);
        if (kind == 0) {
          for (int u = 0; u <= c; ++u) t = fma(F[c * r + u], x[perm[u]], t);
          l = fma(t, t, l);
        } else {
          for (int u = 0; u < r; ++u) t = fma(F[c * r + u], x[u], t);
          l = fma(x[c], t, l);
        }
      }
      const int64_t row = row0 + threadIdx.x;
      if (lev) lev[row] = (double)l;
      if (q) {
        double p = (double)l / (double)r;
        p = p > 0.0 ? (p < 1.0 ? p : 1.0) : 0.0;
        const uint64_t qi = __double2ull_rn(p * 4611686018427387904.0);  // 2^62
        q[row] = qi;
        my_max = qi > my_max ? qi : my_max;
        my_nz += qi > 0;
      }
    }
    if (A_out) {
      for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
        const int c = i % r;
        const FT v = A[row0 * r + i];
        A_out[row0 * r + i] = lam[c] > FT(0) ? v / lam[c] : v;
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
int gram_rows(const FT* A, int64_t n, int r, double* G, cudaStream_t st) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (n <= 0) return CPA_OK;
  const int np = r * (r + 1) / 2;
  const unsigned grid = grid_cap(ceil_div(n, kGramRows), 4);
  const size_t smem = sizeof(FT) * kGramRows * r;
  if (np <= kGramThreads)
    k_gram_rows<FT, 1><<<grid, kGramThreads, smem, st>>>(A, n, r, G);
  else if (np <= 4 * kGramThreads)
    k_gram_rows<FT, 4><<<grid, kGramThreads, smem, st>>>(A, n, r, G);
  else
    k_gram_rows<FT, 9><<<grid, kGramThreads, smem, st>>>(A, n, r, G);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}
template int gram_rows<double>(const double*, int64_t, int, double*, cudaStream_t);
template int gram_rows<float>(const float*, int64_t, int, double*, cudaStream_t);

int factor_spd(const double* G, int r, int normalize, int pivot, double rel_tol, SmallFactor* out,
               int* warn, int warn_bit, cudaStream_t st, DistInfo* zero_info) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  const size_t smem = sizeof(double) * (2 * r * r + 2 * r);
  static bool attr_done = false;
  if (!attr_done) {
    CPA_CUDA_TRY(cudaFuncSetAttribute(k_factor_spd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(double) * (2 * kMaxRank * kMaxRank + 2 * kMaxRank))));
    attr_done = true;
  }
  k_factor_spd<<<1, kFactorThreads, smem, st>>>(G, r, normalize, pivot, rel_tol, out, warn, warn_bit,
                                                zero_info);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

template <class FT>
int lev_rows(const FT* A, int64_t n, int r, const SmallFactor* f, double* lev, uint64_t* q,
             DistInfo* info, FT* A_out, cudaStream_t st) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (n <= 0) return CPA_OK;
  if (n >= kManyRows) {
    const size_t smem = sizeof(FT) * ((size_t)r * r + 2 * r + (size_t)kRowThreads * (r + 1));
    static bool attr = false;
    if (!attr) {
      CPA_CUDA_TRY(cudaFuncSetAttribute(k_lev_rows_tpr<FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(sizeof(FT) * (kMaxRank * kMaxRank + 2 * kMaxRank +
                                                            kRowThreads * (kMaxRank + 1)))));
      attr = true;
    }
    const unsigned grid = grid_cap(ceil_div(n, kRowThreads), 8);
    k_lev_rows_tpr<FT><<<grid, kRowThreads, smem, st>>>(A, n, r, f, lev, q, info, A_out);
  } else {
    const size_t smem = sizeof(FT) * ((size_t)r * r + 2 * r);
    const unsigned grid = grid_cap(ceil_div(n, kRowThreads / 32), 16);
    k_lev_rows<FT><<<grid, kRowThreads, smem, st>>>(A, n, r, f, lev, q, info, A_out);
  }
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}
template int lev_rows<double>(const double*, int64_t, int, const SmallFactor*, double*, uint64_t*,
                              DistInfo*, double*, cudaStream_t);
template int lev_rows<float>(const float*, int64_t, int, const SmallFactor*, double*, uint64_t*,
                             DistInfo*, float*, cudaStream_t);

template <class FT>
int solve_rows(const FT* M, int64_t n, int r, const SmallFactor* f, FT* A, cudaStream_t st,
               double* zero_gram) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (n <= 0) return CPA_OK;
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
