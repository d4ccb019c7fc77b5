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

template <int PMAX>
__global__ void __launch_bounds__(kGramThreads) k_gram_rows(const double* __restrict__ A,
                                                            int64_t n, int r,
                                                            double* __restrict__ G) {
  extern __shared__ double tile[];  // kGramRows * r
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
    const double* src = A + row0 * r;
    for (int i = threadIdx.x; i < kGramRows * r; i += kGramThreads)
      tile[i] = i < rows * r ? src[i] : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
      const int p = threadIdx.x + q * kGramThreads;
      if (p < np) {
        double s = 0.0;
        for (int i = 0; i < rows; ++i) s = fma(tile[i * r + pa[q]], tile[i * r + pb[q]], s);
        acc[q] += s;
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
constexpr int kFactorThreads = 128;

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

__global__ void __launch_bounds__(kFactorThreads) k_factor_spd(const double* __restrict__ G,
                                                               int r, int normalize, int pivot,
                                                               double rel_tol,
                                                               SmallFactor* __restrict__ out,
                                                               int* warn, int warn_bit) {
  extern __shared__ double sm[];
  double* S = sm;              // r x r scaled matrix
  double* L = sm + r * r;      // r x r factor / eigenvectors
  double* scale = L + r * r;   // r
  double* dd = scale + r;      // r remaining diagonal (pivoted path)
  __shared__ int ok, rank, piv;
  __shared__ int perm[kMaxRank];
  __shared__ double dmax;
  const int tid = threadIdx.x;
  for (int c = tid; c < r; c += blockDim.x) {
    const double g = G[c * r + c];
    const double lam = g > 0.0 ? sqrt(g) : 0.0;
    out->lambda[c] = lam;
    scale[c] = normalize ? (lam > 0.0 ? 1.0 / lam : 0.0) : 1.0;
    out->scale[c] = scale[c];
    perm[c] = c;
  }
  __syncthreads();
  for (int i = tid; i < r * r; i += blockDim.x) {
    const int a = i / r, b = i % r;
    const double v = G[i] * scale[a] * scale[b];
    S[i] = v;
    out->gram[i] = v;
    L[i] = 0.0;
  }
  if (tid == 0) {
    ok = 1;
    rank = r;
    double m = 0.0;
    for (int c = 0; c < r; ++c) m = fmax(m, G[c * r + c] * scale[c] * scale[c]);
    dmax = m;
  }
  __syncthreads();
  if (pivot) {
    // Cholesky with diagonal pivoting of P^T S P; stops at the numerical rank.
    for (int j = 0; j < r; ++j) {
      for (int i = j + tid; i < r; i += blockDim.x) {
        double d = S[perm[i] * r + perm[i]];
        for (int c = 0; c < j; ++c) d -= L[i * r + c] * L[i * r + c];
        dd[i] = d;
      }
      __syncthreads();
      if (tid == 0) {
        int p = j;
        for (int i = j + 1; i < r; ++i)
          if (dd[i] > dd[p]) p = i;
        if (!(dd[p] > rel_tol * dmax)) {
          rank = j;
        } else {
          if (p != j) {
            const int t = perm[j];
            perm[j] = perm[p];
            perm[p] = t;
            for (int c = 0; c < j; ++c) {
              const double x = L[j * r + c];
              L[j * r + c] = L[p * r + c];
              L[p * r + c] = x;
            }
          }
          L[j * r + j] = sqrt(dd[p]);
        }
        piv = p;
      }
      __syncthreads();
      if (rank == j) break;
      const double ljj = L[j * r + j];
      for (int i = j + 1 + tid; i < r; i += blockDim.x) {
        double t = S[perm[i] * r + perm[j]];
        for (int c = 0; c < j; ++c) t -= L[i * r + c] * L[j * r + c];
        L[i * r + j] = t / ljj;
      }
      __syncthreads();
    }
    for (int i = tid; i < r * r; i += blockDim.x) out->F[i] = L[i];
    for (int c = tid; c < r; c += blockDim.x) out->perm[c] = perm[c];
    if (tid == 0) {
      out->kind = 0;
      out->rank = rank;
      if (rank < r) atomicOr(warn, warn_bit);
    }
    (void)piv;
    return;
  }
  // plain Cholesky, column by column (rows below the pivot in parallel)
  for (int j = 0; j < r; ++j) {
    if (tid == 0) {
      double s = S[j * r + j];
      for (int c = 0; c < j; ++c) s -= L[j * r + c] * L[j * r + c];
      if (!(s > rel_tol * dmax)) ok = 0;
      else L[j * r + j] = sqrt(s);
    }
    __syncthreads();
    if (!ok) break;
    const double ljj = L[j * r + j];
    for (int i = j + 1 + tid; i < r; i += blockDim.x) {
      double t = S[i * r + j];
      for (int c = 0; c < j; ++c) t -= L[i * r + c] * L[j * r + c];
      L[i * r + j] = t / ljj;
    }
    __syncthreads();
  }
  if (ok) {
    for (int i = tid; i < r * r; i += blockDim.x) out->F[i] = L[i];
    for (int c = tid; c < r; c += blockDim.x) out->perm[c] = c;
    if (tid == 0) {
      out->kind = 0;
      out->rank = r;
    }
    return;
  }
  // pseudo-inverse from the eigendecomposition of S
  if (tid == 0) {
    jacobi_eigen_serial(S, L, r);
    double emax = 0.0;
    for (int c = 0; c < r; ++c) emax = fmax(emax, fabs(S[c * r + c]));
    for (int c = 0; c < r; ++c) {
      const double ev = S[c * r + c];
      scale[c] = ev > rel_tol * emax ? 1.0 / ev : 0.0;  // reuse as inverse eigenvalues
    }
    out->kind = 1;
    out->rank = r;
    atomicOr(warn, warn_bit);
  }
  __syncthreads();
  for (int i = tid; i < r * r; i += blockDim.x) {
    const int a = i / r, b = i % r;
    double s = 0.0;
    for (int c = 0; c < r; ++c) s += L[a * r + c] * scale[c] * L[b * r + c];
    out->F[i] = s;
  }
}

// ---- per-row kernels: a block stages kRowThreads rows in shared memory ------
// (coalesced), each thread then works on its own row with runtime loops over r;
// the row stride r + 1 keeps the per-thread accesses spread over the banks.
constexpr int kRowThreads = 128;

__global__ void __launch_bounds__(kRowThreads) k_lev_rows(const double* A, int64_t n, int r,
                                                          const SmallFactor* __restrict__ f,
                                                          double* __restrict__ lev,
                                                          uint64_t* __restrict__ q,
                                                          DistInfo* info, double* A_out) {
  extern __shared__ double smem[];
  double* F = smem;                       // r * r
  double* sc = F + r * r;                 // r
  double* lam = sc + r;                   // r
  double* xs = lam + r;                   // kRowThreads * (r + 1)
  __shared__ int perm[kMaxRank];
  const int ld = r + 1;
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) F[i] = f->F[i];
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    sc[i] = f->scale[i];
    lam[i] = f->lambda[i];
    perm[i] = f->perm[i];
  }
  const int kind = f->kind;
  const int rank = f->rank;
  uint64_t my_max = 0;
  uint32_t my_nz = 0;
  for (int64_t row0 = (int64_t)blockIdx.x * kRowThreads; row0 < n;
       row0 += (int64_t)gridDim.x * kRowThreads) {
    const int rows = (int)(n - row0 < kRowThreads ? n - row0 : kRowThreads);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
      const int rr = i / r, c = i - rr * r;
      xs[rr * ld + c] = A[row0 * r + i];
    }
    __syncthreads();
    if (threadIdx.x < rows) {
      double* x = xs + threadIdx.x * ld;
      double l = 0.0;
      if (kind == 0) {
        // y = L^{-1} P^T (S a) over the first `rank` pivots, l = ||y||^2; y is kept
        // in the spare column block of the thread's own row (x[r] is free)
        for (int c = 0; c < r; ++c) x[c] *= sc[c];
        double* y = xs + (size_t)kRowThreads * ld + threadIdx.x * ld;
        for (int c = 0; c < rank; ++c) {
          double t = x[perm[c]];
          for (int u = 0; u < c; ++u) t -= F[c * r + u] * y[u];
          t = t / F[c * r + c];
          y[c] = t;
          l += t * t;
        }
      } else {
        for (int c = 0; c < r; ++c) x[c] *= sc[c];
        for (int c = 0; c < r; ++c) {
          double t = 0.0;
          for (int u = 0; u < r; ++u) t += F[c * r + u] * x[u];
          l += x[c] * t;
        }
      }
      const int64_t row = row0 + threadIdx.x;
      if (lev) lev[row] = l;
      if (q) {
        double p = l / (double)r;
        p = p > 0.0 ? (p < 1.0 ? p : 1.0) : 0.0;
        const uint64_t qi = __double2ull_rn(p * 4611686018427387904.0);  // 2^62
        q[row] = qi;
        my_max = qi > my_max ? qi : my_max;
        my_nz += qi > 0;
      }
    }
    if (A_out) {  // normalised copy from the original rows (coalesced)
      __syncthreads();
      for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
        const int c = i % r;
        const double v = A[row0 * r + i];
        A_out[row0 * r + i] = lam[c] > 0.0 ? v / lam[c] : v;
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

__global__ void __launch_bounds__(kRowThreads) k_solve_rows(const double* __restrict__ M,
                                                            int64_t n, int r,
                                                            const SmallFactor* __restrict__ f,
                                                            double* __restrict__ A) {
  extern __shared__ double smem[];
  double* F = smem;         // r * r
  double* xs = F + r * r;   // kRowThreads * (r + 1)
  const int ld = r + 1;
  for (int i = threadIdx.x; i < r * r; i += blockDim.x) F[i] = f->F[i];
  const int kind = f->kind;
  for (int64_t row0 = (int64_t)blockIdx.x * kRowThreads; row0 < n;
       row0 += (int64_t)gridDim.x * kRowThreads) {
    const int rows = (int)(n - row0 < kRowThreads ? n - row0 : kRowThreads);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
      const int rr = i / r, c = i - rr * r;
      xs[rr * ld + c] = M[row0 * r + i];
    }
    __syncthreads();
    if (threadIdx.x < rows) {
      double* x = xs + threadIdx.x * ld;
      if (kind == 0) {
        // G = L L^T: L y = m, then L^T x = y (in place)
        for (int c = 0; c < r; ++c) {
          double t = x[c];
          for (int u = 0; u < c; ++u) t -= F[c * r + u] * x[u];
          x[c] = t / F[c * r + c];
        }
        for (int c = r - 1; c >= 0; --c) {
          double t = x[c];
          for (int u = c + 1; u < r; ++u) t -= F[u * r + c] * x[u];
          x[c] = t / F[c * r + c];
        }
      }
    }
    __syncthreads();
    if (kind == 0) {
      for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
        const int rr = i / r, c = i - rr * r;
        A[row0 * r + i] = xs[rr * ld + c];
      }
    } else {
      // pinv path: A = M F straight from global memory (rare fallback)
      for (int i = threadIdx.x; i < rows * r; i += kRowThreads) {
        const int rr = i / r, b = i - rr * r;
        double t = 0.0;
        for (int a = 0; a < r; ++a) t += M[(row0 + rr) * r + a] * F[a * r + b];
        A[row0 * r + i] = t;
      }
    }
  }
}

__global__ void k_scale_columns(double* A, int64_t n, int r, const double* __restrict__ lambda) {
  const int64_t total = n * r;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double l = lambda[i % r];
    if (l > 0.0) A[i] = A[i] / l;
  }
}

}  // namespace

int gram_rows(const double* A, int64_t n, int r, double* G, cudaStream_t st) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (n <= 0) return CPA_OK;
  const int np = r * (r + 1) / 2;
  const unsigned grid = grid_cap(ceil_div(n, kGramRows), 4);
  const size_t smem = sizeof(double) * kGramRows * r;
  if (np <= kGramThreads)
    k_gram_rows<1><<<grid, kGramThreads, smem, st>>>(A, n, r, G);
  else if (np <= 4 * kGramThreads)
    k_gram_rows<4><<<grid, kGramThreads, smem, st>>>(A, n, r, G);
  else
    k_gram_rows<9><<<grid, kGramThreads, smem, st>>>(A, n, r, G);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

int factor_spd(const double* G, int r, int normalize, int pivot, double rel_tol, SmallFactor* out,
               int* warn, int warn_bit, cudaStream_t st) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  const size_t smem = sizeof(double) * (2 * r * r + 2 * r);
  static bool attr_done = false;
  if (!attr_done) {
    CPA_CUDA_TRY(cudaFuncSetAttribute(k_factor_spd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(double) * (2 * kMaxRank * kMaxRank + 2 * kMaxRank))));
    attr_done = true;
  }
  k_factor_spd<<<1, kFactorThreads, smem, st>>>(G, r, normalize, pivot, rel_tol, out, warn, warn_bit);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

int lev_rows(const double* A, int64_t n, int r, const SmallFactor* f, double* lev, uint64_t* q,
             DistInfo* info, double* A_out, cudaStream_t st) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (n <= 0) return CPA_OK;
  const size_t smem = sizeof(double) * ((size_t)r * r + 2 * r + 2 * (size_t)kRowThreads * (r + 1));
  static bool attr = false;
  if (!attr) {
    CPA_CUDA_TRY(cudaFuncSetAttribute(k_lev_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(double) * (kMaxRank * kMaxRank + 2 * kMaxRank +
                                                              2 * kRowThreads * (kMaxRank + 1)))));
    attr = true;
  }
  const unsigned grid = grid_cap(ceil_div(n, kRowThreads), 8);
  k_lev_rows<<<grid, kRowThreads, smem, st>>>(A, n, r, f, lev, q, info, A_out);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

int solve_rows(const double* M, int64_t n, int r, const SmallFactor* f, double* A,
               cudaStream_t st) {
  if (r < 1 || r > kMaxRank) return CPA_ERR_ARG;
  if (n <= 0) return CPA_OK;
  const size_t smem = sizeof(double) * ((size_t)r * r + (size_t)kRowThreads * (r + 1));
  static bool attr = false;
  if (!attr) {
    CPA_CUDA_TRY(cudaFuncSetAttribute(k_solve_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(double) * (kMaxRank * kMaxRank +
                                                              kRowThreads * (kMaxRank + 1)))));
    attr = true;
  }
  const unsigned grid = grid_cap(ceil_div(n, kRowThreads), 8);
  k_solve_rows<<<grid, kRowThreads, smem, st>>>(M, n, r, f, A);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

int scale_columns(double* A, int64_t n, int r, const double* lambda, cudaStream_t st) {
  if (n <= 0) return CPA_OK;
  k_scale_columns<<<grid_cap(ceil_div(n * r, 256), 8), 256, 0, st>>>(A, n, r, lambda);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

int cdf_from_q(uint64_t* q, uint64_t* C, int64_t n, DistInfo* info, void* scan_scratch,
               cudaStream_t st) {
  CPA_TRY(scan_u64<uint64_t>(q, C, DevCount{nullptr, n}, true, &info->T, scan_scratch, st));
  return CPA_OK;
}

}  // namespace cpa
