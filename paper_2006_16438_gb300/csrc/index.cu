// Per-mode fibre index (Section 5.3, "precompute and store the linearized indices
// ... for every mode"), built once per tensor on the GPU.
//
// For mode k every nonzero gets its packed other-mode multi-index (a 64-bit key
// whose order is the order of the linear index of Eq. 2.2).  Nonzeros are sorted by
// (key, i_k) with the device radix sort, so fibre X(:, key) is one contiguous run of
// (i_k, value) pairs with i_k ascending.  Distinct keys and run starts form the
// fibre table; a directory over the top key bits narrows each probe to a few keys.
#include "cpa_internal.cuh"

namespace cpa {

namespace {

__global__ void k_check_range(const int32_t* __restrict__ idx, int64_t nnz, int64_t dim,
                              int* status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = idx[e];
    if (v < 0 || (int64_t)v >= dim) set_status(status, CPA_ERR_COO_RANGE);
  }
}

struct CooPtrs {
  const int32_t* idx[kMaxOrder];
};

// sort key = (packed other-mode key << ik_bits) | i_k when it fits in 64 bits
// (compose = 1), else the packed key alone (compose = 0, i_k sorted in a first pass).
template <class P>
__global__ void k_make_keys(CooPtrs coo, KeyLayout L, int k, int ik_bits, int compose,
                            int64_t nnz, uint64_t* __restrict__ keys, P* __restrict__ perm) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = 0;
    for (int t = 0; t < L.d; ++t) key |= (uint64_t)(uint32_t)coo.idx[L.mode[t]][e] << L.off[t];
    const uint64_t ik = (uint64_t)(uint32_t)coo.idx[k][e];
    keys[e] = compose ? ((key << ik_bits) | ik) : ik;
    perm[e] = (P)e;
  }
}

// Second-pass keys when (key, i_k) does not fit one word: packed key of the nonzero
// at perm[j] (perm already sorted by i_k).
template <class P>
__global__ void k_packed_keys_by_perm(CooPtrs coo, KeyLayout L, int64_t nnz,
                                      const P* __restrict__ perm, uint64_t* __restrict__ keys) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = (int64_t)perm[j];
    uint64_t key = 0;
    for (int t = 0; t < L.d; ++t) key |= (uint64_t)(uint32_t)coo.idx[L.mode[t]][e] << L.off[t];
    keys[j] = key;
  }
}

// Gather the permuted (i_k, value) stream; flag fibre starts; detect duplicates.
template <class P, class VT>
__global__ void k_gather_stream(const int32_t* __restrict__ idx_k, const VT* __restrict__ vals,
                                const P* __restrict__ perm, const uint64_t* __restrict__ skeys,
                                int compose, int ik_bits, int64_t nnz,
                                int32_t* __restrict__ ik_out, VT* __restrict__ val_out,
                                uint32_t* __restrict__ start_flag, int* status) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = (int64_t)perm[j];
    const int32_t ik = idx_k[e];
    ik_out[j] = ik;
    val_out[j] = vals[e];
    const uint64_t key = compose ? (skeys[j] >> ik_bits) : skeys[j];
    uint32_t start = 1;
    if (j > 0) {
      const uint64_t prev = compose ? (skeys[j - 1] >> ik_bits) : skeys[j - 1];
      if (prev == key) {
        start = 0;
        const int32_t ikp = idx_k[(int64_t)perm[j - 1]];
        if (ikp == ik) set_status(status, CPA_ERR_COO_DUP);
      }
    }
    start_flag[j] = start;
  }
}

__global__ void k_write_fibres(const uint64_t* __restrict__ skeys, int compose, int ik_bits,
                               const uint32_t* __restrict__ start_flag,
                               const uint64_t* __restrict__ fid, int64_t nnz,
                               uint64_t* __restrict__ keys, uint64_t* __restrict__ off) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz;
       j += (int64_t)gridDim.x * blockDim.x) {
    if (start_flag[j]) {
      const uint64_t f = fid[j];
      keys[f] = compose ? (skeys[j] >> ik_bits) : skeys[j];
      off[f] = (uint64_t)j;
    }
  }
}

__global__ void k_finish_off(uint64_t* off, int64_t nfib, int64_t nnz) { off[nfib] = (uint64_t)nnz; }

constexpr size_t kFibreHashBudget = size_t(4) << 30;  // bytes of fibre hash table per mode

// dir[b] = first fibre whose key has top bits >= b, for b in [0, 2^dbits]: one
// bisection of the sorted keys per bucket (balanced whatever the key skew).
__global__ void k_directory(const uint64_t* __restrict__ keys, int64_t nfib, int dshift,
                            int64_t nbuckets, uint64_t* __restrict__ dir) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= nbuckets;
       b += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = nfib;
    if (b < nbuckets) {
      while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if ((int64_t)(keys[mid] >> dshift) < b) lo = mid + 1; else hi = mid;
      }
    } else {
      lo = nfib;
    }
    dir[b] = (uint64_t)lo;
  }
}

// Fibre f into the open-addressing table (slots preset to kNoFibre; keys distinct).
__global__ void k_hash_fibres(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ off,
                              int64_t nfib, int hbits, ulonglong2* __restrict__ htab) {
  const uint64_t mask = (1ull << hbits) - 1ull;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nfib;
       f += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys[f], lo = off[f], len = off[f + 1] - lo;
    uint64_t h = fibre_slot(key, hbits);
    for (;;) {  // at most nfib < 2^hbits occupied slots: a free one exists
      const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(&htab[h].x),
                                                (unsigned long long)kNoFibre, (unsigned long long)key);
      if (prev == kNoFibre) {
        htab[h].y = (lo << 24) | len;
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

template <class VT>
__global__ void k_sumsq(const VT* __restrict__ v, int64_t n, double* out) {
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)v[e];
    s += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

inline unsigned grid_for(int64_t n, int threads = 256) {
  int64_t g = ceil_div(n > 0 ? n : 1, threads);
  const int64_t cap = (int64_t)num_sms() * 32;
  return (unsigned)(g < cap ? g : cap);
}

template <class P, class VT>
int build_modes(cpa_index* X, const CooPtrs& coo, const VT* vals, int* d_status,
                cudaStream_t st) {
  const int64_t nnz = X->nnz;
  const int D = X->order;
  // temporaries: two key buffers, two permutation buffers, flags, fibre ids, scratch
  const size_t sort_ws = sort_workspace(nnz);
  const size_t scan_ws = scan_workspace(nnz);
  Arena a;
  for (int pass = 0; pass < 2; ++pass) {
    a.used = 0;
    uint64_t* k0 = a.take<uint64_t>(nnz);
    uint64_t* k1 = a.take<uint64_t>(nnz);
    P* p0 = a.take<P>(nnz);
    P* p1 = a.take<P>(nnz);
    uint32_t* flag = a.take<uint32_t>(nnz);
    uint64_t* fid = a.take<uint64_t>(nnz);
    char* sws = a.take<char>(sort_ws > scan_ws ? sort_ws : scan_ws);
    uint64_t* d_count = a.take<uint64_t>(2);
    if (pass == 0) {
      CPA_CUDA_TRY(cudaMallocAsync((void**)&a.base, a.used, st));
      a.cap = a.used;
      continue;
    }
    const unsigned grid = grid_for(nnz);
    for (int k = 0; k < D; ++k) {
      auto& M = X->mode[k];
      make_layout(D, X->dims, k, &M.L);
      const int ik_bits = ceil_log2(X->dims[k]);
      const int compose = (M.L.total_bits + ik_bits) <= 64;
      int in_alt = 0;
      k_make_keys<P><<<grid, 256, 0, st>>>(coo, M.L, k, ik_bits, compose, nnz, k0, p0);
      CPA_LAUNCH_CHECK();
      uint64_t* sk;
      P* sp;
      if (compose) {
        CPA_TRY(radix_sort<P>(k0, k1, p0, p1, DevCount{nullptr, nnz}, 0,
                              M.L.total_bits + ik_bits, sws, st, &in_alt));
        sk = in_alt ? k1 : k0;
        sp = in_alt ? p1 : p0;
      } else {
        // stable sort by i_k, then stable sort by the packed key
        CPA_TRY(radix_sort<P>(k0, k1, p0, p1, DevCount{nullptr, nnz}, 0, ik_bits, sws, st,
                              &in_alt));
        uint64_t* kk = in_alt ? k1 : k0;
        uint64_t* ko = in_alt ? k0 : k1;
        P* pp = in_alt ? p1 : p0;
        P* po = in_alt ? p0 : p1;
        k_packed_keys_by_perm<P><<<grid, 256, 0, st>>>(coo, M.L, nnz, pp, kk);
        CPA_LAUNCH_CHECK();
        CPA_TRY(radix_sort<P>(kk, ko, pp, po, DevCount{nullptr, nnz}, 0, M.L.total_bits, sws,
                              st, &in_alt));
        sk = in_alt ? ko : kk;
        sp = in_alt ? po : pp;
      }
      // permuted stream
      CPA_CUDA_TRY(cudaMallocAsync(&M.ik, sizeof(int32_t) * (nnz > 0 ? nnz : 1), st));
      X->allocations.push_back(M.ik);
      CPA_CUDA_TRY(cudaMallocAsync(&M.val, sizeof(VT) * (nnz > 0 ? nnz : 1), st));
      X->allocations.push_back(M.val);
      if (nnz > 0) {
        k_gather_stream<P, VT><<<grid, 256, 0, st>>>(coo.idx[k], vals, sp, sk, compose, ik_bits,
                                                     nnz, M.ik, reinterpret_cast<VT*>(M.val),
                                                     flag, d_status);
        CPA_LAUNCH_CHECK();
      }
      CPA_TRY(scan_u64<uint32_t>(flag, fid, DevCount{nullptr, nnz}, false, d_count, sws, st));
      uint64_t nfib = 0;
      int status = 0;
      CPA_CUDA_TRY(cudaMemcpyAsync(&nfib, d_count, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
      CPA_CUDA_TRY(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
      CPA_CUDA_TRY(cudaStreamSynchronize(st));
      if (status < 0) {
        cudaFreeAsync(a.base, st);
        return status;
      }
      M.nfib = (int64_t)nfib;
      CPA_CUDA_TRY(cudaMallocAsync(&M.keys, sizeof(uint64_t) * (nfib > 0 ? nfib : 1), st));
      X->allocations.push_back(M.keys);
      CPA_CUDA_TRY(cudaMallocAsync(&M.off, sizeof(uint64_t) * (nfib + 1), st));
      X->allocations.push_back(M.off);
      if (nnz > 0) {
        k_write_fibres<<<grid, 256, 0, st>>>(sk, compose, ik_bits, flag, fid, nnz, M.keys, M.off);
        CPA_LAUNCH_CHECK();
      }
      k_finish_off<<<1, 1, 0, st>>>(M.off, M.nfib, nnz);
      // directory: about four fibres per bucket
      int dbits = ceil_log2(M.nfib > 0 ? M.nfib : 1) - 2;
      if (dbits < 0) dbits = 0;
      if (dbits > M.L.total_bits) dbits = M.L.total_bits;
      if (dbits > 30) dbits = 30;
      M.dbits = dbits;
      M.dshift = M.L.total_bits - dbits;
      const int64_t nb = 1ll << dbits;
      CPA_CUDA_TRY(cudaMallocAsync(&M.dir, sizeof(uint64_t) * (nb + 1), st));
      X->allocations.push_back(M.dir);
      k_directory<<<grid_for(nb + 1), 256, 0, st>>>(M.keys, M.nfib, M.dshift, nb, M.dir);
      CPA_LAUNCH_CHECK();
      // hash table of the fibres (load <= 1/2) when it fits the budget and the record
      // encoding (fibre start < 2^40, length < 2^24)
      int hb = 4;
      while ((1ll << hb) < 2 * M.nfib) ++hb;
      const size_t hbytes = sizeof(ulonglong2) * ((size_t)1 << hb);
      size_t longest = 0;  // host bound: a fibre is at most dims[k] long
      longest = (size_t)X->dims[k];
      if (M.nfib > 0 && hbytes <= kFibreHashBudget && longest < (1ull << 24) && nnz < (1ll << 40)) {
        M.hbits = hb;
        CPA_CUDA_TRY(cudaMallocAsync(&M.htab, hbytes, st));
        X->allocations.push_back(M.htab);
        CPA_CUDA_TRY(cudaMemsetAsync(M.htab, 0xff, hbytes, st));
        k_hash_fibres<<<grid_for(M.nfib), 256, 0, st>>>(M.keys, M.off, M.nfib, hb, M.htab);
        CPA_LAUNCH_CHECK();
      }
    }
  }
  CPA_CUDA_TRY(cudaFreeAsync(a.base, st));
  return CPA_OK;
}

}  // namespace

int index_build(const cpa_coo* coo, cudaStream_t st, cpa_index** out) {
  if (!coo || !out || coo->order < 2 || coo->order > kMaxOrder || coo->nnz < 0 || !coo->dims ||
      !coo->idx || (coo->nnz > 0 && !coo->vals))
    return CPA_ERR_ARG;
  if (coo->val_dtype != CPA_F32 && coo->val_dtype != CPA_F64) return CPA_ERR_ARG;
  if (coo->nnz >= (1ll << 40)) return CPA_ERR_UNSUPPORTED;
  const int D = coo->order;
  for (int m = 0; m < D; ++m)
    if (coo->dims[m] < 1 || coo->dims[m] > 0x7fffffffll) return CPA_ERR_ARG;
  for (int k = 0; k < D; ++k) {
    KeyLayout L;
    if (!make_layout(D, coo->dims, k, &L)) return CPA_ERR_UNSUPPORTED;
  }
  cpa_index* X = new (std::nothrow) cpa_index();
  if (!X) return CPA_ERR_OOM;
  X->order = D;
  X->nnz = coo->nnz;
  X->val_dtype = coo->val_dtype;
  for (int m = 0; m < D; ++m) X->dims[m] = coo->dims[m];
  const int64_t nnz = coo->nnz;
  const size_t vb = coo->val_dtype == CPA_F32 ? 4 : 8;
  // device copy of the COO if it lives on the host
  std::vector<void*> tmp;
  CooPtrs cp{};
  const void* dvals = coo->vals;
  int rc = CPA_OK;
  int* d_status = nullptr;
  double* d_norm = nullptr;
  auto fail = [&](int code) {
    for (void* p : tmp) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    index_free(X);
    return code;
  };
  if (cudaMallocAsync((void**)&d_status, sizeof(int) + sizeof(double) * 2, st) != cudaSuccess)
    return fail(CPA_ERR_OOM);
  tmp.push_back(d_status);
  d_norm = reinterpret_cast<double*>(reinterpret_cast<char*>(d_status) + 8);
  if (cudaMemsetAsync(d_status, 0, sizeof(int) + sizeof(double) * 2, st) != cudaSuccess)
    return fail(CPA_ERR_CUDA);
  for (int m = 0; m < D; ++m) {
    if (coo->on_device) {
      cp.idx[m] = coo->idx[m];
    } else {
      void* p = nullptr;
      if (cudaMallocAsync(&p, sizeof(int32_t) * (nnz > 0 ? nnz : 1), st) != cudaSuccess)
        return fail(CPA_ERR_OOM);
      tmp.push_back(p);
      if (nnz > 0 &&
          cudaMemcpyAsync(p, coo->idx[m], sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st) !=
              cudaSuccess)
        return fail(CPA_ERR_CUDA);
      cp.idx[m] = reinterpret_cast<const int32_t*>(p);
    }
  }
  if (!coo->on_device) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, vb * (nnz > 0 ? nnz : 1), st) != cudaSuccess) return fail(CPA_ERR_OOM);
    tmp.push_back(p);
    if (nnz > 0 && cudaMemcpyAsync(p, coo->vals, vb * nnz, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(CPA_ERR_CUDA);
    dvals = p;
  }
  if (nnz > 0) {
    for (int m = 0; m < D; ++m) k_check_range<<<grid_for(nnz), 256, 0, st>>>(cp.idx[m], nnz,
                                                                              X->dims[m], d_status);
    if (coo->val_dtype == CPA_F32)
      k_sumsq<float><<<grid_for(nnz), 256, 0, st>>>(reinterpret_cast<const float*>(dvals), nnz, d_norm);
    else
      k_sumsq<double><<<grid_for(nnz), 256, 0, st>>>(reinterpret_cast<const double*>(dvals), nnz, d_norm);
    if (cudaGetLastError() != cudaSuccess) return fail(CPA_ERR_CUDA);
    int status = 0;
    if (cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&X->norm_x2, d_norm, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(CPA_ERR_CUDA);
    if (status < 0) return fail(status);
  }
  if (nnz < (1ll << 32)) {
    if (coo->val_dtype == CPA_F32)
      rc = build_modes<uint32_t, float>(X, cp, reinterpret_cast<const float*>(dvals), d_status, st);
    else
      rc = build_modes<uint32_t, double>(X, cp, reinterpret_cast<const double*>(dvals), d_status, st);
  } else {
    if (coo->val_dtype == CPA_F32)
      rc = build_modes<uint64_t, float>(X, cp, reinterpret_cast<const float*>(dvals), d_status, st);
    else
      rc = build_modes<uint64_t, double>(X, cp, reinterpret_cast<const double*>(dvals), d_status, st);
  }
  if (rc < 0) return fail(rc);
  for (void* p : tmp) cudaFreeAsync(p, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    index_free(X);
    return CPA_ERR_CUDA;
  }
  *out = X;
  return CPA_OK;
}

void index_free(cpa_index* X) {
  if (!X) return;
  cudaDeviceSynchronize();
  if (X->plan) {
    plan_free(X->plan);
    X->plan = nullptr;
  }
  for (void* p : X->allocations) cudaFree(p);
  delete X;
}

namespace {
template <class VT>
__global__ void k_export(KeyLayout L, const uint64_t* __restrict__ pk, int64_t nfib,
                         uint64_t* __restrict__ keys_out) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nfib;
       f += (int64_t)gridDim.x * blockDim.x)
    keys_out[f] = L.linear(pk[f]);
}
}  // namespace

int index_export(const cpa_index* X, int k, uint64_t* keys, uint64_t* off, int32_t* ik, void* val,
                 cudaStream_t st) {
  if (!X || k < 0 || k >= X->order) return CPA_ERR_ARG;
  const auto& M = X->mode[k];
  if (keys && M.nfib > 0) {
    k_export<double><<<grid_for(M.nfib), 256, 0, st>>>(M.L, M.keys, M.nfib, keys);
    CPA_LAUNCH_CHECK();
  }
  if (off)
    CPA_CUDA_TRY(cudaMemcpyAsync(off, M.off, sizeof(uint64_t) * (M.nfib + 1),
                                 cudaMemcpyDeviceToDevice, st));
  if (ik && X->nnz > 0)
    CPA_CUDA_TRY(cudaMemcpyAsync(ik, M.ik, sizeof(int32_t) * X->nnz, cudaMemcpyDeviceToDevice, st));
  if (val && X->nnz > 0)
    CPA_CUDA_TRY(cudaMemcpyAsync(val, M.val, (X->val_dtype == CPA_F32 ? 4 : 8) * X->nnz,
                                 cudaMemcpyDeviceToDevice, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  return CPA_OK;
}


// ---------------------------------------------------------------------------
// Range-finder initialisation (App. F): one warp per drawn fibre; lane c adds
// x * omega(j, c) (and column c + 32) into row i of A for every nonzero (i, x) of the
// fibre (FP64 atomics: rows are shared between fibres).
// ---------------------------------------------------------------------------
namespace {

template <class VT>
__global__ void __launch_bounds__(256) k_rrf(FibreIndex<VT> Xk, int k, int64_t s_init, uint64_t seed,
                                             const double* __restrict__ omega, int r, double* __restrict__ A) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < s_init; j += nw) {
    uint64_t w0 = (uint64_t)j, w1 = 0, w2 = kDomainRrf | (uint64_t)(uint32_t)k, w3 = 0;
    Philox4x64::block(w0, w1, w2, w3, seed, 0ull);
    const int64_t f = (int64_t)__umul64hi(w0, (uint64_t)Xk.nfib);
    const double o0 = lane < r ? omega[j * r + lane] : 0.0;
    const double o1 = lane + 32 < r ? omega[j * r + lane + 32] : 0.0;
    for (uint64_t e = Xk.off[f]; e < Xk.off[f + 1]; ++e) {
      const double x = (double)Xk.val[e];
      double* row = A + (int64_t)Xk.ik[e] * r;
      if (lane < r) atomicAdd(row + lane, x * o0);
      if (lane + 32 < r) atomicAdd(row + lane + 32, x * o1);
    }
  }
}

}  // namespace

int rrf_enqueue(const cpa_index* X, int k, int64_t s_init, uint64_t seed, const double* omega, int r,
                double* A, cudaStream_t st) {
  if (k < 0 || k >= X->order || s_init < 1 || r < 1 || r > kMaxRank || X->nnz < 1 || !omega || !A)
    return CPA_ERR_ARG;
  CPA_CUDA_TRY(cudaMemsetAsync(A, 0, sizeof(double) * (size_t)X->dims[k] * r, st));
  const int64_t want = ceil_div(s_init, 8);
  const unsigned grid = (unsigned)(want < (int64_t)num_sms() * 16 ? want : (int64_t)num_sms() * 16);
  if (X->val_dtype == CPA_F32)
    k_rrf<float><<<grid, 256, 0, st>>>(fibre_view<float>(X, k), k, s_init, seed, omega, r, A);
  else
    k_rrf<double><<<grid, 256, 0, st>>>(fibre_view<double>(X, k), k, s_init, seed, omega, r, A);
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

}  // namespace cpa
