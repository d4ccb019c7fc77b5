// Per-mode fibre index (Section 5.3: the linear indices of every mode are computed
// once and kept), built once per tensor on the GPU.
//
// For mode k every nonzero gets its packed other-mode multi-index (a 64-bit key
// whose order is the order of the linear index of Eq. 2.2).  Nonzeros are sorted by
// (key, i_k) with the device radix sort, so fibre X(:, key) is one contiguous run of
// (i_k, value) pairs with i_k ascending.  Distinct keys and run starts form the
// fibre table; a directory over the top key bits narrows each probe to a few keys.
#include <algorithm>

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

// Nonzeros of one build segment: position e of the COO for local j (pos == null: the
// segment is the whole COO and e = j).
__device__ __forceinline__ int64_t seg_src(const uint64_t* pos, int64_t j) {
  return pos ? (int64_t)pos[j] : j;
}

__device__ __forceinline__ uint64_t packed_key(const CooPtrs& coo, const KeyLayout& L, int64_t e) {
  uint64_t key = 0;
  for (int t = 0; t < L.d; ++t) key |= (uint64_t)(uint32_t)coo.idx[L.mode[t]][e] << L.off[t];
  return key;
}

// Histogram of the top other-mode coordinate (bins of 2^shift values).
__global__ void k_top_hist(const int32_t* __restrict__ itop, int64_t nnz, int shift,
                           unsigned long long* __restrict__ hist) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[(uint32_t)itop[e] >> shift], 1ull);
}

// Positions of the nonzeros whose top coordinate lies in [lo, hi), in any order (the
// sort that follows orders them by their unique (key, i_k)).  A block takes tiles of
// kSelItems coalesced items per thread, counts the tile's matches with warp ballots,
// and reserves the tile's output range with one atomic (one per warp contended on the
// single counter at billions of nonzeros).
constexpr int kSelItems = 8;
__global__ void __launch_bounds__(256) k_seg_select(const int32_t* __restrict__ itop, int64_t nnz, int64_t lo,
                                                    int64_t hi, uint64_t* __restrict__ pos, int64_t cap,
                                                    unsigned long long* __restrict__ cnt, int* status) {
  __shared__ unsigned wsum[32];
  __shared__ unsigned long long bbase;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t tile = (int64_t)blockDim.x * kSelItems;
  for (int64_t t0 = (int64_t)blockIdx.x * tile; t0 < nnz; t0 += (int64_t)gridDim.x * tile) {  // block-uniform
    unsigned bal[kSelItems];
    unsigned mine = 0;
#pragma unroll
    for (int i = 0; i < kSelItems; ++i) {
      const int64_t e = t0 + (int64_t)i * blockDim.x + threadIdx.x;
      bool m = false;
      if (e < nnz) {
        const int64_t v = itop[e];
        m = v >= lo && v < hi;
      }
      bal[i] = __ballot_sync(0xffffffffu, m);
      mine += __popc(bal[i]);
    }
    if (lane == 0) wsum[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned run = 0;
      for (int w = 0; w < nwarps; ++w) {
        const unsigned c = wsum[w];
        wsum[w] = run;
        run += c;
      }
      bbase = run ? atomicAdd(cnt, (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    unsigned long long at = bbase + wsum[warp];
#pragma unroll
    for (int i = 0; i < kSelItems; ++i) {
      if ((bal[i] >> lane) & 1u) {
        const unsigned long long p = at + __popc(bal[i] & ((1u << lane) - 1u));
        if ((int64_t)p < cap) pos[p] = (uint64_t)(t0 + (int64_t)i * blockDim.x + threadIdx.x);
        else set_status(status, CPA_ERR_CUDA);
      }
      at += __popc(bal[i]);
    }
    __syncthreads();  // wsum and bbase are rewritten for the next tile
  }
}

// Packed other-mode keys of a segment (fibre count pass).
__global__ void k_seg_packed_keys(CooPtrs coo, KeyLayout L, const uint64_t* __restrict__ pos, int64_t n,
                                  uint64_t* __restrict__ keys) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    keys[j] = packed_key(coo, L, seg_src(pos, j));
}

// Distinct keys of a sorted array (one atomic per warp).
__global__ void k_count_distinct(const uint64_t* __restrict__ sk, int64_t n, unsigned long long* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < n; j0 += stride) {
    const int64_t j = j0 + lane;
    const bool s = j < n && (j == 0 || sk[j] != sk[j - 1]);
    const unsigned bal = __ballot_sync(0xffffffffu, s);
    if (lane == 0 && bal) atomicAdd(cnt, (unsigned long long)__popc(bal));
  }
}

// sort key = (packed other-mode key << ik_bits) | i_k when it fits in 64 bits
// (compose = 1), else i_k alone (compose = 0: a first pass by i_k, then a stable pass
// by the packed key).  perm[j] = j, the local number of the nonzero.
__global__ void k_make_keys(CooPtrs coo, KeyLayout L, int k, int ik_bits, int compose,
                            const uint64_t* __restrict__ pos, int64_t n, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ perm) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = seg_src(pos, j);
    const uint64_t ik = (uint64_t)(uint32_t)coo.idx[k][e];
    keys[j] = compose ? ((packed_key(coo, L, e) << ik_bits) | ik) : ik;
    perm[j] = (uint32_t)j;
  }
}

// Second-pass keys when (key, i_k) does not fit one word: packed key of the nonzero
// at perm[j] (perm already sorted by i_k).
__global__ void k_packed_keys_by_perm(CooPtrs coo, KeyLayout L, const uint64_t* __restrict__ pos, int64_t n,
                                      const uint32_t* __restrict__ perm, uint64_t* __restrict__ keys) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    keys[j] = packed_key(coo, L, seg_src(pos, (int64_t)perm[j]));
}

// 16-bit value codes (FP32 tensors with at most 65,536 distinct values): a hash set of
// the values' bit patterns, 2^17 slots (load <= 1/2), and the code of each slot.
constexpr int kCodeSetBits = 17;
constexpr int kMaxCodes = 65536;
constexpr uint32_t kNoValue = 0xffffffffu;  // a NaN pattern; a tensor holding it is not coded

struct ValueCoder {
  const uint32_t* set = nullptr;  // null: values stored as they are
  const uint16_t* codes = nullptr;
};

__device__ __forceinline__ uint32_t code_slot(uint32_t bits) {
  return (bits * 0x9E3779B1u) >> (32 - kCodeSetBits);
}

// Insert every value's bit pattern; *full is set (and the insertions stop) once more
// than kMaxCodes distinct patterns are seen, or on the pattern kNoValue.
__global__ void k_value_set(const float* __restrict__ v, int64_t n, uint32_t* set, unsigned* count, int* full) {
  const uint32_t mask = (1u << kCodeSetBits) - 1u;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (*(volatile int*)full) return;
    const uint32_t b = __float_as_uint(v[e]);
    if (b == kNoValue) {
      atomicExch(full, 1);
      return;
    }
    uint32_t h = code_slot(b);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      const uint32_t cur = __ldcg(set + h);
      if (cur == b) break;
      if (cur == kNoValue) {
        const uint32_t prev = atomicCAS(set + h, kNoValue, b);
        if (prev == kNoValue) {
          if (atomicAdd(count, 1u) >= (unsigned)kMaxCodes) atomicExch(full, 1);
          break;
        }
        if (prev == b) break;
      }
      h = (h + 1) & mask;
    }
  }
}

template <class VT, class OT>
__device__ __forceinline__ OT store_value(const ValueCoder& vc, VT x, int* status) {
  if constexpr (std::is_same<OT, uint16_t>::value) {
    const uint32_t b = __float_as_uint((float)x);
    const uint32_t mask = (1u << kCodeSetBits) - 1u;
    uint32_t h = code_slot(b);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      if (vc.set[h] == b) return vc.codes[h];
      h = (h + 1) & mask;
    }
    set_status(status, CPA_ERR_CUDA);  // every value was inserted: not reached
    return 0;
  } else {
    return x;
  }
}

// Gather the permuted (i_k, value) stream of a segment; flag fibre starts (a segment
// starts a fibre: segments are disjoint ranges of the top key field); detect
// duplicates.
template <class VT, class OT>
__global__ void k_gather_stream(const int32_t* __restrict__ idx_k, const VT* __restrict__ vals,
                                const uint64_t* __restrict__ pos, const uint32_t* __restrict__ perm,
                                const uint64_t* __restrict__ skeys, int compose, int ik_bits, int64_t n,
                                ValueCoder vc, int32_t* __restrict__ ik_out, OT* __restrict__ val_out,
                                uint32_t* __restrict__ start_flag, int* status) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = seg_src(pos, (int64_t)perm[j]);
    const int32_t ik = idx_k[e];
    ik_out[j] = ik;
    val_out[j] = store_value<VT, OT>(vc, vals[e], status);
    const uint64_t key = compose ? (skeys[j] >> ik_bits) : skeys[j];
    uint32_t start = 1;
    if (j > 0) {
      const uint64_t prev = compose ? (skeys[j - 1] >> ik_bits) : skeys[j - 1];
      if (prev == key) {
        start = 0;
        const int32_t ikp = idx_k[seg_src(pos, (int64_t)perm[j - 1])];
        if (ikp == ik) set_status(status, CPA_ERR_COO_DUP);
      }
    }
    start_flag[j] = start;
  }
}

// Fibre table entries of a segment: global fibre fbase + fid[j], global start base + j
// (its low off_bits bits).
__global__ void k_write_fibres(const uint64_t* __restrict__ skeys, int compose, int ik_bits,
                               const uint32_t* __restrict__ start_flag,
                               const uint64_t* __restrict__ fid, int64_t n, int64_t fbase, int64_t base,
                               uint64_t off_mask, uint64_t* __restrict__ keys, uint32_t* __restrict__ off) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    if (start_flag[j]) {
      const int64_t f = fbase + (int64_t)fid[j];
      keys[f] = compose ? (skeys[j] >> ik_bits) : skeys[j];
      off[f] = (uint32_t)((uint64_t)(base + j) & off_mask);
    }
  }
}

__global__ void k_finish_off(uint32_t* off, int64_t nfib, int64_t nnz, uint64_t off_mask) {
  off[nfib] = (uint32_t)((uint64_t)nnz & off_mask);
}

constexpr size_t kFibreHashBudget = size_t(4) << 30;  // bytes of fibre hash table per mode
constexpr int kMaxDirBits = 28;                        // directory of at most 2^28 + 1 entries
constexpr int kHistBits = 24;                          // segment planning: at most 2^24 bins

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
__global__ void k_hash_fibres(const uint64_t* __restrict__ keys, OffView off, int64_t nfib, int hbits,
                              ulonglong2* __restrict__ htab) {
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

// Largest number of nonzeros per build segment (scratch is about 44 bytes per
// nonzero of the largest segment); CPA_INDEX_SEGMENT_NNZ overrides the default 2^29.
int64_t index_segment_nnz() {
  const char* e = getenv("CPA_INDEX_SEGMENT_NNZ");
  int64_t v = e ? atoll(e) : 0;
  if (v <= 0) v = int64_t(1) << 29;
  if (v > (int64_t(1) << 31)) v = int64_t(1) << 31;
  return v;
}

// Bits of a stored fibre offset: 32, or fewer if CPA_INDEX_OFFSET_BITS asks (tests use
// it to place the points where the offsets pass a multiple of 2^bits in small tensors).
int index_offset_bits() {
  const char* e = getenv("CPA_INDEX_OFFSET_BITS");
  const int v = e ? atoi(e) : 32;
  return v >= 4 && v <= 32 ? v : 32;
}

// Fibre hash tables are built when they fit their budget unless CPA_INDEX_HASH=0
// (tests use it to send the probes through the directory at small sizes).
bool index_hash_enabled() {
  const char* e = getenv("CPA_INDEX_HASH");
  return !(e && atoi(e) == 0);
}

struct Segment {
  int64_t lo, hi;  // range of the top coordinate
  int64_t n;       // nonzeros
};

// Split the nonzeros of mode k's index into segments by ranges of the top field of
// the packed key (the other mode of highest number), at most seg_max nonzeros each
// unless one histogram bin holds more.  Segments ascend in key order.
int plan_segments(const cpa_index* X, const CooPtrs& coo, const KeyLayout& L, int64_t seg_max,
                  cudaStream_t st, std::vector<Segment>* segs) {
  segs->clear();
  const int64_t nnz = X->nnz;
  const int mtop = L.mode[L.d - 1];
  const int64_t ntop = X->dims[mtop];
  if (nnz <= seg_max) {
    segs->push_back(Segment{0, ntop, nnz});
    return CPA_OK;
  }
  int shift = 0;
  while ((ntop >> shift) >= (int64_t(1) << kHistBits)) ++shift;
  const int64_t nbins = ((ntop - 1) >> shift) + 1;
  unsigned long long* dh = nullptr;
  CPA_CUDA_TRY(cudaMallocAsync((void**)&dh, sizeof(unsigned long long) * nbins, st));
  CPA_CUDA_TRY(cudaMemsetAsync(dh, 0, sizeof(unsigned long long) * nbins, st));
  k_top_hist<<<grid_for(nnz), 256, 0, st>>>(coo.idx[mtop], nnz, shift, dh);
  std::vector<unsigned long long> h((size_t)nbins);
  cudaError_t e0 = cudaGetLastError();
  cudaError_t e1 = e0 == cudaSuccess ? cudaMemcpyAsync(h.data(), dh, sizeof(unsigned long long) * nbins,
                                                       cudaMemcpyDeviceToHost, st)
                                     : e0;
  cudaError_t e2 = cudaFreeAsync(dh, st);
  cudaError_t e3 = cudaStreamSynchronize(st);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return CPA_ERR_CUDA;
  int64_t cur_lo = 0, cur_n = 0;
  for (int64_t b = 0; b < nbins; ++b) {
    const int64_t c = (int64_t)h[(size_t)b];
    if (cur_n > 0 && cur_n + c > seg_max) {
      segs->push_back(Segment{cur_lo, b << shift, cur_n});
      cur_lo = b << shift;
      cur_n = 0;
    }
    cur_n += c;
  }
  if (cur_n > 0 || segs->empty()) segs->push_back(Segment{cur_lo, ntop, cur_n});
  for (const Segment& s : *segs)
    if (s.n >= (int64_t(1) << 32)) return CPA_ERR_UNSUPPORTED;  // local numbers are 32-bit
  return CPA_OK;
}

template <class T>
int index_alloc(cpa_index* X, T** p, size_t count, cudaStream_t st) {
  const size_t bytes = sizeof(T) * (count > 0 ? count : 1);
  CPA_CUDA_TRY(cudaMallocAsync((void**)p, bytes, st));
  X->allocations.push_back(*p);
  X->device_bytes += bytes;
  return CPA_OK;
}

// Mode k of the index, segment by segment.  With more than one segment a first pass
// sorts each segment's packed keys to count its fibres, so that the fibre table is
// allocated once at its final size; the second pass sorts (key, i_k), writes the
// permuted stream at the segment's place and the segment's fibres.
template <class VT, class OT>
int build_mode(cpa_index* X, const CooPtrs& coo, const VT* vals, const ValueCoder& vc, int k, int64_t seg_max,
               int* d_status, cudaStream_t st) {
  const int64_t nnz = X->nnz;
  const int D = X->order;
  auto& M = X->mode[k];
  make_layout(D, X->dims, k, &M.L);
  const int ik_bits = ceil_log2(X->dims[k]);
  const int compose = (M.L.total_bits + ik_bits) <= 64;
  std::vector<Segment> segs;
  CPA_TRY(plan_segments(X, coo, M.L, seg_max, st, &segs));
  const bool multi = segs.size() > 1;
  int64_t smax = 0;
  for (const Segment& s : segs) smax = s.n > smax ? s.n : smax;
  const int32_t* itop = coo.idx[M.L.mode[M.L.d - 1]];
  // scratch for the largest segment
  const size_t sort_ws = sort_workspace(smax);
  const size_t scan_ws = scan_workspace(smax);
  Arena a;
  uint64_t *pos = nullptr, *k0 = nullptr, *k1 = nullptr, *fid = nullptr;
  uint32_t *p0 = nullptr, *p1 = nullptr, *flag = nullptr;
  unsigned long long* d_count = nullptr;
  char* sws = nullptr;
  for (int pass = 0; pass < 2; ++pass) {
    a.used = 0;
    pos = multi ? a.take<uint64_t>(smax) : nullptr;
    k0 = a.take<uint64_t>(smax);
    k1 = a.take<uint64_t>(smax);
    p0 = a.take<uint32_t>(smax);
    p1 = a.take<uint32_t>(smax);
    flag = a.take<uint32_t>(smax);
    fid = a.take<uint64_t>(smax);
    sws = a.take<char>(sort_ws > scan_ws ? sort_ws : scan_ws);
    d_count = a.take<unsigned long long>(2);
    if (pass == 0) {
      CPA_CUDA_TRY(cudaMallocAsync((void**)&a.base, a.used, st));
      a.cap = a.used;
    }
  }
  auto fail = [&](int code) {
    cudaFreeAsync(a.base, st);
    return code;
  };
  auto select = [&](const Segment& s) -> int {
    if (!multi) return CPA_OK;
    if (cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st) != cudaSuccess) return CPA_ERR_CUDA;
    k_seg_select<<<grid_for(nnz), 256, 0, st>>>(itop, nnz, s.lo, s.hi, pos, smax, d_count, d_status);
    unsigned long long got = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&got, d_count, sizeof(got), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return CPA_ERR_CUDA;
    return (int64_t)got == s.n ? CPA_OK : CPA_ERR_CUDA;  // every position of the segment was listed
  };
  // pass 1 (several segments): fibres per segment
  std::vector<int64_t> seg_fib(segs.size(), 0);
  int64_t nfib_total = -1;
  if (multi) {
    nfib_total = 0;
    for (size_t si = 0; si < segs.size(); ++si) {
      const Segment& s = segs[si];
      if (s.n == 0) continue;
      int rc = select(s);
      if (rc < 0) return fail(rc);
      k_seg_packed_keys<<<grid_for(s.n), 256, 0, st>>>(coo, M.L, pos, s.n, k0);
      if (cudaGetLastError() != cudaSuccess) return fail(CPA_ERR_CUDA);
      int in_alt = 0;
      rc = radix_sort<uint32_t>(k0, k1, nullptr, nullptr, DevCount{nullptr, s.n}, 0, M.L.total_bits, sws, st,
                                &in_alt);
      if (rc < 0) return fail(rc);
      unsigned long long cnt = 0;
      if (cudaMemsetAsync(d_count + 1, 0, sizeof(unsigned long long), st) != cudaSuccess) return fail(CPA_ERR_CUDA);
      k_count_distinct<<<grid_for(s.n), 256, 0, st>>>(in_alt ? k1 : k0, s.n, d_count + 1);
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpyAsync(&cnt, d_count + 1, sizeof(cnt), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return fail(CPA_ERR_CUDA);
      seg_fib[si] = (int64_t)cnt;
      nfib_total += (int64_t)cnt;
    }
  }
  // permuted stream
  if (index_alloc(X, &M.ik, (size_t)nnz, st) < 0) return fail(CPA_ERR_OOM);
  OT* val_out = nullptr;
  if (index_alloc(X, &val_out, (size_t)nnz, st) < 0) return fail(CPA_ERR_OOM);
  M.val = val_out;
  if (multi) {
    M.nfib = nfib_total;
    if (index_alloc(X, &M.keys, (size_t)M.nfib, st) < 0 || index_alloc(X, &M.off, (size_t)M.nfib + 1, st) < 0)
      return fail(CPA_ERR_OOM);
  }
  const int off_bits = index_offset_bits();
  const uint64_t off_mask = (off_bits >= 32) ? 0xffffffffull : ((1ull << off_bits) - 1ull);
  if ((nnz >> off_bits) > kMaxWraps) return fail(CPA_ERR_UNSUPPORTED);
  const int nwrap = (int)(nnz >> off_bits);
  int64_t wraps[kMaxWraps];
  for (int w = 0; w < kMaxWraps; ++w) wraps[w] = -1;
  int64_t base = 0, fbase = 0;
  for (size_t si = 0; si < segs.size(); ++si) {
    const Segment& s = segs[si];
    if (s.n == 0) continue;
    int rc = select(s);
    if (rc < 0) return fail(rc);
    const unsigned grid = grid_for(s.n);
    int in_alt = 0;
    k_make_keys<<<grid, 256, 0, st>>>(coo, M.L, k, ik_bits, compose, pos, s.n, k0, p0);
    if (cudaGetLastError() != cudaSuccess) return fail(CPA_ERR_CUDA);
    uint64_t* sk;
    uint32_t* sp;
    if (compose) {
      rc = radix_sort<uint32_t>(k0, k1, p0, p1, DevCount{nullptr, s.n}, 0, M.L.total_bits + ik_bits, sws, st,
                                &in_alt);
      if (rc < 0) return fail(rc);
      sk = in_alt ? k1 : k0;
      sp = in_alt ? p1 : p0;
    } else {
      // stable sort by i_k, then stable sort by the packed key
      rc = radix_sort<uint32_t>(k0, k1, p0, p1, DevCount{nullptr, s.n}, 0, ik_bits, sws, st, &in_alt);
      if (rc < 0) return fail(rc);
      uint64_t* kk = in_alt ? k1 : k0;
      uint64_t* ko = in_alt ? k0 : k1;
      uint32_t* pp = in_alt ? p1 : p0;
      uint32_t* po = in_alt ? p0 : p1;
      k_packed_keys_by_perm<<<grid, 256, 0, st>>>(coo, M.L, pos, s.n, pp, kk);
      if (cudaGetLastError() != cudaSuccess) return fail(CPA_ERR_CUDA);
      rc = radix_sort<uint32_t>(kk, ko, pp, po, DevCount{nullptr, s.n}, 0, M.L.total_bits, sws, st, &in_alt);
      if (rc < 0) return fail(rc);
      sk = in_alt ? ko : kk;
      sp = in_alt ? po : pp;
    }
    k_gather_stream<VT, OT><<<grid, 256, 0, st>>>(coo.idx[k], vals, pos, sp, sk, compose, ik_bits, s.n, vc,
                                                  M.ik + base, val_out + base, flag, d_status);
    if (cudaGetLastError() != cudaSuccess) return fail(CPA_ERR_CUDA);
    rc = scan_u64<uint32_t>(flag, fid, DevCount{nullptr, s.n}, false, reinterpret_cast<uint64_t*>(d_count), sws,
                            st);
    if (rc < 0) return fail(rc);
    uint64_t nf = 0;
    int status = 0;
    if (cudaMemcpyAsync(&nf, d_count, sizeof(uint64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return fail(CPA_ERR_CUDA);
    // wrap points inside this segment: the fibre holding position B = (w + 1) 2^off_bits, or
    // the next one if it starts before B, is fbase + fid[B - base] (fid counts the starts
    // before each position)
    uint64_t fidv[kMaxWraps];
    int wl[kMaxWraps], nwl = 0;
    for (int w = 0; w < nwrap; ++w) {
      const int64_t B = (int64_t)(w + 1) << off_bits;
      if (B >= base && B < base + s.n) {
        if (cudaMemcpyAsync(&fidv[nwl], fid + (B - base), sizeof(uint64_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
          return fail(CPA_ERR_CUDA);
        wl[nwl++] = w;
      }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(CPA_ERR_CUDA);
    if (status < 0) return fail(status);
    for (int q = 0; q < nwl; ++q) wraps[wl[q]] = fbase + (int64_t)fidv[q];
    if (multi) {
      if ((int64_t)nf != seg_fib[si]) return fail(CPA_ERR_CUDA);  // the two passes must agree
    } else {
      M.nfib = (int64_t)nf;
      if (index_alloc(X, &M.keys, (size_t)M.nfib, st) < 0 || index_alloc(X, &M.off, (size_t)M.nfib + 1, st) < 0)
        return fail(CPA_ERR_OOM);
    }
    k_write_fibres<<<grid, 256, 0, st>>>(sk, compose, ik_bits, flag, fid, s.n, fbase, base, off_mask, M.keys,
                                         M.off);
    if (cudaGetLastError() != cudaSuccess) return fail(CPA_ERR_CUDA);
    base += s.n;
    fbase += (int64_t)nf;
  }
  if (M.keys == nullptr) {  // no nonzeros
    M.nfib = 0;
    if (index_alloc(X, &M.keys, 0, st) < 0 || index_alloc(X, &M.off, 1, st) < 0) return fail(CPA_ERR_OOM);
  }
  if (base != nnz || fbase != M.nfib) return fail(CPA_ERR_CUDA);
  k_finish_off<<<1, 1, 0, st>>>(M.off, M.nfib, nnz, off_mask);
  M.off_shift = off_bits;
  M.nwrap = nwrap;
  for (int w = 0; w < kMaxWraps; ++w) M.wrap[w] = w < nwrap ? (wraps[w] < 0 ? M.nfib : wraps[w]) : 0;
  CPA_CUDA_TRY(cudaFreeAsync(a.base, st));
  // directory: about four fibres per bucket
  int dbits = ceil_log2(M.nfib > 0 ? M.nfib : 1) - 2;
  if (dbits < 0) dbits = 0;
  if (dbits > M.L.total_bits) dbits = M.L.total_bits;
  if (dbits > kMaxDirBits) dbits = kMaxDirBits;
  M.dbits = dbits;
  M.dshift = M.L.total_bits - dbits;
  const int64_t nb = 1ll << dbits;
  CPA_TRY(index_alloc(X, &M.dir, (size_t)nb + 1, st));
  k_directory<<<grid_for(nb + 1), 256, 0, st>>>(M.keys, M.nfib, M.dshift, nb, M.dir);
  CPA_LAUNCH_CHECK();
  // hash table of the fibres (load <= 1/2) when it fits the budget and the record
  // encoding (fibre start < 2^40, length < 2^24)
  int hb = 4;
  while ((1ll << hb) < 2 * M.nfib) ++hb;
  const size_t hbytes = sizeof(ulonglong2) * ((size_t)1 << hb);
  const size_t longest = (size_t)X->dims[k];  // a fibre is at most dims[k] long
  if (index_hash_enabled() && M.nfib > 0 && hbytes <= kFibreHashBudget && longest < (1ull << 24) &&
      nnz < (1ll << 40)) {
    M.hbits = hb;
    CPA_TRY(index_alloc(X, &M.htab, (size_t)1 << hb, st));
    CPA_CUDA_TRY(cudaMemsetAsync(M.htab, 0xff, hbytes, st));
    k_hash_fibres<<<grid_for(M.nfib), 256, 0, st>>>(M.keys, off_view(X, k), M.nfib, hb, M.htab);
    CPA_LAUNCH_CHECK();
  }
  return CPA_OK;
}

template <class VT, class OT>
int build_modes(cpa_index* X, const CooPtrs& coo, const VT* vals, const ValueCoder& vc, int* d_status,
                cudaStream_t st) {
  const int64_t seg_max = index_segment_nnz();
  for (int k = 0; k < X->order; ++k) CPA_TRY((build_mode<VT, OT>(X, coo, vals, vc, k, seg_max, d_status, st)));
  return CPA_OK;
}

// Whether to store FP32 values as 16-bit codes: CPA_INDEX_VALUE_CODES=0 never, =1
// whenever the tensor has at most 65,536 distinct values, otherwise (default) also
// only for tensors of at least 2^31 nonzeros.
bool want_value_codes(int64_t nnz) {
  const char* e = getenv("CPA_INDEX_VALUE_CODES");
  if (e && atoi(e) == 0 && e[0] == '0') return false;
  if (e && atoi(e) == 1) return true;
  return nnz >= (int64_t(1) << 31);
}

// Builds the value table of an FP32 tensor: 1 and *vc (device set and codes, to be
// released by the caller through *tmp) if it has at most kMaxCodes distinct values,
// 0 if it has more.  X->vtab gets the distinct values in ascending bit-pattern order.
int make_value_codes(cpa_index* X, const float* vals, int64_t nnz, cudaStream_t st, std::vector<void*>* tmp,
                     ValueCoder* vc) {
  const size_t nslot = size_t(1) << kCodeSetBits;
  uint32_t* set = nullptr;
  uint16_t* codes = nullptr;
  unsigned* cnt = nullptr;
  CPA_CUDA_TRY(cudaMallocAsync((void**)&set, sizeof(uint32_t) * nslot, st));
  tmp->push_back(set);
  CPA_CUDA_TRY(cudaMallocAsync((void**)&codes, sizeof(uint16_t) * nslot, st));
  tmp->push_back(codes);
  CPA_CUDA_TRY(cudaMallocAsync((void**)&cnt, 16, st));
  tmp->push_back(cnt);
  CPA_CUDA_TRY(cudaMemsetAsync(set, 0xff, sizeof(uint32_t) * nslot, st));
  CPA_CUDA_TRY(cudaMemsetAsync(cnt, 0, 16, st));
  int* full = reinterpret_cast<int*>(cnt + 1);
  k_value_set<<<grid_for(nnz), 256, 0, st>>>(vals, nnz, set, cnt, full);
  CPA_LAUNCH_CHECK();
  std::vector<uint32_t> h(nslot);
  unsigned hc[2] = {0, 0};
  CPA_CUDA_TRY(cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaMemcpyAsync(h.data(), set, sizeof(uint32_t) * nslot, cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  if (hc[1] != 0 || hc[0] > (unsigned)kMaxCodes) return 0;
  std::vector<uint32_t> distinct;
  for (uint32_t b : h)
    if (b != kNoValue) distinct.push_back(b);
  std::sort(distinct.begin(), distinct.end());
  std::vector<uint16_t> hcode(nslot, 0);
  const uint32_t mask = (uint32_t)nslot - 1u;
  for (size_t c = 0; c < distinct.size(); ++c) {  // slot of each value, as the device finds it
    uint32_t s = (distinct[c] * 0x9E3779B1u) >> (32 - kCodeSetBits);
    while (h[s] != distinct[c]) s = (s + 1) & mask;
    hcode[s] = (uint16_t)c;
  }
  X->nvtab = (int)distinct.size();
  CPA_TRY(index_alloc(X, &X->vtab, distinct.size(), st));
  CPA_CUDA_TRY(cudaMemcpyAsync(X->vtab, distinct.data(), sizeof(float) * distinct.size(), cudaMemcpyHostToDevice,
                               st));
  CPA_CUDA_TRY(cudaMemcpyAsync(codes, hcode.data(), sizeof(uint16_t) * nslot, cudaMemcpyHostToDevice, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors go out of scope
  vc->set = set;
  vc->codes = codes;
  return 1;
}

}  // namespace

int index_build(const cpa_coo* coo, cudaStream_t st, cpa_index** out) {
  if (!coo || !out || coo->order < 2 || coo->order > kMaxOrder || coo->nnz < 0 || !coo->dims ||
      !coo->idx || (coo->nnz > 0 && !coo->vals))
    return CPA_ERR_ARG;
  if (coo->val_dtype != CPA_F32 && coo->val_dtype != CPA_F64) return CPA_ERR_ARG;
  if (coo->nnz >= (1ll << 35)) return CPA_ERR_UNSUPPORTED;
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
  ValueCoder vc;
  if (coo->val_dtype == CPA_F32 && nnz > 0 && want_value_codes(nnz)) {
    rc = make_value_codes(X, reinterpret_cast<const float*>(dvals), nnz, st, &tmp, &vc);
    if (rc < 0) return fail(rc);
  }
  if (vc.set)
    rc = build_modes<float, uint16_t>(X, cp, reinterpret_cast<const float*>(dvals), vc, d_status, st);
  else if (coo->val_dtype == CPA_F32)
    rc = build_modes<float, float>(X, cp, reinterpret_cast<const float*>(dvals), vc, d_status, st);
  else
    rc = build_modes<double, double>(X, cp, reinterpret_cast<const double*>(dvals), vc, d_status, st);
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
__global__ void k_export(KeyLayout L, const uint64_t* __restrict__ pk, int64_t nfib,
                         uint64_t* __restrict__ keys_out) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nfib;
       f += (int64_t)gridDim.x * blockDim.x)
    keys_out[f] = L.linear(pk[f]);
}

__global__ void k_export_coded(const uint16_t* __restrict__ code, const float* __restrict__ vtab, int64_t n,
                               float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = vtab[code[e]];
}

__global__ void k_export_off(OffView off, int64_t nfib, uint64_t* __restrict__ out) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f <= nfib;
       f += (int64_t)gridDim.x * blockDim.x)
    out[f] = off[f];
}
}  // namespace

int index_export(const cpa_index* X, int k, uint64_t* keys, uint64_t* off, int32_t* ik, void* val,
                 cudaStream_t st) {
  if (!X || k < 0 || k >= X->order) return CPA_ERR_ARG;
  const auto& M = X->mode[k];
  if (keys && M.nfib > 0) {
    k_export<<<grid_for(M.nfib), 256, 0, st>>>(M.L, M.keys, M.nfib, keys);
    CPA_LAUNCH_CHECK();
  }
  if (off) {
    k_export_off<<<grid_for(M.nfib + 1), 256, 0, st>>>(off_view(X, k), M.nfib, off);
    CPA_LAUNCH_CHECK();
  }
  if (ik && X->nnz > 0)
    CPA_CUDA_TRY(cudaMemcpyAsync(ik, M.ik, sizeof(int32_t) * X->nnz, cudaMemcpyDeviceToDevice, st));
  if (val && X->nnz > 0) {
    if (X->vtab) {
      k_export_coded<<<grid_for(X->nnz), 256, 0, st>>>(reinterpret_cast<const uint16_t*>(M.val), X->vtab, X->nnz,
                                                        reinterpret_cast<float*>(val));
      CPA_LAUNCH_CHECK();
    } else {
      CPA_CUDA_TRY(cudaMemcpyAsync(val, M.val, (X->val_dtype == CPA_F32 ? 4 : 8) * X->nnz,
                                   cudaMemcpyDeviceToDevice, st));
    }
  }
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
    const uint64_t e1 = Xk.off[f + 1];
    for (uint64_t e = Xk.off[f]; e < e1; ++e) {
      const double x = (double)Xk.value(e);
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
  with_value_type(X, [&](auto tag) {
    using VT = decltype(tag);
    k_rrf<VT><<<grid, 256, 0, st>>>(fibre_view<VT>(X, k), k, s_init, seed, omega, r, A);
    return 0;
  });
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

}  // namespace cpa
