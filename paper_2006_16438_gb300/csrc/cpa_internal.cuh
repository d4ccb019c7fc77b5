// Internal types and cross-file entry points of the CP-ARLS-LEV CUDA library.
#pragma once

#include <mutex>
#include <type_traits>

#include "cpa_common.cuh"

namespace cpa {
struct Plan;
void plan_free(Plan* p);
}  // namespace cpa

namespace cpa {
// Fibre offsets stored as their low `shift` bits (32 unless a test asks for fewer).
// Offsets ascend with the fibre number, so the high part of off[f] is the number of
// multiples of 2^shift that the offsets have passed by fibre f: wrap[w] is the first
// fibre whose offset is >= (w + 1) 2^shift.  The builder accepts nnz < 8 * 2^shift,
// so there are at most seven.
constexpr int kMaxWraps = 7;
struct OffView {
  const uint32_t* lo = nullptr;  // F_k + 1 entries
  int shift = 32;
  int nwrap = 0;
  int64_t wrap[kMaxWraps] = {};
  __host__ __device__ __forceinline__ uint64_t operator[](int64_t f) const {
    uint64_t hi = 0;
#pragma unroll
    for (int w = 0; w < kMaxWraps; ++w) hi += (w < nwrap && f >= wrap[w]) ? 1ull : 0ull;  // static indices
    return (hi << shift) | (uint64_t)lo[f];
  }
};
}  // namespace cpa

// Opaque index of the C ABI (Section 5.3 fibre index, one per mode).
struct cpa_index {
  int order = 0;
  int64_t dims[cpa::kMaxOrder] = {};
  int64_t nnz = 0;
  int val_dtype = CPA_F64;
  double norm_x2 = 0.0;  // ||X||_F^2, FP64
  struct Mode {
    cpa::KeyLayout L;           // packed layout of the other modes
    int64_t nfib = 0;           // F_k
    uint64_t* keys = nullptr;   // F_k packed keys, ascending
    uint32_t* off = nullptr;    // F_k + 1 offsets into ik/val, low off_shift bits
    int off_shift = 32;
    int nwrap = 0;              // high parts: see cpa::OffView
    int64_t wrap[cpa::kMaxWraps] = {};
    int32_t* ik = nullptr;      // nnz mode-k indices, fibre order (ascending within a fibre)
    void* val = nullptr;        // nnz values (float or double)
    uint64_t* dir = nullptr;    // (1 << dbits) + 1 bucket starts over the top key bits
    int dbits = 0;
    int dshift = 0;
    // open-addressing table of (key, lo << 24 | len), 2^hbits slots (null: directory only)
    ulonglong2* htab = nullptr;
    int hbits = 0;
  } mode[cpa::kMaxOrder];
  // FP32 values stored as 16-bit codes into vtab (ascending distinct values, nvtab <=
  // 65,536) instead of floats; null: values in val_dtype
  float* vtab = nullptr;
  int nvtab = 0;
  std::vector<void*> allocations;
  size_t device_bytes = 0;  // sum of the sizes of `allocations`
  // cached workspace + CUDA graph of one outer iteration (see api.cu)
  cpa::Plan* plan = nullptr;
  std::mutex plan_mu;
};

namespace cpa {

// Empty slot of the fibre hash table (a packed key uses at most 63 bits).
constexpr uint64_t kNoFibre = ~0ull;
// Slot of a packed key in a table of 2^hbits slots (multiplicative hashing).
__host__ __device__ __forceinline__ uint64_t fibre_slot(uint64_t key, int hbits) {
  return (key * 0x9E3779B97F4A7C15ull) >> (64 - hbits);
}

// Arithmetic type of a stored value: the value itself, or the float a 16-bit code
// stands for.
template <class VT>
struct ValueOf {
  using type = VT;
};
template <>
struct ValueOf<uint16_t> {
  using type = float;
};

// Device view of one mode of the index, passed by value to kernels.  VT is the
// stored value type: float, double, or uint16_t (codes into vtab).
template <class VT>
struct FibreIndex {
  const uint64_t* keys;
  OffView off;  // off[f], f <= nfib, as 64-bit offsets
  const int32_t* ik;
  const VT* val;
  const uint64_t* dir;
  int64_t nfib;
  int dshift;
  int dbits;
  const ulonglong2* htab;  // null: probe through the directory
  int hbits;
  const float* vtab;  // values of the codes (VT = uint16_t)

  // Value of the nonzero at stream position e.
  __device__ __forceinline__ typename ValueOf<VT>::type value(uint64_t e) const {
    if constexpr (std::is_same<VT, uint16_t>::value) return vtab[val[e]];
    else return val[e];
  }
  // The same with a streaming (evict-first) load of the stored value.
  __device__ __forceinline__ typename ValueOf<VT>::type value_stream(uint64_t e) const {
    if constexpr (std::is_same<VT, uint16_t>::value) return vtab[__ldcs(val + e)];
    else return __ldcs(val + e);
  }

  // Fibre [*lo, *hi) of a packed key; empty range if the key has no nonzeros.
  // With the hash table a probe is one 16-byte record (key, lo << 24 | len) per slot
  // visited (load <= 1/2); otherwise the directory bucket and a bisection of keys.
  __device__ __forceinline__ void probe(uint64_t key, uint64_t* lo, uint64_t* hi) const {
    if (htab) {
      const uint64_t mask = (1ull << hbits) - 1ull;
      uint64_t h = fibre_slot(key, hbits);
      for (uint64_t step = 0; step <= mask; ++step) {
        const ulonglong2 rec = htab[h];
        if (rec.x == key) {
          *lo = rec.y >> 24;
          *hi = *lo + (rec.y & 0xffffffull);
          return;
        }
        if (rec.x == kNoFibre) break;
        h = (h + 1) & mask;
      }
      *lo = *hi = 0;
      return;
    }
    const uint64_t b = dshift >= 64 ? 0 : (key >> dshift);
    int64_t a = (int64_t)dir[b], z = (int64_t)dir[b + 1];
    while (a < z) {  // lower bound in keys[a, z)
      const int64_t mid = a + ((z - a) >> 1);
      if (keys[mid] < key) a = mid + 1; else z = mid;
    }
    if (a < nfib && keys[a] == key) {
      *lo = off[a];
      *hi = off[a + 1];
    } else {
      *lo = *hi = 0;
    }
  }
};

inline OffView off_view(const cpa_index* X, int k) {
  const auto& M = X->mode[k];
  OffView o;
  o.lo = M.off;
  o.shift = M.off_shift;
  o.nwrap = M.nwrap;
  for (int w = 0; w < kMaxWraps; ++w) o.wrap[w] = M.wrap[w];
  return o;
}

template <class VT>
inline FibreIndex<VT> fibre_view(const cpa_index* X, int k) {
  const auto& M = X->mode[k];
  return FibreIndex<VT>{M.keys, off_view(X, k), M.ik, reinterpret_cast<const VT*>(M.val), M.dir,
                        M.nfib, M.dshift, M.dbits, M.htab, M.hbits, X->vtab};
}

// Calls fn with a value of the index's stored value type (uint16_t for coded values).
template <class Fn>
inline int with_value_type(const cpa_index* X, Fn&& fn) {
  if (X->vtab) return fn(uint16_t());
  if (X->val_dtype == CPA_F32) return fn(float());
  return fn(double());
}

// index.cu
int index_build(const cpa_coo* coo, cudaStream_t st, cpa_index** out);
void index_free(cpa_index* X);
int index_export(const cpa_index* X, int k, uint64_t* keys, uint64_t* off, int32_t* ik,
                 void* val, cudaStream_t st);
// Range-finder initial factor of mode k (App. F): A (n_k x r, zeroed here) =
// X_(k)(:, S) omega with S = s_init fibres of mode k drawn uniformly (Philox domain
// kDomainRrf | k, word 0 of counter (j, 0, ., 0), position floor(u F_k / 2^64) in key
// order).  omega: s_init x r device doubles.
int rrf_enqueue(const cpa_index* X, int k, int64_t s_init, uint64_t seed, const double* omega, int r,
                double* A, cudaStream_t st);

}  // namespace cpa
