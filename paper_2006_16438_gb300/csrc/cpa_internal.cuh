// Internal types and cross-file entry points of the CP-ARLS-LEV CUDA library.
#pragma once

#include <mutex>

#include "cpa_common.cuh"

namespace cpa {
struct Plan;
void plan_free(Plan* p);
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
    uint64_t* off = nullptr;    // F_k + 1 offsets into ik/val
    int32_t* ik = nullptr;      // nnz mode-k indices, fibre order (ascending within a fibre)
    void* val = nullptr;        // nnz values (float or double)
    uint64_t* dir = nullptr;    // (1 << dbits) + 1 bucket starts over the top key bits
    int dbits = 0;
    int dshift = 0;
    // open-addressing table of (key, lo << 24 | len), 2^hbits slots (null: directory only)
    ulonglong2* htab = nullptr;
    int hbits = 0;
  } mode[cpa::kMaxOrder];
  std::vector<void*> allocations;
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

// Device view of one mode of the index, passed by value to kernels.
template <class VT>
struct FibreIndex {
  const uint64_t* keys;
  const uint64_t* off;
  const int32_t* ik;
  const VT* val;
  const uint64_t* dir;
  int64_t nfib;
  int dshift;
  int dbits;
  const ulonglong2* htab;  // null: probe through the directory
  int hbits;

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

template <class VT>
inline FibreIndex<VT> fibre_view(const cpa_index* X, int k) {
  const auto& M = X->mode[k];
  return FibreIndex<VT>{M.keys, M.off, M.ik, reinterpret_cast<const VT*>(M.val), M.dir,
                        M.nfib, M.dshift, M.dbits, M.htab, M.hbits};
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
