// Shared device/host helpers of the CP-ARLS-LEV CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "../../include/cpa.h"

namespace cpa {

constexpr int kMaxOrder = 8;
constexpr int kMaxRank = 64;
constexpr int kWarp = 32;

// ---------------------------------------------------------------------------
// Device-side status: kernels record the first error here instead of trapping.
// ---------------------------------------------------------------------------
// Comparisons of doubles through their bit patterns.  For non-negative, non-NaN
// values the IEEE patterns order like the values, so an integer compare gives the
// exact result; GB300's FP64 compare (and min/max) has a dependent latency of about
// 200 cycles against a few for the integer forms.
__device__ __forceinline__ bool nonneg_gt(double a, double b) {  // a > b, a and b >= 0
  return __double_as_longlong(a) > __double_as_longlong(b);
}
// a > 0, false for -0, negative values and NaN
__device__ __forceinline__ bool pos_finite(double a) {
  const long long v = __double_as_longlong(a);
  return v > 0 && v < 0x7ff0000000000000ll;
}

// Asynchronous 8-byte global -> shared copy (cp.async, no register round trip) and
// the wait for all of this thread's outstanding ones.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void set_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 64x64->128
// multiplies with the published multipliers, xor-mixing with the round key, which
// is advanced by the two published Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct Philox4x64 {
  static constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ull;
  static constexpr uint64_t kMulB = 0xCA5A826395121157ull;
  static constexpr uint64_t kWeylA = 0x9E3779B97F4A7C15ull;
  static constexpr uint64_t kWeylB = 0xBB67AE8584CAA73Bull;

  __device__ __forceinline__ static void block(uint64_t& w0, uint64_t& w1, uint64_t& w2,
                                               uint64_t& w3, uint64_t ka, uint64_t kb) {
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
      const uint64_t a_lo = kMulA * w0, a_hi = __umul64hi(kMulA, w0);
      const uint64_t b_lo = kMulB * w2, b_hi = __umul64hi(kMulB, w2);
      const uint64_t n0 = b_hi ^ w1 ^ ka;
      const uint64_t n2 = a_hi ^ w3 ^ kb;
      w0 = n0;
      w1 = b_lo;
      w2 = n2;
      w3 = a_lo;
      ka += kWeylA;
      kb += kWeylB;
    }
  }
};

// Domain tags of the draws in the third counter word: Khatri-Rao row sampling, the
// element sample of the estimated fit and the fibre draws of the range-finder
// initialisation.
constexpr uint64_t kDomainSample = 1ull << 32;
constexpr uint64_t kDomainFit = 2ull << 32;
constexpr uint64_t kDomainRrf = 3ull << 32;

// ---------------------------------------------------------------------------
// Packed multi-index: other mode t occupies bits [off_t, off_t + bits_t) of a
// 64-bit word.  The packing keeps the order of the linear index of Eq. 2.2 (both
// compare i_{d-1} first, then i_{d-2}, ...), so sorted packed keys are sorted
// linear keys and decoding needs only shifts and masks.
// ---------------------------------------------------------------------------
struct KeyLayout {
  int d;                        // number of other modes
  int mode[kMaxOrder];          // other modes, ascending
  int bits[kMaxOrder];
  int off[kMaxOrder];
  int total_bits;
  int64_t n[kMaxOrder];         // sizes of the other modes
  uint64_t stride[kMaxOrder];   // linear-key strides prod_{u<t} n_u

  __host__ __device__ __forceinline__ uint32_t get(uint64_t packed, int t) const {
    return (uint32_t)((packed >> off[t]) & ((1ull << bits[t]) - 1ull));
  }
  __host__ __device__ __forceinline__ uint64_t linear(uint64_t packed) const {
    uint64_t key = 0;
    for (int t = 0; t < d; ++t) key += (uint64_t)get(packed, t) * stride[t];
    return key;
  }
};

inline int ceil_log2(int64_t n) {
  int b = 0;
  while (b < 63 && (1ll << b) < n) ++b;
  return b < 1 ? 1 : b;
}

// Layout of the other modes of an update of mode k (k = -1: all `order` modes given
// in `dims` are "other" modes, used by the stage entry points).
inline bool make_layout(int order, const int64_t* dims, int k, KeyLayout* L) {
  memset(L, 0, sizeof(*L));
  int t = 0, off = 0;
  uint64_t stride = 1;
  for (int m = 0; m < order; ++m) {
    if (m == k) continue;
    L->mode[t] = m;
    L->n[t] = dims[m];
    L->bits[t] = ceil_log2(dims[m]);
    L->off[t] = off;
    L->stride[t] = stride;
    off += L->bits[t];
    stride *= (uint64_t)dims[m];
    ++t;
  }
  L->d = t;
  L->total_bits = off;
  return off <= 63;
}

// ---------------------------------------------------------------------------
// Deterministic sums across the blocks of a grid.  Each block stores its partial
// values (width of them) at part[blockIdx.x * width + i]; the block that arrives
// last (a ticket counter) adds every block's partials in block order and re-arms
// the ticket.  The result depends only on the grid size, so kernels that reduce
// this way take grids that do not depend on the SM count or an SM budget.
// ---------------------------------------------------------------------------
constexpr int kSumMaxBlocks = 608;  // largest grid of a block-ordered sum (4 per SM of a GB300)

struct BlockSums {
  unsigned* ticket = nullptr;  // zero between uses
  double* part = nullptr;      // max_blocks * width
  int max_blocks = 0;
};
constexpr size_t block_sums_bytes(int max_blocks, int width) {
  return 256 + sizeof(double) * (size_t)max_blocks * (size_t)(width > 0 ? width : 1);
}
// Views a zeroed region of block_sums_bytes(max_blocks, width) bytes at p.
inline BlockSums block_sums_at(void* p, int max_blocks) {
  BlockSums s;
  s.ticket = reinterpret_cast<unsigned*>(p);
  s.part = reinterpret_cast<double*>(reinterpret_cast<char*>(p) + 256);
  s.max_blocks = max_blocks;
  return s;
}

// Called by every thread of every block once the block's partials are stored;
// true in the one block that arrives last, which may then read all partials (with
// ld.global.cg, past the non-coherent L1).
__device__ __forceinline__ bool last_block_to_arrive(unsigned* ticket) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}
// Sum over blocks b = 0..nb-1 of part[b * width + i] in a fixed order (four
// interleaved chains, then (c0 + c1) + (c2 + c3)), so FP64 add latency overlaps.
__device__ __forceinline__ double ordered_block_sum(const double* part, int nb, int width, int i) {
  double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
  int b = 0;
  for (; b + 3 < nb; b += 4) {
    c0 += __ldcg(part + (size_t)b * width + i);
    c1 += __ldcg(part + (size_t)(b + 1) * width + i);
    c2 += __ldcg(part + (size_t)(b + 2) * width + i);
    c3 += __ldcg(part + (size_t)(b + 3) * width + i);
  }
  for (; b < nb; ++b) c0 += __ldcg(part + (size_t)b * width + i);
  return (c0 + c1) + (c2 + c3);
}
// Re-arms the ticket (by thread 0 of the last block, after its reads).
__device__ __forceinline__ void rearm_ticket(unsigned* ticket) {
  if (threadIdx.x == 0) *ticket = 0u;
}

// ---------------------------------------------------------------------------
// Device arena: one cudaMallocAsync block carved into aligned pieces.  A first
// pass with base == nullptr only measures.
// ---------------------------------------------------------------------------
struct Arena {
  char* base = nullptr;
  size_t used = 0;
  size_t cap = 0;
  template <class T>
  T* take(size_t count) {
    size_t at = (used + 255) & ~size_t(255);
    used = at + count * sizeof(T) + 1;
    return base ? reinterpret_cast<T*>(base + at) : nullptr;
  }
  // Workspace of a block-ordered sum (its ticket must be zeroed before first use).
  BlockSums take_sums(int max_blocks, int width) {
    char* p = take<char>(block_sums_bytes(max_blocks, width));
    BlockSums s;
    if (p) s = block_sums_at(p, max_blocks);
    s.max_blocks = max_blocks;
    return s;
  }
};

// ---------------------------------------------------------------------------
// Kernel attributes (the opt-in to large dynamic shared memory) belong to each
// device's context: set_attr_once runs `set` once per device, the current one.
// `done` holds a bit per device (devices >= 64: set at every call).  Two host threads
// may both run `set` for a device the first time; the call is idempotent.
// ---------------------------------------------------------------------------
template <class Fn>
inline cudaError_t set_attr_once(std::atomic<unsigned long long>& done, Fn&& set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = set();
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// ---------------------------------------------------------------------------
// Error plumbing
// ---------------------------------------------------------------------------
#define CPA_CUDA_TRY(expr)                                                        \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      if (getenv("CPA_VERBOSE"))                                                  \
        fprintf(stderr, "cpa: %s failed at %s:%d: %s\n", #expr, __FILE__, __LINE__, \
                cudaGetErrorString(_e));                                          \
      return _e == cudaErrorMemoryAllocation ? CPA_ERR_OOM : CPA_ERR_CUDA;        \
    }                                                                             \
  } while (0)

#define CPA_TRY(expr)            \
  do {                           \
    int _rc = (expr);            \
    if (_rc < 0) return _rc;     \
  } while (0)

#define CPA_LAUNCH_CHECK() CPA_CUDA_TRY(cudaGetLastError())

// SMs that grid sizes are computed for: the device's count, or a smaller budget set
// by the caller (per host thread) while it captures work that shares the GPU with
// other concurrent work (the batched entry point).
inline int& sm_budget_override() {
  static thread_local int v = 0;
  return v;
}
// The device's SM count, whatever the budget.
inline int device_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}
inline int num_sms() {
  if (sm_budget_override() > 0) return sm_budget_override();
  return device_sms();
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Record a timing event; inside a stream capture it becomes an event-record node of
// the graph (cudaEventRecordExternal), so it is re-recorded at every replay.
inline cudaError_t record_event(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(st, &cs);
  if (err != cudaSuccess) return err;
  if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  return cudaEventRecord(e, st);
}

// Count of items known only on the device (or a fixed host count if dptr is null).
struct DevCount {
  const int64_t* dptr = nullptr;
  int64_t max = 0;
  __device__ __forceinline__ int64_t get() const {
    if (!dptr) return max;
    int64_t v = *dptr;
    return v < max ? (v < 0 ? 0 : v) : max;
  }
};

// ---------------------------------------------------------------------------
// Scan and radix sort (scan_sort.cu).  Both take a device scratch buffer of the
// size their *_workspace function returns for the largest count they will see.
// ---------------------------------------------------------------------------
size_t scan_workspace(int64_t n_max);
// Optional extra outputs of a scan, written by the scan's own kernels:
//   end:   out[count] = total (an exclusive scan with its closing entry);
//   ratio: ratio[i] = in[i] / total as IEEE doubles (a probability vector).
struct ScanExtras {
  bool end = false;
  double* ratio = nullptr;
};
// out[i] = sum_{j<i} in[j] (exclusive) or sum_{j<=i} in[j] (inclusive) for
// i < count; *total (device, may be null) = sum of all.  in may equal out.
template <class T>
int scan_u64(const T* in, uint64_t* out, DevCount count, bool inclusive, uint64_t* total,
             void* scratch, cudaStream_t st, ScanExtras extras = ScanExtras());

size_t sort_workspace(int64_t n_max);
// Stable LSD radix sort (8-bit digits) of keys, and values if vals != null, on key
// bits [begin_bit, end_bit).  Ping-pongs between the buffer pairs; *in_alt is set
// to 1 if the sorted result is in keys_alt/vals_alt, 0 if in keys/vals.
template <class V>
int radix_sort(uint64_t* keys, uint64_t* keys_alt, V* vals, V* vals_alt, DevCount count,
               int begin_bit, int end_bit, void* scratch, cudaStream_t st, int* in_alt);

}  // namespace cpa
