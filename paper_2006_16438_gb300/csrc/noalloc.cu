// cpa_leverage_noalloc: the leverage-score computation of cpa_leverage with its
// scratch memory (the r x r Gram matrix, its factorisation and a warning word) in a
// file-scope device array instead of a per-call allocation.
//
// Who needs this: callers that may not allocate device memory once they are
// running -- for example a serving process that reserves the GPU's memory for its
// own pool at start-up (a library cudaMalloc would then fail or fragment that pool),
// or a latency-critical loop where cudaMalloc/cudaFree would synchronise the device.
// They pass only their input and output buffers.
//
// The array is loaded with the library and every GPU that loads it keeps it until
// the process exits (kScratchBytes per device).  All calls share it: concurrent
// calls whose work overlaps on a GPU race on it and must not be issued.
#include <mutex>

#include "dense.cuh"

namespace {

using cpa::SmallFactor;

// Largest scratch this entry point uses: r <= 64 (cpa::kMaxRank).  Layout: the r x r
// Gram, its factorisation, a warning word, then the block partial sums of the Gram
// (the rest of the array: at least 57 blocks at r = 64, the full grid at r <= 36).
constexpr size_t kScratchBytes = 1024 * 1024;
constexpr size_t kGramOff = 0;
constexpr size_t kFactorOff = 32 * 1024;  // r*r doubles <= 32 KiB before it
constexpr size_t kWarnOff = kFactorOff + ((sizeof(SmallFactor) + 255) / 256) * 256;
constexpr size_t kSumsOff = kWarnOff + 256;
static_assert(sizeof(double) * cpa::kMaxRank * cpa::kMaxRank <= kFactorOff, "Gram does not fit");
static_assert(kSumsOff + cpa::block_sums_bytes(32, cpa::kMaxRank * (cpa::kMaxRank + 1) / 2) <= kScratchBytes,
              "scratch layout exceeds the array");

// Blocks of the Gram whose partial sums fit the rest of the array at rank r.
int sums_blocks(int r) {
  const size_t width = (size_t)cpa::gram_sums_width(r);
  const size_t fit = (kScratchBytes - kSumsOff - 256) / (sizeof(double) * width);
  return (int)(fit < (size_t)cpa::kSumMaxBlocks ? fit : (size_t)cpa::kSumMaxBlocks);
}

static __device__ __align__(256) unsigned char g_lev_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_lev_scratch on the current device, looked up once per device.
// In host code the symbol g_lev_scratch is only a host-side stand-in, never a device
// address; the address comes from cudaGetSymbolAddress with the device current.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CPA_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return CPA_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_lev_scratch) != cudaSuccess || !p) return CPA_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return CPA_OK;
}

}  // namespace

extern "C" int cpa_leverage_noalloc(const double* A, int64_t n, int32_t r, double* lev,
                                    void* stream) {
  if (!A || !lev || n < 1 || r < 1) return CPA_ERR_ARG;
  if (r > cpa::kMaxRank) return CPA_ERR_UNSUPPORTED;  // the scratch holds r <= 64 only
  cudaStream_t st = (cudaStream_t)stream;
  void* base = nullptr;
  CPA_TRY(scratch_address(&base));
  char* b = reinterpret_cast<char*>(base);
  double* G = reinterpret_cast<double*>(b + kGramOff);
  SmallFactor* f = reinterpret_cast<SmallFactor*>(b + kFactorOff);
  int* warn = reinterpret_cast<int*>(b + kWarnOff);
  const cpa::BlockSums sums = cpa::block_sums_at(b + kSumsOff, sums_blocks(r));
  // the array keeps the previous call's contents: clear the warning word and the
  // ticket of the block sums (re-armed by every completed Gram, cleared here in case
  // an earlier launch did not complete)
  CPA_CUDA_TRY(cudaMemsetAsync(warn, 0, sizeof(int), st));
  CPA_CUDA_TRY(cudaMemsetAsync(sums.ticket, 0, sizeof(unsigned), st));
  CPA_TRY(cpa::gram_rows<double>(A, n, r, G, sums, st));
  CPA_TRY(cpa::factor_spd(G, r, 1, 1, 1e-12, f, warn, CPA_WARN_RANK_DEFICIENT_LEV, st));
  CPA_TRY(cpa::lev_rows<double>(A, n, r, f, lev, nullptr, nullptr, (double*)nullptr, st));
  int hwarn = 0;
  CPA_CUDA_TRY(cudaMemcpyAsync(&hwarn, warn, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPA_CUDA_TRY(cudaStreamSynchronize(st));
  return hwarn;
}
