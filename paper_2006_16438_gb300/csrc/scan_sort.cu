// Device prefix sums and stable LSD radix sort with device-side item counts.
//
// Both are multi-kernel designs: a scan is tile sums -> one-block scan of the tile
// sums -> tile-local scans; a radix pass is a per-tile digit histogram -> scan of
// the (digit-major) histogram -> stable scatter in which each warp ranks its keys
// with per-bit ballots and a per-warp digit counter.  Up to 64 tiles (256K items)
// the middle step is folded into the last kernel (each tile sums its predecessors
// itself), so a scan is 2 launches and a radix pass 2.  Item counts may live on the
// device (DevCount) so that a sequence of launches can be enqueued without a host
// round trip; grids are sized for the maximum count.
#include "cpa_common.cuh"

namespace cpa {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;

// Inclusive scan of one value per thread across the block; *total gets the sum of
// the whole block.  `sm` needs blockDim/32 words.  Ends with a barrier so `sm` can
// be reused at once.
__device__ __forceinline__ uint64_t block_inclusive_scan(uint64_t v, uint64_t* sm,
                                                         uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sm[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < nwarps ? sm[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < nwarps) sm[lane] = w;
  }
  __syncthreads();
  const uint64_t add = warp > 0 ? sm[warp - 1] : 0;
  *total = sm[nwarps - 1];
  __syncthreads();
  return v + add;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(const T* __restrict__ in,
                                                                 DevCount count,
                                                                 uint64_t* __restrict__ tile_sums) {
  __shared__ uint64_t sm[32];
  const int64_t n = count.get();
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint64_t s = 0;
  if (base < n) {
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
      const int64_t g = base + i;
      if (g < n) s += (uint64_t)in[g];
    }
  }
  uint64_t total;
  block_inclusive_scan(s, sm, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tile_offsets(uint64_t* tile_sums,
                                                                    int64_t ntiles,
                                                                    uint64_t* total_out) {
  __shared__ uint64_t sm[32];
  uint64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const uint64_t v = i < ntiles ? tile_sums[i] : 0;
    uint64_t bt;
    const uint64_t inc = block_inclusive_scan(v, sm, &bt);
    if (i < ntiles) tile_sums[i] = carry + inc - v;
    carry += bt;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

constexpr int kFusedTiles = 64;  // up to this many tiles a tile sums its predecessors itself

// fused = 1: tile_off holds raw tile sums and each block adds up the ones before it
// fused = 1: tile_off holds raw tile sums; each block sums its predecessors' (and,
// when the total is needed, all) itself.  fused = 0: tile_off holds offsets and
// *total_out the total, both from k_scan_tile_offsets.
template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const T* in, uint64_t* out,
                                                             DevCount count,
                                                             const uint64_t* __restrict__ tile_off,
                                                             int inclusive, int fused,
                                                             uint64_t* total_out, int write_end,
                                                             double* __restrict__ ratio) {
  __shared__ uint64_t sm[32];
  __shared__ uint64_t base_off, grand;
  const int64_t n = count.get();
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const bool need_total = ratio != nullptr || write_end;
  if (fused) {
    if (threadIdx.x < 32) {
      uint64_t acc = 0, tot = 0;
      for (int t = threadIdx.x; t < (int)gridDim.x; t += 32) {
        const uint64_t v = tile_off[t];
        if (t < (int)blockIdx.x) acc += v;
        tot += v;
      }
      for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
      }
      if (threadIdx.x == 0) {
        base_off = acc;
        grand = tot;
        if (blockIdx.x == gridDim.x - 1 && total_out) *total_out = tot;
      }
    }
    __syncthreads();
  } else if (need_total) {
    if (threadIdx.x == 0) grand = *total_out;
    __syncthreads();
  }
  if (write_end && blockIdx.x == 0 && threadIdx.x == 0) out[n] = grand;
  if (base >= n) return;  // uniform over the block
  const int64_t g0 = base + (int64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems];
  uint64_t local = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (g0 + i < n) ? (uint64_t)in[g0 + i] : 0;
    local += v[i];
  }
  uint64_t bt;
  const uint64_t inc = block_inclusive_scan(local, sm, &bt);
  uint64_t run = (fused ? base_off : tile_off[blockIdx.x]) + inc - local;
  const double Td = ratio ? __ull2double_rn(grand) : 1.0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (g0 + i < n) {
      if (ratio) ratio[g0 + i] = __ddiv_rn(__ull2double_rn(v[i]), Td);
      if (inclusive) {
        run += v[i];
        out[g0 + i] = run;
      } else {
        out[g0 + i] = run;
        run += v[i];
      }
    }
  }
}

// ---- radix sort ------------------------------------------------------------
__device__ __forceinline__ int digit_of(uint64_t k, int shift, uint32_t mask) {
  return (int)((k >> shift) & mask);
}

// Lanes of the warp holding the same digit as this lane (valid lanes only), built
// from one ballot per digit bit.
__device__ __forceinline__ unsigned digit_peers(int d, bool valid, int bits) {
  unsigned peers = __ballot_sync(0xffffffffu, valid);
  for (int b = 0; b < bits; ++b) {
    const bool bit = (d >> b) & 1;
    const unsigned bal = __ballot_sync(0xffffffffu, bit && valid);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t* __restrict__ keys,
                                                             DevCount count, int shift,
                                                             uint32_t mask, int bits,
                                                             uint64_t* __restrict__ hist,
                                                             int64_t ntiles) {
  __shared__ uint32_t h[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += kSortThreads) h[i] = 0;
  __syncthreads();
  const int64_t n = count.get();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const int lane = threadIdx.x & 31;
  if (base < n) {
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
      const int64_t g = base + i;
      const bool valid = g < n;
      const int d = valid ? digit_of(keys[g], shift, mask) : 0;
      const unsigned peers = digit_peers(d, valid, bits);
      if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
    hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// fused = 1: `offsets` holds the raw digit-major histogram (ntiles <= kFusedTiles)
// and each block derives its own output offsets from it.
template <class V, bool kVals>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint64_t* __restrict__ keys_in, uint64_t* __restrict__ keys_out,
    const V* __restrict__ vals_in, V* __restrict__ vals_out, DevCount count, int shift,
    uint32_t mask, int bits, const uint64_t* __restrict__ offsets, int64_t ntiles, int fused) {
  __shared__ uint32_t whist[kSortWarps][kRadix];
  __shared__ uint64_t tile_base[kRadix];
  __shared__ uint64_t sm_scan[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = count.get();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base >= n) return;  // uniform over the block
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads)
    (&whist[0][0])[i] = 0;
  if (fused) {
    // thread d: total of digit d over all tiles, and over the tiles before this one
    const int d = threadIdx.x;  // kSortThreads == kRadix
    uint64_t tot = 0, pre = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
      const uint64_t v = offsets[(int64_t)d * ntiles + t];
      tot += v;
      if (t < blockIdx.x) pre += v;
    }
    uint64_t bt;
    const uint64_t inc = block_inclusive_scan(tot, sm_scan, &bt);
    tile_base[d] = inc - tot + pre;
  } else {
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
      tile_base[d] = offsets[(int64_t)d * ntiles + blockIdx.x];
  }
  __syncthreads();

  uint64_t k[kSortItems];
  V v[kSortItems];
  uint32_t rank[kSortItems];
  int dg[kSortItems];
  const int64_t wbase = base + (int64_t)warp * (kSortItems * 32);
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int64_t g = wbase + i * 32 + lane;
    const bool valid = g < n;
    k[i] = valid ? keys_in[g] : 0ull;
    if (kVals) v[i] = valid ? vals_in[g] : V(0);
    const int d = valid ? digit_of(k[i], shift, mask) : kRadix;
    dg[i] = d;
    const unsigned peers = digit_peers(d, valid, bits);
    const uint32_t before = valid ? whist[warp][d] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) whist[warp][d] += (uint32_t)__popc(peers);
    __syncwarp();
    rank[i] = before + (uint32_t)__popc(peers & lt_mask);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t t = whist[w][d];
      whist[w][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    if (dg[i] < kRadix) {
      const uint64_t pos = tile_base[dg[i]] + whist[warp][dg[i]] + rank[i];
      keys_out[pos] = k[i];
      if (kVals) vals_out[pos] = v[i];
    }
  }
}

}  // namespace

size_t scan_workspace(int64_t n_max) {
  const int64_t ntiles = ceil_div(n_max > 0 ? n_max : 1, kScanTile);
  return (size_t)(ntiles + 1) * sizeof(uint64_t) + 256;
}

template <class T>
int scan_u64(const T* in, uint64_t* out, DevCount count, bool inclusive, uint64_t* total,
             void* scratch, cudaStream_t st, ScanExtras ex) {
  const int64_t ntiles = ceil_div(count.max > 0 ? count.max : 1, kScanTile);
  uint64_t* tile_sums = reinterpret_cast<uint64_t*>(scratch);
  // the non-fused path keeps the total in scratch when the caller gives none
  uint64_t* tot = total ? total : tile_sums + ntiles;
  k_scan_tile_sums<T><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, count, tile_sums);
  if (ntiles <= kFusedTiles) {
    // the tile kernel sums its predecessors' totals itself (and writes the total)
    k_scan_tiles<T><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, count, tile_sums,
                                                                inclusive ? 1 : 0, 1, total,
                                                                ex.end ? 1 : 0, ex.ratio);
  } else {
    k_scan_tile_offsets<<<1, kScanThreads, 0, st>>>(tile_sums, ntiles, tot);
    k_scan_tiles<T><<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, out, count, tile_sums,
                                                                inclusive ? 1 : 0, 0, tot,
                                                                ex.end ? 1 : 0, ex.ratio);
  }
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

template int scan_u64<uint64_t>(const uint64_t*, uint64_t*, DevCount, bool, uint64_t*, void*,
                                 cudaStream_t, ScanExtras);
template int scan_u64<uint32_t>(const uint32_t*, uint64_t*, DevCount, bool, uint64_t*, void*,
                                 cudaStream_t, ScanExtras);

size_t sort_workspace(int64_t n_max) {
  const int64_t ntiles = ceil_div(n_max > 0 ? n_max : 1, kSortTile);
  const int64_t nh = ntiles * kRadix;
  return (size_t)nh * sizeof(uint64_t) + 256 + scan_workspace(nh);
}

template <class V>
int radix_sort(uint64_t* keys, uint64_t* keys_alt, V* vals, V* vals_alt, DevCount count,
               int begin_bit, int end_bit, void* scratch, cudaStream_t st, int* in_alt) {
  *in_alt = 0;
  if (count.max <= 0 || end_bit <= begin_bit) return CPA_OK;
  const int64_t ntiles = ceil_div(count.max, kSortTile);
  const int64_t nh = ntiles * kRadix;
  uint64_t* hist = reinterpret_cast<uint64_t*>(scratch);
  void* scan_scratch = reinterpret_cast<char*>(scratch) + (((size_t)nh * 8 + 255) & ~size_t(255));
  uint64_t* src_k = keys;
  uint64_t* dst_k = keys_alt;
  V* src_v = vals;
  V* dst_v = vals_alt;
  int alt = 0;
  const int fused = ntiles <= kFusedTiles ? 1 : 0;
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    const int w = end_bit - shift < 8 ? end_bit - shift : 8;
    const uint32_t mask = (1u << w) - 1u;
    k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, st>>>(src_k, count, shift, mask, w, hist,
                                                            ntiles);
    if (!fused)
      CPA_TRY(scan_u64<uint64_t>(hist, hist, DevCount{nullptr, nh}, false, nullptr, scan_scratch,
                                 st));
    if (vals)
      k_radix_scatter<V, true><<<(unsigned)ntiles, kSortThreads, 0, st>>>(
          src_k, dst_k, src_v, dst_v, count, shift, mask, w, hist, ntiles, fused);
    else
      k_radix_scatter<V, false><<<(unsigned)ntiles, kSortThreads, 0, st>>>(
          src_k, dst_k, nullptr, nullptr, count, shift, mask, w, hist, ntiles, fused);
    CPA_LAUNCH_CHECK();
    uint64_t* tk = src_k;
    src_k = dst_k;
    dst_k = tk;
    V* tv = src_v;
    src_v = dst_v;
    dst_v = tv;
    alt ^= 1;
  }
  *in_alt = alt;
  return CPA_OK;
}

template int radix_sort<uint64_t>(uint64_t*, uint64_t*, uint64_t*, uint64_t*, DevCount, int, int,
                                  void*, cudaStream_t, int*);
template int radix_sort<uint32_t>(uint64_t*, uint64_t*, uint32_t*, uint32_t*, DevCount, int, int,
                                  void*, cudaStream_t, int*);

}  // namespace cpa
