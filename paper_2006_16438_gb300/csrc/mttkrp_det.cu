// Reproducible FP64 sampled MTTKRP (KrpSamp + TnsrSamp of Section 5.3): the same M as
// the atomic kernels of mttkrp.cu, with every sum taken in one fixed order, so two
// runs give M bit for bit (and with it the factors, leverage scores and samples of
// all later iterations).
//
//   1. k_det_prep: per kept sample j its fibre [lo_j, lo_j + len_j) in the mode-k
//      index (probe) and u_j = w_j^2 prod_t A_{m_t}(i_t, :) (FP64).
//   2. scan: item offsets off_j = sum_{j' < j} len_j' (the sampled nonzeros listed in
//      sample order, each fibre's nonzeros in their index order).
//   3. k_det_expand: item p -> key (i_k | j << 32), value x (FP64 bits); one thread
//      per item, its sample found by bisection of the offsets.
//   4. stable radix sort by i_k: a row's items keep ascending j.
//   5. k_det_tiles: fixed tiles of kDetTile sorted items, a warp each (lane c holds
//      column c); a row's items are summed in order in four interleaved chains
//      (item q of the row's run in the tile feeds chain q % 4; the chains are added
//      as (c0 + c1) + (c2 + c3)).  Rows inside one tile are written to M; the parts of
//      a row that crosses tile boundaries are stored as carries.
//   6. k_det_fixup: for each row that crosses a boundary, the tile where it starts
//      adds its carry and the following tiles' carries in tile order.
// The tiles depend on the item count only, never on the SM count.
#include <stdlib.h>

#include "mttkrp.cuh"

namespace cpa {

namespace {

constexpr int kThreads = 256;

// Per sample: fibre start and length, and u_j.  A warp takes 32 consecutive samples
// (lane l probes sample l), then forms the u rows one sample at a time (lane c holds
// column c).  The sampled-nonzero count is added to ctr[0].
template <class VT, int CPL>
__global__ void __launch_bounds__(kThreads) k_det_prep(FibreIndex<VT> X, FactorPtrs F, KeyLayout L, int r,
                                                       const uint64_t* __restrict__ idx,
                                                       const double* __restrict__ wgt, DevCount sbar,
                                                       double* __restrict__ U, uint64_t* __restrict__ los,
                                                       uint32_t* __restrict__ len_out,
                                                       unsigned long long* __restrict__ ctr,
                                                       const SmallFactor* __restrict__ fold) {
  __shared__ double Fs[kMaxRank * kMaxRank];
  if (fold) {
    for (int i = threadIdx.x; i < r * r; i += blockDim.x) Fs[i] = fold->F[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int64_t n = sbar.get();
  const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
  uint64_t my_nnz = 0;
  for (int64_t base = gw * 32; base < n; base += nw * 32) {
    const int64_t j = base + lane;
    uint64_t key = 0, lo = 0, hi = 0;
    double w = 0.0;
    if (j < n) {
      key = idx[j];
      X.probe(key, &lo, &hi);
      w = wgt[j];
      los[j] = lo;
      len_out[j] = (uint32_t)(hi - lo);
    }
    my_nnz += hi - lo;
    const int cnt = (int)(n - base < 32 ? n - base : 32);
    for (int q = 0; q < cnt; ++q) {
      const int64_t jq = base + q;
      const uint64_t kq = __shfl_sync(0xffffffffu, key, q);
      const double wq = __shfl_sync(0xffffffffu, w, q);
      double zr[CPL];
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int c = lane + 32 * v;
        double z = 0.0;
        if (c < r) {
          z = wq * wq;
          for (int t = 0; t < L.d; ++t)
            z *= static_cast<const double*>(F.A[L.mode[t]])[(int64_t)L.get(kq, t) * r + c];
        }
        zr[v] = z;
      }
      if (fold) {  // v_c = sum_u z_u Fs(u, c) in the order u = 0..r-1
        double acc[CPL];
#pragma unroll
        for (int v = 0; v < CPL; ++v) acc[v] = 0.0;
#pragma unroll
        for (int h = 0; h < CPL; ++h)
          for (int uu = 0; uu < 32; ++uu) {
            const int u = 32 * h + uu;
            const double zu = __shfl_sync(0xffffffffu, zr[h], uu);
            if (u < r) {
#pragma unroll
              for (int v = 0; v < CPL; ++v) {
                const int c = lane + 32 * v;
                if (c < r) acc[v] = fma(zu, Fs[u * r + c], acc[v]);
              }
            }
          }
#pragma unroll
        for (int v = 0; v < CPL; ++v) zr[v] = acc[v];
      }
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int c = lane + 32 * v;
        if (c < r) U[jq * r + c] = zr[v];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) my_nnz += __shfl_xor_sync(0xffffffffu, my_nnz, o);
  if (lane == 0 && my_nnz) atomicAdd(&ctr[0], (unsigned long long)my_nnz);
}

// Item p of the sample-ordered list: its sample j (largest j with off[j] <= p among
// the n samples), the nonzero e = los[j] + p - off[j]; key = i_k | j << 32.
template <class VT>
__global__ void __launch_bounds__(kThreads) k_det_expand(FibreIndex<VT> X, DevCount sbar,
                                                         const uint64_t* __restrict__ off,
                                                         const uint64_t* __restrict__ los,
                                                         DevCount items, uint64_t* __restrict__ keys,
                                                         uint64_t* __restrict__ vals) {
  const int64_t n = sbar.get();
  const int64_t total = items.get();
  for (int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x; p < total; p += (int64_t)gridDim.x * kThreads) {
    int64_t a = 0, z = n;  // off[a] <= p < off[z] (off[n] = total)
    while (z - a > 1) {
      const int64_t mid = a + ((z - a) >> 1);
      if ((int64_t)off[mid] <= p) a = mid; else z = mid;
    }
    const uint64_t e = los[a] + (uint64_t)(p - (int64_t)off[a]);
    keys[p] = (uint64_t)(uint32_t)X.ik[e] | ((uint64_t)a << 32);
    vals[p] = (uint64_t)__double_as_longlong((double)X.value(e));
  }
}

__device__ __forceinline__ int64_t item_row(uint64_t key) { return (int64_t)(uint32_t)key; }

// Carries of tile t: slot 0 = the head (the tile's first row, when that row began in
// an earlier tile), slot 1 = the tail (the tile's last row, when it began in this tile
// and continues in the next).  crow[2 t + s] = the row, or -1 for none; cmid[t] = 1
// when the whole tile is one row that also continues in the next tile (its sum is in
// the head slot).
template <int CPL>
__global__ void __launch_bounds__(kThreads) k_det_tiles(const uint64_t* __restrict__ keys,
                                                        const uint64_t* __restrict__ vals, DevCount items,
                                                        const double* __restrict__ U, int r,
                                                        double* __restrict__ M, double* __restrict__ carry,
                                                        int64_t* __restrict__ crow, int* __restrict__ cmid) {
  const int lane = threadIdx.x & 31;
  const int64_t total = items.get();
  const int64_t ntiles = (total + kDetTile - 1) / kDetTile;
  const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t t = gw; t < ntiles; t += nw) {
    const int64_t b = t * kDetTile;
    const int64_t e = b + kDetTile < total ? b + kDetTile : total;
    const int64_t prev_row = b > 0 ? item_row(keys[b - 1]) : -1;
    const int64_t next_row = e < total ? item_row(keys[e]) : -1;
    double c0[CPL], c1[CPL], c2[CPL], c3[CPL];
#pragma unroll
    for (int v = 0; v < CPL; ++v) c0[v] = c1[v] = c2[v] = c3[v] = 0.0;
    int64_t cur = -1, run = 0;
    bool head = true;  // the current run is the tile's first
    int64_t out_head = -1, out_tail = -1;
    int mid = 0;
    auto flush = [&](bool at_end) {
      double s[CPL];
#pragma unroll
      for (int v = 0; v < CPL; ++v) s[v] = (c0[v] + c1[v]) + (c2[v] + c3[v]);
      const bool from_before = head && cur == prev_row;
      const bool into_next = at_end && cur == next_row;
      int slot = -1;
      if (from_before) {
        slot = 0;
        out_head = cur;
        if (into_next) mid = 1;
      } else if (into_next) {
        slot = 1;
        out_tail = cur;
      }
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int c = lane + 32 * v;
        if (c < r) {
          if (slot < 0) M[cur * r + c] = s[v];
          else carry[((size_t)t * 2 + slot) * r + c] = s[v];
        }
        c0[v] = c1[v] = c2[v] = c3[v] = 0.0;
      }
      head = false;
    };
    for (int64_t g = b; g < e; g += 32) {
      const int nb = (int)(e - g < 32 ? e - g : 32);
      uint64_t kl = 0, vl = 0;
      if (lane < nb) {
        kl = keys[g + lane];
        vl = vals[g + lane];
      }
      // eight items at a time: their factor rows are loaded before any is added
      for (int q0 = 0; q0 < nb; q0 += 8) {
        uint64_t kb[8];
        double xb[8], ub[8][CPL];
#pragma unroll
        for (int t8 = 0; t8 < 8; ++t8) {
          const int q = q0 + t8 < nb ? q0 + t8 : nb - 1;
          kb[t8] = __shfl_sync(0xffffffffu, kl, q);
          xb[t8] = __longlong_as_double((long long)__shfl_sync(0xffffffffu, vl, q));
          const int64_t j = (int64_t)(kb[t8] >> 32);
#pragma unroll
          for (int v = 0; v < CPL; ++v) {
            const int c = lane + 32 * v;
            ub[t8][v] = c < r ? U[j * r + c] : 0.0;
          }
        }
#pragma unroll
        for (int t8 = 0; t8 < 8; ++t8) {
          if (q0 + t8 >= nb) break;
          const int64_t row = item_row(kb[t8]);
          if (row != cur) {
            if (cur >= 0) flush(false);
            cur = row;
            run = 0;
          }
          const int ch = (int)(run & 3);
#pragma unroll
          for (int v = 0; v < CPL; ++v) {
            const double x = xb[t8], u = ub[t8][v];
            if (ch == 0) c0[v] = fma(x, u, c0[v]);
            else if (ch == 1) c1[v] = fma(x, u, c1[v]);
            else if (ch == 2) c2[v] = fma(x, u, c2[v]);
            else c3[v] = fma(x, u, c3[v]);
          }
          ++run;
        }
      }
    }
    if (cur >= 0) flush(true);
    if (lane == 0) {
      crow[2 * t] = out_head;
      crow[2 * t + 1] = out_tail;
      cmid[t] = mid;
    }
  }
}

// One warp per tile with a tail: the row's sum is the tail, then the heads of the
// following tiles in order, up to the first tile where the row ends.
template <int CPL>
__global__ void __launch_bounds__(kThreads) k_det_fixup(DevCount items, const double* __restrict__ carry,
                                                        const int64_t* __restrict__ crow,
                                                        const int* __restrict__ cmid, int r,
                                                        double* __restrict__ M) {
  const int lane = threadIdx.x & 31;
  const int64_t total = items.get();
  const int64_t ntiles = (total + kDetTile - 1) / kDetTile;
  const int64_t gw = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t t = gw; t < ntiles; t += nw) {
    const int64_t row = crow[2 * t + 1];
    if (row < 0) continue;
    double s[CPL];
#pragma unroll
    for (int v = 0; v < CPL; ++v) {
      const int c = lane + 32 * v;
      s[v] = c < r ? carry[((size_t)t * 2 + 1) * r + c] : 0.0;
    }
    for (int64_t u = t + 1; u < ntiles; ++u) {
      if (crow[2 * u] != row) break;  // cannot happen: the next tile starts with this row
#pragma unroll
      for (int v = 0; v < CPL; ++v) {
        const int c = lane + 32 * v;
        if (c < r) s[v] += carry[((size_t)u * 2) * r + c];
      }
      if (!cmid[u]) break;
    }
#pragma unroll
    for (int v = 0; v < CPL; ++v) {
      const int c = lane + 32 * v;
      if (c < r) M[row * r + c] = s[v];
    }
  }
}

unsigned grid_for(int64_t work_items, int per_block) {
  int64_t g = (work_items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  const int64_t cap = 1216;  // fixed: independent of the SM count
  return (unsigned)(g < cap ? g : cap);
}

}  // namespace

void det_buffers_carve(Arena& a, int64_t s, int r, int64_t cap, DetBuffers* B) {
  B->cap = cap;
  if (cap <= 0) {
    *B = DetBuffers();
    return;
  }
  const size_t ss = (size_t)(s > 0 ? s : 1);
  const int64_t ntiles = (cap + kDetTile - 1) / kDetTile + 1;
  B->keys = a.take<uint64_t>(cap);
  B->keys_alt = a.take<uint64_t>(cap);
  B->vals = a.take<uint64_t>(cap);
  B->vals_alt = a.take<uint64_t>(cap);
  B->sort_ws = a.take<char>(sort_workspace(cap));
  B->scan_ws = a.take<char>(scan_workspace((int64_t)ss + 1));
  B->off = a.take<uint64_t>(ss + 1);
  B->los = a.take<uint64_t>(ss);
  B->len = a.take<uint32_t>(ss);
  B->total = a.take<uint64_t>(1);
  B->U = a.take<double>(ss * r);
  B->carry = a.take<double>((size_t)ntiles * 2 * r);
  B->crow = a.take<int64_t>((size_t)ntiles * 2);
  B->cmid = a.take<int>((size_t)ntiles);
}

int64_t det_capacity(const cpa_index* X, int precision) {
  if (precision != CPA_FP64) return 0;
  if (const char* e = getenv("CPA_DET_MTTKRP"))  // 0: FP64 atomics whatever the size (tests)
    if (atoi(e) == 0) return 0;
  return X->nnz > 0 && X->nnz <= kDetMaxItems ? X->nnz : 0;
}

int mttkrp_det(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx, const double* wgt,
               DevCount sbar, double* M, unsigned long long* ctr, DetBuffers& B, cudaStream_t st,
               const SmallFactor* fold) {
  if (B.cap <= 0) return CPA_ERR_ARG;
  const KeyLayout& L = X->mode[k].L;
  const int64_t nk = X->dims[k];
  const int rowbits = ceil_log2(nk);
  const DevCount items{reinterpret_cast<const int64_t*>(B.total), B.cap};
  CPA_TRY(with_value_type(X, [&](auto tag) -> int {
    using VT = decltype(tag);
    const FibreIndex<VT> fx = fibre_view<VT>(X, k);
    const unsigned gp = grid_for(sbar.max, kThreads);
    if (r <= 32)
      k_det_prep<VT, 1><<<gp, kThreads, 0, st>>>(fx, F, L, r, idx, wgt, sbar, B.U, B.los, B.len, ctr, fold);
    else
      k_det_prep<VT, 2><<<gp, kThreads, 0, st>>>(fx, F, L, r, idx, wgt, sbar, B.U, B.los, B.len, ctr, fold);
    CPA_LAUNCH_CHECK();
    ScanExtras ex;
    ex.end = true;
    CPA_TRY(scan_u64<uint32_t>(B.len, B.off, sbar, false, B.total, B.scan_ws, st, ex));
    k_det_expand<VT><<<grid_for(B.cap, kThreads), kThreads, 0, st>>>(fx, sbar, B.off, B.los, items, B.keys,
                                                                         B.vals);
    CPA_LAUNCH_CHECK();
    return CPA_OK;
  }));
  int in_alt = 0;
  CPA_TRY(radix_sort<uint64_t>(B.keys, B.keys_alt, B.vals, B.vals_alt, items, 0, rowbits, B.sort_ws, st, &in_alt));
  const uint64_t* sk = in_alt ? B.keys_alt : B.keys;
  const uint64_t* sv = in_alt ? B.vals_alt : B.vals;
  const int64_t ntiles = (B.cap + kDetTile - 1) / kDetTile;
  const unsigned gt = grid_for(ntiles, kThreads / 32);
  if (r <= 32) {
    k_det_tiles<1><<<gt, kThreads, 0, st>>>(sk, sv, items, B.U, r, M, B.carry, B.crow, B.cmid);
    k_det_fixup<1><<<gt, kThreads, 0, st>>>(items, B.carry, B.crow, B.cmid, r, M);
  } else {
    k_det_tiles<2><<<gt, kThreads, 0, st>>>(sk, sv, items, B.U, r, M, B.carry, B.crow, B.cmid);
    k_det_fixup<2><<<gt, kThreads, 0, st>>>(items, B.carry, B.crow, B.cmid, r, M);
  }
  CPA_LAUNCH_CHECK();
  return CPA_OK;
}

}  // namespace cpa
