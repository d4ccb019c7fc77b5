// KrpSamp, TnsrSamp and the sampled normal-equation products (Section 5.2, 5.3).
#pragma once

#include "dense.cuh"

namespace cpa {

// Factor matrices indexed by mode, of the element type of the run (float or double).
struct FactorPtrs {
  const void* A[kMaxOrder];
};

// Buffers of the reproducible FP64 sampled MTTKRP (mttkrp_det.cu) for up to s samples
// and cap sampled nonzeros (cap = 0: not used).
struct DetBuffers {
  int64_t cap = 0;
  uint64_t *keys = nullptr, *keys_alt = nullptr;  // cap: i_k | j << 32, then sorted by i_k
  uint64_t *vals = nullptr, *vals_alt = nullptr;  // cap: the values as FP64 bit patterns
  void* sort_ws = nullptr;
  void* scan_ws = nullptr;
  uint64_t* off = nullptr;    // s + 1 item offsets
  uint64_t* los = nullptr;    // s fibre starts
  uint32_t* len = nullptr;    // s fibre lengths
  uint64_t* total = nullptr;  // sampled nonzeros of the update (device)
  double* U = nullptr;        // s x r: u_j = w_j^2 prod_t A_{m_t}(i_t, :)
  double* carry = nullptr;    // per tile of sorted items: head and tail partial rows
  int64_t* crow = nullptr;
  int* cmid = nullptr;
};
constexpr int kDetTile = 128;                 // sorted items per tile
constexpr int64_t kDetMaxItems = 1ll << 24;   // largest tensor (nonzeros) of the reproducible path

// Device buffers of one sampled MTTKRP for up to s samples.
struct MttkrpBuffers {
  uint64_t* ctr;     // kMttkrpCounters: sampled nonzeros, chunk counter, heavy-list
                     // length, spare, then per row slab its chunk counter, heavy-list
                     // length and heavy-piece counter
  uint64_t* total;   // = ctr: nnz of the sampled right-hand side
  uint32_t* heavy;   // 4 s (16 s with row slabs): (sample, start lo/hi words, length) of
                     // long fibres (row slabs: pieces of long slab ranges)
  // row-slab path (null when no mode's M exceeds one slab): per sample u_j
  // (s x r, run element type), fibre start, and the start of each slab's rows
  // within the fibre (s x 32 u32, slab p at column p, the fibre length at column P)
  void* U = nullptr;
  uint64_t* los = nullptr;
  uint32_t* bnd = nullptr;
  // sticky status word of the run (device; null: a word of ctr) for kernels that can
  // time out (the tensor-core Gram's bounded waits)
  int* status = nullptr;
  // block-ordered sums of the sampled Gram (its ticket is a word of ctr)
  BlockSums gsums;
  // the reproducible FP64 path (det.cap > 0: used for M in FP64 runs)
  DetBuffers det;
};
constexpr int kMttkrpCounters = 6 + 3 * 32;  // words kMttkrpCounters - 2 and - 1: Gram ticket, status
constexpr int kSlabMax = 31;  // most row slabs of one M

// Bytes of M per row slab for ftb-byte elements (96 MB for FP32, 256 MB for FP64, or
// CPA_MTTKRP_SLAB_BYTES; 0 = no slabs): M larger than this is accumulated slab by
// slab, the additions of a pass confined to one slab of rows.
size_t mttkrp_slab_bytes(int ftb);
// Number of row slabs of an n_k x r M of ftb-byte elements (1: no slabs).
int mttkrp_slabs(int64_t nk, int r, int ftb);

void mttkrp_buffers_carve(Arena& a, int64_t s, int r, int ftb, bool slabs, MttkrpBuffers* B,
                          int64_t det_cap = 0);

// Sampled nonzeros the reproducible FP64 path must hold for X (0: X is too large for
// it, or the run is not FP64; M is then accumulated with atomics).
int64_t det_capacity(const cpa_index* X, int precision);
void det_buffers_carve(Arena& a, int64_t s, int r, int64_t cap, DetBuffers* B);
// M (zeroed by the caller) = the sampled MTTKRP in FP64, every sum in a fixed order;
// ctr[0] += sampled nonzeros.
// fold (may be null): the rows summed are u_j F (the solve folded in, see
// sampled_mttkrp_fold).
int mttkrp_det(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx, const double* wgt,
               DevCount sbar, double* M, unsigned long long* ctr, DetBuffers& B, cudaStream_t st,
               const SmallFactor* fold = nullptr);

// Modes of at least this many rows (CPA_FOLD_ROWS overrides; 0 never) take the
// update with the solve folded into the sampled MTTKRP.
int64_t fold_rows();
// Row stride of the accumulation buffer of a folded update: r, rounded up to a
// multiple of 4 for FP32 (16-byte rows for the 16-byte atomics).
inline int fold_ldm(int r, int ftb) { return ftb == 4 ? (r + 3) & ~3 : r; }

// The update of mode k with the normal-equation solve folded in (Alg. 3: A_k =
// argmin ||Z~ A^T - X~^T||): the sampled Gram G (FP64) first, its factor into *fac
// (inverse, or pseudo-inverse with CPA_WARN_SINGULAR_GRAM in *warn), then
// A (n_k x ldm, unnormalised, zeroed here) = X~_(k) (U~ Fs) with U~ the weighted
// sampled Khatri-Rao rows: the same A as M G^-1 without the n_k r^2 solve.
// ev (may be null): events recorded before the Gram and after its factorisation.
template <class FT>
int sampled_mttkrp_fold(const cpa_index* X, int k, const FactorPtrs& F, int r, const uint64_t* idx_packed,
                        const double* wgt, DevCount sbar, FT* A, int ldm, double* G, SmallFactor* fac, int* warn,
                        MttkrpBuffers& B, cudaStream_t st, cudaEvent_t* ev = nullptr);

// A side stream and two events (created without timing) with which the Gram and the
// MTTKRP run as two branches; aux = null runs them one after the other.
struct Fork {
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// G = sum_j y_j y_j^T and M = sum_j wgt_j x(:, key_j) y_j^T over the sbar samples
// (packed keys), with y_j = wgt_j prod_t A_{m_t}(i_t, :), i.e. the sampled normal
// equations of Section 5.3; M, G and B.ctr are cleared here and *B.total receives
// the number of sampled nonzeros.  sbar: device count (max s, the size B was carved for).
// ev (may be null): two timing events recorded on `st` before and after the Gram
// kernel (the branches then run one after the other on `st`).
// FT: element type of the factors and M (double: FP64 path; float: mixed).
template <class FT>
int sampled_mttkrp(const cpa_index* X, int k, const FactorPtrs& F, int r,
                   const uint64_t* idx_packed, const double* wgt, DevCount sbar, FT* M,
                   double* G, MttkrpBuffers& B, cudaStream_t st, cudaEvent_t* ev = nullptr,
                   const Fork* fork = nullptr);

}  // namespace cpa
