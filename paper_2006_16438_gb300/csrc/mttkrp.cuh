// KrpSamp, TnsrSamp and the sampled normal-equation products (Section 5.2, 5.3).
#pragma once

#include "dense.cuh"

namespace cpa {

// Factor matrices indexed by mode, of the element type of the run (float or double).
struct FactorPtrs {
  const void* A[kMaxOrder];
};

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
};
constexpr int kMttkrpCounters = 4 + 3 * 32;
constexpr int kSlabMax = 31;  // most row slabs of one M

// Bytes of M per row slab (128 MB, or CPA_MTTKRP_SLAB_BYTES; 0 = no slabs): M
// larger than this is accumulated slab by slab, the additions of a pass confined to
// one slab of rows.
size_t mttkrp_slab_bytes();
// Number of row slabs of an n_k x r M of ftb-byte elements (1: no slabs).
int mttkrp_slabs(int64_t nk, int r, int ftb);

void mttkrp_buffers_carve(Arena& a, int64_t s, int r, int ftb, bool slabs, MttkrpBuffers* B);

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
