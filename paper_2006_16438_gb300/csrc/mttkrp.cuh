// KrpSamp, TnsrSamp and the sampled normal-equation products (Section 5.2, 5.3).
#pragma once

#include "dense.cuh"

namespace cpa {

// Factor matrices indexed by mode, of the element type of the run (float or double).
struct FactorPtrs {
  const void* A[kMaxOrder];
};

// Buffers of one sampled MTTKRP (device), sized for s samples.
struct MttkrpBuffers {
  void* Y;            // s x r (factor type): y_j = wgt_j * z_j
  uint64_t* lo;       // s: first nonzero of the fibre of sample j in the mode-k stream
  uint32_t* len;      // s: fibre length
  uint64_t* pos;      // s + 1: exclusive prefix of len; pos[sbar] = nnz of the sample
  uint64_t* total;    // 1: nnz of the sampled right-hand side
  char* scratch;      // scan workspace for s items
};

size_t mttkrp_buffers_bytes(int64_t s, int r, int ft_bytes);
void mttkrp_buffers_carve(Arena& a, int64_t s, int r, int ft_bytes, MttkrpBuffers* B);

// G = sum_j y_j y_j^T and M = sum_j wgt_j x(:, key_j) y_j^T over the sbar samples
// (packed keys), with y_j = wgt_j prod_t A_{m_t}(i_t, :); M and G are cleared here.
// sbar: device count (max s).
// ev (may be null): three timing events recorded on `st` after the probe, after
// the KRP/Gram kernel and after the scan (i.e. before the gather-scale-accumulate).
// FT: element type of the factors, Y and M (double: FP64 path; float: mixed).
template <class FT>
int sampled_mttkrp(const cpa_index* X, int k, const FactorPtrs& F, int r,
                   const uint64_t* idx_packed, const double* wgt, DevCount sbar, FT* M,
                   double* G, MttkrpBuffers& B, cudaStream_t st, cudaEvent_t* ev = nullptr);

}  // namespace cpa
