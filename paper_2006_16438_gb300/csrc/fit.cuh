// Exact fit of Eq. 5.1 on the GPU.
#pragma once

#include "mttkrp.cuh"

namespace cpa {

size_t fit_buffers_bytes(int D, int r);
// Enqueue the fit of [[lambda; A_1..A_D]] against X; result in *fit_dev (device).
// scratch: fit_buffers_bytes(D, r) bytes of device memory.
template <class FT>
int fit_enqueue(const cpa_index* X, const FactorPtrs& F, const double* lambda, int r, double* scratch,
                double* fit_dev, cudaStream_t st);

}  // namespace cpa
