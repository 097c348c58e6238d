// Porosity field from a permeability field (Sec. 2.1, Eq. lattice_porosity).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// gamma[i] = clamp(1 - nu_tau / K[i], 0, 1) for n cells; K of dtype kdtype (LBM_DTYPE_*), gamma of
// the compute type (celem bytes). One launch on stream s.
void porous_gamma(const void* K, int kdtype, void* gamma, int celem, long long n, double nu_tau, cudaStream_t s);

}  // namespace lbm
