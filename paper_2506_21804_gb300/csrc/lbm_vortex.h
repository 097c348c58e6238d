// Vortex-method inlet (Sec. 2.2.2): arguments of the per-step update of the inlet velocity field.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

struct VmArgs {
  int ny, nz;          // inlet plane
  int n;               // vortices per step
  double sigma;        // vortex size (cells)
  double I;            // turbulence intensity
  uint64_t seed;       // random-number key
  long long t;         // step counter (random-number counter)
  long long area;      // number of INFLOW cells
  double gden;         // 6 ln 3 - 9 ln 2, formed on the host
  const void* mean;    // compute type [3][ny*nz]: mean inlet profile
  const void* prev;    // compute type [3][ny*nz]: inlet field of the previous step
  void* cur;           // compute type [3][ny*nz]: inlet field of this step (written)
  void* vort;          // compute type [3*n]: y, z, Gamma of this step's vortices (written)
  void* part;          // compute type [2*ceil(n/VM_CHUNK)][ny*nz]: per-chunk partial fields (scratch)
};

constexpr int VM_CHUNK = 32;  // vortices per partial sum

// Three launches on stream s: the vortices of step t, the per-chunk partial fields, the inlet field.
// celem = 4 or 8.
void vm_update(const VmArgs& v, int celem, cudaStream_t s);

}  // namespace lbm
