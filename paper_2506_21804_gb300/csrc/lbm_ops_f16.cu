// Kernel instantiations for population storage type __half.
#include "lbm_impl.cuh"

namespace lbm {
const Ops* ops_f16(int q) {
  if (q == 19) return Impl<19, __half>::table();
  if (q == 27) return Impl<27, __half>::table();
  return nullptr;
}
}  // namespace lbm
