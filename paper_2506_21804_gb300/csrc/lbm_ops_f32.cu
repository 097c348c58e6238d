// Kernel instantiations for population storage type float.
#include "lbm_impl.cuh"

namespace lbm {
const Ops* ops_f32(int q) {
  if (q == 19) return Impl<19, float>::table();
  if (q == 27) return Impl<27, float>::table();
  return nullptr;
}
}  // namespace lbm
