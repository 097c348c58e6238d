// Kernel instantiations for population storage type double.
#include "lbm_impl.cuh"

namespace lbm {
const Ops* ops_f64(int q) {
  if (q == 19) return Impl<19, double>::table();
  if (q == 27) return Impl<27, double>::table();
  return nullptr;
}
}  // namespace lbm
