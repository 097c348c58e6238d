// Kernel instantiations for population storage type __nv_bfloat16.
#include "lbm_impl.cuh"

namespace lbm {
const Ops* ops_bf16(int q) {
  if (q == 19) return Impl<19, __nv_bfloat16>::table();
  if (q == 27) return Impl<27, __nv_bfloat16>::table();
  return nullptr;
}
}  // namespace lbm
