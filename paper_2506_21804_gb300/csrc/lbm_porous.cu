// Porous-medium inputs (Sec. 2.1): the Forchheimer permeability of a measured sample and the
// lattice porosity of Eq. lattice_porosity from a per-cell permeability field.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/lbm.h"
#include "lbm_porous.h"

namespace lbm {
namespace {

// gamma = clamp(1 - nu tau / K, 0, 1) (lattice units, dx = 1; K = +inf gives 1, K <= 0 or NaN gives 0).
// K of dtype KT, gamma in the compute type C.
template <class KT, class C>
__global__ void k_perm_gamma(const KT* K, C* gamma, long long n, double nu_tau) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double k = double(K[i]);
  // K = +inf: fluid; K <= 0 or NaN (no valid permeability): impermeable
  double g = isinf(k) && k > 0.0 ? 1.0 : (k > 0.0 ? 1.0 - nu_tau / k : 0.0);
  g = g < 0.0 ? 0.0 : (g > 1.0 ? 1.0 : g);
  gamma[i] = C(g);
}

}  // namespace

void porous_gamma(const void* K, int kdtype, void* gamma, int celem, long long n, double nu_tau, cudaStream_t s) {
  const unsigned g = unsigned((n + 255) / 256);
  if (kdtype == LBM_DTYPE_F64) {
    if (celem == 8) k_perm_gamma<double, double><<<g, 256, 0, s>>>(static_cast<const double*>(K), static_cast<double*>(gamma), n, nu_tau);
    else k_perm_gamma<double, float><<<g, 256, 0, s>>>(static_cast<const double*>(K), static_cast<float*>(gamma), n, nu_tau);
  } else {
    if (celem == 8) k_perm_gamma<float, double><<<g, 256, 0, s>>>(static_cast<const float*>(K), static_cast<double*>(gamma), n, nu_tau);
    else k_perm_gamma<float, float><<<g, 256, 0, s>>>(static_cast<const float*>(K), static_cast<float*>(gamma), n, nu_tau);
  }
}

}  // namespace lbm

extern "C" double lbm_forchheimer_permeability(double mu, double Q, double A, double L, double dP, double rho, double K_beta) {
  const double inertial = std::isinf(K_beta) ? 0.0 : rho / K_beta * Q * Q / (A * A);
  const double br = dP / L - inertial;
  if (!(br > 0.0) || !(A > 0.0) || !(L > 0.0)) return NAN;
  return mu * Q / (A * br);
}
