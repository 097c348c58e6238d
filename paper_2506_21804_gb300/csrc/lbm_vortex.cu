// Vortex-method turbulent inlet (Sec. 2.2.2): before each step, n seed points are drawn on the inlet
// plane with counter-based random numbers, each carries a circulation set by the local turbulent
// kinetic energy, and the inlet velocity of the step is the mean profile plus the in-plane field of
// the vortices plus a streamwise fluctuation from the linear kinematic (Langevin) model. The inlet
// boundary condition of the step then imposes this field.
//
//   k_i = 3/2 (|u_mean(p_i)| I)^2,   Gamma_i = 4 s_i sqrt(pi k_i A / ((6 ln 3 - 9 ln 2) n)),
//   u_v(x) = (1/2pi) sum_i Gamma_i ((p_i - x) x e_x) (1 - e^{-a}) e^{-a} / |p_i - x|^2,  a = |p_i - x|^2/(2 sigma^2),
//   u'_x = -(u_v . grad U)/|grad U|   (U: streamwise inlet velocity of the previous step),
//
// with A the number of INFLOW cells, positions uniform on [-1/2, ny - 1/2) x [-1/2, nz - 1/2) (cell
// centres at integer coordinates), k_i from the cell containing p_i, grad U by central differences
// over the plane positions (one-sided at the edges).
//
// Random numbers: the SplitMix64 output function (Steele, Lea, Flood 2014) of
// seed + (1 + counter) * 0x9E3779B97F4A7C15, top 53 bits scaled to [0, 1); counter of vortex i,
// component c (0: y, 1: z, 2: sign) at step t: (t n + i) 4 + c. Positions and circulations are
// formed in double precision with explicitly rounded operations (no contraction), the plane field
// in the compute type: partial sums over chunks of VM_CHUNK vortices (one CTA row per chunk), then
// their sum in chunk order (deterministic).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "lbm_vortex.h"

namespace lbm {
namespace {

__device__ __forceinline__ uint64_t sm64_out(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double sm64_uniform(uint64_t seed, uint64_t counter) {
  const uint64_t r = sm64_out(seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull);
  return __dmul_rn(double(r >> 11), 1.0 / 9007199254740992.0);
}

template <class C>
__global__ void k_vm_gen(const VmArgs v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const uint64_t base = (uint64_t(v.t) * uint64_t(v.n) + uint64_t(i)) * 4ull;
  const double y = __dadd_rn(-0.5, __dmul_rn(double(v.ny), sm64_uniform(v.seed, base + 0)));
  const double z = __dadd_rn(-0.5, __dmul_rn(double(v.nz), sm64_uniform(v.seed, base + 1)));
  const double sg = sm64_uniform(v.seed, base + 2) < 0.5 ? 1.0 : -1.0;
  int iy = int(floor(__dadd_rn(y, 0.5))), iz = int(floor(__dadd_rn(z, 0.5)));
  iy = iy < 0 ? 0 : (iy > v.ny - 1 ? v.ny - 1 : iy);
  iz = iz < 0 ? 0 : (iz > v.nz - 1 ? v.nz - 1 : iz);
  const long long pl = (long long)v.ny * v.nz, p = iy + (long long)v.ny * iz;
  const C* um = static_cast<const C*>(v.mean);
  double um2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double ua = double(um[a * pl + p]);
    um2 = __dadd_rn(um2, __dmul_rn(ua, ua));
  }
  const double k = __dmul_rn(__dmul_rn(__dmul_rn(1.5, um2), v.I), v.I);
  const double den = __dmul_rn(v.gden, double(v.n));
  const double gam = __dmul_rn(__dmul_rn(4.0, sg), sqrt(__ddiv_rn(__dmul_rn(__dmul_rn(M_PI, k), double(v.area)), den)));
  C* out = static_cast<C*>(v.vort);
  out[3 * i] = C(y);
  out[3 * i + 1] = C(z);
  out[3 * i + 2] = C(gam);
}

template <class C> __device__ __forceinline__ C vexp(C x) { return exp(x); }
template <> __device__ __forceinline__ float vexp<float>(float x) { return expf(x); }

constexpr int VM_THREADS = 256;

// Partial in-plane field of vortex chunk blockIdx.y (VM_CHUNK vortices) at every plane position.
template <class C>
__global__ void __launch_bounds__(VM_THREADS) k_vm_partial(const VmArgs v) {
  __shared__ C sv[3 * VM_CHUNK];
  const long long pl = (long long)v.ny * v.nz;
  const int c0 = blockIdx.y * VM_CHUNK;
  const int m = v.n - c0 < VM_CHUNK ? v.n - c0 : VM_CHUNK;
  const C* vort = static_cast<const C*>(v.vort);
  for (int j = threadIdx.x; j < 3 * m; j += blockDim.x) sv[j] = vort[3 * c0 + j];
  __syncthreads();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= pl) return;
  const C yc = C(int(p % v.ny)), zc = C(int(p / v.ny));
  const C inv2s2 = C(1) / (C(2) * C(v.sigma) * C(v.sigma));
  const C inv2pi = C(1.0 / (2.0 * M_PI));
  C uy = C(0), uz = C(0);
  for (int j = 0; j < m; ++j) {
    const C ry = sv[3 * j] - yc, rz = sv[3 * j + 1] - zc;
    const C r2 = ry * ry + rz * rz;
    if (r2 == C(0)) continue;
    const C e = vexp(-r2 * inv2s2);
    const C f = sv[3 * j + 2] * (C(1) - e) * e * inv2pi / r2;
    uy += f * rz;
    uz -= f * ry;
  }
  C* part = static_cast<C*>(v.part);
  part[(2 * (long long)blockIdx.y) * pl + p] = uy;
  part[(2 * (long long)blockIdx.y + 1) * pl + p] = uz;
}

// Sum of the chunk partials in chunk order, streamwise fluctuation, inlet field of the step.
template <class C>
__global__ void __launch_bounds__(VM_THREADS) k_vm_finish(const VmArgs v) {
  const long long pl = (long long)v.ny * v.nz;
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= pl) return;
  const int y = int(p % v.ny), z = int(p / v.ny);
  const C* part = static_cast<const C*>(v.part);
  const int nch = (v.n + VM_CHUNK - 1) / VM_CHUNK;
  C uy = C(0), uz = C(0);
  for (int c = 0; c < nch; ++c) {
    uy += part[(2 * (long long)c) * pl + p];
    uz += part[(2 * (long long)c + 1) * pl + p];
  }
  const C* U = static_cast<const C*>(v.prev);  // streamwise component first
  auto at = [&](int yy, int zz) { return U[yy + (long long)v.ny * zz]; };
  C gy = C(0), gz = C(0);
  if (v.ny > 1) {
    if (y == 0) gy = at(1, z) - at(0, z);
    else if (y == v.ny - 1) gy = at(y, z) - at(y - 1, z);
    else gy = C(0.5) * (at(y + 1, z) - at(y - 1, z));
  }
  if (v.nz > 1) {
    if (z == 0) gz = at(y, 1) - at(y, 0);
    else if (z == v.nz - 1) gz = at(y, z) - at(y, z - 1);
    else gz = C(0.5) * (at(y, z + 1) - at(y, z - 1));
  }
  const C gn = sqrt(gy * gy + gz * gz);
  const C ux = gn > C(0) ? -(uy * gy + uz * gz) / gn : C(0);
  const C* um = static_cast<const C*>(v.mean);
  C* cur = static_cast<C*>(v.cur);
  cur[p] = um[p] + ux;
  cur[pl + p] = um[pl + p] + uy;
  cur[2 * pl + p] = um[2 * pl + p] + uz;
}

}  // namespace

void vm_update(const VmArgs& v, int celem, cudaStream_t s) {
  if (v.n <= 0) return;
  const long long pl = (long long)v.ny * v.nz;
  const unsigned gb = unsigned((v.n + 127) / 128), gp = unsigned((pl + VM_THREADS - 1) / VM_THREADS);
  const dim3 gpart(gp, unsigned((v.n + VM_CHUNK - 1) / VM_CHUNK));
  if (celem == 8) {
    k_vm_gen<double><<<gb, 128, 0, s>>>(v);
    k_vm_partial<double><<<gpart, VM_THREADS, 0, s>>>(v);
    k_vm_finish<double><<<gp, VM_THREADS, 0, s>>>(v);
  } else {
    k_vm_gen<float><<<gb, 128, 0, s>>>(v);
    k_vm_partial<float><<<gpart, VM_THREADS, 0, s>>>(v);
    k_vm_finish<float><<<gp, VM_THREADS, 0, s>>>(v);
  }
}

}  // namespace lbm
