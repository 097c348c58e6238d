// Device-side building blocks of the fused collide-and-stream update: velocity sets, storage
// codecs, the AA-pattern slot map, and the per-cell physics (moments, equilibrium, Smagorinsky
// relaxation, regularised boundaries, Spalding wall model).
//
// Populations are stored as deviations h_i = f_i - w_i from the rest state in structure-of-arrays
// form, one array per population index. Propagation is the in-place AA pattern: an even step
// reads and writes only the cell's own slots (writing f*_i into slot opp(i)), an odd step reads
// each incoming population from the slot where the previous even step left it and writes each
// outgoing population into the same slot, where the next even step finds it. Boundary
// substitutions (bounce-back, specular slip, open-face unknowns) only change which slot a
// direction uses, so every slot is still read and written by exactly one cell per step.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <type_traits>
#include <utility>

namespace lbm {

// ---- type byte -----------------------------------------------------------------------------------
constexpr uint8_t T_KIND = 7;    // bits 0-2: kind
constexpr uint8_t T_REF = 8;     // wall-model reference cell (writes its velocity)
constexpr uint8_t T_NEAR = 16;   // some source position is solid or outside the domain
constexpr uint8_t T_LIST = 32;   // on the boundary list
constexpr uint8_t T_INLINE = 64; // list cell updated inside the interior kernel (fused mode)
constexpr uint8_t T_GHOST = 128; // ghost plane of a slab sub-domain: classified, never updated
enum { K_FLUID = 0, K_SOLID = 1, K_WALL = 2, K_INFLOW = 3, K_OUTFLOW = 4 };
enum { F_PERIODIC = 0, F_WALL = 1, F_SLIP = 2, F_OPEN = 3 };
constexpr unsigned ST_NAN = 1u, ST_BADMASK = 2u;

// ---- velocity sets (Sec. 2.2, Fig. "lattice"), ordering of include/lbm.h -------------------------
template <int Q> struct Lat;
template <> struct Lat<19> {
  static constexpr int Q = 19, H = 9, Wden = 36;
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int t[19] = {0, 1, 0, 0, 1, 1, 1, 1, 0, 0, -1, 0, 0, -1, -1, -1, -1, 0, 0};
    return t[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int t[19] = {0, 0, 1, 0, 1, -1, 0, 0, 1, 1, 0, -1, 0, -1, 1, 0, 0, -1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr int cz(int i) {
    constexpr int t[19] = {0, 0, 0, 1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 0, 0, -1, 1, -1, 1};
    return t[i];
  }
  __host__ __device__ static constexpr int W(int i) {  // 36 w_i
    constexpr int t[19] = {12, 2, 2, 2, 1, 1, 1, 1, 1, 1, 2, 2, 2, 1, 1, 1, 1, 1, 1};
    return t[i];
  }
};
template <> struct Lat<27> {
  static constexpr int Q = 27, H = 13, Wden = 216;
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int t[27] = {0, 1, 0, 0, 1, 1, 1, 1, 0, 0, 1, 1, 1, 1, -1, 0, 0, -1, -1, -1, -1, 0, 0, -1, -1, -1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int t[27] = {0, 0, 1, 0, 1, -1, 0, 0, 1, 1, 1, 1, -1, -1, 0, -1, 0, -1, 1, 0, 0, -1, -1, -1, -1, 1, 1};
    return t[i];
  }
  __host__ __device__ static constexpr int cz(int i) {
    constexpr int t[27] = {0, 0, 0, 1, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, -1, 0, 0, -1, 1, -1, 1, -1, 1, -1, 1};
    return t[i];
  }
  __host__ __device__ static constexpr int W(int i) {  // 216 w_i
    constexpr int t[27] = {64, 16, 16, 16, 4, 4, 4, 4, 4, 4, 1, 1, 1, 1, 16, 16, 16, 4, 4, 4, 4, 4, 4, 1, 1, 1, 1};
    return t[i];
  }
};
template <int Q> __host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= Lat<Q>::H ? i + Lat<Q>::H : i - Lat<Q>::H);
}
template <int Q, class C> __device__ __forceinline__ constexpr C wgt(int i) {
  return C(Lat<Q>::W(i)) / C(Lat<Q>::Wden);
}
// Direction index of a velocity (components in {-1,0,1}); -1 if absent from the set.
template <int Q> __device__ __forceinline__ int dir_of(int x, int y, int z) {
  int r = -1;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    if (Lat<Q>::cx(i) == x && Lat<Q>::cy(i) == y && Lat<Q>::cz(i) == z) r = i;
  return r;
}

// Compile-time integer usable as an index in device code.
template <int V> struct IC {
  static constexpr int value = V;
  __host__ __device__ constexpr operator int() const { return V; }
};
// Compile-time loop: f(IC<I>) for I = B..E-1.
template <int B, int E, class F> __device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(IC<B>{});
    sfor<B + 1, E>(f);
  }
}

// ---- storage codecs --------------------------------------------------------------------------------
template <class S> struct Codec;
template <> struct Codec<double> {
  using C = double;
  static __device__ __forceinline__ C ld(const double* p) { return *p; }
  static __device__ __forceinline__ void st(double* p, C v) { *p = v; }
};
template <> struct Codec<float> {
  using C = float;
  static __device__ __forceinline__ C ld(const float* p) { return *p; }
  static __device__ __forceinline__ void st(float* p, C v) { *p = v; }
};
template <> struct Codec<__half> {
  using C = float;
  static __device__ __forceinline__ C ld(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ void st(__half* p, C v) { *p = __float2half_rn(v); }
};
template <> struct Codec<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ C ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, C v) { *p = __float2bfloat16_rn(v); }
};

// ---- kernel arguments (plain data, copied by value into the launch) ---------------------------------
// A scalar parameter in both precisions, rounded to float once on the host: FP32 kernels read the
// float copy, so no double-to-float conversion runs per thread (the FP64 pipe is narrow).
struct Param {
  double d;
  float f;
  template <class C>
  __host__ __device__ __forceinline__ C get() const {
    if constexpr (std::is_same<C, float>::value) return f;
    else return C(d);
  }
  __host__ Param& operator=(double v) {
    d = v;
    f = float(v);
    return *this;
  }
};

// Division of n < 2^31 by a fixed d >= 1 with a precomputed multiplier (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): n / d = (umulhi(m, n) + n) >> l with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1; the sum stays below 2^32 for n < 2^31.
struct FastDiv {
  unsigned m;
  int l;
  static FastDiv make(unsigned d) {
    FastDiv f{0u, 0};
    while ((1ull << f.l) < d) ++f.l;
    f.m = unsigned(((1ull << 32) * ((1ull << f.l) - d)) / d + 1);
    return f;
  }
  __device__ __forceinline__ unsigned div(unsigned n) const { return (__umulhi(m, n) + n) >> l; }
};

struct Args {
  void* f;                 // population deviations, population p of cell m at f + p*stride + m
  long long stride;        // elements between population arrays
  const uint8_t* type;     // classified type byte per cell
  const void* gamma;       // porosity per cell (compute type) or null
  int nx, ny, nz;
  long long nxy, N;
  int face[6];
  Param tau0;              // molecular relaxation time
  Param nu0;               // molecular viscosity (tau0 - 1/2)/3, formed in double precision
  Param smag;              // 18 sqrt(2) C_S^2
  int use_smag;            // smag > 0
  Param cs2smag;           // C_S^2
  Param fx, fy, fz;        // body force
  unsigned* status;        // sticky device status bits
  // boundary list
  const long long* lcell;  // cell index per entry
  const int* lxyz;         // x, y, z per entry
  const unsigned long long* lcode;  // 2 bits per direction: 0 streaming, 1 bounce-back slot, 2 general
  int n_list;
  const void* wnrm;        // C[3] unit normal per entry (WALL entries)
  const void* wyw;         // C wall distance per entry
  const int* wref;         // list position of the reference cell, -1 none
  const void* ref_rd;      // C[3] per entry, reference velocities of the previous step
  void* ref_wr;            // C[3] per entry, written by reference cells this step
  const void* uin;         // C[3][ny*nz] inlet velocity
  Param rho_out;
  Param drho_out;          // rho_out - 1, formed in double precision
  int wm;                  // wall model on
  int fuse;                // 1: list cells flagged T_INLINE are updated by the interior kernel; the
                           //    boundary-list kernel then runs over the other entries only
  int inline_all;          // fused mode with the BGK collision: the interior kernel updates every list
                           //    cell (no boundary-list kernel)
  const int* lidx;         // list position of every cell (-1 off the list)
  const unsigned long long* ccode;  // slot codes of every list and NEAR cell, by cell index
  const int* lsub;         // list positions handled by the boundary-list kernel (fused mode)
  int n_sub;
  const int* lbc;          // list positions of INFLOW/OUTFLOW entries
  int n_bc;
  const int* lwall;        // list positions of WALL entries (wall-state pass)
  int n_wall;
  void* wst;               // wall-model state per list entry (WALL_STATE values)
  int kernel;              // interior kernel: 0 plain, 2 staged (bulk copies into shared memory) where the shape allows
  int idx32;               // 1: every population index q*stride fits in 32 bits (32-bit index arithmetic)
  int debug_stall;         // 1: the staged kernel also waits on a barrier nobody completes (tests the bounded wait)
  Param kappa, E;
  // hybrid recursive regularised collision
  int model;               // 0 BGK, 1 HRR
  int hybrid;              // HRR with sigma < 1 (the finite-difference strain is needed)
  Param sigma;             // hybridisation factor
  const void* uvel_rd;     // C[3][N] velocity field of the previous step
  void* uvel_wr;           // C[3][N] velocity field written by this step
  int pairs;               // interior kernel over cell pairs (nx even, 32-bit indices, few mixed warps)
  // outlet fringe zone: strength s(x) per x-plane (compute type, nx values; 0 before the layer) or null
  const void* fringe;
  int fr_x0;               // first plane of the layer
  int ghost;               // slab sub-domain with ghost planes (cells flagged T_GHOST are skipped)
  // launch shape of the HRR one-cell kernel (cell_at): 1-D CTAs of lc_t threads; when xcols (x faces
  // not periodic) the first lc_cols CTAs update the planes x = 0 and x = nx - 1 column by column and
  // the row CTAs after them skip those planes, so no row warp carries a face cell
  int xcols;
  unsigned lc_t, lc_gx, lc_gy, lc_cols;
  FastDiv lc_dgx, lc_dny, lc_dgy;
};

// ---- AA-pattern slot map ------------------------------------------------------------------------------
// Slot of direction i of cell (x,y,z): population index p and cell m. Before an odd step slot
// (p, m) holds f_i(x); during the odd step it receives f*_opp(i)(x). Rules:
//   source x - c_i inside (after periodic wrap), not solid -> (opp(i), x - c_i)   [streaming]
//   source solid                                          -> (i, x)             [bounce-back]
//   source beyond any open or bounce-back face            -> (i, x)             [unknown / BB]
//   source beyond full-slip faces only                    -> (opp(j), x') with x' the source
//     with the crossed coordinates set back to x's, j = c_i with crossed components reversed;
//     (i, x) if x' is solid.
template <int Q>
__device__ __forceinline__ void slot_of(const Args& a, int x, int y, int z, long long n, int i, int& p, long long& m) {
  int sx = x - Lat<Q>::cx(i), sy = y - Lat<Q>::cy(i), sz = z - Lat<Q>::cz(i);
  int crossed = 0;
  if (sx < 0) { if (a.face[0] == F_PERIODIC) sx += a.nx; else crossed |= 1; }
  else if (sx >= a.nx) { if (a.face[1] == F_PERIODIC) sx -= a.nx; else crossed |= 2; }
  if (sy < 0) { if (a.face[2] == F_PERIODIC) sy += a.ny; else crossed |= 4; }
  else if (sy >= a.ny) { if (a.face[3] == F_PERIODIC) sy -= a.ny; else crossed |= 8; }
  if (sz < 0) { if (a.face[4] == F_PERIODIC) sz += a.nz; else crossed |= 16; }
  else if (sz >= a.nz) { if (a.face[5] == F_PERIODIC) sz -= a.nz; else crossed |= 32; }
  if (crossed == 0) {
    long long s = sx + (long long)a.nx * sy + a.nxy * sz;
    if ((a.type[s] & T_KIND) == K_SOLID) { p = i; m = n; }
    else { p = opp<Q>(i); m = s; }
    return;
  }
  bool allslip = true;
#pragma unroll
  for (int f = 0; f < 6; ++f)
    if ((crossed >> f & 1) && a.face[f] != F_SLIP) allslip = false;
  if (!allslip) { p = i; m = n; return; }
  int jx = Lat<Q>::cx(i), jy = Lat<Q>::cy(i), jz = Lat<Q>::cz(i);
  if (crossed & 3) { sx = x; jx = -jx; }
  if (crossed & 12) { sy = y; jy = -jy; }
  if (crossed & 48) { sz = z; jz = -jz; }
  long long s = sx + (long long)a.nx * sy + a.nxy * sz;
  if ((a.type[s] & T_KIND) == K_SOLID) { p = i; m = n; return; }
  p = opp<Q>(dir_of<Q>(jx, jy, jz));
  m = s;
}

// ---- per-cell physics ------------------------------------------------------------------------------------
// Products with the integer lattice components written so that zero terms never appear: IEEE
// arithmetic does not allow a compiler to drop 0*x or 0+x, so the tables are folded here.
template <int A, class C> __device__ __forceinline__ C cmul(C v) {
  if constexpr (A == 1) return v;
  else if constexpr (A == -1) return -v;
  else return C(A) * v;
}
template <int X, int Y, int Z, class C> __device__ __forceinline__ C cdot(C x, C y, C z) {
  if constexpr (X == 0 && Y == 0 && Z == 0) return C(0);
  else if constexpr (Y == 0 && Z == 0) return cmul<X>(x);
  else if constexpr (X == 0 && Z == 0) return cmul<Y>(y);
  else if constexpr (X == 0 && Y == 0) return cmul<Z>(z);
  else if constexpr (Z == 0) return cmul<X>(x) + cmul<Y>(y);
  else if constexpr (Y == 0) return cmul<X>(x) + cmul<Z>(z);
  else if constexpr (X == 0) return cmul<Y>(y) + cmul<Z>(z);
  else return cmul<X>(x) + cmul<Y>(y) + cmul<Z>(z);
}
template <int Q, int I, class C> __device__ __forceinline__ C cdot_i(C x, C y, C z) {
  return cdot<Lat<Q>::cx(I), Lat<Q>::cy(I), Lat<Q>::cz(I)>(x, y, z);
}

// Equilibrium deviation f_i^eq(rho, v) - w_i = w_i (drho + rho (3 c.v + 4.5 (c.v)^2 - 1.5 v.v)).
template <int Q, class C, int I>
__device__ __forceinline__ C heq(C drho, C rho, C vx, C vy, C vz, C vsq) {
  if constexpr (I == 0) {
    return wgt<Q, C>(I) * (drho - rho * (C(1.5) * vsq));
  } else {
    const C cv = cdot_i<Q, I>(vx, vy, vz);
    return wgt<Q, C>(I) * (drho + rho * (C(3) * cv + C(4.5) * cv * cv - C(1.5) * vsq));
  }
}

template <int Q, class C>
__device__ __forceinline__ void sums(const C* h, C& drho, C& jx, C& jy, C& jz) {
  drho = jx = jy = jz = C(0);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    drho += h[i];
    if (Lat<Q>::cx(i)) jx += C(Lat<Q>::cx(i)) * h[i];
    if (Lat<Q>::cy(i)) jy += C(Lat<Q>::cy(i)) * h[i];
    if (Lat<Q>::cz(i)) jz += C(Lat<Q>::cz(i)) * h[i];
  });
}

// Q_i : A (A symmetric, given by its six components) with Q_i = c_i c_i - I/3.
template <int Q, class C, int I>
__device__ __forceinline__ C qcontract(C axx, C ayy, C azz, C axy, C axz, C ayz) {
  constexpr int cx = Lat<Q>::cx(I), cy = Lat<Q>::cy(I), cz = Lat<Q>::cz(I);
  C r = -(axx + ayy + azz) * C(1.0 / 3.0);
  if constexpr (cx != 0) r += axx;
  if constexpr (cy != 0) r += ayy;
  if constexpr (cz != 0) r += azz;
  if constexpr (cx * cy != 0) r += cmul<2 * cx * cy>(axy);
  if constexpr (cx * cz != 0) r += cmul<2 * cx * cz>(axz);
  if constexpr (cy * cz != 0) r += cmul<2 * cy * cz>(ayz);
  return r;
}

template <class C> __device__ __forceinline__ C rcp(C x) { return C(1) / x; }
template <> __device__ __forceinline__ float rcp<float>(float x) { return __fdividef(1.0f, x); }

// BGK + Smagorinsky + porosity + exact-difference force on the deviations h (in place).
// Returns the density and the reported velocity u + F/(2 rho).
//
// Written over opposite pairs (i, i + H): with s = h_i + h_i', d = h_i - h_i' the moments are
// drho = h_0 + sum s, j = sum c d, sum c c h = sum c c s; and with
//   h*_i = f^eq_i(v) - w_i + k (h_i - (f^eq_i(u) - w_i)),   k = 1 - 1/tau,
// f^eq_i(v) - k f^eq_i(u) - (1 - k) w_i = w_i [sym +- anti] where the sign flips with c_i:
//   sym  = (1 - k) drho - 1.5 rho (v.v - k u.u) + 4.5 rho ((c.v)^2 - k (c.u)^2)
//   anti = 3 rho (c.v - k c.u).
template <int Q, class C>
__device__ __forceinline__ void collide_fluid(C* h, C gamma, const Args& a, C& rho_o, C& urx, C& ury, C& urz) {
  constexpr int H = Lat<Q>::H;
  C drho = h[0], jx = C(0), jy = C(0), jz = C(0);
  C sxx = C(0), syy = C(0), szz = C(0), sxy = C(0), sxz = C(0), syz = C(0);
  sfor<1, H + 1>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    const C sp = h[i] + h[i + H], dp = h[i] - h[i + H];
    drho += sp;
    if constexpr (cx != 0) { jx += cmul<cx>(dp); sxx += sp; }
    if constexpr (cy != 0) { jy += cmul<cy>(dp); syy += sp; }
    if constexpr (cz != 0) { jz += cmul<cz>(dp); szz += sp; }
    if constexpr (cx * cy != 0) sxy += cmul<cx * cy>(sp);
    if constexpr (cx * cz != 0) sxz += cmul<cx * cz>(sp);
    if constexpr (cy * cz != 0) syz += cmul<cy * cz>(sp);
  });
  const C rho = C(1) + drho, ir = rcp(rho);
  const C ux = jx * ir, uy = jy * ir, uz = jz * ir;
  const C usq = ux * ux + uy * uy + uz * uz;
  C tau = a.tau0.get<C>();
  if (a.use_smag != 0) {
    // Pi^neq = sum c c h - drho/3 I - rho u u (second moment of the 2nd-order equilibrium).
    const C d3 = drho * C(1.0 / 3.0);
    const C pxx = sxx - d3 - rho * ux * ux, pyy = syy - d3 - rho * uy * uy, pzz = szz - d3 - rho * uz * uz;
    const C pxy = sxy - rho * ux * uy, pxz = sxz - rho * ux * uz, pyz = syz - rho * uy * uz;
    const C pn = sqrt(pxx * pxx + pyy * pyy + pzz * pzz + C(2) * (pxy * pxy + pxz * pxz + pyz * pyz));
    const C t0 = a.tau0.get<C>();
    tau = C(0.5) * (t0 + sqrt(t0 * t0 + a.smag.get<C>() * pn * ir));
  }
  const C k = C(1) - rcp(tau);
  const C vx = gamma * ux + a.fx.get<C>() * ir, vy = gamma * uy + a.fy.get<C>() * ir, vz = gamma * uz + a.fz.get<C>() * ir;
  const C vsq = vx * vx + vy * vy + vz * vz;
  const C base = (C(1) - k) * drho - C(1.5) * rho * (vsq - k * usq);
  const C r45 = C(4.5) * rho, r3 = C(3) * rho;
  h[0] = k * h[0] + wgt<Q, C>(0) * base;
  sfor<1, H + 1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const C cu = cdot_i<Q, i>(ux, uy, uz), cv = cdot_i<Q, i>(vx, vy, vz);
    const C sym = base + r45 * (cv * cv - k * (cu * cu));
    const C anti = r3 * (cv - k * cu);
    h[i] = k * h[i] + wgt<Q, C>(i) * (sym + anti);
    h[i + H] = k * h[i + H] + wgt<Q, C>(i) * (sym - anti);
  });
  rho_o = rho;
  const C hf = C(0.5) * ir;
  urx = ux + a.fx.get<C>() * hf;
  ury = uy + a.fy.get<C>() * hf;
  urz = uz + a.fz.get<C>() * hf;
}

// ---- the same collision on two cells at once with packed FP32 instructions -------------------------------
// Lane x of every float2 belongs to one cell, lane y to the other. The packed add, multiply and fused
// multiply-add round each lane exactly as their scalar forms, so this is the FP32 collision above
// with half the arithmetic instructions; reciprocals and square roots run per lane.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp(a.x), rcp(a.y)); }
__device__ __forceinline__ float2 sqrt2(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
// acc + S v for a compile-time sign S = +-1
template <int S> __device__ __forceinline__ float2 acc2(float2 acc, float2 v) {
  if constexpr (S > 0) return add2(acc, v);
  else return sub2(acc, v);
}
// sigma_i (c_i . v) with sigma_i the sign of the first non-zero component of c_i
template <int Q, int I> __device__ __forceinline__ float2 cdot2(float2 x, float2 y, float2 z) {
  constexpr int cx = Lat<Q>::cx(I), cy = Lat<Q>::cy(I), cz = Lat<Q>::cz(I);
  constexpr int sg = cx != 0 ? cx : (cy != 0 ? cy : cz);
  constexpr int ax = sg * cx, ay = sg * cy, az = sg * cz;
  if constexpr (ax != 0) {
    float2 r = x;
    if constexpr (ay != 0) r = acc2<ay>(r, y);
    if constexpr (az != 0) r = acc2<az>(r, z);
    return r;
  } else if constexpr (ay != 0) {
    float2 r = y;
    if constexpr (az != 0) r = acc2<az>(r, z);
    return r;
  } else {
    return z;
  }
}
template <int Q, int I> __host__ __device__ constexpr int csign() {
  return Lat<Q>::cx(I) != 0 ? Lat<Q>::cx(I) : (Lat<Q>::cy(I) != 0 ? Lat<Q>::cy(I) : Lat<Q>::cz(I));
}

// Returns false when either cell's density or velocity is not finite. get(i) yields population i of
// both cells (read twice: for the moments and for the relaxation), put(i, v) stores its new value.
template <int Q, class Get, class Put>
__device__ __forceinline__ bool collide_fluid_x2(Get&& get, Put&& put, float2 gamma, const Args& a) {
  constexpr int H = Lat<Q>::H;
  const float2 z2 = bc2(0.f);
  float2 drho = get(0), jx = z2, jy = z2, jz = z2;
  float2 sxx = z2, syy = z2, szz = z2, sxy = z2, sxz = z2, syz = z2;
  sfor<1, H + 1>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    const float2 hi = get(i), ho = get(i + H);
    const float2 sp = add2(hi, ho), dp = sub2(hi, ho);
    drho = add2(drho, sp);
    if constexpr (cx != 0) { jx = acc2<cx>(jx, dp); sxx = add2(sxx, sp); }
    if constexpr (cy != 0) { jy = acc2<cy>(jy, dp); syy = add2(syy, sp); }
    if constexpr (cz != 0) { jz = acc2<cz>(jz, dp); szz = add2(szz, sp); }
    if constexpr (cx * cy != 0) sxy = acc2<cx * cy>(sxy, sp);
    if constexpr (cx * cz != 0) sxz = acc2<cx * cz>(sxz, sp);
    if constexpr (cy * cz != 0) syz = acc2<cy * cz>(syz, sp);
  });
  const float2 one = bc2(1.f);
  const float2 rho = add2(one, drho), ir = rcp2(rho);
  const float2 ux = mul2(jx, ir), uy = mul2(jy, ir), uz = mul2(jz, ir);
  const float2 usq = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
  const float t0 = a.tau0.f;
  float2 tau = bc2(t0);
  if (a.use_smag != 0) {
    const float2 d3 = mul2(drho, bc2(1.f / 3.f));
    const float2 rux = mul2(rho, ux), ruy = mul2(rho, uy), ruz = mul2(rho, uz);
    const float2 pxx = sub2(sxx, fma2(rux, ux, d3)), pyy = sub2(syy, fma2(ruy, uy, d3)), pzz = sub2(szz, fma2(ruz, uz, d3));
    const float2 pxy = sub2(sxy, mul2(rux, uy)), pxz = sub2(sxz, mul2(rux, uz)), pyz = sub2(syz, mul2(ruy, uz));
    const float2 off = fma2(pxy, pxy, fma2(pxz, pxz, mul2(pyz, pyz)));
    const float2 pn = sqrt2(fma2(bc2(2.f), off, fma2(pxx, pxx, fma2(pyy, pyy, mul2(pzz, pzz)))));
    tau = mul2(bc2(0.5f), add2(bc2(t0), sqrt2(fma2(bc2(a.smag.f), mul2(pn, ir), bc2(t0 * t0)))));
  }
  const float2 itau = rcp2(tau);
  const float2 k = sub2(one, itau), nk = sub2(itau, one);
  const float2 vx = fma2(gamma, ux, mul2(bc2(a.fx.f), ir));
  const float2 vy = fma2(gamma, uy, mul2(bc2(a.fy.f), ir));
  const float2 vz = fma2(gamma, uz, mul2(bc2(a.fz.f), ir));
  const float2 vsq = fma2(vx, vx, fma2(vy, vy, mul2(vz, vz)));
  const float2 base = sub2(mul2(itau, drho), mul2(mul2(bc2(1.5f), rho), fma2(nk, usq, vsq)));
  const float2 r45 = mul2(bc2(4.5f), rho), r3 = mul2(bc2(3.f), rho);
  put(0, fma2(k, get(0), mul2(bc2(wgt<Q, float>(0)), base)));
  sfor<1, H + 1>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const float2 cu = cdot2<Q, i>(ux, uy, uz), cv = cdot2<Q, i>(vx, vy, vz);
    const float2 sym = fma2(r45, fma2(nk, mul2(cu, cu), mul2(cv, cv)), base);
    const float2 anti = mul2(r3, fma2(nk, cu, cv));
    const float2 w = bc2(wgt<Q, float>(i));
    const float2 p = mul2(w, add2(sym, anti)), m = mul2(w, sub2(sym, anti));
    if constexpr (csign<Q, i>() > 0) {
      put(i, fma2(k, get(i), p));
      put(i + H, fma2(k, get(i + H), m));
    } else {
      put(i, fma2(k, get(i), m));
      put(i + H, fma2(k, get(i + H), p));
    }
  });
  const float2 chk = add2(add2(abs2(rho), abs2(ux)), add2(abs2(uy), abs2(uz)));
  return chk.x < 1e30f && chk.y < 1e30f;
}

// The BGK collision of a fluid cell and the sigma = 0 update of a wall-model cell as one instruction
// stream, for warps that mix the two (the mixed path of the interior kernel). In the opposite-pair
// form of collide_fluid, with k the relaxation factor, v the homogenised velocity, g a weight and S a
// strain,
//   h*_i = k h_i + w_i [base + 4.5 rho ((c.v)^2 - k (c.u)^2) + g Q_i : S  +-  3 rho (c.v - k c.u)],
//   base = (1 - k) drho - 1.5 rho (v.v - k u.u).
// Fluid lanes (ws == nullptr): k = 1 - 1/tau_eff, v = gamma u + F/rho, g = 0, i.e. collide_fluid.
// Wall lanes: k = 0, v = u^B + F/rho, g = -3 rho (tau - 1), S the modelled strain, i.e.
// f* = f^eq(rho, v) + (1 - 1/tau) f^(1,FD) with f^(1,FD)_i = -(w_i rho tau / cs^2) Q_i : S
// (collide_wall_state). Returns the density and the reported velocity u + F/(2 rho).
template <int Q, class C>
__device__ __forceinline__ void collide_unified(C* h, C gamma, const Args& a, const C* ws, C& rho_o, C& urx, C& ury,
                                                C& urz) {
  constexpr int H = Lat<Q>::H;
  C drho = h[0], jx = C(0), jy = C(0), jz = C(0);
  C sxx = C(0), syy = C(0), szz = C(0), sxy = C(0), sxz = C(0), syz = C(0);
  sfor<1, H + 1>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    const C sp = h[i] + h[i + H], dp = h[i] - h[i + H];
    drho += sp;
    if constexpr (cx != 0) { jx += cmul<cx>(dp); sxx += sp; }
    if constexpr (cy != 0) { jy += cmul<cy>(dp); syy += sp; }
    if constexpr (cz != 0) { jz += cmul<cz>(dp); szz += sp; }
    if constexpr (cx * cy != 0) sxy += cmul<cx * cy>(sp);
    if constexpr (cx * cz != 0) sxz += cmul<cx * cz>(sp);
    if constexpr (cy * cz != 0) syz += cmul<cy * cz>(sp);
  });
  const C rho = C(1) + drho, ir = rcp(rho);
  const C ux = jx * ir, uy = jy * ir, uz = jz * ir;
  const C usq = ux * ux + uy * uy + uz * uz;
  C tau = a.tau0.get<C>();
  if (a.use_smag != 0) {
    const C d3 = drho * C(1.0 / 3.0);
    const C pxx = sxx - d3 - rho * ux * ux, pyy = syy - d3 - rho * uy * uy, pzz = szz - d3 - rho * uz * uz;
    const C pxy = sxy - rho * ux * uy, pxz = sxz - rho * ux * uz, pyz = syz - rho * uy * uz;
    const C pn = sqrt(pxx * pxx + pyy * pyy + pzz * pzz + C(2) * (pxy * pxy + pxz * pxz + pyz * pyz));
    const C t0 = a.tau0.get<C>();
    tau = C(0.5) * (t0 + sqrt(t0 * t0 + a.smag.get<C>() * pn * ir));
  }
  C k = C(1) - rcp(tau);
  C vx = gamma * ux, vy = gamma * uy, vz = gamma * uz;
  C g = C(0), qxx = C(0), qyy = C(0), qzz = C(0), qxy = C(0), qxz = C(0), qyz = C(0);
  if (ws != nullptr) {
    k = C(0);
    vx = ws[0]; vy = ws[1]; vz = ws[2];
    g = -C(3) * rho * (ws[3] - C(1));
    qxx = ws[4]; qyy = ws[5]; qzz = ws[6]; qxy = ws[7]; qxz = ws[8]; qyz = ws[9];
  }
  vx += a.fx.get<C>() * ir; vy += a.fy.get<C>() * ir; vz += a.fz.get<C>() * ir;
  const C vsq = vx * vx + vy * vy + vz * vz;
  const C base = (C(1) - k) * drho - C(1.5) * rho * (vsq - k * usq);
  const C r45 = C(4.5) * rho, r3 = C(3) * rho;
  const C tr3 = (qxx + qyy + qzz) * C(1.0 / 3.0);
  h[0] = k * h[0] + wgt<Q, C>(0) * (base - g * tr3);
  sfor<1, H + 1>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    const C cu = cdot_i<Q, i>(ux, uy, uz), cv = cdot_i<Q, i>(vx, vy, vz);
    C qs = -tr3;  // Q_i : S, the same for i and its opposite
    if constexpr (cx != 0) qs += qxx;
    if constexpr (cy != 0) qs += qyy;
    if constexpr (cz != 0) qs += qzz;
    if constexpr (cx * cy != 0) qs += cmul<2 * cx * cy>(qxy);
    if constexpr (cx * cz != 0) qs += cmul<2 * cx * cz>(qxz);
    if constexpr (cy * cz != 0) qs += cmul<2 * cy * cz>(qyz);
    const C sym = base + r45 * (cv * cv - k * (cu * cu)) + g * qs;
    const C anti = r3 * (cv - k * cu);
    h[i] = k * h[i] + wgt<Q, C>(i) * (sym + anti);
    h[i + H] = k * h[i + H] + wgt<Q, C>(i) * (sym - anti);
  });
  rho_o = rho;
  const C hf = C(0.5) * ir;
  urx = ux + a.fx.get<C>() * hf;
  ury = uy + a.fy.get<C>() * hf;
  urz = uz + a.fz.get<C>() * hf;
}

// Regularised reconstruction: unknown populations (known(i) false) take the non-equilibrium part
// of their opposite; all populations become f^eq + w_i/(2 cs^4) Q_i : Pi^neq.
template <int Q, class C, class Known>
__device__ __forceinline__ void regularise(C* h, C drho, C rho, C ux, C uy, C uz) {
  const C usq = ux * ux + uy * uy + uz * uz;
  C ne[Q];
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    ne[i] = h[i] - heq<Q, C, i>(drho, rho, ux, uy, uz, usq);
  });
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (!Known{}(i)) ne[i] = ne[opp<Q>(i)];
  });
  C pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    if (cx) pxx += ne[i];
    if (cy) pyy += ne[i];
    if (cz) pzz += ne[i];
    if (cx * cy) pxy += C(cx * cy) * ne[i];
    if (cx * cz) pxz += C(cx * cz) * ne[i];
    if (cy * cz) pyz += C(cy * cz) * ne[i];
  });
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    h[i] = heq<Q, C, i>(drho, rho, ux, uy, uz, usq) +
           wgt<Q, C>(i) * C(4.5) * qcontract<Q, C, i>(pxx, pyy, pzz, pxy, pxz, pyz);
  });
}

template <int Q> struct KnownInlet { __host__ __device__ constexpr bool operator()(int i) const { return Lat<Q>::cx(i) <= 0; } };
template <int Q> struct KnownOutlet { __host__ __device__ constexpr bool operator()(int i) const { return Lat<Q>::cx(i) >= 0; } };

// Velocity inlet (inward normal +x): rho (1 - u_x) = sum_{c_x=0} f + 2 sum_{c_x<0} f.
// With f = h + w and sum_{c_x=0} w + 2 sum_{c_x<0} w = 1 the right side is 1 + s, s the same sums
// over h; the density deviation is formed without cancellation as (s + u_x) / (1 - u_x).
template <int Q, class C>
__device__ __forceinline__ void bc_inlet(C* h, C ubx, C uby, C ubz) {
  C s = C(0);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (Lat<Q>::cx(i) == 0) s += h[i];
    if (Lat<Q>::cx(i) < 0) s += C(2) * h[i];
  });
  const C den = C(1) - ubx;
  const C drho = (s + ubx) / den;
  regularise<Q, C, KnownInlet<Q>>(h, drho, C(1) + drho, ubx, uby, ubz);
}

// Pressure outlet (inward normal -x): rho = rho_out, rho_out (1 + u_x) = sum_{c_x=0} f + 2 sum_{c_x>0} f,
// tangential velocity 0; u_x = (s - (rho_out - 1)) / rho_out with s the deviation sums.
template <int Q, class C>
__device__ __forceinline__ void bc_outlet(C* h, C rho_out, C drho_out) {
  C s = C(0);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (Lat<Q>::cx(i) == 0) s += h[i];
    if (Lat<Q>::cx(i) > 0) s += C(2) * h[i];
  });
  const C ux = (s - drho_out) / rho_out;
  regularise<Q, C, KnownOutlet<Q>>(h, drho_out, rho_out, ux, C(0), C(0));
}

// ---- Spalding wall function, Eq. (spaldingfunct) -----------------------------------------------------
template <class C> __device__ __forceinline__ C cexp(C x) { return exp(x); }
template <> __device__ __forceinline__ float cexp<float>(float x) { return expf(x); }
template <class C> __device__ __forceinline__ C clog(C x) { return log(x); }
template <> __device__ __forceinline__ float clog<float>(float x) { return logf(x); }

template <class C> __device__ __forceinline__ C sp_y(C u, C k, C E) {
  const C x = k * u;
  return u + (cexp(x) - C(1) - x - x * x * C(0.5) - x * x * x * C(1.0 / 6.0)) / E;
}
template <class C> __device__ __forceinline__ C sp_dy(C u, C k, C E) {
  const C x = k * u;
  return C(1) + k * (cexp(x) - C(1) - x - x * x * C(0.5)) / E;
}
template <class C> __device__ __forceinline__ C newton_tol() { return std::is_same<C, double>::value ? C(1e-14) : C(1e-6); }

// u+ with u+ * y+(u+) = Re; Newton from the right of the root (monotone for this convex function).
template <class C> __device__ C sp_solve_re(C Re, C k, C E) {
  if (!(Re > C(0))) return C(0);
  C u = sqrt(Re);
  if (k * u > C(10)) {
    const C u1 = clog(C(2) * E * Re) / k;
    if (u1 < u && u1 * sp_y(u1, k, E) - Re >= C(0)) u = u1;
  }
  for (int it = 0; it < 30; ++it) {
    const C y = sp_y(u, k, E);
    const C du = (u * y - Re) / (y + u * sp_dy(u, k, E));
    u -= du;
    if (fabs(du) <= newton_tol<C>() * fabs(u)) break;
  }
  return u;
}
// u+ with y+(u+) = yp.
template <class C> __device__ C sp_solve_y(C yp, C k, C E) {
  if (!(yp > C(0))) return C(0);
  C u = yp;
  if (k * u > C(10)) {
    const C u1 = clog(C(2) * E * yp) / k;
    if (u1 < u && sp_y(u1, k, E) - yp >= C(0)) u = u1;
  }
  for (int it = 0; it < 30; ++it) {
    const C du = (sp_y(u, k, E) - yp) / sp_dy(u, k, E);
    u -= du;
    if (fabs(du) <= newton_tol<C>() * fabs(u)) break;
  }
  return u;
}

// Wall-model state of a WALL cell (Sec. 2.2.1): from the reference velocity ur at distance yw + 1
// along the unit normal n, the solid velocity u^B, the modelled strain S = (du/dn)/2 (t n^T + n t^T)
// with du/dn = (u_tau^2/nu) / (dy+/du+)(u+_w), and tau = tau0 + 3 C_S^2 |du/dn|.
// Layout of the 10 values: u^B (3), tau, S_xx, S_yy, S_zz, S_xy, S_xz, S_yz.
constexpr int WALL_STATE = 10;

template <class C>
__device__ __forceinline__ void wall_state(const Args& a, const C* nrm, C yw, const C* ur, bool has_ref, C* ws) {
  C ubx = 0, uby = 0, ubz = 0, dudn = 0, tx = 0, ty = 0, tz = 0;
  const C nx = nrm[0], ny = nrm[1], nz = nrm[2];
  if (has_ref && (nx != C(0) || ny != C(0) || nz != C(0))) {
    const C un = ur[0] * nx + ur[1] * ny + ur[2] * nz;
    const C utx = ur[0] - un * nx, uty = ur[1] - un * ny, utz = ur[2] - un * nz;
    const C U = sqrt(utx * utx + uty * uty + utz * utz);
    if (U >= C(1e-12)) {
      tx = utx / U; ty = uty / U; tz = utz / U;
      const C k = a.kappa.get<C>(), E = a.E.get<C>();
      const C nu = a.nu0.get<C>();
      const C upr = sp_solve_re<C>(U * (yw + C(1)) / nu, k, E);
      const C utau = U / upr;
      const C upw = sp_solve_y<C>(yw * utau / nu, k, E);
      const C ub = utau * upw;
      ubx = ub * tx; uby = ub * ty; ubz = ub * tz;
      dudn = (utau * utau / nu) / sp_dy<C>(upw, k, E);
    }
  }
  const C hd = C(0.5) * dudn;
  ws[0] = ubx; ws[1] = uby; ws[2] = ubz;
  ws[3] = a.tau0.get<C>() + C(3) * a.cs2smag.get<C>() * fabs(dudn);
  ws[4] = hd * C(2) * tx * nx; ws[5] = hd * C(2) * ty * ny; ws[6] = hd * C(2) * tz * nz;
  ws[7] = hd * (tx * ny + nx * ty); ws[8] = hd * (tx * nz + nx * tz); ws[9] = hd * (ty * nz + ny * tz);
}

// sigma = 0 reconstruction of a WALL cell from its wall-model state:
// f* = f^eq(rho, u^B + F/rho) + (1 - 1/tau) f^(1,FD), f^(1,FD)_i = -(w_i rho tau / cs^2) Q_i : S.
template <int Q, class C>
__device__ __forceinline__ void collide_wall_state(C* h, const Args& a, const C* ws, C& rho_o, C& urx, C& ury, C& urz) {
  C drho, jx, jy, jz;
  sums<Q, C>(h, drho, jx, jy, jz);
  const C rho = C(1) + drho, ir = rcp(rho);
  rho_o = rho;
  const C hf = C(0.5) * ir;
  urx = jx * ir + a.fx.get<C>() * hf;
  ury = jy * ir + a.fy.get<C>() * hf;
  urz = jz * ir + a.fz.get<C>() * hf;
  const C tau = ws[3];
  const C sxx = ws[4], syy = ws[5], szz = ws[6], sxy = ws[7], sxz = ws[8], syz = ws[9];
  const C vx = ws[0] + a.fx.get<C>() * ir, vy = ws[1] + a.fy.get<C>() * ir, vz = ws[2] + a.fz.get<C>() * ir;
  const C vsq = vx * vx + vy * vy + vz * vz;
  const C g = -C(3) * rho * (tau - C(1));  // (1 - 1/tau) * (-rho tau / cs^2)
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    h[i] = heq<Q, C, i>(drho, rho, vx, vy, vz, vsq) + g * wgt<Q, C>(i) * qcontract<Q, C, i>(sxx, syy, szz, sxy, sxz, syz);
  });
}

// Both in one (boundary-list path).
template <int Q, class C>
__device__ __forceinline__ void collide_wall(C* h, const Args& a, const C* nrm, C yw, const C* ur, bool has_ref, C& rho_o,
                                             C& urx, C& ury, C& urz) {
  C ws[WALL_STATE];
  wall_state<C>(a, nrm, yw, ur, has_ref, ws);
  collide_wall_state<Q, C>(h, a, ws, rho_o, urx, ury, urz);
}

template <class C> __device__ __forceinline__ bool finite_all(C a, C b, C c, C d) {
  return fabs(a) + fabs(b) + fabs(c) + fabs(d) < C(1e30);
}

}  // namespace lbm
