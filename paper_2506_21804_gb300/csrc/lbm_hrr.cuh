// Hybrid recursive regularised (HRR) collision of Sec. 2.2 (Eq. hlbm with the Hermite expansion of
// the non-equilibrium part), on the deviations h_i = f_i - w_i:
//
//   f*_i = f^eq_i(rho, u_eq) + (1 - 1/tau) f^(1)_i,
//   f^eq_i = w_i [rho + 3 rho c.u + 4.5 rho (c.u)^2 - 1.5 rho u.u] + third-order term of rho u u u,
//   f^(1)_i = 4.5 w_i Q_i : A2 + third-order term of A3,   Q_i = c_i c_i - I/3,
//   A2 = sigma Pi^neq + (1 - sigma) (-2/3) rho tau S^FD,   A3_abc = u_a A2_bc + u_b A2_ac + u_c A2_ab,
//
// with u_eq the homogenised velocity plus the exact-difference force shift, u (in A3) the homogenised
// velocity, Pi^neq the local non-equilibrium stress and S^FD the finite-difference strain of the
// previous step's velocity field.
//
// Third-order term. With unit speeds the polynomials H_aaa vanish; the velocity sets carry the six
// mixed H_aab = (c_a^2 - 1/3) c_b, and D3Q27 also H_xyz = c_x c_y c_z. The term of a symmetric
// tensor a is w_i sum_k H_k(c_i) b_k with b = G^{-1} a over the carried polynomials, G the Gram
// matrix sum_i w_i H_k H_l, so that the lattice third moments of the term equal the components of a.
// D3Q27: G is diagonal (2/27 for the mixed, 1/27 for H_xyz), b_aab = 13.5 a_aab, b_xyz = 27 a_xyz,
// which is the Hermite term H^(3) : a / (6 cs^6). D3Q19: G pairs H_xxy with H_zzy, H_xxz with H_yyz
// and H_yyx with H_zzx, each block (1/27) [[2, -1], [-1, 2]] with inverse 9 [[2, 1], [1, 2]].
// The code below carries bp_k = b_k / 3 and the integer m_k(c) = 3 H_aab(c) = (3 c_a^2 - 1) c_b.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// mixed polynomial k = 0..5: H_aab with (a, b) = (x,y), (z,y), (x,z), (y,z), (y,x), (z,x); D3Q19's
// Gram blocks are the index pairs (0,1), (2,3), (4,5).
__host__ __device__ constexpr int h3_a(int k) {
  constexpr int t[6] = {0, 2, 0, 1, 1, 2};
  return t[k];
}
__host__ __device__ constexpr int h3_b(int k) {
  constexpr int t[6] = {1, 1, 2, 2, 0, 0};
  return t[k];
}
template <int Q> __host__ __device__ constexpr int ccomp(int i, int a) {
  return a == 0 ? Lat<Q>::cx(i) : (a == 1 ? Lat<Q>::cy(i) : Lat<Q>::cz(i));
}
// m_k(c_i) = 3 H_aab(c_i)
template <int Q, int I, int K> __host__ __device__ constexpr int h3_m() {
  return (3 * ccomp<Q>(I, h3_a(K)) * ccomp<Q>(I, h3_a(K)) - 1) * ccomp<Q>(I, h3_b(K));
}

// r + M v for a compile-time small integer M
template <int M, class C> __device__ __forceinline__ C acc_m(C r, C v) {
  if constexpr (M == 0) return r;
  else if constexpr (M == 1) return r + v;
  else if constexpr (M == -1) return r - v;
  else return r + C(M) * v;
}

// Second-order coefficients A = (xx, yy, zz, xy, xz, yz).
// Overwrites h with the post-collision deviations; drho = rho - 1.
template <int Q, class C>
__device__ __forceinline__ void hrr_relax(C* h, C drho, C rho, C uex, C uey, C uez, C uhx, C uhy, C uhz, C k,
                                          const C* A) {
  constexpr int H = Lat<Q>::H;
  const C Axx = A[0], Ayy = A[1], Azz = A[2], Axy = A[3], Axz = A[4], Ayz = A[5];
  const C usq = uex * uex + uey * uey + uez * uez;
  const C base = drho - C(1.5) * rho * usq - C(1.5) * k * (Axx + Ayy + Azz);
  const C r45 = C(4.5) * rho, r3 = C(3) * rho, k45 = C(4.5) * k;
  // third-order tensor of equilibrium plus relaxed non-equilibrium, mixed components
  const C rxx = rho * uex * uex, ryy = rho * uey * uey, rzz = rho * uez * uez;
  const C a_xxy = rxx * uey + k * (C(2) * uhx * Axy + uhy * Axx);
  const C a_zzy = rzz * uey + k * (C(2) * uhz * Ayz + uhy * Azz);
  const C a_xxz = rxx * uez + k * (C(2) * uhx * Axz + uhz * Axx);
  const C a_yyz = ryy * uez + k * (C(2) * uhy * Ayz + uhz * Ayy);
  const C a_yyx = ryy * uex + k * (C(2) * uhy * Axy + uhx * Ayy);
  const C a_zzx = rzz * uex + k * (C(2) * uhz * Axz + uhx * Azz);
  C bp[6], bxyz = C(0);
  if constexpr (Q == 19) {
    bp[0] = C(3) * (C(2) * a_xxy + a_zzy);
    bp[1] = C(3) * (a_xxy + C(2) * a_zzy);
    bp[2] = C(3) * (C(2) * a_xxz + a_yyz);
    bp[3] = C(3) * (a_xxz + C(2) * a_yyz);
    bp[4] = C(3) * (C(2) * a_yyx + a_zzx);
    bp[5] = C(3) * (a_yyx + C(2) * a_zzx);
  } else {
    bp[0] = C(4.5) * a_xxy;
    bp[1] = C(4.5) * a_zzy;
    bp[2] = C(4.5) * a_xxz;
    bp[3] = C(4.5) * a_yyz;
    bp[4] = C(4.5) * a_yyx;
    bp[5] = C(4.5) * a_zzx;
    const C a_xyz = rho * uex * uey * uez + k * (uhx * Ayz + uhy * Axz + uhz * Axy);
    bxyz = C(27) * a_xyz;
  }
  h[0] = wgt<Q, C>(0) * base;
  sfor<1, H + 1>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    const C cu = cdot_i<Q, i>(uex, uey, uez);
    // c . (k A) . c without the zero terms
    C cac = C(0);
    if constexpr (cx != 0) cac += Axx;
    if constexpr (cy != 0) cac += Ayy;
    if constexpr (cz != 0) cac += Azz;
    if constexpr (cx * cy != 0) cac += cmul<2 * cx * cy>(Axy);
    if constexpr (cx * cz != 0) cac += cmul<2 * cx * cz>(Axz);
    if constexpr (cy * cz != 0) cac += cmul<2 * cy * cz>(Ayz);
    const C sym = base + r45 * (cu * cu) + k45 * cac;
    C t3 = r3 * cu;
    t3 = acc_m<h3_m<Q, i, 0>()>(t3, bp[0]);
    t3 = acc_m<h3_m<Q, i, 1>()>(t3, bp[1]);
    t3 = acc_m<h3_m<Q, i, 2>()>(t3, bp[2]);
    t3 = acc_m<h3_m<Q, i, 3>()>(t3, bp[3]);
    t3 = acc_m<h3_m<Q, i, 4>()>(t3, bp[4]);
    t3 = acc_m<h3_m<Q, i, 5>()>(t3, bp[5]);
    if constexpr (Q == 27) t3 = acc_m<cx * cy * cz>(t3, bxyz);
    h[i] = wgt<Q, C>(i) * (sym + t3);
    h[i + H] = wgt<Q, C>(i) * (sym - t3);
  });
}

// HRR update of a fluid cell (local moments, Smagorinsky tau from Pi^neq, hybrid A2 with the
// finite-difference strain S = (xx, yy, zz, xy, xz, yz), unused when sigma = 1). Returns the density
// and the reported velocity u + F/(2 rho).
template <int Q, class C>
__device__ __forceinline__ void collide_hrr(C* h, C gamma, const Args& a, const C* S, C& rho_o, C& urx, C& ury, C& urz) {
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
  // Pi^neq = sum c c h - drho/3 I - rho u u
  const C d3 = drho * C(1.0 / 3.0);
  C A[6];
  A[0] = sxx - d3 - rho * ux * ux;
  A[1] = syy - d3 - rho * uy * uy;
  A[2] = szz - d3 - rho * uz * uz;
  A[3] = sxy - rho * ux * uy;
  A[4] = sxz - rho * ux * uz;
  A[5] = syz - rho * uy * uz;
  C tau = a.tau0.get<C>();
  if (a.use_smag != 0) {
    const C pn = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2] + C(2) * (A[3] * A[3] + A[4] * A[4] + A[5] * A[5]));
    const C t0 = a.tau0.get<C>();
    tau = C(0.5) * (t0 + sqrt(t0 * t0 + a.smag.get<C>() * pn * ir));
  }
  if (a.hybrid != 0) {
    const C sg = a.sigma.get<C>();
    const C fd = (C(1) - sg) * (C(-2.0 / 3.0) * rho * tau);
    sfor<0, 6>([&](auto I) { A[I] = sg * A[I] + fd * S[I]; });
  }
  const C k = C(1) - rcp(tau);
  const C uhx = gamma * ux, uhy = gamma * uy, uhz = gamma * uz;
  hrr_relax<Q, C>(h, drho, rho, uhx + a.fx.get<C>() * ir, uhy + a.fy.get<C>() * ir, uhz + a.fz.get<C>() * ir, uhx, uhy,
                  uhz, k, A);
  rho_o = rho;
  const C hf = C(0.5) * ir;
  urx = ux + a.fx.get<C>() * hf;
  ury = uy + a.fy.get<C>() * hf;
  urz = uz + a.fz.get<C>() * hf;
}

// HRR form of the WALL-cell update (sigma = 0): third-order equilibrium at u^B + F/rho, A2 =
// -2/3 rho tau S from the wall-model strain, A3 expanded around u^B.
template <int Q, class C>
__device__ __forceinline__ void collide_wall_hrr(C* h, const Args& a, const C* ws, C& rho_o, C& urx, C& ury, C& urz) {
  C drho, jx, jy, jz;
  sums<Q, C>(h, drho, jx, jy, jz);
  const C rho = C(1) + drho, ir = rcp(rho);
  rho_o = rho;
  const C hf = C(0.5) * ir;
  urx = jx * ir + a.fx.get<C>() * hf;
  ury = jy * ir + a.fy.get<C>() * hf;
  urz = jz * ir + a.fz.get<C>() * hf;
  const C tau = ws[3];
  const C g = C(-2.0 / 3.0) * rho * tau;
  C A[6];
  sfor<0, 6>([&](auto I) { A[I] = g * ws[4 + I]; });
  hrr_relax<Q, C>(h, drho, rho, ws[0] + a.fx.get<C>() * ir, ws[1] + a.fy.get<C>() * ir, ws[2] + a.fz.get<C>() * ir,
                  ws[0], ws[1], ws[2], C(1) - rcp(tau), A);
}

// ---- the HRR update of two cells at once with packed FP32 instructions (16-bit paired kernel) --------
// r + M v for a compile-time small integer M, packed lanes
template <int M> __device__ __forceinline__ float2 accm2(float2 r, float2 v) {
  if constexpr (M == 0) return r;
  else if constexpr (M == 1) return add2(r, v);
  else if constexpr (M == -1) return sub2(r, v);
  else return fma2(bc2(float(M)), v, r);
}

// hrr_relax for two cells (lane x, lane y); same formulas, each lane rounded as the scalar form.
template <int Q>
__device__ __forceinline__ void hrr_relax_x2(float2* h, float2 drho, float2 rho, float2 uex, float2 uey, float2 uez,
                                             float2 uhx, float2 uhy, float2 uhz, float2 k, const float2* A) {
  constexpr int H = Lat<Q>::H;
  const float2 Axx = A[0], Ayy = A[1], Azz = A[2], Axy = A[3], Axz = A[4], Ayz = A[5];
  const float2 usq = fma2(uex, uex, fma2(uey, uey, mul2(uez, uez)));
  const float2 c15 = bc2(1.5f), two = bc2(2.f);
  const float2 base = sub2(sub2(drho, mul2(mul2(c15, rho), usq)), mul2(mul2(c15, k), add2(add2(Axx, Ayy), Azz)));
  const float2 r45 = mul2(bc2(4.5f), rho), r3 = mul2(bc2(3.f), rho), k45 = mul2(bc2(4.5f), k);
  const float2 rxx = mul2(mul2(rho, uex), uex), ryy = mul2(mul2(rho, uey), uey), rzz = mul2(mul2(rho, uez), uez);
  const float2 a_xxy = fma2(rxx, uey, mul2(k, fma2(mul2(two, uhx), Axy, mul2(uhy, Axx))));
  const float2 a_zzy = fma2(rzz, uey, mul2(k, fma2(mul2(two, uhz), Ayz, mul2(uhy, Azz))));
  const float2 a_xxz = fma2(rxx, uez, mul2(k, fma2(mul2(two, uhx), Axz, mul2(uhz, Axx))));
  const float2 a_yyz = fma2(ryy, uez, mul2(k, fma2(mul2(two, uhy), Ayz, mul2(uhz, Ayy))));
  const float2 a_yyx = fma2(ryy, uex, mul2(k, fma2(mul2(two, uhy), Axy, mul2(uhx, Ayy))));
  const float2 a_zzx = fma2(rzz, uex, mul2(k, fma2(mul2(two, uhz), Axz, mul2(uhx, Azz))));
  float2 bp[6], bxyz = bc2(0.f);
  if constexpr (Q == 19) {
    const float2 c3 = bc2(3.f);
    bp[0] = mul2(c3, fma2(two, a_xxy, a_zzy));
    bp[1] = mul2(c3, fma2(two, a_zzy, a_xxy));
    bp[2] = mul2(c3, fma2(two, a_xxz, a_yyz));
    bp[3] = mul2(c3, fma2(two, a_yyz, a_xxz));
    bp[4] = mul2(c3, fma2(two, a_yyx, a_zzx));
    bp[5] = mul2(c3, fma2(two, a_zzx, a_yyx));
  } else {
    const float2 c45 = bc2(4.5f);
    bp[0] = mul2(c45, a_xxy);
    bp[1] = mul2(c45, a_zzy);
    bp[2] = mul2(c45, a_xxz);
    bp[3] = mul2(c45, a_yyz);
    bp[4] = mul2(c45, a_yyx);
    bp[5] = mul2(c45, a_zzx);
    const float2 a_xyz = fma2(mul2(mul2(rho, uex), uey), uez, mul2(k, fma2(uhx, Ayz, fma2(uhy, Axz, mul2(uhz, Axy)))));
    bxyz = mul2(bc2(27.f), a_xyz);
  }
  h[0] = mul2(bc2(wgt<Q, float>(0)), base);
  sfor<1, H + 1>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    static_assert(csign<Q, i>() > 0, "the first half of the velocity set has a positive leading component");
    const float2 cu = cdot2<Q, i>(uex, uey, uez);
    float2 cac = bc2(0.f);
    if constexpr (cx != 0) cac = add2(cac, Axx);
    if constexpr (cy != 0) cac = add2(cac, Ayy);
    if constexpr (cz != 0) cac = add2(cac, Azz);
    if constexpr (cx * cy != 0) cac = accm2<2 * cx * cy>(cac, Axy);
    if constexpr (cx * cz != 0) cac = accm2<2 * cx * cz>(cac, Axz);
    if constexpr (cy * cz != 0) cac = accm2<2 * cy * cz>(cac, Ayz);
    const float2 sym = fma2(k45, cac, fma2(r45, mul2(cu, cu), base));
    float2 t3 = mul2(r3, cu);
    t3 = accm2<h3_m<Q, i, 0>()>(t3, bp[0]);
    t3 = accm2<h3_m<Q, i, 1>()>(t3, bp[1]);
    t3 = accm2<h3_m<Q, i, 2>()>(t3, bp[2]);
    t3 = accm2<h3_m<Q, i, 3>()>(t3, bp[3]);
    t3 = accm2<h3_m<Q, i, 4>()>(t3, bp[4]);
    t3 = accm2<h3_m<Q, i, 5>()>(t3, bp[5]);
    if constexpr (Q == 27) t3 = accm2<cx * cy * cz>(t3, bxyz);
    const float2 w = bc2(wgt<Q, float>(i));
    h[i] = mul2(w, add2(sym, t3));
    h[i + H] = mul2(w, sub2(sym, t3));
  });
}

// collide_hrr for two cells; S holds the six strain components of both cells (unused when sigma =
// 1). Returns false when either cell's density or velocity is not finite; ur* = reported velocity.
template <int Q>
__device__ __forceinline__ bool collide_hrr_x2(float2* h, float2 gamma, const Args& a, const float2* S, float2& urx,
                                               float2& ury, float2& urz) {
  constexpr int H = Lat<Q>::H;
  const float2 z2 = bc2(0.f);
  float2 drho = h[0], jx = z2, jy = z2, jz = z2;
  float2 sxx = z2, syy = z2, szz = z2, sxy = z2, sxz = z2, syz = z2;
  sfor<1, H + 1>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    const float2 sp = add2(h[i], h[i + H]), dp = sub2(h[i], h[i + H]);
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
  const float2 d3 = mul2(drho, bc2(1.f / 3.f));
  const float2 rux = mul2(rho, ux), ruy = mul2(rho, uy), ruz = mul2(rho, uz);
  float2 A[6];
  A[0] = sub2(sxx, fma2(rux, ux, d3));
  A[1] = sub2(syy, fma2(ruy, uy, d3));
  A[2] = sub2(szz, fma2(ruz, uz, d3));
  A[3] = sub2(sxy, mul2(rux, uy));
  A[4] = sub2(sxz, mul2(rux, uz));
  A[5] = sub2(syz, mul2(ruy, uz));
  const float t0 = a.tau0.f;
  float2 tau = bc2(t0);
  if (a.use_smag != 0) {
    const float2 off = fma2(A[3], A[3], fma2(A[4], A[4], mul2(A[5], A[5])));
    const float2 pn = sqrt2(fma2(bc2(2.f), off, fma2(A[0], A[0], fma2(A[1], A[1], mul2(A[2], A[2])))));
    tau = mul2(bc2(0.5f), add2(bc2(t0), sqrt2(fma2(bc2(a.smag.f), mul2(pn, ir), bc2(t0 * t0)))));
  }
  if (a.hybrid != 0) {
    const float2 sg = bc2(a.sigma.f);
    const float2 fd = mul2(sub2(one, sg), mul2(bc2(-2.f / 3.f), mul2(rho, tau)));
    sfor<0, 6>([&](auto I) { A[I] = fma2(sg, A[I], mul2(fd, S[I])); });
  }
  const float2 k = sub2(one, rcp2(tau));
  const float2 uhx = mul2(gamma, ux), uhy = mul2(gamma, uy), uhz = mul2(gamma, uz);
  hrr_relax_x2<Q>(h, drho, rho, fma2(bc2(a.fx.f), ir, uhx), fma2(bc2(a.fy.f), ir, uhy), fma2(bc2(a.fz.f), ir, uhz), uhx,
                  uhy, uhz, k, A);
  const float2 hf = mul2(bc2(0.5f), ir);
  urx = fma2(bc2(a.fx.f), hf, ux);
  ury = fma2(bc2(a.fy.f), hf, uy);
  urz = fma2(bc2(a.fz.f), hf, uz);
  const float2 chk = add2(add2(abs2(rho), abs2(urx)), add2(abs2(ury), abs2(urz)));
  return chk.x < 1e30f && chk.y < 1e30f;
}

// Finite-difference strain (xx, yy, zz, xy, xz, yz) of cell (x, y, z) from the previous step's
// velocity field (3 component arrays of N). A neighbour x +- e_b is usable when it lies inside the
// domain after periodic wrap and is not SOLID: central difference with both, one-sided with one,
// zero with none. Cells that are not NEAR have all six neighbours usable.
template <class C>
__device__ __forceinline__ void strain_fd(const Args& a, int x, int y, int z, long long n, bool near, C* S) {
  const C* u = static_cast<const C*>(a.uvel_rd);
  const long long N = a.N;
  const int pos[3] = {x, y, z};
  const int ext[3] = {a.nx, a.ny, a.nz};
  const long long str[3] = {1, a.nx, a.nxy};
  C g[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    long long mp, mm;
    bool okp = true, okm = true;
    const int p = pos[b];
    if (p + 1 < ext[b]) mp = n + str[b];
    else if (a.face[2 * b + 1] == F_PERIODIC) mp = n - (long long)(ext[b] - 1) * str[b];
    else { okp = false; mp = n; }
    if (p > 0) mm = n - str[b];
    else if (a.face[2 * b] == F_PERIODIC) mm = n + (long long)(ext[b] - 1) * str[b];
    else { okm = false; mm = n; }
    if (near) {
      if (okp && (a.type[mp] & T_KIND) == K_SOLID) okp = false;
      if (okm && (a.type[mm] & T_KIND) == K_SOLID) okm = false;
    }
    const C hw = (okp && okm) ? C(0.5) : ((okp || okm) ? C(1) : C(0));
    if (!okp) mp = n;
    if (!okm) mm = n;
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c][b] = hw * (u[c * N + mp] - u[c * N + mm]);
  }
  S[0] = g[0][0];
  S[1] = g[1][1];
  S[2] = g[2][2];
  S[3] = C(0.5) * (g[0][1] + g[1][0]);
  S[4] = C(0.5) * (g[0][2] + g[2][0]);
  S[5] = C(0.5) * (g[1][2] + g[2][1]);
}

// Velocity-field record of the step (reported velocity of every updated cell).
template <class C>
__device__ __forceinline__ void record_velocity(const Args& a, long long n, C ux, C uy, C uz) {
  C* w = static_cast<C*>(a.uvel_wr);
  w[n] = ux;
  w[a.N + n] = uy;
  w[2 * a.N + n] = uz;
}

}  // namespace lbm
