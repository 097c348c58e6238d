// Hand-written reverse mode of the per-cell update (differentiation extension).
//
// The step is S_{t+1} = P(C(S_t)) with C the per-cell collision (boundary reconstruction, then
// BGK + Smagorinsky + porosity + force) and P the streaming permutation with its substitutions.
// The adjoint pulls mu = P^T lambda_{t+1} through the same slot map and applies C'^T per cell:
//   f*_i = f^eq_i(rho, v) + k (f_i - f^eq_i(rho, u)),  u = j/rho,  v = gamma u + F/rho,
//   k = 1 - 1/tau,  tau = (tau0 + sqrt(tau0^2 + K |Pi|/rho))/2,  K = 18 sqrt(2) C_S^2,
//   Pi = sum c c f - rho/3 I - rho u u   (six independent components, Frobenius norm |Pi|).
// With f^eq_i = w_i rho A_i(v), A_i(v) = 1 + 3 c.v + 4.5 (c.v)^2 - 1.5 v.v, every sum over
// populations of mu_i w_i (...) reduces to the moments m0, m1, m2 of mu_i w_i.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

struct AdjArgs {
  const void* fst;     // S_t, natural layout, storage type
  const void* lam_in;  // lambda_{t+1}, natural layout, compute type
  void* lam_out;       // lambda_t
  double* dgam;        // dJ/dgamma accumulator (FP64, N) or null
  double* duin;        // dJ/du_in accumulator (FP64, 3 ny nz) or null
  int add_dj;          // add the objective weights to lambda_t (window step)
  int xa, xb;
  double wa, wb;
};

template <int Q, class C>
struct WMoments {
  C m0, m1x, m1y, m1z, mxx, myy, mzz, mxy, mxz, myz;
};

template <int Q, class C>
__device__ __forceinline__ WMoments<Q, C> wmoments(const C* g) {
  WMoments<Q, C> m{};
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    const C v = wgt<Q, C>(i) * g[i];
    m.m0 += v;
    if (cx) m.m1x += C(cx) * v;
    if (cy) m.m1y += C(cy) * v;
    if (cz) m.m1z += C(cz) * v;
    if (cx) m.mxx += v;
    if (cy) m.myy += v;
    if (cz) m.mzz += v;
    if (cx * cy) m.mxy += C(cx * cy) * v;
    if (cx * cz) m.mxz += C(cx * cz) * v;
    if (cy * cz) m.myz += C(cy * cz) * v;
  });
  return m;
}

// sum_i g_i w_i A_i(v) and d/dv_a of sum_i g_i w_i rho A_i(v).
template <int Q, class C>
__device__ __forceinline__ void a_terms(const WMoments<Q, C>& m, C rho, C vx, C vy, C vz, C& A, C& gx, C& gy, C& gz) {
  const C vsq = vx * vx + vy * vy + vz * vz;
  const C m2vx = m.mxx * vx + m.mxy * vy + m.mxz * vz;
  const C m2vy = m.mxy * vx + m.myy * vy + m.myz * vz;
  const C m2vz = m.mxz * vx + m.myz * vy + m.mzz * vz;
  A = m.m0 + C(3) * (m.m1x * vx + m.m1y * vy + m.m1z * vz) + C(4.5) * (m2vx * vx + m2vy * vy + m2vz * vz) - C(1.5) * vsq * m.m0;
  gx = rho * (C(3) * m.m1x + C(9) * m2vx - C(3) * vx * m.m0);
  gy = rho * (C(3) * m.m1y + C(9) * m2vy - C(3) * vy * m.m0);
  gz = rho * (C(3) * m.m1z + C(9) * m2vz - C(3) * vz * m.m0);
}

// Reverse of collide_fluid: h = pre-collision deviations (after boundary reconstruction),
// mu = dJ/dh*, returns lam = dJ/dh and adds dJ/dgamma to ggam.
template <int Q, class C>
__device__ __forceinline__ void collide_fluid_vjp(const C* h, C gamma, const Args& a, const C* mu, C* lam, C& ggam) {
  C drho, jx, jy, jz;
  sums<Q, C>(h, drho, jx, jy, jz);
  const C rho = C(1) + drho, ir = C(1) / rho;
  const C ux = jx * ir, uy = jy * ir, uz = jz * ir;
  C tau = a.tau0.get<C>();
  C pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0, pn = 0, sD = 0;
  const bool smag = a.use_smag != 0;
  if (smag) {
    C sxx = 0, syy = 0, szz = 0, sxy = 0, sxz = 0, syz = 0;
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
      if (cx) sxx += h[i];
      if (cy) syy += h[i];
      if (cz) szz += h[i];
      if (cx * cy) sxy += C(cx * cy) * h[i];
      if (cx * cz) sxz += C(cx * cz) * h[i];
      if (cy * cz) syz += C(cy * cz) * h[i];
    });
    const C d3 = drho * C(1.0 / 3.0);
    pxx = sxx - d3 - rho * ux * ux; pyy = syy - d3 - rho * uy * uy; pzz = szz - d3 - rho * uz * uz;
    pxy = sxy - rho * ux * uy; pxz = sxz - rho * ux * uz; pyz = syz - rho * uy * uz;
    pn = sqrt(pxx * pxx + pyy * pyy + pzz * pzz + C(2) * (pxy * pxy + pxz * pxz + pyz * pyz));
    const C t0 = a.tau0.get<C>();
    sD = sqrt(t0 * t0 + a.smag.get<C>() * pn * ir);
    tau = C(0.5) * (t0 + sD);
  }
  const C k = C(1) - C(1) / tau;
  const C vx = gamma * ux + a.fx.get<C>() * ir, vy = gamma * uy + a.fy.get<C>() * ir, vz = gamma * uz + a.fz.get<C>() * ir;

  const WMoments<Q, C> m = wmoments<Q, C>(mu);
  C smh = C(0);
  sfor<0, Q>([&](auto I) { smh += mu[I] * h[I]; });
  C Av, gvx, gvy, gvz, Au, gux, guy, guz;
  a_terms<Q, C>(m, rho, vx, vy, vz, Av, gvx, gvy, gvz);
  a_terms<Q, C>(m, rho, ux, uy, uz, Au, gux, guy, guz);
  gux *= -k; guy *= -k; guz *= -k;
  C grho = Av - k * Au;
  const C G = smh - (rho * Au - m.m0);  // dJ/dk
  // v = gamma u + F / rho
  gux += gamma * gvx; guy += gamma * gvy; guz += gamma * gvz;
  ggam += ux * gvx + uy * gvy + uz * gvz;
  grho -= (a.fx.get<C>() * gvx + a.fy.get<C>() * gvy + a.fz.get<C>() * gvz) * ir * ir;
  C gjx = 0, gjy = 0, gjz = 0;
  C gsxx = 0, gsyy = 0, gszz = 0, gsxy = 0, gsxz = 0, gsyz = 0;
  if (smag) {
    const C gtau = G / (tau * tau);
    const C Ks = a.smag.get<C>();
    const C gpn = gtau * Ks / (C(4) * sD) * ir;
    grho -= gtau * Ks * pn / (C(4) * sD) * ir * ir;
    if (pn > C(0)) {
      const C s = gpn / pn;
      gsxx = s * pxx; gsyy = s * pyy; gszz = s * pzz;
      gsxy = C(2) * s * pxy; gsxz = C(2) * s * pxz; gsyz = C(2) * s * pyz;
      grho += -(gsxx + gsyy + gszz) * C(1.0 / 3.0) +
              (gsxx * jx * jx + gsyy * jy * jy + gszz * jz * jz + gsxy * jx * jy + gsxz * jx * jz + gsyz * jy * jz) * ir * ir;
      gjx -= (C(2) * gsxx * jx + gsxy * jy + gsxz * jz) * ir;
      gjy -= (C(2) * gsyy * jy + gsxy * jx + gsyz * jz) * ir;
      gjz -= (C(2) * gszz * jz + gsxz * jx + gsyz * jy) * ir;
    }
  }
  // u = j / rho
  gjx += gux * ir; gjy += guy * ir; gjz += guz * ir;
  grho -= (gux * ux + guy * uy + guz * uz) * ir;
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    C v = k * mu[i] + grho;
    if constexpr (i != 0) v += cdot_i<Q, i>(gjx, gjy, gjz);
    if constexpr (cx != 0) v += gsxx;
    if constexpr (cy != 0) v += gsyy;
    if constexpr (cz != 0) v += gszz;
    if constexpr (cx * cy != 0) v += cmul<cx * cy>(gsxy);
    if constexpr (cx * cz != 0) v += cmul<cx * cz>(gsxz);
    if constexpr (cy * cz != 0) v += cmul<cy * cz>(gsyz);
    lam[i] = v;
  });
}

// Reverse of the regularised reconstruction with (rho, u) given: gout = dJ/dh' (output populations);
// returns gne-derived direct gradients gh (known populations only), and the gradients of the
// equilibrium with respect to rho and u.
template <int Q, class C, class Known>
__device__ __forceinline__ void regularise_vjp(C rho, C ux, C uy, C uz, const C* gout, C* gh, C& grho, C& gux, C& guy,
                                               C& guz) {
  C gpxx = 0, gpyy = 0, gpzz = 0, gpxy = 0, gpxz = 0, gpyz = 0;
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    const C g = wgt<Q, C>(i) * C(4.5) * gout[i];
    gpxx += C(cx * cx - 1.0 / 3.0) * g;
    gpyy += C(cy * cy - 1.0 / 3.0) * g;
    gpzz += C(cz * cz - 1.0 / 3.0) * g;
    if (cx * cy) gpxy += C(2 * cx * cy) * g;
    if (cx * cz) gpxz += C(2 * cx * cz) * g;
    if (cy * cz) gpyz += C(2 * cy * cz) * g;
  });
  C gne[Q];
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value, cx = Lat<Q>::cx(i), cy = Lat<Q>::cy(i), cz = Lat<Q>::cz(i);
    C v = C(0);
    if constexpr (cx != 0) v += gpxx;
    if constexpr (cy != 0) v += gpyy;
    if constexpr (cz != 0) v += gpzz;
    if constexpr (cx * cy != 0) v += cmul<cx * cy>(gpxy);
    if constexpr (cx * cz != 0) v += cmul<cx * cz>(gpxz);
    if constexpr (cy * cz != 0) v += cmul<cy * cz>(gpyz);
    gne[i] = v;
  });
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (!Known{}(i)) {
      gne[opp<Q>(i)] += gne[i];
      gne[i] = C(0);
    }
  });
  C gheq[Q];
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    gh[i] = gne[i];
    gheq[i] = gout[i] - gne[i];
  });
  const WMoments<Q, C> m = wmoments<Q, C>(gheq);
  a_terms<Q, C>(m, rho, ux, uy, uz, grho, gux, guy, guz);
}

// Reverse of bc_inlet: h = gathered deviations, gout = dJ/dh'; lam = dJ/dh; gub += dJ/du_b.
// Forward: s = sum_{c_x=0} h + 2 sum_{c_x<0} h, drho = (s + u_x)/(1 - u_x), rho = 1 + drho.
template <int Q, class C>
__device__ __forceinline__ void bc_inlet_vjp(const C* h, C ubx, C uby, C ubz, const C* gout, C* lam, C* gub) {
  C s = C(0);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (Lat<Q>::cx(i) == 0) s += h[i];
    if (Lat<Q>::cx(i) < 0) s += C(2) * h[i];
  });
  const C den = C(1) - ubx;
  const C rho = C(1) + (s + ubx) / den;
  C grho, gux, guy, guz;
  regularise_vjp<Q, C, KnownInlet<Q>>(rho, ubx, uby, ubz, gout, lam, grho, gux, guy, guz);
  // rho = (1 + s) / (1 - u_x): d rho/ds = 1/den, d rho/du_x = (1 + s)/den^2
  const C gs = grho / den;
  gux += grho * (C(1) + s) / (den * den);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (Lat<Q>::cx(i) == 0) lam[i] += gs;
    if (Lat<Q>::cx(i) < 0) lam[i] += C(2) * gs;
  });
  gub[0] += gux; gub[1] += guy; gub[2] += guz;
}

// Reverse of bc_outlet (u_x = (s - (rho_out - 1))/rho_out).
template <int Q, class C>
__device__ __forceinline__ void bc_outlet_vjp(const C* h, C rho_out, C drho_out, const C* gout, C* lam) {
  C s = C(0);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (Lat<Q>::cx(i) == 0) s += h[i];
    if (Lat<Q>::cx(i) > 0) s += C(2) * h[i];
  });
  const C ux = (s - drho_out) / rho_out;
  C grho, gux, guy, guz;
  regularise_vjp<Q, C, KnownOutlet<Q>>(rho_out, ux, C(0), C(0), gout, lam, grho, gux, guy, guz);
  const C gs = gux / rho_out;
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (Lat<Q>::cx(i) == 0) lam[i] += gs;
    if (Lat<Q>::cx(i) > 0) lam[i] += C(2) * gs;
  });
}

}  // namespace lbm
