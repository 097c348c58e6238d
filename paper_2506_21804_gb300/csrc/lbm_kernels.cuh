// Kernel templates of the fused collide-and-stream step and of the state access, reduction and
// adjoint passes. Instantiated per storage type in lbm_ops_<storage>.cu.
#pragma once

#include "lbm_device.cuh"
#include "lbm_hrr.cuh"
#include "lbm_adjoint.cuh"
#include "lbm_ops.h"

namespace lbm {

constexpr int BULK_THREADS = 128;
constexpr int LIST_THREADS = 128;

enum { LOAD_LOCAL = 0, LOAD_SLOTS = 1 };
enum { STORE_MIRROR = 0, STORE_SLOTS = 1 };

// Cell of the calling thread in a launch of cell_grid: first a.lc_cols column CTAs (each face plane
// x = 0, x = nx - 1 taken along y, lc_t cells of one z per CTA, the two faces alternating), then the row
// CTAs (lc_gx per x-row, rows in y-then-z order). Row threads on the face planes get skip when the
// column CTAs own those planes. in: the coordinates lie in the grid.
struct CellAt {
  int x, y, z;
  bool in, skip;
};
__device__ __forceinline__ CellAt cell_at(const Args& a) {
  CellAt c;
  const unsigned b = blockIdx.x;
  if (b < a.lc_cols) {
    const unsigned r = b >> 1, z = a.lc_dgy.div(r);
    c.x = (b & 1u) ? a.nx - 1 : 0;
    c.y = int((r - z * a.lc_gy) * a.lc_t + threadIdx.x);
    c.z = int(z);
    c.skip = false;
  } else {
    const unsigned br = b - a.lc_cols, row = a.lc_dgx.div(br), z = a.lc_dny.div(row);
    c.x = int((br - row * a.lc_gx) * a.lc_t + threadIdx.x);
    c.y = int(row - z * unsigned(a.ny));
    c.z = int(z);
    c.skip = a.xcols && (c.x == 0 || c.x == a.nx - 1);
  }
  c.in = c.x < a.nx && c.y < a.ny && c.z < a.nz;
  return c;
}

__device__ __forceinline__ void cell_coords(const Args& a, long long n, int& x, int& y, int& z) {
  if (a.N < (1LL << 31)) {  // 32-bit divisions (a 64-bit one is a long instruction sequence)
    const unsigned un = unsigned(n), r = un / unsigned(a.nx);
    x = int(un - r * unsigned(a.nx));
    z = int(r / unsigned(a.ny));
    y = int(r - unsigned(z) * unsigned(a.ny));
    return;
  }
  const long long r = n / a.nx;
  x = int(n - r * a.nx);
  z = int(r / a.ny);
  y = int(r - (long long)z * a.ny);
}

template <class C> __device__ __forceinline__ C gamma_at(const Args& a, long long n) {
  return a.gamma ? static_cast<const C*>(a.gamma)[n] : C(1);
}

// Neighbour index offsets of an interior cell in 32-bit arithmetic (periodic wrap folded into the
// six per-axis deltas); valid when every population index fits in 32 bits (Args::idx32).
struct Nbr32 {
  unsigned n;
  int dxm, dxp, dym, dyp, dzm, dzp;
  __device__ __forceinline__ Nbr32(const Args& a, int x, int y, int z, long long n_) {
    n = unsigned(n_);
    const int nx = a.nx, nxy = int(a.nxy);
    dxm = x == 0 ? nx - 1 : -1;
    dxp = x == nx - 1 ? 1 - nx : 1;
    dym = y == 0 ? (a.ny - 1) * nx : -nx;
    dyp = y == a.ny - 1 ? (1 - a.ny) * nx : nx;
    dzm = z == 0 ? (a.nz - 1) * nxy : -nxy;
    dzp = z == a.nz - 1 ? (1 - a.nz) * nxy : nxy;
  }
  // index of population p at the cell displaced by (dx, dy, dz)
  template <int DX, int DY, int DZ>
  __device__ __forceinline__ unsigned at(unsigned pbase) const {
    unsigned r = pbase + n;
    if constexpr (DX < 0) r += unsigned(dxm);
    if constexpr (DX > 0) r += unsigned(dxp);
    if constexpr (DY < 0) r += unsigned(dym);
    if constexpr (DY > 0) r += unsigned(dyp);
    if constexpr (DZ < 0) r += unsigned(dzm);
    if constexpr (DZ > 0) r += unsigned(dzp);
    return r;
  }
};

// Neighbour indices of the cell group x0 .. x0 + W - 1 (W = 2 pairs, 4 quads; x0 a multiple of W) in a
// launch whose CTA lies in one x-row (y = blockIdx.y, z = blockIdx.z): the y and z displacements with
// their periodic wrap are the same for every thread of the CTA, so they are computed once per warp,
// and only x0 - 1 (cell 0) and x0 + W (cell W - 1) can wrap per thread.
template <int W>
struct RowNbr {
  unsigned un, unm, unp;   // index of x0; the same with the x-wrap of x0 - 1 / x0 + W folded in
  int dym, dyp, dzm, dzp;  // uniform over the CTA
  __device__ __forceinline__ RowNbr(const Args& a, int x0, int y, int z, unsigned un_) {
    un = un_;
    unm = x0 == 0 ? un_ + unsigned(a.nx) : un_;
    unp = x0 + W == a.nx ? un_ - unsigned(a.nx) : un_;
    const int nx = a.nx, nxy = int(a.nxy);
    dym = y == 0 ? (a.ny - 1) * nx : -nx;
    dyp = y == a.ny - 1 ? (1 - a.ny) * nx : nx;
    dzm = z == 0 ? (a.nz - 1) * nxy : -nxy;
    dzp = z == a.nz - 1 ? (1 - a.nz) * nxy : nxy;
  }
  // index of population p at cell x0 + CELL displaced by (DX, DY, DZ)
  template <int CELL, int DX, int DY, int DZ>
  __device__ __forceinline__ unsigned at(unsigned pbase) const {
    unsigned u = pbase;
    if constexpr (DY < 0) u += unsigned(dym);
    if constexpr (DY > 0) u += unsigned(dyp);
    if constexpr (DZ < 0) u += unsigned(dzm);
    if constexpr (DZ > 0) u += unsigned(dzp);
    if constexpr (CELL == 0 && DX < 0) return u + unm - 1u;
    else if constexpr (CELL == W - 1 && DX > 0) return u + unp + unsigned(W);
    else return u + un + unsigned(CELL + DX);
  }
};

// L2 prefetch ahead of a row-form launch (16-bit storage). CTAs start in order of their linear index,
// so CTA L is followed by CTA L + LBM_PF_CTAS about half a CTA lifetime later; threads 0 .. Q of CTA L
// each ask the copy engine for one contiguous run of that later CTA's cells (the Q population arrays
// and the type bytes) with one bulk L2 prefetch, which needs no register and no wait, so the later
// CTA's loads find their lines in L2. The 16-bit kernels are bound by latency rather than bandwidth
// and gain from it (256^3 FP16 channel: 61.1 -> 62.8 GLUPS); the FP32 kernels, already near the
// bandwidth roofline, measured slower with it and do not prefetch. The runs start on 16-byte
// boundaries when nx is a multiple of 16 (else nothing is prefetched).
#ifndef LBM_PF_CTAS
#define LBM_PF_CTAS 512
#endif
template <int Q, class S>
__device__ __forceinline__ void row_prefetch(const Args& a, int cells_per_cta) {
  if constexpr (LBM_PF_CTAS > 0 && sizeof(S) == 2) {
    const int i = int(threadIdx.x);
    if (i > Q || (a.nx & 15)) return;
    const long long L = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z) + LBM_PF_CTAS;
    const long long row = L / gridDim.x;
    if (row >= (long long)a.ny * a.nz) return;
    const int x_begin = int(L - row * gridDim.x) * cells_per_cta;
    const int cells = min(cells_per_cta, a.nx - x_begin);
    const long long n = row * a.nx + x_begin;
    const char* p;
    unsigned bytes;
    if (i < Q) {
      p = reinterpret_cast<const char*>(static_cast<const S*>(a.f) + (long long)i * a.stride + n);
      bytes = unsigned(cells) * unsigned(sizeof(S));
    } else {
      p = reinterpret_cast<const char*>(a.type + n);
      bytes = unsigned(cells);
    }
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
  }
}

// Gather the Q deviations of cell n. LOAD_LOCAL: h_i from slot (i, n) of src (natural layout);
// LOAD_SLOTS: h_i from the AA slot of direction i (state after an even step).
template <int Q, class S, int LOAD>
__device__ __forceinline__ void gather(const Args& a, const S* src, int x, int y, int z, long long n, bool near,
                                       typename Codec<S>::C* h) {
  using C = typename Codec<S>::C;
  if constexpr (LOAD == LOAD_LOCAL) {
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      h[i] = Codec<S>::ld(src + (long long)i * a.stride + n);
    });
  } else {
    if (!near && a.idx32) {
      const Nbr32 nb(a, x, y, z, n);
      const unsigned us = unsigned(a.stride);
      sfor<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        h[i] = Codec<S>::ld(src + nb.template at<-Lat<Q>::cx(i), -Lat<Q>::cy(i), -Lat<Q>::cz(i)>(unsigned(opp<Q>(i)) * us));
      });
    } else if (!near) {
      const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
      const long long y0 = (long long)y * a.nx;
      const long long ym = (long long)(y == 0 ? a.ny - 1 : y - 1) * a.nx, yp = (long long)(y == a.ny - 1 ? 0 : y + 1) * a.nx;
      const long long z0 = (long long)z * a.nxy;
      const long long zm = (long long)(z == 0 ? a.nz - 1 : z - 1) * a.nxy, zp = (long long)(z == a.nz - 1 ? 0 : z + 1) * a.nxy;
      sfor<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int dx = -Lat<Q>::cx(i), dy = -Lat<Q>::cy(i), dz = -Lat<Q>::cz(i);
        const long long s = (dx < 0 ? xm : dx > 0 ? xp : x) + (dy < 0 ? ym : dy > 0 ? yp : y0) + (dz < 0 ? zm : dz > 0 ? zp : z0);
        h[i] = Codec<S>::ld(src + (long long)opp<Q>(i) * a.stride + s);
      });
    } else {
      sfor<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        int p;
        long long m;
        slot_of<Q>(a, x, y, z, n, i, p, m);
        h[i] = Codec<S>::ld(src + (long long)p * a.stride + m);
      });
    }
  }
}

// Write the post-collision deviations h*. STORE_MIRROR: h*_i into slot (opp(i), n) of dst (even
// step); STORE_SLOTS: h*_opp(i) into the AA slot of direction i (odd step, or out-of-place push
// into a natural-layout array).
template <int Q, class S, int STORE>
__device__ __forceinline__ void scatter(const Args& a, S* dst, int x, int y, int z, long long n, bool near,
                                        const typename Codec<S>::C* h) {
  if constexpr (STORE == STORE_MIRROR) {
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      Codec<S>::st(dst + (long long)opp<Q>(i) * a.stride + n, h[i]);
    });
  } else {
    if (!near && a.idx32) {
      const Nbr32 nb(a, x, y, z, n);
      const unsigned us = unsigned(a.stride);
      sfor<0, Q>([&](auto I) {
        constexpr int k = decltype(I)::value;  // outgoing direction: f*_k goes to slot (k, x + c_k)
        Codec<S>::st(dst + nb.template at<Lat<Q>::cx(k), Lat<Q>::cy(k), Lat<Q>::cz(k)>(unsigned(k) * us), h[k]);
      });
    } else if (!near) {
      const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
      const long long y0 = (long long)y * a.nx;
      const long long ym = (long long)(y == 0 ? a.ny - 1 : y - 1) * a.nx, yp = (long long)(y == a.ny - 1 ? 0 : y + 1) * a.nx;
      const long long z0 = (long long)z * a.nxy;
      const long long zm = (long long)(z == 0 ? a.nz - 1 : z - 1) * a.nxy, zp = (long long)(z == a.nz - 1 ? 0 : z + 1) * a.nxy;
      sfor<0, Q>([&](auto I) {
        constexpr int k = decltype(I)::value;  // outgoing direction: f*_k goes to slot (k, x + c_k)
        constexpr int dx = Lat<Q>::cx(k), dy = Lat<Q>::cy(k), dz = Lat<Q>::cz(k);
        const long long s = (dx < 0 ? xm : dx > 0 ? xp : x) + (dy < 0 ? ym : dy > 0 ? yp : y0) + (dz < 0 ? zm : dz > 0 ? zp : z0);
        Codec<S>::st(dst + (long long)k * a.stride + s, h[k]);
      });
    } else {
      sfor<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        int p;
        long long m;
        slot_of<Q>(a, x, y, z, n, i, p, m);
        Codec<S>::st(dst + (long long)p * a.stride + m, h[opp<Q>(i)]);
      });
    }
  }
}

// Odd-step access of a boundary-list cell with precomputed per-direction slot codes: 0 the plain
// (periodic-wrapped) neighbour slot, 1 the cell's own bounce-back slot (i, n), 2 the general rule.
struct Nbr {
  int x, xm, xp;
  long long y0, ym, yp, z0, zm, zp;
  __device__ __forceinline__ Nbr(const Args& a, int x_, int y, int z) {
    x = x_;
    xm = x == 0 ? a.nx - 1 : x - 1;
    xp = x == a.nx - 1 ? 0 : x + 1;
    y0 = (long long)y * a.nx;
    ym = (long long)(y == 0 ? a.ny - 1 : y - 1) * a.nx;
    yp = (long long)(y == a.ny - 1 ? 0 : y + 1) * a.nx;
    z0 = (long long)z * a.nxy;
    zm = (long long)(z == 0 ? a.nz - 1 : z - 1) * a.nxy;
    zp = (long long)(z == a.nz - 1 ? 0 : z + 1) * a.nxy;
  }
  __device__ __forceinline__ long long at(int dx, int dy, int dz) const {
    return (dx < 0 ? xm : dx > 0 ? xp : x) + (dy < 0 ? ym : dy > 0 ? yp : y0) + (dz < 0 ? zm : dz > 0 ? zp : z0);
  }
};

// Bit mask of the directions whose code is 2 (the general rule is needed).
__device__ __forceinline__ bool has_general(unsigned long long code) { return (code & 0xAAAAAAAAAAAAAAAAull) != 0; }

template <int Q, class S>
__device__ __forceinline__ void gather_coded(const Args& a, const S* src, int x, int y, int z, long long n,
                                             unsigned long long code, typename Codec<S>::C* h) {
  if (!has_general(code) && a.idx32) {
    // codes 0/1 only: the plain neighbour slot or the cell's own slot, chosen without branches
    const Nbr32 nb(a, x, y, z, n);
    const unsigned us = unsigned(a.stride), un = unsigned(n);
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const unsigned plain = nb.template at<-Lat<Q>::cx(i), -Lat<Q>::cy(i), -Lat<Q>::cz(i)>(unsigned(opp<Q>(i)) * us);
      const unsigned own = unsigned(i) * us + un;
      h[i] = Codec<S>::ld(src + (((code >> (2 * i)) & 1ull) ? own : plain));
    });
    return;
  }
  const Nbr nb(a, x, y, z);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int c = int(code >> (2 * i)) & 3;
    int p;
    long long m;
    if (c == 0) { p = opp<Q>(i); m = nb.at(-Lat<Q>::cx(i), -Lat<Q>::cy(i), -Lat<Q>::cz(i)); }
    else if (c == 1) { p = i; m = n; }
    else slot_of<Q>(a, x, y, z, n, i, p, m);
    h[i] = Codec<S>::ld(src + (long long)p * a.stride + m);
  });
}

template <int Q, class S>
__device__ __forceinline__ void scatter_coded(const Args& a, S* dst, int x, int y, int z, long long n,
                                              unsigned long long code, const typename Codec<S>::C* h) {
  if (!has_general(code) && a.idx32) {
    const Nbr32 nb(a, x, y, z, n);
    const unsigned us = unsigned(a.stride), un = unsigned(n);
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const unsigned plain = nb.template at<-Lat<Q>::cx(i), -Lat<Q>::cy(i), -Lat<Q>::cz(i)>(unsigned(opp<Q>(i)) * us);
      const unsigned own = unsigned(i) * us + un;
      Codec<S>::st(dst + (((code >> (2 * i)) & 1ull) ? own : plain), h[opp<Q>(i)]);
    });
    return;
  }
  const Nbr nb(a, x, y, z);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const int c = int(code >> (2 * i)) & 3;
    int p;
    long long m;
    if (c == 0) { p = opp<Q>(i); m = nb.at(-Lat<Q>::cx(i), -Lat<Q>::cy(i), -Lat<Q>::cz(i)); }
    else if (c == 1) { p = i; m = n; }
    else slot_of<Q>(a, x, y, z, n, i, p, m);
    Codec<S>::st(dst + (long long)p * a.stride + m, h[opp<Q>(i)]);
  });
}

// Slot code of a cell for the adjoint and recompute passes: list and NEAR cells read theirs from the
// per-cell code array; other cells use plain slots.
__device__ __forceinline__ unsigned long long cell_code(const Args& a, long long n, uint8_t t) {
  return (t & (T_LIST | T_NEAR)) ? a.ccode[n] : 0ull;
}

template <class C> __device__ __forceinline__ const C* cptr(const void* p) { return static_cast<const C*>(p); }
template <class C> __device__ __forceinline__ C* cptr(void* p) { return static_cast<C*>(p); }

// Outlet fringe zone (Sec. 3.2: the fixed-pressure outlet has a fringe zone in front of it; the
// paper gives no parameters, so the layer is a reading): in the last planes x >= fr_x0 the
// post-collision deviations of every cell other than INFLOW/OUTFLOW relax towards the equilibrium at
// the outlet density and the cell's reported velocity, h*_i <- h*_i - s(x) (h*_i - (f^eq_i(rho_out, u)
// - w_i)), with s(x) = s_max xi^p tabulated per plane on the host.
template <int Q, class C>
__device__ __forceinline__ void apply_fringe(const Args& a, int x, int kind, C urx, C ury, C urz, C* h) {
  if (a.fringe == nullptr || x < a.fr_x0 || kind == K_INFLOW || kind == K_OUTFLOW) return;
  const C s = static_cast<const C*>(a.fringe)[x];
  const C ro = a.rho_out.get<C>(), dro = a.drho_out.get<C>();
  const C usq = urx * urx + ury * ury + urz * urz;
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    h[i] -= s * (h[i] - heq<Q, C, i>(dro, ro, urx, ury, urz, usq));
  });
}

// Boundary reconstruction of INFLOW/OUTFLOW cells (in place on h).
template <int Q, class C>
__device__ __forceinline__ void apply_bc(const Args& a, int kind, int y, int z, C* h) {
  if (kind == K_INFLOW) {
    const C* ub = cptr<C>(a.uin);
    const long long pl = (long long)a.ny * a.nz, p = y + (long long)a.ny * z;
    bc_inlet<Q, C>(h, ub[p], ub[pl + p], ub[2 * pl + p]);
  } else if (kind == K_OUTFLOW) {
    bc_outlet<Q, C>(h, a.rho_out.get<C>(), a.drho_out.get<C>());
  }
}

// Collision of a cell of any non-solid kind (boundary reconstruction first, then fluid or wall
// model). k = list entry for reference-velocity bookkeeping (-1: not a list cell).
template <int Q, class C, bool HRR = false>
__device__ __forceinline__ void collide_any(const Args& a, int kind, uint8_t t, int x, int y, int z, long long n, int k, C* h) {
  apply_bc<Q, C>(a, kind, y, z, h);
  C rho, urx, ury, urz;
  if (kind == K_WALL && a.wm) {
    // fused mode: the wall-model state pass has already solved every WALL entry of this step
    C ws_own[WALL_STATE];
    const C* ws = cptr<C>(a.wst) + (long long)WALL_STATE * k;
    if (!a.fuse) {
      const C* nr = cptr<C>(a.wnrm) + 3 * (long long)k;
      const int r = a.wref[k];
      const C* ur = r >= 0 ? cptr<C>(a.ref_rd) + 3 * (long long)r : nullptr;
      C z3[3] = {C(0), C(0), C(0)};
      wall_state<C>(a, nr, cptr<C>(a.wyw)[k], r >= 0 ? ur : z3, r >= 0, ws_own);
      ws = ws_own;
    }
    if constexpr (HRR) collide_wall_hrr<Q, C>(h, a, ws, rho, urx, ury, urz);
    else collide_wall_state<Q, C>(h, a, ws, rho, urx, ury, urz);
  } else if constexpr (HRR) {
    C Sfd[6] = {C(0), C(0), C(0), C(0), C(0), C(0)};
    if (a.hybrid) strain_fd<C>(a, x, y, z, n, (t & T_NEAR) != 0, Sfd);
    collide_hrr<Q, C>(h, gamma_at<C>(a, n), a, Sfd, rho, urx, ury, urz);
  } else {
    collide_fluid<Q, C>(h, gamma_at<C>(a, n), a, rho, urx, ury, urz);
  }
  apply_fringe<Q, C>(a, x, kind, urx, ury, urz, h);
  if ((t & T_REF) && k >= 0) {
    C* w = cptr<C>(a.ref_wr) + 3 * (long long)k;
    w[0] = urx; w[1] = ury; w[2] = urz;
  }
  if constexpr (HRR) record_velocity<C>(a, n, urx, ury, urz);
  if (!finite_all<C>(rho, urx, ury, urz)) atomicOr(a.status, ST_NAN);
}

// ---- the step kernels ----------------------------------------------------------------------------------
// A list cell updated inside the interior kernel (fused mode): its entry gives the slot codes, the
// precomputed wall-model state and the reference-buffer position. Inlet/outlet lanes add their
// boundary reconstruction before the collision; the collision itself is shared with plain lanes.
template <int Q, class S, bool ODD, bool HRR = false>
__device__ __forceinline__ void list_cell_inline(const Args& a, S* f, int x, int y, int z, long long n, uint8_t t) {
  using C = typename Codec<S>::C;
  const int k = a.lidx[n];
  const int kind = t & T_KIND;
  C h[Q];
  unsigned long long code = 0;
  if constexpr (ODD) {
    code = a.lcode[k];
    gather_coded<Q, S>(a, f, x, y, z, n, code, h);
  } else {
    gather<Q, S, LOAD_LOCAL>(a, f, x, y, z, n, false, h);
  }
  if (kind == K_INFLOW || kind == K_OUTFLOW) apply_bc<Q, C>(a, kind, y, z, h);
  C rho, urx, ury, urz;
  if constexpr (HRR) {
    if (kind == K_WALL && a.wm) {
      collide_wall_hrr<Q, C>(h, a, cptr<C>(a.wst) + (long long)WALL_STATE * k, rho, urx, ury, urz);
    } else {
      C Sfd[6] = {C(0), C(0), C(0), C(0), C(0), C(0)};
      if (a.hybrid) strain_fd<C>(a, x, y, z, n, (t & T_NEAR) != 0, Sfd);
      collide_hrr<Q, C>(h, gamma_at<C>(a, n), a, Sfd, rho, urx, ury, urz);
    }
    record_velocity<C>(a, n, urx, ury, urz);
  } else {
    if (kind == K_WALL && a.wm) collide_wall_state<Q, C>(h, a, cptr<C>(a.wst) + (long long)WALL_STATE * k, rho, urx, ury, urz);
    else collide_fluid<Q, C>(h, gamma_at<C>(a, n), a, rho, urx, ury, urz);
  }
  apply_fringe<Q, C>(a, x, kind, urx, ury, urz, h);
  if (t & T_REF) {
    C* w = cptr<C>(a.ref_wr) + 3 * (long long)k;
    w[0] = urx; w[1] = ury; w[2] = urz;
  }
  if (!finite_all<C>(rho, urx, ury, urz)) atomicOr(a.status, ST_NAN);
  if constexpr (ODD) scatter_coded<Q, S>(a, f, x, y, z, n, code, h);
  else scatter<Q, S, STORE_MIRROR>(a, f, x, y, z, n, false, h);
}

// Interior kernel: every FLUID cell off the boundary list, and in fused mode also the list cells
// flagged T_INLINE (inlet/outlet cells, and WALL and reference cells in 32-cell x-groups dense in
// list cells, where the extra path costs little divergence). Threads map to (x, y, z).
//
// Occupancy target (CTAs of 128 threads per SM): D3Q19 10 on even steps (<= 51 registers) and 8 on
// odd steps (<= 64), D3Q27 8 and 7 (measured on the 512x512x256 canopy with every odd-step warp on the
// mixed path: D3Q27 odd 5, 6, 7, 8 gave 24.0, 24.8, 25.3, 25.0 GLUPS; D3Q19 odd 7, 8, 10 gave 34.4,
// 35.1, 34.0); the register cap falls on the rarely taken list-cell path. The FP64 (reference) form
// is left unconstrained.
#ifndef LBM_BULK_MINB19_EVEN
#define LBM_BULK_MINB19_EVEN 10
#endif
#ifndef LBM_BULK_MINB19_ODD
#define LBM_BULK_MINB19_ODD 8
#endif
#ifndef LBM_BULK_MINB27_EVEN
#define LBM_BULK_MINB27_EVEN 8
#endif
#ifndef LBM_BULK_MINB27_ODD
#define LBM_BULK_MINB27_ODD 7
#endif
template <int Q, class S, bool ODD> constexpr int bulk_min_blocks() {
  return sizeof(S) == 8 ? 1
                        : (Q == 19 ? (ODD ? LBM_BULK_MINB19_ODD : LBM_BULK_MINB19_EVEN)
                                   : (ODD ? LBM_BULK_MINB27_ODD : LBM_BULK_MINB27_EVEN));
}

template <int Q, class S, bool ODD, bool HRR = false>
__device__ __forceinline__ void bulk_cell(const Args& a, S* f, int x, int y, int z, long long n, uint8_t t) {
  using C = typename Codec<S>::C;
  if (t & (T_LIST | T_KIND | T_GHOST)) {
    // list cells updated here (T_INLINE, or every list cell when inline_all); solid cells, ghost
    // cells and the list cells of the boundary-list kernel are skipped
    if ((t & (T_LIST | T_GHOST)) == T_LIST && a.fuse && ((t & T_INLINE) || a.inline_all))
      list_cell_inline<Q, S, ODD, HRR>(a, f, x, y, z, n, t);
    return;
  }
  const bool near = (t & T_NEAR) != 0;
  C h[Q];
  gather<Q, S, ODD ? LOAD_SLOTS : LOAD_LOCAL>(a, f, x, y, z, n, near, h);
  C rho, urx, ury, urz;
  if constexpr (HRR) {
    C S6[6] = {C(0), C(0), C(0), C(0), C(0), C(0)};
    if (a.hybrid) strain_fd<C>(a, x, y, z, n, near, S6);
    collide_hrr<Q, C>(h, gamma_at<C>(a, n), a, S6, rho, urx, ury, urz);
    record_velocity<C>(a, n, urx, ury, urz);
  } else {
    collide_fluid<Q, C>(h, gamma_at<C>(a, n), a, rho, urx, ury, urz);
  }
  apply_fringe<Q, C>(a, x, K_FLUID, urx, ury, urz, h);
  if (!finite_all<C>(rho, urx, ury, urz)) atomicOr(a.status, ST_NAN);
  scatter<Q, S, ODD ? STORE_SLOTS : STORE_MIRROR>(a, f, x, y, z, n, near, h);
}
// Mixed path of the BGK interior kernel (fused mode, every list cell inline): one instruction stream
// for every non-solid kind. Even steps gather and scatter the cell's own slots whatever its kind; odd
// steps use per-lane slot codes (0 for plain cells; list and NEAR cells read theirs by cell index from
// the per-cell code array), so lanes of different kinds only diverge in the inlet/outlet
// reconstruction, the wall-state load and the slip rule.
template <int Q, class S, bool ODD>
__device__ __forceinline__ void mixed_cell(const Args& a, S* f, int x, int y, int z, long long n, uint8_t t) {
  using C = typename Codec<S>::C;
  const int kind = t & T_KIND;
  if (kind == K_SOLID || (t & T_GHOST)) return;
  const bool list = (t & T_LIST) != 0;
  C h[Q];
  unsigned long long code = 0;
  // the slot codes come by cell index, so their load does not wait for the list position's
  if constexpr (ODD) code = (t & (T_LIST | T_NEAR)) ? a.ccode[n] : 0ull;
  const int k = list ? a.lidx[n] : -1;
  if constexpr (ODD) {
    gather_coded<Q, S>(a, f, x, y, z, n, code, h);
  } else {
    gather<Q, S, LOAD_LOCAL>(a, f, x, y, z, n, false, h);
  }
  if (kind == K_INFLOW || kind == K_OUTFLOW) apply_bc<Q, C>(a, kind, y, z, h);
  const C* ws = (kind == K_WALL && a.wm) ? cptr<C>(a.wst) + (long long)WALL_STATE * k : nullptr;
  C rho, urx, ury, urz;
  collide_unified<Q, C>(h, gamma_at<C>(a, n), a, ws, rho, urx, ury, urz);
  apply_fringe<Q, C>(a, x, kind, urx, ury, urz, h);
  if (t & T_REF) {
    C* w = cptr<C>(a.ref_wr) + 3 * (long long)k;
    w[0] = urx; w[1] = ury; w[2] = urz;
  }
  if (!finite_all<C>(rho, urx, ury, urz)) atomicOr(a.status, ST_NAN);
  if constexpr (ODD) scatter_coded<Q, S>(a, f, x, y, z, n, code, h);
  else scatter<Q, S, STORE_MIRROR>(a, f, x, y, z, n, false, h);
}

// On even steps the warp decides its path with one ballot: 32 plain FLUID cells (no list entry, no
// solid or outside source) take the plain path; any other warp takes the mixed path when every list
// cell is updated here (BGK, fused mode), else the per-cell dispatch of bulk_cell. Blocks are whole
// warps, and every thread reaches the ballot before any returns.
template <int Q, class S, bool ODD>
__global__ void __launch_bounds__(BULK_THREADS, (bulk_min_blocks<Q, S, ODD>())) k_bulk(const Args a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const bool in = x < a.nx && y < a.ny;
  const long long n = x + (long long)y * a.nx + (long long)z * a.nxy;
  const uint8_t t = in ? a.type[n] : uint8_t(0);
  // Odd steps send every warp down the mixed path (with every list cell inline): one code path for
  // the neighbour-slot step instead of two. Measured on the 512x512x256 canopy: D3Q27 23.9 -> 24.8
  // GLUPS, D3Q19 unchanged (35.1); the same on even steps lost (D3Q19 34.3).
  const bool plain_warp = ODD ? false : __all_sync(0xffffffffu, t == 0);
  if (!in) return;
  S* f = static_cast<S*>(a.f);
  if (!plain_warp && a.inline_all) {
    mixed_cell<Q, S, ODD>(a, f, x, y, z, n, t);
    return;
  }
  bulk_cell<Q, S, ODD>(a, f, x, y, z, n, t);
}
// Interior kernel of the HRR collision (same cell set and slot handling as k_bulk), launched in the
// column-split shape of cell_at: with non-periodic x faces the inlet/outlet planes run in CTAs of
// their own, so no row warp waits on one lane's boundary reconstruction and HRR collision
// (512x512x256 canopy, HRR sigma = 1/2 with the vortex inlet: 20.3 -> 21.9 GLUPS; the same launch
// shape measured slower for the BGK and adjoint kernels, whose face lanes cost less than the strided
// column accesses).
template <int Q, class S, bool ODD>
__global__ void __launch_bounds__(BULK_THREADS) k_bulk_hrr(const Args a) {
  const CellAt c = cell_at(a);
  const int x = c.x, y = c.y, z = c.z;
  if (!c.in || c.skip) return;
  const long long n = x + (long long)y * a.nx + (long long)z * a.nxy;
  bulk_cell<Q, S, ODD, true>(a, static_cast<S*>(a.f), x, y, z, n, a.type[n]);
}

// ---- 16-bit storage, two cells per thread -------------------------------------------------------------
// A pair register holds the same population of cells x0 (low half) and x0 + 1 (high half).
template <class S> struct Pair;
template <> struct Pair<__half> {
  using V = __half2;
  static __device__ __forceinline__ V ld(const __half* p) { return *reinterpret_cast<const __half2*>(p); }
  static __device__ __forceinline__ void st(__half* p, V v) { *reinterpret_cast<__half2*>(p) = v; }
  static __device__ __forceinline__ V make(__half lo, __half hi) { return __halves2half2(lo, hi); }
  static __device__ __forceinline__ __half lo(V v) { return __low2half(v); }
  static __device__ __forceinline__ __half hi(V v) { return __high2half(v); }
  static __device__ __forceinline__ float lof(V v) { return __low2float(v); }
  static __device__ __forceinline__ float hif(V v) { return __high2float(v); }
  static __device__ __forceinline__ V with_lo(V v, float x) { return __halves2half2(__float2half_rn(x), __high2half(v)); }
  static __device__ __forceinline__ V with_hi(V v, float x) { return __halves2half2(__low2half(v), __float2half_rn(x)); }
  static __device__ __forceinline__ V pack(float lo, float hi) { return __floats2half2_rn(lo, hi); }
};
// FP32 storage: the pair is a float2 (8-byte accesses), packing and unpacking are moves.
template <> struct Pair<float> {
  using V = float2;
  static __device__ __forceinline__ V ld(const float* p) { return *reinterpret_cast<const float2*>(p); }
  static __device__ __forceinline__ void st(float* p, V v) { *reinterpret_cast<float2*>(p) = v; }
  static __device__ __forceinline__ V make(float lo, float hi) { return make_float2(lo, hi); }
  static __device__ __forceinline__ float lo(V v) { return v.x; }
  static __device__ __forceinline__ float hi(V v) { return v.y; }
  static __device__ __forceinline__ float lof(V v) { return v.x; }
  static __device__ __forceinline__ float hif(V v) { return v.y; }
  static __device__ __forceinline__ V pack(float lo, float hi) { return make_float2(lo, hi); }
};
template <> struct Pair<__nv_bfloat16> {
  using V = __nv_bfloat162;
  static __device__ __forceinline__ V ld(const __nv_bfloat16* p) { return *reinterpret_cast<const __nv_bfloat162*>(p); }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, V v) { *reinterpret_cast<__nv_bfloat162*>(p) = v; }
  static __device__ __forceinline__ V make(__nv_bfloat16 lo, __nv_bfloat16 hi) { return __halves2bfloat162(lo, hi); }
  static __device__ __forceinline__ __nv_bfloat16 lo(V v) { return __low2bfloat16(v); }
  static __device__ __forceinline__ __nv_bfloat16 hi(V v) { return __high2bfloat16(v); }
  static __device__ __forceinline__ float lof(V v) { return __low2float(v); }
  static __device__ __forceinline__ float hif(V v) { return __high2float(v); }
  static __device__ __forceinline__ V with_lo(V v, float x) { return __halves2bfloat162(__float2bfloat16_rn(x), __high2bfloat16(v)); }
  static __device__ __forceinline__ V with_hi(V v, float x) { return __halves2bfloat162(__low2bfloat16(v), __float2bfloat16_rn(x)); }
  static __device__ __forceinline__ V pack(float lo, float hi) { return __floats2bfloat162_rn(lo, hi); }
};

// Interior kernel for 16-bit storage (nx even, 32-bit indices): the thread owns cells x0 = 2j and
// x0 + 1. Directions without an x-component move both cells' values with one 32-bit access, the
// others with two 16-bit accesses; the pair stays packed in 16-bit pair registers and the two cells
// collide together in packed FP32 lanes. Pairs holding a cell that is not plain FLUID take the
// per-cell path.
template <int Q, class S, bool ODD>
__device__ __forceinline__ void pair_load(const Args& a, const S* f, int x0, int y, int z, typename Pair<S>::V* raw) {
  using P = Pair<S>;
  using NB = RowNbr<2>;
  const unsigned us = unsigned(a.stride);
  const unsigned un = unsigned(x0 + y * a.nx) + unsigned(z) * unsigned(a.nxy);
  if constexpr (!ODD) {
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      raw[i] = P::ld(f + (unsigned(i) * us + un));
    });
  } else {
    const NB nb(a, x0, y, z, un);
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int cx = -Lat<Q>::cx(i), cy = -Lat<Q>::cy(i), cz = -Lat<Q>::cz(i);
      const unsigned pb = unsigned(opp<Q>(i)) * us;
      if constexpr (cx == 0) raw[i] = P::ld(f + nb.template at<0, 0, cy, cz>(pb));
      else raw[i] = P::make(f[nb.template at<0, cx, cy, cz>(pb)], f[nb.template at<1, cx, cy, cz>(pb)]);
    });
  }
}

template <int Q, class S, bool ODD, bool HRR = false>
__device__ __forceinline__ void pair_update(const Args& a, S* f, int x0, int y, int z, typename Pair<S>::V* raw) {
  using P = Pair<S>;
  using NB = RowNbr<2>;
  const unsigned us = unsigned(a.stride);
  const unsigned un = unsigned(x0 + y * a.nx) + unsigned(z) * unsigned(a.nxy);
  bool ok;
  const float2 gam = a.gamma ? make_float2(static_cast<const float*>(a.gamma)[un], static_cast<const float*>(a.gamma)[un + 1])
                             : bc2(1.f);
  if constexpr (HRR) {
    // both cells are plain (not NEAR): all six neighbours of each are usable for the strain
    float2 S2[6];
    if (a.hybrid) {
      float s0[6], s1[6];
      strain_fd<float>(a, x0, y, z, un, false, s0);
      strain_fd<float>(a, x0 + 1, y, z, un + 1, false, s1);
      sfor<0, 6>([&](auto I) { S2[I] = make_float2(s0[I], s1[I]); });
    } else {
      sfor<0, 6>([&](auto I) { S2[I] = bc2(0.f); });
    }
    float2 h[Q], ux, uy, uz;
    sfor<0, Q>([&](auto I) { h[I] = make_float2(P::lof(raw[I]), P::hif(raw[I])); });
    ok = collide_hrr_x2<Q>(h, gam, a, S2, ux, uy, uz);
    sfor<0, Q>([&](auto I) { raw[I] = P::pack(h[I].x, h[I].y); });
    float2* w = static_cast<float2*>(a.uvel_wr);  // N even, x0 even: pairs are 8-byte aligned
    const long long N2 = a.N / 2, p2 = un / 2;
    w[p2] = ux;
    w[N2 + p2] = uy;
    w[2 * N2 + p2] = uz;
  } else {
    float2 h[Q];
    sfor<0, Q>([&](auto I) { h[I] = make_float2(P::lof(raw[I]), P::hif(raw[I])); });
    ok = collide_fluid_x2<Q>([&](int i) { return h[i]; }, [&](int i, float2 v) { h[i] = v; }, gam, a);
    sfor<0, Q>([&](auto I) { raw[I] = P::pack(h[I].x, h[I].y); });
  }
  if (!ok) atomicOr(a.status, ST_NAN);
  // An opaque copy of x0: the store addresses are recomputed here rather than held live across the
  // collision (y and z are uniform over the CTA).
  int x0c;
  const int yc = y, zc = z;
  asm volatile("mov.b32 %0, %1;" : "=r"(x0c) : "r"(x0));
  const unsigned un2 = unsigned(x0c + yc * a.nx) + unsigned(zc) * unsigned(a.nxy);
  if constexpr (!ODD) {
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      P::st(f + (unsigned(opp<Q>(i)) * us + un2), raw[i]);
    });
  } else {
    const NB nb(a, x0c, yc, zc, un2);
    sfor<0, Q>([&](auto I) {
      constexpr int k = decltype(I)::value;  // f*_k goes to slot (k, x + c_k)
      constexpr int cx = Lat<Q>::cx(k), cy = Lat<Q>::cy(k), cz = Lat<Q>::cz(k);
      const unsigned pb = unsigned(k) * us;
      if constexpr (cx == 0) {
        P::st(f + nb.template at<0, 0, cy, cz>(pb), raw[k]);
      } else {
        f[nb.template at<0, cx, cy, cz>(pb)] = P::lo(raw[k]);
        f[nb.template at<1, cx, cy, cz>(pb)] = P::hi(raw[k]);
      }
    });
  }
}

#ifndef LBM_BULK2_MINB_EVEN
#define LBM_BULK2_MINB_EVEN 7
#endif
#ifndef LBM_BULK2_MINB_ODD
#define LBM_BULK2_MINB_ODD 7
#endif
// The pair kernel (BGK or HRR collision) over CTAs that each lie in one x-row (grid
// (ceil(nx / 2 / blockDim.x), ny, nz), 1-D blocks): y and z come from the block index, so the
// neighbour displacements of the odd step are computed once per warp instead of per thread.
template <int Q, class S, bool ODD, bool HRR = false>
__global__ void __launch_bounds__(BULK_THREADS, (Q == 19 && !HRR ? (ODD ? LBM_BULK2_MINB_ODD : LBM_BULK2_MINB_EVEN) : 4))
    k_bulk2r(const Args a) {
  row_prefetch<Q, S>(a, 2 * blockDim.x);
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x0 >= a.nx) return;
  const long long n0 = x0 + (long long)y * a.nx + (long long)z * a.nxy;
  S* f = static_cast<S*>(a.f);
  const unsigned short tt = *reinterpret_cast<const unsigned short*>(a.type + n0);
  if (tt) {
    bulk_cell<Q, S, ODD, HRR>(a, f, x0, y, z, n0, uint8_t(tt & 0xff));
    bulk_cell<Q, S, ODD, HRR>(a, f, x0 + 1, y, z, n0 + 1, uint8_t(tt >> 8));
    return;
  }
  typename Pair<S>::V raw[Q];
  pair_load<Q, S, ODD>(a, f, x0, y, z, raw);
  pair_update<Q, S, ODD, HRR>(a, f, x0, y, z, raw);
}

// ---- 16-bit storage, four cells per thread ---------------------------------------------------------------
// Even steps only: the thread owns cells x0 = 4j .. x0 + 3 (nx a multiple of 4) and moves 8 bytes per
// population, the bytes a thread of the FP32 pair kernel keeps in flight; every access is local and
// aligned. The quad collides as two pairs in turn (packed FP32 lanes, the pair kernel's arithmetic).
// Odd steps run the pair kernel: an x-shifted quad needs two 16-bit accesses and an aligned word per
// population, which measured slower than pairs (spills at this register budget).
template <class V> __device__ __forceinline__ V as_pair(unsigned u) {
  V v;
  __builtin_memcpy(&v, &u, sizeof(v));
  return v;
}
template <class V> __device__ __forceinline__ unsigned as_word(V v) {
  unsigned u;
  __builtin_memcpy(&u, &v, sizeof(u));
  return u;
}

// Collision of one pair held in 16-bit pair registers (cells at un, un + 1); false if not finite.
// Each read decodes the 16-bit pair again (an opaque copy keeps the two decodes apart), so the
// decoded populations are not held across the collision.
template <int Q, class S>
__device__ __forceinline__ bool pair_collide(const Args& a, unsigned un, typename Pair<S>::V* raw) {
  using P = Pair<S>;
  using V = typename P::V;
  const float2 gam = a.gamma ? make_float2(static_cast<const float*>(a.gamma)[un], static_cast<const float*>(a.gamma)[un + 1])
                             : bc2(1.f);
  return collide_fluid_x2<Q>(
      [&](int i) {
        unsigned w = as_word(raw[i]);
        asm volatile("" : "+r"(w));
        const V v = as_pair<V>(w);
        return make_float2(P::lof(v), P::hif(v));
      },
      [&](int i, float2 v) { raw[i] = P::pack(v.x, v.y); }, gam, a);
}

// Six CTAs of 128 threads per SM (80 registers): measured against 4 (128 registers), 5 (96) and 7
// (72, more spilling) on the 256^3 FP16 channel.
#ifndef LBM_BULK4_MINB
#define LBM_BULK4_MINB 6
#endif
// Row form (as k_bulk2r): CTAs of 1-D blocks inside one x-row, y and z from the block index.
template <int Q, class S>
__global__ void __launch_bounds__(BULK_THREADS, LBM_BULK4_MINB) k_bulk4r(const Args a) {
  static_assert(sizeof(S) == 2 && Q == 19, "four cells per thread: D3Q19, 16-bit storage");
  row_prefetch<Q, S>(a, 4 * blockDim.x);
  const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x0 >= a.nx) return;
  const long long n0 = x0 + (long long)y * a.nx + (long long)z * a.nxy;
  S* f = static_cast<S*>(a.f);
  const unsigned tt = *reinterpret_cast<const unsigned*>(a.type + n0);
  if (tt) {
#pragma unroll 1
    for (int c = 0; c < 4; ++c) bulk_cell<Q, S, false>(a, f, x0 + c, y, z, n0 + c, uint8_t(tt >> (8 * c)));
    return;
  }
  using V = typename Pair<S>::V;
  V ra[Q], rb[Q];
  const unsigned un = unsigned(n0), us = unsigned(a.stride);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const uint2 v = *reinterpret_cast<const uint2*>(f + (unsigned(i) * us + un));
    ra[i] = as_pair<V>(v.x);
    rb[i] = as_pair<V>(v.y);
  });
  bool ok = pair_collide<Q, S>(a, un, ra);
  ok = pair_collide<Q, S>(a, un + 2u, rb) && ok;
  if (!ok) atomicOr(a.status, ST_NAN);
  // an opaque copy of x0: the store addresses are recomputed, not held live across the collision
  int x0c;
  asm volatile("mov.b32 %0, %1;" : "=r"(x0c) : "r"(x0));
  const unsigned un2 = unsigned(x0c + y * a.nx) + unsigned(z) * unsigned(a.nxy);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    *reinterpret_cast<uint2*>(f + (unsigned(opp<Q>(i)) * us + un2)) = make_uint2(as_word(ra[i]), as_word(rb[i]));
  });
}

// Wall-model state of every WALL entry from the previous step's reference velocities (fused mode).
template <class C>
__global__ void k_wall_state(const Args a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n_wall) return;
  const int k = a.lwall[j];
  const int r = a.wref[k];
  const C z3[3] = {C(0), C(0), C(0)};
  const C* ur = r >= 0 ? cptr<C>(a.ref_rd) + 3 * (long long)r : z3;
  wall_state<C>(a, cptr<C>(a.wnrm) + 3 * (long long)k, cptr<C>(a.wyw)[k], ur, r >= 0,
                cptr<C>(a.wst) + (long long)WALL_STATE * k);
}

// Boundary-list kernel, one thread per list entry: every entry, or in fused mode the entries not
// handled inline (Args::lsub: INFLOW/OUTFLOW entries and list cells in sparse x-groups).
template <int Q, class S, bool ODD, bool HRR = false>
__global__ void __launch_bounds__(LIST_THREADS) k_list(const Args a) {
  using C = typename Codec<S>::C;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int nj = a.lsub ? a.n_sub : a.n_list;
  if (j >= nj) return;
  const int k = a.lsub ? a.lsub[j] : j;
  const long long n = a.lcell[k];
  const int x = a.lxyz[3 * k], y = a.lxyz[3 * k + 1], z = a.lxyz[3 * k + 2];
  const uint8_t t = a.type[n];
  if (t & T_GHOST) return;  // a neighbouring sub-domain's cell
  const int kind = t & T_KIND;
  S* f = static_cast<S*>(a.f);
  C h[Q];
  if constexpr (ODD) {
    const unsigned long long code = a.lcode[k];
    gather_coded<Q, S>(a, f, x, y, z, n, code, h);
    collide_any<Q, C, HRR>(a, kind, t, x, y, z, n, k, h);
    scatter_coded<Q, S>(a, f, x, y, z, n, code, h);
  } else {
    gather<Q, S, LOAD_LOCAL>(a, f, x, y, z, n, false, h);
    collide_any<Q, C, HRR>(a, kind, t, x, y, z, n, k, h);
    scatter<Q, S, STORE_MIRROR>(a, f, x, y, z, n, false, h);
  }
}

// Out-of-place step for the adjoint's recomputation: natural-layout state fin -> natural-layout fout.
// The wall model is excluded by the host.
template <int Q, class S>
__device__ __forceinline__ void oop_cell(const Args& a, const S* fin, S* fout, int x, int y, int z, long long n, uint8_t t) {
  using C = typename Codec<S>::C;
  const int kind = t & T_KIND;
  C h[Q];
  gather<Q, S, LOAD_LOCAL>(a, fin, x, y, z, n, false, h);
  apply_bc<Q, C>(a, kind, y, z, h);
  C rho, urx, ury, urz;
  collide_fluid<Q, C>(h, gamma_at<C>(a, n), a, rho, urx, ury, urz);
  if (!finite_all<C>(rho, urx, ury, urz)) atomicOr(a.status, ST_NAN);
  if (!(t & (T_LIST | T_NEAR))) scatter<Q, S, STORE_SLOTS>(a, fout, x, y, z, n, false, h);
  else scatter_coded<Q, S>(a, fout, x, y, z, n, cell_code(a, n, t), h);
}

template <int Q, class S>
__global__ void __launch_bounds__(BULK_THREADS) k_step_oop(const Args a, const S* __restrict__ fin, S* __restrict__ fout) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  const long long n = x + (long long)y * a.nx + (long long)z * a.nxy;
  const uint8_t t = a.type[n];
  if ((t & T_KIND) == K_SOLID) return;
  oop_cell<Q, S>(a, fin, fout, x, y, z, n, t);
}

// ---- state access ------------------------------------------------------------------------------------
template <class C> __device__ __forceinline__ C load_in(const void* p, int dtype, long long i) {
  return dtype == 0 ? C(static_cast<const double*>(p)[i]) : C(static_cast<const float*>(p)[i]);
}
__device__ __forceinline__ void store_out(void* p, int dtype, long long i, double v) {
  if (dtype == 0) static_cast<double*>(p)[i] = v;
  else static_cast<float*>(p)[i] = float(v);
}

template <int Q, class S>
__global__ void k_init_eq(const Args a, const void* rho, const void* u, int dtype) {
  using C = typename Codec<S>::C;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  S* f = static_cast<S*>(a.f);
  const bool solid = (a.type[n] & T_KIND) == K_SOLID;
  const C r = load_in<C>(rho, dtype, n);
  const C ux = load_in<C>(u, dtype, n), uy = load_in<C>(u, dtype, a.N + n), uz = load_in<C>(u, dtype, 2 * a.N + n);
  const C usq = ux * ux + uy * uy + uz * uz;
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const C v = solid ? C(0) : heq<Q, C, i>(r - C(1), r, ux, uy, uz, usq);
    Codec<S>::st(f + (long long)i * a.stride + n, v);
  });
}

// Reported macroscopic state of cell n: boundary reconstruction, rho, u = j/rho + F/(2 rho).
template <int Q, class S>
__device__ __forceinline__ void cell_macro(const Args& a, long long n, bool swapped, typename Codec<S>::C& rho,
                                           typename Codec<S>::C* u) {
  using C = typename Codec<S>::C;
  int x, y, z;
  cell_coords(a, n, x, y, z);
  const uint8_t t = a.type[n];
  const S* f = static_cast<const S*>(a.f);
  C h[Q];
  if (swapped) gather<Q, S, LOAD_SLOTS>(a, f, x, y, z, n, true, h);
  else gather<Q, S, LOAD_LOCAL>(a, f, x, y, z, n, false, h);
  apply_bc<Q, C>(a, t & T_KIND, y, z, h);
  C drho, jx, jy, jz;
  sums<Q, C>(h, drho, jx, jy, jz);
  rho = C(1) + drho;
  const C ir = C(1) / rho, hf = C(0.5) * ir;
  u[0] = jx * ir + a.fx.get<C>() * hf;
  u[1] = jy * ir + a.fy.get<C>() * hf;
  u[2] = jz * ir + a.fz.get<C>() * hf;
}

template <int Q, class S>
__global__ void k_moments(const Args a, int swapped, void* rho, void* u, int dtype) {
  using C = typename Codec<S>::C;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  if ((a.type[n] & T_KIND) == K_SOLID || (a.type[n] & T_GHOST)) {
    if (rho) store_out(rho, dtype, n, 0.0);
    for (int c = 0; c < 3; ++c) store_out(u, dtype, c * a.N + n, 0.0);
    return;
  }
  C r, uu[3];
  cell_macro<Q, S>(a, n, swapped != 0, r, uu);
  if (rho) store_out(rho, dtype, n, double(r));
  for (int c = 0; c < 3; ++c) store_out(u, dtype, c * a.N + n, double(uu[c]));
}

template <int Q, class S>
__global__ void k_get_pops(const Args a, int swapped, void* out, int dtype) {
  using C = typename Codec<S>::C;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  if ((a.type[n] & T_KIND) == K_SOLID || (a.type[n] & T_GHOST)) {
    sfor<0, Q>([&](auto I) { store_out(out, dtype, (long long)I * a.N + n, 0.0); });
    return;
  }
  int x, y, z;
  cell_coords(a, n, x, y, z);
  const S* f = static_cast<const S*>(a.f);
  C h[Q];
  if (swapped) gather<Q, S, LOAD_SLOTS>(a, f, x, y, z, n, true, h);
  else gather<Q, S, LOAD_LOCAL>(a, f, x, y, z, n, false, h);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    store_out(out, dtype, (long long)i * a.N + n, double(h[i]) + double(Lat<Q>::W(i)) / double(Lat<Q>::Wden));
  });
}

template <int Q, class S>
__global__ void k_set_pops(const Args a, int swapped, const void* in, int dtype) {
  using C = typename Codec<S>::C;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  if ((a.type[n] & T_KIND) == K_SOLID) return;
  int x, y, z;
  cell_coords(a, n, x, y, z);
  S* f = static_cast<S*>(a.f);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const double v = dtype == 0 ? static_cast<const double*>(in)[(long long)i * a.N + n]
                                : double(static_cast<const float*>(in)[(long long)i * a.N + n]);
    const C hv = C(v - double(Lat<Q>::W(i)) / double(Lat<Q>::Wden));
    if (swapped) {
      int p;
      long long m;
      slot_of<Q>(a, x, y, z, n, i, p, m);
      Codec<S>::st(f + (long long)p * a.stride + m, hv);
    } else {
      Codec<S>::st(f + (long long)i * a.stride + n, hv);
    }
  });
}

// Reference buffer from the current state: entry k of a reference cell gets its reported velocity.
template <int Q, class S>
__global__ void k_ref_fill(const Args a, int swapped, void* ref) {
  using C = typename Codec<S>::C;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_list) return;
  const long long n = a.lcell[k];
  C* r = cptr<C>(ref) + 3 * (long long)k;
  if (!(a.type[n] & T_REF)) { r[0] = r[1] = r[2] = C(0); return; }
  C rho, u[3];
  cell_macro<Q, S>(a, n, swapped != 0, rho, u);
  r[0] = u[0]; r[1] = u[1]; r[2] = u[2];
}

// FP64 mass and momentum: grid-stride accumulation per thread, warp shuffles, one partial per block.
template <int Q, class S>
__global__ void __launch_bounds__(256) k_reduce(const Args a, int swapped, double* partial) {
  using C = typename Codec<S>::C;
  double s[4] = {0, 0, 0, 0};
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N; n += (long long)gridDim.x * blockDim.x) {
    if ((a.type[n] & T_KIND) == K_SOLID || (a.type[n] & T_GHOST)) continue;
    C r, u[3];
    cell_macro<Q, S>(a, n, swapped != 0, r, u);
    const double rd = double(r);
    s[0] += rd;
    s[1] += rd * double(u[0]);
    s[2] += rd * double(u[1]);
    s[3] += rd * double(u[2]);
  }
  __shared__ double sm[8][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
    for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
    for (int c = 0; c < 4; ++c) sm[w][c] = s[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 4; ++c) {
      double t = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sm[i][c];
      partial[4 * (long long)blockIdx.x + c] = t;
    }
  }
}

// Wall normals and distances of the list entries from the integer normal sums.
template <class C>
__global__ void k_list_aux(const Args a, const int* nsum, const float* wall_dist, C* wnrm, C* wyw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_list) return;
  const long long n = a.lcell[k];
  const int v0 = nsum[3 * k], v1 = nsum[3 * k + 1], v2 = nsum[3 * k + 2];
  const C vn = sqrt(C(v0) * C(v0) + C(v1) * C(v1) + C(v2) * C(v2));
  if (vn > C(0)) {
    wnrm[3 * k] = -C(v0) / vn;
    wnrm[3 * k + 1] = -C(v1) / vn;
    wnrm[3 * k + 2] = -C(v2) / vn;
  } else {
    wnrm[3 * k] = wnrm[3 * k + 1] = wnrm[3 * k + 2] = C(0);
  }
  wyw[k] = wall_dist ? C(wall_dist[n]) : C(0.5);
}

// Objective plane sums: partial[b] = wa * sum_{x=xa} rho + wb * sum_{x=xb} rho over the non-solid
// cells of block b's share of the two planes (256 cells per block); k_plane_final adds the partials
// to the accumulator in a fixed order.
template <int Q, class S>
__global__ void __launch_bounds__(256) k_plane_rho(const Args a, const S* state, int swapped, int xa, int xb,
                                                   double* partial, double wa, double wb) {
  using C = typename Codec<S>::C;
  Args b = a;
  b.f = const_cast<S*>(state);
  const long long pl = (long long)a.ny * a.nz;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double s = 0.0;
  if (q < 2 * pl) {
    const int which = q >= pl;
    const long long p = which ? q - pl : q;
    const int y = int(p % a.ny), z = int(p / a.ny);
    const int x = which ? xb : xa;
    const long long n = x + (long long)y * a.nx + (long long)z * a.nxy;
    if ((a.type[n] & T_KIND) != K_SOLID) {
      C h[Q];
      if (swapped) gather<Q, S, LOAD_SLOTS>(b, state, x, y, z, n, true, h);
      else gather<Q, S, LOAD_LOCAL>(b, state, x, y, z, n, false, h);
      C drho = C(0);
      sfor<0, Q>([&](auto I) { drho += h[I]; });
      s = (which ? wb : wa) * (1.0 + double(drho));
    }
  }
  __shared__ double sm[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sm[i];
    partial[blockIdx.x] = t;
  }
}

static __global__ void k_plane_final(const double* partial, int nblk, double* acc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0;
  for (int b = 0; b < nblk; ++b) t += partial[b];
  *acc += t;
}

// ---- adjoint reverse step ---------------------------------------------------------------------------------
// lam_out(n) = (d f*(n) / d f(n))^T mu(n) (+ objective weights), mu_k(n) = lam_in at the slot that
// f*_k(n) streams into; gamma and inlet-velocity sensitivities accumulate in FP64 over all steps.
template <int Q, class S>
__device__ __forceinline__ void reverse_cell(const Args& a, const AdjArgs& d, int x, int y, int z, long long n, uint8_t t) {
  using C = typename Codec<S>::C;
  const int kind = t & T_KIND;
  const unsigned long long code = cell_code(a, n, t);
  // mu_opp(i) from the slot of direction i (where f*_opp(i) streamed to) of the natural-layout lam_in
  C mu[Q];
  {
    C tmp[Q];
    gather_coded<Q, C>(a, cptr<C>(d.lam_in), x, y, z, n, code, tmp);
    sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      mu[opp<Q>(i)] = tmp[i];
    });
  }
  C lam[Q], ggam = C(0), gub[3] = {C(0), C(0), C(0)};
  const C gam = gamma_at<C>(a, n);
  const bool bc = kind == K_INFLOW || kind == K_OUTFLOW;
  // boundary reconstruction forward (inlet/outlet lanes only), then the collision reverse for all
  // lanes together, then the reconstruction reverse (inlet/outlet lanes only, which read the
  // populations again rather than keep them live through the collision reverse)
  C hb[Q];
  gather<Q, S, LOAD_LOCAL>(a, static_cast<const S*>(d.fst), x, y, z, n, false, hb);
  if (bc) apply_bc<Q, C>(a, kind, y, z, hb);
  C gh[Q];
  collide_fluid_vjp<Q, C>(hb, gam, a, mu, gh, ggam);
  if (kind == K_INFLOW) {
    C h[Q];
    gather<Q, S, LOAD_LOCAL>(a, static_cast<const S*>(d.fst), x, y, z, n, false, h);
    const C* ub = cptr<C>(a.uin);
    const long long pl = (long long)a.ny * a.nz, p = y + (long long)a.ny * z;
    bc_inlet_vjp<Q, C>(h, ub[p], ub[pl + p], ub[2 * pl + p], gh, lam, gub);
  } else if (kind == K_OUTFLOW) {
    C h[Q];
    gather<Q, S, LOAD_LOCAL>(a, static_cast<const S*>(d.fst), x, y, z, n, false, h);
    bc_outlet_vjp<Q, C>(h, a.rho_out.get<C>(), a.drho_out.get<C>(), gh, lam);
  } else {
    sfor<0, Q>([&](auto I) { lam[I] = gh[I]; });
  }
  if (d.add_dj) {
    const C w = C(x == d.xa ? d.wa : 0.0) + C(x == d.xb ? d.wb : 0.0);
    sfor<0, Q>([&](auto I) { lam[I] += w; });
  }
  C* lo = cptr<C>(d.lam_out);
  sfor<0, Q>([&](auto I) { lo[(long long)I * a.stride + n] = lam[I]; });
  if (d.dgam) d.dgam[n] += double(ggam);
  if (kind == K_INFLOW && d.duin) {
    const long long pl = (long long)a.ny * a.nz, p = y + (long long)a.ny * z;
    atomicAdd(d.duin + p, double(gub[0]));
    atomicAdd(d.duin + pl + p, double(gub[1]));
    atomicAdd(d.duin + 2 * pl + p, double(gub[2]));
  }
}

// Reverse step over every cell (inlet/outlet cells included: their extra boundary-condition reverse
// costs less as a divergent branch than as a separate, latency-bound pass over a sparse plane).
#ifndef LBM_REVERSE_MINB
#define LBM_REVERSE_MINB 8
#endif
template <int Q, class S>
__global__ void __launch_bounds__(BULK_THREADS, LBM_REVERSE_MINB) k_reverse(const Args a, const AdjArgs d) {
  using C = typename Codec<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  const long long n = x + (long long)y * a.nx + (long long)z * a.nxy;
  const uint8_t t = a.type[n];
  const int kind = t & T_KIND;
  if (kind == K_SOLID) {
    C* lo = cptr<C>(d.lam_out);
    sfor<0, Q>([&](auto I) { lo[(long long)I * a.stride + n] = C(0); });
    return;
  }
  reverse_cell<Q, S>(a, d, x, y, z, n, t);
}

// Adjoint seed lambda_T = dJ/dS_T: weight wa on every population of the non-solid cells of plane
// x = xa, wb on plane x = xb, zero elsewhere.
template <class C>
__global__ void k_seed(const Args a, C* lam, int xa, int xb, double wa, double wb, int q) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const int x = int(n % a.nx);
  C w = C(0);
  if ((a.type[n] & T_KIND) != K_SOLID) w = C(x == xa ? wa : 0.0) + C(x == xb ? wb : 0.0);
  for (int i = 0; i < q; ++i) lam[(long long)i * a.stride + n] = w;
}

template <class A, class B>
__global__ void k_convert(const A* in, B* out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = B(in[i]);
}

}  // namespace lbm
