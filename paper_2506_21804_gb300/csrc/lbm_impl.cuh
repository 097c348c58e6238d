// Host launchers of one (lattice, storage) instantiation and its Ops table.
#pragma once

#include <cstdio>

#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"

namespace lbm {

// ---- host launchers ------------------------------------------------------------------------------------
inline dim3 bulk_block(const Args& a) {
  int bx = a.nx >= 128 ? 128 : ((a.nx + 31) / 32) * 32;
  int by = BULK_THREADS / bx;
  if (by < 1) by = 1;
  return dim3(bx, by, 1);
}
inline dim3 bulk_grid(const Args& a) {
  dim3 b = bulk_block(a);
  return dim3((a.nx + b.x - 1) / b.x, (a.ny + b.y - 1) / b.y, a.nz);
}
inline unsigned blocks_for(long long n, int t) { return unsigned((n + t - 1) / t); }
// Grid of the HRR one-cell kernel (cell_at): the column CTAs of the x-face planes, then the row CTAs.
inline unsigned cell_grid(const Args& a) { return a.lc_cols + a.lc_gx * unsigned(a.ny) * unsigned(a.nz); }
// Threads of a 1-D CTA lying in one x-row that holds `groups` cell groups (pairs or quads) per row:
// whole warps, at most BULK_THREADS.
inline unsigned row_threads(int groups) {
  const int t = ((groups + 31) / 32) * 32;
  return unsigned(t < BULK_THREADS ? t : BULK_THREADS);
}


template <int Q, class S>
struct Impl {
  using C = typename Codec<S>::C;
  // Shared-memory layout of the staged kernel, or stages = 0 when the shape does not allow it.
  static TmaLayout tma_layout(const Args& a) {
    TmaLayout L{};
    // FP64 (reference form) and slab sub-domains (ghost planes) stay with the plain kernel
    if (a.kernel != 2 || a.nx % TMA_W != 0 || sizeof(S) == 8 || a.ghost) return L;
    L.pop_bytes = unsigned(TMA_W * sizeof(S));
    L.type_off = unsigned(Q) * L.pop_bytes;
    unsigned end = L.type_off + unsigned(TMA_W);
    if (a.gamma) {
      L.gamma_off = (end + 15u) & ~15u;
      end = L.gamma_off + unsigned(TMA_W * sizeof(C));
    }
    L.stage_bytes = (end + 127u) & ~127u;
    L.tx_bytes = unsigned(Q) * L.pop_bytes + unsigned(TMA_W) + (a.gamma ? unsigned(TMA_W * sizeof(C)) : 0u);
    // two stages: the copies of one tile land while the other is computed; shared memory is better
    // spent on more resident CTAs (latency hiding for the collision) than on deeper rings
    L.stages = 2;
    return L;
  }
  template <bool ODD>
  static bool launch_tma(const Args& a, const TmaLayout& L, cudaStream_t s) {
    auto kern = k_bulk_tma<Q, S, ODD>;
    const size_t dyn = (size_t)L.stages * L.stage_bytes;
    static size_t configured = 0;
    static int per_sm = 0;
    static int nsm = 0;
    if (configured != dyn) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dyn)) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TMA_W + 32, dyn) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return false;
      }
      configured = dyn;
    }
    const long long tiles = (long long)a.ny * a.nz * (a.nx / TMA_W);
    long long grid = (long long)per_sm * nsm;
    if (grid > tiles) grid = tiles;
    kern<<<unsigned(grid), TMA_W + 32, dyn, s>>>(a, L, a.debug_stall);
    return true;
  }
  static void step_bulk(const Args& a, int odd, cudaStream_t s) {
    if (a.model != 0) {
      if constexpr (sizeof(S) <= 4) {
        if (a.pairs && a.N % 2 == 0) {
          const unsigned t2 = row_threads(a.nx / 2);
          const dim3 g2((a.nx / 2 + t2 - 1) / t2, a.ny, a.nz);
          if (odd) k_bulk2r<Q, S, true, true><<<g2, t2, 0, s>>>(a);
          else k_bulk2r<Q, S, false, true><<<g2, t2, 0, s>>>(a);
          return;
        }
      }
      if (odd) k_bulk_hrr<Q, S, true><<<cell_grid(a), a.lc_t, 0, s>>>(a);
      else k_bulk_hrr<Q, S, false><<<cell_grid(a), a.lc_t, 0, s>>>(a);
      return;
    }
    const TmaLayout L = tma_layout(a);
    if (L.stages >= 2) {
      if (odd ? launch_tma<true>(a, L, s) : launch_tma<false>(a, L, s)) return;
    }
    if constexpr (sizeof(S) <= 4) {
      if (a.pairs) {
        // Row form: 1-D CTAs inside one x-row. 16-bit D3Q19 storage runs four cells per thread on
        // even steps (nx a multiple of 4); odd steps, and every step of the other forms, run cell
        // pairs (measured on the 256^3 FP16 channel per 8.4M cells: even 111 us vs 121 us, odd 156 us
        // vs 149 us, quads vs pairs).
        if constexpr (sizeof(S) == 2 && Q == 19) {
          if (a.nx % 4 == 0 && !odd) {
            const unsigned t4 = row_threads(a.nx / 4);
            k_bulk4r<Q, S><<<dim3((a.nx / 4 + t4 - 1) / t4, a.ny, a.nz), t4, 0, s>>>(a);
            return;
          }
        }
        const unsigned t2 = row_threads(a.nx / 2);
        const dim3 g2((a.nx / 2 + t2 - 1) / t2, a.ny, a.nz);
        if (odd) k_bulk2r<Q, S, true><<<g2, t2, 0, s>>>(a);
        else k_bulk2r<Q, S, false><<<g2, t2, 0, s>>>(a);
        return;
      }
    }
    if (odd) k_bulk<Q, S, true><<<bulk_grid(a), bulk_block(a), 0, s>>>(a);
    else k_bulk<Q, S, false><<<bulk_grid(a), bulk_block(a), 0, s>>>(a);
  }
  static void step_list(const Args& a, int odd, cudaStream_t s) {
    const int nj = a.lsub ? a.n_sub : a.n_list;
    if (nj <= 0 || a.inline_all) return;
    if (a.model != 0) {
      if (odd) k_list<Q, S, true, true><<<blocks_for(nj, LIST_THREADS), LIST_THREADS, 0, s>>>(a);
      else k_list<Q, S, false, true><<<blocks_for(nj, LIST_THREADS), LIST_THREADS, 0, s>>>(a);
      return;
    }
    if (odd) k_list<Q, S, true><<<blocks_for(nj, LIST_THREADS), LIST_THREADS, 0, s>>>(a);
    else k_list<Q, S, false><<<blocks_for(nj, LIST_THREADS), LIST_THREADS, 0, s>>>(a);
  }
  static void wall_pass(const Args& a, cudaStream_t s) {
    if (a.n_wall <= 0) return;
    k_wall_state<C><<<blocks_for(a.n_wall, 128), 128, 0, s>>>(a);
  }
  static void init_eq(const Args& a, const void* rho, const void* u, int dtype, cudaStream_t s) {
    k_init_eq<Q, S><<<blocks_for(a.N, 256), 256, 0, s>>>(a, rho, u, dtype);
  }
  static void moments(const Args& a, int swapped, void* rho, void* u, int dtype, cudaStream_t s) {
    k_moments<Q, S><<<blocks_for(a.N, 128), 128, 0, s>>>(a, swapped, rho, u, dtype);
  }
  static void get_pops(const Args& a, int swapped, void* out, int dtype, cudaStream_t s) {
    k_get_pops<Q, S><<<blocks_for(a.N, 128), 128, 0, s>>>(a, swapped, out, dtype);
  }
  static void set_pops(const Args& a, int swapped, const void* in, int dtype, cudaStream_t s) {
    k_set_pops<Q, S><<<blocks_for(a.N, 128), 128, 0, s>>>(a, swapped, in, dtype);
  }
  static void ref_fill(const Args& a, int swapped, void* ref, cudaStream_t s) {
    if (a.n_list <= 0) return;
    k_ref_fill<Q, S><<<blocks_for(a.n_list, 128), 128, 0, s>>>(a, swapped, ref);
  }
  static void reduce(const Args& a, int swapped, double* partial, int nblk, cudaStream_t s) {
    k_reduce<Q, S><<<nblk, 256, 0, s>>>(a, swapped, partial);
  }
  static void list_aux(const Args& a, const int* nsum, const float* wd, void* wnrm, void* wyw, cudaStream_t s) {
    if (a.n_list <= 0) return;
    k_list_aux<C><<<blocks_for(a.n_list, 128), 128, 0, s>>>(a, nsum, wd, static_cast<C*>(wnrm), static_cast<C*>(wyw));
  }
  static void step_oop(const Args& a, const void* fin, void* fout, cudaStream_t s) {
    k_step_oop<Q, S><<<bulk_grid(a), bulk_block(a), 0, s>>>(a, static_cast<const S*>(fin), static_cast<S*>(fout));
  }
  static void reverse(const Args& a, const AdjArgs& d, cudaStream_t s) {
    k_reverse<Q, S><<<bulk_grid(a), bulk_block(a), 0, s>>>(a, d);
  }
  // acc += the plane sums; scratch holds one partial per 256 plane cells (2 ny nz / 256 doubles)
  static void plane_rho(const Args& a, const void* state, int swapped, int xa, int xb, double* acc, double* scratch,
                        double wa, double wb, cudaStream_t s) {
    const long long cells = 2LL * a.ny * a.nz;
    const int nblk = int((cells + 255) / 256);
    k_plane_rho<Q, S><<<nblk, 256, 0, s>>>(a, static_cast<const S*>(state), swapped, xa, xb, scratch, wa, wb);
    k_plane_final<<<1, 32, 0, s>>>(scratch, nblk, acc);
  }
  static void seed(const Args& a, void* lam, int xa, int xb, double wa, double wb, cudaStream_t s) {
    k_seed<C><<<blocks_for(a.N, 256), 256, 0, s>>>(a, static_cast<C*>(lam), xa, xb, wa, wb, Q);
  }
  static void convert(const void* in, int idt, void* out, int odt, long long n, cudaStream_t s) {
    const unsigned g = blocks_for(n, 256);
    if (idt == 0 && odt == 0) k_convert<double, double><<<g, 256, 0, s>>>((const double*)in, (double*)out, n);
    else if (idt == 0) k_convert<double, float><<<g, 256, 0, s>>>((const double*)in, (float*)out, n);
    else if (odt == 0) k_convert<float, double><<<g, 256, 0, s>>>((const float*)in, (double*)out, n);
    else k_convert<float, float><<<g, 256, 0, s>>>((const float*)in, (float*)out, n);
  }
  static const Ops* table() {
    static const Ops ops = {Q,        int(sizeof(S)), int(sizeof(C)), step_bulk, step_list, wall_pass, init_eq,   moments,
                            get_pops, set_pops,       ref_fill,       reduce,    list_aux,  step_oop,  reverse,
                            plane_rho, seed,           convert};
    return &ops;
  }
};

}  // namespace lbm
