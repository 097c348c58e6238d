// Interior-cell step kernel with the populations of 128-cell x-segments staged in shared memory by
// bulk asynchronous copies (cp.async.bulk, completion through mbarriers); nx a multiple of 128.
//
// A persistent CTA walks the tiles t = blockIdx.x + j*gridDim.x (tile = row r = t / nseg, segment
// t % nseg of TMA_W cells); tile j goes to stage j % S of a ring of S shared-memory stages. The CTA
// has one consumer thread per cell of the segment plus one producer warp: the producer issues the copies of tile j into stage s once every consumer warp has
// released tile j - S from it (an "empty" barrier with one arrival per consumer warp), the
// consumers wait on the stage's "full" barrier (transaction count of the copies), copy their
// cell's populations to registers, release the stage and compute. No CTA-wide barrier is used in
// the loop, so warps run ahead of each other by up to S tiles. Per tile and direction i the
// copied segment is the same x-range of the source row: on an even step the cell's own row of
// population i, on an odd step row (y - c_iy, z - c_iz) of population opp(i), from which cell x
// takes element x - c_ix; the first and last cell of the segment read the one element that lies
// outside it directly from global memory. Copied elements that this tile's cells do not own are
// never used, and no cell writes a slot it does not own (the AA pattern gives each slot one
// owner), so the copies never race with another CTA's stores. Results
// go straight to global memory with coalesced per-cell stores. Cells next to solids or outer faces
// (NEAR) read through the general slot map instead of the staged row.
//
// Every wait is bounded in time; a wait that runs out sets ST_TIMEOUT in the status word, waits
// (again bounded) for the copies this CTA has issued, and ends the kernel.
#pragma once

#include "lbm_kernels.cuh"  // gather, scatter, collide_fluid

namespace lbm {

constexpr unsigned ST_TIMEOUT = 4u;
constexpr unsigned long long WAIT_LIMIT_NS = 1000000000ull;  // 1 s

__device__ __forceinline__ unsigned smem_addr(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, at most WAIT_LIMIT_NS; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > WAIT_LIMIT_NS) return false;
  }
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned), completing
// on the barrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

struct TmaLayout {
  int stages;
  unsigned pop_bytes;    // nx * sizeof(S)
  unsigned stage_bytes;  // Q * pop_bytes + type row + gamma row, rounded up to 128
  unsigned gamma_off;    // offset of the gamma row in a stage (0: none)
  unsigned type_off;
  unsigned tx_bytes;     // bytes delivered per tile
};

constexpr int TMA_MAX_STAGES = 8;
constexpr int TMA_W = 128;  // cells per tile (consumer threads per CTA)

template <int Q, class S, bool ODD>
__global__ void __launch_bounds__(TMA_W + 32, 6) k_bulk_tma(const Args a, const TmaLayout L, int debug_stall) {
  using C = typename Codec<S>::C;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned long long full[TMA_MAX_STAGES], empty[TMA_MAX_STAGES];
  __shared__ unsigned long long never;
  const int tid = threadIdx.x;
  const int nseg = a.nx / TMA_W;
  const long long ntiles = (long long)a.ny * a.nz * nseg;
  const long long G = gridDim.x;
  S* f = static_cast<S*>(a.f);
  if (tid == 0) {
    for (int s = 0; s < L.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TMA_W / 32);
    }
    mbar_init(&never, 1);
    fence_mbar_init();
  }
  __syncthreads();

  if (tid >= TMA_W) {
    // ---- producer warp (one thread) ----
    if (tid != TMA_W) return;
    long long j = 0;
    bool ok = true;
    for (;; ++j) {
      const long long tile = blockIdx.x + j * G;
      if (tile >= ntiles) break;
      const int s = int(j % L.stages);
      if (j >= L.stages && !mbar_wait_bounded(&empty[s], unsigned(((j / L.stages) - 1) & 1))) {
        ok = false;
        break;
      }
      const long long r = tile / nseg;
      const int x0 = int(tile - r * nseg) * TMA_W;
      unsigned char* st = smem + (size_t)s * L.stage_bytes;
      const int y = int(r % a.ny), z = int(r / a.ny);
      fence_proxy_async();
      mbar_expect_tx(&full[s], L.tx_bytes);
      sfor<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        long long row;
        int p;
        if constexpr (ODD) {
          int sy = y - Lat<Q>::cy(i), sz = z - Lat<Q>::cz(i);
          sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
          sz = sz < 0 ? sz + a.nz : (sz >= a.nz ? sz - a.nz : sz);
          row = sy + (long long)a.ny * sz;
          p = opp<Q>(i);
        } else {
          row = r;
          p = i;
        }
        bulk_g2s(st + (size_t)i * L.pop_bytes, f + (long long)p * a.stride + row * a.nx + x0, L.pop_bytes, &full[s]);
      });
      bulk_g2s(st + L.type_off, a.type + r * a.nx + x0, (unsigned)TMA_W, &full[s]);
      if (L.gamma_off)
        bulk_g2s(st + L.gamma_off, static_cast<const C*>(a.gamma) + r * a.nx + x0, unsigned(TMA_W * sizeof(C)), &full[s]);
    }
    if (!ok) atomicOr(a.status, ST_TIMEOUT);
    // the copies of the last (up to S) issued tiles must land before the CTA may exit
    for (long long k = (j > L.stages ? j - L.stages : 0); k < j; ++k)
      mbar_wait_bounded(&full[k % L.stages], unsigned((k / L.stages) & 1));
    return;
  }

  // ---- consumers: one thread per cell of the segment ----
  const int xi = tid;
  const int lane = tid & 31;
  for (long long j = 0;; ++j) {
    const long long tile = blockIdx.x + j * G;
    if (tile >= ntiles) break;
    const int s = int(j % L.stages);
    bool ok = mbar_wait_bounded(&full[s], unsigned((j / L.stages) & 1));
    if (ok && debug_stall && j == 0) ok = mbar_wait_bounded(&never, 0);
    if (!ok) {
      atomicOr(a.status, ST_TIMEOUT);
      return;
    }
    const long long r = tile / nseg;
    const int x = int(tile - r * nseg) * TMA_W + xi;
    const int y = int(r % a.ny), z = int(r / a.ny);
    const long long n = r * a.nx + x;
    const unsigned char* st = smem + (size_t)s * L.stage_bytes;
    const uint8_t t = st[L.type_off + xi];
    const bool active = !(t & (T_LIST | T_KIND));
    const bool near = (t & T_NEAR) != 0;
    C h[Q];
    C gam = C(1);
    if (active && !near) {
      const S* sp = reinterpret_cast<const S*>(st);
      if constexpr (ODD) {
        const bool lo = xi == 0, hi = xi == TMA_W - 1;
        const int xm = x == 0 ? a.nx - 1 : x - 1, xp = x == a.nx - 1 ? 0 : x + 1;
        sfor<0, Q>([&](auto I) {
          constexpr int i = decltype(I)::value;
          constexpr int cx = Lat<Q>::cx(i);
          if constexpr (cx == 0) {
            h[i] = Codec<S>::ld(sp + (size_t)i * TMA_W + xi);
          } else {
            // source x - c_ix: in the segment unless this is its first (c_ix > 0) or last (c_ix < 0) cell
            const bool edge = cx > 0 ? lo : hi;
            if (!edge) {
              h[i] = Codec<S>::ld(sp + (size_t)i * TMA_W + xi - cx);
            } else {
              int sy = y - Lat<Q>::cy(i), sz = z - Lat<Q>::cz(i);
              sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
              sz = sz < 0 ? sz + a.nz : (sz >= a.nz ? sz - a.nz : sz);
              const long long src = (cx > 0 ? xm : xp) + (long long)a.nx * sy + a.nxy * sz;
              h[i] = Codec<S>::ld(f + (long long)opp<Q>(i) * a.stride + src);
            }
          }
        });
      } else {
        sfor<0, Q>([&](auto I) {
          constexpr int i = decltype(I)::value;
          h[i] = Codec<S>::ld(sp + (size_t)i * TMA_W + xi);
        });
      }
      if (L.gamma_off) gam = reinterpret_cast<const C*>(st + L.gamma_off)[xi];
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (!active) continue;
    if (near) {
      gather<Q, S, ODD ? LOAD_SLOTS : LOAD_LOCAL>(a, f, x, y, z, n, true, h);
      gam = gamma_at<C>(a, n);
    }
    C rho, urx, ury, urz;
    collide_fluid<Q, C>(h, gam, a, rho, urx, ury, urz);
    apply_fringe<Q, C>(a, x, K_FLUID, urx, ury, urz, h);
    if (!finite_all<C>(rho, urx, ury, urz)) atomicOr(a.status, ST_NAN);
    scatter<Q, S, ODD ? STORE_SLOTS : STORE_MIRROR>(a, f, x, y, z, n, near, h);
  }
}

}  // namespace lbm
