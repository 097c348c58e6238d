// One-time integer work on the geometry: cell classification, wall-model reference cells, the
// ascending boundary-cell list (warp ballots and per-block offsets), the list's integer wall-normal
// sums and reference positions, and the debug source map. All results are exact integers.
#include "lbm_device.cuh"
#include "lbm_ops.h"

namespace lbm {
namespace {

constexpr int CELLS_PER_BLOCK = 256;

struct Pos {
  int x, y, z;
  int crossed;  // non-periodic faces beyond which the position lies (bit f for face f)
};

__device__ __forceinline__ Pos wrap(const GeoArgs& g, int x, int y, int z) {
  Pos p{x, y, z, 0};
  if (p.x < 0) { if (g.face[0] == F_PERIODIC) p.x += g.nx; else p.crossed |= 1; }
  else if (p.x >= g.nx) { if (g.face[1] == F_PERIODIC) p.x -= g.nx; else p.crossed |= 2; }
  if (p.y < 0) { if (g.face[2] == F_PERIODIC) p.y += g.ny; else p.crossed |= 4; }
  else if (p.y >= g.ny) { if (g.face[3] == F_PERIODIC) p.y -= g.ny; else p.crossed |= 8; }
  if (p.z < 0) { if (g.face[4] == F_PERIODIC) p.z += g.nz; else p.crossed |= 16; }
  else if (p.z >= g.nz) { if (g.face[5] == F_PERIODIC) p.z -= g.nz; else p.crossed |= 32; }
  return p;
}

__device__ __forceinline__ long long lin(const GeoArgs& g, const Pos& p) {
  return p.x + (long long)g.nx * p.y + g.nxy * p.z;
}

__device__ __forceinline__ bool beyond_wall_face(const GeoArgs& g, int crossed) {
  bool w = false;
#pragma unroll
  for (int f = 0; f < 6; ++f)
    if ((crossed >> f & 1) && g.face[f] == F_WALL) w = true;
  return w;
}

// Coordinates of cell n; 32-bit divisions whenever the grid has fewer than 2^31 cells (a 64-bit
// integer division is a long instruction sequence on the GPU).
__device__ __forceinline__ void coords(const GeoArgs& g, long long n, int& x, int& y, int& z) {
  if (g.N < (1LL << 31)) {
    const unsigned un = unsigned(n), r = un / unsigned(g.nx);
    x = int(un - r * unsigned(g.nx));
    z = int(r / unsigned(g.ny));
    y = int(r - unsigned(z) * unsigned(g.ny));
    return;
  }
  const long long r = n / g.nx;
  x = int(n - r * g.nx);
  z = int(r / g.ny);
  y = int(r - (long long)z * g.ny);
}

// Integer wall-normal sum v = sum over solid-like neighbours x + c_i of W_i c_i, from the type bytes.
template <int Q>
__device__ __forceinline__ void normal_sum(const GeoArgs& g, const uint8_t* type, int x, int y, int z, int v[3]) {
  v[0] = v[1] = v[2] = 0;
  sfor<1, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const Pos p = wrap(g, x + Lat<Q>::cx(i), y + Lat<Q>::cy(i), z + Lat<Q>::cz(i));
    const bool solid = p.crossed ? beyond_wall_face(g, p.crossed) : ((type[lin(g, p)] & T_KIND) == K_SOLID);
    if (solid) {
      v[0] += Lat<Q>::W(i) * Lat<Q>::cx(i);
      v[1] += Lat<Q>::W(i) * Lat<Q>::cy(i);
      v[2] += Lat<Q>::W(i) * Lat<Q>::cz(i);
    }
  });
}

// Reference cell of a WALL cell: one step along the dominant axis of n = -v (ties: lowest axis),
// provided that cell is a FLUID cell away from every boundary (kind FLUID, T_NEAR clear: no solid or
// outside streaming source); -1 otherwise, and when v = 0. Reading of Sec. 2.2.1: the wall law's
// reference point has to lie in the flow; in gaps one or two cells wide it would sit on the opposite
// wall or on a domain face (such WALL cells get u^B = 0).
__device__ __forceinline__ long long ref_cell(const GeoArgs& g, const uint8_t* type, int x, int y, int z, const int v[3]) {
  if (v[0] == 0 && v[1] == 0 && v[2] == 0) return -1;
  int a = 0;
  if (abs(v[1]) > abs(v[a])) a = 1;
  if (abs(v[2]) > abs(v[a])) a = 2;
  int d[3] = {0, 0, 0};
  d[a] = v[a] > 0 ? -1 : 1;
  const Pos p = wrap(g, x + d[0], y + d[1], z + d[2]);
  if (p.crossed) return -1;
  const long long r = lin(g, p);
  if ((type[r] & (T_KIND | T_NEAR)) != K_FLUID) return -1;
  return r;
}

// Smallest index of a mask byte that is not a valid code (0, 1, 3, 4); *first_bad stays ~0 if none.
__global__ void k_check_mask(const uint8_t* __restrict__ m, long long N, unsigned long long* first_bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += stride) {
    const uint8_t v = m[n];
    if (!(v == 0 || v == 1 || v == 3 || v == 4)) atomicMin(first_bad, (unsigned long long)n);
  }
}

template <int Q>
__global__ void k_classify(const GeoArgs g, const uint8_t* mask, uint8_t* type, unsigned* status) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  int x, y, z;
  coords(g, n, x, y, z);
  uint8_t m = mask[n];
  if (!(m == 0 || m == 1 || m == 3 || m == 4)) {
    atomicOr(status, ST_BADMASK);
    m = 0;
  }
  if (m == 1) { type[n] = K_SOLID | ((z < g.gh_lo || z >= g.nz - g.gh_hi) ? T_GHOST : 0); return; }
  bool wall = false, near = false;
  if (x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1 && z > 0 && z < g.nz - 1) {
    // away from the faces no source position wraps or leaves the domain: plain index offsets
    sfor<1, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if (mask[n + Lat<Q>::cx(i) + (long long)g.nx * Lat<Q>::cy(i) + g.nxy * Lat<Q>::cz(i)] == 1) wall = true;
    });
    near = wall;
  } else sfor<1, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    // neighbour x + c_i (solid neighbour => WALL)
    const Pos p = wrap(g, x + Lat<Q>::cx(i), y + Lat<Q>::cy(i), z + Lat<Q>::cz(i));
    if (p.crossed) {
      near = true;
      if (beyond_wall_face(g, p.crossed)) wall = true;
    } else if (mask[lin(g, p)] == 1) {
      wall = true;
      near = true;
    }
  });
  uint8_t kind = m == 3 ? K_INFLOW : m == 4 ? K_OUTFLOW : (wall ? K_WALL : K_FLUID);
  const bool ghost = z < g.gh_lo || z >= g.nz - g.gh_hi;
  type[n] = kind | (near ? T_NEAR : 0) | (ghost ? T_GHOST : 0);
}

template <int Q>
__global__ void k_mark_ref(const GeoArgs g, uint8_t* type) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  if ((type[n] & T_KIND) != K_WALL) return;
  int x, y, z;
  coords(g, n, x, y, z);
  int v[3];
  normal_sum<Q>(g, type, x, y, z, v);
  const long long r = ref_cell(g, type, x, y, z, v);
  if (r < 0) return;
  unsigned* word = reinterpret_cast<unsigned*>(type + (r & ~3LL));
  atomicOr(word, unsigned(T_REF) << (8 * (r & 3)));
}

__device__ __forceinline__ bool on_list(uint8_t t) {
  const int k = t & T_KIND;
  return k == K_WALL || k == K_INFLOW || k == K_OUTFLOW || (t & T_REF);
}

__global__ void k_list_count(const GeoArgs g, uint8_t* type, int* counts) {
  const long long n = blockIdx.x * (long long)CELLS_PER_BLOCK + threadIdx.x;
  bool f = false;
  if (n < g.N) {
    const uint8_t t = type[n];
    f = on_list(t);
    if (f) type[n] = t | T_LIST;
  }
  const int c = __syncthreads_count(f);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void k_list_write(const GeoArgs g, const uint8_t* type, const int* offsets, long long* lcell) {
  __shared__ int wcount[CELLS_PER_BLOCK / 32];
  const long long n = blockIdx.x * (long long)CELLS_PER_BLOCK + threadIdx.x;
  const bool f = n < g.N && (type[n] & T_LIST);
  const unsigned b = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wcount[w] = __popc(b);
  __syncthreads();
  int base = offsets[blockIdx.x];
  for (int i = 0; i < w; ++i) base += wcount[i];
  if (f) lcell[base + __popc(b & ((1u << lane) - 1u))] = n;
}

// 2-bit odd-step slot code of every direction of the cell at (x, y, z): 0 the plain (periodic-wrapped)
// neighbour slot, 1 the cell's own bounce-back slot (solid source, or a source across a face that is
// not all slip), 2 the slip rule.
template <int Q>
__device__ __forceinline__ unsigned long long slot_code(const GeoArgs& g, const uint8_t* type, int x, int y, int z) {
  unsigned long long code = 0;
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const Pos p = wrap(g, x - Lat<Q>::cx(i), y - Lat<Q>::cy(i), z - Lat<Q>::cz(i));
    unsigned long long c;
    if (p.crossed) {
      bool allslip = true;
      for (int f = 0; f < 6; ++f)
        if ((p.crossed >> f & 1) && g.face[f] != F_SLIP) allslip = false;
      c = allslip ? 2ull : 1ull;
    } else {
      c = ((type[lin(g, p)] & T_KIND) == K_SOLID) ? 1ull : 0ull;
    }
    code |= c << (2 * i);
  });
  return code;
}

// Per list entry: coordinates, integer wall-normal sum and reference position (WALL entries), and
// the slot code of every direction.
template <int Q>
__global__ void k_list_meta(const GeoArgs g, const uint8_t* type, const long long* lcell, int n_list, int* nsum, int* wref,
                            int* lxyz, unsigned long long* lcode) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_list) return;
  const long long n = lcell[k];
  int x, y, z;
  coords(g, n, x, y, z);
  lxyz[3 * k] = x;
  lxyz[3 * k + 1] = y;
  lxyz[3 * k + 2] = z;
  lcode[k] = slot_code<Q>(g, type, x, y, z);
  nsum[3 * k] = nsum[3 * k + 1] = nsum[3 * k + 2] = 0;
  wref[k] = -1;
  if ((type[n] & T_KIND) != K_WALL) return;
  int v[3];
  normal_sum<Q>(g, type, x, y, z, v);
  nsum[3 * k] = v[0];
  nsum[3 * k + 1] = v[1];
  nsum[3 * k + 2] = v[2];
  const long long r = ref_cell(g, type, x, y, z, v);
  if (r < 0) return;
  int lo = 0, hi = n_list - 1;  // the reference cell is on the (ascending) list
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (lcell[mid] < r) lo = mid + 1;
    else hi = mid;
  }
  wref[k] = (lcell[lo] == r) ? lo : -1;
}

template <int Q>
__global__ void k_source_map(const Args a, int64_t* sdir, int64_t* scell) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const bool solid = (a.type[n] & T_KIND) == K_SOLID;
  const long long r = n / a.nx;
  const int x = int(n - r * a.nx), z = int(r / a.ny), y = int(r - (long long)z * a.ny);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if (solid) {
      sdir[(long long)i * a.N + n] = -1;
      scell[(long long)i * a.N + n] = -1;
      return;
    }
    int p;
    long long m;
    slot_of<Q>(a, x, y, z, n, i, p, m);
    // after an even step slot (p, m) holds f*_opp(p)(m)
    sdir[(long long)i * a.N + n] = opp<Q>(p);
    scell[(long long)i * a.N + n] = m;
  });
}

// Slots that the non-solid cells of plane z_from use in an odd step and that lie in plane z_to:
// slot_of of every (cell, direction) of z_from, kept (p, m) when m is in z_to, else (-1, -1).
// Outputs q * nx * ny values each, direction-major.
template <int Q>
__global__ void k_plane_slots(const Args a, int z_from, int z_to, int* sp, long long* sm) {
  const long long pos = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (pos >= a.nxy) return;
  const long long n = pos + a.nxy * z_from;
  const bool solid = (a.type[n] & T_KIND) == K_SOLID;
  const int x = int(pos % a.nx), y = int(pos / a.nx);
  sfor<0, Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    int p = -1;
    long long m = -1;
    if (!solid) {
      slot_of<Q>(a, x, y, z_from, n, i, p, m);
      if (m / a.nxy != z_to) { p = -1; m = -1; }
    }
    sp[(long long)i * a.nxy + pos] = p;
    sm[(long long)i * a.nxy + pos] = m;
  });
}

// Inline (fused-mode) choice per 32-cell x-group of a row: INFLOW/OUTFLOW cells always; WALL and
// reference cells when the group holds at least inline_min list cells. One thread per group.
__global__ void k_inline_mark(const GeoArgs g, uint8_t* type, int inline_min) {
  const int groups = (g.nx + 31) / 32;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= (long long)groups * g.ny * g.nz) return;
  const long long row = j / groups;
  const int g0 = int(j - row * groups) * 32;
  const int g1 = g0 + 32 < g.nx ? g0 + 32 : g.nx;
  uint8_t* t = type + row * g.nx;
  int cnt = 0;
  for (int x = g0; x < g1; ++x) cnt += (t[x] & T_LIST) != 0;
  for (int x = g0; x < g1; ++x) {
    const uint8_t v = t[x];
    if (!(v & T_LIST)) continue;
    const int kind = v & T_KIND;
    if (kind == K_INFLOW || kind == K_OUTFLOW || cnt >= inline_min) t[x] = uint8_t(v | T_INLINE);
  }
}

// Sub-lists of the boundary list, in list order: 0 entries not updated inline, 1 WALL entries (the
// wall-model state pass), 2 INFLOW/OUTFLOW entries. Two passes like the list itself: per-block counts, then
// writes at exclusive offsets (entries ranked inside a warp by ballot).
__device__ __forceinline__ void sub_flags(const uint8_t* type, const long long* lcell, int k, int n_list, bool f[3]) {
  f[0] = f[1] = f[2] = false;
  if (k >= n_list) return;
  const uint8_t t = type[lcell[k]];
  const int kind = t & T_KIND;
  f[0] = !(t & T_INLINE);
  f[1] = kind == K_WALL;
  f[2] = kind == K_INFLOW || kind == K_OUTFLOW;
}

constexpr int SUB_THREADS = 256;

__global__ void __launch_bounds__(SUB_THREADS) k_sub_count(const uint8_t* type, const long long* lcell, int n_list, int* counts) {
  __shared__ int wc[SUB_THREADS / 32][3];
  const int k = blockIdx.x * SUB_THREADS + threadIdx.x;
  bool f[3];
  sub_flags(type, lcell, k, n_list, f);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = 0; c < 3; ++c) {
    const unsigned b = __ballot_sync(0xffffffffu, f[c]);
    if (lane == 0) wc[w][c] = __popc(b);
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    int sum = 0;
    for (int i = 0; i < SUB_THREADS / 32; ++i) sum += wc[i][threadIdx.x];
    counts[3 * blockIdx.x + threadIdx.x] = sum;
  }
}

__global__ void __launch_bounds__(SUB_THREADS) k_sub_write(const uint8_t* type, const long long* lcell, int n_list,
                                                           const int* offsets, int* lsub, int* lwall, int* lbc) {
  __shared__ int wo[SUB_THREADS / 32][3];
  const int k = blockIdx.x * SUB_THREADS + threadIdx.x;
  bool f[3];
  sub_flags(type, lcell, k, n_list, f);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned b[3];
  for (int c = 0; c < 3; ++c) {
    b[c] = __ballot_sync(0xffffffffu, f[c]);
    if (lane == 0) wo[w][c] = __popc(b[c]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 3; ++c) {
      int run = offsets[3 * blockIdx.x + c];
      for (int i = 0; i < SUB_THREADS / 32; ++i) {
        const int v = wo[i][c];
        wo[i][c] = run;
        run += v;
      }
    }
  }
  __syncthreads();
  int* dst[3] = {lsub, lwall, lbc};
  for (int c = 0; c < 3; ++c)
    if (f[c]) dst[c][wo[w][c] + __popc(b[c] & ((1u << lane) - 1u))] = k;
}

// Groups of 64 cells along x (the cells of one warp of the paired kernels) that mix plain cell
// pairs (both cells plain FLUID, type byte 0) with pairs that take the per-cell path: such a warp
// runs both paths. out[0] += groups, out[1] += mixed groups. nx even.
__global__ void k_pair_mix(const GeoArgs g, const uint8_t* type, unsigned long long* out) {
  const int groups = (g.nx + 63) / 64;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned long long mixed = 0, tot = 0;
  if (j < (long long)groups * g.ny * g.nz) {
    const long long row = j / groups;
    const int g0 = int(j - row * groups) * 64;
    const int g1 = g0 + 64 < g.nx ? g0 + 64 : g.nx;
    const unsigned short* t2 = reinterpret_cast<const unsigned short*>(type + row * g.nx);
    bool plain = false, other = false;
    for (int x = g0; x < g1; x += 2) {
      if (t2[x >> 1] == 0) plain = true;
      else other = true;
    }
    tot = 1;
    mixed = (plain && other) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_down_sync(0xffffffffu, tot, o);
    mixed += __shfl_down_sync(0xffffffffu, mixed, o);
  }
  if ((threadIdx.x & 31) == 0 && tot) {
    atomicAdd(&out[0], tot);
    atomicAdd(&out[1], mixed);
  }
}

// Counts of WALL, reference, INFLOW, OUTFLOW and SOLID cells.
__global__ void k_count_kinds(const uint8_t* type, long long N, unsigned long long* out) {
  __shared__ unsigned long long sc[5];
  if (threadIdx.x < 5) sc[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long c[5] = {0, 0, 0, 0, 0};
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    const uint8_t t = type[n];
    const int k = t & T_KIND;
    c[0] += k == K_WALL;
    c[1] += (t & T_REF) != 0;
    c[2] += k == K_INFLOW;
    c[3] += k == K_OUTFLOW;
    c[4] += k == K_SOLID;
  }
  for (int i = 0; i < 5; ++i) {
    unsigned long long v = c[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sc[i], v);
  }
  __syncthreads();
  if (threadIdx.x < 5) atomicAdd(&out[threadIdx.x], sc[threadIdx.x]);
}

__global__ void k_list_index(const long long* lcell, int n_list, int* lidx) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n_list) lidx[lcell[k]] = k;
}

__global__ void k_reduce_final(const double* partial, int nblk, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[4] = {0, 0, 0, 0};
  for (int b = 0; b < nblk; ++b)
    for (int c = 0; c < 4; ++c) s[c] += partial[4 * b + c];
  for (int c = 0; c < 4; ++c) out[c] = s[c];
}

inline unsigned nblocks(long long n, int t) { return unsigned((n + t - 1) / t); }

}  // namespace

void geo_classify(const GeoArgs& g, const uint8_t* mask, uint8_t* type, unsigned* status, cudaStream_t s) {
  if (g.q == 19) k_classify<19><<<nblocks(g.N, 256), 256, 0, s>>>(g, mask, type, status);
  else k_classify<27><<<nblocks(g.N, 256), 256, 0, s>>>(g, mask, type, status);
}

void geo_mark_ref(const GeoArgs& g, uint8_t* type, cudaStream_t s) {
  if (g.q == 19) k_mark_ref<19><<<nblocks(g.N, 256), 256, 0, s>>>(g, type);
  else k_mark_ref<27><<<nblocks(g.N, 256), 256, 0, s>>>(g, type);
}

int geo_count_blocks(const GeoArgs& g) { return int(nblocks(g.N, CELLS_PER_BLOCK)); }

void geo_list_count(const GeoArgs& g, uint8_t* type, int* counts, cudaStream_t s) {
  k_list_count<<<nblocks(g.N, CELLS_PER_BLOCK), CELLS_PER_BLOCK, 0, s>>>(g, type, counts);
}

void geo_list_write(const GeoArgs& g, const uint8_t* type, const int* offsets, long long* lcell, cudaStream_t s) {
  k_list_write<<<nblocks(g.N, CELLS_PER_BLOCK), CELLS_PER_BLOCK, 0, s>>>(g, type, offsets, lcell);
}

void geo_list_meta(const GeoArgs& g, const uint8_t* type, const long long* lcell, int n_list, int* nsum, int* wref,
                   int* lxyz, unsigned long long* lcode, cudaStream_t s) {
  if (n_list <= 0) return;
  if (g.q == 19) k_list_meta<19><<<nblocks(n_list, 128), 128, 0, s>>>(g, type, lcell, n_list, nsum, wref, lxyz, lcode);
  else k_list_meta<27><<<nblocks(n_list, 128), 128, 0, s>>>(g, type, lcell, n_list, nsum, wref, lxyz, lcode);
}

void geo_source_map(const GeoArgs& g, const uint8_t* type, int64_t* sdir, int64_t* scell, cudaStream_t s) {
  Args a{};
  a.type = type;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
  a.nxy = g.nxy; a.N = g.N;
  for (int f = 0; f < 6; ++f) a.face[f] = g.face[f];
  if (g.q == 19) k_source_map<19><<<nblocks(g.N, 128), 128, 0, s>>>(a, sdir, scell);
  else k_source_map<27><<<nblocks(g.N, 128), 128, 0, s>>>(a, sdir, scell);
}

void geo_plane_slots(const GeoArgs& g, const uint8_t* type, int z_from, int z_to, int* sp, long long* sm,
                     cudaStream_t s) {
  Args a{};
  a.type = type;
  a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
  a.nxy = g.nxy; a.N = g.N;
  for (int f = 0; f < 6; ++f) a.face[f] = g.face[f];
  if (g.q == 19) k_plane_slots<19><<<nblocks(g.nxy, 128), 128, 0, s>>>(a, z_from, z_to, sp, sm);
  else k_plane_slots<27><<<nblocks(g.nxy, 128), 128, 0, s>>>(a, z_from, z_to, sp, sm);
}

void geo_inline_mark(const GeoArgs& g, uint8_t* type, int inline_min, cudaStream_t s) {
  const long long groups = (long long)((g.nx + 31) / 32) * g.ny * g.nz;
  k_inline_mark<<<nblocks(groups, 256), 256, 0, s>>>(g, type, inline_min);
}

void geo_check_mask(const uint8_t* mask, long long N, unsigned long long* first_bad, cudaStream_t s) {
  cudaMemsetAsync(first_bad, 0xFF, sizeof(unsigned long long), s);
  long long blocks = nblocks(N, 256);
  if (blocks > 8 * 1216) blocks = 8 * 1216;
  k_check_mask<<<unsigned(blocks), 256, 0, s>>>(mask, N, first_bad);
}

int geo_sub_blocks(int n_list) { return int(nblocks(n_list, SUB_THREADS)); }

void geo_sub_count(const uint8_t* type, const long long* lcell, int n_list, int* counts, cudaStream_t s) {
  if (n_list <= 0) return;
  k_sub_count<<<nblocks(n_list, SUB_THREADS), SUB_THREADS, 0, s>>>(type, lcell, n_list, counts);
}

void geo_sub_write(const uint8_t* type, const long long* lcell, int n_list, const int* offsets, int* lsub, int* lwall,
                   int* lbc, cudaStream_t s) {
  if (n_list <= 0) return;
  k_sub_write<<<nblocks(n_list, SUB_THREADS), SUB_THREADS, 0, s>>>(type, lcell, n_list, offsets, lsub, lwall, lbc);
}

void geo_pair_mix(const GeoArgs& g, const uint8_t* type, unsigned long long* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), s);
  const long long groups = (long long)((g.nx + 63) / 64) * g.ny * g.nz;
  k_pair_mix<<<nblocks(groups, 256), 256, 0, s>>>(g, type, out);
}

void geo_count_kinds(const uint8_t* type, long long N, unsigned long long* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, 5 * sizeof(unsigned long long), s);
  long long blocks = nblocks(N, 256);
  if (blocks > 4 * 1216) blocks = 4 * 1216;
  k_count_kinds<<<unsigned(blocks), 256, 0, s>>>(type, N, out);
}

// Slot codes of the list and NEAR cells, by cell index, so that the interior kernel's mixed path reads
// a cell's codes directly from its index rather than through its list position. Only those entries
// are written (and read); the others keep whatever they held.
template <int Q>
__global__ void k_cell_code(const GeoArgs g, const uint8_t* type, unsigned long long* ccode) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= g.N) return;
  const uint8_t t = type[n];
  if (!(t & (T_LIST | T_NEAR)) || (t & T_KIND) == K_SOLID) return;
  int x, y, z;
  coords(g, n, x, y, z);
  ccode[n] = slot_code<Q>(g, type, x, y, z);
}

void geo_cell_code(const GeoArgs& g, const uint8_t* type, unsigned long long* ccode, cudaStream_t s) {
  if (g.q == 19) k_cell_code<19><<<nblocks(g.N, 256), 256, 0, s>>>(g, type, ccode);
  else k_cell_code<27><<<nblocks(g.N, 256), 256, 0, s>>>(g, type, ccode);
}

void geo_list_index(const long long* lcell, int n_list, int* lidx, cudaStream_t s) {
  if (n_list <= 0) return;
  k_list_index<<<nblocks(n_list, 256), 256, 0, s>>>(lcell, n_list, lidx);
}

template <class T>
__global__ void k_halo_copy(bool gather, T* base, const long long* __restrict__ off, long long n, int width, T* buf) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const long long o = off[j];
  for (int c = 0; c < width; ++c) {
    if (gather) buf[j * width + c] = base[o + c];
    else base[o + c] = buf[j * width + c];
  }
}

void halo_copy(bool gather, void* base, const long long* off, long long n, int width, int elem, void* buf,
               cudaStream_t s) {
  if (n <= 0) return;
  const unsigned g = nblocks(n, 256);
  if (elem == 2) k_halo_copy<uint16_t><<<g, 256, 0, s>>>(gather, static_cast<uint16_t*>(base), off, n, width, static_cast<uint16_t*>(buf));
  else if (elem == 4) k_halo_copy<uint32_t><<<g, 256, 0, s>>>(gather, static_cast<uint32_t*>(base), off, n, width, static_cast<uint32_t*>(buf));
  else k_halo_copy<unsigned long long><<<g, 256, 0, s>>>(gather, static_cast<unsigned long long*>(base), off, n, width, static_cast<unsigned long long*>(buf));
}

void reduce_final(const double* partial, int nblk, double* out, cudaStream_t s) {
  k_reduce_final<<<1, 32, 0, s>>>(partial, nblk, out);
}

}  // namespace lbm
