// Host-side table of the kernel launchers of one (lattice, storage) instantiation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {
struct Args;

struct AdjArgs;

struct Ops {
  int q;
  int elem;      // bytes per stored population value
  int celem;     // bytes per compute value (float or double)
  // one step: interior kernel then boundary-list kernel; parity odd = step counter & 1
  void (*step_bulk)(const Args&, int odd, cudaStream_t);
  void (*step_list)(const Args&, int odd, cudaStream_t);
  // fused mode: wall-model state of the WALL entries before the interior kernel
  void (*wall_pass)(const Args&, cudaStream_t);
  // state access; swapped = state stored in the after-even-step form
  void (*init_eq)(const Args&, const void* rho, const void* u, int dtype, cudaStream_t);
  void (*moments)(const Args&, int swapped, void* rho, void* u, int dtype, cudaStream_t);
  void (*get_pops)(const Args&, int swapped, void* out, int dtype, cudaStream_t);
  void (*set_pops)(const Args&, int swapped, const void* in, int dtype, cudaStream_t);
  void (*ref_fill)(const Args&, int swapped, void* ref, cudaStream_t);
  // FP64 reduction: writes nblk partials of (mass, mom x, y, z)
  void (*reduce)(const Args&, int swapped, double* partial, int nblk, cudaStream_t);
  // list auxiliary data (normals, wall distances) from integer normal sums
  void (*list_aux)(const Args&, const int* nsum, const float* wall_dist, void* wnrm, void* wyw, cudaStream_t);
  // adjoint: out-of-place forward from a natural-layout state, reverse step, objective plane sums
  void (*step_oop)(const Args&, const void* fin, void* fout, cudaStream_t);
  void (*reverse)(const Args&, const AdjArgs&, cudaStream_t);
  void (*plane_rho)(const Args&, const void* state, int swapped, int xa, int xb, double* acc, double* scratch,
                    double wa, double wb, cudaStream_t);
  void (*seed)(const Args&, void* lam, int xa, int xb, double wa, double wb, cudaStream_t);
  void (*convert)(const void* in, int in_dtype, void* out, int out_dtype, long long n, cudaStream_t);
};

const Ops* ops_f64(int q);
const Ops* ops_f32(int q);
const Ops* ops_f16(int q);
const Ops* ops_bf16(int q);

// Geometry kernels (storage independent)
struct GeoArgs {
  int nx, ny, nz;
  long long nxy, N;
  int face[6];
  int q;
  int gh_lo, gh_hi;  // ghost z-planes below and above (slab sub-domain), flagged T_GHOST
};
void geo_classify(const GeoArgs&, const uint8_t* mask, uint8_t* type, unsigned* status, cudaStream_t);
// odd-step slots (p, m) of the non-solid cells of plane z_from that lie in plane z_to ((-1, -1) else),
// q * nx * ny entries each, direction-major
void geo_plane_slots(const GeoArgs&, const uint8_t* type, int z_from, int z_to, int* sp, long long* sm,
                     cudaStream_t);
// smallest index of an invalid mask code (first_bad = ~0 when every code is valid)
void geo_check_mask(const uint8_t* mask, long long N, unsigned long long* first_bad, cudaStream_t);
void geo_mark_ref(const GeoArgs&, uint8_t* type, cudaStream_t);
// list compaction: per-block counts (blocks of 256 cells), then scatter with block offsets
int geo_count_blocks(const GeoArgs&);
void geo_list_count(const GeoArgs&, uint8_t* type, int* counts, cudaStream_t);
void geo_list_write(const GeoArgs&, const uint8_t* type, const int* offsets, long long* lcell, cudaStream_t);
void geo_list_meta(const GeoArgs&, const uint8_t* type, const long long* lcell, int n_list, int* nsum, int* wref,
                   int* lxyz, unsigned long long* lcode, cudaStream_t);
// list position of every cell (-1 off the list)
void geo_list_index(const long long* lcell, int n_list, int* lidx, cudaStream_t);
// odd-step slot codes of every list and NEAR cell (the other entries are not written)
void geo_cell_code(const GeoArgs&, const uint8_t* type, unsigned long long* ccode, cudaStream_t);
// inline (fused-mode) flags per 32-cell x-group; sub-lists of the boundary list (3 per-block counts,
// then writes at offsets: not-inline, WALL, INFLOW/OUTFLOW); counts of WALL, reference,
// INFLOW, OUTFLOW and SOLID cells
void geo_inline_mark(const GeoArgs&, uint8_t* type, int inline_min, cudaStream_t);
int geo_sub_blocks(int n_list);
void geo_sub_count(const uint8_t* type, const long long* lcell, int n_list, int* counts, cudaStream_t);
void geo_sub_write(const uint8_t* type, const long long* lcell, int n_list, const int* offsets, int* lsub, int* lwall,
                   int* lbc, cudaStream_t);
void geo_count_kinds(const uint8_t* type, long long N, unsigned long long* out, cudaStream_t);
// 64-cell x-groups and the groups mixing plain pairs with per-cell pairs (nx even): out[0], out[1]
void geo_pair_mix(const GeoArgs&, const uint8_t* type, unsigned long long* out, cudaStream_t);
// source map (debug): for each (i, n): source population and cell, -1 for solid cells
void geo_source_map(const GeoArgs&, const uint8_t* type, int64_t* src_dir, int64_t* src_cell, cudaStream_t);
// halo copies of a slab sub-domain: gather (buf[j*width + c] = base[off[j] + c]) or scatter (the
// reverse) of n entries of width values of elem bytes (2, 4 or 8; raw bits)
void halo_copy(bool gather, void* base, const long long* off, long long n, int width, int elem, void* buf,
               cudaStream_t);
// FP64 final reduction of nblk partials (4 doubles each) into out[4], fixed order
void reduce_final(const double* partial, int nblk, double* out, cudaStream_t);
}  // namespace lbm
