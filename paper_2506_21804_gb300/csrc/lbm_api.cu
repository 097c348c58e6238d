// Host side of the C ABI declared in include/lbm.h: context lifetime, argument validation, device
// memory, geometry set-up, step orchestration, state access, checkpoints and the adjoint driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_adjoint.cuh"
#include "lbm_device.cuh"
#include "lbm_ops.h"
#include "lbm_vortex.h"
#include "lbm_porous.h"

using namespace lbm;

namespace {
thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  // (re)allocate to at least `bytes`; contents undefined
  cudaError_t ensure(size_t bytes) {
    if (bytes <= n && p) return cudaSuccess;
    release();
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) n = bytes;
    return e;
  }
};

constexpr int RED_BLOCKS = 1024;
constexpr uint32_t SAVE_MAGIC = 0x4C424D32u;  // "LBM2"

struct SaveHeader {
  uint32_t magic, q, storage, model;
  int64_t nx, ny, nz, n_list, t;
  uint64_t fbytes, rbytes, ubytes;  // populations, one reference buffer, HRR velocity field (0: none)
  double sigma;
  uint64_t vbytes;                  // vortex-inlet field of the last step (0: none)
};
}  // namespace

struct lbm_ctx {
  int q = 19, nx = 0, ny = 0, nz = 0;
  long long N = 0, stride = 0;
  int storage = LBM_F32;
  double tau0 = 0.6, cs = 0.0;
  int face[6] = {0, 0, 0, 0, 0, 0};
  double force[3] = {0, 0, 0};
  double rho_out = 1.0;
  bool wm = false;
  double kappa = 0.41, E = 9.52;
  int kernel = 0;       // LBM_OPT_KERNEL value
  int debug_stall = 0;  // LBM_OPT_DEBUG_STALL value
  int model = LBM_BGK;  // collision model
  double sigma = 1.0;   // HRR hybridisation factor
  bool uvel_stale = true;  // the HRR velocity field must be rebuilt from the state before the next step
  // vortex-method inlet (off when vm_n == 0)
  int vm_n = 0;
  double vm_sigma = 4.0, vm_I = 0.1;
  unsigned long long vm_seed = 0;
  int vm_which = 0;  // 0: the current inlet field is uin_a
  int device = 0;
  cudaStream_t stream = 0;
  const Ops* ops = nullptr;
  long long t = 0;
  long long launches = 0;  // kernels launched by the step calls (lbm_step, lbm_step_timed)
  unsigned status_seen = 0;
  // device buffers
  DevBuf f, type, mask, wdist, gamma, uin, lcell, nsum, wref, lxyz, lcode, wnrm, wyw, ref0, ref1, status, red, redout, stage;
  DevBuf lidx, lsub, lwall, lbc, wst, ccode;
  DevBuf uvel0, uvel1;  // HRR velocity fields (step t reads uvel[t & 1], writes the other)
  DevBuf uin_a, uin_b, vort, vpart;  // vortex inlet: current/previous inlet fields, vortex list, partial fields
  DevBuf fringe;  // outlet fringe zone: strength per x-plane (compute type)
  // slab sub-domain: ghost z-planes below/above, and per side (z-, z+) and halo list (0 real-plane
  // slots, 1 ghost-plane slots, 2 reference cells sent, 3 reference cells received) the device
  // offsets of the entries and their canonical form (slot * nx * ny + plane position, or position)
  int gh_lo = 0, gh_hi = 0;
  DevBuf halo_off[2][4];
  std::vector<int64_t> halo_map[2][4];
  int fr_L = 0;
  double fr_smax = 0.0, fr_p = 2.0;
  DevBuf geo_counts, geo_sub, geo_kinds;  // geometry set-up scratch (per-block counts, kind counters)
  double pair_mixed = 1.0;  // fraction of 64-cell x-groups mixing plain and per-cell pairs
  int n_sub = 0, n_wall = 0, n_bc = 0;
  bool has_gamma = false, has_wdist = false;
  int n_list = 0;
  long long counts[8] = {0};  // wall, ref, inflow, outflow, solid
  std::vector<double> uin_host;
  std::vector<uint8_t> type_host;  // host copy of the type bytes, valid when type_host_valid
  bool type_host_valid = false;
  unsigned* status_h = nullptr;
  double* red_h = nullptr;
  // adjoint state
  DevBuf lamA, lamB, dgam, duin, plane;
  DevBuf hist;  // every state of the last forward run (checkpoint interval 1), T + 1 states
  std::vector<DevBuf> ckpts, ring;
  int adj_T = 0, adj_W = 0, adj_xa = 0, adj_xb = 0, adj_ck = 0;
  double adj_wa = 0, adj_wb = 0;
  long long adj_t0 = -1;
  double adj_ms[3] = {0, 0, 0};

  ~lbm_ctx() {
    for (auto& side : halo_off)
      for (auto& b : side) b.release();
    DevBuf* all[] = {&fringe, &geo_counts, &geo_sub, &geo_kinds, &uin_a, &uin_b, &vort, &vpart, &uvel0, &uvel1, &lidx, &lsub, &lwall, &lbc, &wst, &ccode, &f, &type, &mask, &wdist, &gamma, &uin, &lcell, &nsum, &wref, &lxyz, &lcode, &wnrm, &wyw, &ref0, &ref1, &status, &red,
                     &redout, &stage, &lamA, &lamB, &dgam, &duin, &plane};
    for (DevBuf* b : all) b->release();
    for (auto& b : ckpts) b.release();
    for (auto& b : ring) b.release();
    if (status_h) cudaFreeHost(status_h);
    if (red_h) cudaFreeHost(red_h);
  }
};

namespace {

const Ops* pick_ops(int q, int storage) {
  switch (storage) {
    case LBM_F64: return ops_f64(q);
    case LBM_F32: return ops_f32(q);
    case LBM_F16: return ops_f16(q);
    case LBM_BF16: return ops_bf16(q);
  }
  return nullptr;
}

GeoArgs geo_args(const lbm_ctx* c) {
  GeoArgs g{};
  g.nx = c->nx; g.ny = c->ny; g.nz = c->nz;
  g.nxy = (long long)c->nx * c->ny;
  g.N = c->N;
  for (int i = 0; i < 6; ++i) g.face[i] = c->face[i];
  g.q = c->q;
  g.gh_lo = c->gh_lo;
  g.gh_hi = c->gh_hi;
  return g;
}

// The paired interior kernel (two cells per thread, packed FP32 collision) runs when nx is even, the
// indices fit 32 bits, the storage is not FP64, and few warps would mix plain pairs with pairs on the
// per-cell path (a mixed warp runs both): at most PAIR_MIX_MAX of the 64-cell x-groups mixed (the
// plane channel: none; a city canopy or a duct with inlet and outlet planes: many).
#ifndef LBM_PAIR_MIX_MAX
#define LBM_PAIR_MIX_MAX 0.02
#endif
bool pairs_selected(const lbm_ctx* c) {
  const bool idx32 = (unsigned long long)c->q * (unsigned long long)c->stride < (1ull << 32) && c->N < (1ll << 31);
  if (c->storage == LBM_F64 || c->nx % 2 != 0 || !idx32 || c->kernel != 0 || c->fr_L > 0) return false;
  return c->pair_mixed <= LBM_PAIR_MIX_MAX;
}

Args make_args(const lbm_ctx* c) {
  Args a{};
  a.f = c->f.p;
  a.stride = c->stride;
  a.type = static_cast<const uint8_t*>(c->type.p);
  a.gamma = c->has_gamma ? c->gamma.p : nullptr;
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
  a.nxy = (long long)c->nx * c->ny;
  a.N = c->N;
  for (int i = 0; i < 6; ++i) a.face[i] = c->face[i];
  a.tau0 = c->tau0;
  a.nu0 = (c->tau0 - 0.5) / 3.0;
  a.smag = 18.0 * std::sqrt(2.0) * c->cs * c->cs;
  a.use_smag = a.smag.d > 0.0;
  a.cs2smag = c->cs * c->cs;
  a.fx = c->force[0]; a.fy = c->force[1]; a.fz = c->force[2];
  a.status = static_cast<unsigned*>(c->status.p);
  a.lcell = static_cast<const long long*>(c->lcell.p);
  a.lxyz = static_cast<const int*>(c->lxyz.p);
  a.lcode = static_cast<const unsigned long long*>(c->lcode.p);
  a.n_list = c->n_list;
  a.wnrm = c->wnrm.p;
  a.wyw = c->wyw.p;
  a.wref = static_cast<const int*>(c->wref.p);
  // step t reads the reference velocities written in step t-1 and writes its own
  a.ref_rd = (c->t & 1) ? c->ref0.p : c->ref1.p;
  a.ref_wr = (c->t & 1) ? c->ref1.p : c->ref0.p;
  a.uin = c->vm_n > 0 ? (c->vm_which == 0 ? c->uin_a.p : c->uin_b.p) : c->uin.p;
  a.rho_out = c->rho_out;
  a.drho_out = c->rho_out - 1.0;
  a.wm = c->wm ? 1 : 0;
  a.kappa = c->kappa;
  a.E = c->E;
  a.kernel = c->kernel;
  a.fuse = c->kernel == 0 ? 1 : 0;
  a.inline_all = (a.fuse && c->model == LBM_BGK) ? 1 : 0;
  a.lidx = static_cast<const int*>(c->lidx.p);
  a.ccode = static_cast<const unsigned long long*>(c->ccode.p);
  a.lsub = a.fuse ? static_cast<const int*>(c->lsub.p) : nullptr;
  a.n_sub = c->n_sub;
  a.lwall = static_cast<const int*>(c->lwall.p);
  a.lbc = static_cast<const int*>(c->lbc.p);
  a.n_bc = c->n_bc;
  a.n_wall = c->n_wall;
  a.wst = c->wst.p;
  a.idx32 = ((unsigned long long)c->q * (unsigned long long)c->stride < (1ull << 32) && c->N < (1ll << 31)) ? 1 : 0;
  a.debug_stall = c->debug_stall;
  a.model = c->model;
  a.hybrid = (c->model == LBM_HRR && c->sigma < 1.0) ? 1 : 0;
  a.sigma = c->sigma;
  a.uvel_rd = (c->t & 1) ? c->uvel1.p : c->uvel0.p;
  a.uvel_wr = (c->t & 1) ? c->uvel0.p : c->uvel1.p;
  a.pairs = pairs_selected(c) ? 1 : 0;
  a.fringe = c->fr_L > 0 ? c->fringe.p : nullptr;
  a.ghost = (c->gh_lo > 0 || c->gh_hi > 0) ? 1 : 0;
  // HRR one-cell kernel: CTAs of whole warps along x, the x-face planes in columns of their own when
  // the x faces are not periodic (their cells are inlet, outlet, wall or slip cells)
  a.xcols = (c->face[0] != F_PERIODIC && c->nx >= 3) ? 1 : 0;
  {
    const unsigned t = unsigned(std::min(128, (c->nx + 31) / 32 * 32));
    a.lc_t = t;
    a.lc_gx = (unsigned(c->nx) + t - 1) / t;
    a.lc_gy = (unsigned(c->ny) + t - 1) / t;
    a.lc_cols = a.xcols ? 2u * a.lc_gy * unsigned(c->nz) : 0u;
    a.lc_dgx = FastDiv::make(a.lc_gx);
    a.lc_dny = FastDiv::make(unsigned(c->ny));
    a.lc_dgy = FastDiv::make(a.lc_gy);
  }
  a.fr_x0 = c->nx - c->fr_L;
  return a;
}

bool is_device_ptr(const void* p, int device) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == device;
}

// Pointer check: host (any kind) is fine; device pointers must be on the context's device.
int check_ptr(const lbm_ctx* c, const void* p, const char* what) {
  if (!p) return fail(LBM_EINVAL, "%s: null pointer", what);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return LBM_OK;
  }
  if ((at.type == cudaMemoryTypeDevice) && at.device != c->device)
    return fail(LBM_EINVAL, "%s: device pointer on device %d, context on device %d", what, at.device, c->device);
  return LBM_OK;
}

size_t dsize(int dtype) { return dtype == LBM_DTYPE_F64 ? 8 : 4; }

// Device address of page-locked host memory that kernels may read and write directly (over the
// CPU-GPU link, one pass, no staging copy), or null for any other pointer.
#ifndef LBM_MAPPED_HOST
#define LBM_MAPPED_HOST 1
#endif
void* mapped_host(const void* p) {
  if (!LBM_MAPPED_HOST || !p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int read_status(lbm_ctx* c) {
  CK(cudaMemcpyAsync(c->status_h, c->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->status_seen |= *c->status_h;
  return LBM_OK;
}

int status_code(lbm_ctx* c) {
  if (c->status_seen & 4u)
    return fail(LBM_ETIMEOUT, "a bounded wait in the staged step kernel ran out; the state is incomplete (re-initialise)");
  if (c->status_seen & ST_NAN) return fail(LBM_ENAN, "non-finite density or momentum seen by a step");
  return LBM_OK;
}

// Copy `bytes` from a host or device pointer into device buffer dst (stream-ordered).
int upload(lbm_ctx* c, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
  if (!is_device_ptr(src, c->device)) CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int alloc_state(lbm_ctx* c) {
  c->stride = (c->N + 127) / 128 * 128;
  CK(c->f.ensure((size_t)c->q * c->stride * c->ops->elem));
  CK(cudaMemsetAsync(c->f.p, 0, (size_t)c->q * c->stride * c->ops->elem, c->stream));
  return LBM_OK;
}

// Compute-type inlet velocity buffer from the host copy.
int upload_uin(lbm_ctx* c) {
  const size_t n = 3 * (size_t)c->ny * c->nz;
  CK(c->uin.ensure(n * c->ops->celem));
  if (c->ops->celem == 8) {
    CK(cudaMemcpyAsync(c->uin.p, c->uin_host.data(), n * 8, cudaMemcpyHostToDevice, c->stream));
  } else {
    std::vector<float> tmp(n);
    for (size_t i = 0; i < n; ++i) tmp[i] = float(c->uin_host[i]);
    CK(cudaMemcpyAsync(c->uin.p, tmp.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int build_halo(lbm_ctx* c);

// Classification and boundary list from the device mask; list auxiliary data in compute type.
int build_geometry(lbm_ctx* c) {
  const GeoArgs g = geo_args(c);
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(c->status.p, 0, sizeof(unsigned), s));
  geo_classify(g, static_cast<const uint8_t*>(c->mask.p), static_cast<uint8_t*>(c->type.p), static_cast<unsigned*>(c->status.p), s);
  geo_mark_ref(g, static_cast<uint8_t*>(c->type.p), s);
  const int nb = geo_count_blocks(g);
  DevBuf& counts = c->geo_counts;  // kept between calls: a geometry change allocates nothing new
  CK(counts.ensure((size_t)nb * sizeof(int)));
  geo_list_count(g, static_cast<uint8_t*>(c->type.p), static_cast<int*>(counts.p), s);
  std::vector<int> hc(nb);
  CK(cudaMemcpyAsync(hc.data(), counts.p, nb * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->status_h, c->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*c->status_h & ST_BADMASK) {
    return fail(LBM_EINVAL, "mask holds codes other than 0 (fluid), 1 (solid), 3 (inflow), 4 (outflow)");
  }
  long long total = 0;
  for (int b = 0; b < nb; ++b) {
    int v = hc[b];
    hc[b] = int(total);
    total += v;
  }
  if (total > 0x7fffffffLL) {
    return fail(LBM_EINVAL, "boundary list too long (%lld entries)", total);
  }
  c->n_list = int(total);
  CK(cudaMemcpyAsync(counts.p, hc.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
  const size_t nl = std::max<size_t>(1, (size_t)c->n_list);
  CK(c->lcell.ensure(nl * sizeof(long long)));
  geo_list_write(g, static_cast<const uint8_t*>(c->type.p), static_cast<const int*>(counts.p), static_cast<long long*>(c->lcell.p), s);
  CK(c->nsum.ensure(nl * 3 * sizeof(int)));
  CK(c->wref.ensure(nl * sizeof(int)));
  CK(c->lxyz.ensure(nl * 3 * sizeof(int)));
  CK(c->lcode.ensure(nl * sizeof(unsigned long long)));
  geo_list_meta(g, static_cast<const uint8_t*>(c->type.p), static_cast<const long long*>(c->lcell.p), c->n_list,
                static_cast<int*>(c->nsum.p), static_cast<int*>(c->wref.p), static_cast<int*>(c->lxyz.p),
                static_cast<unsigned long long*>(c->lcode.p), s);
  CK(c->wnrm.ensure(nl * 3 * c->ops->celem));
  CK(c->wyw.ensure(nl * c->ops->celem));
  CK(c->ref0.ensure(nl * 3 * c->ops->celem));
  CK(c->ref1.ensure(nl * 3 * c->ops->celem));
  CK(cudaMemsetAsync(c->ref0.p, 0, nl * 3 * c->ops->celem, s));
  CK(cudaMemsetAsync(c->ref1.p, 0, nl * 3 * c->ops->celem, s));
  Args a = make_args(c);
  c->ops->list_aux(a, static_cast<const int*>(c->nsum.p), c->has_wdist ? static_cast<const float*>(c->wdist.p) : nullptr,
                   c->wnrm.p, c->wyw.p, s);
  CK(cudaGetLastError());
  // list position of every cell, and the sub-lists of INFLOW/OUTFLOW and WALL entries
  CK(c->lidx.ensure((size_t)c->N * sizeof(int)));
  CK(cudaMemsetAsync(c->lidx.p, 0xFF, (size_t)c->N * sizeof(int), s));
  geo_list_index(static_cast<const long long*>(c->lcell.p), c->n_list, static_cast<int*>(c->lidx.p), s);
  CK(c->ccode.ensure((size_t)c->N * sizeof(unsigned long long)));
  geo_cell_code(g, static_cast<const uint8_t*>(c->type.p), static_cast<unsigned long long*>(c->ccode.p), s);
  CK(c->wst.ensure(nl * WALL_STATE * c->ops->celem));
  CK(cudaMemsetAsync(c->wst.p, 0, nl * WALL_STATE * c->ops->celem, s));
  {
    // Inline (fused-mode) choice: INFLOW/OUTFLOW cells are always updated by the interior kernel
    // (their extra work is a short reconstruction before the shared collision); WALL and reference
    // cells when their 32-cell x-group holds at least INLINE_MIN list cells. Isolated WALL and
    // reference cells stay with the boundary-list kernel. Then the sub-lists of the boundary list.
#ifndef LBM_INLINE_MIN
#define LBM_INLINE_MIN 8
#endif
    constexpr int INLINE_MIN = LBM_INLINE_MIN;
    uint8_t* type = static_cast<uint8_t*>(c->type.p);
    const long long* lcell = static_cast<const long long*>(c->lcell.p);
    geo_inline_mark(g, type, INLINE_MIN, s);
    const int sb = std::max(1, geo_sub_blocks(c->n_list));
    DevBuf& sc = c->geo_sub;
    CK(sc.ensure((size_t)sb * 3 * sizeof(int)));
    std::vector<int> hs(3 * (size_t)sb, 0);
    if (c->n_list) {
      geo_sub_count(type, lcell, c->n_list, static_cast<int*>(sc.p), s);
      CK(cudaMemcpyAsync(hs.data(), sc.p, hs.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    int tot[3] = {0, 0, 0};
    for (int b = 0; b < sb; ++b)
      for (int k = 0; k < 3; ++k) {
        const int v = hs[3 * b + k];
        hs[3 * b + k] = tot[k];
        tot[k] += v;
      }
    c->n_sub = tot[0]; c->n_wall = tot[1]; c->n_bc = tot[2];
    CK(c->lsub.ensure(std::max<size_t>(1, (size_t)tot[0]) * sizeof(int)));
    CK(c->lwall.ensure(std::max<size_t>(1, (size_t)tot[1]) * sizeof(int)));
    CK(c->lbc.ensure(std::max<size_t>(1, (size_t)tot[2]) * sizeof(int)));
    if (c->n_list) {
      CK(cudaMemcpyAsync(sc.p, hs.data(), hs.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      geo_sub_write(type, lcell, c->n_list, static_cast<const int*>(sc.p), static_cast<int*>(c->lsub.p),
                    static_cast<int*>(c->lwall.p), static_cast<int*>(c->lbc.p), s);
    }
    // cell-kind counters
    DevBuf& kc = c->geo_kinds;
    CK(kc.ensure(5 * sizeof(unsigned long long)));
    geo_count_kinds(type, c->N, static_cast<unsigned long long*>(kc.p), s);
    unsigned long long hk[5];
    CK(cudaMemcpyAsync(hk, kc.p, sizeof(hk), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    for (int i = 0; i < 5; ++i) c->counts[i] = (long long)hk[i];
    c->pair_mixed = 1.0;
    if (c->nx % 2 == 0) {
      geo_pair_mix(g, type, static_cast<unsigned long long*>(kc.p), s);
      unsigned long long pm[2];
      CK(cudaMemcpyAsync(pm, kc.p, sizeof(pm), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      c->pair_mixed = pm[0] ? double(pm[1]) / double(pm[0]) : 1.0;
    }
  }
  c->type_host_valid = false;
  if (c->gh_lo > 0 || c->gh_hi > 0) return build_halo(c);
  return LBM_OK;
}

// Host copy of the type bytes (fetched on first use after a geometry change).
const std::vector<uint8_t>& host_types(lbm_ctx* c) {
  if (!c->type_host_valid) {
    c->type_host.resize(c->N);
    cudaMemcpyAsync(c->type_host.data(), c->type.p, c->N, cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    c->type_host_valid = true;
  }
  return c->type_host;
}

// Halo lists of a slab sub-domain (the z decomposition of Sec. 3.1), per side s (0: z-, 1: z+), with
// zr the real boundary plane and zg the adjacent ghost plane, entries over the plane positions
// pos = x + nx y ascending, then slots p ascending:
//   0: slots (p, zr cell) that the non-solid cells of zg use in an odd step (slot_of). After an even
//      step they hold the post-collision populations opp(p) that leave through the cut; after an odd
//      step the neighbour's populations that arrived there. A slot that a cell of zr uses itself
//      (bounce-back from a solid cell across the cut) is not on the list.
//   1: slots (p, zg cell) that the non-solid cells of zr use: the neighbour's leaving populations
//      (before an odd step), then the ones this sub-domain sent into them (after it).
//   2: zr cells that a WALL cell of zg takes as reference cell; 3: zg cells that a WALL cell of zr
//      takes as reference cell (their wall-model reference velocities cross the cut).
// The neighbour's list 1 (3) on the other side of the same cut is this list 0 (2), entry by entry.
int build_halo(lbm_ctx* c) {
  const std::vector<uint8_t>& th = host_types(c);
  const long long nxy = (long long)c->nx * c->ny;
  std::vector<long long> lcell(std::max(1, c->n_list));
  std::vector<int> wref(std::max(1, c->n_list));
  if (c->n_list > 0) {
    CK(cudaMemcpy(lcell.data(), c->lcell.p, sizeof(long long) * c->n_list, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(wref.data(), c->wref.p, sizeof(int) * c->n_list, cudaMemcpyDeviceToHost));
  }
  for (int side = 0; side < 2; ++side) {
    const int g = side == 0 ? c->gh_lo : c->gh_hi;
    const long long zr = side == 0 ? c->gh_lo : c->nz - c->gh_hi - 1;
    const long long zg = side == 0 ? c->gh_lo - 1 : c->nz - c->gh_hi;
    std::vector<int64_t> map[4], off[4];
    if (g > 0) {
      // list 0: the slots of zr that the cells of zg use in an odd step; list 1: the slots of zg that
      // the cells of zr use (the slot map of every cell, computed on the device for the two planes)
      const GeoArgs ga = geo_args(c);
      DevBuf sp, sm;
      CK(sp.ensure((size_t)c->q * nxy * sizeof(int)));
      CK(sm.ensure((size_t)c->q * nxy * sizeof(long long)));
      std::vector<int> hp((size_t)c->q * nxy);
      std::vector<long long> hm((size_t)c->q * nxy);
      for (int lst = 0; lst < 2; ++lst) {
        const int zf = int(lst == 0 ? zg : zr), zt = int(lst == 0 ? zr : zg);
        geo_plane_slots(ga, static_cast<const uint8_t*>(c->type.p), zf, zt, static_cast<int*>(sp.p),
                        static_cast<long long*>(sm.p), c->stream);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(hp.data(), sp.p, hp.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(hm.data(), sm.p, hm.size() * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        std::vector<std::pair<long long, int>> e;  // (pos in the target plane, slot)
        for (size_t k = 0; k < hp.size(); ++k)
          if (hp[k] >= 0) e.emplace_back(hm[k] - nxy * zt, hp[k]);
        std::sort(e.begin(), e.end());
        for (const auto& v : e) {
          map[lst].push_back((int64_t)v.second * nxy + v.first);
          off[lst].push_back((int64_t)v.second * c->stride + v.first + nxy * zt);
        }
      }
      sp.release();
      sm.release();
      // list positions of the cells of the two planes, and the reference relations across the cut
      std::vector<int> kpos_r(nxy, -1), kpos_g(nxy, -1);
      std::vector<uint8_t> hit2(nxy, 0), hit3(nxy, 0);
      for (int k = 0; k < c->n_list; ++k) {
        const long long n = lcell[k], z = n / nxy;
        if (z == zr) kpos_r[n - nxy * zr] = k;
        if (z == zg) kpos_g[n - nxy * zg] = k;
      }
      for (int k = 0; k < c->n_list; ++k) {
        const long long w = lcell[k], z = w / nxy;
        if ((th[w] & T_KIND) != K_WALL || wref[k] < 0) continue;
        const long long r = lcell[wref[k]], zr_ = r / nxy;
        if (z == zg && zr_ == zr) hit2[r - nxy * zr] = 1;
        if (z == zr && zr_ == zg) hit3[r - nxy * zg] = 1;
      }
      for (long long pos = 0; pos < nxy; ++pos) {
        if (hit2[pos]) {
          map[2].push_back(pos);
          off[2].push_back(3 * (int64_t)kpos_r[pos]);
        }
        if (hit3[pos]) {
          map[3].push_back(pos);
          off[3].push_back(3 * (int64_t)kpos_g[pos]);
        }
      }
    }
    for (int lst = 0; lst < 4; ++lst) {
      c->halo_map[side][lst] = map[lst];
      CK(c->halo_off[side][lst].ensure(std::max<size_t>(1, off[lst].size()) * sizeof(int64_t)));
      if (!off[lst].empty())
        CK(cudaMemcpy(c->halo_off[side][lst].p, off[lst].data(), off[lst].size() * sizeof(int64_t),
                      cudaMemcpyHostToDevice));
    }
  }
  return LBM_OK;
}

// One time step: in fused mode the wall-model states of the WALL entries first, then the interior
// kernel, then the boundary-list kernel. Events (optional) bracket the interior kernel.
int fill_uvel(lbm_ctx* c);

// Vortex inlet: the inlet field restarts from the mean profile.
int vm_reset(lbm_ctx* c) {
  if (c->vm_n <= 0) return LBM_OK;
  const size_t pb = 3 * (size_t)c->ny * c->nz * c->ops->celem;
  CK(c->uin_a.ensure(pb));
  CK(c->uin_b.ensure(pb));
  CK(c->vort.ensure(3 * (size_t)c->vm_n * c->ops->celem));
  CK(c->vpart.ensure(2 * (size_t)((c->vm_n + VM_CHUNK - 1) / VM_CHUNK) * c->ny * c->nz * c->ops->celem));
  CK(cudaMemcpyAsync(c->uin_a.p, c->uin.p, pb, cudaMemcpyDeviceToDevice, c->stream));
  c->vm_which = 0;
  return LBM_OK;
}

// Vortex inlet: the inlet field of step t from the vortices of step t and the previous field.
void vm_step(lbm_ctx* c) {
  VmArgs v{};
  v.ny = c->ny; v.nz = c->nz; v.n = c->vm_n;
  v.sigma = c->vm_sigma; v.I = c->vm_I; v.seed = c->vm_seed; v.t = c->t;
  v.area = c->counts[2];
  v.gden = 6.0 * std::log(3.0) - 9.0 * std::log(2.0);
  v.mean = c->uin.p;
  v.prev = c->vm_which == 0 ? c->uin_a.p : c->uin_b.p;
  v.cur = c->vm_which == 0 ? c->uin_b.p : c->uin_a.p;
  v.vort = c->vort.p;
  v.part = c->vpart.p;
  vm_update(v, c->ops->celem, c->stream);
  c->vm_which ^= 1;
}

void launch_step(lbm_ctx* c, cudaEvent_t before_bulk = nullptr, cudaEvent_t after_bulk = nullptr) {
  if (c->model == LBM_HRR && c->uvel_stale) {
    fill_uvel(c);
    ++c->launches;
  }
  if (c->vm_n > 0) {
    vm_step(c);
    c->launches += 3;  // vortex generation, partial fields, final field
  }
  const Args a = make_args(c);
  const int odd = int(c->t & 1);
  if (a.fuse && a.wm && a.n_wall > 0) {
    c->ops->wall_pass(a, c->stream);
    ++c->launches;
  }
  if (before_bulk) cudaEventRecord(before_bulk, c->stream);
  c->ops->step_bulk(a, odd, c->stream);
  ++c->launches;
  if (after_bulk) cudaEventRecord(after_bulk, c->stream);
  if (!a.inline_all && (a.lsub ? a.n_sub : a.n_list) > 0) {
    c->ops->step_list(a, odd, c->stream);
    ++c->launches;
  }
  ++c->t;
}

// State to rest (f = w), step counter 0, reference buffers from that state.
int reset_state(lbm_ctx* c) {
  c->uvel_stale = true;
  if (vm_reset(c) != LBM_OK) return LBM_ECUDA;
  CK(cudaMemsetAsync(c->f.p, 0, (size_t)c->q * c->stride * c->ops->elem, c->stream));
  c->t = 0;
  c->adj_t0 = -1;
  const size_t nl = std::max<size_t>(1, (size_t)c->n_list);
  CK(cudaMemsetAsync(c->ref0.p, 0, nl * 3 * c->ops->celem, c->stream));
  CK(cudaMemsetAsync(c->ref1.p, 0, nl * 3 * c->ops->celem, c->stream));
  return LBM_OK;
}

// HRR velocity field of the current state (reported velocity of every cell) into the buffer the
// next step reads.
int fill_uvel(lbm_ctx* c) {
  const size_t bytes = 3 * (size_t)c->N * c->ops->celem;
  CK(c->uvel0.ensure(bytes));
  CK(c->uvel1.ensure(bytes));
  Args a = make_args(c);
  c->ops->moments(a, int(c->t & 1), nullptr, const_cast<void*>(a.uvel_rd),
                  c->ops->celem == 8 ? LBM_DTYPE_F64 : LBM_DTYPE_F32, c->stream);
  CK(cudaGetLastError());
  c->uvel_stale = false;
  return LBM_OK;
}

int fill_refs(lbm_ctx* c) {
  c->uvel_stale = true;
  if (vm_reset(c) != LBM_OK) return LBM_ECUDA;
  Args a = make_args(c);
  const int sw = int(c->t & 1);
  c->ops->ref_fill(a, sw, c->ref0.p, c->stream);
  c->ops->ref_fill(a, sw, c->ref1.p, c->stream);
  CK(cudaGetLastError());
  return LBM_OK;
}

// Convert a caller array (dtype, host or device) into a device buffer of the compute type.
int upload_compute(lbm_ctx* c, DevBuf& dst, const void* src, int dtype, size_t count) {
  const size_t bytes = count * dsize(dtype);
  CK(dst.ensure(count * c->ops->celem));
  CK(c->stage.ensure(bytes));
  CK(cudaMemcpyAsync(c->stage.p, src, bytes, cudaMemcpyDefault, c->stream));
  c->ops->convert(c->stage.p, dtype, dst.p, c->ops->celem == 8 ? LBM_DTYPE_F64 : LBM_DTYPE_F32, (long long)count, c->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int valid_dtype(int dtype) { return dtype == LBM_DTYPE_F32 || dtype == LBM_DTYPE_F64; }

}  // namespace

// =================================================================================================
extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

lbm_ctx* lbm_create(int lattice, int nx, int ny, int nz, double tau, double c_smag) {
  if (lattice != 19 && lattice != 27) { fail(LBM_EINVAL, "lattice must be 19 or 27"); return nullptr; }
  if (nx < 1 || ny < 1 || nz < 1) { fail(LBM_EINVAL, "grid sizes must be >= 1"); return nullptr; }
  if ((long long)nx * ny > 0x7fffffffLL || nz > 65535 || ny > 65535) {
    fail(LBM_EINVAL, "grid too large for the launch shape (nx*ny < 2^31, ny <= 65535, nz <= 65535)");
    return nullptr;
  }
  if (!(tau > 0.5) || !std::isfinite(tau)) { fail(LBM_EINVAL, "tau must be > 1/2"); return nullptr; }
  if (!(c_smag >= 0.0) || !std::isfinite(c_smag)) { fail(LBM_EINVAL, "c_smag must be >= 0"); return nullptr; }
  lbm_ctx* c = new lbm_ctx();
  c->q = lattice; c->nx = nx; c->ny = ny; c->nz = nz;
  c->N = (long long)nx * ny * nz;
  c->tau0 = tau; c->cs = c_smag;
  c->ops = pick_ops(lattice, LBM_F32);
  c->uin_host.assign(3 * (size_t)ny * nz, 0.0);
  auto bail = [&](const char* what, cudaError_t e) {
    fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    delete c;
    return nullptr;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess) return bail("cudaGetDevice", e);
  if ((e = cudaMallocHost(&c->status_h, sizeof(unsigned))) != cudaSuccess) return bail("cudaMallocHost", e);
  if ((e = cudaMallocHost(&c->red_h, 4 * sizeof(double))) != cudaSuccess) return bail("cudaMallocHost", e);
  if ((e = c->status.ensure(sizeof(unsigned))) != cudaSuccess) return bail("status", e);
  if ((e = c->red.ensure(RED_BLOCKS * 4 * sizeof(double))) != cudaSuccess) return bail("reduction", e);
  if ((e = c->redout.ensure(4 * sizeof(double))) != cudaSuccess) return bail("reduction", e);
  if ((e = c->type.ensure(((size_t)c->N + 3) / 4 * 4)) != cudaSuccess) return bail("type", e);
  if ((e = c->mask.ensure((size_t)c->N)) != cudaSuccess) return bail("mask", e);
  cudaMemset(c->mask.p, 0, c->N);
  cudaMemset(c->type.p, 0, ((size_t)c->N + 3) / 4 * 4);
  cudaMemset(c->status.p, 0, sizeof(unsigned));
  if (alloc_state(c) != LBM_OK) { delete c; return nullptr; }
  if (upload_uin(c) != LBM_OK || build_geometry(c) != LBM_OK || reset_state(c) != LBM_OK) { delete c; return nullptr; }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) { fail(LBM_ECUDA, "create: %s", cudaGetErrorString(cudaGetLastError())); delete c; return nullptr; }
  return c;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  delete c;
}

int lbm_set_stream(lbm_ctx* c, void* s) {
  if (!c) return fail(LBM_EINVAL, "null context");
  c->stream = static_cast<cudaStream_t>(s);
  return LBM_OK;
}

int lbm_set_precision(lbm_ctx* c, int storage) {
  if (!c) return fail(LBM_EINVAL, "null context");
  const Ops* o = pick_ops(c->q, storage);
  if (!o) return fail(LBM_EINVAL, "storage must be LBM_F64, LBM_F32, LBM_F16 or LBM_BF16");
  CK(cudaStreamSynchronize(c->stream));
  // compute-typed side buffers follow the new compute type
  std::vector<double> g;
  if (c->has_gamma) {
    g.resize(c->N);
    CK(c->stage.ensure((size_t)c->N * 8));
    c->ops->convert(c->gamma.p, c->ops->celem == 8 ? LBM_DTYPE_F64 : LBM_DTYPE_F32, c->stage.p, LBM_DTYPE_F64, c->N, c->stream);
    CK(cudaMemcpyAsync(g.data(), c->stage.p, (size_t)c->N * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  c->storage = storage;
  c->ops = o;
  c->f.release();
  c->gamma.release();
  int rc;
  if ((rc = alloc_state(c)) != LBM_OK) return rc;
  if ((rc = upload_uin(c)) != LBM_OK) return rc;
  if (c->has_gamma && (rc = upload_compute(c, c->gamma, g.data(), LBM_DTYPE_F64, c->N)) != LBM_OK) return rc;
  c->wnrm.release(); c->wyw.release(); c->ref0.release(); c->ref1.release();
  c->uvel0.release(); c->uvel1.release();
  c->uin_a.release(); c->uin_b.release(); c->vort.release(); c->vpart.release();
  if (c->fr_L > 0) {
    c->fringe.release();
    if ((rc = lbm_set_fringe(c, c->fr_L, c->fr_smax, c->fr_p)) != LBM_OK) return rc;
  }
  if ((rc = build_geometry(c)) != LBM_OK) return rc;
  return reset_state(c);
}

int lbm_set_faces(lbm_ctx* c, const int kinds[6]) {
  if (!c || !kinds) return fail(LBM_EINVAL, "null argument");
  for (int f = 0; f < 6; ++f)
    if (kinds[f] < 0 || kinds[f] > 3) return fail(LBM_EINVAL, "face kind %d out of range", kinds[f]);
  for (int a = 0; a < 3; ++a)
    if ((kinds[2 * a] == LBM_FACE_PERIODIC) != (kinds[2 * a + 1] == LBM_FACE_PERIODIC))
      return fail(LBM_EINVAL, "periodic faces must come in pairs (axis %d)", a);
  CK(cudaStreamSynchronize(c->stream));
  for (int f = 0; f < 6; ++f) c->face[f] = kinds[f];
  int rc = build_geometry(c);
  if (rc != LBM_OK) return rc;
  return reset_state(c);
}

int lbm_set_periodic(lbm_ctx* c, int px, int py, int pz) {
  if (!c) return fail(LBM_EINVAL, "null context");
  int k[6] = {px ? 0 : 1, px ? 0 : 1, py ? 0 : 1, py ? 0 : 1, pz ? 0 : 1, pz ? 0 : 1};
  return lbm_set_faces(c, k);
}

int lbm_set_geometry(lbm_ctx* c, const uint8_t* mask, const float* wall_dist) {
  if (!c) return fail(LBM_EINVAL, "null context");
  int rc;
  if ((rc = check_ptr(c, mask, "mask")) != LBM_OK) return rc;
  if (wall_dist && (rc = check_ptr(c, wall_dist, "wall_dist")) != LBM_OK) return rc;
  CK(cudaStreamSynchronize(c->stream));
  // The mask goes to a staging buffer and its codes are checked there, on the device; only a valid
  // mask replaces the current one, so a rejected call changes nothing.
  {
    cudaStream_t s = c->stream;
    CK(c->stage.ensure((size_t)c->N));
    CK(c->geo_kinds.ensure(5 * sizeof(unsigned long long)));
    CK(cudaMemcpyAsync(c->stage.p, mask, (size_t)c->N, cudaMemcpyDefault, s));
    unsigned long long* first_bad = static_cast<unsigned long long*>(c->geo_kinds.p);
    geo_check_mask(static_cast<const uint8_t*>(c->stage.p), c->N, first_bad, s);
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bad, first_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (bad != ~0ull) {
      uint8_t v = 0;
      CK(cudaMemcpy(&v, static_cast<const uint8_t*>(c->stage.p) + bad, 1, cudaMemcpyDeviceToHost));
      return fail(LBM_EINVAL, "mask[%lld] = %d: codes are 0 fluid, 1 solid, 3 inflow, 4 outflow", (long long)bad, int(v));
    }
    CK(cudaMemcpyAsync(c->mask.p, c->stage.p, (size_t)c->N, cudaMemcpyDeviceToDevice, s));
  }
  if (wall_dist) {
    CK(c->wdist.ensure((size_t)c->N * sizeof(float)));
    if ((rc = upload(c, c->wdist.p, wall_dist, (size_t)c->N * sizeof(float))) != LBM_OK) return rc;
    c->has_wdist = true;
  } else {
    c->has_wdist = false;
  }
  if ((rc = build_geometry(c)) != LBM_OK) {
    cudaMemsetAsync(c->mask.p, 0, c->N, c->stream);
    build_geometry(c);
    reset_state(c);
    return rc;
  }
  return reset_state(c);
}

int lbm_set_force(lbm_ctx* c, double fx, double fy, double fz) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!std::isfinite(fx) || !std::isfinite(fy) || !std::isfinite(fz)) return fail(LBM_EINVAL, "force must be finite");
  c->force[0] = fx; c->force[1] = fy; c->force[2] = fz;
  return LBM_OK;
}

int lbm_set_inflow_ex(lbm_ctx* c, const void* u_in, int dtype) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!valid_dtype(dtype)) return fail(LBM_EINVAL, "dtype must be LBM_DTYPE_F32 or LBM_DTYPE_F64");
  int rc;
  if ((rc = check_ptr(c, u_in, "u_in")) != LBM_OK) return rc;
  const size_t n = 3 * (size_t)c->ny * c->nz;
  CK(cudaStreamSynchronize(c->stream));
  std::vector<unsigned char> tmp(n * dsize(dtype));
  CK(cudaMemcpy(tmp.data(), u_in, tmp.size(), cudaMemcpyDefault));
  for (size_t i = 0; i < n; ++i) {
    const double v = dtype == LBM_DTYPE_F64 ? reinterpret_cast<const double*>(tmp.data())[i]
                                            : double(reinterpret_cast<const float*>(tmp.data())[i]);
    if (!std::isfinite(v) || (i < (size_t)c->ny * c->nz && v >= 1.0)) return fail(LBM_EINVAL, "u_in[%zu] = %g invalid", i, v);
    c->uin_host[i] = v;
  }
  if ((rc = upload_uin(c)) != LBM_OK) return rc;
  return vm_reset(c);
}
int lbm_set_inflow(lbm_ctx* c, const float* u_in) { return lbm_set_inflow_ex(c, u_in, LBM_DTYPE_F32); }

int lbm_set_outflow(lbm_ctx* c, double rho_out) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!(rho_out > 0.0) || !std::isfinite(rho_out)) return fail(LBM_EINVAL, "rho_out must be > 0");
  c->rho_out = rho_out;
  return LBM_OK;
}

int lbm_set_fringe(lbm_ctx* c, int L, double s_max, double p) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (L < 0 || L > c->nx) return fail(LBM_EINVAL, "fringe length %d outside 0..nx = %d", L, c->nx);
  if (!(s_max >= 0.0 && s_max <= 1.0)) return fail(LBM_EINVAL, "fringe strength must lie in [0, 1]");
  if (!(p >= 0.0) || !std::isfinite(p)) return fail(LBM_EINVAL, "fringe exponent must be finite and >= 0");
  if (L == 0) {
    c->fringe.release();
    c->fr_L = 0;
    return LBM_OK;
  }
  // s(x) = s_max xi^p, xi = (x - (nx - L) + 1) / L on the layer, 0 before it (formed in double)
  std::vector<double> sd(c->nx, 0.0);
  for (int x = c->nx - L; x < c->nx; ++x) sd[x] = s_max * std::pow(double(x - (c->nx - L) + 1) / double(L), p);
  CK(c->fringe.ensure((size_t)c->nx * c->ops->celem));
  if (c->ops->celem == 8) {
    CK(cudaMemcpyAsync(c->fringe.p, sd.data(), (size_t)c->nx * 8, cudaMemcpyHostToDevice, c->stream));
  } else {
    std::vector<float> sf(sd.begin(), sd.end());
    CK(cudaMemcpyAsync(c->fringe.p, sf.data(), (size_t)c->nx * 4, cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  c->fr_L = L;
  c->fr_smax = s_max;
  c->fr_p = p;
  return LBM_OK;
}

int lbm_set_ghost_planes(lbm_ctx* c, int lo, int hi) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!(lo == 0 || lo == 2) || !(hi == 0 || hi == 2) || lo + hi >= c->nz)
    return fail(LBM_EINVAL, "ghost planes: 0 or 2 per side and fewer than nz = %d in total", c->nz);
  if ((lo || hi) && (c->model != LBM_BGK || c->vm_n > 0))
    return fail(LBM_ESTATE, "slab sub-domains run the BGK collision with a steady inlet");
  CK(cudaStreamSynchronize(c->stream));
  c->gh_lo = lo;
  c->gh_hi = hi;
  int rc;
  if ((rc = build_geometry(c)) != LBM_OK) return rc;
  return reset_state(c);
}

// element bytes and width of a halo list entry, and the array it lives in
static int halo_target(lbm_ctx* c, int side, int list, bool pack, void** base, int* width, int* elem, long long* n) {
  if (side < 0 || side > 1 || list < 0 || list > 3) return fail(LBM_EINVAL, "side must be 0 or 1, list 0..3");
  if (pack && list == 3) return fail(LBM_EINVAL, "list 3 (reference cells received) is unpacked only");
  if (!pack && list == 2) return fail(LBM_EINVAL, "list 2 (reference cells sent) is packed only");
  *n = (long long)c->halo_map[side][list].size();
  if (list <= 1) {
    *base = c->f.p;
    *width = 1;
    *elem = c->ops->elem;
  } else {
    // the reference buffer the last step wrote, which the next step reads
    *base = const_cast<void*>(make_args(c).ref_rd);
    *width = 3;
    *elem = c->ops->celem;
  }
  return LBM_OK;
}

int lbm_halo_count(lbm_ctx* c, int side, int list, int64_t* n) {
  if (!c || !n) return fail(LBM_EINVAL, "null argument");
  if (side < 0 || side > 1 || list < 0 || list > 3) return fail(LBM_EINVAL, "side must be 0 or 1, list 0..3");
  *n = (int64_t)c->halo_map[side][list].size();
  return LBM_OK;
}

int lbm_halo_pack(lbm_ctx* c, int side, int list, void* buf) {
  if (!c) return fail(LBM_EINVAL, "null context");
  void* base;
  int width, elem, rc;
  long long n;
  if ((rc = halo_target(c, side, list, true, &base, &width, &elem, &n)) != LBM_OK) return rc;
  if (n == 0) return LBM_OK;
  if ((rc = check_ptr(c, buf, "buf")) != LBM_OK) return rc;
  const size_t bytes = (size_t)n * width * elem;
  const long long* off = static_cast<const long long*>(c->halo_off[side][list].p);
  if (is_device_ptr(buf, c->device)) {
    halo_copy(true, base, off, n, width, elem, buf, c->stream);
  } else {
    CK(c->stage.ensure(bytes));
    halo_copy(true, base, off, n, width, elem, c->stage.p, c->stream);
    CK(cudaMemcpyAsync(buf, c->stage.p, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  CK(cudaGetLastError());
  return LBM_OK;
}

int lbm_halo_unpack(lbm_ctx* c, int side, int list, const void* buf) {
  if (!c) return fail(LBM_EINVAL, "null context");
  void* base;
  int width, elem, rc;
  long long n;
  if ((rc = halo_target(c, side, list, false, &base, &width, &elem, &n)) != LBM_OK) return rc;
  if (n == 0) return LBM_OK;
  if ((rc = check_ptr(c, buf, "buf")) != LBM_OK) return rc;
  const size_t bytes = (size_t)n * width * elem;
  const long long* off = static_cast<const long long*>(c->halo_off[side][list].p);
  if (is_device_ptr(buf, c->device)) {
    halo_copy(false, base, off, n, width, elem, const_cast<void*>(buf), c->stream);
  } else {
    CK(c->stage.ensure(bytes));
    CK(cudaMemcpyAsync(c->stage.p, buf, bytes, cudaMemcpyHostToDevice, c->stream));
    halo_copy(false, base, off, n, width, elem, c->stage.p, c->stream);
    CK(cudaStreamSynchronize(c->stream));
  }
  CK(cudaGetLastError());
  return LBM_OK;
}

int lbm_set_porosity_ex(lbm_ctx* c, const void* gamma, int dtype) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!gamma) {
    c->has_gamma = false;
    return LBM_OK;
  }
  if (!valid_dtype(dtype)) return fail(LBM_EINVAL, "dtype must be LBM_DTYPE_F32 or LBM_DTYPE_F64");
  int rc;
  if ((rc = check_ptr(c, gamma, "gamma")) != LBM_OK) return rc;
  CK(cudaStreamSynchronize(c->stream));
  if ((rc = upload_compute(c, c->gamma, gamma, dtype, c->N)) != LBM_OK) return rc;
  c->has_gamma = true;
  return LBM_OK;
}
int lbm_set_porosity(lbm_ctx* c, const float* gamma) { return lbm_set_porosity_ex(c, gamma, LBM_DTYPE_F32); }

int lbm_set_permeability_ex(lbm_ctx* c, const void* K, int dtype) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!valid_dtype(dtype)) return fail(LBM_EINVAL, "dtype must be LBM_DTYPE_F32 or LBM_DTYPE_F64");
  int rc;
  if ((rc = check_ptr(c, K, "K")) != LBM_OK) return rc;
  const size_t bytes = (size_t)c->N * dsize(dtype);
  CK(cudaStreamSynchronize(c->stream));
  CK(c->stage.ensure(bytes));
  CK(cudaMemcpyAsync(c->stage.p, K, bytes, cudaMemcpyDefault, c->stream));
  CK(c->gamma.ensure((size_t)c->N * c->ops->celem));
  const double nu = (c->tau0 - 0.5) / 3.0;
  porous_gamma(c->stage.p, dtype, c->gamma.p, c->ops->celem, c->N, nu * c->tau0, c->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  c->has_gamma = true;
  return LBM_OK;
}
int lbm_set_permeability(lbm_ctx* c, const float* K) { return lbm_set_permeability_ex(c, K, LBM_DTYPE_F32); }

int lbm_set_wall_model(lbm_ctx* c, double kappa, double E) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!(kappa > 0.0)) {
    c->wm = false;
    return LBM_OK;
  }
  if (!(E > 0.0) || !std::isfinite(E) || !std::isfinite(kappa)) return fail(LBM_EINVAL, "E must be > 0");
  c->wm = true;
  c->kappa = kappa;
  c->E = E;
  return LBM_OK;
}

int lbm_init_equilibrium_ex(lbm_ctx* c, const void* rho, const void* u, int dtype) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!valid_dtype(dtype)) return fail(LBM_EINVAL, "dtype must be LBM_DTYPE_F32 or LBM_DTYPE_F64");
  int rc;
  if ((rc = check_ptr(c, rho, "rho")) != LBM_OK) return rc;
  if ((rc = check_ptr(c, u, "u")) != LBM_OK) return rc;
  const size_t es = dsize(dtype);
  const size_t bytes = (size_t)c->N * es;
  // page-locked host fields are read by the kernel in place; other memory is staged on the device
  const void* src_rho = mapped_host(rho);
  const void* src_u = mapped_host(u);
  if (!src_rho || !src_u) {
    CK(c->stage.ensure(4 * bytes));
    CK(cudaMemcpyAsync(c->stage.p, rho, bytes, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(static_cast<char*>(c->stage.p) + bytes, u, 3 * bytes, cudaMemcpyDefault, c->stream));
    src_rho = c->stage.p;
    src_u = static_cast<char*>(c->stage.p) + bytes;
  }
  c->t = 0;
  c->adj_t0 = -1;
  Args a = make_args(c);
  c->ops->init_eq(a, src_rho, src_u, dtype, c->stream);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(c->status.p, 0, sizeof(unsigned), c->stream));
  c->status_seen = 0;
  if ((rc = fill_refs(c)) != LBM_OK) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}
int lbm_init_equilibrium(lbm_ctx* c, const float* rho, const float* u) {
  return lbm_init_equilibrium_ex(c, rho, u, LBM_DTYPE_F32);
}

int lbm_step(lbm_ctx* c, int n) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (n < 0) return fail(LBM_EINVAL, "n must be >= 0");
  for (int s = 0; s < n; ++s) launch_step(c);
  CK(cudaGetLastError());
  return status_code(c);
}

int lbm_step_timed(lbm_ctx* c, int n, double ms[3]) {
  if (!c || !ms) return fail(LBM_EINVAL, "null argument");
  if (n < 1) return fail(LBM_EINVAL, "n must be >= 1");
  std::vector<cudaEvent_t> ev(4 * (size_t)n);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (int s = 0; s < n; ++s) {
    CK(cudaEventRecord(ev[4 * s], c->stream));
    launch_step(c, ev[4 * s + 1], ev[4 * s + 2]);
    CK(cudaEventRecord(ev[4 * s + 3], c->stream));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  for (int s = 0; s < n; ++s) {
    float all = 0, bulk = 0;
    CK(cudaEventElapsedTime(&all, ev[4 * s], ev[4 * s + 3]));
    CK(cudaEventElapsedTime(&bulk, ev[4 * s + 1], ev[4 * s + 2]));
    ms[0] += bulk;
    ms[1] += all - bulk;
  }
  float tot = 0;
  CK(cudaEventElapsedTime(&tot, ev[0], ev[4 * (size_t)n - 1]));
  ms[2] += tot;
  for (auto& e : ev) cudaEventDestroy(e);
  int rc = read_status(c);
  if (rc != LBM_OK) return rc;
  return status_code(c);
}

int lbm_sync(lbm_ctx* c) {
  if (!c) return fail(LBM_EINVAL, "null context");
  int rc = read_status(c);
  if (rc != LBM_OK) return rc;
  return status_code(c);
}

int lbm_moments_ex(lbm_ctx* c, void* rho, void* u, int dtype) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!valid_dtype(dtype)) return fail(LBM_EINVAL, "dtype must be LBM_DTYPE_F32 or LBM_DTYPE_F64");
  int rc;
  if ((rc = check_ptr(c, rho, "rho")) != LBM_OK) return rc;
  if ((rc = check_ptr(c, u, "u")) != LBM_OK) return rc;
  const size_t bytes = (size_t)c->N * dsize(dtype);
  Args a = make_args(c);
  const int sw = int(c->t & 1);
  const bool dev = is_device_ptr(rho, c->device) && is_device_ptr(u, c->device);
  void* mrho = mapped_host(rho);
  void* mu = mapped_host(u);
  if (dev) {
    c->ops->moments(a, sw, rho, u, dtype, c->stream);
    CK(cudaGetLastError());
  } else if (mrho && mu) {
    // page-locked host fields: the kernel writes them in place
    c->ops->moments(a, sw, mrho, mu, dtype, c->stream);
    CK(cudaGetLastError());
  } else {
    CK(c->stage.ensure(4 * bytes));
    c->ops->moments(a, sw, c->stage.p, static_cast<char*>(c->stage.p) + bytes, dtype, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(rho, c->stage.p, bytes, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(u, static_cast<char*>(c->stage.p) + bytes, 3 * bytes, cudaMemcpyDefault, c->stream));
  }
  if ((rc = read_status(c)) != LBM_OK) return rc;
  return status_code(c);
}
int lbm_moments(lbm_ctx* c, float* rho, float* u) { return lbm_moments_ex(c, rho, u, LBM_DTYPE_F32); }

int lbm_reduce(lbm_ctx* c, double* mass, double mom[3]) {
  if (!c || !mass || !mom) return fail(LBM_EINVAL, "null argument");
  Args a = make_args(c);
  c->ops->reduce(a, int(c->t & 1), static_cast<double*>(c->red.p), RED_BLOCKS, c->stream);
  reduce_final(static_cast<const double*>(c->red.p), RED_BLOCKS, static_cast<double*>(c->redout.p), c->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->red_h, c->redout.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  int rc = read_status(c);
  if (rc != LBM_OK) return rc;
  *mass = c->red_h[0];
  mom[0] = c->red_h[1]; mom[1] = c->red_h[2]; mom[2] = c->red_h[3];
  return status_code(c);
}

int lbm_get_populations(lbm_ctx* c, void* f, int dtype) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!valid_dtype(dtype)) return fail(LBM_EINVAL, "dtype must be LBM_DTYPE_F32 or LBM_DTYPE_F64");
  int rc;
  if ((rc = check_ptr(c, f, "f")) != LBM_OK) return rc;
  const size_t bytes = (size_t)c->q * c->N * dsize(dtype);
  Args a = make_args(c);
  if (is_device_ptr(f, c->device)) {
    c->ops->get_pops(a, int(c->t & 1), f, dtype, c->stream);
    CK(cudaGetLastError());
  } else {
    CK(c->stage.ensure(bytes));
    c->ops->get_pops(a, int(c->t & 1), c->stage.p, dtype, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(f, c->stage.p, bytes, cudaMemcpyDefault, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const void* f, int dtype) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!valid_dtype(dtype)) return fail(LBM_EINVAL, "dtype must be LBM_DTYPE_F32 or LBM_DTYPE_F64");
  int rc;
  if ((rc = check_ptr(c, f, "f")) != LBM_OK) return rc;
  const size_t bytes = (size_t)c->q * c->N * dsize(dtype);
  CK(c->stage.ensure(bytes));
  CK(cudaMemcpyAsync(c->stage.p, f, bytes, cudaMemcpyDefault, c->stream));
  Args a = make_args(c);
  c->ops->set_pops(a, int(c->t & 1), c->stage.p, dtype, c->stream);
  CK(cudaGetLastError());
  c->adj_t0 = -1;
  if ((rc = fill_refs(c)) != LBM_OK) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_set_option(lbm_ctx* c, int option, int value) {
  if (!c) return fail(LBM_EINVAL, "null context");
  switch (option) {
    case LBM_OPT_KERNEL:
      if (value != 0 && value != 2) return fail(LBM_EINVAL, "LBM_OPT_KERNEL takes 0 (plain) or 2 (staged)");
      c->kernel = value;
      return LBM_OK;
    case LBM_OPT_DEBUG_STALL:
      if (value != 0 && value != 1) return fail(LBM_EINVAL, "LBM_OPT_DEBUG_STALL takes 0 or 1");
      c->debug_stall = value;
      return LBM_OK;
  }
  return fail(LBM_EINVAL, "unknown option %d", option);
}

int lbm_interior_kernel(lbm_ctx* c) {
  if (!c) {
    fail(LBM_EINVAL, "null context");
    return -1;
  }
  if (c->kernel == 2) return 2;
  if (!pairs_selected(c)) return 0;
  const bool quads = (c->storage == LBM_F16 || c->storage == LBM_BF16) && c->q == 19 && c->model == LBM_BGK &&
                     c->nx % 4 == 0;
  return quads ? 3 : 1;
}

int lbm_launch_count(lbm_ctx* c, int64_t* n) {
  if (!c || !n) return fail(LBM_EINVAL, "null argument");
  *n = c->launches;
  return LBM_OK;
}

int lbm_info(lbm_ctx* c, int64_t out[10]) {
  if (!c || !out) return fail(LBM_EINVAL, "null argument");
  out[0] = c->N; out[1] = c->n_list; out[2] = c->counts[0]; out[3] = c->counts[1]; out[4] = c->counts[2];
  out[5] = c->counts[3]; out[6] = c->counts[4]; out[7] = c->t; out[8] = c->storage; out[9] = c->q;
  return LBM_OK;
}

int lbm_debug_dump(lbm_ctx* c, int which, int64_t* out, size_t count) {
  if (!c || !out) return fail(LBM_EINVAL, "null argument");
  CK(cudaStreamSynchronize(c->stream));
  size_t need = 0;
  switch (which) {
    case 0: need = c->N; break;
    case 1: case 2: need = c->n_list; break;
    case 3: need = 3 * (size_t)c->n_list; break;
    case 4: case 5: need = (size_t)c->q * c->N; break;
    default:
      if (which < 6 || which > 13) return fail(LBM_EINVAL, "which must be 0..13");
      need = c->halo_map[(which - 6) / 4][(which - 6) % 4].size();
  }
  if (count < need) return fail(LBM_EINVAL, "output holds %zu values, %zu needed", count, need);
  if (which == 0) {
    const std::vector<uint8_t>& th = host_types(c);
    for (long long n = 0; n < c->N; ++n) out[n] = th[n];
    return LBM_OK;
  }
  if (which == 1) {
    std::vector<long long> v(need);
    if (need) CK(cudaMemcpy(v.data(), c->lcell.p, need * sizeof(long long), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < need; ++i) out[i] = v[i];
    return LBM_OK;
  }
  if (which >= 6) {
    const std::vector<int64_t>& m = c->halo_map[(which - 6) / 4][(which - 6) % 4];
    for (size_t i = 0; i < need; ++i) out[i] = m[i];
    return LBM_OK;
  }
  if (which == 2 || which == 3) {
    std::vector<int> v(need);
    if (need) CK(cudaMemcpy(v.data(), which == 2 ? c->wref.p : c->nsum.p, need * sizeof(int), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < need; ++i) out[i] = v[i];
    return LBM_OK;
  }
  DevBuf tmp;
  CK(tmp.ensure(2 * need * sizeof(int64_t)));
  geo_source_map(geo_args(c), static_cast<const uint8_t*>(c->type.p), static_cast<int64_t*>(tmp.p),
                 static_cast<int64_t*>(tmp.p) + need, c->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, static_cast<int64_t*>(tmp.p) + (which == 4 ? 0 : need), need * sizeof(int64_t),
                     cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  tmp.release();
  return LBM_OK;
}

int lbm_save(lbm_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return fail(LBM_EINVAL, "null argument");
  const size_t fb = (size_t)c->q * c->stride * c->ops->elem;
  const size_t rb = std::max<size_t>(1, (size_t)c->n_list) * 3 * c->ops->celem;
  const size_t ub = c->model == LBM_HRR ? 3 * (size_t)c->N * c->ops->celem : 0;
  const size_t vb = c->vm_n > 0 ? 3 * (size_t)c->ny * c->nz * c->ops->celem : 0;
  const size_t total = sizeof(SaveHeader) + fb + 2 * rb + ub + vb;
  if (!buf) {
    *len = total;
    return LBM_OK;
  }
  if (*len < total) return fail(LBM_EINVAL, "buffer holds %zu bytes, %zu needed", *len, total);
  if (ub && c->uvel_stale) {
    int rc = fill_uvel(c);
    if (rc != LBM_OK) return rc;
  }
  SaveHeader h{};
  h.magic = SAVE_MAGIC; h.q = c->q; h.storage = c->storage; h.model = c->model;
  h.nx = c->nx; h.ny = c->ny; h.nz = c->nz; h.n_list = c->n_list; h.t = c->t;
  h.fbytes = fb; h.rbytes = rb; h.ubytes = ub; h.sigma = c->sigma; h.vbytes = vb;
  char* p = static_cast<char*>(buf);
  std::memcpy(p, &h, sizeof(h));
  CK(cudaMemcpyAsync(p + sizeof(h), c->f.p, fb, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(p + sizeof(h) + fb, c->ref0.p, rb, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(p + sizeof(h) + fb + rb, c->ref1.p, rb, cudaMemcpyDefault, c->stream));
  if (ub) {
    const void* src = (c->t & 1) ? c->uvel1.p : c->uvel0.p;
    CK(cudaMemcpyAsync(p + sizeof(h) + fb + 2 * rb, src, ub, cudaMemcpyDefault, c->stream));
  }
  if (vb) {
    const void* src = c->vm_which == 0 ? c->uin_a.p : c->uin_b.p;
    CK(cudaMemcpyAsync(p + sizeof(h) + fb + 2 * rb + ub, src, vb, cudaMemcpyDefault, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  *len = total;
  return LBM_OK;
}

int lbm_load(lbm_ctx* c, const void* buf, size_t len) {
  if (!c || !buf) return fail(LBM_EINVAL, "null argument");
  if (len < sizeof(SaveHeader)) return fail(LBM_EINVAL, "buffer too short");
  SaveHeader h;
  std::memcpy(&h, buf, sizeof(h));
  const size_t fb = (size_t)c->q * c->stride * c->ops->elem;
  const size_t rb = std::max<size_t>(1, (size_t)c->n_list) * 3 * c->ops->celem;
  const size_t ub = c->model == LBM_HRR ? 3 * (size_t)c->N * c->ops->celem : 0;
  const size_t vb = c->vm_n > 0 ? 3 * (size_t)c->ny * c->nz * c->ops->celem : 0;
  if (h.magic != SAVE_MAGIC || int(h.q) != c->q || int(h.storage) != c->storage || h.nx != c->nx || h.ny != c->ny ||
      h.nz != c->nz || h.n_list != c->n_list || h.fbytes != fb || h.rbytes != rb || int(h.model) != c->model ||
      h.ubytes != ub || h.vbytes != vb || len < sizeof(h) + fb + 2 * rb + ub + vb)
    return fail(LBM_EINVAL, "checkpoint does not match this context (lattice, size, storage, geometry or collision model)");
  const char* p = static_cast<const char*>(buf);
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpyAsync(c->f.p, p + sizeof(h), fb, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(c->ref0.p, p + sizeof(h) + fb, rb, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(c->ref1.p, p + sizeof(h) + fb + rb, rb, cudaMemcpyDefault, c->stream));
  c->t = h.t;
  if (ub) {
    CK(c->uvel0.ensure(ub));
    CK(c->uvel1.ensure(ub));
    void* dst = (c->t & 1) ? c->uvel1.p : c->uvel0.p;
    CK(cudaMemcpyAsync(dst, p + sizeof(h) + fb + 2 * rb, ub, cudaMemcpyDefault, c->stream));
    c->uvel_stale = false;
  }
  if (vb) {
    int rc = vm_reset(c);
    if (rc != LBM_OK) return rc;
    CK(cudaMemcpyAsync(c->uin_a.p, p + sizeof(h) + fb + 2 * rb + ub, vb, cudaMemcpyDefault, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  c->adj_t0 = -1;
  return LBM_OK;
}

// Vortex-method inlet: n vortices per step (0 switches it off), vortex size sigma (cells), turbulence
// intensity, random-number seed.
int lbm_set_vortex_inlet(lbm_ctx* c, int n, double sigma, double intensity, unsigned long long seed) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (n < 0 || n > (1 << 20)) return fail(LBM_EINVAL, "n must lie in [0, 2^20]");
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(LBM_EINVAL, "sigma must be > 0");
  if (!(intensity >= 0.0) || !std::isfinite(intensity)) return fail(LBM_EINVAL, "intensity must be >= 0");
  if (n > 0 && (c->gh_lo || c->gh_hi)) return fail(LBM_ESTATE, "slab sub-domains run with a steady inlet");
  c->vm_n = n; c->vm_sigma = sigma; c->vm_I = intensity; c->vm_seed = seed;
  if (n == 0) {
    c->uin_a.release(); c->uin_b.release(); c->vort.release(); c->vpart.release();
    return LBM_OK;
  }
  int rc = vm_reset(c);
  if (rc != LBM_OK) return rc;
  CK(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

// Collision model: LBM_BGK, or LBM_HRR with hybridisation factor sigma in [0, 1].
int lbm_set_collision(lbm_ctx* c, int model, double sigma) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (model != LBM_BGK && model != LBM_HRR) return fail(LBM_EINVAL, "model must be LBM_BGK or LBM_HRR");
  if (model != LBM_BGK && (c->gh_lo || c->gh_hi)) return fail(LBM_ESTATE, "slab sub-domains run the BGK collision");
  if (!(sigma >= 0.0 && sigma <= 1.0)) return fail(LBM_EINVAL, "sigma must lie in [0, 1]");
  c->model = model;
  c->sigma = sigma;
  c->uvel_stale = true;
  if (model == LBM_BGK) {
    c->uvel0.release();
    c->uvel1.release();
  }
  return LBM_OK;
}

// ---- adjoint ---------------------------------------------------------------------------------------------
static int adj_check(lbm_ctx* c, int xa, int xb, double* wa, double* wb, int W) {
  if (c->model != LBM_BGK) return fail(LBM_ESTATE, "the adjoint is defined for the BGK collision only");
  if (c->fr_L > 0) return fail(LBM_ESTATE, "the adjoint is defined without the outlet fringe zone");
  if (c->gh_lo || c->gh_hi) return fail(LBM_ESTATE, "the adjoint is defined on a whole domain, not a slab sub-domain");
  if (c->vm_n > 0) return fail(LBM_ESTATE, "the adjoint is defined for a steady inlet only");
  if (c->wm) return fail(LBM_ESTATE, "the wall model is not differentiated; switch it off (kappa <= 0)");
  if (xa < 0 || xa >= c->nx || xb < 0 || xb >= c->nx || xa == xb) return fail(LBM_EINVAL, "objective planes out of range");
  long long na = 0, nb = 0;
  const std::vector<uint8_t>& th = host_types(c);
  for (long long n = 0; n < c->N; ++n) {
    const int x = int(n % c->nx);
    if (x != xa && x != xb) continue;
    const int k = th[n] & T_KIND;
    if (k == K_SOLID) continue;
    if (k == K_INFLOW || k == K_OUTFLOW) return fail(LBM_EINVAL, "objective plane x=%d holds boundary cells", x);
    (x == xa ? na : nb)++;
  }
  if (na == 0 || nb == 0) return fail(LBM_EINVAL, "objective plane without fluid cells");
  *wa = (1.0 / 3.0) / (double(W) * na);
  *wb = -(1.0 / 3.0) / (double(W) * nb);
  return LBM_OK;
}

int lbm_objective_forward(lbm_ctx* c, int T, int W, int xa, int xb, int ckpt, double* J) {
  if (!c || !J) return fail(LBM_EINVAL, "null argument");
  if (T < 1 || W < 1 || W > T) return fail(LBM_EINVAL, "need 1 <= W <= T");
  if (!(ckpt == 1 || (ckpt >= 2 && !(ckpt & 1))))
    return fail(LBM_EINVAL, "checkpoint interval must be 1 (every state) or even and >= 2");
  if (ckpt == 1 && (T & 1)) return fail(LBM_EINVAL, "keeping every state needs an even T");
  if (c->t & 1) return fail(LBM_ESTATE, "the forward run must start after an even number of steps");
  double wa, wb;
  int rc = adj_check(c, xa, xb, &wa, &wb, W);
  if (rc != LBM_OK) return rc;
  if (ckpt == 1) {
    // Every state kept in HBM (T + 1 states of q * stride values): the forward steps out of place
    // from state s into state s + 1 (the same one read and one write per population as the in-place
    // step), and the backward runs the reverse sweep alone, with no recomputation.
    const size_t sb1 = (size_t)c->q * c->stride * c->ops->elem;
    cudaError_t e = c->hist.ensure((size_t)(T + 1) * sb1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->hist.release();
      return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "state history (%zu bytes): %s",
                  (size_t)(T + 1) * sb1, cudaGetErrorString(e));
    }
    char* H = static_cast<char*>(c->hist.p);
    CK(cudaMemsetAsync(c->redout.p, 0, sizeof(double), c->stream));
    const size_t plane_blocks1 = (2 * (size_t)c->ny * c->nz + 255) / 256;
    CK(c->plane.ensure(plane_blocks1 * sizeof(double)));
    cudaEvent_t f0, f1;
    CK(cudaEventCreate(&f0));
    CK(cudaEventCreate(&f1));
    CK(cudaEventRecord(f0, c->stream));
    CK(cudaMemcpyAsync(H, c->f.p, sb1, cudaMemcpyDeviceToDevice, c->stream));  // even t: natural layout
    const Args a = make_args(c);
    for (int s1 = 0; s1 < T; ++s1) {
      c->ops->step_oop(a, H + (size_t)s1 * sb1, H + (size_t)(s1 + 1) * sb1, c->stream);
      ++c->launches;
      if (s1 + 1 > T - W)
        c->ops->plane_rho(a, H + (size_t)(s1 + 1) * sb1, 0, xa, xb, static_cast<double*>(c->redout.p),
                          static_cast<double*>(c->plane.p), wa, wb, c->stream);
    }
    // T even: the final state in the natural layout is the in-place layout after an even count
    CK(cudaMemcpyAsync(c->f.p, H + (size_t)T * sb1, sb1, cudaMemcpyDeviceToDevice, c->stream));
    c->t += T;
    CK(cudaEventRecord(f1, c->stream));
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->red_h, c->redout.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((rc = read_status(c)) != LBM_OK) return rc;
    float fms = 0;
    CK(cudaEventElapsedTime(&fms, f0, f1));
    c->adj_ms[2] = fms;
    cudaEventDestroy(f0);
    cudaEventDestroy(f1);
    *J = c->red_h[0];
    c->adj_T = T; c->adj_W = W; c->adj_xa = xa; c->adj_xb = xb; c->adj_ck = 1;
    c->adj_wa = wa; c->adj_wb = wb;
    c->adj_t0 = c->t;
    return status_code(c);
  }
  const int nck = (T + ckpt - 1) / ckpt;
  const size_t sb = (size_t)c->q * c->stride * c->ops->elem;
  if ((int)c->ckpts.size() < nck) c->ckpts.resize(nck);
  for (int k = 0; k < nck; ++k) {
    cudaError_t e = c->ckpts[k].ensure(sb);
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "checkpoints: %s", cudaGetErrorString(e));
  }
  CK(cudaMemsetAsync(c->redout.p, 0, sizeof(double), c->stream));
  const size_t plane_blocks = (2 * (size_t)c->ny * c->nz + 255) / 256;
  CK(c->plane.ensure(plane_blocks * sizeof(double)));
  cudaEvent_t f0, f1;
  CK(cudaEventCreate(&f0));
  CK(cudaEventCreate(&f1));
  CK(cudaEventRecord(f0, c->stream));
  for (int s = 0; s < T; ++s) {
    if (s % ckpt == 0) CK(cudaMemcpyAsync(c->ckpts[s / ckpt].p, c->f.p, sb, cudaMemcpyDeviceToDevice, c->stream));
    launch_step(c);
    if (s + 1 > T - W) {
      const Args b = make_args(c);
      c->ops->plane_rho(b, c->f.p, int(c->t & 1), xa, xb, static_cast<double*>(c->redout.p),
                        static_cast<double*>(c->plane.p), wa, wb, c->stream);
    }
  }
  CK(cudaEventRecord(f1, c->stream));
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->red_h, c->redout.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if ((rc = read_status(c)) != LBM_OK) return rc;
  float fms = 0;
  CK(cudaEventElapsedTime(&fms, f0, f1));
  c->adj_ms[2] = fms;
  cudaEventDestroy(f0);
  cudaEventDestroy(f1);
  *J = c->red_h[0];
  c->adj_T = T; c->adj_W = W; c->adj_xa = xa; c->adj_xb = xb; c->adj_ck = ckpt;
  c->adj_wa = wa; c->adj_wb = wb;
  c->adj_t0 = c->t;
  return status_code(c);
}

int lbm_objective_backward(lbm_ctx* c, double* dJ_dgamma, double* dJ_duin) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (c->adj_t0 != c->t) return fail(LBM_ESTATE, "no forward run to differentiate (run lbm_objective_forward first)");
  if (c->fr_L > 0) return fail(LBM_ESTATE, "the adjoint is defined without the outlet fringe zone");
  if (c->gh_lo || c->gh_hi) return fail(LBM_ESTATE, "the adjoint is defined on a whole domain, not a slab sub-domain");
  if (c->model != LBM_BGK) return fail(LBM_ESTATE, "the adjoint is defined for the BGK collision only");
  if (c->vm_n > 0) return fail(LBM_ESTATE, "the adjoint is defined for a steady inlet only");
  if (c->wm) return fail(LBM_ESTATE, "the wall model is not differentiated");
  int rc0;
  if (dJ_dgamma && (rc0 = check_ptr(c, dJ_dgamma, "dJ_dgamma")) != LBM_OK) return rc0;
  if (dJ_duin && (rc0 = check_ptr(c, dJ_duin, "dJ_duin")) != LBM_OK) return rc0;
  const int T = c->adj_T, W = c->adj_W, ck = c->adj_ck;
  const bool keep_all = ck == 1;  // every state kept by the forward run: one segment, no recomputation
  const int seg_len = keep_all ? T : ck;
  const int nck = (T + seg_len - 1) / seg_len;
  const size_t sb = (size_t)c->q * c->stride * c->ops->elem;
  const size_t lb = (size_t)c->q * c->stride * c->ops->celem;
  const size_t pl = 3 * (size_t)c->ny * c->nz;
  if (!keep_all && (int)c->ring.size() < ck) c->ring.resize(ck);
  for (int k = 1; !keep_all && k < ck; ++k) {
    cudaError_t e = c->ring[k].ensure(sb);
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "ring: %s", cudaGetErrorString(e));
  }
  CK(c->lamA.ensure(lb));
  CK(c->lamB.ensure(lb));
  CK(c->dgam.ensure((size_t)c->N * sizeof(double)));
  CK(c->duin.ensure(pl * sizeof(double)));
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(c->dgam.p, 0, (size_t)c->N * sizeof(double), s));
  CK(cudaMemsetAsync(c->duin.p, 0, pl * sizeof(double), s));
  Args a = make_args(c);
  c->ops->seed(a, c->lamA.p, c->adj_xa, c->adj_xb, c->adj_wa, c->adj_wb, s);
  void* lin = c->lamA.p;
  void* lout = c->lamB.p;
  cudaEvent_t e0, e1, e2;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventCreate(&e2));
  float rec_ms = 0, rev_ms = 0;
  for (int seg = nck - 1; seg >= 0; --seg) {
    const int t0 = seg * seg_len;
    const int L = std::min(T, t0 + seg_len) - t0;
    std::vector<const void*> st(L);
    CK(cudaEventRecord(e0, s));
    if (keep_all) {
      for (int j = 0; j < L; ++j) st[j] = static_cast<const char*>(c->hist.p) + (size_t)j * sb;
    } else {
      st[0] = c->ckpts[seg].p;
      for (int j = 1; j < L; ++j) {
        c->ops->step_oop(a, st[j - 1], c->ring[j].p, s);
        st[j] = c->ring[j].p;
      }
    }
    CK(cudaEventRecord(e1, s));
    for (int j = L - 1; j >= 0; --j) {
      const int t = t0 + j;
      AdjArgs d{};
      d.fst = st[j];
      d.lam_in = lin;
      d.lam_out = lout;
      d.dgam = static_cast<double*>(c->dgam.p);
      d.duin = static_cast<double*>(c->duin.p);
      d.add_dj = (t > T - W) ? 1 : 0;
      d.xa = c->adj_xa; d.xb = c->adj_xb; d.wa = c->adj_wa; d.wb = c->adj_wb;
      c->ops->reverse(a, d, s);
      std::swap(lin, lout);
    }
    CK(cudaEventRecord(e2, s));
    CK(cudaEventSynchronize(e2));
    float m0 = 0, m1 = 0;
    CK(cudaEventElapsedTime(&m0, e0, e1));
    CK(cudaEventElapsedTime(&m1, e1, e2));
    rec_ms += m0;
    rev_ms += m1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  CK(cudaGetLastError());
  c->adj_ms[0] = keep_all ? 0.0 : rec_ms;  // nothing is recomputed when every state was kept
  c->adj_ms[1] = keep_all ? rev_ms + rec_ms : rev_ms;
  // the FP64 accumulators go to the caller's arrays as they are (host or device memory)
  if (dJ_dgamma) CK(cudaMemcpyAsync(dJ_dgamma, c->dgam.p, (size_t)c->N * sizeof(double), cudaMemcpyDefault, s));
  if (dJ_duin) CK(cudaMemcpyAsync(dJ_duin, c->duin.p, pl * sizeof(double), cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  int rc = read_status(c);
  if (rc != LBM_OK) return rc;
  return status_code(c);
}

int lbm_adjoint_step(lbm_ctx* c, const void* lam_in, void* lam_out, int dtype, double* dgamma, double* duin) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!valid_dtype(dtype)) return fail(LBM_EINVAL, "dtype must be LBM_DTYPE_F32 or LBM_DTYPE_F64");
  if (c->model != LBM_BGK) return fail(LBM_ESTATE, "the adjoint is defined for the BGK collision only");
  if (c->vm_n > 0) return fail(LBM_ESTATE, "the adjoint is defined for a steady inlet only");
  if (c->wm) return fail(LBM_ESTATE, "the wall model is not differentiated");
  if (c->t & 1) return fail(LBM_ESTATE, "the reverse step needs the state after an even number of steps");
  if (c->fr_L > 0) return fail(LBM_ESTATE, "the adjoint is defined without the outlet fringe zone");
  if (c->gh_lo || c->gh_hi) return fail(LBM_ESTATE, "the adjoint is defined on a whole domain, not a slab sub-domain");
  int rc;
  if ((rc = check_ptr(c, lam_in, "lam_in")) != LBM_OK) return rc;
  if ((rc = check_ptr(c, lam_out, "lam_out")) != LBM_OK) return rc;
  if (dgamma && (rc = check_ptr(c, dgamma, "dgamma")) != LBM_OK) return rc;
  if (duin && (rc = check_ptr(c, duin, "duin")) != LBM_OK) return rc;
  const size_t cnt = (size_t)c->q * c->N;
  const size_t lb = (size_t)c->q * c->stride * c->ops->celem;
  const size_t pl = 3 * (size_t)c->ny * c->nz;
  const int cd = c->ops->celem == 8 ? LBM_DTYPE_F64 : LBM_DTYPE_F32;
  cudaStream_t s = c->stream;
  CK(c->lamA.ensure(lb));
  CK(c->lamB.ensure(lb));
  CK(c->dgam.ensure((size_t)c->N * sizeof(double)));
  CK(c->duin.ensure(pl * sizeof(double)));
  CK(cudaMemsetAsync(c->dgam.p, 0, (size_t)c->N * sizeof(double), s));
  CK(cudaMemsetAsync(c->duin.p, 0, pl * sizeof(double), s));
  // caller layout q*N -> padded q*stride
  CK(c->stage.ensure(cnt * 8));
  CK(cudaMemcpyAsync(c->stage.p, lam_in, cnt * dsize(dtype), cudaMemcpyDefault, s));
  for (int i = 0; i < c->q; ++i)
    c->ops->convert(static_cast<const char*>(c->stage.p) + (size_t)i * c->N * dsize(dtype), dtype,
                    static_cast<char*>(c->lamA.p) + (size_t)i * c->stride * c->ops->celem, cd, c->N, s);
  Args a = make_args(c);
  AdjArgs d{};
  d.fst = c->f.p;
  d.lam_in = c->lamA.p;
  d.lam_out = c->lamB.p;
  d.dgam = static_cast<double*>(c->dgam.p);
  d.duin = static_cast<double*>(c->duin.p);
  c->ops->reverse(a, d, s);
  for (int i = 0; i < c->q; ++i)
    c->ops->convert(static_cast<const char*>(c->lamB.p) + (size_t)i * c->stride * c->ops->celem, cd,
                    static_cast<char*>(c->stage.p) + (size_t)i * c->N * dsize(dtype), dtype, c->N, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(lam_out, c->stage.p, cnt * dsize(dtype), cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  if (dgamma) CK(cudaMemcpyAsync(dgamma, c->dgam.p, (size_t)c->N * sizeof(double), cudaMemcpyDefault, s));
  if (duin) CK(cudaMemcpyAsync(duin, c->duin.p, pl * sizeof(double), cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  return LBM_OK;
}

int lbm_adjoint_timing(lbm_ctx* c, double ms[3]) {
  if (!c || !ms) return fail(LBM_EINVAL, "null argument");
  ms[0] = c->adj_ms[0];
  ms[1] = c->adj_ms[1];
  ms[2] = c->adj_ms[2];
  return LBM_OK;
}

}  // extern "C"
