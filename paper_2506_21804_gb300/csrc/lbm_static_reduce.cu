// Mass and momentum of a caller-owned population array with no allocation at all: the per-chunk
// partial sums live in a file-scope device array instead of memory obtained from cudaMalloc.
//
// Some callers cannot let a library allocate device memory: applications that hand all device
// memory to their own pool allocator and forbid other allocations, codes that run close to the
// memory limit (a cudaMalloc could fail exactly when a diagnostic is needed), and step loops that
// must not pay for an allocation between two time steps. This entry point serves them; the
// context-based lbm_reduce keeps its own scratch buffer.
//
// The static array is created when the library is loaded and every GPU that loads the library keeps
// it until the process exits. Its device address is looked up once per device (first call made on
// that device, with the device current) through cudaGetSymbolAddress; host code never passes the
// array's own name to a kernel, since in host code that name denotes a host-side stand-in. A
// cudaDeviceReset unloads the module and invalidates the cached address, so this entry point must
// not be used on a device after it has been reset.
// Every call shares the array: calls whose work overlaps on the GPU (other streams, other host
// threads) race on it. Each call overwrites every partial it later reads, so nothing has to be
// cleared between calls.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace {

constexpr long long kChunk = 65536;  // cells per partial sum (one CTA)
constexpr int kMaxChunks = LBM_REDUCE_STATIC_MAX_CELLS / 65536;
static_assert((long long)kMaxChunks * kChunk == LBM_REDUCE_STATIC_MAX_CELLS, "chunking");

// 4 partial sums (mass, momentum x, y, z) per chunk, then 4 for the result.
static __device__ __align__(256) double g_scratch[4 * kMaxChunks + 4];

std::mutex g_mu;
void* g_addr[256] = {nullptr};
thread_local std::string g_err_static;

template <int Q, class T>
__global__ void __launch_bounds__(256) k_static_partial(const T* __restrict__ f, const uint8_t* __restrict__ mask,
                                                        long long N, double* part) {
  const long long begin = blockIdx.x * kChunk;
  long long end = begin + kChunk;
  if (end > N) end = N;
  double s[4] = {0, 0, 0, 0};
  for (long long n = begin + threadIdx.x; n < end; n += blockDim.x) {
    if (mask && mask[n] == 1) continue;
    lbm::sfor<0, Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const double v = double(f[(long long)i * N + n]);
      s[0] += v;
      if constexpr (lbm::Lat<Q>::cx(i) != 0) s[1] += double(lbm::Lat<Q>::cx(i)) * v;
      if constexpr (lbm::Lat<Q>::cy(i) != 0) s[2] += double(lbm::Lat<Q>::cy(i)) * v;
      if constexpr (lbm::Lat<Q>::cz(i) != 0) s[3] += double(lbm::Lat<Q>::cz(i)) * v;
    });
  }
  __shared__ double sm[8][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
    for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_down_sync(0xffffffffu, s[c], o);
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 4; ++c) sm[threadIdx.x >> 5][c] = s[c];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; ++c) {
      double t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w][c];
      part[4 * (long long)blockIdx.x + c] = t;
    }
}

// Fixed-order sum of the partials (one thread), so results do not depend on scheduling.
__global__ void k_static_final(const double* part, int nchunks, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[4] = {0, 0, 0, 0};
  for (int b = 0; b < nchunks; ++b)
    for (int c = 0; c < 4; ++c) s[c] += part[4 * b + c];
  for (int c = 0; c < 4; ++c) out[c] = s[c];
}

// 1: device or managed memory of device `dev`; 2: device or managed memory of another device;
// 0: anything else (host memory, registered or not).
int pointer_kind(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return 0;
  return at.device == dev ? 1 : 2;
}

int fail_static(int code, const std::string& msg) {
  g_err_static = msg;
  return code;
}

}  // namespace

extern "C" const char* lbm_reduce_static_error(void) { return g_err_static.c_str(); }

extern "C" int lbm_reduce_static(int lattice, const void* f, int dtype, const uint8_t* mask, int64_t n_cells,
                                 double* out, void* stream) {
  if (lattice != 19 && lattice != 27) return fail_static(LBM_EINVAL, "lattice must be 19 or 27");
  if (dtype != LBM_DTYPE_F32 && dtype != LBM_DTYPE_F64) return fail_static(LBM_EINVAL, "dtype must be LBM_DTYPE_F32 or LBM_DTYPE_F64");
  if (!f || !out) return fail_static(LBM_EINVAL, "null pointer");
  if (n_cells < 1 || n_cells > LBM_REDUCE_STATIC_MAX_CELLS)
    return fail_static(LBM_EINVAL, "n_cells = " + std::to_string((long long)n_cells) + " outside 1.." +
                                       std::to_string((long long)LBM_REDUCE_STATIC_MAX_CELLS) +
                                       " (the static scratch holds one partial sum per 65536 cells)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_static(LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return fail_static(LBM_EINVAL, "device ordinal out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      e = cudaGetSymbolAddress(&g_addr[dev], g_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        return fail_static(LBM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    scratch = g_addr[dev];
  }
  // f and mask are read by the kernel, so they must be device-accessible memory of this device
  // (device or managed); out is written by the kernel when it is such memory, else it is host memory
  // and receives the result by a copy.
  const int kf = pointer_kind(f, dev);
  if (kf != 1) return fail_static(LBM_EINVAL, kf == 2 ? "f is device memory of another device" : "f must be device memory of the current device");
  if (mask) {
    const int km = pointer_kind(mask, dev);
    if (km != 1) return fail_static(LBM_EINVAL, km == 2 ? "mask is device memory of another device" : "mask must be device memory of the current device (or NULL)");
  }
  const int ko = pointer_kind(out, dev);
  if (ko == 2) return fail_static(LBM_EINVAL, "out is device memory of another device");
  const bool out_dev = ko == 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* part = static_cast<double*>(scratch);
  double* result = part + 4 * kMaxChunks;
  const int nchunks = int((n_cells + kChunk - 1) / kChunk);
  if (lattice == 19) {
    if (dtype == LBM_DTYPE_F64) k_static_partial<19, double><<<nchunks, 256, 0, s>>>(static_cast<const double*>(f), mask, n_cells, part);
    else k_static_partial<19, float><<<nchunks, 256, 0, s>>>(static_cast<const float*>(f), mask, n_cells, part);
  } else {
    if (dtype == LBM_DTYPE_F64) k_static_partial<27, double><<<nchunks, 256, 0, s>>>(static_cast<const double*>(f), mask, n_cells, part);
    else k_static_partial<27, float><<<nchunks, 256, 0, s>>>(static_cast<const float*>(f), mask, n_cells, part);
  }
  k_static_final<<<1, 32, 0, s>>>(part, nchunks, out_dev ? out : result);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_static(LBM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  if (!out_dev) {
    e = cudaMemcpyAsync(out, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_static(LBM_ECUDA, std::string("copy of the result: ") + cudaGetErrorString(e));
  }
  return LBM_OK;
}
