// Allocation-free statistics of one velocity component (fs_component_stats_noalloc).
//
// Who needs this: code that may not call cudaMalloc at all -- for example a
// host application whose device memory is owned by its own pool allocator
// and forbids outside allocations, or a monitoring hook inside a timed loop
// where an allocation's implicit device synchronisation is not allowed.
// Such callers cannot create an fs_grid (fs_create_grid allocates), so this
// entry point takes plain pointers and keeps its reduction scratch in a
// fixed, file-scope device array that exists from library load to process
// exit on every device that loads the library.
//
// It is the allocation-free counterpart of the kinetic-energy / max|u| part of
// fs_diagnostics, which accumulates into scratch owned by a grid.
#include <cuda_runtime.h>

#include <mutex>

#include "fs_internal.cuh"

namespace {

constexpr int kChunk = 8192;          // elements reduced by one CTA
constexpr int kMaxChunks = 4096;      // partial slots in the static scratch
constexpr int kThreads = 256;

// Two doubles per chunk: partial sum of 0.5 u^2 w and partial max |u|.  64 KiB.
static __device__ __align__(256) double g_noalloc_partials[2 * kMaxChunks];

// A symbol's device address belongs to a CUDA context, not to a device: the
// address is cached per device together with the context it was looked up in,
// and looked up again when another context is current on that device (a
// driver-API context, or the primary context re-created after
// cudaDeviceReset).
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct ScratchAddr {
  void* ctx;
  double* addr;
};
ScratchAddr g_partials_addr[kMaxDevices] = {};

typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn g_ctx_get_current = nullptr;   // the driver's cuCtxGetCurrent

template <typename T>
__global__ void chunk_stats_kernel(const T* __restrict__ u, long long n, int ex, int ey, double vol,
                                   const double* __restrict__ wy, double* __restrict__ partials) {
  __shared__ double ss[kThreads], sm[kThreads];
  const long long base = (long long)blockIdx.x * kChunk;
  const long long end = base + kChunk < n ? base + kChunk : n;
  double s = 0.0, m = 0.0;
  for (long long t = base + threadIdx.x; t < end; t += blockDim.x) {
    const double v = (double)u[t];
    double w = vol;
    if (wy) w *= wy[(int)((t / ex) % ey)];
    s += 0.5 * v * v * w;
    m = fmax(m, fabs(v));
  }
  ss[threadIdx.x] = s;
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ss[threadIdx.x] += ss[threadIdx.x + o];
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // every used slot is overwritten, so stale contents of a previous call never leak in
    partials[2 * blockIdx.x] = ss[0];
    partials[2 * blockIdx.x + 1] = sm[0];
  }
}

__global__ void finish_stats_kernel(const double* __restrict__ partials, int nchunks, double* __restrict__ out) {
  __shared__ double ss[kThreads], sm[kThreads];
  double s = 0.0, m = 0.0;
  for (int b = threadIdx.x; b < nchunks; b += blockDim.x) {
    s += partials[2 * b];
    m = fmax(m, partials[2 * b + 1]);
  }
  ss[threadIdx.x] = s;
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ss[threadIdx.x] += ss[threadIdx.x + o];
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = ss[0];
    out[1] = sm[0];
  }
}

// Device address of the static scratch in the current context, looked up once per
// (device, context).
int scratch_address(double** addr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fs::cuda_check(e, "fs_component_stats_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fs::set_error(FS_ERR_UNSUPPORTED, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_ctx_get_current) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fs::set_error(FS_ERR_CUDA, "fs_component_stats_noalloc: cuCtxGetCurrent not found");
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
  }
  void* ctx = nullptr;
  if (g_ctx_get_current(&ctx) != 0) ctx = nullptr;
  ScratchAddr& a = g_partials_addr[dev];
  if (!ctx || !a.addr || a.ctx != ctx) {
    // the lookup also makes the runtime's context current when none is yet
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return fs::cuda_check(e, "fs_component_stats_noalloc: cudaGetSymbolAddress");
    if (g_ctx_get_current(&ctx) != 0 || !ctx)
      return fs::set_error(FS_ERR_CUDA, "fs_component_stats_noalloc: no current CUDA context");
    a.ctx = ctx;
    a.addr = static_cast<double*>(p);
  }
  *addr = a.addr;
  return FS_OK;
}

}  // namespace

extern "C" int fs_component_stats_noalloc(const void* u, int precision, const int ext[3], double vol,
                                          const double* wy, double* out, void* stream) {
  if (!u || !ext || !out) return fs::set_error(FS_ERR_ARG, "fs_component_stats_noalloc: NULL argument");
  if (precision != FS_FP64 && precision != FS_MIXED)
    return fs::set_error(FS_ERR_ARG, "fs_component_stats_noalloc: unknown precision");
  if (ext[0] < 1 || ext[1] < 1 || ext[2] < 1)
    return fs::set_error(FS_ERR_ARG, "fs_component_stats_noalloc: extents must be >= 1");
  // the element count, checked against the scratch's capacity before each product
  constexpr long long kMaxElems = (long long)kChunk * kMaxChunks;
  long long n = ext[0];
  bool too_big = n > kMaxElems;
  if (!too_big) {
    n *= ext[1];
    too_big = n > kMaxElems;
  }
  if (!too_big) {
    n *= ext[2];
    too_big = n > kMaxElems;
  }
  if (too_big)
    return fs::set_error(FS_ERR_ARG, "fs_component_stats_noalloc: field has more than 33554432 elements "
                                     "(4096 chunks of 8192), the size of its fixed scratch");
  const long long nchunks = (n + kChunk - 1) / kChunk;
  double* partials = nullptr;
  int rc = scratch_address(&partials);
  if (rc != FS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == FS_MIXED)
    chunk_stats_kernel<float><<<(int)nchunks, kThreads, 0, s>>>((const float*)u, n, ext[0], ext[1], vol, wy, partials);
  else
    chunk_stats_kernel<double><<<(int)nchunks, kThreads, 0, s>>>((const double*)u, n, ext[0], ext[1], vol, wy,
                                                                 partials);
  finish_stats_kernel<<<1, kThreads, 0, s>>>(partials, (int)nchunks, out);
  return fs::cuda_check(cudaGetLastError(), "fs_component_stats_noalloc launch");
}
