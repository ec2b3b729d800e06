// Allocation-free variant of the norm reduction (mw3_norms_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while an application's
// device memory is fixed up front (a pre-sized arena or memory pool shared with
// other work), code called from inside a region where allocation is forbidden or
// would stall other streams, or a host that must not take the driver's allocation
// lock. The regular norm kernels of the propagation write their per-chunk partial
// sums into a scratch buffer that the context allocates; this entry point instead
// keeps that scratch in a file-scope device array, so a call allocates nothing.
//
// The array (kNoAllocMaxSegments x kNoAllocChunks doubles = 128 KB) is created on
// every GPU that loads the library and stays there until the process exits. Host
// code cannot use the array's name as a device address: on the first call for a
// device, with that device current, its address is looked up with
// cudaGetSymbolAddress and cached together with the CUDA context that was current;
// a later call under another context (after cudaDeviceReset, or once the primary
// context was destroyed and made again) looks the address up anew. Make the first
// call of each context before any stream capture.
// Every call shares the one array and overwrites it completely (each chunk writes its
// own slot before the final pass reads it, so nothing has to start at zero); calls
// whose kernels overlap on the GPU (different streams, no ordering) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mw3.h"

namespace {

constexpr int kNoAllocMaxSegments = 64;
constexpr int kNoAllocChunks = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partial[kNoAllocMaxSegments * kNoAllocChunks];

// per device: the array's device address and the context it was looked up under
double* g_partial_addr[kMaxDevices] = {};
CUcontext g_partial_ctx[kMaxDevices] = {};
std::mutex g_partial_mu;

// the current CUDA context through the driver's entry point (the library does not link
// libcuda); nullptr when it cannot be had
CUcontext current_context() {
  using CtxGetFn = CUresult (*)(CUcontext*);
  static CtxGetFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetFn>(f);
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// partial[s][chunk] = sum of x^2 over a fixed contiguous chunk of segment s
__global__ void __launch_bounds__(256) k_segment_partial(const double* __restrict__ x,
                                                         long seg_len, double* __restrict__ partial) {
  __shared__ double red[256];
  const int s = blockIdx.y;
  const long per = (seg_len + kNoAllocChunks - 1) / kNoAllocChunks;
  const long a = per * blockIdx.x;
  const long z = (a + per < seg_len) ? a + per : seg_len;
  const double* xs = x + (long)s * seg_len;
  double acc = 0;
  for (long i = a + threadIdx.x; i < z; i += blockDim.x) acc += xs[i] * xs[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(long)s * kNoAllocChunks + blockIdx.x] = red[0];
}

// out[s] = ordered sum of the partials of segment s (deterministic)
__global__ void k_segment_final(const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  const int s = blockIdx.x;
  double acc = 0;
  for (int i = 0; i < kNoAllocChunks; ++i) acc += partial[(long)s * kNoAllocChunks + i];
  out[s] = acc;
}

}  // namespace

extern "C" int mw3_norms_noalloc(const double* x, long seg_len, int nseg, double* out, void* stream) {
  if (!x || !out || seg_len < 0) return MW3_ERR_BAD_ARG;
  if (nseg < 1 || nseg > kNoAllocMaxSegments) return MW3_ERR_BAD_ARG;  // scratch holds 64 segments
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MW3_ERR_CUDA;
  double* partial = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_partial_mu);
    // the symbol lookup below makes the device's primary context current if none is, so
    // the context is read after it
    if (g_partial_addr[dev]) {
      const CUcontext ctx = current_context();
      if (!ctx || ctx != g_partial_ctx[dev]) g_partial_addr[dev] = nullptr;
    }
    if (!g_partial_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) return MW3_ERR_CUDA;
      g_partial_addr[dev] = static_cast<double*>(p);
      g_partial_ctx[dev] = current_context();
    }
    partial = g_partial_addr[dev];
  }
  // each launch's own status: cudaLaunchKernel returns the status of this launch, so an
  // error left pending by earlier, unrelated work on the thread is neither reported as
  // this call's failure nor consumed here
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    void* args[] = {(void*)&x, (void*)&seg_len, (void*)&partial};
    if (cudaLaunchKernel((const void*)k_segment_partial, dim3(kNoAllocChunks, nseg), dim3(256),
                         args, 0, st) != cudaSuccess)
      return MW3_ERR_CUDA;
  }
  {
    const double* pc = partial;
    void* args[] = {(void*)&pc, (void*)&out};
    if (cudaLaunchKernel((const void*)k_segment_final, dim3(nseg), dim3(32), args, 0, st) !=
        cudaSuccess)
      return MW3_ERR_CUDA;
  }
  return MW3_OK;
}
