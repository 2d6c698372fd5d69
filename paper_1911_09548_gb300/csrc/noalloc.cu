// Allocation-free l2 norm of a device vector: a variant of the library's
// deterministic two-stage norm (the stopping test of the solver) whose scratch
// (one partial sum per block, plus the final sum) lives in a file-scope device
// array instead of memory the caller or a handle allocated.
//
// The array is a module global: every GPU that loads the library holds it
// (kNoAllocMaxBlocks + 1 doubles = 256 KiB + 8 B) until the process exits, and
// every call shares it.  Host code cannot use the array's name as a device
// address, so its address is fetched with cudaGetSymbolAddress once per device,
// on the first call made while that device is current.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/st_mg.h"
#include "device.h"

namespace stmg {
void set_last_error(const char* msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int64_t kPerBlock = (int64_t)kThreads * kPerThread;   // elements summed by one block
constexpr int64_t kNoAllocMaxBlocks = 32768;                    // scratch partial sums
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 1];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Block b sums v[b*kPerBlock, (b+1)*kPerBlock) in a fixed order into partial[b].
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(const double* __restrict__ v, int64_t n,
                                                              double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kPerBlock;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
    if (i < n) s = fma(v[i], v[i], s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// out[0] = sqrt(sum of partial[0..nb)) in a fixed order.
__global__ void __launch_bounds__(kThreads) k_noalloc_final(const double* __restrict__ partial, int nb,
                                                            double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += kThreads) s += partial[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    out[0] = sqrt(t);
  }
}

int noalloc_fail(int code, const char* msg) {
  stmg::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int st_mg_norm2_noalloc(const double* v_dev, int64_t n, void* stream, double* norm_dev) {
  if (!v_dev || !norm_dev || n < 0) return noalloc_fail(ST_MG_ERR_INVALID_ARG, "st_mg_norm2_noalloc: null pointer or n < 0");
  if ((reinterpret_cast<uintptr_t>(v_dev) & 7u) || (reinterpret_cast<uintptr_t>(norm_dev) & 7u))
    return noalloc_fail(ST_MG_ERR_INVALID_ARG, "st_mg_norm2_noalloc: pointers must be 8-byte aligned");
  const int64_t nb = (n + kPerBlock - 1) / kPerBlock;
  if (nb > kNoAllocMaxBlocks)
    return noalloc_fail(ST_MG_ERR_INVALID_ARG,
                        "st_mg_norm2_noalloc: n exceeds the maximum of 134217728 elements (fixed scratch size)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(ST_MG_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(ST_MG_ERR_INVALID_ARG, "st_mg_norm2_noalloc: device ordinal >= 64");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return noalloc_fail(ST_MG_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (nb > 0) {
    k_noalloc_partial<<<(unsigned)nb, kThreads, 0, st>>>(v_dev, n, scratch);
    stmg::count_launches(1);
  }
  // nb == 0: nothing was written, the final kernel sums zero partials and stores 0
  k_noalloc_final<<<1, kThreads, 0, st>>>(scratch, (int)nb, norm_dev);
  stmg::count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(ST_MG_ERR_CUDA, cudaGetErrorString(e));
  return ST_MG_OK;
}
