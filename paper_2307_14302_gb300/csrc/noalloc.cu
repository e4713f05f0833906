// noalloc.cu -- total water volume from caller-owned device arrays, without allocating.
//
// dgswe_volume reduces in library-allocated scratch memory.  This variant does the same
// two-pass FP64 reduction (Neumaier-compensated per thread, fixed-order merges, per-block
// partial sums, one final block) with its partials held in a file-scope device array instead,
// so a call never allocates or frees device memory.  That matters to callers that cannot call
// cudaMalloc/cudaFree: code whose device memory all comes from its own pool or caching
// allocator, and loops that must not stall on the implicit device synchronisation of cudaFree.
// The scratch array's device address is looked up once per device and kept; it is stale after a
// cudaDeviceReset of that device.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "dgswe.h"

namespace dg {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 16;
constexpr long long NA_CHUNK = (long long)NA_THREADS * NA_PER_THREAD;  // elements per block
constexpr int NA_MAX_PARTIALS = 4096;                                  // blocks per call
constexpr long long NA_MAX_ELEMENTS = NA_CHUNK * NA_MAX_PARTIALS;      // 16,777,216

// (sum, compensation) of each block of the current call; 64 KiB on every device that loads the
// library, for the life of the process.  Shared by all calls: overlapping calls race.
static __device__ __align__(256) double g_na_scratch[2 * NA_MAX_PARTIALS];

__device__ __forceinline__ void na_add(double& s, double& c, double v) {
  const double t = s + v;
  c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
  s = t;
}

// merge the (s, c) pairs of a warp in a fixed pattern
__device__ __forceinline__ void na_warp(double& s, double& c) {
  for (int o = 16; o > 0; o >>= 1) {
    const double s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
    na_add(s, c, s2);
    c += c2;
  }
}

__global__ void __launch_bounds__(NA_THREADS) na_partial(const double* w0, const double* area, long long n,
                                                         double* part) {
  const long long base = (long long)blockIdx.x * NA_CHUNK;
  double s = 0.0, c = 0.0;
  for (int k = 0; k < NA_PER_THREAD; ++k) {
    const long long i = base + (long long)k * NA_THREADS + threadIdx.x;
    if (i < n) na_add(s, c, area[i] * (w0[i] * 0.7071067811865476));  // mean = mode 0 / sqrt(2)
  }
  na_warp(s, c);
  __shared__ double sh[2][NA_THREADS / 32];
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = s;
    sh[1][threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NA_THREADS / 32; ++w) {
      na_add(s, c, sh[0][w]);
      c += sh[1][w];
    }
    part[2 * blockIdx.x] = s;  // every slot of this call is written before it is read
    part[2 * blockIdx.x + 1] = c;
  }
}

__global__ void __launch_bounds__(NA_THREADS) na_final(const double* part, int nb, double* out) {
  double s = 0.0, c = 0.0;
  for (int b = threadIdx.x; b < nb; b += NA_THREADS) {
    na_add(s, c, part[2 * b]);
    c += part[2 * b + 1];
  }
  na_warp(s, c);
  __shared__ double sh[2][NA_THREADS / 32];
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = s;
    sh[1][threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NA_THREADS / 32; ++w) {
      na_add(s, c, sh[0][w]);
      c += sh[1][w];
    }
    out[0] = s + c;
  }
}

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
double* g_na_ptr[NA_MAX_DEVICES] = {};

int na_fail(int code, const char* msg) {
  dg::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int dgswe_volume_sum_noalloc(const double* w0, const double* area, int64_t n, double* out,
                                        void* cuda_stream) {
  if (!w0 || !area || !out) return na_fail(DGSWE_EINVAL, "volume_sum_noalloc: null device pointer");
  if (n < 0 || n > NA_MAX_ELEMENTS) {
    char buf[160];
    snprintf(buf, sizeof buf, "volume_sum_noalloc: n = %lld is outside [0, %lld], the capacity of its fixed scratch",
             (long long)n, NA_MAX_ELEMENTS);
    return na_fail(DGSWE_EINVAL, buf);
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
    return na_fail(DGSWE_ECUDA, "volume_sum_noalloc: no current CUDA device");
  double* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the scratch array
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_na_scratch);
      if (e != cudaSuccess) {
        std::string m = std::string("volume_sum_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
        return na_fail(DGSWE_ECUDA, m.c_str());
      }
      g_na_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nb = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
  if (nb > 0) na_partial<<<nb, NA_THREADS, 0, s>>>(w0, area, (long long)n, scratch);
  na_final<<<1, NA_THREADS, 0, s>>>(scratch, nb, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::string m = std::string("volume_sum_noalloc: launch failed: ") + cudaGetErrorString(e);
    return na_fail(DGSWE_ECUDA, m.c_str());
  }
  return 0;
}
