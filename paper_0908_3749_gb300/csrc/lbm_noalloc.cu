// lbm_noalloc.cu -- conservation totals of a population array without any
// device allocation (lbm_audit_noalloc in include/lbm.h).
//
// The reduction needs scratch for one partial sum per thread block and an
// arrival counter. Here that scratch is a file-scope __device__ array of
// fixed size, so the entry point never calls cudaMalloc: callers that cannot
// allocate device memory (an allocator-free embedding, a memory pool that is
// fully reserved, a real-time loop that must not allocate) can still audit a
// state. Every GPU that loads this library holds the array until the process
// exits. All calls share it: two calls whose kernels overlap on the GPU (on
// different streams or from different host threads) race on it and give wrong
// totals; issue them in one stream, one after another.
//
// Host code must not use the array's name as an address: in host code the
// symbol is a stand-in, not a device pointer. The device address is looked
// up once per device with cudaGetSymbolAddress, with that device current, on
// the first call made on it; make that first call before any stream capture
// that might include the entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "d2v16.cuh"

using namespace d2v16;

namespace {

constexpr int NA_X = 32, NA_Y = 8, NA_N = NA_X * NA_Y;

struct NoAllocScratch {
  double partial[LBM_NOALLOC_MAX_BLOCKS][4];
  unsigned int arrive;
};

__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__global__ void __launch_bounds__(NA_N) k_audit_noalloc(const R* __restrict__ f, int nx, int ny,
                                                        long long pitch, double area,
                                                        NoAllocScratch* sc, double* totals,
                                                        const Coeffs<double> K) {
  __shared__ double sm[NA_N / 32][4];
  __shared__ int s_last;
  const int x = blockIdx.x * NA_X + threadIdx.x;
  const int y = blockIdx.y * NA_Y + threadIdx.y;
  const int t = threadIdx.y * NA_X + threadIdx.x;
  const long long plane = pitch * ny;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (x < nx && y < ny) {
    const long long c = (long long)y * pitch + x;
    double g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = (double)f[i * plane + c];
    Groups<double> d;
    transform(g, d);
    const Cons<double> m = conserved(K, d);
    v[0] = m.rho; v[1] = m.jx; v[2] = m.jy; v[3] = m.e;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = na_warp_sum(v[k]);
  if ((t & 31) == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) sm[t >> 5][k] = v[k];
  __syncthreads();
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (t < 4) {
    double s = 0.0;
    for (int w = 0; w < NA_N / 32; ++w) s += sm[w][t];
    sc->partial[bid][t] = s;
  }
  __syncthreads();
  if (t == 0) {
    __threadfence();
    s_last = atomicAdd(&sc->arrive, 1u) == (unsigned)nblocks - 1;
  }
  __syncthreads();
  if (s_last && t < 32) {
    __threadfence();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double s = 0.0;
      for (int b = t; b < nblocks; b += 32) s += __ldcg(&sc->partial[b][k]);
      s = na_warp_sum(s);
      if (t == 0) totals[k] = s * area;
    }
    if (t == 0) sc->arrive = 0;
  }
}

// Device address of the scratch array, looked up once per device.
constexpr int MAX_DEVICES = 64;
NoAllocScratch* g_scratch_addr[MAX_DEVICES] = {};
std::mutex g_scratch_mutex;
thread_local std::string g_noalloc_error = "no error";

int na_fail(int code, const std::string& m) {
  g_noalloc_error = m;
  return code;
}

}  // namespace

extern "C" {

int lbm_audit_noalloc(const void* f, int precision, int nx, int ny, long long pitch,
                      double dx, double dy, double* totals, void* cuda_stream) {
  if (!f || !totals) return na_fail(LBM_ERR_INVALID, "lbm_audit_noalloc: NULL pointer");
  if (precision != LBM_FP64 && precision != LBM_FP32)
    return na_fail(LBM_ERR_INVALID, "lbm_audit_noalloc: precision must be LBM_FP64 or LBM_FP32");
  if (nx < 1 || ny < 1 || pitch < nx)
    return na_fail(LBM_ERR_INVALID, "lbm_audit_noalloc: need nx, ny >= 1 and pitch >= nx");
  if (!(std::isfinite(dx) && std::isfinite(dy)))
    return na_fail(LBM_ERR_INVALID, "lbm_audit_noalloc: dx, dy must be finite");
  const dim3 grid((nx + NA_X - 1) / NA_X, (ny + NA_Y - 1) / NA_Y);
  const long long nblocks = (long long)grid.x * grid.y;
  if (nblocks > LBM_NOALLOC_MAX_BLOCKS)
    return na_fail(LBM_ERR_INVALID,
                   "lbm_audit_noalloc: grid needs " + std::to_string(nblocks) +
                       " blocks of 32 x 8 nodes, more than the fixed scratch holds (" +
                       std::to_string(LBM_NOALLOC_MAX_BLOCKS) + ")");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return na_fail(LBM_ERR_UNSUPPORTED, "device ordinal too large");
  NoAllocScratch* sc = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return na_fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = (NoAllocScratch*)p;
    }
    sc = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // The arrival counter must start at zero whatever the last call left.
  e = cudaMemsetAsync(&sc->arrive, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return na_fail(LBM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  const double area = dx * dy;
  Coeffs<double> K;
  memset(&K, 0, sizeof(K));
  fill_forward(K);  // only the forward blocks are used by the totals
  if (precision == LBM_FP64)
    k_audit_noalloc<double><<<grid, dim3(NA_X, NA_Y), 0, s>>>((const double*)f, nx, ny, pitch,
                                                               area, sc, totals, K);
  else
    k_audit_noalloc<float><<<grid, dim3(NA_X, NA_Y), 0, s>>>((const float*)f, nx, ny, pitch,
                                                              area, sc, totals, K);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(LBM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return LBM_OK;
}

const char* lbm_audit_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

}  // extern "C"
