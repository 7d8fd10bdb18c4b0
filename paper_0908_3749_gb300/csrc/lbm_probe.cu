// lbm_probe.cu -- measured fused multiply-add rates of the device
// (lbm_probe_fma_rate in include/lbm_probe.h): the denominators of the
// arithmetic rooflines of the FP64 step (FP64 units) and of the double-word
// step (FP32 units).
//
// Each thread runs 8 independent chains a <- a * b + c, enough independent
// work per warp to cover the units' latency; every multiprocessor runs 8
// blocks of 8 warps. The chains' final values are compared with a value they
// cannot take, so the compiler keeps every operation and nothing is written.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/lbm.h"
#include "../../include/lbm_probe.h"

namespace {

constexpr int PROBE_THREADS = 256, PROBE_BLOCKS_PER_SM = 8, CHAINS = 8;

template <int KIND>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(long long iters, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if constexpr (KIND == LBM_PROBE_FP64) {
    double a[CHAINS];
    const double b = 1.0 - 1e-12 * (t & 7), c = 1e-9;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 1.0 + 1e-3 * k + 1e-7 * (t & 1023);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
  } else if constexpr (KIND == LBM_PROBE_FP32) {
    float a[CHAINS];
    const float b = 1.0f - 1e-7f * (t & 7), c = 1e-6f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = 1.0f + 1e-3f * k + 1e-7f * (t & 1023);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) a[k] = __fmaf_rn(a[k], b, c);
    }
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
  } else {
    float2 a[CHAINS];
    const float2 b = make_float2(1.0f - 1e-7f * (t & 7), 1.0f - 2e-7f * (t & 7));
    const float2 c = make_float2(1e-6f, 2e-6f);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k)
      a[k] = make_float2(1.0f + 1e-3f * k + 1e-7f * (t & 1023), 1.0f - 1e-3f * k);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < CHAINS; ++k) a[k] = __ffma2_rn(a[k], b, c);
    }
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k].x + a[k].y;
  }
  if (s == -12345.0) out[t & 1023] = s;  // never true: keeps the chains live
}

// Launch of `iters` iterations of kind KIND on `blocks` blocks; elapsed ms.
template <int KIND>
cudaError_t timed(int blocks, long long iters, double* buf, cudaStream_t s, cudaEvent_t e0,
                  cudaEvent_t e1, float* ms) {
  cudaEventRecord(e0, s);
  k_fma_probe<KIND><<<blocks, PROBE_THREADS, 0, s>>>(iters, buf);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  return e;
}

template <int KIND>
cudaError_t rate(double millis, double* out, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * PROBE_BLOCKS_PER_SM;
  double* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&buf, 1024 * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  long long iters = 1024;
  // Calibrate: grow the iteration count until a launch takes >= 1/4 of the
  // target, then scale to the target (bounded: at most 2^26 iterations).
  while (e == cudaSuccess) {
    e = timed<KIND>(blocks, iters, buf, s, e0, e1, &ms);
    if (e != cudaSuccess || ms >= 0.25f * (float)millis || iters >= (1ll << 26)) break;
    iters *= 4;
  }
  if (e == cudaSuccess && ms > 0.f)
    iters = std::min(1ll << 26, std::max(1ll, (long long)(iters * (millis / ms))));
  const double lanes = KIND == LBM_PROBE_FP32X2 ? 2.0 : 1.0;
  double best = 0.0;
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    e = timed<KIND>(blocks, iters, buf, s, e0, e1, &ms);
    if (e == cudaSuccess && ms > 0.f)
      best = std::max(best, (double)blocks * PROBE_THREADS * CHAINS * lanes * (double)iters /
                                (ms * 1e-3));
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  *out = best;
  return e;
}

}  // namespace

extern "C" int lbm_probe_fma_rate(int kind, double millis, double* fma_per_s, void* cuda_stream) {
  if (!fma_per_s || !(millis >= 1.0 && millis <= 2000.0)) return LBM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e;
  switch (kind) {
    case LBM_PROBE_FP64: e = rate<LBM_PROBE_FP64>(millis, fma_per_s, s); break;
    case LBM_PROBE_FP32: e = rate<LBM_PROBE_FP32>(millis, fma_per_s, s); break;
    case LBM_PROBE_FP32X2: e = rate<LBM_PROBE_FP32X2>(millis, fma_per_s, s); break;
    default: return LBM_ERR_INVALID;
  }
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
