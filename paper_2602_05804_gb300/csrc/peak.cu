// Measured fused-multiply-add throughput of the GPU: the denominators of the
// arithmetic rooflines of the near-field and M2L kernels.
//
// Every thread runs eight independent FMA chains (enough independent work per
// warp scheduler to hide the pipe latency), every SM is filled with 32 warps,
// and the chains' operands come from kernel arguments so that nothing folds at
// compile time.  One launch is calibrated to last about `target_ms`; the best
// of `reps` launches, timed with CUDA events on the caller's stream, gives the
// rate (2 flops per FMA, 4 per packed FP32 FMA).
#include <algorithm>

#include "sfmm_internal.cuh"

namespace {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 4;

template <int FORM>  // 0 FP64, 1 FP32, 2 packed FP32
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(int iters, double b, double c, double* sink) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (FORM == 0) {
    double a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = 1.0 + 1e-3 * (k + (tid & 7));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
    if (s == 12345.678) sink[tid] = s;  // never true; keeps the chains live
  } else if constexpr (FORM == 1) {
    const float bf = (float)b, cf = (float)c;
    float a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = 1.0f + 1e-3f * (k + (tid & 7));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = __fmaf_rn(a[k], bf, cf);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
    if (s == 12345.678f) sink[tid] = s;
  } else {
    const float2 b2 = make_float2((float)b, (float)b), c2 = make_float2((float)c, (float)c);
    float2 a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = make_float2(1.0f + 1e-3f * k, 1.0f + 1e-3f * (tid & 7));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k].x + a[k].y;
    if (s == 12345.678f) sink[tid] = s;
  }
}

int launch_peak(int form, int blocks, int iters, cudaStream_t st, double* sink) {
  const double b = 0.9999999, c = 1e-7;  // a stays near 1: no overflow, no subnormals
  switch (form) {
    case 0: k_fma_peak<0><<<blocks, PEAK_THREADS, 0, st>>>(iters, b, c, sink); break;
    case 1: k_fma_peak<1><<<blocks, PEAK_THREADS, 0, st>>>(iters, b, c, sink); break;
    default: k_fma_peak<2><<<blocks, PEAK_THREADS, 0, st>>>(iters, b, c, sink); break;
  }
  return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ECUDA;
}

}  // namespace

extern "C" int sfmm_fma_peak(int device, int form, void* stream, double target_ms, int reps, double* tflops,
                             double* ms) {
  if (form < 0 || form > 2 || !tflops || reps < 1 || reps > 1000 || !(target_ms > 0.0 && target_ms <= 1000.0))
    return SFMM_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SFMM_EINVAL;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = sfmm::num_sms(device) * PEAK_BLOCKS_PER_SM;
  const double threads = (double)blocks * PEAK_THREADS;
  const double flops_per_iter = threads * PEAK_CHAINS * (form == 2 ? 4.0 : 2.0);
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SFMM_OK;
  double best = 0.0, best_ms = 0.0;
  if (cudaMalloc(&sink, sizeof(double) * (size_t)threads) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    rc = SFMM_ECUDA;
  }
  // calibrate: a short launch, then scale the iteration count to target_ms
  int iters = (form == 0) ? 64 : 4096;
  for (int pass = 0; rc == SFMM_OK && pass < 2; ++pass) {
    float t = 0.f;
    if ((rc = launch_peak(form, blocks, iters, st, sink))) break;  // warm-up of this size
    cudaEventRecord(e0, st);
    if ((rc = launch_peak(form, blocks, iters, st, sink))) break;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      rc = SFMM_ECUDA;
      break;
    }
    const double scale = std::min(target_ms / std::max((double)t, 1e-3), 1000.0);
    iters = (int)std::min(std::max((double)iters * scale, 16.0), 2.0e8);
  }
  for (int r = 0; rc == SFMM_OK && r < reps; ++r) {
    float t = 0.f;
    cudaEventRecord(e0, st);
    if ((rc = launch_peak(form, blocks, iters, st, sink))) break;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      rc = SFMM_ECUDA;
      break;
    }
    const double rate = flops_per_iter * iters / (t * 1e-3) / 1e12;
    if (rate > best) {
      best = rate;
      best_ms = t;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (rc) cudaGetLastError();
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  *tflops = best;
  if (ms) *ms = best_ms;
  return rc;
}
