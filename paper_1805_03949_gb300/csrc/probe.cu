// probe.cu -- arithmetic peaks of the current GPU, measured: the FP64 and FP32
// denominators of the assembly roofline (its HBM denominator is a copy rate
// measured outside the library).
//
// Every SM runs warps of independent fused multiply-add chains long enough
// that launch and tail costs vanish; the rate is the FMA count x 2 over the
// kernel's CUDA-event time.  The chains are x <- x m + c with |m| < 1, so the
// values stay normal and finite whatever the length.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "element.cuh"
#include "fea_internal.cuh"

namespace fea {

// the kernels' own precision conversions, elementwise (dir 0: FP32 -> FP64
// exact widening; dir 1: FP64 -> FP32 rounded to nearest even), by integer
// instructions as in the assembly kernels
__global__ void k_convert(int dir, const void* in, void* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (dir == 0)
      static_cast<double*>(out)[i] = f32_to_f64_exact(static_cast<const float*>(in)[i]);
    else
      static_cast<float*>(out)[i] = f64_to_f32_rn(static_cast<const double*>(in)[i]);
  }
}

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int64_t iters, T* out) {
  T x[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = (T)(threadIdx.x + 1 + k) * (T)1e-3;
  const T m = (T)0.9990234375, c = (T)1.220703125e-4;  // both exact in FP32 and FP64
  for (int64_t it = 0; it < iters; it += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kProbeChains; ++k) x[k] = fma(x[k], m, c);
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int run_probe(int64_t iters, double* flops, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  FEA_CUDA(cudaGetDevice(&dev));
  FEA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  FEA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, kProbeThreads, 0));
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  T* out = nullptr;
  FEA_CUDA(cudaMalloc(&out, sizeof(T) * (size_t)grid * kProbeThreads));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FEA_OK;
  float ms = 0.0f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = fail(FEA_ERR_CUDA, "fea_peak_probe: cudaEventCreate failed");
  } else {
    k_fma_probe<T><<<grid, kProbeThreads, 0, s>>>(iters / 8 + 4, out);  // warm-up (clocks, caches)
    cudaEventRecord(e0, s);
    k_fma_probe<T><<<grid, kProbeThreads, 0, s>>>(iters, out);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) rc = cuda_fail(e, "fea_peak_probe");
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == FEA_OK) {
    const int64_t iters4 = (iters + 3) / 4 * 4;
    *flops = 2.0 * kProbeChains * (double)iters4 * grid * kProbeThreads / (ms * 1e-3);
  }
  return rc;
}

}  // namespace fea

extern "C" int fea_convert(int dir, const void* in, void* out, int64_t n, void* stream) {
  using namespace fea;
  if ((dir != 0 && dir != 1) || n < 0 || (n > 0 && (!in || !out)))
    return fail(FEA_ERR_ARG, "fea_convert: dir 0 or 1, n >= 0, buffers not null");
  if (n == 0) return FEA_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_convert<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(dir, in, out, n);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

extern "C" int fea_peak_probe(int kind, int64_t iters, double* flops, void* stream) {
  using namespace fea;
  if (!flops || iters < 4 || (kind != 0 && kind != 1))
    return fail(FEA_ERR_ARG, "fea_peak_probe: kind 0 (FP64) or 1 (FP32), iters >= 4, flops not null");
  cudaStream_t s = (cudaStream_t)stream;
  return kind == 0 ? run_probe<double>(iters, flops, s) : run_probe<float>(iters, flops, s);
}
