// Arithmetic throughput probe used as the roofline denominator for ALU-bound kernels:
// a grid of 8 independent FMA chains per thread, timed with CUDA events. Also the element
// kernels' pivot inverse square root evaluated on given inputs, for its accuracy test.
#include <cuda_runtime.h>

#include "hyb_device.h"
#include "hyb_internal.h"

namespace hyb {
namespace {

template <typename T>
__global__ void fma_chains_kernel(T* out, int iters, T a, T b) {
  T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
int measure(cudaStream_t s, int iters, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYB_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HYB_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  T* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(T) * blocks * threads, s) != cudaSuccess) return HYB_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, s);
    fma_chains_kernel<T><<<blocks, threads, 0, s>>>(out, iters, (T)0.999, (T)1e-3);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaFreeAsync(out, s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return HYB_ERR_CUDA;
  *tflops = 2.0 * 32.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return HYB_OK;
}

__global__ void rsqrt_probe_kernel(int64_t n, const double* x, double* out, int* ok) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = dev::rsqrt_h3(x[i]);
    ok[i] = dev::positive_normal(x[i]) ? 1 : 0;
  }
}

}  // namespace
}  // namespace hyb

extern "C" int hyb_rsqrt_probe(int64_t n, const double* x, double* out, int* positive_normal, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!x || !out || !positive_normal))) return HYB_ERR_INVALID_ARG;
  if (n == 0) return HYB_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int64_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  hyb::rsqrt_probe_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, x, out, positive_normal);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? HYB_OK : HYB_ERR_CUDA;
}

extern "C" int hyb_measure_fma_peak(int fp64, void* cuda_stream, double* tflops) {
  if (!tflops) return HYB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return fp64 ? hyb::measure<double>(s, 2000, tflops) : hyb::measure<float>(s, 32000, tflops);
}
