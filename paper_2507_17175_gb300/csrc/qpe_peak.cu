// FMA throughput of the FP64 and FP32 units (include/qpe_peak.h): the
// measured denominators of the ALU-bound kernels' roofline.
#include <cuda_runtime.h>

#include "../../include/qpe_peak.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;
constexpr int kChains = 8;

// 8 independent chains x = x * a + b per thread; a and b keep |x| bounded
// (a < 1), and the results go to memory so nothing is removed.
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_loop_kernel(T* __restrict__ out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(int64_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" qpe_status qpe_measure_fma_peak(int32_t fp64, int32_t iters, int32_t repeats, void* scratch,
                                           size_t scratch_bytes, size_t* scratch_bytes_needed, double* tflops,
                                           void* cuda_stream) {
  if (iters < 1 || iters > (1 << 20) || repeats < 1 || repeats > 100) return QPE_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QPE_ERR_CUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QPE_ERR_CUDA;
  const int64_t ctas = (int64_t)nsm * kCtasPerSm;
  const size_t need = (size_t)ctas * kThreads * 8;
  if (scratch_bytes_needed) *scratch_bytes_needed = need;
  if (!scratch) return QPE_OK;  // a size query
  if (!tflops) return QPE_ERR_ARG;
  if (scratch_bytes < need) return QPE_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return QPE_ERR_CUDA;
  auto launch = [&]() {
    if (fp64)
      fma_loop_kernel<double><<<(unsigned)ctas, kThreads, 0, s>>>(static_cast<double*>(scratch), iters, 0.999, 1e-3);
    else
      fma_loop_kernel<float><<<(unsigned)ctas, kThreads, 0, s>>>(static_cast<float*>(scratch), iters, 0.999f, 1e-3f);
  };
  launch();  // warm-up
  float best_ms = 0.f;
  cudaError_t e = cudaGetLastError();
  for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (r == 0 || ms < best_ms)) best_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || best_ms <= 0.f) return QPE_ERR_CUDA;
  const double flop = 2.0 * kChains * (double)iters * (double)ctas * kThreads;
  *tflops = flop / (best_ms * 1e-3) / 1e12;
  return QPE_OK;
}
