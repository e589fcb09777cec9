// qpe_readout_static: the histogram + readout reduction for callers that
// cannot allocate device memory.
//
// The regular path needs a workspace from the caller (qpe_plan / qpe_bind).
// Some callers cannot provide one: code that runs where device allocation is
// forbidden or unsafe (inside a region that must not synchronise or grow the
// memory pool, under a fixed memory budget, or in a host library that never
// owns device memory). For them this entry point keeps its only scratch, the
// per-block partial results of the reduction, in a fixed array compiled into
// the library. The caller passes the final statevector and receives the
// histogram and the readout in its own buffers; nothing is allocated.
#include <cuda_runtime.h>

#include <mutex>

#include "qpe_internal.cuh"

namespace {

constexpr int kRowsPerBlock = 256;  // rows of the state reduced by one CTA
constexpr int kMaxBlocks = 8192;    // -> at most 2^21 rows (Nmeas <= 21)

// Scratch shared by every call on a device: one partial per CTA. Every slot a
// call reads is written earlier in the same call, so nothing needs clearing;
// calls whose kernels overlap on the GPU overwrite each other's partials.
static __device__ __align__(256) qpe::Partial g_readout_scratch[kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
qpe::Partial* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in for it).
cudaError_t scratch_address(qpe::Partial** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_readout_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<qpe::Partial*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// P[y] = sum_t |X[y][t]|^2 for the rows of this CTA; partial readout into parts[blockIdx.x]
template <typename C>
__global__ void __launch_bounds__(256) static_partials_kernel(const C* __restrict__ X, double* __restrict__ probs,
                                                              qpe::Partial* __restrict__ parts, int64_t N, int logd) {
  const int d = 1 << logd;
  const int lanes = d < 32 ? d : 32;  // lanes per row
  const int rows_per_warp = 32 / lanes;
  const int per = d / lanes;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock;
  double best = -1.0, wsum = 0.0, psum = 0.0;
  int64_t by = INT64_MAX;
  for (int rr = warp * rows_per_warp; rr < kRowsPerBlock; rr += 8 * rows_per_warp) {
    const int64_t y = r0 + rr + lane / lanes;
    const int sub = lane % lanes;
    double acc = 0.0;
    if (rr + lane / lanes < kRowsPerBlock && y < N) {
      const C* row = X + (y << logd);
      for (int k = 0; k < per; ++k) {
        const C v = row[sub + k * lanes];
        acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
      }
    }
    for (int off = lanes >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (sub == 0 && rr + lane / lanes < kRowsPerBlock && y < N) {
      probs[y] = acc;
      qpe::better(best, by, acc, y);
      wsum += acc * (double)y;
      psum += acc;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int64_t oy = __shfl_xor_sync(0xffffffffu, by, off);
    qpe::better(best, by, ob, oy);
    wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
    psum += __shfl_xor_sync(0xffffffffu, psum, off);
  }
  __shared__ qpe::Partial sp[8];
  if (lane == 0) sp[warp] = qpe::Partial{best, by, wsum, psum};
  __syncthreads();
  if (threadIdx.x == 0) {
    qpe::Partial r = sp[0];
    for (int w = 1; w < 8; ++w) {
      qpe::better(r.best, r.besty, sp[w].best, sp[w].besty);
      r.wsum += sp[w].wsum;
      r.psum += sp[w].psum;
    }
    parts[blockIdx.x] = r;
  }
}

// The same merge and readout as the plan path's finalize; a non-finite sum or
// a histogram without any comparable bin reports argmax = -1 and a NaN
// phase_argmax.
__global__ void __launch_bounds__(256) static_finish_kernel(const qpe::Partial* __restrict__ parts, int count,
                                                            qpe_readout_t* __restrict__ out, int n) {
  const qpe::Partial m = qpe::reduce_partials_256(parts, count);
  if (threadIdx.x == 0) {
    const double N = ldexp(1.0, n);
    const bool ok = qpe::readout_finite(m);
    qpe_readout_t o;
    o.argmax = ok ? m.besty : -1;
    o.phase_argmax = ok ? (double)m.besty / N : __longlong_as_double(0x7ff8000000000000LL);
    o.phase_mean = m.wsum / N;
    o.total = m.psum;
    *out = o;
  }
}

}  // namespace

extern "C" qpe_status qpe_readout_static(const void* final_state, int32_t nmat, int32_t nmeas, int32_t prec,
                                         double* probs, qpe_readout_t* readout, void* cuda_stream) {
  if (!final_state || !probs || !readout) return QPE_ERR_ARG;
  if (nmat < 1 || nmat > 12 || nmeas < 1 || nmeas > 30) return QPE_ERR_ARG;
  if (prec < QPE_FP64 || prec > QPE_C64_TF32X3) return QPE_ERR_ARG;
  const int64_t N = int64_t(1) << nmeas;
  const int64_t blocks = (N + kRowsPerBlock - 1) / kRowsPerBlock;
  if (blocks > kMaxBlocks) return QPE_ERR_WORKSPACE;  // the fixed scratch holds 8192 partials: Nmeas <= 21
  qpe::Partial* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return QPE_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (prec == QPE_FP64)
    static_partials_kernel<double2><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const double2*>(final_state), probs,
                                                                      scratch, N, nmat);
  else
    static_partials_kernel<float2><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float2*>(final_state), probs,
                                                                     scratch, N, nmat);
  if (cudaGetLastError() != cudaSuccess) return QPE_ERR_CUDA;
  static_finish_kernel<<<1, 256, 0, s>>>(scratch, (int)blocks, readout, nmeas);
  if (cudaGetLastError() != cudaSuccess) return QPE_ERR_CUDA;
  return QPE_OK;
}
