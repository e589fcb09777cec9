// Grouped kernels for batched plans (many QPE instances of uneven Nmat and
// Nmeas in one plan). Each grouped launch covers one step for every instance
// that needs it, with CTAs mapped to (instance, tile) through a work list in
// the workspace:
//   squaring step k   every instance with Nmeas > k: P_k = P_(k-1)^2 (FP64),
//                      8 x 8 output tiles, plus the complex64 copy;
//   tables / seeds    every fused instance (Nmat <= 6);
//   level rounds      see level2_grouped_kernel (qpe_level.cu);
//   finalize          one CTA per fused instance.
#include <cuda_runtime.h>

#include "qpe_internal.cuh"

namespace qpe {

namespace {

template <typename C>
__device__ __forceinline__ C ldgc(const C* p) { return __ldg(p); }

}  // namespace

// P_k = P_(k-1)^2 for every listed instance: 8 x 8 output tile per CTA, the
// inner index split over 4 thread layers and summed in shared memory.
__global__ void __launch_bounds__(256) square_grouped_kernel(const SqItem* __restrict__ items, int nitems) {
  pdl_begin();
  __shared__ double2 red[4][8][8];
  const SqItem it = items[find_item(items, nitems, blockIdx.x)];
  const int64_t t = blockIdx.x - it.tile0;
  const int d = it.d;
  const int nt = (d + 7) / 8;
  const int by = (int)(t / nt), bx = (int)(t % nt);
  const int tx = threadIdx.x & 7, ty = (threadIdx.x >> 3) & 7, tz = threadIdx.x >> 6;
  const int row = by * 8 + ty, col = bx * 8 + tx;
  double2 acc = make_double2(0.0, 0.0);
  if (row < d && col < d) {
    const double2* arow = it.A + (int64_t)row * d;
    for (int k = tz; k < d; k += 4) cfma(acc, ldgc(arow + k), ldgc(it.A + (int64_t)k * d + col));
  }
  red[tz][ty][tx] = acc;
  __syncthreads();
  if (tz == 0 && row < d && col < d) {
    double2 s = red[0][ty][tx];
    for (int z = 1; z < 4; ++z) s = cadd(s, red[z][ty][tx]);
    const int64_t o = (int64_t)row * d + col;
    it.C[o] = s;
    if (it.C32) it.C32[o] = make_float2((float)s.x, (float)s.y);
    if (it.A32) {
      const double2 v = it.A[o];
      it.A32[o] = make_float2((float)v.x, (float)v.y);
    }
  }
  pdl_trigger();
}

__device__ __forceinline__ int64_t sq_first(const SqItem& it, int v) {
  return v == 0 ? it.tile0 : (v == 1 ? it.tile16 : it.tile32);
}

// P_k = P_(k-1)^2 for every listed instance: T x T output tile per CTA (256
// threads, TM x TM outputs each), 16-wide k slabs of the row and column
// panels staged in shared memory. V selects the item's CTA numbering.
template <int T, int TM, int V>
__global__ void __launch_bounds__(256) square_grouped_smem_kernel(const SqItem* __restrict__ items, int nitems) {
  pdl_begin();
  constexpr int BK = 16;
  constexpr int TPD = T / TM;  // threads per tile dimension (16)
  __shared__ double2 As[BK][T + 1];  // As[kk][r] = A[r0 + r][k0 + kk]
  __shared__ double2 Bs[BK][T + 1];  // Bs[kk][c] = A[k0 + kk][c0 + c]
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sq_first(items[mid], V) <= (int64_t)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  const SqItem it = items[lo];
  const int64_t t = blockIdx.x - sq_first(it, V);
  const int d = it.d;
  const int nt = (d + T - 1) / T;
  const int r0 = (int)(t / nt) * T, c0 = (int)(t % nt) * T;
  const int tc = threadIdx.x % TPD, tr = threadIdx.x / TPD;
  const double2 zero = make_double2(0.0, 0.0);
  double2 acc[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = zero;
  for (int k0 = 0; k0 < d; k0 += BK) {
    for (int idx = threadIdx.x; idx < T * BK; idx += 256) {
      const int r = idx / BK, kk = idx % BK;
      As[kk][r] = (r0 + r < d && k0 + kk < d) ? ldgc(it.A + (int64_t)(r0 + r) * d + k0 + kk) : zero;
      const int kb = idx / T, cb = idx % T;
      Bs[kb][cb] = (k0 + kb < d && c0 + cb < d) ? ldgc(it.A + (int64_t)(k0 + kb) * d + c0 + cb) : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a[TM], b[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tr + i * TPD];
#pragma unroll
      for (int j = 0; j < TM; ++j) b[j] = Bs[kk][tc + j * TPD];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      const int row = r0 + tr + i * TPD, col = c0 + tc + j * TPD;
      if (row >= d || col >= d) continue;
      const int64_t o = (int64_t)row * d + col;
      it.C[o] = acc[i][j];
      if (it.C32) it.C32[o] = make_float2((float)acc[i][j].x, (float)acc[i][j].y);
      if (it.A32) {
        const double2 v = it.A[o];
        it.A32[o] = make_float2((float)v.x, (float)v.y);
      }
    }
  pdl_trigger();
}

// complex64 copy of P_0 for instances with Nmeas = 1 (no squaring writes it)
__global__ void convert_grouped_kernel(const SqItem* __restrict__ items, int nitems) {
  pdl_begin();
  const SqItem it = items[find_item(items, nitems, blockIdx.x)];
  const int64_t t = blockIdx.x - it.tile0;
  const int64_t dd = (int64_t)it.d * it.d;
  for (int64_t i = t * 256 + threadIdx.x; i < dd && i < (t + 1) * 256; i += blockDim.x) {
    const double2 v = it.A[i];
    it.A32[i] = make_float2((float)v.x, (float)v.y);
  }
  pdl_trigger();
}

// Level tables of every fused instance (same layout and arithmetic as
// level_table_kernel): one CTA per (instance, level, m_b, block of rows).
template <typename C>
__global__ void __launch_bounds__(256) table_grouped_kernel(const TabItem<C>* __restrict__ items, int nitems) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TabItem<C> it = items[find_item(items, nitems, blockIdx.x)];
  const int64_t b = blockIdx.x - it.tile0;
  const int D = 1 << it.logd;
  const int TB = D < 16 ? D : 16;
  const int nrb = D / TB;
  C* Pb = reinterpret_cast<C*>(smem_raw);
  C* V = Pb + D * D;
  C* Vn = V + TB * D;
  const int mb = (int)(b / nrb), rb = (int)(b % nrb);
  const int i0 = rb * TB;
  const int64_t DD = (int64_t)D * D;
  const int tid = threadIdx.x;
  bool started = false;
  for (int j = 0; j < it.r; ++j) {
    if (!((mb >> j) & 1)) continue;
    const C* Pj = it.P + (int64_t)(it.off + j) * DD;
    if (!started) {
      for (int e = tid; e < TB * D; e += blockDim.x) V[e] = ldgc(Pj + (int64_t)i0 * D + e);
      started = true;
      continue;
    }
    __syncthreads();
    for (int e = tid; e < D * D; e += blockDim.x) Pb[e] = ldgc(Pj + e);
    __syncthreads();
    const int q4 = D >= 4 ? D / 4 : 1;
    for (int e = tid; e < TB * q4; e += blockDim.x) {
      const int rr = e / q4, k0 = e - rr * q4;
      const int nk = D >= 4 ? 4 : D;
      C acc[4] = {mk((typename real_of<C>::type)0, (typename real_of<C>::type)0),
                  mk((typename real_of<C>::type)0, (typename real_of<C>::type)0),
                  mk((typename real_of<C>::type)0, (typename real_of<C>::type)0),
                  mk((typename real_of<C>::type)0, (typename real_of<C>::type)0)};
      for (int l = 0; l < D; ++l) {
        const C v = V[rr * D + l];
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < nk) cfma(acc[t], v, Pb[l * D + k0 + t * q4]);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nk) Vn[rr * D + k0 + t * q4] = acc[t];
    }
    __syncthreads();
    for (int e = tid; e < TB * D; e += blockDim.x) V[e] = Vn[e];
  }
  if (!started) {
    for (int e = tid; e < TB * D; e += blockDim.x) {
      const int rr = e / D, k = e - rr * D;
      V[e] = (k == i0 + rr) ? mk((typename real_of<C>::type)1, (typename real_of<C>::type)0)
                            : mk((typename real_of<C>::type)0, (typename real_of<C>::type)0);
    }
  }
  __syncthreads();
  const int ROWS = (1 << it.r) << it.logd;
  for (int e = tid; e < TB * D; e += blockDim.x) {
    const int k = e / TB, rr = e - k * TB;
    it.tab[(int64_t)k * ROWS + mb * D + i0 + rr] = V[rr * D + k];
  }
  pdl_trigger();
}

// psi (complex128) -> the deepest level's seed, one CTA per fused instance
template <typename C>
__global__ void seed_grouped_kernel(const SeedItem<C>* __restrict__ items) {
  pdl_begin();
  const SeedItem<C> it = items[blockIdx.x];
  for (int i = threadIdx.x; i < it.d; i += blockDim.x) it.seed[i] = to_c(it.psi[i], (C*)nullptr);
  pdl_trigger();
}

// readout of every fused instance from its level partials, one CTA each
__global__ void __launch_bounds__(256) finalize_grouped_kernel(const FinItem* __restrict__ items) {
  pdl_begin();
  const FinItem it = items[blockIdx.x];
  const Partial m = reduce_partials_256(it.parts, it.count);
  if (threadIdx.x == 0) {
    const double N = ldexp(1.0, it.nmeas);
    Scalars s;
    s.argmax = m.besty;
    s.phase_argmax = (double)m.besty / N;
    s.phase_mean = m.wsum / N;
    s.total = m.psum;
    s.best = m.best;
    s.err = readout_finite(m) ? 0 : (int)QPE_ERR_NUMERIC;
    s.pad = 0;
    *it.out = s;
  }
  pdl_trigger();
}

// ------------------------------------------------------------- launchers
int launch_square_grouped(const SqItem* items, int nitems, int64_t tiles, int variant, cudaStream_t s) {
  if (nitems <= 0) return 0;
  cudaError_t e;
  switch (variant) {
    case 1: e = launch_k(square_grouped_smem_kernel<16, 1, 1>, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems); break;
    case 2: e = launch_k(square_grouped_smem_kernel<32, 2, 2>, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems); break;
    default: e = launch_k(square_grouped_kernel, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems); break;
  }
  return e == cudaSuccess ? 1 : -1;
}

int launch_convert_grouped(const SqItem* items, int nitems, int64_t tiles, cudaStream_t s) {
  if (nitems <= 0) return 0;
  return launch_k(convert_grouped_kernel, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems) == cudaSuccess ? 1
                                                                                                                : -1;
}

template <typename C>
int launch_table_grouped(const TabItem<C>* items, int nitems, int64_t blocks, int max_logd, cudaStream_t s) {
  if (nitems <= 0) return 0;
  const size_t D = size_t(1) << max_logd;
  const size_t TB = D < 16 ? D : 16;
  const size_t smem = (D * D + 2 * TB * D) * sizeof(C);
  return launch_k(table_grouped_kernel<C>, dim3((unsigned)blocks), dim3(256), smem, s, items, nitems) == cudaSuccess
             ? 1
             : -1;
}

template <typename C>
int launch_seed_grouped(const SeedItem<C>* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return 0;
  return launch_k(seed_grouped_kernel<C>, dim3((unsigned)nitems), dim3(64), 0, s, items) == cudaSuccess ? 1 : -1;
}

int launch_finalize_grouped(const FinItem* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return 0;
  return launch_k(finalize_grouped_kernel, dim3((unsigned)nitems), dim3(256), 0, s, items) == cudaSuccess ? 1 : -1;
}

cudaError_t configure_batched_kernels() {
  cudaError_t e = cudaFuncSetAttribute(table_grouped_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (64 * 64 + 2 * 16 * 64) * 16);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(table_grouped_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (64 * 64 + 2 * 16 * 64) * 8);
}

template int launch_table_grouped<float2>(const TabItem<float2>*, int, int64_t, int, cudaStream_t);
template int launch_table_grouped<double2>(const TabItem<double2>*, int, int64_t, int, cudaStream_t);
template int launch_seed_grouped<float2>(const SeedItem<float2>*, int, cudaStream_t);
template int launch_seed_grouped<double2>(const SeedItem<double2>*, int, cudaStream_t);

}  // namespace qpe
