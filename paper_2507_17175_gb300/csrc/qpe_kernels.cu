// CUDA kernels of the QPE emulator (sm_103a).
//
// Stages (Fig. 1, left to right):
//   powers   P_k = U^(2^k) by FP64 repeated squaring (P_{k+1} = P_k P_k).
//   sweep    Hadamard layer + controlled-U^(2^k): row m of the N x d state
//            becomes 2^(-n/2) U^m psi. Two schedules:
//              doubling  S[m + 2^j] = P_j S[m] for m < 2^j, j = 0..n-1
//                        (every row receives exactly the controlled gates of
//                        its set bits, lowest bit first, as in the circuit;
//                        each distinct row value is computed once);
//              gate      for k = 0..n-1, every row with bit k set is
//                        replaced by P_k times itself (one pass per gate).
//   fft      QFT^-1 on the measurement register = a batched DFT along m with
//            kernel exp(-2 pi i m y / N), decimation in frequency, in place,
//            in passes of up to 2^9 points staged in shared memory.
//   reduce   P[y] = sum_t |X[y][t]|^2 with digit-reversal undone, plus the
//            readout: argmax (lowest y on ties) and sum_y P[y] y / N.
#include <cuda_runtime.h>
#include <math.h>

#include "qpe_internal.cuh"

namespace qpe {

namespace {

__device__ __forceinline__ double2 ld(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld(const float2* p) { return __ldg(p); }

// omega_N^e = exp(-2 pi i e / N) from the two-level table: e = hi * 2^h + lo.
template <typename C>
__device__ __forceinline__ C twiddle(const C* lo, const C* hi, int h, int64_t e) {
  const int64_t mask = (int64_t(1) << h) - 1;
  return cmul(ld(lo + (e & mask)), ld(hi + (e >> h)));
}

// ------------------------------------------------------------- twiddles
__global__ void twiddle_tables_kernel(double2* lo64, double2* hi64, float2* lo32, float2* hi32,
                                      int n, int h) {
  pdl_begin();
  const int64_t nlo = int64_t(1) << h;
  const int64_t nhi = int64_t(1) << (n - h);
  const double N = ldexp(1.0, n);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlo + nhi;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i < nlo ? i : ((i - nlo) << h);
    double s, c;
    sincospi(-2.0 * (double)e / N, &s, &c);  // exact argument: e < N = 2^n
    const double2 v = make_double2(c, s);
    const float2 f = make_float2((float)c, (float)s);
    if (i < nlo) {
      lo64[i] = v;
      lo32[i] = f;
    } else {
      hi64[i - nlo] = v;
      hi32[i - nlo] = f;
    }
  }
}

// --------------------------------------------------------------- powers
// C = A * A for a d x d complex128 matrix, d <= 256. Each CTA owns a TS x TS
// output tile; its KS thread layers split the inner index and are summed in
// shared memory, so even d = 64 spreads over hundreds of CTAs.
// C32 / A32 (optional): complex64 copies of the result / of the input, each
// element written by the thread that owns that output position.
template <int TS, int KS>
__global__ void __launch_bounds__(TS * TS * KS) square_small_kernel(const double2* __restrict__ A,
                                                                    double2* __restrict__ C, int d,
                                                                    float2* __restrict__ C32,
                                                                    float2* __restrict__ A32) {
  pdl_begin();
  __shared__ double2 red[KS][TS][TS];
  const int tx = threadIdx.x % TS;
  const int ty = (threadIdx.x / TS) % TS;
  const int tz = threadIdx.x / (TS * TS);
  const int row = blockIdx.y * TS + ty;
  const int col = blockIdx.x * TS + tx;
  const int kper = d / KS;
  double2 acc = make_double2(0.0, 0.0);
  const double2* arow = A + (int64_t)row * d;
  for (int k = tz * kper; k < (tz + 1) * kper; ++k) cfma(acc, ld(arow + k), ld(A + (int64_t)k * d + col));
  red[tz][ty][tx] = acc;
  __syncthreads();
  if (tz == 0) {
    double2 s = red[0][ty][tx];
    for (int z = 1; z < KS; ++z) s = cadd(s, red[z][ty][tx]);
    const int64_t o = (int64_t)row * d + col;
    C[o] = s;
    if (C32) C32[o] = make_float2((float)s.x, (float)s.y);
    if (A32) {
      const double2 v = A[o];
      A32[o] = make_float2((float)v.x, (float)v.y);
    }
  }
  pdl_trigger();
}

// Unitarity check of U (the FP64 P_0): G = U^dagger U in 16 x 16 output
// tiles, 16-row slabs of U staged in shared memory; any |G_ij - delta_ij| above
// tol (or not finite) sets *err to QPE_ERR_NUMERIC, keeping an earlier error.
__global__ void __launch_bounds__(256) unitarity_kernel(const double2* __restrict__ U, int d, double tol,
                                                        int* __restrict__ err) {
  pdl_begin();
  __shared__ double2 Ui[16][17];  // U[k0 + r][i0 + c]
  __shared__ double2 Uj[16][17];  // U[k0 + r][j0 + c]
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  const double2 zero = make_double2(0.0, 0.0);
  double2 acc = zero;
  for (int k0 = 0; k0 < d; k0 += 16) {
    const int k = k0 + ty;
    Ui[ty][tx] = (k < d && i0 + tx < d) ? U[(int64_t)k * d + i0 + tx] : zero;
    Uj[ty][tx] = (k < d && j0 + tx < d) ? U[(int64_t)k * d + j0 + tx] : zero;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const double2 a = Ui[kk][ty];  // U[k][i]
      const double2 b = Uj[kk][tx];  // U[k][j]
      acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));   // Re(conj(a) b)
      acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));  // Im(conj(a) b)
    }
    __syncthreads();
  }
  const int i = i0 + ty, j = j0 + tx;
  if (i < d && j < d) {
    const double re = acc.x - (i == j ? 1.0 : 0.0);
    if (!(re * re + acc.y * acc.y <= tol * tol)) atomicCAS(err, 0, (int)QPE_ERR_NUMERIC);
  }
  pdl_trigger();
}

// C = A * A for d >= 512: 32 x 32 output tiles, 16-wide k slabs in shared
// memory, 2 x 2 outputs per thread.
__global__ void __launch_bounds__(256) square_tiled_kernel(const double2* __restrict__ A,
                                                           double2* __restrict__ C, int d,
                                                           float2* __restrict__ C32, float2* __restrict__ A32) {
  pdl_begin();
  constexpr int T = 32, BK = 16;
  __shared__ double2 As[BK][T + 1];
  __shared__ double2 Bs[BK][T + 1];
  const int tid = threadIdx.x;
  const int tc = tid % 16, tr = tid / 16;
  const int r0 = blockIdx.y * T, c0 = blockIdx.x * T;
  double2 acc[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < d; k0 += BK) {
    for (int idx = tid; idx < T * BK; idx += 256) {
      const int r = idx / BK, kk = idx % BK;
      As[kk][r] = ld(A + (int64_t)(r0 + r) * d + k0 + kk);
      const int kb = idx / T, cb = idx % T;
      Bs[kb][cb] = ld(A + (int64_t)(k0 + kb) * d + c0 + cb);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const double2 a0 = As[kk][tr], a1 = As[kk][tr + 16];
      const double2 b0 = Bs[kk][tc], b1 = Bs[kk][tc + 16];
      cfma(acc[0][0], a0, b0);
      cfma(acc[0][1], a0, b1);
      cfma(acc[1][0], a1, b0);
      cfma(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int64_t o = (int64_t)(r0 + tr + 16 * i) * d + c0 + tc + 16 * j;
      C[o] = acc[i][j];
      if (C32) C32[o] = make_float2((float)acc[i][j].x, (float)acc[i][j].y);
      if (A32) {
        const double2 v = A[o];
        A32[o] = make_float2((float)v.x, (float)v.y);
      }
    }
  pdl_trigger();
}

__global__ void convert_c128_to_c64_kernel(const double2* __restrict__ in, float2* __restrict__ out,
                                           int64_t count) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

// ---------------------------------------------------------------- sweep
// rows [0, rows) of S = scale * psi
template <typename C>
__global__ void init_rows_kernel(C* __restrict__ S, const double2* __restrict__ psi, int64_t rows, int logd,
                                 double scale) {
  pdl_begin();
  const int64_t total = rows << logd;
  const int64_t dmask = (int64_t(1) << logd) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = psi[i & dmask];
    S[i] = to_c(make_double2(v.x * scale, v.y * scale), (C*)nullptr);
  }
}

// Logical row r of a controlled-gate GEMM -> physical rows read and written.
struct DoublingRows {  // level j: read row r, write row r + 2^j
  int64_t half;
  __device__ __forceinline__ int64_t in(int64_t r) const { return r; }
  __device__ __forceinline__ int64_t out(int64_t r) const { return r + half; }
};
struct GateRows {  // gate k: the r-th row with bit k set, in place
  int k;
  __device__ __forceinline__ int64_t in(int64_t r) const {
    const int64_t low = r & ((int64_t(1) << k) - 1);
    return ((r >> k) << (k + 1)) | (int64_t(1) << k) | low;
  }
  __device__ __forceinline__ int64_t out(int64_t r) const { return in(r); }
};

// out_row(r)[i] = sum_c P[i][c] * in_row(r)[c] for logical rows r < M:
// a complex GEMM (M x d) * P^T with BM x BN tiles, BK-deep k slabs staged in
// shared memory and TM x TN outputs per thread. When BN == d one CTA owns
// whole rows, so in-place updates (GateRows) are safe: every read of a row
// happens before the CTA's epilogue writes it.
template <typename C, int BM, int BN, int BK, int TM, int TN, typename Rows>
__device__ __forceinline__ void rows_times_pt_tile(C* __restrict__ S, const C* __restrict__ P, int64_t M, int d,
                                                   Rows rows, int64_t bx, int by) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int TCOLS = BN / TN;
  __shared__ C As[BK][BM + 1];
  __shared__ C Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tc = tid % TCOLS, tr = tid / TCOLS;
  const int64_t r0 = bx * BM;
  const int c0 = by * BN;
  C acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = mk((typename real_of<C>::type)0, (typename real_of<C>::type)0);

  for (int k0 = 0; k0 < d; k0 += BK) {
    for (int idx = tid; idx < BM * BK; idx += NT) {
      const int r = idx / BK, kk = idx % BK;
      const int64_t lr = r0 + r;
      C v = mk((typename real_of<C>::type)0, (typename real_of<C>::type)0);
      if (lr < M) v = S[rows.in(lr) * d + k0 + kk];
      As[kk][r] = v;
    }
    for (int idx = tid; idx < BN * BK; idx += NT) {
      const int c = idx / BK, kk = idx % BK;
      Bs[kk][c] = ld(P + (int64_t)(c0 + c) * d + k0 + kk);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tr + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tc + j * TCOLS];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t lr = r0 + tr + i * (BM / TM);
    if (lr >= M) continue;
    C* orow = S + rows.out(lr) * d + c0;
#pragma unroll
    for (int j = 0; j < TN; ++j) orow[tc + j * TCOLS] = acc[i][j];
  }
}

template <typename C, int BM, int BN, int BK, int TM, int TN, typename Rows>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    rows_times_pt_kernel(C* __restrict__ S, const C* __restrict__ P, int64_t M, int d, Rows rows) {
  pdl_begin();
  rows_times_pt_tile<C, BM, BN, BK, TM, TN, Rows>(S, P, M, d, rows, blockIdx.x, blockIdx.y);
}

// One doubling level of every listed instance (batched plans): CTAs map to
// (instance, row tile, column tile) through tile0, the item's first CTA.
template <typename C, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    doubling_grouped_kernel(const DblItem<C>* __restrict__ items, int nitems) {
  pdl_begin();
  const DblItem<C> it = items[find_item(items, nitems, blockIdx.x)];
  const int64_t t = blockIdx.x - it.tile0;
  const int nby = it.d / BN;
  rows_times_pt_tile<C, BM, BN, BK, TM, TN, DoublingRows>(it.S, it.P, it.M, it.d, DoublingRows{it.M}, t / nby,
                                                          (int)(t % nby));
}

// ------------------------------------------------------------------ fft
// One decimation-in-frequency pass over the middle axis of X viewed as
// [B][R][Q] (Q = L * d contiguous elements): for each block and each of the Q
// columns, a length-R DFT over the middle axis (kernel omega_R^(a y)), then
// the twiddle omega_(R L)^(b y) with b = column / d the row offset inside the
// block, stored in place at digit y. Each CTA stages an R x W slab in shared
// memory and runs log2(R) radix-2 stages on it.

__device__ __forceinline__ int bitrev(int x, int bits) { return bits ? (__brev(x) >> (32 - bits)) : 0; }

// K consecutive radix-2 DIF stages on the rows row0 + j 2^logs (j < 2^K) of
// column w, in registers (see fft_pass_kernel).
template <typename C, int K>
__device__ __forceinline__ void fft_group(C* tile, const C* twp, int W, int w, int row0, int logm, int logs,
                                          int logr) {
  constexpr int RK = 1 << K;
  C x[RK];
#pragma unroll
  for (int j = 0; j < RK; ++j) x[j] = tile[(row0 + (j << logs)) * W + w];
#pragma unroll
  for (int lt = 0; lt < K; ++lt) {
    const int logh = logm - lt - 1;  // global half size h = 2^logh
#pragma unroll
    for (int j = 0; j < RK; ++j) {
      const int hh = RK >> (lt + 1);
      if (j & hh) continue;
      const C x0 = x[j], x1 = x[j + hh];
      x[j] = cadd(x0, x1);
      const C dlt = csub(x0, x1);
      const int pos = (row0 + (j << logs)) & ((1 << logh) - 1);
      x[j + hh] = pos ? cmul(dlt, twp[pos << (logr - logh - 1)]) : dlt;
    }
  }
#pragma unroll
  for (int j = 0; j < RK; ++j) tile[(row0 + (j << logs)) * W + w] = x[j];
}

template <typename C>
__device__ __forceinline__ void fft_pass_block(C* __restrict__ X, const C* __restrict__ tw_lo,
                                               const C* __restrict__ tw_hi, const FftArgs& a, int64_t bid) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = reinterpret_cast<C*>(smem_raw);
  using R_t = typename real_of<C>::type;
  const int R = 1 << a.logr;
  const int W = 1 << a.logw;
  const int64_t slices_log = a.logq - a.logw;
  const int64_t blk = bid >> slices_log;
  const int64_t qs = bid & ((int64_t(1) << slices_log) - 1);
  C* base = X + (blk << (a.logr + a.logq)) + (qs << a.logw);
  const int RW = R * W;
  C* twp = tile + RW;  // w_R^e = omega_N^(e << (n - logr)), e < R / 2: the pass's twiddles
  // the tile arrives by asynchronous 16-byte copies (every thread's copies in
  // flight at once) while the twiddles are computed
  constexpr int V = 16 / (int)sizeof(C);  // elements per copy
  if (W >= V) {
    for (int idx = threadIdx.x * V; idx < RW; idx += blockDim.x * V) {
      const int r = idx >> a.logw, w = idx & (W - 1);
      cp_async16(tile + idx, base + ((int64_t)r << a.logq) + w);
    }
  } else {
    for (int idx = threadIdx.x; idx < RW; idx += blockDim.x) {
      const int r = idx >> a.logw, w = idx & (W - 1);
      cp_async_elem(tile + idx, base + ((int64_t)r << a.logq) + w, true);
    }
  }
  cp_async_commit();
  for (int e = threadIdx.x; e < (R >> 1); e += blockDim.x)
    twp[e] = twiddle(tw_lo, tw_hi, a.htw, (int64_t)e << (a.n + a.tw_sh - a.logr));
  cp_async_wait<0>();
  __syncthreads();
  // Radix-2 DIF stages s = 0 .. logr - 1 (stage s pairs rows p and p + h,
  // h = 2^(logr - s - 1), twiddle omega_(2h)^(p mod h) on the difference),
  // three at a time in registers: rows base + j S, j < 2^K, meet only each
  // other within those K stages. The butterflies and twiddles are those of
  // the stage-by-stage order, so the result is the same bit for bit.
  for (int s0 = 0; s0 < a.logr; s0 += 3) {
    const int K = a.logr - s0 < 3 ? a.logr - s0 : 3;
    const int logm = a.logr - s0;  // sub-blocks of 2^logm rows
    const int logs = logm - K;     // stride S = 2^logs between a task's rows
    const int tasks = (R >> K) << a.logw;
    for (int t = threadIdx.x; t < tasks; t += blockDim.x) {
      const int w = t & (W - 1);
      const int rest = t >> a.logw;
      const int q = rest & ((1 << logs) - 1);
      const int b0 = rest >> logs;
      const int row0 = (b0 << logm) + q;
      switch (K) {
        case 1: fft_group<C, 1>(tile, twp, W, w, row0, logm, logs, a.logr); break;
        case 2: fft_group<C, 2>(tile, twp, W, w, row0, logm, logs, a.logr); break;
        default: fft_group<C, 3>(tile, twp, W, w, row0, logm, logs, a.logr); break;
      }
    }
    __syncthreads();
  }
  const int64_t rl_mask = (int64_t(1) << (a.logr + a.logq - a.logd)) - 1;  // R*L - 1
  for (int idx = threadIdx.x; idx < RW; idx += blockDim.x) {
    const int i = idx >> a.logw, w = idx & (W - 1);
    const int ya = bitrev(i, a.logr);
    C v = tile[idx];
    if (!a.last) {
      const int64_t q = (qs << a.logw) + w;
      const int64_t b = q >> a.logd;
      const int64_t e = ((b * ya) & rl_mask) << (a.logb + a.tw_sh);  // omega_(RL)^(b ya) = omega_N^(b ya B)
      if (e) v = cmul(v, twiddle(tw_lo, tw_hi, a.htw, e));
    }
    if (a.scale != 1.0) v = cscale(v, (R_t)a.scale);
    base[((int64_t)ya << a.logq) + w] = v;
  }
}

template <typename C>
__global__ void __launch_bounds__(256) fft_pass_kernel(C* __restrict__ X, const C* __restrict__ tw_lo,
                                                       const C* __restrict__ tw_hi, FftArgs a) {
  pdl_begin();
  fft_pass_block<C>(X, tw_lo, tw_hi, a, blockIdx.x);
}

// One QFT^-1 pass of every listed instance (each item its own pass arguments).
template <typename C>
__global__ void __launch_bounds__(256) fft_pass_grouped_kernel(const FftItem<C>* __restrict__ items, int nitems) {
  pdl_begin();
  const int i = find_item(items, nitems, blockIdx.x);
  fft_pass_block<C>(items[i].X, items[i].lo, items[i].hi, items[i].a, blockIdx.x - items[i].tile0);
}

// --------------------------------------------------------------- reduce

// Position p of the in-place DIF output -> outcome y: the pass that ran
// first (top bits of p) produced the least significant digit of y.
__device__ __forceinline__ int64_t pos_to_y(const Digits& g, int n, int64_t p) {
  int64_t y = 0;
  int rem = n, sh = 0;
  for (int i = 0; i < g.count; ++i) {
    rem -= g.logr[i];
    const int64_t dig = (p >> rem) & ((int64_t(1) << g.logr[i]) - 1);
    y |= dig << sh;
    sh += g.logr[i];
  }
  return y;
}

__device__ __forceinline__ int64_t y_to_pos(const Digits& g, int n, int64_t y) {
  int64_t p = 0;
  int rem = n, sh = 0;
  for (int i = 0; i < g.count; ++i) {
    rem -= g.logr[i];
    const int64_t dig = (y >> sh) & ((int64_t(1) << g.logr[i]) - 1);
    p |= dig << rem;
    sh += g.logr[i];
  }
  return p;
}

template <typename C>
__device__ __forceinline__ void reduce_block(const C* __restrict__ X, double* __restrict__ hist,
                                             Partial* __restrict__ part_out, int64_t N, int logd, int n,
                                             const Digits& g, double scale, int64_t bidx, int64_t nblk) {
  const int d = 1 << logd;
  const int lpr = d < 32 ? d : 32;  // lanes per row
  const int rpw = 32 / lpr;         // rows per warp step
  const int per = d / lpr;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t gw = bidx * 8 + warp;
  const int64_t tw = nblk * 8;
  double best = -1.0, wsum = 0.0, psum = 0.0;
  int64_t by = INT64_MAX;
  // complex64 rows narrower than a warp (many rows): the per-row readout stays
  // off the FP64 units (float argmax, Kahan-compensated FP32 sums, bit-exact
  // widening of the stored value)
  const bool narrow32 = sizeof(C) == 8 && lpr < 32;
  float best_f = -1.f, wsum_f = 0.f, wcomp_f = 0.f, psum_f = 0.f, pcomp_f = 0.f;
  // rows of at most 64 bytes: one thread per outcome y, in y order (coalesced
  // histogram stores), reading the row at y's digit-reversed position (whole
  // 32-byte sectors); every lane runs the readout
  const bool per_y = d * (int)sizeof(C) <= 64;
  // Blocked digit reversal (at least two digits, the lowest of y >= 5 bits):
  // a tile is the outcomes y sharing their middle bits, 32 consecutive values
  // of y's lowest bits times K values of its highest digit. The rows are read
  // as K consecutive positions (y's highest digit is the position's lowest)
  // for each of the 32, |X|^2 goes through shared memory, and the bins are
  // written as 32 consecutive y for each of the K.
  const int lb = g.count >= 2 ? g.logr[g.count - 1] : 0;
  const bool blocked = per_y && g.count >= 2 && g.logr[0] >= 5 && blockDim.x == 256;
  if (blocked) {
    __shared__ double tile[32 * 129];
    float* tile_f = reinterpret_cast<float*>(tile);
    const int K = lb < 7 ? (1 << lb) : 128;
    const int kc_count = (1 << lb) / K;
    const int mid_bits = n - 5 - lb;
    const int64_t ntiles = (int64_t(kc_count)) << mid_bits;
    const int shift_hi = n - lb;
    for (int64_t t = bidx; t < ntiles; t += nblk) {
      const int kc = (int)(t % kc_count);
      const int64_t mbits = t / kc_count;
      const int64_t ybase = (mbits << 5);
      // reads: k fastest across the threads (consecutive positions)
      for (int e = threadIdx.x; e < 32 * K; e += 256) {
        const int k = e % K, ylo = e / K;
        const int64_t y = ybase + ylo + (int64_t(kc * K + k) << shift_hi);
        const C* row = X + (y_to_pos(g, n, y) << logd);
        if constexpr (sizeof(C) == 8) {
          float f = 0.f;
          for (int q = 0; q < d; ++q) {
            const C v = __ldg(row + q);
            f = fmaf(v.x, v.x, fmaf(v.y, v.y, f));
          }
          tile_f[ylo * 129 + k] = f * (float)scale;  // scale is a power of two
        } else {
          double acc = 0.0;
          for (int q = 0; q < d; ++q) {
            const C v = __ldg(row + q);
            acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
          }
          tile[ylo * 129 + k] = acc * scale;
        }
      }
      __syncthreads();
      // writes: 32 consecutive y across the threads
      for (int e = threadIdx.x; e < 32 * K; e += 256) {
        const int ylo = e & 31, k = e >> 5;
        const int64_t y = ybase + ylo + (int64_t(kc * K + k) << shift_hi);
        if constexpr (sizeof(C) == 8) {
          const float v = tile_f[ylo * 129 + k];
          hist[y] = widen_nonneg(v);
          if (v > best_f || (v == best_f && y < by)) {
            best_f = v;
            by = y;
          }
          float t1 = v * (float)y - wcomp_f;
          float t2 = wsum_f + t1;
          wcomp_f = (t2 - wsum_f) - t1;
          wsum_f = t2;
          t1 = v - pcomp_f;
          t2 = psum_f + t1;
          pcomp_f = (t2 - psum_f) - t1;
          psum_f = t2;
        } else {
          const double v = tile[ylo * 129 + k];
          hist[y] = v;
          better(best, by, v, y);
          wsum += v * (double)y;
          psum += v;
        }
      }
      __syncthreads();  // the tile is reused
    }
  } else if (per_y) {
    const int64_t tstep = nblk * blockDim.x;
    for (int64_t y = bidx * blockDim.x + threadIdx.x; y < N; y += tstep) {
      const C* row = X + (y_to_pos(g, n, y) << logd);
      if constexpr (sizeof(C) == 8) {
        float f = 0.f;
        for (int k = 0; k < d; ++k) {
          const C v = __ldg(row + k);
          f = fmaf(v.x, v.x, fmaf(v.y, v.y, f));
        }
        const float v = f * (float)scale;  // scale is a power of two
        hist[y] = widen_nonneg(v);
        if (v > best_f || (v == best_f && y < by)) {
          best_f = v;
          by = y;
        }
        float t1 = v * (float)y - wcomp_f;
        float t2 = wsum_f + t1;
        wcomp_f = (t2 - wsum_f) - t1;
        wsum_f = t2;
        t1 = v - pcomp_f;
        t2 = psum_f + t1;
        pcomp_f = (t2 - psum_f) - t1;
        psum_f = t2;
      } else {
        double acc = 0.0;
        for (int k = 0; k < d; ++k) {
          const C v = __ldg(row + k);
          acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
        const double v = acc * scale;
        hist[y] = v;
        better(best, by, v, y);
        wsum += v * (double)y;
        psum += v;
      }
    }
  }
  for (int64_t p0 = per_y ? N : gw * rpw; p0 < N; p0 += tw * rpw) {
    const int64_t p = p0 + lane / lpr;
    const int sub = lane % lpr;
    double acc = 0.0;
    float fsum = 0.f;  // complex64: this lane's FP32 partial of the row
    if (p < N) {
      const C* row = X + (p << logd);
      if constexpr (sizeof(C) == 8) {
        // complex64: squares and the lane's partial sum (d / 32 <= 128 terms) in
        // FP32 with Kahan compensation, two elements per 16-byte load when a
        // lane owns >= 2; the sum across rows (the readout) is FP64
        float f = 0.f;
        if (per >= 2) {
          float comp = 0.f;  // Kahan compensation of the running FP32 sum
          for (int k = 0; k < per; k += 2) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(row + 2 * sub + k * lpr));
            const float term = fmaf(v.x, v.x, v.y * v.y) + fmaf(v.z, v.z, v.w * v.w);
            const float y = term - comp;
            const float t = f + y;
            comp = (t - f) - y;
            f = t;
          }
        } else {
          const C v = row[sub];
          f = fmaf(v.x, v.x, v.y * v.y);
        }
        fsum = f;
      } else {
        for (int k = 0; k < per; ++k) {
          const C v = row[sub + k * lpr];
          acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
      }
    }
    // sum over the row's lanes (every lane takes part; lanes past N carry 0)
    if (sizeof(C) == 8 && lpr < 32) {
      // rows narrower than a warp (d < 32, many rows): in FP32 (<= 4 rounding
      // steps of nonnegative terms, < 3e-7 relative), off the FP64 units
      for (int off = lpr >> 1; off > 0; off >>= 1) fsum += __shfl_xor_sync(0xffffffffu, fsum, off);
      acc = (double)fsum;
    } else {
      if (sizeof(C) == 8) acc = (double)fsum;
      for (int off = lpr >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    }
    if (sub == 0 && p < N) {
      const int64_t y = pos_to_y(g, n, p);
      if (narrow32) {
        const float v = fsum * (float)scale;  // scale is a power of two
        hist[y] = widen_nonneg(v);
        if (v > best_f || (v == best_f && y < by)) {
          best_f = v;
          by = y;
        }
        float t1 = v * (float)y - wcomp_f;
        float t2 = wsum_f + t1;
        wcomp_f = (t2 - wsum_f) - t1;
        wsum_f = t2;
        t1 = v - pcomp_f;
        t2 = psum_f + t1;
        pcomp_f = (t2 - psum_f) - t1;
        psum_f = t2;
      } else {
        const double v = acc * scale;
        hist[y] = v;
        better(best, by, v, y);
        wsum += v * (double)y;
        psum += v;
      }
    }
  }
  if (narrow32 || (per_y && sizeof(C) == 8)) {
    best = best_f < 0.f ? -1.0 : widen_nonneg(best_f);
    wsum = (double)wsum_f;
    psum = (double)psum_f;
  }
  // warp then block reduction (fixed order: deterministic)
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int64_t oy = __shfl_xor_sync(0xffffffffu, by, off);
    better(best, by, ob, oy);
    wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
    psum += __shfl_xor_sync(0xffffffffu, psum, off);
  }
  __shared__ Partial sp[8];
  if (lane == 0) sp[warp] = Partial{best, by, wsum, psum};
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial r = sp[0];
    for (int w = 1; w < 8; ++w) {
      better(r.best, r.besty, sp[w].best, sp[w].besty);
      r.wsum += sp[w].wsum;
      r.psum += sp[w].psum;
    }
    *part_out = r;
  }
}

template <typename C>
__global__ void __launch_bounds__(256) reduce_kernel(const C* __restrict__ X, double* __restrict__ hist,
                                                     Partial* __restrict__ parts, int64_t N, int logd, int n,
                                                     Digits g, double scale) {
  pdl_begin();
  reduce_block<C>(X, hist, parts + blockIdx.x, N, logd, n, g, scale, blockIdx.x, gridDim.x);
}

// The histogram and readout partials of every listed instance: item i owns
// CTAs [tile0, tile0 + nblk) and its own partial slots.
template <typename C>
__global__ void __launch_bounds__(256) reduce_grouped_kernel(const RedItem<C>* __restrict__ items, int nitems) {
  pdl_begin();
  const int i = find_item(items, nitems, blockIdx.x);
  const RedItem<C>& it = items[i];
  const int64_t b = blockIdx.x - it.tile0;
  reduce_block<C>(it.X, it.hist, it.parts + b, it.N, it.logd, it.n, it.g, 1.0, b, it.nblk);
}

// Row 0 of every listed instance's state = 2^(-n/2) psi (one CTA each).
template <typename C>
__global__ void init_grouped_kernel(const InitItem<C>* __restrict__ items) {
  pdl_begin();
  const InitItem<C> it = items[blockIdx.x];
  for (int i = threadIdx.x; i < it.d; i += blockDim.x) {
    const double2 v = it.psi[i];
    it.S[i] = to_c(make_double2(v.x * it.scale, v.y * it.scale), (C*)nullptr);
  }
}

__global__ void __launch_bounds__(256) finalize_kernel(const Partial* __restrict__ parts, int count,
                                                       Scalars* __restrict__ out, int n) {
  pdl_begin();
  const Partial m = reduce_partials_256(parts, count);
  if (threadIdx.x == 0) {
    const double N = ldexp(1.0, n);
    Scalars s;
    s.argmax = m.besty;
    s.phase_argmax = (double)m.besty / N;
    s.phase_mean = m.wsum / N;
    s.total = m.psum;
    s.best = m.best;
    s.err = readout_finite(m) ? 0 : (int)QPE_ERR_NUMERIC;
    s.pad = 0;
    *out = s;
  }
}

template <typename C>
__global__ void unpermute_kernel(const C* __restrict__ X, C* __restrict__ out, int64_t N, int logd, int n,
                                 Digits g) {
  pdl_begin();
  const int64_t total = N << logd;
  const int64_t dmask = (int64_t(1) << logd) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i >> logd;
    out[i] = X[(y_to_pos(g, n, y) << logd) | (i & dmask)];
  }
}

inline int grid_for(int64_t work, int threads, int cap = 152 * 16) {
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

inline int ilog2(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}

template <typename C>
C* at(char* ws, size_t off) {
  return reinterpret_cast<C*>(ws + off);
}

Digits digits_of(const FftPlan& f) {
  Digits g;
  g.count = f.passes;
  for (int i = 0; i < kMaxPasses; ++i) g.logr[i] = i < f.passes ? f.logr_list[i] : 0;
  return g;
}

}  // namespace

// ------------------------------------------------------ sharded plain schedule
// Rank r of G = 2^sh holds the rows m = r + G i (i < N / G). Its local state
// after the controlled gates is row i = 2^(-n/2) U^(r + G i) psi; the local
// QFT^-1 passes give F_r[y'] = 2^(-n/2) sum_i w_(N/G)^(i y') S[r + G i] for
// y' < N / G (positions in digit order), and
//   X[y' + (N / G) q] = sum_r w_G^(r q) (w_N^(r y') F_r[y']),
// one length-G DFT across the ranks per (y', column). The pack kernel forms
// w_N^(r y') F_r[y'] and sorts it by the rank that owns y' (y' = s mod G):
// send[s][y' >> sh][t]. After the all-to-all, rank s holds recv[r][i][t] =
// w_N^(r y') F_r[y'] for y' = s + G i, and the combine kernel runs the G-point
// DFTs, the |.|^2 sums over t and the readout of its outcomes
// y = s + G (i + (N / G^2) q).
template <typename C>
__global__ void __launch_bounds__(256) shard_pack_kernel(const C* __restrict__ F, C* __restrict__ send, int64_t nloc,
                                                         int logd, int nloc_bits, int sh, int rank, Digits g,
                                                         const C* __restrict__ tw_lo, const C* __restrict__ tw_hi,
                                                         int htw, int n) {
  pdl_begin();
  const int64_t total = nloc << logd;
  const int64_t per_peer = nloc >> sh;
  const int64_t dmask = (int64_t(1) << logd) - 1;
  const int64_t nmask = (int64_t(1) << n) - 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e >> logd, t = e & dmask;
    const int64_t yp = pos_to_y(g, nloc_bits, p);
    C v = F[e];
    const int64_t ex = ((int64_t)rank * yp) & nmask;
    if (ex) v = cmul(v, twiddle(tw_lo, tw_hi, htw, ex));
    const int64_t dest = yp & ((int64_t(1) << sh) - 1);
    send[((dest * per_peer + (yp >> sh)) << logd) + t] = v;
  }
  pdl_trigger();
}

// One warp per local row i of this rank's outcomes; G-point DFT over the
// source ranks for every column, |.|^2 summed over the columns.
template <typename C>
__global__ void __launch_bounds__(256) shard_combine_kernel(const C* __restrict__ recv, double* __restrict__ hist,
                                                            Partial* __restrict__ parts, int64_t per_peer, int logd,
                                                            int sh, int rank, int n, const C* __restrict__ tw_lo,
                                                            const C* __restrict__ tw_hi, int htw) {
  pdl_begin();
  const int d = 1 << logd, G = 1 << sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double best = -1.0, wsum = 0.0, psum = 0.0;
  int64_t by = INT64_MAX;
  const int64_t warps = (int64_t)gridDim.x * 8;
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < per_peer; i += warps) {
    for (int q = 0; q < G; ++q) {
      double acc = 0.0;
      for (int t = lane; t < d; t += 32) {
        C x = mk((typename real_of<C>::type)0, (typename real_of<C>::type)0);
        for (int r = 0; r < G; ++r) {
          const C v = recv[(((int64_t)r * per_peer + i) << logd) + t];
          const int64_t ex = (int64_t)((r * q) & (G - 1)) << (n - sh);  // w_G^(r q) = w_N^(r q N / G)
          x = cadd(x, ex ? cmul(v, twiddle(tw_lo, tw_hi, htw, ex)) : v);
        }
        acc += (double)x.x * (double)x.x + (double)x.y * (double)x.y;
      }
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) {
        const int64_t j = i + per_peer * q;
        const int64_t y = rank + ((int64_t)j << sh);
        hist[j] = acc;
        better(best, by, acc, y);
        wsum += acc * (double)y;
        psum += acc;
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int64_t oy = __shfl_xor_sync(0xffffffffu, by, off);
    better(best, by, ob, oy);
    wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
    psum += __shfl_xor_sync(0xffffffffu, psum, off);
  }
  __shared__ Partial sp[8];
  if (lane == 0) sp[warp] = Partial{best, by, wsum, psum};
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial r = sp[0];
    for (int w = 1; w < 8; ++w) merge_partial(r, sp[w]);
    parts[blockIdx.x] = r;
  }
  pdl_trigger();
}

// ============================================================ launchers
int launch_twiddles(const Instance& in, char* ws, cudaStream_t s) {
  const int64_t total = (int64_t(1) << in.htw) + (int64_t(1) << (in.nmeas - in.htw));
  const cudaError_t e = launch_k(twiddle_tables_kernel, dim3(grid_for(total, 256)), dim3(256), 0, s,
                                 at<double2>(ws, in.off_tw_lo64), at<double2>(ws, in.off_tw_hi64),
                                 at<float2>(ws, in.off_tw_lo32), at<float2>(ws, in.off_tw_hi32), in.nmeas, in.htw);
  return e == cudaSuccess ? 1 : -1;
}

static int launch_square(const double2* A, double2* C, int d, float2* C32, float2* A32, cudaStream_t s) {
  cudaError_t e;
  switch (d) {
    case 2: e = launch_k(square_small_kernel<2, 2>, dim3(1, 1), dim3(8), 0, s, A, C, d, C32, A32); break;
    case 4: e = launch_k(square_small_kernel<4, 4>, dim3(1, 1), dim3(64), 0, s, A, C, d, C32, A32); break;
    case 8: e = launch_k(square_small_kernel<4, 8>, dim3(2, 2), dim3(128), 0, s, A, C, d, C32, A32); break;
    case 16: e = launch_k(square_small_kernel<4, 16>, dim3(4, 4), dim3(256), 0, s, A, C, d, C32, A32); break;
    case 32: e = launch_k(square_small_kernel<4, 16>, dim3(8, 8), dim3(256), 0, s, A, C, d, C32, A32); break;
    case 64: e = launch_k(square_small_kernel<4, 16>, dim3(16, 16), dim3(256), 0, s, A, C, d, C32, A32); break;
    case 128: e = launch_k(square_small_kernel<8, 4>, dim3(16, 16), dim3(256), 0, s, A, C, d, C32, A32); break;
    case 256: e = launch_k(square_small_kernel<8, 4>, dim3(32, 32), dim3(256), 0, s, A, C, d, C32, A32); break;
    default: e = launch_k(square_tiled_kernel, dim3(d / 32, d / 32), dim3(256), 0, s, A, C, d, C32, A32); break;
  }
  return e == cudaSuccess ? 1 : -1;
}

int launch_check_unitary(const Instance& in, char* ws, cudaStream_t s) {
  const unsigned t = (unsigned)((in.d + 15) / 16);
  return launch_k(unitarity_kernel, dim3(t, t), dim3(256), 0, s, (const double2*)at<double2>(ws, in.off_pow64),
                  (int)in.d, 1e-8, at<int>(ws, in.off_err)) == cudaSuccess
             ? 1
             : -1;
}

int launch_powers(const Instance& in, char* ws, bool want_c64, cudaStream_t s) {
  const int64_t dd = in.d * in.d;
  double2* P = at<double2>(ws, in.off_pow64);
  float2* P32 = want_c64 ? at<float2>(ws, in.off_pow32) : nullptr;
  int launches = 0;
  for (int k = 1; k < in.nmeas; ++k) {
    // complex64 copies ride along: P_k from the squaring that makes it, P_0 from the first one
    if (in.oz_square) {
      const int r = launch_square_oz(in, ws, k, want_c64, s);
      if (r < 0) return -1;
      launches += r;
      continue;
    }
    if (launch_square(P + (k - 1) * dd, P + k * dd, (int)in.d, P32 ? P32 + k * dd : nullptr,
                      (P32 && k == 1) ? P32 : nullptr, s) < 0)
      return -1;
    ++launches;
  }
  if (want_c64 && in.nmeas == 1) {
    if (launch_k(convert_c128_to_c64_kernel, dim3(grid_for(dd, 256)), dim3(256), 0, s, (const double2*)P, P32,
                 dd) != cudaSuccess)
      return -1;
    ++launches;
  }
  return launches;
}

template <typename C, typename Rows>
static int launch_rows_times_pt(C* S, const C* P, int64_t M, int d, Rows rows, cudaStream_t s) {
  if (M <= 0) return 0;
  cudaError_t err = cudaSuccess;
#define QPE_GEMM(BM, BN, BK, TM, TN)                                                          \
  do {                                                                                        \
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)(d / BN));                              \
    err = launch_k(rows_times_pt_kernel<C, BM, BN, BK, TM, TN, Rows>, grid, dim3((BM / TM) * (BN / TN)), 0, s, \
                   S, P, M, d, rows);                                                                      \
  } while (0)
  switch (d) {
    case 2: QPE_GEMM(256, 2, 2, 2, 1); break;
    case 4: QPE_GEMM(256, 4, 4, 4, 1); break;
    case 8: QPE_GEMM(256, 8, 8, 4, 2); break;
    case 16: QPE_GEMM(256, 16, 8, 4, 4); break;
    case 32: QPE_GEMM(128, 32, 8, 4, 4); break;
    default: QPE_GEMM(64, 64, 8, 4, 4); break;
  }
#undef QPE_GEMM
  return err == cudaSuccess ? 1 : -1;
}

template <typename C>
int launch_sweep(const Instance& in, char* ws, bool gate_mode, cudaStream_t s, int prec) {
  const bool tc = prec == QPE_C64_TF32X3 || prec == QPE_C64_FP16X2;
  C* S = at<C>(ws, in.off_state);
  const C* P = (sizeof(C) == 16) ? at<C>(ws, in.off_pow64) : at<C>(ws, in.off_pow32);
  const int64_t dd = in.d * in.d;
  const int logd = in.nmat;
  const double scale = 1.0 / sqrt(ldexp(1.0, in.nmeas));  // Hadamard layer: 2^(-n/2)
  int launches = 0;
  const int64_t init_rows = gate_mode ? in.N : 1;
  if (launch_k(init_rows_kernel<C>, dim3(grid_for(init_rows << logd, 256)), dim3(256), 0, s, S,
               (const double2*)at<double2>(ws, in.off_psi), init_rows, logd, scale) != cudaSuccess)
    return -1;
  ++launches;
  if (in.shard_log > 0) {
    // rank r: rows 0 .. G-1 = U^m psi (m < G) by the doubling of the low sh
    // measurement qubits, row r moved to row 0, then the doubling of the high
    // n - sh qubits over the local rows (local row i = U^(r + G i) psi)
    const int sh = in.shard_log;
    for (int j = 0; j < sh; ++j) {
      const int r = launch_rows_times_pt<C>(S, P + j * dd, int64_t(1) << j, (int)in.d, DoublingRows{int64_t(1) << j}, s);
      if (r < 0) return -1;
      launches += r;
    }
    if (in.shard_rank != 0 &&
        cudaMemcpyAsync(S, S + ((int64_t)in.shard_rank << logd), sizeof(C) << logd, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
      return -1;
    for (int j = 0; j < in.nmeas - sh; ++j) {
      int r;
      if (tc && in.d >= 32 && (int64_t(1) << j) >= 128)
        r = launch_tc_level(in, ws, prec, j, s, sh);
      else if (sizeof(C) == 16 && in.oz_gates && (int64_t(1) << j) >= 128)
        r = launch_oz_gate_level(in, ws, j, sh, s);
      else
        r = launch_rows_times_pt<C>(S, P + (j + sh) * dd, int64_t(1) << j, (int)in.d, DoublingRows{int64_t(1) << j},
                                    s);
      if (r < 0) return -1;
      launches += r;
    }
    return launches;
  }
  const bool repeat_u = prec < 0;  // controlled-U applied 2^j times (gate schedule only)
  for (int j = 0; j < in.nmeas; ++j) {
    int r = 0;
    if (gate_mode && repeat_u) {
      for (int64_t rep = 0; rep < (int64_t(1) << j); ++rep) {
        const int rr = launch_rows_times_pt<C>(S, P, in.N / 2, (int)in.d, GateRows{j}, s);
        if (rr < 0) return -1;
        r += rr;
      }
    } else if (gate_mode)
      r = launch_rows_times_pt<C>(S, P + j * dd, in.N / 2, (int)in.d, GateRows{j}, s);
    else if (tc && in.d >= 32 && (int64_t(1) << j) >= 128)
      r = launch_tc_level(in, ws, prec, j, s);  // tensor cores once a level fills 128-row tiles
    else if (sizeof(C) == 16 && in.oz_gates && (int64_t(1) << j) >= 128)
      r = launch_oz_gate_level(in, ws, j, 0, s);  // FP64: exact digit products on the tensor cores
    else
      r = launch_rows_times_pt<C>(S, P + j * dd, int64_t(1) << j, (int)in.d, DoublingRows{int64_t(1) << j}, s);
    if (r < 0) return -1;
    launches += r;
  }
  return launches;
}

FftPlan make_fft_plan(int nmeas, int64_t d, size_t esize) {
  FftPlan f;
  const int logd = ilog2(d);
  const int logwmax = ilog2((int64_t)(128 / esize));  // 128-byte column slabs
  const int max_bits = 9;                            // R * W * esize <= 64 KiB
  const int passes = (nmeas + max_bits - 1) / max_bits;
  f.passes = passes;
  int used = 0;
  for (int i = 0; i < passes; ++i) {
    const int r = nmeas / passes + (i < nmeas % passes ? 1 : 0);
    FftPass& p = f.p[i];
    p.logr = r;
    p.B = int64_t(1) << used;
    used += r;
    p.L = int64_t(1) << (nmeas - used);
    p.Q = p.L * d;
    const int logq = ilog2(p.Q);
    const int logw = logq < logwmax ? logq : logwmax;
    p.W = int64_t(1) << logw;
    f.logr_list[i] = r;
    (void)logd;
  }
  return f;
}

int64_t fft_position_to_y(const FftPlan& f, int nmeas, int64_t p) {
  int64_t y = 0;
  int rem = nmeas, sh = 0;
  for (int i = 0; i < f.passes; ++i) {
    rem -= f.logr_list[i];
    const int64_t dig = (p >> rem) & ((int64_t(1) << f.logr_list[i]) - 1);
    y |= dig << sh;
    sh += f.logr_list[i];
  }
  return y;
}

FftArgs fft_pass_args(const Instance& in, int i, int64_t* blocks, size_t* smem, size_t esize) {
  const FftPass& p = in.fft.p[i];
  FftArgs a;
  a.logr = p.logr;
  a.logw = ilog2(p.W);
  a.logq = ilog2(p.Q);
  a.logd = in.nmat;
  a.n = in.nmeas - in.shard_log;  // a sharded plan transforms its N / 2^shard_log local rows
  a.tw_sh = in.shard_log;
  a.htw = in.htw;
  a.logb = ilog2(p.B);
  a.last = (i == in.fft.passes - 1);
  a.scale = a.last ? 1.0 / sqrt(ldexp(1.0, in.nmeas)) : 1.0;  // QFT^-1 normalisation 2^(-n/2) in the last pass
  *blocks = p.B * (p.Q / p.W);
  *smem = ((size_t)(int64_t(1) << p.logr) * p.W + ((size_t)1 << p.logr) / 2) * esize;
  return a;
}

template <typename C>
int launch_fft(const Instance& in, char* ws, cudaStream_t s) {
  C* X = at<C>(ws, in.off_state);
  const C* lo = (sizeof(C) == 16) ? at<C>(ws, in.off_tw_lo64) : at<C>(ws, in.off_tw_lo32);
  const C* hi = (sizeof(C) == 16) ? at<C>(ws, in.off_tw_hi64) : at<C>(ws, in.off_tw_hi32);
  int launches = 0;
  for (int i = 0; i < in.fft.passes; ++i) {
    int64_t blocks = 0;
    size_t smem = 0;
    const FftArgs a = fft_pass_args(in, i, &blocks, &smem, sizeof(C));
    if (launch_k(fft_pass_kernel<C>, dim3((unsigned)blocks), dim3(256), smem, s, X, lo, hi, a) != cudaSuccess)
      return -1;
    ++launches;
  }
  return launches;
}

Digits fft_digits(const FftPlan& f) { return digits_of(f); }

int64_t reduce_blocks(const Instance& in) {
  const int64_t rows_per_block_step = 8 * (32 / (in.d < 32 ? in.d : 32));
  const int64_t b = std::min<int64_t>(kReduceBlocks, (in.N + rows_per_block_step - 1) / rows_per_block_step);
  return b < 1 ? 1 : b;
}

void doubling_tile(int d, int* BM, int* BN) {
  switch (d) {
    case 2: *BM = 256; *BN = 2; break;
    case 4: *BM = 256; *BN = 4; break;
    case 8: *BM = 256; *BN = 8; break;
    case 16: *BM = 256; *BN = 16; break;
    case 32: *BM = 128; *BN = 32; break;
    default: *BM = 64; *BN = 64; break;
  }
}

template <typename C>
int launch_init_grouped(const InitItem<C>* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return 0;
  return launch_k(init_grouped_kernel<C>, dim3((unsigned)nitems), dim3(256), 0, s, items) == cudaSuccess ? 1 : -1;
}

// one doubling round for the items of one tile class (d, or 64 for d >= 64)
template <typename C>
int launch_doubling_grouped(const DblItem<C>* items, int nitems, int64_t tiles, int dclass, cudaStream_t s) {
  if (nitems <= 0) return 0;
  cudaError_t e;
  switch (dclass) {
    case 2: e = launch_k(doubling_grouped_kernel<C, 256, 2, 2, 2, 1>, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems); break;
    case 4: e = launch_k(doubling_grouped_kernel<C, 256, 4, 4, 4, 1>, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems); break;
    case 8: e = launch_k(doubling_grouped_kernel<C, 256, 8, 8, 4, 2>, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems); break;
    case 16: e = launch_k(doubling_grouped_kernel<C, 256, 16, 8, 4, 4>, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems); break;
    case 32: e = launch_k(doubling_grouped_kernel<C, 128, 32, 8, 4, 4>, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems); break;
    default: e = launch_k(doubling_grouped_kernel<C, 64, 64, 8, 4, 4>, dim3((unsigned)tiles), dim3(256), 0, s, items, nitems); break;
  }
  return e == cudaSuccess ? 1 : -1;
}

template <typename C>
int launch_fft_grouped(const FftItem<C>* items, int nitems, int64_t blocks, size_t smem, cudaStream_t s) {
  if (nitems <= 0) return 0;
  return launch_k(fft_pass_grouped_kernel<C>, dim3((unsigned)blocks), dim3(256), smem, s, items, nitems) ==
                 cudaSuccess
             ? 1
             : -1;
}

template <typename C>
int launch_reduce_grouped(const RedItem<C>* items, int nitems, int64_t blocks, cudaStream_t s) {
  if (nitems <= 0) return 0;
  return launch_k(reduce_grouped_kernel<C>, dim3((unsigned)blocks), dim3(256), 0, s, items, nitems) == cudaSuccess
             ? 1
             : -1;
}

template <typename C>
int launch_shard_pack(const Instance& in, char* ws, cudaStream_t s) {
  const int nb = in.nmeas - in.shard_log;
  const int64_t nloc = int64_t(1) << nb;
  const C* lo = (sizeof(C) == 16) ? at<C>(ws, in.off_tw_lo64) : at<C>(ws, in.off_tw_lo32);
  const C* hi = (sizeof(C) == 16) ? at<C>(ws, in.off_tw_hi64) : at<C>(ws, in.off_tw_hi32);
  return launch_k(shard_pack_kernel<C>, dim3(grid_for(nloc << in.nmat, 256)), dim3(256), 0, s,
                  (const C*)at<C>(ws, in.off_state), at<C>(ws, in.off_send), nloc, in.nmat, nb, in.shard_log,
                  in.shard_rank, digits_of(in.fft), lo, hi, in.htw, in.nmeas) == cudaSuccess
             ? 1
             : -1;
}

template <typename C>
int launch_shard_combine(const Instance& in, char* ws, cudaStream_t s, int* blocks_out) {
  const int64_t per_peer = int64_t(1) << (in.nmeas - 2 * in.shard_log);
  const C* lo = (sizeof(C) == 16) ? at<C>(ws, in.off_tw_lo64) : at<C>(ws, in.off_tw_lo32);
  const C* hi = (sizeof(C) == 16) ? at<C>(ws, in.off_tw_hi64) : at<C>(ws, in.off_tw_hi32);
  int blocks = (int)std::min<int64_t>(kReduceBlocks, (per_peer + 7) / 8);
  if (blocks < 1) blocks = 1;
  *blocks_out = blocks;
  return launch_k(shard_combine_kernel<C>, dim3(blocks), dim3(256), 0, s, (const C*)at<C>(ws, in.off_recv),
                  at<double>(ws, in.off_hist), at<Partial>(ws, in.off_partials), per_peer, in.nmat, in.shard_log,
                  in.shard_rank, in.nmeas, lo, hi, in.htw) == cudaSuccess
             ? 1
             : -1;
}

template <typename C>
int launch_reduce(const Instance& in, char* ws, cudaStream_t s) {
  const Digits g = digits_of(in.fft);
  const int64_t rows_per_block_step = 8 * (32 / (in.d < 32 ? in.d : 32));
  int blocks = (int)std::min<int64_t>(kReduceBlocks, (in.N + rows_per_block_step - 1) / rows_per_block_step);
  if (blocks < 1) blocks = 1;
  if (launch_k(reduce_kernel<C>, dim3(blocks), dim3(256), 0, s, (const C*)at<C>(ws, in.off_state),
               at<double>(ws, in.off_hist), at<Partial>(ws, in.off_partials), in.N, in.nmat, in.nmeas, g,
               1.0) != cudaSuccess)
    return -1;
  if (launch_finalize(in, ws, blocks, s) < 0) return -1;
  return 2;
}

int launch_finalize(const Instance& in, char* ws, int count, cudaStream_t s) {
  return launch_k(finalize_kernel, dim3(1), dim3(256), 0, s, (const Partial*)at<Partial>(ws, in.off_partials), count,
                  at<Scalars>(ws, in.off_scalars), in.nmeas) == cudaSuccess
             ? 1
             : -1;
}

template <typename C>
int launch_unpermute(const Instance& in, const char* ws, void* out, cudaStream_t s) {
  const Digits g = digits_of(in.fft);
  return launch_k(unpermute_kernel<C>, dim3(grid_for(in.N * in.d, 256)), dim3(256), 0, s,
                  reinterpret_cast<const C*>(ws + in.off_state), reinterpret_cast<C*>(out), in.N, in.nmat, in.nmeas,
                  g) == cudaSuccess
             ? 1
             : -1;
}

// Dynamic shared memory above 48 KiB needs an opt-in per kernel.
cudaError_t configure_kernels() {
  cudaError_t e = configure_level_kernels();
  if (e != cudaSuccess) return e;
  // tile (<= 64 KiB) + the pass's twiddles (<= 256 entries)
  e = cudaFuncSetAttribute(fft_pass_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024 + 4096);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fft_pass_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024 + 4096);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fft_pass_grouped_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           64 * 1024 + 4096);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fft_pass_grouped_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              64 * 1024 + 4096);
}

template int launch_sweep<float2>(const Instance&, char*, bool, cudaStream_t, int);
template int launch_sweep<double2>(const Instance&, char*, bool, cudaStream_t, int);
template int launch_fft<float2>(const Instance&, char*, cudaStream_t);
template int launch_fft<double2>(const Instance&, char*, cudaStream_t);
template int launch_reduce<float2>(const Instance&, char*, cudaStream_t);
#define QPE_GROUPED_INST(C)                                                                             \
  template int launch_init_grouped<C>(const InitItem<C>*, int, cudaStream_t);                          \
  template int launch_doubling_grouped<C>(const DblItem<C>*, int, int64_t, int, cudaStream_t);         \
  template int launch_fft_grouped<C>(const FftItem<C>*, int, int64_t, size_t, cudaStream_t);           \
  template int launch_reduce_grouped<C>(const RedItem<C>*, int, int64_t, cudaStream_t);
QPE_GROUPED_INST(float2)
QPE_GROUPED_INST(double2)
#undef QPE_GROUPED_INST
template int launch_shard_pack<float2>(const Instance&, char*, cudaStream_t);
template int launch_shard_pack<double2>(const Instance&, char*, cudaStream_t);
template int launch_shard_combine<float2>(const Instance&, char*, cudaStream_t, int*);
template int launch_shard_combine<double2>(const Instance&, char*, cudaStream_t, int*);
template int launch_reduce<double2>(const Instance&, char*, cudaStream_t);
template int launch_unpermute<float2>(const Instance&, const char*, void*, cudaStream_t);
template int launch_unpermute<double2>(const Instance&, const char*, void*, cudaStream_t);

}  // namespace qpe
