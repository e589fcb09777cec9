// FP64 levels of the fused schedule on the tcgen05 tensor cores, d = 16 and
// 8-point levels (QPE_FLAG_LEVEL_TC with QPE_FP64), with the accuracy of FP64
// arithmetic.
//
// A level takes, for every pencil y_a, the level below's Z[y_a] (16 complex
// values) and forms T[m_b][i] = sum_k M[m_b][i][k] Z[y_a][k] for m_b < 8
// (M[m_b] the level's table) and X[y_a + N_a y_b][i] = sum_(m_b)
// w_8^(m_b y_b) (w_N'^(m_b y_a) T[m_b][i]). The top level (MODE 1) keeps only
// the histogram bin sum_i |X|^2 / N^2 and the readout; a lower level (MODE 0)
// writes X, the next level's Z.
//
// The contraction is one real product per tile of 128 pencils: A = the Z rows
// (K = 32 reals, re / im interleaved), B = the table's real embedding with
// rows n = 16 i + 2 m_b + c (c: re / im of T). Both are split into 7 balanced
// 8-bit digits (the Ozaki scheme): A per pencil at its own power-of-two scale
// 2^tau, B at one scale 2^sigma, x = 2^(tau - 55) sum_(s<7) a_s 2^(8 (6 - s)),
// |a_s| <= 128 (exact in bf16). The 28 digit pairs (s, t) of weight
// w = s + t <= 6 are formed; a pair's products are integers of at most 2^14,
// so a weight's accumulator (w + 1 pairs over K = 32) stays below 2^22 and is
// exact in FP32. With acc_w the weight sums,
//   T = 2^(tau + sigma - 62) E,  E = sum_w acc_w 2^(8 (6 - w)),
// |T| < 32 2^(tau + sigma), so |E| < 2^67. The omitted digit pairs and the
// digit rounding lie at 2^-53 of |Z| |M| K, the error bound of an FP64 dot
// product.
//
// GB300 issues an FP64 instruction at 1/32 of the rate of a 32-bit integer
// one, so the epilogue stays in 64-bit fixed point until |X|^2: the drain
// reads each accumulator as an int (a magic-number addition in FP32), forms
// W = floor(E / 2^10) (|W| < 2^57 + 1, units 2^(tau + sigma - 52)),
// multiplies by the twiddles held in Q61 (round(w 2^61), split at bit 31 into
// int32 halves so that every partial product is one 32 x 32 -> 64-bit
// multiply-add; at most 3 units off), runs the 8-point DFT on the integers
// (|X| < 8 sqrt(2) 2^57 < 2^61; the factor cos(pi / 4) also in Q61) and turns
// X into FP64 (the hardware conversion, rounded to nearest; the unit's power
// of two goes into the exponent bits, or, for |X|^2, into the histogram's
// scale once per tile). The fixed point's truncations are a few units, 2^-55
// of the pencil's bound |T| < 2^(tau + sigma + 5), below the contraction's
// own error. |X|^2 and the readout run in FP64; a lower level (MODE 0) stores
// X in FP64.
//
// Roles (640 threads, one CTA per SM, persistent over the tiles):
//   warps 0-2   producers: Z rows -> digit tiles (shared memory, 128-byte
//               swizzled K-major, two digits per 128-byte row), two threads
//               per pencil (eight complex values each); the pencils'
//               twiddles w_N^(m_b y_a) and scales (two buffers);
//   warp 3      tensor memory, and lane 0 issues the MMAs and the table's
//               copies: per chunk of two columns i (32 table rows), 28 pairs
//               x 2 K-steps of M = 128, N = 32 into seven weight accumulators
//               (224 columns; two chunk buffers, even chunks in one, odd in
//               the other); the digits of two tiles in shared memory (the
//               producers run a tile ahead) and the table's chunk images
//               streamed from L2 through a four-stage ring (bulk copies);
//   warps 4-19  drain: four warps per tensor-memory lane quarter (four per
//               SM sub-partition, for the integer epilogue's latencies),
//               warp k takes column 2 c + (k & 1) of the chunks
//               c with c & 1 = k >> 1; weights -> fixed point, twiddle, DFT,
//               FP64, then |X|^2 (the four warps' sums meet through tensor
//               memory columns 448-495) or the store of X.
// Every wait is a bounded mbarrier wait; an expired wait sets QPE_ERR_TIMEOUT.
#include "qpe_internal.cuh"
#include "qpe_tcgen05.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace qpe {
using namespace tcg;

namespace {

constexpr int kOtL = 8, kOtD = 16, kOtS = 7;
constexpr int kOtRows = 128;                   // pencils per tile (MMA M)
constexpr int kOtN = 2 * kOtD * kOtL;          // 256 table rows
constexpr int kOtChunks = kOtD / 2;            // two columns i (32 table rows) per chunk
constexpr int kOtThreads = 640;
constexpr int kOtProducers = 96;
constexpr uint32_t kOtSlabA = kOtRows * 128;   // digits [2q | 2q+1] of 128 pencils, 16 KiB
constexpr uint32_t kOtBSlab = 32 * 128;        // digits [2q | 2q+1] of one chunk's 32 rows, 4 KiB
constexpr uint32_t kOtBChunk = 4 * kOtBSlab;   // one chunk's seven digits, 16 KiB
constexpr int kOtBStages = 4;                  // ring of table chunks
constexpr uint32_t kOtBufCols = kOtS * 32;     // one chunk's seven weight accumulators (two buffers)
constexpr uint32_t kOtSqCol = 2 * kOtBufCols;  // columns 448 .. 495: the hand-over of the partial sums
constexpr size_t kOtBBytes = (size_t)kOtChunks * kOtBChunk;  // the table's image in global memory, 128 KiB
constexpr size_t kOtABytes = 4 * (size_t)kOtSlabA;           // one tile's digits (two buffers)
constexpr size_t kOtTwBytes = (size_t)kOtRows * (kOtL - 1) * sizeof(int4);
constexpr size_t kOtSmem =
    2 * kOtABytes + kOtBStages * (size_t)kOtBChunk + 2 * kOtTwBytes + 2 * kOtRows * sizeof(int) + 1024;
static_assert(kOtSmem <= 227 * 1024, "shared memory of the FP64 top level");

// v 2^e for an FP64 v that is zero or normal, by adding e to the exponent
// field; results below 2^-1022 flush to 0
__device__ __forceinline__ double ot_scale2(double v, int e) {
  const long long b = __double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ff);
  return (E == 0 || E + e <= 0) ? 0.0 : __longlong_as_double(b + ((long long)e << 52));
}

// A weight accumulator (an exact integer |acc| < 2^22 in FP32) plus 1.5 2^23
// in FP32 is exact and has the bits acc + M, M = 0x4B400000.
__device__ __forceinline__ uint32_t ot_acc_bits(uint32_t u) {
  return __float_as_uint(__fadd_rn(__uint_as_float(u), 12582912.0f));
}

// The drain's fixed point W = floor(E / 2^10) of one T component from its
// seven weight sums, E = sum_w acc_w 2^(8 (6 - w)), T = 2^(tau + sigma - 62) E.
// With b_w = acc_w + M, the low part acc_5 2^8 + acc_6 = b_5 2^8 + b_6 - 257 M
// (exact in int32), and the rest sum_(w<5) b_w 2^(8 (6 - w) - 10) minus
// M sum_(w<5) 2^(8 (6 - w) - 10), modulo 2^64 (W itself fits).
__device__ __forceinline__ long long ot_weights_fix(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3, uint32_t u4,
                                                    uint32_t u5, uint32_t u6) {
  constexpr unsigned long long kMW = 0xe2e2e2e2d0000000ull;  // M (2^38 + 2^30 + 2^22 + 2^14 + 2^6) mod 2^64
  const int r = (int)(ot_acc_bits(u5) * 256u + ot_acc_bits(u6) - 0x8b400000u) >> 10;  // 257 M mod 2^32
  unsigned long long w = (unsigned long long)(long long)r - kMW;
  w += (unsigned long long)ot_acc_bits(u4) * 64u;
  w += (unsigned long long)ot_acc_bits(u3) * 16384u;
  w += (unsigned long long)ot_acc_bits(u2) * 4194304u;
  w += (unsigned long long)ot_acc_bits(u1) * 1073741824u;
  w += (unsigned long long)(ot_acc_bits(u0) * 64u) << 32;
  return (long long)w;
}

// (wr + i wi) (qr + i qi) 2^-61 for a twiddle in Q61 (q = round(w 2^61)),
// with both operands split at bit 31 (h = x >> 31, l = x mod 2^31): the
// products l l 2^-61 (below 2) are dropped and the middle sum is floored.
// q = (qr h, qr l, qi h, qi l).
__device__ __forceinline__ void ot_tw_fix(long long& wr, long long& wi, int4 q) {
  const int rh = (int)(wr >> 31), rl = (int)(wr & 0x7fffffff);
  const int ih = (int)(wi >> 31), il = (int)(wi & 0x7fffffff);
  const long long sr = (long long)rh * q.y + (long long)rl * q.x - (long long)ih * q.w - (long long)il * q.z;
  const long long si = (long long)rh * q.w + (long long)rl * q.z + (long long)ih * q.y + (long long)il * q.x;
  wr = 2 * ((long long)rh * q.x - (long long)ih * q.z) + (sr >> 30);
  wi = 2 * ((long long)rh * q.z + (long long)ih * q.x) + (si >> 30);
}

// x cos(pi / 4) in the same fixed point (cos(pi / 4) 2^61 rounded, split as in
// ot_tw_fix)
__device__ __forceinline__ long long ot_rot_fix(long long x) {
  constexpr long long kC = 1630477228166597777LL;  // round(2^61 / sqrt(2))
  constexpr int ch = (int)(kC >> 31), cl = (int)(kC & 0x7fffffff);
  const int xh = (int)(x >> 31), xl = (int)(x & 0x7fffffff);
  return 2 * ((long long)xh * ch) + (((long long)xh * cl + (long long)xl * ch) >> 30);
}

// 8-point DFT X[k] = sum_n x[n] exp(-2 pi i n k / 8) on fixed-point values
// (re, im interleaved: x[2 n], x[2 n + 1]), natural order in and out (radix-2
// decimation in frequency; -i by exchange, (+-1 - i) / sqrt 2 by ot_rot_fix)
__device__ __forceinline__ void ot_dft8_fix(long long (&x)[16]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const long long ur = x[2 * p], ui = x[2 * p + 1], vr = x[2 * p + 8], vi = x[2 * p + 9];
    x[2 * p] = ur + vr;
    x[2 * p + 1] = ui + vi;
    const long long dr = ur - vr, di = ui - vi;
    if (p == 0) { x[8] = dr; x[9] = di; }
    if (p == 1) { x[10] = ot_rot_fix(dr + di); x[11] = ot_rot_fix(di - dr); }
    if (p == 2) { x[12] = di; x[13] = -dr; }
    if (p == 3) { x[14] = ot_rot_fix(di - dr); x[15] = -ot_rot_fix(dr + di); }
  }
#pragma unroll
  for (int g = 0; g < 8; g += 4) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int a = 2 * (g + p), b = 2 * (g + p + 2);
      const long long ur = x[a], ui = x[a + 1], vr = x[b], vi = x[b + 1];
      x[a] = ur + vr;
      x[a + 1] = ui + vi;
      if (p == 0) { x[b] = ur - vr; x[b + 1] = ui - vi; }
      else { x[b] = ui - vi; x[b + 1] = vr - ur; }
    }
  }
#pragma unroll
  for (int g = 0; g < 8; g += 2) {
    const long long ur = x[2 * g], ui = x[2 * g + 1], vr = x[2 * g + 2], vi = x[2 * g + 3];
    x[2 * g] = ur + vr;
    x[2 * g + 1] = ui + vi;
    x[2 * g + 2] = ur - vr;
    x[2 * g + 3] = ui - vi;
  }
  long long t;
  t = x[2]; x[2] = x[8]; x[8] = t;
  t = x[3]; x[3] = x[9]; x[9] = t;
  t = x[6]; x[6] = x[12]; x[12] = t;
  t = x[7]; x[7] = x[13]; x[13] = t;
}

// the largest exponent field among the values, as the scale exponent t with
// |x| < 2^t; zero or subnormal only: 0 (their digits are zero)
__device__ __forceinline__ int ot_scale_exp(int emax) {
  if (emax == 0) return 0;
  const int t = emax - 1022;
  return t < -960 ? -960 : t;
}

// round(x 2^(55 - t)) for |x| 2^(55 - t) < 2^62 (digits: |x| < 2^t; the Q61
// twiddles: t = -6, |x| <= 1) by integer operations on x's bits (x =
// M 2^(E - 1075), M the 53-bit significand; halves round away from zero);
// zero and subnormal x give 0
__device__ __forceinline__ long long ot_fixed(double x, int t) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0) return 0;
  const long long M = (b & 0xfffffffffffffLL) | 0x10000000000000LL;
  const int k = E - 1020 - t;  // x 2^(55 - t) = M 2^k (k <= 2 for |x| < 2^t, <= 9 for the twiddles)
  long long F = 0;
  if (k >= 0)
    F = M << k;
  else if (k > -54)
    F = (M + (1LL << (-k - 1))) >> (-k);
  return b < 0 ? -F : F;
}

// balanced base-256 digits of round(x 2^(55 - t)), most significant first
__device__ __forceinline__ void ot_digits(double x, int t, int (&dg)[kOtS]) {
  long long F = ot_fixed(x, t);  // |F| <= 2^55
#pragma unroll
  for (int s = kOtS - 1; s >= 1; --s) {
    int r = (int)(F & 255);
    if (r >= 128) r -= 256;
    dg[s] = r;
    F = (F - r) >> 8;
  }
  dg[0] = (int)F;
}

// bf16 bits of a small integer (|v| <= 256: exact in the upper half of the float)
__device__ __forceinline__ uint32_t ot_bf16(int v) { return __float_as_uint((float)v) >> 16; }

// The balanced digits of F = round(x 2^(55 - t)) (|F| <= 2^55) from the plain
// base-256 digits of F + B, B = 128 sum_(s<7) 2^(8 s) (0 <= F + B < 2^57):
// digit s is byte 6 - s of F + B minus 128 (the top one takes bits 48..56).
// Each becomes a float by the magic-number form 2^23 + d minus 2^23 + 128
// (exact), whose upper half is its bf16; w[s] packs digit s of x0 (low half)
// and x1 (high half).
constexpr unsigned long long kOtBias = 0x80808080808080ull;
__device__ __forceinline__ float ot_byte_digit(uint32_t word, uint32_t sel) {
  return __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7540u | sel)) - 8388736.0f;
}
__device__ __forceinline__ void ot_digit_pairs(double x0, double x1, int t, uint32_t (&w)[kOtS]) {
  const unsigned long long u0 = (unsigned long long)ot_fixed(x0, t) + kOtBias;
  const unsigned long long u1 = (unsigned long long)ot_fixed(x1, t) + kOtBias;
  const uint32_t l0 = (uint32_t)u0, h0 = (uint32_t)(u0 >> 32), l1 = (uint32_t)u1, h1 = (uint32_t)(u1 >> 32);
  const float t0 = __uint_as_float(0x4B000000u | (h0 >> 16)) - 8388736.0f;
  const float t1 = __uint_as_float(0x4B000000u | (h1 >> 16)) - 8388736.0f;
  w[0] = __byte_perm(__float_as_uint(t0), __float_as_uint(t1), 0x7632);
#pragma unroll
  for (int s = 1; s < kOtS; ++s) {
    const int byte = 6 - s;
    const float f0 = ot_byte_digit(byte >= 4 ? h0 : l0, (uint32_t)(byte & 3));
    const float f1 = ot_byte_digit(byte >= 4 ? h1 : l1, (uint32_t)(byte & 3));
    w[s] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
  }
}

__device__ __forceinline__ double2 ot_cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// The MMAs of one chunk: pair (S, T) into weight S + T (32 columns each), two
// K = 16 steps of the 32-wide digit (digit s sits in half s & 1 of slab s >> 1).
template <int S, int T>
__device__ __forceinline__ void ot_pairs(uint32_t d0, uint64_t a0, uint64_t b0, uint32_t idesc) {
  if constexpr (S < kOtS) {
    if constexpr (S + T < kOtS) {
      const uint64_t ad = a0 + (uint64_t)((S >> 1) * (kOtSlabA >> 4) + (S & 1) * 4);
      const uint64_t bd = b0 + (uint64_t)((T >> 1) * (kOtBSlab >> 4) + (T & 1) * 4);
      const uint32_t d = d0 + (uint32_t)((S + T) * 32);
      umma_k<kTcBF16>(d, ad, bd, idesc, S == 0 ? 0u : 1u);
      umma_k<kTcBF16>(d, ad + 2, bd + 2, idesc, 1u);
      ot_pairs<S, T + 1>(d0, a0, b0, idesc);
    } else {
      ot_pairs<S + 1, 0>(d0, a0, b0, idesc);
    }
  }
}

// The table's digits: rows n = 16 i + 2 m_b + c, K index k2 = 2 k + c'
// (value Re M, -Im M, Im M, Re M for (c, c') = (0,0), (0,1), (1,0), (1,1)),
// as the shared-memory image of each chunk (columns 2 c, 2 c + 1): [chunk c]
// [slab q][row n mod 32][128 bytes, 128-byte swizzled], digit 2q in the first 64
// bytes of a row and 2q + 1 in the second (the unused digit 7 zero); sigma
// (|M| < 2^sigma) after the image. One CTA.
__global__ void __launch_bounds__(256) oz_top_table_kernel(const double2* __restrict__ tab,
                                                           unsigned short* __restrict__ out, int* __restrict__ sigma) {
  pdl_begin();
  __shared__ int emax_s;
  if (threadIdx.x == 0) emax_s = 0;
  __syncthreads();
  int em = 0;
  for (int e = threadIdx.x; e < kOtD * kOtL * kOtD; e += blockDim.x) {
    const double2 m = tab[e];
    em = max(em, (int)((__double_as_longlong(m.x) >> 52) & 0x7ff));
    em = max(em, (int)((__double_as_longlong(m.y) >> 52) & 0x7ff));
  }
  atomicMax(&emax_s, em);
  __syncthreads();
  const int sg = ot_scale_exp(emax_s);
  for (int e = threadIdx.x; e < kOtN * 32; e += blockDim.x) {
    const int n = e >> 5, k2 = e & 31;
    const int i = n >> 4, mb = (n >> 1) & 7, c = n & 1;
    const int k = k2 >> 1, cp = k2 & 1;
    const double2 m = tab[k * (kOtL * kOtD) + mb * kOtD + i];
    const double v = c == 0 ? (cp == 0 ? m.x : -m.y) : (cp == 0 ? m.y : m.x);
    int dg[kOtS];
    ot_digits(v, sg, dg);
#pragma unroll
    for (int s = 0; s < kOtS + 1; ++s) {
      const int byte = 2 * ((s & 1) * 32 + k2);  // within the 128-byte row
      const uint32_t off = (uint32_t)(i >> 1) * kOtBChunk + (uint32_t)(s >> 1) * kOtBSlab + sw128_offset(n & 31, byte >> 4) +
                           (uint32_t)(byte & 15);
      out[off >> 1] = s < kOtS ? (unsigned short)ot_bf16(dg[s]) : (unsigned short)0;
    }
  }
  if (threadIdx.x == 0) *sigma = sg;
  pdl_trigger();
}

struct OzTopArgs {
  const double2* seeds;  // Z of the level below (compact when that level is sharded)
  double2* xout;         // MODE 0: X of this level
  const unsigned char* btab;  // the table's image, one 16 KiB chunk per two columns i
  const int* sigma;
  const double2* tw_lo;
  const double2* tw_hi;
  double* hist;
  Partial* parts;
  int* err;
  int64_t npencils;  // local pencils (a power of two)
  int64_t tile_begin, tile_end;  // this launch's tiles of 128 pencils (one partial tile below 128 pencils)
  int nmeas, logna, htw, sh, rk, seed_sh, seed_rk;
  double pscale;   // 1 / N^2
};

template <int MODE>
__global__ void __launch_bounds__(kOtThreads, 1) level_oz_kernel(OzTopArgs a) {
  pdl_begin();
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  unsigned char* As = base;                     // [2] tiles' digits
  unsigned char* Bs = base + 2 * kOtABytes;     // [kOtBStages] table chunks
  int4* twS = reinterpret_cast<int4*>(Bs + kOtBStages * kOtBChunk);  // [2][128][7] twiddles in Q61, split at bit 31
  int* tauS = reinterpret_cast<int*>(twS + 2 * kOtRows * (kOtL - 1));  // [2][128]
  __shared__ uint64_t a_full[2], a_empty[2], tw_empty[2], b_full[kOtBStages], b_empty[kOtBStages], t_full[2],
      t_empty[2], sq_full, sq_empty, mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ Partial sp[4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&a_full[b], 2 * kOtRows);  // one arrival per producer item
      mbar_init(&a_empty[b], 1);
      mbar_init(&tw_empty[b], 16);         // every drain warp
    }
    for (int b = 0; b < kOtBStages; ++b) {
      mbar_init(&b_full[b], 1);
      mbar_init(&b_empty[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&t_full[b], 1);
      mbar_init(&t_empty[b], 8);  // the drain warps of the buffer's chunks, two per lane quarter
    }
    mbar_init(&sq_full, 12);
    mbar_init(&sq_empty, 4);
    mbar_init(&mma_done, 1);
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 3) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* vfail = &fail;
  const int lna = a.logna - a.sh;
  const int64_t tw_mask = (int64_t(1) << a.htw) - 1;
  const int lvl_shift = a.nmeas - a.logna - 3;
  const int sigma = *a.sigma;
  const int64_t lvl_mask = (int64_t(1) << (a.logna + 3)) - 1;

  if (warp < 3) {
    // ------------------------------------------------------------ producers
    // item u < 256 of a tile: half u & 1 (complex values 8 (u & 1) .. + 7) of
    // pencil u >> 1; items u and u ^ 1 run in adjacent lanes of one round
    int it = 0;
    for (int64_t t = a.tile_begin + blockIdx.x; t < a.tile_end; t += gridDim.x, ++it) {
      const int tb = it & 1;  // digit, twiddle and scale buffers of this tile
      if (it >= 2 && (!mbar_wait(&a_empty[tb], ((it >> 1) - 1) & 1) ||
                      !mbar_wait(&tw_empty[tb], ((it >> 1) - 1) & 1))) {
        atomicExch(&fail, 1);
        break;
      }
      if (*vfail) break;
      unsigned char* At = As + tb * kOtABytes;
      for (int u = threadIdx.x; u < 2 * kOtRows; u += kOtProducers) {
        const int p = u >> 1, half = u & 1;
        const int64_t j = t * kOtRows + p;
        const bool have = j < a.npencils;  // rows past a partial tile's pencils: zero digits
        const double2* src = a.seeds + (have ? ((a.seed_rk + (j << a.seed_sh)) << 4) + 8 * half : 0);
        double2 z[kOtD / 2];
        int emax = 0;
#pragma unroll
        for (int k = 0; k < kOtD / 2; ++k) {
          z[k] = have ? __ldg(src + k) : make_double2(0.0, 0.0);
          emax = max(emax, (int)((__double_as_longlong(z[k].x) >> 52) & 0x7ff));
          emax = max(emax, (int)((__double_as_longlong(z[k].y) >> 52) & 0x7ff));
        }
        emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
        const int tau = ot_scale_exp(emax);
        // digit s of reals 4 g .. 4 g + 3 (two complex values) -> the half g & 1
        // of chunk (s & 1) 4 + (g >> 1) of slab s >> 1
#pragma unroll
        for (int gg = 0; gg < 4; ++gg) {
          const int g = 4 * half + gg;
          uint32_t wa[kOtS], wb[kOtS];
          ot_digit_pairs(z[2 * gg].x, z[2 * gg].y, tau, wa);
          ot_digit_pairs(z[2 * gg + 1].x, z[2 * gg + 1].y, tau, wb);
#pragma unroll
          for (int s = 0; s < kOtS; ++s)
            *reinterpret_cast<uint2*>(At + (s >> 1) * kOtSlabA + sw128_offset(p, (s & 1) * 4 + (g >> 1)) +
                                      (g & 1) * 8) = make_uint2(wa[s], wb[s]);
        }
        {  // the twiddles w_N^(m_b y_a): m_b = 1 .. 4 by half 0 (with the scale), 5 .. 7 by half 1
          const int64_t ya = a.rk + (j << a.sh);
          int4* tw = twS + (tb * kOtRows + p) * (kOtL - 1);
          const int m0 = half == 0 ? 1 : 5, m1 = half == 0 ? 5 : kOtL;
          for (int m = m0; m < m1; ++m) {
            const int64_t ex = (((int64_t)m * ya) & lvl_mask) << lvl_shift;
            const double2 w = ot_cmul(__ldg(a.tw_lo + (ex & tw_mask)), __ldg(a.tw_hi + (ex >> a.htw)));
            const long long qr = ot_fixed(w.x, -6), qi = ot_fixed(w.y, -6);  // round(w 2^61)
            tw[m - 1] =
                make_int4((int)(qr >> 31), (int)(qr & 0x7fffffff), (int)(qi >> 31), (int)(qi & 0x7fffffff));
          }
          if (half == 0) tauS[tb * kOtRows + p] = tau + sigma - 30;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&a_full[tb]);
      }
    }
  } else if (warp == 3) {
    // ------------------------------------------------------------ MMA issuer
    // Per tile, 8 chunks (two columns i each) into the two tensor-memory
    // buffers in turn; the table's chunk image streams through a ring of
    // kOtBStages stages by bulk copies, kOtBStages - 2 chunks ahead (a stage
    // is refilled once the MMAs of the chunk two back, its last reader, are done).
    if (lane == 0) {
      const uint32_t idesc = make_idesc<kTcBF16, 32>();
      const int64_t first = a.tile_begin + blockIdx.x;
      const int64_t ntile = first < a.tile_end ? (a.tile_end - first + gridDim.x - 1) / gridDim.x : 0;
      const int64_t total = ntile * kOtChunks;
      int64_t issued = 0, g = 0;
      bool ok = true;
      auto issue = [&](int64_t gq) {
        const int st = (int)(gq % kOtBStages);
        if (gq >= kOtBStages && !mbar_wait(&b_empty[st], (uint32_t)(((gq / kOtBStages) - 1) & 1))) return false;
        mbar_expect_tx(&b_full[st], kOtBChunk);
        bulk_load(Bs + st * kOtBChunk, a.btab + (size_t)(gq % kOtChunks) * kOtBChunk, kOtBChunk, &b_full[st]);
        return true;
      };
      while (ok && issued < total && issued < kOtBStages - 2) {
        ok = issue(issued);
        issued += ok ? 1 : 0;
      }
      int it = 0;
      for (int64_t t = first; t < a.tile_end && ok; t += gridDim.x, ++it) {
        const int ab = it & 1;
        if (!mbar_wait(&a_full[ab], (it >> 1) & 1) || *vfail) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t a0 = sw128_desc(smem_u32(As + ab * kOtABytes));
        for (int c = 0; c < kOtChunks; ++c, ++g) {
          if (issued < total) {
            if (!(ok = issue(issued))) break;
            ++issued;
          }
          const int st = (int)(g % kOtBStages);
          const int buf = c & 1;
          if (!mbar_wait(&b_full[st], (uint32_t)((g / kOtBStages) & 1)) ||
              (g >= 2 && !mbar_wait(&t_empty[buf], (uint32_t)(((g >> 1) - 1) & 1)))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          ot_pairs<0, 0>(tmem + (uint32_t)buf * kOtBufCols, a0, sw128_desc(smem_u32(Bs + st * kOtBChunk)), idesc);
          umma_commit(&t_full[buf]);
          umma_commit(&b_empty[st]);
        }
        if (!ok) break;
        umma_commit(&a_empty[ab]);
      }
      if (!ok) atomicExch(&fail, 1);
      // every table copy issued has landed and every MMA issued has finished
      // before shared and tensor memory are released
      for (int64_t gq = g; gq < issued; ++gq)
        if (!mbar_wait(&b_full[gq % kOtBStages], (uint32_t)((gq / kOtBStages) & 1))) atomicExch(&fail, 1);
      umma_commit(&mma_done);
      if (!mbar_wait(&mma_done, 0)) atomicExch(&fail, 1);
    }
  } else {
    // ------------------------------------------------------------ drain
    const int q = warp & 3;          // tensor-memory lane quarter
    const int k = (warp - 4) >> 2;   // 0 .. 3
    const int h = k & 1;             // column i = 2 c + h of chunk c
    const int par = k >> 1;          // the chunks c with c & 1 = par (tensor-memory buffer par)
    const int row = q * 32 + lane;   // pencil of this thread within the tile
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    double best = -1.0, wsum = 0.0, psum = 0.0;
    int64_t besty = INT64_MAX;
    int it = 0;
    uint32_t uses = 0;  // fills of buffer par consumed so far
    bool ok = true;
    for (int64_t t = a.tile_begin + blockIdx.x; t < a.tile_end && ok; t += gridDim.x, ++it) {
      const int tb = it & 1;
      bool got = mbar_wait(&a_full[tb], (it >> 1) & 1);  // this tile's twiddles and scales are written
      if (!__all_sync(0xffffffffu, got && !*vfail)) {
        ok = false;
        break;
      }
      const int4* tw = twS + (tb * kOtRows + row) * (kOtL - 1);
      // X in units of 2^(tau + sigma - 52) (the fixed point below)
      const int e2 = tauS[tb * kOtRows + row] - 22;
      const int64_t jt = t * kOtRows + row;  // local pencil index
      double acc[kOtL];
#pragma unroll
      for (int y = 0; y < kOtL; ++y) acc[y] = 0.0;
      for (int c = par; c < kOtChunks; c += 2, ++uses) {
        got = mbar_wait(&t_full[par], uses & 1);
        got = __all_sync(0xffffffffu, got && !*vfail) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!got) {
          ok = false;
          break;
        }
        const uint32_t col = lane_base + (uint32_t)par * kOtBufCols + (uint32_t)(h * 16);
        // T[m_b] (columns 2 m_b + c of this half) as 64-bit fixed point, four
        // values at a time (the seven weights' loads in flight together)
        long long x[16];
#pragma unroll
        for (int grp = 0; grp < 4; ++grp) {
          uint32_t v[kOtS][4];
#pragma unroll
          for (int w = 0; w < kOtS; ++w) tmem_ld4_async(col + (uint32_t)(w * 32 + grp * 4), v[w]);
          tmem_wait7x4(v);
#pragma unroll
          for (int e = 0; e < 4; ++e)
            x[4 * grp + e] = ot_weights_fix(v[0][e], v[1][e], v[2][e], v[3][e], v[4][e], v[5][e], v[6][e]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&t_empty[par]);
        // twiddles w_N^(m_b y_a) (m_b >= 1), then the 8-point DFT over m_b
#pragma unroll
        for (int m = 1; m < kOtL; ++m) ot_tw_fix(x[2 * m], x[2 * m + 1], tw[m - 1]);
        ot_dft8_fix(x);
        if (MODE == 0) {
          const int i = 2 * c + h;
          if (jt < a.npencils) {
#pragma unroll
            for (int y = 0; y < kOtL; ++y)
              a.xout[((jt + ((int64_t)y << lna)) << 4) + i] =
                  make_double2(ot_scale2(__ll2double_rn(x[2 * y]), e2), ot_scale2(__ll2double_rn(x[2 * y + 1]), e2));
          }
        } else {
#pragma unroll
          for (int y = 0; y < kOtL; ++y) {
            const double re = __ll2double_rn(x[2 * y]), im = __ll2double_rn(x[2 * y + 1]);
            acc[y] = fma(re, re, fma(im, im, acc[y]));  // in units of 2^(2 e2)
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&tw_empty[tb]);  // done with this tile's twiddles and scales
      if (!ok) break;
      if (MODE == 0) continue;
      // the four partial sums of a bin meet in tensor memory: warps k = 1 .. 3
      // of a lane quarter store theirs in columns 448 + 16 (k - 1), warp 0 adds
      const uint32_t sqc = lane_base + kOtSqCol;
      if (k != 0) {
        got = it < 1 || mbar_wait(&sq_empty, (it - 1) & 1);
        if (!__all_sync(0xffffffffu, got && !*vfail)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t w[16];
#pragma unroll
        for (int y = 0; y < kOtL; ++y) {
          w[2 * y] = (uint32_t)__double2loint(acc[y]);
          w[2 * y + 1] = (uint32_t)__double2hiint(acc[y]);
        }
        tmem_st16(sqc + (uint32_t)(16 * (k - 1)), w);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&sq_full);
      } else {
        got = mbar_wait(&sq_full, it & 1);
        if (!__all_sync(0xffffffffu, got && !*vfail)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int o = 0; o < 3; ++o) {
          uint32_t w[16];
          tmem_ld16(sqc + (uint32_t)(16 * o), w);
#pragma unroll
          for (int y = 0; y < kOtL; ++y) acc[y] += __hiloint2double((int)w[2 * y + 1], (int)w[2 * y]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&sq_empty);
        const double f = a.pscale * ldexp(1.0, e2) * ldexp(1.0, e2);  // the units and 1 / N^2
        const int64_t j = jt;
        if (j < a.npencils) {
#pragma unroll
          for (int y = 0; y < kOtL; ++y) {
            const double pv = acc[y] * f;
            const int64_t yl = j + ((int64_t)y << lna);
            a.hist[yl] = pv;
            const int64_t yy = a.rk + (yl << a.sh);
            better(best, besty, pv, yy);
            wsum = fma(pv, (double)yy, wsum);
            psum += pv;
          }
        }
      }
    }
    if (!ok) atomicExch(&fail, 1);
    if (MODE == 1 && k == 0) {  // readout partial of this CTA: the four k = 0 warps
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int64_t oy = __shfl_xor_sync(0xffffffffu, besty, off);
        better(best, besty, ob, oy);
        wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
        psum += __shfl_xor_sync(0xffffffffu, psum, off);
      }
      if (lane == 0) sp[q] = Partial{best, besty, wsum, psum};
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    if (MODE == 1) {
      Partial r = sp[0];
      for (int w = 1; w < 4; ++w) merge_partial(r, sp[w]);
      a.parts[blockIdx.x] = r;
    }
    if (fail) atomicExch(a.err, (int)QPE_ERR_TIMEOUT);
  }
  if (warp == 3)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  pdl_trigger();
}

}  // namespace

size_t oz_top_table_bytes() { return kOtBBytes + 256; }

cudaError_t configure_oz_top_kernel() {
  cudaError_t e = cudaFuncSetAttribute(level_oz_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOtSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(level_oz_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOtSmem);
}

// One FP64 level on the tensor cores: the level table's digits, then the
// persistent kernel (one CTA per SM, at most one per tile). top: the final
// level (histogram + readout partials; *grid_out = the partials), otherwise
// X into la.xout. A top level whose instance has a host histogram runs in
// kHostChunks tile ranges; after each, a copy stream forked from s copies
// that range's bins to the host while the next range computes, and s joins
// it at the end. Returns the launches or -1.
int launch_oz_level(const Instance& in, char* ws, const LevelArgs<double2>& la, bool top, cudaStream_t s,
                    cudaEvent_t* top_ev, int64_t* grid_out) {
  char* btab = ws + in.off_tctab;
  int* sigma = reinterpret_cast<int*>(btab + kOtBBytes);
  if (launch_k(oz_top_table_kernel, dim3(1), dim3(256), 0, s, la.tab, reinterpret_cast<unsigned short*>(btab),
               sigma) != cudaSuccess)
    return -1;
  OzTopArgs a{};
  a.seeds = la.seeds;
  a.xout = la.xout;
  a.btab = reinterpret_cast<const unsigned char*>(btab);
  a.sigma = sigma;
  a.tw_lo = la.tw_lo;
  a.tw_hi = la.tw_hi;
  a.hist = la.hist;
  a.err = reinterpret_cast<int*>(ws + in.off_err);
  a.npencils = int64_t(1) << (la.logna - la.sh);
  const int64_t ntiles = (a.npencils + kOtRows - 1) / kOtRows;
  a.nmeas = la.nmeas;
  a.logna = la.logna;
  a.htw = la.htw;
  a.sh = la.sh;
  a.rk = la.rk;
  a.seed_sh = la.seed_sh;
  a.seed_rk = la.seed_rk;
  a.pscale = la.pscale;
  const int lna = la.logna - la.sh;
  const bool chunked = top && in.host_hist && in.copy_stream;
  const int parts = chunked ? (int)std::min<int64_t>(kHostChunks, ntiles) : 1;
  int64_t nparts = 0;
  int launches = 1;
  if (top && top_ev && record_event(top_ev[0], s) != cudaSuccess) return -1;
  for (int c = 0; c < parts; ++c) {
    a.tile_begin = ntiles * c / parts;
    a.tile_end = ntiles * (c + 1) / parts;
    int64_t grid = in.nsm > 0 ? in.nsm : 1;
    if (grid > a.tile_end - a.tile_begin) grid = a.tile_end - a.tile_begin;
    if (grid > kReduceBlocks / parts) grid = kReduceBlocks / parts;
    a.parts = la.parts + nparts;  // each part's CTAs write their own readout partials
    nparts += grid;
    const cudaError_t e = top ? launch_k(level_oz_kernel<1>, dim3((unsigned)grid), dim3(kOtThreads), kOtSmem, s, a)
                              : launch_k(level_oz_kernel<0>, dim3((unsigned)grid), dim3(kOtThreads), kOtSmem, s, a);
    if (e != cudaSuccess) return -1;
    ++launches;
    if (chunked) {
      // bins j + (y << lna) of this part's pencils j, for every y < 8
      if (cudaEventRecord(in.copy_ev[c], s) != cudaSuccess) return -1;
      if (cudaStreamWaitEvent(in.copy_stream, in.copy_ev[c], 0) != cudaSuccess) return -1;
      const int64_t j0 = a.tile_begin * kOtRows;
      const int64_t j1 = std::min<int64_t>(a.tile_end * kOtRows, a.npencils);
      for (int y = 0; y < kOtL; ++y) {
        const int64_t o = j0 + ((int64_t)y << lna);
        if (cudaMemcpyAsync(in.host_hist + o, la.hist + o, (size_t)(j1 - j0) * sizeof(double), cudaMemcpyDeviceToHost,
                            in.copy_stream) != cudaSuccess)
          return -1;
      }
    }
  }
  if (top && top_ev && record_event(top_ev[1], s) != cudaSuccess) return -1;
  if (chunked) {  // s waits for the last copies
    if (cudaEventRecord(in.copy_ev[kHostChunks], in.copy_stream) != cudaSuccess) return -1;
    if (cudaStreamWaitEvent(s, in.copy_ev[kHostChunks], 0) != cudaSuccess) return -1;
  }
  if (grid_out) *grid_out = nparts;
  return launches;
}

// whether launch_oz_level copies the instance's histogram to the host itself
bool oz_top_copies_host_histogram(const Instance& in) {
  return in.tc_top && in.tc_top_prec == QPE_FP64 && in.host_hist && in.copy_stream;
}

}  // namespace qpe
