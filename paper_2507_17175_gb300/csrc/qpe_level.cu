// Fused QPE kernels for small target registers (d = 2^Nmat <= 64): the
// controlled-U^(2^k) gates, the QFT^-1 and the |amp|^2 reduction of one
// "level" in a single launch, with no pass over the full state in HBM.
//
// Write m = m_b + L m_a (m_b: the low r bits, L = 2^r; m_a: the high bits,
// N_a = N / L values) and y = y_a + N_a y_b. After the Hadamard layer and the
// controlled gates (Fig. 1) row m of the state is 2^(-n/2) U^m psi, and the
// unnormalised QFT^-1 output is
//
//   X[y] = sum_m w_N^(m y) U^m psi
//        = sum_{m_b} w_L^(m_b y_b) [ w_N^(m_b y_a) U^(m_b) Z[y_a] ],
//   Z[y_a] = sum_{m_a} w_(N_a)^(m_a y_a) (U^L)^(m_a) psi,     w_K = exp(-2 pi i / K)
//
// because w_N^(L m_a y) depends on y only through y_a. Z is the same problem
// for U^L = U^(2^r) on the high n - r measurement qubits, so levels recurse:
// the deepest level starts from psi, each level's X is the next one's Z, and
// the top level reduces |X|^2 / N^2 into the histogram P[y].
//
// The controlled gates of the r low measurement qubits act on Z[y_a] through
// the table M[m_b] = U_l^(m_b) = prod_{j in bits(m_b)} P_(off+j), m_b < L <= 32
// (built once per run by level_table_kernel). A CTA takes G consecutive y_a
// per iteration (persistent loop) and computes
//   T[g][m_b] = w_(N_level)^(m_b y_a) M[m_b] Z[y_a]       (register-tiled GEMM)
// then one length-L DFT over m_b per (g, column) in registers, and writes
// either X (natural order of y) or the histogram with the readout partials;
// the G consecutive y_a make the histogram and X writes contiguous.
#include <cuda_runtime.h>
#include <math.h>

#include "qpe_internal.cuh"

namespace qpe {

__constant__ double2 c_w32_64[32];  // exp(-2 pi i k / 32)
__constant__ float2 c_w32_32[32];

namespace {

template <typename C>
__device__ __forceinline__ C w32(int k);
template <>
__device__ __forceinline__ double2 w32<double2>(int k) { return c_w32_64[k]; }
template <>
__device__ __forceinline__ float2 w32<float2>(int k) { return c_w32_32[k]; }

template <typename C>
__device__ __forceinline__ C ldg(const C* p) { return __ldg(p); }

template <typename C>
__device__ __forceinline__ C tw_lookup(const C* lo, const C* hi, int h, int64_t e) {
  const int64_t mask = (int64_t(1) << h) - 1;
  return cmul(ldg(lo + (e & mask)), ldg(hi + (e >> h)));
}

template <typename C>
__device__ __forceinline__ C czero() {
  return mk((typename real_of<C>::type)0, (typename real_of<C>::type)0);
}

// In-register length-R DFT (R = 2^K <= 32), forward kernel w_R^(j j'),
// output in natural order.
template <typename C, int K>
__device__ __forceinline__ void dft_reg(C (&x)[1 << K]) {
  constexpr int R = 1 << K;
  // radix-2 decimation in frequency; output lands in bit-reversed order
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int h = R >> (s + 1);
#pragma unroll
    for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
      for (int p = 0; p < h; ++p) {
        const C a = x[g + p], b = x[g + p + h];
        x[g + p] = cadd(a, b);
        const C dl = csub(a, b);
        // w_(2h)^p = w_32^(p * 32 / (2h))
        x[g + p + h] = (p == 0) ? dl : cmul(dl, w32<C>(p * (32 / (2 * h))));
      }
    }
  }
  // undo the bit reversal
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int rv = 0;
#pragma unroll
    for (int b = 0; b < K; ++b) rv |= ((i >> b) & 1) << (K - 1 - b);
    if (rv > i) {
      const C t = x[i];
      x[i] = x[rv];
      x[rv] = t;
    }
  }
}

// One in-place DIF radix-2^K pass over the rows of tile (L rows, row stride
// RS elements, D columns): sub-blocks of M = 2^hi rows, stride S = M / 2^K.
// For each (block, q, column) the 2^K elements q + j S are transformed, the
// output digit j' is twisted by w_M^(q j') and stored back at q + j' S.
template <typename C, int K>
__device__ __forceinline__ void radix_pass(C* tile, int RS, int D, int logd, int hi, const C* twL, int logL) {
  constexpr int R = 1 << K;
  const int M = 1 << hi;
  const int S = M >> K;
  const int logS = hi - K;
  const int L = 1 << logL;
  const int items = (L >> K) << logd;  // (L / R) groups x D columns
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int c = it & (D - 1);
    const int g = it >> logd;
    const int b0 = g >> logS;
    const int q = g & (S - 1);
    const int base = b0 * M + q;
    C x[R];
#pragma unroll
    for (int j = 0; j < R; ++j) x[j] = tile[(base + j * S) * RS + c];
    dft_reg<C, K>(x);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      C v = x[j];
      if (j && q) {
        const int e = ((q * j) & (M - 1)) << (logL - hi);  // w_M^(q j) = w_L^(q j L / M)
        v = cmul(v, twL[e]);
      }
      tile[(base + j * S) * RS + c] = v;
    }
  }
}

template <typename C>
__device__ __forceinline__ void radix_dispatch(int k, C* tile, int RS, int D, int logd, int hi, const C* twL,
                                               int logL) {
  switch (k) {
    case 1: radix_pass<C, 1>(tile, RS, D, logd, hi, twL, logL); break;
    case 2: radix_pass<C, 2>(tile, RS, D, logd, hi, twL, logL); break;
    case 3: radix_pass<C, 3>(tile, RS, D, logd, hi, twL, logL); break;
    case 4: radix_pass<C, 4>(tile, RS, D, logd, hi, twL, logL); break;
    default: radix_pass<C, 5>(tile, RS, D, logd, hi, twL, logL); break;
  }
}

__device__ __forceinline__ int brev_bits(int x, int bits) { return bits ? (int)(__brev((unsigned)x) >> (32 - bits)) : 0; }

// Position p of the in-tile DIF output -> frequency index y_b: the pass that
// ran first (top bits of p) produced the least significant digit.
__device__ __forceinline__ int tile_pos_to_freq(int p, int r, int kmax) {
  int y = 0, rem = r, sh = 0;
  while (rem > 0) {
    const int k = rem < kmax ? rem : kmax;
    rem -= k;
    const int dig = (p >> rem) & ((1 << k) - 1);
    y |= dig << sh;
    sh += k;
  }
  return y;
}

// float -> double by integer bit manipulation (for finite, non-negative
// normal or zero inputs, as squared magnitudes are), avoiding the FP64 pipe.
__device__ __forceinline__ double widen_nonneg(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = u >> 23;
  if (ex == 0) return 0.0;  // zero or subnormal: below 1.2e-38, far under every tolerance
  if (ex == 0xff) return (double)f;
  const unsigned long long bits =
      ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

template <typename C>
struct Acc;  // per-row |x|^2 accumulator type
template <>
struct Acc<float2> {
  using T = float;
};
template <>
struct Acc<double2> {
  using T = double;
};

}  // namespace

// ----------------------------------------------------------- configuration
// Per (d, precision): L_max = 2^logl rows per pencil, G pencils per CTA
// iteration, TR x TG outputs (rows x pencils) per thread in the GEMM, and
// whether the level table fits in shared memory. 256 threads; every config
// gives (L_max d / TR) (G / TG) = 256 GEMM units and stays under ~100 KiB.
struct LvCfg {
  int logl, G, TR, TG;
  bool tab_smem;
};

__host__ __device__ constexpr LvCfg lv_cfg(int logd, bool dbl) {
  return dbl ? (logd == 1   ? LvCfg{5, 32, 2, 4, true}
                : logd == 2 ? LvCfg{5, 16, 4, 2, true}
                : logd == 3 ? LvCfg{4, 16, 4, 2, true}
                : logd == 4 ? LvCfg{3, 16, 4, 2, true}
                : logd == 5 ? LvCfg{3, 8, 4, 2, false}
                            : LvCfg{2, 8, 4, 2, false})
             : (logd == 1   ? LvCfg{5, 64, 2, 8, true}
                : logd == 2 ? LvCfg{5, 32, 4, 4, true}
                : logd == 3 ? LvCfg{5, 16, 4, 4, true}
                : logd == 4 ? LvCfg{4, 16, 4, 4, true}
                : logd == 5 ? LvCfg{3, 16, 4, 4, false}
                            : LvCfg{3, 8, 4, 4, false});
}

template <typename C, int K, int N>
__device__ __forceinline__ void dft_k(C (&x)[N]) {
  constexpr int R = 1 << K;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int h = R >> (s + 1);
#pragma unroll
    for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
      for (int p = 0; p < h; ++p) {
        const C u = x[g + p], v = x[g + p + h];
        x[g + p] = cadd(u, v);
        const C dl = csub(u, v);
        x[g + p + h] = (p == 0) ? dl : cmul(dl, w32<C>(p * (32 / (2 * h))));
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int rv = 0;
#pragma unroll
    for (int b = 0; b < K; ++b) rv |= ((i >> b) & 1) << (K - 1 - b);
    if (rv > i) {
      const C t = x[i];
      x[i] = x[rv];
      x[rv] = t;
    }
  }
}

// length-2^r DFT of x[0 .. 2^r), natural order in and out (2^r <= N)
template <typename C, int N>
__device__ __forceinline__ void dft_r(C (&x)[N], int r) {
  switch (r) {
    case 1: dft_k<C, 1, N>(x); break;
    case 2: if constexpr (N >= 4) dft_k<C, 2, N>(x); break;
    case 3: if constexpr (N >= 8) dft_k<C, 3, N>(x); break;
    case 4: if constexpr (N >= 16) dft_k<C, 4, N>(x); break;
    case 5: if constexpr (N >= 32) dft_k<C, 5, N>(x); break;
    default: break;
  }
}

// ------------------------------------------------------------------ kernel
template <typename C, int LOGD, int MODE>
__global__ void __launch_bounds__(256, sizeof(C) == 8 ? 2 : 1) level2_kernel(LevelArgs<C> a) {
  using R_t = typename real_of<C>::type;
  using A_t = typename Acc<C>::T;
  constexpr LvCfg cfg = lv_cfg(LOGD, sizeof(C) == 16);
  constexpr int D = 1 << LOGD, G = cfg.G, TR = cfg.TR, TG = cfg.TG;
  constexpr int LMAX = 1 << cfg.logl;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = a.r;
  const int L = 1 << r;
  const int ROWS = L * D;
  C* T = reinterpret_cast<C*>(smem_raw);        // [G][L][D]
  C* Zs = T + G * LMAX * D;                      // [G][D]
  C* twS = Zs + G * D;                           // [G][L]
  C* tabS = twS + G * LMAX;                      // [D][L D] (tab_smem)
  A_t* sq = reinterpret_cast<A_t*>(tabS + (cfg.tab_smem ? D * LMAX * D : 0));  // [L][D][G+1]
  const C* tab = cfg.tab_smem ? tabS : a.tab;
  const int tid = threadIdx.x;

  if (cfg.tab_smem)
    for (int e = tid; e < D * ROWS; e += blockDim.x) tabS[e] = ldg(a.tab + e);

  const int64_t Na = int64_t(1) << a.logna;
  const int64_t iters = (Na + G - 1) / G;
  const int lvl_shift = a.nmeas - a.logna - r;
  const int64_t lvl_mask = (int64_t(1) << (a.logna + r)) - 1;

  double best = -1.0, wsum = 0.0, psum = 0.0;
  int64_t besty = INT64_MAX;
  float wsum_f = 0.f, wcomp_f = 0.f, psum_f = 0.f, pcomp_f = 0.f;

  for (int64_t it = blockIdx.x; it < iters; it += gridDim.x) {
    const int64_t ya0 = it * G;
    __syncthreads();  // previous iteration's buffers consumed
    for (int e = tid; e < G * D; e += blockDim.x) {
      const int g = e >> LOGD;
      Zs[e] = (ya0 + g < Na) ? ldg(a.seeds + ((ya0 + g) << LOGD) + (e & (D - 1))) : czero<C>();
    }
    for (int e = tid; e < G * L; e += blockDim.x) {
      const int g = e >> r, mb = e & (L - 1);
      const int64_t ya = ya0 + g;
      C w = mk((R_t)1, (R_t)0);
      if (mb && ya) w = tw_lookup(a.tw_lo, a.tw_hi, a.htw, (((int64_t)mb * ya) & lvl_mask) << lvl_shift);
      twS[e] = w;
    }
    __syncthreads();
    // T[g][m_b][i] = w^(m_b y_a) sum_k M[m_b][i][k] Z[g][k]
    {
      const int nrg = ROWS / TR;
      const int units = nrg * (G / TG);
      for (int u = tid; u < units; u += blockDim.x) {
        const int rg = u % nrg, gg = u / nrg;
        const int row0 = rg * TR;
        const int mb = row0 >> LOGD;
        C acc[TR][TG];
#pragma unroll
        for (int t = 0; t < TR; ++t)
#pragma unroll
          for (int g = 0; g < TG; ++g) acc[t][g] = czero<C>();
#pragma unroll 4
        for (int k = 0; k < D; ++k) {
          C av[TR], zv[TG];
          const C* tp = tab + k * ROWS + row0;
#pragma unroll
          for (int t = 0; t < TR; ++t) av[t] = cfg.tab_smem ? tp[t] : ldg(tp + t);
#pragma unroll
          for (int g = 0; g < TG; ++g) zv[g] = Zs[(gg * TG + g) * D + k];
#pragma unroll
          for (int t = 0; t < TR; ++t)
#pragma unroll
            for (int g = 0; g < TG; ++g) cfma(acc[t][g], av[t], zv[g]);
        }
#pragma unroll
        for (int g = 0; g < TG; ++g) {
          const int gi = gg * TG + g;
          const C w = twS[gi * L + mb];
          C* out = T + (gi * L) * D + row0;
#pragma unroll
          for (int t = 0; t < TR; ++t) out[t] = cmul(acc[t][g], w);
        }
      }
    }
    __syncthreads();
    // length-L DFT over m_b for every (g, column)
    for (int p = tid; p < G * D; p += blockDim.x) {
      const int g = p >> LOGD, i = p & (D - 1);
      C x[LMAX];
#pragma unroll
      for (int m = 0; m < LMAX; ++m)
        if (m < L) x[m] = T[(g * L + m) * D + i];
      dft_r<C, LMAX>(x, r);
      const int64_t ya = ya0 + g;
      if (MODE == 0) {
        if (ya < Na) {
#pragma unroll
          for (int yb = 0; yb < LMAX; ++yb)
            if (yb < L) a.xout[((ya + ((int64_t)yb << a.logna)) << LOGD) + i] = x[yb];
        }
      } else {
#pragma unroll
        for (int yb = 0; yb < LMAX; ++yb)
          if (yb < L) sq[(yb * D + i) * (G + 1) + g] = (A_t)x[yb].x * (A_t)x[yb].x + (A_t)x[yb].y * (A_t)x[yb].y;
        if (MODE == 2 && ya < Na) {
#pragma unroll
          for (int yb = 0; yb < LMAX; ++yb)
            if (yb < L) a.xout[((ya + ((int64_t)yb << a.logna)) << LOGD) + i] = cscale(x[yb], (R_t)a.xscale);
        }
      }
    }
    if (MODE != 0) {
      __syncthreads();
      for (int q = tid; q < G * L; q += blockDim.x) {
        const int g = q % G, yb = q / G;
        const int64_t ya = ya0 + g;
        if (ya >= Na) continue;
        A_t s = 0;
#pragma unroll 8
        for (int i = 0; i < D; ++i) s += sq[(yb * D + i) * (G + 1) + g];
        const int64_t y = ya + ((int64_t)yb << a.logna);
        if (sizeof(C) == 8) {
          const float v = (float)s * (float)a.pscale;  // pscale = 1/N^2, a power of two
          a.hist[y] = widen_nonneg(v);
          if ((double)v > best || ((double)v == best && y < besty)) {
            best = v;
            besty = y;
          }
          const float yv = v * (float)y;  // P y (finalize divides by N), Kahan-compensated
          float t1 = yv - wcomp_f;
          float t2 = wsum_f + t1;
          wcomp_f = (t2 - wsum_f) - t1;
          wsum_f = t2;
          t1 = v - pcomp_f;
          t2 = psum_f + t1;
          pcomp_f = (t2 - psum_f) - t1;
          psum_f = t2;
        } else {
          const double v = (double)s * a.pscale;
          a.hist[y] = v;
          if (v > best || (v == best && y < besty)) {
            best = v;
            besty = y;
          }
          wsum += v * (double)y;
          psum += v;
        }
      }
    }
  }
  if (MODE != 0) {
    if (sizeof(C) == 8) {
      wsum = (double)wsum_f;
      psum = (double)psum_f;
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int64_t oy = __shfl_xor_sync(0xffffffffu, besty, off);
      if (ob > best || (ob == best && oy < besty)) {
        best = ob;
        besty = oy;
      }
      wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
      psum += __shfl_xor_sync(0xffffffffu, psum, off);
    }
    __shared__ Partial sp[8];
    const int lane = tid & 31, warp = tid >> 5;
    __syncthreads();
    if (lane == 0) sp[warp] = Partial{best, besty, wsum, psum};
    __syncthreads();
    if (tid == 0) {
      Partial res = sp[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        if (sp[w].best > res.best || (sp[w].best == res.best && sp[w].besty < res.besty)) {
          res.best = sp[w].best;
          res.besty = sp[w].besty;
        }
        res.wsum += sp[w].wsum;
        res.psum += sp[w].psum;
      }
      a.parts[blockIdx.x] = res;
    }
  }
}

// Level tables: tab_l[k][m_b d + i] = (U_l^(m_b))[i][k], U_l = P_(off_l), for
// m_b < 2^(r_l). One warp per (level, m_b, i): the row e_i^T prod P_(off+j)
// over the set bits j of m_b, as a chain of vector-matrix products.
template <typename C>
__global__ void __launch_bounds__(256) level_table_kernel(const C* __restrict__ P, char* __restrict__ ws,
                                                          TableJobs jobs, int logd) {
  const int D = 1 << logd;
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t base = 0;
  int li = -1;
  for (int l = 0; l < jobs.count; ++l) {
    const int64_t rows = (int64_t(1) << jobs.r[l]) << logd;
    if (w < base + rows) {
      li = l;
      break;
    }
    base += rows;
  }
  if (li < 0) return;
  const int row = (int)(w - base);
  const int mb = row >> logd, i = row & (D - 1);
  const int L = 1 << jobs.r[li];
  C* tab = reinterpret_cast<C*>(ws + jobs.tab_off[li]);
  const int64_t DD = (int64_t)D * D;
  // v: lane holds columns k = lane, lane + 32 (D <= 64)
  C v0 = czero<C>(), v1 = czero<C>();
  bool started = false;
  for (int j = 0; j < jobs.r[li]; ++j) {
    if (!((mb >> j) & 1)) continue;
    const C* Pj = P + (int64_t)(jobs.off[li] + j) * DD;
    if (!started) {
      if (lane < D) v0 = ldg(Pj + (int64_t)i * D + lane);
      if (lane + 32 < D) v1 = ldg(Pj + (int64_t)i * D + lane + 32);
      started = true;
      continue;
    }
    C n0 = czero<C>(), n1 = czero<C>();
    for (int l = 0; l < D; ++l) {
      const C vl = l < 32 ? mk(__shfl_sync(0xffffffffu, v0.x, l), __shfl_sync(0xffffffffu, v0.y, l))
                          : mk(__shfl_sync(0xffffffffu, v1.x, l - 32), __shfl_sync(0xffffffffu, v1.y, l - 32));
      if (lane < D) cfma(n0, vl, ldg(Pj + (int64_t)l * D + lane));
      if (lane + 32 < D) cfma(n1, vl, ldg(Pj + (int64_t)l * D + lane + 32));
    }
    v0 = n0;
    v1 = n1;
  }
  if (!started) {  // m_b = 0: identity row
    v0 = (lane == i) ? mk((typename real_of<C>::type)1, (typename real_of<C>::type)0) : czero<C>();
    v1 = (lane + 32 == i) ? mk((typename real_of<C>::type)1, (typename real_of<C>::type)0) : czero<C>();
  }
  const int ROWS = L << logd;
  if (lane < D) tab[(int64_t)lane * ROWS + row] = v0;
  if (lane + 32 < D) tab[(int64_t)(lane + 32) * ROWS + row] = v1;
}

template <typename C>
__global__ void seed_psi_kernel(const double2* __restrict__ psi, C* __restrict__ out, int d) {
  for (int i = threadIdx.x; i < d; i += blockDim.x) out[i] = to_c(psi[i], (C*)nullptr);
}

// --------------------------------------------------------------- host side
size_t level_smem_bytes(int logd, int r, size_t esize) {
  (void)r;
  const LvCfg c = lv_cfg(logd, esize == 16);
  const size_t D = size_t(1) << logd, L = size_t(1) << c.logl;
  const size_t acc = esize == 8 ? 4 : 8;
  size_t b = (size_t)c.G * L * D * esize + (size_t)c.G * D * esize + (size_t)c.G * L * esize;
  if (c.tab_smem) b += D * L * D * esize;
  b += L * D * (c.G + 1) * acc;
  return b;
}

int level_max_bits(int logd, size_t esize, size_t smem_cap) {
  (void)smem_cap;
  return lv_cfg(logd, esize == 16).logl;
}

std::vector<Level> make_levels(int nmeas, int logd, size_t esize, int rtop) {
  const int rmax = level_max_bits(logd, esize, kLevelSmemCap);
  std::vector<Level> lv;
  int remaining = nmeas, off = 0;
  bool top = true;
  while (remaining > 0) {
    int r = top ? (rtop > 0 ? rtop : rmax) : rmax;
    if (r > rmax) r = rmax;
    if (r > remaining) r = remaining;
    Level L{};
    L.off = off;
    L.r = r;
    L.logna = remaining - r;
    lv.push_back(L);
    off += r;
    remaining -= r;
    top = false;
  }
  return lv;
}

#define QPE_LV_ALL(X, C) X(C, 1, 0) X(C, 1, 1) X(C, 1, 2) X(C, 2, 0) X(C, 2, 1) X(C, 2, 2) \
  X(C, 3, 0) X(C, 3, 1) X(C, 3, 2) X(C, 4, 0) X(C, 4, 1) X(C, 4, 2) X(C, 5, 0) X(C, 5, 1) X(C, 5, 2) \
  X(C, 6, 0) X(C, 6, 1) X(C, 6, 2)

static cudaError_t set_level_attrs() {
  cudaError_t e;
#define QPE_ATTR(C, LD, M)                                                                                  \
  e = cudaFuncSetAttribute(level2_kernel<C, LD, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                           (int)level_smem_bytes(LD, 0, sizeof(C)));                                        \
  if (e != cudaSuccess) return e;
  QPE_LV_ALL(QPE_ATTR, float2)
  QPE_LV_ALL(QPE_ATTR, double2)
#undef QPE_ATTR
  return cudaSuccess;
}

cudaError_t configure_level_kernels() {
  double2 w64[32];
  float2 w32v[32];
  for (int k = 0; k < 32; ++k) {
    // exp(-2 pi i k / 32) from the host math library
    const double ang = -2.0 * M_PI * (double)k / 32.0;
    w64[k] = make_double2(cos(ang), sin(ang));
    w32v[k] = make_float2((float)w64[k].x, (float)w64[k].y);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_w32_64, w64, sizeof(w64));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyToSymbol(c_w32_32, w32v, sizeof(w32v));
  if (e != cudaSuccess) return e;
  return set_level_attrs();
}

template <typename C, int M>
static void launch_level2(int logd, unsigned grid, size_t smem, cudaStream_t s, const LevelArgs<C>& a) {
  switch (logd) {
    case 1: level2_kernel<C, 1, M><<<grid, 256, smem, s>>>(a); break;
    case 2: level2_kernel<C, 2, M><<<grid, 256, smem, s>>>(a); break;
    case 3: level2_kernel<C, 3, M><<<grid, 256, smem, s>>>(a); break;
    case 4: level2_kernel<C, 4, M><<<grid, 256, smem, s>>>(a); break;
    case 5: level2_kernel<C, 5, M><<<grid, 256, smem, s>>>(a); break;
    default: level2_kernel<C, 6, M><<<grid, 256, smem, s>>>(a); break;
  }
}

template <typename C>
int launch_levels(const Instance& in, char* ws, bool keep_state, cudaStream_t s) {
  const size_t esize = sizeof(C);
  const C* P = reinterpret_cast<const C*>(ws + (esize == 16 ? in.off_pow64 : in.off_pow32));
  const C* tlo = reinterpret_cast<const C*>(ws + (esize == 16 ? in.off_tw_lo64 : in.off_tw_lo32));
  const C* thi = reinterpret_cast<const C*>(ws + (esize == 16 ? in.off_tw_hi64 : in.off_tw_hi32));
  int launches = 0;
  const int nl = (int)in.levels.size();
  // tables of every level
  {
    TableJobs jobs{};
    jobs.count = nl;
    int64_t warps = 0;
    for (int li = 0; li < nl; ++li) {
      jobs.off[li] = in.levels[li].off;
      jobs.r[li] = in.levels[li].r;
      jobs.tab_off[li] = in.levels[li].tab_off;
      warps += (int64_t(1) << in.levels[li].r) << in.nmat;
    }
    const int64_t blocks = (warps * 32 + 255) / 256;
    level_table_kernel<C><<<(unsigned)blocks, 256, 0, s>>>(P, ws, jobs, in.nmat);
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    ++launches;
  }
  C* seed = reinterpret_cast<C*>(ws + in.zbuf_seed_off);
  seed_psi_kernel<C><<<1, 64, 0, s>>>(reinterpret_cast<const double2*>(ws + in.off_psi), seed, (int)in.d);
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  ++launches;
  const LvCfg cfg = lv_cfg(in.nmat, esize == 16);
  const size_t smem = level_smem_bytes(in.nmat, 0, esize);
  const C* cur_seed = seed;
  for (int li = nl - 1; li >= 0; --li) {
    const Level& L = in.levels[li];
    LevelArgs<C> a{};
    a.seeds = cur_seed;
    a.tab = reinterpret_cast<const C*>(ws + L.tab_off);
    a.off = L.off;
    a.r = L.r;
    a.logna = L.logna;
    a.logd = in.nmat;
    a.nmeas = in.nmeas;
    a.tw_lo = tlo;
    a.tw_hi = thi;
    a.htw = in.htw;
    a.pscale = ldexp(1.0, -2 * in.nmeas);
    a.inv_n = ldexp(1.0, -in.nmeas);
    a.xscale = 1.0;
    const int64_t Na = int64_t(1) << L.logna;
    const int64_t iters = (Na + cfg.G - 1) / cfg.G;
    int64_t grid = iters < in.level_grid ? iters : in.level_grid;
    if (li > 0) {
      C* out = reinterpret_cast<C*>(ws + in.off_zbuf[li & 1]);
      a.xout = out;
      launch_level2<C, 0>(in.nmat, (unsigned)grid, smem, s, a);
      cur_seed = out;
    } else {
      a.hist = reinterpret_cast<double*>(ws + in.off_hist);
      a.parts = reinterpret_cast<Partial*>(ws + in.off_partials);
      if (grid > kReduceBlocks) grid = kReduceBlocks;
      if (keep_state) {
        a.xout = reinterpret_cast<C*>(ws + in.off_state);
        a.xscale = ldexp(1.0, -in.nmeas);  // physical final state: X / N
        launch_level2<C, 2>(in.nmat, (unsigned)grid, smem, s, a);
      } else {
        launch_level2<C, 1>(in.nmat, (unsigned)grid, smem, s, a);
      }
      if (cudaPeekAtLastError() != cudaSuccess) return -1;
      ++launches;
      finalize_readout(in, ws, (int)grid, s);
      if (cudaPeekAtLastError() != cudaSuccess) return -1;
      ++launches;
      break;
    }
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    ++launches;
  }
  return launches;
}

template <typename C>
int level_occupancy(int logd, int r) {
  (void)r;
  int blocks = 0;
  const size_t smem = level_smem_bytes(logd, 0, sizeof(C));
  cudaError_t e;
  switch (logd) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_kernel<C, 1, 1>, 256, smem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_kernel<C, 2, 1>, 256, smem); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_kernel<C, 3, 1>, 256, smem); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_kernel<C, 4, 1>, 256, smem); break;
    case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_kernel<C, 5, 1>, 256, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_kernel<C, 6, 1>, 256, smem); break;
  }
  if (e != cudaSuccess) return 1;
  return blocks > 0 ? blocks : 1;
}
template int level_occupancy<float2>(int, int);
template int level_occupancy<double2>(int, int);

template int launch_levels<float2>(const Instance&, char*, bool, cudaStream_t);
template int launch_levels<double2>(const Instance&, char*, bool, cudaStream_t);

}  // namespace qpe
