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

#include <cuda_fp16.h>

#include "qpe_internal.cuh"
#include "qpe_tcgen05.cuh"

namespace qpe {

using tcg::kTcFP16;
using tcg::kTcTF32;

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

// count contiguous complex elements (16-byte aligned, count * sizeof(C) a multiple of 16)
template <typename C>
__device__ __forceinline__ void cp_async_block(C* smem, const C* gmem, int count, int tid, int nthreads) {
  constexpr int V = 16 / (int)sizeof(C);
  for (int e = tid * V; e < count; e += nthreads * V) cp_async16(smem + e, gmem + e);
}

template <typename C>
__device__ __forceinline__ C czero() {
  return mk((typename real_of<C>::type)0, (typename real_of<C>::type)0);
}

// The complex64 schedules' readout of one thread: bin values in FP32 (the
// histogram stores them widened, bit-exactly), the argmax compared in FP32,
// and Kahan-compensated FP32 sums of P y and P (off GB300's slow FP64 units).
struct HistAcc32 {
  float best = -1.f;
  int64_t besty = INT64_MAX;
  float wsum = 0.f, wcomp = 0.f, psum = 0.f, pcomp = 0.f;
  __device__ __forceinline__ void add(float v, int64_t y) {
    if (v > best || (v == best && y < besty)) {
      best = v;
      besty = y;
    }
    // P y (the finalize divides by N); y < 2^30 converts through int32 (an
    // int64 conversion would run on the slow FP64 pipe)
    float t1 = v * __int2float_rn((int)y) - wcomp;
    float t2 = wsum + t1;
    wcomp = (t2 - wsum) - t1;
    wsum = t2;
    t1 = v - pcomp;
    t2 = psum + t1;
    pcomp = (t2 - psum) - t1;
    psum = t2;
  }
};

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
  bool tab_smem;  // final level: whole table resident in shared memory
  int DI0, G0;    // other levels: columns per CTA (table slice in shared memory), pencils per iteration
};

__host__ __device__ constexpr LvCfg lv_cfg(int logd, bool dbl) {
  return dbl ? (logd == 1   ? LvCfg{5, 32, 2, 4, true, 2, 32}
                : logd == 2 ? LvCfg{5, 16, 4, 2, true, 4, 16}
                : logd == 3 ? LvCfg{4, 16, 4, 2, true, 8, 16}
                : logd == 4 ? LvCfg{3, 16, 4, 2, true, 8, 32}
                : logd == 5 ? LvCfg{3, 8, 4, 2, false, 8, 32}
                            : LvCfg{2, 8, 4, 2, false, 8, 32})
             : (logd == 1   ? LvCfg{5, 64, 2, 8, true, 2, 64}
                : logd == 2 ? LvCfg{5, 32, 4, 4, true, 4, 32}
                : logd == 3 ? LvCfg{5, 16, 4, 4, true, 8, 16}
                : logd == 4 ? LvCfg{4, 16, 4, 4, true, 8, 32}
                : logd == 5 ? LvCfg{3, 16, 4, 4, false, 8, 64}
                            : LvCfg{4, 8, 2, 8, false, 8, 32});
}

// Per-MODE view of the configuration: the final level (MODE 1/2) takes whole
// rows (the histogram sums over all d columns); the others take DI0 columns.
template <int LOGD, bool DBL, int MODE>
struct LvShape {
  static constexpr LvCfg c = lv_cfg(LOGD, DBL);
  static constexpr int D = 1 << LOGD;
  static constexpr int DI = MODE == 0 ? c.DI0 : D;
  static constexpr int G = MODE == 0 ? c.G0 : c.G;
  static constexpr int LMAX = 1 << c.logl;
  static constexpr bool TAB_SMEM = MODE == 0 ? true : c.tab_smem;
  // FP64 with the table in shared memory: complex products with three real
  // multiplications (Gauss), the table's Re + Im kept beside it (d >= 8: the
  // short-DFT shapes have the registers for the third accumulator)
  static constexpr bool THREE_M = DBL && TAB_SMEM && LOGD >= 3;
  static constexpr size_t smem(size_t esize) {
    const size_t acc = esize == 8 ? 4 : 8;
    size_t b = (size_t)G * LMAX * DI * esize + (size_t)G * D * esize + 2 * (size_t)G * LMAX * esize;
    if (TAB_SMEM) b += (size_t)D * LMAX * DI * esize;
    if (THREE_M) b += (size_t)D * LMAX * DI * (esize / 2);
    if (MODE != 0) b += (size_t)LMAX * D * (G + 1) * acc;
    return b;
  }
};

// 4 consecutive complex values through 16-byte accesses
__device__ __forceinline__ void load4(const float2* p, float2 (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 2);
  v[0] = make_float2(a.x, a.y);
  v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y);
  v[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4(const double2* p, double2 (&v)[4]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) v[t] = p[t];
}
__device__ __forceinline__ void ldg4(const float2* p, float2 (&v)[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p + 2));
  v[0] = make_float2(a.x, a.y);
  v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y);
  v[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void ldg4(const double2* p, double2 (&v)[4]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) v[t] = __ldg(p + t);
}
__device__ __forceinline__ void store4(float2* p, const float2 (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  *reinterpret_cast<float4*>(p + 2) = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}
__device__ __forceinline__ void store4(double2* p, const double2 (&v)[4]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) p[t] = v[t];
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

// Butterfly reduce-scatter of NV values over the lanes whose index bits below
// 2 O differ: each step keeps half of the values (the upper half on lanes with
// bit O set) and adds the partner's copy of that half. With NV >= lanes, lane
// li ends holding the sums for indices yb0 .. yb0 + NV / lanes - 1; with fewer
// values than lanes the remaining steps are plain all-reduce steps.
template <int O, int NV, typename A, int N>
__device__ __forceinline__ void reduce_scatter_step(A (&v)[N], int li, int& yb0) {
  if constexpr (O >= 1) {
    if constexpr (NV > 1) {
      constexpr int H = NV / 2;
      const bool up = (li & O) != 0;
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const A send = up ? v[j] : v[j + H];
        const A keep = up ? v[j + H] : v[j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      if (up) yb0 += H;
      reduce_scatter_step<O / 2, H>(v, li, yb0);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
      reduce_scatter_step<O / 2, 1>(v, li, yb0);
    }
  }
}
template <int O, int NV, typename A, int N>
__device__ __forceinline__ void reduce_scatter(A (&v)[N], int li, int& yb0) {
  reduce_scatter_step<O, NV>(v, li, yb0);
}

// ------------------------------------------------------------------ kernel
// One CTA's share of a level: column group cg, pencil-group iterations
// it_begin, it_begin + it_step, ... < it_end. MODE != 0 writes this share's
// readout partial to *part_out.
template <typename C, int LOGD, int MODE>
__device__ __forceinline__ void level_body(const LevelArgs<C>& a, int cg, int64_t it_begin, int64_t it_end,
                                           int64_t it_step, Partial* part_out) {
  using R_t = typename real_of<C>::type;
  using A_t = typename Acc<C>::T;
  using S = LvShape<LOGD, sizeof(C) == 16, MODE>;
  constexpr LvCfg cfg = S::c;
  constexpr int D = S::D, DI = S::DI, G = S::G, TR = cfg.TR, TG = cfg.TG, LMAX = S::LMAX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int r = a.r;
  const int L = 1 << r;
  const int ROWS = L * DI;  // GEMM rows of this CTA: (m_b, column in group)
  C* T = reinterpret_cast<C*>(smem_raw);  // [G][L][DI]
  C* ZsT = T + G * LMAX * DI;             // [D][G]  (k-major: seeds of the G pencils)
  C* twLo = ZsT + G * D;                  // [G][L] low factor of w^(m_b y_a)
  C* twHi = twLo + G * LMAX;              // [G][L] high factor
  C* tabS = twHi + G * LMAX;              // [D][L DI] (TAB_SMEM)
  R_t* tabSum = reinterpret_cast<R_t*>(tabS + (S::TAB_SMEM ? D * LMAX * DI : 0));  // [D][L DI] Re + Im (THREE_M)
  A_t* sq = reinterpret_cast<A_t*>(tabSum + (S::THREE_M ? D * LMAX * DI : 0));      // [L][D][G+1] (MODE != 0)
  const C* tab = S::TAB_SMEM ? tabS : a.tab;
  const int tab_ld = S::TAB_SMEM ? ROWS : L * D;  // row stride (per k) of the table in use
  const int tid = threadIdx.x;

  __syncthreads();  // shared memory of a previous share (grouped launches) fully consumed
  const int i_base = cg * DI;
  const int tab_col0 = S::TAB_SMEM ? 0 : i_base;
  if (S::TAB_SMEM) {
    // slice: tabS[k][m_b DI + ii] = tab[k][m_b D + i_base + ii], asynchronous,
    // completed by the first iteration's wait
    constexpr int V = 16 / (int)sizeof(C);  // elements per 16-byte copy
    if constexpr (DI % V == 0) {
      for (int e = tid * V; e < D * ROWS; e += blockDim.x * V) {
        const int k = e / ROWS, rr = e - k * ROWS;
        const int mb = rr / DI, ii = rr - mb * DI;
        cp_async16(tabS + e, a.tab + (int64_t)k * (L * D) + mb * D + i_base + ii);
      }
    } else {
      for (int e = tid; e < D * ROWS; e += blockDim.x) {
        const int k = e / ROWS, rr = e - k * ROWS;
        const int mb = rr / DI, ii = rr - mb * DI;
        cp_async_elem(tabS + e, a.tab + (int64_t)k * (L * D) + mb * D + i_base + ii, true);
      }
    }
  }

  const int lna = a.logna - a.sh;              // local pencils: 2^lna (all of them when not sharded)
  const int64_t Na = int64_t(1) << lna;
  const int lvl_shift = a.nmeas - a.logna - r;
  const int64_t lvl_mask = (int64_t(1) << (a.logna + r)) - 1;

  double best = -1.0, wsum = 0.0, psum = 0.0;
  int64_t besty = INT64_MAX;
  HistAcc32 h32;

  // histogram bin of local index yl (outcome y = rk + (yl << sh)) <- s / N^2,
  // with the readout partials (argmax, Kahan sums) over the outcome y
  auto account = [&](A_t s, int64_t yl) {
    const int64_t y = a.rk + (yl << a.sh);
    if (sizeof(C) == 8) {
      const float v = (float)s * (float)a.pscale;  // pscale = 1/N^2, a power of two
      a.hist[yl] = widen_nonneg(v);
      h32.add(v, y);
    } else {
      const double v = (double)s * a.pscale;
      a.hist[yl] = v;
      if (v > best || (v == best && y < besty)) {
        best = v;
        besty = y;
      }
      wsum += v * (double)y;
      psum += v;
    }
  };

  // seeds Z[y_a] (k-major) and the two table factors of w^(m_b y_a) of the
  // pencil group `itg`, as asynchronous copies (w^0 = lo[0] hi[0] = 1 exactly)
  const int64_t tw_mask = (int64_t(1) << a.htw) - 1;
  auto issue_group = [&](int64_t itg) {
    const int64_t yg = itg * G;
    const int gv = (int)(Na - yg < G ? Na - yg : G);
    for (int e = tid; e < G * D; e += blockDim.x) {
      const int g = e / D, k = e - g * D;
      const bool valid = g < gv;
      cp_async_elem(ZsT + k * G + g, a.seeds + (valid ? ((a.seed_rk + ((yg + g) << a.seed_sh)) << LOGD) + k : 0),
                    valid);
    }
    for (int e = tid; e < G * L; e += blockDim.x) {
      const int g = e >> r, mb = e & (L - 1);
      const int64_t ya_true = a.rk + ((yg + g) << a.sh);
      const int64_t ex = (((int64_t)mb * ya_true) & lvl_mask) << lvl_shift;
      cp_async_elem(twLo + e, a.tw_lo + (ex & tw_mask), true);
      cp_async_elem(twHi + e, a.tw_hi + (ex >> a.htw), true);
    }
    cp_async_commit();
  };
  if (it_begin < it_end) issue_group(it_begin);

  for (int64_t it = it_begin; it < it_end; it += it_step) {
    const int64_t ya0 = it * G;
    const int gvalid = (int)(Na - ya0 < G ? Na - ya0 : G);
    cp_async_wait<0>();
    __syncthreads();  // this group's copies (and the table slice) landed; the previous iteration is consumed
    if constexpr (S::THREE_M) {
      if (it == it_begin) {  // Re + Im of the table slice, once per share
        for (int e = tid; e < D * ROWS; e += blockDim.x) tabSum[e] = tabS[e].x + tabS[e].y;
        __syncthreads();
      }
    }
    // T[g][m_b][ii] = w^(m_b y_a) sum_k M[m_b][i_base + ii][k] Z[g][k]
    {
      const int nrg = ROWS / TR;
      const int ngg = (gvalid + TG - 1) / TG;
      const int units = nrg * ngg;
      for (int u = tid; u < units; u += blockDim.x) {
        const int rg = u % nrg, gg = u / nrg;
        const int row0 = rg * TR;  // (m_b, ii) row in this CTA's numbering
        const int mb = row0 / DI;
        const int ii0 = row0 - mb * DI;
        const int trow = S::TAB_SMEM ? row0 : mb * D + tab_col0 + ii0;
        C acc[TR][TG];
#pragma unroll
        for (int t = 0; t < TR; ++t)
#pragma unroll
          for (int g = 0; g < TG; ++g) acc[t][g] = czero<C>();
        if constexpr (S::THREE_M) {
          // (a_r + i a_i)(z_r + i z_i) = (a_r z_r - a_i z_i) + i ((a_r + a_i)(z_r + z_i) - a_r z_r - a_i z_i):
          // three FMA chains per output instead of four
          R_t p1[TR][TG], p2[TR][TG], p3[TR][TG];
#pragma unroll
          for (int t = 0; t < TR; ++t)
#pragma unroll
            for (int g = 0; g < TG; ++g) p1[t][g] = p2[t][g] = p3[t][g] = (R_t)0;
#pragma unroll 4
          for (int k = 0; k < D; ++k) {
            const C* tp = tab + k * tab_ld + trow;
            const R_t* sp3 = tabSum + k * tab_ld + trow;
            const C* zp = ZsT + k * G + gg * TG;
            C av[TR], zv[TG];
            R_t as[TR], zs[TG];
#pragma unroll
            for (int t = 0; t < TR; ++t) {
              av[t] = tp[t];
              as[t] = sp3[t];
            }
#pragma unroll
            for (int g = 0; g < TG; ++g) {
              zv[g] = zp[g];
              zs[g] = zv[g].x + zv[g].y;
            }
#pragma unroll
            for (int t = 0; t < TR; ++t)
#pragma unroll
              for (int g = 0; g < TG; ++g) {
                p1[t][g] = fma(av[t].x, zv[g].x, p1[t][g]);
                p2[t][g] = fma(av[t].y, zv[g].y, p2[t][g]);
                p3[t][g] = fma(as[t], zs[g], p3[t][g]);
              }
          }
#pragma unroll
          for (int t = 0; t < TR; ++t)
#pragma unroll
            for (int g = 0; g < TG; ++g) acc[t][g] = mk(p1[t][g] - p2[t][g], p3[t][g] - p1[t][g] - p2[t][g]);
        } else {
#pragma unroll 4
        for (int k = 0; k < D; ++k) {
          C av[TR], zv[TG];
          const C* tp = tab + k * tab_ld + trow;
          if constexpr (TR == 4) {
            if (S::TAB_SMEM)
              load4(tp, av);
            else
              ldg4(tp, av);
          } else if constexpr (TR == 2 && sizeof(C) == 8) {
            const float4 v2 = S::TAB_SMEM ? *reinterpret_cast<const float4*>(tp)
                                          : __ldg(reinterpret_cast<const float4*>(tp));
            av[0] = mk((R_t)v2.x, (R_t)v2.y);
            av[1] = mk((R_t)v2.z, (R_t)v2.w);
          } else {
#pragma unroll
            for (int t = 0; t < TR; ++t) av[t] = S::TAB_SMEM ? tp[t] : ldg(tp + t);
          }
          const C* zp = ZsT + k * G + gg * TG;
          if constexpr (TG == 4) {
            load4(zp, zv);
          } else if constexpr (TG == 8) {
            load4(zp, *reinterpret_cast<C(*)[4]>(&zv[0]));
            load4(zp + 4, *reinterpret_cast<C(*)[4]>(&zv[4]));
          } else {
#pragma unroll
            for (int g = 0; g < TG; ++g) zv[g] = zp[g];
          }
#pragma unroll
          for (int t = 0; t < TR; ++t)
#pragma unroll
            for (int g = 0; g < TG; ++g) cfma(acc[t][g], av[t], zv[g]);
        }
        }
#pragma unroll
        for (int g = 0; g < TG; ++g) {
          const int gi = gg * TG + g;
          const C w = cmul(twLo[gi * L + mb], twHi[gi * L + mb]);
          C* out = T + (gi * L + mb) * DI + ii0;
          if constexpr (TR == 4) {
            C ov[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) ov[t] = cmul(acc[t][g], w);
            store4(out, ov);
          } else {
#pragma unroll
            for (int t = 0; t < TR; ++t) out[t] = cmul(acc[t][g], w);
          }
        }
      }
    }
    __syncthreads();
    // the GEMM was the only reader of ZsT / twLo / twHi: fetch the next group now
    if (it + it_step < it_end) issue_group(it + it_step);
    // length-L DFT over m_b for every (g, column)
    // Final level with d <= 32 columns and a full-width level: the d lanes of a
    // pencil hold its columns, so the sums over columns are a butterfly
    // reduce-scatter over shuffles (no shared-memory pass, no extra barrier).
    constexpr bool kShuffleHist = MODE != 0 && D <= 32;
    if constexpr (kShuffleHist) if (r == cfg.logl) {
      for (int pb = 0; pb < G * D; pb += blockDim.x) {  // same trip count on every lane
        const int p = pb + tid;
        const bool act = p < G * D;  // G D is a multiple of 32: whole warps
        const int g = p / D, ii = p - g * D;
        const bool valid = act && g < gvalid;
        C x[LMAX];
        A_t v[LMAX];
#pragma unroll
        for (int m = 0; m < LMAX; ++m) x[m] = act ? T[(g * LMAX + m) * D + ii] : czero<C>();
        dft_k<C, cfg.logl, LMAX>(x);
#pragma unroll
        for (int m = 0; m < LMAX; ++m) v[m] = (A_t)x[m].x * (A_t)x[m].x + (A_t)x[m].y * (A_t)x[m].y;
        if (MODE == 2 && valid) {
#pragma unroll
          for (int yb = 0; yb < LMAX; ++yb)
            a.xout[((ya0 + g + ((int64_t)yb << lna)) << LOGD) + ii] = cscale(x[yb], (R_t)a.xscale);
        }
        int yb0 = 0;
        reduce_scatter<D / 2, LMAX>(v, ii, yb0);
        constexpr int NV = LMAX >= D ? LMAX / D : 1;  // column sums left on each lane
        if (valid && (LMAX >= D || ii % (D / LMAX) == 0)) {
#pragma unroll
          for (int j = 0; j < NV; ++j) account(v[j], ya0 + g + ((int64_t)(yb0 + j) << lna));
        }
      }
      continue;
    }
    for (int p = tid; p < gvalid * DI; p += blockDim.x) {
      const int g = p / DI, ii = p - g * DI;
      C x[LMAX];
#pragma unroll
      for (int m = 0; m < LMAX; ++m)
        if (m < L) x[m] = T[(g * L + m) * DI + ii];
      dft_r<C, LMAX>(x, r);
      const int64_t ya = ya0 + g;
      const int i = i_base + ii;
      if (MODE == 0) {
#pragma unroll
        for (int yb = 0; yb < LMAX; ++yb)
          if (yb < L) a.xout[((ya + ((int64_t)yb << lna)) << LOGD) + i] = x[yb];
      } else {
#pragma unroll
        for (int yb = 0; yb < LMAX; ++yb)
          if (yb < L) sq[(yb * D + i) * (G + 1) + g] = (A_t)x[yb].x * (A_t)x[yb].x + (A_t)x[yb].y * (A_t)x[yb].y;
        if (MODE == 2) {
#pragma unroll
          for (int yb = 0; yb < LMAX; ++yb)
            if (yb < L) a.xout[((ya + ((int64_t)yb << lna)) << LOGD) + i] = cscale(x[yb], (R_t)a.xscale);
        }
      }
    }
    if (MODE != 0) {
      __syncthreads();
      for (int q = tid; q < G * L; q += blockDim.x) {
        const int g = q % G, yb = q / G;
        if (g >= gvalid) continue;
        A_t s = 0;
#pragma unroll 8
        for (int i = 0; i < D; ++i) s += sq[(yb * D + i) * (G + 1) + g];
        account(s, ya0 + g + ((int64_t)yb << lna));
      }
    }
  }
  cp_async_wait<0>();  // a share with no iterations still issued its slice copies
  if (MODE != 0) {
    if (sizeof(C) == 8) {
      best = h32.best;
      besty = h32.besty;
      wsum = (double)h32.wsum;
      psum = (double)h32.psum;
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
      *part_out = res;
    }
  }
}

// CTAs per SM the register allocation aims for: two for complex64 and for the
// FP64 d = 16 levels (whose shared memory also admits two), one for the other
// FP64 shapes (their register tiles and DFTs need more than 128 registers)
template <typename C, int LOGD>
__host__ __device__ constexpr int level_min_blocks() {
  return (sizeof(C) == 8 || LOGD == 4) ? 2 : 1;
}

template <typename C, int LOGD, int MODE>
__global__ void __launch_bounds__(256, level_min_blocks<C, LOGD>()) level2_kernel(LevelArgs<C> a) {
  pdl_begin();
  using S = LvShape<LOGD, sizeof(C) == 16, MODE>;
  constexpr int NCG = S::D / S::DI;
  const int64_t iters = ((int64_t(1) << (a.logna - a.sh)) + S::G - 1) / S::G;
  level_body<C, LOGD, MODE>(a, (int)(blockIdx.x % NCG), blockIdx.x / NCG, iters, gridDim.x / NCG,
                            a.parts + blockIdx.x);
  pdl_trigger();
}

// Grouped form: one launch runs many (instance, level) shares listed in
// items[]; each CTA walks the list with a grid stride.
template <typename C, int LOGD, int MODE>
__global__ void __launch_bounds__(256, level_min_blocks<C, LOGD>())
    level2_grouped_kernel(const LevelArgs<C>* __restrict__ args, const GroupItem* __restrict__ items, int nitems) {
  pdl_begin();
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const GroupItem it = items[w];
    const LevelArgs<C> a = args[it.arg];
    level_body<C, LOGD, MODE>(a, it.cg, it.it_begin, it.it_end, 1, a.parts + it.part);
  }
  pdl_trigger();
}

// Level tables: tab_l[k][m_b d + i] = (U_l^(m_b))[i][k], U_l = P_(off_l), for
// m_b < 2^(r_l). One CTA per (level, m_b, block of TB rows): the rows
// e_i^T prod_{j in bits(m_b)} P_(off+j) as a chain of (TB x d) x (d x d)
// products, each factor staged in shared memory.
template <typename C>
__global__ void __launch_bounds__(256) level_table_kernel(const C* __restrict__ P, char* __restrict__ ws,
                                                          TableJobs jobs, int logd) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int D = 1 << logd;
  const int TB = D < 16 ? D : 16;  // rows per CTA
  const int nrb = D / TB;
  C* Pb0 = reinterpret_cast<C*>(smem_raw);  // two D x D factors (double buffer)
  C* V = Pb0 + 2 * D * D;                    // TB x D running rows
  C* Vn = V + TB * D;
  // locate (level, m_b, row block)
  int64_t b = blockIdx.x;
  int li = -1;
  for (int l = 0; l < jobs.count; ++l) {
    const int64_t cnt = (int64_t(1) << jobs.r[l]) * nrb;
    if (b < cnt) {
      li = l;
      break;
    }
    b -= cnt;
  }
  if (li < 0) return;
  const int mb = (int)(b / nrb), rb = (int)(b % nrb);
  const int i0 = rb * TB;
  const int64_t DD = (int64_t)D * D;
  const int tid = threadIdx.x;
  // the factors P_(off+j), j in bits(m_b), in increasing j
  int js[8];
  int nf = 0;
  for (int j = 0; j < jobs.r[li]; ++j)
    if ((mb >> j) & 1) js[nf++] = j;
  const C* Pbase = P + (int64_t)jobs.off[li] * DD;
  if (nf == 0) {  // m_b = 0: identity rows
    for (int e = tid; e < TB * D; e += blockDim.x) {
      const int rr = e / D, k = e - rr * D;
      V[e] = (k == i0 + rr) ? mk((typename real_of<C>::type)1, (typename real_of<C>::type)0) : czero<C>();
    }
  } else {
    // rows i0.. of the first factor, and the second factor, in flight together
    cp_async_block(V, Pbase + js[0] * DD + (int64_t)i0 * D, TB * D, tid, blockDim.x);
    if (nf > 1) cp_async_block(Pb0, Pbase + js[1] * DD, D * D, tid, blockDim.x);
    cp_async_commit();
    for (int f = 1; f < nf; ++f) {
      const C* Pb = Pb0 + (f & 1 ? 0 : D * D);
      if (f + 1 < nf) {  // next factor into the other buffer while this one is used
        cp_async_block(Pb0 + (f & 1 ? D * D : 0), Pbase + js[f + 1] * DD, D * D, tid, blockDim.x);
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      // each thread: 4 outputs (row rr, columns k0..k0+3 spaced by D/4), 4 independent chains
      const int q4 = D >= 4 ? D / 4 : 1;
      for (int e = tid; e < TB * q4; e += blockDim.x) {
        const int rr = e / q4, k0 = e - rr * q4;
        const int nk = D >= 4 ? 4 : D;
        C acc[4] = {czero<C>(), czero<C>(), czero<C>(), czero<C>()};
#pragma unroll 4
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
      C* tmp = V;
      V = Vn;
      Vn = tmp;
    }
    cp_async_wait<0>();
  }
  __syncthreads();
  const int L = 1 << jobs.r[li];
  const int ROWS = L << logd;
  C* tab = reinterpret_cast<C*>(ws + jobs.tab_off[li]);
  for (int e = tid; e < TB * D; e += blockDim.x) {
    const int k = e / TB, rr = e - k * TB;  // consecutive threads: consecutive rows (contiguous in tab)
    tab[(int64_t)k * ROWS + mb * D + i0 + rr] = V[rr * D + k];
  }
  pdl_trigger();
}

template <typename C>
__global__ void seed_psi_kernel(const double2* __restrict__ psi, C* __restrict__ out, int d) {
  pdl_begin();
  for (int i = threadIdx.x; i < d; i += blockDim.x) out[i] = to_c(psi[i], (C*)nullptr);
  pdl_trigger();
}

// ------------------------------------------- top level on the tensor cores
// The top level of the fused schedule for d = 16 (L = 16) under the split
// precisions QPE_C64_FP16X2 and QPE_C64_TF32X3. The level's contraction
//   T[y_a][m_b][i] = sum_k M[m_b][i][k] Z[y_a][k]
// is one real GEMM per tile of 128 pencils y_a:
//   A (128 x 32): row y_a = the 32 floats (re, im interleaved) of Z[y_a],
//   B (512 x 32): row n = (i, m_b, c) = the real embedding of M, n-major
//                 (c = 0 real part: (Re M, -Im M); c = 1: (Im M, Re M)),
//   D = A B^T (128 x 512, FP32 in tensor memory): column n of row y_a is the
//       real (c = 0) or imaginary part of T[y_a][m_b][i],
// as split products. FP16x2: two passes, A_hi B_hi, then [A_hi | A_lo] times
// [B_lo | B_hi] over K = 64 (both cross products in one pass); each A row is
// scaled by a power of two into fp16's range (largest |entry| in
// [2^14, 2^15)) and B by 2^14, and the drain multiplies by the exact inverse;
// the 128-byte rows [hi | lo] are the K-major, 128-byte-swizzled layout the
// MMA reads, B in both orders. TF32x3: A_hi, A_lo, B_hi, B_lo are separate
// 128-byte rows (32 tf32 values) and three products A_hi B_hi + A_hi B_lo +
// A_lo B_hi; no scaling; one A stage (shared memory). B stays in shared memory
// for the whole launch.
//
// Roles (384 threads, one CTA per SM, persistent over tiles; 12 warps leave
// 168 registers per thread):
//   warps 0..2   load the tile's Z rows (rows p and p + 96), split and store
//                them into one of two A stages, and store the row's 16
//                twiddles w_N^(m_b y_a) times the row's inverse scale
//   warp 3       allocates tensor memory; lane 0 issues the MMAs: columns
//                [0, 256) (i < 8) into tensor-memory half 0, [256, 512) into
//                half 1, so the MMAs of one half overlap the drain of the other
//   warps 4..11  drain: thread (set s, lane group q, lane) owns pencil
//                y_a = 32 q + lane of the tile and the columns i of set s
//                (4 per half); for each i it loads the 16 values T[m_b]
//                (32 floats, one tcgen05.ld, issued while the previous column's
//                DFT runs), multiplies by the stored twiddles, runs the
//                length-16 DFT over m_b in registers and adds |X|^2
//                into 16 bin sums; set 1 hands its sums to set 0 through
//                shared memory, set 0 writes the histogram and the readout.
// Every wait is an mbarrier wait with a poll limit; on expiry the CTA records
// QPE_ERR_TIMEOUT, frees its tensor memory and returns.
constexpr int kTcL = 16, kTcD = 16;   // DFT length and target dimension of this kernel
constexpr int kTcRows = 128;          // pencils per tile (MMA M)
constexpr int kTcN = 2 * kTcD * kTcL; // 512 GEMM columns
constexpr int kTcThreads = 384;
constexpr int kTcProducers = 96;      // threads of warps 0..2
constexpr int kTcSqStride = 17;       // padded row of the hand-over buffer
constexpr int kTcTwStride = 18;       // padded twiddle row (complex; 16-byte aligned, no bank conflicts)
constexpr size_t kTcBBytes = (size_t)kTcN * 128;  // one B operand (order or part), 64 KiB
// A stages and the bytes of one (fp16: rows [hi | lo]; tf32: a hi tile and a lo tile)
template <int KIND>
__host__ __device__ constexpr int tc_stages() { return KIND == kTcFP16 ? 2 : 1; }
template <int KIND>
__host__ __device__ constexpr size_t tc_a_bytes() { return (size_t)kTcRows * 128 * (KIND == kTcFP16 ? 1 : 2); }
template <int KIND>
__host__ __device__ constexpr size_t tc_top_smem() {
  return 2 * kTcBBytes + tc_stages<KIND>() * tc_a_bytes<KIND>() +
         tc_stages<KIND>() * (size_t)kTcRows * kTcTwStride * 8 + 2 * (size_t)kTcRows * kTcSqStride * 4 + 1024;
}

struct TcTopArgs {
  const float2* seeds;       // Z of the level below (compact when the level below is sharded)
  const uint4* btab;         // 128 KiB: fp16 rows [hi | lo] then [lo | hi], or tf32 rows hi then lo
  const float2* tw_lo;
  const float2* tw_hi;
  double* hist;
  Partial* parts;
  int* err;
  int64_t ntiles;            // local pencils / 128
  int nmeas, logna, htw, sh, rk, seed_sh, seed_rk;
  double pscale;
};

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// B rows of the top level's table (tab[k][m_b d + i] = M[m_b][i][k],
// complex64). FP16x2: scaled by 2^14, split into fp16 hi / lo, rows [hi | lo]
// then [lo | hi] (64 halves each). TF32x3: split into tf32 hi / lo, the hi rows
// then the lo rows (32 floats each).
template <int KIND>
__global__ void __launch_bounds__(256) tc_top_table_kernel(const float2* __restrict__ tab, void* __restrict__ outp) {
  pdl_begin();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kTcN * 32; e += gridDim.x * blockDim.x) {
    const int n = e >> 5, kk = e & 31;
    const int i = n >> 5, mb = (n >> 1) & 15, c = n & 1;
    const int k = kk >> 1, cp = kk & 1;
    const float2 m = tab[k * (kTcL * kTcD) + mb * kTcD + i];
    const float v = c == 0 ? (cp == 0 ? m.x : -m.y) : (cp == 0 ? m.y : m.x);
    if constexpr (KIND == kTcFP16) {
      __half* out = static_cast<__half*>(outp);
      const float vs = v * 16384.0f;  // 2^14, exact
      const __half hi = __float2half_rn(vs);
      const __half lo = __float2half_rn(vs - __half2float(hi));
      out[(size_t)n * 64 + kk] = hi;             // [hi | lo]
      out[(size_t)n * 64 + 32 + kk] = lo;
      out[(size_t)(kTcN + n) * 64 + kk] = lo;    // [lo | hi]
      out[(size_t)(kTcN + n) * 64 + 32 + kk] = hi;
    } else {
      float* out = static_cast<float*>(outp);
      const float hi = tf32_rna(v);
      out[(size_t)n * 32 + kk] = hi;
      out[(size_t)(kTcN + n) * 32 + kk] = tf32_rna(v - hi);
    }
  }
  pdl_trigger();
}

template <int KIND>
__global__ void __launch_bounds__(kTcThreads, 1) level_tc_top_kernel(TcTopArgs a) {
  using namespace tcg;
  pdl_begin();
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  constexpr int NST = tc_stages<KIND>();
  constexpr size_t AB = tc_a_bytes<KIND>();
  unsigned char* Bs = base;                            // two B operands, 64 KiB each
  unsigned char* As = base + 2 * kTcBBytes;            // NST A stages
  float2* twS = reinterpret_cast<float2*>(As + NST * AB);  // [NST][128][18]: scaled twiddles per row
  float* sq = reinterpret_cast<float*>(twS + NST * kTcRows * kTcTwStride);  // [2][128][17]
  __shared__ uint64_t a_full[2], a_empty[2], t_full[2], t_empty[2], sq_full[2], sq_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ Partial sp[4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&a_full[b], kTcRows);
      mbar_init(&a_empty[b], 1 + 8);
      mbar_init(&t_full[b], 1);
      mbar_init(&t_empty[b], 8);
      mbar_init(&sq_full[b], kTcRows);
      mbar_init(&sq_empty[b], kTcRows);
    }
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 3) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // both orders of B into shared memory, swizzled (16-byte chunks)
  {
    const uint4* src = a.btab;
    for (int q = threadIdx.x; q < 2 * kTcN * 8; q += kTcThreads) {
      const int which = q / (kTcN * 8), n = (q >> 3) % kTcN, c = q & 7;
      *reinterpret_cast<uint4*>(Bs + which * kTcBBytes + sw128_offset(n, c)) = __ldg(src + q);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const int lna = a.logna - a.sh;
  volatile int* vfail = &fail;
  const int64_t tw_mask = (int64_t(1) << a.htw) - 1;
  const int lvl_shift = a.nmeas - a.logna - 4;
  const int64_t lvl_mask = (int64_t(1) << (a.logna + 4)) - 1;

  if (warp < 3) {
    // ---------------------------------------------------------- producer
    int it = 0;
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++it) {
      const int b = it % NST;
      if (it >= NST && !mbar_wait(&a_empty[b], ((it / NST) - 1) & 1)) {
        atomicExch(&fail, 1);
        break;
      }
      if (*vfail) break;
      for (int p = threadIdx.x; p < kTcRows; p += kTcProducers) {  // tile rows of this thread
      const int64_t j = t * kTcRows + p;
      const float4* src = reinterpret_cast<const float4*>(a.seeds + ((a.seed_rk + (j << a.seed_sh)) << 4));
      float x[32];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 v = __ldg(src + c);
        x[4 * c] = v.x;
        x[4 * c + 1] = v.y;
        x[4 * c + 2] = v.z;
        x[4 * c + 3] = v.w;
      }
      float sc = 1.f, invr = 1.f;
      if constexpr (KIND == kTcFP16) {
        float mx = 0.f;
#pragma unroll
        for (int c = 0; c < 32; ++c) mx = fmaxf(mx, fabsf(x[c]));
        // floor(log2(mx)) from the exponent field; zero or tiny rows keep scale 1
        const int ex = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 127;
        const int e = (ex < -100 || ex > 100) ? 0 : 14 - ex;
        sc = __uint_as_float((uint32_t)(127 + e) << 23);
        invr = __uint_as_float((uint32_t)(127 - e - 14) << 23);  // undoes both operand scales
      }
      {
        const int64_t ya = a.rk + (j << a.sh);
        float2* tw = twS + (b * kTcRows + p) * kTcTwStride;
#pragma unroll
        for (int mb = 0; mb < kTcL; mb += 2) {
          float2 w[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int64_t ex = (((int64_t)(mb + u) * ya) & lvl_mask) << lvl_shift;
            w[u] = cscale(cmul(__ldg(a.tw_lo + (ex & tw_mask)), __ldg(a.tw_hi + (ex >> a.htw))), invr);
          }
          *reinterpret_cast<float4*>(tw + mb) = make_float4(w[0].x, w[0].y, w[1].x, w[1].y);
        }
      }
      unsigned char* row = As + b * AB;
      if constexpr (KIND == kTcFP16) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float x0 = x[8 * c + 2 * h] * sc, x1 = x[8 * c + 2 * h + 1] * sc;
            const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
            const __half l0 = __float2half_rn(x0 - __half2float(h0)), l1 = __float2half_rn(x1 - __half2float(h1));
            hw[h] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
            lw[h] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
          }
          *reinterpret_cast<uint4*>(row + sw128_offset(p, c)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(row + sw128_offset(p, 4 + c)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
      } else {  // tf32: the hi tile, then the lo tile 16 KiB on
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float hv[4], lv[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            hv[h] = tf32_rna(x[4 * c + h]);
            lv[h] = tf32_rna(x[4 * c + h] - hv[h]);
          }
          *reinterpret_cast<float4*>(row + sw128_offset(p, c)) = make_float4(hv[0], hv[1], hv[2], hv[3]);
          *reinterpret_cast<float4*>(row + kTcRows * 128 + sw128_offset(p, c)) =
              make_float4(lv[0], lv[1], lv[2], lv[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&a_full[b]);
      }
    }
  } else if (warp == 3) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc<KIND, 256>();
      const uint32_t b1 = smem_u32(Bs), b2 = smem_u32(Bs + kTcBBytes);
      int it = 0;
      for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++it) {
        const int b = it % NST;
        if (!mbar_wait(&a_full[b], (it / NST) & 1)) {
          atomicExch(&fail, 1);
          break;
        }
        if (*vfail) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t ad = sw128_desc(smem_u32(As + b * AB));
        bool ok = true;
        for (int h = 0; h < 2; ++h) {
          if (it >= 1 && !mbar_wait(&t_empty[h], (it - 1) & 1)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t bd1 = sw128_desc(b1 + (uint32_t)h * 32768u), bd2 = sw128_desc(b2 + (uint32_t)h * 32768u);
          const uint32_t d = tmem + (uint32_t)(h * 256);
          if constexpr (KIND == kTcFP16) {
            umma_k<kTcFP16>(d, ad, bd1, idesc, 0u);          // A_hi B_hi, K = 0..15
            umma_k<kTcFP16>(d, ad + 2, bd1 + 2, idesc, 1u);  //            K = 16..31
#pragma unroll
            for (int k = 0; k < 4; ++k) umma_k<kTcFP16>(d, ad + 2 * k, bd2 + 2 * k, idesc, 1u);  // cross, K = 64
          } else {
            const uint64_t adl = sw128_desc(smem_u32(As + b * AB + kTcRows * 128));  // A_lo tile
#pragma unroll
            for (int k = 0; k < 4; ++k) umma_k<kTcTF32>(d, ad + 2 * k, bd1 + 2 * k, idesc, k == 0 ? 0u : 1u);  // hi hi
#pragma unroll
            for (int k = 0; k < 4; ++k) umma_k<kTcTF32>(d, ad + 2 * k, bd2 + 2 * k, idesc, 1u);   // hi lo
#pragma unroll
            for (int k = 0; k < 4; ++k) umma_k<kTcTF32>(d, adl + 2 * k, bd1 + 2 * k, idesc, 1u);  // lo hi
          }
          umma_commit(&t_full[h]);
        }
        if (!ok) {
          atomicExch(&fail, 1);
          break;
        }
        umma_commit(&a_empty[b]);
      }
    }
  } else {
    // ---------------------------------------------------------- drain
    const int dw = warp - 4;
    const int set = dw >> 2, lg = warp & 3;
    const int row = lg * 32 + lane;
    const float pscale = (float)a.pscale;  // 1/N^2, a power of two
    HistAcc32 h32;
    int it = 0;
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++it) {
      const int b = it % NST;   // A / twiddle stage
      const int bq = it & 1;    // hand-over buffer
      const int64_t j = t * kTcRows + row;
      const float4* tr = reinterpret_cast<const float4*>(twS + (b * kTcRows + row) * kTcTwStride);
      float acc[kTcL];
#pragma unroll
      for (int yb = 0; yb < kTcL; ++yb) acc[yb] = 0.f;
      bool ok = true;
      for (int h = 0; h < 2 && ok; ++h) {
        bool got = mbar_wait(&t_full[h], it & 1);
        got = __all_sync(0xffffffffu, got && !*vfail) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!got) {
          ok = false;
          break;
        }
        // the stage's twiddles are read from shared memory at every use (no
        // registers held for them); the stage is released after the last half
        const uint32_t col0 = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(h * 256 + set * 4 * 32);
        uint32_t v[32];
        tmem_ld32_async(col0, v);
        tmem_wait32(v);
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {  // column i = 8 h + 4 set + q
          float2 x[kTcL];
#pragma unroll
          for (int mb = 0; mb < kTcL; mb += 2) {
            const float4 w = tr[mb >> 1];
            x[mb] = cmul(make_float2(__uint_as_float(v[2 * mb]), __uint_as_float(v[2 * mb + 1])), make_float2(w.x, w.y));
            x[mb + 1] = cmul(make_float2(__uint_as_float(v[2 * mb + 2]), __uint_as_float(v[2 * mb + 3])),
                             make_float2(w.z, w.w));
          }
          if (q < 3) tmem_ld32_async(col0 + (uint32_t)((q + 1) * 32), v);  // next column while this DFT runs
          dft_k<float2, 4, kTcL>(x);
#pragma unroll
          for (int yb = 0; yb < kTcL; ++yb) acc[yb] = fmaf(x[yb].x, x[yb].x, fmaf(x[yb].y, x[yb].y, acc[yb]));
          if (q < 3) tmem_wait32(v);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&t_empty[h]);
          if (h == 1) mbar_arrive(&a_empty[b]);  // this warp is done with the stage's twiddles
        }
      }
      if (!ok || *vfail) {
        atomicExch(&fail, 1);
        break;
      }
      float* sqb = sq + bq * kTcRows * kTcSqStride + row * kTcSqStride;
      if (set == 1) {
        if (it >= 2 && !mbar_wait(&sq_empty[bq], ((it >> 1) - 1) & 1)) {
          atomicExch(&fail, 1);
          break;
        }
#pragma unroll
        for (int yb = 0; yb < kTcL; ++yb) sqb[yb] = acc[yb];
        mbar_arrive(&sq_full[bq]);
      } else {
        if (!mbar_wait(&sq_full[bq], (it >> 1) & 1)) {
          atomicExch(&fail, 1);
          break;
        }
#pragma unroll
        for (int yb = 0; yb < kTcL; ++yb) acc[yb] += sqb[yb];
        mbar_arrive(&sq_empty[bq]);
#pragma unroll
        for (int yb = 0; yb < kTcL; ++yb) {
          const int64_t yl = j + ((int64_t)yb << lna);
          const float pv = acc[yb] * pscale;
          a.hist[yl] = widen_nonneg(pv);
          h32.add(pv, a.rk + (yl << a.sh));
        }
      }
    }
    if (set == 0) {  // readout partial of this CTA: the four set-0 warps
      double best = h32.best, wsum = (double)h32.wsum, psum = (double)h32.psum;
      int64_t besty = h32.besty;
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int64_t oy = __shfl_xor_sync(0xffffffffu, besty, off);
        better(best, besty, ob, oy);
        wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
        psum += __shfl_xor_sync(0xffffffffu, psum, off);
      }
      if (lane == 0) sp[lg] = Partial{best, besty, wsum, psum};
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial r = sp[0];
    for (int w = 1; w < 4; ++w) merge_partial(r, sp[w]);
    a.parts[blockIdx.x] = r;
    if (fail) atomicExch(a.err, (int)QPE_ERR_TIMEOUT);
  }
  if (warp == 3)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  pdl_trigger();
}

// --------------------------------------------------------------- host side
size_t tc_top_table_bytes() { return 2 * kTcBBytes; }

// The tensor-core top level: its table operands, then the persistent kernel
// (one CTA per SM, at most one per tile). Returns launches or -1.
static int launch_tc_top(const Instance& in, char* ws, const LevelArgs<float2>& la, cudaStream_t s,
                         cudaEvent_t* top_ev, int64_t* grid_out) {
  void* btab = ws + in.off_tctab;
  const bool fp16 = in.tc_top_prec == QPE_C64_FP16X2;
  if ((fp16 ? launch_k(tc_top_table_kernel<kTcFP16>, dim3(64), dim3(256), 0, s, la.tab, btab)
            : launch_k(tc_top_table_kernel<kTcTF32>, dim3(64), dim3(256), 0, s, la.tab, btab)) != cudaSuccess)
    return -1;
  TcTopArgs a{};
  a.seeds = la.seeds;
  a.btab = static_cast<const uint4*>(btab);
  a.tw_lo = la.tw_lo;
  a.tw_hi = la.tw_hi;
  a.hist = la.hist;
  a.parts = la.parts;
  a.err = reinterpret_cast<int*>(ws + in.off_err);
  a.ntiles = (int64_t(1) << (la.logna - la.sh)) / kTcRows;
  a.nmeas = la.nmeas;
  a.logna = la.logna;
  a.htw = la.htw;
  a.sh = la.sh;
  a.rk = la.rk;
  a.seed_sh = la.seed_sh;
  a.seed_rk = la.seed_rk;
  a.pscale = la.pscale;
  int64_t grid = in.nsm > 0 ? in.nsm : 1;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid > kReduceBlocks) grid = kReduceBlocks;
  if (top_ev && record_event(top_ev[0], s) != cudaSuccess) return -1;
  if ((fp16 ? launch_k(level_tc_top_kernel<kTcFP16>, dim3((unsigned)grid), dim3(kTcThreads), tc_top_smem<kTcFP16>(),
                       s, a)
            : launch_k(level_tc_top_kernel<kTcTF32>, dim3((unsigned)grid), dim3(kTcThreads), tc_top_smem<kTcTF32>(),
                       s, a)) != cudaSuccess)
    return -1;
  if (top_ev && record_event(top_ev[1], s) != cudaSuccess) return -1;
  *grid_out = grid;
  return 2;
}

template <int LD, int M>
static size_t smem_of(size_t esize) {
  return esize == 16 ? LvShape<LD, true, M>::smem(esize) : LvShape<LD, false, M>::smem(esize);
}

size_t level_smem_bytes(int logd, int mode, size_t esize) {
  const int m = mode == 0 ? 0 : 1;
  switch (logd) {
    case 1: return m ? smem_of<1, 1>(esize) : smem_of<1, 0>(esize);
    case 2: return m ? smem_of<2, 1>(esize) : smem_of<2, 0>(esize);
    case 3: return m ? smem_of<3, 1>(esize) : smem_of<3, 0>(esize);
    case 4: return m ? smem_of<4, 1>(esize) : smem_of<4, 0>(esize);
    case 5: return m ? smem_of<5, 1>(esize) : smem_of<5, 0>(esize);
    default: return m ? smem_of<6, 1>(esize) : smem_of<6, 0>(esize);
  }
}

int level_max_bits(int logd, size_t esize, size_t smem_cap) {
  (void)smem_cap;
  return lv_cfg(logd, esize == 16).logl;
}

bool level_sharded(const Instance& in, int li) {
  return in.shard_log > 0 && in.levels[li].logna >= in.shard_log;
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
                           (int)level_smem_bytes(LD, M, sizeof(C)));                                        \
  if (e != cudaSuccess) return e;                                                                           \
  e = cudaFuncSetAttribute(level2_grouped_kernel<C, LD, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                           (int)level_smem_bytes(LD, M, sizeof(C)));                                        \
  if (e != cudaSuccess) return e;
  QPE_LV_ALL(QPE_ATTR, float2)
  QPE_LV_ALL(QPE_ATTR, double2)
#undef QPE_ATTR
  return cudaSuccess;
}

cudaError_t configure_level_kernels() {
  {
    cudaError_t e0 = cudaFuncSetAttribute(level_table_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (2 * 64 * 64 + 2 * 16 * 64) * 16);
    if (e0 != cudaSuccess) return e0;
    e0 = cudaFuncSetAttribute(level_table_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (2 * 64 * 64 + 2 * 16 * 64) * 8);
    if (e0 != cudaSuccess) return e0;
  }
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
  e = cudaFuncSetAttribute(level_tc_top_kernel<kTcFP16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_top_smem<kTcFP16>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(level_tc_top_kernel<kTcTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_top_smem<kTcTF32>());
  if (e != cudaSuccess) return e;
  return set_level_attrs();
}

template <typename C, int M>
static void launch_level2(int logd, unsigned grid, size_t smem, cudaStream_t s, const LevelArgs<C>& a) {
  switch (logd) {
    case 1: launch_k(level2_kernel<C, 1, M>, dim3(grid), dim3(256), smem, s, a); break;
    case 2: launch_k(level2_kernel<C, 2, M>, dim3(grid), dim3(256), smem, s, a); break;
    case 3: launch_k(level2_kernel<C, 3, M>, dim3(grid), dim3(256), smem, s, a); break;
    case 4: launch_k(level2_kernel<C, 4, M>, dim3(grid), dim3(256), smem, s, a); break;
    case 5: launch_k(level2_kernel<C, 5, M>, dim3(grid), dim3(256), smem, s, a); break;
    default: launch_k(level2_kernel<C, 6, M>, dim3(grid), dim3(256), smem, s, a); break;
  }
}

template <typename C>
static int launch_level_tables(const Instance& in, char* ws, int first, int count, cudaStream_t s) {
  const size_t esize = sizeof(C);
  const C* P = reinterpret_cast<const C*>(ws + (esize == 16 ? in.off_pow64 : in.off_pow32));
  TableJobs jobs{};
  jobs.count = count;
  const int D = (int)in.d;
  const int TB = D < 16 ? D : 16;
  int64_t blocks = 0;
  for (int j = 0; j < count; ++j) {
    const Level& L = in.levels[first + j];
    jobs.off[j] = L.off;
    jobs.r[j] = L.r;
    jobs.tab_off[j] = L.tab_off;
    blocks += (int64_t(1) << L.r) * (D / TB);
  }
  const size_t smem = (2 * (size_t)D * D + 2 * (size_t)TB * D) * esize;
  return launch_k(level_table_kernel<C>, dim3((unsigned)blocks), dim3(256), smem, s, P, ws, jobs, in.nmat) ==
                 cudaSuccess
             ? 1
             : -1;
}

template <typename C>
int launch_levels(const Instance& in, char* ws, bool keep_state, cudaStream_t s, cudaEvent_t* top_ev) {
  const size_t esize = sizeof(C);
  const C* tlo = reinterpret_cast<const C*>(ws + (esize == 16 ? in.off_tw_lo64 : in.off_tw_lo32));
  const C* thi = reinterpret_cast<const C*>(ws + (esize == 16 ? in.off_tw_hi64 : in.off_tw_hi32));
  int launches = 0;
  const int nl = (int)in.levels.size();
  if (launch_level_tables<C>(in, ws, 0, nl, s) < 0) return -1;
  ++launches;
  C* seed = reinterpret_cast<C*>(ws + in.zbuf_seed_off);
  if (launch_k(seed_psi_kernel<C>, dim3(1), dim3(64), 0, s, reinterpret_cast<const double2*>(ws + in.off_psi), seed,
               (int)in.d) != cudaSuccess)
    return -1;
  ++launches;
  const LvCfg cfg = lv_cfg(in.nmat, esize == 16);
  const C* cur_seed = seed;
  for (int li = nl - 1; li >= 0; --li) {
    const Level& L = in.levels[li];
    const bool sharded = level_sharded(in, li);
    const bool below_sharded = li + 1 < nl && level_sharded(in, li + 1);
    LevelArgs<C> a{};
    a.sh = sharded ? in.shard_log : 0;
    a.rk = sharded ? in.shard_rank : 0;
    a.seed_sh = (sharded && !below_sharded) ? in.shard_log : 0;
    a.seed_rk = (sharded && !below_sharded) ? in.shard_rank : 0;
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
    const int64_t Na = int64_t(1) << (L.logna - a.sh);  // pencils this rank computes
    if (li > 0) {
      // column groups x pencil groups; the grid is a multiple of the group count
      const int64_t ncg = in.d / cfg.DI0;
      const int64_t iters = (Na + cfg.G0 - 1) / cfg.G0;
      int64_t per = in.level_grid / ncg;
      if (per < 1) per = 1;
      if (per > iters) per = iters;
      C* out = reinterpret_cast<C*>(ws + in.off_zbuf[li & 1]);
      a.xout = out;
      bool on_tc = false;
      if constexpr (sizeof(C) == 16) {
        // FP64 with QPE_FLAG_LEVEL_TC: an 8-point level of at least 128 pencils
        // in all (the same levels with or without sharding)
        if (in.oz_levels && L.r == 3 && L.logna >= 7) {
          if (launch_oz_level(in, ws, a, false, s, nullptr, nullptr) < 0) return -1;
          ++launches;  // the table's digits; the level kernel is counted below
          on_tc = true;
        }
      }
      if (!on_tc) launch_level2<C, 0>(in.nmat, (unsigned)(per * ncg), level_smem_bytes(in.nmat, 0, esize), s, a);
      cur_seed = out;
    } else {
      const size_t smem = level_smem_bytes(in.nmat, 1, esize);
      const int64_t iters = (Na + cfg.G - 1) / cfg.G;
      int64_t grid = iters < in.level_grid ? iters : in.level_grid;
      a.hist = reinterpret_cast<double*>(ws + in.off_hist);
      a.parts = reinterpret_cast<Partial*>(ws + in.off_partials);
      if (grid > kReduceBlocks) grid = kReduceBlocks;
      if (in.tc_top) {
        int r;
        if constexpr (sizeof(C) == 8)
          r = launch_tc_top(in, ws, a, s, top_ev, &grid);
        else
          r = launch_oz_level(in, ws, a, true, s, top_ev, &grid);
        if (r < 0) return -1;
        launches += r;
        finalize_readout(in, ws, (int)grid, s);
        if (cudaPeekAtLastError() != cudaSuccess) return -1;
        ++launches;
        break;
      }
      if (top_ev && record_event(top_ev[0], s) != cudaSuccess) return -1;
      if (keep_state) {
        a.xout = reinterpret_cast<C*>(ws + in.off_state);
        a.xscale = ldexp(1.0, -in.nmeas);  // physical final state: X / N
        launch_level2<C, 2>(in.nmat, (unsigned)grid, smem, s, a);
      } else {
        launch_level2<C, 1>(in.nmat, (unsigned)grid, smem, s, a);
      }
      if (cudaPeekAtLastError() != cudaSuccess) return -1;
      ++launches;
      if (top_ev && record_event(top_ev[1], s) != cudaSuccess) return -1;
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
  const size_t smem = level_smem_bytes(logd, 1, sizeof(C));
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

void level_shape(int logd, int mode, size_t esize, int* DI, int* G) {
  const LvCfg c = lv_cfg(logd, esize == 16);
  *DI = mode == 0 ? c.DI0 : (1 << logd);
  *G = mode == 0 ? c.G0 : c.G;
}

template <typename C, int M>
static cudaError_t launch_grouped_m(int logd, unsigned grid, size_t smem, cudaStream_t s, const LevelArgs<C>* args,
                                    const GroupItem* items, int n) {
  switch (logd) {
    case 1: return launch_k(level2_grouped_kernel<C, 1, M>, dim3(grid), dim3(256), smem, s, args, items, n);
    case 2: return launch_k(level2_grouped_kernel<C, 2, M>, dim3(grid), dim3(256), smem, s, args, items, n);
    case 3: return launch_k(level2_grouped_kernel<C, 3, M>, dim3(grid), dim3(256), smem, s, args, items, n);
    case 4: return launch_k(level2_grouped_kernel<C, 4, M>, dim3(grid), dim3(256), smem, s, args, items, n);
    case 5: return launch_k(level2_grouped_kernel<C, 5, M>, dim3(grid), dim3(256), smem, s, args, items, n);
    default: return launch_k(level2_grouped_kernel<C, 6, M>, dim3(grid), dim3(256), smem, s, args, items, n);
  }
}

template <typename C>
int launch_level_grouped(const LevelLaunch& L, const LevelArgs<C>* args, const GroupItem* items, cudaStream_t s) {
  if (L.nitems <= 0) return 0;
  const size_t smem = level_smem_bytes(L.logd, L.mode, sizeof(C));
  cudaError_t e;
  if (L.mode == 0)
    e = launch_grouped_m<C, 0>(L.logd, (unsigned)L.grid, smem, s, args, items, L.nitems);
  else if (L.mode == 1)
    e = launch_grouped_m<C, 1>(L.logd, (unsigned)L.grid, smem, s, args, items, L.nitems);
  else
    e = launch_grouped_m<C, 2>(L.logd, (unsigned)L.grid, smem, s, args, items, L.nitems);
  return e == cudaSuccess ? 1 : -1;
}
template int launch_level_grouped<float2>(const LevelLaunch&, const LevelArgs<float2>*, const GroupItem*, cudaStream_t);
template int launch_level_grouped<double2>(const LevelLaunch&, const LevelArgs<double2>*, const GroupItem*,
                                           cudaStream_t);

template <typename C, int M>
static int occ_m(int logd) {
  int blocks = 0;
  const size_t smem = level_smem_bytes(logd, M, sizeof(C));
  cudaError_t e;
  switch (logd) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_grouped_kernel<C, 1, M>, 256, smem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_grouped_kernel<C, 2, M>, 256, smem); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_grouped_kernel<C, 3, M>, 256, smem); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_grouped_kernel<C, 4, M>, 256, smem); break;
    case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_grouped_kernel<C, 5, M>, 256, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, level2_grouped_kernel<C, 6, M>, 256, smem); break;
  }
  return (e == cudaSuccess && blocks > 0) ? blocks : 1;
}

template <typename C>
int level_grouped_occupancy(int logd, int mode) {
  return mode == 0 ? occ_m<C, 0>(logd) : (mode == 1 ? occ_m<C, 1>(logd) : occ_m<C, 2>(logd));
}
template int level_grouped_occupancy<float2>(int, int);
template int level_grouped_occupancy<double2>(int, int);

template int launch_levels<float2>(const Instance&, char*, bool, cudaStream_t, cudaEvent_t*);
template int launch_levels<double2>(const Instance&, char*, bool, cudaStream_t, cudaEvent_t*);

}  // namespace qpe
