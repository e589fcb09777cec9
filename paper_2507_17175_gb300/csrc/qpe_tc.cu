// Tensor-core controlled-gate GEMM for large target registers (sm_103a
// tcgen05 + TMA), used by the split-precision plans (QPE_C64_TF32X3,
// QPE_C64_FP16X2) in the doubling schedule:
//
//   rows [2^j, 2^(j+1)) of the state  =  rows [0, 2^j)  x  P_j^T,
//
// written over reals: a complex64 row is 2d interleaved floats (re, im, ...)
// and P_j becomes the 2d x 2d real matrix B with B[2i][2k] = Re P[i][k],
// B[2i][2k+1] = -Im P[i][k], B[2i+1][2k] = Im P[i][k], B[2i+1][2k+1] = Re P[i][k]
// (stored n-major: row n holds the weights of output column n), so
// out[m][n] = sum_kk A[m][kk] B[n][kk]. Each operand x is split into
// hi = round(x) and lo = round(x - hi) in the tensor type (tf32 or fp16);
// the product A B^T is accumulated in FP32 in tensor memory as
// A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T (the lo lo term is below the FP32
// accumulator's resolution). The hi.hi pass and the cross pass (the two cross
// products into one accumulator, i.e. [A_hi | A_lo] [B_lo ; B_hi]^T over a
// doubled K) are the two passes of the FP16x2 scheme. fp16 has 5 exponent
// bits, so its operands are scaled by powers of two first: each A row so that
// its largest |entry| lies in [2^14, 2^15), B (entries of a unitary, |.| <= 1)
// by 2^14; the drain multiplies each output row by the exact inverse.
//
// Kernel: one CTA per 128 x BN output tile (BN <= 128), 320 threads. Warp 0
// lane 0 issues TMA loads of the K-slabs A_hi, A_lo, B_hi, B_lo (128-byte
// swizzled, one ring stage per K-block, 3 or 4 stages); warp 1 lane 0
// issues tcgen05.mma (M = 128, N = BN, K = 32 bytes per instruction) into
// double-buffered FP32 tensor-memory accumulators (hi.hi drained after every
// two instructions, the cross terms every 8 K-blocks); warps 2..9 drain each
// finished buffer with tcgen05.ld into FP32 registers (correctly rounded adds)
// and store the rows at the end. Every mbarrier wait
// is bounded; on expiry the CTA records QPE_ERR_TIMEOUT in the device error
// word, frees its tensor memory and returns.
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "qpe_internal.cuh"
#include "qpe_tcgen05.cuh"

namespace qpe {

namespace {

constexpr int kStages = 4;  // most stages of any ring below

// Stages of the controlled-gate GEMM's ring: one stage holds the four operand
// tiles of a K-block (A_hi, A_lo, B_hi, B_lo), 64 KiB for BN = 128.
template <int BN>
__host__ __device__ constexpr int tc_stages() { return BN == 128 ? 3 : 4; }
}  // namespace

using namespace tcg;

// D[m][n] (FP32, leading dimension ldd floats) for rows m < M of the tile grid
// = sum over the 3 operand pairs of A_pair[m][:] . B_pair[n][:], K = 2d.
//
// The tensor-core accumulator drops low-order bits on every accumulation
// step, so nothing is left to accumulate there for long: the dominant
// hi.hi product goes, two MMA instructions (32 elements of K for 16-bit
// types) at a time, to one of two "main" tensor-memory buffers and is added
// into correctly rounded FP32 registers right after; the two cross products
// (about 2^-11 smaller) go to one of two "cross" buffers drained every KPC
// K-blocks. Eight drain warps do the adds while the next MMAs run. (Draining
// after every instruction instead halves the histogram error again but makes
// the kernel drain-bound, about twice slower.)
//   warp 0 lane 0   TMA producer (one stage = the four operand tiles of a K-block)
//   warp 1 lane 0   MMA issuer
//   warps 2..9      drain + epilogue; warp w owns tensor-memory lanes
//                   32 (w % 4) .. +31, i.e. tile rows 32 (w % 4) .. +31, and
//                   the column half (w - 2) / 4 of the tile
// Tiles are visited in groups of kGroupM row tiles by all column tiles so the
// operand panels in flight stay in L2.
constexpr int kGroupM = 8;
constexpr int kKPC = 8;  // K-blocks per cross-term chunk
constexpr int kMS = 2;   // hi.hi drains per K-block (every 2 MMA instructions)
constexpr int kTcDrainWarps = 8;  // 4 lane quarters x 2 column halves

template <int KIND, int BN>
__device__ __forceinline__ void tc_gemm_tile(const CUtensorMap* mapAhi, const CUtensorMap* mapAlo,
                                             const CUtensorMap* mapBhi, const CUtensorMap* mapBlo,
                                             float* __restrict__ D, int64_t ldd, int64_t M, int K,
                                             int* __restrict__ err, const float* __restrict__ row_scale,
                                             int64_t bid) {
  constexpr int ESZ = KIND == kTcTF32 ? 4 : 2;
  constexpr int BK = 128 / ESZ;       // K elements per 128-byte swizzle row
  constexpr int A_BYTES = kBM * 128;  // 16 KiB
  constexpr int B_BYTES = BN * 128;
  constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);  // A_hi, A_lo, B_hi, B_lo of one K-block
  constexpr int QS = tc_stages<BN>();
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* ring =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full_bar[kStages], empty_bar[kStages];
  __shared__ uint64_t main_full[2], main_empty[2], cross_full[2], cross_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped raster: kGroupM row tiles x all column tiles per group
  const int64_t m_tiles = (M + kBM - 1) / kBM;
  const int n_tiles = (int)(ldd / BN);
  int64_t m_tile, n_tile;
  {
    const int64_t per_group = (int64_t)kGroupM * n_tiles;
    const int64_t g = bid / per_group;
    const int64_t first = g * kGroupM;
    const int64_t gm = (m_tiles - first) < kGroupM ? (m_tiles - first) : kGroupM;
    const int64_t local = bid - g * per_group;
    m_tile = first + local % gm;
    n_tile = local / gm;
  }
  const int64_t m0 = m_tile * kBM;
  const int n0 = (int)n_tile * BN;
  const int kblocks = K / BK;
  const int nchunks_x = (kblocks + kKPC - 1) / kKPC;

  if (threadIdx.x == 0) {
    for (int s = 0; s < QS; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&main_full[b], 1);
      mbar_init(&main_empty[b], kTcDrainWarps);
      mbar_init(&cross_full[b], 1);
      mbar_init(&cross_empty[b], kTcDrainWarps);
    }
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)(4 * BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // tensor-memory columns: main buffers [0, 2 BN), cross buffers [2 BN, 4 BN)

  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < kblocks; ++kb) {
        const int st = kb % QS;
        if (kb >= QS && !mbar_wait(&empty_bar[st], ((kb / QS) - 1) & 1)) {
          atomicExch(&fail, 1);
          break;
        }
        if (*((volatile int*)&fail)) break;
        unsigned char* sa = ring + st * STAGE_BYTES;
        mbar_expect_tx(&full_bar[st], STAGE_BYTES);
        tma_load_2d(sa, mapAhi, &full_bar[st], kb * BK, (int)m0);
        tma_load_2d(sa + A_BYTES, mapAlo, &full_bar[st], kb * BK, (int)m0);
        tma_load_2d(sa + 2 * A_BYTES, mapBhi, &full_bar[st], kb * BK, n0);
        tma_load_2d(sa + 2 * A_BYTES + B_BYTES, mapBlo, &full_bar[st], kb * BK, n0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc<KIND, BN>();
      for (int kb = 0; kb < kblocks; ++kb) {
        const int cx = kb / kKPC, bx = cx & 1;    // cross chunk and its buffer
        const bool cx_first = (kb % kKPC) == 0;
        const bool cx_last = (kb % kKPC) == kKPC - 1 || kb == kblocks - 1;
        if (cx_first && cx >= 2 && !mbar_wait(&cross_empty[bx], ((cx >> 1) - 1) & 1)) {
          atomicExch(&fail, 1);
          break;
        }
        const int st = kb % QS;
        if (!mbar_wait(&full_bar[st], (kb / QS) & 1)) {
          atomicExch(&fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = smem_u32(ring + st * STAGE_BYTES);
        bool ok = true;
        {  // hi.hi: kMS groups of 4 / kMS instructions, each group into its own main buffer
          const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + 2 * A_BYTES);
          for (int gs = 0; gs < kMS; ++gs) {
            const int j = kb * kMS + gs, bm = j & 1;
            if (j >= 2 && !mbar_wait(&main_empty[bm], ((j >> 1) - 1) & 1)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < 4 / kMS; ++kk) {
              const int k = gs * (4 / kMS) + kk;
              umma_k<KIND>(tmem + (uint32_t)(bm * BN), ad + 2 * k, bd + 2 * k, idesc, kk == 0 ? 0u : 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&main_full[bm]))
                         : "memory");
          }
        }
        if (!ok) {
          atomicExch(&fail, 1);
          break;
        }
        for (int pr = 1; pr < 3; ++pr) {  // (hi, lo), (lo, hi) into the cross buffer
          const uint64_t ad = sw128_desc(pr == 2 ? sa + A_BYTES : sa);
          const uint64_t bd = sw128_desc(sa + 2 * A_BYTES + (pr == 1 ? B_BYTES : 0));
          const uint32_t acc_addr = tmem + (uint32_t)((2 + bx) * BN);
#pragma unroll
          for (int k = 0; k < 4; ++k) {  // 32 bytes of K per instruction
            const bool fresh = k == 0 && pr == 1 && cx_first;
            umma_k<KIND>(acc_addr, ad + 2 * k, bd + 2 * k, idesc, fresh ? 0u : 1u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&empty_bar[st]))
                     : "memory");
        if (cx_last)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&cross_full[bx]))
                       : "memory");
      }
    }
  } else {
    // drain warps: add finished buffers into FP32 registers
    const int lg = warp & 3;  // tensor-memory lane group (fixed by the warp's rank)
    constexpr int CW = BN / 2;  // columns of this drain warp
    const int ch = (warp - 2) >> 2;  // column half
    float acc[CW];
#pragma unroll
    for (int i = 0; i < CW; ++i) acc[i] = 0.f;
    bool ok = true;
    auto drain = [&](uint64_t* full, uint64_t* empty, uint32_t parity, uint32_t col0) -> bool {
      bool got = mbar_wait(full, parity);
      got = __all_sync(0xffffffffu, got && !*((volatile int*)&fail)) != 0;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!got) return false;
#pragma unroll
      for (int q = 0; q < CW / 32; ++q) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + col0 + (uint32_t)(ch * CW + q * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
            "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[q * 32 + i] += __uint_as_float(v[i]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(empty)) : "memory");
      return true;
    };
    for (int kb = 0; kb < kblocks && ok; ++kb) {
      for (int gs = 0; gs < kMS && ok; ++gs) {
        const int j = kb * kMS + gs, bm = j & 1;
        ok = drain(&main_full[bm], &main_empty[bm], (j >> 1) & 1, (uint32_t)(bm * BN));
      }
      const int cx = kb / kKPC, bx = cx & 1;
      const bool cx_last = (kb % kKPC) == kKPC - 1 || kb == kblocks - 1;
      if (ok && cx_last) ok = drain(&cross_full[bx], &cross_empty[bx], (cx >> 1) & 1, (uint32_t)((2 + bx) * BN));
    }
    (void)nchunks_x;
    const int64_t row = m0 + lg * 32 + lane;
    if (ok && row < M) {
      if constexpr (KIND == kTcFP16) {  // undo the power-of-two operand scales (exact)
        const float sc = row_scale[row];
#pragma unroll
        for (int i = 0; i < CW; ++i) acc[i] *= sc;
      }
      float4* dst = reinterpret_cast<float4*>(D + row * ldd + n0 + ch * CW);
#pragma unroll
      for (int q = 0; q < CW / 4; ++q) dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
    if (!ok) atomicExch(&fail, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (fail && threadIdx.x == 0) atomicExch(err, (int)QPE_ERR_TIMEOUT);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(4 * BN))
                 : "memory");
  }
}

template <int KIND, int BN>
__global__ void __launch_bounds__(64 + 32 * kTcDrainWarps, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapAhi, const __grid_constant__ CUtensorMap mapAlo,
                   const __grid_constant__ CUtensorMap mapBhi, const __grid_constant__ CUtensorMap mapBlo,
                   float* __restrict__ D, int64_t ldd, int64_t M, int K, int* __restrict__ err,
                   const float* __restrict__ row_scale) {
  pdl_begin();
  tc_gemm_tile<KIND, BN>(&mapAhi, &mapAlo, &mapBhi, &mapBlo, D, ldd, M, K, err, row_scale, blockIdx.x);
  pdl_trigger();
}

// Acquire a tensor map that the host wrote into global memory before the
// launch, for the TMA (tensor-map) proxy.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(m))
               : "memory");
}

// One doubling level on the tensor cores for every listed instance (batched
// plans): item i owns CTAs [tile0, tile0 + tiles) of the launch; its four
// operand tensor maps live in the item (global memory, written at bind).
template <int KIND, int BN>
__global__ void __launch_bounds__(64 + 32 * kTcDrainWarps, 1)
    tc_gemm_grouped_kernel(const TcGemmItem* __restrict__ items, int nitems) {
  pdl_begin();
  const int i = find_item(items, nitems, blockIdx.x);
  const TcGemmItem* it = items + i;
  if (threadIdx.x == 0) {
    tensormap_acquire(&it->mAh);
    tensormap_acquire(&it->mAl);
    tensormap_acquire(&it->mBh);
    tensormap_acquire(&it->mBl);
  }
  __syncthreads();
  tc_gemm_tile<KIND, BN>(&it->mAh, &it->mAl, &it->mBh, &it->mBl, it->D, it->ldd, it->M, it->K, it->err,
                         it->row_scale, blockIdx.x - it->tile0);
  pdl_trigger();
}

// ------------------------------------------------------- operand splits
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// A rows (complex64 = 2d interleaved floats) -> tf32 hi / lo
__global__ void split_rows_tf32_kernel(const float* __restrict__ src, float* __restrict__ hi, float* __restrict__ lo,
                                       int64_t count) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float x = src[i];
    const float h = tf32_round(x);
    hi[i] = h;
    lo[i] = tf32_round(x - h);
  }
  pdl_trigger();
}

// A rows -> fp16 hi / lo after scaling each row by 2^e so that its largest
// |entry| lies in [2^14, 2^15); inv_scale[row] = 2^-(e + 14) undoes both
// operand scales. One warp per row (width floats, a multiple of 4).
// one row (width floats) by one warp
__device__ __forceinline__ void split_row_fp16(const float* __restrict__ src, __half* __restrict__ hi,
                                               __half* __restrict__ lo, float* __restrict__ inv_scale, int64_t r,
                                               int width, int lane) {
  {
    const float* row = src + r * width;
    float mx = 0.f;
    for (int c = lane * 4; c < width; c += 128) {
      const float4 v = *reinterpret_cast<const float4*>(row + c);
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // floor(log2(mx)) from the exponent field; zero / tiny rows keep scale 1
    const int ex = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 127;
    const int e = (ex < -100 || ex > 100) ? 0 : 14 - ex;
    const float sc = __uint_as_float((uint32_t)(127 + e) << 23);
    if (lane == 0) inv_scale[r] = __uint_as_float((uint32_t)(127 - e - 14) << 23);
    for (int c = lane * 4; c < width; c += 128) {
      const float4 v = *reinterpret_cast<const float4*>(row + c);
      const float x[4] = {v.x * sc, v.y * sc, v.z * sc, v.w * sc};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const __half h = __float2half_rn(x[t]);
        hi[r * width + c + t] = h;
        lo[r * width + c + t] = __float2half_rn(x[t] - __half2float(h));
      }
    }
  }
}

__global__ void split_rows_fp16_kernel(const float* __restrict__ src, __half* __restrict__ hi,
                                       __half* __restrict__ lo, float* __restrict__ inv_scale, int64_t rows,
                                       int width) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps)
    split_row_fp16(src, hi, lo, inv_scale, r, width, lane);
  pdl_trigger();
}

// P (d x d complex128) -> real embedding B (2d x 2d, n-major) split hi / lo
// element e of P's real embedding (2d x 2d, n-major) split into hi / lo
template <int KIND>
__device__ __forceinline__ void embed_split_elem(const double2* __restrict__ P, void* __restrict__ hi,
                                                 void* __restrict__ lo, int d, int64_t e) {
  const int64_t n2 = 2 * (int64_t)d;
  const int64_t n = e / n2, kk = e - n * n2;
  const int64_t i = n >> 1, k = kk >> 1;
  const double2 p = P[i * d + k];
  const int c = (int)(n & 1), cp = (int)(kk & 1);
  // [[re, -im], [im, re]]
  const double v = c == 0 ? (cp == 0 ? p.x : -p.y) : (cp == 0 ? p.y : p.x);
  if constexpr (KIND == kTcTF32) {
    const float h = tf32_round((float)v);
    reinterpret_cast<float*>(hi)[e] = h;
    reinterpret_cast<float*>(lo)[e] = tf32_round((float)(v - (double)h));
  } else {
    static_assert(KIND == kTcFP16, "gate GEMM operands are tf32 or fp16");
    const double vs = v * 16384.0;  // 2^14, exact
    const __half h = __float2half_rn((float)vs);
    reinterpret_cast<__half*>(hi)[e] = h;
    reinterpret_cast<__half*>(lo)[e] = __float2half_rn((float)(vs - (double)__half2float(h)));
  }
}

template <int KIND>
__global__ void embed_split_kernel(const double2* __restrict__ P, void* __restrict__ hi, void* __restrict__ lo,
                                   int d) {
  pdl_begin();
  const int64_t n2 = 2 * (int64_t)d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2 * n2; e += (int64_t)gridDim.x * blockDim.x)
    embed_split_elem<KIND>(P, hi, lo, d, e);
  pdl_trigger();
}

// The operand splits of one tensor-core level for every listed instance:
// warps take the A rows of all items (row0 numbering), threads the embedding
// elements of all items (e0 numbering).
template <int KIND>
__global__ void split_grouped_kernel(const TcSplitItem* __restrict__ items, int nitems, int64_t rows, int64_t elems) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const TcSplitItem& it = items[find_item(items, nitems, r)];
    const int64_t lr = r - it.row0;
    if constexpr (KIND == kTcFP16) {
      split_row_fp16(it.S, static_cast<__half*>(it.hi), static_cast<__half*>(it.lo), it.inv_scale, lr, it.width,
                     lane);
    } else {
      const float* row = it.S + lr * it.width;
      float* h = static_cast<float*>(it.hi) + lr * it.width;
      float* l = static_cast<float*>(it.lo) + lr * it.width;
      for (int c = lane; c < it.width; c += 32) {
        const float x = row[c];
        const float hv = tf32_round(x);
        h[c] = hv;
        l[c] = tf32_round(x - hv);
      }
    }
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < elems; e += (int64_t)gridDim.x * blockDim.x) {
    int lo_i = 0, hi_i = nitems - 1;  // item with e0 <= e
    while (lo_i < hi_i) {
      const int mid = (lo_i + hi_i + 1) >> 1;
      if (items[mid].e0 <= e)
        lo_i = mid;
      else
        hi_i = mid - 1;
    }
    const TcSplitItem& it = items[lo_i];
    embed_split_elem<KIND>(it.P, it.bhi, it.blo, it.d, e - it.e0);
  }
  pdl_trigger();
}

// ------------------------------------- FP64-accurate squaring (Ozaki scheme)
// P_(k+1) = P_k^2 on the tensor cores with the accuracy of an FP64 product.
// Over reals, with E = [[Re P, -Im P], [Im P, Re P]] (2d x 2d), the first d
// columns of E^2 are [Re P^2 ; Im P^2]; so out = E (2d x 2d) times
// B^T, B[n][kk] = E[kk][n] (n < d, K-major). Every entry of row m of E is
// written as x = 2^(tau_m - 55) sum_{s=0..6} a_s 2^(8 (6 - s)) with balanced
// integer digits |a_s| <= 128 (round to nearest at 2^(tau_m - 55), |x| <
// 2^tau_m), and every entry of column n of B likewise (digits b_t) with
// sigma_n. Digits are exact in bf16 and the product of two is an exact integer
// of at most 2^14, so tcgen05 MMAs with FP32 accumulation sum them exactly as
// long as every partial sum stays below 2^24. A digit pair (s, t) has weight
// w = s + t: out = 2^(tau_m + sigma_n + 2) sum_w acc_w 2^(-8 w - 16), acc_w
// the integer sum of the pairs of weight w over K. The pairs with w <= 6 are
// formed (28 bf16 products); the rest lie below 2^-53 of 2^(tau + sigma) K.
constexpr int kOzS = 7;       // digits per operand entry
constexpr int kOzBeta = 8;    // bits per digit

__device__ __forceinline__ double pow2d(int e) {  // 2^e for -1022 <= e <= 1023
  return __longlong_as_double((long long)(1023 + e) << 52);
}

// exponent t with 0 < |x| < 2^t for the largest |x| of a row or column; tiny
// or zero lines get a floor (their digits are all zero)
__device__ __forceinline__ int oz_exponent(double mx) {
  if (!(mx > 0x1p-900)) return -900;
  const int eb = (int)((__double_as_longlong(mx) >> 52) & 0x7ff) - 1023;
  return eb + 1;
}

// tau[i]: scale of rows i and i + d of E (from row i of P); sig[j]: of column
// j of [Re P ; Im P]. A non-finite entry sets the error word.
__device__ __forceinline__ void oz_scale_block(const double2* __restrict__ P, int d, int* __restrict__ tau,
                                               int* __restrict__ sig, int* __restrict__ err, int b) {
  double mx = 0.0;
  bool finite = true;
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    const double2 p = b < d ? P[(int64_t)b * d + k] : P[(int64_t)k * d + (b - d)];
    finite = finite && isfinite(p.x) && isfinite(p.y);
    mx = fmax(mx, fmax(fabs(p.x), fabs(p.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ double wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  if (__syncthreads_or(!finite) && threadIdx.x == 0) atomicCAS(err, 0, (int)QPE_ERR_NUMERIC);
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, wm[w]);
    mx = fmax(mx, wm[0]);
    const int e = oz_exponent(mx);
    if (b < d)
      tau[b] = e;
    else
      sig[b - d] = e;
  }
}

__global__ void __launch_bounds__(256) oz_scale_kernel(const double2* __restrict__ P, int d, int* __restrict__ tau,
                                                       int* __restrict__ sig, int* __restrict__ err) {
  pdl_begin();
  oz_scale_block(P, d, tau, sig, err, blockIdx.x);
  pdl_trigger();
}

// balanced base-2^8 digits of x at scale 2^t, most significant first:
// out[s * stride], s = 0 .. kOzS - 1
__device__ __forceinline__ void oz_digits(double x, int t, __nv_bfloat16* out, int64_t stride) {
  long long F = __double2ll_rn(x * pow2d(kOzS * kOzBeta - 1 - t));  // |F| < 2^55
#pragma unroll
  for (int s = kOzS - 1; s >= 1; --s) {
    long long r = F & 255;
    if (r >= 128) r -= 256;
    out[(int64_t)s * stride] = __float2bfloat16_rn((float)r);
    F = (F - r) / 256;
  }
  out[0] = __float2bfloat16_rn((float)F);
}

// digits of E (rows 2d, K = 2d) per slice: A[(s 2d + m) 2d + kk]; also the
// complex64 copy of P when A32 is given
__device__ __forceinline__ void oz_slice_a_elem(const double2* __restrict__ P, int d, const int* __restrict__ tau,
                                                __nv_bfloat16* __restrict__ A, float2* __restrict__ A32, int64_t e) {
  const int64_t d2 = 2 * (int64_t)d, stride = d2 * d2;
  {
    const int64_t i = e / d, j = e - i * d;
    const double2 p = P[e];
    if (A32) A32[e] = make_float2((float)p.x, (float)p.y);
    const int t = tau[i];
    oz_digits(p.x, t, A + i * d2 + j, stride);             // E[i][j]     = Re
    oz_digits(p.x, t, A + (i + d) * d2 + j + d, stride);   // E[i+d][j+d] = Re
    oz_digits(-p.y, t, A + i * d2 + j + d, stride);        // E[i][j+d]   = -Im
    oz_digits(p.y, t, A + (i + d) * d2 + j, stride);       // E[i+d][j]   = Im
  }
}

__global__ void __launch_bounds__(256) oz_slice_a_kernel(const double2* __restrict__ P, int d,
                                                         const int* __restrict__ tau, __nv_bfloat16* __restrict__ A,
                                                         float2* __restrict__ A32) {
  pdl_begin();
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < dd; e += (int64_t)gridDim.x * blockDim.x)
    oz_slice_a_elem(P, d, tau, A, A32, e);
  pdl_trigger();
}

// digits of B (rows d, K = 2d): B[(s d + n) 2d + kk] = digits of E[kk][n]
__device__ __forceinline__ void oz_slice_b_elem(const double2* __restrict__ P, int d, const int* __restrict__ sig,
                                                __nv_bfloat16* __restrict__ B, int64_t e) {
  const int64_t d2 = 2 * (int64_t)d, stride = (int64_t)d * d2;
  {
    const int64_t n = e / d, kk = e - n * d;  // consecutive threads: consecutive kk (contiguous writes)
    const double2 p = P[kk * d + n];
    const int t = sig[n];
    oz_digits(p.x, t, B + n * d2 + kk, stride);      // E[kk][n]   = Re P[kk][n]
    oz_digits(p.y, t, B + n * d2 + kk + d, stride);  // E[kk+d][n] = Im P[kk][n]
  }
}

__global__ void __launch_bounds__(256) oz_slice_b_kernel(const double2* __restrict__ P, int d,
                                                         const int* __restrict__ sig, __nv_bfloat16* __restrict__ B) {
  pdl_begin();
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < dd; e += (int64_t)gridDim.x * blockDim.x)
    oz_slice_b_elem(P, d, sig, B, e);
  pdl_trigger();
}


// Digits of state row r for a gate level: [Re S_r | Im S_r] (2d reals) at the
// row's own scale tau[r], A[(s M + r) 2d + k]; the whole CTA takes part. A
// non-finite entry sets the error word.
__device__ __forceinline__ void oz_slice_row(const double2* __restrict__ S, int64_t M, int d, int* __restrict__ tau,
                                             __nv_bfloat16* __restrict__ A, int* __restrict__ err, int64_t r) {
  __shared__ double wm[8];
  __shared__ int t_s;
  const double2* row = S + r * d;
  double mx = 0.0;
  bool finite = true;
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    const double2 p = row[k];
    finite = finite && isfinite(p.x) && isfinite(p.y);
    mx = fmax(mx, fmax(fabs(p.x), fabs(p.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  if (__syncthreads_or(!finite) && threadIdx.x == 0) atomicCAS(err, 0, (int)QPE_ERR_NUMERIC);
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, wm[w]);
    t_s = oz_exponent(fmax(mx, wm[0]));
    tau[r] = t_s;
  }
  __syncthreads();
  const int t = t_s;
  const int64_t stride = M * 2 * (int64_t)d;
  __nv_bfloat16* out = A + r * 2 * (int64_t)d;
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    const double2 p = row[k];
    oz_digits(p.x, t, out + k, stride);
    oz_digits(p.y, t, out + d + k, stride);
  }
  __syncthreads();  // wm and t_s are reused by the next row
}

__global__ void __launch_bounds__(256) oz_slice_rows_kernel(const double2* __restrict__ S, int64_t M, int d,
                                                            int* __restrict__ tau, __nv_bfloat16* __restrict__ A,
                                                            int* __restrict__ err) {
  pdl_begin();
  for (int64_t r = blockIdx.x; r < M; r += gridDim.x) oz_slice_row(S, M, d, tau, A, err, r);
  pdl_trigger();
}

// The state rows of every listed instance (batched gate level): global row
// g of the launch is row g - tile0 of its item.
__global__ void __launch_bounds__(256) oz_slice_rows_grouped_kernel(const RowSliceItem* __restrict__ items,
                                                                    int nitems, int64_t rows) {
  pdl_begin();
  for (int64_t g = blockIdx.x; g < rows; g += gridDim.x) {
    const RowSliceItem& it = items[find_item(items, nitems, g)];
    oz_slice_row(it.S, it.M, it.d, it.tau, static_cast<__nv_bfloat16*>(it.A), it.err, g - it.tile0);
  }
  pdl_trigger();
}

// One CTA per 128 x 64 tile of out (rows m0.. of E, columns n0.. < d).
// K-block by K-block (64 elements of K), every digit tile is loaded once: the
// seven B digit tiles of the K-block (resident, two buffers) and the seven A
// digit tiles one after another through a ring; A digit s meets B digits
// t = 0 .. 6 - s, and pair (s, t) goes into the tensor-memory accumulator of
// weight w = s + t (64 columns each, 448 in all). Weight w is complete for the
// K-block once A digit w has been used, so the weights finish in order and
// the drain of one overlaps the MMAs of the next.
// An accumulator holds (w + 1) pairs per K-block, each at most 64 * 2^14, so
// it stays an exact FP32 integer (below 2^24) over a window of win_w
// K-blocks, (w + 1) * win_w < 16; the drain reads it once per window.
// Drain warps 2 .. 9 (two per tensor-memory lane quarter, 32 columns each)
// convert the window sums to integers and add them into two int64 sums per
// column, hi = sum_(w <= 2) acc_w 2^(8 (2 - w)) and lo = sum_(w >= 3) acc_w
// 2^(8 (6 - w)) (below 2^44 and 2^54 for K <= 8192); at the end
// val = hi 2^-32 + lo 2^-64 and out = val 2^(tau_m + sigma_n + 2).
// Warp 0 lane 0 issues the TMA loads, warp 1 lane 0 the MMAs.
constexpr int kOzBN = 64;
constexpr int kOzAStages = 6;
constexpr int kOzThreads = 320;
constexpr int kOzA = kBM * 128;              // one A digit tile, 16 KiB
constexpr int kOzB = kOzBN * 128;            // one B digit tile, 8 KiB
constexpr int kOzBSet = kOzS * kOzB;         // the seven B digit tiles of a K-block
// Window of weight w's accumulator in K-blocks (8, 4, 4, 2, 2, 2, 2) and its
// phase: window j of weight w covers the K-blocks kb with
// (kb + off_w) >> log2(win_w) = j (the first one shorter when off_w > 0). The
// phases spread the drains over the K-blocks (two or three at each boundary)
// instead of all seven at once.
template <int W>
__host__ __device__ constexpr int oz_log_win() { return W == 0 ? 3 : (W <= 2 ? 2 : 1); }
template <int W>
__host__ __device__ constexpr int oz_win() { return 1 << oz_log_win<W>(); }
template <int W>
__host__ __device__ constexpr int oz_off() { return W == 0 ? 2 : (W == 1 ? 1 : (W == 2 ? 3 : (W & 1) ^ 1)); }
static_assert((0 + 1) * oz_win<0>() < 16 && (2 + 1) * oz_win<2>() < 16 && (6 + 1) * oz_win<6>() < 16,
              "window sums must stay below 2^24");

template <int W>
__device__ __forceinline__ int oz_window(int kb) { return (kb + oz_off<W>()) >> oz_log_win<W>(); }
template <int W>
__device__ __forceinline__ bool oz_window_start(int kb) {
  return kb == 0 || ((kb + oz_off<W>()) & (oz_win<W>() - 1)) == 0;
}
template <int W>
__device__ __forceinline__ bool oz_window_end(int kb, int kblocks) {
  return ((kb + 1 + oz_off<W>()) & (oz_win<W>() - 1)) == 0 || kb + 1 == kblocks;
}

// The MMAs of A digit S against B digits T .. 6 - S (one K-block): pair
// (S, T) into the accumulator of weight S + T, four K = 16 steps. The first
// pair of a window (S = 0) overwrites the accumulator, after waiting for the
// drain of the window before. False if that wait runs out.
template <int S, int T>
__device__ __forceinline__ bool oz_mma_pairs(uint32_t tmem, uint64_t ad, uint64_t bd0, uint32_t idesc, int kb,
                                             uint64_t* acc_empty) {
  if constexpr (S + T < kOzS) {
    constexpr int w = S + T;
    bool fresh = false;
    if constexpr (S == 0) {
      fresh = oz_window_start<w>(kb);
      if (fresh && kb > 0) {
        if (!mbar_wait(&acc_empty[w], (oz_window<w>(kb) - 1) & 1)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
    }
    const uint64_t bd = bd0 + (uint64_t)(T * (kOzB >> 4));
#pragma unroll
    for (int k = 0; k < 4; ++k)
      umma_k<kTcBF16>(tmem + (uint32_t)(w * kOzBN), ad + 2 * k, bd + 2 * k, idesc, (fresh && k == 0) ? 0u : 1u);
    return oz_mma_pairs<S, T + 1>(tmem, ad, bd0, idesc, kb, acc_empty);
  }
  return true;
}

// A digits S .. 6 of one K-block: wait for the digit's ring stage, its pairs,
// release the stage, and signal weight S complete at the end of its window.
template <int S>
__device__ __forceinline__ bool oz_mma_digits(uint32_t tmem, uint64_t a_desc0, uint64_t bd0, uint32_t idesc, int kb,
                                              int kblocks, int& stage, uint32_t& phase, uint64_t* a_full,
                                              uint64_t* a_empty, uint64_t* acc_full, uint64_t* acc_empty) {
  if constexpr (S < kOzS) {
    if (!mbar_wait(&a_full[stage], phase)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint64_t ad = a_desc0 + (uint64_t)(stage * (kOzA >> 4));
    if (!oz_mma_pairs<S, 0>(tmem, ad, bd0, idesc, kb, acc_empty)) return false;
    umma_commit(&a_empty[stage]);
    if (oz_window_end<S>(kb, kblocks)) umma_commit(&acc_full[S]);  // weight S is complete
    if (++stage == kOzAStages) {
      stage = 0;
      phase ^= 1u;
    }
    return oz_mma_digits<S + 1>(tmem, a_desc0, bd0, idesc, kb, kblocks, stage, phase, a_full, a_empty, acc_full,
                                acc_empty);
  }
  return true;
}

// Drain of weight W at the end of its window: 32 columns of this warp's lane
// quarter into the int64 sums (weights 0-2 into hi, 3-6 into lo, shifted by
// their place). False if the wait runs out or another role failed.
template <int W>
__device__ __forceinline__ bool oz_drain_weight(uint32_t taddr, int kb, uint64_t* acc_full, uint64_t* acc_empty,
                                                const int* fail, int lane, long long (&hi)[32],
                                                long long (&lo)[32]) {
  bool got = mbar_wait(&acc_full[W], oz_window<W>(kb) & 1);
  got = __all_sync(0xffffffffu, got && !*((volatile const int*)fail)) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!got) return false;
  uint32_t v[32];
  tmem_ld32(taddr + (uint32_t)(W * kOzBN), v);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncwarp();
  if (lane == 0) mbar_arrive(&acc_empty[W]);
  constexpr int sh = 8 * ((W <= 2 ? 2 : 6) - W);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const long long x = (long long)__float2int_rn(__uint_as_float(v[i])) << sh;
    if constexpr (W <= 2)
      hi[i] += x;
    else
      lo[i] += x;
  }
  return true;
}

template <int W>
__device__ __forceinline__ bool oz_drain_kblock(uint32_t taddr, int kb, int kblocks, uint64_t* acc_full,
                                                uint64_t* acc_empty, const int* fail, int lane, long long (&hi)[32],
                                                long long (&lo)[32]) {
  if constexpr (W < kOzS) {
    if (oz_window_end<W>(kb, kblocks) && !oz_drain_weight<W>(taddr, kb, acc_full, acc_empty, fail, lane, hi, lo))
      return false;
    return oz_drain_kblock<W + 1>(taddr, kb, kblocks, acc_full, acc_empty, fail, lane, hi, lo);
  }
  return true;
}

__device__ __forceinline__ void oz_square_tile(const CUtensorMap* mapA, const CUtensorMap* mapB, const OzArgs& a,
                                               int bid) {
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  unsigned char* bset = base;                 // 2 x kOzBSet
  unsigned char* aring = base + 2 * kOzBSet;  // kOzAStages x kOzA
  __shared__ uint64_t a_full[kOzAStages], a_empty[kOzAStages], b_full[2], b_empty[2];
  __shared__ uint64_t acc_full[kOzS], acc_empty[kOzS], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = a.d, d2 = 2 * d;
  // squaring: out (2d x d) = E B^T; gate level: out (M x 2d) = A E(P)^T
  const int mrows = a.M ? (int)a.M : d2, ncols = a.M ? d2 : d;
  const int m_tiles = mrows / kBM, n_tiles = ncols / kOzBN;
  int m_tile, n_tile;
  {
    const int per_group = kGroupM * n_tiles;
    const int g = bid / per_group;
    const int first = g * kGroupM;
    const int gm = (m_tiles - first) < kGroupM ? (m_tiles - first) : kGroupM;
    const int local = bid - g * per_group;
    m_tile = first + local % gm;
    n_tile = local / gm;
  }
  const int m0 = m_tile * kBM, n0 = n_tile * kOzBN;
  const int kblocks = d2 / 64;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzAStages; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&b_full[b], 1);
      mbar_init(&b_empty[b], 1);
    }
    for (int w = 0; w < kOzS; ++w) {
      mbar_init(&acc_full[w], 1);
      mbar_init(&acc_empty[w], 8);
    }
    mbar_init(&mma_done, 1);
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  int a_issued = 0, b_issued = 0;  // producer: loads issued (to wait for them after a failure)
  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int kb = 0; kb < kblocks; ++kb) {
        const int bb = kb & 1;
        if (kb >= 2 && !mbar_wait(&b_empty[bb], ((kb >> 1) - 1) & 1)) {
          atomicExch(&fail, 1);
          break;
        }
        if (*((volatile int*)&fail)) break;
        mbar_expect_tx(&b_full[bb], kOzBSet);
        for (int t = 0; t < kOzS; ++t)
          tma_load_2d(bset + bb * kOzBSet + t * kOzB, mapB, &b_full[bb], kb * 64, t * ncols + n0);
        ++b_issued;
        bool go = true;
        for (int s = 0; s < kOzS; ++s, ++it) {
          const int st = it % kOzAStages;
          if (it >= kOzAStages && !mbar_wait(&a_empty[st], ((it / kOzAStages) - 1) & 1)) {
            atomicExch(&fail, 1);
            go = false;
            break;
          }
          if (*((volatile int*)&fail)) {
            go = false;
            break;
          }
          mbar_expect_tx(&a_full[st], kOzA);
          tma_load_2d(aring + st * kOzA, mapA, &a_full[st], kb * 64, s * mrows + m0);
          ++a_issued;
        }
        if (!go) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc<kTcBF16, kOzBN>();
      const uint64_t a_desc0 = sw128_desc(smem_u32(aring)), b_desc0 = sw128_desc(smem_u32(bset));
      int stage = 0;
      uint32_t phase = 0;
      for (int kb = 0; kb < kblocks; ++kb) {
        const int bb = kb & 1;
        if (!mbar_wait(&b_full[bb], (kb >> 1) & 1)) {
          atomicExch(&fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t bd0 = b_desc0 + (uint64_t)(bb * (kOzBSet >> 4));
        if (!oz_mma_digits<0>(tmem, a_desc0, bd0, idesc, kb, kblocks, stage, phase, a_full, a_empty, acc_full,
                              acc_empty)) {
          atomicExch(&fail, 1);
          break;
        }
        umma_commit(&b_empty[bb]);
      }
      // every MMA issued has finished before tensor memory is released
      umma_commit(&mma_done);
      if (!mbar_wait(&mma_done, 0)) atomicExch(&fail, 1);
    }
  } else {
    const int q = warp & 3;          // tensor-memory lane quarter
    const int h = (warp - 2) >> 2;   // column half
    const int row = q * 32 + lane;   // tile row of this thread
    long long hi[32], lo[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) hi[i] = lo[i] = 0;
    bool ok = true;
    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 32);
    for (int kb = 0; kb < kblocks && ok; ++kb)
      ok = oz_drain_kblock<0>(taddr, kb, kblocks, acc_full, acc_empty, &fail, lane, hi, lo);
    if (ok && a.M) {
      // gate level: product row r -> state row row_out + r; this thread's 32
      // columns are all real (n < d) or all imaginary parts
      const int64_t r = m0 + row;
      const int t = a.tau[r];
      const int c0 = n0 + h * 32, im = c0 >= d ? 1 : 0, j0 = c0 - im * d;
      double* vr = reinterpret_cast<double*>(a.S + (a.row_out + r) * d + j0) + im;
#pragma unroll
      for (int n = 0; n < 32; ++n) {
        const double val = fma((double)lo[n], 0x1p-64, (double)hi[n] * 0x1p-32);
        const int e = t + a.sig[j0 + n] + 2;
        vr[2 * n] = val == 0.0 ? 0.0 : val * pow2d(e < -1022 ? -1022 : e);
      }
    } else if (ok) {
      const int gm = m0 + row;  // row of E: real part of P row gm, or imaginary part of row gm - d
      const int i = gm < d ? gm : gm - d;
      const int t = a.tau[i];
      double* vr = reinterpret_cast<double*>(a.C + (int64_t)i * d + n0 + h * 32) + (gm < d ? 0 : 1);
#pragma unroll
      for (int n = 0; n < 32; ++n) {
        const int col = n0 + h * 32 + n;
        const double val = fma((double)lo[n], 0x1p-64, (double)hi[n] * 0x1p-32);
        const int e = t + a.sig[col] + 2;
        const double c = val == 0.0 ? 0.0 : val * pow2d(e < -1022 ? -1022 : e);
        vr[2 * n] = c;
        if (a.C32) reinterpret_cast<float*>(a.C32 + (int64_t)i * d + col)[gm < d ? 0 : 1] = (float)c;
      }
    } else {
      atomicExch(&fail, 1);
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && fail) {
    // copies still in flight land before the CTA's shared memory is released
    const int na = a_issued < kOzAStages ? a_issued : kOzAStages;
    for (int j = a_issued - na; j < a_issued; ++j) mbar_wait(&a_full[j % kOzAStages], (j / kOzAStages) & 1);
    const int nb = b_issued < 2 ? b_issued : 2;
    for (int j = b_issued - nb; j < b_issued; ++j) mbar_wait(&b_full[j & 1], (j >> 1) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (fail && threadIdx.x == 0) atomicExch(a.err, (int)QPE_ERR_TIMEOUT);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

__global__ void __launch_bounds__(kOzThreads, 1) oz_square_kernel(const __grid_constant__ CUtensorMap mapA,
                                                                  const __grid_constant__ CUtensorMap mapB, OzArgs a) {
  pdl_begin();
  oz_square_tile(&mapA, &mapB, a, blockIdx.x);
  pdl_trigger();
}

// One squaring step of every listed instance (batched plans): scales, digit
// slices, then the digit-product GEMM with per-item tensor maps.
__global__ void __launch_bounds__(256) oz_scale_grouped_kernel(const OzItem* __restrict__ items, int nitems) {
  pdl_begin();
  int lo = 0, hi = nitems - 1;  // item whose scale blocks [sb0, sb0 + 2d) hold this CTA
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].sb0 <= (int64_t)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  const OzItem& it = items[lo];
  oz_scale_block(it.P, it.a.d, const_cast<int*>(it.a.tau), const_cast<int*>(it.a.sig), it.a.err,
                 (int)(blockIdx.x - it.sb0));
  pdl_trigger();
}

__global__ void __launch_bounds__(256) oz_slice_grouped_kernel(const OzItem* __restrict__ items, int nitems,
                                                               int64_t elems) {
  pdl_begin();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < elems; e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nitems - 1;  // item whose elements [e0, e0 + d^2) hold e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].e0 <= e)
        lo = mid;
      else
        hi = mid - 1;
    }
    const OzItem& it = items[lo];
    const int64_t le = e - it.e0;
    oz_slice_a_elem(it.P, it.a.d, it.a.tau, static_cast<__nv_bfloat16*>(it.A), it.A32, le);
    oz_slice_b_elem(it.P, it.a.d, it.a.sig, static_cast<__nv_bfloat16*>(it.B), le);
  }
  pdl_trigger();
}

__global__ void __launch_bounds__(kOzThreads, 1) oz_square_grouped_kernel(const OzItem* __restrict__ items, int nitems) {
  pdl_begin();
  const OzItem* it = items + find_item(items, nitems, blockIdx.x);
  if (threadIdx.x == 0) {
    tensormap_acquire(&it->mA);
    tensormap_acquire(&it->mB);
  }
  __syncthreads();
  oz_square_tile(&it->mA, &it->mB, it->a, (int)(blockIdx.x - it->tile0));
  pdl_trigger();
}


// ------------------------------------------------------------ host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D K-major operand [rows][K], box = (128 bytes of K) x box_rows, 128 B swizzle
bool make_map(CUtensorMap* m, void* base, int kind, int64_t rows, int64_t K, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esz = kind == kTcTF32 ? 4 : 2;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * esz};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r =
      fn(m,
         kind == kTcTF32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
         : kind == kTcBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
         2, base, dims,
         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int KIND, int BN>
size_t tc_smem() {
  return (size_t)tc_stages<BN>() * 2 * (kBM * 128 + BN * 128) + 1024;
}

// two sets of B digit tiles, the A ring, 1 KiB for the alignment
size_t oz_smem() { return (size_t)2 * kOzBSet + (size_t)kOzAStages * kOzA + 1024; }

}  // namespace

cudaError_t configure_tc_kernels() {
  cudaError_t e;
#define QPE_TC_ATTR(K, BN)                                                                                        \
  e = cudaFuncSetAttribute(tc_gemm_kernel<K, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<K, BN>()); \
  if (e != cudaSuccess) return e;
  QPE_TC_ATTR(kTcTF32, 64)
  QPE_TC_ATTR(kTcTF32, 128)
  QPE_TC_ATTR(kTcFP16, 64)
  QPE_TC_ATTR(kTcFP16, 128)
#undef QPE_TC_ATTR
  e = cudaFuncSetAttribute(tc_gemm_grouped_kernel<kTcTF32, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem<kTcTF32, 128>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(tc_gemm_grouped_kernel<kTcFP16, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem<kTcFP16, 128>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(oz_square_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(oz_square_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem());
}

// Workspace of the tensor-core squaring: row / column scales and the digit
// slices of E (kOzS x 2d x 2d) and of B (kOzS x d x 2d), bf16.
size_t oz_square_bytes(int nmat) {
  const size_t d = (size_t)1 << nmat;
  return 256 + 2 * d * sizeof(int) + 256 + (size_t)kOzS * (4 * d * d + 2 * d * d) * 2;
}

// P_k = P_(k-1)^2 on the tensor cores (d >= 256): scales, digit slices, GEMM.
// want_c64 also writes the complex64 copies (P_k, and P_0 when k = 1).
int launch_square_oz(const Instance& in, char* ws, int k, bool want_c64, cudaStream_t s) {
  const int d = (int)in.d;
  const int64_t dd = in.d * in.d;
  const double2* P = reinterpret_cast<const double2*>(ws + in.off_pow64) + (k - 1) * dd;
  double2* C = reinterpret_cast<double2*>(ws + in.off_pow64) + k * dd;
  float2* P32 = want_c64 ? reinterpret_cast<float2*>(ws + in.off_pow32) : nullptr;
  char* base = ws + in.off_ozsq;
  int* tau = reinterpret_cast<int*>(base);
  int* sig = tau + d;
  __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(base + ((2 * (size_t)d * sizeof(int) + 255) & ~size_t(255)));
  __nv_bfloat16* B = A + (size_t)kOzS * 4 * dd;
  int* err = reinterpret_cast<int*>(ws + in.off_err);
  cudaError_t e = launch_k(oz_scale_kernel, dim3(2 * d), dim3(256), 0, s, P, d, tau, sig, err);
  const unsigned eb = (unsigned)std::min<int64_t>((dd + 255) / 256, 152 * 16);
  if (e == cudaSuccess)
    e = launch_k(oz_slice_a_kernel, dim3(eb), dim3(256), 0, s, P, d, (const int*)tau, A,
                 (P32 && k == 1) ? P32 : (float2*)nullptr);
  if (e == cudaSuccess) e = launch_k(oz_slice_b_kernel, dim3(eb), dim3(256), 0, s, P, d, (const int*)sig, B);
  if (e != cudaSuccess) return -1;
  CUtensorMap mA, mB;
  if (!make_map(&mA, A, kTcBF16, (int64_t)kOzS * 2 * d, 2 * (int64_t)d, kBM) ||
      !make_map(&mB, B, kTcBF16, (int64_t)kOzS * d, 2 * (int64_t)d, kOzBN))
    return -1;
  OzArgs a{tau, sig, C, P32 ? P32 + k * dd : nullptr, d, err};
  const unsigned grid = (unsigned)((2 * d / kBM) * (d / kOzBN));
  e = launch_k(oz_square_kernel, dim3(grid), dim3(kOzThreads), oz_smem(), s, mA, mB, a);
  return e == cudaSuccess ? 4 : -1;
}

// Workspace of the FP64 gate levels on the tensor cores: the state rows'
// scales and digit slices of the largest level (M = rows / 2).
size_t oz_gate_bytes(int nmat, int64_t rows) {
  const size_t d = (size_t)1 << nmat, M = (size_t)(rows / 2);
  return ((M * sizeof(int) + 255) & ~size_t(255)) + (size_t)kOzS * M * 2 * d * 2 + 256;
}

// Doubling level j of the FP64 plain schedule on the tensor cores (d >= 256,
// M = 2^j >= 128): S[M + r] = P_(j + pow_off) S[r] for r < M as digit products,
// A = the digits of state rows 0 .. M-1, B = the digits of E(P). Returns the
// launches or -1.
int launch_oz_gate_level(const Instance& in, char* ws, int j, int pow_off, cudaStream_t s) {
  const int d = (int)in.d;
  const int64_t dd = in.d * in.d, M = int64_t(1) << j;
  const double2* P = reinterpret_cast<const double2*>(ws + in.off_pow64) + (j + pow_off) * dd;
  double2* S = reinterpret_cast<double2*>(ws + in.off_state);
  int* err = reinterpret_cast<int*>(ws + in.off_err);
  // B: E(P)'s rows at the scales of P's rows (the squaring's first-operand slices)
  char* base = ws + in.off_ozsq;
  int* tauP = reinterpret_cast<int*>(base);
  int* sigP = tauP + d;
  __nv_bfloat16* B = reinterpret_cast<__nv_bfloat16*>(base + ((2 * (size_t)d * sizeof(int) + 255) & ~size_t(255)));
  // A: the state rows
  char* gbase = ws + in.off_ozgate;
  const int64_t Mmax = (in.N >> in.shard_log) / 2;
  int* tauA = reinterpret_cast<int*>(gbase);
  __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(gbase + ((Mmax * sizeof(int) + 255) & ~size_t(255)));
  cudaError_t e = launch_k(oz_scale_kernel, dim3(2 * d), dim3(256), 0, s, P, d, tauP, sigP, err);
  const unsigned eb = (unsigned)std::min<int64_t>((dd + 255) / 256, 152 * 16);
  if (e == cudaSuccess)
    e = launch_k(oz_slice_a_kernel, dim3(eb), dim3(256), 0, s, P, d, (const int*)tauP, B, (float2*)nullptr);
  if (e == cudaSuccess)
    e = launch_k(oz_slice_rows_kernel, dim3((unsigned)std::min<int64_t>(M, 152 * 8)), dim3(256), 0, s,
                 (const double2*)S, M, d, tauA, A, err);
  if (e != cudaSuccess) return -1;
  CUtensorMap mA, mB;
  if (!make_map(&mA, A, kTcBF16, (int64_t)kOzS * M, 2 * (int64_t)d, kBM) ||
      !make_map(&mB, B, kTcBF16, (int64_t)kOzS * 2 * d, 2 * (int64_t)d, kOzBN))
    return -1;
  OzArgs a{};
  a.tau = tauA;
  a.sig = tauP;
  a.d = d;
  a.err = err;
  a.M = M;
  a.S = S;
  a.row_out = M;
  const unsigned grid = (unsigned)((M / kBM) * (2 * d / kOzBN));
  e = launch_k(oz_square_kernel, dim3(grid), dim3(kOzThreads), oz_smem(), s, mA, mB, a);
  return e == cudaSuccess ? 4 : -1;
}

size_t oz_gate_round_bytes(const Instance& in, int j) {
  const size_t M = (size_t)1 << j, d = (size_t)in.d;
  return ((M * sizeof(int) + 255) & ~size_t(255)) + (((size_t)kOzS * M * 2 * d * 2 + 255) & ~size_t(255));
}

int64_t oz_gate_tiles(const Instance& in, int j) { return ((int64_t(1) << j) / kBM) * (2 * in.d / kOzBN); }

bool oz_gate_items(const Instance& in, char* ws, int j, char* rowbuf, OzItem* pit, RowSliceItem* rit, OzItem* git) {
  // P_j's digits in the squaring's layout (the item of squaring step j + 1 reads P_j)
  if (!oz_square_item(in, ws, j + 1, false, pit)) return false;
  const int d = (int)in.d;
  const int64_t M = int64_t(1) << j;
  int* tauA = reinterpret_cast<int*>(rowbuf);
  __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(rowbuf + ((M * sizeof(int) + 255) & ~size_t(255)));
  double2* S = ws ? reinterpret_cast<double2*>(ws + in.off_state) : nullptr;
  int* err = ws ? reinterpret_cast<int*>(ws + in.off_err) : nullptr;
  *rit = RowSliceItem{S, M, d, tauA, A, err, 0};
  *git = OzItem{};
  git->a.tau = tauA;
  git->a.sig = pit->a.tau;  // E(P)'s row n scaled like row n mod d of P
  git->a.d = d;
  git->a.err = err;
  git->a.M = M;
  git->a.S = S;
  git->a.row_out = M;
  if (!ws) return true;
  return make_map(&git->mA, A, kTcBF16, (int64_t)kOzS * M, 2 * (int64_t)d, kBM) &&
         make_map(&git->mB, pit->A, kTcBF16, (int64_t)kOzS * 2 * d, 2 * (int64_t)d, kOzBN);
}

// One batched FP64 gate level: P_j's scales and digits per instance, the
// state rows' digits, the digit-product GEMM; four grouped launches.
int launch_oz_gate_grouped(const OzItem* pits, const RowSliceItem* rits, const OzItem* gits, const GateRound& R,
                           cudaStream_t s) {
  if (R.g_n <= 0) return 0;
  const unsigned eb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((R.elems + 255) / 256, 152 * 16));
  cudaError_t e = launch_k(oz_scale_grouped_kernel, dim3((unsigned)R.sblocks), dim3(256), 0, s, pits, R.p_n);
  if (e == cudaSuccess) e = launch_k(oz_slice_grouped_kernel, dim3(eb), dim3(256), 0, s, pits, R.p_n, R.elems);
  if (e == cudaSuccess)
    e = launch_k(oz_slice_rows_grouped_kernel, dim3((unsigned)std::min<int64_t>(R.rows, 152 * 16)), dim3(256), 0, s,
                 rits, R.r_n, R.rows);
  if (e == cudaSuccess)
    e = launch_k(oz_square_grouped_kernel, dim3((unsigned)R.tiles), dim3(kOzThreads), oz_smem(), s, gits, R.g_n);
  return e == cudaSuccess ? 4 : -1;
}

// Split buffers (bytes) a plan of this precision needs for the largest level.
size_t tc_split_bytes(int prec, int nmat, int nmeas) {
  if (prec != QPE_C64_TF32X3 && prec != QPE_C64_FP16X2) return 0;
  const size_t esz = prec == QPE_C64_TF32X3 ? 4 : 2;
  const size_t d2 = (size_t)2 << nmat;
  const size_t rows = nmeas >= 1 ? ((size_t)1 << (nmeas - 1)) : 1;
  const size_t scales = prec == QPE_C64_FP16X2 ? rows * sizeof(float) : 0;  // per-row inverse scales
  return 2 * rows * d2 * esz + 2 * d2 * d2 * esz + scales;
}

// One doubling level j on the tensor cores: rows [half, 2 half) = rows
// [0, half) x P_j^T. Returns launches, or -1 (launch error / tensor map).
int launch_tc_level(const Instance& in, char* ws, int prec, int j, cudaStream_t s, int pow_off) {
  const int kind = prec == QPE_C64_TF32X3 ? kTcTF32 : kTcFP16;
  const size_t esz = kind == kTcTF32 ? 4 : 2;
  const int64_t half = int64_t(1) << j;
  const int64_t d2 = 2 * in.d;
  char* Ahi = ws + in.off_tcsplit;
  char* Alo = Ahi + (size_t)(int64_t(1) << (in.nmeas - 1)) * d2 * esz;
  char* Bhi = Alo + (size_t)(int64_t(1) << (in.nmeas - 1)) * d2 * esz;
  char* Blo = Bhi + (size_t)d2 * d2 * esz;
  float* inv_scale = reinterpret_cast<float*>(Blo + (size_t)d2 * d2 * esz);  // FP16x2 only
  float* S = reinterpret_cast<float*>(ws + in.off_state);
  const double2* Pj = reinterpret_cast<const double2*>(ws + in.off_pow64) + (int64_t)(j + pow_off) * in.d * in.d;
  int launches = 0;
  cudaError_t e;
  const int64_t cnt = half * d2;
  const int gblocks = (int)std::min<int64_t>((cnt + 255) / 256, 152 * 16);
  if (kind == kTcFP16) {
    const int rblocks = (int)std::min<int64_t>((half + 7) / 8, 152 * 16);  // 8 warps (rows) per block
    e = launch_k(split_rows_fp16_kernel, dim3(rblocks), dim3(256), 0, s, (const float*)S,
                 reinterpret_cast<__half*>(Ahi), reinterpret_cast<__half*>(Alo), inv_scale, half, (int)d2);
  } else {
    e = launch_k(split_rows_tf32_kernel, dim3(gblocks), dim3(256), 0, s, (const float*)S, reinterpret_cast<float*>(Ahi),
                 reinterpret_cast<float*>(Alo), cnt);
  }
  if (e != cudaSuccess) return -1;
  ++launches;
  const int eblocks = (int)std::min<int64_t>((d2 * d2 + 255) / 256, 152 * 16);
  e = kind == kTcTF32 ? launch_k(embed_split_kernel<kTcTF32>, dim3(eblocks), dim3(256), 0, s, Pj, (void*)Bhi,
                                 (void*)Blo, (int)in.d)
                      : launch_k(embed_split_kernel<kTcFP16>, dim3(eblocks), dim3(256), 0, s, Pj, (void*)Bhi,
                                 (void*)Blo, (int)in.d);
  if (e != cudaSuccess) return -1;
  ++launches;
  const int BN = d2 >= 128 ? 128 : (int)d2;
  CUtensorMap mAh, mAl, mBh, mBl;
  if (!make_map(&mAh, Ahi, kind, half, d2, kBM) || !make_map(&mAl, Alo, kind, half, d2, kBM) ||
      !make_map(&mBh, Bhi, kind, d2, d2, BN) || !make_map(&mBl, Blo, kind, d2, d2, BN))
    return -1;
  float* Dout = S + half * d2;
  int* err = reinterpret_cast<int*>(ws + in.off_err);
  const dim3 grid((unsigned)(((half + kBM - 1) / kBM) * (d2 / BN)));  // grouped raster inside the kernel
#define QPE_TC_LAUNCH(K, B)                                                                                    \
  e = launch_k(tc_gemm_kernel<K, B>, grid, dim3(64 + 32 * kTcDrainWarps), tc_smem<K, B>(), s, mAh, mAl, mBh, mBl, \
               Dout, (int64_t)d2, \
               half, (int)d2, err, (const float*)inv_scale)
  if (kind == kTcTF32) {
    if (BN == 128)
      QPE_TC_LAUNCH(kTcTF32, 128);
    else
      QPE_TC_LAUNCH(kTcTF32, 64);
  } else {
    if (BN == 128)
      QPE_TC_LAUNCH(kTcFP16, 128);
    else
      QPE_TC_LAUNCH(kTcFP16, 64);
  }
#undef QPE_TC_LAUNCH
  if (e != cudaSuccess) return -1;
  return launches + 1;
}

// ------------------------------------------------ grouped tensor-core level
// Fills the operand buffers, tensor maps and numbering of instance `in`'s
// level j for a grouped launch (tensor maps only when ws is a bound workspace).
bool tc_level_items(const Instance& in, char* ws, int prec, int j, TcSplitItem* sp, TcGemmItem* gm) {
  const int kind = prec == QPE_C64_TF32X3 ? kTcTF32 : kTcFP16;
  const size_t esz = kind == kTcTF32 ? 4 : 2;
  const int64_t half = int64_t(1) << j;
  const int64_t d2 = 2 * in.d;
  char* Ahi = ws + in.off_tcsplit;
  char* Alo = Ahi + (size_t)(int64_t(1) << (in.nmeas - 1)) * d2 * esz;
  char* Bhi = Alo + (size_t)(int64_t(1) << (in.nmeas - 1)) * d2 * esz;
  char* Blo = Bhi + (size_t)d2 * d2 * esz;
  float* inv_scale = reinterpret_cast<float*>(Blo + (size_t)d2 * d2 * esz);
  float* S = reinterpret_cast<float*>(ws + in.off_state);
  sp->S = S;
  sp->hi = Ahi;
  sp->lo = Alo;
  sp->inv_scale = inv_scale;
  sp->P = reinterpret_cast<const double2*>(ws + in.off_pow64) + (int64_t)j * in.d * in.d;
  sp->bhi = Bhi;
  sp->blo = Blo;
  sp->rows = half;
  sp->width = (int)d2;
  sp->d = (int)in.d;
  gm->D = S + half * d2;
  gm->ldd = d2;
  gm->M = half;
  gm->K = (int)d2;
  gm->err = reinterpret_cast<int*>(ws + in.off_err);
  gm->row_scale = inv_scale;
  if (!ws) return true;
  return make_map(&gm->mAh, Ahi, kind, half, d2, kBM) && make_map(&gm->mAl, Alo, kind, half, d2, kBM) &&
         make_map(&gm->mBh, Bhi, kind, d2, d2, 128) && make_map(&gm->mBl, Blo, kind, d2, d2, 128);
}

int64_t tc_level_tiles(const Instance& in, int j) {
  const int64_t half = int64_t(1) << j;
  return ((half + kBM - 1) / kBM) * (2 * in.d / 128);
}

// split + embed of every item, then the GEMM of every item (BN = 128: every
// grouped instance has 2d >= 128)
int launch_tc_level_grouped(int prec, const TcSplitItem* sp, const TcGemmItem* gm, int nitems, int64_t rows,
                            int64_t elems, int64_t tiles, cudaStream_t s) {
  if (nitems <= 0) return 0;
  const int kind = prec == QPE_C64_TF32X3 ? kTcTF32 : kTcFP16;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((elems + 255) / 256, 152 * 16));
  cudaError_t e = kind == kTcTF32 ? launch_k(split_grouped_kernel<kTcTF32>, dim3(blocks), dim3(256), 0, s, sp, nitems,
                                             rows, elems)
                                  : launch_k(split_grouped_kernel<kTcFP16>, dim3(blocks), dim3(256), 0, s, sp, nitems,
                                             rows, elems);
  if (e != cudaSuccess) return -1;
  e = kind == kTcTF32 ? launch_k(tc_gemm_grouped_kernel<kTcTF32, 128>, dim3((unsigned)tiles),
                                 dim3(64 + 32 * kTcDrainWarps), tc_smem<kTcTF32, 128>(), s, gm, nitems)
                      : launch_k(tc_gemm_grouped_kernel<kTcFP16, 128>, dim3((unsigned)tiles),
                                 dim3(64 + 32 * kTcDrainWarps), tc_smem<kTcFP16, 128>(), s, gm, nitems);
  return e == cudaSuccess ? 2 : -1;
}

// One instance's squaring step k for a grouped launch (tensor maps only when
// ws is a bound workspace); its scale blocks, slice elements and GEMM CTAs.
bool oz_square_item(const Instance& in, char* ws, int k, bool want_c64, OzItem* it) {
  const int d = (int)in.d;
  const int64_t dd = in.d * in.d;
  it->P = reinterpret_cast<const double2*>(ws + in.off_pow64) + (k - 1) * dd;
  float2* P32 = want_c64 ? reinterpret_cast<float2*>(ws + in.off_pow32) : nullptr;
  char* base = ws + in.off_ozsq;
  int* tau = reinterpret_cast<int*>(base);
  __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(base + ((2 * (size_t)d * sizeof(int) + 255) & ~size_t(255)));
  __nv_bfloat16* B = A + (size_t)kOzS * 4 * dd;
  it->A = A;
  it->B = B;
  it->A32 = (P32 && k == 1) ? P32 : nullptr;
  it->a = OzArgs{tau, tau + d, reinterpret_cast<double2*>(ws + in.off_pow64) + k * dd, P32 ? P32 + k * dd : nullptr, d,
                 reinterpret_cast<int*>(ws + in.off_err)};
  if (!ws) return true;
  return make_map(&it->mA, A, kTcBF16, (int64_t)kOzS * 2 * d, 2 * (int64_t)d, kBM) &&
         make_map(&it->mB, B, kTcBF16, (int64_t)kOzS * d, 2 * (int64_t)d, kOzBN);
}

int64_t oz_square_tiles(const Instance& in) { return (2 * in.d / kBM) * (in.d / kOzBN); }

int launch_square_oz_grouped(const OzItem* items, int nitems, int64_t sblocks, int64_t elems, int64_t tiles,
                             cudaStream_t s) {
  if (nitems <= 0) return 0;
  const unsigned eb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((elems + 255) / 256, 152 * 16));
  cudaError_t e = launch_k(oz_scale_grouped_kernel, dim3((unsigned)sblocks), dim3(256), 0, s, items, nitems);
  if (e == cudaSuccess) e = launch_k(oz_slice_grouped_kernel, dim3(eb), dim3(256), 0, s, items, nitems, elems);
  if (e == cudaSuccess)
    e = launch_k(oz_square_grouped_kernel, dim3((unsigned)tiles), dim3(kOzThreads), oz_smem(), s, items, nitems);
  return e == cudaSuccess ? 3 : -1;
}

// ------------------------------------------- expiry of a bounded wait
// The exit path every tensor-core kernel takes when one of its mbarrier waits
// runs out, exercised on purpose: warp 0 holds tensor memory, warp 1 waits
// with a poll limit of `polls` on a barrier that nothing arrives at (no TMA
// copy and no MMA is in flight), the CTA records QPE_ERR_TIMEOUT in the error
// word, warp 0 frees the tensor memory and the kernel returns.
__global__ void __launch_bounds__(64, 1) wait_expiry_kernel(int* __restrict__ err, uint32_t polls) {
  pdl_begin();
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(32u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (warp == 1 && lane == 0 && !mbar_wait(&bar, 0, polls)) atomicExch(&fail, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (fail && threadIdx.x == 0) atomicExch(err, (int)QPE_ERR_TIMEOUT);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u) : "memory");
  pdl_trigger();
}

int launch_wait_expiry(const Instance& in, char* ws, uint32_t polls, cudaStream_t s) {
  return launch_k(wait_expiry_kernel, dim3(1), dim3(64), 0, s, reinterpret_cast<int*>(ws + in.off_err), polls) ==
                 cudaSuccess
             ? 1
             : -1;
}

}  // namespace qpe
