// Internal declarations of the QPE emulator: complex helpers, workspace
// layout, and the kernel launchers the C ABI calls. Not part of the ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qpe.h"

namespace qpe {

// Global -> shared copies that do not stall the issuing thread: every thread
// issues all of its copies, then waits once (cp.async groups).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// one complex element; valid == false stores zeros (no bytes are read)
__device__ __forceinline__ void cp_async_elem(float2* smem, const float2* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2* smem, const double2* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
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

// ------------------------------------------------ programmatic dependent launch
// Every kernel of a run starts with pdl_wait(), which returns once the
// previous grid in the stream has completed and its writes are visible, and
// ends by letting its successor be scheduled (pdl_trigger(), or implicitly at
// exit). With programmatic launches enabled (the default; QPE_PDL=0 in the
// environment at qpe_bind turns them off), a dependent kernel's launch
// overlaps the tail of its predecessor; otherwise launch_k() is an ordinary
// launch and both instructions are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_begin() { pdl_wait(); }

extern bool g_pdl_enabled;

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = g_pdl_enabled ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------- complex
template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C>
__host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C>
__host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C>
__host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
template <typename C>
__host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
template <typename C, typename R>
__host__ __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }

__device__ __forceinline__ float2 to_c(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_c(double2 v, double2*) { return v; }

// ------------------------------------------------------------ fft plan
constexpr int kMaxPasses = 8;

struct FftPass {
  int logr;      // this pass's DFT length R = 2^logr
  int64_t B;     // independent blocks (N / (R * L))
  int64_t L;     // row stride between the R elements of one DFT
  int64_t Q;     // L * d: contiguous elements per (block, digit)
  int64_t W;     // elements of Q each CTA takes
};

struct FftPlan {
  int passes = 0;
  FftPass p[kMaxPasses];
  int logr_list[kMaxPasses];  // digit widths from the top of m downwards
};

// Arguments of one QFT^-1 pass (fft_pass_kernel): a length-2^logr DFT over
// the middle axis of the state viewed as [B][R][Q].
struct FftArgs {
  int logr;
  int logw;    // W = 2^logw columns per CTA
  int logq;    // Q = 2^logq
  int logd;
  int n;       // log2 of the transform length
  int htw;
  int logb;    // B = 2^logb blocks
  int last;    // 1: no inter-pass twiddle
  int tw_sh;   // log2(N / transform length): a shard's local transform reads the N-point tables
  double scale;
};

// Digit widths of the passes, top of m first (position -> outcome order).
struct Digits {
  int count;
  int logr[kMaxPasses];
};

// item index i with items[i].tile0 <= b < items[i + 1].tile0 (tile0 ascending):
// the grouped kernels map a CTA to the work item it belongs to
template <typename T>
__device__ __forceinline__ int find_item(const T* items, int n, int64_t b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].tile0 <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Device-side scalars of one instance (readout + error word).
struct Scalars {
  int64_t argmax;
  double phase_argmax;
  double phase_mean;
  double total;      // sum_y P[y]
  double best;       // P[argmax]
  int32_t err;       // qpe_status raised on the device, 0 if none
  int32_t pad;
};

// Per-block partial of the readout reduction.
struct Partial {
  double best;
  int64_t besty;
  double wsum;   // sum P[y] * y
  double psum;   // sum P[y]
};

constexpr int kReduceBlocks = 1216;  // 152 SMs x 8
constexpr int kHostChunks = 8;       // parts of a top level whose histogram is copied out while the next computes

// The readout's merge rule, used by every kernel that combines partials: the
// larger probability wins, an exact tie goes to the lower y, and a NaN best is
// replaced by whatever comes next (so a non-finite histogram cannot freeze it).
__device__ __forceinline__ void better(double& best, int64_t& by, double v, int64_t y) {
  if (v > best || (v == best && y < by) || (best != best)) {
    best = v;
    by = y;
  }
}
__device__ __forceinline__ void merge_partial(Partial& m, const Partial& o) {
  better(m.best, m.besty, o.best, o.besty);
  m.wsum += o.wsum;
  m.psum += o.psum;
}
// parts[0 .. count) merged by one CTA of 256 threads in a fixed order (the
// result is deterministic); every thread must call it; thread 0 gets the result.
__device__ __forceinline__ Partial reduce_partials_256(const Partial* __restrict__ parts, int count) {
  __shared__ Partial sp[256];
  Partial r{-1.0, INT64_MAX, 0.0, 0.0};
  for (int i = threadIdx.x; i < count; i += 256) merge_partial(r, parts[i]);
  sp[threadIdx.x] = r;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) merge_partial(sp[threadIdx.x], sp[threadIdx.x + s]);
    __syncthreads();
  }
  return sp[0];
}
// A readout whose sums are not finite (or that saw no bin at all) has no
// defined argmax.
__device__ __forceinline__ bool readout_finite(const Partial& m) {
  return isfinite(m.psum) && isfinite(m.wsum) && isfinite(m.best) && m.besty != INT64_MAX;
}

// One level of the fused small-d schedule: the controlled gates of
// measurement qubits off .. off + r - 1 and a length-2^r DFT, for N_a = 2^logna
// seeds.
struct Level {
  int off, r, logna;
  size_t tab_off;  // workspace offset of this level's table U_l^(m_b), m_b < 2^r
};

constexpr int kMaxLevels = 32;
// state_stage of a sharded plain plan between qpe_run and qpe_shard_finish
constexpr int kStageExchange = 5;
struct TableJobs {
  int count;
  int off[kMaxLevels];
  int r[kMaxLevels];
  size_t tab_off[kMaxLevels];
};

constexpr size_t kLevelSmemCap = 110 * 1024;  // two CTAs per SM

// A share of a grouped level launch: LevelArgs index, column group, a range
// of pencil-group iterations, and the slot of its readout partial.
struct GroupItem {
  int arg;
  int cg;
  int64_t it_begin, it_end;
  int64_t part;
};

// Sharded levels (a plan for rank rk of 2^sh ranks): the level computes only
// the y_a = rk + 2^sh j, j < N_a / 2^sh, and keeps its outputs compact: the
// value of outcome y (y = rk mod 2^sh) sits at local index y >> sh. Seeds are
// read at seed_rk + (j << seed_sh): (0, 0) when the level below is sharded
// too (compact), (rk, sh) when it was computed whole. Unsharded levels have
// sh = rk = seed_sh = seed_rk = 0.
template <typename C>
struct LevelArgs {
  const C* seeds;  // N_a x d: Z of the level below (psi for the deepest level)
  const C* tab;    // [k][m_b d + i] = (U_l^(m_b))[i][k]
  int off, r, logna, logd, nmeas, htw;
  int sh, rk, seed_sh, seed_rk;
  const C* tw_lo;
  const C* tw_hi;
  C* xout;         // MODE 0: X of this level; MODE 2: physical final state
  double* hist;    // MODE 1/2
  Partial* parts;  // MODE 1/2
  double pscale;   // 1 / N^2
  double inv_n;    // 1 / N
  double xscale;
};

// One problem instance inside a plan: its shape and workspace offsets.
struct Instance {
  int nmat, nmeas;
  int64_t d, N;
  int htw;              // split point of the two-level twiddle table
  size_t off_pow64;     // nmeas x d x d complex128
  size_t off_pow32;     // nmeas x d x d complex64 (complex64 plans)
  size_t off_psi;       // d complex128
  size_t off_state;     // N x d elements
  size_t off_hist;      // N doubles
  size_t off_tw_lo64, off_tw_hi64, off_tw_lo32, off_tw_hi32;
  size_t off_partials;  // kReduceBlocks Partials
  size_t off_scalars;   // Scalars
  size_t off_err = 0;   // int32 device error word (bounded waits)
  size_t off_tcsplit = 0;  // split operands of the tensor-core levels
  size_t off_ozsq = 0;     // scales + digit slices of the tensor-core squaring
  bool oz_gates = false;   // FP64 plain doubling levels on the tensor cores (QPE_FLAG_LEVEL_TC, d >= 256)
  size_t off_ozgate = 0;   // their state-row scales and digit slices
  bool oz_square = false;  // U^(2^k) squared on the tensor cores (QPE_FLAG_SQUARE_TC, d >= 256)
  size_t state_bytes;
  bool has_state = true;  // the workspace holds an N x d state buffer
  FftPlan fft;
  // fused small-d schedule
  bool fused = false;
  std::vector<Level> levels;  // top level first
  size_t off_zbuf[2] = {0, 0};
  size_t zbuf_seed_off = 0;
  int64_t level_grid = 0;     // persistent grid (set at bind)
  // sharded plans: this rank (shard_rank of 2^shard_log) owns the outcomes
  // y = shard_rank mod 2^shard_log; its histogram (and kept state) hold them
  // compactly, y at local index y >> shard_log
  int shard_log = 0, shard_rank = 0;
  bool shard_plain = false;           // sharded plain schedule: one exchange per run
  size_t off_send = 0, off_recv = 0;  // its all-to-all buffers, [2^shard_log][N / 4^shard_log][d] each
  // top level of the fused schedule on the tensor cores (FP16x2 / TF32x3, or
  // FP64 with QPE_FLAG_LEVEL_TC; d = 16)
  bool tc_top = false;
  int tc_top_prec = 0;
  bool oz_levels = false;  // FP64: every 8-point level with a 128-pencil tile per rank on the tensor cores
  size_t off_tctab = 0;    // the table operands (fp16 / tf32 splits, or the FP64 table's digit slabs)
  // qpe_set_host_histogram: every run also copies the histogram into this
  // page-locked host buffer (overlapped with the FP64 tensor-core top level,
  // which then runs in kHostChunks parts); its copy stream and fork / join events
  double* host_hist = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev[9] = {};
  int nsm = 0;           // multiprocessors of the bound device
  bool keep_state = false;
  bool loaded = false;
  bool powers_done = false;
  int state_stage = 0;  // last stage whose output the state buffer holds
  bool state_natural = false;  // state buffer rows are in natural order of y
  bool state_valid = true;     // false after a fused run without KEEP_STATE
};

// ---------------------------------------------------------- batched plans
struct SqItem {  // one instance's squaring step: C = A^2 (FP64), complex64 copies
  const double2* A;
  double2* C;
  float2* C32;
  float2* A32;
  int d, pad;
  int64_t tile0;  // first CTA of this item in the grouped launch (8 x 8 tiles)
  int64_t tile16, tile32;  // the same with 16 x 16 and 32 x 32 tiles
};
template <typename C>
struct TabItem {  // one (instance, level) table
  const C* P;
  C* tab;
  int off, r, logd, pad;
  int64_t tile0;
};
template <typename C>
struct SeedItem {
  const double2* psi;
  C* seed;
  int d, pad;
};
struct FinItem {
  const Partial* parts;
  Scalars* out;
  int count, nmeas;
};

// Work items of the batched plain schedule (instances run together, one
// launch per step): row 0 of each state, one doubling level, one QFT^-1 pass,
// the histogram.
template <typename C>
struct InitItem {
  C* S;
  const double2* psi;
  double scale;
  int d, pad;
};
template <typename C>
struct DblItem {  // rows [M, 2M) = rows [0, M) x P^T
  C* S;
  const C* P;
  int64_t M;
  int d, pad;
  int64_t tile0;
};
template <typename C>
struct FftItem {
  C* X;
  const C* lo;
  const C* hi;
  FftArgs a;
  int64_t tile0;
};
template <typename C>
struct RedItem {
  const C* X;
  double* hist;
  Partial* parts;
  int64_t N;
  int logd, n;
  Digits g;
  int64_t tile0, nblk;
};

struct LevelLaunch {  // one grouped level launch
  int logd, mode;
  int arg_off, item_off, nitems;
  int64_t grid;
};

// One instance's doubling level on the tensor cores in a grouped launch: its
// operand tensor maps (A hi / lo rows, B hi / lo embedding; 64-byte aligned in
// global memory), output and error word.
struct TcGemmItem {
  CUtensorMap mAh, mAl, mBh, mBl;
  float* D;
  int64_t ldd, M;
  int K, pad;
  int* err;
  const float* row_scale;
  int64_t tile0;
};
// One instance's operand split for the grouped tensor-core level: the rows
// [0, rows) of its state into hi / lo (warp per row), and U^(2^j)'s embedding.
struct TcSplitItem {
  const float* S;
  void* hi;
  void* lo;
  float* inv_scale;
  const double2* P;
  void* bhi;
  void* blo;
  int64_t rows, row0;  // rows of A, first row in the launch's numbering
  int64_t e0;          // first embedding element in the launch's numbering
  int width, d;
  int64_t tile0;       // = row0 (for find_item over rows)
};
struct TcRound {  // one level j across the tensor-core instances
  int j, item_off, nitems;
  int64_t rows, elems, tiles;
};

// The digit-product GEMM of the tensor-core squaring (P_(k+1) = P_k^2).
struct OzArgs {
  const int* tau;  // row scales of the first operand (rows of E; state rows for a gate level)
  const int* sig;  // scales of the second operand's rows (columns n of E; for a gate level the rows of
                   // E(P), row n scaled like row n mod d of P)
  double2* C;      // squaring: P_(k+1), complex128 d x d
  float2* C32;     // its complex64 copy, or null
  int d;
  int* err;
  // a gate level (M > 0): out = A B^T with A the digits of state rows 0 .. M-1
  // ([Re | Im], K = 2d) and B those of E(P) (N = 2d rows); row r of out is
  // row row_out + r of S (columns n < d the real parts, n >= d the imaginary)
  int64_t M = 0;
  double2* S = nullptr;
  int64_t row_out = 0;
};
// One instance's squaring step in a grouped launch: the digit slices' tensor
// maps, P_k, the slice buffers, and the item's first scale block, first slice
// element and first GEMM CTA in the launches' numbering.
struct OzItem {
  CUtensorMap mA, mB;
  OzArgs a;
  const double2* P;
  void* A;
  void* B;
  float2* A32;
  int64_t sb0, e0, tile0;
};
// The state rows 0 .. M-1 of one instance cut into digits for a batched FP64
// gate level (row scales and digit planes in the round's shared buffer);
// tile0 = its first row in the launch's numbering.
struct RowSliceItem {
  const double2* S;
  int64_t M;
  int d;
  int* tau;
  void* A;
  int* err;
  int64_t tile0;
};
struct GateRound {  // FP64 doubling level j on the tensor cores across the batched instances
  int j;
  int p_off, p_n;            // P_j's scale + slicing items (OzItem, squaring layout)
  int64_t sblocks, elems;
  int r_off, r_n;            // the state rows' slicing items
  int64_t rows;
  int g_off, g_n;            // the digit-product GEMM items (OzItem with a gate level's OzArgs)
  int64_t tiles;
};
struct OzStep {  // squaring step k across the tensor-core instances
  int k, item_off, nitems;
  int64_t sblocks, elems, tiles;
};

struct DblRound {  // one grouped doubling launch: level j of the items of one tile class
  int j, dclass, item_off, nitems;
  int64_t tiles;
};
struct FftRound {  // one grouped QFT^-1 pass launch
  int item_off, nitems;
  int64_t blocks;
  size_t smem;
};

struct BatchMeta {
  int maxn = 0;
  // plain instances (Nmat > 6, or QPE_FLAG_PLAIN), run together step by step
  std::vector<char> init_items, dbl_items, fft_items, red_items;  // typed by the plan's precision
  std::vector<DblRound> dbl_rounds;
  std::vector<OzItem> oz_items;  // tensor-core squarings, grouped per step
  std::vector<OzStep> oz_steps;
  std::vector<OzItem> gate_p, gate_g;  // FP64 gate levels on the tensor cores, grouped per level
  std::vector<RowSliceItem> gate_r;
  std::vector<GateRound> gate_rounds;
  size_t gate_buf_bytes = 0, off_gatebuf = 0, off_gate_p = 0, off_gate_g = 0, off_gate_r = 0;
  std::vector<TcSplitItem> tc_split;  // tensor-core levels (j >= 7, 2d >= 128), grouped per level
  std::vector<TcGemmItem> tc_gemm;
  std::vector<TcRound> tc_rounds;
  std::vector<FftRound> fft_rounds;
  std::vector<FinItem> fin_plain;
  int ninit = 0, nred = 0, maxn_plain = 0;
  int64_t red_blocks = 0;
  size_t off_init = 0, off_dbl = 0, off_fft = 0, off_red = 0, off_finp = 0, off_tcsp = 0, off_tcgm = 0, off_oz = 0;
  // squaring: items of step k at [sq_begin[k], sq_begin[k] + sq_count[k])
  std::vector<SqItem> sq;
  std::vector<int> sq_begin, sq_count;
  std::vector<int64_t> sq_tiles, sq_tiles16, sq_tiles32;  // CTAs per step, per tile variant
  std::vector<SqItem> conv;
  int64_t conv_tiles = 0;
  // fused instances
  std::vector<int> fused, plain;
  std::vector<char> tab_items, seed_items, level_args;  // typed by the plan's precision
  int ntab = 0, nseed = 0, max_logd = 1;
  int64_t tab_blocks = 0;
  std::vector<GroupItem> items;
  std::vector<LevelLaunch> launches;
  std::vector<FinItem> fin;
  // workspace offsets of the uploaded lists
  size_t off_sq = 0, off_conv = 0, off_tab = 0, off_seed = 0, off_args = 0, off_items = 0, off_fin = 0;
  size_t bytes = 0;
};

// variant 0: 8 x 8 output tiles, inner index split 4 ways; 1: 16 x 16 tiles and
// 2: 32 x 32 tiles, both with 16-wide k slabs staged in shared memory
int launch_square_grouped(const SqItem* items, int nitems, int64_t tiles, int variant, cudaStream_t s);
int launch_convert_grouped(const SqItem* items, int nitems, int64_t tiles, cudaStream_t s);
template <typename C>
int launch_table_grouped(const TabItem<C>* items, int nitems, int64_t blocks, int max_logd, cudaStream_t s);
template <typename C>
int launch_seed_grouped(const SeedItem<C>* items, int nitems, cudaStream_t s);
int launch_finalize_grouped(const FinItem* items, int nitems, cudaStream_t s);
template <typename C>
int launch_level_grouped(const LevelLaunch& L, const LevelArgs<C>* args, const GroupItem* items, cudaStream_t s);
template <typename C>
int level_grouped_occupancy(int logd, int mode);
cudaError_t configure_batched_kernels();
// host view of the level configuration: (columns per CTA, pencils per iteration)
void level_shape(int logd, int mode, size_t esize, int* DI, int* G);

}  // namespace qpe

struct qpe_plan_s {
  int prec;
  uint32_t flags;
  std::vector<qpe::Instance> inst;
  size_t ws_bytes = 0;
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  bool bound = false;
  int64_t last_launches = 0;
  cudaGraphExec_t graph_exec = nullptr;
  cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // QPE_FLAG_TIMING
  bool timed_kernel = false;  // ev[5], ev[6] bracket the top-level fused kernel of the last run
  int sq_variant = 0;            // batched squaring tile variant (autotuned or forced)
  float tune_ms[3] = {0, 0, 0};  // the autotuner's timing of each variant (ms)
  bool batched = false;
  qpe::BatchMeta bm;
  bool timed_run = false;  // the last enqueue recorded all five events
  std::string last_error;
};

namespace qpe {

// Launchers (qpe_kernels.cu). Each returns the number of kernels enqueued or
// -1 on a launch error (cudaGetLastError is left for the caller to read).
int launch_twiddles(const Instance& in, char* ws, cudaStream_t s);
int launch_powers(const Instance& in, char* ws, bool want_c64, cudaStream_t s);
// U^dagger U = I to 1e-8 per entry, else the instance's error word = QPE_ERR_NUMERIC
int launch_check_unitary(const Instance& in, char* ws, cudaStream_t s);
template <typename C> int launch_sweep(const Instance& in, char* ws, bool gate_mode, cudaStream_t s, int prec = 1);
// doubling level j on the tensor cores with the power P_(j + pow_off)
int launch_tc_level(const Instance& in, char* ws, int prec, int j, cudaStream_t s, int pow_off = 0);
// a bounded wait that runs out after `polls` polls (records QPE_ERR_TIMEOUT)
int launch_wait_expiry(const Instance& in, char* ws, uint32_t polls, cudaStream_t s);
// grouped tensor-core level (batched plans): one instance's items, its CTA
// count, and the two launches (operand splits, GEMM) for all items
bool tc_level_items(const Instance& in, char* ws, int prec, int j, TcSplitItem* sp, TcGemmItem* gm);
int64_t tc_level_tiles(const Instance& in, int j);
int launch_tc_level_grouped(int prec, const TcSplitItem* sp, const TcGemmItem* gm, int nitems, int64_t rows,
                            int64_t elems, int64_t tiles, cudaStream_t s);
size_t oz_square_bytes(int nmat);
// grouped tensor-core squaring (batched plans): one instance's item, its GEMM
// CTAs, and the three launches (scales, slices, GEMM) for all items of a step
bool oz_square_item(const Instance& in, char* ws, int k, bool want_c64, OzItem* it);
int64_t oz_square_tiles(const Instance& in);
int launch_square_oz_grouped(const OzItem* items, int nitems, int64_t sblocks, int64_t elems, int64_t tiles,
                             cudaStream_t s);
int launch_square_oz(const Instance& in, char* ws, int k, bool want_c64, cudaStream_t s);
size_t tc_split_bytes(int prec, int nmat, int nmeas);
cudaError_t configure_tc_kernels();
template <typename C> int launch_fft(const Instance& in, char* ws, cudaStream_t s);
template <typename C> int launch_reduce(const Instance& in, char* ws, cudaStream_t s);
// sharded plain schedule: twiddle and sort the local transform by owner rank
// into the send buffer; after the caller's all-to-all, the cross-rank DFT,
// histogram and readout partials of this rank's outcomes
template <typename C> int launch_shard_pack(const Instance& in, char* ws, cudaStream_t s);
template <typename C> int launch_shard_combine(const Instance& in, char* ws, cudaStream_t s, int* blocks);
template <typename C> int launch_unpermute(const Instance& in, const char* ws, void* out, cudaStream_t s);

template <typename C>
int launch_levels(const Instance& in, char* ws, bool keep_state, cudaStream_t s, cudaEvent_t* top_ev = nullptr);
cudaError_t record_event(cudaEvent_t ev, cudaStream_t s);
int launch_finalize(const Instance& in, char* ws, int count, cudaStream_t s);
inline void finalize_readout(const Instance& in, char* ws, int count, cudaStream_t s) {
  launch_finalize(in, ws, count, s);
}
size_t level_smem_bytes(int logd, int mode, size_t esize);
size_t tc_top_table_bytes();
// the FP64 top level on the tensor cores (d = 16, 8-point top level)
size_t oz_top_table_bytes();
cudaError_t configure_oz_top_kernel();
int launch_oz_level(const Instance& in, char* ws, const LevelArgs<double2>& la, bool top, cudaStream_t s,
                    cudaEvent_t* top_ev, int64_t* grid_out);
bool oz_top_copies_host_histogram(const Instance& in);
// FP64 plain doubling levels on the tensor cores
size_t oz_gate_bytes(int nmat, int64_t rows);
int launch_oz_gate_level(const Instance& in, char* ws, int j, int pow_off, cudaStream_t s);
// batched: bytes of one level's row digits in the round buffer; the three items
// of instance `in` at level j (rowbuf: its part of the round buffer; maps and
// pointers only when ws is a bound workspace); the round's grouped launches
size_t oz_gate_round_bytes(const Instance& in, int j);
bool oz_gate_items(const Instance& in, char* ws, int j, char* rowbuf, OzItem* pit, RowSliceItem* rit, OzItem* git);
int64_t oz_gate_tiles(const Instance& in, int j);
int launch_oz_gate_grouped(const OzItem* pits, const RowSliceItem* rits, const OzItem* gits, const GateRound& R,
                           cudaStream_t s);
int level_max_bits(int logd, size_t esize, size_t smem_cap);
std::vector<Level> make_levels(int nmeas, int logd, size_t esize, int rtop);
// a level of a sharded plan computes only this rank's outcomes when it has at
// least 2^shard_log pencils; smaller (deeper) levels are computed whole
bool level_sharded(const Instance& in, int li);
cudaError_t configure_level_kernels();
template <typename C> int level_occupancy(int logd, int r);

// The batched plain schedule's grouped launches (one per step across instances).
template <typename C> int launch_init_grouped(const InitItem<C>* items, int nitems, cudaStream_t s);
template <typename C>
int launch_doubling_grouped(const DblItem<C>* items, int nitems, int64_t tiles, int dclass, cudaStream_t s);
template <typename C>
int launch_fft_grouped(const FftItem<C>* items, int nitems, int64_t blocks, size_t smem, cudaStream_t s);
template <typename C> int launch_reduce_grouped(const RedItem<C>* items, int nitems, int64_t blocks, cudaStream_t s);
// pass i's arguments, CTA count and shared memory; the plain histogram's CTA
// count; the doubling GEMM's row / column tile for a target dimension d
FftArgs fft_pass_args(const Instance& in, int i, int64_t* blocks, size_t* smem, size_t esize);
Digits fft_digits(const FftPlan& f);
int64_t reduce_blocks(const Instance& in);
void doubling_tile(int d, int* BM, int* BN);

// Host helpers shared with the ABI layer.
int64_t fft_position_to_y(const FftPlan& f, int nmeas, int64_t p);
FftPlan make_fft_plan(int nmeas, int64_t d, size_t esize);

}  // namespace qpe
