/*
 * qpe.h - C ABI of the GB300 (sm_103a) statevector emulator for the Quantum
 * Phase Estimation circuit (QPE; Sec. 2 and Fig. 1 of "GPU benchmark through
 * QPE emulator with cuQuantum for practical quantum applications").
 *
 * The circuit: Nmeas measurement qubits start in |0>, the Nmat-qubit target
 * register holds psi. A Hadamard acts on every measurement qubit, measurement
 * qubit k (k = 0 is the top wire of Fig. 1) controls U^(2^k) on the target
 * register, QFT^-1 acts on the measurement register, and the measurement
 * register is read out; the eigenphase phi of U (eigenvalue exp(2 pi i phi),
 * Sec. 2) is estimated from the outcome distribution either by the most
 * probable outcome or by the probability-weighted average (Sec. 4.2).
 *
 * Data layout (all device memory is caller-owned):
 *   - d = 2^Nmat, N = 2^Nmeas.
 *   - U: d x d complex128, row-major, interleaved (re, im) doubles.
 *   - psi: d complex128.
 *   - The state is an N x d row-major matrix S[m][t], flat index m*d + t
 *     (measurement register = high bits); measurement qubit k is bit k of m.
 *     Element type: complex128 for QPE_FP64 plans, complex64 otherwise.
 *   - The histogram P[y], y in [0, N), is float64 in natural order of y.
 *
 * Conventions:
 *   - QFT^-1 is F^dagger[y][m] = 2^(-n/2) exp(-2 pi i m y / N) including the
 *     final swaps, so an eigenphase phi peaks at y = N phi.
 *   - psi is not renormalised: sum_y P[y] = ||psi||^2.
 *   - Every call returns a qpe_status; no C++ exception crosses the ABI. A
 *     plan is not thread-safe; distinct plans are independent.
 *   - The library never allocates device memory: qpe_plan reports the
 *     workspace size, the caller allocates it and passes it to qpe_bind.
 *     Host-side allocation happens only inside qpe_plan (the plan object) and
 *     in qpe_state's host-output path (a temporary for the reordering).
 *   - All device work is enqueued on the stream given to qpe_bind. Calls that
 *     return data to host memory synchronise that stream.
 */
#ifndef QPE_H
#define QPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qpe_plan_s* qpe_plan_t;

typedef enum {
  QPE_OK = 0,
  QPE_ERR_ARG = 1,         /* null pointer, bad enum, argument out of range      */
  QPE_ERR_SHAPE = 2,       /* nmat/nmeas/instance do not match the plan          */
  QPE_ERR_WORKSPACE = 3,   /* workspace null, too small or not 256-byte aligned  */
  QPE_ERR_UNSUPPORTED = 4, /* valid request this build does not implement        */
  QPE_ERR_CUDA = 5,        /* a CUDA runtime call failed (see qpe_last_error)    */
  QPE_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out                 */
  QPE_ERR_NUMERIC = 7,     /* NaN/Inf detected in the histogram                  */
  QPE_ERR_STATE = 8        /* call out of order (e.g. run before bind/load)      */
} qpe_status;

typedef enum {
  QPE_FP64 = 0,       /* complex128 state, FP64 arithmetic everywhere           */
  QPE_C64_FP32 = 1,   /* complex64 state, FP32 arithmetic for the controlled    */
                      /* gates and QFT^-1; U^(2^k) squaring and the readout     */
                      /* stay FP64                                              */
  QPE_C64_BF16X3 = 2, /* refused by every plan (QPE_ERR_UNSUPPORTED): bf16      */
                      /* hi/lo splits keep ~16 significand bits per operand,    */
                      /* and the histogram's L1 error then grows past 1e-6 with  */
                      /* the number of gate levels (measured up to 1.6e-6 at     */
                      /* Nmeas = 18); the value stays reserved                   */
  QPE_C64_FP16X2 = 3, /* complex64 state; controlled gates on the tcgen05       */
                      /* tensor cores with fp16 hi/lo splits (~22 bits) and FP32 */
                      /* accumulation in two passes (hi.hi, then both cross      */
                      /* products over a doubled K); rows of the state are       */
                      /* scaled by powers of two into fp16's range and U's       */
                      /* embedding by 2^14; squaring and readout stay FP64.      */
                      /* nmat >= 5: plain schedule, gate GEMMs on the tensor    */
                      /* cores; nmat = 4: fused schedule with its top level     */
                      /* (gates of the 4 low measurement qubits, 16-point DFT,  */
                      /* histogram) on the tensor cores when it has >= 128      */
                      /* pencils; otherwise (nmat <= 3, or too few pencils) the  */
                      /* fused complex64 schedule on the CUDA cores              */
  QPE_C64_TF32X3 = 4  /* as QPE_C64_FP16X2 with tf32 hi/lo splits (~21 bits),   */
                      /* no scaling, and three products A_hi B_hi + A_hi B_lo +  */
                      /* A_lo B_hi (nmat = 4: the same fused tensor-core top     */
                      /* level)                                                  */
} qpe_precision;

/* Plan flags. */
#define QPE_FLAG_GATE_SWEEP 0x1u /* schedule the controlled gates one per      */
                                 /* measurement qubit over all rows whose bit  */
                                 /* k is set (gate-faithful; d <= 64), instead */
                                 /* of the default doubling schedule           */
#define QPE_FLAG_GRAPH 0x2u      /* qpe_run captures its launches into a CUDA  */
                                 /* graph on first use and replays it         */
#define QPE_FLAG_TIMING 0x4u     /* record a CUDA event before each stage and  */
                                 /* after the last one (read: qpe_stage_times) */
#define QPE_FLAG_PLAIN 0x8u      /* materialise the N x d state after the      */
                                 /* controlled gates and run QFT^-1 and the    */
                                 /* reduction as separate passes over it; the  */
                                 /* default for nmat <= 6 is the fused         */
                                 /* schedule (see qpe_run), whose workspace    */
                                 /* has no N x d state buffer unless           */
                                 /* QPE_FLAG_KEEP_STATE is set, so stage-by-   */
                                 /* stage runs and qpe_load_state need PLAIN   */
#define QPE_FLAG_KEEP_STATE 0x10u /* fused schedule: also write the final     */
                                  /* statevector (one extra state write)      */
#define QPE_FLAG_REPEAT_U 0x20u  /* with QPE_FLAG_GATE_SWEEP: apply U itself   */
                                 /* 2^k times for measurement qubit k instead */
                                 /* of U^(2^k) once (the construction the     */
                                 /* paper's cost argument assumes, Sec. 4.1); */
                                 /* nmeas <= 14                               */
#define QPE_FLAG_AUTOTUNE 0x80u /* batched plans: qpe_bind times the grouped */
                                /* FP64 squaring with 8 x 8, 16 x 16 and 32 x  */
                                /* 32 output tiles on the plan's own first     */
                                /* squaring step and keeps the fastest (the    */
                                /* environment variable QPE_SQUARE_TILE = 8,   */
                                /* 16 or 32 forces one instead)                */
#define QPE_FLAG_SQUARE_TC 0x100u /* U^(2^k) squarings of d >= 256 on the  */
                                  /* tcgen05 tensor cores with FP64-grade     */
                                  /* accuracy: 7 balanced 8-bit digits per     */
                                  /* entry (row / column power-of-two scales), */
                                  /* 28 exact bf16 digit products accumulated  */
                                  /* in integers (the Ozaki scheme); single-   */
                                  /* instance plans                            */
#define QPE_FLAG_LEVEL_TC 0x200u /* QPE_FP64: contractions on the tcgen05   */
                                 /* tensor cores with FP64-grade accuracy (7  */
                                 /* balanced 8-bit digits per operand at      */
                                 /* power-of-two row scales, 28 exact bf16    */
                                 /* digit products folded in integers): with  */
                                 /* nmat = 4 the fused schedule's 8-point     */
                                 /* levels of >= 128 pencils, the top level   */
                                 /* included (QPE_INFO_TC_TOP_LEVEL tells;    */
                                 /* twiddles and DFT in 64-bit fixed point,   */
                                 /* |X|^2 and readout in FP64; single-        */
                                 /* instance and sharded plans); with         */
                                 /* nmat >= 8 the plain schedule's doubling   */
                                 /* levels of >= 128 rows (single-instance,   */
                                 /* sharded and batched plans: one grouped    */
                                 /* round per level across the instances);    */
                                 /* ignored elsewhere                         */
#define QPE_FLAG_CHECK_UNITARY 0x40u /* the POWERS stage first forms U^dagger */
                                     /* U in FP64; if any entry of            */
                                     /* U^dagger U - I exceeds 1e-8 in        */
                                     /* modulus (or is not finite) the run's  */
                                     /* device error word is set and          */
                                     /* qpe_sync / qpe_probs return           */
                                     /* QPE_ERR_NUMERIC. 8 d^3 FP64 flop.     */

typedef struct {
  int32_t nmat;   /* target-register qubits, 1..12 (d = 2^nmat)                 */
  int32_t nmeas;  /* measurement qubits, 1..30 (N = 2^nmeas)                    */
  int32_t prec;   /* a qpe_precision                                           */
  uint32_t flags; /* QPE_FLAG_*                                                */
} qpe_plan_desc;

/* Stages of one run, in order (Fig. 1 left to right). */
typedef enum {
  QPE_STAGE_POWERS = 1, /* P_k = U^(2^k), k < Nmeas, by FP64 repeated squaring  */
  QPE_STAGE_SWEEP = 2,  /* Hadamard layer + all controlled-U^(2^k) gates: row m */
                        /* of the state becomes 2^(-n/2) U^m psi               */
  QPE_STAGE_FFT = 3,    /* QFT^-1 on the measurement register                   */
  QPE_STAGE_REDUCE = 4  /* P[y] = sum_t |X[y][t]|^2, argmax, weighted mean      */
} qpe_stage;

/* Introspection keys for qpe_query. */
typedef enum {
  QPE_INFO_WORKSPACE_BYTES = 1,
  QPE_INFO_STATE_BYTES = 2,     /* bytes of one instance's state                */
  QPE_INFO_FFT_PASSES = 3,      /* passes over the state the QFT^-1 takes      */
  QPE_INFO_LAST_LAUNCHES = 4,   /* kernels enqueued by the last qpe_run*       */
  QPE_INFO_INSTANCES = 5,
  QPE_INFO_SQUARE_TILE = 6,     /* batched plans: output tile edge (8, 16, 32)  */
                                /* of the grouped FP64 squaring in use         */
  QPE_INFO_LEVELS = 7,          /* fused schedule: number of levels (0 when    */
                                /* the plan runs another schedule)            */
  QPE_INFO_TOP_LEVEL_BITS = 8,  /* fused schedule: r of the top level, i.e.    */
                                /* its DFT length is 2^r (0 otherwise)         */
  QPE_INFO_TC_TOP_LEVEL = 9     /* 1 when the fused top level runs on the      */
                                /* tensor cores (split precision, nmat = 4)     */
} qpe_info;

/*
 * qpe_plan: validate a problem and size its workspace. Host only; touches no
 * GPU. On success *out is a new plan and *workspace_bytes the device bytes
 * qpe_bind needs. Errors: QPE_ERR_ARG for null pointers or nmat/nmeas/prec
 * out of range; QPE_ERR_UNSUPPORTED for combinations not built
 * (QPE_C64_BF16X3 in any plan; the split precisions with the gate-by-gate
 * schedule;
 * QPE_FLAG_GATE_SWEEP with nmat > 6; QPE_FLAG_REPEAT_U without
 * QPE_FLAG_GATE_SWEEP or with nmeas > 14).
 */
qpe_status qpe_plan(const qpe_plan_desc* desc, size_t* workspace_bytes, qpe_plan_t* out);

/*
 * qpe_plan_batched: one plan for `count` independent problems of uneven
 * nmat/nmeas (descs[i]; all with the same prec and flags; GATE_SWEEP is not
 * available here, QPE_ERR_UNSUPPORTED; TIMING gives the coarse split of
 * qpe_stage_times). Instances are addressed by index 0..count-1 in qpe_load /
 * qpe_probs / qpe_state. A run groups the work across instances: every launch
 * covers one step for every instance that needs it, its CTAs mapped to
 * (instance, tile) through work lists built at qpe_bind and kept in the
 * workspace. Steps: each U^(2^k) squaring (FP64 units; with
 * QPE_FLAG_SQUARE_TC the instances with d >= 256 on the tensor cores, their
 * digit-slice tensor maps in the work list); for nmat <= 6 the fused tables,
 * levels and readouts; for the plain instances (nmat > 6, or QPE_FLAG_PLAIN)
 * row 0, each doubling level (CUDA cores, one launch per tile class; under
 * the split precisions the levels of >= 128 rows and 2d >= 128 on the tensor
 * cores, per-item tensor maps), each QFT^-1 pass, the histograms and the
 * readouts. The number of launches depends on the largest nmeas and the tile
 * classes present, not on the number of instances. Under the split
 * precisions (QPE_C64_FP16X2 / TF32X3) instances with nmat <= 6 keep the
 * fused complex64 schedule. Only whole runs (qpe_run) are supported. Host
 * only, like qpe_plan.
 */
qpe_status qpe_plan_batched(const qpe_plan_desc* descs, int32_t count, size_t* workspace_bytes, qpe_plan_t* out);

/*
 * qpe_plan_shard: the plan of rank `rank` of `world` processes (world a power
 * of two, 1 .. 1024; 0 <= rank < world; QPE_ERR_ARG otherwise) that share one
 * problem, one GPU each. The paper runs on one GPU and names its memory as
 * the limit of the qubit count (Sec. 1); this splits the work of one run.
 * Rank r ends up with the outcomes y = r (mod world). Each rank reads U and
 * psi in full (qpe_load) and squares U itself. Two forms:
 *   - fused schedule (nmat <= 6, not QPE_FLAG_PLAIN; QPE_FP64, QPE_C64_FP32,
 *     or a split precision with nmat <= 4): the top level writes X[y] for
 *     y = y_a + N_a y_b from Z[y_a] alone (see qpe_run), and y = y_a
 *     (mod world) whenever world divides N_a, so every level with at least
 *     `world` pencils computes only this rank's y_a, from the same rank's
 *     share of the level below; smaller (deeper) levels are computed whole
 *     by every rank. No data moves between ranks during a run. Needs a top
 *     level with at least `world` pencils.
 *   - plain schedule (nmat > 6, QPE_FLAG_PLAIN, or a split precision with
 *     nmat >= 5): rank r holds the state rows m = r + world i (the low
 *     log2(world) measurement bits fixed), applies their controlled gates,
 *     and transforms them locally (QFT^-1 over the high bits); qpe_run stops
 *     there, with this rank's twiddled transform sorted by owner rank in a
 *     send buffer (qpe_shard_buffers). The caller then exchanges N / world^2
 *     rows with every other rank (an all-to-all of equal chunks: send chunk
 *     s goes to rank s, which stores it as its receive chunk r), and
 *     qpe_shard_finish runs the cross-rank length-world DFT, the histogram and
 *     the readout of this rank's outcomes. Needs N >= world^2; no
 *     QPE_FLAG_KEEP_STATE, no stage-by-stage runs, no qpe_state (the final
 *     state stays distributed).
 * After qpe_run (and, for the plain form, the exchange and qpe_shard_finish)
 * on every rank:
 *   - qpe_probs returns this rank's N / world bins compactly: probs[j] =
 *     P[rank + world j]; its argmax is the most probable of them (as a global
 *     y), phase_mean their share of sum_y P[y] y / N;
 *   - qpe_state (QPE_FLAG_KEEP_STATE) returns the N / world rows y = rank +
 *     world j in that order;
 *   - qpe_shard_readout gives the partial that qpe_merge_shard_readouts
 *     combines into the readout of the whole histogram.
 * Gathering the histograms is the caller's (e.g. an all-gather of N / world
 * doubles per rank, then P[r + world j] = part_r[j]). QPE_FLAG_GATE_SWEEP,
 * REPEAT_U and the requirements above not met: QPE_ERR_UNSUPPORTED. Host
 * only, like qpe_plan; world = 1 gives the ordinary plan.
 */
qpe_status qpe_plan_shard(const qpe_plan_desc* desc, int32_t rank, int32_t world, size_t* workspace_bytes,
                          qpe_plan_t* out);

/*
 * qpe_bind: attach caller-owned device memory and a CUDA stream (a
 * cudaStream_t, or NULL for the legacy default stream) to a plan. The
 * workspace must stay allocated until qpe_destroy or the next qpe_bind, be
 * 256-byte aligned and hold at least the size qpe_plan reported
 * (QPE_ERR_WORKSPACE otherwise). Builds the plan's twiddle tables on the
 * stream. QPE_FLAG_GRAPH plans need a non-NULL stream (QPE_ERR_ARG).
 */
qpe_status qpe_bind(qpe_plan_t plan, void* d_workspace, size_t bytes, void* cuda_stream);

/*
 * qpe_load: copy U (d x d complex128 row-major) and psi (d complex128) into
 * the workspace (the paper's host-to-device transfer, Sec. 4.3). ptr_is_device
 * = 0: host pointers; 1: device pointers. The caller keeps ownership of its
 * buffers. nmat/nmeas must equal the plan's (QPE_ERR_SHAPE); instance must be
 * 0 for single-problem plans.
 */
qpe_status qpe_load(qpe_plan_t plan, int32_t instance, const void* U, const void* psi,
                    int32_t nmat, int32_t nmeas, int32_t ptr_is_device);

/*
 * qpe_run: enqueue one whole run (all four stages) on the bound stream.
 * Asynchronous: no host synchronisation and no allocation. Requires bind and
 * load (QPE_ERR_STATE).
 *
 * Schedules. For nmat <= 6, unless QPE_FLAG_PLAIN or QPE_FLAG_GATE_SWEEP is
 * set, the controlled gates, QFT^-1 and the histogram run fused: with
 * m = m_b + 2^r m_a, X[y] = sum_{m_b} w_N^(m_b y) U^(m_b) Z[y mod N/2^r] where
 * Z is the same QPE for U^(2^r) on the high measurement qubits, so the work
 * recurses over levels of r <= 10 bits and the N x d state is never written
 * unless QPE_FLAG_KEEP_STATE asks for the final statevector. Otherwise the
 * state is materialised after the controlled gates (doubling or gate-by-gate
 * schedule) and transformed and reduced in separate passes.
 */
qpe_status qpe_run(qpe_plan_t plan);

/*
 * qpe_run_stages: enqueue stages first..last (qpe_stage values) only. Used to
 * check one step at a time: e.g. (SWEEP, SWEEP) after qpe_load_state-free
 * runs, or (FFT, REDUCE) after qpe_load_state. The POWERS stage must have run
 * (in this or an earlier call since the last qpe_load) before SWEEP.
 */
qpe_status qpe_run_stages(qpe_plan_t plan, int32_t first, int32_t last);

/*
 * qpe_probs: read the measurement histogram and the readout. probs (N
 * doubles, natural order of y) may be NULL to skip it; argmax is the most
 * probable outcome (lowest y on exact ties), phase_argmax = argmax / N, and
 * phase_mean = sum_y P[y] y / N (the weighted average of Sec. 4.2). Scalar
 * outputs may be NULL. ptr_is_device applies to probs only; the scalars are
 * always host pointers. Synchronises the stream and returns QPE_ERR_NUMERIC
 * if the device flagged a non-finite histogram.
 */
qpe_status qpe_probs(qpe_plan_t plan, int32_t instance, double* probs, int64_t* argmax,
                     double* phase_argmax, double* phase_mean, int32_t ptr_is_device);

/*
 * qpe_state: copy the current state (N x d, element type of the plan) in
 * natural row order: after SWEEP, row m = 2^(-n/2) U^m psi; after FFT, row y
 * is the final statevector (the paper's output file, Sec. 3). Host output
 * synchronises and reorders on the host; device output is reordered by a
 * kernel on the stream. After a fused qpe_run the final state exists only
 * with QPE_FLAG_KEEP_STATE (QPE_ERR_STATE otherwise).
 */
qpe_status qpe_state(qpe_plan_t plan, int32_t instance, void* out, int32_t ptr_is_device);

/*
 * qpe_load_state: overwrite the state with N x d elements (plan element type,
 * natural order); the next stage to run on it is FFT. For step-by-step checks.
 */
qpe_status qpe_load_state(qpe_plan_t plan, int32_t instance, const void* in, int32_t ptr_is_device);

/*
 * qpe_powers: copy P_k = U^(2^k) (d x d complex128) after the POWERS stage.
 */
qpe_status qpe_powers(qpe_plan_t plan, int32_t instance, int32_t k, void* out, int32_t ptr_is_device);

/* qpe_query: integer facts about a plan (qpe_info keys); -1 on a bad key. */
int64_t qpe_query(qpe_plan_t plan, int32_t key);

/*
 * qpe_stage_times: milliseconds each stage of the last qpe_run took on the
 * bound stream (ms[0..3] = POWERS, SWEEP, FFT, REDUCE), from CUDA events the
 * library records around its own launches. Needs QPE_FLAG_TIMING (QPE_ERR_STATE
 * otherwise). Batched plans split a run into every squaring step; the fused
 * instances' levels and the plain instances' doubling levels; the plain
 * instances' QFT^-1 passes; their histograms and every readout.
 * Synchronises the stream.
 */
qpe_status qpe_stage_times(qpe_plan_t plan, double* ms);

/*
 * qpe_kernel_time: milliseconds of the last qpe_run's dominant kernel on the
 * bound stream, from a CUDA event pair around that launch (QPE_FLAG_TIMING,
 * single instance): the top level of the fused schedule (the launch that
 * applies the controlled gates of the low measurement qubits to every row,
 * runs its QFT^-1 digit and writes the histogram). *kernel_id receives 1 for
 * that kernel, or 0 (and *ms = 0) when the last run used another schedule.
 * Synchronises the stream.
 */
qpe_status qpe_kernel_time(qpe_plan_t plan, double* ms, int32_t* kernel_id);

/* qpe_sync: wait for the bound stream and report device-side error flags. */
qpe_status qpe_sync(qpe_plan_t plan);

/*
 * qpe_selftest_timeout: run the failure path of a bounded device-side wait on
 * purpose. Enqueues one kernel that holds tensor memory while one thread
 * waits, with a limit of `polls` polls (1 .. 2^20, else QPE_ERR_ARG), on an
 * mbarrier that nothing arrives at; when the limit runs out the kernel does
 * what every tcgen05 kernel of the library does on an expired wait: it
 * records QPE_ERR_TIMEOUT in the instance's device error word, frees its
 * tensor memory and returns. No copy or MMA is in flight while it waits. The
 * next qpe_sync or qpe_probs reports QPE_ERR_TIMEOUT; the next whole qpe_run
 * clears the word. Single-instance plans only (QPE_ERR_UNSUPPORTED for
 * batched plans); requires qpe_bind. Not part of the paper's method: it
 * tests the library's failure detection.
 */
qpe_status qpe_selftest_timeout(qpe_plan_t plan, int32_t instance, uint32_t polls);

/* qpe_destroy: free the host-side plan (and its CUDA graph, if any). Does not
 * touch the caller's workspace. NULL is accepted. */
qpe_status qpe_destroy(qpe_plan_t plan);

/* Readout written by qpe_readout_static (device memory, caller-owned). */
typedef struct {
  int64_t argmax;      /* most probable outcome, lowest y on exact ties; -1    */
                       /* when the histogram is not finite (a NaN or Inf in    */
                       /* the state), which the caller tests through total     */
  double phase_argmax; /* argmax / N (NaN when argmax is -1)                  */
  double phase_mean;   /* sum_y P[y] y / N                                    */
  double total;        /* sum_y P[y]                                          */
} qpe_readout_t;

/*
 * qpe_readout_static: histogram and readout of a final statevector without
 * any device allocation and without a plan. The paper has no counterpart;
 * this serves callers that cannot allocate device memory (code where an
 * allocation would synchronise or grow a memory pool that must stay fixed,
 * or a host library that never owns device memory), so it needs no
 * workspace: its only scratch, the per-block partial results, is a fixed
 * array inside the library (256 KiB on every GPU that loads it, held until
 * the process exits).
 *
 * final_state: device pointer to the N x d final statevector in natural row
 * order (complex128 for QPE_FP64, complex64 for the other precisions), as
 * qpe_state returns it. Outputs, device pointers owned by the caller: probs
 * (N doubles, P[y] = sum_t |X[y][t]|^2) and *readout. Enqueued on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream); no host
 * synchronisation. Nmeas above 21 is rejected with QPE_ERR_WORKSPACE (the
 * fixed scratch holds 8192 partials of 256 rows each); bad pointers or
 * shapes with QPE_ERR_ARG. The first call on each device looks up the
 * scratch's device address (cudaGetSymbolAddress); make that first call
 * outside any stream capture. All calls on a device share the scratch: two
 * calls whose kernels may overlap on the GPU (different streams, no
 * ordering between them) race on it.
 */
qpe_status qpe_readout_static(const void* final_state, int32_t nmat, int32_t nmeas, int32_t prec, double* probs,
                              qpe_readout_t* readout, void* cuda_stream);

/* One rank's share of the readout of a sharded run (qpe_plan_shard). */
typedef struct {
  int64_t argmax;         /* most probable outcome among this rank's bins (global y) */
  double p_argmax;        /* its probability                                         */
  double phase_mean_part; /* sum over this rank's bins of P[y] y / N                 */
  double total;           /* sum over this rank's bins of P[y]                       */
  int32_t nmeas;
  int32_t rank;
} qpe_shard_readout_t;

/*
 * qpe_shard_readout: this rank's readout partial after qpe_run (host output;
 * synchronises the stream; QPE_ERR_NUMERIC / QPE_ERR_TIMEOUT as qpe_probs).
 */
qpe_status qpe_shard_readout(qpe_plan_t plan, qpe_shard_readout_t* out);

/*
 * qpe_shard_buffers: device pointers of a sharded plain plan's all-to-all
 * buffers in its workspace and the bytes exchanged with each rank: send holds
 * world chunks of *bytes_per_peer bytes (chunk s for rank s), recv receives
 * world chunks (chunk r from rank r). After qpe_run the send buffer is ready
 * on the bound stream; the receive buffer must be filled before
 * qpe_shard_finish is enqueued. Fused sharded plans exchange nothing: NULL
 * pointers and 0 bytes.
 */
qpe_status qpe_shard_buffers(qpe_plan_t plan, void** send, void** recv, size_t* bytes_per_peer);

/*
 * qpe_shard_finish: after the exchange, enqueue the rest of a sharded plain
 * run on the bound stream (the cross-rank DFT, this rank's histogram and
 * readout partial); QPE_ERR_STATE unless qpe_run came first. For a fused
 * sharded plan it only checks that qpe_run came first.
 */
qpe_status qpe_shard_finish(qpe_plan_t plan);

/*
 * qpe_merge_shard_readouts: the readout of the whole histogram from the
 * `world` partials of one sharded run (host only, any order of parts): the
 * argmax by the plan path's rule (larger probability, then the lower y on an
 * exact tie), phase_argmax = argmax / N, phase_mean and total summed in the
 * order of parts. QPE_ERR_SHAPE if the parts disagree on nmeas,
 * QPE_ERR_NUMERIC if any part holds a value that is not finite.
 */
qpe_status qpe_merge_shard_readouts(const qpe_shard_readout_t* parts, int32_t world, qpe_readout_t* out);

/*
 * qpe_host_alloc / qpe_host_free: page-locked host memory (cudaHostAlloc) of
 * `bytes` bytes for a plan's host-side inputs and outputs (U, psi, the
 * histogram of qpe_probs, the state of qpe_state). Copies between the device
 * and such memory run at the host link's rate, which is not the case for every
 * page-locked buffer (on GB300 hosts, a large buffer pinned by another route
 * may be read or written at a fraction of it). The caller owns the memory
 * and frees it with qpe_host_free (not with free()). QPE_ERR_ARG for
 * bytes == 0 or ptr == NULL; QPE_ERR_CUDA if the allocation fails, with
 * *ptr = NULL. qpe_host_free(NULL) is QPE_OK.
 */
qpe_status qpe_host_alloc(size_t bytes, void** ptr);
qpe_status qpe_host_free(void* ptr);

/*
 * qpe_set_host_histogram: every following whole run of `instance` also copies
 * its histogram (N / 2^shard_log doubles, local index order as qpe_probs) into
 * `host`, page-locked memory from qpe_host_alloc that stays valid while it is
 * set. Where the top level allows it (the FP64 top level on the tensor cores,
 * QPE_FLAG_LEVEL_TC) the copy overlaps the computation: that level runs in
 * eight tile ranges and a copy stream forked from the plan's stream moves each
 * range's bins while the next range computes, joining the plan's stream before
 * the run ends; otherwise it follows the run on the plan's stream. The copy is
 * complete when qpe_sync or qpe_probs returns; qpe_probs with probs == host
 * does not copy again. host = NULL stops the copies. QPE_ERR_ARG if host is
 * not page-locked host memory, QPE_ERR_STATE before qpe_bind,
 * QPE_ERR_UNSUPPORTED for batched plans and sharded plans of the plain
 * schedule. A graph-replayed plan captures the new copies at its next run.
 */
qpe_status qpe_set_host_histogram(qpe_plan_t plan, int32_t instance, double* host);

const char* qpe_status_string(qpe_status s);
/* Last error message recorded on the plan ("" if none; static text for NULL). */
const char* qpe_last_error(qpe_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* QPE_H */
