// C ABI of the QPE emulator: plan validation, workspace layout, stage
// scheduling, readback. Declarations and contracts are in include/qpe.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "qpe_internal.cuh"

namespace qpe {
cudaError_t configure_kernels();
bool g_pdl_enabled = false;
}

#ifndef QPE_MAX_FUSED_NMAT
#define QPE_MAX_FUSED_NMAT 6
#endif

using qpe::Instance;

namespace {

constexpr int kMaxNmat = 12;
constexpr int kMaxNmeas = 30;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

bool is_c64(int prec) { return prec != QPE_FP64; }
// split-precision tensor-core plans (complex64 state, tcgen05 U-application)
bool is_tc(int prec) { return prec == QPE_C64_TF32X3 || prec == QPE_C64_FP16X2; }
size_t elem_size(int prec) { return is_c64(prec) ? 8 : 16; }

qpe_status fail(qpe_plan_t p, qpe_status st, const std::string& msg) {
  if (p) p->last_error = msg;
  return st;
}

qpe_status cuda_fail(qpe_plan_t p, cudaError_t e, const char* where) {
  return fail(p, QPE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

// Lays out one instance starting at byte offset `base`; returns the end.
// Batched plans keep instances with Nmat <= 6 on the fused complex64 schedule
// under the split precisions; those apply to the plain instances' gate GEMMs.
size_t layout_instance(Instance& in, int prec, uint32_t flags, size_t base, bool batched = false) {
  const int64_t d = in.d, N = in.N;
  size_t off = align_up(base);
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  in.off_pow64 = take((size_t)in.nmeas * d * d * 16);
  in.off_pow32 = is_c64(prec) ? take((size_t)in.nmeas * d * d * 8) : 0;
  in.off_psi = take((size_t)d * 16);
  in.fused = in.nmat <= QPE_MAX_FUSED_NMAT && !(flags & (QPE_FLAG_PLAIN | QPE_FLAG_GATE_SWEEP)) &&
             (!is_tc(prec) || batched || in.nmat <= 4);
  in.keep_state = (flags & QPE_FLAG_KEEP_STATE) != 0;
  if (in.nmat <= QPE_MAX_FUSED_NMAT) in.levels = qpe::make_levels(in.nmeas, in.nmat, elem_size(prec), 0);
  // the fused schedule never materialises the N x d state unless asked to keep
  // it; a sharded plan keeps (and histograms) only its own N / 2^shard_log rows
  in.state_bytes = (size_t)(N >> in.shard_log) * d * elem_size(prec);
  in.has_state = !in.fused || in.keep_state;
  in.off_state = in.has_state ? take(in.state_bytes) : 0;
  in.off_hist = take((size_t)(N >> in.shard_log) * 8);
  in.htw = (in.nmeas + 1) / 2;
  const size_t nlo = size_t(1) << in.htw, nhi = size_t(1) << (in.nmeas - in.htw);
  in.off_tw_lo64 = take(nlo * 16);
  in.off_tw_hi64 = take(nhi * 16);
  in.off_tw_lo32 = take(nlo * 8);
  in.off_tw_hi32 = take(nhi * 8);
  in.off_partials = take(sizeof(qpe::Partial) * qpe::kReduceBlocks);
  in.off_scalars = take(sizeof(qpe::Scalars));
  in.off_err = take(sizeof(int));
  if (is_tc(prec) && !in.fused) in.off_tcsplit = take(qpe::tc_split_bytes(prec, in.nmat, in.nmeas));
  // sharded plain schedule: all-to-all buffers of the local transform
  in.shard_plain = !in.fused && in.shard_log > 0;
  if (in.shard_plain) {
    in.off_send = take(in.state_bytes);
    in.off_recv = take(in.state_bytes);
  }
  in.oz_square = (flags & QPE_FLAG_SQUARE_TC) && in.nmat >= 8 && in.nmeas >= 2;
  // FP64 plain doubling levels of at least 128 rows on the tensor cores
  // (a batched plan's instances share one row-digit buffer per level instead)
  in.oz_gates = prec == QPE_FP64 && (flags & QPE_FLAG_LEVEL_TC) && !in.fused && in.nmat >= 8 &&
                !(flags & QPE_FLAG_GATE_SWEEP) && in.nmeas - in.shard_log >= 8;
  if (in.oz_square || in.oz_gates) in.off_ozsq = take(qpe::oz_square_bytes(in.nmat));
  if (in.oz_gates && !batched) in.off_ozgate = take(qpe::oz_gate_bytes(in.nmat, (int64_t)(N >> in.shard_log)));
  // the fused top level on the tensor cores, d = 16, histogram only: a split
  // precision with a 16-point top level and at least one tile of 128 pencils
  // per rank, or FP64 (QPE_FLAG_LEVEL_TC) with an 8-point one of at least 128
  // pencils in all (a rank with fewer runs one partial tile, so that sharded
  // and unsharded plans take the same arithmetic)
  const bool tc_top_ok = in.fused && !batched && in.nmat == 4 && !in.keep_state && !in.levels.empty();
  const bool fp64_top = prec == QPE_FP64 && (flags & QPE_FLAG_LEVEL_TC) && tc_top_ok && in.levels[0].r == 3 &&
                        in.levels[0].logna >= 7;
  in.tc_top = (tc_top_ok && is_tc(prec) && in.levels[0].r == 4 && in.levels[0].logna - in.shard_log >= 7) ||
              fp64_top;
  in.tc_top_prec = prec;
  // FP64: the lower 8-point levels too (each one that fills 128-pencil tiles)
  in.oz_levels = prec == QPE_FP64 && (flags & QPE_FLAG_LEVEL_TC) && in.fused && !batched && in.nmat == 4;
  if (in.tc_top || in.oz_levels)
    in.off_tctab = take(in.oz_levels ? qpe::oz_top_table_bytes() : qpe::tc_top_table_bytes());
  in.fft = qpe::make_fft_plan(in.nmeas - (in.shard_plain ? in.shard_log : 0), d, elem_size(prec));
  if (in.nmat <= QPE_MAX_FUSED_NMAT) {
    // level buffers for the fused schedule (also allotted to plain plans so a
    // plan's layout does not depend on its schedule flags)
    size_t zb[2] = {0, 0};
    for (size_t li = 1; li < in.levels.size(); ++li) {
      const qpe::Level& L = in.levels[li];
      const int lsh = qpe::level_sharded(in, (int)li) ? in.shard_log : 0;
      const size_t bytes = ((size_t)1 << (L.logna + L.r - lsh)) * d * elem_size(prec);
      zb[li & 1] = std::max(zb[li & 1], bytes);
    }
    in.off_zbuf[0] = take(zb[0] ? zb[0] : 16);
    in.off_zbuf[1] = take(zb[1] ? zb[1] : 16);
    in.zbuf_seed_off = take((size_t)d * elem_size(prec));
    for (qpe::Level& L : in.levels) L.tab_off = take(((size_t)d << L.r) * d * elem_size(prec));
  }
  return off;
}

qpe_status check_desc(const qpe_plan_desc* desc, bool batched = false) {
  if (!desc) return QPE_ERR_ARG;
  if (desc->nmat < 1 || desc->nmat > kMaxNmat) return QPE_ERR_ARG;
  if (desc->nmeas < 1 || desc->nmeas > kMaxNmeas) return QPE_ERR_ARG;
  if (desc->prec < QPE_FP64 || desc->prec > QPE_C64_TF32X3) return QPE_ERR_ARG;
  if (desc->flags & ~(QPE_FLAG_GATE_SWEEP | QPE_FLAG_GRAPH | QPE_FLAG_TIMING | QPE_FLAG_PLAIN | QPE_FLAG_KEEP_STATE |
                      QPE_FLAG_REPEAT_U | QPE_FLAG_CHECK_UNITARY | QPE_FLAG_AUTOTUNE | QPE_FLAG_SQUARE_TC |
                      QPE_FLAG_LEVEL_TC))
    return QPE_ERR_ARG;
  if ((desc->flags & QPE_FLAG_REPEAT_U) && (!(desc->flags & QPE_FLAG_GATE_SWEEP) || desc->nmeas > 14))
    return QPE_ERR_UNSUPPORTED;
  // bf16 hi/lo splits keep ~16 bits per operand: the histogram's L1 error
  // against FP64 then exceeds 1e-6 after enough gate levels (1.6e-6 measured
  // at Nmeas = 18), so the library does not offer that precision
  if (desc->prec == QPE_C64_BF16X3) return QPE_ERR_UNSUPPORTED;
  if (is_tc(desc->prec) && (desc->flags & QPE_FLAG_GATE_SWEEP)) return QPE_ERR_UNSUPPORTED;
  if ((desc->flags & QPE_FLAG_GATE_SWEEP) && desc->nmat > 6) return QPE_ERR_UNSUPPORTED;
  return QPE_OK;
}

// What a non-zero device error word means.
const char* err_word_message(int derr) {
  return derr == QPE_ERR_NUMERIC ? "U is not unitary to 1e-8 (QPE_FLAG_CHECK_UNITARY)"
                                 : "a bounded device wait expired during the run";
}

qpe_status get_instance(qpe_plan_t p, int32_t i, Instance** out) {
  if (!p) return QPE_ERR_ARG;
  if (i < 0 || i >= (int32_t)p->inst.size()) return fail(p, QPE_ERR_SHAPE, "instance index out of range");
  *out = &p->inst[i];
  return QPE_OK;
}

cudaMemcpyKind kind_to_device(int32_t ptr_is_device) {
  return ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_from_device(int32_t ptr_is_device) {
  return ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

}  // namespace

namespace qpe {
// Records a timing event; inside stream capture it must become an event
// record node of the graph (cudaEventRecordExternal), outside it is a plain
// record (the external flag is rejected on a stream that is not capturing).
cudaError_t record_event(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, s);
}
}  // namespace qpe

namespace {
using qpe::record_event;

// Enqueue stages first..last for every instance; returns launches or sets error.
qpe_status enqueue_batched(qpe_plan_t p, int64_t* launches);

qpe_status enqueue_stages(qpe_plan_t p, int first, int last, int64_t* launches) {
  if (p->batched) {
    if (first != QPE_STAGE_POWERS || last != QPE_STAGE_REDUCE)
      return fail(p, QPE_ERR_UNSUPPORTED, "batched plans run whole (POWERS..REDUCE) only");
    return enqueue_batched(p, launches);
  }
  int64_t n = 0;
  const bool c64 = is_c64(p->prec);
  const bool gate = (p->flags & QPE_FLAG_GATE_SWEEP) != 0;
  const bool timing = (p->flags & QPE_FLAG_TIMING) && p->inst.size() == 1 && p->ev[0];
  p->timed_run = timing && first == QPE_STAGE_POWERS && last == QPE_STAGE_REDUCE;
  p->timed_kernel = false;
  const bool check_u = (p->flags & QPE_FLAG_CHECK_UNITARY) != 0;
  for (Instance& in : p->inst) {
    if (!in.loaded) return fail(p, QPE_ERR_STATE, "qpe_load has not been called for every instance");
    // the error word covers one run: cleared where a whole run, or the first
    // stage that can set it, begins
    if (first == QPE_STAGE_POWERS || (first == QPE_STAGE_SWEEP && (is_tc(p->prec) || in.oz_gates))) {
      cudaError_t e = cudaMemsetAsync(p->ws + in.off_err, 0, sizeof(int), p->stream);
      if (e != cudaSuccess) return cuda_fail(p, e, "error word reset");
    }
    if (check_u && first == QPE_STAGE_POWERS) {
      if (qpe::launch_check_unitary(in, p->ws, p->stream) < 0) return cuda_fail(p, cudaGetLastError(), "unitarity check");
      ++n;
    }
    if (in.shard_plain) {
      // this rank's part of a run up to the exchange: powers, the controlled
      // gates of its rows, its local QFT^-1 passes, the sorted send buffer
      if (first != QPE_STAGE_POWERS || last != QPE_STAGE_REDUCE)
        return fail(p, QPE_ERR_UNSUPPORTED, "sharded plans of the plain schedule run whole (qpe_run)");
      const int prec_arg = p->prec;
      int r = qpe::launch_powers(in, p->ws, c64, p->stream);
      if (r >= 0) {
        n += r;
        r = c64 ? qpe::launch_sweep<float2>(in, p->ws, false, p->stream, prec_arg)
                : qpe::launch_sweep<double2>(in, p->ws, false, p->stream, prec_arg);
      }
      if (r >= 0) {
        n += r;
        r = c64 ? qpe::launch_fft<float2>(in, p->ws, p->stream) : qpe::launch_fft<double2>(in, p->ws, p->stream);
      }
      if (r >= 0) {
        n += r;
        r = c64 ? qpe::launch_shard_pack<float2>(in, p->ws, p->stream)
                : qpe::launch_shard_pack<double2>(in, p->ws, p->stream);
      }
      if (r < 0) return cuda_fail(p, cudaGetLastError(), "kernel launch");
      n += r;
      in.powers_done = true;
      in.state_stage = qpe::kStageExchange;
      in.state_natural = false;
      in.state_valid = false;
      continue;
    }
    if (in.fused && first <= QPE_STAGE_SWEEP && last == QPE_STAGE_REDUCE) {
      // fused schedule: POWERS, then the levels (gates + QFT^-1 + histogram)
      for (int st = first; st <= QPE_STAGE_REDUCE; ++st) {
        if (timing) {
          cudaError_t e = record_event(p->ev[st - 1], p->stream);
          if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventRecord");
        }
        int r = 0;
        if (st == QPE_STAGE_POWERS) {
          r = qpe::launch_powers(in, p->ws, c64, p->stream);
          in.powers_done = true;
        } else if (st == QPE_STAGE_SWEEP) {
          if (!in.powers_done) return fail(p, QPE_ERR_STATE, "SWEEP before POWERS");
          cudaEvent_t* kev = timing ? &p->ev[5] : nullptr;
          r = c64 ? qpe::launch_levels<float2>(in, p->ws, in.keep_state, p->stream, kev)
                  : qpe::launch_levels<double2>(in, p->ws, in.keep_state, p->stream, kev);
          p->timed_kernel = timing;
        }
        if (r < 0) return cuda_fail(p, cudaGetLastError(), "kernel launch");
        n += r;
      }
      if (timing) {
        cudaError_t e = record_event(p->ev[QPE_STAGE_REDUCE], p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventRecord");
      }
      if (in.host_hist && !qpe::oz_top_copies_host_histogram(in)) {
        cudaError_t e = cudaMemcpyAsync(in.host_hist, p->ws + in.off_hist, (size_t)(in.N >> in.shard_log) * 8,
                                        cudaMemcpyDeviceToHost, p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "host histogram copy");
      }
      in.state_stage = QPE_STAGE_REDUCE;
      in.state_natural = true;
      in.state_valid = in.keep_state;
      continue;
    }
    if (!in.has_state && last >= QPE_STAGE_SWEEP)
      return fail(p, QPE_ERR_STATE,
                  "this fused plan has no state buffer for stage-by-stage runs; plan with QPE_FLAG_PLAIN or "
                  "QPE_FLAG_KEEP_STATE");
    for (int st = first; st <= last; ++st) {
      if (timing) {
        cudaError_t e = record_event(p->ev[st - 1], p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventRecord");
      }
      int r = 0;
      switch (st) {
        case QPE_STAGE_POWERS:
          r = qpe::launch_powers(in, p->ws, c64, p->stream);
          in.powers_done = true;
          break;
        case QPE_STAGE_SWEEP:
          if (!in.powers_done) return fail(p, QPE_ERR_STATE, "SWEEP before POWERS");
          {
            const int prec_arg = (p->flags & QPE_FLAG_REPEAT_U) ? -1 : p->prec;  // -1: repeat U 2^k times
            r = c64 ? qpe::launch_sweep<float2>(in, p->ws, gate, p->stream, prec_arg)
                    : qpe::launch_sweep<double2>(in, p->ws, gate, p->stream, prec_arg);
          }
          in.state_stage = QPE_STAGE_SWEEP;
          in.state_natural = true;
          in.state_valid = true;
          break;
        case QPE_STAGE_FFT:
          if (in.state_stage != QPE_STAGE_SWEEP) return fail(p, QPE_ERR_STATE, "FFT needs the state after SWEEP");
          if (!in.state_valid) return fail(p, QPE_ERR_STATE, "no materialised state to transform");
          r = c64 ? qpe::launch_fft<float2>(in, p->ws, p->stream) : qpe::launch_fft<double2>(in, p->ws, p->stream);
          in.state_stage = QPE_STAGE_FFT;
          in.state_natural = false;
          break;
        case QPE_STAGE_REDUCE:
          if ((in.state_stage != QPE_STAGE_FFT && in.state_stage != QPE_STAGE_REDUCE) || in.state_natural ||
              !in.state_valid)
            return fail(p, QPE_ERR_STATE, "REDUCE needs the state after FFT");
          r = c64 ? qpe::launch_reduce<float2>(in, p->ws, p->stream)
                  : qpe::launch_reduce<double2>(in, p->ws, p->stream);
          in.state_stage = QPE_STAGE_REDUCE;
          break;
        default:
          return fail(p, QPE_ERR_ARG, "bad stage");
      }
      if (r < 0) return cuda_fail(p, cudaGetLastError(), "kernel launch");
      n += r;
    }
    if (timing) {
      cudaError_t e = record_event(p->ev[last], p->stream);
      if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventRecord");
    }
    if (in.host_hist && last == QPE_STAGE_REDUCE) {
      cudaError_t e = cudaMemcpyAsync(in.host_hist, p->ws + in.off_hist, (size_t)(in.N >> in.shard_log) * 8,
                                      cudaMemcpyDeviceToHost, p->stream);
      if (e != cudaSuccess) return cuda_fail(p, e, "host histogram copy");
    }
  }
  *launches = n;
  return QPE_OK;
}


// (Re)builds a batched plan's work lists. With ws == nullptr only the counts
// matter (plan time, for sizing); at bind the device pointers are filled in.
void build_batch_meta(qpe_plan_t p, char* ws, int nsm) {
  qpe::BatchMeta& bm = p->bm;
  const bool c64 = is_c64(p->prec);
  const size_t esize = elem_size(p->prec);
  bm.sq.clear();
  bm.conv.clear();
  bm.fused.clear();
  bm.plain.clear();
  bm.tab_items.clear();
  bm.seed_items.clear();
  bm.level_args.clear();
  bm.items.clear();
  bm.launches.clear();
  bm.fin.clear();
  bm.init_items.clear();
  bm.dbl_items.clear();
  bm.fft_items.clear();
  bm.red_items.clear();
  bm.dbl_rounds.clear();
  bm.oz_items.clear();
  bm.oz_steps.clear();
  bm.gate_p.clear();
  bm.gate_g.clear();
  bm.gate_r.clear();
  bm.gate_rounds.clear();
  bm.gate_buf_bytes = 0;
  bm.tc_split.clear();
  bm.tc_gemm.clear();
  bm.tc_rounds.clear();
  bm.fft_rounds.clear();
  bm.fin_plain.clear();
  bm.ninit = bm.nred = bm.maxn_plain = 0;
  bm.red_blocks = 0;
  bm.maxn = 0;
  for (const Instance& in : p->inst) bm.maxn = std::max(bm.maxn, in.nmeas);
  bm.sq_begin.assign(bm.maxn + 1, 0);
  bm.sq_count.assign(bm.maxn + 1, 0);
  bm.sq_tiles.assign(bm.maxn + 1, 0);
  bm.sq_tiles16.assign(bm.maxn + 1, 0);
  bm.sq_tiles32.assign(bm.maxn + 1, 0);
  for (int k = 1; k < bm.maxn; ++k) {
    bm.sq_begin[k] = (int)bm.sq.size();
    int64_t tiles = 0, tiles16 = 0, tiles32 = 0;
    for (Instance& in : p->inst) {
      if (in.nmeas <= k || in.oz_square) continue;  // tensor-core squarings are launched per instance
      const int64_t dd = in.d * in.d;
      double2* P = reinterpret_cast<double2*>(ws + in.off_pow64);
      float2* P32 = c64 ? reinterpret_cast<float2*>(ws + in.off_pow32) : nullptr;
      qpe::SqItem it{};
      it.A = P + (k - 1) * dd;
      it.C = P + k * dd;
      it.C32 = P32 ? P32 + k * dd : nullptr;
      it.A32 = (P32 && k == 1) ? P32 : nullptr;
      it.d = (int)in.d;
      it.tile0 = tiles;
      it.tile16 = tiles16;
      it.tile32 = tiles32;
      tiles += ((in.d + 7) / 8) * ((in.d + 7) / 8);
      tiles16 += ((in.d + 15) / 16) * ((in.d + 15) / 16);
      tiles32 += ((in.d + 31) / 32) * ((in.d + 31) / 32);
      bm.sq.push_back(it);
    }
    bm.sq_count[k] = (int)bm.sq.size() - bm.sq_begin[k];
    // the tensor-core squarings of this step, one grouped launch set
    qpe::OzStep O{};
    O.k = k;
    O.item_off = (int)bm.oz_items.size();
    for (Instance& in : p->inst) {
      if (in.nmeas <= k || !in.oz_square) continue;
      qpe::OzItem oz{};
      if (!qpe::oz_square_item(in, ws, k, c64, &oz)) throw std::runtime_error("tensor map");
      oz.sb0 = O.sblocks;
      oz.e0 = O.elems;
      oz.tile0 = O.tiles;
      O.sblocks += 2 * in.d;
      O.elems += in.d * in.d;
      O.tiles += qpe::oz_square_tiles(in);
      bm.oz_items.push_back(oz);
    }
    O.nitems = (int)bm.oz_items.size() - O.item_off;
    if (O.nitems > 0) bm.oz_steps.push_back(O);
    bm.sq_tiles[k] = tiles;
    bm.sq_tiles16[k] = tiles16;
    bm.sq_tiles32[k] = tiles32;
  }
  bm.conv_tiles = 0;
  if (c64)
    for (Instance& in : p->inst)
      if (in.nmeas == 1) {
        qpe::SqItem it{};
        it.A = reinterpret_cast<double2*>(ws + in.off_pow64);
        it.A32 = reinterpret_cast<float2*>(ws + in.off_pow32);
        it.d = (int)in.d;
        it.tile0 = bm.conv_tiles;
        bm.conv_tiles += (in.d * in.d + 255) / 256;
        bm.conv.push_back(it);
      }
  for (size_t i = 0; i < p->inst.size(); ++i) (p->inst[i].fused ? bm.fused : bm.plain).push_back((int)i);
  // tables and seeds of the fused instances
  bm.ntab = 0;
  bm.tab_blocks = 0;
  bm.max_logd = 1;
  bm.nseed = 0;
  auto push_bytes = [](std::vector<char>& v, const void* src, size_t n) {
    const size_t o = v.size();
    v.resize(o + n);
    std::memcpy(v.data() + o, src, n);
  };
  for (int i : bm.fused) {
    const Instance& in = p->inst[i];
    bm.max_logd = std::max(bm.max_logd, in.nmat);
    const int D = (int)in.d, TB = D < 16 ? D : 16;
    for (const qpe::Level& L : in.levels) {
      if (c64) {
        qpe::TabItem<float2> t{};
        t.P = reinterpret_cast<const float2*>(ws + in.off_pow32);
        t.tab = reinterpret_cast<float2*>(ws + L.tab_off);
        t.off = L.off;
        t.r = L.r;
        t.logd = in.nmat;
        t.tile0 = bm.tab_blocks;
        push_bytes(bm.tab_items, &t, sizeof(t));
      } else {
        qpe::TabItem<double2> t{};
        t.P = reinterpret_cast<const double2*>(ws + in.off_pow64);
        t.tab = reinterpret_cast<double2*>(ws + L.tab_off);
        t.off = L.off;
        t.r = L.r;
        t.logd = in.nmat;
        t.tile0 = bm.tab_blocks;
        push_bytes(bm.tab_items, &t, sizeof(t));
      }
      bm.tab_blocks += (int64_t(1) << L.r) * (D / TB);
      ++bm.ntab;
    }
    if (c64) {
      qpe::SeedItem<float2> sd{reinterpret_cast<const double2*>(ws + in.off_psi),
                               reinterpret_cast<float2*>(ws + in.zbuf_seed_off), D, 0};
      push_bytes(bm.seed_items, &sd, sizeof(sd));
    } else {
      qpe::SeedItem<double2> sd{reinterpret_cast<const double2*>(ws + in.off_psi),
                                reinterpret_cast<double2*>(ws + in.zbuf_seed_off), D, 0};
      push_bytes(bm.seed_items, &sd, sizeof(sd));
    }
    ++bm.nseed;
  }
  // level rounds, deepest first; one grouped launch per (round, d, top/other)
  int maxl = 0;
  for (int i : bm.fused) maxl = std::max(maxl, (int)p->inst[i].levels.size());
  std::vector<int> part_count(p->inst.size(), 0);
  const size_t asz = c64 ? sizeof(qpe::LevelArgs<float2>) : sizeof(qpe::LevelArgs<double2>);
  for (int t = 0; t < maxl; ++t) {
    for (int top = 0; top < 2; ++top) {
      for (int logd = 1; logd <= QPE_MAX_FUSED_NMAT; ++logd) {
        qpe::LevelLaunch LL{};
        LL.logd = logd;
        LL.arg_off = (int)(bm.level_args.size() / asz);
        LL.item_off = (int)bm.items.size();
        int nargs = 0;
        for (int i : bm.fused) {
          Instance& in = p->inst[i];
          const int nl = (int)in.levels.size();
          if (in.nmat != logd || t >= nl) continue;
          const int li = nl - 1 - t;
          if ((li == 0) != (top == 1)) continue;
          const int mode = li == 0 ? (in.keep_state ? 2 : 1) : 0;
          LL.mode = mode;
          const qpe::Level& L = in.levels[li];
          char* seeds = (li == nl - 1) ? ws + in.zbuf_seed_off : ws + in.off_zbuf[(li + 1) & 1];
          char* P = ws + (c64 ? in.off_tw_lo32 : in.off_tw_lo64);
          char* Ph = ws + (c64 ? in.off_tw_hi32 : in.off_tw_hi64);
          char* xout = li > 0 ? ws + in.off_zbuf[li & 1] : (in.keep_state ? ws + in.off_state : nullptr);
          const double xscale = (li == 0 && in.keep_state) ? ldexp(1.0, -in.nmeas) : 1.0;
#define QPE_FILL_ARGS(CT)                                                   \
  {                                                                         \
    qpe::LevelArgs<CT> a{};                                                 \
    a.seeds = reinterpret_cast<const CT*>(seeds);                           \
    a.tab = reinterpret_cast<const CT*>(ws + L.tab_off);                    \
    a.off = L.off;                                                          \
    a.r = L.r;                                                              \
    a.logna = L.logna;                                                      \
    a.logd = in.nmat;                                                       \
    a.nmeas = in.nmeas;                                                     \
    a.htw = in.htw;                                                         \
    a.tw_lo = reinterpret_cast<const CT*>(P);                               \
    a.tw_hi = reinterpret_cast<const CT*>(Ph);                              \
    a.xout = reinterpret_cast<CT*>(xout);                                   \
    a.hist = reinterpret_cast<double*>(ws + in.off_hist);                   \
    a.parts = reinterpret_cast<qpe::Partial*>(ws + in.off_partials);        \
    a.pscale = ldexp(1.0, -2 * in.nmeas);                                   \
    a.inv_n = ldexp(1.0, -in.nmeas);                                        \
    a.xscale = xscale;                                                      \
    push_bytes(bm.level_args, &a, sizeof(a));                               \
  }
          if (c64)
            QPE_FILL_ARGS(float2)
          else
            QPE_FILL_ARGS(double2)
#undef QPE_FILL_ARGS
          int DI = 0, G = 0;
          qpe::level_shape(logd, mode, elem_size(p->prec), &DI, &G);
          const int ncg = (int)(in.d / DI);
          const int64_t iters = ((int64_t(1) << L.logna) + G - 1) / G;
          int64_t ch = 4;
          if (mode != 0) ch = std::max<int64_t>(4, (iters + qpe::kReduceBlocks - 1) / qpe::kReduceBlocks);
          for (int cg = 0; cg < ncg; ++cg)
            for (int64_t c0 = 0; c0 < iters; c0 += ch) {
              qpe::GroupItem gi{};
              gi.arg = nargs;
              gi.cg = cg;
              gi.it_begin = c0;
              gi.it_end = std::min(iters, c0 + ch);
              gi.part = mode != 0 ? part_count[i]++ : 0;
              bm.items.push_back(gi);
            }
          if (mode != 0) {
            qpe::FinItem f{};
            f.parts = reinterpret_cast<const qpe::Partial*>(ws + in.off_partials);
            f.out = reinterpret_cast<qpe::Scalars*>(ws + in.off_scalars);
            f.count = part_count[i];
            f.nmeas = in.nmeas;
            bm.fin.push_back(f);
          }
          ++nargs;
        }
        LL.nitems = (int)bm.items.size() - LL.item_off;
        if (LL.nitems > 0) {
          int occ = 1;
          if (nsm > 0)
            occ = c64 ? qpe::level_grouped_occupancy<float2>(logd, LL.mode)
                      : qpe::level_grouped_occupancy<double2>(logd, LL.mode);
          LL.grid = std::min<int64_t>(LL.nitems, (int64_t)std::max(nsm, 1) * occ);
          bm.launches.push_back(LL);
        }
      }
    }
  }
  // plain instances: row 0, the doubling rounds, the QFT^-1 passes, the
  // histogram, the readout, each one grouped launch across the instances
  {
    std::vector<int> pl = bm.plain;
    for (int i : pl) bm.maxn_plain = std::max(bm.maxn_plain, p->inst[i].nmeas);
    auto build_plain = [&](auto tag) {
      using C = decltype(tag);
      for (int i : pl) {
        const Instance& in = p->inst[i];
        qpe::InitItem<C> it{};
        it.S = reinterpret_cast<C*>(ws + in.off_state);
        it.psi = reinterpret_cast<const double2*>(ws + in.off_psi);
        it.scale = 1.0 / std::sqrt(std::ldexp(1.0, in.nmeas));
        it.d = (int)in.d;
        push_bytes(bm.init_items, &it, sizeof(it));
        ++bm.ninit;
      }
      // level j of an instance runs on the tensor cores once it fills 128-row
      // tiles and 128-column tiles (2d >= 128), on the CUDA cores otherwise;
      // FP64 with QPE_FLAG_LEVEL_TC: as exact digit products for d >= 256
      auto on_tc = [&](const Instance& in, int j) {
        return is_tc(p->prec) && (int64_t(1) << j) >= 128 && in.d >= 64;
      };
      auto on_oz = [&](const Instance& in, int j) { return in.oz_gates && (int64_t(1) << j) >= 128; };
      for (int j = 0; j < bm.maxn_plain; ++j) {
        {
          // the instances' row digits share one buffer per level (its largest
          // total sizes the buffer)
          qpe::GateRound G{};
          G.j = j;
          G.p_off = (int)bm.gate_p.size();
          G.r_off = (int)bm.gate_r.size();
          G.g_off = (int)bm.gate_g.size();
          size_t bytes = 0;
          for (int i : pl) {
            const Instance& in = p->inst[i];
            if (in.nmeas <= j || !on_oz(in, j)) continue;
            qpe::OzItem pit{}, git{};
            qpe::RowSliceItem rit{};
            char* rowbuf = ws ? ws + bm.off_gatebuf + bytes : nullptr;
            if (!qpe::oz_gate_items(in, ws, j, rowbuf, &pit, &rit, &git)) throw std::runtime_error("tensor map");
            pit.sb0 = G.sblocks;
            pit.e0 = G.elems;
            G.sblocks += 2 * in.d;
            G.elems += in.d * in.d;
            rit.tile0 = G.rows;
            G.rows += int64_t(1) << j;
            git.tile0 = G.tiles;
            G.tiles += qpe::oz_gate_tiles(in, j);
            bytes += qpe::oz_gate_round_bytes(in, j);
            bm.gate_p.push_back(pit);
            bm.gate_r.push_back(rit);
            bm.gate_g.push_back(git);
          }
          G.p_n = (int)bm.gate_p.size() - G.p_off;
          G.r_n = (int)bm.gate_r.size() - G.r_off;
          G.g_n = (int)bm.gate_g.size() - G.g_off;
          if (G.g_n > 0) bm.gate_rounds.push_back(G);
          bm.gate_buf_bytes = std::max(bm.gate_buf_bytes, bytes);
        }
        {
          qpe::TcRound T{};
          T.j = j;
          T.item_off = (int)bm.tc_split.size();
          for (int i : pl) {
            const Instance& in = p->inst[i];
            if (in.nmeas <= j || !on_tc(in, j)) continue;
            qpe::TcSplitItem sp{};
            qpe::TcGemmItem gm{};
            if (!qpe::tc_level_items(in, ws, p->prec, j, &sp, &gm)) throw std::runtime_error("tensor map");
            sp.row0 = sp.tile0 = T.rows;
            sp.e0 = T.elems;
            gm.tile0 = T.tiles;
            T.rows += sp.rows;
            T.elems += (2 * in.d) * (2 * in.d);
            T.tiles += qpe::tc_level_tiles(in, j);
            bm.tc_split.push_back(sp);
            bm.tc_gemm.push_back(gm);
          }
          T.nitems = (int)bm.tc_split.size() - T.item_off;
          if (T.nitems > 0) bm.tc_rounds.push_back(T);
        }
        for (int dclass : {2, 4, 8, 16, 32, 64}) {
          qpe::DblRound R{};
          R.j = j;
          R.dclass = dclass;
          R.item_off = (int)(bm.dbl_items.size() / sizeof(qpe::DblItem<C>));
          int64_t tiles = 0;
          for (int i : pl) {
            const Instance& in = p->inst[i];
            if (in.nmeas <= j || on_tc(in, j) || on_oz(in, j) || std::min<int64_t>(in.d, 64) != dclass) continue;
            int BM = 0, BN = 0;
            qpe::doubling_tile((int)in.d, &BM, &BN);
            qpe::DblItem<C> it{};
            it.S = reinterpret_cast<C*>(ws + in.off_state);
            it.P = reinterpret_cast<const C*>(ws + (c64 ? in.off_pow32 : in.off_pow64)) + (int64_t)j * in.d * in.d;
            it.M = int64_t(1) << j;
            it.d = (int)in.d;
            it.tile0 = tiles;
            tiles += ((it.M + BM - 1) / BM) * (in.d / BN);
            push_bytes(bm.dbl_items, &it, sizeof(it));
          }
          R.nitems = (int)(bm.dbl_items.size() / sizeof(qpe::DblItem<C>)) - R.item_off;
          R.tiles = tiles;
          if (R.nitems > 0) bm.dbl_rounds.push_back(R);
        }
      }
      int maxp = 0;
      for (int i : pl) maxp = std::max(maxp, p->inst[i].fft.passes);
      for (int pass = 0; pass < maxp; ++pass) {
        qpe::FftRound R{};
        R.item_off = (int)(bm.fft_items.size() / sizeof(qpe::FftItem<C>));
        int64_t blocks = 0;
        size_t smem = 0;
        for (int i : pl) {
          const Instance& in = p->inst[i];
          if (in.fft.passes <= pass) continue;
          qpe::FftItem<C> it{};
          int64_t nb = 0;
          size_t sm = 0;
          it.a = qpe::fft_pass_args(in, pass, &nb, &sm, sizeof(C));
          it.X = reinterpret_cast<C*>(ws + in.off_state);
          it.lo = reinterpret_cast<const C*>(ws + (c64 ? in.off_tw_lo32 : in.off_tw_lo64));
          it.hi = reinterpret_cast<const C*>(ws + (c64 ? in.off_tw_hi32 : in.off_tw_hi64));
          it.tile0 = blocks;
          blocks += nb;
          smem = std::max(smem, sm);
          push_bytes(bm.fft_items, &it, sizeof(it));
        }
        R.nitems = (int)(bm.fft_items.size() / sizeof(qpe::FftItem<C>)) - R.item_off;
        R.blocks = blocks;
        R.smem = smem;
        if (R.nitems > 0) bm.fft_rounds.push_back(R);
      }
      for (int i : pl) {
        const Instance& in = p->inst[i];
        qpe::RedItem<C> it{};
        it.X = reinterpret_cast<const C*>(ws + in.off_state);
        it.hist = reinterpret_cast<double*>(ws + in.off_hist);
        it.parts = reinterpret_cast<qpe::Partial*>(ws + in.off_partials);
        it.N = in.N;
        it.logd = in.nmat;
        it.n = in.nmeas;
        it.g = qpe::fft_digits(in.fft);
        it.nblk = qpe::reduce_blocks(in);
        it.tile0 = bm.red_blocks;
        bm.red_blocks += it.nblk;
        push_bytes(bm.red_items, &it, sizeof(it));
        ++bm.nred;
        qpe::FinItem f{};
        f.parts = it.parts;
        f.out = reinterpret_cast<qpe::Scalars*>(ws + in.off_scalars);
        f.count = (int)it.nblk;
        f.nmeas = in.nmeas;
        bm.fin_plain.push_back(f);
      }
    };
    if (c64)
      build_plain(float2{});
    else
      build_plain(double2{});
  }
}

// Workspace offsets of the uploaded lists, after the instances' regions.
size_t place_batch_meta(qpe::BatchMeta& bm, size_t off) {
  auto take = [&](size_t bytes) {
    const size_t o = align_up(off);
    off = align_up(o + std::max<size_t>(bytes, 16));
    return o;
  };
  bm.off_sq = take(bm.sq.size() * sizeof(qpe::SqItem));
  bm.off_conv = take(bm.conv.size() * sizeof(qpe::SqItem));
  bm.off_tab = take(bm.tab_items.size());
  bm.off_seed = take(bm.seed_items.size());
  bm.off_args = take(bm.level_args.size());
  bm.off_items = take(bm.items.size() * sizeof(qpe::GroupItem));
  bm.off_fin = take(bm.fin.size() * sizeof(qpe::FinItem));
  bm.off_init = take(bm.init_items.size());
  bm.off_dbl = take(bm.dbl_items.size());
  bm.off_fft = take(bm.fft_items.size());
  bm.off_red = take(bm.red_items.size());
  bm.off_finp = take(bm.fin_plain.size() * sizeof(qpe::FinItem));
  bm.off_oz = take(bm.oz_items.size() * sizeof(qpe::OzItem));
  bm.off_tcsp = take(bm.tc_split.size() * sizeof(qpe::TcSplitItem));
  bm.off_tcgm = take(bm.tc_gemm.size() * sizeof(qpe::TcGemmItem));
  bm.off_gate_p = take(bm.gate_p.size() * sizeof(qpe::OzItem));
  bm.off_gate_g = take(bm.gate_g.size() * sizeof(qpe::OzItem));
  bm.off_gate_r = take(bm.gate_r.size() * sizeof(qpe::RowSliceItem));
  bm.off_gatebuf = take(bm.gate_buf_bytes);
  return off;
}

qpe_status upload_batch_meta(qpe_plan_t p) {
  qpe::BatchMeta& bm = p->bm;
  struct Blk {
    size_t off;
    const void* src;
    size_t n;
  } blks[] = {{bm.off_sq, bm.sq.data(), bm.sq.size() * sizeof(qpe::SqItem)},
              {bm.off_conv, bm.conv.data(), bm.conv.size() * sizeof(qpe::SqItem)},
              {bm.off_tab, bm.tab_items.data(), bm.tab_items.size()},
              {bm.off_seed, bm.seed_items.data(), bm.seed_items.size()},
              {bm.off_args, bm.level_args.data(), bm.level_args.size()},
              {bm.off_items, bm.items.data(), bm.items.size() * sizeof(qpe::GroupItem)},
              {bm.off_fin, bm.fin.data(), bm.fin.size() * sizeof(qpe::FinItem)},
              {bm.off_init, bm.init_items.data(), bm.init_items.size()},
              {bm.off_dbl, bm.dbl_items.data(), bm.dbl_items.size()},
              {bm.off_fft, bm.fft_items.data(), bm.fft_items.size()},
              {bm.off_red, bm.red_items.data(), bm.red_items.size()},
              {bm.off_finp, bm.fin_plain.data(), bm.fin_plain.size() * sizeof(qpe::FinItem)},
              {bm.off_oz, bm.oz_items.data(), bm.oz_items.size() * sizeof(qpe::OzItem)},
              {bm.off_gate_p, bm.gate_p.data(), bm.gate_p.size() * sizeof(qpe::OzItem)},
              {bm.off_gate_g, bm.gate_g.data(), bm.gate_g.size() * sizeof(qpe::OzItem)},
              {bm.off_gate_r, bm.gate_r.data(), bm.gate_r.size() * sizeof(qpe::RowSliceItem)},
              {bm.off_tcsp, bm.tc_split.data(), bm.tc_split.size() * sizeof(qpe::TcSplitItem)},
              {bm.off_tcgm, bm.tc_gemm.data(), bm.tc_gemm.size() * sizeof(qpe::TcGemmItem)}};
  for (const Blk& b : blks) {
    if (!b.n) continue;
    cudaError_t e = cudaMemcpyAsync(p->ws + b.off, b.src, b.n, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "upload of batched work lists");
  }
  return QPE_OK;
}

// One whole batched run: grouped squaring steps, grouped fused levels, then
// the plain schedule instance by instance.
// CTAs of the grouped squaring launch of step k with the given tile variant
int64_t square_tiles(const qpe::BatchMeta& bm, int k, int variant) {
  return variant == 1 ? bm.sq_tiles16[k] : (variant == 2 ? bm.sq_tiles32[k] : bm.sq_tiles[k]);
}

// The squaring tile autotuner of batched plans: every variant runs the plan's
// own first squaring step (all instances with Nmeas > 1, at their own d) once
// to warm up and twice under CUDA events; the fastest is kept. It runs at bind
// time, before any input is loaded: the arithmetic does not depend on the
// values, and the outputs it writes are recomputed by every qpe_run.
qpe_status autotune_square(qpe_plan_t p) {
  const qpe::BatchMeta& bm = p->bm;
  if (bm.maxn < 2 || bm.sq_count[1] == 0) return QPE_OK;
  const qpe::SqItem* items = reinterpret_cast<const qpe::SqItem*>(p->ws + bm.off_sq) + bm.sq_begin[1];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int best = 0;
  for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
    if (qpe::launch_square_grouped(items, bm.sq_count[1], square_tiles(bm, 1, v), v, p->stream) < 0) {
      e = cudaGetLastError();
      break;
    }
    e = cudaEventRecord(e0, p->stream);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r)
      if (qpe::launch_square_grouped(items, bm.sq_count[1], square_tiles(bm, 1, v), v, p->stream) < 0)
        e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    p->tune_ms[v] = ms / 2;
    if (e == cudaSuccess && p->tune_ms[v] < p->tune_ms[best]) best = v;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(p, e, "squaring autotune");
  p->sq_variant = best;
  return QPE_OK;
}

qpe_status enqueue_batched(qpe_plan_t p, int64_t* launches) {
  qpe::BatchMeta& bm = p->bm;
  const bool c64 = is_c64(p->prec);
  char* ws = p->ws;
  int64_t n = 0;
  auto chk = [&](int r) {
    if (r < 0) return false;
    n += r;
    return true;
  };
  for (Instance& in : p->inst)
    if (!in.loaded) return fail(p, QPE_ERR_STATE, "qpe_load has not been called for every instance");
  // QPE_FLAG_TIMING: events at the start, after the squarings, after the gates
  // (fused levels whole, plain doubling levels), after the plain QFT^-1 passes
  // and at the end (plain histograms and every readout)
  const bool timing = (p->flags & QPE_FLAG_TIMING) && p->ev[0];
  p->timed_run = timing;
  auto mark = [&](int i) { return !timing || record_event(p->ev[i], p->stream) == cudaSuccess; };
  if (!mark(0)) return cuda_fail(p, cudaGetLastError(), "cudaEventRecord");
  // error words of the instances whose kernels can set them, cleared per run
  for (Instance& in : p->inst)
    if (in.oz_square || in.oz_gates || (is_tc(p->prec) && !in.fused)) {
      cudaError_t e = cudaMemsetAsync(ws + in.off_err, 0, sizeof(int), p->stream);
      if (e != cudaSuccess) return cuda_fail(p, e, "error word reset");
    }
  if (p->flags & QPE_FLAG_CHECK_UNITARY) {
    for (Instance& in : p->inst) {
      cudaError_t e = cudaMemsetAsync(ws + in.off_err, 0, sizeof(int), p->stream);
      if (e != cudaSuccess) return cuda_fail(p, e, "error word reset");
      if (!chk(qpe::launch_check_unitary(in, ws, p->stream))) return cuda_fail(p, cudaGetLastError(), "unitarity check");
    }
  }
  for (int k = 1; k < bm.maxn; ++k) {
    if (!chk(qpe::launch_square_grouped(reinterpret_cast<const qpe::SqItem*>(ws + bm.off_sq) + bm.sq_begin[k],
                                        bm.sq_count[k], square_tiles(bm, k, p->sq_variant), p->sq_variant,
                                        p->stream)))
      return cuda_fail(p, cudaGetLastError(), "grouped squaring");
    for (const qpe::OzStep& O : bm.oz_steps)
      if (O.k == k && !chk(qpe::launch_square_oz_grouped(reinterpret_cast<const qpe::OzItem*>(ws + bm.off_oz) +
                                                             O.item_off,
                                                         O.nitems, O.sblocks, O.elems, O.tiles, p->stream)))
        return cuda_fail(p, cudaGetLastError(), "tensor-core squaring");
  }
  if (!chk(qpe::launch_convert_grouped(reinterpret_cast<const qpe::SqItem*>(ws + bm.off_conv), (int)bm.conv.size(),
                                       bm.conv_tiles, p->stream)))
    return cuda_fail(p, cudaGetLastError(), "grouped conversion");
  if (!mark(1)) return cuda_fail(p, cudaGetLastError(), "cudaEventRecord");
  if (!bm.fused.empty()) {
    int r;
    if (c64)
      r = qpe::launch_table_grouped<float2>(reinterpret_cast<const qpe::TabItem<float2>*>(ws + bm.off_tab), bm.ntab,
                                            bm.tab_blocks, bm.max_logd, p->stream);
    else
      r = qpe::launch_table_grouped<double2>(reinterpret_cast<const qpe::TabItem<double2>*>(ws + bm.off_tab),
                                             bm.ntab, bm.tab_blocks, bm.max_logd, p->stream);
    if (!chk(r)) return cuda_fail(p, cudaGetLastError(), "grouped tables");
    r = c64 ? qpe::launch_seed_grouped<float2>(reinterpret_cast<const qpe::SeedItem<float2>*>(ws + bm.off_seed),
                                               bm.nseed, p->stream)
            : qpe::launch_seed_grouped<double2>(reinterpret_cast<const qpe::SeedItem<double2>*>(ws + bm.off_seed),
                                                bm.nseed, p->stream);
    if (!chk(r)) return cuda_fail(p, cudaGetLastError(), "grouped seeds");
    const qpe::GroupItem* items = reinterpret_cast<const qpe::GroupItem*>(ws + bm.off_items);
    for (const qpe::LevelLaunch& L : bm.launches) {
      if (c64)
        r = qpe::launch_level_grouped<float2>(
            L, reinterpret_cast<const qpe::LevelArgs<float2>*>(ws + bm.off_args) + L.arg_off, items + L.item_off,
            p->stream);
      else
        r = qpe::launch_level_grouped<double2>(
            L, reinterpret_cast<const qpe::LevelArgs<double2>*>(ws + bm.off_args) + L.arg_off, items + L.item_off,
            p->stream);
      if (!chk(r)) return cuda_fail(p, cudaGetLastError(), "grouped level");
    }
    if (!chk(qpe::launch_finalize_grouped(reinterpret_cast<const qpe::FinItem*>(ws + bm.off_fin), (int)bm.fin.size(),
                                          p->stream)))
      return cuda_fail(p, cudaGetLastError(), "grouped finalize");
    for (int i : bm.fused) {
      Instance& in = p->inst[i];
      in.powers_done = true;
      in.state_stage = QPE_STAGE_REDUCE;
      in.state_natural = true;
      in.state_valid = in.keep_state;
    }
  }
  if (!bm.plain.empty()) {
    // the plain instances step by step, each step one grouped launch
    auto run_plain = [&](auto tag) -> bool {
      using C = decltype(tag);
      if (!chk(qpe::launch_init_grouped<C>(reinterpret_cast<const qpe::InitItem<C>*>(ws + bm.off_init), bm.ninit,
                                           p->stream)))
        return false;
      for (int j = 0; j < bm.maxn_plain; ++j) {
        for (const qpe::DblRound& R : bm.dbl_rounds)
          if (R.j == j &&
              !chk(qpe::launch_doubling_grouped<C>(reinterpret_cast<const qpe::DblItem<C>*>(ws + bm.off_dbl) + R.item_off,
                                                   R.nitems, R.tiles, R.dclass, p->stream)))
            return false;
        for (const qpe::GateRound& G : bm.gate_rounds)
          if (G.j == j &&
              !chk(qpe::launch_oz_gate_grouped(reinterpret_cast<const qpe::OzItem*>(ws + bm.off_gate_p) + G.p_off,
                                               reinterpret_cast<const qpe::RowSliceItem*>(ws + bm.off_gate_r) + G.r_off,
                                               reinterpret_cast<const qpe::OzItem*>(ws + bm.off_gate_g) + G.g_off, G,
                                               p->stream)))
            return false;
        for (const qpe::TcRound& T : bm.tc_rounds)
          if (T.j == j &&
              !chk(qpe::launch_tc_level_grouped(
                  p->prec, reinterpret_cast<const qpe::TcSplitItem*>(ws + bm.off_tcsp) + T.item_off,
                  reinterpret_cast<const qpe::TcGemmItem*>(ws + bm.off_tcgm) + T.item_off, T.nitems, T.rows, T.elems,
                  T.tiles, p->stream)))
            return false;
      }
      if (!mark(2)) return false;
      for (const qpe::FftRound& R : bm.fft_rounds)
        if (!chk(qpe::launch_fft_grouped<C>(reinterpret_cast<const qpe::FftItem<C>*>(ws + bm.off_fft) + R.item_off,
                                            R.nitems, R.blocks, R.smem, p->stream)))
          return false;
      if (!mark(3)) return false;
      if (!chk(qpe::launch_reduce_grouped<C>(reinterpret_cast<const qpe::RedItem<C>*>(ws + bm.off_red), bm.nred,
                                             bm.red_blocks, p->stream)))
        return false;
      return chk(qpe::launch_finalize_grouped(reinterpret_cast<const qpe::FinItem*>(ws + bm.off_finp),
                                              (int)bm.fin_plain.size(), p->stream));
    };
    if (!(c64 ? run_plain(float2{}) : run_plain(double2{}))) return cuda_fail(p, cudaGetLastError(), "plain instances");
    for (int i : bm.plain) {
      Instance& in = p->inst[i];
      in.powers_done = true;
      in.state_stage = QPE_STAGE_REDUCE;
      in.state_natural = false;
      in.state_valid = true;
    }
  } else if (!mark(2) || !mark(3)) {
    return cuda_fail(p, cudaGetLastError(), "cudaEventRecord");
  }
  if (!mark(4)) return cuda_fail(p, cudaGetLastError(), "cudaEventRecord");
  *launches = n;
  return QPE_OK;
}

}  // namespace

extern "C" {

const char* qpe_status_string(qpe_status s) {
  switch (s) {
    case QPE_OK: return "QPE_OK";
    case QPE_ERR_ARG: return "QPE_ERR_ARG: invalid argument";
    case QPE_ERR_SHAPE: return "QPE_ERR_SHAPE: shape does not match the plan";
    case QPE_ERR_WORKSPACE: return "QPE_ERR_WORKSPACE: workspace missing, misaligned or too small";
    case QPE_ERR_UNSUPPORTED: return "QPE_ERR_UNSUPPORTED: combination not implemented";
    case QPE_ERR_CUDA: return "QPE_ERR_CUDA: CUDA runtime error";
    case QPE_ERR_TIMEOUT: return "QPE_ERR_TIMEOUT: bounded device wait expired";
    case QPE_ERR_NUMERIC: return "QPE_ERR_NUMERIC: non-finite histogram";
    case QPE_ERR_STATE: return "QPE_ERR_STATE: call out of order";
  }
  return "QPE_ERR_?: unknown status";
}

const char* qpe_last_error(qpe_plan_t p) { return p ? p->last_error.c_str() : "null plan"; }

qpe_status qpe_plan(const qpe_plan_desc* desc, size_t* workspace_bytes, qpe_plan_t* out) {
  if (!desc || !workspace_bytes || !out) return QPE_ERR_ARG;
  *out = nullptr;
  const qpe_status st = check_desc(desc);
  if (st != QPE_OK) return st;
  qpe_plan_s* p = new (std::nothrow) qpe_plan_s();
  if (!p) return QPE_ERR_ARG;
  p->prec = desc->prec;
  p->flags = desc->flags;
  Instance in{};
  in.nmat = desc->nmat;
  in.nmeas = desc->nmeas;
  in.d = int64_t(1) << desc->nmat;
  in.N = int64_t(1) << desc->nmeas;
  p->ws_bytes = layout_instance(in, p->prec, p->flags, 0);
  p->inst.push_back(in);
  *workspace_bytes = p->ws_bytes;
  *out = p;
  return QPE_OK;
}

qpe_status qpe_plan_shard(const qpe_plan_desc* desc, int32_t rank, int32_t world, size_t* workspace_bytes,
                          qpe_plan_t* out) {
  if (!desc || !workspace_bytes || !out) return QPE_ERR_ARG;
  *out = nullptr;
  if (world < 1 || world > 1024 || (world & (world - 1)) != 0 || rank < 0 || rank >= world) return QPE_ERR_ARG;
  const qpe_status st = check_desc(desc);
  if (st != QPE_OK) return st;
  int sh = 0;
  while ((1 << sh) < world) ++sh;
  if (desc->flags & (QPE_FLAG_GATE_SWEEP | QPE_FLAG_REPEAT_U)) return QPE_ERR_UNSUPPORTED;
  const bool plain = desc->nmat > QPE_MAX_FUSED_NMAT || (desc->flags & QPE_FLAG_PLAIN) ||
                     (is_tc(desc->prec) && desc->nmat > 4);
  if (plain) {
    // rows m = rank (mod world), one exchange of N / world^2 rows per pair of
    // ranks: needs N >= world^2; the final state stays distributed
    if (desc->nmeas < 2 * sh || (desc->flags & QPE_FLAG_KEEP_STATE)) return QPE_ERR_UNSUPPORTED;
  } else {
    // the fused form partitions the outcomes; the top level must have at
    // least `world` pencils
    const std::vector<qpe::Level> lv = qpe::make_levels(desc->nmeas, desc->nmat, elem_size(desc->prec), 0);
    if (lv.empty() || lv[0].logna < sh) return QPE_ERR_UNSUPPORTED;
  }
  qpe_plan_s* p = new (std::nothrow) qpe_plan_s();
  if (!p) return QPE_ERR_ARG;
  p->prec = desc->prec;
  p->flags = desc->flags;
  Instance in{};
  in.nmat = desc->nmat;
  in.nmeas = desc->nmeas;
  in.d = int64_t(1) << desc->nmat;
  in.N = int64_t(1) << desc->nmeas;
  in.shard_log = sh;
  in.shard_rank = rank;
  p->ws_bytes = layout_instance(in, p->prec, p->flags, 0);
  p->inst.push_back(in);
  *workspace_bytes = p->ws_bytes;
  *out = p;
  return QPE_OK;
}

qpe_status qpe_shard_readout(qpe_plan_t p, qpe_shard_readout_t* out) {
  if (!p || !out) return fail(p, QPE_ERR_ARG, "null pointer");
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  if (p->batched) return fail(p, QPE_ERR_UNSUPPORTED, "batched plans have no shard readout");
  Instance& in = p->inst[0];
  if (in.state_stage != QPE_STAGE_REDUCE) return fail(p, QPE_ERR_STATE, "REDUCE has not run");
  qpe::Scalars s;
  int derr = 0;
  cudaError_t e = cudaMemcpyAsync(&s, p->ws + in.off_scalars, sizeof(s), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&derr, p->ws + in.off_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "qpe_shard_readout copy");
  if (derr) return fail(p, (qpe_status)derr, err_word_message(derr));
  out->argmax = s.argmax;
  out->p_argmax = s.best;
  out->phase_mean_part = s.phase_mean;
  out->total = s.total;
  out->nmeas = in.nmeas;
  out->rank = in.shard_rank;
  if (s.err) return fail(p, (qpe_status)s.err, "device flagged a non-finite histogram");
  return QPE_OK;
}

qpe_status qpe_shard_buffers(qpe_plan_t p, void** send, void** recv, size_t* bytes_per_peer) {
  if (!p || !send || !recv || !bytes_per_peer) return fail(p, QPE_ERR_ARG, "null pointer");
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  if (p->batched) return fail(p, QPE_ERR_UNSUPPORTED, "batched plans are not sharded");
  const Instance& in = p->inst[0];
  *send = in.shard_plain ? p->ws + in.off_send : nullptr;
  *recv = in.shard_plain ? p->ws + in.off_recv : nullptr;
  *bytes_per_peer = in.shard_plain ? in.state_bytes >> in.shard_log : 0;
  return QPE_OK;
}

qpe_status qpe_shard_finish(qpe_plan_t p) {
  if (!p) return QPE_ERR_ARG;
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  if (p->batched) return fail(p, QPE_ERR_UNSUPPORTED, "batched plans are not sharded");
  Instance& in = p->inst[0];
  if (!in.shard_plain) {
    if (in.state_stage != QPE_STAGE_REDUCE) return fail(p, QPE_ERR_STATE, "qpe_run has not run");
    return QPE_OK;  // the fused form needs no exchange
  }
  if (in.state_stage != qpe::kStageExchange) return fail(p, QPE_ERR_STATE, "qpe_run (and the exchange) first");
  int blocks = 0;
  const int r = is_c64(p->prec) ? qpe::launch_shard_combine<float2>(in, p->ws, p->stream, &blocks)
                                : qpe::launch_shard_combine<double2>(in, p->ws, p->stream, &blocks);
  if (r < 0 || qpe::launch_finalize(in, p->ws, blocks, p->stream) < 0)
    return cuda_fail(p, cudaGetLastError(), "shard combine");
  in.state_stage = QPE_STAGE_REDUCE;
  return QPE_OK;
}

qpe_status qpe_host_alloc(size_t bytes, void** ptr) {
  if (!ptr) return QPE_ERR_ARG;
  *ptr = nullptr;
  if (bytes == 0) return QPE_ERR_ARG;
  if (cudaHostAlloc(ptr, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return QPE_ERR_CUDA;
  }
  return QPE_OK;
}

qpe_status qpe_host_free(void* ptr) {
  if (!ptr) return QPE_OK;
  return cudaFreeHost(ptr) == cudaSuccess ? QPE_OK : QPE_ERR_CUDA;
}

qpe_status qpe_merge_shard_readouts(const qpe_shard_readout_t* parts, int32_t world, qpe_readout_t* out) {
  if (!parts || !out || world < 1) return QPE_ERR_ARG;
  int64_t am = -1;
  double best = -1.0, mean = 0.0, total = 0.0;
  for (int32_t i = 0; i < world; ++i) {
    const qpe_shard_readout_t& q = parts[i];
    if (q.nmeas != parts[0].nmeas) return QPE_ERR_SHAPE;
    if (!std::isfinite(q.p_argmax) || !std::isfinite(q.phase_mean_part) || !std::isfinite(q.total))
      return QPE_ERR_NUMERIC;
    // the plan path's rule: larger probability, then lower outcome on a tie
    if (am < 0 || q.p_argmax > best || (q.p_argmax == best && q.argmax < am)) {
      best = q.p_argmax;
      am = q.argmax;
    }
    mean += q.phase_mean_part;
    total += q.total;
  }
  out->argmax = am;
  out->phase_argmax = std::ldexp((double)am, -parts[0].nmeas);
  out->phase_mean = mean;
  out->total = total;
  return QPE_OK;
}

qpe_status qpe_plan_batched(const qpe_plan_desc* descs, int32_t count, size_t* workspace_bytes, qpe_plan_t* out) {
  if (!descs || !workspace_bytes || !out || count < 1) return QPE_ERR_ARG;
  *out = nullptr;
  for (int32_t i = 0; i < count; ++i) {
    const qpe_status st = check_desc(&descs[i], true);
    if (st != QPE_OK) return st;
    if (descs[i].prec != descs[0].prec || descs[i].flags != descs[0].flags) return QPE_ERR_ARG;
  }
  if (descs[0].flags & QPE_FLAG_GATE_SWEEP) return QPE_ERR_UNSUPPORTED;
  qpe_plan_s* p = new (std::nothrow) qpe_plan_s();
  if (!p) return QPE_ERR_ARG;
  p->prec = descs[0].prec;
  p->flags = descs[0].flags;
  p->batched = true;
  size_t off = 0;
  try {
    for (int32_t i = 0; i < count; ++i) {
      Instance in{};
      in.nmat = descs[i].nmat;
      in.nmeas = descs[i].nmeas;
      in.d = int64_t(1) << in.nmat;
      in.N = int64_t(1) << in.nmeas;
      off = layout_instance(in, p->prec, p->flags, off, true);
      p->inst.push_back(in);
    }
    build_batch_meta(p, nullptr, 0);
  } catch (...) {
    delete p;
    return QPE_ERR_ARG;
  }
  p->ws_bytes = place_batch_meta(p->bm, off);
  *workspace_bytes = p->ws_bytes;
  *out = p;
  return QPE_OK;
}

qpe_status qpe_bind(qpe_plan_t p, void* d_ws, size_t bytes, void* stream) {
  if (!p) return QPE_ERR_ARG;
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) % kAlign) != 0 || bytes < p->ws_bytes)
    return fail(p, QPE_ERR_WORKSPACE, "workspace must be non-null, 256-byte aligned and >= qpe_plan's size");
  if ((p->flags & QPE_FLAG_GRAPH) && !stream)
    return fail(p, QPE_ERR_ARG, "QPE_FLAG_GRAPH needs a non-default stream");
  cudaError_t e = qpe::configure_kernels();
  if (e == cudaSuccess) e = qpe::configure_batched_kernels();
  if (e == cudaSuccess && (is_tc(p->prec) || (p->flags & (QPE_FLAG_SQUARE_TC | QPE_FLAG_LEVEL_TC))))
    e = qpe::configure_tc_kernels();
  if (e == cudaSuccess && (p->flags & QPE_FLAG_LEVEL_TC)) e = qpe::configure_oz_top_kernel();
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute");
  {
    const char* v = getenv("QPE_PDL");
    qpe::g_pdl_enabled = !(v && v[0] == '0');
  }
  if (p->graph_exec) {
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  p->ws = static_cast<char*>(d_ws);
  p->stream = static_cast<cudaStream_t>(stream);
  if ((p->flags & QPE_FLAG_TIMING) && !p->ev[0]) {
    for (cudaEvent_t& ev : p->ev) {
      e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventCreate");
    }
  }
  int nsm = 0, dev = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(p, e, "device query");
  for (Instance& in : p->inst) {
    in.nsm = nsm;
    if (!in.levels.empty()) {
      int occ = 1;
      for (const qpe::Level& L : in.levels) {
        const int o = is_c64(p->prec) ? qpe::level_occupancy<float2>(in.nmat, L.r)
                                      : qpe::level_occupancy<double2>(in.nmat, L.r);
        occ = std::max(occ, o);
      }
      in.level_grid = (int64_t)nsm * occ;
    }
    in.loaded = false;
    in.powers_done = false;
    in.state_stage = 0;
    e = cudaMemsetAsync(p->ws + in.off_err, 0, sizeof(int), p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "error word reset");
    if (qpe::launch_twiddles(in, p->ws, p->stream) < 0) return cuda_fail(p, cudaGetLastError(), "twiddle tables");
  }
  if (p->batched) {
    try {
      build_batch_meta(p, p->ws, nsm);
    } catch (...) {
      return fail(p, QPE_ERR_CUDA, "batched work lists: tensor map encoding failed");
    }
    qpe_status st = upload_batch_meta(p);
    if (st != QPE_OK) return st;
    const char* forced = getenv("QPE_SQUARE_TILE");  // 8, 16 or 32: skip the autotuner
    if (forced && forced[0]) {
      const int t = atoi(forced);
      p->sq_variant = t == 16 ? 1 : (t == 32 ? 2 : 0);
    } else if (p->flags & QPE_FLAG_AUTOTUNE) {
      st = autotune_square(p);
      if (st != QPE_OK) return st;
    }
  }
  p->bound = true;
  return QPE_OK;
}

qpe_status qpe_load(qpe_plan_t p, int32_t instance, const void* U, const void* psi, int32_t nmat, int32_t nmeas,
                    int32_t ptr_is_device) {
  if (!p || !U || !psi) return fail(p, QPE_ERR_ARG, "null pointer");
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  Instance* in;
  qpe_status st = get_instance(p, instance, &in);
  if (st != QPE_OK) return st;
  if (nmat != in->nmat || nmeas != in->nmeas) return fail(p, QPE_ERR_SHAPE, "nmat/nmeas differ from the plan");
  cudaError_t e = cudaMemcpyAsync(p->ws + in->off_pow64, U, (size_t)in->d * in->d * 16, kind_to_device(ptr_is_device),
                                  p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->ws + in->off_psi, psi, (size_t)in->d * 16, kind_to_device(ptr_is_device), p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "qpe_load copy");
  in->loaded = true;
  in->powers_done = false;
  in->state_stage = 0;
  return QPE_OK;
}

qpe_status qpe_run_stages(qpe_plan_t p, int32_t first, int32_t last) {
  if (!p) return QPE_ERR_ARG;
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  if (first < QPE_STAGE_POWERS || last > QPE_STAGE_REDUCE || first > last)
    return fail(p, QPE_ERR_ARG, "stages must satisfy POWERS <= first <= last <= REDUCE");
  int64_t launches = 0;
  const qpe_status st = enqueue_stages(p, first, last, &launches);
  if (st == QPE_OK) p->last_launches = launches;
  return st;
}

qpe_status qpe_run(qpe_plan_t p) {
  if (!p) return QPE_ERR_ARG;
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  if (!(p->flags & QPE_FLAG_GRAPH)) return qpe_run_stages(p, QPE_STAGE_POWERS, QPE_STAGE_REDUCE);
  for (Instance& in : p->inst)
    if (!in.loaded) return fail(p, QPE_ERR_STATE, "qpe_load has not been called for every instance");
  if (!p->graph_exec) {
    cudaError_t e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaStreamBeginCapture");
    int64_t launches = 0;
    qpe_status st = enqueue_stages(p, QPE_STAGE_POWERS, QPE_STAGE_REDUCE, &launches);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(p->stream, &g);
    if (st != QPE_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&p->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p->graph_exec = nullptr;
      return cuda_fail(p, e, "cudaGraphInstantiate");
    }
    p->last_launches = launches;
  } else {
    // the captured graph replays the same stages; keep the host-side
    // stage bookkeeping in step with it
    for (Instance& in : p->inst) {
      in.powers_done = true;
      in.state_stage = in.shard_plain ? qpe::kStageExchange : QPE_STAGE_REDUCE;
    }
  }
  cudaError_t e = cudaGraphLaunch(p->graph_exec, p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaGraphLaunch");
  return QPE_OK;
}

qpe_status qpe_sync(qpe_plan_t p) {
  if (!p) return QPE_ERR_ARG;
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaStreamSynchronize");
  for (const Instance& in : p->inst) {
    if (!in.loaded) continue;
    int derr = 0;
    e = cudaMemcpy(&derr, p->ws + in.off_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p, e, "read error word");
    if (derr) return fail(p, (qpe_status)derr, err_word_message(derr));
    if (in.state_stage != QPE_STAGE_REDUCE) continue;
    qpe::Scalars s;
    e = cudaMemcpy(&s, p->ws + in.off_scalars, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p, e, "read readout scalars");
    if (s.err) return fail(p, (qpe_status)s.err, "device flagged a non-finite histogram");
  }
  return QPE_OK;
}

qpe_status qpe_probs(qpe_plan_t p, int32_t instance, double* probs, int64_t* argmax, double* phase_argmax,
                     double* phase_mean, int32_t ptr_is_device) {
  if (!p) return QPE_ERR_ARG;
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  Instance* in;
  qpe_status st = get_instance(p, instance, &in);
  if (st != QPE_OK) return st;
  if (in->state_stage != QPE_STAGE_REDUCE) return fail(p, QPE_ERR_STATE, "REDUCE has not run");
  cudaError_t e = cudaSuccess;
  if (probs && probs != in->host_hist)  // the host histogram buffer already holds the run's bins
    e = cudaMemcpyAsync(probs, p->ws + in->off_hist, (size_t)(in->N >> in->shard_log) * 8,
                        kind_from_device(ptr_is_device), p->stream);
  qpe::Scalars s;
  int derr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&s, p->ws + in->off_scalars, sizeof(s), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&derr, p->ws + in->off_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "qpe_probs copy");
  if (derr) return fail(p, (qpe_status)derr, err_word_message(derr));
  if (argmax) *argmax = s.argmax;
  if (phase_argmax) *phase_argmax = s.phase_argmax;
  if (phase_mean) *phase_mean = s.phase_mean;
  if (s.err) return fail(p, (qpe_status)s.err, "device flagged a non-finite histogram");
  return QPE_OK;
}

qpe_status qpe_state(qpe_plan_t p, int32_t instance, void* out, int32_t ptr_is_device) {
  if (!p || !out) return fail(p, QPE_ERR_ARG, "null pointer");
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  Instance* in;
  qpe_status st = get_instance(p, instance, &in);
  if (st != QPE_OK) return st;
  if (in->shard_plain) return fail(p, QPE_ERR_UNSUPPORTED, "a sharded plain plan's final state stays distributed");
  if (in->state_stage == 0) return fail(p, QPE_ERR_STATE, "no state computed yet");
  if (!in->state_valid)
    return fail(p, QPE_ERR_STATE, "the fused schedule keeps the final state only with QPE_FLAG_KEEP_STATE");
  const bool c64 = is_c64(p->prec);
  const bool permuted = !in->state_natural;
  cudaError_t e;
  if (!permuted) {
    e = cudaMemcpyAsync(out, p->ws + in->off_state, in->state_bytes, kind_from_device(ptr_is_device), p->stream);
    if (e == cudaSuccess && !ptr_is_device) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "qpe_state copy");
    return QPE_OK;
  }
  if (ptr_is_device) {
    const int r = c64 ? qpe::launch_unpermute<float2>(*in, p->ws, out, p->stream)
                      : qpe::launch_unpermute<double2>(*in, p->ws, out, p->stream);
    if (r < 0) return cuda_fail(p, cudaGetLastError(), "unpermute kernel");
    return QPE_OK;
  }
  // host output: copy position-ordered rows, reorder on the host
  std::vector<char> tmp;
  try {
    tmp.resize(in->state_bytes);
  } catch (...) {
    return fail(p, QPE_ERR_ARG, "host memory for the reordering copy");
  }
  e = cudaMemcpyAsync(tmp.data(), p->ws + in->off_state, in->state_bytes, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "qpe_state copy");
  const size_t row = (size_t)in->d * elem_size(p->prec);
  for (int64_t pos = 0; pos < in->N; ++pos) {
    const int64_t y = qpe::fft_position_to_y(in->fft, in->nmeas, pos);
    std::memcpy(static_cast<char*>(out) + (size_t)y * row, tmp.data() + (size_t)pos * row, row);
  }
  return QPE_OK;
}

qpe_status qpe_load_state(qpe_plan_t p, int32_t instance, const void* src, int32_t ptr_is_device) {
  if (!p || !src) return fail(p, QPE_ERR_ARG, "null pointer");
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  Instance* in;
  qpe_status st = get_instance(p, instance, &in);
  if (st != QPE_OK) return st;
  if (!in->has_state) return fail(p, QPE_ERR_STATE, "this fused plan has no state buffer; plan with QPE_FLAG_PLAIN");
  if (in->shard_plain) return fail(p, QPE_ERR_UNSUPPORTED, "sharded plans run whole");
  cudaError_t e =
      cudaMemcpyAsync(p->ws + in->off_state, src, in->state_bytes, kind_to_device(ptr_is_device), p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "qpe_load_state copy");
  in->loaded = true;
  in->state_stage = QPE_STAGE_SWEEP;
  in->state_natural = true;
  in->state_valid = true;
  return QPE_OK;
}

qpe_status qpe_powers(qpe_plan_t p, int32_t instance, int32_t k, void* out, int32_t ptr_is_device) {
  if (!p || !out) return fail(p, QPE_ERR_ARG, "null pointer");
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  Instance* in;
  qpe_status st = get_instance(p, instance, &in);
  if (st != QPE_OK) return st;
  if (k < 0 || k >= in->nmeas) return fail(p, QPE_ERR_ARG, "k out of range");
  if (!in->powers_done) return fail(p, QPE_ERR_STATE, "POWERS has not run");
  const size_t bytes = (size_t)in->d * in->d * 16;
  cudaError_t e = cudaMemcpyAsync(out, p->ws + in->off_pow64 + (size_t)k * bytes, bytes,
                                  kind_from_device(ptr_is_device), p->stream);
  if (e == cudaSuccess && !ptr_is_device) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "qpe_powers copy");
  return QPE_OK;
}

int64_t qpe_query(qpe_plan_t p, int32_t key) {
  if (!p || p->inst.empty()) return -1;
  switch (key) {
    case QPE_INFO_WORKSPACE_BYTES: return (int64_t)p->ws_bytes;
    case QPE_INFO_STATE_BYTES: return (int64_t)p->inst[0].state_bytes;
    case QPE_INFO_FFT_PASSES: return p->inst[0].fft.passes;
    case QPE_INFO_LAST_LAUNCHES: return p->last_launches;
    case QPE_INFO_INSTANCES: return (int64_t)p->inst.size();
    case QPE_INFO_SQUARE_TILE: return p->sq_variant == 1 ? 16 : (p->sq_variant == 2 ? 32 : 8);
    case QPE_INFO_LEVELS: return p->inst[0].fused ? (int64_t)p->inst[0].levels.size() : 0;
    case QPE_INFO_TOP_LEVEL_BITS: return p->inst[0].fused ? p->inst[0].levels[0].r : 0;
    case QPE_INFO_TC_TOP_LEVEL: return p->inst[0].tc_top ? 1 : 0;
  }
  return -1;
}

qpe_status qpe_stage_times(qpe_plan_t p, double* ms) {
  if (!p || !ms) return fail(p, QPE_ERR_ARG, "null pointer");
  if (!(p->flags & QPE_FLAG_TIMING) || !p->ev[0])
    return fail(p, QPE_ERR_STATE, "plan was not created with QPE_FLAG_TIMING and bound");
  if (!p->timed_run) return fail(p, QPE_ERR_STATE, "no whole qpe_run has been timed yet");
  cudaError_t e = cudaEventSynchronize(p->ev[4]);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventSynchronize");
  for (int i = 0; i < 4; ++i) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventElapsedTime");
    ms[i] = t;
  }
  return QPE_OK;
}

qpe_status qpe_kernel_time(qpe_plan_t p, double* ms, int32_t* kernel_id) {
  if (!p || !ms || !kernel_id) return fail(p, QPE_ERR_ARG, "null pointer");
  if (!(p->flags & QPE_FLAG_TIMING) || p->inst.size() != 1 || !p->ev[0])
    return fail(p, QPE_ERR_STATE, "plan was not created with QPE_FLAG_TIMING (single instance) and bound");
  *ms = 0.0;
  *kernel_id = 0;
  if (!p->timed_kernel) return QPE_OK;
  cudaError_t e = cudaEventSynchronize(p->ev[6]);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventSynchronize");
  float t = 0.f;
  e = cudaEventElapsedTime(&t, p->ev[5], p->ev[6]);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaEventElapsedTime");
  *ms = t;
  *kernel_id = 1;
  return QPE_OK;
}

qpe_status qpe_selftest_timeout(qpe_plan_t p, int32_t instance, uint32_t polls) {
  if (!p) return QPE_ERR_ARG;
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  if (p->batched) return fail(p, QPE_ERR_UNSUPPORTED, "the wait-expiry self-test takes single-instance plans");
  if (polls < 1 || polls > (1u << 20)) return fail(p, QPE_ERR_ARG, "polls must be in 1 .. 2^20");
  Instance* in;
  qpe_status st = get_instance(p, instance, &in);
  if (st != QPE_OK) return st;
  cudaError_t e = qpe::configure_tc_kernels();
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute");
  if (qpe::launch_wait_expiry(*in, p->ws, polls, p->stream) < 0)
    return cuda_fail(p, cudaGetLastError(), "wait-expiry kernel");
  return QPE_OK;
}

qpe_status qpe_set_host_histogram(qpe_plan_t p, int32_t instance, double* host) {
  if (!p) return QPE_ERR_ARG;
  if (!p->bound) return fail(p, QPE_ERR_STATE, "qpe_bind first");
  if (p->batched) return fail(p, QPE_ERR_UNSUPPORTED, "batched plans hand out histograms with qpe_probs");
  Instance* in;
  qpe_status st = get_instance(p, instance, &in);
  if (st != QPE_OK) return st;
  if (in->shard_plain) return fail(p, QPE_ERR_UNSUPPORTED, "a sharded plain plan's histogram comes after the exchange");
  if (host) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess || at.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      return fail(p, QPE_ERR_ARG, "the host histogram must be page-locked host memory (qpe_host_alloc)");
    }
    if (!in->copy_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&in->copy_stream, cudaStreamNonBlocking);
      for (int c = 0; e == cudaSuccess && c <= qpe::kHostChunks; ++c)
        e = cudaEventCreateWithFlags(&in->copy_ev[c], cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(p, e, "copy stream");
    }
  }
  in->host_hist = host;
  if (p->graph_exec) {  // the next run captures the new copies
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  return QPE_OK;
}

qpe_status qpe_destroy(qpe_plan_t p) {
  if (!p) return QPE_OK;
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  for (Instance& in : p->inst) {
    for (cudaEvent_t ev : in.copy_ev)
      if (ev) cudaEventDestroy(ev);
    if (in.copy_stream) cudaStreamDestroy(in.copy_stream);
  }
  for (cudaEvent_t ev : p->ev)
    if (ev) cudaEventDestroy(ev);
  delete p;
  return QPE_OK;
}

}  // extern "C"
