// C ABI of the QPE emulator: plan validation, workspace layout, stage
// scheduling, readback. Declarations and contracts are in include/qpe.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
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
size_t elem_size(int prec) { return is_c64(prec) ? 8 : 16; }

qpe_status fail(qpe_plan_t p, qpe_status st, const std::string& msg) {
  if (p) p->last_error = msg;
  return st;
}

qpe_status cuda_fail(qpe_plan_t p, cudaError_t e, const char* where) {
  return fail(p, QPE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

// Lays out one instance starting at byte offset `base`; returns the end.
size_t layout_instance(Instance& in, int prec, uint32_t flags, size_t base) {
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
  in.state_bytes = (size_t)N * d * elem_size(prec);
  in.off_state = take(in.state_bytes);
  in.off_hist = take((size_t)N * 8);
  in.htw = (in.nmeas + 1) / 2;
  const size_t nlo = size_t(1) << in.htw, nhi = size_t(1) << (in.nmeas - in.htw);
  in.off_tw_lo64 = take(nlo * 16);
  in.off_tw_hi64 = take(nhi * 16);
  in.off_tw_lo32 = take(nlo * 8);
  in.off_tw_hi32 = take(nhi * 8);
  in.off_partials = take(sizeof(qpe::Partial) * qpe::kReduceBlocks);
  in.off_scalars = take(sizeof(qpe::Scalars));
  in.fft = qpe::make_fft_plan(in.nmeas, d, elem_size(prec));
  in.fused = in.nmat <= QPE_MAX_FUSED_NMAT && !(flags & (QPE_FLAG_PLAIN | QPE_FLAG_GATE_SWEEP));
  in.keep_state = (flags & QPE_FLAG_KEEP_STATE) != 0;
  if (in.nmat <= QPE_MAX_FUSED_NMAT) {
    // level buffers for the fused schedule (also allotted to plain plans so a
    // plan's layout does not depend on its schedule flags)
    in.levels = qpe::make_levels(in.nmeas, in.nmat, elem_size(prec), 0);
    size_t zb[2] = {0, 0};
    for (size_t li = 1; li < in.levels.size(); ++li) {
      const qpe::Level& L = in.levels[li];
      const size_t bytes = ((size_t)1 << (L.logna + L.r)) * d * elem_size(prec);
      zb[li & 1] = std::max(zb[li & 1], bytes);
    }
    in.off_zbuf[0] = take(zb[0] ? zb[0] : 16);
    in.off_zbuf[1] = take(zb[1] ? zb[1] : 16);
    in.zbuf_seed_off = take((size_t)d * elem_size(prec));
    for (qpe::Level& L : in.levels) L.tab_off = take(((size_t)d << L.r) * d * elem_size(prec));
  }
  return off;
}

qpe_status check_desc(const qpe_plan_desc* desc) {
  if (!desc) return QPE_ERR_ARG;
  if (desc->nmat < 1 || desc->nmat > kMaxNmat) return QPE_ERR_ARG;
  if (desc->nmeas < 1 || desc->nmeas > kMaxNmeas) return QPE_ERR_ARG;
  if (desc->prec < QPE_FP64 || desc->prec > QPE_C64_TF32X3) return QPE_ERR_ARG;
  if (desc->flags & ~(QPE_FLAG_GATE_SWEEP | QPE_FLAG_GRAPH | QPE_FLAG_TIMING | QPE_FLAG_PLAIN | QPE_FLAG_KEEP_STATE))
    return QPE_ERR_ARG;
  if (desc->prec > QPE_C64_FP32) return QPE_ERR_UNSUPPORTED;
  if ((desc->flags & QPE_FLAG_GATE_SWEEP) && desc->nmat > 6) return QPE_ERR_UNSUPPORTED;
  return QPE_OK;
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
qpe_status enqueue_stages(qpe_plan_t p, int first, int last, int64_t* launches) {
  int64_t n = 0;
  const bool c64 = is_c64(p->prec);
  const bool gate = (p->flags & QPE_FLAG_GATE_SWEEP) != 0;
  const bool timing = (p->flags & QPE_FLAG_TIMING) && p->inst.size() == 1 && p->ev[0];
  p->timed_run = timing && first == QPE_STAGE_POWERS && last == QPE_STAGE_REDUCE;
  p->timed_kernel = false;
  for (Instance& in : p->inst) {
    if (!in.loaded) return fail(p, QPE_ERR_STATE, "qpe_load has not been called for every instance");
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
      in.state_stage = QPE_STAGE_REDUCE;
      in.state_natural = true;
      in.state_valid = in.keep_state;
      continue;
    }
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
          r = c64 ? qpe::launch_sweep<float2>(in, p->ws, gate, p->stream)
                  : qpe::launch_sweep<double2>(in, p->ws, gate, p->stream);
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
  }
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

qpe_status qpe_bind(qpe_plan_t p, void* d_ws, size_t bytes, void* stream) {
  if (!p) return QPE_ERR_ARG;
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) % kAlign) != 0 || bytes < p->ws_bytes)
    return fail(p, QPE_ERR_WORKSPACE, "workspace must be non-null, 256-byte aligned and >= qpe_plan's size");
  if ((p->flags & QPE_FLAG_GRAPH) && !stream)
    return fail(p, QPE_ERR_ARG, "QPE_FLAG_GRAPH needs a non-default stream");
  cudaError_t e = qpe::configure_kernels();
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
    if (qpe::launch_twiddles(in, p->ws, p->stream) < 0) return cuda_fail(p, cudaGetLastError(), "twiddle tables");
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
      in.state_stage = QPE_STAGE_REDUCE;
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
    if (in.state_stage != QPE_STAGE_REDUCE) continue;
    qpe::Scalars s;
    e = cudaMemcpy(&s, p->ws + in.off_scalars, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p, e, "read error word");
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
  if (probs)
    e = cudaMemcpyAsync(probs, p->ws + in->off_hist, (size_t)in->N * 8, kind_from_device(ptr_is_device), p->stream);
  qpe::Scalars s;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&s, p->ws + in->off_scalars, sizeof(s), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "qpe_probs copy");
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
  }
  return -1;
}

qpe_status qpe_stage_times(qpe_plan_t p, double* ms) {
  if (!p || !ms) return fail(p, QPE_ERR_ARG, "null pointer");
  if (!(p->flags & QPE_FLAG_TIMING) || p->inst.size() != 1 || !p->ev[0])
    return fail(p, QPE_ERR_STATE, "plan was not created with QPE_FLAG_TIMING (single instance) and bound");
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

qpe_status qpe_destroy(qpe_plan_t p) {
  if (!p) return QPE_OK;
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  for (cudaEvent_t ev : p->ev)
    if (ev) cudaEventDestroy(ev);
  delete p;
  return QPE_OK;
}

}  // extern "C"
