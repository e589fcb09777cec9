"""Python binding of libqpe.so (include/qpe.h): argument marshalling only.

Every step of a QPE run executes in the library's CUDA kernels. PyTorch
supplies device memory (the workspace and any device-side outputs) and the
CUDA stream; this module never computes any part of the circuit itself and
has no CPU fallback: importing it fails if libqpe.so is missing.

Typical use::

    plan = Plan(nmat=6, nmeas=16, prec=C64_FP32)
    plan.load(U, psi)              # numpy complex128 (host) or torch cuda tensors
    plan.run()
    probs, argmax, phi_max, phi_mean = plan.probs()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libqpe.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"libqpe.so not found at {_LIB_PATH}: build it first "
        "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")

_lib = ctypes.CDLL(_LIB_PATH)

# ----------------------------------------------------------------- constants
OK, ERR_ARG, ERR_SHAPE, ERR_WORKSPACE, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT, ERR_NUMERIC, ERR_STATE = range(9)
FP64, C64_FP32, C64_BF16X3, C64_FP16X2, C64_TF32X3 = range(5)
FLAG_GATE_SWEEP = 0x1
FLAG_GRAPH = 0x2
FLAG_TIMING = 0x4
FLAG_PLAIN = 0x8
FLAG_KEEP_STATE = 0x10
FLAG_REPEAT_U = 0x20
FLAG_CHECK_UNITARY = 0x40
FLAG_AUTOTUNE = 0x80
FLAG_SQUARE_TC = 0x100
FLAG_LEVEL_TC = 0x200
STAGE_POWERS, STAGE_SWEEP, STAGE_FFT, STAGE_REDUCE = 1, 2, 3, 4
INFO_WORKSPACE_BYTES, INFO_STATE_BYTES, INFO_FFT_PASSES, INFO_LAST_LAUNCHES, INFO_INSTANCES = 1, 2, 3, 4, 5
INFO_SQUARE_TILE = 6
INFO_LEVELS, INFO_TOP_LEVEL_BITS, INFO_TC_TOP_LEVEL = 7, 8, 9


class PlanDesc(ctypes.Structure):
    _fields_ = [("nmat", ctypes.c_int32), ("nmeas", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class Readout(ctypes.Structure):
    _fields_ = [("argmax", ctypes.c_int64), ("phase_argmax", ctypes.c_double),
                ("phase_mean", ctypes.c_double), ("total", ctypes.c_double)]


class ShardReadout(ctypes.Structure):
    _fields_ = [("argmax", ctypes.c_int64), ("p_argmax", ctypes.c_double), ("phase_mean_part", ctypes.c_double),
                ("total", ctypes.c_double), ("nmeas", ctypes.c_int32), ("rank", ctypes.c_int32)]

    def as_tuple(self):
        return (int(self.argmax), float(self.p_argmax), float(self.phase_mean_part), float(self.total),
                int(self.nmeas), int(self.rank))

    @classmethod
    def from_tuple(cls, t):
        return cls(int(t[0]), float(t[1]), float(t[2]), float(t[3]), int(t[4]), int(t[5]))


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_sig = {
    "qpe_plan": (ctypes.c_int, [ctypes.POINTER(PlanDesc), ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_vp)]),
    "qpe_plan_batched": (ctypes.c_int, [ctypes.POINTER(PlanDesc), ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t),
                                        ctypes.POINTER(_vp)]),
    "qpe_plan_shard": (ctypes.c_int, [ctypes.POINTER(PlanDesc), _i32, _i32, ctypes.POINTER(ctypes.c_size_t),
                                      ctypes.POINTER(_vp)]),
    "qpe_shard_readout": (ctypes.c_int, [_vp, ctypes.POINTER(ShardReadout)]),
    "qpe_merge_shard_readouts": (ctypes.c_int, [ctypes.POINTER(ShardReadout), _i32, ctypes.POINTER(Readout)]),
    "qpe_shard_buffers": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t)]),
    "qpe_shard_finish": (ctypes.c_int, [_vp]),
    "qpe_bind": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _vp]),
    "qpe_load": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i32, _i32, _i32]),
    "qpe_run": (ctypes.c_int, [_vp]),
    "qpe_run_stages": (ctypes.c_int, [_vp, _i32, _i32]),
    "qpe_probs": (ctypes.c_int, [_vp, _i32, _vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), _i32]),
    "qpe_state": (ctypes.c_int, [_vp, _i32, _vp, _i32]),
    "qpe_load_state": (ctypes.c_int, [_vp, _i32, _vp, _i32]),
    "qpe_powers": (ctypes.c_int, [_vp, _i32, _i32, _vp, _i32]),
    "qpe_query": (ctypes.c_int64, [_vp, _i32]),
    "qpe_sync": (ctypes.c_int, [_vp]),
    "qpe_stage_times": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "qpe_kernel_time": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    "qpe_destroy": (ctypes.c_int, [_vp]),
    "qpe_selftest_timeout": (ctypes.c_int, [_vp, _i32, ctypes.c_uint32]),
    "qpe_readout_static": (ctypes.c_int, [_vp, _i32, _i32, _i32, _vp, _vp, _vp]),
    "qpe_measure_fma_peak": (ctypes.c_int, [_i32, _i32, _i32, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                                            ctypes.POINTER(ctypes.c_double), _vp]),
    "qpe_host_alloc": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "qpe_set_host_histogram": (ctypes.c_int, [_vp, _i32, _vp]),
    "qpe_host_free": (ctypes.c_int, [_vp]),
    "qpe_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "qpe_last_error": (ctypes.c_char_p, [_vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

LIB = _lib
LIB_PATH = _LIB_PATH


class QpeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


def status_string(st: int) -> str:
    return _lib.qpe_status_string(st).decode()


class _HostBuffer:
    """Owner of one qpe_host_alloc block; freed when the last array over it goes."""

    def __init__(self, nbytes: int):
        self.ptr = _vp()
        st = _lib.qpe_host_alloc(nbytes, ctypes.byref(self.ptr))
        if st != OK:
            raise QpeError(st, f"qpe_host_alloc({nbytes}): {status_string(st)}")
        self.nbytes = nbytes

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value:
            _lib.qpe_host_free(self.ptr)
            self.ptr = _vp()


def host_array(shape, dtype=np.float64) -> np.ndarray:
    """A numpy array in page-locked host memory from qpe_host_alloc (device
    copies into and out of it run at the host link's rate); the memory is freed
    with the last reference to the array."""
    dtype = np.dtype(dtype)
    count = int(np.prod(shape))
    buf = _HostBuffer(max(1, count) * dtype.itemsize)
    raw = (ctypes.c_char * (max(1, count) * dtype.itemsize)).from_address(buf.ptr.value)
    raw._qpe_buffer = buf  # the array's base (the ctypes block) keeps the allocation alive
    return np.frombuffer(raw, dtype=dtype, count=count).reshape(shape)


def plan_workspace(nmat: int, nmeas: int, prec: int = C64_FP32, flags: int = 0):
    """Host-only: (status, workspace_bytes, raw plan handle)."""
    desc = PlanDesc(nmat, nmeas, prec, flags)
    ws = ctypes.c_size_t(0)
    h = _vp()
    st = _lib.qpe_plan(ctypes.byref(desc), ctypes.byref(ws), ctypes.byref(h))
    return st, ws.value, h


def plan_shard_workspace(nmat: int, nmeas: int, prec: int, flags: int, rank: int, world: int):
    """Host-only: (status, workspace_bytes, raw plan handle) of rank ``rank``
    of ``world`` (qpe_plan_shard)."""
    desc = PlanDesc(nmat, nmeas, prec, flags)
    ws = ctypes.c_size_t(0)
    h = _vp()
    st = _lib.qpe_plan_shard(ctypes.byref(desc), rank, world, ctypes.byref(ws), ctypes.byref(h))
    return st, ws.value, h


def merge_shard_readouts(parts):
    """Readout of the whole histogram from every rank's ShardReadout (or its
    as_tuple()): (argmax, phase_argmax, phase_mean, total); host only."""
    parts = [p if isinstance(p, ShardReadout) else ShardReadout.from_tuple(p) for p in parts]
    arr = (ShardReadout * len(parts))(*parts)
    out = Readout()
    st = _lib.qpe_merge_shard_readouts(arr, len(parts), ctypes.byref(out))
    if st != OK:
        raise QpeError(st, f"qpe_merge_shard_readouts: {status_string(st)}")
    return int(out.argmax), float(out.phase_argmax), float(out.phase_mean), float(out.total)


def interleave_shards(parts):
    """The whole histogram from the ranks' compact slices (rank r holds
    P[r + world j] at j): P[r + world j] = parts[r][j]. Works on numpy arrays
    or torch tensors of equal length."""
    world = len(parts)
    if isinstance(parts[0], np.ndarray):
        return np.stack(parts, axis=1).reshape(-1)
    import torch
    return torch.stack(list(parts), dim=1).reshape(-1)


def gather_shards(dist, local, part: ShardReadout, group=None):
    """(whole histogram, argmax, phase_argmax, phase_mean) of a sharded run:
    every rank's compact histogram slice ``local`` (a float64 tensor, N / world
    bins) is all-gathered and interleaved, and the ranks' readout partials
    merged by qpe_merge_shard_readouts. NCCL groups gather device tensors,
    others (gloo) host tensors."""
    import torch
    world = dist.get_world_size(group)
    if dist.get_backend(group) != "nccl":
        local = local.cpu()
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local.contiguous(), group=group)
    mine = torch.tensor(part.as_tuple()[:4], dtype=torch.float64, device=local.device)
    allp = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(allp, mine, group=group)
    pieces = [ShardReadout(int(t[0].item()), float(t[1]), float(t[2]), float(t[3]), part.nmeas, r)
              for r, t in enumerate(allp)]
    am, pa, pm, _ = merge_shard_readouts(pieces)
    return interleave_shards(parts), am, pa, pm


def readout_static(final_state, nmat: int, nmeas: int, prec: int, probs, readout, stream=None) -> int:
    """Histogram + readout of a device-resident final statevector through the
    entry point that allocates nothing (qpe_readout_static). ``probs`` is a
    float64 CUDA tensor of N elements and ``readout`` a 32-byte CUDA tensor
    receiving (int64 argmax, phase_argmax, phase_mean, total). Returns the
    qpe_status."""
    import torch
    if not (1 <= nmat <= 12 and 1 <= nmeas <= 30):
        raise ValueError("nmat must be in 1..12 and nmeas in 1..30")
    want = torch.complex128 if prec == FP64 else torch.complex64
    n_amp, n_out = (1 << nmat) << nmeas, 1 << nmeas
    for name, t, dt, count in (("final_state", final_state, want, n_amp), ("probs", probs, torch.float64, n_out),
                               ("readout", readout, None, None)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if dt is not None and (t.dtype != dt or t.numel() < count):
            raise ValueError(f"{name} must be {dt} with at least {count} elements")
    if readout.numel() * readout.element_size() < 32:
        raise ValueError("readout must hold at least 32 bytes")
    s = 0 if stream is None else stream.cuda_stream
    return _lib.qpe_readout_static(final_state.data_ptr(), nmat, nmeas, prec, probs.data_ptr(), readout.data_ptr(),
                                   s or None)


def measure_fma_peak(fp64: bool, iters: int, repeats: int = 5, device=None, stream=None) -> float:
    """TFLOP/s of fused multiply-adds on the FP64 (fp64=True) or FP32 units,
    measured by the library's FMA loop kernel with CUDA events
    (include/qpe_peak.h); scratch from torch."""
    import torch
    need = ctypes.c_size_t(0)
    st = _lib.qpe_measure_fma_peak(int(fp64), iters, repeats, None, 0, ctypes.byref(need), None, None)
    if st != OK:
        raise QpeError(st, f"qpe_measure_fma_peak: {status_string(st)}")
    dev = torch.device(device if device is not None else "cuda")
    scratch = torch.empty(need.value, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream(dev) if stream is None else stream
    tf = ctypes.c_double(0.0)
    st = _lib.qpe_measure_fma_peak(int(fp64), iters, repeats, scratch.data_ptr(), need.value, None,
                                   ctypes.byref(tf), s.cuda_stream)
    if st != OK:
        raise QpeError(st, f"qpe_measure_fma_peak: {status_string(st)}")
    return tf.value


def plan_batched_workspace(shapes, prec: int = C64_FP32, flags: int = 0):
    """Host-only: (status, workspace_bytes, raw handle) for [(nmat, nmeas), ...]."""
    arr = (PlanDesc * len(shapes))(*[PlanDesc(a, b, prec, flags) for a, b in shapes])
    ws = ctypes.c_size_t(0)
    h = _vp()
    st = _lib.qpe_plan_batched(arr, len(shapes), ctypes.byref(ws), ctypes.byref(h))
    return st, ws.value, h


def _ptr(x):
    """(address, is_device) of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), 1 if x.is_cuda else 0
    raise TypeError(f"unsupported buffer type {type(x)}")


class Plan:
    """One QPE problem bound to a torch-allocated workspace and stream."""

    def __init__(self, nmat: int, nmeas: int, prec: int = C64_FP32, flags: int = 0,
                 device=None, stream=None, workspace=None):
        import torch
        self.nmat, self.nmeas, self.prec, self.flags = nmat, nmeas, prec, flags
        self.d, self.N = 1 << nmat, 1 << nmeas
        st, self.ws_bytes, self._h = plan_workspace(nmat, nmeas, prec, flags)
        if st != OK:
            raise QpeError(st, f"qpe_plan: {status_string(st)}")
        self.device = torch.device(device if device is not None else "cuda")
        if stream is None:
            stream = torch.cuda.Stream(device=self.device) if (flags & FLAG_GRAPH) else \
                torch.cuda.current_stream(self.device)
        self.stream = stream
        if workspace is None:
            workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.workspace = workspace
        self._check(_lib.qpe_bind(self._h, workspace.data_ptr(), self.ws_bytes, stream.cuda_stream), "qpe_bind")

    # -------------------------------------------------------------- helpers
    def _check(self, st: int, what: str):
        if st != OK:
            msg = _lib.qpe_last_error(self._h).decode() if self._h else ""
            raise QpeError(st, f"{what}: {status_string(st)} {msg}")

    @property
    def handle(self):
        return self._h

    @property
    def state_dtype(self):
        return np.complex128 if self.prec == FP64 else np.complex64

    def query(self, key: int) -> int:
        return int(_lib.qpe_query(self._h, key))

    # ------------------------------------------------------------------ API
    def load(self, U, psi, instance: int = 0):
        """Copy U (d x d complex128) and psi (d complex128) in; numpy arrays
        are host buffers, CUDA tensors device buffers."""
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
            psi = np.ascontiguousarray(psi, dtype=np.complex128)
        pu, du = _ptr(U)
        pp, dp = _ptr(psi)
        if du != dp:
            raise ValueError("U and psi must both be host or both be device buffers")
        self._keep = (U, psi)
        self._check(_lib.qpe_load(self._h, instance, pu, pp, self.nmat, self.nmeas, du), "qpe_load")

    def set_host_histogram(self, host, instance: int = 0):
        """Every following run also copies the histogram into ``host`` (a
        host_array of N float64, or None to stop), overlapped with the
        computation where the top level allows it."""
        ptr = None if host is None else host.ctypes.data
        self._check(_lib.qpe_set_host_histogram(self._h, instance, ptr), "qpe_set_host_histogram")
        self._host_hist = host

    def run(self):
        self._check(_lib.qpe_run(self._h), "qpe_run")

    def run_stages(self, first: int, last: int):
        self._check(_lib.qpe_run_stages(self._h, first, last), "qpe_run_stages")

    def sync(self):
        self._check(_lib.qpe_sync(self._h), "qpe_sync")

    def probs(self, out=None, instance: int = 0, want_hist: bool = True):
        """(histogram or None, argmax, phase_argmax, phase_mean). ``out`` may be
        a float64 numpy array or CUDA tensor of N elements."""
        am = ctypes.c_int64(0)
        pa = ctypes.c_double(0.0)
        pm = ctypes.c_double(0.0)
        if want_hist and out is None:
            out = np.empty(self.N, dtype=np.float64)
        ptr, dev = (0, 0) if out is None else _ptr(out)
        self._check(_lib.qpe_probs(self._h, instance, ptr or None, ctypes.byref(am), ctypes.byref(pa),
                                   ctypes.byref(pm), dev), "qpe_probs")
        return out, am.value, pa.value, pm.value

    def state(self, out=None, instance: int = 0):
        if out is None:
            out = np.empty((self.N, self.d), dtype=self.state_dtype)
        ptr, dev = _ptr(out)
        self._check(_lib.qpe_state(self._h, instance, ptr, dev), "qpe_state")
        return out

    def load_state(self, S, instance: int = 0):
        if isinstance(S, np.ndarray):
            S = np.ascontiguousarray(S, dtype=self.state_dtype)
        ptr, dev = _ptr(S)
        self._keep_state = S
        self._check(_lib.qpe_load_state(self._h, instance, ptr, dev), "qpe_load_state")

    def power(self, k: int, instance: int = 0) -> np.ndarray:
        out = np.empty((self.d, self.d), dtype=np.complex128)
        self._check(_lib.qpe_powers(self._h, instance, k, out.ctypes.data, 0), "qpe_powers")
        return out

    def stage_times(self):
        """ms of (powers, sweep, fft, reduce) in the last qpe_run (FLAG_TIMING)."""
        ms = (ctypes.c_double * 4)()
        self._check(_lib.qpe_stage_times(self._h, ms), "qpe_stage_times")
        return list(ms)

    def kernel_time(self):
        """(ms, kernel id) of the last run's dominant kernel (FLAG_TIMING);
        id 1 = the top level of the fused schedule, 0 = not timed."""
        ms = ctypes.c_double(0.0)
        kid = ctypes.c_int32(0)
        self._check(_lib.qpe_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(kid)), "qpe_kernel_time")
        return ms.value, kid.value

    def selftest_timeout(self, polls: int = 64, instance: int = 0):
        """Enqueue the library's bounded-wait expiry on purpose: the next sync
        or probs reports ERR_TIMEOUT, the next whole run clears it."""
        self._check(_lib.qpe_selftest_timeout(self._h, instance, polls), "qpe_selftest_timeout")

    def close(self):
        if getattr(self, "_h", None):
            _lib.qpe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ShardedPlan(Plan):
    """Rank ``rank`` of ``world`` processes sharing one QPE problem
    (qpe_plan_shard): this rank computes the outcomes y = rank (mod world).
    ``probs()`` returns its N / world bins compactly; ``shard_readout()`` its
    readout partial for merge_shard_readouts; ``gather(dist)`` all-gathers the
    whole histogram over a torch.distributed process group."""

    def __init__(self, nmat: int, nmeas: int, prec: int, flags: int, rank: int, world: int,
                 device=None, stream=None, workspace=None):
        import torch
        self.nmat, self.nmeas, self.prec, self.flags = nmat, nmeas, prec, flags
        self.rank, self.world = rank, world
        self.d, self.N = 1 << nmat, 1 << nmeas
        st, self.ws_bytes, self._h = plan_shard_workspace(nmat, nmeas, prec, flags, rank, world)
        if st != OK:
            raise QpeError(st, f"qpe_plan_shard: {status_string(st)}")
        self.device = torch.device(device if device is not None else "cuda")
        if stream is None:
            stream = torch.cuda.Stream(device=self.device) if (flags & FLAG_GRAPH) else \
                torch.cuda.current_stream(self.device)
        self.stream = stream
        if workspace is None:
            workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.workspace = workspace
        self._check(_lib.qpe_bind(self._h, workspace.data_ptr(), self.ws_bytes, stream.cuda_stream), "qpe_bind")

    def probs(self, out=None, instance: int = 0, want_hist: bool = True):
        if want_hist and out is None:
            out = np.empty(self.N // self.world, dtype=np.float64)
        return super().probs(out, instance, want_hist)

    def state(self, out=None, instance: int = 0):
        if out is None:
            out = np.empty((self.N // self.world, self.d), dtype=self.state_dtype)
        return super().state(out, instance)

    def buffers(self):
        """(send, recv) uint8 views of the all-to-all buffers inside the
        workspace (world chunks of equal size each), or (None, None) when the
        plan exchanges nothing (fused form)."""
        sp, rp, nb = _vp(), _vp(), ctypes.c_size_t(0)
        self._check(_lib.qpe_shard_buffers(self._h, ctypes.byref(sp), ctypes.byref(rp), ctypes.byref(nb)),
                    "qpe_shard_buffers")
        if nb.value == 0:
            return None, None
        base = self.workspace.data_ptr()
        n = nb.value * self.world
        so, ro = sp.value - base, rp.value - base
        return self.workspace[so:so + n], self.workspace[ro:ro + n]

    def finish(self):
        self._check(_lib.qpe_shard_finish(self._h), "qpe_shard_finish")

    def run_exchange(self, dist, group=None):
        """One whole sharded run with its exchange over a torch.distributed
        group: qpe_run, an all-to-all of the send buffer (NCCL on device
        buffers; other backends through host copies), qpe_shard_finish."""
        import torch
        self.run()
        send, recv = self.buffers()
        if send is not None:
            if dist.get_backend(group) == "nccl":
                torch.cuda.current_stream(self.device).wait_stream(self.stream)
                dist.all_to_all_single(recv, send, group=group)
                self.stream.wait_stream(torch.cuda.current_stream(self.device))
            else:
                self.stream.synchronize()
                hs = send.cpu()
                hr = torch.empty_like(hs)
                dist.all_to_all_single(hr, hs, group=group)
                with torch.cuda.stream(self.stream):
                    recv.copy_(hr, non_blocking=False)
        self.finish()

    def shard_readout(self) -> ShardReadout:
        r = ShardReadout()
        self._check(_lib.qpe_shard_readout(self._h, ctypes.byref(r)), "qpe_shard_readout")
        return r

    def gather(self, dist, group=None):
        """(whole histogram, argmax, phase_argmax, phase_mean) over the process
        group (see gather_shards)."""
        import torch
        local = torch.empty(self.N // self.world, dtype=torch.float64, device=self.device)
        super().probs(local)
        return gather_shards(dist, local, self.shard_readout(), group)


class BatchedPlan(Plan):
    """Many independent QPE problems of uneven shape in one plan (grouped
    launches per step across instances). ``shapes`` = [(nmat, nmeas), ...]."""

    def __init__(self, shapes, prec: int = C64_FP32, flags: int = 0, device=None, stream=None, workspace=None):
        import torch
        self.shapes = [(int(a), int(b)) for a, b in shapes]
        self.prec, self.flags = prec, flags
        st, self.ws_bytes, self._h = plan_batched_workspace(self.shapes, prec, flags)
        if st != OK:
            raise QpeError(st, f"qpe_plan_batched: {status_string(st)}")
        self.device = torch.device(device if device is not None else "cuda")
        if stream is None:
            stream = torch.cuda.Stream(device=self.device) if (flags & FLAG_GRAPH) else \
                torch.cuda.current_stream(self.device)
        self.stream = stream
        if workspace is None:
            workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.workspace = workspace
        self._keep_inputs = {}
        self._check(_lib.qpe_bind(self._h, workspace.data_ptr(), self.ws_bytes, stream.cuda_stream), "qpe_bind")

    def load(self, instance: int, U, psi):
        nmat, nmeas = self.shapes[instance]
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
            psi = np.ascontiguousarray(psi, dtype=np.complex128)
        pu, du = _ptr(U)
        pp, dp = _ptr(psi)
        self._keep_inputs[instance] = (U, psi)
        self._check(_lib.qpe_load(self._h, instance, pu, pp, nmat, nmeas, du), "qpe_load")

    def probs(self, instance: int = 0, out=None, want_hist: bool = True):
        nmat, nmeas = self.shapes[instance]
        am = ctypes.c_int64(0)
        pa = ctypes.c_double(0.0)
        pm = ctypes.c_double(0.0)
        if want_hist and out is None:
            out = np.empty(1 << nmeas, dtype=np.float64)
        ptr, dev = (0, 0) if out is None else _ptr(out)
        self._check(_lib.qpe_probs(self._h, instance, ptr or None, ctypes.byref(am), ctypes.byref(pa),
                                   ctypes.byref(pm), dev), "qpe_probs")
        return out, am.value, pa.value, pm.value

    def state(self, instance: int = 0, out=None):
        nmat, nmeas = self.shapes[instance]
        if out is None:
            out = np.empty((1 << nmeas, 1 << nmat), dtype=self.state_dtype)
        ptr, dev = _ptr(out)
        self._check(_lib.qpe_state(self._h, instance, ptr, dev), "qpe_state")
        return out
