"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (max-abs on probabilities): FP64 path 1e-10, complex64 path 1e-5,
argmax identical. Against closed forms at large Nmeas the FP64 floor of the
constructed input applies: its eigenphases carry ~u sqrt(d) of rounding,
which the readout multiplies by N, so those comparisons use
max(1e-10, 2 N u sqrt(d)).
"""
import numpy as np
import pytest

from oracle import fejer, gates, readout
from paper_2507_17175_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64 = np.finfo(np.float64).eps / 2
TOL = {0: 1e-10, 1: 1e-5}  # FP64, C64_FP32


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2507_17175_gb300 import qpe
    return qpe


_cache = {}


def oracle_probs(inst):
    key = inst.name
    if key not in _cache:
        _cache[key] = gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)
    return _cache[key]


def run_plan(q, inst, prec, flags=0):
    plan = q.Plan(inst.nmat, inst.nmeas, prec, flags)
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, pa, pm = plan.probs()
    return plan, P, am, pa, pm


# ------------------------------------------------------------ end to end
PLAIN, KEEP = 0x8, 0x10


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("flags", [0, 1, 2, PLAIN, PLAIN | 2])
def test_c1_exact_phase(q, prec, flags):
    inst = W.c1()
    plan, P, am, pa, pm = run_plan(q, inst, prec, flags)
    ref = oracle_probs(inst)
    assert np.abs(P - ref).max() <= TOL[prec]
    k0 = int(inst.meta["k"][0])
    assert am == k0 and pa == k0 / 64.0
    assert abs(pm - readout.phase_weighted_mean(ref)) <= 64 * TOL[prec]
    tgt = np.zeros(64)
    tgt[k0] = 1.0
    assert np.abs(P - tgt).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("flags", [0, 1, PLAIN])
def test_c2_vs_gate_by_gate_and_fejer(q, prec, flags):
    inst = W.c2()
    plan, P, am, pa, pm = run_plan(q, inst, prec, flags)
    ref = oracle_probs(inst)
    err = np.abs(P - ref).max()
    assert err <= TOL[prec], err
    assert am == readout.argmax_lowest(ref)
    assert pa == readout.phase_max_norm(ref)
    assert abs(pm - readout.phase_weighted_mean(ref)) <= (1e-9 if prec == 0 else 1e-4)
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas)
    assert np.abs(P - Q).max() <= TOL[prec]
    assert abs(P.sum() - 1.0) <= (1e-10 if prec == 0 else 1e-4)


def test_c2_graph_replay_is_deterministic(q):
    inst = W.c2()
    plan = q.Plan(inst.nmat, inst.nmeas, q.C64_FP32, q.FLAG_GRAPH)
    plan.load(inst.U, inst.psi)
    outs = []
    for _ in range(3):
        plan.run()
        outs.append(plan.probs()[0].copy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    assert np.abs(outs[0] - oracle_probs(inst)).max() <= 1e-5


# ------------------------------------------------------------ single steps
@pytest.mark.parametrize("nmat,nmeas", [(1, 5), (3, 9), (6, 16), (8, 10), (10, 6)])
def test_powers_stage(q, nmat, nmeas):
    rng = np.random.default_rng(100 + nmat)
    U = W.haar_unitary(rng, 1 << nmat)
    psi = U[:, 0].copy()
    plan = q.Plan(nmat, nmeas, q.C64_FP32)
    plan.load(U, psi)
    plan.run_stages(q.STAGE_POWERS, q.STAGE_POWERS)
    ref = gates.powers_by_squaring(U, nmeas)
    for k in range(nmeas):
        got = plan.power(k)
        want = np.linalg.matrix_power(U, 1 << k)
        assert np.abs(got - ref[k]).max() <= 64 * (1 << k) * U64 * (1 << nmat)
        assert np.abs(got - want).max() <= 64 * (1 << k) * U64 * (1 << nmat)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("flags", [PLAIN, 1])
@pytest.mark.parametrize("nmat,nmeas", [(1, 1), (2, 7), (4, 11), (6, 9)])
def test_sweep_stage_rows(q, prec, flags, nmat, nmeas):
    """After the Hadamard layer and the controlled gates, row m of the state
    equals the oracle's gate-by-gate row (2^(-n/2) U^m psi)."""
    rng = np.random.default_rng(7 * nmat + nmeas)
    U = W.haar_unitary(rng, 1 << nmat)
    psi = W.random_state(rng, 1 << nmat, 1)[:, 0]
    plan = q.Plan(nmat, nmeas, prec, flags)
    plan.load(U, psi)
    plan.run_stages(q.STAGE_POWERS, q.STAGE_SWEEP)
    S = plan.state()
    ref = gates.qpe_after_sweeps(U, psi, nmeas)
    scale = 1.0 / np.sqrt(1 << nmeas)
    tol = (1e-12 if prec == 0 else 2e-6) * scale * np.abs(psi).max() * (1 << nmat)
    assert np.abs(S - ref).max() <= tol


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nmat,nmeas", [(1, 1), (2, 2), (1, 9), (3, 10), (2, 13), (4, 19), (6, 16), (9, 11),
                                        (1, 18)])
def test_fft_stage_vs_numpy(q, prec, nmat, nmeas):
    """QFT^-1 stage on an arbitrary loaded state == numpy.fft.fft(axis=0,
    norm="ortho") (covers 1..3 passes and ragged digit splits)."""
    rng = np.random.default_rng(nmat * 100 + nmeas)
    S = W.random_state(rng, 1 << nmeas, 1 << nmat)
    plan = q.Plan(nmat, nmeas, prec, PLAIN)
    dt = np.complex128 if prec == 0 else np.complex64
    plan.load(np.eye(1 << nmat, dtype=np.complex128), np.ones(1 << nmat, dtype=np.complex128))
    plan.load_state(S.astype(dt))
    plan.run_stages(q.STAGE_FFT, q.STAGE_FFT)
    X = plan.state()
    ref = np.fft.fft(S.astype(dt).astype(np.complex128), axis=0, norm="ortho")
    tol = (1e-13 if prec == 0 else 3e-6) * np.sqrt(nmeas) * np.abs(ref).max()
    assert np.abs(X - ref).max() <= tol


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nmat,nmeas", [(1, 3), (3, 10), (5, 19), (7, 8)])
def test_reduce_stage(q, prec, nmat, nmeas):
    """Histogram, argmax and weighted mean from a loaded state == numpy on the
    numpy-transformed state."""
    rng = np.random.default_rng(nmat + 31 * nmeas)
    S = W.random_state(rng, 1 << nmeas, 1 << nmat)
    S /= np.linalg.norm(S)
    dt = np.complex128 if prec == 0 else np.complex64
    plan = q.Plan(nmat, nmeas, prec, PLAIN)
    plan.load(np.eye(1 << nmat, dtype=np.complex128), np.ones(1 << nmat, dtype=np.complex128))
    plan.load_state(S.astype(dt))
    plan.run_stages(q.STAGE_FFT, q.STAGE_REDUCE)
    P, am, pa, pm = plan.probs()
    X = np.fft.fft(S.astype(dt).astype(np.complex128), axis=0, norm="ortho")
    ref = gates.probabilities(X)
    assert np.abs(P - ref).max() <= (1e-12 if prec == 0 else 1e-5) * ref.max()
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 10 * TOL[prec]:
        assert am == readout.argmax_lowest(ref)
    assert am == int(np.argmax(P))
    assert abs(pm - readout.phase_weighted_mean(ref)) <= 1e-6


def test_reduce_ties_go_to_lowest_index(q):
    """A delta input on a 2-qubit register transforms into exactly equal
    amplitudes (twiddles are 1 and -i, exact), so every outcome ties: the
    argmax must be 0."""
    S = np.zeros((4, 2), dtype=np.complex128)
    S[0, 0] = 1.0
    plan = q.Plan(1, 2, q.FP64, PLAIN)
    plan.load(np.eye(2, dtype=np.complex128), np.ones(2, dtype=np.complex128))
    plan.load_state(S)
    plan.run_stages(q.STAGE_FFT, q.STAGE_REDUCE)
    P, am, pa, pm = plan.probs()
    assert np.all(P == 0.25) and am == 0 and pa == 0.0
    assert pm == pytest.approx((0 + 1 + 2 + 3) / 4 / 4)


@pytest.mark.parametrize("flags", [KEEP, PLAIN])
def test_state_readback_device_matches_host(q, flags):
    import torch
    inst = W.c1()
    plan, *_ = run_plan(q, inst, q.FP64, flags)
    host = plan.state()
    dev = torch.empty((64, 4), dtype=torch.complex128, device="cuda")
    plan.state(dev)
    torch.cuda.synchronize()
    assert np.array_equal(host, dev.cpu().numpy())
    ref = gates.qpe_final_state(inst.U, inst.psi, inst.nmeas)
    assert np.abs(host - ref).max() <= 1e-12


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nmat,nmeas", [(1, 12), (2, 14), (3, 11), (4, 13), (5, 10), (6, 9), (2, 20), (4, 19),
                                        (6, 17), (1, 1), (3, 2)])
def test_fused_levels_vs_oracle(q, prec, nmat, nmeas):
    """The fused schedule (levels of r <= 10 measurement qubits, recursing
    through Z tables) against the gate-by-gate oracle: histogram, readout and
    the kept final statevector. Sizes cover one, two and three levels."""
    rng = np.random.default_rng(1000 * nmat + nmeas)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    plan = q.Plan(nmat, nmeas, prec, KEEP)
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, pa, pm = plan.probs()
    X = plan.state()
    ref_state = gates.qpe_final_state(inst.U, inst.psi, nmeas)
    ref = gates.probabilities(ref_state)
    assert np.abs(P - ref).max() <= TOL[prec]
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 10 * TOL[prec]:
        assert am == readout.argmax_lowest(ref)
    assert abs(pm - readout.phase_weighted_mean(ref)) <= (1e-9 if prec == 0 else 2e-5)
    # FP64: U^(2^(n-1)) carries ~2^(n-1) u of rounding on both sides
    amp_tol = max(1e-12, 16 * (1 << nmeas) * U64) if prec == 0 else 3e-6
    assert np.abs(X - ref_state).max() <= amp_tol
    # without KEEP_STATE the same histogram, and the state is not available
    plan2 = q.Plan(nmat, nmeas, prec)
    plan2.load(inst.U, inst.psi)
    plan2.run()
    P2, am2, _, _ = plan2.probs()
    assert np.array_equal(P, P2) and am == am2
    with pytest.raises(q.QpeError) as e:
        plan2.state()
    assert e.value.status == q.ERR_STATE


def test_fused_plan_without_state_buffer(q):
    """A default (fused) plan reserves no N x d state: stage-by-stage runs
    and qpe_load_state say so instead of touching memory it does not have."""
    st_f, ws_f, h = q.plan_workspace(4, 20, q.C64_FP32)
    q.LIB.qpe_destroy(h)
    st_p, ws_p, h = q.plan_workspace(4, 20, q.C64_FP32, PLAIN)
    q.LIB.qpe_destroy(h)
    assert ws_p - ws_f >= (1 << 20) * 16 * 8
    plan = q.Plan(2, 6, q.C64_FP32)
    U = np.eye(4, dtype=np.complex128)
    plan.load(U, U[0].copy())
    with pytest.raises(q.QpeError) as e:
        plan.run_stages(q.STAGE_POWERS, q.STAGE_SWEEP)
    assert e.value.status == q.ERR_STATE
    with pytest.raises(q.QpeError) as e:
        plan.load_state(np.zeros((64, 4), dtype=np.complex64))
    assert e.value.status == q.ERR_STATE


def test_device_inputs(q):
    import torch
    inst = W.c2()
    plan = q.Plan(inst.nmat, inst.nmeas, q.C64_FP32)
    plan.load(torch.from_numpy(inst.U).cuda(), torch.from_numpy(inst.psi).cuda())
    plan.run()
    out = torch.empty(inst.N, dtype=torch.float64, device="cuda")
    _, am, _, _ = plan.probs(out)
    assert np.abs(out.cpu().numpy() - oracle_probs(inst)).max() <= 1e-5


# ------------------------------------------------------------ edge cases
@pytest.mark.parametrize("prec", [0, 1])
def test_smallest_problem(q, prec):
    """Nmat = Nmeas = 1 (2 qubits) against the whole-circuit matrix."""
    from oracle import circuit_matrix
    rng = np.random.default_rng(1)
    U = W.haar_unitary(rng, 2)
    psi = np.array([0.6, 0.8j])
    plan = q.Plan(1, 1, prec)
    plan.load(U, psi)
    plan.run()
    P, am, _, _ = plan.probs()
    ref = gates.probabilities(circuit_matrix.qpe_final_state(U, psi, 1))
    assert np.abs(P - ref).max() <= TOL[prec]


def test_unnormalised_psi_keeps_its_norm(q):
    rng = np.random.default_rng(2)
    inst = W.haar_instance(rng, 3, 12, superposition=True)
    plan = q.Plan(3, 12, q.FP64)
    plan.load(inst.U, 2.0 * inst.psi)
    plan.run()
    P, *_ = plan.probs()
    assert abs(P.sum() - 4.0) <= 1e-10


def test_nan_input_is_reported(q):
    U = np.eye(4, dtype=np.complex128)
    U[1, 1] = np.nan
    plan = q.Plan(2, 5, q.C64_FP32)
    plan.load(U, np.ones(4, dtype=np.complex128) / 2)
    plan.run()
    with pytest.raises(q.QpeError) as e:
        plan.probs()
    assert e.value.status == q.ERR_NUMERIC


def test_gpu_error_paths(q):
    import torch
    st, ws, h = q.plan_workspace(2, 6, q.FP64)
    small = torch.empty(ws // 2, dtype=torch.uint8, device="cuda")
    assert q.LIB.qpe_bind(h, small.data_ptr(), ws // 2, None) == q.ERR_WORKSPACE
    q.LIB.qpe_destroy(h)
    plan = q.Plan(2, 6, q.FP64, PLAIN)
    U = np.eye(4, dtype=np.complex128)
    with pytest.raises(q.QpeError) as e:
        plan._check(q.LIB.qpe_load(plan.handle, 0, U.ctypes.data, U.ctypes.data, 3, 6, 0), "load")
    assert e.value.status == q.ERR_SHAPE
    with pytest.raises(q.QpeError) as e:
        plan._check(q.LIB.qpe_load(plan.handle, 1, U.ctypes.data, U.ctypes.data, 2, 6, 0), "load")
    assert e.value.status == q.ERR_SHAPE
    with pytest.raises(q.QpeError) as e:
        plan.run()
    assert e.value.status == q.ERR_STATE
    plan.load(U, U[0].copy())
    with pytest.raises(q.QpeError) as e:
        plan.run_stages(q.STAGE_SWEEP, q.STAGE_SWEEP)
    assert e.value.status == q.ERR_STATE
    with pytest.raises(q.QpeError) as e:
        plan.probs()
    assert e.value.status == q.ERR_STATE


# ------------------------------------------------- full-size workloads
def _fejer_sample(inst, P, tol, am):
    N = inst.N
    rng = np.random.default_rng(4242)
    ref_am = int(np.argmax(fejer.probabilities(inst.phases, inst.weights, inst.nmeas,
                                               y=np.arange(N)))) if N <= (1 << 22) else None
    top = np.argsort(P)[-64:] if N <= (1 << 24) else None
    ys = rng.integers(0, N, 4096)
    if top is not None:
        ys = np.concatenate([ys, top])
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas, y=ys)
    assert np.abs(P[ys] - Q).max() <= tol
    if ref_am is not None:
        assert am == ref_am


def test_c3_complex64_vs_fejer(q):
    """Nmat = 12, Nmeas = 20 (32 qubits, 32 GiB complex64 state)."""
    inst = W.c3()
    plan, P, am, pa, pm = run_plan(q, inst, q.C64_FP32)
    _fejer_sample(inst, P, 1e-5, am)
    # the most probable outcome: the closed form's maximum lies next to N phi_0
    y0 = int(np.floor(inst.N * inst.phases[0]))
    cand = [(y0 + k) % inst.N for k in (-1, 0, 1, 2)]
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas, y=np.array(cand))
    assert am == cand[int(np.argmax(Q))]


@pytest.mark.parametrize("prec,nmeas", [(1, 30), (0, 30)])
def test_c5_vs_fejer(q, prec, nmeas):
    """Nmat = 4, superposition input (Dirichlet weights): the histogram is the
    weighted sum of Fejer kernels, at full size (34 qubits) on the complex64
    and on the FP64 path, in the launch configuration the benchmark times."""
    import torch
    inst = W.c5(nmeas)
    plan = q.Plan(inst.nmat, inst.nmeas, prec)
    plan.load(inst.U, inst.psi)
    plan.run()
    out = torch.empty(inst.N, dtype=torch.float64, device="cuda")
    _, am, pa, pm = plan.probs(out)
    N = inst.N
    rng = np.random.default_rng(5)
    ys = np.concatenate([rng.integers(0, N, 1 << 16),
                         np.floor(N * inst.phases).astype(np.int64) % N,
                         (np.floor(N * inst.phases).astype(np.int64) + 1) % N])
    got = out[torch.from_numpy(ys).cuda()].cpu().numpy()
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas, y=ys)
    tol = TOL[prec] if prec == 1 else fp64_floor(inst)
    assert np.abs(got - Q).max() <= tol
    # argmax: the closed form's maximum lies in the bins next to some N phi_j
    y0 = np.floor(N * inst.phases).astype(np.int64)
    cand = np.unique(np.concatenate([(y0 + k) % N for k in (-1, 0, 1, 2)]))
    Qc = fejer.probabilities(inst.phases, inst.weights, inst.nmeas, y=cand)
    order = np.argsort(Qc)
    if Qc[order[-1]] - Qc[order[-2]] > 10 * tol:
        assert am == cand[order[-1]]
    total = float(out.sum().item())
    assert abs(total - 1.0) <= (1e-4 if prec == 1 else 1e-8)
    del out
    plan.close()
    del plan
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nmat,nmeas", [(11, 4), (12, 3)])
def test_largest_target_registers_vs_oracle(q, prec, nmat, nmeas):
    """Nmat = 11 and 12 (d = 2048, 4096: the plain schedule with the doubling
    GEMMs of the largest U) against the gate-by-gate oracle, whole histogram,
    superposition input."""
    rng = np.random.default_rng(31 * nmat + nmeas)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    plan, P, am, pa, pm = run_plan(q, inst, prec)
    ref = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    assert np.abs(P - ref).max() <= TOL[prec]
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 10 * TOL[prec]:
        assert am == readout.argmax_lowest(ref)
    assert abs(pm - readout.phase_weighted_mean(ref)) <= (1e-9 if prec == 0 else 2e-5)


def fp64_floor(inst):
    """The FP64 floor of a constructed input against its closed form: U =
    V diag V^dagger carries rounding of ~u sqrt(d) per eigenphase, which the
    readout multiplies by N (U^(2^(n-1)) turns a phase error delta into
    2^(n-1) delta)."""
    return max(1e-10, 2 * inst.N * U64 * np.sqrt(inst.d))


def test_c3_fp64_vs_fejer(q):
    """C3 (Nmat = 12, Nmeas = 20, 32 qubits, 64 GiB complex128 state) on the
    all-FP64 path, every bin against the closed form, to the input's FP64
    floor."""
    import torch
    inst = W.c3()
    plan, P, am, pa, pm = run_plan(q, inst, q.FP64)
    Q = fejer.probabilities(inst.phases, inst.weights, inst.nmeas)
    tol = fp64_floor(inst)
    assert np.abs(P - Q).max() <= tol
    order = np.argsort(Q)
    if Q[order[-1]] - Q[order[-2]] > 10 * tol:
        assert am == order[-1]
    assert abs(pm - readout.phase_weighted_mean(Q)) <= 1e-8
    plan.close()
    del plan
    torch.cuda.empty_cache()


# ------------------------------------------------ paper-faithful variants
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("nmat,nmeas", [(2, 6), (3, 9), (5, 8)])
def test_repeated_u_gates(q, prec, nmat, nmeas):
    """Controlled-U applied 2^k times per measurement qubit (no squaring, the
    construction Sec. 4.1's cost argument assumes) gives the same
    distribution as the oracle."""
    rng = np.random.default_rng(nmat + 3 * nmeas)
    inst = W.haar_instance(rng, nmat, nmeas, superposition=True)
    plan = q.Plan(nmat, nmeas, prec, 0x1 | 0x20)
    plan.load(inst.U, inst.psi)
    plan.run()
    P, am, _, _ = plan.probs()
    ref = gates.qpe_probabilities(inst.U, inst.psi, nmeas)
    assert np.abs(P - ref).max() <= TOL[prec]
    top2 = np.sort(ref)[-2:]
    if top2[1] - top2[0] > 10 * TOL[prec]:
        assert am == readout.argmax_lowest(ref)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("flags", [0, 0x1, 0x8])
def test_paper_analytic_family(q, prec, flags):
    """The analytic problem of Sec. 3 (phases j / 2^Nmat, non-unitary
    U = P Lambda P^-1, eigenvector x_j as input): probability 1 at
    y = j 2^(Nmeas - Nmat), as the golden cases state."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_exact_phases.txt")
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        nmat, nmeas, j, y, p = (int(v) if i < 4 else float(v) for i, v in enumerate(line.split()))
        inst = W.analytic_instance(nmat, nmeas, j)
        plan = q.Plan(nmat, nmeas, prec, flags)
        plan.load(inst.U, inst.psi)
        plan.run()
        P, am, _, _ = plan.probs()
        assert am == y
        assert abs(P[y] - p) <= (1e-10 if prec == 0 else 2e-5)


def test_host_buffers_from_the_library(q):
    """qpe.host_array (qpe_host_alloc, page-locked) as the host side of
    qpe_load and qpe_probs: the same histogram and readout as numpy buffers."""
    rng = np.random.default_rng(91)
    inst = W.haar_instance(rng, 3, 12, superposition=True)
    U_h = q.host_array(inst.U.shape, np.complex128)
    U_h[...] = inst.U
    psi_h = q.host_array(inst.psi.shape, np.complex128)
    psi_h[...] = inst.psi
    hist_h = q.host_array(inst.N, np.float64)
    plan = q.Plan(inst.nmat, inst.nmeas, q.FP64)
    plan.load(U_h, psi_h)
    plan.run()
    _, am, pa, pm = plan.probs(hist_h)
    P, am2, pa2, pm2 = plan.probs()
    assert np.array_equal(hist_h, P) and (am, pa, pm) == (am2, pa2, pm2)
    assert np.abs(P - gates.qpe_probabilities(inst.U, inst.psi, inst.nmeas)).max() <= 1e-10
    del hist_h, U_h, psi_h
