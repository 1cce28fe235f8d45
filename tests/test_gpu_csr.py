"""Parity of the general sparse operator kind (PXA_CSR: dq/dt = A q, RK4, initial-condition
control, J = 0.5 ||q(T) - g||^2), of the terminal objective's target on the 1D
advection-diffusion problem, and of FP32 stepping of that problem, with the CPU oracle.

Tolerances: FP64 paths 1e-10 (element-wise, tests/parity.py); Paraexp with the RK4
stepper's own propagator reproduces serial stepping up to the Krylov tolerance (held to
1e-10 against the oracle's serial stepping); FP32 stepping of K = 512 CN steps 1e-4
(K u_32 = 3e-5)."""
import numpy as np
import pytest

import oracle as O
from paper_2004_00546_gb300 import inputs as I
from parity import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X(cuda_ok):
    from paper_2004_00546_gb300 import pxa

    return pxa


@pytest.fixture(scope="module")
def torch():
    import torch as t

    return t


def dev(torch, a, dtype=None):
    import torch as t

    return t.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def csr_ctx(X, torch, rp, col, val, T, K, P, phi, m=30, sub=1):
    ctx = X.Context()
    keep = (dev(torch, rp, torch.int64), dev(torch, col, torch.int32), dev(torch, val, torch.float64))
    ctx.set_operator_csr(*keep)
    ctx.set_time(T, K, X.RK4, P)
    ctx.set_krylov(m, 1e-12, phi, sub)
    return ctx, keep


def adv2d_csr(n, nu):
    """The 2D advection-diffusion operator of Sec. 4.2 (5-point stencil, a seeded
    divergence-free velocity) in CSR form, its columns taken from the oracle's operator."""
    u, v = I.streamfunction_velocity(n, n, 3, 77)
    N = n * n
    cols = [O.ad2_apply(e.reshape(n, n), u, v, nu).reshape(-1) for e in np.eye(N)]
    D = np.stack(cols, 1)
    rp, col, val = [0], [], []
    for r in range(N):
        nz = np.nonzero(D[r])[0]
        col.extend(nz.tolist())
        val.extend(D[r, nz].tolist())
        rp.append(len(col))
    return np.array(rp, np.int64), np.array(col, np.int32), np.array(val)


CASES = {
    "random_n200": lambda: (I.sparse_operator(200, 4, 901), 0.5, 400, 8),
    "ragged_n37": lambda: (I.sparse_operator(37, 1, 902), 0.3, 60, 3),
    "adv2d_16sq": lambda: (adv2d_csr(16, 2e-2), 0.4, 256, 4),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("target", [False, True])
def test_csr_gradient_matches_oracle(X, torch, case, target):
    (rp, col, val), T, K, P = CASES[case]()
    n = rp.size - 1
    q0 = I.grf_k2(max(n, 16), 33)[:n]
    g = I.grf_k2(max(n, 16), 34)[:n] if target else None
    Js, gs, _ = O.csr_gradient_serial(rp, col, val, q0, T, K, g)
    Je, ge, _ = O.csr_gradient_paraexp(rp, col, val, q0, T, K, P, O.CSR_PHI_EXP, g)
    for phi, ref in ((X.PHI_STEPPER, (Js, gs)), (X.PHI_EXP, (Je, ge))):
        ctx, keep = csr_ctx(X, torch, rp, col, val, T, K, P, phi, sub=2 if phi == X.PHI_EXP else 1)
        qd = dev(torch, q0, torch.float64)
        ctx.set_control(qd)
        if target:
            gd = dev(torch, g, torch.float64)
            ctx.set_objective(X.OBJ_TERMINAL_L2, gd)
        out = torch.empty_like(qd)
        for mode in (X.PARAEXP, X.SERIAL):
            J = ctx.gradient(mode, out)
            Jr, gr = (Js, gs) if mode == X.SERIAL else ref
            assert abs(J - Jr) / Jr < 1e-10, (case, phi, mode)
            assert rel(out.cpu().numpy(), gr) < 1e-10, (case, phi, mode)
        assert ctx.stats()["krylov_err_max"] <= 1e-12
        ctx.close()


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("target", [False, True])
def test_csr_series_chain_matches_serial_stepping(X, torch, case, target):
    """PXA_PROP_POLY: both chains carry the summed homogeneous problems with the RK4 stepper's
    segment propagator as its power series in kk dt A (A^T for the adjoint), cut where the
    max-norm tail bound falls below 1e-12: Paraexp equals the oracle's serial stepping to
    1e-10 point by point, with operator products only (no inner products)."""
    (rp, col, val), T, K, P = CASES[case]()
    n = rp.size - 1
    q0 = I.grf_k2(max(n, 16), 33)[:n]
    g = I.grf_k2(max(n, 16), 34)[:n] if target else None
    Js, gs, _ = O.csr_gradient_serial(rp, col, val, q0, T, K, g)
    ctx, keep = csr_ctx(X, torch, rp, col, val, T, K, P, X.PHI_STEPPER)
    ctx.set_propagator(X.PROP_POLY, 200)
    qd = dev(torch, q0, torch.float64)
    ctx.set_control(qd)
    if target:
        ctx.set_objective(X.OBJ_TERMINAL_L2, dev(torch, g, torch.float64))
    out = torch.empty_like(qd)
    J = ctx.gradient(X.PARAEXP, out)
    st = ctx.stats()
    assert st["prop_degree"] > 0 and st["prop_tail"] <= 1e-12, st
    assert abs(J - Js) / Js < 1e-10, (case, J, Js)
    assert rel(out.cpu().numpy(), gs) < 1e-10, case
    ctx.close()


def test_csr_series_chain_segments_and_global_workspace(X, torch):
    """n = 8000 (the chain's three vectors exceed a block's shared memory) and subintervals
    long enough that the series runs in several segments per subinterval."""
    rp, col, val = I.sparse_operator(8000, 4, 903)
    T, K, P = 1.6, 512, 4
    q0 = np.sin(np.arange(8000) * 0.01)
    Js, gs, _ = O.csr_gradient_serial(rp, col, val, q0, T, K)
    ctx, keep = csr_ctx(X, torch, rp, col, val, T, K, P, X.PHI_STEPPER, m=24)
    ctx.set_propagator(X.PROP_POLY, 200)
    qd = dev(torch, q0, torch.float64)
    ctx.set_control(qd)
    out = torch.empty_like(qd)
    J = ctx.gradient(X.PARAEXP, out)
    st = ctx.stats()
    assert st["prop_substeps"] > 1, st
    assert abs(J - Js) / Js < 1e-10 and rel(out.cpu().numpy(), gs) < 1e-10
    ctx.close()


def test_csr_lanes_in_global_memory_and_graph_replay(X, torch):
    """n = 8000: a lane's four vectors exceed a block's shared memory, so the lanes step
    in a global workspace; Paraexp with the stepper propagator against serial stepping of
    the oracle, launched one by one and as graph replays (bit-identical)."""
    rp, col, val = I.sparse_operator(8000, 4, 903)
    T, K, P = 0.2, 64, 4
    q0 = np.sin(np.arange(8000) * 0.01)
    Js, gs, _ = O.csr_gradient_serial(rp, col, val, q0, T, K)
    ctx, keep = csr_ctx(X, torch, rp, col, val, T, K, P, X.PHI_STEPPER, m=24)
    qd = dev(torch, q0, torch.float64)
    ctx.set_control(qd)
    res = []
    for graph in (False, True):
        ctx.set_graph(graph)
        out = torch.empty_like(qd)
        J = ctx.gradient(X.PARAEXP, out)
        assert abs(J - Js) / Js < 1e-10 and rel(out.cpu().numpy(), gs) < 1e-10
        res.append(out.cpu().numpy())
    assert np.array_equal(res[0], res[1])
    ctx.close()


def test_csr_split_solves_equal_the_gradient(X, torch):
    (rp, col, val), T, K, P = CASES["random_n200"]()
    q0 = I.grf_k2(200, 35)
    ctx, keep = csr_ctx(X, torch, rp, col, val, T, K, P, X.PHI_STEPPER)
    qd = dev(torch, q0, torch.float64)
    ctx.set_control(qd)
    g1, g2 = torch.empty_like(qd), torch.empty_like(qd)
    J1 = ctx.gradient(X.PARAEXP, g1)
    J2 = ctx.solve_direct(X.PARAEXP)
    ctx.solve_adjoint(X.PARAEXP, g2)
    assert J1 == J2 and torch.equal(g1, g2)
    ctx.close()


def test_terminal_target_on_advdiff1d(X, torch):
    """J = 0.5 ||q(T) - g||^2 on the 1D advection-diffusion problem: the oracle's q(T) and
    gradient without a target, minus (M^K)^T g by the oracle's exact DFT CN power."""
    n, c, nu, T, K, P = 128, 1.0, 0.01, 0.5, 512, 4
    q0 = I.grf_k2(n, 36)
    g = I.grf_k2(n, 37)
    _, g0, qT = O.ad1_cn_gradient_serial(q0, c, nu, T, K)
    Jr = 0.5 * np.sum((qT - g) ** 2)
    gr = g0 - O.ad1_phi_dft(g, c, nu, O.PHI_CN, dt=T / K, steps=K, transpose=True)
    for prop in (X.PROP_KRYLOV, X.PROP_BAND):
        ctx = X.Context()
        ctx.set_operator(X.ADVDIFF_1D, n, c=c, nu=nu)
        ctx.set_time(T, K, X.CN, P)
        ctx.set_krylov(30, 1e-12, X.PHI_STEPPER, 1)
        ctx.set_propagator(prop, 150)
        qd, gd = dev(torch, q0, torch.float64), dev(torch, g, torch.float64)
        ctx.set_control(qd)
        ctx.set_objective(X.OBJ_TERMINAL_L2, gd)
        out = torch.empty_like(qd)
        for mode in (X.PARAEXP, X.SERIAL):
            J = ctx.gradient(mode, out)
            assert abs(J - Jr) / Jr < 1e-10 and rel(out.cpu().numpy(), gr) < 1e-10, (prop, mode)
        ctx.close()


def test_objective_kinds_follow_the_operator(X, torch):
    ctx = X.Context()
    with pytest.raises(X.PxaError) as ei:
        ctx.set_objective(X.OBJ_TERMINAL_L2)
    assert ei.value.code == X.ERR_STATE
    ctx.set_operator(X.BURGERS_1D, 64, nu=0.01)
    with pytest.raises(X.PxaError):
        ctx.set_objective(X.OBJ_TERMINAL_L2)
    with pytest.raises(X.PxaError):
        ctx.set_objective(X.OBJ_INTEGRAL_TRACKING)  # needs a target
    ctx.set_objective(X.OBJ_INTEGRAL_TRACKING, torch.zeros(64, dtype=torch.float64, device="cuda"))
    with pytest.raises(X.PxaError):
        ctx.set_precision(X.F32)  # Burgers steps in FP64 only
    ctx.set_operator(X.ADVDIFF_1D, 64, c=1.0, nu=0.01)
    with pytest.raises(X.PxaError):
        ctx.set_objective(X.OBJ_INTEGRAL_TRACKING, torch.zeros(64, dtype=torch.float64, device="cuda"))
    ctx.close()


@pytest.mark.parametrize("phi", ["stepper", "exp"])
def test_advdiff1d_fp32_stepping_matches_oracle(X, torch, phi):
    """pxa_set_precision(F32) on the 1D advection-diffusion problem (FP32 lanes, FP64
    superposition): J and the gradient within the FP32 tolerance of the FP64 oracle
    (serial CN for serial stepping and for the stepper's propagator, the oracle's Paraexp
    with exp(tau A) for the exponential)."""
    n, c, nu, T, K, P = 256, 1.0, 0.01, 1.0, 512, 8
    q0 = I.grf_k2(n, 38)
    Js, gs, _ = O.ad1_cn_gradient_serial(q0, c, nu, T, K)
    Je, ge, _ = O.ad1_cn_gradient_paraexp(q0, c, nu, T, K, P, O.PHI_EXP)
    ctx = X.Context()
    ctx.set_operator(X.ADVDIFF_1D, n, c=c, nu=nu)
    ctx.set_time(T, K, X.CN, P)
    ctx.set_krylov(30, 1e-8, X.PHI_STEPPER if phi == "stepper" else X.PHI_EXP, 1)
    ctx.set_precision(X.F32)
    qd = dev(torch, q0, torch.float64)
    ctx.set_control(qd)
    out = torch.empty_like(qd)
    for mode in (X.PARAEXP, X.SERIAL):
        J = ctx.gradient(mode, out)
        Jr, gr = (Js, gs) if (mode == X.SERIAL or phi == "stepper") else (Je, ge)
        assert abs(J - Jr) / Jr < 1e-4 and rel(out.cpu().numpy(), gr) < 1e-4, (phi, mode)
    with pytest.raises(X.PxaError):
        ctx.solve_direct(X.PARAEXP)
    # the FP64 path of the same context after switching back
    ctx.set_precision(X.F64)
    J = ctx.gradient(X.SERIAL, out)
    assert abs(J - Js) / Js < 1e-10 and rel(out.cpu().numpy(), gs) < 1e-10
    ctx.close()
