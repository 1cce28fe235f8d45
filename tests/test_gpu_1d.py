"""Parity of the CUDA path (through the C ABI) with the CPU oracle, 1D problems.

Tolerances: FP64 throughout; the CUDA path must match the oracle within 1e-10
relative (the gradient, J and building blocks), and Paraexp with the stepper's own
propagator must match serial stepping within 1e-8 (the accuracy gate of the
benchmark). Building blocks that involve no long recursions are held to 1e-13.
"""
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


def dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def ad1_ctx(X, n, c, nu, T, K, P, m=30, tol=1e-11, phi=None, sub=1):
    ctx = X.Context()
    ctx.set_operator(X.ADVDIFF_1D, n, c=c, nu=nu)
    ctx.set_time(T, K, X.CN, P)
    ctx.set_krylov(m, tol, X.PHI_STEPPER if phi is None else phi, sub)
    return ctx


# ---- building blocks ----------------------------------------------------------------
@pytest.mark.parametrize("n", [3, 31, 256, 1000, 4096])
def test_apply_operator_matches_oracle(X, torch, n):
    ctx = ad1_ctx(X, n, 1.0, 0.01, 1.0, 16, 1)
    x = I.grf_k2(max(n, 4), 3)[:n] if n >= 4 else np.array([0.3, -1.0, 2.0])
    xd = dev(torch, x)
    y = torch.empty_like(xd)
    for tr in (False, True):
        ctx.apply_operator(xd, y, transpose=tr)
        ref = O.ad1_apply(x, 1.0, 0.01, transpose=tr)
        assert rel(host(y), ref) < 1e-13


@pytest.mark.parametrize("n,steps", [(31, 7), (256, 100), (1000, 33)])
def test_cn_step_matches_oracle(X, torch, n, steps):
    T, K = 1.0, 4096
    ctx = ad1_ctx(X, n, 1.0, 0.01, T, K, 1)
    x = I.grf_k2(n if n % 2 == 0 else n + 1, 5)[:n]
    xd = dev(torch, x)
    y = torch.empty_like(xd)
    for tr in (False, True):
        ctx.step(xd, y, steps, transpose=tr)
        ref = x.copy()
        for _ in range(steps):
            ref = O.ad1_cn_step_T(ref, 1.0, 0.01, T / K) if tr else O.ad1_cn_step(ref, 1.0, 0.01, T / K)
        assert rel(host(y), ref) < 1e-12


@pytest.mark.parametrize("phi", ["exp", "stepper"])
@pytest.mark.parametrize("sub", [1, 4])
def test_krylov_expv_matches_exact_propagator(X, torch, phi, sub):
    n, c, nu, T, K = 256, 1.0, 0.01, 1.0, 4096
    ctx = ad1_ctx(X, n, c, nu, T, K, 8, m=30, tol=1e-10,
                  phi=X.PHI_EXP if phi == "exp" else X.PHI_STEPPER)
    v = I.grf_k2(n, 9)
    span = 512
    xd = dev(torch, v)
    y = torch.empty_like(xd)
    for tr in (False, True):
        err = ctx.expv(xd, y, span, substeps=sub, transpose=tr)
        if phi == "exp":
            ref = O.ad1_phi_dft(v, c, nu, O.PHI_EXP, t=span * T / K, transpose=tr)
        else:
            ref = O.ad1_phi_dft(v, c, nu, O.PHI_CN, dt=T / K, steps=span, transpose=tr)
        assert rel(host(y), ref) < 1e-10
        assert err < 1e-10


def test_krylov_not_converged_is_reported(X, torch):
    """A Krylov space far too small for the span must come back as NOT_CONVERGED,
    raised on the host from the device status word (no fault, context stays usable)."""
    n = 256
    ctx = ad1_ctx(X, n, 1.0, 0.01, 1.0, 4096, 1, m=3, tol=1e-12, phi=X.PHI_EXP)
    xd = dev(torch, I.grf_k2(n, 1))
    y = torch.empty_like(xd)
    with pytest.raises(X.PxaError) as ei:
        ctx.expv(xd, y, 4096)
    assert ei.value.code == X.ERR_NOT_CONVERGED
    ctx.set_krylov(30, 1e-10, X.PHI_EXP, 1)
    ctx.expv(xd, y, 64)  # the same context keeps working


# ---- full direct-adjoint loops, 1D advection-diffusion --------------------------------
C1 = dict(n=256, c=1.0, nu=0.01, T=1.0, K=4096, P=8, m=30)


@pytest.fixture(scope="module")
def c1_oracle():
    p = I.advdiff1d_problem()
    J, g, qT = O.ad1_cn_gradient_serial(p["q0"], p["c"], p["nu"], p["T"], C1["K"])
    return p, J, g


def test_c1_serial_matches_oracle(X, torch, c1_oracle):
    p, J, g = c1_oracle
    ctx = ad1_ctx(X, C1["n"], C1["c"], C1["nu"], C1["T"], C1["K"], C1["P"])
    q0 = dev(torch, p["q0"])
    ctx.set_control(q0)
    gd = torch.empty_like(q0)
    Jg = ctx.gradient(X.SERIAL, gd)
    assert abs(Jg - J) / J < 1e-10
    assert rel(host(gd), g) < 1e-10


@pytest.mark.parametrize("sub", [1, 2])
def test_c1_paraexp_stepper_matches_serial_and_oracle(X, torch, c1_oracle, sub):
    p, J, g = c1_oracle
    ctx = ad1_ctx(X, C1["n"], C1["c"], C1["nu"], C1["T"], C1["K"], C1["P"], m=C1["m"], sub=sub)
    q0 = dev(torch, p["q0"])
    ctx.set_control(q0)
    gd = torch.empty_like(q0)
    Jg = ctx.gradient(X.PARAEXP, gd)
    # accuracy gate against serial stepping
    assert abs(Jg - J) / J < 1e-8
    assert rel(host(gd), g) < 1e-8
    # against the oracle's Paraexp with the exact stepper propagator
    Jo, go, _ = O.ad1_cn_gradient_paraexp(p["q0"], p["c"], p["nu"], p["T"], C1["K"], C1["P"], O.PHI_CN)
    assert abs(Jg - Jo) / Jo < 1e-10
    assert rel(host(gd), go) < 1e-10


def test_c1_paraexp_exp_matches_oracle(X, torch, c1_oracle):
    p, _, _ = c1_oracle
    ctx = ad1_ctx(X, C1["n"], C1["c"], C1["nu"], C1["T"], C1["K"], C1["P"], m=30, phi=X.PHI_EXP)
    q0 = dev(torch, p["q0"])
    ctx.set_control(q0)
    gd = torch.empty_like(q0)
    Jg = ctx.gradient(X.PARAEXP, gd)
    Jo, go, _ = O.ad1_cn_gradient_paraexp(p["q0"], p["c"], p["nu"], p["T"], C1["K"], C1["P"], O.PHI_EXP)
    assert abs(Jg - Jo) / Jo < 1e-10
    assert rel(host(gd), go) < 1e-10


@pytest.mark.parametrize("n,K,P,nu,sub", [(1000, 1000, 5, 0.002, 4), (37, 60, 3, 0.02, 1),
                                          (256, 512, 1, 0.01, 1), (2048, 256, 16, 1e-4, 1)])
def test_c1_ragged_sizes(X, torch, n, K, P, nu, sub):
    c, T = 0.8, 0.5
    q0 = I.grf_k2(n + (n % 2), 77)[:n]
    J, g, _ = O.ad1_cn_gradient_serial(q0, c, nu, T, K)
    ctx = ad1_ctx(X, n, c, nu, T, K, P, m=40, tol=1e-10, sub=sub)
    qd = dev(torch, q0)
    ctx.set_control(qd)
    gd = torch.empty_like(qd)
    Js = ctx.gradient(X.SERIAL, gd)
    assert abs(Js - J) / J < 1e-10 and rel(host(gd), g) < 1e-10
    Jp = ctx.gradient(X.PARAEXP, gd)
    assert abs(Jp - J) / J < 1e-8 and rel(host(gd), g) < 1e-8


def test_c1_graph_replay_and_host_entry(X, torch, c1_oracle):
    p, J, g = c1_oracle
    ctx = ad1_ctx(X, C1["n"], C1["c"], C1["nu"], C1["T"], C1["K"], C1["P"])
    q0 = dev(torch, p["q0"])
    ctx.set_control(q0)
    g1 = torch.empty_like(q0)
    J1 = ctx.gradient(X.PARAEXP, g1)
    ctx.set_graph(True)
    g2 = torch.empty_like(q0)
    J2 = ctx.gradient(X.PARAEXP, g2)
    J3 = ctx.gradient(X.PARAEXP, g2)  # replay of the captured graph
    assert J1 == J2 == J3
    assert torch.equal(g1, g2)
    # the captured graph's kernel nodes: at least the lanes, the chain and a superposition
    # in each direction
    assert ctx.stats()["graph_kernels"] >= 6
    gh = np.empty(C1["n"])
    Jh = ctx.gradient_host(X.PARAEXP, np.ascontiguousarray(p["q0"]), gh)
    assert Jh == J1
    assert np.array_equal(gh, host(g1))


def test_c1_autotune_keeps_parity(X, torch, c1_oracle):
    p, J, g = c1_oracle
    ctx = ad1_ctx(X, C1["n"], C1["c"], C1["nu"], C1["T"], C1["K"], C1["P"])
    q0 = dev(torch, p["q0"])
    ctx.set_control(q0)
    gd = torch.empty_like(q0)
    ms = ctx.autotune(X.PARAEXP, gd)
    assert ms > 0
    st = ctx.stats()
    assert st["krylov_m"] in (16, 20, 24, 30, 36, 40) and st["krylov_substeps"] in (1, 2, 4, 8)
    Jg = ctx.gradient(X.PARAEXP, gd)
    assert abs(Jg - J) / J < 1e-8 and rel(host(gd), g) < 1e-8


def test_split_solves_match_gradient_and_check_order(X, torch, c1_oracle):
    p, J, g = c1_oracle
    ctx = ad1_ctx(X, C1["n"], C1["c"], C1["nu"], C1["T"], C1["K"], C1["P"])
    q0 = dev(torch, p["q0"])
    ctx.set_control(q0)
    gd = torch.empty_like(q0)
    with pytest.raises(X.PxaError) as ei:
        ctx.solve_adjoint(X.PARAEXP, gd)
    assert ei.value.code == X.ERR_STATE
    for mode in (X.SERIAL, X.PARAEXP):
        Jd = ctx.solve_direct(mode)
        ctx.solve_adjoint(mode, gd)
        g2 = torch.empty_like(q0)
        Jf = ctx.gradient(mode, g2)
        assert Jd == Jf and torch.equal(gd, g2)
    ctx.solve_direct(X.SERIAL)
    with pytest.raises(X.PxaError):
        ctx.solve_adjoint(X.PARAEXP, gd)  # mode mismatch


# ---- 1D viscous Burgers ------------------------------------------------------------------
def bu1_ctx(X, n, nu, T, K, P, M=25, m=30, tol=1e-10, phi=None, memory=None):
    ctx = X.Context()
    ctx.set_operator(X.BURGERS_1D, n, nu=nu)
    ctx.set_time(T, K, X.RK4, P)
    ctx.set_krylov(m, tol, X.PHI_EXP if phi is None else phi, 1)
    if phi is None or phi == X.PHI_EXP:
        ctx.set_magnus(M)
    if memory is not None:
        ctx.set_memory(memory)
    return ctx


@pytest.mark.parametrize("n", [3, 64, 1000])
def test_burgers_building_blocks(X, torch, n):
    ctx = bu1_ctx(X, n, 0.01, 1.0, 100, 1)
    rng = np.random.default_rng(n)
    u, x = rng.standard_normal(n), rng.standard_normal(n)
    ud, xd = dev(torch, u), dev(torch, x)
    y = torch.empty_like(ud)
    ctx.burgers_rhs(ud, y)
    assert rel(host(y), O.bu1_rhs(u, 0.01)) < 1e-13
    ctx.burgers_jac_T(ud, xd, y)
    assert rel(host(y), O.bu1_jac(u, x, 0.01, transpose=True)) < 1e-13


@pytest.fixture(scope="module")
def bu_small():
    n, nu, T, K = 200, 0.01, 0.3, 600
    f = 3.0 * I.fourier1d(n, 8, 61)
    g = I.fourier1d(n, 8, 62)
    J, grad = O.bu1_gradient_serial(f, g, nu, T, K)
    return dict(n=n, nu=nu, T=T, K=K, f=f, g=g, J=J, grad=grad)


@pytest.mark.parametrize("memory", ["full", "checkpoints"])
def test_burgers_serial_matches_oracle(X, torch, bu_small, memory):
    b = bu_small
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], 6,
                  memory=X.STORE_FULL if memory == "full" else X.STORE_CHECKPOINTS)
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    J = ctx.gradient(X.SERIAL, out)
    assert abs(J - b["J"]) / b["J"] < 1e-10
    assert rel(host(out), b["grad"]) < 1e-10


@pytest.mark.parametrize("memory", ["full", "checkpoints"])
@pytest.mark.parametrize("P", [1, 6, 20])
def test_burgers_paraexp_stepper_chain_is_exact(X, torch, bu_small, memory, P):
    b = bu_small
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], P, phi=X.PHI_STEPPER,
                  memory=X.STORE_FULL if memory == "full" else X.STORE_CHECKPOINTS)
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    J = ctx.gradient(X.PARAEXP, out)
    assert abs(J - b["J"]) / b["J"] < 1e-10
    assert rel(host(out), b["grad"]) < 1e-10


@pytest.mark.parametrize("memory", ["full", "checkpoints"])
def test_burgers_paraexp_magnus_matches_oracle(X, torch, bu_small, memory):
    b = bu_small
    P, M, m = 6, 10, 30
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], P, M=M, m=m,
                  memory=X.STORE_FULL if memory == "full" else X.STORE_CHECKPOINTS)
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    J = ctx.gradient(X.PARAEXP, out)
    Jo, go = O.bu1_gradient_hybrid(b["f"], b["g"], b["nu"], b["T"], b["K"], P, O.HOM_MAGNUS, M, m)
    assert abs(J - Jo) / Jo < 1e-10
    assert rel(host(out), go) < 1e-10
    # the Magnus approximation itself stays close to serial stepping at this step size
    assert rel(host(out), b["grad"]) < 1e-6


@pytest.mark.parametrize("C", [1, 2, 3, 8, 16])
def test_burgers_cluster_sizes(X, torch, bu_small, C):
    """Every cluster size gives the same gradient; n = 200 with C = 16 leaves a last
    chunk (5 points) smaller than the reverse step's halo, so halos span two CTAs."""
    b = bu_small
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], 6, phi=X.PHI_STEPPER)
    ctx.set_cluster(C, C, C)
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    for mode in (X.SERIAL, X.PARAEXP):
        J = ctx.gradient(mode, out)
        assert abs(J - b["J"]) / b["J"] < 1e-10
        assert rel(host(out), b["grad"]) < 1e-10


def test_burgers_cluster_checkpoint_recompute(X, torch, bu_small):
    b = bu_small
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], 6, phi=X.PHI_STEPPER, memory=X.STORE_CHECKPOINTS)
    ctx.set_cluster(4, 3, 4)
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    J = ctx.gradient(X.PARAEXP, out)
    assert abs(J - b["J"]) / b["J"] < 1e-10
    assert rel(host(out), b["grad"]) < 1e-10


def test_burgers_autotune_and_split_solves(X, torch, bu_small):
    b = bu_small
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], 6, phi=X.PHI_STEPPER)
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    assert ctx.autotune(X.PARAEXP, out) > 0
    J = ctx.solve_direct(X.PARAEXP)
    ctx.solve_adjoint(X.PARAEXP, out)
    assert abs(J - b["J"]) / b["J"] < 1e-10
    assert rel(host(out), b["grad"]) < 1e-10


# ---- full size 1D Burgers (n = 1024, K = 20000, P = 32) ---------------------------------
@pytest.fixture(scope="module")
def bu_full():
    p = I.burgers1d_problem()
    J, grad = O.bu1_gradient_serial(p["f"], p["g"], p["nu"], p["T"], 20000)
    return dict(p=p, J=J, grad=grad)


def test_burgers_full_size_serial_and_stepper_paraexp(X, torch, bu_full):
    p = bu_full["p"]
    ctx = bu1_ctx(X, 1024, p["nu"], p["T"], 20000, 32, phi=X.PHI_STEPPER)
    fd, gd_ = dev(torch, p["f"]), dev(torch, p["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    J = ctx.gradient(X.SERIAL, out)
    assert abs(J - bu_full["J"]) / bu_full["J"] < 1e-10
    assert rel(host(out), bu_full["grad"]) < 1e-10
    J = ctx.gradient(X.PARAEXP, out)
    assert abs(J - bu_full["J"]) / bu_full["J"] < 1e-10
    assert rel(host(out), bu_full["grad"]) < 1e-10


def test_burgers_full_size_magnus_matches_oracle(X, torch, bu_full):
    p = bu_full["p"]
    M, m = 25, 20
    ctx = bu1_ctx(X, 1024, p["nu"], p["T"], 20000, 32, M=M, m=m, tol=1e-9)
    fd, gd_ = dev(torch, p["f"]), dev(torch, p["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    J = ctx.gradient(X.PARAEXP, out)
    Jo, go = O.bu1_gradient_hybrid(p["f"], p["g"], p["nu"], p["T"], 20000, 32, O.HOM_MAGNUS, M, 30)
    assert abs(J - Jo) / Jo < 1e-10
    assert rel(host(out), go) < 1e-9


@pytest.mark.parametrize("impl", ["banded", "banded_pair", "banded_single", "restep"])
@pytest.mark.parametrize("memory", ["full", "checkpoints"])
@pytest.mark.parametrize("P", [1, 6])
def test_burgers_adjoint_evaluations_match_oracle(X, torch, bu_small, impl, memory, P):
    """The banded adjoint (rows of M_s^T formed once per step; the chain with four-step
    products M_s^T ... M_{s+3}^T, two-step products or one step per exchange) and the
    stage-by-stage reverse sweep are the same linear map: all match the oracle's serial
    gradient, in serial and Paraexp modes, with full storage and with checkpoint
    recompute."""
    b = bu_small
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], P, phi=X.PHI_STEPPER,
                  memory=X.STORE_FULL if memory == "full" else X.STORE_CHECKPOINTS)
    ctx.set_adjoint({"banded": X.ADJ_BANDED, "banded_pair": X.ADJ_BANDED_PAIR,
                     "banded_single": X.ADJ_BANDED_SINGLE, "restep": X.ADJ_RESTEP}[impl])
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    for mode in (X.SERIAL, X.PARAEXP):
        J = ctx.gradient(mode, out)
        assert abs(J - b["J"]) / b["J"] < 1e-10
        assert rel(host(out), b["grad"]) < 1e-10
    assert ctx.stats()["adjoint_band"] == (0 if impl == "restep" else 1)


@pytest.mark.parametrize("n,C", [(3, 1), (8, 2), (64, 16), (37, 5)])
def test_burgers_banded_small_grids_and_chunks(X, torch, n, C):
    """Grids down to 3 points (one CTA whose halo wraps the periodic grid more than once)
    and clusters whose chunks hold exactly the 4-point halo, with sin(omega t) forcing."""
    nu, T, K, P = 0.05, 0.2, 120, 4
    f = I.fourier1d(n, max(1, min(8, n // 2 - 1)), 71) if n > 4 else np.array([0.3, -0.2, 0.5][:n])
    g = I.fourier1d(n, max(1, min(8, n // 2 - 1)), 72) if n > 4 else np.array([0.1, 0.4, -0.3][:n])
    J0, g0 = O.bu1_gradient_serial(f, g, nu, T, K, omega=2.0)
    ctx = bu1_ctx(X, n, nu, T, K, P, phi=X.PHI_STEPPER)
    ctx.set_cluster(1, C, C)
    fd, gd_ = dev(torch, f), dev(torch, g)
    ctx.set_control(fd, 2.0)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    for mode in (X.SERIAL, X.PARAEXP):
        J = ctx.gradient(mode, out)
        assert abs(J - J0) / J0 < 1e-10
        assert rel(host(out), g0) < 1e-10
    st = ctx.stats()
    assert st["adjoint_band"] == 1


@pytest.mark.parametrize("P,phi", [(6, "stepper"), (1, "stepper"), (6, "exp")])
def test_burgers_overlapped_phases_match_sequential(X, torch, bu_small, P, phi):
    """The chunked direct with the band records and adjoint lanes on a second stream
    (hybrid overlap) gives the gradient of the sequential schedule: the same trajectory
    bit for bit, J up to the summation order of its chunk partials."""
    b = bu_small
    ph = X.PHI_STEPPER if phi == "stepper" else X.PHI_EXP
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    res = {}
    for ov in (True, False):
        ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], P, M=10, phi=ph)
        ctx.set_overlap(ov)
        ctx.set_control(fd)
        ctx.set_target(gd_)
        out = torch.empty_like(fd)
        mode = X.SERIAL if P == 1 else X.PARAEXP
        J = ctx.gradient(mode, out)
        res[ov] = (J, host(out))
        if phi == "stepper":
            assert abs(J - b["J"]) / b["J"] < 1e-10
            assert rel(host(out), b["grad"]) < 1e-10
        ctx.close()
    assert abs(res[True][0] - res[False][0]) <= 1e-14 * abs(res[False][0])
    assert np.array_equal(res[True][1], res[False][1])


@pytest.mark.parametrize("qd,qs", [(1, 1), (2, 4), (4, 2)])
@pytest.mark.parametrize("C", [4, 16])
def test_burgers_exchange_groups(X, torch, bu_small, qd, qs, C):
    """Every number of steps per halo exchange (1, 2, 4) of the direct and of the banded
    sweeps gives the oracle's gradient; the grid of 200 points over 16 CTAs leaves chunks
    of 13 and 5 points, so the group size falls back where the 4q halo does not fit."""
    b = bu_small
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], 6, phi=X.PHI_STEPPER)
    ctx.set_cluster(C, C, C)
    ctx.set_groups(qd, qs)
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    ctx.set_control(fd, 1.5)
    ctx.set_target(gd_)
    J0, g0 = O.bu1_gradient_serial(b["f"], b["g"], b["nu"], b["T"], b["K"], omega=1.5)
    out = torch.empty_like(fd)
    for mode in (X.SERIAL, X.PARAEXP):
        J = ctx.gradient(mode, out)
        assert abs(J - J0) / J0 < 1e-10
        assert rel(host(out), g0) < 1e-10


@pytest.mark.parametrize("P", [1, 6])
def test_burgers_partition_keeps_the_gradient(X, torch, bu_small, P):
    """Geometric chunk partitions of the overlapped direct solve (Eq. nonEquiP, rounded
    to whole subintervals) change only when the adjoint work is done: the gradient is
    bit for bit that of equal chunks, J differs by the summation order of its partials,
    and both match the oracle."""
    b = bu_small
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    mode = X.SERIAL if P == 1 else X.PARAEXP
    res = []
    for r in (0.0, 0.37, 0.59, 0.9):
        ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], P, phi=X.PHI_STEPPER)
        ctx.set_partition(r)
        ctx.set_control(fd)
        ctx.set_target(gd_)
        out = torch.empty_like(fd)
        J = ctx.gradient(mode, out)
        st = ctx.stats()
        assert st["chunks"] == (8 if P == 1 else 6)
        assert abs(st["partition_r"] - r) < 1e-6
        assert abs(J - b["J"]) / b["J"] < 1e-10
        assert rel(host(out), b["grad"]) < 1e-10
        res.append((J, host(out)))
        ctx.close()
    for J, g in res[1:]:
        assert abs(J - res[0][0]) <= 1e-14 * abs(res[0][0])
        assert np.array_equal(g, res[0][1])


def test_burgers_autotune_measures_the_partition_ratio(X, torch, bu_small):
    """The autotuner's third pass measures k = tau_adj / tau_direct and keeps one of
    r = 0, k/(k+1), k or a fixed ratio; the tuned context still gives the oracle's
    gradient."""
    b = bu_small
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], 6, phi=X.PHI_STEPPER)
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    ctx.set_control(fd)
    ctx.set_target(gd_)
    out = torch.empty_like(fd)
    ctx.autotune(X.PARAEXP, out)
    st = ctx.stats()
    k = st["tau_ratio"]
    assert k > 0.0
    cands = [0.0, k / (k + 1.0)] + ([k] if k < 0.95 else []) + [0.6, 0.7, 0.8, 0.9]
    assert min(abs(st["partition_r"] - c) for c in cands) < 1e-5
    J = ctx.gradient(X.PARAEXP, out)
    assert abs(J - b["J"]) / b["J"] < 1e-10
    assert rel(host(out), b["grad"]) < 1e-10
    ctx.close()


@pytest.mark.parametrize("n,C,K,P", [(200, 4, 630, 6), (200, 8, 600, 6), (100, 1, 632, 8),
                                      (48, 3, 210, 3), (512, 16, 400, 5), (290, 4, 630, 6),
                                      (1000, 9, 400, 5)])
def test_burgers_four_step_chain(X, torch, n, C, K, P):
    """The chain with four-step product bands (33 taps split over four warps, 16-point
    halos) on clusters from one CTA (halo wrapping the grid) to 16, with subinterval
    lengths that are not multiples of 4 (so the plan mixes four-, two- and one-step
    entries around the lane values), gives the oracle's gradient like the two-step
    chain. The point groups cover one to four groups of 32 per CTA, with a shorter last
    CTA (290 over 4, 1000 over 9): the edge group and the interior groups split the
    points differently in each."""
    nu, T = 0.02, 0.25
    f = 2.0 * I.fourier1d(n, 8, 81)
    g = I.fourier1d(n, 8, 82)
    J0, g0 = O.bu1_gradient_serial(f, g, nu, T, K, omega=1.5)
    fd, gd_ = dev(torch, f), dev(torch, g)
    res = {}
    for impl in (X.ADJ_BANDED, X.ADJ_BANDED_PAIR):
        ctx = bu1_ctx(X, n, nu, T, K, P, phi=X.PHI_STEPPER)
        ctx.set_adjoint(impl)
        ctx.set_cluster(0, 0, C)
        ctx.set_control(fd, 1.5)
        ctx.set_target(gd_)
        out = torch.empty_like(fd)
        for mode in (X.SERIAL, X.PARAEXP):
            J = ctx.gradient(mode, out)
            assert abs(J - J0) / J0 < 1e-10
            assert rel(host(out), g0) < 1e-10, (impl, mode)
            res[(impl, mode)] = host(out)
        assert ctx.stats()["cluster_chain"] == C
        ctx.close()
    for mode in (X.SERIAL, X.PARAEXP):
        assert rel(res[(X.ADJ_BANDED, mode)], res[(X.ADJ_BANDED_PAIR, mode)]) < 1e-12


# ---- multi-checkpoint scheme (Sec. 3.5) ----------------------------------------------------
@pytest.mark.parametrize("n,C,K,P,nint", [(200, 4, 630, 6, 5), (100, 1, 600, 4, 3), (48, 3, 210, 3, 7),
                                           (512, 16, 400, 5, 2), (64, 2, 105, 1, 5), (64, 2, 120, 4, 30),
                                           (96, 4, 132, 2, 6)])
def test_burgers_multi_checkpoint_matches_oracle(X, torch, n, C, K, P, nint):
    """The rough pass keeps nint + 1 checkpoints; every interval is re-stepped and solved by
    the Paraexp adjoint over its own P subintervals from the adjoint value its upper
    neighbour left. Intervals starting on rows that are not multiples of 2 or 4 (pair and
    four-step records offset), one-step subintervals (a lane value on every row), odd
    interval counts (the two buffer sets end unevenly), clusters of 1 to 16 CTAs, serial
    and Paraexp modes, with sin(omega t) forcing: the gradient is the oracle's and that of
    full storage."""
    nu, T = 0.02, 0.25
    f = 2.0 * I.fourier1d(n, 8, 91)
    g = I.fourier1d(n, 8, 92)
    J0, g0 = O.bu1_gradient_serial(f, g, nu, T, K, omega=1.5)
    fd, gd_ = dev(torch, f), dev(torch, g)
    for impl in (X.ADJ_BANDED, X.ADJ_BANDED_PAIR):
        ref = bu1_ctx(X, n, nu, T, K, P, phi=X.PHI_STEPPER)
        ref.set_adjoint(impl)
        ref.set_cluster(0, 0, C)
        ref.set_control(fd, 1.5)
        ref.set_target(gd_)
        ctx = bu1_ctx(X, n, nu, T, K, P, phi=X.PHI_STEPPER)
        ctx.set_adjoint(impl)
        ctx.set_cluster(0, 0, C)
        ctx.set_checkpoints(nint)
        ctx.set_control(fd, 1.5)
        ctx.set_target(gd_)
        out, out_ref = torch.empty_like(fd), torch.empty_like(fd)
        for mode in (X.SERIAL, X.PARAEXP):
            J = ctx.gradient(mode, out)
            ref.gradient(mode, out_ref)
            assert abs(J - J0) / J0 < 1e-10
            assert rel(host(out), g0) < 1e-10, (impl, mode)
            assert rel(host(out), host(out_ref)) < 1e-12, (impl, mode)
        st = ctx.stats()
        assert st["checkpoint_intervals"] == nint
        assert st["cluster_chain"] == C
        ctx.close()
        ref.close()


def test_burgers_multi_checkpoint_graph_split_and_memory(X, torch, bu_small):
    """Graph replay, a direct solve followed by the adjoint solve, and the workspace: two
    interval buffer sets take a fraction of the full-storage workspace."""
    b = bu_small
    fd, gd_ = dev(torch, b["f"]), dev(torch, b["g"])
    full = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], 6, phi=X.PHI_STEPPER)
    full.set_control(fd)
    full.set_target(gd_)
    out = torch.empty_like(fd)
    full.gradient(X.PARAEXP, out)
    ws_full = full.stats()["workspace_bytes"]
    full.close()
    ctx = bu1_ctx(X, b["n"], b["nu"], b["T"], b["K"], 6, phi=X.PHI_STEPPER)
    ctx.set_checkpoints(10)
    ctx.set_control(fd)
    ctx.set_target(gd_)
    ctx.set_graph(True)
    for _ in range(2):
        J = ctx.gradient(X.PARAEXP, out)
        assert abs(J - b["J"]) / b["J"] < 1e-10
        assert rel(host(out), b["grad"]) < 1e-10
    ctx.set_graph(False)
    out2 = torch.zeros_like(fd)
    J = ctx.solve_direct(X.PARAEXP)
    ctx.solve_adjoint(X.PARAEXP, out2)
    assert abs(J - b["J"]) / b["J"] < 1e-10
    assert rel(host(out2), host(out)) < 1e-14
    assert ctx.stats()["workspace_bytes"] < 0.35 * ws_full
    # K = 600 is not a multiple of 7 x 6; the exponential propagator is not supported
    ctx.set_checkpoints(7)
    with pytest.raises(X.PxaError):
        ctx.gradient(X.PARAEXP, out)
    ctx.set_checkpoints(5)
    ctx.set_krylov(30, 1e-10, X.PHI_EXP, 1)
    with pytest.raises(X.PxaError):
        ctx.gradient(X.PARAEXP, out)
    ctx.close()


# ---- real Leja points method (Sec. 4.1) ----------------------------------------------------
@pytest.mark.parametrize("phi", ["exp", "stepper"])
@pytest.mark.parametrize("n,c,nu,span", [(256, 1.0, 0.01, 512), (64, 1.0, 0.0, 1200), (128, 0.0, 0.05, 800),
                                         (1000, 1.0, 0.002, 4096), (37, 2.0, 0.1, 300)])
def test_relpm_expv_matches_exact_propagators(X, torch, n, c, nu, span, phi):
    """exp(t A) v (Newton interpolation of phi) and the CN power R(dt A)^k v (interpolated
    directly), and their transposes, by the real Leja points method (pure advection:
    degenerate focal interval; pure diffusion; mixed; stiff) against the closed-form
    Fourier propagators."""
    T, K = 1.0, 4096
    ph = X.PHI_EXP if phi == "exp" else X.PHI_STEPPER
    ctx = ad1_ctx(X, n, c, nu, T, K, 8, m=30, tol=1e-13, phi=ph)
    ctx.set_propagator(X.PROP_RELPM, 150)
    v = I.grf_k2(n, 9)
    xd = dev(torch, v)
    y = torch.empty_like(xd)
    for tr in (False, True):
        err = ctx.expv(xd, y, span, transpose=tr)
        if phi == "exp":
            ref = O.ad1_phi_dft(v, c, nu, O.PHI_EXP, t=span * T / K, transpose=tr)
        else:
            ref = O.ad1_phi_dft(v, c, nu, O.PHI_CN, dt=T / K, steps=span, transpose=tr)
        assert rel(host(y), ref) < 1e-11
        assert err < 1e-12


def test_relpm_not_converged_is_reported(X, torch):
    n = 256
    ctx = ad1_ctx(X, n, 1.0, 0.01, 1.0, 4096, 1, m=30, tol=1e-14, phi=X.PHI_EXP)
    ctx.set_propagator(X.PROP_RELPM, 4)
    xd = dev(torch, I.grf_k2(n, 1))
    y = torch.empty_like(xd)
    with pytest.raises(X.PxaError) as ei:
        ctx.expv(xd, y, 4096)
    assert ei.value.code == X.ERR_NOT_CONVERGED
    ctx.set_propagator(X.PROP_KRYLOV, 120)
    ctx.set_krylov(30, 1e-10, X.PHI_EXP, 1)
    ctx.expv(xd, y, 64)  # the same context keeps working


@pytest.mark.parametrize("n,nu,K,P", [(256, 0.01, 4096, 8), (100, 0.0, 512, 4), (333, 0.05, 1024, 16)])
def test_relpm_paraexp_gradient_matches_oracle(X, torch, n, nu, K, P):
    """The Paraexp loop with ReLPM homogeneous exponentials (Eq. hom, Eq. adjHomNormal)
    equals the oracle's Paraexp with the exact exponential, and the Krylov path."""
    c, T = 1.0, 1.0
    q0 = I.grf_k2(n, 21)
    Jo, go, _ = O.ad1_cn_gradient_paraexp(q0, c, nu, T, K, P, O.PHI_EXP)
    qd = dev(torch, q0)
    res = {}
    for prop in (X.PROP_RELPM, X.PROP_KRYLOV):
        ctx = ad1_ctx(X, n, c, nu, T, K, P, m=40, tol=1e-12, phi=X.PHI_EXP)
        ctx.set_propagator(prop, 150)
        if prop == X.PROP_KRYLOV:
            ctx.set_krylov(40, 1e-12, X.PHI_EXP, 4)
        ctx.set_control(qd)
        out = torch.empty_like(qd)
        J = ctx.gradient(X.PARAEXP, out)
        assert abs(J - Jo) / Jo < 1e-10
        assert rel(host(out), go) < 1e-10
        res[prop] = host(out)
        ctx.close()
    assert rel(res[X.PROP_RELPM], res[X.PROP_KRYLOV]) < 1e-10


@pytest.mark.parametrize("n,nu,K,P", [(256, 0.01, 4096, 8), (100, 0.0, 512, 4), (333, 0.05, 1024, 16)])
def test_relpm_stepper_paraexp_equals_serial_stepping(X, torch, n, nu, K, P):
    """With the CN power interpolated by ReLPM, the Paraexp loop reproduces serial CN
    stepping (the oracle's serial gradient) to 1e-10."""
    c, T = 1.0, 1.0
    q0 = I.grf_k2(n, 23)
    Jo, go, _ = O.ad1_cn_gradient_serial(q0, c, nu, T, K)
    ctx = ad1_ctx(X, n, c, nu, T, K, P, m=30, tol=1e-13, phi=X.PHI_STEPPER)
    ctx.set_propagator(X.PROP_RELPM, 150)
    qd = dev(torch, q0)
    ctx.set_control(qd)
    out = torch.empty_like(qd)
    J = ctx.gradient(X.PARAEXP, out)
    assert abs(J - Jo) / Jo < 1e-10
    assert rel(host(out), go) < 1e-10


# ---- lanes stepping with the product band of M^q ------------------------------------------------
@pytest.mark.parametrize("n,nu,K,P", [(256, 0.01, 4096, 8), (100, 0.0, 512, 4), (333, 0.05, 1024, 16),
                                      (64, 0.02, 96, 16), (17, 0.1, 64, 64)])
def test_lane_product_bands_keep_the_gradient(X, torch, n, nu, K, P):
    """The lanes apply the band of M^q, q CN steps at a time (q = 1, 2, 4 or the widest
    dividing K/P): serial stepping and Paraexp with the stepper propagator match the
    oracle's serial CN gradient for every q, and q = 4 is refused where K/P = 6."""
    c, T = 1.0, 1.0
    q0 = I.grf_k2(n, 29)
    Jo, go, _ = O.ad1_cn_gradient_serial(q0, c, nu, T, K)
    qd = dev(torch, q0)
    k = K // P
    for q in (1, 2, 4, 0):
        ctx = ad1_ctx(X, n, c, nu, T, K, P, m=30, tol=1e-12, phi=X.PHI_STEPPER)
        ctx.set_propagator(X.PROP_BAND, 150)
        ctx.set_lane_steps(q)
        ctx.set_control(qd)
        out = torch.empty_like(qd)
        if q and k % q:
            with pytest.raises(X.PxaError):
                ctx.gradient(X.PARAEXP, out)
            ctx.close()
            continue
        for mode in (X.SERIAL, X.PARAEXP):
            J = ctx.gradient(mode, out)
            assert abs(J - Jo) / Jo < 1e-10, (q, mode)
            assert rel(host(out), go) < 1e-10, (q, mode)
        st = ctx.stats()
        assert st["lane_steps"] == (q if q else (4 if k % 4 == 0 else 2 if k % 2 == 0 else 1))
        assert st["lane_band_taps"] >= st["band_taps"]
        ctx.close()


# ---- the subinterval propagator as a circulant band -------------------------------------------
@pytest.mark.parametrize("phi", ["exp", "stepper"])
@pytest.mark.parametrize("n,c,nu,span", [(256, 1.0, 0.01, 512), (64, 1.0, 0.0, 1200), (128, 0.0, 0.05, 800),
                                         (1000, 1.0, 0.002, 4096), (37, 2.0, 0.1, 300), (4096, 1.0, 0.02, 2048)])
def test_band_expv_matches_exact_propagators(X, torch, n, c, nu, span, phi):
    """exp(t A) v and the CN power R(dt A)^k v, and their transposes, applied as one
    circulant band whose taps come from the propagator's eigenvalues (pure advection, pure
    diffusion, mixed, stiff, a long grid), against the closed-form Fourier propagators."""
    T, K = 1.0, 4096
    ph = X.PHI_EXP if phi == "exp" else X.PHI_STEPPER
    ctx = ad1_ctx(X, n, c, nu, T, K, 8, m=30, tol=1e-13, phi=ph)
    ctx.set_propagator(X.PROP_BAND, 150)
    v = I.grf_k2(n, 19)
    xd = dev(torch, v)
    y = torch.empty_like(xd)
    for tr in (False, True):
        ctx.expv(xd, y, span, transpose=tr)
        if phi == "exp":
            ref = O.ad1_phi_dft(v, c, nu, O.PHI_EXP, t=span * T / K, transpose=tr)
        else:
            ref = O.ad1_phi_dft(v, c, nu, O.PHI_CN, dt=T / K, steps=span, transpose=tr)
        assert rel(host(y), ref) < 1e-12, tr


@pytest.mark.parametrize("n,nu,K,P", [(256, 0.01, 4096, 8), (100, 0.0, 512, 4), (333, 0.05, 1024, 16),
                                      (17, 0.1, 64, 64)])
def test_band_paraexp_gradient_matches_oracle(X, torch, n, nu, K, P):
    """The Paraexp loop with the band of exp(tau A) equals the oracle's Paraexp with the
    exact exponential; with the band of M^(K/P) it equals the oracle's serial CN stepping
    (graph replay included)."""
    c, T = 1.0, 1.0
    q0 = I.grf_k2(n, 27)
    qd = dev(torch, q0)
    for phi in (X.PHI_EXP, X.PHI_STEPPER):
        if phi == X.PHI_EXP:
            Jo, go, _ = O.ad1_cn_gradient_paraexp(q0, c, nu, T, K, P, O.PHI_EXP)
        else:
            Jo, go, _ = O.ad1_cn_gradient_serial(q0, c, nu, T, K)
        ctx = ad1_ctx(X, n, c, nu, T, K, P, m=30, tol=1e-12, phi=phi)
        ctx.set_propagator(X.PROP_BAND, 150)
        ctx.set_control(qd)
        out = torch.empty_like(qd)
        for graph in (False, True):
            ctx.set_graph(graph)
            J = ctx.gradient(X.PARAEXP, out)
            assert abs(J - Jo) / Jo < 1e-10
            assert rel(host(out), go) < 1e-10, (phi, graph)
        ctx.close()


@pytest.mark.parametrize("n,nu", [(4608, 0.01), (5000, 0.002), (64, 0.05), (2304 * 3 + 4, 0.0)])
def test_cn_lanes_1d_streaming_matches_oracle(X, torch, n, nu):
    """FP32 CN band lanes with their states in global memory (tiles of 2304 points,
    periodic halos across tile and lane ends, a partial last tile) against the oracle's
    FP64 CN steps, within FP32 roundoff."""
    c, T, K, steps, lanes = 1.0, 1.0, 4096, 7, 3
    ctx = ad1_ctx(X, n, c, nu, T, K, 1)
    q0 = I.grf_k2(n, 31)
    qd = dev(torch, q0)
    ctx.set_control(qd)
    out = torch.empty(lanes * n, dtype=torch.float64, device="cuda")
    ms = ctx.cn_lanes_1d(lanes, steps, out)
    assert ms > 0.0
    ref = q0.copy()
    for _ in range(steps):
        ref = O.ad1_cn_step(ref, c, nu, T / K)
    o = host(out).reshape(lanes, n)
    for l in range(lanes):
        assert rel(o[l], ref) < 1e-5


def test_bounded_wait_runs_out_and_the_context_stays_usable(X, torch):
    """The failure path of the bounded device waits: a thread block waits on an mbarrier
    that nothing completes (no copy, no peer) and gives up after the context's wait
    limit (2^20 cycles, about 0.5 ms), which the host reads as PXA_ERR_TIMEOUT; a Burgers
    gradient on the same context, whose cluster halo exchanges wait under the same short
    limit, then matches the oracle."""
    n, nu, T, K, P = 256, 0.02, 0.05, 100, 4
    f = I.fourier1d(n, 8, 61)
    tg = I.fourier1d(n, 8, 62)
    ctx = X.Context()
    ctx.set_operator(X.BURGERS_1D, n, nu=nu)
    ctx.set_time(T, K, X.RK4, P)
    ctx.set_krylov(20, 1e-10, X.PHI_STEPPER, 1)
    fd, td = dev(torch, f), dev(torch, tg)
    ctx.set_control(fd)
    ctx.set_target(td)
    with pytest.raises(X.PxaError):
        ctx.set_wait_limit(100)  # below 1024 cycles
    ctx.set_wait_limit(1 << 20)
    for _ in range(2):
        with pytest.raises(X.PxaError) as ei:
            ctx.wait_probe()
        assert ei.value.code == X.ERR_TIMEOUT
    out = torch.empty_like(fd)
    J = ctx.gradient(X.PARAEXP, out)
    Jo, go = O.bu1_gradient_serial(f, tg, nu, T, K)
    assert abs(J - Jo) / Jo < 1e-10 and rel(host(out), go) < 1e-10
    ctx.set_wait_limit(0)
    with pytest.raises(X.PxaError) as ei:  # the default limit (2^31 cycles, about 1 s)
        ctx.wait_probe()
    assert ei.value.code == X.ERR_TIMEOUT
    ctx.close()


# ---- iterative nonlinear Paraexp direct (Sec. 3.2, Alg. 2) --------------------------------
NL_CASES = {"n32": (32, 0.05, 0.5, 128, 4, 3.0, 1.5), "n256": (256, 0.02, 0.25, 400, 8, 2.0, 0.0),
            "n1000": (1000, 0.02, 0.1, 200, 10, 1.0, 2.0)}


def nl_setup(X, torch, case):
    n, nu, T, K, P, amp, om = NL_CASES[case]
    f = amp * I.fourier1d(n, 8, 71)
    ctx = bu1_ctx(X, n, nu, T, K, P, phi=X.PHI_STEPPER)
    fd = dev(torch, f)
    ctx.set_control(fd, om)
    traj = torch.empty((K + 1, n), dtype=torch.float64, device="cuda")
    return ctx, fd, traj, f


@pytest.mark.parametrize("case", sorted(NL_CASES))
def test_nl_paraexp_matches_the_oracle_iteration_by_iteration(X, torch, case):
    """After 1, 2 and 3 iterations from q(t) = 0 the GPU iterate equals the oracle's point
    by point (1e-10 of its largest value) and so do the iterations' changes."""
    n, nu, T, K, P, amp, om = NL_CASES[case]
    ctx, fd, traj, f = nl_setup(X, torch, case)
    for iters in (1, 2, 3):
        tr_o, ch_o, _ = O.bu1_nl_paraexp_direct(f, nu, T, K, P, omega=om, tol=1e-300, max_iter=iters)
        ch, ok = ctx.nl_paraexp(traj, tol=1e-300, max_iter=iters)
        assert not ok and len(ch) == iters == len(ch_o)
        assert rel(traj.cpu().numpy(), tr_o) < 1e-10, (case, iters)
        assert np.all(np.abs(ch - ch_o) <= 1e-10 * np.maximum(ch_o, 1e-3)), (ch, ch_o)
    ctx.close()


@pytest.mark.parametrize("case", sorted(NL_CASES))
def test_nl_paraexp_converges_to_the_serial_rk4_trajectory(X, torch, case):
    """Iterated to a change of 1e-12 the iterate is the serial RK4 trajectory (the
    iteration's fixed point), in as many iterations as the oracle takes (within one)."""
    n, nu, T, K, P, amp, om = NL_CASES[case]
    ctx, fd, traj, f = nl_setup(X, torch, case)
    g = I.fourier1d(n, 8, 72)
    _, _, ts = O.bu1_gradient_serial(f, g, nu, T, K, omega=om, want_traj=True)
    _, ch_o, ok_o = O.bu1_nl_paraexp_direct(f, nu, T, K, P, omega=om, tol=1e-12, max_iter=60)
    ch, ok = ctx.nl_paraexp(traj, tol=1e-12, max_iter=60)
    assert ok and ok_o and abs(len(ch) - len(ch_o)) <= 1 and ch[-1] <= 1e-12
    assert rel(traj.cpu().numpy(), ts) < 1e-10
    # the serial trajectory as the guess is a fixed point: one iteration changes nothing
    guess = dev(torch, ts)
    ch1, ok1 = ctx.nl_paraexp(traj, guess=guess, tol=1e-12, max_iter=1)
    assert ok1 and ch1[0] < 1e-13 and rel(traj.cpu().numpy(), ts) < 1e-13
    ctx.close()
