"""2D advection-diffusion (FP32 stepping on TMA halo tiles) against the FP64 oracle.

Tolerance: the stepping is FP32 (unit roundoff 6e-8) and the objective and gradient
accumulate FP32 step results in FP64; over K <= 64 steps the relative error of J
and of the gradient stays below K * 1e-6, so these tests hold them to 1e-4 (the
per-result FP32 tolerance), and the FP32 lane states to 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from paper_2004_00546_gb300 import inputs as I
from parity import rel

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module")
def env(cuda_ok):
    import torch

    from paper_2004_00546_gb300 import pxa as X

    return torch, X


def problem(n, seed=2006, kv=4, kf=4):
    u, v = I.streamfunction_velocity(n, n, kv, seed)
    f = I.fourier2d(n, n, kf, seed + 1)
    ft = I.fourier2d(n, n, kf, seed + 2)
    return u, v, f, ft


def ctx2d(torch, X, n, nu, T, K, P, u, v, f, ft, omega=1.0):
    ctx = X.Context()
    ud, vd = torch.as_tensor(u, device="cuda"), torch.as_tensor(v, device="cuda")
    ctx.set_operator_2d(n, n, ud, vd, nu)
    ctx.set_time(T, K, X.RK4, P)
    ctx.set_krylov(20, 1e-10, X.PHI_STEPPER, 1)
    fd = torch.as_tensor(f, device="cuda")
    td = torch.as_tensor(ft, device="cuda")
    ctx.set_control(fd.reshape(-1), omega)
    ctx.set_target(td.reshape(-1))
    return ctx


@pytest.mark.parametrize("n", [8, 64, 72])
def test_rk4_lanes_match_oracle_steps(env, n):
    """Each lane starts from zero at step l*steps and takes `steps` FP32 RK4 steps with
    the forcing s(t)(f - f_true); compare every lane with the oracle's FP64 steps."""
    torch, X = env
    nu, T, K = 0.01, 0.2, 64
    u, v, f, ft = problem(n)
    ctx = ctx2d(torch, X, n, nu, T, K, 1, u, v, f, ft)
    lanes, steps = 5, 7
    out = torch.empty(lanes * n * n, dtype=torch.float64, device="cuda")
    ms = ctx.rk4_lanes_2d(lanes, steps, out)
    assert ms > 0
    got = out.cpu().numpy().reshape(lanes, n, n)
    dt = T / K
    d = f - ft
    for l in range(lanes):
        q = np.zeros((n, n))
        for s in range(steps):
            q = O.ad2_rk4_step(q, u, v, nu, dt, d, t=(l * steps + s) * dt, omega=1.0)
        assert rel(got[l], q) < 1e-5


@pytest.mark.parametrize("n,K,P", [(64, 48, 6), (72, 40, 4), (8, 30, 3), (120, 24, 4)])
def test_gradient_serial_and_paraexp_match_oracle(env, n, K, P):
    """Serial and Paraexp gradients against the oracle. The adjoint lanes run as a
    register wavefront on 56-column strips and row segments from 64 points on: at 64,
    72 and 120 the last strip (and at 72 and 120 the last segment) overlaps the one
    before it, and only its own points add to the lane gradients."""
    torch, X = env
    nu, T = 0.02, 0.3
    u, v, f, ft = problem(n)
    J_ref, g_ref = O.ad2_gradient_serial(f, ft, u, v, nu, T, K, omega=1.0)
    ctx = ctx2d(torch, X, n, nu, T, K, P, u, v, f, ft)
    grad = torch.empty(n * n, dtype=torch.float64, device="cuda")
    for mode in (X.SERIAL, X.PARAEXP):
        J = ctx.gradient(mode, grad)
        assert abs(J - J_ref) / J_ref < TOL32
        assert rel(grad.cpu().numpy().reshape(n, n), g_ref) < TOL32


def test_paraexp_equals_serial_to_fp32_roundoff(env):
    """The hybrid Paraexp adjoint with the stepper's own propagator is an exact
    reorganisation of serial stepping: the two GPU gradients agree to FP32 roundoff."""
    torch, X = env
    n, nu, T, K, P = 64, 0.01, 0.25, 64, 8
    u, v, f, ft = problem(n, seed=77)
    ctx = ctx2d(torch, X, n, nu, T, K, P, u, v, f, ft)
    gs = torch.empty(n * n, dtype=torch.float64, device="cuda")
    gp = torch.empty_like(gs)
    Js = ctx.gradient(X.SERIAL, gs)
    Jp = ctx.gradient(X.PARAEXP, gp)
    assert Js == Jp  # the direct solve is the same serial kernel sequence
    assert rel(gp.cpu().numpy(), gs.cpu().numpy()) < 1e-5


def test_full_size_c3_central_fd_16_directions(env):
    """512 x 512 grid, nu = 1e-3, T = 1, K = 1024 RK4 steps, P = 64, velocity from a
    |k| <= 8 streamfunction, s(t) = sin t. The objective is quadratic in the forcing, so
    the central difference with a unit step equals <grad, d> exactly; FP32 stepping
    limits the check to 1e-3 relative on 16 random directions."""
    torch, X = env
    n, nu, T, K, P = 512, 1e-3, 1.0, 1024, 64
    u, v = I.streamfunction_velocity(n, n, 8, 2006)
    x = I.grid1d(n)
    Xg, Yg = np.meshgrid(x, x)
    ft = np.sin(Xg) * np.sin(Yg)
    f = np.ones((n, n))
    ctx = ctx2d(torch, X, n, nu, T, K, P, u, v, f, ft)
    grad = torch.empty(n * n, dtype=torch.float64, device="cuda")
    ctx.gradient(X.PARAEXP, grad)
    g = grad.cpu().numpy()
    rng = np.random.default_rng(16)
    base = f.copy()
    for _ in range(16):
        d = rng.standard_normal((n, n)) * 0.1
        for sign, store in ((1, "p"), (-1, "m")):
            ctl = torch.as_tensor((base + sign * d).reshape(-1), device="cuda")
            ctx.set_control(ctl, 1.0)
            val = ctx.solve_direct(X.PARAEXP)
            if store == "p":
                Jp = val
            else:
                Jm = val
        fd = (Jp - Jm) / 2.0
        dd = float(np.sum(g * d.reshape(-1)))
        assert abs(fd - dd) < 1e-3 * abs(dd), (fd, dd)


@pytest.mark.parametrize("n,T,K,P,tol,rough", [(64, 0.35, 24, 2, 100.0, True), (64, 0.35, 24, 2, 1.0, True),
                                                (64, 0.35, 24, 2, 1e-10, True), (64, 0.3, 48, 6, 1e-10, False),
                                                (72, 0.3, 40, 4, 1e-10, False), (120, 0.3, 48, 8, 1e-10, False),
                                                (8, 0.3, 30, 3, 1e-10, False)])
def test_poly_chain_matches_oracle_at_its_degree(env, n, T, K, P, tol, rough):
    """The chain by the stepper's propagator as a power series (PXA_PROP_POLY) against the
    oracle's hybrid loop cut at the same degree m, point by point. With white-noise
    forcings and a subinterval near the series' reach (k ||dt A^T|| = 3.96), a loose
    tolerance makes the series short (m = 4) and its cut moves the gradient by ~2e-3, far
    above the FP32 tolerance: the GPU must evaluate the same truncated polynomials, not
    merely land near serial stepping. At the default tolerance it matches serial
    stepping as well."""
    torch, X = env
    nu = 0.02
    u, v, f, ft = problem(n)
    if rough:
        rng = np.random.default_rng(5)
        f, ft = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    ctx = ctx2d(torch, X, n, nu, T, K, P, u, v, f, ft)
    ctx.set_krylov(20, tol, X.PHI_STEPPER, 1)
    ctx.set_propagator(X.PROP_POLY, 200)
    grad = torch.empty(n * n, dtype=torch.float64, device="cuda")
    J = ctx.gradient(X.PARAEXP, grad)
    st = ctx.stats()
    m = st["prop_degree"]
    assert m > 0 and m % 4 == 0 and st["prop_substeps"] == 1, st
    J_ref, g_ref = O.ad2_gradient_hybrid_poly(f, ft, u, v, nu, T, K, P, m, omega=1.0)
    assert abs(J - J_ref) / J_ref < TOL32
    g = grad.cpu().numpy().reshape(n, n)
    assert rel(g, g_ref) < TOL32, (m, rel(g, g_ref))
    _, g_ser = O.ad2_gradient_serial(f, ft, u, v, nu, T, K, omega=1.0)
    if tol >= 100.0:
        assert m == 4 and rel(g_ref, g_ser) > 1e-3
    if tol <= 1e-7:
        assert rel(g, g_ser) < TOL32


def test_poly_chain_segments_within_a_subinterval(env):
    """A long subinterval (K/P = 64 steps, kk * ||dt A^T|| > 4) is split into several
    series segments; the gradient still matches serial stepping (the oracle)."""
    torch, X = env
    n, nu, T, K, P = 64, 0.02, 1.6, 256, 4
    u, v, f, ft = problem(n, seed=91)
    ctx = ctx2d(torch, X, n, nu, T, K, P, u, v, f, ft)
    ctx.set_propagator(X.PROP_POLY, 200)
    grad = torch.empty(n * n, dtype=torch.float64, device="cuda")
    ctx.gradient(X.PARAEXP, grad)
    st = ctx.stats()
    assert st["prop_substeps"] > 1 and st["prop_tail"] <= 1e-7, st
    _, g_ser = O.ad2_gradient_serial(f, ft, u, v, nu, T, K, omega=1.0)
    assert rel(grad.cpu().numpy().reshape(n, n), g_ser) < TOL32


def test_poly_chain_full_size_against_the_stepper_chain(env):
    """C3's size (512^2, K = 1024, P = 64): the series chain against the stepper chain on
    the GPU, point by point, and serial stepping; both are FP32 reorganisations of the same
    discrete adjoint, the series cut with tail bound <= 1e-7."""
    torch, X = env
    n, nu, T, K, P = 512, 1e-3, 1.0, 1024, 64
    u, v = I.streamfunction_velocity(n, n, 8, 2006)
    x = I.grid1d(n)
    Xg, Yg = np.meshgrid(x, x)
    ft = np.sin(Xg) * np.sin(Yg)
    f = np.ones((n, n))
    grads = {}
    for name, prop in (("stepper", None), ("poly", X.PROP_POLY)):
        ctx = ctx2d(torch, X, n, nu, T, K, P, u, v, f, ft)
        if prop is not None:
            ctx.set_propagator(prop, 200)
        g = torch.empty(n * n, dtype=torch.float64, device="cuda")
        ctx.gradient(X.PARAEXP, g)
        grads[name] = g.cpu().numpy()
        if prop is not None:
            st = ctx.stats()
            assert st["prop_degree"] > 0 and st["prop_tail"] <= 1e-7, st
        ctx.close()
    ctx = ctx2d(torch, X, n, nu, T, K, 1, u, v, f, ft)
    g = torch.empty(n * n, dtype=torch.float64, device="cuda")
    ctx.gradient(X.SERIAL, g)
    grads["serial"] = g.cpu().numpy()
    assert rel(grads["poly"], grads["stepper"]) < TOL32
    assert rel(grads["poly"], grads["serial"]) < TOL32
