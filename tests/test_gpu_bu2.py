"""Parity of the 2D viscous Burgers path (Sec. 4.3: FP32 RK4 direct, the exact discrete
adjoint of the RK4 map, initial-state control, J = 0.5 ||q(T) - q_target||^2 in FP64)
with the FP64 oracle, and the 20-iteration L-BFGS loop with the per-iteration error.

Tolerance from the arithmetic: FP32 stepping of K steps loses about K u_32 relative
(u_32 = 2^-24); the tests hold J, q(T) and the gradient to max(1e-4, 4 K u_32), point by
point. At the full size (256^2, K = 5120) the oracle's direct alone takes minutes, so the
gradient is checked there against central differences of the GPU objective along seeded
directions (a property at any size), to 2e-2."""
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


def ctx_bu2(X, n, nu, T, K, P=4):
    ctx = X.Context()
    ctx.set_operator_burgers_2d(n, nu)
    ctx.set_time(T, K, X.RK4, P)
    return ctx


def split(x, n):
    return x[:n * n].reshape(n, n), x[n * n:].reshape(n, n)


@pytest.mark.parametrize("n,nu,T,K", [(16, 0.05, 0.2, 40), (32, 0.02, 0.1, 100), (48, 0.01, 0.05, 64)])
def test_bu2_gradient_matches_oracle(X, torch, n, nu, T, K):
    p = I.burgers2d_problem(n=n, seed=31, kmax=4, amp=1.0)
    tU, tV = O.bu2_direct(*split(0.8 * p["true_ic"], n), nu, T, K)
    target = np.concatenate([tU.ravel(), tV.ravel()])
    q0 = p["other_ic"]
    Jo, gU, gV = O.bu2_gradient_serial(*split(q0, n), tU, tV, nu, T, K)
    go = np.concatenate([gU.ravel(), gV.ravel()])
    tol = max(1e-4, 4 * K * 2.0 ** -24)
    ctx = ctx_bu2(X, n, nu, T, K)
    qd, td = torch.as_tensor(q0, device="cuda"), torch.as_tensor(target, device="cuda")
    ctx.set_control(qd)
    ctx.set_target(td)
    res = {}
    for mode in (X.SERIAL, X.PARAEXP):
        g = torch.empty_like(qd)
        J = ctx.gradient(mode, g)
        assert abs(J - Jo) / Jo < tol, (mode, J, Jo)
        assert rel(g.cpu().numpy(), go) < tol, mode
        res[mode] = g.cpu().numpy()
    assert np.array_equal(res[X.SERIAL], res[X.PARAEXP])  # the same kernels (terminal objective)
    # the direct's final state against the oracle's
    qT = torch.empty_like(qd)
    ctx.direct_state(qd, qT)
    oU, oV = O.bu2_direct(*split(q0, n), nu, T, K)
    assert rel(qT.cpu().numpy(), np.concatenate([oU.ravel(), oV.ravel()])) < tol
    ctx.close()


def test_bu2_lbfgs_per_iteration_error(X, torch):
    """20 L-BFGS iterations from the zero initial state towards the target made from a true
    initial state: J decreases monotonically and at every accepted iterate the GPU's J and
    gradient match the FP64 oracle's at that iterate (the per-iteration error, FP32
    tolerance relative to the first gradient, whose terms dominate the rounding)."""
    from paper_2004_00546_gb300 import lbfgs

    n, nu, T, K = 32, 0.02, 0.1, 100
    p = I.burgers2d_problem(n=n, seed=32, kmax=4, amp=1.0)
    tU, tV = O.bu2_direct(*split(0.8 * p["true_ic"], n), nu, T, K)
    ctx = ctx_bu2(X, n, nu, T, K)
    td = torch.as_tensor(np.concatenate([tU.ravel(), tV.ravel()]), device="cuda")
    ctx.set_target(td)
    res = lbfgs.minimize(ctx, torch.zeros(2 * n * n, dtype=torch.float64, device="cuda"), iters=20,
                         mode=X.PARAEXP, keep_iterates=True)
    assert len(res.J) >= 10
    assert all(b <= a for a, b in zip(res.J, res.J[1:]))
    assert res.J[-1] < 0.1 * res.J[0]
    tol = max(1e-4, 4 * K * 2.0 ** -24)
    g0 = None
    for it, xk in enumerate(res.iterates):
        Jo, gU, gV = O.bu2_gradient_serial(*split(xk.cpu().numpy(), n), tU, tV, nu, T, K)
        go = np.concatenate([gU.ravel(), gV.ravel()])
        g0 = np.abs(go).max() if g0 is None else g0
        gk = torch.empty_like(xk)
        ctx.set_control(xk)
        Jk = ctx.gradient(X.PARAEXP, gk)
        assert abs(Jk - Jo) <= tol * Jo + 1e-6 * res.J[0], it
        assert np.abs(gk.cpu().numpy() - go).max() <= tol * np.abs(go).max() + tol * g0, it
    ctx.close()


def test_bu2_full_size_gradient_against_central_differences(X, torch):
    """The configured workload (256^2, nu = 2e-3, T = 1, K = 5120, initial fields of
    amplitude 0.15): along three seeded directions, the central difference of the GPU
    objective with a step of 1e-2 of the state's size matches the gradient's directional
    derivative to 2e-2 (FP32 stepping)."""
    n, nu, T, K = 256, 2e-3, 1.0, 5120
    p = I.burgers2d_problem(n=n)
    ctx = ctx_bu2(X, n, nu, T, K, P=128)
    ic_true = torch.as_tensor(p["true_ic"], device="cuda")
    target = torch.empty_like(ic_true)
    ctx.direct_state(ic_true, target)
    ctx.set_target(target)
    x = torch.as_tensor(p["other_ic"], device="cuda")
    g = torch.empty_like(x)
    ctx.set_control(x)
    J = ctx.gradient(X.PARAEXP, g)
    assert J > 0 and bool(torch.isfinite(g).all())
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = torch.as_tensor(rng.standard_normal(2 * n * n), device="cuda")
        eps = 1e-2 * 0.15
        ctx.set_control(x + eps * d)
        Jp = ctx.solve_direct(X.PARAEXP)
        ctx.set_control(x - eps * d)
        Jm = ctx.solve_direct(X.PARAEXP)
        fd = (Jp - Jm) / (2 * eps)
        ex = float(torch.dot(g, d))
        assert abs(fd - ex) < 2e-2 * abs(ex), (fd, ex)
    ctx.close()
