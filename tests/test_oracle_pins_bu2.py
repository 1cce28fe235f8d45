"""Pins of the oracle's 2D viscous Burgers problem (Sec. 4.3: the vector field (u, v),
advective central differences, classical RK4, initial-condition control, terminal
objective J = 0.5 ||q(T) - q_target||^2): the right-hand side on fields whose central
differences have closed forms (each advection term -u u_x, -v u_y, -u v_x, -v v_y
exercised on its own, with its sign), the Jacobian by central differences (exact: N is
quadratic), the transpose against a dense brute-force transpose, one RK4 step against the
amplification polynomial on a small-amplitude Fourier mode, and the gradient against
Richardson-extrapolated central differences of J."""
import numpy as np
import pytest

import oracle as O
from paper_2004_00546_gb300 import inputs as I


def grid(n, L=2 * np.pi):
    x = L * np.arange(n) / n
    X, Y = np.meshgrid(x, x)  # X varies along columns (x fastest), Y along rows
    return X, Y


def sym(k, n, L=2 * np.pi):
    h = L / n
    kt = np.sin(2 * np.pi * k / L * h) / h
    dd = 4 * np.sin(np.pi * k / L * h) ** 2 / h ** 2
    return kt, dd


def bound(n, amp2, amp, nu, L=2 * np.pi):
    h = L / n
    return 1e-13 * (amp2 / h + nu * amp / h ** 2)


@pytest.mark.parametrize("n,k,l,A,B,nu", [(16, 2, 3, 1.3, 0.7, 0.02), (48, 5, 1, 0.8, 1.5, 0.005)])
def test_bu2_rhs_self_advection_closed_form(n, k, l, A, B, nu):
    """U = A sin(k x), V = B cos(l y): -u u_x = -A^2 k~ sin cos, -v v_y = +B^2 l~ sin(ly) cos(ly),
    and the cross terms vanish (u_y = 0, v_x = 0)."""
    X, Y = grid(n)
    U, V = A * np.sin(k * X), B * np.cos(l * Y)
    kt, dk = sym(k, n)
    lt, dl = sym(l, n)
    oU, oV = O.bu2_rhs(U, V, nu)
    refU = -A * A * kt * np.sin(k * X) * np.cos(k * X) - nu * A * dk * np.sin(k * X)
    refV = B * B * lt * np.sin(l * Y) * np.cos(l * Y) - nu * B * dl * np.cos(l * Y)
    tol = bound(n, max(A, B) ** 2, max(A, B), nu)
    assert np.abs(oU - refU).max() < tol and np.abs(oV - refV).max() < tol


@pytest.mark.parametrize("n,k,A,C,nu", [(20, 3, 1.1, 0.6, 0.01), (64, 7, 0.9, -1.2, 0.003)])
def test_bu2_rhs_cross_advection_closed_form(n, k, A, C, nu):
    """U = A sin(k y), V = C: -v u_y = -C A k~ cos(k y) (and N_v = 0); U = C, V = A sin(k x):
    -u v_x = -C A k~ cos(k x) (and N_u = 0)."""
    X, Y = grid(n)
    kt, dk = sym(k, n)
    tol = bound(n, abs(A * C) + A * A, A, nu)
    oU, oV = O.bu2_rhs(A * np.sin(k * Y), np.full((n, n), C), nu)
    assert np.abs(oU - (-C * A * kt * np.cos(k * Y) - nu * A * dk * np.sin(k * Y))).max() < tol
    assert np.abs(oV).max() < tol
    oU, oV = O.bu2_rhs(np.full((n, n), C), A * np.sin(k * X), nu)
    assert np.abs(oU).max() < tol
    assert np.abs(oV - (-C * A * kt * np.cos(k * X) - nu * A * dk * np.sin(k * X))).max() < tol


def test_bu2_jacobian_central_fd_exact():
    rng = np.random.default_rng(3)
    for n in (3, 12):
        U, V, W1, W2 = (rng.standard_normal((n, n)) for _ in range(4))
        for eps in (1.0, 0.25):
            pU, pV = O.bu2_rhs(U + eps * W1, V + eps * W2, 0.03)
            mU, mV = O.bu2_rhs(U - eps * W1, V - eps * W2, 0.03)
            j1, j2 = O.bu2_jac(U, V, W1, W2, 0.03)
            sc = max(np.abs(j1).max(), np.abs(j2).max())
            assert np.abs((pU - mU) / (2 * eps) - j1).max() < 1e-11 * sc
            assert np.abs((pV - mV) / (2 * eps) - j2).max() < 1e-11 * sc


@pytest.mark.parametrize("n", [3, 5, 6])
def test_bu2_jacobian_transpose_matches_dense_brute_force(n):
    rng = np.random.default_rng(n)
    U, V = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    N2 = 2 * n * n
    E = np.eye(N2)
    cols = []
    for e in E:
        j1, j2 = O.bu2_jac(U, V, e[:n * n].reshape(n, n), e[n * n:].reshape(n, n), 0.05)
        cols.append(np.concatenate([j1.ravel(), j2.ravel()]))
    D = np.stack(cols, 1)
    colsT = []
    for e in E:
        t1, t2 = O.bu2_jac(U, V, e[:n * n].reshape(n, n), e[n * n:].reshape(n, n), 0.05, transpose=True)
        colsT.append(np.concatenate([t1.ravel(), t2.ravel()]))
    DT = np.stack(colsT, 1)
    assert np.abs(DT - D.T).max() < 1e-12 * np.abs(D).max()


def test_bu2_rk4_step_is_the_amplification_polynomial_at_small_amplitude():
    """At amplitude 1e-14 the advection terms are below rounding: one step multiplies a
    mode of u by R(dt lambda), lambda = -nu (d~_k + d~_l) the 5-point Laplacian's symbol."""
    n, nu, k, l = 16, 0.2, 2, 3
    X, Y = grid(n)
    eps = 1e-14
    U = eps * np.cos(k * X + l * Y)
    V = 0.5 * eps * np.sin(l * X)
    _, dk = sym(k, n)
    _, dl = sym(l, n)
    for dt in (0.02, 0.05):
        z = -dt * nu * (dk + dl)
        R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
        zv = -dt * nu * sym(l, n)[1]
        Rv = 1 + zv + zv * zv / 2 + zv ** 3 / 6 + zv ** 4 / 24
        oU, oV = O.bu2_rk4_step(U, V, nu, dt)
        assert np.abs(oU - R * U).max() < 1e-12 * eps
        assert np.abs(oV - Rv * V).max() < 1e-12 * eps


def test_bu2_gradient_central_fd_richardson():
    n, nu, T, K = 8, 0.05, 0.2, 40
    q0U = 0.6 * I.fourier2d(n, n, 2, 11)
    q0V = 0.6 * I.fourier2d(n, n, 2, 12)
    tU, tV = O.bu2_direct(0.8 * I.fourier2d(n, n, 2, 13), 0.8 * I.fourier2d(n, n, 2, 14), nu, T, K)
    J, gU, gV = O.bu2_gradient_serial(q0U, q0V, tU, tV, nu, T, K)
    assert J > 0
    rng = np.random.default_rng(5)
    for _ in range(3):
        dU, dV = rng.standard_normal((n, n)), rng.standard_normal((n, n))

        def cfd(e):
            Jp = O.bu2_gradient_serial(q0U + e * dU, q0V + e * dV, tU, tV, nu, T, K)[0]
            Jm = O.bu2_gradient_serial(q0U - e * dU, q0V - e * dV, tU, tV, nu, T, K)[0]
            return (Jp - Jm) / (2 * e)

        rich = (4 * cfd(1e-3) - cfd(2e-3)) / 3
        ex = np.sum(gU * dU) + np.sum(gV * dV)
        assert abs(rich - ex) < 1e-8 * abs(ex)


def test_bu2_gradient_vanishes_at_the_target_initial_state():
    n, nu, T, K = 8, 0.05, 0.2, 40
    aU, aV = 0.8 * I.fourier2d(n, n, 2, 13), 0.8 * I.fourier2d(n, n, 2, 14)
    tU, tV = O.bu2_direct(aU, aV, nu, T, K)
    J, gU, gV = O.bu2_gradient_serial(aU, aV, tU, tV, nu, T, K)
    assert J < 1e-28 and np.abs(gU).max() < 1e-14 and np.abs(gV).max() < 1e-14
