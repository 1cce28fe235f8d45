"""Pins of the oracle's polynomial propagator (the RK4 stepper's propagator over a
subinterval as a power series in dt*A, cut after degree m; Eq. hom / adjHomNormal with
operator applications only, like the paper's ReLPM of Sec. 4.1).

What fixes them, independently of the code under test:
- a scalar problem dy/dt = lam*y (+ s(t)) stepped by the four RK4 stages written out
  here: k steps of the homogeneous problem from 1 give R(dt lam)^k, and k steps of the
  forced problem from 0 give the forcing polynomial b(dt lam);
- RK4 matches exp to fourth order, so the first five coefficients of R(z)^k are
  k^i/i!, and the last one is 24^-k;
- with s = 1 the forcing polynomial telescopes to dt (R(z)^k - 1)/z;
- the whole polynomial (no truncation) applied with the 2D operator equals k RK4 steps
  of the oracle's stepper, and the hybrid loop with it equals serial stepping;
- the truncation error obeys the power-series tail bound sum_{i>m} a_i rho^i with
  rho the max-norm of dt*A^T (all a_i are positive).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2004_00546_gb300 import inputs as I


def scalar_rk4(lam, dt, k, y0, s=None, t0=0.0):
    """k classical RK4 steps of dy/dt = lam*y + s(t) (s None: homogeneous), in complex."""
    y = complex(y0)
    for j in range(k):
        t = t0 + j * dt
        f = (lambda tt: 0.0) if s is None else s
        k1 = lam * y + f(t)
        k2 = lam * (y + 0.5 * dt * k1) + f(t + 0.5 * dt)
        k3 = lam * (y + 0.5 * dt * k2) + f(t + 0.5 * dt)
        k4 = lam * (y + dt * k3) + f(t + dt)
        y = y + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


def peval(c, z):
    return sum(ci * z**i for i, ci in enumerate(c))


def pscale(c, z):
    """sum |c_i| |z|^i: the size of the largest partial sums of a power-series evaluation,
    which bounds its rounding error (times a few units of roundoff)."""
    return sum(abs(ci) * abs(z) ** i for i, ci in enumerate(c))


@pytest.mark.parametrize("k", [1, 2, 7, 16])
def test_power_coeffs_equal_scalar_rk4_stepping(k):
    a = O.rk4_power_coeffs(k)
    assert a.shape == (4 * k + 1,)
    dt = 0.05
    for lam in (-3.0, 2.5, -1.0 + 4.0j, -20.0 + 1.5j):
        ref = scalar_rk4(lam, dt, k, 1.0)
        assert abs(peval(a, dt * lam) - ref) <= 1e-14 * k * (pscale(a, dt * lam) + abs(ref))


@pytest.mark.parametrize("k", [1, 3, 16, 40])
def test_power_coeffs_match_exp_to_order_four_and_leading_term(k):
    a = O.rk4_power_coeffs(k)
    for i in range(5):
        assert abs(a[i] - k**i / math.factorial(i)) <= 1e-15 * k**i / math.factorial(i)
    assert abs(a[-1] - 24.0 ** (-k)) <= 1e-14 * 24.0 ** (-k)
    # every coefficient of R^k lies between 0 and that of exp(k z)
    for i in range(len(a)):
        assert 0.0 < a[i] <= (1 + 1e-14) * k**i / math.factorial(i)


@pytest.mark.parametrize("omega,t0", [(0.0, 0.0), (1.0, 0.0), (1.0, 0.37), (3.7, 1.25)])
@pytest.mark.parametrize("k", [1, 4, 16])
def test_forcing_coeffs_equal_scalar_forced_rk4(k, omega, t0):
    dt = 0.03
    b = O.rk4_forcing_coeffs(k, dt, t0, omega)
    assert b.shape == (4 * k,)
    s = (lambda t: 1.0) if omega == 0.0 else (lambda t: math.sin(omega * t))
    for lam in (-2.0, 3.0, -0.5 + 6.0j, -15.0):
        ref = scalar_rk4(lam, dt, k, 0.0, s=s, t0=t0)
        assert abs(peval(b, dt * lam) - ref) <= 1e-14 * k * (pscale(b, dt * lam) + abs(ref))


@pytest.mark.parametrize("k", [1, 5, 16])
def test_forcing_coeffs_unit_forcing_telescope(k):
    """s = 1: sum_j g(z) R^(k-1-j) with g = dt (R - 1)/z telescopes to dt (R^k - 1)/z."""
    dt = 0.02
    a = O.rk4_power_coeffs(k)
    b = O.rk4_forcing_coeffs(k, dt, 0.0, 0.0)
    # (R^k - 1)/z has the coefficients of R^k shifted down by one
    assert np.allclose(b, dt * a[1:], rtol=1e-14, atol=0.0)


def velocity(n, seed=2006, kv=4):
    return I.streamfunction_velocity(n, n, kv, seed)


def rho_T(u, v, nu, dt, n):
    """max-norm of dt*A^T (largest absolute row sum of the transposed stencil)."""
    h = 2 * np.pi / n
    d = nu / h**2
    aw = np.abs(-np.roll(u, 1, axis=1) / (2 * h) + d)
    ae = np.abs(np.roll(u, -1, axis=1) / (2 * h) + d)
    as_ = np.abs(-np.roll(v, 1, axis=0) / (2 * h) + d)
    an = np.abs(np.roll(v, -1, axis=0) / (2 * h) + d)
    return dt * float((aw + ae + as_ + an + 4 * d).max())


@pytest.mark.parametrize("transpose", [False, True])
def test_whole_polynomial_equals_k_rk4_steps_2d(transpose):
    n, nu, dt, k = 12, 0.02, 0.01, 6
    u, v = velocity(n)
    x = I.fourier2d(n, n, 4, 5)
    a = O.rk4_power_coeffs(k)
    got = O.ad2_poly_apply(x, u, v, nu, dt, a, transpose=transpose)
    zero = np.zeros_like(x)
    if not transpose:
        ref = x.copy()
        for _ in range(k):
            ref = O.ad2_rk4_step(ref, u, v, nu, dt, zero)
    else:
        # A^T stepping: the RK4 step of the transposed operator, by dense transpose
        N = n * n
        E = np.eye(N)
        AT = np.column_stack([O.ad2_apply(E[:, j].reshape(n, n), u, v, nu, transpose=True).ravel()
                              for j in range(N)])
        Z = dt * AT
        R = np.eye(N) + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24
        ref = (np.linalg.matrix_power(R, k) @ x.ravel()).reshape(n, n)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("m", [4, 8, 12])
def test_truncation_within_the_power_series_tail_bound(m):
    n, nu, dt, k = 16, 0.01, 0.02, 16
    u, v = velocity(n)
    x = I.fourier2d(n, n, 6, 9)
    a = O.rk4_power_coeffs(k)
    full = O.ad2_poly_apply(x, u, v, nu, dt, a, transpose=True)
    cut = O.ad2_poly_apply(x, u, v, nu, dt, a[: m + 1], transpose=True)
    rho = rho_T(u, v, nu, dt, n)
    bound = sum(a[i] * rho**i for i in range(m + 1, len(a))) * np.abs(x).max()
    err = np.abs(cut - full).max()
    assert err <= bound * (1 + 1e-9) + 1e-15
    assert err > 0.0


@pytest.mark.parametrize("n,K,P", [(12, 24, 4), (16, 30, 5), (9, 16, 8)])
def test_hybrid_whole_polynomial_equals_serial_stepping(n, K, P):
    """m = 0 (the whole polynomials): the hybrid loop is an exact reorganisation of the
    serial loop, J identical, gradient to rounding (point by point)."""
    nu, T = 0.02, 0.3
    u, v = velocity(n)
    f = I.fourier2d(n, n, 3, 31)
    ft = I.fourier2d(n, n, 3, 32)
    Js, gs = O.ad2_gradient_serial(f, ft, u, v, nu, T, K, omega=1.0)
    Jh, gh = O.ad2_gradient_hybrid_poly(f, ft, u, v, nu, T, K, P, 0, omega=1.0)
    assert Jh == Js
    assert np.abs(gh - gs).max() <= 1e-12 * np.abs(gs).max()


def test_hybrid_truncated_error_falls_with_the_degree():
    n, nu, T, K, P = 16, 0.01, 0.5, 64, 4
    u, v = velocity(n)
    f = I.fourier2d(n, n, 3, 41)
    ft = I.fourier2d(n, n, 3, 42)
    _, gs = O.ad2_gradient_serial(f, ft, u, v, nu, T, K, omega=1.0)
    errs = []
    for m in (2, 4, 6, 8, 12):
        _, g = O.ad2_gradient_hybrid_poly(f, ft, u, v, nu, T, K, P, m, omega=1.0)
        errs.append(np.abs(g - gs).max() / np.abs(gs).max())
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[0] > 1e-5 and errs[-2] < 1e-11 and errs[-1] < 1e-14, errs


def test_hybrid_single_part_is_serial():
    """P = 1: no homogeneous problems; the one lane is the serial adjoint."""
    n, nu, T, K = 10, 0.03, 0.2, 12
    u, v = velocity(n)
    f = I.fourier2d(n, n, 3, 51)
    ft = I.fourier2d(n, n, 3, 52)
    Js, gs = O.ad2_gradient_serial(f, ft, u, v, nu, T, K, omega=1.0)
    Jh, gh = O.ad2_gradient_hybrid_poly(f, ft, u, v, nu, T, K, 1, 5, omega=1.0)
    assert Jh == Js
    assert np.abs(gh - gs).max() <= 1e-13 * np.abs(gs).max()
