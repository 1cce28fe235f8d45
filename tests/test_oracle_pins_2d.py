"""Pins of the 2D oracle (advection-diffusion with a frozen velocity field, Sec. 4.2)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2004_00546_gb300 import inputs as I


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def test_constant_velocity_fourier_symbol_and_rk4_amplification():
    n, nu, c1, c2 = 32, 0.03, 0.7, -0.4
    h = 2 * np.pi / n
    u = np.full((n, n), c1)
    v = np.full((n, n), c2)
    X, Y = np.meshgrid(np.arange(n) * h, np.arange(n) * h)
    for k, l in ((1, 0), (3, 5), (16, 7)):
        z = np.exp(1j * (k * X + l * Y))
        lam = (-1j * c1 * np.sin(k * h) / h - 1j * c2 * np.sin(l * h) / h
               - 4 * nu / h**2 * (np.sin(k * h / 2) ** 2 + np.sin(l * h / 2) ** 2))
        Az = O.ad2_apply(z.real, u, v, nu) + 1j * O.ad2_apply(z.imag, u, v, nu)
        assert np.abs(Az - lam * z).max() < 1e-12 * (abs(lam) + 1)
        dt = 0.01
        w = dt * lam
        R = 1 + w + w**2 / 2 + w**3 / 6 + w**4 / 24
        zero = np.zeros((n, n))
        st = O.ad2_rk4_step(z.real, u, v, nu, dt, zero) + 1j * O.ad2_rk4_step(z.imag, u, v, nu, dt, zero)
        assert np.abs(st - R * z).max() < 1e-13


def test_transpose_dense_brute_force_variable_velocity():
    n, nu = 5, 0.1
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    E = np.eye(n * n)
    A = np.column_stack([O.ad2_apply(E[:, j].reshape(n, n), u, v, nu).ravel() for j in range(n * n)])
    AT = np.column_stack([O.ad2_apply(E[:, j].reshape(n, n), u, v, nu, transpose=True).ravel()
                          for j in range(n * n)])
    assert np.abs(AT - A.T).max() < 1e-12 * np.abs(A).max()


def test_velocity_normalised_and_laplacian_conserves_sum():
    """The streamfunction velocity is scaled to max(|u|, |v|) = 1, and with zero
    velocity the operator (pure Laplacian) conserves the sum of the field."""
    u, v = I.streamfunction_velocity(64, 64, 8, 2006)
    assert abs(max(np.abs(u).max(), np.abs(v).max()) - 1.0) < 1e-14
    q = I.fourier2d(64, 64, 6, 7)
    zero = np.zeros_like(u)
    assert abs(O.ad2_apply(q, zero, zero, 0.5).sum()) < 1e-9 * np.abs(q).sum()


def test_gradient_central_fd_exact_linear_quadratic():
    n, nu, T, K = 24, 0.02, 0.2, 40
    u, v = I.streamfunction_velocity(n, n, 4, 11)
    ft = I.fourier2d(n, n, 3, 12)
    f = I.fourier2d(n, n, 3, 13)
    J, g = O.ad2_gradient_serial(f, ft, u, v, nu, T, K, omega=1.0)
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.standard_normal((n, n))
        Jp = O.ad2_gradient_serial(f + d, ft, u, v, nu, T, K, omega=1.0)[0]
        Jm = O.ad2_gradient_serial(f - d, ft, u, v, nu, T, K, omega=1.0)[0]
        assert abs((Jp - Jm) / 2 - np.sum(g * d)) < 1e-10 * abs(np.sum(g * d))


def test_gradient_vanishes_at_the_true_forcing():
    n, nu, T, K = 16, 0.05, 0.1, 20
    u, v = I.streamfunction_velocity(n, n, 3, 21)
    ft = I.fourier2d(n, n, 3, 22)
    J, g = O.ad2_gradient_serial(ft, ft, u, v, nu, T, K)
    assert J == 0.0 and np.abs(g).max() == 0.0


@pytest.mark.parametrize("omega,t,dt", [(0.0, 0.0, 0.1), (1.0, 0.3, 0.05), (2.5, 1.1, 0.02)])
def test_rk4_forcing_stage_times_simpson(omega, t, dt):
    """With no velocity and no viscosity A = 0, and one RK4 step of dq/dt = s(t) f adds
    Simpson's rule of s over [t, t + dt] times f: the forcing is sampled at t, at t + dt/2
    (stages 2 and 3) and at t + dt (s = 1 when omega = 0)."""
    n = 8
    z = np.zeros((n, n))
    f, q = I.fourier2d(n, n, 3, 5), I.fourier2d(n, n, 3, 6)
    s = (lambda x: 1.0) if omega == 0.0 else (lambda x: math.sin(omega * x))
    got = O.ad2_rk4_step(q, z, z, 0.0, dt, f, t=t, omega=omega)
    ref = q + dt / 6.0 * (s(t) + 4.0 * s(t + dt / 2) + s(t + dt)) * f
    assert np.abs(got - ref).max() <= 1e-15 * np.abs(ref).max()


@pytest.mark.parametrize("omega", [0.0, 1.3])
def test_gradient_closed_form_without_transport(omega):
    """A = 0 (no velocity, no viscosity): q_k = c_k (f - f_true), c_k the Simpson weights of
    s summed over the first k steps, so J = (dt/T) sum_k c_k^2 ||f - f_true||^2 and
    grad J = 2 (dt/T) sum_k c_k^2 (f - f_true). This fixes the objective's normalisation
    and the adjoint's forcing quadrature without the oracle's adjoint code."""
    n, T, K = 6, 0.7, 14
    dt = T / K
    z = np.zeros((n, n))
    f, ft = I.fourier2d(n, n, 3, 7), I.fourier2d(n, n, 3, 8)
    s = (lambda x: 1.0) if omega == 0.0 else (lambda x: math.sin(omega * x))
    c = S = 0.0
    for k in range(K):
        t = k * dt
        c += dt / 6.0 * (s(t) + 4.0 * s(t + dt / 2) + s(t + dt))
        S += c * c
    d = f - ft
    J, g = O.ad2_gradient_serial(f, ft, z, z, 0.0, T, K, omega=omega)
    assert J == pytest.approx(dt / T * S * float(np.sum(d * d)), rel=1e-13)
    gref = 2.0 * dt / T * S * d
    assert np.abs(g - gref).max() <= 1e-13 * np.abs(gref).max()
