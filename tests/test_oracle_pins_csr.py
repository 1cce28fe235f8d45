"""Pins of the oracle's general sparse (CSR) problem: dq/dt = A q with classical RK4,
initial-condition control and J = 0.5 ||q(T) - g||^2, serial stepping and Paraexp
(Alg. 1). Each test checks the oracle against something other than itself: the RK4
amplification polynomial on Fourier modes of a circulant operator, a dense brute-force
transpose, central differences that are exact for a quadratic objective of linear
dynamics, serial stepping reproduced by the stepper's own propagator, and the order-4
convergence of the exponential propagator's Paraexp to serial stepping."""
import numpy as np
import pytest

import oracle as O
from paper_2004_00546_gb300 import inputs as I


def stencil_csr(n, c, nu, L=2 * np.pi):
    """The 1D advection-diffusion operator of Sec. 4.2 (central differences) in CSR form."""
    h = L / n
    am, a0, ap = c / (2 * h) + nu / h ** 2, -2 * nu / h ** 2, -c / (2 * h) + nu / h ** 2
    i = np.arange(n)
    col = np.stack([(i - 1) % n, i, (i + 1) % n], 1).ravel().astype(np.int32)
    val = np.tile([am, a0, ap], n)
    rp = np.arange(0, 3 * n + 1, 3, dtype=np.int64)
    return rp, col, val


def dense(rp, col, val):
    n = rp.size - 1
    D = np.zeros((n, n))
    for r in range(n):
        for k in range(rp[r], rp[r + 1]):
            D[r, col[k]] += val[k]
    return D


@pytest.mark.parametrize("k,dt", [(1, 1e-3), (5, 4e-3), (12, 2e-3)])
def test_csr_rk4_step_is_the_rk4_polynomial_on_fourier_modes(k, dt):
    """A circulant A has the eigenvectors e^{i k x} with the central-difference symbol
    lambda_k; one RK4 step multiplies the mode by R(dt lambda_k), R(z) = 1 + z + z^2/2 +
    z^3/6 + z^4/24 (real and imaginary parts checked separately)."""
    n, c, nu = 64, 1.0, 0.02
    rp, col, val = stencil_csr(n, c, nu)
    h = 2 * np.pi / n
    th = 2 * np.pi * k / n
    lam = -1j * c * np.sin(th) / h - 4 * nu / h ** 2 * np.sin(th / 2) ** 2
    z = dt * lam
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    x = th * np.arange(n)
    got_c = O.csr_rk4_step(rp, col, val, np.cos(x), dt)
    got_s = O.csr_rk4_step(rp, col, val, np.sin(x), dt)
    assert np.abs(got_c - np.real(R * np.exp(1j * x))).max() < 1e-13
    assert np.abs(got_s - np.imag(R * np.exp(1j * x))).max() < 1e-13


def test_csr_rk4_step_with_a_constant_source_is_affine():
    """RK4 of dq/dt = A q + b with b = A q0 equals RK4 of dq/dt = A q started at q + q0,
    minus q0 (affine equivariance: the substitution of Eq. linzero is exact)."""
    rp, col, val = I.sparse_operator(40, 4, 11)
    q0 = np.random.default_rng(1).standard_normal(40)
    q = np.random.default_rng(2).standard_normal(40)
    b = dense(rp, col, val) @ q0
    a = O.csr_rk4_step(rp, col, val, q, 0.05, src=b)
    ref = O.csr_rk4_step(rp, col, val, q + q0, 0.05) - q0
    assert np.abs(a - ref).max() < 1e-13 * np.abs(ref).max()


def test_csr_transpose_matches_dense_transpose():
    for n, per in ((1, 0), (7, 2), (50, 5)):
        rp, col, val = I.sparse_operator(n, per, 100 + n)
        rpT, colT, valT = O.csr_transpose(rp, col, val)
        assert np.array_equal(dense(rpT, colT, valT), dense(rp, col, val).T)
        assert rpT[-1] == rp[-1]


@pytest.mark.parametrize("target", [False, True])
def test_csr_serial_gradient_central_fd_exact(target):
    """J is quadratic in q0 and the dynamics are linear, so the central difference with
    eps = 1 is exact: (J(q0 + d) - J(q0 - d)) / 2 = <grad, d> (P5)."""
    n, T, K = 30, 0.4, 40
    rp, col, val = I.sparse_operator(n, 3, 21)
    q0 = np.random.default_rng(3).standard_normal(n)
    g = np.random.default_rng(4).standard_normal(n) if target else None
    J, grad, qT = O.csr_gradient_serial(rp, col, val, q0, T, K, g)
    assert abs(J - 0.5 * np.sum((qT - (g if target else 0)) ** 2)) < 1e-13 * J
    for s in range(3):
        d = np.random.default_rng(10 + s).standard_normal(n)
        Jp = O.csr_gradient_serial(rp, col, val, q0 + d, T, K, g)[0]
        Jm = O.csr_gradient_serial(rp, col, val, q0 - d, T, K, g)[0]
        assert abs((Jp - Jm) / 2 - grad @ d) < 1e-11 * max(1.0, abs(grad @ d), J)


def test_csr_serial_gradient_is_the_transposed_map_brute_force():
    """grad = (M^K)^T (q(T) - g) with M = R(dt A) formed densely from unit vectors."""
    n, T, K = 12, 0.3, 9
    rp, col, val = I.sparse_operator(n, 2, 31)
    dt = T / K
    M = np.stack([O.csr_rk4_step(rp, col, val, e, dt) for e in np.eye(n)], 1)
    q0 = np.random.default_rng(5).standard_normal(n)
    g = np.random.default_rng(6).standard_normal(n)
    MK = np.linalg.matrix_power(M, K)
    J, grad, qT = O.csr_gradient_serial(rp, col, val, q0, T, K, g)
    assert np.abs(qT - MK @ q0).max() < 1e-13 * np.abs(qT).max()
    assert np.abs(grad - MK.T @ (MK @ q0 - g)).max() < 1e-12 * np.abs(grad).max()


@pytest.mark.parametrize("P", [1, 2, 5, 8])
def test_csr_paraexp_with_the_stepper_propagator_is_serial_stepping(P):
    """Paraexp with the RK4 stepper's own R(dt A)^(K/P) reproduces serial stepping (P4)."""
    n, T, K = 24, 0.5, 40
    rp, col, val = I.sparse_operator(n, 3, 41)
    q0 = np.random.default_rng(7).standard_normal(n)
    g = np.random.default_rng(8).standard_normal(n)
    Js, gs, qs = O.csr_gradient_serial(rp, col, val, q0, T, K, g)
    Jp, gp, qp = O.csr_gradient_paraexp(rp, col, val, q0, T, K, P, O.CSR_PHI_RK4, g)
    assert abs(Jp - Js) < 1e-12 * Js
    assert np.abs(qp - qs).max() < 1e-12 * np.abs(qs).max()
    assert np.abs(gp - gs).max() < 1e-12 * np.abs(gs).max()


def test_csr_paraexp_exp_converges_to_serial_with_order_four():
    """With the exact exponential on the homogeneous parts, Paraexp differs from serial
    RK4 only by the RK4 error of the propagated boundary values, which falls as dt^4:
    halving dt divides the gradient difference by about 16."""
    n, T, P = 16, 0.5, 4
    rp, col, val = I.sparse_operator(n, 3, 51, shift=2.0)
    q0 = np.random.default_rng(9).standard_normal(n)
    diffs = []
    for K in (8, 16, 32):
        _, gs, _ = O.csr_gradient_serial(rp, col, val, q0, T, K)
        _, ge, _ = O.csr_gradient_paraexp(rp, col, val, q0, T, K, P, O.CSR_PHI_EXP)
        diffs.append(np.linalg.norm(ge - gs))
    r1, r2 = diffs[0] / diffs[1], diffs[1] / diffs[2]
    assert 12.0 < r1 < 20.0 and 12.0 < r2 < 20.0, diffs


def test_csr_paraexp_exp_superposition_with_dft_exponentials():
    """On the circulant stencil in CSR form the homogeneous propagator exp(tau A) is also
    the naive-DFT diagonalisation (pinned against numpy's FFT elsewhere): q(T) =
    q0 + w_{P-1} + sum_j exp((P - j) tau A) w_{j-1}, with the lanes w stepped by RK4."""
    n, c, nu, T, K, P = 32, 1.0, 0.02, 0.5, 64, 4
    rp, col, val = stencil_csr(n, c, nu)
    q0 = I.grf_k2(n, 12)
    k, dt, tau = K // P, T / K, T / P
    src = dense(rp, col, val) @ q0
    w = []
    for _ in range(P):
        x = np.zeros(n)
        for _ in range(k):
            x = O.csr_rk4_step(rp, col, val, x, dt, src=src)
        w.append(x)
    qT = q0 + w[P - 1]
    for j in range(1, P):
        qT = qT + O.ad1_phi_dft(w[j - 1], c, nu, O.PHI_EXP, t=(P - j) * tau)
    _, _, qp = O.csr_gradient_paraexp(rp, col, val, q0, T, K, P, O.CSR_PHI_EXP)
    assert np.abs(qp - qT).max() < 1e-12 * np.abs(qT).max()
