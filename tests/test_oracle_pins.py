"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form,
an invariant, a library routine used as a textbook reference, brute force on a
tiny case, or a hand-worked example under tests/golden/. The tolerances follow
from FP64 rounding of the operations involved.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from paper_2004_00546_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def symbol_ad1(k, n, c, nu, L=2 * np.pi):
    """Closed-form symbol of the central-difference advection-diffusion operator:
    lambda_k = -i c sin(k h)/h - (4 nu / h^2) sin^2(k h / 2), k in units of 2 pi / L."""
    h = L / n
    th = 2 * np.pi * k / n
    return -1j * c * np.sin(th) / h - 4 * nu / h**2 * np.sin(th / 2) ** 2


# ---- operator and stepper closed forms (P1) --------------------------------------
@pytest.mark.parametrize("n,k", [(3, 1), (31, 5), (256, 7), (256, 127)])
def test_ad1_fourier_eigenvalue(n, k):
    c, nu = 1.0, 0.01
    x = I.grid1d(n) * 1.0
    th = 2 * np.pi * k / n * np.arange(n)
    lam = symbol_ad1(k, n, c, nu)
    # A e^{i k x} = lam e^{i k x}: real and imaginary parts separately
    Ac = O.ad1_apply(np.cos(th), c, nu)
    As = O.ad1_apply(np.sin(th), c, nu)
    ref_c = np.real(lam * np.exp(1j * th))
    ref_s = np.imag(lam * np.exp(1j * th))
    scale = abs(lam) + 1e-300
    assert np.abs(Ac - ref_c).max() / scale < 1e-12
    assert np.abs(As - ref_s).max() / scale < 1e-12
    del x


@pytest.mark.parametrize("k", [1, 8, 40, 127])
def test_cn_amplification_decay_and_phase(k):
    """One CN step multiplies mode k by r_k = (1 + dt lam/2)/(1 - dt lam/2); K steps give
    |r_k|^K decay and K arg(r_k) phase."""
    n, c, nu, T, K = 256, 1.0, 0.01, 1.0, 64
    dt = T / K
    th = 2 * np.pi * k / n * np.arange(n)
    z = np.exp(1j * th)
    lam = symbol_ad1(k, n, c, nu)
    r = (1 + dt * lam / 2) / (1 - dt * lam / 2)
    qr, qi = np.cos(th), np.sin(th)
    for _ in range(K):
        qr = O.ad1_cn_step(qr, c, nu, dt)
        qi = O.ad1_cn_step(qi, c, nu, dt)
    got = qr + 1j * qi
    ref = r**K * z
    assert np.abs(got - ref).max() < 1e-13 * max(1.0, abs(r) ** K) + 1e-15
    # decay and phase separately
    amp = np.abs(got).mean()
    # rounding leaves ~K*eps of the unit initial amplitude in a mode that decayed below it
    assert abs(amp - abs(r) ** K) <= 1e-12 * abs(r) ** K + K * 2e-16


def test_symbol_tends_to_pde_mode():
    """As h -> 0 the discrete symbol approaches the PDE's -i c k - nu k^2 at O(h^2)."""
    c, nu, k = 1.0, 0.01, 3
    errs = []
    for n in (64, 128, 256):
        lam = symbol_ad1(k, n, c, nu)
        # oracle eigenvalue from the stencil applied to the mode
        th = 2 * np.pi * k / n * np.arange(n)
        Az = O.ad1_apply(np.cos(th), c, nu) + 1j * O.ad1_apply(np.sin(th), c, nu)
        lam_oracle = (Az / np.exp(1j * th)).mean()
        assert abs(lam_oracle - lam) < 1e-10 * abs(lam)
        errs.append(abs(lam_oracle - (-1j * c * k - nu * k * k)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


# ---- exact propagators by DFT against numpy's FFT (library) ---------------------
@pytest.mark.parametrize("mode", [O.PHI_EXP, O.PHI_CN, O.PHI_RK4])
@pytest.mark.parametrize("transpose", [False, True])
def test_phi_dft_vs_fft_closed_form(mode, transpose):
    n, c, nu = 96, 1.0, 0.02
    v = I.grf_k2(n, 11)
    t, dt, steps = 0.3, 0.3 / 37, 37
    out = O.ad1_phi_dft(v, c, nu, mode, t=t, dt=dt, steps=steps, transpose=transpose)
    k = np.fft.fftfreq(n, 1.0 / n)
    lam = symbol_ad1(k, n, c, nu)
    if transpose:
        lam = np.conj(lam)  # A real: A^T has the conjugate symbol on e^{ikx}
    if mode == O.PHI_EXP:
        phi = np.exp(t * lam)
    elif mode == O.PHI_CN:
        phi = ((1 + dt * lam / 2) / (1 - dt * lam / 2)) ** steps
    else:
        z = dt * lam
        phi = (1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24) ** steps
    ref = np.real(np.fft.ifft(phi * np.fft.fft(v)))
    assert rel(out, ref) < 1e-13


def test_cn_stepping_equals_stepper_power():
    n, c, nu, dt, steps = 64, 1.0, 0.01, 1.0 / 512, 50
    v = I.grf_k2(n, 3)
    x = v.copy()
    for _ in range(steps):
        x = O.ad1_cn_step(x, c, nu, dt)
    assert rel(x, O.ad1_phi_dft(v, c, nu, O.PHI_CN, dt=dt, steps=steps)) < 1e-13


# ---- C1 gradient in closed form (P2) ---------------------------------------------
def test_c1_gradient_closed_form_full_size():
    """J = 0.5 sum_k |r_k|^{2K} |q0_k|^2 / n and g = F^{-1}(|r_k|^{2K} F q0)."""
    p = I.advdiff1d_problem()
    n, c, nu, T, K = p["n"], p["c"], p["nu"], p["T"], 4096
    q0 = p["q0"]
    J, g, qT = O.ad1_cn_gradient_serial(q0, c, nu, T, K)
    k = np.fft.fftfreq(n, 1.0 / n)
    lam = symbol_ad1(k, n, c, nu)
    dt = T / K
    r = (1 + dt * lam / 2) / (1 - dt * lam / 2)
    qh = np.fft.fft(q0)
    J_ref = 0.5 * np.sum(np.abs(r) ** (2 * K) * np.abs(qh) ** 2) / n
    g_ref = np.real(np.fft.ifft(np.abs(r) ** (2 * K) * qh))
    qT_ref = np.real(np.fft.ifft(r**K * qh))
    # 8192 sequential CN solves: rounding grows like K * eps (~1e-12); 1e-11 bounds it
    assert abs(J - J_ref) / J_ref < 1e-11
    assert rel(g, g_ref) < 1e-11
    assert rel(qT, qT_ref) < 1e-11


# ---- duality <A u, v> = <u, A^T v> (P3) -------------------------------------------
def test_duality_operators_and_steps():
    rng = np.random.default_rng(5)
    for n in (3, 17, 256):
        u, v = rng.standard_normal(n), rng.standard_normal(n)
        for c, nu in ((1.0, 0.01), (-0.7, 0.3), (0.0, 1.0)):
            lhs = v @ O.ad1_apply(u, c, nu)
            rhs = u @ O.ad1_apply(v, c, nu, transpose=True)
            assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(O.ad1_apply(u, c, nu)) * np.linalg.norm(v)
            dt = 1.0 / 300
            lhs = v @ O.ad1_cn_step(u, c, nu, dt)
            rhs = u @ O.ad1_cn_step_T(v, c, nu, dt)
            assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(u) * np.linalg.norm(v)
        U = rng.standard_normal(n)
        lhs = v @ O.bu1_jac(U, u, 0.01)
        rhs = u @ O.bu1_jac(U, v, 0.01, transpose=True)
        assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(O.bu1_jac(U, u, 0.01)) * np.linalg.norm(v)


def test_transposes_match_dense_brute_force():
    """Brute force on a tiny grid: assemble each operator column by column and compare
    the oracle's transpose with the dense matrix transpose."""
    n, c, nu, dt = 7, 0.9, 0.05, 0.01
    E = np.eye(n)
    A = np.column_stack([O.ad1_apply(E[:, j], c, nu) for j in range(n)])
    AT = np.column_stack([O.ad1_apply(E[:, j], c, nu, transpose=True) for j in range(n)])
    assert np.abs(AT - A.T).max() < 1e-12 * np.abs(A).max()
    M = np.column_stack([O.ad1_cn_step(E[:, j], c, nu, dt) for j in range(n)])
    MT = np.column_stack([O.ad1_cn_step_T(E[:, j], c, nu, dt) for j in range(n)])
    Md = np.linalg.solve(np.eye(n) - dt / 2 * A, np.eye(n) + dt / 2 * A)
    assert np.abs(M - Md).max() < 1e-14 and np.abs(MT - Md.T).max() < 1e-14
    U = np.random.default_rng(0).standard_normal(n)
    Jm = np.column_stack([O.bu1_jac(U, E[:, j], nu) for j in range(n)])
    JT = np.column_stack([O.bu1_jac(U, E[:, j], nu, transpose=True) for j in range(n)])
    assert np.abs(JT - Jm.T).max() < 1e-12 * np.abs(Jm).max()


# ---- superposition: Paraexp with the stepper propagator = serial stepping (P4) ---
@pytest.mark.parametrize("P", [1, 2, 8])
def test_paraexp_stepper_reproduces_serial_c1(P):
    p = I.advdiff1d_problem()
    args = (p["q0"], p["c"], p["nu"], p["T"], 4096)
    J, g, qT = O.ad1_cn_gradient_serial(*args)
    Jp, gp, qTp = O.ad1_cn_gradient_paraexp(*args, P, O.PHI_CN)
    assert abs(J - Jp) / J < 1e-12
    assert rel(gp, g) < 1e-12
    assert rel(qTp, qT) < 1e-12


def test_paraexp_exp_mode_is_exact_exponential_superposition():
    """EXP mode: with the exact exponential on the homogeneous parts the result equals
    the closed form built from the CN inhomogeneous lanes and e^{lam t}."""
    p = I.advdiff1d_problem(n=64)
    c, nu, T, K, P = p["c"], p["nu"], p["T"], 512, 4
    q0 = p["q0"]
    J, g, qT = O.ad1_cn_gradient_paraexp(q0, c, nu, T, K, P, O.PHI_EXP)
    n = q0.size
    k = np.fft.fftfreq(n, 1.0 / n)
    lam = symbol_ad1(k, n, c, nu)
    dt, kk, tau = T / K, K // P, T / P
    r = (1 + dt * lam / 2) / (1 - dt * lam / 2)
    # inhomogeneous lane end state in Fourier: (r^kk - 1) q0_hat (affine CN of the shifted problem)
    qh = np.fft.fft(q0)
    e = (r**kk - 1) * qh
    qT_h = qh + e + sum(np.exp((P - j) * tau * lam) * e for j in range(1, P))
    assert rel(np.real(np.fft.ifft(qT_h)), qT) < 1e-12
    lamT = qT_h
    ea = (np.conj(r) ** kk - 1) * lamT
    g_h = lamT + ea + sum(np.exp(j * tau * np.conj(lam)) * ea for j in range(1, P))
    assert rel(np.real(np.fft.ifft(g_h)), g) < 1e-12
    assert abs(J - 0.5 * np.sum(np.abs(qT_h) ** 2) / n) < 1e-12 * J


# ---- finite differences (P5, P6, P7) -------------------------------------------------
def test_central_fd_exact_for_quadratic_c1():
    p = I.advdiff1d_problem()
    args = (p["c"], p["nu"], p["T"], 4096)
    q0 = p["q0"]
    J, g, _ = O.ad1_cn_gradient_serial(q0, *args)
    rng = np.random.default_rng(7)
    for _ in range(4):
        d = rng.standard_normal(q0.size)
        Jp = O.ad1_cn_gradient_serial(q0 + d, *args)[0]
        Jm = O.ad1_cn_gradient_serial(q0 - d, *args)[0]
        assert abs((Jp - Jm) / 2 - g @ d) < 1e-11 * max(1.0, abs(g @ d)) + 1e-12 * J


def test_burgers_jacobian_central_fd_exact():
    rng = np.random.default_rng(8)
    for n in (3, 64):
        u, w = rng.standard_normal(n), rng.standard_normal(n)
        for eps in (1.0, 0.1):
            fd = (O.bu1_rhs(u + eps * w, 0.02) - O.bu1_rhs(u - eps * w, 0.02)) / (2 * eps)
            ex = O.bu1_jac(u, w, 0.02)
            assert np.abs(fd - ex).max() < 1e-11 * np.abs(ex).max()


def test_burgers_gradient_central_fd_richardson():
    n, nu, T, K = 48, 0.05, 0.5, 400
    f = I.fourier1d(n, 4, 21)
    g = I.fourier1d(n, 4, 22)
    u0 = 0.5 * I.fourier1d(n, 3, 23)
    J, grad = O.bu1_gradient_serial(f, g, nu, T, K, u0=u0)
    rng = np.random.default_rng(9)
    for _ in range(3):
        d = rng.standard_normal(n)

        def cfd(eps):
            Jp = O.bu1_gradient_serial(f + eps * d, g, nu, T, K, u0=u0)[0]
            Jm = O.bu1_gradient_serial(f - eps * d, g, nu, T, K, u0=u0)[0]
            return (Jp - Jm) / (2 * eps)

        rich = (4 * cfd(1e-3) - cfd(2e-3)) / 3
        assert abs(rich - grad @ d) < 1e-8 * abs(grad @ d) + 1e-12


def test_burgers_forcing_omega_gradient_fd():
    """Time-dependent forcing s(t) = sin(omega t): the stage times enter the gradient."""
    n, nu, T, K = 32, 0.05, 0.6, 300
    f = I.fourier1d(n, 3, 31)
    g = I.fourier1d(n, 3, 32)
    J, grad = O.bu1_gradient_serial(f, g, nu, T, K, omega=3.0)
    d = np.random.default_rng(3).standard_normal(n)

    def cfd(eps):
        Jp = O.bu1_gradient_serial(f + eps * d, g, nu, T, K, omega=3.0)[0]
        Jm = O.bu1_gradient_serial(f - eps * d, g, nu, T, K, omega=3.0)[0]
        return (Jp - Jm) / (2 * eps)

    rich = (4 * cfd(1e-3) - cfd(2e-3)) / 3
    assert abs(rich - grad @ d) < 1e-8 * abs(grad @ d)


def test_rk4_step_order_four_on_linear_problem():
    """On a tiny-amplitude Fourier mode the quadratic term is below rounding, so one RK4
    step must multiply the mode by the degree-4 Taylor polynomial R(z) of exp(z),
    z = dt * lambda_k of the diffusion symbol."""
    n, nu = 32, 0.3
    f = np.zeros(n)
    th = 2 * np.pi * 2 / n * np.arange(n)
    eps = 1e-14  # relative size of u u_x is ~ eps * k * dt: below 1e-13
    u = eps * np.cos(th)
    lam = -4 * nu / (2 * np.pi / n) ** 2 * np.sin(np.pi * 2 / n) ** 2
    for dt in (0.05, 0.1):
        z = dt * lam
        got = O.bu1_rk4_step(u, f, nu, dt)
        ref = (1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24) * u
        assert np.abs(got - ref).max() < 1e-12 * eps


# ---- invariants (P8) -------------------------------------------------------------------
def test_mean_conserved_and_energy_nonincreasing():
    p = I.advdiff1d_problem(n=128)
    q0 = p["q0"] + 0.37  # non-zero mean
    c, nu, dt = 1.0, 0.01, 1.0 / 256
    assert abs(O.ad1_apply(q0, c, nu).sum()) < 1e-10
    q = q0.copy()
    e_prev = q @ q
    for _ in range(40):
        q = O.ad1_cn_step(q, c, nu, dt)
        assert q @ q <= e_prev * (1 + 1e-14)
        e_prev = q @ q
    assert abs(q.sum() - q0.sum()) < 1e-11 * abs(q0).sum()
    e = O.ad1_phi_dft(q0, c, nu, O.PHI_EXP, t=0.7)
    assert abs(e.sum() - q0.sum()) < 1e-11 * abs(q0).sum()
    assert e @ e <= q0 @ q0


# ---- dense exponential and Krylov (P10) --------------------------------------------------
def test_expm_closed_forms_and_library():
    th = 0.8
    R = O.expm(np.array([[0.0, -th], [th, 0.0]]))
    assert np.abs(R - np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])).max() < 1e-15
    N = np.diag(np.ones(4), 1)  # nilpotent 5x5 Jordan block
    EN = O.expm(2.0 * N)
    ref = np.zeros((5, 5))
    for i in range(5):
        for j in range(i, 5):
            ref[i, j] = 2.0 ** (j - i) / math.factorial(j - i)
    assert np.abs(EN - ref).max() < 1e-14
    rng = np.random.default_rng(4)
    for d, s in ((6, 0.5), (20, 3.0), (33, 12.0)):
        A = s * rng.standard_normal((d, d)) / np.sqrt(d)
        E = O.expm(A)
        assert np.abs(E - scipy.linalg.expm(A)).max() < 1e-12 * np.abs(E).max()


def test_expm_circulant_matches_dft():
    """expm of a small circulant equals the DFT closed form."""
    n, c, nu, t = 12, 1.0, 0.05, 0.4
    E = np.eye(n)
    A = np.column_stack([O.ad1_apply(E[:, j], c, nu) for j in range(n)])
    Ex = O.expm(t * A)
    v = I.grf_k2(n, 1)
    assert rel(Ex @ v, O.ad1_phi_dft(v, c, nu, O.PHI_EXP, t=t)) < 1e-13


@pytest.mark.parametrize("t,m", [(0.02, 20), (0.05, 30), (0.125, 40)])
def test_krylov_expv_converges_to_exact(t, m):
    p = I.advdiff1d_problem()
    v = p["q0"]
    e, p1 = O.ad1_krylov_expv(v, 1.0, 0.01, t, m)
    ee = O.ad1_phi_dft(v, 1.0, 0.01, O.PHI_EXP, t=t)
    assert rel(e, ee) < 1e-11
    # phi_1(tA) v: (exp(tA) - I) (tA)^{-1} v on the mean-free part; check (tA) phi1 = exp - I
    tAp = t * O.ad1_apply(p1, 1.0, 0.01)
    assert rel(tAp, ee - v) < 1e-10


# ---- hybrid Burgers adjoint (P4 for the hybrid form, P9 Magnus order) ---------------------
def test_hybrid_stepper_homogeneous_equals_serial():
    n, nu, T, K = 64, 0.02, 0.4, 400
    f = I.fourier1d(n, 6, 41)
    g = I.fourier1d(n, 6, 42)
    J, grad = O.bu1_gradient_serial(f, g, nu, T, K)
    for P in (1, 4, 10):
        Jh, gh = O.bu1_gradient_hybrid(f, g, nu, T, K, P, O.HOM_STEPPER)
        assert Jh == J
        assert rel(gh, grad) < 1e-13


def test_magnus_homogeneous_order_four():
    n, nu, T, K, P = 64, 0.02, 0.5, 800, 4
    f = I.fourier1d(n, 6, 51)
    g = I.fourier1d(n, 6, 52)
    _, grad = O.bu1_gradient_hybrid(f, g, nu, T, K, P, O.HOM_STEPPER)
    errs = []
    for M in (40, 20, 10):
        _, gm = O.bu1_gradient_hybrid(f, g, nu, T, K, P, O.HOM_MAGNUS, M, 30)
        errs.append(rel(gm, grad))
    o1 = math.log2(errs[0] / errs[1])
    o2 = math.log2(errs[1] / errs[2])
    assert 3.7 < o1 < 4.3 and 3.7 < o2 < 4.3, errs


# ---- partition formula (P11) ---------------------------------------------------------------
def _golden(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return np.array([float(r[1]) for r in rows])


def test_partition_hand_worked_example():
    assert np.abs(O.partition_nonequi(7.0, 3, 1.0) - _golden("partition_k1_N3_T7.txt")).max() < 1e-14


def test_partition_paper_ratio():
    Tn = O.partition_nonequi(1.0, 4, 2.11)
    assert np.abs(Tn - _golden("partition_k2.11_N4_T1.txt")).max() < 2e-5
    w = np.diff(Tn)
    assert np.allclose(w[1:] / w[:-1], 2.11 / 3.11, rtol=1e-13)
    assert Tn[0] == 0.0 and abs(Tn[-1] - 1.0) < 1e-15


# ---- real Leja points method (Sec. 4.1) ----------------------------------------------------
def test_leja_points_sequence():
    """Leja points of [-2, 2]: 2, -2, 0 first; every point maximises the product of its
    distances to the earlier ones over the interval (checked on a fine grid); the points
    are distinct and, like Chebyshev points, crowd towards the ends (arcsine law)."""
    xi = O.leja_points(120)
    assert xi[0] == 2.0 and xi[1] == -2.0 and abs(xi[2]) < 1e-12
    assert len(set(np.round(xi, 12))) == len(xi) and np.all(np.abs(xi) <= 2.0)
    grid = np.linspace(-2.0, 2.0, 20001)
    for j in range(1, 25):
        prod = lambda x: np.sum(np.log(np.abs(x[:, None] - xi[None, :j]) + 1e-300), axis=1)
        assert prod(np.array([xi[j]]))[0] >= prod(grid).max() - 1e-3
    # arcsine law: the fraction of points in |x| > sqrt(2) tends to 1/2
    frac = np.mean(np.abs(xi) > np.sqrt(2.0))
    assert 0.4 < frac < 0.6


@pytest.mark.parametrize("n,c,nu,t", [(256, 1.0, 0.01, 0.125), (64, 1.0, 0.0, 0.3), (128, 0.0, 0.05, 0.2),
                                      (200, 2.0, 0.003, 1.0), (31, 1.0, 0.1, 0.5), (512, 1.0, 0.05, 0.25)])
def test_relpm_matches_the_exact_exponential(n, c, nu, t):
    """ReLPM (pure advection: degenerate focal interval; pure diffusion; mixed; stiff)
    against exp(t A) from the closed-form Fourier symbol."""
    v = I.grf_k2(n, 3)
    y, deg, sub = O.ad1_relpm_expv(v, c, nu, t, tol=1e-13)
    ye = O.ad1_phi_dft(v, c, nu, O.PHI_EXP, t=t)
    assert np.linalg.norm(y - ye) / np.linalg.norm(ye) < 1e-12
    assert 2 <= deg <= 120 and sub >= 1


def test_relpm_error_follows_its_tolerance():
    v = I.grf_k2(256, 4)
    ye = O.ad1_phi_dft(v, 1.0, 0.01, O.PHI_EXP, t=0.125)
    errs = []
    for tol in (1e-4, 1e-8, 1e-12):
        y, deg, _ = O.ad1_relpm_expv(v, 1.0, 0.01, 0.125, tol=tol)
        errs.append((np.linalg.norm(y - ye) / np.linalg.norm(v), deg))
    assert errs[0][0] > errs[1][0] > errs[2][0]
    assert errs[0][1] < errs[1][1] < errs[2][1]
    for (e, _), tol in zip(errs, (1e-4, 1e-8, 1e-12)):
        assert e < 10 * tol
    with pytest.raises(ValueError):  # the Newton series cannot converge in 4 terms
        O.ad1_relpm_expv(v, 1.0, 0.01, 0.125, tol=1e-14, mmax=4)


# ---- iterative nonlinear Paraexp direct (Sec. 3.2, Alg. 2) -------------------------------
# The iteration's linear problems take the serial direct's RK4 steps with the nonlinear
# source taken at the RK4 stages of the previous iterate, so its fixed point is the serial
# RK4 trajectory (the oracle's pinned serial direct): a dropped source term, a wrong
# Jacobian or a lost lane value in the carry moves the fixed point.
@pytest.mark.parametrize("P,omega", [(1, 0.0), (4, 0.0), (8, 1.5), (32, 1.5)])
def test_nl_paraexp_fixed_point_is_the_serial_rk4_trajectory(P, omega):
    n, nu, T, K = 32, 0.05, 0.5, 128
    f = 3.0 * I.fourier1d(n, 8, 61)
    g = I.fourier1d(n, 8, 62)
    u0 = 0.5 * I.fourier1d(n, 4, 63)
    _, _, tr = O.bu1_gradient_serial(f, g, nu, T, K, omega=omega, u0=u0, want_traj=True)
    traj, errs, ok = O.bu1_nl_paraexp_direct(f, nu, T, K, P, omega=omega, u0=u0, guess=tr, max_iter=1)
    assert ok and len(errs) == 1 and errs[0] < 1e-14
    assert np.abs(traj - tr).max() / np.abs(tr).max() < 1e-14


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16])
def test_nl_paraexp_converges_to_the_serial_rk4_trajectory(P):
    """From the guess q(t) = q0 the iterates converge to the serial RK4 trajectory."""
    n, nu, T, K = 32, 0.05, 0.5, 128
    f = 3.0 * I.fourier1d(n, 8, 71)
    g = I.fourier1d(n, 8, 72)
    u0 = 0.5 * I.fourier1d(n, 4, 73)
    _, _, tr = O.bu1_gradient_serial(f, g, nu, T, K, omega=1.5, u0=u0, want_traj=True)
    traj, errs, ok = O.bu1_nl_paraexp_direct(f, nu, T, K, P, omega=1.5, u0=u0, tol=1e-13, max_iter=60)
    assert ok and errs[-1] <= 1e-13
    assert np.all(np.diff(np.log(errs[1:])) < 0)  # contracting after the first iterate
    assert np.abs(traj - tr).max() / np.abs(tr).max() < 1e-12


def test_nl_paraexp_iterations_fall_with_the_subintervals_and_the_nonlinearity():
    """Averaging the Jacobian over shorter subintervals makes each linearisation closer to
    the local one (fewer iterations); a nearly linear problem converges at once."""
    n, nu, T, K = 32, 0.05, 0.5, 128
    g = I.fourier1d(n, 8, 62)
    f = 10.0 * I.fourier1d(n, 8, 61)
    its = []
    for P in (1, 4, 16):
        _, errs, ok = O.bu1_nl_paraexp_direct(f, nu, T, K, P, max_iter=60)
        assert ok
        its.append(len(errs))
    assert its[0] > its[1] > its[2]
    _, errs, ok = O.bu1_nl_paraexp_direct(1e-6 * f, nu, T, K, 4, max_iter=60)
    assert ok and len(errs) <= 4
    _, errs, ok = O.bu1_nl_paraexp_direct(f, nu, T, K, 4, max_iter=2)
    assert not ok and len(errs) == 2


# ---- sparse matrix-vector product in CSR form --------------------------------------------
def _csr_of_dense(A):
    rows = [np.nonzero(A[i])[0] for i in range(A.shape[0])]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    col = np.concatenate(rows).astype(np.int32) if rp[-1] else np.zeros(0, np.int32)
    val = np.concatenate([A[i, r] for i, r in enumerate(rows)]) if rp[-1] else np.zeros(0)
    return rp, col, val


@pytest.mark.parametrize("n,density", [(1, 1.0), (37, 0.05), (200, 0.2)])
def test_spmv_csr_equals_the_dense_product(n, density):
    """Random sparse matrices (empty rows included) against the dense matrix-vector
    product."""
    rng = np.random.default_rng(n)
    A = (rng.random((n, n)) < density) * rng.standard_normal((n, n))
    A[n // 2] = 0.0  # an empty row
    rp, col, val = _csr_of_dense(A)
    x = rng.standard_normal(n)
    assert np.abs(O.spmv_csr(rp, col, val, x) - A @ x).max() <= 1e-14 * max(1.0, np.abs(A).sum(1).max())


def test_spmv_csr_of_the_advection_diffusion_stencil_is_the_operator():
    """The 1D advection-diffusion stencil assembled in CSR form applies the operator A of
    the oracle's own stencil code."""
    n, c, nu = 64, 1.0, 0.01
    h = 2.0 * np.pi / n
    am, a0, ap = c / (2 * h) + nu / h ** 2, -2 * nu / h ** 2, -c / (2 * h) + nu / h ** 2
    i = np.arange(n)
    col = np.stack([(i - 1) % n, i, (i + 1) % n], 1).ravel().astype(np.int32)
    val = np.tile([am, a0, ap], n)
    rp = np.arange(0, 3 * n + 1, 3, dtype=np.int64)
    q = I.grf_k2(n, 7)
    ref = O.ad1_apply(q, c, nu)
    assert np.linalg.norm(O.spmv_csr(rp, col, val, q) - ref) / np.linalg.norm(ref) < 1e-14


def test_nl_paraexp_diverges_on_the_burgers_workload():
    """Alg. 2 from the guess q(t) = q0 on the 1D Burgers workload (n = 1024, nu = 0.005,
    T = 2, K = 20000, P = 32, the benchmark's forcing): the iterates' changes stop falling
    after the third iterate and turn non-finite; the paper warns that convergence is not
    guaranteed, and this is why the iterative direct is not built on the GPU."""
    p = I.burgers1d_problem(n=1024)
    _, errs, ok = O.bu1_nl_paraexp_direct(p["f"], 0.005, 2.0, 20000, 32, max_iter=6)
    assert not ok
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert not np.isfinite(errs[-1]) or errs[-1] >= errs[2]


# ---- Burgers advection term, Jacobian and RK4 stage times in closed form (P6, R2) -------
def _cd_symbols(k, n, L=2 * np.pi):
    """Central differences on a Fourier mode of wavenumber k (k in units of 2 pi / L):
    delta_x maps sin/cos(k x) to k~ cos/-sin with k~ = sin(k h)/h, and the 3-point
    Laplacian multiplies the mode by -d~ with d~ = 4 sin^2(k h / 2) / h^2."""
    h = L / n
    kt = np.sin(2 * np.pi * k / L * h) / h
    dt_ = 4 * np.sin(2 * np.pi * k / L * h / 2) ** 2 / h**2
    return kt, dt_


def _round_bound(n, amp_sq, amp, nu, L=2 * np.pi):
    """Rounding bound of a central-difference evaluation of mode samples: the samples
    carry absolute errors ~1e-16 x amplitude (and ~1e-16 x k x in their arguments), which
    the differences divide by 2h and h^2."""
    h = L / n
    return 1e-13 * (amp_sq / h + nu * amp / h**2)


@pytest.mark.parametrize("n,k,A,nu", [(16, 3, 1.0, 0.0), (64, 5, 1.7, 0.02), (1024, 16, 0.8, 0.005),
                                      (37, 11, 2.0, 0.1)])
def test_burgers_rhs_of_a_sine_mode_closed_form(n, k, A, nu):
    """u = A sin(k x): (u_x)_i = A k~ cos(k x_i), (u_xx)_i = -A d~ sin(k x_i), so the
    advective central-difference Burgers term is -u_i (u_x)_i = -A^2 k~ sin cos (Sec. 4.3,
    R2) and the diffusion term -nu A d~ sin(k x_i). O(1) amplitude: the quadratic term is
    of the same size as the linear one, so its sign and its advective (not conservative)
    form are both tested; the conservative form -(u^2)_x / 2 by central differences would
    give -A^2 sin(2 k h) sin(2 k x) / (4 h) instead."""
    x = 2 * np.pi * np.arange(n) / n
    kt, dd = _cd_symbols(k, n)
    u = A * np.sin(k * x)
    ref = -A * A * kt * np.sin(k * x) * np.cos(k * x) - nu * A * dd * np.sin(k * x)
    got = O.bu1_rhs(u, nu)
    scale = A * A * abs(kt) + nu * A * dd
    assert np.abs(got - ref).max() < _round_bound(n, A * A, A, nu)
    cons = -A * A * np.sin(2 * k * 2 * np.pi / n) * np.sin(2 * k * x) / (4 * 2 * np.pi / n)
    assert np.abs(got - (cons - nu * A * dd * np.sin(k * x))).max() > 1e-6 * scale


@pytest.mark.parametrize("n,k,A,B,nu", [(32, 2, 1.3, 0.4, 0.01), (200, 9, 0.6, -1.1, 0.003)])
def test_burgers_rhs_of_a_shifted_cosine_closed_form(n, k, A, B, nu):
    """u = A cos(k x) + B: -u u_x = (A cos + B) A k~ sin(k x) and nu u_xx = -nu A d~ cos(k x);
    the mean B advects the mode, which the product form carries exactly."""
    x = 2 * np.pi * np.arange(n) / n
    kt, dd = _cd_symbols(k, n)
    u = A * np.cos(k * x) + B
    ref = (A * np.cos(k * x) + B) * A * kt * np.sin(k * x) - nu * A * dd * np.cos(k * x)
    got = O.bu1_rhs(u, nu)
    assert np.abs(got - ref).max() < _round_bound(n, abs(A) * (abs(A) + abs(B)), abs(A), nu)


@pytest.mark.parametrize("n,k,l,A,B,nu", [(48, 3, 5, 1.2, 0.7, 0.02), (256, 7, 1, 0.9, 1.4, 0.005)])
def test_burgers_jacobian_closed_form_linearisation(n, k, l, A, B, nu):
    """Linearisation of N(u) = -u u_x + nu u_xx about u = A sin(k x) in direction
    w = B cos(l x): J(u) w = -w u_x - u w_x + nu w_xx
      = -B cos(l x) A k~ cos(k x) + A sin(k x) B l~ sin(l x) - nu B e~ cos(l x),
    k~, l~ and e~ the central-difference symbols of k and l. The transposed Jacobian must
    satisfy <J w, z> = <w, J^T z> with the closed-form J w."""
    x = 2 * np.pi * np.arange(n) / n
    kt, _ = _cd_symbols(k, n)
    lt, ee = _cd_symbols(l, n)
    u = A * np.sin(k * x)
    w = B * np.cos(l * x)
    ref = (-B * np.cos(l * x) * A * kt * np.cos(k * x) + A * np.sin(k * x) * B * lt * np.sin(l * x)
           - nu * B * ee * np.cos(l * x))
    got = O.bu1_jac(u, w, nu)
    scale = abs(A * B) * (abs(kt) + abs(lt)) + nu * abs(B) * ee
    assert np.abs(got - ref).max() < _round_bound(n, abs(A * B), abs(B), nu)
    z = np.random.default_rng(n + k).standard_normal(n)
    assert abs(ref @ z - w @ O.bu1_jac(u, z, nu, transpose=True)) < 1e-12 * scale * np.abs(z).sum()


@pytest.mark.parametrize("omega,t,dt", [(0.0, 0.0, 0.1), (3.0, 0.37, 0.05), (40.0, 1.1, 0.01),
                                        (1.0, 0.0, 0.5)])
def test_burgers_rk4_forcing_stage_times_simpson(omega, t, dt):
    """du/dt = s(t) f with a spatially uniform state and forcing (N(u) = 0 for uniform u):
    the classical RK4 step is then Simpson's rule, u(t + dt) = u(t) + dt/6 (s(t)
    + 4 s(t + dt/2) + s(t + dt)) f. A forcing sampled at the wrong stage times fails it."""
    n, nu = 24, 0.05
    c0, fc = 0.8, -1.3
    u = np.full(n, c0)
    f = np.full(n, fc)
    s = (lambda tt: 1.0) if omega == 0.0 else (lambda tt: math.sin(omega * tt))
    ref = c0 + dt / 6 * (s(t) + 4 * s(t + dt / 2) + s(t + dt)) * fc
    got = O.bu1_rk4_step(u, f, nu, dt, t=t, omega=omega)
    assert np.abs(got - ref).max() < 1e-15 * max(1.0, abs(ref))
    # the stage times really matter here: the left-point and mid-point rules differ
    if omega != 0.0:
        assert abs(c0 + dt * s(t) * fc - ref) > 1e-8 and abs(c0 + dt * s(t + dt / 2) * fc - ref) > 1e-12


def test_burgers_tracking_objective_of_a_uniform_trajectory():
    """A uniform initial state and a uniform forcing stay uniform: u_j = u0 + j dt fc
    exactly (Simpson of a constant), so the tracking objective of Eq. cost in the
    rectangle rule J = (1/T) sum_{j=1..K} dt ||u_j - g||^2 has the closed form
    (1/K) sum_j sum_i (u0 + j dt fc - g_i)^2."""
    n, nu, T, K = 20, 0.01, 0.5, 50
    dt = T / K
    u0, fc = 0.3, 0.9
    g = I.fourier1d(n, 3, 41)
    J, _ = O.bu1_gradient_serial(np.full(n, fc), g, nu, T, K, u0=np.full(n, u0))
    ref = sum(((u0 + j * dt * fc - g) ** 2).sum() for j in range(1, K + 1)) / K
    assert abs(J - ref) < 1e-13 * ref
