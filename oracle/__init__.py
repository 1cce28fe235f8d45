"""Plain serial FP64 CPU oracle for the Paraexp direct-adjoint loop (arXiv 2004.00546).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code with
the CUDA library in ``paper_2004_00546_gb300``; the two meet only through the
seeded input generators, which hold none of the method's arithmetic.

Every function here is a thin ctypes marshaller over ``pxo.c``; the arithmetic
lives in C (see the comments there for the passage each function follows).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pxo.c")
_LIB_PATH = os.path.join(_HERE, "libpxo.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ``pxo.c`` into ``libpxo.so`` with plain gcc (no vendor libraries)."""
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], cwd=_HERE
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            sigs = {
                "pxo_ad1_apply": [_i, _d, _d, _d, _p, _p],
                "pxo_ad1_apply_T": [_i, _d, _d, _d, _p, _p],
                "pxo_ad1_cn_step": [_i, _d, _d, _d, _d, _p, _p, _p],
                "pxo_ad1_cn_step_T": [_i, _d, _d, _d, _d, _p, _p],
                "pxo_ad1_phi_dft": [_i, _d, _d, _d, _i, _d, _d, _i64, _i, _p, _p],
                "pxo_ad1_cn_gradient_serial": [_i, _d, _d, _d, _d, _i64, _p, _p, _p, _p],
                "pxo_ad1_cn_gradient_paraexp": [_i, _d, _d, _d, _d, _i64, _i, _i, _p, _p, _p, _p],
                "pxo_bu1_rhs": [_i, _d, _d, _p, _p],
                "pxo_bu1_jac": [_i, _d, _d, _p, _p, _p],
                "pxo_bu1_jac_T": [_i, _d, _d, _p, _p, _p],
                "pxo_bu1_rk4_step": [_i, _d, _d, _d, _d, _d, _p, _p, _p],
                "pxo_bu1_gradient_serial": [_i, _d, _d, _d, _i64, _d, _p, _p, _p, _p, _p, _p],
                "pxo_bu1_gradient_hybrid": [_i, _d, _d, _d, _i64, _d, _i, _i, _i, _i, _p, _p, _p,
                                            _p, _p],
                "pxo_spmv_csr": [_i64, _i64, _p, _p, _p, _p, _p],
                "pxo_bu1_nl_paraexp": [_i, _d, _d, _d, _i64, _i, _d, _p, _p, _p, _d, _i, _p, _p, _p],
                "pxo_expm": [_i, _p, _p],
                "pxo_ad1_krylov_expv": [_i, _d, _d, _d, _d, _i, _p, _p, _p],
                "pxo_partition_nonequi": [_d, _i, _d, _p],
                "pxo_leja_points": [_i, _p],
                "pxo_ad1_relpm_expv": [_i, _d, _d, _d, _d, _d, _i, _p, _p, _p, _p],
                "pxo_ad2_apply": [_i, _i, _d, _d, _p, _p, _p, _p],
                "pxo_ad2_apply_T": [_i, _i, _d, _d, _p, _p, _p, _p],
                "pxo_ad2_rk4_step": [_i, _i, _d, _d, _p, _p, _d, _d, _d, _p, _p, _p],
                "pxo_ad2_gradient_serial": [_i, _i, _d, _d, _p, _p, _d, _i64, _d, _p, _p, _p, _p],
                "pxo_csr_transpose": [_i64, _p, _p, _p, _p, _p, _p],
                "pxo_rk4_power_coeffs": [_i, _p],
                "pxo_rk4_forcing_coeffs": [_i, _d, _d, _d, _p],
                "pxo_ad2_poly_apply": [_i, _i, _d, _d, _p, _p, _d, _i, _i, _p, _p, _p],
                "pxo_ad2_gradient_hybrid_poly": [_i, _i, _d, _d, _p, _p, _d, _i64, _d, _p, _p, _i, _i, _p,
                                                 _p],
                "pxo_bu2_rhs": [_i, _d, _d, _p, _p, _p, _p],
                "pxo_bu2_jac": [_i, _d, _d, _p, _p, _p, _p, _p, _p],
                "pxo_bu2_jac_T": [_i, _d, _d, _p, _p, _p, _p, _p, _p],
                "pxo_bu2_rk4_step": [_i, _d, _d, _d, _p, _p, _p, _p],
                "pxo_bu2_direct": [_i, _d, _d, _d, _i64, _p, _p, _p, _p],
                "pxo_bu2_gradient_serial": [_i, _d, _d, _d, _i64, _p, _p, _p, _p, _p, _p, _p],
                "pxo_csr_rk4_step": [_i64, _p, _p, _p, _d, _p, _p, _p],
                "pxo_csr_gradient_serial": [_i64, _p, _p, _p, _d, _i64, _p, _p, _p, _p, _p],
                "pxo_csr_gradient_paraexp": [_i64, _p, _p, _p, _d, _i64, _i, _i, _p, _p, _p, _p, _p],
            }
            for name, argt in sigs.items():
                fn = getattr(L, name)
                fn.argtypes = argt
                fn.restype = _i
            _lib = L
    return _lib


def _in(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_p)


def _check(rc: int, name: str):
    if rc != 0:
        raise ValueError(f"{name}: invalid arguments (rc={rc})")


TWO_PI = 2.0 * np.pi


# ---- 1D advection-diffusion ------------------------------------------------
def ad1_apply(q, c, nu, L=TWO_PI, transpose=False):
    q = _in(q)
    out = np.empty_like(q)
    fn = lib().pxo_ad1_apply_T if transpose else lib().pxo_ad1_apply
    _check(fn(q.size, L, c, nu, _ptr(q), _ptr(out)), "ad1_apply")
    return out


def ad1_cn_step(q, c, nu, dt, src=None, L=TWO_PI):
    q = _in(q)
    s = None if src is None else _in(src)
    out = np.empty_like(q)
    _check(lib().pxo_ad1_cn_step(q.size, L, c, nu, dt, _ptr(q), _ptr(s), _ptr(out)), "cn_step")
    return out


def ad1_cn_step_T(q, c, nu, dt, L=TWO_PI):
    q = _in(q)
    out = np.empty_like(q)
    _check(lib().pxo_ad1_cn_step_T(q.size, L, c, nu, dt, _ptr(q), _ptr(out)), "cn_step_T")
    return out


PHI_EXP, PHI_CN, PHI_RK4 = 0, 1, 2


def ad1_phi_dft(v, c, nu, mode, t=0.0, dt=0.0, steps=0, transpose=False, L=TWO_PI):
    v = _in(v)
    out = np.empty_like(v)
    _check(lib().pxo_ad1_phi_dft(v.size, L, c, nu, mode, t, dt, int(steps), int(transpose),
                                 _ptr(v), _ptr(out)), "phi_dft")
    return out


def ad1_cn_gradient_serial(q0, c, nu, T, K, L=TWO_PI):
    q0 = _in(q0)
    J = ctypes.c_double()
    g = np.empty_like(q0)
    qT = np.empty_like(q0)
    _check(lib().pxo_ad1_cn_gradient_serial(q0.size, L, c, nu, T, int(K), _ptr(q0),
                                            ctypes.byref(J), _ptr(g), _ptr(qT)), "cn_serial")
    return J.value, g, qT


def ad1_cn_gradient_paraexp(q0, c, nu, T, K, P, phi_mode, L=TWO_PI):
    q0 = _in(q0)
    J = ctypes.c_double()
    g = np.empty_like(q0)
    qT = np.empty_like(q0)
    _check(lib().pxo_ad1_cn_gradient_paraexp(q0.size, L, c, nu, T, int(K), int(P), int(phi_mode),
                                             _ptr(q0), ctypes.byref(J), _ptr(g), _ptr(qT)),
           "cn_paraexp")
    return J.value, g, qT


def leja_points(m):
    out = np.empty(m)
    _check(lib().pxo_leja_points(m, _ptr(out)), "leja_points")
    return out


def ad1_relpm_expv(v, c, nu, t, tol=1e-13, mmax=120, L=TWO_PI):
    """exp(t A) v by the real Leja points method; returns (y, degree, substeps). Raises
    when the Newton series has not converged within mmax terms."""
    v = _in(v)
    y = np.empty_like(v)
    deg = ctypes.c_int()
    sub = ctypes.c_int()
    _check(lib().pxo_ad1_relpm_expv(v.size, L, c, nu, t, tol, mmax, _ptr(v), _ptr(y),
                                     ctypes.byref(deg), ctypes.byref(sub)), "relpm_expv")
    return y, deg.value, sub.value


def ad1_krylov_expv(v, c, nu, t, m, L=TWO_PI):
    v = _in(v)
    e = np.empty_like(v)
    p1 = np.empty_like(v)
    _check(lib().pxo_ad1_krylov_expv(v.size, L, c, nu, t, m, _ptr(v), _ptr(e), _ptr(p1)),
           "krylov_expv")
    return e, p1


# ---- 1D Burgers -------------------------------------------------------------
def bu1_rhs(u, nu, L=TWO_PI):
    u = _in(u)
    out = np.empty_like(u)
    _check(lib().pxo_bu1_rhs(u.size, L, nu, _ptr(u), _ptr(out)), "bu1_rhs")
    return out


def bu1_jac(u, w, nu, L=TWO_PI, transpose=False):
    u, w = _in(u), _in(w)
    out = np.empty_like(u)
    fn = lib().pxo_bu1_jac_T if transpose else lib().pxo_bu1_jac
    _check(fn(u.size, L, nu, _ptr(u), _ptr(w), _ptr(out)), "bu1_jac")
    return out


def bu1_rk4_step(u, f, nu, dt, t=0.0, omega=0.0, L=TWO_PI):
    u, f = _in(u), _in(f)
    out = np.empty_like(u)
    _check(lib().pxo_bu1_rk4_step(u.size, L, nu, dt, t, omega, _ptr(f), _ptr(u), _ptr(out)),
           "bu1_rk4_step")
    return out


def bu1_gradient_serial(f, g, nu, T, K, omega=0.0, u0=None, L=TWO_PI, want_traj=False):
    f, g = _in(f), _in(g)
    u0a = None if u0 is None else _in(u0)
    J = ctypes.c_double()
    grad = np.empty_like(f)
    traj = np.empty((int(K) + 1, f.size)) if want_traj else None
    _check(lib().pxo_bu1_gradient_serial(f.size, L, nu, T, int(K), omega, _ptr(u0a), _ptr(f),
                                         _ptr(g), ctypes.byref(J), _ptr(grad), _ptr(traj)),
           "bu1_serial")
    return (J.value, grad, traj) if want_traj else (J.value, grad)


HOM_MAGNUS, HOM_STEPPER = 0, 1


def bu1_gradient_hybrid(f, g, nu, T, K, P, hom_mode=HOM_MAGNUS, M_mag=25, m_kry=30, omega=0.0,
                        u0=None, L=TWO_PI):
    f, g = _in(f), _in(g)
    u0a = None if u0 is None else _in(u0)
    J = ctypes.c_double()
    grad = np.empty_like(f)
    _check(lib().pxo_bu1_gradient_hybrid(f.size, L, nu, T, int(K), omega, int(P), int(hom_mode),
                                         int(M_mag), int(m_kry), _ptr(u0a), _ptr(f), _ptr(g),
                                         ctypes.byref(J), _ptr(grad)), "bu1_hybrid")
    return J.value, grad


def spmv_csr(row_ptr, col, val, x):
    """y = A x for A in CSR form (the definition); rows = len(row_ptr) - 1, columns = len(x)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    va, xa = _in(val), _in(x)
    y = np.empty(rp.size - 1)
    _check(lib().pxo_spmv_csr(rp.size - 1, xa.size, rp.ctypes.data_as(_p), cl.ctypes.data_as(_p), _ptr(va),
                              _ptr(xa), _ptr(y)), "spmv_csr")
    return y


def bu1_nl_paraexp_direct(f, nu, T, K, P, omega=0.0, u0=None, guess=None, tol=1e-12, max_iter=50,
                          L=TWO_PI):
    """Iterative nonlinear Paraexp direct (Sec. 3.2, Alg. 2): returns (trajectory (K+1, n),
    errors of the iterations, converged)."""
    f = _in(f)
    n = f.size
    u0a = None if u0 is None else _in(u0)
    ga = None if guess is None else _in(guess)
    traj = np.empty((int(K) + 1, n))
    errs = np.zeros(int(max_iter))
    it = ctypes.c_int(0)
    rc = lib().pxo_bu1_nl_paraexp(n, L, nu, T, int(K), int(P), omega, _ptr(u0a), _ptr(f), _ptr(ga),
                                  float(tol), int(max_iter), _ptr(traj), _ptr(errs), ctypes.byref(it))
    if rc < 0:
        _check(rc, "bu1_nl_paraexp")
    return traj, errs[:it.value].copy(), rc == 0


# ---- small helpers -----------------------------------------------------------
def expm(A):
    A = _in(A)
    d = A.shape[0]
    E = np.empty_like(A)
    _check(lib().pxo_expm(d, _ptr(A), _ptr(E)), "expm")
    return E


def partition_nonequi(T, N, k):
    out = np.empty(N + 1)
    _check(lib().pxo_partition_nonequi(T, N, k, _ptr(out)), "partition_nonequi")
    return out


# ---- 2D advection-diffusion (arrays shaped (ny, nx)) -------------------------------------
def ad2_apply(q, u, v, nu, L=TWO_PI, transpose=False):
    q, u, v = _in(q), _in(u), _in(v)
    ny, nx = q.shape
    out = np.empty_like(q)
    fn = lib().pxo_ad2_apply_T if transpose else lib().pxo_ad2_apply
    _check(fn(nx, ny, L, nu, _ptr(u), _ptr(v), _ptr(q), _ptr(out)), "ad2_apply")
    return out


def ad2_rk4_step(q, u, v, nu, dt, f, t=0.0, omega=0.0, L=TWO_PI):
    q, u, v, f = _in(q), _in(u), _in(v), _in(f)
    ny, nx = q.shape
    out = np.empty_like(q)
    _check(lib().pxo_ad2_rk4_step(nx, ny, L, nu, _ptr(u), _ptr(v), dt, t, omega, _ptr(f), _ptr(q),
                                  _ptr(out)), "ad2_rk4_step")
    return out


def ad2_gradient_serial(f, f_true, u, v, nu, T, K, omega=1.0, L=TWO_PI):
    f, ft, u, v = _in(f), _in(f_true), _in(u), _in(v)
    ny, nx = f.shape
    J = ctypes.c_double()
    g = np.empty_like(f)
    _check(lib().pxo_ad2_gradient_serial(nx, ny, L, nu, _ptr(u), _ptr(v), T, int(K), omega, _ptr(f),
                                         _ptr(ft), ctypes.byref(J), _ptr(g)), "ad2_serial")
    return J.value, g


# ---- polynomial propagator of the homogeneous parts (RK4 stepper's power series) ----
def rk4_power_coeffs(k):
    """Coefficients a[0..4k] of R(z)^k, R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24."""
    a = np.empty(4 * k + 1)
    _check(lib().pxo_rk4_power_coeffs(int(k), _ptr(a)), "rk4_power_coeffs")
    return a


def rk4_forcing_coeffs(k, dt, t0, omega):
    """Coefficients b[0..4k-1] of the forcing-gradient polynomial of k RK4 steps from t0."""
    b = np.empty(4 * k)
    _check(lib().pxo_rk4_forcing_coeffs(int(k), dt, t0, omega, _ptr(b)), "rk4_forcing_coeffs")
    return b


def ad2_poly_apply(x, u, v, nu, dt, coeffs, transpose=False, L=TWO_PI):
    """sum_j coeffs[j] (dt A)^j x (A^T with transpose) for the 2D operator."""
    x, u, v, c = _in(x), _in(u), _in(v), _in(coeffs)
    ny, nx = x.shape
    out = np.empty_like(x)
    _check(lib().pxo_ad2_poly_apply(nx, ny, L, nu, _ptr(u), _ptr(v), dt, int(bool(transpose)), len(c) - 1,
                                    _ptr(c), _ptr(x), _ptr(out)), "ad2_poly_apply")
    return out


def ad2_gradient_hybrid_poly(f, f_true, u, v, nu, T, K, P, m, omega=1.0, L=TWO_PI):
    """Hybrid loop with the homogeneous adjoint by the power series cut after degree m
    (m <= 0: the whole polynomials, i.e. serial stepping reorganised)."""
    f, ft, u, v = _in(f), _in(f_true), _in(u), _in(v)
    ny, nx = f.shape
    J = ctypes.c_double()
    g = np.empty_like(f)
    _check(lib().pxo_ad2_gradient_hybrid_poly(nx, ny, L, nu, _ptr(u), _ptr(v), T, int(K), omega, _ptr(f),
                                              _ptr(ft), int(P), int(m), ctypes.byref(J), _ptr(g)),
           "ad2_hybrid_poly")
    return J.value, g


# ---- general sparse operator in CSR form -------------------------------------
def _csr(rp, col, val):
    return (np.ascontiguousarray(rp, dtype=np.int64), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


def csr_transpose(rp, col, val):
    rp, col, val = _csr(rp, col, val)
    n = rp.size - 1
    rpT = np.empty_like(rp)
    colT = np.empty(max(col.size, 1), dtype=np.int32)
    valT = np.empty(max(val.size, 1))
    _check(lib().pxo_csr_transpose(n, _ptr(rp), _ptr(col), _ptr(val), _ptr(rpT), _ptr(colT), _ptr(valT)),
           "csr_transpose")
    return rpT, colT[:col.size], valT[:val.size]


def csr_rk4_step(rp, col, val, q, dt, src=None):
    rp, col, val = _csr(rp, col, val)
    q = _in(q)
    s = None if src is None else _in(src)
    out = np.empty_like(q)
    _check(lib().pxo_csr_rk4_step(q.size, _ptr(rp), _ptr(col), _ptr(val), dt, _ptr(s), _ptr(q), _ptr(out)),
           "csr_rk4_step")
    return out


def csr_gradient_serial(rp, col, val, q0, T, K, g=None):
    rp, col, val = _csr(rp, col, val)
    q0 = _in(q0)
    ga = None if g is None else _in(g)
    J = ctypes.c_double()
    grad = np.empty_like(q0)
    qT = np.empty_like(q0)
    _check(lib().pxo_csr_gradient_serial(q0.size, _ptr(rp), _ptr(col), _ptr(val), T, int(K), _ptr(q0), _ptr(ga),
                                         ctypes.byref(J), _ptr(grad), _ptr(qT)), "csr_serial")
    return J.value, grad, qT


CSR_PHI_EXP, CSR_PHI_RK4 = 0, 2


def csr_gradient_paraexp(rp, col, val, q0, T, K, P, phi_mode, g=None):
    rp, col, val = _csr(rp, col, val)
    q0 = _in(q0)
    ga = None if g is None else _in(g)
    J = ctypes.c_double()
    grad = np.empty_like(q0)
    qT = np.empty_like(q0)
    _check(lib().pxo_csr_gradient_paraexp(q0.size, _ptr(rp), _ptr(col), _ptr(val), T, int(K), int(P),
                                          int(phi_mode), _ptr(q0), _ptr(ga), ctypes.byref(J), _ptr(grad),
                                          _ptr(qT)), "csr_paraexp")
    return J.value, grad, qT


# ---- 2D viscous Burgers (fields shaped (n, n), x fastest) ------------------------------
def _sq(a):
    a = _in(a)
    assert a.ndim == 2 and a.shape[0] == a.shape[1]
    return a


def bu2_rhs(U, V, nu, L=TWO_PI):
    U, V = _sq(U), _sq(V)
    oU, oV = np.empty_like(U), np.empty_like(V)
    _check(lib().pxo_bu2_rhs(U.shape[0], L, nu, _ptr(U), _ptr(V), _ptr(oU), _ptr(oV)), "bu2_rhs")
    return oU, oV


def bu2_jac(U, V, W1, W2, nu, L=TWO_PI, transpose=False):
    U, V, W1, W2 = _sq(U), _sq(V), _sq(W1), _sq(W2)
    o1, o2 = np.empty_like(U), np.empty_like(V)
    fn = lib().pxo_bu2_jac_T if transpose else lib().pxo_bu2_jac
    _check(fn(U.shape[0], L, nu, _ptr(U), _ptr(V), _ptr(W1), _ptr(W2), _ptr(o1), _ptr(o2)), "bu2_jac")
    return o1, o2


def bu2_rk4_step(U, V, nu, dt, L=TWO_PI):
    U, V = _sq(U), _sq(V)
    oU, oV = np.empty_like(U), np.empty_like(V)
    _check(lib().pxo_bu2_rk4_step(U.shape[0], L, nu, dt, _ptr(U), _ptr(V), _ptr(oU), _ptr(oV)), "bu2_rk4_step")
    return oU, oV


def bu2_direct(U0, V0, nu, T, K, L=TWO_PI):
    U0, V0 = _sq(U0), _sq(V0)
    UT, VT = np.empty_like(U0), np.empty_like(V0)
    _check(lib().pxo_bu2_direct(U0.shape[0], L, nu, T, int(K), _ptr(U0), _ptr(V0), _ptr(UT), _ptr(VT)), "bu2_direct")
    return UT, VT


def bu2_gradient_serial(U0, V0, Ut, Vt, nu, T, K, L=TWO_PI):
    U0, V0, Ut, Vt = _sq(U0), _sq(V0), _sq(Ut), _sq(Vt)
    J = ctypes.c_double()
    gU, gV = np.empty_like(U0), np.empty_like(V0)
    rc = lib().pxo_bu2_gradient_serial(U0.shape[0], L, nu, T, int(K), _ptr(U0), _ptr(V0), _ptr(Ut), _ptr(Vt),
                                       ctypes.byref(J), _ptr(gU), _ptr(gV))
    _check(rc, "bu2_gradient_serial")
    return J.value, gU, gV
