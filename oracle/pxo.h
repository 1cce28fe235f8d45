/*
 * pxo — plain, serial, FP64 CPU oracle for the Paraexp direct-adjoint loop
 * (Skene, Eggl & Schmid, "A parallel-in-time approach for accelerating
 * direct-adjoint studies", arXiv 2004.00546).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the independent reference that the
 * CUDA path is checked against. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Conventions (all functions):
 *   - host pointers, FP64, caller-owned; nothing is retained after return;
 *   - periodic grid x_i = i*h, h = L/n, n >= 3 (periodic central differences need
 *     three distinct neighbours); functions return 0 on success, -1 on invalid
 *     arguments (null pointer, n < 3, K < 1, P < 1, K % P != 0, ...).
 *   - "transpose" means the plain matrix transpose (discrete adjoint, Sec. 2:
 *     the discrete adjoint operator is the conjugate transpose; everything is real).
 */
#ifndef PXO_H
#define PXO_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* ---- 1D linear advection-diffusion, Sec. 4.2 (1D restriction) -------------
 * (A q)_i = -c (q_{i+1}-q_{i-1})/(2h) + nu (q_{i+1}-2 q_i+q_{i-1})/h^2.      */
int pxo_ad1_apply(int n, double L, double c, double nu, const double* q, double* out);
int pxo_ad1_apply_T(int n, double L, double c, double nu, const double* q, double* out);

/* Crank–Nicolson step (I - dt/2 A) out = (I + dt/2 A) q + dt*src (src may be NULL),
 * solved as a periodic tridiagonal system by Sherman–Morrison + Thomas.          */
int pxo_ad1_cn_step(int n, double L, double c, double nu, double dt, const double* q,
                    const double* src, double* out);
/* Transposed CN map: out = (I + dt/2 A^T)(I - dt/2 A^T)^{-1} q.                  */
int pxo_ad1_cn_step_T(int n, double L, double c, double nu, double dt, const double* q,
                      double* out);

/* Exact homogeneous propagator of the circulant A by a naive O(n^2) DFT.
 * mode 0 (EXP):     out = exp(t A) v                (t = time span)
 * mode 1 (STEPPER): out = R_CN(dt A)^steps v,  R_CN(z) = (1+z/2)/(1-z/2)
 * mode 2 (STEPPER): out = R_RK4(dt A)^steps v, R_RK4(z) = 1+z+z^2/2+z^3/6+z^4/24
 * transpose != 0 uses A^T.                                                     */
int pxo_ad1_phi_dft(int n, double L, double c, double nu, int mode, double t, double dt,
                    int64_t steps, int transpose, const double* v, double* out);

/* Serial direct-adjoint loop, IC control, J = 0.5 ||q(T)||^2, CN with K steps.
 * Returns J in *J, dJ/dq0 in grad (n), q(T) in qT (may be NULL).                 */
int pxo_ad1_cn_gradient_serial(int n, double L, double c, double nu, double T, int64_t K,
                               const double* q0, double* J, double* grad, double* qT);

/* Paraexp direct-adjoint loop (Alg. 1; Eqs. linzero, linInhomEqus, hom, fullsol0,
 * adjInhom, adjHomNormal, fulladjsol) for the same problem, equal partition into P
 * parts; inhomogeneous parts stepped with CN, homogeneous parts with the exact DFT
 * propagator of mode phi_mode (0 = exp, 1 = CN stepper).                          */
int pxo_ad1_cn_gradient_paraexp(int n, double L, double c, double nu, double T, int64_t K,
                                int P, int phi_mode, const double* q0, double* J,
                                double* grad, double* qT);

/* ---- 1D viscous Burgers, Sec. 4.3 (1D restriction) -------------------------
 * N(u)_i = -u_i (u_{i+1}-u_{i-1})/(2h) + nu (u_{i+1}-2u_i+u_{i-1})/h^2          */
int pxo_bu1_rhs(int n, double L, double nu, const double* u, double* out);
/* Jacobian dN/du at u applied to w, and its transpose.                          */
int pxo_bu1_jac(int n, double L, double nu, const double* u, const double* w, double* out);
int pxo_bu1_jac_T(int n, double L, double nu, const double* u, const double* w, double* out);

/* One classical RK4 step of du/dt = N(u) + s(t) f at time t; s(t) = sin(omega t),
 * or s = 1 when omega == 0.                                                      */
int pxo_bu1_rk4_step(int n, double L, double nu, double dt, double t, double omega,
                     const double* f, const double* u, double* out);

/* Serial direct-adjoint loop for forcing control f, u(0) = u0 (NULL = 0),
 * J = (1/T) sum_{j=1..K} dt ||u_j - g||^2 (rectangle rule of Eq. cost).
 * Exact discrete adjoint of the RK4 map (reverse sweep of the four stages).
 * traj (optional, (K+1)*n) receives u_0..u_K.                                    */
int pxo_bu1_gradient_serial(int n, double L, double nu, double T, int64_t K, double omega,
                            const double* u0, const double* f, const double* g, double* J,
                            double* grad, double* traj);

/* y = A x for A in CSR form, `rows` rows over `cols` columns:
 * y_i = sum_{k = row_ptr[i]}^{row_ptr[i+1]-1} val_k x_{col_k} (the definition, one row
 * after another); -1 for a column index outside [0, cols).                       */
int pxo_spmv_csr(int64_t rows, int64_t cols, const int64_t* row_ptr, const int32_t* col, const double* val,
                 const double* x, double* y);

/* Iterative nonlinear Paraexp direct (Sec. 3.2, Alg. 2, Eqs. nl, nlIter, nonlinTrans,
 * Jacobians, nlHomIter, fullsolIter) on P equal subintervals, forcing s(t) f, u(0) = u0
 * (NULL = 0). Split: A = nu d2/dx2, N(q) = -q dq/dx. Each iteration averages the
 * Jacobian of N over every subinterval at iterate q_i, solves the P inhomogeneous
 * problems from zero, carries the homogeneous problems (the stepper's own propagator)
 * and sums them into q_{i+1}; the linear problems take the serial direct's RK4 steps with
 * their source taken at the nonlinear RK4 stages of q_i, so that the fixed point is the
 * serial RK4 trajectory. Initial guess: guess ((K+1)*n) or q = u0 at every step. Stops
 * when max_s ||q_{i+1}(t_s) - q_i(t_s)|| <= tol max_s ||q_{i+1}(t_s)||, or after
 * max_iter iterations. traj ((K+1)*n) receives the last iterate, errs (max_iter) the
 * error of every iteration, *iters their number. Returns 0 when converged, 1 when not,
 * -1 on bad arguments, -2 when out of memory.                                      */
int pxo_bu1_nl_paraexp(int n, double L, double nu, double T, int64_t K, int P, double omega,
                       const double* u0, const double* f, const double* guess, double tol,
                       int max_iter, double* traj, double* errs, int* iters);

/* Hybrid serial-direct / parallel-adjoint loop (Sec. 3.3; Eqs. seriesDirect,
 * hybadjinhom, adjHomNormal, fullAdjSolHyb) with the equal partition into P parts.
 * Adjoint inhomogeneous parts: exact discrete RK4 adjoint per subinterval.
 * Adjoint homogeneous parts (chained through the subintervals):
 *   hom_mode 0: 4th-order Magnus steps of M_mag RK4 steps each (two Gauss nodes,
 *               U interpolated by 4-point Lagrange in time), exp and phi_1 by a
 *               Krylov space of dimension m_kry (Saad 1992) and a dense exponential;
 *   hom_mode 1: exact transposed RK4 stepping (consistency reference).           */
int pxo_bu1_gradient_hybrid(int n, double L, double nu, double T, int64_t K, double omega,
                            int P, int hom_mode, int M_mag, int m_kry, const double* u0,
                            const double* f, const double* g, double* J, double* grad);

/* ---- 2D linear advection-diffusion with a frozen velocity field (Sec. 4.2) ----
 * Grid [ny][nx] row-major (x fastest), h = L/nx = L/ny (nx == ny required), periodic:
 * (A q)_{j,i} = -u_{j,i} (q_{j,i+1}-q_{j,i-1})/(2h) - v_{j,i} (q_{j+1,i}-q_{j-1,i})/(2h)
 *              + nu (q_{j,i+1}+q_{j,i-1}+q_{j+1,i}+q_{j-1,i}-4 q_{j,i})/h^2.          */
int pxo_ad2_apply(int nx, int ny, double L, double nu, const double* u, const double* v,
                  const double* q, double* out);
int pxo_ad2_apply_T(int nx, int ny, double L, double nu, const double* u, const double* v,
                    const double* q, double* out);
/* One RK4 step of dq/dt = A q + s(t) f at time t, s(t) = sin(omega t) (1 if omega == 0). */
int pxo_ad2_rk4_step(int nx, int ny, double L, double nu, const double* u, const double* v,
                     double dt, double t, double omega, const double* f, const double* q,
                     double* out);
/* Serial direct-adjoint loop, forcing control f, zero initial value, tracking of the
 * trajectory driven by f_true: J = (1/T) sum_{j=1..K} dt ||q_j(f) - q_j(f_true)||^2.
 * By linearity q(f) - q(f_true) is the response to the forcing f - f_true, which is
 * what is stepped. Exact discrete adjoint of the RK4 map. */
int pxo_ad2_gradient_serial(int nx, int ny, double L, double nu, const double* u,
                            const double* v, double T, int64_t K, double omega,
                            const double* f, const double* f_true, double* J, double* grad);

/* ---- polynomial propagator of the homogeneous parts (Eq. hom / adjHomNormal with
 * operator applications only, as the ReLPM of Sec. 4.1): the RK4 stepper's propagator
 * over k steps is R(dt A)^k, R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24.
 * a[0..4k]: coefficients of R(z)^k (long double products, rounded once).          */
int pxo_rk4_power_coeffs(int k, double* a);
/* b[0..4k-1]: coefficients of b(z) = sum_{j<k} g_j(z) R(z)^{k-1-j}, g_j(dt A) =
 * d u_{j+1}/d f for RK4 step j (times t0 + j dt) of du/dt = A u + s(t) f, s(t) =
 * sin(omega t) (1 if omega == 0). b(dt A^T) h is the forcing gradient that the
 * homogeneous adjoint started from h at the end of the k steps contributes.        */
int pxo_rk4_forcing_coeffs(int k, double dt, double t0, double omega, double* b);
/* out = sum_{j=0}^{m} c[j] (dt B)^j x, B = A (transpose == 0) or A^T, the 2D
 * advection-diffusion operator; the powers formed one after another.             */
int pxo_ad2_poly_apply(int nx, int ny, double L, double nu, const double* u, const double* v, double dt,
                       int transpose, int m, const double* c, const double* x, double* out);
/* The hybrid loop (Sec. 3.3) of pxo_ad2_gradient_serial's problem on P equal parts:
 * serial direct; adjoint lanes by the exact discrete RK4 adjoint from zero; the
 * summed homogeneous adjoint problems carried down subinterval by subinterval with
 * the power series of R(dt A^T)^(K/P) and of the forcing-gradient polynomial, both
 * cut after degree m (m <= 0 or m >= 4K/P: the whole polynomials, which reproduces
 * serial stepping).                                                               */
int pxo_ad2_gradient_hybrid_poly(int nx, int ny, double L, double nu, const double* u, const double* v,
                                 double T, int64_t K, double omega, const double* f, const double* f_true,
                                 int P, int m, double* J, double* grad);

/* ---- small dense and Krylov building blocks ------------------------------- */
/* Dense matrix exponential (row-major d x d), scaling and squaring of a Taylor
 * series evaluated in long double.                                              */
int pxo_expm(int d, const double* A, double* E);
/* Krylov approximation (Saad 1992) of exp(t A) v and, optionally, t*phi_1(t A) v
 * for the 1D advection-diffusion operator (m = Krylov dimension).                */
int pxo_ad1_krylov_expv(int n, double L, double c, double nu, double t, int m,
                        const double* v, double* out_exp, double* out_phi1);

/* Real Leja points method (Sec. 4.1): m Leja points of [-2, 2] (xi_0 = 2, each next one
 * maximising the product of distances to the previous ones).                    */
int pxo_leja_points(int m, double* xi);
/* exp(t A) v for the 1D advection-diffusion operator by ReLPM: Newton interpolation of
 * phi(z) = (e^z - 1)/z at Leja points of the focal interval of the spectral ellipse,
 * exp(B) v = v + B phi(B) v, substeps keeping the ellipse's capacity <= 4, degree up to
 * mmax until the last two Newton terms fall below tol ||v||. Returns 0, -1 (bad
 * arguments) or -2 (not converged); *degree_out / *substeps_out (may be NULL).       */
int pxo_ad1_relpm_expv(int n, double L, double c, double nu, double t, double tol, int mmax,
                       const double* v, double* out, int* degree_out, int* substeps_out);

/* Non-equidistant partition of Eq. nonEquiP: T_j = T (1 - r^j)/(1 - r^N),
 * r = k/(k+1); out has N+1 entries.                                              */
int pxo_partition_nonequi(double T, int N, double k, double* out);

/* General sparse linear operator in CSR form (row_ptr int64, col int32, val FP64):
 * dq/dt = A q with classical RK4, control q(0), J = 0.5 ||q(T) - g||^2 (g may be NULL). */
int pxo_csr_transpose(int64_t n, const int64_t* rp, const int32_t* col, const double* val, int64_t* rpT,
                      int32_t* colT, double* valT);
int pxo_csr_rk4_step(int64_t n, const int64_t* rp, const int32_t* col, const double* val, double dt,
                     const double* src, const double* q, double* out);
int pxo_csr_gradient_serial(int64_t n, const int64_t* rp, const int32_t* col, const double* val, double T,
                            int64_t K, const double* q0, const double* g, double* J, double* grad,
                            double* qT);
/* phi_mode 0: exp(tau A) (Eq. hom); 2: the RK4 stepper's R(dt A)^(K/P). n <= 2048. */
int pxo_csr_gradient_paraexp(int64_t n, const int64_t* rp, const int32_t* col, const double* val, double T,
                             int64_t K, int P, int phi_mode, const double* q0, const double* g, double* J,
                             double* grad, double* qT);

/* 2D viscous Burgers on an n x n periodic grid (arrays [n][n], x fastest), RK4, control =
 * the initial state, J = 0.5 ||q(T) - q_target||^2. */
int pxo_bu2_rhs(int n, double L, double nu, const double* U, const double* V, double* oU, double* oV);
int pxo_bu2_jac(int n, double L, double nu, const double* U, const double* V, const double* W1, const double* W2,
                double* o1, double* o2);
int pxo_bu2_jac_T(int n, double L, double nu, const double* U, const double* V, const double* Z1, const double* Z2,
                  double* o1, double* o2);
int pxo_bu2_rk4_step(int n, double L, double nu, double dt, const double* U, const double* V, double* oU,
                     double* oV);
int pxo_bu2_direct(int n, double L, double nu, double T, int64_t K, const double* U0, const double* V0, double* UT,
                   double* VT);
int pxo_bu2_gradient_serial(int n, double L, double nu, double T, int64_t K, const double* U0, const double* V0,
                            const double* Ut, const double* Vt, double* J, double* gU, double* gV);

#ifdef __cplusplus
}
#endif
#endif
