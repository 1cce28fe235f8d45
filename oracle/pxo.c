/*
 * pxo.c — plain serial FP64 CPU oracle for the Paraexp direct-adjoint loop
 * (Skene, Eggl & Schmid, arXiv 2004.00546).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path. Written for a reader
 * checking it against the paper by eye: one loop per definition, no blocking,
 * no fusion, no reordering beyond what each equation states.
 *
 * Readings of the paper that this file fixes (the paper leaves them open):
 *   - grid: periodic, L = 2*pi by default (caller passes L), x_i = i*h, h = L/n;
 *   - space: second-order central differences (Sec. 4.2 and 4.3);
 *   - time: Crank–Nicolson or classical RK4 with fixed dt (the paper used an
 *     adaptive RK45; fixed steps make the discrete adjoint exact);
 *   - adjoint: the exact transpose of the discrete direct map (Sec. 2: the
 *     discrete adjoint operator is the conjugate transpose);
 *   - homogeneous propagation: exact exponential / exact stepper powers by DFT
 *     for circulant operators; 4th-order Magnus with Krylov exponentials for the
 *     linear time-varying Burgers adjoint (Sec. 4.1 allows exponential steps for
 *     time-varying problems "with smaller time-steps").
 */
#include "pxo.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PXO_PI 3.14159265358979323846

static int bad_grid(int n, double L) { return n < 3 || !(L > 0.0); }

/* ------------------------------------------------------------------------- */
/* 1D advection-diffusion operator (Sec. 4.2, restricted to one dimension).  */
/* Stencil: (A q)_i = a_m q_{i-1} + a_0 q_i + a_p q_{i+1} with               */
/*   a_m = c/(2h) + nu/h^2, a_0 = -2 nu/h^2, a_p = -c/(2h) + nu/h^2.         */
/* ------------------------------------------------------------------------- */
static void ad1_coeffs(int n, double L, double c, double nu, double* am, double* a0,
                       double* ap) {
  double h = L / n;
  *am = c / (2.0 * h) + nu / (h * h);
  *a0 = -2.0 * nu / (h * h);
  *ap = -c / (2.0 * h) + nu / (h * h);
}

int pxo_ad1_apply(int n, double L, double c, double nu, const double* q, double* out) {
  if (bad_grid(n, L) || !q || !out) return -1;
  double am, a0, ap;
  ad1_coeffs(n, L, c, nu, &am, &a0, &ap);
  for (int i = 0; i < n; ++i) {
    int im = (i - 1 + n) % n, ip = (i + 1) % n;
    out[i] = am * q[im] + a0 * q[i] + ap * q[ip];
  }
  return 0;
}

int pxo_ad1_apply_T(int n, double L, double c, double nu, const double* q, double* out) {
  if (bad_grid(n, L) || !q || !out) return -1;
  double am, a0, ap;
  ad1_coeffs(n, L, c, nu, &am, &a0, &ap);
  /* A^T has the row stencil (a_p, a_0, a_m): column i of A holds a_m at row i+1
   * and a_p at row i-1. */
  for (int i = 0; i < n; ++i) {
    int im = (i - 1 + n) % n, ip = (i + 1) % n;
    out[i] = ap * q[im] + a0 * q[i] + am * q[ip];
  }
  return 0;
}

/* Solve the periodic tridiagonal system
 *   lo*x_{i-1} + di*x_i + up*x_{i+1} = r_i   (indices mod n)
 * by Sherman–Morrison around a plain Thomas elimination. */
static void cyclic_tridiag_solve(int n, double lo, double di, double up, const double* r,
                                 double* x) {
  /* T = B + p q^T with p = gamma e_0 + lo_corner e_{n-1}, q = e_0 + (up_corner/gamma) e_{n-1}.
   * Row 0 of T holds lo at column n-1 (corner), row n-1 holds up at column 0. */
  double gamma = -di;
  double corner_top = lo;    /* T[0][n-1] */
  double corner_bot = up;    /* T[n-1][0] */
  double* bdiag = (double*)malloc(sizeof(double) * n);
  double* cprime = (double*)malloc(sizeof(double) * n);
  double* y = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * n);
  double* pvec = (double*)calloc(n, sizeof(double));
  for (int i = 0; i < n; ++i) bdiag[i] = di;
  bdiag[0] = di - gamma;
  bdiag[n - 1] = di - corner_bot * corner_top / gamma;
  pvec[0] = gamma;
  pvec[n - 1] = corner_bot;
  /* Thomas on B for two right-hand sides: r and p. */
  for (int pass = 0; pass < 2; ++pass) {
    const double* rhs = pass == 0 ? r : pvec;
    double* sol = pass == 0 ? y : z;
    double denom = bdiag[0];
    cprime[0] = up / denom;
    sol[0] = rhs[0] / denom;
    for (int i = 1; i < n; ++i) {
      denom = bdiag[i] - lo * cprime[i - 1];
      cprime[i] = (i < n - 1) ? up / denom : 0.0;
      sol[i] = (rhs[i] - lo * sol[i - 1]) / denom;
    }
    for (int i = n - 2; i >= 0; --i) sol[i] -= cprime[i] * sol[i + 1];
  }
  double qy = y[0] + (corner_top / gamma) * y[n - 1];
  double qz = z[0] + (corner_top / gamma) * z[n - 1];
  double fac = qy / (1.0 + qz);
  for (int i = 0; i < n; ++i) x[i] = y[i] - fac * z[i];
  free(bdiag);
  free(cprime);
  free(y);
  free(z);
  free(pvec);
}

int pxo_ad1_cn_step(int n, double L, double c, double nu, double dt, const double* q,
                    const double* src, double* out) {
  if (bad_grid(n, L) || !q || !out) return -1;
  double am, a0, ap;
  ad1_coeffs(n, L, c, nu, &am, &a0, &ap);
  double th = 0.5 * dt;
  double* rhs = (double*)malloc(sizeof(double) * n);
  /* rhs = (I + dt/2 A) q + dt*src */
  for (int i = 0; i < n; ++i) {
    int im = (i - 1 + n) % n, ip = (i + 1) % n;
    double Aq = am * q[im] + a0 * q[i] + ap * q[ip];
    rhs[i] = q[i] + th * Aq + (src ? dt * src[i] : 0.0);
  }
  /* (I - dt/2 A): lower = -th*am, diag = 1 - th*a0, upper = -th*ap */
  cyclic_tridiag_solve(n, -th * am, 1.0 - th * a0, -th * ap, rhs, out);
  free(rhs);
  return 0;
}

int pxo_ad1_cn_step_T(int n, double L, double c, double nu, double dt, const double* q,
                      double* out) {
  if (bad_grid(n, L) || !q || !out) return -1;
  double am, a0, ap;
  ad1_coeffs(n, L, c, nu, &am, &a0, &ap);
  double th = 0.5 * dt;
  double* y = (double*)malloc(sizeof(double) * n);
  /* M^T = (I + th A^T)(I - th A^T)^{-1}; A^T has lower ap, upper am. */
  cyclic_tridiag_solve(n, -th * ap, 1.0 - th * a0, -th * am, q, y);
  for (int i = 0; i < n; ++i) {
    int im = (i - 1 + n) % n, ip = (i + 1) % n;
    double ATy = ap * y[im] + a0 * y[i] + am * y[ip];
    out[i] = y[i] + th * ATy;
  }
  free(y);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Exact propagators of the circulant A by a naive DFT.                      */
/* e_k(i) = exp(2 pi I k i / n) is an eigenvector: A e_k = lam_k e_k with     */
/* lam_k = a_0 + a_m w^{-k} + a_p w^{k}, w = exp(2 pi I / n).                 */
/* ------------------------------------------------------------------------- */
static double complex cpow_int(double complex z, int64_t e) {
  double complex r = 1.0;
  while (e > 0) {
    if (e & 1) r *= z;
    z *= z;
    e >>= 1;
  }
  return r;
}

int pxo_ad1_phi_dft(int n, double L, double c, double nu, int mode, double t, double dt,
                    int64_t steps, int transpose, const double* v, double* out) {
  if (bad_grid(n, L) || !v || !out || mode < 0 || mode > 2 || steps < 0) return -1;
  double am, a0, ap;
  ad1_coeffs(n, L, c, nu, &am, &a0, &ap);
  if (transpose) {
    double tmp = am;
    am = ap;
    ap = tmp;
  }
  double complex* vh = (double complex*)malloc(sizeof(double complex) * n);
  /* forward DFT: vh_k = sum_i v_i exp(-2 pi I k i / n) */
  for (int k = 0; k < n; ++k) {
    double complex s = 0.0;
    for (int i = 0; i < n; ++i) {
      double ang = -2.0 * PXO_PI * (double)(((int64_t)k * i) % n) / n;
      s += v[i] * (cos(ang) + I * sin(ang));
    }
    double ang = 2.0 * PXO_PI * k / n;
    double complex w = cos(ang) + I * sin(ang);
    double complex lam = a0 + am / w + ap * w;
    double complex phi;
    if (mode == 0) {
      phi = cexp(t * lam);
    } else if (mode == 1) {
      double complex z = dt * lam;
      phi = cpow_int((1.0 + 0.5 * z) / (1.0 - 0.5 * z), steps);
    } else {
      double complex z = dt * lam;
      phi = cpow_int(1.0 + z + z * z / 2.0 + z * z * z / 6.0 + z * z * z * z / 24.0, steps);
    }
    vh[k] = phi * s;
  }
  /* inverse DFT */
  for (int i = 0; i < n; ++i) {
    double complex s = 0.0;
    for (int k = 0; k < n; ++k) {
      double ang = 2.0 * PXO_PI * (double)(((int64_t)k * i) % n) / n;
      s += vh[k] * (cos(ang) + I * sin(ang));
    }
    out[i] = creal(s) / n;
  }
  free(vh);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Serial direct-adjoint loop, IC control, terminal objective (Sec. 2).      */
/* ------------------------------------------------------------------------- */
int pxo_ad1_cn_gradient_serial(int n, double L, double c, double nu, double T, int64_t K,
                               const double* q0, double* J, double* grad, double* qT) {
  if (bad_grid(n, L) || K < 1 || !q0 || !J || !grad) return -1;
  double dt = T / (double)K;
  double* q = (double*)malloc(sizeof(double) * n);
  double* tmp = (double*)malloc(sizeof(double) * n);
  memcpy(q, q0, sizeof(double) * n);
  for (int64_t s = 0; s < K; ++s) {
    pxo_ad1_cn_step(n, L, c, nu, dt, q, NULL, tmp);
    memcpy(q, tmp, sizeof(double) * n);
  }
  double acc = 0.0;
  for (int i = 0; i < n; ++i) acc += q[i] * q[i];
  *J = 0.5 * acc;
  if (qT) memcpy(qT, q, sizeof(double) * n);
  /* adjoint terminal condition (Eq. adjFinalTime): lambda_K = dJ/dq(T) = q(T) */
  for (int64_t s = 0; s < K; ++s) {
    pxo_ad1_cn_step_T(n, L, c, nu, dt, q, tmp);
    memcpy(q, tmp, sizeof(double) * n);
  }
  /* IC gradient (Eq. initupdate): dL/dq0 = lambda(0) */
  memcpy(grad, q, sizeof(double) * n);
  free(q);
  free(tmp);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Paraexp direct-adjoint loop (Alg. 1), global homogeneous form (Eq. hom).  */
/* ------------------------------------------------------------------------- */
int pxo_ad1_cn_gradient_paraexp(int n, double L, double c, double nu, double T, int64_t K,
                                int P, int phi_mode, const double* q0, double* J,
                                double* grad, double* qT) {
  if (bad_grid(n, L) || K < 1 || P < 1 || K % P != 0 || !q0 || !J || !grad) return -1;
  if (phi_mode != 0 && phi_mode != 1) return -1;
  double dt = T / (double)K;
  int64_t k = K / P;
  double tau = T / P; /* equal partition T_p = p*tau (Alg. 1) */
  size_t nb = sizeof(double) * n;
  double* e = (double*)malloc(nb * P);     /* inhomogeneous end states q_{I,p}(T_{p+1}) */
  double* src = (double*)malloc(nb);
  double* x = (double*)malloc(nb);
  double* tmp = (double*)malloc(nb);
  double* qTv = (double*)malloc(nb);

  /* Eq. linzero: q~ = q - q0 has zero IC and the source A q0. Its CN step is
   * (I - dt/2 A) q~' = (I + dt/2 A) q~ + dt A q0. */
  pxo_ad1_apply(n, L, c, nu, q0, src);
  /* Eq. linInhomEqus: P independent zero-IC problems on [T_p, T_{p+1}]. */
  for (int p = 0; p < P; ++p) {
    memset(x, 0, nb);
    for (int64_t s = 0; s < k; ++s) {
      pxo_ad1_cn_step(n, L, c, nu, dt, x, src, tmp);
      memcpy(x, tmp, nb);
    }
    memcpy(e + (size_t)p * n, x, nb);
  }
  /* Eq. fullsol0 at t = T: q(T) = q0 + q_{I,P-1}(T) + sum_{j=1}^{P-1} q_{H,j}(T),
   * Eq. hom: q_{H,j} propagates q_{I,j-1}(T_j) over [T_j, T]. */
  for (int i = 0; i < n; ++i) qTv[i] = q0[i] + e[(size_t)(P - 1) * n + i];
  for (int j = 1; j < P; ++j) {
    int64_t span_steps = (int64_t)(P - j) * k;
    pxo_ad1_phi_dft(n, L, c, nu, phi_mode, (P - j) * tau, dt, span_steps, 0,
                    e + (size_t)(j - 1) * n, tmp);
    for (int i = 0; i < n; ++i) qTv[i] += tmp[i];
  }
  double acc = 0.0;
  for (int i = 0; i < n; ++i) acc += qTv[i] * qTv[i];
  *J = 0.5 * acc;
  if (qT) memcpy(qT, qTv, nb);

  /* Adjoint (Eq. adjInhom): lambda~ = lambda - lambda(T), lambda(T) = q(T).
   * The transposed CN recursion lambda_s = M^T lambda_{s+1} becomes
   * lambda~_s = M^T lambda~_{s+1} + (M^T - I) lambda(T). */
  pxo_ad1_cn_step_T(n, L, c, nu, dt, qTv, tmp);
  for (int i = 0; i < n; ++i) src[i] = tmp[i] - qTv[i];
  for (int p = 0; p < P; ++p) {
    memset(x, 0, nb);
    for (int64_t s = 0; s < k; ++s) {
      pxo_ad1_cn_step_T(n, L, c, nu, dt, x, tmp);
      for (int i = 0; i < n; ++i) x[i] = tmp[i] + src[i];
    }
    memcpy(e + (size_t)p * n, x, nb); /* lambda~_{I,p}(T_p) */
  }
  /* Eq. fulladjsol at t = 0 with the global homogeneous form (Eq. adjHomNormal):
   * lambda(0) = lambda(T) + lambda~_{I,0}(0) + sum_{j=1}^{P-1} exp-propagation of
   * lambda~_{I,j}(T_j) over [0, T_j] with A^T. */
  for (int i = 0; i < n; ++i) grad[i] = qTv[i] + e[i];
  for (int j = 1; j < P; ++j) {
    int64_t span_steps = (int64_t)j * k;
    pxo_ad1_phi_dft(n, L, c, nu, phi_mode, j * tau, dt, span_steps, 1, e + (size_t)j * n, tmp);
    for (int i = 0; i < n; ++i) grad[i] += tmp[i];
  }
  free(e);
  free(src);
  free(x);
  free(tmp);
  free(qTv);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* 1D viscous Burgers (Sec. 4.3, restricted to one dimension).               */
/* ------------------------------------------------------------------------- */
int pxo_bu1_rhs(int n, double L, double nu, const double* u, double* out) {
  if (bad_grid(n, L) || !u || !out) return -1;
  double h = L / n;
  for (int i = 0; i < n; ++i) {
    int im = (i - 1 + n) % n, ip = (i + 1) % n;
    double ux = (u[ip] - u[im]) / (2.0 * h);
    double uxx = (u[ip] - 2.0 * u[i] + u[im]) / (h * h);
    out[i] = -u[i] * ux + nu * uxx;
  }
  return 0;
}

/* Linearisation about u (the 1D form of the linearised Burgers equations of
 * Sec. 4.3): J(u) w = -w * du/dx - u * dw/dx + nu * d2w/dx2, all by central FD. */
int pxo_bu1_jac(int n, double L, double nu, const double* u, const double* w, double* out) {
  if (bad_grid(n, L) || !u || !w || !out) return -1;
  double h = L / n;
  for (int i = 0; i < n; ++i) {
    int im = (i - 1 + n) % n, ip = (i + 1) % n;
    double ux = (u[ip] - u[im]) / (2.0 * h);
    double wx = (w[ip] - w[im]) / (2.0 * h);
    double wxx = (w[ip] - 2.0 * w[i] + w[im]) / (h * h);
    out[i] = -w[i] * ux - u[i] * wx + nu * wxx;
  }
  return 0;
}

/* Transpose of J(u), assembled column by column: w_j enters row j (through
 * -ux_j w_j and -2 nu/h^2 w_j), row j-1 (through -u_{j-1}/(2h) and nu/h^2) and
 * row j+1 (through +u_{j+1}/(2h) and nu/h^2). */
int pxo_bu1_jac_T(int n, double L, double nu, const double* u, const double* w, double* out) {
  if (bad_grid(n, L) || !u || !w || !out) return -1;
  double h = L / n;
  for (int j = 0; j < n; ++j) {
    int jm = (j - 1 + n) % n, jp = (j + 1) % n;
    double uxj = (u[jp] - u[jm]) / (2.0 * h);
    double diag = -uxj - 2.0 * nu / (h * h);
    /* entry J[j-1][j] = -u_{j-1}/(2h) + nu/h^2 ; entry J[j+1][j] = u_{j+1}/(2h) + nu/h^2 */
    double from_row_m = -u[jm] / (2.0 * h) + nu / (h * h);
    double from_row_p = u[jp] / (2.0 * h) + nu / (h * h);
    out[j] = diag * w[j] + from_row_m * w[jm] + from_row_p * w[jp];
  }
  return 0;
}

static double forcing_s(double omega, double t) { return omega == 0.0 ? 1.0 : sin(omega * t); }

int pxo_bu1_rk4_step(int n, double L, double nu, double dt, double t, double omega,
                     const double* f, const double* u, double* out) {
  if (bad_grid(n, L) || !f || !u || !out) return -1;
  size_t nb = sizeof(double) * n;
  double* k1 = (double*)malloc(nb);
  double* k2 = (double*)malloc(nb);
  double* k3 = (double*)malloc(nb);
  double* k4 = (double*)malloc(nb);
  double* y = (double*)malloc(nb);
  double s1 = forcing_s(omega, t), s2 = forcing_s(omega, t + 0.5 * dt),
         s4 = forcing_s(omega, t + dt);
  pxo_bu1_rhs(n, L, nu, u, k1);
  for (int i = 0; i < n; ++i) k1[i] += s1 * f[i];
  for (int i = 0; i < n; ++i) y[i] = u[i] + 0.5 * dt * k1[i];
  pxo_bu1_rhs(n, L, nu, y, k2);
  for (int i = 0; i < n; ++i) k2[i] += s2 * f[i];
  for (int i = 0; i < n; ++i) y[i] = u[i] + 0.5 * dt * k2[i];
  pxo_bu1_rhs(n, L, nu, y, k3);
  for (int i = 0; i < n; ++i) k3[i] += s2 * f[i];
  for (int i = 0; i < n; ++i) y[i] = u[i] + dt * k3[i];
  pxo_bu1_rhs(n, L, nu, y, k4);
  for (int i = 0; i < n; ++i) k4[i] += s4 * f[i];
  for (int i = 0; i < n; ++i)
    out[i] = u[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  free(k1);
  free(k2);
  free(k3);
  free(k4);
  free(y);
  return 0;
}

/* One reverse sweep of the RK4 step taken at u_s (time t): given lam = dJ/du_{s+1},
 * returns M_s^T lam in lam_out and adds G_s^T lam (G_s = du_{s+1}/df) to gacc. */
static void bu1_rk4_adjoint_step(int n, double L, double nu, double dt, double t,
                                 double omega, const double* f, const double* u,
                                 const double* lam, double* lam_out, double* gacc) {
  size_t nb = sizeof(double) * n;
  double* Y2 = (double*)malloc(nb);
  double* Y3 = (double*)malloc(nb);
  double* Y4 = (double*)malloc(nb);
  double* kk = (double*)malloc(nb);
  double* mu = (double*)malloc(nb);
  double* nv = (double*)malloc(nb);
  double s1 = forcing_s(omega, t), s2 = forcing_s(omega, t + 0.5 * dt),
         s4 = forcing_s(omega, t + dt);
  /* recompute the stage states */
  pxo_bu1_rhs(n, L, nu, u, kk);
  for (int i = 0; i < n; ++i) Y2[i] = u[i] + 0.5 * dt * (kk[i] + s1 * f[i]);
  pxo_bu1_rhs(n, L, nu, Y2, kk);
  for (int i = 0; i < n; ++i) Y3[i] = u[i] + 0.5 * dt * (kk[i] + s2 * f[i]);
  pxo_bu1_rhs(n, L, nu, Y3, kk);
  for (int i = 0; i < n; ++i) Y4[i] = u[i] + dt * (kk[i] + s2 * f[i]);
  /* reverse of the four stages */
  for (int i = 0; i < n; ++i) lam_out[i] = lam[i];
  /* stage 4: kbar4 = dt/6 lam */
  for (int i = 0; i < n; ++i) mu[i] = dt / 6.0 * lam[i];
  for (int i = 0; i < n; ++i) gacc[i] += s4 * mu[i];
  pxo_bu1_jac_T(n, L, nu, Y4, mu, nv); /* Ybar4 */
  for (int i = 0; i < n; ++i) lam_out[i] += nv[i];
  /* stage 3: kbar3 = dt/3 lam + dt Ybar4 */
  for (int i = 0; i < n; ++i) mu[i] = dt / 3.0 * lam[i] + dt * nv[i];
  for (int i = 0; i < n; ++i) gacc[i] += s2 * mu[i];
  pxo_bu1_jac_T(n, L, nu, Y3, mu, nv); /* Ybar3 */
  for (int i = 0; i < n; ++i) lam_out[i] += nv[i];
  /* stage 2: kbar2 = dt/3 lam + dt/2 Ybar3 */
  for (int i = 0; i < n; ++i) mu[i] = dt / 3.0 * lam[i] + 0.5 * dt * nv[i];
  for (int i = 0; i < n; ++i) gacc[i] += s2 * mu[i];
  pxo_bu1_jac_T(n, L, nu, Y2, mu, nv); /* Ybar2 */
  for (int i = 0; i < n; ++i) lam_out[i] += nv[i];
  /* stage 1: kbar1 = dt/6 lam + dt/2 Ybar2 */
  for (int i = 0; i < n; ++i) mu[i] = dt / 6.0 * lam[i] + 0.5 * dt * nv[i];
  for (int i = 0; i < n; ++i) gacc[i] += s1 * mu[i];
  pxo_bu1_jac_T(n, L, nu, u, mu, nv); /* Ybar1 */
  for (int i = 0; i < n; ++i) lam_out[i] += nv[i];
  free(Y2);
  free(Y3);
  free(Y4);
  free(kk);
  free(mu);
  free(nv);
}

static double bu1_direct(int n, double L, double nu, double T, int64_t K, double omega,
                         const double* u0, const double* f, const double* g, double* traj) {
  double dt = T / (double)K;
  size_t nb = sizeof(double) * n;
  if (u0)
    memcpy(traj, u0, nb);
  else
    memset(traj, 0, nb);
  double J = 0.0;
  for (int64_t s = 0; s < K; ++s) {
    double* cur = traj + (size_t)s * n;
    double* nxt = traj + (size_t)(s + 1) * n;
    pxo_bu1_rk4_step(n, L, nu, dt, s * dt, omega, f, cur, nxt);
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc += (nxt[i] - g[i]) * (nxt[i] - g[i]);
    J += dt / T * acc;
  }
  return J;
}

/* ------------------------------------------------------------------------- */
/* Sparse matrix-vector product in CSR form (the definition).                */
/* ------------------------------------------------------------------------- */
int pxo_spmv_csr(int64_t rows, int64_t cols, const int64_t* row_ptr, const int32_t* col, const double* val,
                 const double* x, double* y) {
  if (rows < 1 || cols < 1 || !row_ptr || !col || !val || !x || !y) return -1;
  for (int64_t i = 0; i < rows; ++i) {
    double s = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      if (col[k] < 0 || col[k] >= cols) return -1;
      s += val[k] * x[col[k]];
    }
    y[i] = s;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Iterative nonlinear Paraexp direct (Sec. 3.2, Alg. 2).                    */
/* ------------------------------------------------------------------------- */
/* Source of the linearised problems at a stage (Eq. nonlinTrans): N(Y) - J Y + c f with
 * N(Y) = -Y dY/dx and J = dN/dq at qbar, J Y = -Y dqbar/dx - qbar dY/dx. */
static void nl_source(int n, double L, const double* qbar, const double* Y, double c,
                      const double* f, double* out) {
  double h = L / n;
  for (int i = 0; i < n; ++i) {
    int im = (i - 1 + n) % n, ip = (i + 1) % n;
    double Yx = (Y[ip] - Y[im]) / (2.0 * h);
    double qx = (qbar[ip] - qbar[im]) / (2.0 * h);
    out[i] = -Y[i] * Yx + (Y[i] * qx + qbar[i] * Yx) + c * f[i];
  }
}

/* One RK4 step of dy/dt = (A + J) y + S_q (stage sources S[0..3], NULL = none) from y,
 * with (A + J) w = pxo_bu1_jac(qbar, w) (diffusion plus the averaged Jacobian of N). */
static void nl_lin_step(int n, double L, double nu, double dt, const double* qbar, double* const S[4],
                        double* y, double* k, double* ys, double* acc) {
  static const double cst[4] = {0.5, 0.5, 1.0, 0.0};
  static const double wgt[4] = {1.0, 2.0, 2.0, 1.0};
  for (int i = 0; i < n; ++i) acc[i] = 0.0;
  memcpy(ys, y, sizeof(double) * n);
  for (int q = 0; q < 4; ++q) {
    pxo_bu1_jac(n, L, nu, qbar, ys, k);
    if (S[0])
      for (int i = 0; i < n; ++i) k[i] += S[q][i];
    for (int i = 0; i < n; ++i) acc[i] += wgt[q] * k[i];
    if (q < 3)
      for (int i = 0; i < n; ++i) ys[i] = y[i] + cst[q] * dt * k[i];
  }
  for (int i = 0; i < n; ++i) y[i] += dt / 6.0 * acc[i];
}

int pxo_bu1_nl_paraexp(int n, double L, double nu, double T, int64_t K, int P, double omega,
                       const double* u0, const double* f, const double* guess, double tol,
                       int max_iter, double* traj, double* errs, int* iters) {
  if (bad_grid(n, L) || !f || !traj || !iters || K < 1 || P < 1 || K % P != 0 || max_iter < 1 ||
      !(tol > 0.0))
    return -1;
  const int64_t k = K / P;
  const double dt = T / (double)K;
  const size_t nb = sizeof(double) * n, rows = (size_t)(K + 1) * n;
  double* Q = traj;                               /* iterate q_i, then q_{i+1} */
  double* Qn = (double*)malloc(sizeof(double) * rows);
  double* V = (double*)malloc(sizeof(double) * rows); /* lane solutions (Eq. nonlinTrans) */
  double* qbar = (double*)malloc(nb * (size_t)P); /* qbar_p of every subinterval */
  double* S[4];
  double* Y = (double*)malloc(nb);
  double* kk = (double*)malloc(nb);
  double* ys = (double*)malloc(nb);
  double* acc = (double*)malloc(nb);
  double* y = (double*)malloc(nb);
  for (int q = 0; q < 4; ++q) S[q] = (double*)malloc(nb);
  int bad = !Qn || !V || !qbar || !Y || !kk || !ys || !acc || !y;
  for (int q = 0; q < 4; ++q) bad = bad || !S[q];
  int rc = -2;
  if (bad) goto done;
  /* Alg. 2: the initial guess of the direct solution */
  for (int64_t s = 0; s <= K; ++s) {
    double* row = Q + (size_t)s * n;
    if (guess)
      memcpy(row, guess + (size_t)s * n, nb);
    else if (u0)
      memcpy(row, u0, nb);
    else
      memset(row, 0, nb);
  }
  rc = 1;
  *iters = 0;
  for (int it = 0; it < max_iter; ++it) {
    /* lanes (Eq. nonlinTrans) on every subinterval from zero */
    for (int p = 0; p < P; ++p) {
      const int64_t a = (int64_t)p * k;
      /* Eq. Jacobians: dN/dq is linear in q, so its average over [T_p, T_{p+1}] is dN/dq
       * at the average of q_i there (trapezoid rule over the step states) */
      double* qb = qbar + (size_t)p * n;
      for (int i = 0; i < n; ++i) {
        double sum = 0.5 * (Q[(size_t)a * n + i] + Q[(size_t)(a + k) * n + i]);
        for (int64_t s = a + 1; s < a + k; ++s) sum += Q[(size_t)s * n + i];
        qb[i] = sum / (double)k;
      }
      /* the lane starts from zero at T_p; row a of V keeps lane p-1's end value */
      memset(y, 0, nb);
      for (int64_t s = a; s < a + k; ++s) {
        const double t = (double)s * dt;
        const double c1 = forcing_s(omega, t), c2 = forcing_s(omega, t + 0.5 * dt),
                     c4 = forcing_s(omega, t + dt);
        const double* qs = Q + (size_t)s * n;
        /* the nonlinear RK4 stages of q_i(t_s) and the sources there */
        nl_source(n, L, qb, qs, c1, f, S[0]);
        pxo_bu1_rhs(n, L, nu, qs, kk);
        for (int i = 0; i < n; ++i) Y[i] = qs[i] + 0.5 * dt * (kk[i] + c1 * f[i]);
        nl_source(n, L, qb, Y, c2, f, S[1]);
        pxo_bu1_rhs(n, L, nu, Y, kk);
        for (int i = 0; i < n; ++i) Y[i] = qs[i] + 0.5 * dt * (kk[i] + c2 * f[i]);
        nl_source(n, L, qb, Y, c2, f, S[2]);
        pxo_bu1_rhs(n, L, nu, Y, kk);
        for (int i = 0; i < n; ++i) Y[i] = qs[i] + dt * (kk[i] + c2 * f[i]);
        nl_source(n, L, qb, Y, c4, f, S[3]);
        nl_lin_step(n, L, nu, dt, qb, S, y, kk, ys, acc);
        memcpy(V + (size_t)(s + 1) * n, y, nb);
      }
    }
    /* homogeneous problems (Eq. nlHomIter), carried as their sum from T_p with the
     * stepper's own propagator, and the sum Eq. fullsolIter on every step */
    double* const none[4] = {NULL, NULL, NULL, NULL};
    if (u0)
      memcpy(y, u0, nb); /* q_{i+1}(0) = q0 */
    else
      memset(y, 0, nb);
    for (int p = 0; p < P; ++p) {
      const int64_t a = (int64_t)p * k;
      const double* qb = qbar + (size_t)p * n;
      memcpy(Qn + (size_t)a * n, y, nb); /* q_{i+1}(T_p): lane value 0 plus the carried sum */
      for (int64_t s = a; s < a + k; ++s) {
        nl_lin_step(n, L, nu, dt, qb, none, y, kk, ys, acc);
        double* row = Qn + (size_t)(s + 1) * n;
        const double* v = V + (size_t)(s + 1) * n;
        for (int i = 0; i < n; ++i) row[i] = v[i] + y[i];
      }
      memcpy(y, Qn + (size_t)(a + k) * n, nb); /* the carried sum at T_{p+1} */
    }
    /* the error of the iteration, then q_i <- q_{i+1} */
    double dmax = 0.0, qmax = 0.0;
    for (int64_t s = 0; s <= K; ++s) {
      double d2 = 0.0, q2 = 0.0;
      for (int i = 0; i < n; ++i) {
        double d = Qn[(size_t)s * n + i] - Q[(size_t)s * n + i];
        d2 += d * d;
        q2 += Qn[(size_t)s * n + i] * Qn[(size_t)s * n + i];
      }
      if (d2 > dmax) dmax = d2;
      if (q2 > qmax) qmax = q2;
    }
    const double err = qmax > 0.0 ? sqrt(dmax / qmax) : sqrt(dmax);
    if (errs) errs[it] = err;
    memcpy(Q, Qn, sizeof(double) * rows);
    *iters = it + 1;
    if (!(err == err) || isinf(err)) break; /* diverged to non-finite values */
    if (err <= tol) {
      rc = 0;
      break;
    }
  }
done:
  free(Qn);
  free(V);
  free(qbar);
  free(Y);
  free(kk);
  free(ys);
  free(acc);
  free(y);
  for (int q = 0; q < 4; ++q) free(S[q]);
  return rc;
}

int pxo_bu1_gradient_serial(int n, double L, double nu, double T, int64_t K, double omega,
                            const double* u0, const double* f, const double* g, double* J,
                            double* grad, double* traj) {
  if (bad_grid(n, L) || K < 1 || !f || !g || !J || !grad) return -1;
  double dt = T / (double)K;
  size_t nb = sizeof(double) * n;
  double* U = traj ? traj : (double*)malloc(nb * (size_t)(K + 1));
  if (!U) return -1;
  *J = bu1_direct(n, L, nu, T, K, omega, u0, f, g, U);
  double* lam = (double*)malloc(nb);
  double* tmp = (double*)malloc(nb);
  memset(grad, 0, nb);
  /* lambda_K = dJ/du_K = (2 dt/T)(u_K - g) */
  for (int i = 0; i < n; ++i) lam[i] = 2.0 * dt / T * (U[(size_t)K * n + i] - g[i]);
  for (int64_t s = K - 1; s >= 0; --s) {
    bu1_rk4_adjoint_step(n, L, nu, dt, s * dt, omega, f, U + (size_t)s * n, lam, tmp, grad);
    for (int i = 0; i < n; ++i)
      lam[i] = tmp[i] + (s >= 1 ? 2.0 * dt / T * (U[(size_t)s * n + i] - g[i]) : 0.0);
  }
  if (!traj) free(U);
  free(lam);
  free(tmp);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Dense exponential: scaling and squaring of a Taylor series, long double.  */
/* ------------------------------------------------------------------------- */
int pxo_expm(int d, const double* A, double* E) {
  if (d < 1 || !A || !E) return -1;
  size_t dd = (size_t)d * d;
  long double* X = (long double*)malloc(sizeof(long double) * dd);
  long double* S = (long double*)malloc(sizeof(long double) * dd);
  long double* Tm = (long double*)malloc(sizeof(long double) * dd);
  long double* W = (long double*)malloc(sizeof(long double) * dd);
  long double nrm = 0.0L; /* max column sum */
  for (int j = 0; j < d; ++j) {
    long double cs = 0.0L;
    for (int i = 0; i < d; ++i) cs += fabsl((long double)A[(size_t)i * d + j]);
    if (cs > nrm) nrm = cs;
  }
  int sq = 0;
  long double scale = 1.0L;
  while (nrm * scale > 0.125L) {
    scale *= 0.5L;
    ++sq;
  }
  for (size_t i = 0; i < dd; ++i) X[i] = (long double)A[i] * scale;
  /* S = I + X + X^2/2! + ... + X^30/30!  (||X|| <= 1/8: the tail is far below
   * long double rounding) */
  for (size_t i = 0; i < dd; ++i) S[i] = 0.0L;
  for (int i = 0; i < d; ++i) S[(size_t)i * d + i] = 1.0L;
  memcpy(Tm, S, sizeof(long double) * dd);
  for (int term = 1; term <= 30; ++term) {
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        long double acc = 0.0L;
        for (int l = 0; l < d; ++l) acc += Tm[(size_t)i * d + l] * X[(size_t)l * d + j];
        W[(size_t)i * d + j] = acc / term;
      }
    memcpy(Tm, W, sizeof(long double) * dd);
    for (size_t i = 0; i < dd; ++i) S[i] += Tm[i];
  }
  for (int s = 0; s < sq; ++s) {
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        long double acc = 0.0L;
        for (int l = 0; l < d; ++l) acc += S[(size_t)i * d + l] * S[(size_t)l * d + j];
        W[(size_t)i * d + j] = acc;
      }
    memcpy(S, W, sizeof(long double) * dd);
  }
  for (size_t i = 0; i < dd; ++i) E[i] = (double)S[i];
  free(X);
  free(S);
  free(Tm);
  free(W);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Krylov approximation of exp(B) v and phi_1(B) v (Sec. 4.1, Saad 1992):    */
/* Arnoldi with modified Gram–Schmidt builds V_{m+1}, H_m; then              */
/*   exp(B) v   ~ beta V_m exp(H_m) e_1,                                      */
/*   phi_1(B) v ~ beta V_m phi_1(H_m) e_1,                                    */
/* both read off one dense exponential of [[H_m, e_1], [0, 0]].               */
/* ------------------------------------------------------------------------- */
typedef void (*pxo_matvec)(void* ctx, const double* x, double* y);

static void krylov_exp_phi1(int n, int m, pxo_matvec op, void* ctx, const double* v,
                            double* out_exp, double* out_phi1) {
  size_t nb = sizeof(double) * n;
  double beta = 0.0;
  for (int i = 0; i < n; ++i) beta += v[i] * v[i];
  beta = sqrt(beta);
  if (beta == 0.0) {
    if (out_exp) memset(out_exp, 0, nb);
    if (out_phi1) memset(out_phi1, 0, nb);
    return;
  }
  if (m > n) m = n;
  double* V = (double*)malloc(nb * (size_t)(m + 1));
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  for (int i = 0; i < n; ++i) V[i] = v[i] / beta;
  int mm = m; /* dimension actually used (smaller on a happy breakdown) */
  for (int j = 0; j < m; ++j) {
    double* w = V + (size_t)(j + 1) * n;
    op(ctx, V + (size_t)j * n, w);
    for (int i = 0; i <= j; ++i) {
      double hij = 0.0;
      for (int l = 0; l < n; ++l) hij += V[(size_t)i * n + l] * w[l];
      H[(size_t)i * m + j] = hij;
      for (int l = 0; l < n; ++l) w[l] -= hij * V[(size_t)i * n + l];
    }
    double hn = 0.0;
    for (int l = 0; l < n; ++l) hn += w[l] * w[l];
    hn = sqrt(hn);
    H[(size_t)(j + 1) * m + j] = hn;
    if (hn <= 1e-14 * beta) { /* happy breakdown: the space is invariant */
      mm = j + 1;
      break;
    }
    for (int l = 0; l < n; ++l) w[l] /= hn;
  }
  /* dense exponential of the (mm+1) x (mm+1) augmented matrix */
  int d = mm + 1;
  double* Aug = (double*)calloc((size_t)d * d, sizeof(double));
  double* E = (double*)malloc(sizeof(double) * d * d);
  for (int i = 0; i < mm; ++i)
    for (int j = 0; j < mm; ++j) Aug[(size_t)i * d + j] = H[(size_t)i * m + j];
  Aug[(size_t)0 * d + mm] = 1.0; /* e_1 in the last column */
  pxo_expm(d, Aug, E);
  if (out_exp) {
    for (int l = 0; l < n; ++l) {
      double acc = 0.0;
      for (int i = 0; i < mm; ++i) acc += V[(size_t)i * n + l] * E[(size_t)i * d + 0];
      out_exp[l] = beta * acc;
    }
  }
  if (out_phi1) {
    for (int l = 0; l < n; ++l) {
      double acc = 0.0;
      for (int i = 0; i < mm; ++i) acc += V[(size_t)i * n + l] * E[(size_t)i * d + mm];
      out_phi1[l] = beta * acc;
    }
  }
  free(V);
  free(H);
  free(Aug);
  free(E);
}

typedef struct {
  int n;
  double L, c, nu, t;
} ad1_op_ctx;

static void ad1_scaled_op(void* vctx, const double* x, double* y) {
  ad1_op_ctx* cx = (ad1_op_ctx*)vctx;
  pxo_ad1_apply(cx->n, cx->L, cx->c, cx->nu, x, y);
  for (int i = 0; i < cx->n; ++i) y[i] *= cx->t;
}

int pxo_ad1_krylov_expv(int n, double L, double c, double nu, double t, int m,
                        const double* v, double* out_exp, double* out_phi1) {
  if (bad_grid(n, L) || m < 1 || !v || (!out_exp && !out_phi1)) return -1;
  ad1_op_ctx cx = {n, L, c, nu, t};
  krylov_exp_phi1(n, m, ad1_scaled_op, &cx, v, out_exp, out_phi1);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Real Leja points method (Sec. 4.1): exp(B) v = v + B phi(B) v with        */
/* phi(z) = (e^z - 1)/z, and phi(B) v by Newton interpolation of phi at      */
/* real Leja points of a focal interval [mu - f, mu + f] of the spectrum.    */
/* ------------------------------------------------------------------------- */

/* Leja points on [-2, 2]: xi_0 = 2; each further point maximises the product of its
 * distances to the points chosen so far (searched on a uniform grid of 2^16 + 1
 * points, which is all an interpolation sequence needs). */
int pxo_leja_points(int m, double* xi) {
  if (m < 1 || !xi) return -1;
  const int G = 65537;
  double* logd = (double*)calloc(G, sizeof(double)); /* sum of log distances per grid point */
  char* used = (char*)calloc(G, 1);
  int cur = G - 1; /* the grid point +2 */
  for (int j = 0; j < m; ++j) {
    xi[j] = -2.0 + 4.0 * cur / (G - 1);
    used[cur] = 1;
    int best = -1;
    double bv = -INFINITY;
    for (int g = 0; g < G; ++g) {
      if (used[g]) continue;
      double x = -2.0 + 4.0 * g / (G - 1);
      logd[g] += log(fabs(x - xi[j]));
      if (logd[g] > bv) {
        bv = logd[g];
        best = g;
      }
    }
    cur = best;
  }
  free(logd);
  free(used);
  return 0;
}

/* Newton divided differences D_j = phi[z_0, .., z_j] of phi(z) = (e^z - 1)/z at the
 * nodes z_0..z_m (coincident nodes allowed): by Opitz's theorem they form the first
 * column of phi(Z), Z lower bidiagonal with the nodes on the diagonal and ones below it,
 * and phi(Z) e_1 is the last column of exp([[Z, e_1], [0, 0]]). */
static int relpm_divdiff(int m, const double* z, double* D) {
  const int d = m + 2;
  double* A = (double*)calloc((size_t)d * d, sizeof(double));
  double* E = (double*)malloc(sizeof(double) * (size_t)d * d);
  for (int i = 0; i <= m; ++i) {
    A[(size_t)i * d + i] = z[i];
    if (i > 0) A[(size_t)i * d + (i - 1)] = 1.0;
  }
  A[(size_t)0 * d + (m + 1)] = 1.0;
  int rc = pxo_expm(d, A, E);
  for (int i = 0; i <= m; ++i) D[i] = E[(size_t)i * d + (m + 1)];
  free(A);
  free(E);
  return rc;
}

int pxo_ad1_relpm_expv(int n, double L, double c, double nu, double t, double tol, int mmax,
                       const double* v, double* out, int* degree_out, int* substeps_out) {
  if (bad_grid(n, L) || mmax < 2 || mmax > 200 || !(tol > 0.0) || !v || !out) return -1;
  double am, a0, ap;
  ad1_coeffs(n, L, c, nu, &am, &a0, &ap);
  /* spectrum of A: the ellipse a0 + (am + ap) cos th + i (ap - am) sin th, th in
   * [0, 2 pi): centre a0, real semi-axis |am + ap|, imaginary semi-axis |ap - am| */
  const double alpha = fabs(am + ap), beta = fabs(ap - am);
  const double mu_t = a0;                                   /* centre (per unit time) */
  const double f_t = sqrt(fmax(alpha * alpha - beta * beta, 0.0)); /* focal half-length */
  /* capacity of the smallest confocal ellipse containing the spectrum: (A + B)/2 with
   * B = beta, A = sqrt(beta^2 + f^2) >= alpha; substeps keep it <= 4 per substep */
  const double cap = 0.5 * (fmax(alpha, sqrt(beta * beta + f_t * f_t)) + beta);
  int nsub = (int)ceil(t * cap / 4.0 - 1e-12);
  if (nsub < 1) nsub = 1;
  const double ts = t / nsub;
  double* xi = (double*)malloc(sizeof(double) * (mmax + 1));
  double* z = (double*)malloc(sizeof(double) * (mmax + 1));
  double* D = (double*)malloc(sizeof(double) * (mmax + 1));
  pxo_leja_points(mmax + 1, xi);
  for (int j = 0; j <= mmax; ++j) z[j] = ts * mu_t + 0.5 * ts * f_t * xi[j];
  relpm_divdiff(mmax, z, D);
  double* x = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  double* y = (double*)malloc(sizeof(double) * n);
  memcpy(x, v, sizeof(double) * n);
  int deg_max = 0, ok = 1;
  for (int sub = 0; sub < nsub; ++sub) {
    double vn = 0.0;
    for (int i = 0; i < n; ++i) vn += x[i] * x[i];
    vn = sqrt(vn);
    /* p = sum_j D_j prod_{i<j} (B - z_i I) x,  B = ts A */
    memcpy(w, x, sizeof(double) * n);
    for (int i = 0; i < n; ++i) p[i] = D[0] * w[i];
    double prev = fabs(D[0]) * vn;
    int j = 1, conv = 0;
    for (; j <= mmax; ++j) {
      pxo_ad1_apply(n, L, c, nu, w, y);
      double wn = 0.0;
      for (int i = 0; i < n; ++i) {
        w[i] = ts * y[i] - z[j - 1] * w[i];
        wn += w[i] * w[i];
      }
      wn = sqrt(wn);
      for (int i = 0; i < n; ++i) p[i] += D[j] * w[i];
      /* a-posteriori estimate: the last two terms of the Newton series */
      const double est = fabs(D[j]) * wn;
      if (est + prev <= tol * vn) {
        conv = 1;
        break;
      }
      prev = est;
    }
    if (!conv) ok = 0;
    if (j > deg_max) deg_max = j;
    /* exp(B) x = x + B phi(B) x */
    pxo_ad1_apply(n, L, c, nu, p, y);
    for (int i = 0; i < n; ++i) x[i] = x[i] + ts * y[i];
  }
  memcpy(out, x, sizeof(double) * n);
  if (degree_out) *degree_out = deg_max;
  if (substeps_out) *substeps_out = nsub;
  free(xi);
  free(z);
  free(D);
  free(x);
  free(w);
  free(p);
  free(y);
  return ok ? 0 : -2;
}

/* ------------------------------------------------------------------------- */
/* Hybrid serial-direct / parallel-adjoint loop for 1D Burgers (Sec. 3.3).   */
/* ------------------------------------------------------------------------- */

/* 4-point Lagrange interpolation of the stored trajectory at time t. */
static void interp_traj(int n, int64_t K, double dt, const double* U, double t, double* out) {
  double s = t / dt;
  int64_t i0 = (int64_t)floor(s) - 1;
  if (i0 < 0) i0 = 0;
  if (i0 > K - 3) i0 = K - 3;
  double w[4];
  for (int a = 0; a < 4; ++a) {
    double c = 1.0;
    for (int b = 0; b < 4; ++b)
      if (b != a) c *= (s - (double)(i0 + b)) / (double)(a - b);
    w[a] = c;
  }
  for (int i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int a = 0; a < 4; ++a) acc += w[a] * U[(size_t)(i0 + a) * n + i];
    out[i] = acc;
  }
}

/* Magnus operator of one backward step for the adjoint (time reversed so that it
 * runs forward in tau): Omega x = (H/2)(B1 + B2) x + (sqrt(3)/12) H^2 (B2 B1 - B1 B2) x
 * with B_i = J(U(t_i))^T at the two Gauss nodes. */
typedef struct {
  int n;
  double L, nu, H;
  const double* U1;
  const double* U2;
  double* t1;
  double* t2;
  double* t3;
} magnus_ctx;

static void magnus_op(void* vctx, const double* x, double* y) {
  magnus_ctx* m = (magnus_ctx*)vctx;
  int n = m->n;
  double c2 = sqrt(3.0) / 12.0 * m->H * m->H;
  pxo_bu1_jac_T(n, m->L, m->nu, m->U1, x, m->t1);     /* B1 x */
  pxo_bu1_jac_T(n, m->L, m->nu, m->U2, x, m->t2);     /* B2 x */
  pxo_bu1_jac_T(n, m->L, m->nu, m->U2, m->t1, m->t3); /* B2 B1 x */
  for (int i = 0; i < n; ++i) y[i] = 0.5 * m->H * (m->t1[i] + m->t2[i]) + c2 * m->t3[i];
  pxo_bu1_jac_T(n, m->L, m->nu, m->U1, m->t2, m->t3); /* B1 B2 x */
  for (int i = 0; i < n; ++i) y[i] -= c2 * m->t3[i];
}

int pxo_bu1_gradient_hybrid(int n, double L, double nu, double T, int64_t K, double omega,
                            int P, int hom_mode, int M_mag, int m_kry, const double* u0,
                            const double* f, const double* g, double* J, double* grad) {
  if (bad_grid(n, L) || K < 4 || P < 1 || K % P != 0 || !f || !g || !J || !grad) return -1;
  int64_t k = K / P;
  if (hom_mode != 0 && hom_mode != 1) return -1;
  if (hom_mode == 0 && (M_mag < 1 || k % M_mag != 0 || m_kry < 1)) return -1;
  double dt = T / (double)K;
  size_t nb = sizeof(double) * n;
  double* U = (double*)malloc(nb * (size_t)(K + 1));
  if (!U) return -1;
  /* Eq. seriesDirect: the direct problem is solved in series; all states kept. */
  *J = bu1_direct(n, L, nu, T, K, omega, u0, f, g, U);

  double* w = (double*)malloc(nb * P); /* lambda_{I,p}(T_p) */
  double* lam = (double*)malloc(nb);
  double* tmp = (double*)malloc(nb);
  memset(grad, 0, nb);
  /* Eq. hybadjinhom: each subinterval's adjoint from a zero value at T_{p+1},
   * driven only by the objective's source (no absorbed terminal value). */
  for (int p = 0; p < P; ++p) {
    int64_t s0 = (int64_t)p * k, s1 = (int64_t)(p + 1) * k;
    for (int i = 0; i < n; ++i) lam[i] = 2.0 * dt / T * (U[(size_t)s1 * n + i] - g[i]);
    for (int64_t s = s1 - 1; s >= s0; --s) {
      bu1_rk4_adjoint_step(n, L, nu, dt, s * dt, omega, f, U + (size_t)s * n, lam, tmp, grad);
      for (int i = 0; i < n; ++i)
        lam[i] = tmp[i] + (s > s0 ? 2.0 * dt / T * (U[(size_t)s * n + i] - g[i]) : 0.0);
    }
    memcpy(w + (size_t)p * n, lam, nb);
  }
  /* Homogeneous parts (Eq. adjHomNormal): by linearity the problems active on
   * [T_p, T_{p+1}] are summed and carried down one subinterval at a time:
   * h enters subinterval p at T_{p+1} as sum_{j>p} (propagated lambda_{I,j}(T_j)). */
  double* h = (double*)calloc(n, sizeof(double));
  double* U1 = (double*)malloc(nb);
  double* U2 = (double*)malloc(nb);
  double* ex = (double*)malloc(nb);
  double* ph = (double*)malloc(nb);
  double* t1 = (double*)malloc(nb);
  double* t2 = (double*)malloc(nb);
  double* t3 = (double*)malloc(nb);
  for (int p = P - 2; p >= 0; --p) {
    for (int i = 0; i < n; ++i) h[i] += w[(size_t)(p + 1) * n + i];
    int64_t s0 = (int64_t)p * k, s1 = (int64_t)(p + 1) * k;
    if (hom_mode == 1) {
      for (int64_t s = s1 - 1; s >= s0; --s) {
        bu1_rk4_adjoint_step(n, L, nu, dt, s * dt, omega, f, U + (size_t)s * n, h, tmp, grad);
        memcpy(h, tmp, nb);
      }
    } else {
      double H = M_mag * dt;
      double g1 = 0.5 - sqrt(3.0) / 6.0, g2 = 0.5 + sqrt(3.0) / 6.0;
      for (int64_t s = s1; s > s0; s -= M_mag) {
        double ttop = s * dt;
        /* tau runs backward in t: node tau_i = tau_0 + g_i H  <=>  t_i = ttop - g_i H */
        double tn1 = ttop - g1 * H, tn2 = ttop - g2 * H;
        interp_traj(n, K, dt, U, tn1, U1);
        interp_traj(n, K, dt, U, tn2, U2);
        magnus_ctx mc = {n, L, nu, H, U1, U2, t1, t2, t3};
        krylov_exp_phi1(n, m_kry, magnus_op, &mc, h, ex, ph);
        /* gradient integral d(gamma)/d(tau) = s(t) lambda, augmented Magnus:
         * gamma += W phi_1(Omega) lambda with
         * W = (H/2)(s1+s2) I + (sqrt(3)/12) H^2 (s2 B1 - s1 B2). */
        double sa = forcing_s(omega, tn1), sb = forcing_s(omega, tn2);
        double c2 = sqrt(3.0) / 12.0 * H * H;
        pxo_bu1_jac_T(n, L, nu, U1, ph, t1);
        pxo_bu1_jac_T(n, L, nu, U2, ph, t2);
        for (int i = 0; i < n; ++i)
          grad[i] += 0.5 * H * (sa + sb) * ph[i] + c2 * (sb * t1[i] - sa * t2[i]);
        memcpy(h, ex, nb);
      }
    }
  }
  free(h);
  free(U1);
  free(U2);
  free(ex);
  free(ph);
  free(t1);
  free(t2);
  free(t3);
  free(U);
  free(w);
  free(lam);
  free(tmp);
  return 0;
}

int pxo_partition_nonequi(double T, int N, double k, double* out) {
  if (N < 1 || !(k > 0.0) || !out) return -1;
  double r = k / (k + 1.0);
  double den = 1.0 - pow(r, N);
  for (int j = 0; j <= N; ++j) out[j] = T * (1.0 - pow(r, j)) / den;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* 2D linear advection-diffusion with a frozen velocity field (Sec. 4.2).     */
/* ------------------------------------------------------------------------- */
static int bad_grid2(int nx, int ny, double L) { return nx < 3 || ny < 3 || nx != ny || !(L > 0.0); }

int pxo_ad2_apply(int nx, int ny, double L, double nu, const double* u, const double* v,
                  const double* q, double* out) {
  if (bad_grid2(nx, ny, L) || !u || !v || !q || !out) return -1;
  double h = L / nx;
  for (int j = 0; j < ny; ++j) {
    int jm = (j - 1 + ny) % ny, jp = (j + 1) % ny;
    for (int i = 0; i < nx; ++i) {
      int im = (i - 1 + nx) % nx, ip = (i + 1) % nx;
      size_t c = (size_t)j * nx + i;
      double qx = (q[(size_t)j * nx + ip] - q[(size_t)j * nx + im]) / (2.0 * h);
      double qy = (q[(size_t)jp * nx + i] - q[(size_t)jm * nx + i]) / (2.0 * h);
      double lap = (q[(size_t)j * nx + ip] + q[(size_t)j * nx + im] + q[(size_t)jp * nx + i] +
                    q[(size_t)jm * nx + i] - 4.0 * q[c]) / (h * h);
      out[c] = -u[c] * qx - v[c] * qy + nu * lap;
    }
  }
  return 0;
}

/* Transpose, entry by entry: A[(j,i),(j,i+1)] = -u_{j,i}/(2h) + nu/h^2,
 * A[(j,i),(j,i-1)] = +u_{j,i}/(2h) + nu/h^2, likewise in y with v, and
 * A[(j,i),(j,i)] = -4 nu/h^2. So (A^T l)_{j,i} = sum over the four neighbours r of
 * A[r,(j,i)] l_r: the west neighbour's row holds (j,i) as its east entry, etc. */
int pxo_ad2_apply_T(int nx, int ny, double L, double nu, const double* u, const double* v,
                    const double* q, double* out) {
  if (bad_grid2(nx, ny, L) || !u || !v || !q || !out) return -1;
  double h = L / nx;
  for (int j = 0; j < ny; ++j) {
    int jm = (j - 1 + ny) % ny, jp = (j + 1) % ny;
    for (int i = 0; i < nx; ++i) {
      int im = (i - 1 + nx) % nx, ip = (i + 1) % nx;
      size_t c = (size_t)j * nx + i;
      size_t w = (size_t)j * nx + im, e = (size_t)j * nx + ip;
      size_t s = (size_t)jm * nx + i, n = (size_t)jp * nx + i;
      /* neighbour west (j,i-1): its row has (j,i) as its east neighbour */
      double a_w = -u[w] / (2.0 * h) + nu / (h * h);
      /* neighbour east (j,i+1): (j,i) is its west neighbour */
      double a_e = u[e] / (2.0 * h) + nu / (h * h);
      double a_s = -v[s] / (2.0 * h) + nu / (h * h);
      double a_n = v[n] / (2.0 * h) + nu / (h * h);
      out[c] = a_w * q[w] + a_e * q[e] + a_s * q[s] + a_n * q[n] - 4.0 * nu / (h * h) * q[c];
    }
  }
  return 0;
}

int pxo_ad2_rk4_step(int nx, int ny, double L, double nu, const double* u, const double* v,
                     double dt, double t, double omega, const double* f, const double* q,
                     double* out) {
  if (bad_grid2(nx, ny, L) || !u || !v || !f || !q || !out) return -1;
  size_t N = (size_t)nx * ny, nb = sizeof(double) * N;
  double *k1 = malloc(nb), *k2 = malloc(nb), *k3 = malloc(nb), *k4 = malloc(nb), *y = malloc(nb);
  double s1 = forcing_s(omega, t), s2 = forcing_s(omega, t + 0.5 * dt), s4 = forcing_s(omega, t + dt);
  pxo_ad2_apply(nx, ny, L, nu, u, v, q, k1);
  for (size_t i = 0; i < N; ++i) k1[i] += s1 * f[i];
  for (size_t i = 0; i < N; ++i) y[i] = q[i] + 0.5 * dt * k1[i];
  pxo_ad2_apply(nx, ny, L, nu, u, v, y, k2);
  for (size_t i = 0; i < N; ++i) k2[i] += s2 * f[i];
  for (size_t i = 0; i < N; ++i) y[i] = q[i] + 0.5 * dt * k2[i];
  pxo_ad2_apply(nx, ny, L, nu, u, v, y, k3);
  for (size_t i = 0; i < N; ++i) k3[i] += s2 * f[i];
  for (size_t i = 0; i < N; ++i) y[i] = q[i] + dt * k3[i];
  pxo_ad2_apply(nx, ny, L, nu, u, v, y, k4);
  for (size_t i = 0; i < N; ++i) k4[i] += s4 * f[i];
  for (size_t i = 0; i < N; ++i) out[i] = q[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  free(k1); free(k2); free(k3); free(k4); free(y);
  return 0;
}

int pxo_ad2_gradient_serial(int nx, int ny, double L, double nu, const double* u,
                            const double* v, double T, int64_t K, double omega,
                            const double* f, const double* f_true, double* J, double* grad) {
  if (bad_grid2(nx, ny, L) || K < 1 || !u || !v || !f || !f_true || !J || !grad) return -1;
  size_t N = (size_t)nx * ny, nb = sizeof(double) * N;
  double dt = T / (double)K;
  double* d = malloc(nb);
  double* traj = malloc(nb * (size_t)(K + 1));
  if (!d || !traj) return -1;
  for (size_t i = 0; i < N; ++i) d[i] = f[i] - f_true[i];
  /* direct: the response e to the forcing f - f_true from e(0) = 0 */
  memset(traj, 0, nb);
  double Jacc = 0.0;
  for (int64_t s = 0; s < K; ++s) {
    pxo_ad2_rk4_step(nx, ny, L, nu, u, v, dt, s * dt, omega, d, traj + (size_t)s * N,
                     traj + (size_t)(s + 1) * N);
    double acc = 0.0;
    for (size_t i = 0; i < N; ++i) acc += traj[(size_t)(s + 1) * N + i] * traj[(size_t)(s + 1) * N + i];
    Jacc += dt / T * acc;
  }
  *J = Jacc;
  /* adjoint: reverse of the four stages of the linear RK4 map */
  double *lam = malloc(nb), *mu = malloc(nb), *nv = malloc(nb), *acc = malloc(nb);
  memset(grad, 0, nb);
  for (size_t i = 0; i < N; ++i) lam[i] = 2.0 * dt / T * traj[(size_t)K * N + i];
  for (int64_t s = K - 1; s >= 0; --s) {
    double t = s * dt;
    double s1 = forcing_s(omega, t), s2 = forcing_s(omega, t + 0.5 * dt), s4 = forcing_s(omega, t + dt);
    for (size_t i = 0; i < N; ++i) acc[i] = lam[i];
    for (size_t i = 0; i < N; ++i) mu[i] = dt / 6.0 * lam[i];            /* kbar4 */
    for (size_t i = 0; i < N; ++i) grad[i] += s4 * mu[i];
    pxo_ad2_apply_T(nx, ny, L, nu, u, v, mu, nv);                        /* Ybar4 */
    for (size_t i = 0; i < N; ++i) { acc[i] += nv[i]; mu[i] = dt / 3.0 * lam[i] + dt * nv[i]; }
    for (size_t i = 0; i < N; ++i) grad[i] += s2 * mu[i];
    pxo_ad2_apply_T(nx, ny, L, nu, u, v, mu, nv);                        /* Ybar3 */
    for (size_t i = 0; i < N; ++i) { acc[i] += nv[i]; mu[i] = dt / 3.0 * lam[i] + 0.5 * dt * nv[i]; }
    for (size_t i = 0; i < N; ++i) grad[i] += s2 * mu[i];
    pxo_ad2_apply_T(nx, ny, L, nu, u, v, mu, nv);                        /* Ybar2 */
    for (size_t i = 0; i < N; ++i) { acc[i] += nv[i]; mu[i] = dt / 6.0 * lam[i] + 0.5 * dt * nv[i]; }
    for (size_t i = 0; i < N; ++i) grad[i] += s1 * mu[i];
    pxo_ad2_apply_T(nx, ny, L, nu, u, v, mu, nv);                        /* Ybar1 */
    for (size_t i = 0; i < N; ++i)
      lam[i] = acc[i] + nv[i] + (s >= 1 ? 2.0 * dt / T * traj[(size_t)s * N + i] : 0.0);
  }
  free(d); free(traj); free(lam); free(mu); free(nv); free(acc);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Homogeneous parts by a polynomial propagator (Eq. hom / Eq. adjHomNormal  */
/* with a propagator that needs only operator applications, as the paper's  */
/* ReLPM of Sec. 4.1 does). The stepper's own propagator over a subinterval  */
/* of k classical RK4 steps is the polynomial R(dt A)^k,                     */
/*   R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24,                                  */
/* of degree 4k; its power series is cut after degree m. The forcing         */
/* gradient that the homogeneous adjoint contributes over the subinterval    */
/* (Eq. paramupdate summed over its steps) is a second polynomial in the     */
/* same operator:                                                            */
/*   b(z) = sum_{j=0}^{k-1} g_j(z) R(z)^{k-1-j},                             */
/*   g_j(z) = dt [ (s1 + 4 s2 + s4)/6 + z (s1/6 + s2/3) + z^2 (s1 + s2)/12    */
/*               + z^3 s1/24 ],                                              */
/* where g_j(dt A) = d u_{j+1} / d f is the derivative of RK4 step j of      */
/* du/dt = A u + s(t) f with respect to f (s1, s2, s4 = s(t) at the step's   */
/* stage times t_j, t_j + dt/2, t_j + dt), and b(dt A^T) h is the sum of     */
/* g_j(dt A)^T lambda_{j+1} along the homogeneous adjoint                    */
/* lambda_j = R(dt A)^T lambda_{j+1} started from h at the subinterval's end.*/
/* ------------------------------------------------------------------------- */

/* c (degree da + db) = a (degree da) * b (degree db), long double. */
static void poly_mul_ld(const long double* a, int da, const long double* b, int db, long double* c) {
  for (int i = 0; i <= da + db; ++i) c[i] = 0.0L;
  for (int i = 0; i <= da; ++i)
    for (int j = 0; j <= db; ++j) c[i + j] += a[i] * b[j];
}

/* pw[j][0..4j] = coefficients of R(z)^j for j = 0..k (pw: (k+1) x (4k+1), zero padded). */
static void rk4_powers_ld(int k, long double* pw) {
  const long double R[5] = {1.0L, 1.0L, 0.5L, 1.0L / 6.0L, 1.0L / 24.0L};
  const int w = 4 * k + 1;
  for (int i = 0; i < (k + 1) * w; ++i) pw[i] = 0.0L;
  pw[0] = 1.0L;
  for (int j = 1; j <= k; ++j) poly_mul_ld(pw + (size_t)(j - 1) * w, 4 * (j - 1), R, 4, pw + (size_t)j * w);
}

int pxo_rk4_power_coeffs(int k, double* a) {
  if (k < 1 || !a) return -1;
  const int w = 4 * k + 1;
  long double* pw = malloc(sizeof(long double) * (size_t)(k + 1) * w);
  if (!pw) return -1;
  rk4_powers_ld(k, pw);
  for (int i = 0; i < w; ++i) a[i] = (double)pw[(size_t)k * w + i];
  free(pw);
  return 0;
}

int pxo_rk4_forcing_coeffs(int k, double dt, double t0, double omega, double* b) {
  if (k < 1 || !b || !(dt > 0.0)) return -1;
  const int w = 4 * k + 1;
  long double* pw = malloc(sizeof(long double) * (size_t)(k + 1) * w);
  long double* acc = malloc(sizeof(long double) * (size_t)w);
  long double* term = malloc(sizeof(long double) * (size_t)(w + 3));
  if (!pw || !acc || !term) {
    free(pw); free(acc); free(term);
    return -1;
  }
  rk4_powers_ld(k, pw);
  for (int i = 0; i < w; ++i) acc[i] = 0.0L;
  for (int j = 0; j < k; ++j) {
    double t = t0 + j * dt;
    long double s1 = forcing_s(omega, t), s2 = forcing_s(omega, t + 0.5 * dt), s4 = forcing_s(omega, t + dt);
    long double g[4] = {(long double)dt * (s1 + 4.0L * s2 + s4) / 6.0L, (long double)dt * (s1 / 6.0L + s2 / 3.0L),
                        (long double)dt * (s1 + s2) / 12.0L, (long double)dt * s1 / 24.0L};
    const int e = k - 1 - j; /* g_j(z) R(z)^e, degree 3 + 4e <= 4k - 1 */
    poly_mul_ld(g, 3, pw + (size_t)e * w, 4 * e, term);
    for (int i = 0; i <= 3 + 4 * e; ++i) acc[i] += term[i];
  }
  for (int i = 0; i < 4 * k; ++i) b[i] = (double)acc[i];
  free(pw); free(acc); free(term);
  return 0;
}

int pxo_ad2_poly_apply(int nx, int ny, double L, double nu, const double* u, const double* v, double dt,
                       int transpose, int m, const double* c, const double* x, double* out) {
  if (bad_grid2(nx, ny, L) || !u || !v || m < 0 || !c || !x || !out) return -1;
  size_t N = (size_t)nx * ny, nb = sizeof(double) * N;
  double *p = malloc(nb), *q = malloc(nb);
  if (!p || !q) {
    free(p); free(q);
    return -1;
  }
  memcpy(p, x, nb);                                   /* p = (dt A)^0 x */
  for (size_t i = 0; i < N; ++i) out[i] = c[0] * p[i];
  for (int j = 1; j <= m; ++j) {                      /* p = (dt A)^j x */
    if (transpose) pxo_ad2_apply_T(nx, ny, L, nu, u, v, p, q);
    else pxo_ad2_apply(nx, ny, L, nu, u, v, p, q);
    for (size_t i = 0; i < N; ++i) p[i] = dt * q[i];
    for (size_t i = 0; i < N; ++i) out[i] += c[j] * p[i];
  }
  free(p); free(q);
  return 0;
}

/* One reverse step of the exact discrete adjoint of the RK4 map (as in the serial loop
 * above): lam <- R(dt A)^T lam, grad += g_s(dt A)^T lam (the stage terms at the
 * incoming lam), no objective source. */
static void ad2_adjoint_step(int nx, int ny, double L, double nu, const double* u, const double* v,
                             double dt, double t, double omega, double* lam, double* grad,
                             double* mu, double* nv, double* acc) {
  size_t N = (size_t)nx * ny;
  double s1 = forcing_s(omega, t), s2 = forcing_s(omega, t + 0.5 * dt), s4 = forcing_s(omega, t + dt);
  for (size_t i = 0; i < N; ++i) acc[i] = lam[i];
  for (size_t i = 0; i < N; ++i) mu[i] = dt / 6.0 * lam[i];            /* kbar4 */
  for (size_t i = 0; i < N; ++i) grad[i] += s4 * mu[i];
  pxo_ad2_apply_T(nx, ny, L, nu, u, v, mu, nv);
  for (size_t i = 0; i < N; ++i) { acc[i] += nv[i]; mu[i] = dt / 3.0 * lam[i] + dt * nv[i]; }
  for (size_t i = 0; i < N; ++i) grad[i] += s2 * mu[i];              /* kbar3 */
  pxo_ad2_apply_T(nx, ny, L, nu, u, v, mu, nv);
  for (size_t i = 0; i < N; ++i) { acc[i] += nv[i]; mu[i] = dt / 3.0 * lam[i] + 0.5 * dt * nv[i]; }
  for (size_t i = 0; i < N; ++i) grad[i] += s2 * mu[i];              /* kbar2 */
  pxo_ad2_apply_T(nx, ny, L, nu, u, v, mu, nv);
  for (size_t i = 0; i < N; ++i) { acc[i] += nv[i]; mu[i] = dt / 6.0 * lam[i] + 0.5 * dt * nv[i]; }
  for (size_t i = 0; i < N; ++i) grad[i] += s1 * mu[i];              /* kbar1 */
  pxo_ad2_apply_T(nx, ny, L, nu, u, v, mu, nv);
  for (size_t i = 0; i < N; ++i) lam[i] = acc[i] + nv[i];
}

int pxo_ad2_gradient_hybrid_poly(int nx, int ny, double L, double nu, const double* u, const double* v,
                                 double T, int64_t K, double omega, const double* f, const double* f_true,
                                 int P, int m, double* J, double* grad) {
  if (bad_grid2(nx, ny, L) || K < 1 || P < 1 || K % P != 0 || !u || !v || !f || !f_true || !J || !grad)
    return -1;
  const int64_t k = K / P;
  const int deg = 4 * (int)k;
  if (m <= 0 || m > deg) m = deg;
  size_t N = (size_t)nx * ny, nb = sizeof(double) * N;
  double dt = T / (double)K, src = 2.0 * dt / T;
  double *d = malloc(nb), *traj = malloc(nb * (size_t)(K + 1));
  double *lam = malloc(nb), *mu = malloc(nb), *nv = malloc(nb), *acc = malloc(nb);
  double *W = malloc(nb * (size_t)P), *h = malloc(nb), *hp = malloc(nb), *pw = malloc(nb), *q = malloc(nb);
  double *a = malloc(sizeof(double) * (size_t)(deg + 1)), *b = malloc(sizeof(double) * (size_t)deg);
  if (!d || !traj || !lam || !mu || !nv || !acc || !W || !h || !hp || !pw || !q || !a || !b) return -1;
  /* Eq. seriesDirect: serial RK4 of the response to f - f_true, every state kept */
  for (size_t i = 0; i < N; ++i) d[i] = f[i] - f_true[i];
  memset(traj, 0, nb);
  double Jacc = 0.0;
  for (int64_t s = 0; s < K; ++s) {
    pxo_ad2_rk4_step(nx, ny, L, nu, u, v, dt, s * dt, omega, d, traj + (size_t)s * N,
                     traj + (size_t)(s + 1) * N);
    double sq = 0.0;
    for (size_t i = 0; i < N; ++i) sq += traj[(size_t)(s + 1) * N + i] * traj[(size_t)(s + 1) * N + i];
    Jacc += dt / T * sq;
  }
  *J = Jacc;
  memset(grad, 0, nb);
  /* Eq. hybadjinhom: lane p from zero at its top row (p+1)k, where it takes the
   * objective's source, down to row pk, adding the source of rows pk+1 .. (p+1)k-1 */
  for (int p = 0; p < P; ++p) {
    int64_t top = (int64_t)(p + 1) * k;
    for (size_t i = 0; i < N; ++i) lam[i] = src * traj[(size_t)top * N + i];
    for (int64_t s = top - 1; s >= (int64_t)p * k; --s) {
      ad2_adjoint_step(nx, ny, L, nu, u, v, dt, s * dt, omega, lam, grad, mu, nv, acc);
      if (s > (int64_t)p * k)
        for (size_t i = 0; i < N; ++i) lam[i] += src * traj[(size_t)s * N + i];
    }
    memcpy(W + (size_t)p * N, lam, nb); /* w_p = lambda_{I,p} at row pk */
  }
  /* Eq. adjHomNormal, local form: h carries the summed homogeneous problems from
   * subinterval P-2 down to 0, h <- a(dt A^T)(h + w_{p+1}); their forcing gradient over
   * subinterval p is b_p(dt A^T)(h + w_{p+1}) (a, b cut after degree m) */
  memset(h, 0, nb);
  pxo_rk4_power_coeffs((int)k, a);
  for (int p = P - 2; p >= 0; --p) {
    pxo_rk4_forcing_coeffs((int)k, dt, (double)p * k * dt, omega, b);
    for (size_t i = 0; i < N; ++i) hp[i] = h[i] + W[(size_t)(p + 1) * N + i];
    memcpy(pw, hp, nb);
    for (size_t i = 0; i < N; ++i) { h[i] = a[0] * pw[i]; grad[i] += b[0] * pw[i]; }
    for (int j = 1; j <= m; ++j) {
      pxo_ad2_apply_T(nx, ny, L, nu, u, v, pw, q);
      for (size_t i = 0; i < N; ++i) pw[i] = dt * q[i];
      for (size_t i = 0; i < N; ++i) h[i] += a[j] * pw[i];
      if (j < deg)
        for (size_t i = 0; i < N; ++i) grad[i] += b[j] * pw[i];
    }
  }
  free(d); free(traj); free(lam); free(mu); free(nv); free(acc);
  free(W); free(h); free(hp); free(pw); free(q); free(a); free(b);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Linear problem with a general sparse operator in CSR form (Sec. 2: the    */
/* state equation dq/dt = A q with a constant discretised operator A; the    */
/* paper's Sec. 4 operators are such matrices). Classical RK4, control =     */
/* q(0), objective J = 0.5 ||q(T) - g||^2 (g = 0 when absent), Alg. 1 for     */
/* Paraexp with exact propagators formed densely (small n only).             */
/* ------------------------------------------------------------------------- */
static int csr_bad(int64_t n, const int64_t* rp, const int32_t* col, const double* val) {
  if (n < 1 || !rp || !col || !val || rp[0] != 0) return 1;
  for (int64_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return 1;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (col[k] < 0 || col[k] >= n) return 1;
  }
  return 0;
}

/* A^T in CSR form, entry by entry: entry (i, j, a) of A becomes (j, i, a). */
int pxo_csr_transpose(int64_t n, const int64_t* rp, const int32_t* col, const double* val, int64_t* rpT,
                      int32_t* colT, double* valT) {
  if (csr_bad(n, rp, col, val) || !rpT || !colT || !valT) return -1;
  for (int64_t j = 0; j <= n; ++j) rpT[j] = 0;
  for (int64_t k = 0; k < rp[n]; ++k) rpT[col[k] + 1] += 1;
  for (int64_t j = 0; j < n; ++j) rpT[j + 1] += rpT[j];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t j = 0; j < n; ++j) fill[j] = rpT[j];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      int64_t dst = fill[col[k]]++;
      colT[dst] = (int32_t)i;
      valT[dst] = val[k];
    }
  free(fill);
  return 0;
}

/* y = A x + src (src may be NULL). */
static void csr_apply_src(int64_t n, const int64_t* rp, const int32_t* col, const double* val,
                          const double* x, const double* src, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = src ? src[i] : 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = s;
  }
}

/* One classical RK4 step of dq/dt = A q + src (src constant, may be NULL). */
int pxo_csr_rk4_step(int64_t n, const int64_t* rp, const int32_t* col, const double* val, double dt,
                     const double* src, const double* q, double* out) {
  if (csr_bad(n, rp, col, val) || !q || !out) return -1;
  size_t nb = sizeof(double) * (size_t)n;
  double* k1 = (double*)malloc(nb);
  double* k2 = (double*)malloc(nb);
  double* k3 = (double*)malloc(nb);
  double* k4 = (double*)malloc(nb);
  double* y = (double*)malloc(nb);
  csr_apply_src(n, rp, col, val, q, src, k1);
  for (int64_t i = 0; i < n; ++i) y[i] = q[i] + 0.5 * dt * k1[i];
  csr_apply_src(n, rp, col, val, y, src, k2);
  for (int64_t i = 0; i < n; ++i) y[i] = q[i] + 0.5 * dt * k2[i];
  csr_apply_src(n, rp, col, val, y, src, k3);
  for (int64_t i = 0; i < n; ++i) y[i] = q[i] + dt * k3[i];
  csr_apply_src(n, rp, col, val, y, src, k4);
  for (int64_t i = 0; i < n; ++i) out[i] = q[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  free(k1);
  free(k2);
  free(k3);
  free(k4);
  free(y);
  return 0;
}

/* Reverse sweep of one RK4 step of dq/dt = A q (exact discrete adjoint, the stages
 * in reverse order with A^T given as rpT/colT/valT): lam_out = M^T lam. */
static void csr_rk4_adjoint_step(int64_t n, const int64_t* rpT, const int32_t* colT, const double* valT,
                                 double dt, const double* lam, double* lam_out) {
  size_t nb = sizeof(double) * (size_t)n;
  double* mu = (double*)malloc(nb);
  double* nv = (double*)malloc(nb);
  for (int64_t i = 0; i < n; ++i) lam_out[i] = lam[i];
  /* stage 4: kbar4 = dt/6 lam, Ybar4 = A^T kbar4 */
  for (int64_t i = 0; i < n; ++i) mu[i] = dt / 6.0 * lam[i];
  csr_apply_src(n, rpT, colT, valT, mu, NULL, nv);
  for (int64_t i = 0; i < n; ++i) lam_out[i] += nv[i];
  /* stage 3: kbar3 = dt/3 lam + dt Ybar4 */
  for (int64_t i = 0; i < n; ++i) mu[i] = dt / 3.0 * lam[i] + dt * nv[i];
  csr_apply_src(n, rpT, colT, valT, mu, NULL, nv);
  for (int64_t i = 0; i < n; ++i) lam_out[i] += nv[i];
  /* stage 2: kbar2 = dt/3 lam + dt/2 Ybar3 */
  for (int64_t i = 0; i < n; ++i) mu[i] = dt / 3.0 * lam[i] + 0.5 * dt * nv[i];
  csr_apply_src(n, rpT, colT, valT, mu, NULL, nv);
  for (int64_t i = 0; i < n; ++i) lam_out[i] += nv[i];
  /* stage 1: kbar1 = dt/6 lam + dt/2 Ybar2 */
  for (int64_t i = 0; i < n; ++i) mu[i] = dt / 6.0 * lam[i] + 0.5 * dt * nv[i];
  csr_apply_src(n, rpT, colT, valT, mu, NULL, nv);
  for (int64_t i = 0; i < n; ++i) lam_out[i] += nv[i];
  free(mu);
  free(nv);
}

static double terminal_objective(int64_t n, const double* q, const double* g, double* lam) {
  double J = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double d = q[i] - (g ? g[i] : 0.0);
    J += 0.5 * d * d;
    if (lam) lam[i] = d; /* dJ/dq(T) (Eq. adjFinalTime) */
  }
  return J;
}

/* Serial stepping (the plain definition): K RK4 steps from q0, J, the reverse sweep of
 * every step from lam(T) = q(T) - g, grad = lam(0) (Eq. initupdate). */
int pxo_csr_gradient_serial(int64_t n, const int64_t* rp, const int32_t* col, const double* val, double T,
                            int64_t K, const double* q0, const double* g, double* J, double* grad,
                            double* qT) {
  if (csr_bad(n, rp, col, val) || !(T > 0.0) || K < 1 || !q0 || !J || !grad) return -1;
  size_t nb = sizeof(double) * (size_t)n;
  const double dt = T / (double)K;
  double* q = (double*)malloc(nb);
  double* q2 = (double*)malloc(nb);
  int64_t* rpT = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t* colT = (int32_t*)malloc(sizeof(int32_t) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  double* valT = (double*)malloc(sizeof(double) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  pxo_csr_transpose(n, rp, col, val, rpT, colT, valT);
  memcpy(q, q0, nb);
  for (int64_t s = 0; s < K; ++s) {
    pxo_csr_rk4_step(n, rp, col, val, dt, NULL, q, q2);
    memcpy(q, q2, nb);
  }
  if (qT) memcpy(qT, q, nb);
  *J = terminal_objective(n, q, g, q2); /* q2 = lam(T) */
  for (int64_t s = K - 1; s >= 0; --s) {
    csr_rk4_adjoint_step(n, rpT, colT, valT, dt, q2, q);
    memcpy(q2, q, nb);
  }
  memcpy(grad, q2, nb);
  free(q);
  free(q2);
  free(rpT);
  free(colT);
  free(valT);
  return 0;
}

/* Dense n x n matrix of the CSR operator (row-major). */
static double* csr_dense(int64_t n, const int64_t* rp, const int32_t* col, const double* val) {
  double* D = (double*)calloc((size_t)(n * n), sizeof(double));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) D[i * n + col[k]] += val[k];
  return D;
}

static void dense_matvec(int64_t n, const double* M, int transpose, const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += (transpose ? M[j * n + i] : M[i * n + j]) * x[j];
    y[i] = s;
  }
}

/* Paraexp (Alg. 1) for the CSR problem, with the homogeneous propagator of one
 * subinterval formed densely: phi_mode 0 = exp(tau A) (Eq. hom), 2 = the RK4 stepper's
 * own R(dt A)^(K/P), R(Z) = I + Z + Z^2/2 + Z^3/6 + Z^4/24 (reproduces serial stepping).
 * Inhomogeneous lanes (Eq. linzero, linInhomEqus): zero initial value and the constant
 * source A q0 on every subinterval; homogeneous problems in the global form, each
 * boundary value propagated from T_j to T; superposition Eq. fullsol0; the adjoint
 * mirrored (Eq. adjInhom, adjHomNormal, fulladjsol) with A^T and Phi^T; Eq. initupdate. */
int pxo_csr_gradient_paraexp(int64_t n, const int64_t* rp, const int32_t* col, const double* val, double T,
                             int64_t K, int P, int phi_mode, const double* q0, const double* g, double* J,
                             double* grad, double* qT) {
  if (csr_bad(n, rp, col, val) || !(T > 0.0) || K < 1 || P < 1 || K % P != 0 || !q0 || !J || !grad ||
      (phi_mode != 0 && phi_mode != 2) || n > 2048)
    return -1;
  const int64_t k = K / P;
  const double dt = T / (double)K, tau = T / (double)P;
  size_t nb = sizeof(double) * (size_t)n;
  int64_t* rpT = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t* colT = (int32_t*)malloc(sizeof(int32_t) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  double* valT = (double*)malloc(sizeof(double) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  pxo_csr_transpose(n, rp, col, val, rpT, colT, valT);
  /* the subinterval propagator Phi, densely */
  double* A = csr_dense(n, rp, col, val);
  double* Phi = (double*)malloc(nb * (size_t)n);
  if (phi_mode == 0) {
    for (int64_t e = 0; e < n * n; ++e) A[e] *= tau;
    pxo_expm((int)n, A, Phi);
  } else {
    /* R(dt A) column by column (one RK4 step of each unit vector), then R^k */
    double* R = (double*)malloc(nb * (size_t)n);
    double* e = (double*)calloc((size_t)n, sizeof(double));
    double* col_out = (double*)malloc(nb);
    for (int64_t j = 0; j < n; ++j) {
      e[j] = 1.0;
      pxo_csr_rk4_step(n, rp, col, val, dt, NULL, e, col_out);
      for (int64_t i = 0; i < n; ++i) R[i * n + j] = col_out[i];
      e[j] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) Phi[i * n + j] = (i == j) ? 1.0 : 0.0;
    double* W = (double*)malloc(nb * (size_t)n);
    for (int64_t s = 0; s < k; ++s) { /* Phi <- R Phi */
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
          double acc = 0.0;
          for (int64_t l = 0; l < n; ++l) acc += R[i * n + l] * Phi[l * n + j];
          W[i * n + j] = acc;
        }
      memcpy(Phi, W, nb * (size_t)n);
    }
    free(W);
    free(R);
    free(e);
    free(col_out);
  }
  double* src = (double*)malloc(nb);
  double* w = (double*)malloc(nb * (size_t)P);
  double* x = (double*)malloc(nb);
  double* y = (double*)malloc(nb);
  double* qTT = (double*)malloc(nb);
  double* lamT = (double*)malloc(nb);
  /* direct lanes: q~_p(T_p) = 0, dq~/dt = A q~ + A q0 */
  csr_apply_src(n, rp, col, val, q0, NULL, src);
  for (int p = 0; p < P; ++p) {
    double* wp = w + (size_t)p * n;
    memset(wp, 0, nb);
    for (int64_t s = 0; s < k; ++s) {
      pxo_csr_rk4_step(n, rp, col, val, dt, src, wp, y);
      memcpy(wp, y, nb);
    }
  }
  /* q(T) = q0 + w_{P-1} + sum_{j=1}^{P-1} Phi^{P-j} w_{j-1} */
  for (int64_t i = 0; i < n; ++i) qTT[i] = q0[i] + w[(size_t)(P - 1) * n + i];
  for (int j = 1; j < P; ++j) {
    memcpy(x, w + (size_t)(j - 1) * n, nb);
    for (int r = 0; r < P - j; ++r) {
      dense_matvec(n, Phi, 0, x, y);
      memcpy(x, y, nb);
    }
    for (int64_t i = 0; i < n; ++i) qTT[i] += x[i];
  }
  if (qT) memcpy(qT, qTT, nb);
  *J = terminal_objective(n, qTT, g, lamT);
  /* adjoint lanes: lam~_p(T_{p+1}) = 0, backward k steps with A^T and the source A^T lam(T) */
  csr_apply_src(n, rpT, colT, valT, lamT, NULL, src);
  for (int p = 0; p < P; ++p) {
    double* wp = w + (size_t)p * n;
    memset(wp, 0, nb);
    for (int64_t s = 0; s < k; ++s) {
      pxo_csr_rk4_step(n, rpT, colT, valT, dt, src, wp, y);
      memcpy(wp, y, nb);
    }
  }
  /* grad = lam(0) = lam(T) + w_0 + sum_{j=1}^{P-1} (Phi^T)^j w_j */
  for (int64_t i = 0; i < n; ++i) grad[i] = lamT[i] + w[i];
  for (int j = 1; j < P; ++j) {
    memcpy(x, w + (size_t)j * n, nb);
    for (int r = 0; r < j; ++r) {
      dense_matvec(n, Phi, 1, x, y);
      memcpy(x, y, nb);
    }
    for (int64_t i = 0; i < n; ++i) grad[i] += x[i];
  }
  free(rpT);
  free(colT);
  free(valT);
  free(A);
  free(Phi);
  free(src);
  free(w);
  free(x);
  free(y);
  free(qTT);
  free(lamT);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* 2D viscous Burgers (Sec. 4.3): the vector field (u, v) on an n x n periodic grid   */
/* (arrays [n][n], row = y, x fastest, h = L / n), advective central differences:    */
/*   N_u = -u u_x - v u_y + nu lap u,   N_v = -u v_x - v v_y + nu lap v,              */
/* classical RK4, control = the initial state, J = 0.5 ||q(T) - q_target||^2.        */
/* ------------------------------------------------------------------------- */
#define B2(a, i, j) (a)[(size_t)(((i) + n) % n) * n + (size_t)(((j) + n) % n)]

static double dxc(const double* a, int n, int i, int j, double h) { return (B2(a, i, j + 1) - B2(a, i, j - 1)) / (2.0 * h); }
static double dyc(const double* a, int n, int i, int j, double h) { return (B2(a, i + 1, j) - B2(a, i - 1, j)) / (2.0 * h); }
static double lap(const double* a, int n, int i, int j, double h) {
  return (B2(a, i, j + 1) + B2(a, i, j - 1) + B2(a, i + 1, j) + B2(a, i - 1, j) - 4.0 * B2(a, i, j)) / (h * h);
}

int pxo_bu2_rhs(int n, double L, double nu, const double* U, const double* V, double* oU, double* oV) {
  if (n < 3 || !(L > 0.0) || !U || !V || !oU || !oV) return -1;
  const double h = L / n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double u = B2(U, i, j), v = B2(V, i, j);
      oU[(size_t)i * n + j] = -u * dxc(U, n, i, j, h) - v * dyc(U, n, i, j, h) + nu * lap(U, n, i, j, h);
      oV[(size_t)i * n + j] = -u * dxc(V, n, i, j, h) - v * dyc(V, n, i, j, h) + nu * lap(V, n, i, j, h);
    }
  return 0;
}

/* Linearisation about (U, V) in the direction (W1, W2) (the linearised Burgers operator
 * of Sec. 4.3): J_u = -W1 U_x - U W1_x - W2 U_y - V W1_y + nu lap W1,
 *                J_v = -W1 V_x - U W2_x - W2 V_y - V W2_y + nu lap W2. */
int pxo_bu2_jac(int n, double L, double nu, const double* U, const double* V, const double* W1, const double* W2,
                double* o1, double* o2) {
  if (n < 3 || !(L > 0.0) || !U || !V || !W1 || !W2 || !o1 || !o2) return -1;
  const double h = L / n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double u = B2(U, i, j), v = B2(V, i, j), w1 = B2(W1, i, j), w2 = B2(W2, i, j);
      o1[(size_t)i * n + j] = -w1 * dxc(U, n, i, j, h) - u * dxc(W1, n, i, j, h) - w2 * dyc(U, n, i, j, h) -
                              v * dyc(W1, n, i, j, h) + nu * lap(W1, n, i, j, h);
      o2[(size_t)i * n + j] = -w1 * dxc(V, n, i, j, h) - u * dxc(W2, n, i, j, h) - w2 * dyc(V, n, i, j, h) -
                              v * dyc(W2, n, i, j, h) + nu * lap(W2, n, i, j, h);
    }
  return 0;
}

/* Transpose of the linearisation, term by term: a pointwise factor c (as in -W1 U_x)
 * stays pointwise (-U_x Z1); a factor a in front of a central difference D (as in
 * -U W1_x) becomes D(a Z), since D^T = -D on the periodic grid; the 5-point Laplacian
 * is symmetric:
 *   (J^T Z)_1 = -U_x Z1 + D_x(U Z1) + D_y(V Z1) + nu lap Z1 - V_x Z2,
 *   (J^T Z)_2 = -U_y Z1 + D_x(U Z2) + D_y(V Z2) + nu lap Z2 - V_y Z2. */
int pxo_bu2_jac_T(int n, double L, double nu, const double* U, const double* V, const double* Z1, const double* Z2,
                  double* o1, double* o2) {
  if (n < 3 || !(L > 0.0) || !U || !V || !Z1 || !Z2 || !o1 || !o2) return -1;
  const double h = L / n;
  const size_t nn = (size_t)n * n;
  double* UZ1 = (double*)malloc(sizeof(double) * nn);
  double* VZ1 = (double*)malloc(sizeof(double) * nn);
  double* UZ2 = (double*)malloc(sizeof(double) * nn);
  double* VZ2 = (double*)malloc(sizeof(double) * nn);
  for (size_t e = 0; e < nn; ++e) {
    UZ1[e] = U[e] * Z1[e];
    VZ1[e] = V[e] * Z1[e];
    UZ2[e] = U[e] * Z2[e];
    VZ2[e] = V[e] * Z2[e];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const size_t e = (size_t)i * n + j;
      o1[e] = -dxc(U, n, i, j, h) * Z1[e] + dxc(UZ1, n, i, j, h) + dyc(VZ1, n, i, j, h) + nu * lap(Z1, n, i, j, h) -
              dxc(V, n, i, j, h) * Z2[e];
      o2[e] = -dyc(U, n, i, j, h) * Z1[e] + dxc(UZ2, n, i, j, h) + dyc(VZ2, n, i, j, h) + nu * lap(Z2, n, i, j, h) -
              dyc(V, n, i, j, h) * Z2[e];
    }
  free(UZ1);
  free(VZ1);
  free(UZ2);
  free(VZ2);
  return 0;
}

/* One classical RK4 step of dq/dt = N(q), q = (U, V). */
int pxo_bu2_rk4_step(int n, double L, double nu, double dt, const double* U, const double* V, double* oU,
                     double* oV) {
  if (n < 3 || !(L > 0.0) || !U || !V || !oU || !oV) return -1;
  const size_t nn = (size_t)n * n, nb = sizeof(double) * nn;
  double* kU = (double*)malloc(nb);
  double* kV = (double*)malloc(nb);
  double* aU = (double*)malloc(nb);
  double* aV = (double*)malloc(nb);
  double* yU = (double*)malloc(nb);
  double* yV = (double*)malloc(nb);
  static const double cst[3] = {0.5, 0.5, 1.0};
  static const double wgt[4] = {1.0, 2.0, 2.0, 1.0};
  memcpy(yU, U, nb);
  memcpy(yV, V, nb);
  memset(aU, 0, nb);
  memset(aV, 0, nb);
  for (int q = 0; q < 4; ++q) {
    pxo_bu2_rhs(n, L, nu, yU, yV, kU, kV);
    for (size_t e = 0; e < nn; ++e) {
      aU[e] += wgt[q] * kU[e];
      aV[e] += wgt[q] * kV[e];
    }
    if (q < 3)
      for (size_t e = 0; e < nn; ++e) {
        yU[e] = U[e] + cst[q] * dt * kU[e];
        yV[e] = V[e] + cst[q] * dt * kV[e];
      }
  }
  for (size_t e = 0; e < nn; ++e) {
    oU[e] = U[e] + dt / 6.0 * aU[e];
    oV[e] = V[e] + dt / 6.0 * aV[e];
  }
  free(kU);
  free(kV);
  free(aU);
  free(aV);
  free(yU);
  free(yV);
  return 0;
}

/* Reverse sweep of one RK4 step taken at (U, V): given lam = dJ/dq_{s+1} (l1, l2), adds
 * M_s^T lam to (o1, o2) (which must hold lam on entry): the stage states are recomputed
 * and their transposed Jacobians applied in reverse order. */
static void bu2_rk4_adjoint_step(int n, double L, double nu, double dt, const double* U, const double* V,
                                 const double* l1, const double* l2, double* o1, double* o2) {
  const size_t nn = (size_t)n * n, nb = sizeof(double) * nn;
  double *Y1[4], *Y2[4];
  for (int q = 0; q < 4; ++q) {
    Y1[q] = (double*)malloc(nb);
    Y2[q] = (double*)malloc(nb);
  }
  double* kU = (double*)malloc(nb);
  double* kV = (double*)malloc(nb);
  double* m1 = (double*)malloc(nb);
  double* m2 = (double*)malloc(nb);
  double* n1 = (double*)malloc(nb);
  double* n2 = (double*)malloc(nb);
  static const double cst[3] = {0.5, 0.5, 1.0};
  memcpy(Y1[0], U, nb);
  memcpy(Y2[0], V, nb);
  for (int q = 0; q < 3; ++q) {
    pxo_bu2_rhs(n, L, nu, Y1[q], Y2[q], kU, kV);
    for (size_t e = 0; e < nn; ++e) {
      Y1[q + 1][e] = U[e] + cst[q] * dt * kU[e];
      Y2[q + 1][e] = V[e] + cst[q] * dt * kV[e];
    }
  }
  /* kbar4 = dt/6 lam; Ybar4 = J(Y4)^T kbar4; kbar3 = dt/3 lam + dt Ybar4; ...
   * kbar_q = b_q dt lam + c_q dt Ybar_{q+1}; q(U) receives every Ybar_q */
  static const double bw[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  for (size_t e = 0; e < nn; ++e) {
    n1[e] = 0.0;
    n2[e] = 0.0;
  }
  for (int q = 3; q >= 0; --q) {
    const double c = q < 3 ? cst[q] : 0.0; /* Y_{q+1} = U + c_q dt k_q */
    for (size_t e = 0; e < nn; ++e) {
      m1[e] = bw[q] * dt * l1[e] + c * dt * n1[e];
      m2[e] = bw[q] * dt * l2[e] + c * dt * n2[e];
    }
    pxo_bu2_jac_T(n, L, nu, Y1[q], Y2[q], m1, m2, n1, n2); /* Ybar_q */
    for (size_t e = 0; e < nn; ++e) {
      o1[e] += n1[e];
      o2[e] += n2[e];
    }
  }
  for (int q = 0; q < 4; ++q) {
    free(Y1[q]);
    free(Y2[q]);
  }
  free(kU);
  free(kV);
  free(m1);
  free(m2);
  free(n1);
  free(n2);
}

/* q(T) after K RK4 steps from (U0, V0). */
int pxo_bu2_direct(int n, double L, double nu, double T, int64_t K, const double* U0, const double* V0, double* UT,
                   double* VT) {
  if (n < 3 || !(L > 0.0) || !(T > 0.0) || K < 1 || !U0 || !V0 || !UT || !VT) return -1;
  const size_t nb = sizeof(double) * (size_t)n * n;
  double* a = (double*)malloc(nb);
  double* b = (double*)malloc(nb);
  memcpy(UT, U0, nb);
  memcpy(VT, V0, nb);
  for (int64_t s = 0; s < K; ++s) {
    pxo_bu2_rk4_step(n, L, nu, T / (double)K, UT, VT, a, b);
    memcpy(UT, a, nb);
    memcpy(VT, b, nb);
  }
  free(a);
  free(b);
  return 0;
}

/* Serial stepping (the plain definition): K RK4 steps from (U0, V0) keeping every state,
 * J = 0.5 ||q(T) - q_target||^2, lam(T) = q(T) - q_target, the reverse sweep of every
 * step, grad = lam(0) (initial-condition control, Eq. initupdate). */
int pxo_bu2_gradient_serial(int n, double L, double nu, double T, int64_t K, const double* U0, const double* V0,
                            const double* Ut, const double* Vt, double* J, double* gU, double* gV) {
  if (n < 3 || !(L > 0.0) || !(T > 0.0) || K < 1 || !U0 || !V0 || !Ut || !Vt || !J || !gU || !gV) return -1;
  const size_t nn = (size_t)n * n, nb = sizeof(double) * nn;
  const double dt = T / (double)K;
  double* tr = (double*)malloc(nb * 2 * (size_t)(K + 1));
  if (!tr) return -2;
  memcpy(tr, U0, nb);
  memcpy(tr + nn, V0, nb);
  for (int64_t s = 0; s < K; ++s)
    pxo_bu2_rk4_step(n, L, nu, dt, tr + 2 * nn * s, tr + 2 * nn * s + nn, tr + 2 * nn * (s + 1),
                     tr + 2 * nn * (s + 1) + nn);
  const double* qU = tr + 2 * nn * K;
  const double* qV = qU + nn;
  double acc = 0.0;
  double* l1 = (double*)malloc(nb);
  double* l2 = (double*)malloc(nb);
  double* o1 = (double*)malloc(nb);
  double* o2 = (double*)malloc(nb);
  for (size_t e = 0; e < nn; ++e) {
    l1[e] = qU[e] - Ut[e];
    l2[e] = qV[e] - Vt[e];
    acc += l1[e] * l1[e] + l2[e] * l2[e];
  }
  *J = 0.5 * acc;
  for (int64_t s = K - 1; s >= 0; --s) {
    memcpy(o1, l1, nb);
    memcpy(o2, l2, nb);
    bu2_rk4_adjoint_step(n, L, nu, dt, tr + 2 * nn * s, tr + 2 * nn * s + nn, l1, l2, o1, o2);
    memcpy(l1, o1, nb);
    memcpy(l2, o2, nb);
  }
  memcpy(gU, l1, nb);
  memcpy(gV, l2, nb);
  free(tr);
  free(l1);
  free(l2);
  free(o1);
  free(o2);
  return 0;
}
#undef B2
