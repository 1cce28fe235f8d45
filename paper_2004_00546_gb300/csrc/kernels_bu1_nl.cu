// kernels_bu1_nl.cu — the iterative nonlinear Paraexp direct of Alg. 2 (Sec. 3.2) for the
// 1D viscous Burgers problem: each iteration linearises the problem about the previous
// iterate q_i, solves the linear inhomogeneous problems of every subinterval in parallel
// (Eq. nonlinTrans, with the averaged Jacobian of Eq. Jacobians), carries the homogeneous
// problems (Eq. nlHomIter) and sums them (Eq. fullsolIter) into the next iterate.
//
//   nl_qbar_kernel   qbar_p = the average of q_i over [T_p, T_{p+1}] (trapezoid rule over
//                    the step states): dN/dq is linear in q, so the averaged Jacobian of
//                    Eq. Jacobians is the Jacobian at qbar_p
//   nl_lanes_kernel  one thread block per subinterval: from zero at T_p, k RK4 steps of
//                    dy/dt = (A + J_p) y + S(t), J_p = dN/dq at qbar_p and the source
//                    S = N(Y) - J_p Y + s(t) f evaluated at the RK4 stage states Y of the
//                    nonlinear step of q_i (the stage sources of Eq. nonlinTrans)
//   nl_carry_kernel  the summed homogeneous problems from q0, subinterval after
//                    subinterval, by the stepper's own propagator of (A + J_p), plus the
//                    lanes' values: q_{i+1} at every step
//   nl_change_kernel the iteration's change max_s ||q_{i+1}(t_s) - q_i(t_s)|| relative to
//                    max_s ||q_{i+1}(t_s)||
// One thread per grid point (n <= 1024), the vectors of a step in shared memory.
#include "common.cuh"
#include "kernels_1d.cuh"

namespace pxa {

namespace {

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// N(u)_i = -u_i (u_{i+1} - u_{i-1}) / (2h) + nu (u_{i+1} - 2 u_i + u_{i-1}) / h^2
__device__ __forceinline__ double rhs_at(const double* u, int i, int n, double i2h, double ih2, double nu) {
  const double um = u[wrap(i - 1, n)], u0 = u[i], up = u[wrap(i + 1, n)];
  return -u0 * ((up - um) * i2h) + nu * ((up - 2.0 * u0 + um) * ih2);
}

// (A + J(qbar)) w at i: -w_i qbar_x - qbar_i w_x + nu w_xx (qbx = qbar_x at i)
__device__ __forceinline__ double jac_at(const double* w, int i, int n, double qb, double qbx, double i2h,
                                         double ih2, double nu) {
  const double wm = w[wrap(i - 1, n)], w0 = w[i], wp = w[wrap(i + 1, n)];
  return -w0 * qbx - qb * ((wp - wm) * i2h) + nu * ((wp - 2.0 * w0 + wm) * ih2);
}

// N(Y) - J(qbar) Y + c f at i, with the diffusion terms cancelling:
// -Y Y_x + (Y qbar_x + qbar Y_x) + c f
__device__ __forceinline__ double source_at(const double* Y, int i, int n, double qb, double qbx, double i2h,
                                            double cf) {
  const double Ym = Y[wrap(i - 1, n)], Y0 = Y[i], Yp = Y[wrap(i + 1, n)];
  const double Yx = (Yp - Ym) * i2h;
  return -Y0 * Yx + (Y0 * qbx + qb * Yx) + cf;
}

// One linear RK4 step of dy/dt = (A + J) y + S_q (S_q the stage sources, `with_src`) on
// the block's points; y, ya, yb in shared memory (ya, yb scratch). Ends with a barrier.
__device__ __forceinline__ void lin_step(double* y, double* ya, double* yb, int n, double qb, double qbx,
                                         double i2h, double ih2, double nu, double dt, bool with_src,
                                         const double S[4]) {
  const int i = threadIdx.x;
  const bool on = i < n;
  double acc = 0.0, kk;
  // stage 1 from y
  if (on) {
    kk = jac_at(y, i, n, qb, qbx, i2h, ih2, nu) + (with_src ? S[0] : 0.0);
    acc = acc + kk;
    ya[i] = y[i] + 0.5 * dt * kk;
  }
  __syncthreads();
  if (on) {  // stage 2 from ya
    kk = jac_at(ya, i, n, qb, qbx, i2h, ih2, nu) + (with_src ? S[1] : 0.0);
    acc = acc + 2.0 * kk;
    yb[i] = y[i] + 0.5 * dt * kk;
  }
  __syncthreads();
  if (on) {  // stage 3 from yb
    kk = jac_at(yb, i, n, qb, qbx, i2h, ih2, nu) + (with_src ? S[2] : 0.0);
    acc = acc + 2.0 * kk;
    ya[i] = y[i] + dt * kk;
  }
  __syncthreads();
  if (on) {  // stage 4 from ya
    kk = jac_at(ya, i, n, qb, qbx, i2h, ih2, nu) + (with_src ? S[3] : 0.0);
    acc = acc + kk;
  }
  __syncthreads();  // every stage read of y is done before y changes
  if (on) y[i] = y[i] + dt / 6.0 * acc;
  __syncthreads();
}

}  // namespace

__global__ void nl_qbar_kernel(const double* __restrict__ Q, int n, int64_t k, int P, double* __restrict__ qbar) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)P * n) return;
  const int p = (int)(t / n), i = (int)(t % n);
  const int64_t a = (int64_t)p * k;
  double sum = 0.5 * (Q[(size_t)a * n + i] + Q[(size_t)(a + k) * n + i]);
  for (int64_t s = a + 1; s < a + k; ++s) sum += Q[(size_t)s * n + i];
  qbar[(size_t)p * n + i] = sum / (double)k;
}

// Block p: the lane of subinterval p. V row s+1 (s in [a, a + k)) receives the lane state.
__global__ void nl_lanes_kernel(const double* __restrict__ Q, const double* __restrict__ qbar,
                                const double* __restrict__ f, const double* __restrict__ sc, int n, int64_t k,
                                double dt, double i2h, double ih2, double nu, double* __restrict__ V) {
  extern __shared__ double sm[];
  double* qb_s = sm;        // qbar_p
  double* Y = sm + n;       // stage states of the nonlinear step of q_i
  double* Y2 = sm + 2 * n;
  double* y = sm + 3 * n;   // the lane
  double* ya = sm + 4 * n;
  double* yb = sm + 5 * n;
  const int p = blockIdx.x, i = threadIdx.x;
  const bool on = i < n;
  const int64_t a = (int64_t)p * k;
  if (on) {
    qb_s[i] = qbar[(size_t)p * n + i];
    y[i] = 0.0;
  }
  __syncthreads();
  const double qb = on ? qb_s[i] : 0.0;
  const double qbx = on ? (qb_s[wrap(i + 1, n)] - qb_s[wrap(i - 1, n)]) * i2h : 0.0;
  const double fi = on ? f[i] : 0.0;
  for (int64_t s = a; s < a + k; ++s) {
    const double c1 = sc ? sc[3 * s] : 1.0, c2 = sc ? sc[3 * s + 1] : 1.0, c4 = sc ? sc[3 * s + 2] : 1.0;
    const double* qs = Q + (size_t)s * n;
    double S[4];
    double qsi = 0.0;
    // stage 1 at q_i(t_s): its source and the stage state Y2 = q + dt/2 (N(q) + c1 f)
    if (on) {
      qsi = qs[i];
      S[0] = source_at(qs, i, n, qb, qbx, i2h, c1 * fi);
      Y[i] = qsi + 0.5 * dt * (rhs_at(qs, i, n, i2h, ih2, nu) + c1 * fi);
    }
    __syncthreads();
    if (on) {  // stage 2 at Y
      S[1] = source_at(Y, i, n, qb, qbx, i2h, c2 * fi);
      Y2[i] = qsi + 0.5 * dt * (rhs_at(Y, i, n, i2h, ih2, nu) + c2 * fi);
    }
    __syncthreads();
    if (on) {  // stage 3 at Y2; stage 4's state into Y (stage 2's readers are done)
      S[2] = source_at(Y2, i, n, qb, qbx, i2h, c2 * fi);
      Y[i] = qsi + dt * (rhs_at(Y2, i, n, i2h, ih2, nu) + c2 * fi);
    }
    __syncthreads();
    if (on) S[3] = source_at(Y, i, n, qb, qbx, i2h, c4 * fi);
    __syncthreads();  // Y is rewritten at the next step's stage 1
    lin_step(y, ya, yb, n, qb, qbx, i2h, ih2, nu, dt, true, S);
    if (on) V[(size_t)(s + 1) * n + i] = y[i];
  }
}

// One block: y = q0 (zero); for p: Qn[a] = y; k linear steps of (A + J_p) without
// source, Qn[s+1] = V[s+1] + y; then y = Qn[a + k] (the full value at T_{p+1}).
__global__ void nl_carry_kernel(const double* __restrict__ V, const double* __restrict__ qbar, int n,
                                int64_t k, int P, double dt, double i2h, double ih2, double nu,
                                double* __restrict__ Qn) {
  extern __shared__ double sm[];
  double* qb_s = sm;
  double* y = sm + n;
  double* ya = sm + 2 * n;
  double* yb = sm + 3 * n;
  const int i = threadIdx.x;
  const bool on = i < n;
  if (on) y[i] = 0.0;
  const double none[4] = {0.0, 0.0, 0.0, 0.0};
  for (int p = 0; p < P; ++p) {
    const int64_t a = (int64_t)p * k;
    __syncthreads();
    if (on) {
      qb_s[i] = qbar[(size_t)p * n + i];
      Qn[(size_t)a * n + i] = y[i];
    }
    __syncthreads();
    const double qb = on ? qb_s[i] : 0.0;
    const double qbx = on ? (qb_s[wrap(i + 1, n)] - qb_s[wrap(i - 1, n)]) * i2h : 0.0;
    for (int64_t s = a; s < a + k; ++s) {
      lin_step(y, ya, yb, n, qb, qbx, i2h, ih2, nu, dt, false, none);
      if (on) Qn[(size_t)(s + 1) * n + i] = V[(size_t)(s + 1) * n + i] + y[i];
    }
    __syncthreads();
    if (on) y[i] = Qn[(size_t)(a + k) * n + i];
  }
}

// Block per row s: d2 = ||Qn_s - Q_s||^2, q2 = ||Qn_s||^2; out[0] = max d2, out[1] = max
// q2 (non-negative doubles order like their bit patterns), out[2] set when non-finite.
__global__ void nl_change_kernel(const double* __restrict__ Q, const double* __restrict__ Qn, int n,
                                 double* out) {
  __shared__ double red[40];
  const size_t s = blockIdx.x;
  double d2 = 0.0, q2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double qn = Qn[s * n + i], d = qn - Q[s * n + i];
    d2 = fma(d, d, d2);
    q2 = fma(qn, qn, q2);
  }
  d2 = block_sum(d2, red);
  q2 = block_sum(q2, red);
  if (threadIdx.x == 0) {
    if (!isfinite(d2) || !isfinite(q2)) {
      out[2] = 1.0;
    } else {
      atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(d2));
      atomicMax(reinterpret_cast<unsigned long long*>(out + 1), (unsigned long long)__double_as_longlong(q2));
    }
  }
}

cudaError_t launch_nl_iteration(cudaStream_t st, int n, int64_t K, int P, double L, double nu, double dt,
                                const double* f, const double* sc, const double* Q, double* Qn, double* V,
                                double* qbar, double* change) {
  const int64_t k = K / P;
  const double h = L / n, i2h = 1.0 / (2.0 * h), ih2 = 1.0 / (h * h);
  const int threads = ((n + 31) / 32) * 32;
  const int64_t tot = (int64_t)P * n;
  nl_qbar_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Q, n, k, P, qbar);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sh_l = sizeof(double) * 6 * (size_t)n;
  e = cudaFuncSetAttribute(nl_lanes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh_l);
  if (e != cudaSuccess) return e;
  nl_lanes_kernel<<<P, threads, sh_l, st>>>(Q, qbar, f, sc, n, k, dt, i2h, ih2, nu, V);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sh_c = sizeof(double) * 4 * (size_t)n;
  nl_carry_kernel<<<1, threads, sh_c, st>>>(V, qbar, n, k, P, dt, i2h, ih2, nu, Qn);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(change, 0, 3 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  nl_change_kernel<<<(unsigned)(K + 1), 256, 0, st>>>(Q, Qn, n, change);
  return cudaGetLastError();
}

}  // namespace pxa
