// krylov.cuh — one-thread-block Arnoldi process and Krylov matrix functions
// (Sec. 4.1: exp(B) v ~ V_m exp(H_m) V_m^T v, Saad 1992).
//
// The Krylov basis V (m+1 vectors of length n, leading dimension ldv) lives in
// shared memory when it fits, otherwise in global memory (L2-resident); the code
// is the same through generic pointers. Orthogonalisation is classical
// Gram–Schmidt applied twice (CGS2): the j+1 dot products of one pass are
// independent, so each warp takes a subset of them and reduces with shuffles.
#pragma once
#include "common.cuh"

namespace pxa {

// Shared scratch that one Krylov solve needs (all in shared memory).
struct KrylovScratch {
  double* H;     // (kMaxM+1) x kLD Hessenberg
  double* D0;    // kLD x kLD dense scratch
  double* D1;
  double* D2;
  double* D3;
  double* hcol;  // kDMax doubles
  double* red;   // 40 doubles
  int* ipiv;
  int* flag;
};

// All threads: dots[i] = <V_i, w> for i = 0..cnt-1 (warp-per-dot). Ends with a barrier.
__device__ __forceinline__ void multi_dot(const double* V, int ldv, int cnt, const double* w,
                                          int n, double* dots) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < cnt; i += nw) {
    const double* vi = V + (size_t)i * ldv;
    double s = 0.0;
    for (int p = lane; p < n; p += 32) s = fma(vi[p], w[p], s);
    s = warp_sum(s);
    if (lane == 0) dots[i] = s;
  }
  __syncthreads();
}

// w -= sum_i c[i] V_i (threads over points). Ends with a barrier.
__device__ __forceinline__ void multi_axpy(const double* V, int ldv, int cnt, const double* c,
                                           double* w, int n) {
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    double acc = w[p];
    for (int i = 0; i < cnt; ++i) acc = fma(-c[i], V[(size_t)i * ldv + p], acc);
    w[p] = acc;
  }
  __syncthreads();
}

// Arnoldi with CGS2 on the block-cooperative operator `op` (op.apply(x, y) writes
// y = Op x and ends with a barrier). V_0 = v / ||v||. Returns beta = ||v||; *mm_out
// receives the dimension reached (< m after a happy breakdown, when the Krylov
// space is invariant), H(0..mm, 0..mm-1) is filled. If beta == 0, mm = 0.
template <class Op>
__device__ double arnoldi(Op& op, const double* v, int n, int m, double* V, int ldv,
                          KrylovScratch& ks, int* mm_out) {
  double ss = 0.0;
  for (int p = threadIdx.x; p < n; p += blockDim.x) ss = fma(v[p], v[p], ss);
  double beta = sqrt(block_sum(ss, ks.red));
  for (int e = threadIdx.x; e < (kMaxM + 1) * kLD; e += blockDim.x) ks.H[e] = 0.0;
  if (beta == 0.0) {
    __syncthreads();
    *mm_out = 0;
    return 0.0;
  }
  const double inv = 1.0 / beta;
  for (int p = threadIdx.x; p < n; p += blockDim.x) V[p] = v[p] * inv;
  __syncthreads();
  int mm = m;
  for (int j = 0; j < m; ++j) {
    double* w = V + (size_t)(j + 1) * ldv;
    op.apply(V + (size_t)j * ldv, w);
    // first Gram–Schmidt pass
    multi_dot(V, ldv, j + 1, w, n, ks.hcol);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) ks.H[i * kLD + j] = ks.hcol[i];
    multi_axpy(V, ldv, j + 1, ks.hcol, w, n);
    // second pass (re-orthogonalisation)
    multi_dot(V, ldv, j + 1, w, n, ks.hcol);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) ks.H[i * kLD + j] += ks.hcol[i];
    multi_axpy(V, ldv, j + 1, ks.hcol, w, n);
    double s2 = 0.0;
    for (int p = threadIdx.x; p < n; p += blockDim.x) s2 = fma(w[p], w[p], s2);
    double hn = sqrt(block_sum(s2, ks.red));
    if (threadIdx.x == 0) ks.H[(j + 1) * kLD + j] = hn;
    if (hn <= 1e-14 * beta) {  // happy breakdown: exact in the space built so far
      mm = j + 1;
      __syncthreads();
      break;
    }
    const double ih = 1.0 / hn;
    for (int p = threadIdx.x; p < n; p += blockDim.x) w[p] *= ih;
    __syncthreads();
  }
  *mm_out = mm;
  return beta;
}

// y = beta * V_mm * c (c in shared memory, mm entries). Ends with a barrier.
__device__ __forceinline__ void krylov_combine(const double* V, int ldv, int mm, const double* c,
                                               double beta, double* y, int n) {
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < mm; ++i) acc = fma(c[i], V[(size_t)i * ldv + p], acc);
    y[p] = beta * acc;
  }
  __syncthreads();
}

// Homogeneous propagator on the Krylov space.
//   phi_mode 0 (EXP):       F = exp(H)            (H already carries the time span)
//   phi_mode 1 (CN power):  F = [(I - H/2)^{-1} (I + H/2)]^steps
//   phi_mode 2 (RK4 power): F = [I + H + H^2/2 + H^3/6 + H^4/24]^steps (classical RK4's
//                           amplification polynomial, by Horner's rule)
// with H = dt * H_m for the stepper modes. Writes the first column of F to c[0..mm)
// and returns |F[mm-1][0]| for Saad's a-posteriori estimate beta*h_{mm+1,mm}*|F[mm-1][0]|.
// `want_phi1`: also writes phi_1(H) e_1 to c1 (EXP only), through the augmented
// matrix [[H, e_1], [0, 0]] whose exponential holds phi_1(H) e_1 in its last column.
__device__ inline double hessenberg_phi(KrylovScratch& ks, int mm, int phi_mode, double hscale,
                                        int64_t steps, bool want_phi1, double* c, double* c1) {
  const int d = (phi_mode == 0 && want_phi1) ? mm + 1 : mm;
  // D0 = hscale * H_mm (padded)
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    int i = e / d, j = e % d;
    double v = 0.0;
    if (i < mm && j < mm) v = hscale * ks.H[i * kLD + j];
    if (want_phi1 && phi_mode == 0 && j == mm && i == 0) v = 1.0;
    ks.D0[i * kLD + j] = v;
  }
  __syncthreads();
  double* F = ks.D1;
  if (phi_mode == 0) {
    dense_expm(ks.D1, ks.D0, ks.D2, ks.D3, d, ks.red);  // D1 = exp(D0)
  } else if (phi_mode == 2) {
    // R(Z) = I + Z (I + Z/2 (I + Z/3 (I + Z/4))), Z = D0
    for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
      int i = e / d, j = e % d;
      ks.D2[i * kLD + j] = (i == j ? 1.0 : 0.0) + 0.25 * ks.D0[i * kLD + j];
    }
    __syncthreads();
    dense_gemm(ks.D3, ks.D0, ks.D2, d, 1.0 / 3.0, 1.0);
    dense_gemm(ks.D2, ks.D0, ks.D3, d, 0.5, 1.0);
    dense_gemm(ks.D1, ks.D0, ks.D2, d, 1.0, 1.0);  // D1 = R
    F = dense_pow(ks.D1, ks.D0, ks.D2, ks.D3, d, steps);  // F = R^steps
  } else {
    // R = (I - Z/2)^{-1} (I + Z/2): A = I - Z/2 in D2, B = I + Z/2 in D1
    for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
      int i = e / d, j = e % d;
      double z = 0.5 * ks.D0[i * kLD + j];
      ks.D2[i * kLD + j] = (i == j ? 1.0 : 0.0) - z;
      ks.D1[i * kLD + j] = (i == j ? 1.0 : 0.0) + z;
    }
    __syncthreads();
    dense_solve(ks.D2, ks.D1, d, ks.hcol, ks.ipiv);  // D1 = R
    F = dense_pow(ks.D1, ks.D0, ks.D2, ks.D3, d, steps);  // F = R^steps
  }
  for (int i = threadIdx.x; i < mm; i += blockDim.x) {
    c[i] = F[i * kLD + 0];
    if (want_phi1 && phi_mode == 0) c1[i] = F[i * kLD + mm];
  }
  __syncthreads();
  return fabs(F[(mm - 1) * kLD + 0]);
}

// One-block operator used inside the Arnoldi process: y = A x (stencil am, a0, ap).
struct Ad1Op {
  int n;
  double am, a0, ap;
  __device__ void apply(const double* x, double* y) {
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      int im = p == 0 ? n - 1 : p - 1, ip = p == n - 1 ? 0 : p + 1;
      y[p] = am * x[im] + a0 * x[p] + ap * x[ip];
    }
    __syncthreads();
  }
};

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  if (v > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Shared layout of a one-block Krylov solve (see ks_layout_bytes on the host side).
__device__ __forceinline__ KrylovScratch ks_carve(double*& cur) {
  KrylovScratch ks;
  ks.H = cur;
  cur += (kMaxM + 1) * kLD;
  ks.D0 = cur;
  cur += kLD * kLD;
  ks.D1 = cur;
  cur += kLD * kLD;
  ks.D2 = cur;
  cur += kLD * kLD;
  ks.D3 = cur;
  cur += kLD * kLD;
  ks.hcol = cur;
  cur += kDMax;
  ks.red = cur;
  cur += 40;
  ks.ipiv = reinterpret_cast<int*>(cur);
  ks.flag = ks.ipiv + 1;
  cur += 2;
  return ks;
}

// Krylov propagation of one vector h over `nsub` substeps:
//   EXP:     h <- exp(hscale * A) h per substep  (hscale = substep length)
//   STEPPER: h <- R_CN(hscale * A)^steps h        (hscale = dt)
template <class Op>
__device__ void krylov_propagate(Op& op, double* hvec, int n, int m, double* V, int ldv,
                                 KrylovScratch& ks, double* c, double* c1, int phi_mode,
                                 double hscale, int64_t steps, int nsub, double tol,
                                 int* status, double* errmax) {
  for (int sub = 0; sub < nsub; ++sub) {
    int mm = 0;
    double beta = arnoldi(op, hvec, n, m, V, ldv, ks, &mm);
    if (mm == 0) return;  // zero vector stays zero
    double fm = hessenberg_phi(ks, mm, phi_mode, hscale, steps, false, c, c1);
    // Saad's a-posteriori estimate relative to ||h||: span * h_{m+1,m} * |[phi(H)]_{m,1}|,
    // span = the time the substep covers; zero after a happy breakdown
    const double span = phi_mode == 0 ? hscale : hscale * (double)steps;
    double err = (mm == m) ? span * ks.H[m * kLD + (m - 1)] * fm : 0.0;
    if (threadIdx.x == 0) {
      atomic_max_pos(errmax, err);
      if (!(err <= tol)) set_status(status, PXA_ERR_NOT_CONVERGED);
    }
    krylov_combine(V, ldv, mm, c, beta, hvec, n);
  }
}

}  // namespace pxa
