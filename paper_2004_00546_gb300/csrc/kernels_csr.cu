// kernels_csr.cu — the general sparse operator kind (PXA_CSR): dq/dt = A q for a
// constant matrix A in CSR form (Sec. 2: the discretised state equation), classical RK4,
// initial-condition control and the terminal objective J = 0.5 ||q(T) - g||^2.
//
//   csr_rk4_lanes_kernel   Eq. linInhomEqus / Eq. adjInhom: one thread block per lane
//                          steps dq/dt = A q + b from its initial value (zero for the
//                          Paraexp lanes, whose constant source b = A q0 is the shift of
//                          Eq. linzero); the adjoint lanes run the same kernel with A^T
//                          (for a constant A one transposed RK4 step is the RK4 step of
//                          A^T: the amplification polynomial commutes with transposition).
//   csr_chain_kernel       Eq. hom / Eq. adjHomNormal: the summed homogeneous problems
//                          carried subinterval by subinterval with Krylov exp(tau A) or the
//                          RK4 stepper's own R(dt A)^(K/P) on the Hessenberg matrix.
//   csr_superpose_kernel   Eq. fullsol0 at T, J and lambda(T) = q(T) - g (Eq. adjFinalTime).
//
// A lane's four vectors (state, two stage inputs, stage sum) sit in shared memory when
// they fit, else in a global workspace (L2-resident); one thread per row forms the row's
// dot product, and a block barrier separates the stages.
#include "common.cuh"
#include "kernels_csr.cuh"
#include "krylov.cuh"

namespace pxa {

namespace {

// Block-cooperative y = A x (+ b) over all rows; no barrier.
struct CsrRows {
  int n;
  const int64_t* __restrict__ rp;
  const int32_t* __restrict__ col;
  const double* __restrict__ val;
  __device__ __forceinline__ double row(int i, const double* x) const {
    double s = 0.0;
    const int64_t e1 = rp[i + 1];
    for (int64_t k = rp[i]; k < e1; ++k) s = fma(val[k], x[col[k]], s);
    return s;
  }
};

// Operator of the Arnoldi process: y = A x, ending with a barrier.
struct CsrOp {
  CsrRows A;
  __device__ void apply(const double* x, double* y) {
    for (int i = threadIdx.x; i < A.n; i += blockDim.x) y[i] = A.row(i, x);
    __syncthreads();
  }
};

}  // namespace

// Lane l: u = x0[l] (x0 == NULL: zero), k RK4 steps of du/dt = A u + b (b may be NULL),
// out[l] = u. Vectors: shared memory (in_smem) or work + 4 n l.
__global__ void csr_rk4_lanes_kernel(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                     const double* __restrict__ val, const double* __restrict__ b, double dt,
                                     int64_t k, const double* __restrict__ x0, double* __restrict__ out,
                                     double* __restrict__ work, int in_smem) {
  extern __shared__ double sm[];
  const int lane = blockIdx.x;
  double* base = in_smem ? sm : work + (size_t)4 * n * lane;
  double* u = base;
  double* ya = base + n;
  double* yb = base + 2 * (size_t)n;
  double* acc = base + 3 * (size_t)n;
  const CsrRows A{n, rp, col, val};
  const double h2 = 0.5 * dt, dt6 = dt / 6.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) u[i] = x0 ? x0[(size_t)lane * n + i] : 0.0;
  __syncthreads();
  for (int64_t s = 0; s < k; ++s) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // stage 1 (from u)
      const double kk = A.row(i, u) + (b ? b[i] : 0.0);
      acc[i] = kk;
      yb[i] = fma(h2, kk, u[i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // stage 2 (from yb)
      const double kk = A.row(i, yb) + (b ? b[i] : 0.0);
      acc[i] = fma(2.0, kk, acc[i]);
      ya[i] = fma(h2, kk, u[i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // stage 3 (from ya)
      const double kk = A.row(i, ya) + (b ? b[i] : 0.0);
      acc[i] = fma(2.0, kk, acc[i]);
      yb[i] = fma(dt, kk, u[i]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // stage 4 (from yb); u[i] is this thread's
      const double kk = A.row(i, yb) + (b ? b[i] : 0.0);
      u[i] = fma(dt6, acc[i] + kk, u[i]);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[(size_t)lane * n + i] = u[i];
}

// h = 0; for i < count: h += E[first + i stride]; h = Phi h, Phi by Krylov over nsub
// substeps (phi_mode 0: exp(hscale A) per substep; 2: R(hscale A)^steps_per_sub).
__global__ void csr_chain_kernel(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const double* __restrict__ E, int first,
                                 int stride, int count, double* __restrict__ hout, double* Vglob, int m,
                                 int phi_mode, double hscale, int64_t steps_per_sub, int nsub, double tol,
                                 int v_in_smem, int* status, double* errmax) {
  extern __shared__ double sm[];
  double* cur = sm;
  KrylovScratch ks = ks_carve(cur);
  double* c = cur;
  cur += kDMax;
  double* c1 = cur;
  cur += kDMax;
  double* hvec = cur;
  cur += n;
  double* V = v_in_smem ? cur : Vglob;
  CsrOp op{CsrRows{n, rp, col, val}};
  for (int p = threadIdx.x; p < n; p += blockDim.x) hvec[p] = 0.0;
  __syncthreads();
  for (int i = 0; i < count; ++i) {
    const double* e = E + (size_t)(first + i * stride) * n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) hvec[p] += e[p];
    __syncthreads();
    krylov_propagate(op, hvec, n, m, V, n, ks, c, c1, phi_mode, hscale, steps_per_sub, nsub, tol, status,
                     errmax);
  }
  for (int p = threadIdx.x; p < n; p += blockDim.x) hout[p] = hvec[p];
}

// h = 0; for i < count: h += E[first + i stride]; then `sub` times h <- sum_{j<=m} a_j
// (tau A)^j h (the RK4 stepper's propagator over a segment as its power series, cut after
// degree m; the powers formed one after another). Vectors h, the power and its successor in
// shared memory when they fit (3 n doubles), else in `work` (3 n doubles).
__global__ void csr_series_chain_kernel(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                        const double* __restrict__ val, const double* __restrict__ E, int first,
                                        int stride, int count, double* __restrict__ hout,
                                        const double* __restrict__ a, int m, int sub, double tau,
                                        double* __restrict__ work, int in_smem) {
  extern __shared__ double sm[];
  double* h = in_smem ? sm : work;
  double* pw = h + n;
  double* nx = pw + n;
  const CsrRows A{n, rp, col, val};
  for (int p = threadIdx.x; p < n; p += blockDim.x) h[p] = 0.0;
  __syncthreads();
  for (int i = 0; i < count; ++i) {
    const double* e = E + (size_t)(first + i * stride) * n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      h[p] += e[p];
      pw[p] = h[p];
      h[p] *= a[0];
    }
    __syncthreads();
    for (int s = 0; s < sub; ++s) {
      if (s > 0) {
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
          pw[p] = h[p];
          h[p] *= a[0];
        }
        __syncthreads();
      }
      for (int j = 1; j <= m; ++j) {
        for (int p = threadIdx.x; p < n; p += blockDim.x) nx[p] = tau * A.row(p, pw);
        __syncthreads();
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
          pw[p] = nx[p];
          h[p] = fma(a[j], nx[p], h[p]);
        }
        __syncthreads();
      }
    }
  }
  for (int p = threadIdx.x; p < n; p += blockDim.x) hout[p] = h[p];
}

// q(T) = q0 + elast + hsum (each may be NULL), lamT = q(T) - g (g may be NULL),
// J = 0.5 ||lamT||^2.
__global__ void csr_superpose_kernel(int n, const double* __restrict__ q0, const double* __restrict__ elast,
                                     const double* __restrict__ hsum, const double* __restrict__ g,
                                     double* __restrict__ lamT, double* __restrict__ Jdev, int* status) {
  __shared__ double red[40];
  double acc = 0.0;
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const double v = (q0 ? q0[p] : 0.0) + (elast ? elast[p] : 0.0) + (hsum ? hsum[p] : 0.0);
    const double d = v - (g ? g[p] : 0.0);
    lamT[p] = d;
    acc = fma(d, d, acc);
  }
  const double J = 0.5 * block_sum(acc, red);
  if (threadIdx.x == 0) {
    *Jdev = J;
    if (!isfinite(J)) set_status(status, PXA_ERR_NONFINITE);
  }
}

size_t csr_lane_smem_bytes(int n) { return sizeof(double) * 4 * (size_t)n; }

bool csr_lanes_fit_smem(int n) { return csr_lane_smem_bytes(n) <= 200 * 1024; }

cudaError_t launch_csr_rk4_lanes(cudaStream_t st, int lanes, int n, const int64_t* rp, const int32_t* col,
                                 const double* val, const double* b, double dt, int64_t k, const double* x0,
                                 double* out, double* work) {
  const int in_smem = csr_lanes_fit_smem(n) ? 1 : 0;
  const size_t sh = in_smem ? csr_lane_smem_bytes(n) : 0;
  cudaError_t e = cudaFuncSetAttribute(csr_rk4_lanes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  const int threads = n >= 1024 ? 1024 : ((n + 31) / 32) * 32;
  csr_rk4_lanes_kernel<<<lanes, threads < 64 ? 64 : threads, sh, st>>>(n, rp, col, val, b, dt, k, x0, out, work,
                                                                       in_smem);
  return cudaGetLastError();
}

cudaError_t launch_csr_chain(cudaStream_t st, int n, const int64_t* rp, const int32_t* col, const double* val,
                             const double* E, int first, int stride, int count, double* hout, double* Vglob,
                             int m, int phi_mode, double hscale, int64_t steps_per_sub, int nsub, double tol,
                             int v_in_smem, int* status, double* errmax) {
  const size_t sh = krylov_smem_bytes(n, m, n, v_in_smem != 0);
  cudaError_t e = cudaFuncSetAttribute(csr_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  const int threads = n >= 512 ? 512 : 256;
  csr_chain_kernel<<<1, threads, sh, st>>>(n, rp, col, val, E, first, stride, count, hout, Vglob, m, phi_mode,
                                           hscale, steps_per_sub, nsub, tol, v_in_smem, status, errmax);
  return cudaGetLastError();
}

cudaError_t launch_csr_series_chain(cudaStream_t st, int n, const int64_t* rp, const int32_t* col,
                                    const double* val, const double* E, int first, int stride, int count,
                                    double* hout, const double* a, int m, int sub, double tau, double* work) {
  const size_t sh = sizeof(double) * 3 * (size_t)n;
  const bool in_smem = sh <= 200 * 1024;
  if (in_smem) {
    cudaError_t e = cudaFuncSetAttribute(csr_series_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
  }
  const int threads = n >= 512 ? 512 : 256;
  csr_series_chain_kernel<<<1, threads, in_smem ? sh : 0, st>>>(n, rp, col, val, E, first, stride, count, hout, a,
                                                                m, sub, tau, work, in_smem ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_csr_superpose(cudaStream_t st, int n, const double* q0, const double* elast,
                                 const double* hsum, const double* g, double* lamT, double* Jdev, int* status) {
  csr_superpose_kernel<<<1, 1024, 0, st>>>(n, q0, elast, hsum, g, lamT, Jdev, status);
  return cudaGetLastError();
}

}  // namespace pxa
