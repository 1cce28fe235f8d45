// kernels_1d.cu — device kernels of the 1D Paraexp direct-adjoint loop.
//
// Mapping to the paper (Skene, Eggl & Schmid, arXiv 2004.00546):
//   cn_lanes_kernel          Eq. linInhomEqus / Eq. adjInhom: one thread block per
//                            subinterval ("lane"), zero initial value, CN steps of the
//                            shifted problem of Eq. linzero. With one lane and no
//                            source it is plain serial stepping.
//   ad1_chain_kernel         Eq. hom / Eq. adjHomNormal: Krylov exponential (or CN
//                            stepper power) of the summed homogeneous problems,
//                            carried subinterval by subinterval.
//   ad1_relpm_chain_kernel   the same chain with the real Leja points method (Sec. 4.1):
//                            Newton interpolation of phi(z) = (e^z - 1)/z.
//   ad1_superpose_*          Eq. fullsol0 and Eq. fulladjsol at the end points,
//                            J, the adjoint terminal value (Eq. adjFinalTime) and the
//                            initial-condition gradient (Eq. initupdate).
//   (the RK4 direct, adjoint lanes and stepper chain run on thread-block clusters,
//    see kernels_bu1_cluster.cu)
//   bu1_magnus_chain_kernel  Eq. adjHomNormal for the linear time-varying adjoint:
//                            4th-order Magnus steps, Krylov exp and phi_1.
//   sum_lanes_kernel         Eq. fullAdjSolHyb integrated against s(t): the forcing
//                            gradient of Eq. paramupdate.
#include <cooperative_groups.h>

#include "common.cuh"
#include "krylov.cuh"
#include "kernels_1d.cuh"

namespace cg = cooperative_groups;

namespace pxa {

// ----------------------------------------------------------------------------
// Circulant band stepper: x <- M x + src, (M x)_i = sum_{j=-r..r} m_j x_{i+j} (M^T: taps
// reversed), `steps` times, one thread-block cluster of CNL_CL CTAs per lane. A step costs
// n (2r+1) FP64 FMAs, microseconds on one SM (its FP64 units take one warp instruction per
// 64 cycles whatever the active lanes), so the lane is spread over the cluster: every CTA
// keeps the whole vector (X0, X1 with r-point halos, refreshed with every write so that
// the inner loop has no wrap-around test), forms the outputs of its slice 64 points per
// pass (two point groups, the taps of each point split over four warps whose partial
// sums are added in a fixed order), and writes them with their halo copies into the next
// buffer of every CTA through distributed shared memory; one cluster barrier ends a step
// and keeps any CTA from writing into a buffer that another may still read.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void put_halo(T* buf, int n, int r, int p, T v) {
  buf[r + p] = v;
  if (p < r) buf[r + n + p] = v;
  if (p >= n - r) buf[p - n + r] = v;
}

constexpr int CNL_CL = 8;         // CTAs per lane
constexpr int CNL_THREADS = 256;  // 8 warps: 2 point groups x 4 tap groups
constexpr int CNL_TG = 4;

__global__ void __launch_bounds__(CNL_THREADS) cn_lanes_kernel(int n, int r, const double* __restrict__ taps,
                                                               int transpose, int64_t steps,
                                                               const double* __restrict__ x0,
                                                               const double* __restrict__ src,
                                                               double* __restrict__ out) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm[];
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int lane = (int)blockIdx.x / C;
  const int w = 2 * r + 1;
  double* tp = sm;
  double* xa = tp + w;            // the current vector (same offset in every CTA)
  double* xb = xa + n + 2 * r;    // the next one
  double* sr = xb + n + 2 * r;    // [n] the source (own slice)
  double* part = sr + n;          // [8 warps][32] partial sums
  const int nc = (n + C - 1) / C, p0 = rank * nc, p1 = min(n, p0 + nc);
  const int wid = (int)threadIdx.x >> 5, ln = (int)threadIdx.x & 31;
  const int tg = wid % CNL_TG, pg = wid / CNL_TG;
  const int j0 = tg * w / CNL_TG, j1 = (tg + 1) * w / CNL_TG;  // this warp's run of taps
  for (int j = threadIdx.x; j < w; j += blockDim.x) tp[j] = transpose ? taps[w - 1 - j] : taps[j];
  for (int p = threadIdx.x; p < n; p += blockDim.x) put_halo(xa, n, r, p, x0 ? x0[p] : 0.0);
  for (int p = p0 + (int)threadIdx.x; p < p1; p += blockDim.x) sr[p] = src ? src[p] : 0.0;
  cl.sync();  // every CTA of the cluster runs before any remote write
  for (int64_t s = 0; s < steps; ++s) {
    for (int pb = p0; pb < p1; pb += 64) {
      const int p = pb + 32 * pg + ln;
      double acc = 0.0;
      if (p < p1) {
        const double* xp = xa + p;  // xp[r + j] = x_{p+j}
        for (int j = j0; j < j1; ++j) acc = fma(tp[j], xp[j], acc);
      }
      part[wid * 32 + ln] = acc;
      __syncthreads();
      if (tg == 0 && p < p1) {
        const double* pp = part + pg * CNL_TG * 32 + ln;
        const double y = sr[p] + ((pp[0] + pp[32]) + (pp[64] + pp[96]));
        for (int d = 0; d < C; ++d) put_halo(cl.map_shared_rank(xb, d), n, r, p, y);
      }
      __syncthreads();  // part is reused by the next pass
    }
    cl.sync();
    double* t = xa;
    xa = xb;
    xb = t;
  }
  for (int p = p0 + (int)threadIdx.x; p < p1; p += blockDim.x) out[(size_t)lane * n + p] = xa[r + p];
}

// y = M x - x (or M^T x - x) for the circulant band: the source of the shifted lanes.
__global__ void band_minus_identity_kernel(int n, int r, const double* __restrict__ taps,
                                           int transpose, const double* __restrict__ x,
                                           double* __restrict__ y) {
  const int w = 2 * r + 1;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int jj = 0; jj < w; ++jj) {
      int idx = p + jj - r;
      idx += (idx < 0) ? n : 0;
      idx -= (idx >= n) ? n : 0;
      s = fma(transpose ? taps[w - 1 - jj] : taps[jj], x[idx], s);
    }
    y[p] = s - x[p];
  }
}

// y = A x or A^T x (3-point periodic stencil am, a0, ap).
__global__ void ad1_apply_kernel(int n, double am, double a0, double ap, int transpose,
                                 const double* __restrict__ x, double* __restrict__ y) {
  if (transpose) {
    double t = am;
    am = ap;
    ap = t;
  }
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    int im = p == 0 ? n - 1 : p - 1, ip = p == n - 1 ? 0 : p + 1;
    y[p] = am * x[im] + a0 * x[p] + ap * x[ip];
  }
}

// Chain of homogeneous propagations (summed problems, carried lane by lane):
//   h = 0; for i in 0..count-1: h += E[first + i*stride]; h = Phi h.
__global__ void ad1_chain_kernel(int n, double am, double a0, double ap, int transpose,
                                 const double* __restrict__ E, int first, int stride, int count,
                                 double* __restrict__ hout, double* Vglob, int m, int phi_mode,
                                 double hscale, int64_t steps_per_sub, int nsub, double tol,
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
  const int ldv = n;
  if (transpose) {
    double t = am;
    am = ap;
    ap = t;
  }
  Ad1Op op{n, am, a0, ap};
  for (int p = threadIdx.x; p < n; p += blockDim.x) hvec[p] = 0.0;
  __syncthreads();
  for (int i = 0; i < count; ++i) {
    const double* e = E + (size_t)(first + i * stride) * n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) hvec[p] += e[p];
    __syncthreads();
    krylov_propagate(op, hvec, n, m, V, ldv, ks, c, c1, phi_mode, hscale, steps_per_sub, nsub,
                     tol, status, errmax);
  }
  for (int p = threadIdx.x; p < n; p += blockDim.x) hout[p] = hvec[p];
}

// Real Leja points method (Sec. 4.1): h <- exp(ts A)^nsub h, each substep as
// h + ts A p with p = phi(ts A) h, phi(z) = (e^z - 1)/z, interpolated in Newton form at
// the nodes z_j (Leja points of the spectrum's focal interval, scaled by ts):
//   w_0 = h, w_j = (ts A - z_{j-1}) w_{j-1}, p = sum_j D_j w_j,
// stopping when the last two terms fall below tol ||h||. With `direct` the interpolated
// function is the substep's propagator itself (the CN power) and h <- p. Vectors w, p, t in shared
// memory (n each); D, z: the divided differences and nodes (mmax + 1 each).
template <class Op>
__device__ void relpm_propagate(Op& op, double* h, double* w, double* p, double* t, int n,
                                const double* D, const double* z, int mmax, double ts, int nsub,
                                int direct, double tol, double* red, int* status, double* errmax) {
  for (int sub = 0; sub < nsub; ++sub) {
    double ss = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = h[i];
      w[i] = v;
      p[i] = D[0] * v;
      ss = fma(v, v, ss);
    }
    const double hn = sqrt(block_sum(ss, red));
    if (hn == 0.0) continue;  // h stays zero
    double prev = fabs(D[0]) * hn, est = 0.0;
    bool conv = false;
    for (int j = 1; j <= mmax; ++j) {
      op.apply(w, t);  // t = A w (ends with a barrier)
      double s2 = 0.0;
      const double zj = z[j - 1], dj = D[j];
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = fma(ts, t[i], -zj * w[i]);
        w[i] = v;
        p[i] = fma(dj, v, p[i]);
        s2 = fma(v, v, s2);
      }
      est = fabs(dj) * sqrt(block_sum(s2, red));  // (the block sum ends with a barrier)
      if (est + prev <= tol * hn) {
        conv = true;
        break;
      }
      prev = est;
    }
    if (threadIdx.x == 0) {
      atomic_max_pos(errmax, (est + prev) / hn);
      if (!conv) set_status(status, PXA_ERR_NOT_CONVERGED);
    }
    if (direct) {  // the interpolated function is the propagator itself: h <- p
      for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = p[i];
    } else {  // phi: h <- h + ts A p
      op.apply(p, t);
      for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = fma(ts, t[i], h[i]);
    }
    __syncthreads();
  }
}

// Shared layout of the ReLPM kernels: h, w, p, t [n], D, z [mmax + 1], red [40].
__device__ __forceinline__ void relpm_carve(double* sm, int n, int mmax, const double* Dg, const double* zg,
                                            double*& h, double*& w, double*& p, double*& t, double*& D,
                                            double*& z, double*& red) {
  h = sm;
  w = h + n;
  p = w + n;
  t = p + n;
  D = t + n;
  z = D + mmax + 1;
  red = z + mmax + 1;
  for (int j = threadIdx.x; j <= mmax; j += blockDim.x) {
    D[j] = Dg[j];
    z[j] = zg[j];
  }
}

// The chain of Eq. hom / Eq. adjHomNormal with ReLPM exponentials (as ad1_chain_kernel):
//   h = 0; for i in 0..count-1: h += E[first + i*stride]; h = exp(tau A) h.
__global__ void ad1_relpm_chain_kernel(int n, double am, double a0, double ap, int transpose,
                                       const double* __restrict__ E, int first, int stride, int count,
                                       double* __restrict__ hout, const double* __restrict__ Dg,
                                       const double* __restrict__ zg, int mmax, double ts, int nsub,
                                       int direct, double tol, int* status, double* errmax) {
  extern __shared__ double sm[];
  double *h, *w, *p, *t, *D, *z, *red;
  relpm_carve(sm, n, mmax, Dg, zg, h, w, p, t, D, z, red);
  if (transpose) {
    const double x = am;
    am = ap;
    ap = x;
  }
  Ad1Op op{n, am, a0, ap};
  for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = 0.0;
  __syncthreads();
  for (int l = 0; l < count; ++l) {
    const double* e = E + (size_t)(first + l * stride) * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] += e[i];
    __syncthreads();
    relpm_propagate(op, h, w, p, t, n, D, z, mmax, ts, nsub, direct, tol, red, status, errmax);
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) hout[i] = h[i];
}

// Eq. hom / Eq. adjHomNormal with the subinterval propagator B itself as a circulant band
// (exp(tau A) or the CN power M^(K/P); periodic grid, constant coefficients):
// h = 0; for l < count: h += E[first + l stride]; h = B h (B^T: taps reversed).
// One thread-block cluster: B's band can span the whole circulant, so every CTA keeps the
// whole vector (buffers X0, X1 with r-point halos as in cn_lanes_kernel); in link l
// each CTA adds E's row to its copy of X[l % 2], forms the outputs of its slice of points
// (32 at a time, each point's taps split over the CTA's warps, whose partial sums warp 0
// adds in a fixed order: an FP64 warp instruction costs the same with idle lanes, so the
// split, not the lane count, sets the time) and writes them, with their halo copies,
// into X[(l + 1) % 2] of every CTA of the cluster through distributed shared memory.
// The cluster barrier that ends a link makes the new vector complete everywhere and
// keeps any CTA from writing into a buffer that another may still read.
__global__ void ad1_band_chain_kernel(int n, int r, const double* __restrict__ taps, int transpose,
                                      const double* __restrict__ E, int first, int stride, int count,
                                      double* __restrict__ hout) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm[];
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int w = 2 * r + 1;
  double* tp = sm;
  double* xa = tp + w;              // the current vector (same offset in every CTA)
  double* xb = xa + n + 2 * r;      // the next one
  double* part = xb + n + 2 * r;    // [warps][32] partial sums
  const int nc = (n + C - 1) / C, p0 = rank * nc, p1 = min(n, p0 + nc);
  const int G = (int)blockDim.x / 32, lane = (int)threadIdx.x & 31, g = (int)threadIdx.x >> 5;
  const int j0 = g * w / G, j1 = (g + 1) * w / G;  // this warp's run of taps
  for (int j = threadIdx.x; j < w; j += blockDim.x) tp[j] = transpose ? taps[w - 1 - j] : taps[j];
  for (int p = threadIdx.x; p < n; p += blockDim.x) put_halo(xa, n, r, p, 0.0);
  cl.sync();  // every CTA of the cluster runs before any remote write
  for (int l = 0; l < count; ++l) {
    const double* e = E + (size_t)(first + l * stride) * n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) put_halo(xa, n, r, p, xa[r + p] + e[p]);
    __syncthreads();
    for (int pb = p0; pb < p1; pb += 32) {
      const int p = pb + lane;
      double acc = 0.0;
      if (p < p1) {
        const double* xp = xa + p;  // xp[r + j] = x_{p+j}
        for (int j = j0; j < j1; ++j) acc = fma(tp[j], xp[j], acc);
      }
      part[g * 32 + lane] = acc;
      __syncthreads();
      if (g == 0 && p < p1) {
        double y = part[lane];
        for (int q = 1; q < G; ++q) y += part[q * 32 + lane];
        for (int d = 0; d < C; ++d) put_halo(cl.map_shared_rank(xb, d), n, r, p, y);
      }
      __syncthreads();  // part is reused by the next 32 points
    }
    cl.sync();
    double* t = xa;
    xa = xb;
    xb = t;
  }
  for (int p = p0 + (int)threadIdx.x; p < p1; p += blockDim.x) hout[p] = xa[r + p];
}

cudaError_t launch_ad1_band_chain(cudaStream_t st, int n, int r, const double* taps, int transpose,
                                  const double* E, int first, int stride, int count, double* hout) {
  constexpr int CL = 8;  // CTAs of the cluster (portable size)
  const size_t sh = sizeof(double) * ((size_t)(2 * r + 1) + 2 * (size_t)(n + 2 * r) + 256);
  cudaError_t e = cudaFuncSetAttribute(ad1_band_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = sh;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ad1_band_chain_kernel, n, r, taps, transpose, E, first, stride, count, hout);
}

// One vector: y = exp(ts A)^nsub x (building block).
__global__ void ad1_relpm_expv_kernel(int n, double am, double a0, double ap, int transpose,
                                      const double* __restrict__ x, double* __restrict__ y,
                                      const double* __restrict__ Dg, const double* __restrict__ zg, int mmax,
                                      double ts, int nsub, int direct, double tol, int* status,
                                      double* errmax) {
  extern __shared__ double sm[];
  double *h, *w, *p, *t, *D, *z, *red;
  relpm_carve(sm, n, mmax, Dg, zg, h, w, p, t, D, z, red);
  if (transpose) {
    const double s = am;
    am = ap;
    ap = s;
  }
  Ad1Op op{n, am, a0, ap};
  for (int i = threadIdx.x; i < n; i += blockDim.x) h[i] = x[i];
  __syncthreads();
  relpm_propagate(op, h, w, p, t, n, D, z, mmax, ts, nsub, direct, tol, red, status, errmax);
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = h[i];
}

// Direct superposition at t = T (Eq. fullsol0): q(T) = q0 + e_{P-1} + hsum;
// J = 0.5 ||q(T) - g||^2 (g = 0 when NULL); qT receives lambda_K = q(T) - g
// (Eq. adjFinalTime) and srcT the adjoint lanes' source (M^T - I) lambda_K of the shifted
// adjoint (Eq. adjInhom, discrete form).
__global__ void ad1_superpose_direct_kernel(int n, int r, const double* __restrict__ taps,
                                            const double* __restrict__ q0,
                                            const double* __restrict__ elast,
                                            const double* __restrict__ hsum,
                                            const double* __restrict__ g,
                                            double* __restrict__ qT, double* __restrict__ srcT,
                                            double* __restrict__ Jdev, int* status) {
  extern __shared__ double sm[];
  double* red = sm;
  double* q = sm + 40;
  const int w = 2 * r + 1;
  double acc = 0.0;
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    // lambda(T) = dJ/dq(T) = q(T) - g for J = 0.5 ||q(T) - g||^2 (g = 0 when absent)
    double v = (q0 ? q0[p] : 0.0) + (elast ? elast[p] : 0.0) + (hsum ? hsum[p] : 0.0) - (g ? g[p] : 0.0);
    q[p] = v;
    qT[p] = v;
    acc = fma(v, v, acc);
  }
  double J = 0.5 * block_sum(acc, red);
  if (threadIdx.x == 0) {
    *Jdev = J;
    if (!isfinite(J)) set_status(status, PXA_ERR_NONFINITE);
  }
  if (srcT) {
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      // (M^T x)_p = sum_j m_{-j} x_{p+j} = sum_j taps[w-1-(r+j)] x_{p+j}
      double s = 0.0;
      for (int jj = 0; jj < w; ++jj) {
        int off = jj - r;
        int idx = p + off;
        idx += (idx < 0) ? n : 0;
        idx -= (idx >= n) ? n : 0;
        s = fma(taps[w - 1 - jj], q[idx], s);
      }
      srcT[p] = s - q[p];
    }
  }
}

// Adjoint superposition at t = 0 (Eq. fulladjsol) and the IC gradient
// (Eq. initupdate): grad = lambda_K + e_0 + hsum.
__global__ void ad1_superpose_adjoint_kernel(int n, const double* __restrict__ lamK,
                                             const double* __restrict__ e0,
                                             const double* __restrict__ hsum,
                                             double* __restrict__ grad, int* status) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double v = (lamK ? lamK[p] : 0.0) + (e0 ? e0[p] : 0.0) + (hsum ? hsum[p] : 0.0);
    grad[p] = v;
    if (!isfinite(v)) set_status(status, PXA_ERR_NONFINITE);
  }
}

// Krylov propagation of a single vector (building block for tests).
__global__ void ad1_expv_kernel(int n, double am, double a0, double ap, int transpose,
                                const double* __restrict__ x, double* __restrict__ y,
                                double* Vglob, int m, int phi_mode, double hscale,
                                int64_t steps_per_sub, int nsub, double tol, int v_in_smem,
                                int* status, double* errmax) {
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
  if (transpose) {
    double t = am;
    am = ap;
    ap = t;
  }
  Ad1Op op{n, am, a0, ap};
  for (int p = threadIdx.x; p < n; p += blockDim.x) hvec[p] = x[p];
  __syncthreads();
  krylov_propagate(op, hvec, n, m, V, n, ks, c, c1, phi_mode, hscale, steps_per_sub, nsub, tol,
                   status, errmax);
  for (int p = threadIdx.x; p < n; p += blockDim.x) y[p] = hvec[p];
}

// ============================================================================
// 1D viscous Burgers
// ============================================================================
// N(y)_p on a halo-1 buffer (y[p+1] is point p).
__device__ __forceinline__ double bu1_rhs_at(const Bu1Grid& g, const double* y, int p) {
  double ym = y[p], y0 = y[p + 1], yp = y[p + 2];
  double ux = (yp - ym) * g.inv2h;
  double uxx = (yp - 2.0 * y0 + ym) * g.invh2;
  return -y0 * ux + g.nu * uxx;
}

// (J(U)^T x)_p on halo-1 buffers: column p of J(U) holds -dU_p - 2nu/h^2 on the
// diagonal, -U_{p-1}/(2h) + nu/h^2 in row p-1 and U_{p+1}/(2h) + nu/h^2 in row p+1.
__device__ __forceinline__ double bu1_jacT_at(const Bu1Grid& g, const double* U, const double* x,
                                              int p) {
  double Um = U[p], Up = U[p + 2];
  double diag = -(Up - Um) * g.inv2h - 2.0 * g.nu * g.invh2;
  double from_m = -Um * g.inv2h + g.nu * g.invh2;
  double from_p = Up * g.inv2h + g.nu * g.invh2;
  return diag * x[p + 1] + from_m * x[p] + from_p * x[p + 2];
}

__device__ __forceinline__ void put1(double* buf, int n, int p, double v) {
  buf[p + 1] = v;
  if (p == 0) buf[n + 1] = v;
  if (p == n - 1) buf[0] = v;
}

__device__ __forceinline__ double forcing_s(double omega, double t) {
  return omega == 0.0 ? 1.0 : sin(omega * t);
}

// Address of direct state row s: contiguous rows (lane_k == 0) or the per-lane
// recompute layout, where lane l holds rows l*k .. l*k+k in a block of k+1 rows.
__device__ __forceinline__ const double* row_ptr(const double* base, int n, int64_t s,
                                                 int64_t lane_k, int lanes) {
  if (lane_k == 0) return base + (size_t)s * n;
  int64_t l = s / lane_k;
  if (l > lanes - 1) l = lanes - 1;
  return base + ((size_t)l * (size_t)(lane_k + 1) + (size_t)(s - l * lane_k)) * n;
}

// Magnus operator of one backward step of the adjoint (time reversed, tau = t_top - t):
//   Omega x = (H/2)(B1 + B2) x + (sqrt(3)/12) H^2 (B2 B1 - B1 B2) x,
// B_i = J(U(t_i))^T at the Gauss nodes t_i = t_top - g_i H, g_{1,2} = 1/2 -+ sqrt(3)/6.
struct MagnusOp {
  Bu1Grid g;
  double H, c2;
  const double* U1;  // halo-1
  const double* U2;  // halo-1
  double* t1;        // halo-1 scratch
  double* t2;        // halo-1 scratch
  double* xs;        // halo-1 copy of x
  __device__ void apply(const double* x, double* y) {
    const int n = g.n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) put1(xs, n, p, x[p]);
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      put1(t1, n, p, bu1_jacT_at(g, U1, xs, p));
      put1(t2, n, p, bu1_jacT_at(g, U2, xs, p));
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      double b21 = bu1_jacT_at(g, U2, t1, p);
      double b12 = bu1_jacT_at(g, U1, t2, p);
      y[p] = 0.5 * H * (t1[p + 1] + t2[p + 1]) + c2 * (b21 - b12);
    }
    __syncthreads();
  }
};

// 4-point Lagrange interpolation in time of the stored trajectory (rows 0..K).
__device__ __forceinline__ void interp_rows(const double* traj, int n, int64_t K, double dt,
                                            double t, double* out_halo, int64_t lane_k,
                                            int lanes) {
  double s = t / dt;
  int64_t i0 = (int64_t)floor(s) - 1;
  if (i0 < 0) i0 = 0;
  if (i0 > K - 3) i0 = K - 3;
  double w[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double c = 1.0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (b != a) c *= (s - (double)(i0 + b)) / (double)(a - b);
    w[a] = c;
  }
  const double* r0 = row_ptr(traj, n, i0, lane_k, lanes);
  const double* r1 = row_ptr(traj, n, i0 + 1, lane_k, lanes);
  const double* r2 = row_ptr(traj, n, i0 + 2, lane_k, lanes);
  const double* r3 = row_ptr(traj, n, i0 + 3, lane_k, lanes);
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    double acc = w[0] * r0[p];
    acc = fma(w[1], r1[p], acc);
    acc = fma(w[2], r2[p], acc);
    acc = fma(w[3], r3[p], acc);
    put1(out_halo, n, p, acc);
  }
}

// Homogeneous adjoint chain (summed problems carried from subinterval P-2 down to 0)
// with 4th-order Magnus steps of M RK4 steps each; the gradient integral of the
// homogeneous part rides on the augmented system [lambda; gamma]:
//   gamma <- gamma + W phi_1(Omega) lambda,  lambda <- exp(Omega) lambda,
//   W = (H/2)(s1 + s2) I + (sqrt(3)/12) H^2 (s2 B1 - s1 B2).
template <int PPT>
__global__ void bu1_magnus_chain_kernel(Bu1Grid g, double dt, int64_t K, int P, int64_t k,
                                        int M, double omega, const double* __restrict__ traj,
                                        int64_t lane_k, const double* __restrict__ W,
                                        double* __restrict__ gH, double* Vglob, int m,
                                        double tol, int v_in_smem, int* status,
                                        double* errmax) {
  extern __shared__ double sm[];
  const int n = g.n;
  double* cur = sm;
  KrylovScratch ks = ks_carve(cur);
  double* c = cur;
  cur += kDMax;
  double* c1 = cur;
  cur += kDMax;
  double* U1 = cur;
  cur += n + 2;
  double* U2 = cur;
  cur += n + 2;
  double* t1 = cur;
  cur += n + 2;
  double* t2 = cur;
  cur += n + 2;
  double* xs = cur;
  cur += n + 2;
  double* hvec = cur;
  cur += n;
  double* V = v_in_smem ? cur : Vglob;
  const double H = M * dt;
  const double c2 = sqrt(3.0) / 12.0 * H * H;
  const double g1 = 0.5 - sqrt(3.0) / 6.0, g2 = 0.5 + sqrt(3.0) / 6.0;
  MagnusOp op{g, H, c2, U1, U2, t1, t2, xs};
  double gacc[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) gacc[q] = 0.0;
  for (int p = threadIdx.x; p < n; p += blockDim.x) hvec[p] = 0.0;
  __syncthreads();
  for (int lane = P - 2; lane >= 0; --lane) {
    const double* w = W + (size_t)(lane + 1) * n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) hvec[p] += w[p];
    __syncthreads();
    const int64_t s0 = (int64_t)lane * k, s1 = s0 + k;
    for (int64_t s = s1; s > s0; s -= M) {
      const double ttop = (double)s * dt;
      const double tn1 = ttop - g1 * H, tn2 = ttop - g2 * H;
      interp_rows(traj, n, K, dt, tn1, U1, lane_k, P);
      interp_rows(traj, n, K, dt, tn2, U2, lane_k, P);
      __syncthreads();
      int mm = 0;
      double beta = arnoldi(op, hvec, n, m, V, n, ks, &mm);
      if (mm == 0) continue;
      double fm = hessenberg_phi(ks, mm, 0, 1.0, 0, true, c, c1);
      double err = (mm == m) ? ks.H[m * kLD + (m - 1)] * fm : 0.0;
      if (threadIdx.x == 0) {
        atomic_max_pos(errmax, err);
        if (!(err <= tol)) set_status(status, PXA_ERR_NOT_CONVERGED);
      }
      // phi_1(Omega) lambda into xs (halo), then the gradient contribution
      for (int p = threadIdx.x; p < n; p += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < mm; ++i) acc = fma(c1[i], V[(size_t)i * n + p], acc);
        put1(xs, n, p, beta * acc);
      }
      __syncthreads();
      const double sa = forcing_s(omega, tn1), sb = forcing_s(omega, tn2);
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        int p = threadIdx.x + q * blockDim.x;
        if (p < n) {
          double b1 = bu1_jacT_at(g, U1, xs, p);
          double b2 = bu1_jacT_at(g, U2, xs, p);
          gacc[q] += 0.5 * H * (sa + sb) * xs[p + 1] + c2 * (sb * b1 - sa * b2);
        }
      }
      krylov_combine(V, n, mm, c, beta, hvec, n);
    }
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    int p = threadIdx.x + q * blockDim.x;
    if (p < n) gH[p] = gacc[q];
  }
}

// grad = sum_{lane} G[lane] + extra (forcing gradient of Eq. paramupdate).
__global__ void sum_lanes_kernel(int n, int lanes, const double* __restrict__ G,
                                 const double* __restrict__ extra, double* __restrict__ grad,
                                 int* status) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double acc = extra ? extra[p] : 0.0;
    for (int l = 0; l < lanes; ++l) acc += G[(size_t)l * n + p];
    grad[p] = acc;
    if (!isfinite(acc)) set_status(status, PXA_ERR_NONFINITE);
  }
}

__global__ void bu1_rhs_kernel(Bu1Grid g, const double* __restrict__ u, double* __restrict__ y) {
  const int n = g.n;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    int im = p == 0 ? n - 1 : p - 1, ip = p == n - 1 ? 0 : p + 1;
    double b[3] = {u[im], u[p], u[ip]};
    y[p] = bu1_rhs_at(g, b, 0);
  }
}

__global__ void bu1_jacT_kernel(Bu1Grid g, const double* __restrict__ U,
                                const double* __restrict__ x, double* __restrict__ y) {
  const int n = g.n;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    int im = p == 0 ? n - 1 : p - 1, ip = p == n - 1 ? 0 : p + 1;
    double ub[3] = {U[im], U[p], U[ip]};
    double xb[3] = {x[im], x[p], x[ip]};
    y[p] = bu1_jacT_at(g, ub, xb, 0);
  }
}

// ---- host-side launch wrappers ------------------------------------------------
size_t ks_layout_doubles() {
  return (size_t)(kMaxM + 1) * kLD + 4 * (size_t)kLD * kLD + kDMax + 40 + 2;
}

cudaError_t launch_cn_lanes(cudaStream_t st, int lanes, int threads, int n, int r,
                            const double* taps, int transpose, int64_t steps, const double* x0,
                            const double* src, double* out) {
  (void)threads;  // the cluster kernel's block shape is fixed
  const size_t sh = sizeof(double) * ((size_t)(2 * r + 1) + 2 * (size_t)(n + 2 * r) + n + 8 * 32);
  cudaError_t e = cudaFuncSetAttribute(cn_lanes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(lanes * CNL_CL);
  cfg.blockDim = dim3(CNL_THREADS);
  cfg.dynamicSmemBytes = sh;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CNL_CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cn_lanes_kernel, n, r, taps, transpose, steps, x0, src, out);
}

cudaError_t launch_band_minus_identity(cudaStream_t st, int n, int r, const double* taps,
                                       int transpose, const double* x, double* y) {
  int threads = 256, blocks = (n + threads - 1) / threads;
  band_minus_identity_kernel<<<blocks, threads, 0, st>>>(n, r, taps, transpose, x, y);
  return cudaGetLastError();
}

cudaError_t launch_ad1_apply(cudaStream_t st, int n, double am, double a0, double ap,
                             int transpose, const double* x, double* y) {
  int threads = 256, blocks = (n + threads - 1) / threads;
  ad1_apply_kernel<<<blocks, threads, 0, st>>>(n, am, a0, ap, transpose, x, y);
  return cudaGetLastError();
}

size_t krylov_smem_bytes(int n, int m, int extra_vecs, bool v_in_smem) {
  size_t d = ks_layout_doubles() + 2 * kDMax + (size_t)extra_vecs;
  if (v_in_smem) d += (size_t)(m + 1) * n;
  return d * sizeof(double);
}

cudaError_t launch_ad1_chain(cudaStream_t st, int threads, int n, double am, double a0, double ap,
                             int transpose, const double* E, int first, int stride, int count,
                             double* hout, double* Vglob, int m, int phi_mode, double hscale,
                             int64_t steps_per_sub, int nsub, double tol, int v_in_smem,
                             int* status, double* errmax) {
  size_t sh = krylov_smem_bytes(n, m, n, v_in_smem != 0);
  cudaError_t e = cudaFuncSetAttribute(ad1_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  ad1_chain_kernel<<<1, threads, sh, st>>>(n, am, a0, ap, transpose, E, first, stride, count,
                                            hout, Vglob, m, phi_mode, hscale, steps_per_sub, nsub,
                                            tol, v_in_smem, status, errmax);
  return cudaGetLastError();
}

static size_t relpm_smem(int n, int mmax) { return sizeof(double) * (4 * (size_t)n + 2 * (size_t)(mmax + 1) + 40); }

cudaError_t launch_ad1_relpm_chain(cudaStream_t st, int threads, int n, double am, double a0, double ap,
                                   int transpose, const double* E, int first, int stride, int count,
                                   double* hout, const double* D, const double* z, int mmax, double ts,
                                   int nsub, int direct, double tol, int* status, double* errmax) {
  const size_t sh = relpm_smem(n, mmax);
  cudaError_t e = cudaFuncSetAttribute(ad1_relpm_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  ad1_relpm_chain_kernel<<<1, threads, sh, st>>>(n, am, a0, ap, transpose, E, first, stride, count, hout, D, z,
                                                  mmax, ts, nsub, direct, tol, status, errmax);
  return cudaGetLastError();
}

cudaError_t launch_ad1_relpm_expv(cudaStream_t st, int threads, int n, double am, double a0, double ap,
                                  int transpose, const double* x, double* y, const double* D, const double* z,
                                  int mmax, double ts, int nsub, int direct, double tol, int* status,
                                  double* errmax) {
  const size_t sh = relpm_smem(n, mmax);
  cudaError_t e = cudaFuncSetAttribute(ad1_relpm_expv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  ad1_relpm_expv_kernel<<<1, threads, sh, st>>>(n, am, a0, ap, transpose, x, y, D, z, mmax, ts, nsub, direct,
                                                 tol, status, errmax);
  return cudaGetLastError();
}

cudaError_t launch_ad1_expv(cudaStream_t st, int threads, int n, double am, double a0, double ap,
                            int transpose, const double* x, double* y, double* Vglob, int m,
                            int phi_mode, double hscale, int64_t steps_per_sub, int nsub,
                            double tol, int v_in_smem, int* status, double* errmax) {
  size_t sh = krylov_smem_bytes(n, m, n, v_in_smem != 0);
  cudaError_t e = cudaFuncSetAttribute(ad1_expv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  ad1_expv_kernel<<<1, threads, sh, st>>>(n, am, a0, ap, transpose, x, y, Vglob, m, phi_mode,
                                           hscale, steps_per_sub, nsub, tol, v_in_smem, status,
                                           errmax);
  return cudaGetLastError();
}

cudaError_t launch_ad1_superpose_direct(cudaStream_t st, int threads, int n, int r,
                                        const double* taps, const double* q0, const double* elast,
                                        const double* hsum, const double* g, double* qT, double* srcT,
                                        double* J, int* status) {
  size_t sh = sizeof(double) * (40 + (size_t)n);
  if (sh > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(ad1_superpose_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
  }
  ad1_superpose_direct_kernel<<<1, threads, sh, st>>>(n, r, taps, q0, elast, hsum, g, qT, srcT, J,
                                                       status);
  return cudaGetLastError();
}

cudaError_t launch_ad1_superpose_adjoint(cudaStream_t st, int n, const double* lamK,
                                         const double* e0, const double* hsum, double* grad,
                                         int* status) {
  int threads = 256, blocks = (n + threads - 1) / threads;
  ad1_superpose_adjoint_kernel<<<blocks, threads, 0, st>>>(n, lamK, e0, hsum, grad, status);
  return cudaGetLastError();
}

template <int PPT>
static cudaError_t launch_mag_t(cudaStream_t st, int threads, size_t sh, Bu1Grid g, double dt,
                                int64_t K, int P, int64_t k, int M, double omega,
                                const double* traj, int64_t lane_k, const double* W, double* gH, double* Vglob,
                                int m, double tol, int v_in_smem, int* status, double* errmax) {
  cudaError_t e = cudaFuncSetAttribute(bu1_magnus_chain_kernel<PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  bu1_magnus_chain_kernel<PPT><<<1, threads, sh, st>>>(g, dt, K, P, k, M, omega, traj, lane_k, W, gH, Vglob,
                                                       m, tol, v_in_smem, status, errmax);
  return cudaGetLastError();
}

cudaError_t launch_bu1_magnus_chain(cudaStream_t st, int threads, Bu1Grid g, double dt, int64_t K,
                                    int P, int64_t k, int M, double omega, const double* traj,
                                    int64_t lane_k, const double* W, double* gH, double* Vglob, int m, double tol,
                                    int v_in_smem, int* status, double* errmax) {
  size_t sh = krylov_smem_bytes(g.n, m, 5 * (g.n + 2) + g.n, v_in_smem != 0);
  int ppt = (g.n + threads - 1) / threads;
  if (ppt <= 1) return launch_mag_t<1>(st, threads, sh, g, dt, K, P, k, M, omega, traj, lane_k, W, gH, Vglob, m, tol, v_in_smem, status, errmax);
  if (ppt <= 2) return launch_mag_t<2>(st, threads, sh, g, dt, K, P, k, M, omega, traj, lane_k, W, gH, Vglob, m, tol, v_in_smem, status, errmax);
  if (ppt <= 4) return launch_mag_t<4>(st, threads, sh, g, dt, K, P, k, M, omega, traj, lane_k, W, gH, Vglob, m, tol, v_in_smem, status, errmax);
  return cudaErrorInvalidValue;
}

cudaError_t launch_sum_lanes(cudaStream_t st, int n, int lanes, const double* G, const double* extra,
                             double* grad, int* status) {
  int threads = 256, blocks = (n + threads - 1) / threads;
  sum_lanes_kernel<<<blocks, threads, 0, st>>>(n, lanes, G, extra, grad, status);
  return cudaGetLastError();
}

cudaError_t launch_bu1_rhs(cudaStream_t st, Bu1Grid g, const double* u, double* y) {
  int threads = 256, blocks = (g.n + threads - 1) / threads;
  bu1_rhs_kernel<<<blocks, threads, 0, st>>>(g, u, y);
  return cudaGetLastError();
}

cudaError_t launch_bu1_jacT(cudaStream_t st, Bu1Grid g, const double* U, const double* x, double* y) {
  int threads = 256, blocks = (g.n + threads - 1) / threads;
  bu1_jacT_kernel<<<blocks, threads, 0, st>>>(g, U, x, y);
  return cudaGetLastError();
}

}  // namespace pxa
