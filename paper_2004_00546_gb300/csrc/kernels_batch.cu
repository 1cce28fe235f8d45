// kernels_batch.cu — Alg. 1 for many independent 1D advection-diffusion problems at once
// (uneven grid sizes and viscosities), one launch per phase over the whole batch.
//
//   batch_cn_lanes_kernel          Eq. linInhomEqus / Eq. adjInhom for every (problem,
//                                  subinterval) pair: a persistent grid takes the lanes
//                                  from a cost-sorted list (largest first) through an
//                                  atomic counter; each lane steps the Crank-Nicolson
//                                  band in FP32 with FP32 accumulation in shared memory.
//                                  With one lane per problem and no source it is plain
//                                  serial stepping.
//   batch_band_src_kernel          the lanes' constant source (M - I) x of Eq. linzero
//                                  (FP64 band), per problem.
//   batch_chain_kernel             Eq. hom / Eq. adjHomNormal: one thread block per
//                                  problem carries the summed homogeneous problems link
//                                  by link with the Krylov exponential exp(tau A) in FP64
//                                  (substeps per problem from its stiffness).
//   batch_cn_chain_kernel          the same with the stepper's own propagator (the local
//                                  chained form, FP32 band), for the problems where it is
//                                  cheaper than the Krylov exponential.
//   batch_superpose_*              Eq. fullsol0 / Eq. fulladjsol, J_i = 0.5 ||q_i(T)||^2,
//                                  the adjoint terminal value and the IC gradient, FP64.
#include <algorithm>

#include "common.cuh"
#include "krylov.cuh"
#include "kernels_batch.cuh"
#include "kernels_1d.cuh"

namespace pxa {

namespace {

__device__ __forceinline__ void put_halo32(float* buf, int n, int r, int p, float v) {
  buf[r + p] = v;
  if (p < r) buf[r + n + p] = v;
  if (p >= n - r) buf[p - n + r] = v;
}

__device__ __forceinline__ int wrapb(int g, int n) {
  g %= n;
  return g < 0 ? g + n : g;
}

}  // namespace

// ---- lanes ----------------------------------------------------------------------------
// One CN step of the FP32 band on the block's points. Thread t owns the PPT consecutive
// points t*PPT .. t*PPT+PPT-1 (PPT odd, so that the threads of a warp read shared memory
// at a stride coprime with the 32 banks) and keeps a window of 2*PPT state values in
// registers: taps are taken PPT at a time (the band is zero-padded to a multiple of
// PPT), each tap and each new state value is read from shared memory once and feeds PPT
// FMAs. xa[i] = x_{i-r}; the tap j of point p reads xa[p + j].
template <int PPT>
__device__ __forceinline__ void band_step32(const float* __restrict__ tp, int wp, const float* __restrict__ xa,
                                            float* __restrict__ xb, const float* __restrict__ sr, int n,
                                            int r) {
  const int b = threadIdx.x * PPT;
  if (b >= n) return;
  float acc[PPT], w1[PPT], w2[PPT];
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    acc[u] = (sr && b + u < n) ? sr[b + u] : 0.f;
    w1[u] = xa[b + u];
  }
  for (int jb = 0; jb < wp; jb += PPT) {
#pragma unroll
    for (int u = 0; u < PPT; ++u) w2[u] = xa[b + jb + PPT + u];
#pragma unroll
    for (int jj = 0; jj < PPT; ++jj) {
      const float tj = tp[jb + jj];
#pragma unroll
      for (int u = 0; u < PPT; ++u) acc[u] = fmaf(tj, u + jj < PPT ? w1[u + jj] : w2[u + jj - PPT], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < PPT; ++u) w1[u] = w2[u];
  }
#pragma unroll
  for (int u = 0; u < PPT; ++u)
    if (b + u < n) put_halo32(xb, n, r, b + u, acc[u]);
}

// Shared layout of one lane: taps [wp] (zero beyond 2r+1), xa and xb [n + 2r + 2 PPT]
// (the tail past the halo is zero: it meets only the zero taps), src [n].
template <int PPT>
__device__ __forceinline__ void lane_layout(float* smf, int n, int r, int w, float*& tp, int& wp, float*& xa,
                                            float*& xb, float*& sr) {
  wp = ((w + PPT - 1) / PPT) * PPT;
  tp = smf;
  xa = tp + ((wp + 3) & ~3);
  const int len = n + 2 * r + 2 * PPT;
  xb = xa + len;
  sr = xb + len;
  for (int j = threadIdx.x; j < 2 * PPT; j += blockDim.x) {
    xa[n + 2 * r + j] = 0.f;
    xb[n + 2 * r + j] = 0.f;
  }
}

// items[it] = {problem, lane}. A lane takes `steps` CN steps of its problem's FP32 band
// (transposed when `transpose`) from x0 (FP64 packed, NULL = zero) with the constant
// source src (FP64 packed, NULL = none) and writes its end state (FP64) to
// out + off * lanes + lane * n. Shared: taps[2 r + 1], xa, xb [n + 2 r], src [n].
template <int PPT>
__global__ void __launch_bounds__(BATCH_THREADS) batch_cn_lanes_kernel(
    const BatchInst* __restrict__ inst, const int2* __restrict__ items, int nitems, int* counter,
    const float* __restrict__ taps32, int transpose, int64_t steps, const double* __restrict__ x0,
    const double* __restrict__ src, double* __restrict__ out, int lanes) {
  extern __shared__ float smf[];
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = cur;
    if (it >= nitems) return;  // the same for every thread of the block
    const int2 wk = items[it];
    const BatchInst I = inst[wk.x];
    const int n = I.n, r = I.r32, w = 2 * r + 1;
    float *tp, *xa, *xb, *sr;
    int wp;
    lane_layout<PPT>(smf, n, r, w, tp, wp, xa, xb, sr);
    const float* tg = taps32 + I.t32;
    for (int j = threadIdx.x; j < wp; j += blockDim.x) tp[j] = j < w ? (transpose ? tg[w - 1 - j] : tg[j]) : 0.f;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      put_halo32(xa, n, r, p, x0 ? (float)x0[I.off + p] : 0.f);
      sr[p] = src ? (float)src[I.off + p] : 0.f;
    }
    __syncthreads();
    for (int64_t s = 0; s < steps; ++s) {
      band_step32<PPT>(tp, wp, xa, xb, src ? sr : nullptr, n, r);
      __syncthreads();
      float* t = xa;
      xa = xb;
      xb = t;
    }
    double* o = out + I.off * lanes + (int64_t)wk.y * n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) o[p] = (double)xa[r + p];
    __syncthreads();  // shared memory and `cur` are reused by the next lane
  }
}

// ---- homogeneous chains with the stepper's own propagator (the local chained form) ---
// items[it] = {problem, 0}: x = 0; for l < links: x += E[first + l * stride] (FP64 lane end
// states, packed with `lanes` lanes per problem); x <- M^steps x (M^T when `transpose`) in
// FP32; the result goes to hout (FP64 packed). This is the homogeneous propagation of
// Eq. hom / Eq. adjHomNormal with the stepper's own propagator, carried subinterval by
// subinterval: by `steps` CN steps, or (power == 1) by one application of the circulant
// band of M^(K/P) itself (the problem's rp, tpw), whose taps the host takes from the
// eigenvalues R_k^(K/P). A link then costs one band product instead of K/P.
template <int PPT>
__global__ void __launch_bounds__(BATCH_THREADS) batch_cn_chain_kernel(
    const BatchInst* __restrict__ inst, const int2* __restrict__ items, int nitems, int* counter,
    const float* __restrict__ taps32, int transpose, int64_t steps, const double* __restrict__ E,
    int lanes, int first, int stride, int links, double* __restrict__ hout, int power) {
  extern __shared__ float smf[];
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = cur;
    if (it >= nitems) return;  // the same for every thread of the block
    const BatchInst I = inst[items[it].x];
    const int n = I.n, r = power ? I.rp : I.r32, w = 2 * r + 1;
    const int64_t nst = power ? 1 : steps;
    float *tp, *xa, *xb, *sr;
    int wp;
    lane_layout<PPT>(smf, n, r, w, tp, wp, xa, xb, sr);
    const float* tg = taps32 + (power ? I.tpw : I.t32);
    const double* Ei = E + I.off * lanes;
    for (int j = threadIdx.x; j < wp; j += blockDim.x) tp[j] = j < w ? (transpose ? tg[w - 1 - j] : tg[j]) : 0.f;
    for (int p = threadIdx.x; p < n; p += blockDim.x) put_halo32(xa, n, r, p, 0.f);
    __syncthreads();
    for (int l = 0; l < links; ++l) {
      const double* e = Ei + (int64_t)(first + l * stride) * n;
      for (int p = threadIdx.x; p < n; p += blockDim.x) put_halo32(xa, n, r, p, xa[r + p] + (float)e[p]);
      __syncthreads();
      for (int64_t s = 0; s < nst; ++s) {
        band_step32<PPT>(tp, wp, xa, xb, nullptr, n, r);
        __syncthreads();
        float* t = xa;
        xa = xb;
        xb = t;
      }
    }
    for (int p = threadIdx.x; p < n; p += blockDim.x) hout[I.off + p] = (double)xa[r + p];
    __syncthreads();  // shared memory and `cur` are reused by the next problem
  }
}

// ---- sources --------------------------------------------------------------------------
// Grid (point blocks, problems): y_i = (M_i - I) x_i, or (M_i^T - I) x_i, FP64 band.
__global__ void batch_band_src_kernel(const BatchInst* __restrict__ inst, const double* __restrict__ taps64,
                                      int transpose, const double* __restrict__ x, double* __restrict__ y) {
  const BatchInst I = inst[blockIdx.y];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= I.n) return;
  const int r = I.r64, w = 2 * r + 1;
  const double* tg = taps64 + I.t64;
  const double* xi = x + I.off;
  double acc = 0.0;
  for (int jj = 0; jj < w; ++jj) {
    // (M x)_p = sum_j m_j x_{p+j}; (M^T x)_p = sum_j m_{-j} x_{p+j}
    const double t = transpose ? tg[w - 1 - jj] : tg[jj];
    acc = fma(t, xi[wrapb(p + jj - r, I.n)], acc);
  }
  y[I.off + p] = acc - xi[p];
}

// ---- homogeneous chains ---------------------------------------------------------------
// One block per problem of the list `which`: h = 0; for l < links: h += E[first + l * stride];
// h = exp(tau A) h (A^T when `transpose`), each exponential in nsub Krylov substeps of
// length hsub.
__global__ void batch_chain_kernel(
    const BatchInst* __restrict__ inst, const int* __restrict__ which, int m, int transpose,
    const double* __restrict__ E, int lanes, int first, int stride, int links, double* __restrict__ hout,
    double* __restrict__ Vg, double tol, int* status, double* errmax) {
  extern __shared__ double smd[];
  const BatchInst I = inst[which[blockIdx.x]];
  const int n = I.n;
  double* cur = smd;
  KrylovScratch ks = ks_carve(cur);
  double* c = cur;
  cur += kDMax;
  double* c1 = cur;
  cur += kDMax;
  double* hvec = cur;
  Ad1Op op{n, transpose ? I.ap : I.am, I.a0, transpose ? I.am : I.ap};
  double* V = Vg + I.voff;
  const double* Ei = E + I.off * lanes;
  for (int p = threadIdx.x; p < n; p += blockDim.x) hvec[p] = 0.0;
  __syncthreads();
  for (int l = 0; l < links; ++l) {
    const double* e = Ei + (int64_t)(first + l * stride) * n;
    for (int p = threadIdx.x; p < n; p += blockDim.x) hvec[p] += e[p];
    __syncthreads();
    krylov_propagate(op, hvec, n, m, V, n, ks, c, c1, 0, I.hsub, 1, I.nsub, tol, status, errmax);
  }
  for (int p = threadIdx.x; p < n; p += blockDim.x) hout[I.off + p] = hvec[p];
}

// ---- superposition ------------------------------------------------------------------
// One block per problem: qT = q0 + E[last] + h (each term optional), J_i = 0.5 ||qT||^2,
// srcT = (M^T - I) qT (the adjoint lanes' source) when srcT is given.
__global__ void __launch_bounds__(BATCH_THREADS) batch_superpose_direct_kernel(
    const BatchInst* __restrict__ inst, const double* __restrict__ taps64, const double* __restrict__ q0,
    const double* __restrict__ E, int lanes, int last, const double* __restrict__ h,
    double* __restrict__ qT, double* __restrict__ srcT, double* __restrict__ J, int* status) {
  __shared__ double red[40];
  const int i = blockIdx.x;
  const BatchInst I = inst[i];
  const int n = I.n;
  const double* el = E + I.off * lanes + (int64_t)last * n;
  double acc = 0.0;
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const double v = (q0 ? q0[I.off + p] : 0.0) + el[p] + (h ? h[I.off + p] : 0.0);
    qT[I.off + p] = v;
    acc = fma(v, v, acc);
  }
  const double Ji = 0.5 * block_sum(acc, red);
  if (threadIdx.x == 0) {
    J[i] = Ji;
    if (!isfinite(Ji)) set_status(status, PXA_ERR_NONFINITE);
  }
  __syncthreads();  // qT complete before the band reads neighbours
  if (srcT) {
    const int r = I.r64, w = 2 * r + 1;
    const double* tg = taps64 + I.t64;
    const double* q = qT + I.off;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      double s = 0.0;
      for (int jj = 0; jj < w; ++jj) s = fma(tg[w - 1 - jj], q[wrapb(p + jj - r, n)], s);
      srcT[I.off + p] = s - q[p];
    }
  }
}

// Grid (point blocks, problems): grad = lamK + EA[0] + h (each optional but EA).
__global__ void batch_superpose_adjoint_kernel(const BatchInst* __restrict__ inst,
                                               const double* __restrict__ lamK,
                                               const double* __restrict__ EA, int lanes,
                                               const double* __restrict__ h, double* __restrict__ grad,
                                               int* status) {
  const BatchInst I = inst[blockIdx.y];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= I.n) return;
  const double v = (lamK ? lamK[I.off + p] : 0.0) + EA[I.off * lanes + p] + (h ? h[I.off + p] : 0.0);
  grad[I.off + p] = v;
  if (!isfinite(v)) set_status(status, PXA_ERR_NONFINITE);
}

// ---- one persistent launch with device-side dependencies --------------------------------
// The whole Paraexp gradient of every problem as one launch: a persistent grid takes work
// items from a queue through an atomic counter. Items (int4 {type, problem, lane, 0}):
//   FLOW_SRC        the lanes' source (M - I) q0_i of Eq. linzero (FP64 band)
//   FLOW_LANE       one direct lane (Eq. linInhomEqus), after its problem's source
//   FLOW_CHAIN_SUP  the direct chain (Eq. hom) and the superposition (Eq. fullsol0, J_i,
//                   the adjoint lanes' source (M^T - I) q_i(T)), after all P lanes
//   FLOW_ALANE      one adjoint lane (Eq. adjInhom), after the superposition
//   FLOW_ACHAIN_GRAD the adjoint chain (Eq. adjHomNormal) and the gradient (Eq. fulladjsol,
//                   Eq. initupdate), after all P adjoint lanes
// A finished item publishes its results (every thread fences its writes, then one thread
// adds to the problem's counter in `flags`); an item first waits, one thread polling with
// acquire loads and a bounded spin (PXA_ERR_TIMEOUT after ~2^31 cycles), for its counter
// to reach the target. The queue lists every item after the items it depends on, and a
// block claims an item only while it runs, so every awaited item is held by a running
// block that waits only on earlier items: the waits end. Results read from other blocks
// go through L2 (__ldcg). The arithmetic of each item is that of the phase kernels above,
// so the results are bit-identical to theirs.
enum { FLOW_SRC = 0, FLOW_LANE = 1, FLOW_CHAIN_SUP = 2, FLOW_ALANE = 3, FLOW_ACHAIN_GRAD = 4 };

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits (bounded) until *flag >= target; ends with a block barrier.
__device__ __forceinline__ void flow_wait(const int* flag, int target, int* status) {
  if (threadIdx.x == 0 && ld_acquire(flag) < target) {
    const long long t0 = clock64();
    for (int it = 1;; ++it) {
      if (ld_acquire(flag) >= target) break;
      __nanosleep(64);
      if ((it & 63) == 0) {
        if (*(volatile int*)status != 0) break;
        if (clock64() - t0 > (1LL << 31)) {
          set_status(status, PXA_ERR_TIMEOUT);
          break;
        }
      }
    }
  }
  __syncthreads();
}

// Every thread fences its global writes; after the barrier one thread publishes.
__device__ __forceinline__ void flow_signal(int* flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(flag, 1);
}

template <int PPT>
__global__ void __launch_bounds__(BATCH_THREADS) batch_flow_kernel(
    const BatchInst* __restrict__ inst, const int4* __restrict__ items, int nitems, int* counter, int* flags,
    int count, int P, const float* __restrict__ taps32, const double* __restrict__ taps64, int64_t k,
    const double* __restrict__ q0, double* src, double* E, double* qT, double* srcT, double* EA,
    double* __restrict__ J, double* __restrict__ grad, int* status) {
  extern __shared__ float smf[];
  __shared__ int cur;
  __shared__ double red[40];
  int* const f_src = flags;
  int* const f_lanes = flags + count;
  int* const f_sup = flags + 2 * count;
  int* const f_alanes = flags + 3 * count;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = cur;
    if (it >= nitems) return;  // the same for every thread of the block
    const int4 wk = items[it];
    const int type = wk.x, i = wk.y, lane = wk.z;
    const BatchInst I = inst[i];
    const int n = I.n;
    if (type == FLOW_SRC) {
      const int r = I.r64, w = 2 * r + 1;
      const double* tg = taps64 + I.t64;
      const double* xi = q0 + I.off;
      for (int p = threadIdx.x; p < n; p += blockDim.x) {
        double acc = 0.0;
        for (int jj = 0; jj < w; ++jj) acc = fma(tg[jj], xi[wrapb(p + jj - r, n)], acc);
        src[I.off + p] = acc - xi[p];
      }
      flow_signal(f_src + i);
    } else if (type == FLOW_LANE || type == FLOW_ALANE) {
      const bool adj = type == FLOW_ALANE;
      flow_wait(adj ? f_sup + i : f_src + i, 1, status);
      const double* sg = adj ? srcT : src;
      const int r = I.r32, w = 2 * r + 1;
      float *tp, *xa, *xb, *sr;
      int wp;
      lane_layout<PPT>(smf, n, r, w, tp, wp, xa, xb, sr);
      const float* tg = taps32 + I.t32;
      for (int j = threadIdx.x; j < wp; j += blockDim.x) tp[j] = j < w ? (adj ? tg[w - 1 - j] : tg[j]) : 0.f;
      for (int p = threadIdx.x; p < n; p += blockDim.x) {
        put_halo32(xa, n, r, p, 0.f);
        sr[p] = (float)__ldcg(sg + I.off + p);
      }
      __syncthreads();
      for (int64_t s = 0; s < k; ++s) {
        band_step32<PPT>(tp, wp, xa, xb, sr, n, r);
        __syncthreads();
        float* t = xa;
        xa = xb;
        xb = t;
      }
      double* o = (adj ? EA : E) + I.off * P + (int64_t)lane * n;
      for (int p = threadIdx.x; p < n; p += blockDim.x) o[p] = (double)xa[r + p];
      flow_signal((adj ? f_alanes : f_lanes) + i);
    } else {
      // the chain of the summed homogeneous problems (direct: links over E[0 .. P-2];
      // adjoint: over EA[P-1 .. 1] with the transposed band), then the superposition
      const bool adj = type == FLOW_ACHAIN_GRAD;
      flow_wait(adj ? f_alanes + i : f_lanes + i, P, status);
      const bool power = I.rp > 0;
      const int r = power ? I.rp : I.r32, w = 2 * r + 1;
      const int64_t nst = power ? 1 : k;
      float *tp, *xa, *xb, *sr;
      int wp;
      lane_layout<PPT>(smf, n, r, w, tp, wp, xa, xb, sr);
      const float* tg = taps32 + (power ? I.tpw : I.t32);
      const double* Ei = (adj ? EA : E) + I.off * P;
      for (int j = threadIdx.x; j < wp; j += blockDim.x) tp[j] = j < w ? (adj ? tg[w - 1 - j] : tg[j]) : 0.f;
      for (int p = threadIdx.x; p < n; p += blockDim.x) put_halo32(xa, n, r, p, 0.f);
      __syncthreads();
      const int first = adj ? P - 1 : 0, stride = adj ? -1 : 1;
      for (int l = 0; l < P - 1; ++l) {
        const double* e = Ei + (int64_t)(first + l * stride) * n;
        for (int p = threadIdx.x; p < n; p += blockDim.x) put_halo32(xa, n, r, p, xa[r + p] + (float)__ldcg(e + p));
        __syncthreads();
        for (int64_t s = 0; s < nst; ++s) {
          band_step32<PPT>(tp, wp, xa, xb, nullptr, n, r);
          __syncthreads();
          float* t = xa;
          xa = xb;
          xb = t;
        }
      }
      if (!adj) {
        // qT = q0 + E[P-1] + h, J_i = 0.5 ||qT||^2, srcT = (M^T - I) qT
        const double* el = Ei + (int64_t)(P - 1) * n;
        double acc = 0.0;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
          const double v = q0[I.off + p] + __ldcg(el + p) + (P > 1 ? (double)xa[r + p] : 0.0);
          qT[I.off + p] = v;
          acc = fma(v, v, acc);
        }
        const double Ji = 0.5 * block_sum(acc, red);
        if (threadIdx.x == 0) {
          J[i] = Ji;
          if (!isfinite(Ji)) set_status(status, PXA_ERR_NONFINITE);
        }
        __syncthreads();  // qT complete before the band reads neighbours
        const int r6 = I.r64, w6 = 2 * r6 + 1;
        const double* t6 = taps64 + I.t64;
        const double* q = qT + I.off;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
          double s2 = 0.0;
          for (int jj = 0; jj < w6; ++jj) s2 = fma(t6[w6 - 1 - jj], q[wrapb(p + jj - r6, n)], s2);
          srcT[I.off + p] = s2 - q[p];
        }
        flow_signal(f_sup + i);
      } else {
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
          const double v = __ldcg(qT + I.off + p) + __ldcg(Ei + p) + (P > 1 ? (double)xa[r + p] : 0.0);
          grad[I.off + p] = v;
          if (!isfinite(v)) set_status(status, PXA_ERR_NONFINITE);
        }
        __syncthreads();  // shared memory and `cur` are reused by the next item
      }
    }
  }
}

// ---- launch wrappers ------------------------------------------------------------------
namespace {
constexpr int PPT_SMALL = 9, PPT_LARGE = 17;  // odd: coprime with the 32 shared-memory banks
bool small_lanes(int nmax) { return nmax <= PPT_SMALL * BATCH_THREADS; }
}  // namespace

size_t batch_lanes_smem(int nmax, int rmax) {
  const int ppt = small_lanes(nmax) ? PPT_SMALL : PPT_LARGE;
  const int wp = ((2 * rmax + 1 + ppt - 1) / ppt) * ppt;
  return sizeof(float) * ((size_t)((wp + 3) & ~3) + 2 * (size_t)(nmax + 2 * rmax + 2 * ppt) + (size_t)nmax);
}

int batch_lanes_grid(int device, int nmax, int rmax) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const size_t sh = batch_lanes_smem(nmax, rmax);
  const void* fn = small_lanes(nmax) ? (const void*)batch_cn_lanes_kernel<PPT_SMALL>
                                     : (const void*)batch_cn_lanes_kernel<PPT_LARGE>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, BATCH_THREADS, sh);
  if (per < 1) per = 1;
  return (sms > 0 ? sms : 1) * per;
}

cudaError_t launch_batch_cn_lanes(cudaStream_t st, int grid, const BatchInst* inst, const int2* items,
                                  int nitems, int* counter, const float* taps32, int transpose,
                                  int64_t steps, const double* x0, const double* src, double* out,
                                  int lanes, int nmax, int rmax) {
  const size_t sh = batch_lanes_smem(nmax, rmax);
  const bool small = small_lanes(nmax);
  const void* fn = small ? (const void*)batch_cn_lanes_kernel<PPT_SMALL> : (const void*)batch_cn_lanes_kernel<PPT_LARGE>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (small)
    batch_cn_lanes_kernel<PPT_SMALL><<<grid, BATCH_THREADS, sh, st>>>(inst, items, nitems, counter, taps32, transpose,
                                                               steps, x0, src, out, lanes);
  else
    batch_cn_lanes_kernel<PPT_LARGE><<<grid, BATCH_THREADS, sh, st>>>(inst, items, nitems, counter, taps32, transpose,
                                                                steps, x0, src, out, lanes);
  return cudaGetLastError();
}

cudaError_t launch_batch_band_src(cudaStream_t st, const BatchInst* inst, int count, int nmax,
                                  const double* taps64, int transpose, const double* x, double* y) {
  dim3 grid((nmax + 255) / 256, count);
  batch_band_src_kernel<<<grid, 256, 0, st>>>(inst, taps64, transpose, x, y);
  return cudaGetLastError();
}

cudaError_t launch_batch_chain(cudaStream_t st, const BatchInst* inst, const int* which, int count, int nmax,
                               int m, int transpose, const double* E, int lanes, int first, int stride,
                               int links, double* hout, double* V, double tol, int* status,
                               double* errmax) {
  if (links <= 0 || count <= 0) return cudaSuccess;
  const size_t sh = krylov_smem_bytes(nmax, m, nmax, false);
  cudaError_t e = cudaFuncSetAttribute(batch_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  batch_chain_kernel<<<count, BATCH_THREADS, sh, st>>>(inst, which, m, transpose, E, lanes, first, stride,
                                                        links, hout, V, tol, status, errmax);
  return cudaGetLastError();
}

cudaError_t launch_batch_cn_chain(cudaStream_t st, int grid, const BatchInst* inst, const int2* items,
                                  int nitems, int* counter, const float* taps32, int transpose,
                                  int64_t steps, const double* E, int lanes, int first, int stride,
                                  int links, double* hout, int nmax, int rmax, int power) {
  if (nitems <= 0 || links <= 0) return cudaSuccess;
  const size_t sh = batch_lanes_smem(nmax, rmax);
  const bool small = small_lanes(nmax);
  const void* fn = small ? (const void*)batch_cn_chain_kernel<PPT_SMALL> : (const void*)batch_cn_chain_kernel<PPT_LARGE>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (small)
    batch_cn_chain_kernel<PPT_SMALL><<<grid, BATCH_THREADS, sh, st>>>(inst, items, nitems, counter, taps32, transpose, steps,
                                                               E, lanes, first, stride, links, hout, power);
  else
    batch_cn_chain_kernel<PPT_LARGE><<<grid, BATCH_THREADS, sh, st>>>(inst, items, nitems, counter, taps32, transpose,
                                                                steps, E, lanes, first, stride, links, hout, power);
  return cudaGetLastError();
}

cudaError_t launch_batch_superpose_direct(cudaStream_t st, const BatchInst* inst, int count, int nmax,
                                          const double* taps64, const double* q0, const double* E,
                                          int lanes, int last, const double* h, double* qT,
                                          double* srcT, double* J, int* status) {
  (void)nmax;
  batch_superpose_direct_kernel<<<count, BATCH_THREADS, 0, st>>>(inst, taps64, q0, E, lanes, last, h, qT,
                                                                  srcT, J, status);
  return cudaGetLastError();
}

cudaError_t launch_batch_superpose_adjoint(cudaStream_t st, const BatchInst* inst, int count, int nmax,
                                           const double* lamK, const double* EA, int lanes,
                                           const double* h, double* grad, int* status) {
  dim3 grid((nmax + 255) / 256, count);
  batch_superpose_adjoint_kernel<<<grid, 256, 0, st>>>(inst, lamK, EA, lanes, h, grad, status);
  return cudaGetLastError();
}

size_t batch_flow_smem(int nmax, int rmax, int rpmax) {
  return std::max(batch_lanes_smem(nmax, rmax), batch_lanes_smem(nmax, std::max(rpmax, rmax)));
}

int batch_flow_grid(int device, int nmax, int rmax, int rpmax) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const size_t sh = batch_flow_smem(nmax, rmax, rpmax);
  const void* fn = small_lanes(nmax) ? (const void*)batch_flow_kernel<PPT_SMALL> : (const void*)batch_flow_kernel<PPT_LARGE>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, BATCH_THREADS, sh);
  if (per < 1) per = 1;
  return (sms > 0 ? sms : 1) * per;
}

cudaError_t launch_batch_flow(cudaStream_t st, int grid, const BatchInst* inst, const int4* items, int nitems,
                              int* state, int count, int P, const float* taps32, const double* taps64, int64_t k,
                              const double* q0, double* src, double* E, double* qT, double* srcT, double* EA,
                              double* J, double* grad, int* status, int nmax, int rmax, int rpmax) {
  const size_t sh = batch_flow_smem(nmax, rmax, rpmax);
  const bool small = small_lanes(nmax);
  const void* fn = small ? (const void*)batch_flow_kernel<PPT_SMALL> : (const void*)batch_flow_kernel<PPT_LARGE>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  // state: [0] the queue counter, [1 ..] the per-problem counters (4 count)
  e = cudaMemsetAsync(state, 0, sizeof(int) * (1 + 4 * (size_t)count), st);
  if (e != cudaSuccess) return e;
  if (small)
    batch_flow_kernel<PPT_SMALL><<<grid, BATCH_THREADS, sh, st>>>(inst, items, nitems, state, state + 1, count, P, taps32,
                                                           taps64, k, q0, src, E, qT, srcT, EA, J, grad, status);
  else
    batch_flow_kernel<PPT_LARGE><<<grid, BATCH_THREADS, sh, st>>>(inst, items, nitems, state, state + 1, count, P, taps32,
                                                            taps64, k, q0, src, E, qT, srcT, EA, J, grad, status);
  return cudaGetLastError();
}

}  // namespace pxa
