// common.cuh — shared device helpers of libpxa (status word, block reductions,
// small dense matrix routines used by the Krylov exponential).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pxa.h"

namespace pxa {

// Kernel nodes of a captured CUDA graph (-1 if the graph cannot be read).
int graph_kernel_nodes(cudaGraph_t g);

constexpr int kMaxM = 48;           // largest Krylov dimension
constexpr int kDMax = kMaxM + 2;    // dense scratch: (m+1) plus the phi_1 augmentation
constexpr int kLD = kDMax;          // leading dimension of dense scratch matrices

// First error wins: later errors do not overwrite the first code.
__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum; `red` is shared scratch of >= 33 doubles. All threads get the sum.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < nw ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Programmatic dependent launch: a kernel launched with the programmatic-serialization
// attribute may start while the kernel before it in the stream still runs. It must wait
// here before it touches anything that kernel writes (or reads what it overwrites);
// before the wait it may only read data written by kernels that finished earlier. Without
// the attribute the wait returns at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel in the stream (if launched with the attribute) start its blocks
// once every block of this grid has passed this point.
__device__ __forceinline__ void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- small dense matrices in shared memory, row-major, leading dimension kLD ----
__device__ __forceinline__ void dense_identity(double* A, int d) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    int i = e / d, j = e % d;
    A[i * kLD + j] = (i == j) ? 1.0 : 0.0;
  }
}

__device__ __forceinline__ void dense_copy(double* dst, const double* src, int d) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    int i = e / d, j = e % d;
    dst[i * kLD + j] = src[i * kLD + j];
  }
}

// C = alpha * A * B + beta_diag * I (C must not alias A or B). Ends with a barrier.
// One entry per thread and pass: the kernels that use it are bound by the SM's FP64
// issue rate, so extra partial sums (more FP64 adds) cost more than they hide.
__device__ __forceinline__ void dense_gemm(double* C, const double* A, const double* B, int d,
                                           double alpha, double beta_diag) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    int i = e / d, j = e % d;
    double acc = 0.0;
    for (int l = 0; l < d; ++l) acc = fma(A[i * kLD + l], B[l * kLD + j], acc);
    C[i * kLD + j] = alpha * acc + (i == j ? beta_diag : 0.0);
  }
  __syncthreads();
}

// Max column-sum norm (1-norm). Ends with a barrier; all threads get the value.
__device__ __forceinline__ double dense_norm1(const double* A, int d, double* red) {
  double m = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += fabs(A[i * kLD + j]);
    m = fmax(m, s);
  }
  m = warp_max(m);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (warp == 0) {
    double s = lane < nw ? red[lane] : 0.0;
    s = warp_max(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// E = exp(X) for a d x d matrix by scaling and squaring of a degree-14 Taylor
// polynomial: X is scaled by 2^-s so that ||X 2^-s||_1 <= 1/4, where the omitted
// tail is below (1/4)^15/15! < 1e-21 relative; the polynomial is evaluated by Horner's
// rule and squared s times. X is overwritten (scaled). T1, T2 are scratch.
__device__ inline void dense_expm(double* E, double* X, double* T1, double* T2, int d,
                                  double* red) {
  double nrm = dense_norm1(X, d, red);
  int s = 0;
  double scale = 1.0;
  while (nrm * scale > 0.25 && s < 60) {
    scale *= 0.5;
    ++s;
  }
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    int i = e / d, j = e % d;
    X[i * kLD + j] *= scale;
  }
  __syncthreads();
  // Horner: E = I + X/14; E = I + X E / k for k = 13 .. 1
  const int deg = 14;
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    int i = e / d, j = e % d;
    E[i * kLD + j] = X[i * kLD + j] / deg + (i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  double* cur = E;
  double* nxt = T1;
  for (int k = deg - 1; k >= 1; --k) {
    dense_gemm(nxt, X, cur, d, 1.0 / k, 1.0);
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int q = 0; q < s; ++q) {
    dense_gemm(nxt, cur, cur, d, 1.0, 0.0);
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  if (cur != E) {
    dense_copy(E, cur, d);
    __syncthreads();
  }
  (void)T2;
}

// Solve A X = B in place (B <- X) by Gauss–Jordan elimination with partial
// pivoting; A is destroyed. `col` is shared scratch of >= kDMax doubles, `ipiv` one int.
__device__ inline void dense_solve(double* A, double* B, int d, double* col, int* ipiv) {
  for (int k = 0; k < d; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + threadIdx.x; i < d; i += 32) {
        double v = fabs(A[i * kLD + k]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) *ipiv = bi;
    }
    __syncthreads();
    int p = *ipiv;
    if (p != k) {
      for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double t = A[k * kLD + j];
        A[k * kLD + j] = A[p * kLD + j];
        A[p * kLD + j] = t;
        t = B[k * kLD + j];
        B[k * kLD + j] = B[p * kLD + j];
        B[p * kLD + j] = t;
      }
    }
    __syncthreads();
    double piv = A[k * kLD + k];
    for (int i = threadIdx.x; i < d; i += blockDim.x) col[i] = A[i * kLD + k];
    __syncthreads();
    double inv = 1.0 / piv;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      A[k * kLD + j] *= inv;
      B[k * kLD + j] *= inv;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
      int i = e / d, j = e % d;
      if (i != k) {
        double f = col[i];
        A[i * kLD + j] -= f * A[k * kLD + j];
        B[i * kLD + j] -= f * B[k * kLD + j];
      }
    }
    __syncthreads();
  }
}

// R^e for a d x d matrix by binary powering with pointer rotation over four buffers
// (R holds the base on entry; E, T1, T2 are scratch; no copies). Returns the buffer
// that holds the result (the identity is written into E when e == 0).
__device__ inline double* dense_pow(double* R, double* E, double* T1, double* T2, int d, int64_t e) {
  double* pool[4] = {R, E, T1, T2};
  int ib = 0, ir = -1;
  if (e <= 0) {
    dense_identity(E, d);
    __syncthreads();
    return E;
  }
  while (e > 0) {
    if (e & 1) {
      if (ir < 0) {
        ir = ib;
      } else {
        int f = 0;
        while (f == ib || f == ir) ++f;
        dense_gemm(pool[f], pool[ir], pool[ib], d, 1.0, 0.0);
        ir = f;
      }
    }
    e >>= 1;
    if (e > 0) {
      int f = 0;
      while (f == ib || f == ir) ++f;
      dense_gemm(pool[f], pool[ib], pool[ib], d, 1.0, 0.0);
      ib = f;
    }
  }
  return pool[ir];
}

}  // namespace pxa
