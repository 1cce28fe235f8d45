// kernels_bu2.cuh — host-side launch wrappers of the 2D viscous Burgers kernels
// (kernels_bu2.cu). Fields are FP32 [2][n][n] (u then v), n % BU2_TILE == 0.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <algorithm>

namespace pxa {

constexpr int BU2_TILE = 16;

size_t bu2_adj_smem_bytes();
// q_{s+1} = one RK4 step of q_s
cudaError_t launch_bu2_step(cudaStream_t st, const float* q, float* qn, int n, double L, double nu, double dt);
// lo = M_s^T lam, the transposed RK4 step map at the stored state q_s
cudaError_t launch_bu2_adj_step(cudaStream_t st, const float* qs, const float* lam, float* lo, int n, double L,
                                double nu, double dt);
// J = 0.5 ||q(T) - target||^2 (FP64, Jpart: (n/BU2_TILE)^2 partials) and lamT = q(T) - target
cudaError_t launch_bu2_terminal(cudaStream_t st, const float* qT, const double* target, int n, float* lamT,
                                double* Jpart, double* J, int* status);
cudaError_t launch_bu2_convert(cudaStream_t st, const double* x, float* y, size_t count);
cudaError_t launch_bu2_convert_back(cudaStream_t st, const float* x, double* y, size_t count, int* status);

}  // namespace pxa
