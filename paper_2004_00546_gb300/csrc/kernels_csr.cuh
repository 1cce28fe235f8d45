// kernels_csr.cuh — host-side launch wrappers of the CSR operator kind (kernels_csr.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pxa {

size_t krylov_smem_bytes(int n, int m, int extra_vecs, bool v_in_smem);
// Bytes of shared memory of one RK4 lane (four vectors) and whether they fit in a block.
size_t csr_lane_smem_bytes(int n);
bool csr_lanes_fit_smem(int n);
// `lanes` blocks: lane l starts from x0[l] (NULL: zero) and takes k RK4 steps of
// du/dt = A u + b (b may be NULL); out[l] = u. work: 4 n lanes doubles, used when the
// lane does not fit in shared memory (may be NULL otherwise).
cudaError_t launch_csr_rk4_lanes(cudaStream_t st, int lanes, int n, const int64_t* rp, const int32_t* col,
                                 const double* val, const double* b, double dt, int64_t k, const double* x0,
                                 double* out, double* work);
// One block: h = 0; for i < count: h += E[first + i stride]; h = Phi h (Krylov); hout = h.
cudaError_t launch_csr_chain(cudaStream_t st, int n, const int64_t* rp, const int32_t* col, const double* val,
                             const double* E, int first, int stride, int count, double* hout, double* Vglob,
                             int m, int phi_mode, double hscale, int64_t steps_per_sub, int nsub, double tol,
                             int v_in_smem, int* status, double* errmax);
// One block: h = 0; for i < count: h += E[first + i stride]; h <- (sum_{j<=m} a_j (tau A)^j)^sub h
// (PXA_PROP_POLY: the RK4 stepper's segment propagator as its power series); hout = h.
// work: 3 n doubles, used when they do not fit in shared memory.
cudaError_t launch_csr_series_chain(cudaStream_t st, int n, const int64_t* rp, const int32_t* col,
                                    const double* val, const double* E, int first, int stride, int count,
                                    double* hout, const double* a, int m, int sub, double tau, double* work);
// q(T) = q0 + elast + hsum, lamT = q(T) - g, J = 0.5 ||lamT||^2 (each input may be NULL).
cudaError_t launch_csr_superpose(cudaStream_t st, int n, const double* q0, const double* elast,
                                 const double* hsum, const double* g, double* lamT, double* Jdev, int* status);

}  // namespace pxa
