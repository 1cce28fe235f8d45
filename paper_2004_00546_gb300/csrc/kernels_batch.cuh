// kernels_batch.cuh — many independent 1D advection-diffusion problems (uneven grids and
// viscosities) solved together: host-side launch wrappers of kernels_batch.cu.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pxa {

// One problem of the batch (device-visible, set up on the host).
struct BatchInst {
  int n;         // grid points
  int r32;       // half-width of the FP32 Crank-Nicolson band used by the lanes
  int r64;       // half-width of the FP64 band used for the sources
  int nsub;      // Krylov substeps per subinterval
  int rp;        // half-width of the FP32 band of M^(K/P), the subinterval propagator (0: none)
  int64_t off;   // first point of the problem in the packed vectors
  int64_t t32;   // first tap of its FP32 band
  int64_t t64;   // first tap of its FP64 band
  int64_t voff;  // first double of its Krylov basis ((m+1) x n)
  int64_t tpw;   // first tap of its subinterval-propagator band (in the FP32 taps)
  double am, a0, ap;  // stencil of A
  double hsub;   // Krylov substep length (tau / nsub)
};

constexpr int BATCH_THREADS = 256;
constexpr int BATCH_MAX_N = 4096;
constexpr int BATCH_MAX_R = 255;  // widest FP32 band a lane keeps in shared memory
constexpr int BATCH_MAX_RP = 1024;  // widest subinterval-propagator band a chain applies

size_t batch_lanes_smem(int nmax, int rmax);
int batch_lanes_grid(int device, int nmax, int rmax);
cudaError_t launch_batch_cn_lanes(cudaStream_t st, int grid, const BatchInst* inst, const int2* items,
                                  int nitems, int* counter, const float* taps32, int transpose,
                                  int64_t steps, const double* x0, const double* src, double* out,
                                  int lanes, int nmax, int rmax);
cudaError_t launch_batch_band_src(cudaStream_t st, const BatchInst* inst, int count, int nmax,
                                  const double* taps64, int transpose, const double* x, double* y);
cudaError_t launch_batch_chain(cudaStream_t st, const BatchInst* inst, const int* which, int count, int nmax,
                               int m, int transpose, const double* E, int lanes, int first, int stride,
                               int links, double* hout, double* V, double tol, int* status,
                               double* errmax);
// power == 1: one application per link of the problem's band of M^(K/P) (rp, tpw)
// instead of `steps` CN steps.
cudaError_t launch_batch_cn_chain(cudaStream_t st, int grid, const BatchInst* inst, const int2* items,
                                  int nitems, int* counter, const float* taps32, int transpose,
                                  int64_t steps, const double* E, int lanes, int first, int stride,
                                  int links, double* hout, int nmax, int rmax, int power);
cudaError_t launch_batch_superpose_direct(cudaStream_t st, const BatchInst* inst, int count, int nmax,
                                          const double* taps64, const double* q0, const double* E,
                                          int lanes, int last, const double* h, double* qT,
                                          double* srcT, double* J, int* status);
cudaError_t launch_batch_superpose_adjoint(cudaStream_t st, const BatchInst* inst, int count, int nmax,
                                           const double* lamK, const double* EA, int lanes,
                                           const double* h, double* grad, int* status);

// The whole Paraexp gradient as one persistent launch with device-side dependencies
// (kernels_batch.cu, batch_flow_kernel). items: the queue (int4 {type, problem, lane, 0},
// every item after the items it depends on); state: 1 + 4 count ints, zeroed here.
size_t batch_flow_smem(int nmax, int rmax, int rpmax);
int batch_flow_grid(int device, int nmax, int rmax, int rpmax);
cudaError_t launch_batch_flow(cudaStream_t st, int grid, const BatchInst* inst, const int4* items, int nitems,
                              int* state, int count, int P, const float* taps32, const double* taps64, int64_t k,
                              const double* q0, double* src, double* E, double* qT, double* srcT, double* EA,
                              double* J, double* grad, int* status, int nmax, int rmax, int rpmax);

}  // namespace pxa
