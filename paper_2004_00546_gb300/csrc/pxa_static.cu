// pxa_static.cu — pxa_expv_static: the Krylov propagation of pxa_expv with its scratch
// (Krylov basis, status word, error estimate) in a fixed device array owned by the
// library, for callers that must not allocate device memory. Nothing here allocates.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/pxa.h"
#include "kernels_1d.cuh"

namespace {

// Layout: [0] status word (int in the first double), [1] error estimate,
// [64 ..] Krylov basis (n * (m+1) doubles). 256-byte aligned.
constexpr int kHeader = 64;
static __device__ __align__(256) double g_expv_scratch[PXA_EXPV_STATIC_MAX_DOUBLES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of g_expv_scratch on `device` (that device must be current).
// Looked up once per device; in host code the array's name is only a host-side
// stand-in, so kernels must be given this address, never &g_expv_scratch.
cudaError_t scratch_on(int device, double** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_expv_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = static_cast<double*>(p);
  }
  *out = g_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" int pxa_expv_static(int device, void* cuda_stream, const pxa_operator_desc* op,
                               double T, int64_t K, int m, double tol, int phi, int transpose,
                               int64_t span_steps, int substeps, const double* x_dev,
                               double* y_dev, double* err_host) {
  if (!op || !x_dev || !y_dev || op->kind != PXA_ADVDIFF_1D || op->n < 3 || op->n > 4096 ||
      !(op->L > 0.0) || !(op->nu >= 0.0) || !(T > 0.0) || K < 1 || m < 2 || m > 48 ||
      !(tol > 0.0) || (phi != PXA_PHI_EXP && phi != PXA_PHI_STEPPER) || span_steps < 1 ||
      substeps < 1 || span_steps % substeps != 0 || device < 0 || device >= kMaxDevices)
    return PXA_ERR_INVALID;
  const int n = op->n;
  if ((int64_t)n * (m + 1) > (int64_t)PXA_EXPV_STATIC_MAX_DOUBLES - kHeader) return PXA_ERR_TOO_LARGE;

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return PXA_ERR_CUDA;
  int rc = PXA_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  do {
    if (cudaSetDevice(device) != cudaSuccess) { rc = PXA_ERR_CUDA; break; }
    double* base = nullptr;
    if (scratch_on(device, &base) != cudaSuccess) { rc = PXA_ERR_CUDA; break; }
    int* status = reinterpret_cast<int*>(base);
    double* errmax = base + 1;
    double* V = base + kHeader;
    // status and the running error maximum must start at zero on every call
    if (cudaMemsetAsync(base, 0, 2 * sizeof(double), st) != cudaSuccess) { rc = PXA_ERR_CUDA; break; }
    const double h = op->L / n;
    const double am = op->c / (2.0 * h) + op->nu / (h * h);
    const double a0 = -2.0 * op->nu / (h * h);
    const double ap = -op->c / (2.0 * h) + op->nu / (h * h);
    const double dt = T / (double)K;
    const int64_t sps = span_steps / substeps;
    const double hscale = phi == PXA_PHI_EXP ? dt * (double)sps : dt;
    if (pxa::launch_ad1_expv(st, 256, n, am, a0, ap, transpose, x_dev, y_dev, V, m, phi, hscale, sps,
                             substeps, tol, /*v_in_smem=*/0, status, errmax) != cudaSuccess) {
      rc = PXA_ERR_CUDA;
      break;
    }
    double hdr[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(hdr, base, sizeof(hdr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = PXA_ERR_CUDA;
      break;
    }
    int code = 0;
    static_assert(sizeof(int) <= sizeof(double), "status fits in the first slot");
    memcpy(&code, &hdr[0], sizeof(int));
    if (err_host) *err_host = hdr[1];
    if (code != 0) rc = code;
  } while (0);
  cudaSetDevice(prev);
  return rc;
}
