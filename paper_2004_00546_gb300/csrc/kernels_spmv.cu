// kernels_spmv.cu — y = A x for an operator in CSR form (the sparse building block of the
// stepping and Arnoldi operators, Sec. 4: the discretised operators are sparse matrices
// with a few entries per row). HBM-bound: per row 8 bytes of row pointer, 12 bytes per
// entry (column index and value), the gathered x and 8 bytes of y.
//
// One thread per row, grid-stride: for the short, uniform rows of stencil operators the
// threads of a warp read neighbouring segments of col/val (the sectors a load leaves
// are taken by the next entry's load from L1) and neighbouring x entries, so HBM sees
// each byte about once.
#include <cuda_runtime.h>

#include <stdint.h>

#include "../../include/pxa.h"

namespace {

__global__ void __launch_bounds__(256) spmv_csr_kernel(int64_t n, const int64_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col,
                                                       const double* __restrict__ val,
                                                       const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k0 = row_ptr[i], k1 = row_ptr[i + 1];
    double s = 0.0;
    for (int64_t k = k0; k < k1; ++k) s = fma(val[k], x[col[k]], s);
    y[i] = s;
  }
}

}  // namespace

extern "C" int pxa_spmv_csr(void* cuda_stream, int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const double* val, const double* x, double* y) {
  if (n < 1 || n > INT32_MAX || !row_ptr || !col || !val || !x || !y) return PXA_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return PXA_ERR_CUDA;
  }
  // enough blocks to keep every SM's load units busy (8 x 256 threads resident per SM)
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 64;
  if (blocks > cap) blocks = cap;
  spmv_csr_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(n, row_ptr, col, val, x, y);
  if (cudaGetLastError() != cudaSuccess) return PXA_ERR_CUDA;
  return PXA_OK;
}
