// kernels_ad1_stream.cu — FP32 Crank–Nicolson band lanes of the 1D advection-diffusion
// problem with the lane states in global memory: the form of Eq. linInhomEqus for grids
// too long to live in shared memory (the batched and 1D lane kernels keep their lanes on
// chip). One launch takes one step of every lane: y_l = M x_l, M the exact circulant CN
// band (taps m_j, |j| <= r), FP32 arithmetic and accumulation.
//
// A persistent grid (SMs x resident blocks) walks the (lane, tile) items, TILE = 2 x 256 x
// PPT points, 256 threads per block. A block stages a tile and the r-point halos on both sides
// (periodic in the lane) in shared memory by cp.async while it steps the previous one:
// each thread steps PPT consecutive points of each half (7, 9 or 11: coprime with the 32
// banks, chosen to pad the band least) with a register window (one shared load per PPT FMAs) into an
// output tile that the block stores with 16-byte vector stores. Global traffic per step: 4 bytes read and 4 written per point,
// plus 2r halo points per tile.
#include "common.cuh"
#include "kernels_1d.cuh"

namespace pxa {

namespace {

constexpr int ST_THREADS = 256;
constexpr int ST_GROUPS = 2;  // groups of 256 x PPT points per tile (halves the per-tile costs)

// points per thread: 7, 9 or 11 (coprime with the 32 banks), whichever pads the band
// (2r + 1 taps) to a multiple of itself with the fewest zero taps
int stream_ppt(int r) {
  const int w = 2 * r + 1;
  int best = 9, waste = 1 << 30;
  for (int p : {11, 9, 7}) {
    const int wv = (w + p - 1) / p * p - w;
    if (wv < waste) {
      waste = wv;
      best = p;
    }
  }
  return best;
}

}  // namespace

__device__ __forceinline__ void cpa16(float* sdst, const float* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cpa4(float* sdst, const float* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Persistent: block b takes the (lane, tile) items b, b + gridDim.x, ...; while it steps
// one tile from shared buffer A, the next tile and its halos stream into buffer B
// (cp.async). Buffers hold xs[i] = x_{t0 + i - r} for i < TILE + 2r and a zero tail, with
// xs + r 16-byte aligned; results go through a separate output tile for 16-byte stores.
template <int ST_PPT>
__global__ void __launch_bounds__(ST_THREADS) ad1_stream_step_kernel(int n, int r, int wp, int lanes,
                                                                     const float* __restrict__ taps,
                                                                     const float* __restrict__ x,
                                                                     float* __restrict__ y) {
  extern __shared__ __align__(16) float sms[];
  constexpr int ST_TILE = ST_GROUPS * ST_THREADS * ST_PPT;  // a multiple of 4
  const int tid = threadIdx.x;
  const int tpl = (n + ST_TILE - 1) / ST_TILE;  // tiles per lane
  const int total = lanes * tpl;
  const int bufw = ((ST_TILE + 2 * r + 3 * ST_PPT + 3) & ~3) + 4;  // floats per input buffer
  float* tp = sms;                                                   // [wp]
  float* ob = tp + ((wp + 3) & ~3);                                  // [TILE], 16-byte aligned
  float* base = ob + ST_TILE;
  float* const xs0 = base + ((4 - (r & 3)) & 3);
  float* const xs1 = xs0 + bufw;
  for (int j = tid; j < wp; j += ST_THREADS) tp[j] = taps[j];
  // the zero tail past a full tile's data (partial tiles zero their own)
  for (int i = tid; i < 3 * ST_PPT; i += ST_THREADS) {
    xs0[2 * r + ST_TILE + i] = 0.f;
    xs1[2 * r + ST_TILE + i] = 0.f;
  }
  auto issue = [&](int item, float* xb) {
    const int lane = item / tpl, tile = item - lane * tpl;
    const int t0 = tile * ST_TILE, cnt = min(ST_TILE, n - t0);
    const float* xl = x + (size_t)lane * n;
    const int nv = cnt >> 2;
    for (int q = tid; q < nv; q += ST_THREADS) cpa16(xb + r + 4 * q, xl + t0 + 4 * q);
    for (int i = 4 * nv + tid; i < cnt; i += ST_THREADS) cpa4(xb + r + i, xl + t0 + i);
    for (int i = tid; i < r; i += ST_THREADS) {
      int gl = t0 - r + i;
      gl += gl < 0 ? n : 0;
      int gr = t0 + cnt + i;
      gr -= gr >= n ? n : 0;
      cpa4(xb + i, xl + gl);
      cpa4(xb + r + cnt + i, xl + gr);
    }
    if (cnt < ST_TILE)
      for (int i = tid; i < ST_TILE - cnt; i += ST_THREADS) xb[2 * r + cnt + i] = 0.f;
  };
  int cur = 0;
  if ((int)blockIdx.x < total) issue(blockIdx.x, xs0);
  cpa_commit();
  const int b = tid * ST_PPT;
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int next = item + gridDim.x;
    if (next < total) issue(next, cur ? xs0 : xs1);
    cpa_commit();
    cpa_wait1();  // this thread's copies of the current tile have landed
    __syncthreads();
#pragma unroll 1
    for (int g = 0; g < ST_GROUPS; ++g) {
      const float* xc = (cur ? xs1 : xs0) + g * ST_THREADS * ST_PPT;
      float acc[ST_PPT], w1[ST_PPT], w2[ST_PPT];
#pragma unroll
      for (int u = 0; u < ST_PPT; ++u) {
        acc[u] = 0.f;
        w1[u] = xc[b + u];
      }
      for (int jb = 0; jb < wp; jb += ST_PPT) {
#pragma unroll
        for (int u = 0; u < ST_PPT; ++u) w2[u] = xc[b + jb + ST_PPT + u];
#pragma unroll
        for (int jj = 0; jj < ST_PPT; ++jj) {
          const float tj = tp[jb + jj];
#pragma unroll
          for (int u = 0; u < ST_PPT; ++u) acc[u] = fmaf(tj, u + jj < ST_PPT ? w1[u + jj] : w2[u + jj - ST_PPT], acc[u]);
        }
#pragma unroll
        for (int u = 0; u < ST_PPT; ++u) w1[u] = w2[u];
      }
#pragma unroll
      for (int u = 0; u < ST_PPT; ++u) ob[g * ST_THREADS * ST_PPT + b + u] = acc[u];
    }
    __syncthreads();  // the output tile is complete; buffer `cur` is free for item + 2 grid
    const int lane = item / tpl, tile = item - lane * tpl;
    const int t0 = tile * ST_TILE, cnt = min(ST_TILE, n - t0);
    float* yl = y + (size_t)lane * n + t0;
    const int nv = cnt >> 2;
    const float4* ov = reinterpret_cast<const float4*>(ob);
    for (int q = tid; q < nv; q += ST_THREADS) reinterpret_cast<float4*>(yl)[q] = ov[q];
    for (int i = 4 * nv + tid; i < cnt; i += ST_THREADS) yl[i] = ob[i];
    cur ^= 1;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// x[l][i] = (float) q0[i] for every lane l; out[l][i] = (double) x[l][i].
__global__ void ad1_stream_fill_kernel(int n, int lanes, const double* __restrict__ q0, float* __restrict__ x) {
  const size_t total = (size_t)n * lanes;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    x[i] = (float)q0[i % n];
}

__global__ void ad1_stream_out_kernel(size_t total, const float* __restrict__ x, double* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)x[i];
}

cudaError_t launch_ad1_stream_fill(cudaStream_t st, int n, int lanes, const double* q0, float* x) {
  ad1_stream_fill_kernel<<<1216, 256, 0, st>>>(n, lanes, q0, x);
  return cudaGetLastError();
}

cudaError_t launch_ad1_stream_out(cudaStream_t st, size_t total, const float* x, double* out) {
  ad1_stream_out_kernel<<<1216, 256, 0, st>>>(total, x, out);
  return cudaGetLastError();
}

size_t ad1_stream_smem(int r) {
  const int p = stream_ppt(r), tile = ST_GROUPS * ST_THREADS * p;
  const int wp = ((2 * r + 1 + p - 1) / p) * p;
  const size_t bufw = (size_t)(((tile + 2 * r + 3 * p + 3) & ~3) + 4);
  return sizeof(float) * ((((size_t)wp + 3) & ~(size_t)3) + tile + 3 + 2 * bufw);
}

int ad1_stream_padded_taps(int r) {
  const int p = stream_ppt(r);
  return ((2 * r + 1 + p - 1) / p) * p;
}

template <int PPT>
static cudaError_t stream_launch(cudaStream_t st, int lanes, int n, int r, const float* taps, const float* x,
                                 float* y) {
  const int wp = ((2 * r + 1 + PPT - 1) / PPT) * PPT;
  const size_t sh = ad1_stream_smem(r);
  const void* fn = (const void*)ad1_stream_step_kernel<PPT>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ad1_stream_step_kernel<PPT>, ST_THREADS, sh);
  const int tile = ST_GROUPS * ST_THREADS * PPT;
  const int items = lanes * ((n + tile - 1) / tile);
  int grid = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  if (grid > items) grid = items;
  ad1_stream_step_kernel<PPT><<<grid, ST_THREADS, sh, st>>>(n, r, wp, lanes, taps, x, y);
  return cudaGetLastError();
}

cudaError_t launch_ad1_stream_step(cudaStream_t st, int lanes, int n, int r, const float* taps_padded,
                                   const float* x, float* y) {
  switch (stream_ppt(r)) {
    case 7: return stream_launch<7>(st, lanes, n, r, taps_padded, x, y);
    case 11: return stream_launch<11>(st, lanes, n, r, taps_padded, x, y);
    default: return stream_launch<9>(st, lanes, n, r, taps_padded, x, y);
  }
}

}  // namespace pxa
