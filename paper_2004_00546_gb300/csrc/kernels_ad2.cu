// kernels_ad2.cu — 2D advection-diffusion with a frozen velocity field (Sec. 4.2),
// FP32 RK4 stepping on halo tiles staged in shared memory by TMA.
//
// State layout (per lane, FP32): a padded array [ny + 2G][nx + 2G], G = 4 ghost
// layers holding periodic copies, so that every tile's halo is a plain rectangle of
// global memory. One CTA owns a TX x TY tile; its (TX+2G) x (TY+2G) halo tile and the
// coefficient tiles (u, v, forcing) arrive by cp.async.bulk.tensor (TMA) completing on
// an mbarrier. The four RK4 stages are fused in shared memory on shrinking regions
// (halo 3, 2, 1, 0), so one time step reads the state once and writes it once: the
// kernel is bound by HBM (FP32: 8 bytes and ~60 flop per point per step). Edge tiles
// also write the periodic ghost copies of their points.
//
// The transposed kernel runs one reverse step of the exact discrete adjoint of the
// linear RK4 map (four applications of A^T fused on halo 3..0 from a halo-4 tile),
// adds the objective's source read from the stored direct trajectory, and
// accumulates the forcing gradient (FP32 per step, FP64 across steps).
//
// Paper mapping: Eq. seriesDirect (serial direct of the hybrid scheme),
// Eq. hybadjinhom (adjoint lanes), Eq. adjHomNormal with the stepper's own
// propagator (homogeneous chain), Eq. paramupdate / Eq. update (forcing gradient).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "common.cuh"
#include "kernels_ad2.cuh"

namespace pxa {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait on an mbarrier phase; false if the limit was reached.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ double forcing_s(double omega, double t) {
  return omega == 0.0 ? 1.0 : sin(omega * t);
}

// acc (hi, lo) += g in FP32 arithmetic: Knuth's two-sum gives the rounding error of hi + g
// exactly, and it is carried in lo (about 2^-44 relative overall, without the FP64 pipe,
// which issues one warp instruction per 64 cycles on GB300). Rounded adds, never fused.
__device__ __forceinline__ float2 df_add(float2 acc, float g) {
  const float s = __fadd_rn(acc.x, g);
  const float bp = __fsub_rn(s, acc.x);
  const float err = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, bp)), __fsub_rn(g, bp));
  return make_float2(s, __fadd_rn(acc.y, err));
}

// (A x)_c on a tile (row pitch BX2): advective central differences + 5-point Laplacian.
__device__ __forceinline__ float A_at(const Ad2Params& p, const float* x, const float* u,
                                      const float* v, int c) {
  float xe = x[c + 1], xw = x[c - 1], xn = x[c + BX2], xs = x[c - BX2], x0 = x[c];
  float qx = (xe - xw) * p.inv2h, qy = (xn - xs) * p.inv2h;
  float lap = (xe + xw + xn + xs - 4.0f * x0) * p.invh2;
  return -u[c] * qx - v[c] * qy + p.nu * lap;
}

// (A^T x)_c: the west neighbour's row holds c as its east entry, and so on.
__device__ __forceinline__ float AT_at(const Ad2Params& p, const float* x, const float* u,
                                       const float* v, int c) {
  const float d = p.nu * p.invh2;
  float aw = -u[c - 1] * p.inv2h + d, ae = u[c + 1] * p.inv2h + d;
  float as = -v[c - BX2] * p.inv2h + d, an = v[c + BX2] * p.inv2h + d;
  return aw * x[c - 1] + ae * x[c + 1] + as * x[c - BX2] + an * x[c + BX2] - 4.0f * d * x[c];
}

// Store value `val` of domain point (x, y) into a padded array and into its periodic
// ghost copies. With nx, ny >= 2G a point has at most one alias per axis.
__device__ __forceinline__ void store_with_ghosts(float* dst, const Ad2Params& p, int x, int y,
                                                  float val) {
  const int X = x + G2, Y = y + G2;
  dst[(size_t)Y * p.Wp + X] = val;
  const bool xl = x < G2, xh = x >= p.nx - G2, yl = y < G2, yh = y >= p.ny - G2;
  if (!(xl | xh | yl | yh)) return;
  const int Xa = xl ? X + p.nx : X - p.nx;
  const int Ya = yl ? Y + p.ny : Y - p.ny;
  const bool hx = xl | xh, hy = yl | yh;
  if (hx) dst[(size_t)Y * p.Wp + Xa] = val;
  if (hy) dst[(size_t)Ya * p.Wp + X] = val;
  if (hx && hy) dst[(size_t)Ya * p.Wp + Xa] = val;
}

struct TileSmem {
  float* coef;  // [3][TILE2] u, v, forcing
  float* q[2];  // double-buffered state tiles
  float* ya;
  float* yb;
  float* acc;
  uint64_t* bar;  // [3]: coef, q[0], q[1]
  double* red;    // 40
  float* sc;      // 8: s(t) at the three stage times, double-buffered by lane parity
};

__device__ __forceinline__ TileSmem carve(unsigned char* raw) {
  TileSmem t;
  float* f = reinterpret_cast<float*>(raw);
  t.coef = f;
  t.q[0] = f + 3 * TILE2;
  t.q[1] = f + 4 * TILE2;
  t.ya = f + 5 * TILE2;
  t.yb = f + 6 * TILE2;
  t.acc = f + 7 * TILE2;
  t.bar = reinterpret_cast<uint64_t*>(f + 8 * TILE2);
  t.red = reinterpret_cast<double*>(t.bar + 4);
  t.sc = reinterpret_cast<float*>(t.red + 40);
  return t;
}

}  // namespace

size_t ad2_smem_bytes() {
  return (size_t)8 * TILE2 * sizeof(float) + 4 * sizeof(uint64_t) + 40 * sizeof(double) + 8 * sizeof(float);
}

// One RK4 time step of dq/dt = A q + s(t) f for a group of lanes on one tile.
//
// Thread layout: 64 columns x 4 row groups. Thread (tx, ty) owns tile column tx + 1
// and RG consecutive rows of the halo-3 region, for every lane and every stage, so
// that the stencil coefficients of its points (cE, cW, cN, cS from u, v; the forcing)
// are computed once per CTA and kept in registers, vertical neighbours come from its
// own registers, and only horizontal neighbours and the two strip ends go through
// shared memory (stage values ping-pong between two tile buffers, one barrier per
// stage). Lane l (global index) is at absolute step l * lane_k + s_local.
// in/out: padded state arrays of the ping-pong pair, tensor-map z = buf * map_lanes + l.
// traj (optional): interior of lane 0's new state as row traj_row. Jpart (WITH_J): the
// eight warps' partials of ||q_new||^2 over the tile (FP32) at
// Jpart[(jrow * tiles + tile) * AD2_J_WARPS + warp]; launch_ad2_reduce_J sums them.
template <bool WITH_J>
__global__ void __launch_bounds__(256, 2) ad2_rk4_kernel(const __grid_constant__ CUtensorMap qmap,
                                                         const __grid_constant__ CUtensorMap cmap,
                                                         Ad2Params p, float* __restrict__ states,
                                                         int lanes, int map_lanes, int lanes_per_cta,
                                                         int buf_in, int64_t lane_k, int64_t s_local,
                                                         const float* __restrict__ sc,
                                                         float* __restrict__ traj, int64_t traj_row,
                                                         float* __restrict__ Jpart, int64_t jrow,
                                                         int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem t = carve(smem_raw);
  const int tile = blockIdx.x;
  const int tbx = tile % p.tiles_x, tby = tile / p.tiles_x;
  const int x0 = tbx * TX2, y0 = tby * TY2;  // padded coordinates of the halo corner
  const int l_begin = blockIdx.y * lanes_per_cta;
  const int l_end = min(lanes, l_begin + lanes_per_cta);
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int col = tx + 1;                       // tile column
  const bool colact = col <= BX2 - 2;           // inside the halo-3 region [1, BX2-1)
  const int row0 = 1 + ty * RG2;                // first owned row
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&t.bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the coefficient tile (written before the sweep) is loaded before the wait for the
  // previous step; the state tile after it
  if (threadIdx.x == 0) {
    mbar_expect_tx(&t.bar[0], 3 * TILE2 * sizeof(float));
    tma_load_3d(t.coef, &cmap, x0, y0, 0, &t.bar[0]);
  }
  grid_dep_trigger();
  float* outbase = states + (size_t)(1 - buf_in) * map_lanes * p.Hp * p.Wp;
  bool ok = mbar_wait(&t.bar[0], 0);
  if (!ok) {
    if (threadIdx.x == 0) set_status(status, PXA_ERR_TIMEOUT);
    // let the copy issued above land (bounded again) before the block can leave
    (void)mbar_wait(&t.bar[0], 0);
    return;
  }
  // per-point stencil coefficients: (A x)_c = cE x_e + cW x_w + cN x_n + cS x_s + cC x_c
  const float d = p.nu * p.invh2, cC = -4.0f * d;
  float cE[RG2], cW[RG2], cN[RG2], cS[RG2], fr[RG2];
#pragma unroll
  for (int i = 0; i < RG2; ++i) {
    const int c = (row0 + i) * BX2 + col;
    const float uu = t.coef[c], vv = t.coef[TILE2 + c];
    cE[i] = -uu * p.inv2h + d;
    cW[i] = uu * p.inv2h + d;
    cN[i] = -vv * p.inv2h + d;
    cS[i] = vv * p.inv2h + d;
    fr[i] = t.coef[2 * TILE2 + c];
  }
  grid_dep_wait();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&t.bar[1], TILE2 * sizeof(float));
    tma_load_3d(t.q[0], &qmap, x0, y0, buf_in * map_lanes + l_begin, &t.bar[1]);
  }
  const float dt = p.dt, hdt = 0.5f * p.dt, sdt = p.dt / 6.0f;
  float* Y0 = t.ya;
  float* Y1 = t.yb;
  // s(t) at the three stage times of lane l's step come from the precomputed table
  // sc[3 step + {0, 1, 2}] (FP64 sin costs thousands of cycles of one warp's FP64 pipe)
  for (int l = l_begin; l < l_end; ++l) {
    const int li = l - l_begin;
    if (threadIdx.x == 0 && l + 1 < l_end) {  // prefetch the next lane's tile
      // order the generic-proxy reads of this buffer (previous lane) before the TMA write
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&t.bar[1 + ((li + 1) & 1)], TILE2 * sizeof(float));
      tma_load_3d(t.q[0] + ((li + 1) & 1) * TILE2, &qmap, x0, y0, buf_in * map_lanes + l + 1, &t.bar[1 + ((li + 1) & 1)]);
    }
    ok = mbar_wait(&t.bar[1 + (li & 1)], (li >> 1) & 1);
    if (!ok) {
      if (threadIdx.x == 0) set_status(status, PXA_ERR_TIMEOUT);
      // this lane's copy and the next lane's prefetch may still be in flight: let them
      // land (bounded again) before the block can leave
      (void)mbar_wait(&t.bar[1 + (li & 1)], (li >> 1) & 1);
      if (l + 1 < l_end) (void)mbar_wait(&t.bar[1 + ((li + 1) & 1)], ((li + 1) >> 1) & 1);
      return;
    }
    const float* Q = t.q[0] + (li & 1) * TILE2;
    const float* scl = sc + 3 * ((int64_t)l * lane_k + s_local);
    const float c1 = __ldg(scl), c2 = __ldg(scl + 1), c4 = __ldg(scl + 2);
    float qv[RG2], acc[RG2], yv[RG2];
#pragma unroll
    for (int i = 0; i < RG2; ++i) qv[i] = Q[(row0 + i) * BX2 + col];
    // stage 1 on the halo-3 region (every owned point): neighbours from the q tile
#pragma unroll
    for (int i = 0; i < RG2; ++i) {
      const int c = (row0 + i) * BX2 + col;
      const float xs = i > 0 ? qv[i - 1] : Q[c - BX2];
      const float xn = i + 1 < RG2 ? qv[i + 1] : Q[c + BX2];
      float k = cE[i] * Q[c + 1] + cW[i] * Q[c - 1] + cN[i] * xn + cS[i] * xs + cC * qv[i] + c1 * fr[i];
      acc[i] = k;
      yv[i] = qv[i] + hdt * k;
      if (colact) Y0[c] = yv[i];
    }
    __syncthreads();
    // stages 2 and 3: every owned point is updated (uniform work, no divergence at the
    // barriers); values on the outer rings that read not-yet-valid neighbours are never
    // used, because the valid region shrinks by one ring per stage and stage 4 stores
    // only the interior. Vertical neighbours come from registers, horizontal ones and
    // the strip ends from the previous stage's buffer.
#pragma unroll
    for (int stg = 2; stg <= 3; ++stg) {
      const float* Xp = stg == 2 ? Y0 : Y1;
      float* Xn = stg == 2 ? Y1 : Y0;
      const float a = stg == 2 ? hdt : dt;
      float prev = 0.0f;
#pragma unroll
      for (int i = 0; i < RG2; ++i) {
        const int c = (row0 + i) * BX2 + col;
        const float cur = yv[i];
        const float xs = i > 0 ? prev : Xp[c - BX2];
        const float xn = i + 1 < RG2 ? yv[i + 1] : Xp[c + BX2];
        prev = cur;
        float k = cE[i] * Xp[c + 1] + cW[i] * Xp[c - 1] + cN[i] * xn + cS[i] * xs + cC * cur + c2 * fr[i];
        acc[i] += 2.0f * k;
        yv[i] = qv[i] + a * k;
        if (colact) Xn[c] = yv[i];
      }
      __syncthreads();
    }
    // stage 4 on the interior: q_new = q + dt/6 (k1 + 2 k2 + 2 k3 + k4)
    float* out = outbase + (size_t)l * p.Hp * p.Wp;
    float jl = 0.0f;  // FP32 within the thread and warp, FP64 across warps and steps
    {
      const float* Xp = Y0;
      const bool cin = col >= G2 && col < G2 + TX2;
      const int x = x0 + col - G2;  // domain column (x0 is the halo corner in padded coordinates)
      float prev = 0.0f;
#pragma unroll
      for (int i = 0; i < RG2; ++i) {
        const int row = row0 + i;
        const int c = row * BX2 + col;
        const float cur = yv[i];
        const float xs = i > 0 ? prev : Xp[c - BX2];
        const float xn = i + 1 < RG2 ? yv[i + 1] : Xp[c + BX2];
        prev = cur;
        const int y = y0 + row - G2;
        if (cin && row >= G2 && row < G2 + TY2 && x < p.nx && y < p.ny) {
          float k = cE[i] * Xp[c + 1] + cW[i] * Xp[c - 1] + cN[i] * xn + cS[i] * xs + cC * cur + c4 * fr[i];
          float qn = qv[i] + sdt * (acc[i] + k);
          store_with_ghosts(out, p, x, y, qn);
          if (traj && l == 0) traj[(size_t)traj_row * p.nx * p.ny + (size_t)y * p.nx + x] = qn;
          if (WITH_J) jl = fmaf(qn, qn, jl);
        }
      }
    }
    if (WITH_J) {
      // no FP64 here (GB300 completes about one FP64 warp instruction per 19 cycles per SM,
      // and a block's serial FP64 sum sat at the end of every step): each warp stores its
      // FP32 partial; the reduction after the sweep adds them in double-float and FP64
      static_assert(AD2_J_WARPS * 32 == 256, "one partial per warp of the 256-thread block");
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) jl += __shfl_xor_sync(0xffffffffu, jl, o);
      if ((threadIdx.x & 31) == 0)
        Jpart[((size_t)jrow * gridDim.x + tile) * AD2_J_WARPS + (threadIdx.x >> 5)] = jl;
    }
    __syncthreads();  // all reads of q[li & 1] and the stage buffers done before reuse
  }
}

// One reverse step of the exact discrete adjoint of the RK4 map for a group of lanes:
// lambda_s = M^T lambda_{s+1} (+ (2dt/T) e_s when with_source and s_local > 0), and
// G += sum of the stage terms s_i kbar_i (the forcing gradient, a double-float accumulator).
// Lane l is at absolute step l * lane_k + s_local (its time lane_base + ...).
__global__ void __launch_bounds__(256) ad2_rk4T_kernel(const __grid_constant__ CUtensorMap qmap,
                                                       const __grid_constant__ CUtensorMap cmap,
                                                       Ad2Params p, float* __restrict__ states,
                                                       int lanes, int map_lanes, int lanes_per_cta,
                                                       int buf_in, int64_t lane_k, int64_t lane_off,
                                                       int64_t s_local, int with_source,
                                                       const float* __restrict__ traj,
                                                       double src_scale, float2* __restrict__ G,
                                                       const float* __restrict__ sc, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem t = carve(smem_raw);
  const int tile = blockIdx.x;
  const int tbx = tile % p.tiles_x, tby = tile / p.tiles_x;
  const int x0 = tbx * TX2, y0 = tby * TY2;
  const int l_begin = blockIdx.y * lanes_per_cta;
  const int l_end = min(lanes, l_begin + lanes_per_cta);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&t.bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&t.bar[0], 3 * TILE2 * sizeof(float));
    tma_load_3d(t.coef, &cmap, x0, y0, 0, &t.bar[0]);
    mbar_expect_tx(&t.bar[1], TILE2 * sizeof(float));
    tma_load_3d(t.q[0], &qmap, x0, y0, buf_in * map_lanes + l_begin, &t.bar[1]);
  }
  const float* u = t.coef;
  const float* v = t.coef + TILE2;
  float* outbase = states + (size_t)(1 - buf_in) * map_lanes * p.Hp * p.Wp;
  bool ok = mbar_wait(&t.bar[0], 0);
  const float dt = p.dt;
  float* ma = t.ya;
  float* mb = t.yb;
  float* Ln = t.acc;
  for (int l = l_begin; l < l_end; ++l) {
    const int li = l - l_begin;
    if (threadIdx.x == 0 && l + 1 < l_end) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&t.bar[1 + ((li + 1) & 1)], TILE2 * sizeof(float));
      tma_load_3d(t.q[0] + ((li + 1) & 1) * TILE2, &qmap, x0, y0, buf_in * map_lanes + l + 1, &t.bar[1 + ((li + 1) & 1)]);
    }
    ok = mbar_wait(&t.bar[1 + (li & 1)], (li >> 1) & 1) && ok;
    if (!ok) {
      if (threadIdx.x == 0) set_status(status, PXA_ERR_TIMEOUT);
      // the coefficient copy, this lane's copy and the next lane's prefetch may still be
      // in flight: let them land (bounded again) before the block can leave
      (void)mbar_wait(&t.bar[0], 0);
      (void)mbar_wait(&t.bar[1 + (li & 1)], (li >> 1) & 1);
      if (l + 1 < l_end) (void)mbar_wait(&t.bar[1 + ((li + 1) & 1)], ((li + 1) >> 1) & 1);
      return;
    }
    const float* L = t.q[0] + (li & 1) * TILE2;
    const int64_t s_abs = lane_off + (int64_t)l * lane_k + s_local;
    // the source and gradient values of this thread's interior points, loaded now so
    // that their global-memory latency passes during the four stencil phases below
    constexpr int NQ = (TX2 * TY2 + 255) / 256;
    float2* Gl = G + (size_t)l * p.nx * p.ny;
    const float* es = traj ? traj + (size_t)s_abs * p.nx * p.ny : nullptr;
    const bool add_src = with_source && s_local > 0 && es;
    float srcv[NQ];
    float2 gold[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int e = threadIdx.x + q * 256;
      const int x = x0 + e % TX2, y = y0 + e / TX2;
      const bool in = e < TX2 * TY2 && x < p.nx && y < p.ny;
      const size_t gi = in ? (size_t)y * p.nx + x : 0;
      srcv[q] = (in && add_src) ? __ldg(es + gi) : 0.0f;
      gold[q] = in ? Gl[gi] : make_float2(0.0f, 0.0f);
    }
    // s(t) at the step's stage times from the precomputed table
    const float* scl = sc + 3 * s_abs;
    const float c1 = __ldg(scl), c2 = __ldg(scl + 1), c4 = __ldg(scl + 2);
    __syncthreads();
    // kbar4 = dt/6 lambda on the whole halo-4 tile
    for (int e = threadIdx.x; e < TILE2; e += blockDim.x) ma[e] = dt / 6.0f * L[e];
    __syncthreads();
    // halo 3: Ybar4 = A^T kbar4; kbar3 = dt/3 lambda + dt Ybar4; Ln = lambda + Ybar4
    for (int e = threadIdx.x; e < (TX2 + 6) * (TY2 + 6); e += blockDim.x) {
      int c = (G2 - 3 + e / (TX2 + 6)) * BX2 + (G2 - 3 + e % (TX2 + 6));
      float nv = AT_at(p, ma, u, v, c);
      mb[c] = dt / 3.0f * L[c] + dt * nv;
      Ln[c] = L[c] + nv;
    }
    __syncthreads();
    // the gradient terms in FP32 per step, kept in registers per interior point below;
    // halo 2: Ybar3 = A^T kbar3; kbar2 = dt/3 lambda + dt/2 Ybar3
    // (kbar4 is still in ma on the interior: read it before ma is overwritten)
    float g4[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      int e = threadIdx.x + q * 256;
      int c = (G2 + e / TX2) * BX2 + (G2 + e % TX2);
      g4[q] = c4 * ma[c] + c2 * mb[c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (TX2 + 4) * (TY2 + 4); e += blockDim.x) {
      int c = (G2 - 2 + e / (TX2 + 4)) * BX2 + (G2 - 2 + e % (TX2 + 4));
      float nv = AT_at(p, mb, u, v, c);
      Ln[c] += nv;
      ma[c] = dt / 3.0f * L[c] + 0.5f * dt * nv;
    }
    __syncthreads();
    // halo 1: Ybar2 = A^T kbar2; kbar1 = dt/6 lambda + dt/2 Ybar2
    for (int e = threadIdx.x; e < (TX2 + 2) * (TY2 + 2); e += blockDim.x) {
      int c = (G2 - 1 + e / (TX2 + 2)) * BX2 + (G2 - 1 + e % (TX2 + 2));
      float nv = AT_at(p, ma, u, v, c);
      Ln[c] += nv;
      mb[c] = dt / 6.0f * L[c] + 0.5f * dt * nv;
    }
    __syncthreads();
    // interior: Ybar1 = A^T kbar1; lambda_s = Ln + Ybar1 (+ source); gradient terms
    float* out = outbase + (size_t)l * p.Hp * p.Wp;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      int e = threadIdx.x + q * 256;
      const int xx = e % TX2, yy = e / TX2;
      const int c = (G2 + yy) * BX2 + (G2 + xx);
      const int x = x0 + xx, y = y0 + yy;
      if (e >= TX2 * TY2 || x >= p.nx || y >= p.ny) continue;
      float nv = AT_at(p, mb, u, v, c);
      float lam = Ln[c] + nv;
      const size_t gi = (size_t)y * p.nx + x;
      if (add_src) lam += (float)src_scale * srcv[q];
      store_with_ghosts(out, p, x, y, lam);
      float gstep = g4[q] + c2 * ma[c] + c1 * mb[c];
      Gl[gi] = df_add(gold[q], gstep);
    }
    __syncthreads();
  }
}

// One reverse step of the exact discrete adjoint of the RK4 map for one lane (the serial
// adjoint and the stepper chain), in the register layout of ad2_rk4_kernel: thread
// (tx, ty) owns tile column tx + 1 and RG2 rows of the halo-3 region, keeps dt times the
// coefficients of A^T at its points in registers, takes vertical neighbours from its own
// registers and horizontal ones (and the strip ends) from the previous stage's tile in
// shared memory. With Z = A^T and lambda the incoming value (step s + 1):
//   kbar4 = dt/6 lambda, kbar3 = dt/3 lambda + dt Z kbar4, kbar2 = dt/3 lambda + dt/2 Z kbar3,
//   kbar1 = dt/6 lambda + dt/2 Z kbar2,
//   lambda_s = lambda + Z (kbar4 + kbar3 + kbar2 + kbar1) (+ src_scale e_s when add_src),
//   G += c4 kbar4 + c2 (kbar3 + kbar2) + c1 kbar1 (c1, c2, c4 = s(t) at the stage times of
// step s, from the table sc), G a double-float (hi, lo) FP32 pair per point (df_add).
// Z kbar4 = dt/6 Z lambda is formed from the lambda tile itself.
__global__ void __launch_bounds__(256, 2) ad2_rk4T1_kernel(const __grid_constant__ CUtensorMap qmap,
                                                           const __grid_constant__ CUtensorMap cmap,
                                                           Ad2Params p, float* __restrict__ states, int buf_in,
                                                           int64_t s_abs, int add_src,
                                                           const float* __restrict__ traj, float src_scale,
                                                           float2* __restrict__ G, const float* __restrict__ sc,
                                                           int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem t = carve(smem_raw);
  const int tile = blockIdx.x;
  const int tbx = tile % p.tiles_x, tby = tile / p.tiles_x;
  const int x0 = tbx * TX2, y0 = tby * TY2;  // padded coordinates of the halo corner
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int col = tx + 1;
  const bool colact = col <= BX2 - 2;
  const int row0 = 1 + ty * RG2;
  if (threadIdx.x == 0) {
    mbar_init(&t.bar[0], 1);
    mbar_init(&t.bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // before the wait for the previous step: the coefficient tile, the source rows of the
  // direct trajectory and the step's forcing factors (all written before the sweep)
  if (threadIdx.x == 0) {
    mbar_expect_tx(&t.bar[0], 3 * TILE2 * sizeof(float));
    tma_load_3d(t.coef, &cmap, x0, y0, 0, &t.bar[0]);
  }
  grid_dep_trigger();
  const bool cin = col >= G2 && col < G2 + TX2;
  const int x = x0 + col - G2;  // domain column
  const size_t N = (size_t)p.nx * p.ny;
  const float* es = (add_src && traj) ? traj + (size_t)s_abs * N : nullptr;
  float srcv[RG2];
#pragma unroll
  for (int i = 0; i < RG2; ++i) {
    const int row = row0 + i, y = y0 + row - G2;
    const bool in = cin && row >= G2 && row < G2 + TY2 && x < p.nx && y < p.ny;
    srcv[i] = (in && es) ? __ldg(es + (size_t)y * p.nx + x) : 0.0f;
  }
  const float c1 = __ldg(sc + 3 * s_abs), c2 = __ldg(sc + 3 * s_abs + 1), c4 = __ldg(sc + 3 * s_abs + 2);
  if (!mbar_wait(&t.bar[0], 0)) {
    if (threadIdx.x == 0) set_status(status, PXA_ERR_TIMEOUT);
    (void)mbar_wait(&t.bar[0], 0);
    return;
  }
  const float* u = t.coef;
  const float* v = t.coef + TILE2;
  const float d = p.nu * p.invh2, dt = p.dt, tc = -4.0f * d;
  float tw[RG2], te[RG2], ts[RG2], tn[RG2];
#pragma unroll
  for (int i = 0; i < RG2; ++i) {
    const int c = (row0 + i) * BX2 + col;
    tw[i] = -u[c - 1] * p.inv2h + d;
    te[i] = u[c + 1] * p.inv2h + d;
    ts[i] = -v[c - BX2] * p.inv2h + d;
    tn[i] = v[c + BX2] * p.inv2h + d;
  }
  // after it: the lambda tile and the gradient values the previous step wrote
  grid_dep_wait();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&t.bar[1], TILE2 * sizeof(float));
    tma_load_3d(t.q[0], &qmap, x0, y0, buf_in, &t.bar[1]);
  }
  float2 gold[RG2];
#pragma unroll
  for (int i = 0; i < RG2; ++i) {
    const int row = row0 + i, y = y0 + row - G2;
    const bool in = cin && row >= G2 && row < G2 + TY2 && x < p.nx && y < p.ny;
    gold[i] = in ? G[(size_t)y * p.nx + x] : make_float2(0.0f, 0.0f);
  }
  if (!mbar_wait(&t.bar[1], 0)) {
    if (threadIdx.x == 0) set_status(status, PXA_ERR_TIMEOUT);
    (void)mbar_wait(&t.bar[1], 0);
    return;
  }
  const float* L = t.q[0];
  float lam[RG2], ln[RG2], kb[RG2], g[RG2];
#pragma unroll
  for (int i = 0; i < RG2; ++i) lam[i] = L[(row0 + i) * BX2 + col];
  // stage 1 (halo 3): Z kbar4 = dt/6 Z lambda
  {
#pragma unroll
    for (int i = 0; i < RG2; ++i) {
      const int c = (row0 + i) * BX2 + col;
      const float xs = i > 0 ? lam[i - 1] : L[c - BX2];
      const float xn = i + 1 < RG2 ? lam[i + 1] : L[c + BX2];
      const float z = tw[i] * L[c - 1] + te[i] * L[c + 1] + ts[i] * xs + tn[i] * xn + tc * lam[i];
      const float nv = (dt / 6.0f) * z;
      kb[i] = (dt / 3.0f) * lam[i] + dt * nv;  // kbar3
      ln[i] = lam[i] + nv;
      g[i] = c4 * ((dt / 6.0f) * lam[i]) + c2 * kb[i];
      if (colact) t.ya[c] = kb[i];
    }
    __syncthreads();
  }
  // stages 2 and 3: Z kbar3 -> kbar2 (halo 2), Z kbar2 -> kbar1 (halo 1)
#pragma unroll
  for (int stg = 2; stg <= 3; ++stg) {
    const float* Xp = stg == 2 ? t.ya : t.yb;
    float* Xn = stg == 2 ? t.yb : t.ya;
    const float wl = stg == 2 ? dt / 3.0f : dt / 6.0f;
    const float cg = stg == 2 ? c2 : c1;
    float nk[RG2];
#pragma unroll
    for (int i = 0; i < RG2; ++i) {
      const int c = (row0 + i) * BX2 + col;
      const float xs = i > 0 ? kb[i - 1] : Xp[c - BX2];
      const float xn = i + 1 < RG2 ? kb[i + 1] : Xp[c + BX2];
      const float nv = tw[i] * Xp[c - 1] + te[i] * Xp[c + 1] + ts[i] * xs + tn[i] * xn + tc * kb[i];
      ln[i] += nv;
      nk[i] = wl * lam[i] + (0.5f * dt) * nv;
      g[i] += cg * nk[i];
      if (colact) Xn[c] = nk[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RG2; ++i) kb[i] = nk[i];
  }
  // stage 4 on the interior: lambda_s = ln + Z kbar1 (+ source); the gradient terms leave
  float* out = states + (size_t)(1 - buf_in) * p.Hp * p.Wp;
  const float* Xp = t.ya;
#pragma unroll
  for (int i = 0; i < RG2; ++i) {
    const int row = row0 + i;
    const int c = row * BX2 + col;
    const int y = y0 + row - G2;
    if (!(cin && row >= G2 && row < G2 + TY2 && x < p.nx && y < p.ny)) continue;
    const float xs = i > 0 ? kb[i - 1] : Xp[c - BX2];
    const float xn = i + 1 < RG2 ? kb[i + 1] : Xp[c + BX2];
    const float nv = tw[i] * Xp[c - 1] + te[i] * Xp[c + 1] + ts[i] * xs + tn[i] * xn + tc * kb[i];
    const float lnew = ln[i] + nv + src_scale * srcv[i];
    store_with_ghosts(out, p, x, y, lnew);
    G[(size_t)y * p.nx + x] = df_add(gold[i], g[i]);
  }
}

// ---- the chain's polynomial propagator (PXA_PROP_POLY) ---------------------------------
// The summed homogeneous adjoint problems of one chain segment of kk RK4 steps are carried
// by the power series of the stepper's own propagator, h <- sum_{i<=m} a_i Z^i h' with
// Z = tau A^T, tau = kk dt (Eq. adjHomNormal with R(dt A^T)^kk, R the RK4 amplification
// polynomial), and the segment's forcing gradient is sum_{i<=m} b_i Z^i h' (Eq. paramupdate
// summed over the segment's steps). One launch forms four powers on one tile: from the halo-4 tile of
// v_{i0} (TMA) the powers v_{i0+1}, .., v_{i0+4} on the halo-3, 2, 1 regions and the
// interior, in the register layout of ad2_rk4_kernel (thread (tx, ty): tile column tx + 1
// and RG2 rows; tau times the coefficients of A^T at its points in registers). Interior
// points add their terms: H = (i0 == 0 ? a_0 v_0 : H) + sum_j a_{i0+j} v_{i0+j} (FP32,
// padded with ghosts; skipped when want_h == 0) and G += (i0 == 0 ? b_0 v_0 : 0) + sum_j
// b_{i0+j} v_{i0+j} (FP32 within the launch, a double-float pair across launches, df_add);
// v_{i0+4} goes to the other plane of V (padded with ghosts). ca / cb hold at least i0 + 5
// coefficients, both FP32 (converting FP64 ones in every thread of every launch kept the
// FP64 pipes 12 % busy in this latency-bound kernel).
__global__ void __launch_bounds__(256, 2) ad2_poly_kernel(const __grid_constant__ CUtensorMap vmap,
                                                          const __grid_constant__ CUtensorMap cmap,
                                                          const __grid_constant__ CUtensorMap hmap,
                                                          const __grid_constant__ CUtensorMap wmap, int w_z,
                                                          Ad2Params p, float tau, float* __restrict__ V,
                                                          int buf_in, int i0, const float* __restrict__ ca,
                                                          const float* __restrict__ cb,
                                                          float* __restrict__ H, int want_h,
                                                          float2* __restrict__ G, int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TileSmem t = carve(smem_raw);
  const int tile = blockIdx.x;
  const int tbx = tile % p.tiles_x, tby = tile / p.tiles_x;
  const int x0 = tbx * TX2, y0 = tby * TY2;  // padded coordinates of the halo corner
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int col = tx + 1;                     // tile column
  const bool colact = col <= BX2 - 2;         // inside the halo-3 region [1, BX2-1)
  const int row0 = 1 + ty * RG2;              // first owned row
  if (threadIdx.x == 0) {
    mbar_init(&t.bar[0], 1);
    mbar_init(&t.bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // before the wait for the previous launch: the coefficient tile and this launch's series
  // coefficients (the same for every thread; all written before the chain)
  if (threadIdx.x == 0) {
    mbar_expect_tx(&t.bar[0], 3 * TILE2 * sizeof(float));
    tma_load_3d(t.coef, &cmap, x0, y0, 0, &t.bar[0]);
  }
  grid_dep_trigger();
  float ka[5], kb[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    ka[j] = __ldg(ca + i0 + j);
    kb[j] = __ldg(cb + i0 + j);
  }
  if (!mbar_wait(&t.bar[0], 0)) {
    if (threadIdx.x == 0) set_status(status, PXA_ERR_TIMEOUT);
    (void)mbar_wait(&t.bar[0], 0);
    return;
  }
  const float* u = t.coef;
  const float* v = t.coef + TILE2;
  // tau (A^T x)_c = tw x_w + te x_e + ts x_s + tn x_n + tc x_c: the west neighbour's row of
  // A holds c as its east entry (-u_w/(2h) + nu/h^2), and so on
  const float d = p.nu * p.invh2, dt = tau, tc = -4.0f * d * dt;
  float tw[RG2], te[RG2], ts[RG2], tn[RG2];
#pragma unroll
  for (int i = 0; i < RG2; ++i) {
    const int c = (row0 + i) * BX2 + col;
    tw[i] = dt * (-u[c - 1] * p.inv2h + d);
    te[i] = dt * (u[c + 1] * p.inv2h + d);
    ts[i] = dt * (-v[c - BX2] * p.inv2h + d);
    tn[i] = dt * (v[c + BX2] * p.inv2h + d);
  }
  // after the wait: the power tile (for a segment's first launch v_0 = h + w: the carried
  // value's tile and the lane value's, added below), and this thread's interior H and G
  // values (loaded now, so that their latency passes during the first three powers)
  grid_dep_wait();
  const bool first = i0 == 0;
  const bool with_w = first && w_z >= 0;
  if (threadIdx.x == 0) {
    mbar_expect_tx(&t.bar[1], (with_w ? 2 : 1) * TILE2 * sizeof(float));
    if (first) {
      tma_load_3d(t.q[0], &hmap, x0, y0, 0, &t.bar[1]);
      if (with_w) tma_load_3d(t.q[1], &wmap, x0, y0, w_z, &t.bar[1]);
    } else {
      tma_load_3d(t.q[0], &vmap, x0, y0, buf_in, &t.bar[1]);
    }
  }
  const bool cin = col >= G2 && col < G2 + TX2;
  const int x = x0 + col - G2;  // domain column
  float hold[RG2];
  float2 gold[RG2];
#pragma unroll
  for (int i = 0; i < RG2; ++i) {
    const int row = row0 + i, y = y0 + row - G2;
    const bool in = cin && row >= G2 && row < G2 + TY2 && x < p.nx && y < p.ny;
    hold[i] = (in && want_h && !first) ? H[(size_t)(y + G2) * p.Wp + (x + G2)] : 0.0f;
    gold[i] = in ? G[(size_t)y * p.nx + x] : make_float2(0.0f, 0.0f);
  }
  if (!mbar_wait(&t.bar[1], 0)) {
    if (threadIdx.x == 0) set_status(status, PXA_ERR_TIMEOUT);
    (void)mbar_wait(&t.bar[1], 0);
    return;
  }
  if (with_w) {
    for (int e = threadIdx.x; e < TILE2; e += blockDim.x) t.q[0][e] += t.q[1][e];
    __syncthreads();
  }
  const float* Xp = t.q[0];
  float xv[RG2], hacc[RG2], gacc[RG2];
#pragma unroll
  for (int i = 0; i < RG2; ++i) {
    xv[i] = Xp[(row0 + i) * BX2 + col];
    hacc[i] = first ? ka[0] * xv[i] : 0.0f;
    gacc[i] = first ? kb[0] * xv[i] : 0.0f;
  }
  // powers 1, 2, 3 on every owned point (the valid region shrinks by one ring per power;
  // ring values that read not-yet-valid neighbours never reach the interior); vertical
  // neighbours from registers, horizontal ones and the strip ends from the previous power
  float* Yn = t.ya;
#pragma unroll
  for (int j = 1; j <= 3; ++j) {
    float yv[RG2];
#pragma unroll
    for (int i = 0; i < RG2; ++i) {
      const int c = (row0 + i) * BX2 + col;
      const float xs = i > 0 ? xv[i - 1] : Xp[c - BX2];
      const float xn = i + 1 < RG2 ? xv[i + 1] : Xp[c + BX2];
      const float y = tw[i] * Xp[c - 1] + te[i] * Xp[c + 1] + ts[i] * xs + tn[i] * xn + tc * xv[i];
      yv[i] = y;
      if (colact) Yn[c] = y;
      hacc[i] = fmaf(ka[j], y, hacc[i]);
      gacc[i] = fmaf(kb[j], y, gacc[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RG2; ++i) xv[i] = yv[i];
    Xp = Yn;
    Yn = Yn == t.ya ? t.yb : t.ya;
  }
  // power 4 on the interior; the interior's terms leave the tile
  float* Vout = V + (size_t)(1 - buf_in) * p.Hp * p.Wp;
#pragma unroll
  for (int i = 0; i < RG2; ++i) {
    const int row = row0 + i;
    const int c = row * BX2 + col;
    const int y = y0 + row - G2;
    if (!(cin && row >= G2 && row < G2 + TY2 && x < p.nx && y < p.ny)) continue;
    const float xs = i > 0 ? xv[i - 1] : Xp[c - BX2];
    const float xn = i + 1 < RG2 ? xv[i + 1] : Xp[c + BX2];
    const float y4 = tw[i] * Xp[c - 1] + te[i] * Xp[c + 1] + ts[i] * xs + tn[i] * xn + tc * xv[i];
    store_with_ghosts(Vout, p, x, y, y4);
    if (want_h) store_with_ghosts(H, p, x, y, fmaf(ka[4], y4, hacc[i]) + hold[i]);
    G[(size_t)y * p.nx + x] = df_add(gold[i], fmaf(kb[4], y4, gacc[i]));
  }
}

// b[s][i], i = 0..m, of chain segment s (steps s kk .. s kk + kk - 1):
// sum_j s(t_j) Q[0][j][i] + s(t_j + dt/2) Q[1][j][i] + s(t_j + dt) Q[2][j][i], t_j =
// (s kk + j) dt, Q = [3][kk][m+1] (FP64; s(t) = sin(omega t), 1 when omega == 0). One block
// per segment, one thread per coefficient (m < blockDim.x).
__global__ void ad2_poly_forcing_kernel(int kk, int m, double dt, double omega, const double* __restrict__ Q,
                                        float* __restrict__ b) {
  __shared__ double sv[3][128];
  const int s = blockIdx.x, i = threadIdx.x;
  double acc = 0.0;
  for (int j0 = 0; j0 < kk; j0 += 128) {
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * 128; e += blockDim.x) {
      const int jj = e / 3, w = e % 3, j = j0 + jj;
      const double tj = ((double)s * kk + j) * dt + (w == 0 ? 0.0 : (w == 1 ? 0.5 * dt : dt));
      sv[w][jj] = j < kk ? forcing_s(omega, tj) : 0.0;
    }
    __syncthreads();
    if (i <= m)
      for (int jj = 0; jj < 128 && j0 + jj < kk; ++jj) {
        const size_t j = (size_t)(j0 + jj);
        acc += sv[0][jj] * Q[(0 * (size_t)kk + j) * (m + 1) + i] + sv[1][jj] * Q[(1 * (size_t)kk + j) * (m + 1) + i] +
               sv[2][jj] * Q[(2 * (size_t)kk + j) * (m + 1) + i];
      }
  }
  if (i <= m) b[(size_t)s * (m + 1) + i] = (float)acc;
}

// Pack u, v (FP64, [ny][nx]) and the forcing f - f_true into the padded FP32
// coefficient array [3][Hp][Wp] with periodic ghosts.
__global__ void ad2_pack_coef_kernel(Ad2Params p, const double* __restrict__ u,
                                     const double* __restrict__ v, const double* __restrict__ f,
                                     const double* __restrict__ ft, float* __restrict__ coef) {
  const size_t plane = (size_t)p.Hp * p.Wp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.nx * p.ny; i += gridDim.x * blockDim.x) {
    int x = i % p.nx, y = i / p.nx;
    store_with_ghosts(coef, p, x, y, (float)u[i]);
    store_with_ghosts(coef + plane, p, x, y, (float)v[i]);
    store_with_ghosts(coef + 2 * plane, p, x, y, (float)(f[i] - (ft ? ft[i] : 0.0)));
  }
}

// The coefficients of A^T at every padded point (periodic indices): (A^T x)_c =
// tE x_E + tW x_W + tN x_N + tS x_S - 4 d x_c with tE = d + a u_E, tW = d - a u_W,
// tN = d + a v_N, tS = d - a v_S (a = 1/(2h), d = nu/h^2): the neighbour's entry of A in
// the column of c. tc = [4][Hp][Wp] FP32 (tE, tW, tN, tS).
__global__ void ad2_pack_coefT_kernel(Ad2Params p, const double* __restrict__ u,
                                      const double* __restrict__ v, float* __restrict__ tc) {
  const size_t plane = (size_t)p.Hp * p.Wp;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= plane) return;
  const int X = (int)(i % p.Wp), Y = (int)(i / p.Wp);
  const int x = ((X - G2) % p.nx + p.nx) % p.nx, y = ((Y - G2) % p.ny + p.ny) % p.ny;
  const int xe = (x + 1) % p.nx, xw = (x + p.nx - 1) % p.nx;
  const int yn = (y + 1) % p.ny, ys = (y + p.ny - 1) % p.ny;
  const float a = p.inv2h, d = p.nu * p.invh2;
  tc[i] = (float)u[(size_t)y * p.nx + xe] * a + d;
  tc[plane + i] = -(float)u[(size_t)y * p.nx + xw] * a + d;
  tc[2 * plane + i] = (float)v[(size_t)yn * p.nx + x] * a + d;
  tc[3 * plane + i] = -(float)v[(size_t)ys * p.nx + x] * a + d;
}

// Fill lanes' padded states: zero (src == nullptr), or scale * row(row0 + l*row_step)
// of the FP32 trajectory (the adjoint's terminal source of each lane), or, when `add`
// is set, state += padded vector `addv` (FP32 padded, per call one lane).
// Lane l (blockIdx.y, strided) gets scale * traj row (row0 + l row_step), ghosts included,
// or zero. FP32 product and 32-bit indices: an FP64 product with its two conversions per
// point (three FP64-pipe instructions) and 64-bit divisions made this 16.8 M-point fill
// take ~0.1 ms at C3's size.
__global__ void ad2_fill_kernel(Ad2Params p, float* __restrict__ states, int lanes,
                                const float* __restrict__ traj, int64_t row0, int64_t row_step,
                                float scale) {
  const size_t plane = (size_t)p.Hp * p.Wp;
  const int N = p.nx * p.ny;
  for (int l = blockIdx.y; l < lanes; l += gridDim.y) {
    float* st = states + (size_t)l * plane;
    const float* src = traj ? traj + (size_t)(row0 + (int64_t)l * row_step) * N : nullptr;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
      const int y = r / p.nx, x = r - y * p.nx;
      store_with_ghosts(st, p, x, y, src ? scale * src[r] : 0.0f);
    }
  }
}

// dst (padded, one lane) += src (padded, one lane), ghosts included.
__global__ void ad2_add_padded_kernel(size_t count, float* __restrict__ dst, const float* __restrict__ src) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    dst[i] += src[i];
}

// First pass of the objective's sum: block b adds the FP32 partials part[b chunk,
// (b + 1) chunk) as a double-float pair (FP32 two-sums, exact to about 2^-44 of the terms)
// and then across the block in FP64 into out[b]. Spread over the SMs because one SM
// completes only about one FP64 warp instruction per 19 cycles on GB300.
__global__ void ad2_reduce_J_part_kernel(const float* __restrict__ part, size_t count, size_t chunk,
                                         double* __restrict__ out) {
  extern __shared__ double red[];
  const size_t b0 = (size_t)blockIdx.x * chunk, b1 = min(count, b0 + chunk);
  float2 acc = make_float2(0.0f, 0.0f);
  for (size_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) acc = df_add(acc, part[i]);
  const double s = block_sum((double)acc.x + (double)acc.y, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// Second pass: J = scale * the sum of the block sums (one block).
__global__ void ad2_reduce_J_kernel(const double* __restrict__ part, size_t count, double scale, double* J,
                                    int* status) {
  extern __shared__ double red[];
  double s = 0.0;
  for (size_t i = threadIdx.x; i < count; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    *J = scale * s;
    if (!isfinite(*J)) set_status(status, PXA_ERR_NONFINITE);
  }
}

// grad = sum over lanes of G[l] (double-float) and Gf[l] (FP32) (+ extra), read out in
// FP64. The terms are added as a double-float (hi, lo) pair by FP32 two-sums, which keeps
// the sum within about 2^-40 of its terms' magnitude (far below the FP32 rounding of the
// terms themselves) without one FP64 add per term and point: 17 M of them at C3's size
// cost ~30 us of the FP64 pipes.
__global__ void ad2_sum_grad_kernel(size_t N, int lanes, const float2* __restrict__ G, int flanes,
                                    const float* __restrict__ Gf, const float2* __restrict__ extra,
                                    double* __restrict__ grad, int* status) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    float2 acc = make_float2(0.0f, 0.0f);
    for (int l = 0; l < lanes; ++l) {
      const float2 v = G[(size_t)l * N + i];
      acc = df_add(df_add(acc, v.x), v.y);
    }
    for (int l = 0; l < flanes; ++l) acc = df_add(acc, Gf[(size_t)l * N + i]);
    double r = (double)acc.x + (double)acc.y;
    if (extra) r += (double)extra[i].x + (double)extra[i].y;
    grad[i] = r;
    if (!isfinite(r)) set_status(status, PXA_ERR_NONFINITE);
  }
}

// ---- host side ----------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3D tiled map over `depth` padded planes [Hp][Wp] of FP32 with box (BX2, BY2, box_depth).
bool ad2_make_map(CUtensorMap* map, float* base, const Ad2Params& p, int depth, int box_depth) {
  return ad2_make_map_box(map, base, p, depth, BX2, BY2, box_depth);
}

bool ad2_make_map_box(CUtensorMap* map, float* base, const Ad2Params& p, int depth, int box_x,
                      int box_y, int box_depth) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)p.Wp, (cuuint64_t)p.Hp, (cuuint64_t)depth};
  cuuint64_t strides[2] = {(cuuint64_t)p.Wp * sizeof(float), (cuuint64_t)p.Wp * p.Hp * sizeof(float)};
  cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_depth};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool ad2_make_map_plain(CUtensorMap* map, void* base, int elem_bytes, int nx, int ny, int depth, int box_x,
                        int box_y) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (elem_bytes != 4 && elem_bytes != 8)) return false;
  cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)depth};
  cuuint64_t strides[2] = {(cuuint64_t)nx * elem_bytes, (cuuint64_t)nx * ny * elem_bytes};
  cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                  base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Launch with or without the programmatic-serialization attribute (the kernel may then
// start while the previous kernel in the stream finishes; see grid_dep_wait).
template <typename... KArgs, typename... Args>
static cudaError_t launch_ex(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                             Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fn, std::forward<Args>(args)...);
}

static cudaError_t set_smem(const void* fn) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ad2_smem_bytes());
}

cudaError_t launch_ad2_rk4(cudaStream_t st, const CUtensorMap& qmap, const CUtensorMap& cmap,
                           const Ad2Params& p, float* states, int lanes, int map_lanes,
                           int lanes_per_cta, int buf_in, int64_t lane_k, int64_t s_local, const float* sc,
                           float* traj, int64_t traj_row, float* Jpart, int64_t jrow, int* status, int pdl) {
  dim3 grid(p.tiles_x * p.tiles_y, (lanes + lanes_per_cta - 1) / lanes_per_cta);
  if (Jpart) {
    cudaError_t e = set_smem((const void*)ad2_rk4_kernel<true>);
    if (e != cudaSuccess) return e;
    return launch_ex(ad2_rk4_kernel<true>, grid, dim3(256), ad2_smem_bytes(), st, pdl != 0, qmap, cmap, p, states,
                     lanes, map_lanes, lanes_per_cta, buf_in, lane_k, s_local, sc, traj, traj_row, Jpart, jrow,
                     status);
  }
  cudaError_t e = set_smem((const void*)ad2_rk4_kernel<false>);
  if (e != cudaSuccess) return e;
  return launch_ex(ad2_rk4_kernel<false>, grid, dim3(256), ad2_smem_bytes(), st, pdl != 0, qmap, cmap, p, states,
                   lanes, map_lanes, lanes_per_cta, buf_in, lane_k, s_local, sc, traj, traj_row, Jpart, jrow,
                   status);
}

cudaError_t launch_ad2_rk4T(cudaStream_t st, const CUtensorMap& qmap, const CUtensorMap& cmap,
                            const Ad2Params& p, float* states, int lanes, int map_lanes,
                            int lanes_per_cta, int buf_in, int64_t lane_k, int64_t lane_off, int64_t s_local,
                            int with_source, const float* traj, double src_scale, float2* G,
                            const float* sc, int* status, int pdl) {
  if (lanes == 1 && map_lanes == 1) {
    // one lane: the register-layout step
    cudaError_t e = set_smem((const void*)ad2_rk4T1_kernel);
    if (e != cudaSuccess) return e;
    const int64_t s_abs = lane_off + s_local;
    return launch_ex(ad2_rk4T1_kernel, dim3(p.tiles_x * p.tiles_y), dim3(256), ad2_smem_bytes(), st, pdl != 0,
                     qmap, cmap, p, states, buf_in, s_abs, (with_source && s_local > 0 && traj) ? 1 : 0, traj,
                     (float)src_scale, G, sc, status);
  }
  cudaError_t e = set_smem((const void*)ad2_rk4T_kernel);
  if (e != cudaSuccess) return e;
  dim3 grid(p.tiles_x * p.tiles_y, (lanes + lanes_per_cta - 1) / lanes_per_cta);
  ad2_rk4T_kernel<<<grid, 256, ad2_smem_bytes(), st>>>(qmap, cmap, p, states, lanes, map_lanes,
                                                       lanes_per_cta, buf_in, lane_k, lane_off, s_local,
                                                       with_source, traj, src_scale, G, sc, status);
  return cudaGetLastError();
}

cudaError_t launch_ad2_poly(cudaStream_t st, const CUtensorMap& vmap, const CUtensorMap& cmap, const CUtensorMap& hmap,
                            const CUtensorMap& wmap, int w_z, const Ad2Params& p, float tau, float* V, int buf_in,
                            int i0, const float* ca, const float* cb, float* H, int want_h, float2* G, int* status,
                            int pdl) {
  cudaError_t e = set_smem((const void*)ad2_poly_kernel);
  if (e != cudaSuccess) return e;
  return launch_ex(ad2_poly_kernel, dim3(p.tiles_x * p.tiles_y), dim3(256), ad2_smem_bytes(), st, pdl != 0, vmap,
                   cmap, hmap, wmap, w_z, p, tau, V, buf_in, i0, ca, cb, H, want_h, G, status);
}

cudaError_t launch_ad2_poly_forcing(cudaStream_t st, int segments, int kk, int m, double dt, double omega,
                                    const double* Q, float* b) {
  if (segments < 1) return cudaSuccess;
  if (m < 0 || m >= 256) return cudaErrorInvalidValue;
  ad2_poly_forcing_kernel<<<segments, 256, 0, st>>>(kk, m, dt, omega, Q, b);
  return cudaGetLastError();
}

cudaError_t launch_ad2_pack_coef(cudaStream_t st, const Ad2Params& p, const double* u,
                                 const double* v, const double* f, const double* ft, float* coef) {
  int threads = 256, blocks = (p.nx * p.ny + threads - 1) / threads;
  ad2_pack_coef_kernel<<<blocks, threads, 0, st>>>(p, u, v, f, ft, coef);
  return cudaGetLastError();
}

cudaError_t launch_ad2_pack_coefT(cudaStream_t st, const Ad2Params& p, const double* u, const double* v,
                                  float* tc) {
  const size_t plane = (size_t)p.Hp * p.Wp;
  ad2_pack_coefT_kernel<<<(unsigned)((plane + 255) / 256), 256, 0, st>>>(p, u, v, tc);
  return cudaGetLastError();
}

cudaError_t launch_ad2_fill(cudaStream_t st, const Ad2Params& p, float* states, int lanes,
                            const float* traj, int64_t row0, int64_t row_step, double scale) {
  if (lanes <= 0) return cudaSuccess;
  const int N = p.nx * p.ny, threads = 256;
  const dim3 grid((unsigned)std::min((N + threads - 1) / threads, 1024), (unsigned)std::min(lanes, 65535));
  ad2_fill_kernel<<<grid, threads, 0, st>>>(p, states, lanes, traj, row0, row_step, (float)scale);
  return cudaGetLastError();
}

cudaError_t launch_ad2_add_padded(cudaStream_t st, size_t count, float* dst, const float* src) {
  int threads = 256;
  int blocks = (int)((count + threads - 1) / threads);
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  ad2_add_padded_kernel<<<blocks, threads, 0, st>>>(count, dst, src);
  return cudaGetLastError();
}

cudaError_t launch_ad2_reduce_J(cudaStream_t st, const float* part, size_t count, double scale, double* scratch,
                                double* J, int* status) {
  size_t chunk = 2048;
  if ((count + chunk - 1) / chunk > (size_t)AD2_REDUCE_J_BLOCKS)
    chunk = (count + AD2_REDUCE_J_BLOCKS - 1) / AD2_REDUCE_J_BLOCKS;
  const size_t nb = count ? (count + chunk - 1) / chunk : 1;
  ad2_reduce_J_part_kernel<<<(unsigned)nb, 256, 40 * sizeof(double), st>>>(part, count, chunk, scratch);
  ad2_reduce_J_kernel<<<1, 1024, 40 * sizeof(double), st>>>(scratch, nb, scale, J, status);
  return cudaGetLastError();
}

cudaError_t launch_ad2_sum_grad(cudaStream_t st, size_t N, int lanes, const float2* G, int flanes, const float* Gf,
                                const float2* extra, double* grad, int* status) {
  int threads = 256;
  int blocks = (int)((N + threads - 1) / threads);
  if (blocks > 4096) blocks = 4096;
  ad2_sum_grad_kernel<<<blocks, threads, 0, st>>>(N, lanes, G, flanes, Gf, extra, grad, status);
  return cudaGetLastError();
}

}  // namespace pxa
