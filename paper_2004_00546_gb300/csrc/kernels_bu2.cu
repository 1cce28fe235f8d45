// kernels_bu2.cu — 2D viscous Burgers (Sec. 4.3): the vector field q = (u, v) on an
// n x n periodic grid, advective central differences
//   N_u = -u u_x - v u_y + nu lap u,   N_v = -u v_x - v v_y + nu lap v,
// classical RK4 in FP32, control = the initial state, J = 0.5 ||q(T) - q_target||^2
// (accumulated in FP64).
//
//   bu2_step_kernel      one RK4 step of the direct problem (Eq. seriesDirect): a thread
//                        block per 16 x 16 tile with a 4-point halo (each stage narrows the
//                        valid region by one point), the stage states in shared memory
//   bu2_adj_step_kernel  one step of the exact discrete adjoint (the transpose of the RK4
//                        step map, the hybrid scheme's adjoint of Sec. 3.3): the stage
//                        states are recomputed from the stored state on a 7-point halo and
//                        the transposed stage Jacobians applied in reverse order
//   bu2_terminal_kernel  J's partial sums and lambda(T) = q(T) - q_target (Eq. adjFinalTime)
// Fields are [2][n][n] (u then v, row = y, x fastest).
#include "common.cuh"
#include "kernels_bu2.cuh"

namespace pxa {

namespace {

constexpr int TS = BU2_TILE;  // interior tile edge (one point per thread)
constexpr int HD = 4;         // halo of one direct step
constexpr int HA = 7;         // halo of the state for one adjoint step
constexpr int HL = 4;         // halo of lambda for one adjoint step
constexpr int WD = TS + 2 * HD;  // 24
constexpr int WA = TS + 2 * HA;  // 30
constexpr int WL = TS + 2 * HL;  // 24

__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

struct Bu2C {
  float i2h, ih2, nu;
};

// N(Y) at (r, c) of a tile of width W (planes Yu, Yv): returns (N_u, N_v)
template <int W>
__device__ __forceinline__ void rhs_tile(const float* Yu, const float* Yv, int r, int c, const Bu2C& k, float& nu_o,
                                         float& nv_o) {
  const int e = r * W + c;
  const float u = Yu[e], v = Yv[e];
  const float ue = Yu[e + 1], uw = Yu[e - 1], un = Yu[e + W], us = Yu[e - W];
  const float ve = Yv[e + 1], vw = Yv[e - 1], vn = Yv[e + W], vs = Yv[e - W];
  nu_o = -u * ((ue - uw) * k.i2h) - v * ((un - us) * k.i2h) + k.nu * ((ue + uw + un + us - 4.0f * u) * k.ih2);
  nv_o = -u * ((ve - vw) * k.i2h) - v * ((vn - vs) * k.i2h) + k.nu * ((ve + vw + vn + vs - 4.0f * v) * k.ih2);
}

// (J(Y)^T Z) at (r, c) (Y on a tile of width WY, Z on a tile of width WZ, the same point
// at offset `off` = (WY - WZ) / 2 in Y's coordinates):
//   o1 = -Y_u,x Z1 + D_x(Y_u Z1) + D_y(Y_v Z1) + nu lap Z1 - Y_v,x Z2,
//   o2 = -Y_u,y Z1 + D_x(Y_u Z2) + D_y(Y_v Z2) + nu lap Z2 - Y_v,y Z2.
template <int WY, int WZ>
__device__ __forceinline__ void jacT_tile(const float* Yu, const float* Yv, const float* Z1, const float* Z2, int r,
                                          int c, const Bu2C& k, float& o1, float& o2) {
  constexpr int off = (WY - WZ) / 2;
  const int ey = (r + off) * WY + (c + off), ez = r * WZ + c;
  const float uE = Yu[ey + 1], uW = Yu[ey - 1], uN = Yu[ey + WY], uS = Yu[ey - WY];
  const float vE = Yv[ey + 1], vW = Yv[ey - 1], vN = Yv[ey + WY], vS = Yv[ey - WY];
  const float z1 = Z1[ez], z1E = Z1[ez + 1], z1W = Z1[ez - 1], z1N = Z1[ez + WZ], z1S = Z1[ez - WZ];
  const float z2 = Z2[ez], z2E = Z2[ez + 1], z2W = Z2[ez - 1], z2N = Z2[ez + WZ], z2S = Z2[ez - WZ];
  const float ux = (uE - uW) * k.i2h, uy = (uN - uS) * k.i2h, vx = (vE - vW) * k.i2h, vy = (vN - vS) * k.i2h;
  o1 = -ux * z1 + (uE * z1E - uW * z1W) * k.i2h + (vN * z1N - vS * z1S) * k.i2h +
       k.nu * ((z1E + z1W + z1N + z1S - 4.0f * z1) * k.ih2) - vx * z2;
  o2 = -uy * z1 + (uE * z2E - uW * z2W) * k.i2h + (vN * z2N - vS * z2S) * k.i2h +
       k.nu * ((z2E + z2W + z2N + z2S - 4.0f * z2) * k.ih2) - vy * z2;
}

// Load plane pairs of a (W x W) tile whose corner is the global point (y0, x0), periodic.
template <int W>
__device__ __forceinline__ void load_tile(const float* __restrict__ q, int n, int y0, int x0, float* Tu, float* Tv) {
  const size_t plane = (size_t)n * n;
  for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
    const int r = e / W, c = e % W;
    const size_t g = (size_t)wrapn(y0 + r, n) * n + wrapn(x0 + c, n);
    Tu[e] = q[g];
    Tv[e] = q[plane + g];
  }
}

}  // namespace

// q_{s+1} = RK4 step of q_s. Grid (n/TS, n/TS), TS*TS threads.
__global__ void __launch_bounds__(BU2_TILE * BU2_TILE) bu2_step_kernel(const float* __restrict__ q,
                                                                       float* __restrict__ qn, int n, Bu2C k,
                                                                       float dt) {
  __shared__ float Qu[WD * WD], Qv[WD * WD], Au[WD * WD], Av[WD * WD], Bu[WD * WD], Bv[WD * WD];
  const int ty = blockIdx.y * TS, tx = blockIdx.x * TS;
  load_tile<WD>(q, n, ty - HD, tx - HD, Qu, Qv);
  __syncthreads();
  const int ir = threadIdx.x / TS + HD, ic = threadIdx.x % TS + HD;  // this thread's interior point
  float accu = 0.f, accv = 0.f, ku, kv;
  const float h2 = 0.5f * dt;
  // stage 1 on [1, WD-1): k1 = N(q), A = q + dt/2 k1
  for (int e = threadIdx.x; e < (WD - 2) * (WD - 2); e += blockDim.x) {
    const int r = e / (WD - 2) + 1, c = e % (WD - 2) + 1;
    rhs_tile<WD>(Qu, Qv, r, c, k, ku, kv);
    Au[r * WD + c] = Qu[r * WD + c] + h2 * ku;
    Av[r * WD + c] = Qv[r * WD + c] + h2 * kv;
  }
  rhs_tile<WD>(Qu, Qv, ir, ic, k, ku, kv);
  accu = ku;
  accv = kv;
  __syncthreads();
  // stage 2 on [2, WD-2): k2 = N(A), B = q + dt/2 k2
  for (int e = threadIdx.x; e < (WD - 4) * (WD - 4); e += blockDim.x) {
    const int r = e / (WD - 4) + 2, c = e % (WD - 4) + 2;
    rhs_tile<WD>(Au, Av, r, c, k, ku, kv);
    Bu[r * WD + c] = Qu[r * WD + c] + h2 * ku;
    Bv[r * WD + c] = Qv[r * WD + c] + h2 * kv;
  }
  rhs_tile<WD>(Au, Av, ir, ic, k, ku, kv);
  accu += 2.f * ku;
  accv += 2.f * kv;
  __syncthreads();
  // stage 3 on [3, WD-3): k3 = N(B), A = q + dt k3
  for (int e = threadIdx.x; e < (WD - 6) * (WD - 6); e += blockDim.x) {
    const int r = e / (WD - 6) + 3, c = e % (WD - 6) + 3;
    rhs_tile<WD>(Bu, Bv, r, c, k, ku, kv);
    Au[r * WD + c] = Qu[r * WD + c] + dt * ku;
    Av[r * WD + c] = Qv[r * WD + c] + dt * kv;
  }
  rhs_tile<WD>(Bu, Bv, ir, ic, k, ku, kv);
  accu += 2.f * ku;
  accv += 2.f * kv;
  __syncthreads();
  // stage 4 on the interior: q_{s+1} = q + dt/6 (k1 + 2 k2 + 2 k3 + k4)
  rhs_tile<WD>(Au, Av, ir, ic, k, ku, kv);
  const size_t g = (size_t)(ty + ir - HD) * n + (tx + ic - HD), plane = (size_t)n * n;
  qn[g] = Qu[ir * WD + ic] + dt / 6.f * (accu + ku);
  qn[plane + g] = Qv[ir * WD + ic] + dt / 6.f * (accv + kv);
}

// lam_out = M_s^T lam for the RK4 step taken at q_s. Grid (n/TS, n/TS), TS*TS threads.
__global__ void __launch_bounds__(BU2_TILE * BU2_TILE) bu2_adj_step_kernel(const float* __restrict__ qs,
                                                                           const float* __restrict__ lam,
                                                                           float* __restrict__ lo, int n, Bu2C k,
                                                                           float dt) {
  extern __shared__ float sm[];
  float* Y1u = sm;  // stage states on the WA x WA tile
  float* Y1v = Y1u + WA * WA;
  float* Y2u = Y1v + WA * WA;
  float* Y2v = Y2u + WA * WA;
  float* Y3u = Y2v + WA * WA;
  float* Y3v = Y3u + WA * WA;
  float* Y4u = Y3v + WA * WA;
  float* Y4v = Y4u + WA * WA;
  float* Lu = Y4v + WA * WA;  // lambda on the WL x WL tile
  float* Lv = Lu + WL * WL;
  float* Mu = Lv + WL * WL;  // kbar of the stage being reversed
  float* Mv = Mu + WL * WL;
  float* Nu = Mv + WL * WL;  // Ybar of the stage just reversed
  float* Nv = Nu + WL * WL;
  const int ty = blockIdx.y * TS, tx = blockIdx.x * TS;
  load_tile<WA>(qs, n, ty - HA, tx - HA, Y1u, Y1v);
  load_tile<WL>(lam, n, ty - HL, tx - HL, Lu, Lv);
  __syncthreads();
  const float h2 = 0.5f * dt;
  float ku, kv;
  // the stage states: Y2 = q + dt/2 N(Y1) on [1, WA-1), Y3 = q + dt/2 N(Y2) on [2, WA-2),
  // Y4 = q + dt N(Y3) on [3, WA-3)
  for (int e = threadIdx.x; e < (WA - 2) * (WA - 2); e += blockDim.x) {
    const int r = e / (WA - 2) + 1, c = e % (WA - 2) + 1;
    rhs_tile<WA>(Y1u, Y1v, r, c, k, ku, kv);
    Y2u[r * WA + c] = Y1u[r * WA + c] + h2 * ku;
    Y2v[r * WA + c] = Y1v[r * WA + c] + h2 * kv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (WA - 4) * (WA - 4); e += blockDim.x) {
    const int r = e / (WA - 4) + 2, c = e % (WA - 4) + 2;
    rhs_tile<WA>(Y2u, Y2v, r, c, k, ku, kv);
    Y3u[r * WA + c] = Y1u[r * WA + c] + h2 * ku;
    Y3v[r * WA + c] = Y1v[r * WA + c] + h2 * kv;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (WA - 6) * (WA - 6); e += blockDim.x) {
    const int r = e / (WA - 6) + 3, c = e % (WA - 6) + 3;
    rhs_tile<WA>(Y3u, Y3v, r, c, k, ku, kv);
    Y4u[r * WA + c] = Y1u[r * WA + c] + dt * ku;
    Y4v[r * WA + c] = Y1v[r * WA + c] + dt * kv;
  }
  // reverse of the four stages (lambda coordinates, WL wide):
  //   kbar4 = dt/6 lam; Ybar4 = J(Y4)^T kbar4            (radius 3)
  //   kbar3 = dt/3 lam + dt Ybar4; Ybar3 = J(Y3)^T kbar3  (radius 2)
  //   kbar2 = dt/3 lam + dt/2 Ybar3; Ybar2 = J(Y2)^T kbar2 (radius 1)
  //   kbar1 = dt/6 lam + dt/2 Ybar2; Ybar1 = J(Y1)^T kbar1 (interior)
  //   lam_out = lam + Ybar4 + Ybar3 + Ybar2 + Ybar1
  for (int e = threadIdx.x; e < WL * WL; e += blockDim.x) {
    Mu[e] = dt / 6.f * Lu[e];
    Mv[e] = dt / 6.f * Lv[e];
  }
  const int ir = threadIdx.x / TS + HL, ic = threadIdx.x % TS + HL;  // interior point (lambda coordinates)
  float ou = Lu[ir * WL + ic], ov = Lv[ir * WL + ic];
  __syncthreads();
  const float* const Ys_u[4] = {Y1u, Y2u, Y3u, Y4u};
  const float* const Ys_v[4] = {Y1v, Y2v, Y3v, Y4v};
  const float bw[4] = {1.f / 6.f, 1.f / 3.f, 1.f / 3.f, 1.f / 6.f};
  const float cw[4] = {0.5f, 0.5f, 1.f, 0.f};  // Y_{q+2} = q + cw[q] dt k_{q+1}
#pragma unroll
  for (int q = 3; q >= 0; --q) {
    const int rad = q;  // Ybar_{q+1} is needed on this radius around the interior
    const int lo_ = HL - rad, w = TS + 2 * rad;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int r = e / w + lo_, c = e % w + lo_;
      float a, bq;
      jacT_tile<WA, WL>(Ys_u[q], Ys_v[q], Mu, Mv, r, c, k, a, bq);
      Nu[r * WL + c] = a;
      Nv[r * WL + c] = bq;
    }
    __syncthreads();
    ou += Nu[ir * WL + ic];
    ov += Nv[ir * WL + ic];
    if (q > 0) {
      // kbar_q of the stage before, on the radius Ybar_q will need it
      const int rad2 = q - 1 + 1, lo2 = HL - rad2, w2 = TS + 2 * rad2;
      for (int e = threadIdx.x; e < w2 * w2; e += blockDim.x) {
        const int r = e / w2 + lo2, c = e % w2 + lo2, ee = r * WL + c;
        Mu[ee] = bw[q - 1] * dt * Lu[ee] + cw[q - 1] * dt * Nu[ee];
        Mv[ee] = bw[q - 1] * dt * Lv[ee] + cw[q - 1] * dt * Nv[ee];
      }
      __syncthreads();
    }
  }
  const size_t g = (size_t)(ty + ir - HL) * n + (tx + ic - HL), plane = (size_t)n * n;
  lo[g] = ou;
  lo[plane + g] = ov;
}

// Per tile: partial of sum (q(T) - target)^2 in FP64 into Jpart[tile]; lamT = q(T) - target.
__global__ void bu2_terminal_kernel(const float* __restrict__ qT, const double* __restrict__ target, int n,
                                    float* __restrict__ lamT, double* __restrict__ Jpart) {
  __shared__ double red[40];
  const size_t plane = (size_t)n * n;
  const int tile = blockIdx.y * gridDim.x + blockIdx.x;
  const int r = blockIdx.y * TS + threadIdx.x / TS, c = blockIdx.x * TS + threadIdx.x % TS;
  const size_t g = (size_t)r * n + c;
  const double du = (double)qT[g] - target[g], dv = (double)qT[plane + g] - target[plane + g];
  lamT[g] = (float)du;
  lamT[plane + g] = (float)dv;
  const double s = block_sum(du * du + dv * dv, red);
  if (threadIdx.x == 0) Jpart[tile] = s;
}

// J = 0.5 sum_tiles Jpart (fixed order, one thread).
__global__ void bu2_sum_kernel(const double* __restrict__ Jpart, int tiles, double* __restrict__ J, int* status) {
  double s = 0.0;
  for (int t = 0; t < tiles; ++t) s += Jpart[t];
  *J = 0.5 * s;
  if (!isfinite(s)) set_status(status, PXA_ERR_NONFINITE);
}

__global__ void bu2_to_f32_kernel(const double* __restrict__ x, float* __restrict__ y, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void bu2_to_f64_kernel(const float* __restrict__ x, double* __restrict__ y, size_t count, int* status) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    y[i] = (double)x[i];
    if (!isfinite(y[i])) set_status(status, PXA_ERR_NONFINITE);
  }
}

static Bu2C bu2c(int n, double L, double nu) {
  const double h = L / n;
  return Bu2C{(float)(1.0 / (2.0 * h)), (float)(1.0 / (h * h)), (float)nu};
}

size_t bu2_adj_smem_bytes() { return sizeof(float) * (8 * (size_t)WA * WA + 6 * (size_t)WL * WL); }

cudaError_t launch_bu2_step(cudaStream_t st, const float* q, float* qn, int n, double L, double nu, double dt) {
  const dim3 grid(n / TS, n / TS);
  bu2_step_kernel<<<grid, TS * TS, 0, st>>>(q, qn, n, bu2c(n, L, nu), (float)dt);
  return cudaGetLastError();
}

cudaError_t launch_bu2_adj_step(cudaStream_t st, const float* qs, const float* lam, float* lo, int n, double L,
                                double nu, double dt) {
  const size_t sh = bu2_adj_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(bu2_adj_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  const dim3 grid(n / TS, n / TS);
  bu2_adj_step_kernel<<<grid, TS * TS, sh, st>>>(qs, lam, lo, n, bu2c(n, L, nu), (float)dt);
  return cudaGetLastError();
}

cudaError_t launch_bu2_terminal(cudaStream_t st, const float* qT, const double* target, int n, float* lamT,
                                double* Jpart, double* J, int* status) {
  const dim3 grid(n / TS, n / TS);
  bu2_terminal_kernel<<<grid, TS * TS, 0, st>>>(qT, target, n, lamT, Jpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bu2_sum_kernel<<<1, 1, 0, st>>>(Jpart, (n / TS) * (n / TS), J, status);
  return cudaGetLastError();
}

cudaError_t launch_bu2_convert(cudaStream_t st, const double* x, float* y, size_t count) {
  bu2_to_f32_kernel<<<(unsigned)std::min<size_t>((count + 255) / 256, 4096), 256, 0, st>>>(x, y, count);
  return cudaGetLastError();
}

cudaError_t launch_bu2_convert_back(cudaStream_t st, const float* x, double* y, size_t count, int* status) {
  bu2_to_f64_kernel<<<(unsigned)std::min<size_t>((count + 255) / 256, 4096), 256, 0, st>>>(x, y, count, status);
  return cudaGetLastError();
}

}  // namespace pxa
