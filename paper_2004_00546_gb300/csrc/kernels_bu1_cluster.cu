// kernels_bu1_cluster.cu — 1D Burgers RK4 direct and exact discrete adjoint on a
// thread-block cluster: one time lane is spread over C CTAs (C SMs), each owning a
// contiguous chunk of the grid.
//
// GB300 has 2 FP64 FMA per clock per SM, so one CTA stepping n = 1024 points is
// bound by a single SM's FP64 rate. Here each CTA steps ~n/C points and the chunks
// exchange halos through distributed shared memory (DSMEM): after a step every CTA
// pushes the boundary values its neighbours need straight into their shared-memory
// halo slots, and one cluster barrier per time step publishes them. The four RK4
// stages need halo 1 each; the halo is widened (4 for the direct step, 7 for the
// adjoint step) and the stages are recomputed redundantly on the overlap, so that a
// whole RK4 step, forward or reversed, needs one exchange. Halo buffers alternate by
// step parity, so a push for step s+1 never lands in a buffer still read in step s.
//
// Paper mapping: Eq. seriesDirect (serial direct), Eq. hybadjinhom (adjoint lanes with
// the objective's source), Eq. adjHomNormal with the stepper's own propagator
// (homogeneous chain, summed problems carried lane by lane).
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels_1d.cuh"

namespace cg = cooperative_groups;

namespace pxa {

namespace {

constexpr int HD = 4;  // halo of the direct RK4 step (stage ranges shrink by 1 per stage)
constexpr int HA = 7;  // halo of the reverse RK4 step (stage states 3 deep + reverse 4 deep)

struct Chunk {
  int n, C, rank, nc, start, cnt;
  __device__ void init(int n_, int C_, int rank_) {
    n = n_;
    C = C_;
    rank = rank_;
    nc = (n + C - 1) / C;
    start = rank * nc;
    cnt = min(nc, n - start);
  }
  __device__ __forceinline__ int gidx(int p) const {  // global index of local p (periodic)
    int g = start + p;
    g %= n;
    return g < 0 ? g + n : g;
  }
};

__device__ __forceinline__ double forcing_s(double omega, double t) {
  return omega == 0.0 ? 1.0 : sin(omega * t);
}

// Push the own-chunk values of `buf` (local layout: buf[H + p], p in [0, cnt)) into
// the halo slots of every CTA of the cluster that needs them (including this CTA
// when the halo wraps onto its own chunk). Any chunk size works: for every target
// rank r and halo slot j, the owner of global point (start_r + j) mod n writes it.
template <int H>
__device__ void push_halo(cg::cluster_group& cl, double* buf, const Chunk& ch) {
  const int slots = 2 * H;
  for (int e = threadIdx.x; e < ch.C * slots; e += blockDim.x) {
    const int r = e / slots, s = e % slots;
    const int nc = ch.nc;
    const int start_r = r * nc;
    const int cnt_r = min(nc, ch.n - start_r);
    const int j = s < H ? s - H : cnt_r + (s - H);  // [-H, 0) then [cnt_r, cnt_r + H)
    int g = (start_r + j) % ch.n;
    if (g < 0) g += ch.n;
    const int owner = g / nc;
    if (owner != ch.rank) continue;
    const double v = buf[H + (g - ch.start)];
    double* dst = cl.map_shared_rank(buf, r);
    dst[H + j] = v;
  }
}

struct Bu1Coef {
  double inv2h, invh2, nu;
};

__device__ __forceinline__ double rhs_at(const Bu1Coef& c, const double* y, int i) {
  double ym = y[i - 1], y0 = y[i], yp = y[i + 1];
  double ux = (yp - ym) * c.inv2h;
  double uxx = (yp - 2.0 * y0 + ym) * c.invh2;
  return -y0 * ux + c.nu * uxx;
}

__device__ __forceinline__ double jacT_at(const Bu1Coef& c, const double* U, const double* x, int i) {
  double Um = U[i - 1], Up = U[i + 1];
  double diag = -(Up - Um) * c.inv2h - 2.0 * c.nu * c.invh2;
  double from_m = -Um * c.inv2h + c.nu * c.invh2;
  double from_p = Up * c.inv2h + c.nu * c.invh2;
  return diag * x[i] + from_m * x[i - 1] + from_p * x[i + 1];
}

// One direct RK4 step on the chunk: u (halo HD, current) -> un (own points).
// ya, yb, acc: local stage buffers (halo HD). ff: forcing (halo HD).
__device__ __forceinline__ void rk4_chunk(const Bu1Coef& c, double dt, double c1, double c2,
                                          double c4, const double* u, double* ya, double* yb,
                                          double* acc, const double* ff, int cnt, double* un) {
  // offsets: local p lives at index HD + p
  for (int p = -3 + (int)threadIdx.x; p < cnt + 3; p += blockDim.x) {
    int i = HD + p;
    double k = rhs_at(c, u, i) + c1 * ff[i];
    acc[i] = k;
    ya[i] = u[i] + 0.5 * dt * k;
  }
  __syncthreads();
  for (int p = -2 + (int)threadIdx.x; p < cnt + 2; p += blockDim.x) {
    int i = HD + p;
    double k = rhs_at(c, ya, i) + c2 * ff[i];
    acc[i] += 2.0 * k;
    yb[i] = u[i] + 0.5 * dt * k;
  }
  __syncthreads();
  for (int p = -1 + (int)threadIdx.x; p < cnt + 1; p += blockDim.x) {
    int i = HD + p;
    double k = rhs_at(c, yb, i) + c2 * ff[i];
    acc[i] += 2.0 * k;
    ya[i] = u[i] + dt * k;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
    int i = HD + p;
    double k = rhs_at(c, ya, i) + c4 * ff[i];
    un[i] = u[i] + dt / 6.0 * (acc[i] + k);
  }
}

}  // namespace

// Address of direct-state row s: contiguous rows (lane_k == 0) or the per-lane
// recompute layout (lane l holds rows l*k .. l*k+k in a block of k+1 rows).
__device__ __forceinline__ const double* crow(const double* base, int n, int64_t s, int64_t lane_k,
                                              int lanes, int own_lane) {
  if (lane_k == 0) return base + (size_t)s * n;
  int64_t l = s / lane_k;
  if (l > lanes - 1) l = lanes - 1;
  if (own_lane >= 0 && s == (int64_t)(own_lane + 1) * lane_k) l = own_lane;  // a lane's top row
  return base + ((size_t)l * (size_t)(lane_k + 1) + (size_t)(s - l * lane_k)) * n;
}

// Reverse RK4 sweep of one lane on one cluster, from step s_top down to s_bot.
// lam: double-buffered halo-HA buffers holding lambda_{s+1}; on return lam[parity]
// holds lambda_{s_bot}. gacc: own-point forcing-gradient accumulator.
// Returns the parity index of the buffer that holds the result.
__device__ int bu1c_reverse_sweep(cg::cluster_group& cl, const Chunk& ch, const Bu1Coef& cf,
                                  double dt, double T, double omega, const double* rows,
                                  int64_t lane_k, int lanes, int own_lane, int64_t s_top,
                                  int64_t s_bot, double* u, double* Y2, double* Y3, double* Y4,
                                  double* ma, double* mb, double* lam0, double* lam1,
                                  const double* ff, const double* gg, double* gacc, int par,
                                  bool with_source) {
  const int n = ch.n, cnt = ch.cnt;
  const double src = 2.0 * dt / T;
  double* lb[2] = {lam0, lam1};
  for (int64_t s = s_top - 1; s >= s_bot; --s) {
    const double t = (double)s * dt;
    const double c1 = forcing_s(omega, t), c2 = forcing_s(omega, t + 0.5 * dt),
                 c4 = forcing_s(omega, t + dt);
    const double* us = crow(rows, n, s, lane_k, lanes, own_lane);
    const double* L = lb[par];
    double* Ln = lb[par ^ 1];
    // u_s with halo HA straight from global memory
    for (int p = -HA + (int)threadIdx.x; p < cnt + HA; p += blockDim.x) u[HA + p] = us[ch.gidx(p)];
    __syncthreads();
    // stage states on shrinking ranges: Y2 on +-6, Y3 on +-5, Y4 on +-4
    for (int p = -6 + (int)threadIdx.x; p < cnt + 6; p += blockDim.x) {
      int i = HA + p;
      Y2[i] = u[i] + 0.5 * dt * (rhs_at(cf, u, i) + c1 * ff[i]);
    }
    __syncthreads();
    for (int p = -5 + (int)threadIdx.x; p < cnt + 5; p += blockDim.x) {
      int i = HA + p;
      Y3[i] = u[i] + 0.5 * dt * (rhs_at(cf, Y2, i) + c2 * ff[i]);
    }
    __syncthreads();
    for (int p = -4 + (int)threadIdx.x; p < cnt + 4; p += blockDim.x) {
      int i = HA + p;
      Y4[i] = u[i] + dt * (rhs_at(cf, Y3, i) + c2 * ff[i]);
      ma[i] = dt / 6.0 * L[i];  // kbar4 on +-4
    }
    __syncthreads();
    // Ybar4 = J(Y4)^T kbar4 on +-3; kbar3 = dt/3 lam + dt Ybar4; lamn accumulates in Ln
    for (int p = -3 + (int)threadIdx.x; p < cnt + 3; p += blockDim.x) {
      int i = HA + p;
      double nv = jacT_at(cf, Y4, ma, i);
      mb[i] = dt / 3.0 * L[i] + dt * nv;
      if (p >= 0 && p < cnt) {
        Ln[i] = L[i] + nv;
        gacc[p] = fma(c4, ma[i], gacc[p]);
      }
    }
    __syncthreads();
    // Ybar3 on +-2; kbar2 = dt/3 lam + dt/2 Ybar3
    for (int p = -2 + (int)threadIdx.x; p < cnt + 2; p += blockDim.x) {
      int i = HA + p;
      double nv = jacT_at(cf, Y3, mb, i);
      if (p >= 0 && p < cnt) {
        Ln[i] += nv;
        gacc[p] = fma(c2, mb[i], gacc[p]);
      }
      ma[i] = dt / 3.0 * L[i] + 0.5 * dt * nv;
    }
    __syncthreads();
    // Ybar2 on +-1; kbar1 = dt/6 lam + dt/2 Ybar2
    for (int p = -1 + (int)threadIdx.x; p < cnt + 1; p += blockDim.x) {
      int i = HA + p;
      double nv = jacT_at(cf, Y2, ma, i);
      if (p >= 0 && p < cnt) {
        Ln[i] += nv;
        gacc[p] = fma(c2, ma[i], gacc[p]);
      }
      mb[i] = dt / 6.0 * L[i] + 0.5 * dt * nv;
    }
    __syncthreads();
    // Ybar1 = J(u_s)^T kbar1 on the chunk; lambda_s = lambda_{s+1} + sum Ybar (+ source)
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
      int i = HA + p;
      double nv = jacT_at(cf, u, mb, i);
      gacc[p] = fma(c1, mb[i], gacc[p]);
      double l = Ln[i] + nv;
      if (with_source && s > s_bot) l = fma(src, u[i] - gg[i], l);
      Ln[i] = l;
    }
    __syncthreads();
    push_halo<HA>(cl, Ln, ch);
    cl.sync();
    par ^= 1;
  }
  return par;
}

// Adjoint lanes on clusters (one cluster per lane): exact discrete RK4 adjoint with the
// objective's source and a zero value above the lane (Eq. hybadjinhom). In checkpoint
// mode the lane first recomputes its rows from checkpoint row `lane` into its block of
// `scratch`. Outputs wout[lane] = lambda(T_lane), gout[lane] = lane's forcing gradient.
__global__ void bu1c_adjoint_lanes_kernel(int n, Bu1Coef cf, double dt, double T, int64_t k,
                                          double omega, const double* __restrict__ f,
                                          const double* __restrict__ gt,
                                          const double* __restrict__ traj,
                                          const double* __restrict__ ckpt, double* scratch,
                                          double* __restrict__ wout, double* __restrict__ gout) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm[];
  Chunk ch;
  ch.init(n, (int)cl.num_blocks(), (int)cl.block_rank());
  const int lanes = gridDim.x / ch.C;
  const int lane = blockIdx.x / ch.C;
  const int64_t s0 = (int64_t)lane * k, s1 = s0 + k;
  const int W = ch.nc + 2 * HA;
  double* u = sm;
  double* Y2 = u + W;
  double* Y3 = Y2 + W;
  double* Y4 = Y3 + W;
  double* ma = Y4 + W;
  double* mb = ma + W;
  double* l0 = mb + W;
  double* l1 = l0 + W;
  double* ff = l1 + W;
  double* gg = ff + W;
  double* gacc = gg + W;  // nc
  for (int p = -HA + (int)threadIdx.x; p < ch.cnt + HA; p += blockDim.x) {
    int g = ch.gidx(p);
    ff[HA + p] = f[g];
    gg[HA + p] = gt[g];
  }
  for (int p = threadIdx.x; p < ch.cnt; p += blockDim.x) gacc[p] = 0.0;
  const double* rows = traj;
  int64_t lane_k = 0;
  if (ckpt) {
    // recompute this lane's rows s0..s1 with the cluster RK4 (halo HD inside the HA buffers)
    double* my = scratch + (size_t)lane * (size_t)(k + 1) * n;
    double* ubuf[2] = {Y2, Y3};
    double* ya = Y4;
    double* yb = ma;
    double* acc = mb;
    // reuse ff/gg with halo HA: the direct helpers index halo HD, so shift by HA - HD
    const int sh = HA - HD;
    for (int p = -HD + (int)threadIdx.x; p < ch.cnt + HD; p += blockDim.x)
      ubuf[0][HD + p] = ckpt[(size_t)lane * n + ch.gidx(p)];
    for (int p = threadIdx.x; p < ch.cnt; p += blockDim.x) my[ch.start + p] = ckpt[(size_t)lane * n + ch.start + p];
    __syncthreads();
    for (int64_t s = s0; s < s1; ++s) {
      double* uu = ubuf[(s - s0) & 1];
      double* un = ubuf[(s - s0 + 1) & 1];
      const double t = (double)s * dt;
      rk4_chunk(cf, dt, forcing_s(omega, t), forcing_s(omega, t + 0.5 * dt),
                forcing_s(omega, t + dt), uu, ya, yb, acc, ff + sh, ch.cnt, un);
      __syncthreads();
      for (int p = threadIdx.x; p < ch.cnt; p += blockDim.x)
        my[(size_t)(s + 1 - s0) * n + ch.start + p] = un[HD + p];
      push_halo<HD>(cl, un, ch);
      __threadfence();
      cl.sync();
    }
    rows = scratch;
    lane_k = k;
  }
  __syncthreads();
  // lambda at the lane's top: the objective's source of u_{s1} (halo from global)
  const double src = 2.0 * dt / T;
  const double* top = crow(rows, n, s1, lane_k, lanes, lane);
  for (int p = -HA + (int)threadIdx.x; p < ch.cnt + HA; p += blockDim.x)
    l0[HA + p] = src * (top[ch.gidx(p)] - gg[HA + p]);
  __syncthreads();
  int par = bu1c_reverse_sweep(cl, ch, cf, dt, T, omega, rows, lane_k, lanes, lane, s1, s0, u, Y2,
                               Y3, Y4, ma, mb, l0, l1, ff, gg, gacc, 0, true);
  const double* L = par ? l1 : l0;
  for (int p = threadIdx.x; p < ch.cnt; p += blockDim.x) {
    wout[(size_t)lane * n + ch.start + p] = L[HA + p];
    gout[(size_t)lane * n + ch.start + p] = gacc[p];
  }
}

// Homogeneous chain with the stepper's own propagator on one cluster: h = 0; for
// lane = P-2 .. 0: h += W[lane+1]; sweep h through the lane without source.
__global__ void bu1c_stepper_chain_kernel(int n, Bu1Coef cf, double dt, double T, int64_t k,
                                          int P, double omega, const double* __restrict__ f,
                                          const double* __restrict__ gt,
                                          const double* __restrict__ rows, int64_t lane_k,
                                          const double* __restrict__ Wl,
                                          double* __restrict__ gH) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double sm[];
  Chunk ch;
  ch.init(n, (int)cl.num_blocks(), (int)cl.block_rank());
  const int W = ch.nc + 2 * HA;
  double* u = sm;
  double* Y2 = u + W;
  double* Y3 = Y2 + W;
  double* Y4 = Y3 + W;
  double* ma = Y4 + W;
  double* mb = ma + W;
  double* l0 = mb + W;
  double* l1 = l0 + W;
  double* ff = l1 + W;
  double* gg = ff + W;
  double* gacc = gg + W;
  for (int p = -HA + (int)threadIdx.x; p < ch.cnt + HA; p += blockDim.x) {
    int g = ch.gidx(p);
    ff[HA + p] = f[g];
    gg[HA + p] = gt[g];
    l0[HA + p] = 0.0;
    l1[HA + p] = 0.0;
  }
  for (int p = threadIdx.x; p < ch.cnt; p += blockDim.x) gacc[p] = 0.0;
  __syncthreads();
  int par = 0;
  for (int lane = P - 2; lane >= 0; --lane) {
    double* L = par ? l1 : l0;
    const double* w = Wl + (size_t)(lane + 1) * n;
    for (int p = -HA + (int)threadIdx.x; p < ch.cnt + HA; p += blockDim.x) L[HA + p] += w[ch.gidx(p)];
    __syncthreads();
    const int64_t s0 = (int64_t)lane * k;
    par = bu1c_reverse_sweep(cl, ch, cf, dt, T, omega, rows, lane_k, P, -1, s0 + k, s0, u, Y2, Y3,
                             Y4, ma, mb, l0, l1, ff, gg, gacc, par, false);
  }
  for (int p = threadIdx.x; p < ch.cnt; p += blockDim.x) gH[ch.start + p] = gacc[p];
}

// ---- launch wrappers ---------------------------------------------------------------
static cudaError_t launch_cluster(const void* fn, int grid, int C, int threads, size_t sh,
                                  cudaStream_t st, void** args) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = sh;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

static int cluster_threads(int n, int C) {
  int nc = (n + C - 1) / C + 2 * HA;
  int t = ((nc + 31) / 32) * 32;
  return t < 64 ? 64 : (t > 1024 ? 1024 : t);
}

bool bu1c_valid_cluster(int n, int C) {
  if (C < 1 || C > 16) return false;
  int nc = (n + C - 1) / C;
  // every CTA owns at least one point (so each is a halo source for its neighbours)
  return (C - 1) * nc < n;
}

cudaError_t launch_bu1c_adjoint_lanes(cudaStream_t st, int C, int lanes, int n, double L, double nu,
                                      double dt, double T, int64_t k, double omega, const double* f,
                                      const double* gt, const double* traj, const double* ckpt,
                                      double* scratch, double* wout, double* gout) {
  double h = L / n;
  Bu1Coef cf{1.0 / (2.0 * h), 1.0 / (h * h), nu};
  int nc = (n + C - 1) / C;
  size_t sh = sizeof(double) * (10 * (size_t)(nc + 2 * HA) + nc);
  void* args[] = {&n, &cf, &dt, &T, &k, &omega, &f, &gt, &traj, &ckpt, &scratch, &wout, &gout};
  return launch_cluster((const void*)bu1c_adjoint_lanes_kernel, lanes * C, C,
                        cluster_threads(n, C), sh, st, args);
}

cudaError_t launch_bu1c_stepper_chain(cudaStream_t st, int C, int n, double L, double nu, double dt,
                                      double T, int64_t k, int P, double omega, const double* f,
                                      const double* gt, const double* rows, int64_t lane_k,
                                      const double* W, double* gH) {
  double h = L / n;
  Bu1Coef cf{1.0 / (2.0 * h), 1.0 / (h * h), nu};
  int nc = (n + C - 1) / C;
  size_t sh = sizeof(double) * (10 * (size_t)(nc + 2 * HA) + nc);
  void* args[] = {&n, &cf, &dt, &T, &k, &P, &omega, &f, &gt, &rows, &lane_k, &W, &gH};
  return launch_cluster((const void*)bu1c_stepper_chain_kernel, C, C, cluster_threads(n, C), sh,
                        st, args);
}

}  // namespace pxa
