// kernels_bu1_band.cu — the discrete adjoint of the 1D Burgers RK4 map as banded step
// matrices (Eq. hybadjinhom and Eq. adjHomNormal with the stepper's own propagator).
//
// One RK4 step u' = u + dt/6 (k1 + 2k2 + 2k3 + k4) of the central-difference Burgers
// operator has a Jacobian M_s = du'/du with nine diagonals (each stage widens the
// stencil by one point), and the adjoint recursion is lambda_s = M_s^T lambda_{s+1} +
// dJ/du_s. On GB300 an FP64 warp instruction holds its sub-partition's FP64 unit for
// 64 cycles whatever the number of active lanes, so the serial reverse sweep costs
// (FP64 instructions per step) x 64 cycles: the stage-by-stage transposed sweep needs
// about 67 of them per step, a precomputed 9-diagonal row of M_s^T needs 9. So:
//
//  1. bu1_band_prepass_kernel (parallel over every step and grid tile): rebuilds the
//     stage states from the stored direct state u_s and writes, for every point i,
//     the record rec[s][i] = { M_s^T[i][i-4..i+4], dJ/du_s[i] } and the transposed
//     stage Jacobian rows of stages 2..4 (for the forcing gradient). Column i of M_s
//     (= row i of M_s^T) is the tangent image of the unit vector e_i through the four
//     stages.
//  2. bu1_band_sweep_kernel (serial in time, one lane per thread-block cluster): the
//     9-tap recursion. Each CTA owns a contiguous chunk; after a step it writes its 4
//     boundary values straight into the neighbours' shared-memory halo with st.async,
//     which completes bytes on the receiver's mbarrier — a point-to-point exchange
//     without a cluster-wide barrier. The records of the coming steps are prefetched
//     into a shared-memory ring with cp.async.
//  3. bu1_band_grad_kernel (parallel): the forcing gradient sum_s G_s^T lambda_{s+1},
//     G_s = du'/df, evaluated by the transposed stage recursion on the stored lambda
//     rows (kbar4 = dt/6 lambda, kbar3 = dt/3 lambda + dt J4^T kbar4, ...), reduced over
//     steps in a fixed order by bu1_band_reduce_kernel.
#include <cooperative_groups.h>

#include "common.cuh"
#include "dsmem.cuh"
#include "kernels_1d.cuh"

namespace cg = cooperative_groups;

namespace pxa {

namespace {

constexpr int RW = BU1_BAND_RECORD;  // doubles per record (9 band taps + source)
constexpr int PT = 128;              // points per tile of the parallel kernels
constexpr int PH = 8;                // direct-state halo of the pre-pass tile
constexpr int PW = PT + 2 * PH;
constexpr int SH = 4;                // lambda halo of the sweep (band half-width)

__device__ __forceinline__ double forcing_s(double omega, double t) {
  return omega == 0.0 ? 1.0 : sin(omega * t);
}

__device__ __forceinline__ int wrapi(int g, int n) {
  g %= n;
  return g < 0 ? g + n : g;
}

// N(y)_i = -y_i (y_{i+1} - y_{i-1}) / (2h) + nu (y_{i+1} - 2 y_i + y_{i-1}) / h^2
__device__ __forceinline__ double burgers_n(double inv2h, double invh2, double nu, double ym,
                                            double y0, double yp) {
  double ux = (yp - ym) * inv2h;
  double uxx = (yp - 2.0 * y0 + ym) * invh2;
  return -y0 * ux + nu * uxx;
}

// Direct-state row s: contiguous rows (lane_k == 0) or the per-lane recompute layout
// (lane l holds rows l*k .. l*k+k in a block of k+1 rows).
__device__ __forceinline__ const double* state_row(const double* base, int n, int64_t s,
                                                   int64_t lane_k, int lanes) {
  if (lane_k == 0) return base + (size_t)s * n;
  int64_t l = s / lane_k;
  if (l > lanes - 1) l = lanes - 1;
  return base + ((size_t)l * (size_t)(lane_k + 1) + (size_t)(s - l * lane_k)) * n;
}

// y = J x for x supported on offsets [-W, W] around local row p; J tridiagonal with row
// coefficients (al, be, ga): (J v)_r = al[r] v_{r-1} + be[r] v_r + ga[r] v_{r+1}.
// y is supported on [-(W+1), W+1]. All offsets are compile-time after unrolling.
template <int W>
__device__ __forceinline__ void jmul(const double* al, const double* be, const double* ga, int p,
                                     const double (&x)[2 * W + 1], double (&y)[2 * W + 3]) {
#pragma unroll
  for (int o = -(W + 1); o <= W + 1; ++o) {
    double acc = 0.0;
    bool any = false;
    if (o - 1 >= -W && o - 1 <= W) {
      acc = al[p + o] * x[o - 1 + W];
      any = true;
    }
    if (o >= -W && o <= W) {
      acc = any ? fma(be[p + o], x[o + W], acc) : be[p + o] * x[o + W];
      any = true;
    }
    if (o + 1 >= -W && o + 1 <= W) acc = any ? fma(ga[p + o], x[o + 1 + W], acc) : ga[p + o] * x[o + 1 + W];
    y[o + W + 1] = acc;
  }
}

}  // namespace

// ---- 1. pre-pass ---------------------------------------------------------------------
// Grid (tiles, step blocks). Rows s in [s_begin, s_end); row K (the final state) only
// gets its source entry. rec: [(K+1)][n][RW]; jt: [K][n][RW].
__global__ void __launch_bounds__(PT) bu1_band_prepass_kernel(
    int n, double inv2h, double invh2, double nu, double dt, double T, double omega,
    const double* __restrict__ f, const double* __restrict__ gt, const double* __restrict__ rows,
    int64_t lane_k, int lanes, int64_t s_begin, int64_t s_end, int64_t K, int steps_per_block,
    double* __restrict__ rec, double* __restrict__ jt) {
  __shared__ double u[PW], y2[PW], y3[PW], y4[PW], ff[PW], gg[PW];
  __shared__ double al[4][PW], be[4][PW], ga[4][PW];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * PT;
  const int64_t sb = s_begin + (int64_t)blockIdx.y * steps_per_block;
  int64_t se = sb + steps_per_block;
  if (se > s_end) se = s_end;
  const double src = 2.0 * dt / T;
  const double h2 = 0.5 * dt, dt6 = dt / 6.0;
  const double a = nu * invh2;
  for (int p = tid - PH; p < PT + PH; p += PT) {
    const int g = wrapi(i0 + p, n);
    ff[PH + p] = f[g];
    gg[PH + p] = gt[g];
  }
  const int pt = i0 + tid;
  const bool own = pt < n;
  for (int64_t s = sb; s < se; ++s) {
    __syncthreads();
    const double* us = state_row(rows, n, s, lane_k, lanes);
    for (int p = tid - PH; p < PT + PH; p += PT) u[PH + p] = us[wrapi(i0 + p, n)];
    __syncthreads();
    const double R = s >= 1 ? src * (u[PH + tid] - gg[PH + tid]) : 0.0;
    if (s == K) {  // final state: the source of lambda_K only
      if (own) {
        double* r = rec + ((size_t)s * n + pt) * RW;
#pragma unroll
        for (int j = 0; j < RW - 1; ++j) r[j] = 0.0;
        r[RW - 1] = R;
      }
      continue;
    }
    const double t = (double)s * dt;
    const double c1 = forcing_s(omega, t), c2 = forcing_s(omega, t + 0.5 * dt),
                 c4 = forcing_s(omega, t + dt);
    // stage states on shrinking ranges: Y2 on +-7, Y3 on +-6, Y4 on +-5
    for (int p = tid - 7; p < PT + 7; p += PT) {
      const int i = PH + p;
      y2[i] = u[i] + h2 * (burgers_n(inv2h, invh2, nu, u[i - 1], u[i], u[i + 1]) + c1 * ff[i]);
    }
    __syncthreads();
    for (int p = tid - 6; p < PT + 6; p += PT) {
      const int i = PH + p;
      y3[i] = u[i] + h2 * (burgers_n(inv2h, invh2, nu, y2[i - 1], y2[i], y2[i + 1]) + c2 * ff[i]);
    }
    __syncthreads();
    for (int p = tid - 5; p < PT + 5; p += PT) {
      const int i = PH + p;
      y4[i] = u[i] + dt * (burgers_n(inv2h, invh2, nu, y3[i - 1], y3[i], y3[i + 1]) + c2 * ff[i]);
    }
    __syncthreads();
    // Jacobian rows of the four stages: stage q on rows +-q (+-4 covers all)
    for (int p = tid - 4; p < PT + 4; p += PT) {
      const int i = PH + p;
      const double* Y[4] = {u, y2, y3, y4};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double yc = Y[q][i];
        al[q][i] = fma(yc, inv2h, a);
        ga[q][i] = fma(-yc, inv2h, a);
        be[q][i] = fma(-(Y[q][i + 1] - Y[q][i - 1]), inv2h, -2.0 * a);
      }
    }
    __syncthreads();
    if (!own) continue;
    const int p = PH + tid;
    // tangent image of e_p: d1 = J1 e, Y2' = e + dt/2 d1, d2 = J2 Y2', Y3' = e + dt/2 d2,
    // d3 = J3 Y3', Y4' = e + dt d3, d4 = J4 Y4'; column = e + dt/6 (d1 + 2 d2 + 2 d3 + d4)
    double d1[3] = {ga[0][p - 1], be[0][p], al[0][p + 1]};
    double v2[3] = {h2 * d1[0], fma(h2, d1[1], 1.0), h2 * d1[2]};
    double d2[5];
    jmul<1>(al[1], be[1], ga[1], p, v2, d2);
    double v3[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) v3[o] = o == 2 ? fma(h2, d2[o], 1.0) : h2 * d2[o];
    double d3[7];
    jmul<2>(al[2], be[2], ga[2], p, v3, d3);
    double v4[7];
#pragma unroll
    for (int o = 0; o < 7; ++o) v4[o] = o == 3 ? fma(dt, d3[o], 1.0) : dt * d3[o];
    double d4[9];
    jmul<3>(al[3], be[3], ga[3], p, v4, d4);
    double col[RW];
#pragma unroll
    for (int o = 0; o < 9; ++o) {
      double sum = d4[o];
      if (o >= 1 && o <= 7) sum = fma(2.0, d3[o - 1], sum);
      if (o >= 2 && o <= 6) sum = fma(2.0, d2[o - 2], sum);
      if (o >= 3 && o <= 5) sum += d1[o - 3];
      col[o] = o == 4 ? fma(dt6, sum, 1.0) : dt6 * sum;
    }
    col[9] = R;
    double2* r2 = reinterpret_cast<double2*>(rec + ((size_t)s * n + pt) * RW);
#pragma unroll
    for (int j = 0; j < RW / 2; ++j) r2[j] = make_double2(col[2 * j], col[2 * j + 1]);
    // transposed stage rows for the forcing gradient: (J_q^T x)_p = ga_q[p-1] x_{p-1} +
    // be_q[p] x_p + al_q[p+1] x_{p+1}, stages q = 2, 3, 4
    double jr[RW];
#pragma unroll
    for (int q = 1; q < 4; ++q) {
      jr[3 * (q - 1) + 0] = ga[q][p - 1];
      jr[3 * (q - 1) + 1] = be[q][p];
      jr[3 * (q - 1) + 2] = al[q][p + 1];
    }
    jr[9] = 0.0;
    double2* j2 = reinterpret_cast<double2*>(jt + ((size_t)s * n + pt) * RW);
#pragma unroll
    for (int j = 0; j < RW / 2; ++j) j2[j] = make_double2(jr[2 * j], jr[2 * j + 1]);
  }
}

// ---- 2. banded reverse sweep --------------------------------------------------------
// Lane mode (chain == 0): cluster l sweeps rows s_hi = (l+1)k down to s_lo = lk from
// lambda_{s_hi} = source(s_hi), adding the source for s > s_lo; it writes rows
// (s_lo, s_hi] to out_rows and lambda_{s_lo} to wout[l].
// Chain mode (chain == 1, one cluster): h_{(P-1)k} = W[P-1], swept down to row 0 without
// source, adding W[j] at rows jk (0 < j < P-1); rows (0, (P-1)k] go to out_rows.
template <int DEPTH>
__global__ void bu1_band_sweep_kernel(int n, const double* __restrict__ rec, int64_t k, int P,
                                      int chain, const double* __restrict__ W,
                                      double* __restrict__ out_rows, double* __restrict__ wout,
                                      int* status) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double smb[];
  __shared__ __align__(8) uint64_t bar[2];
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int nc = (n + C - 1) / C, start = rank * nc, cnt = min(nc, n - start);
  const int lane = chain ? 0 : (int)(blockIdx.x / C);
  const int64_t s_hi = chain ? (int64_t)(P - 1) * k : (int64_t)(lane + 1) * k;
  const int64_t s_lo = chain ? 0 : (int64_t)lane * k;
  const int Wd = nc + 2 * SH;
  double* const lam0 = smb;
  double* const lam1 = smb + Wd;
  double* ring = smb + 2 * Wd;  // [DEPTH][nc][RW]
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool multi = C > 1;
  // the neighbours' chunk sizes, and where my boundary values land in their halos
  const int left = (rank + C - 1) % C, right = (rank + 1) % C;
  const int cnt_left = min(nc, n - left * nc);
  if (multi && tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // lambda_{s_hi} on own points and halo
  for (int p = tid - SH; p < cnt + SH; p += nt) {
    const int g = wrapi(start + p, n);
    const double v = chain ? W[(size_t)(P - 1) * n + g] : rec[((size_t)s_hi * n + g) * RW + (RW - 1)];
    ((s_hi & 1) ? lam1 : lam0)[SH + p] = v;
    if (p >= 0 && p < cnt && out_rows) out_rows[(size_t)s_hi * n + start + p] = v;
  }
  // Prefetch of the records of step s into ring slot `slot`, one commit group per step.
  // Each thread copies the records of exactly the points it consumes, so its own
  // cp.async.wait_group is the only wait the data needs.
  auto prefetch = [&](int64_t s, int slot) {
    if (s >= s_lo) {
      const double* srcp = rec + ((size_t)s * n + start) * RW;
      double* dst = ring + (size_t)slot * nc * RW;
      for (int p = tid; p < cnt; p += nt) {
#pragma unroll
        for (int j = 0; j < RW / 2; ++j) cp_async16(dst + (size_t)p * RW + 2 * j, srcp + (size_t)p * RW + 2 * j);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int j = 0; j < DEPTH - 1; ++j) prefetch(s_hi - 1 - j, j);
  if (multi) {
    if (tid == 0 && s_hi - 1 >= s_lo) mbar_arm(&bar[(s_hi - 1) & 1], 2 * SH * (int)sizeof(double));
    cl.sync();  // barriers initialised and armed, initial lambda in place cluster-wide
  } else {
    __syncthreads();
  }
  uint32_t ph0 = 0u, ph1 = 0u;
  const int64_t steps = s_hi - s_lo;
  // chain: the next row that receives a lane value, W[inj_j] at row inj_j * k
  int inj_j = chain ? P - 2 : 0;
  int64_t inj_row = (int64_t)inj_j * k;
  for (int64_t it = 0; it < steps; ++it) {
    const int64_t s = s_hi - 1 - it;
    prefetch(s - (DEPTH - 1), (int)((uint64_t)(it + DEPTH - 1) % DEPTH));
    cp_async_wait<DEPTH - 1>();
    const int b = (int)(s & 1);
    double* const lb = b ? lam1 : lam0;
    const double* Lp = (b ? lam0 : lam1) + SH;
    double* Ln = lb + SH;
    uint64_t* const bar_b = b ? &bar[1] : &bar[0];
    const double* rs = ring + (size_t)((uint64_t)it % DEPTH) * nc * RW;
    const bool add_src = !chain && s > s_lo;
    const bool inject = chain && inj_j >= 1 && s == inj_row;
    for (int p = tid; p < cnt; p += nt) {
      const double2* r2 = reinterpret_cast<const double2*>(rs + (size_t)p * RW);
      const double2 q0 = r2[0], q1 = r2[1], q2 = r2[2], q3 = r2[3], q4 = r2[4];
      double acc = add_src ? q4.y : 0.0;
      acc = fma(q0.x, Lp[p - 4], acc);
      acc = fma(q0.y, Lp[p - 3], acc);
      acc = fma(q1.x, Lp[p - 2], acc);
      acc = fma(q1.y, Lp[p - 1], acc);
      acc = fma(q2.x, Lp[p], acc);
      acc = fma(q2.y, Lp[p + 1], acc);
      acc = fma(q3.x, Lp[p + 2], acc);
      acc = fma(q3.y, Lp[p + 3], acc);
      acc = fma(q4.x, Lp[p + 4], acc);
      if (inject) acc += W[(size_t)inj_j * n + start + p];
      Ln[p] = acc;
      if (multi) {
        if (p < SH)  // my first points are the left neighbour's right halo
          st_async_f64(map_rank(smem_u32(lb + SH + cnt_left + p), left), acc,
                       map_rank(smem_u32(bar_b), left));
        if (p >= cnt - SH)  // my last points are the right neighbour's left halo
          st_async_f64(map_rank(smem_u32(lb + SH + (p - cnt)), right), acc,
                       map_rank(smem_u32(bar_b), right));
      }
      if (s > s_lo && out_rows) out_rows[(size_t)s * n + start + p] = acc;
      if (s == s_lo && wout) wout[(size_t)lane * n + start + p] = acc;
    }
    if (inject) {
      --inj_j;
      inj_row -= k;
    }
    if (multi) {
      if (tid == 0 && s - 1 >= s_lo) mbar_arm(b ? &bar[0] : &bar[1], 2 * SH * (int)sizeof(double));
      mbar_wait_bounded(bar_b, b ? ph1 : ph0, status);
      if (b) ph1 ^= 1u; else ph0 ^= 1u;
      __syncthreads();
    } else {
      __syncthreads();
      // one CTA holds the whole periodic grid: fill the halo from its own values
      for (int j = tid; j < 2 * SH; j += nt) {
        const int p = j < SH ? j - SH : cnt + (j - SH);
        Ln[p] = Ln[wrapi(p, n)];
      }
      __syncthreads();
    }
  }
  cp_async_wait<0>();
  if (multi) cl.sync();  // no CTA leaves while a neighbour could still address it
}

// ---- 3. forcing gradient --------------------------------------------------------------
// Grid (tiles, step blocks); partial[block_y][n] = sum over the block's steps s of
// (G_s^T lambda_{s+1}), lambda = LI (+ H for rows <= h_top when H is given).
__global__ void __launch_bounds__(PT) bu1_band_grad_kernel(
    int n, double dt, double omega, int64_t K, int64_t h_top, const double* __restrict__ LI,
    const double* __restrict__ H, const double* __restrict__ jt, int steps_per_block,
    double* __restrict__ partial) {
  __shared__ double lam[PT + 6], kb4[PT + 6], kb3[PT + 6], kb2[PT + 6];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * PT;
  const int64_t sb = (int64_t)blockIdx.y * steps_per_block;
  int64_t se = sb + steps_per_block;
  if (se > K) se = K;
  const double dt6 = dt / 6.0, dt3 = dt / 3.0, h2 = 0.5 * dt;
  double acc = 0.0;
  constexpr int O = 3;  // halo offset
  for (int64_t s = sb; s < se; ++s) {
    const double t = (double)s * dt;
    const double c1 = forcing_s(omega, t), c2 = forcing_s(omega, t + 0.5 * dt),
                 c4 = forcing_s(omega, t + dt);
    const size_t row = (size_t)(s + 1) * n;
    const bool withH = H != nullptr && s + 1 <= h_top;
    for (int p = tid - O; p < PT + O; p += PT) {
      const int g = wrapi(i0 + p, n);
      double v = LI[row + g];
      if (withH) v += H[row + g];
      lam[O + p] = v;
      kb4[O + p] = dt6 * v;
    }
    __syncthreads();
    // kbar3 = dt/3 lambda + dt J4^T kbar4 on +-2 (stage-4 rows at jt[.][6..8])
    for (int p = tid - 2; p < PT + 2; p += PT) {
      const double* r = jt + ((size_t)s * n + wrapi(i0 + p, n)) * RW;
      const int i = O + p;
      double x = r[6] * kb4[i - 1];
      x = fma(r[7], kb4[i], x);
      x = fma(r[8], kb4[i + 1], x);
      kb3[i] = fma(dt3, lam[i], dt * x);
    }
    __syncthreads();
    // kbar2 = dt/3 lambda + dt/2 J3^T kbar3 on +-1 (stage 3 at jt[.][3..5])
    for (int p = tid - 1; p < PT + 1; p += PT) {
      const double* r = jt + ((size_t)s * n + wrapi(i0 + p, n)) * RW;
      const int i = O + p;
      double x = r[3] * kb3[i - 1];
      x = fma(r[4], kb3[i], x);
      x = fma(r[5], kb3[i + 1], x);
      kb2[i] = fma(dt3, lam[i], h2 * x);
    }
    __syncthreads();
    // kbar1 = dt/6 lambda + dt/2 J2^T kbar2 (stage 2 at jt[.][0..2]); accumulate
    if (i0 + tid < n) {
      const double* r = jt + ((size_t)s * n + i0 + tid) * RW;
      const int i = O + tid;
      double x = r[0] * kb2[i - 1];
      x = fma(r[1], kb2[i], x);
      x = fma(r[2], kb2[i + 1], x);
      const double kb1 = fma(dt6, lam[i], h2 * x);
      acc = fma(c1, kb1, acc);
      acc = fma(c2, kb2[i] + kb3[i], acc);
      acc = fma(c4, kb4[i], acc);
    }
    __syncthreads();
  }
  if (i0 + tid < n) partial[(size_t)blockIdx.y * n + i0 + tid] = acc;
}

// grad[i] = sum_b partial[b][i] (+ extra[i]), in a fixed order.
__global__ void bu1_band_reduce_kernel(int n, int blocks, const double* __restrict__ partial,
                                       const double* __restrict__ extra, double* __restrict__ grad,
                                       int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int b = 0; b < blocks; ++b) s += partial[(size_t)b * n + i];
  if (extra) s += extra[i];
  grad[i] = s;
  if (!isfinite(s)) set_status(status, PXA_ERR_NONFINITE);
}

// ---- launch wrappers ---------------------------------------------------------------
int bu1_band_steps_per_block(int64_t K, int n) {
  const int tiles = (n + PT - 1) / PT;
  // about 8 blocks per SM of a 152-SM part, at least 4 steps per block
  int64_t per = (K * tiles + 1215) / 1216;
  if (per < 4) per = 4;
  if (per > 256) per = 256;
  return (int)per;
}

cudaError_t launch_bu1_band_prepass(cudaStream_t st, int n, double L, double nu, double dt, double T,
                                    double omega, const double* f, const double* gt,
                                    const double* rows, int64_t lane_k, int lanes, int64_t s_begin,
                                    int64_t s_end, int64_t K, double* rec, double* jt) {
  if (s_end <= s_begin) return cudaSuccess;
  const double h = L / n;
  const int spb = bu1_band_steps_per_block(s_end - s_begin, n);
  dim3 grid((n + PT - 1) / PT, (unsigned)((s_end - s_begin + spb - 1) / spb));
  bu1_band_prepass_kernel<<<grid, PT, 0, st>>>(n, 1.0 / (2.0 * h), 1.0 / (h * h), nu, dt, T, omega,
                                               f, gt, rows, lane_k, lanes, s_begin, s_end, K, spb,
                                               rec, jt);
  return cudaGetLastError();
}

bool bu1_band_valid_cluster(int n, int C) {
  if (C < 1 || C > 16) return false;
  const int nc = (n + C - 1) / C;
  if (nc > BU1_BAND_MAX_CHUNK) return false;
  if (C == 1) return true;
  // every CTA owns at least the 4 points its neighbours need as halo
  return n - (C - 1) * nc >= SH;
}

static int sweep_threads(int nc) {
  int t = ((nc + 31) / 32) * 32;
  return t < 32 ? 32 : (t > 1024 ? 1024 : t);
}

static size_t sweep_smem(int nc, int depth) {
  return sizeof(double) * (2 * (size_t)(nc + 2 * SH) + (size_t)depth * nc * RW);
}

cudaError_t launch_bu1_band_sweep(cudaStream_t st, int C, int clusters, int n, const double* rec,
                                  int64_t k, int P, int chain, const double* W, double* out_rows,
                                  double* wout, int* status) {
  const int nc = (n + C - 1) / C;
  const int depth = sweep_smem(nc, 4) <= 200 * 1024 ? 4 : 2;
  const size_t sh = sweep_smem(nc, depth);
  const void* fn = depth == 4 ? (const void*)bu1_band_sweep_kernel<4> : (const void*)bu1_band_sweep_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {&n, &rec, &k, &P, &chain, &W, &out_rows, &wout, &status};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * clusters);
  cfg.blockDim = dim3(sweep_threads(nc));
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

int bu1_band_grad_blocks(int64_t K, int n) {
  const int spb = bu1_band_steps_per_block(K, n);
  return (int)((K + spb - 1) / spb);
}

cudaError_t launch_bu1_band_grad(cudaStream_t st, int n, double dt, double omega, int64_t K,
                                 int64_t h_top, const double* LI, const double* H, const double* jt,
                                 double* partial, const double* extra, double* grad, int* status) {
  const int spb = bu1_band_steps_per_block(K, n);
  const int blocks = (int)((K + spb - 1) / spb);
  dim3 grid((n + PT - 1) / PT, blocks);
  bu1_band_grad_kernel<<<grid, PT, 0, st>>>(n, dt, omega, K, h_top, LI, H, jt, spb, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bu1_band_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, blocks, partial, extra, grad, status);
  return cudaGetLastError();
}

}  // namespace pxa
