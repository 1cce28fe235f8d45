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
// Lane mode (chain == 0): cluster c sweeps lane l = lane0 + c, rows s_hi = (l+1)k down to
// s_lo = lk, from lambda_{s_hi} = source(s_hi), adding the source for s > s_lo; it writes
// rows (s_lo, s_hi] to out_rows and lambda_{s_lo} to wout[l] (Eq. hybadjinhom).
// Chain mode (chain == 1, one cluster): rows Pk down to 0. On the top subinterval
// ((P-1)k, Pk] it is the top lane itself (source included, nothing above it); below,
// it carries the sum of the homogeneous problems without source, adding the lane value
// W[j] at row jk for j = P-2 .. 1 (Eq. adjHomNormal with the stepper's propagator).
// Rows (0, Pk] go to out_rows. With P = 1 this is the plain serial adjoint.
//
// Steps are taken in groups of Q: a CTA also updates the 4(Q-1) points on each side of
// its chunk (the neighbours' points, redundantly: an FP64 warp instruction costs the
// same with idle lanes), so one exchange of 4Q boundary values per side serves Q steps.
// A group with parity x starts from buffer A_x (halo received from the neighbours),
// alternates through B_x, and writes its last step into A_{x^1}, which the neighbours
// fill next: a neighbour may run up to one group ahead, and only ever writes the halo
// of the buffer that the receiver reads in its next group.
// Per-thread state of the banded sweep (one point per thread).
struct SweepThread {
  int p, cnt, lane, n;
  int steps;         // s_hi - s_lo
  int src_steps;     // the first src_steps steps add the objective's source
  int inj_it;        // step index of the next lane-value injection (chain), else -1
  int inj_j;
  bool own, act, to_left, to_right;
  uint32_t rl0, rl1, rr0, rr1, bl0, bl1, br0, br1;
  const double* pf;  // record of the next prefetch
  double* orow;      // output row of the current step (own points)
  double* my_ring;
  size_t row_stride;
  int slot_stride, inj_stride;
  const double* wrow;  // W[inj_j][g]
  double* wout;
};

// One step (index it, position m within its group of Q) of the banded sweep.
template <int Q, int DEPTH>
__device__ __forceinline__ void band_step(SweepThread& t, int it, int m, int m0, int x,
                                          const double*& in, double* A_x, double* B_x,
                                          double* A_next, bool exchange_after) {
  if (t.act && it + DEPTH - 1 < t.steps) {
    double* d = t.my_ring + ((it + DEPTH - 1) & (DEPTH - 1)) * t.slot_stride;
#pragma unroll
    for (int q = 0; q < RW / 2; ++q) cp_async16(d + 2 * q, t.pf + 2 * q);
  }
  t.pf -= t.row_stride;
  cp_async_commit();
  cp_async_wait<DEPTH - 1>();
  double* const out = m == Q - 1 ? A_next : (((m - m0) & 1) ? A_x : B_x);
  const int w = 4 * (Q - 1 - m);
  const bool inject = it == t.inj_it;
  if (t.p >= -w && t.p < t.cnt + w) {
    const double2* r2 = reinterpret_cast<const double2*>(t.my_ring + (it & (DEPTH - 1)) * t.slot_stride);
    const double2 q0 = r2[0], q1 = r2[1], q2 = r2[2], q3 = r2[3], q4 = r2[4];
    const double* L = in + t.p;
    double acc = it < t.src_steps ? q4.y : 0.0;
    acc = fma(q0.x, L[-4], acc);
    acc = fma(q0.y, L[-3], acc);
    acc = fma(q1.x, L[-2], acc);
    acc = fma(q1.y, L[-1], acc);
    acc = fma(q2.x, L[0], acc);
    acc = fma(q2.y, L[1], acc);
    acc = fma(q3.x, L[2], acc);
    acc = fma(q3.y, L[3], acc);
    acc = fma(q4.x, L[4], acc);
    if (inject) acc += *t.wrow;
    out[t.p] = acc;
    if (m == Q - 1 && exchange_after) {
      if (t.to_left) st_async_f64(x ? t.rl0 : t.rl1, acc, x ? t.bl0 : t.bl1);
      if (t.to_right) st_async_f64(x ? t.rr0 : t.rr1, acc, x ? t.br0 : t.br1);
    }
    if (t.own) {
      if (it < t.steps - 1) {
        if (t.orow) *t.orow = acc;
      } else if (t.wout) {
        *t.wout = acc;
      }
    }
  }
  if (t.orow) t.orow -= t.n;
  if (inject) {
    --t.inj_j;
    t.inj_it = t.inj_j >= 1 ? t.inj_it + t.inj_stride : -1;
    t.wrow -= t.n;
  }
  in = out;
  if (m < Q - 1) __syncthreads();
}

template <int Q, int DEPTH>
__global__ void bu1_band_sweep_kernel(int n, const double* __restrict__ rec, int k, int P,
                                      int chain, int lane0, const double* __restrict__ W,
                                      double* __restrict__ out_rows, double* __restrict__ wout,
                                      int* status) {
  constexpr int HQ = 4 * Q;      // halo of a group
  constexpr int EX = 4 * Q - 4;  // points computed on each side beyond the chunk
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double smb[];
  __shared__ __align__(8) uint64_t bar[2];
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int nc = (n + C - 1) / C, start = rank * nc, cnt = min(nc, n - start);
  const int lane = chain ? 0 : lane0 + (int)(blockIdx.x / C);
  const int s_hi = chain ? P * k : (lane + 1) * k;
  const int s_lo = chain ? 0 : lane * k;
  const int Wd = nc + 2 * HQ;
  double* const A0 = smb + HQ;
  double* const A1 = smb + Wd + HQ;
  double* const B0 = smb + 2 * Wd + HQ;
  double* const B1 = smb + 3 * Wd + HQ;
  const int npts = nc + 2 * EX;       // points handled by the threads
  double* const ring = smb + 4 * Wd;  // [DEPTH][npts][RW]
  const int tid = threadIdx.x, nt = blockDim.x;
  SweepThread t;
  t.p = tid - EX;
  t.cnt = cnt;
  t.lane = lane;
  t.n = n;
  t.act = t.p >= -EX && t.p < cnt + EX;
  t.own = t.p >= 0 && t.p < cnt;
  const int g = wrapi(start + t.p, n);
  const bool multi = C > 1;
  const int left = (rank + C - 1) % C, right = (rank + 1) % C;
  const int cnt_left = min(nc, n - left * nc);
  if (multi && tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // lambda_{s_hi} on own points and halo, into A0 (group 0 starts there)
  for (int q = tid - HQ; q < cnt + HQ; q += nt) {
    const int gq = wrapi(start + q, n);
    const double v = rec[((size_t)s_hi * n + gq) * RW + (RW - 1)];
    A0[q] = v;
    if (q >= 0 && q < cnt && out_rows) out_rows[(size_t)s_hi * n + start + q] = v;
  }
  // remote halo slots (in A0 / A1) of my boundary points
  t.to_left = multi && t.own && t.p < HQ;
  t.to_right = multi && t.own && t.p >= cnt - HQ;
  t.rl0 = t.rl1 = t.rr0 = t.rr1 = t.bl0 = t.bl1 = t.br0 = t.br1 = 0;
  if (t.to_left) {
    t.rl0 = map_rank(smem_u32(A0 + cnt_left + t.p), left);
    t.rl1 = map_rank(smem_u32(A1 + cnt_left + t.p), left);
    t.bl0 = map_rank(smem_u32(&bar[0]), left);
    t.bl1 = map_rank(smem_u32(&bar[1]), left);
  }
  if (t.to_right) {
    t.rr0 = map_rank(smem_u32(A0 + (t.p - cnt)), right);
    t.rr1 = map_rank(smem_u32(A1 + (t.p - cnt)), right);
    t.br0 = map_rank(smem_u32(&bar[0]), right);
    t.br1 = map_rank(smem_u32(&bar[1]), right);
  }
  const int steps = s_hi - s_lo;
  t.steps = steps;
  t.src_steps = chain ? k - 1 : steps - 1;
  // chain: W[j] is added at row j*k for j = P-2 .. 1, i.e. at step index s_hi-1-j*k
  t.inj_j = chain ? P - 2 : 0;
  t.inj_it = (chain && P >= 3) ? 2 * k - 1 : -1;  // row (P-2)k
  t.inj_stride = k;
  t.wrow = (chain && P >= 3) ? W + (size_t)(P - 2) * n + g : nullptr;
  t.wout = (wout && t.own) ? wout + (size_t)lane * n + start + t.p : nullptr;
  t.orow = (out_rows && t.own) ? out_rows + (size_t)(s_hi - 1) * n + start + t.p : nullptr;
  t.row_stride = (size_t)n * RW;
  t.pf = rec + ((size_t)(s_hi - 1) * n + g) * RW;
  t.my_ring = ring + (size_t)(tid < npts ? tid : 0) * RW;
  t.slot_stride = npts * RW;
#pragma unroll
  for (int j = 0; j < DEPTH - 1; ++j) {
    if (t.act && j < steps) {
      double* d = t.my_ring + j * t.slot_stride;
#pragma unroll
      for (int q = 0; q < RW / 2; ++q) cp_async16(d + 2 * q, t.pf + 2 * q);
    }
    t.pf -= t.row_stride;
    cp_async_commit();
  }
  const int groups = (steps + Q - 1) / Q;
  const int rem = steps - (groups - 1) * Q;  // steps of the last group
  if (multi) {
    if (tid == 0 && groups > 1) mbar_arm(&bar[1], 2 * HQ * (int)sizeof(double));
    cl.sync();  // barriers initialised and armed, initial lambda in place cluster-wide
  } else {
    __syncthreads();
  }
  uint32_t ph0 = 0u, ph1 = 0u;
  int it = 0;
  for (int grp = 0; grp < groups; ++grp) {
    const int x = grp & 1;
    double* const Ax = x ? A1 : A0;
    double* const Bx = x ? B1 : B0;
    double* const An = x ? A0 : A1;
    const bool more = grp + 1 < groups;
    const double* in = Ax;
    if (grp + 1 < groups || rem == Q) {
#pragma unroll
      for (int m = 0; m < Q; ++m) band_step<Q, DEPTH>(t, it + m, m, 0, x, in, Ax, Bx, An, more);
      it += Q;
    } else {
      for (int m = Q - rem; m < Q; ++m, ++it) band_step<Q, DEPTH>(t, it, m, Q - rem, x, in, Ax, Bx, An, more);
    }
    if (more) {
      if (multi) {
        // A_{x^1} is complete once the neighbours' 4Q values per side arrived; arm the
        // barrier of the exchange after the next group first
        if (tid == 0 && grp + 2 < groups) mbar_arm(x ? &bar[1] : &bar[0], 2 * HQ * (int)sizeof(double));
        mbar_wait_bounded(x ? &bar[0] : &bar[1], x ? ph0 : ph1, status);
        if (x) ph0 ^= 1u; else ph1 ^= 1u;
        __syncthreads();
      } else {
        __syncthreads();
        // one CTA holds the whole periodic grid: fill the halo from its own values
        for (int j = tid; j < 2 * HQ; j += nt) {
          const int q = j < HQ ? j - HQ : cnt + (j - HQ);
          An[q] = An[wrapi(q, n)];
        }
        __syncthreads();
      }
    }
  }
  cp_async_wait<0>();
  if (multi) cl.sync();  // no CTA leaves while a neighbour could still address it
}

// ---- 3. forcing gradient --------------------------------------------------------------
// Grid (tiles, step blocks); block y covers the steps s_begin + y spb .. (capped at s_end)
// and writes partial[block0 + y][n] = sum over its steps s of (G_s^T lambda_{s+1}),
// lambda = H (every row, when given) + LI (rows <= li_top).
__global__ void __launch_bounds__(PT) bu1_band_grad_kernel(
    int n, double dt, double omega, int64_t s_begin, int64_t s_end, int64_t li_top,
    const double* __restrict__ LI, const double* __restrict__ H, const double* __restrict__ jt,
    int steps_per_block, int block0, double* __restrict__ partial) {
  __shared__ double lam[PT + 6], kb4[PT + 6], kb3[PT + 6], kb2[PT + 6];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * PT;
  const int by = block0 + (int)blockIdx.y;  // row of partial
  const int64_t sb = s_begin + (int64_t)blockIdx.y * steps_per_block;
  int64_t se = sb + steps_per_block;
  if (se > s_end) se = s_end;
  const double dt6 = dt / 6.0, dt3 = dt / 3.0, h2 = 0.5 * dt;
  double acc = 0.0;
  constexpr int O = 3;  // halo offset
  for (int64_t s = sb; s < se; ++s) {
    const double t = (double)s * dt;
    const double c1 = forcing_s(omega, t), c2 = forcing_s(omega, t + 0.5 * dt),
                 c4 = forcing_s(omega, t + dt);
    const size_t row = (size_t)(s + 1) * n;
    const bool withLI = LI != nullptr && s + 1 <= li_top;
    for (int p = tid - O; p < PT + O; p += PT) {
      const int g = wrapi(i0 + p, n);
      double v = H ? H[row + g] : 0.0;
      if (withLI) v += LI[row + g];
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
  if (i0 + tid < n) partial[(size_t)by * n + i0 + tid] = acc;
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
  // about 32 blocks per SM of a 152-SM part (a quarter of them, the last segment of the
  // chain, still fill the GPU), at least 4 steps per block
  int64_t per = (K * tiles + 4863) / 4864;
  if (per < 4) per = 4;
  if (per > 256) per = 256;
  return (int)per;
}

cudaError_t launch_bu1_band_prepass(cudaStream_t st, int n, double L, double nu, double dt, double T,
                                    double omega, const double* f, const double* gt,
                                    const double* rows, int64_t lane_k, int lanes, int64_t s_begin,
                                    int64_t s_end, int64_t K, double* rec, double* jt, int priority) {
  if (s_end <= s_begin) return cudaSuccess;
  const double h = L / n;
  int spb = bu1_band_steps_per_block(s_end - s_begin, n);
  double inv2h = 1.0 / (2.0 * h), invh2 = 1.0 / (h * h);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((n + PT - 1) / PT, (unsigned)((s_end - s_begin + spb - 1) / spb));
  cfg.blockDim = dim3(PT);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = priority;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bu1_band_prepass_kernel, n, inv2h, invh2, nu, dt, T, omega, f, gt,
                            rows, lane_k, lanes, s_begin, s_end, K, spb, rec, jt);
}

bool bu1_band_valid_cluster(int n, int C) {
  if (C < 1 || C > 16) return false;
  const int nc = (n + C - 1) / C;
  if (nc > BU1_BAND_MAX_CHUNK) return false;
  if (C == 1) return true;
  // every CTA owns at least the 4 points its neighbours need as halo
  return n - (C - 1) * nc >= SH;
}

static size_t sweep_smem(int nc, int q, int depth) {
  const int npts = nc + 2 * (4 * q - 4);
  return sizeof(double) * (4 * (size_t)(nc + 8 * q) + (size_t)depth * npts * RW);
}

// Steps per exchange Q in {1, 2, 4}: every CTA must own the 4Q-point halo its neighbours
// need, and the threads (chunk + 2 (4Q - 4) points) must fit in one CTA.
static bool sweep_group_ok(int n, int C, int q) {
  const int nc = (n + C - 1) / C, last = n - (C - 1) * nc;
  if (nc + 2 * (4 * q - 4) > 1024) return false;
  if (q > 1 && C > 1 && last < 4 * q) return false;
  if (q > 1 && C == 1 && n < 4 * q) return false;
  return true;
}

// The requested Q, or the largest valid smaller one. Without a request: Q = 1. Measured
// on GB300 at n = 1024 over 16 CTAs, grouping the 9-tap steps (Q = 4: 88 points on 3
// warps) was slower than one exchange per step (64 points on 2 warps), unlike the RK4
// sweep; the autotuner still tries 2 and 4.
static int sweep_group(int n, int C, int want) {
  if (want == 4 || want == 2 || want == 1)
    for (int q = want; q >= 1; q /= 2)
      if (sweep_group_ok(n, C, q)) return q;
  return 1;
}

template <int Q>
static cudaError_t launch_sweep_q(cudaStream_t st, int C, int clusters, int nc, void** args,
                                  int priority) {
  const int depth = sweep_smem(nc, Q, 4) <= 200 * 1024 ? 4 : 2;
  const size_t sh = sweep_smem(nc, Q, depth);
  const void* fn = depth == 4 ? (const void*)bu1_band_sweep_kernel<Q, 4>
                              : (const void*)bu1_band_sweep_kernel<Q, 2>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  const int npts = nc + 2 * (4 * Q - 4);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * clusters);
  cfg.blockDim = dim3(((npts + 31) / 32) * 32);
  cfg.dynamicSmemBytes = sh;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributePriority;
  at[1].val.priority = priority;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_bu1_band_sweep(cudaStream_t st, int C, int clusters, int lane0, int n,
                                  const double* rec, int64_t k, int P, int chain, const double* W,
                                  double* out_rows, double* wout, int* status, int priority,
                                  int group) {
  if (clusters <= 0) return cudaSuccess;
  const int nc = (n + C - 1) / C;
  int ki = (int)k;  // steps fit in int: K * n records are addressed with size_t
  void* args[] = {&n, &rec, &ki, &P, &chain, &lane0, &W, &out_rows, &wout, &status};
  switch (sweep_group(n, C, group)) {
    case 4: return launch_sweep_q<4>(st, C, clusters, nc, args, priority);
    case 2: return launch_sweep_q<2>(st, C, clusters, nc, args, priority);
    default: return launch_sweep_q<1>(st, C, clusters, nc, args, priority);
  }
}

int bu1_band_grad_blocks(int64_t K, int n) {
  const int spb = bu1_band_steps_per_block(K, n);
  return (int)((K + spb - 1) / spb);
}

cudaError_t launch_bu1_band_grad(cudaStream_t st, int n, double dt, double omega, int64_t K,
                                 int64_t li_top, const double* LI, const double* H, const double* jt,
                                 double* partial, const double* extra, double* grad, int* status) {
  const int blocks = bu1_band_grad_blocks(K, n);
  cudaError_t e = launch_bu1_band_grad_part(st, n, dt, omega, K, li_top, LI, H, jt, partial, 0, blocks, 0);
  if (e != cudaSuccess) return e;
  return launch_bu1_band_grad_reduce(st, n, K, partial, extra, grad, status);
}

cudaError_t launch_bu1_band_grad_part(cudaStream_t st, int n, double dt, double omega, int64_t K,
                                      int64_t li_top, const double* LI, const double* H,
                                      const double* jt, double* partial, int b_lo, int b_hi,
                                      int priority) {
  if (b_hi <= b_lo) return cudaSuccess;
  const int spb = bu1_band_steps_per_block(K, n);
  const int64_t s_end = (int64_t)b_hi * spb < K ? (int64_t)b_hi * spb : K;
  return launch_bu1_band_grad_range(st, n, dt, omega, (int64_t)b_lo * spb, s_end, spb, li_top, LI, H, jt,
                                    partial, b_lo, priority);
}

cudaError_t launch_bu1_band_grad_range(cudaStream_t st, int n, double dt, double omega, int64_t s_begin,
                                       int64_t s_end, int spb, int64_t li_top, const double* LI,
                                       const double* H, const double* jt, double* partial, int block0,
                                       int priority) {
  if (s_end <= s_begin) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((n + PT - 1) / PT, (unsigned)((s_end - s_begin + spb - 1) / spb));
  cfg.blockDim = dim3(PT);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = priority;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bu1_band_grad_kernel, n, dt, omega, s_begin, s_end, li_top, LI, H, jt, spb,
                            block0, partial);
}

cudaError_t launch_bu1_band_grad_reduce(cudaStream_t st, int n, int64_t K, const double* partial,
                                        const double* extra, double* grad, int* status) {
  const int blocks = bu1_band_grad_blocks(K, n);
  bu1_band_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, blocks, partial, extra, grad, status);
  return cudaGetLastError();
}

cudaError_t launch_bu1_band_reduce_blocks(cudaStream_t st, int n, int blocks, const double* partial,
                                          double* grad, int* status) {
  bu1_band_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, blocks, partial, nullptr, grad, status);
  return cudaGetLastError();
}

// lambda at the bottom row of a checkpoint interval: the chain's row (homogeneous carry
// and the bottom lane's value) plus the objective's source of that row.
__global__ void bu1_band_top_kernel(int n, const double* __restrict__ H, const double* __restrict__ rec,
                                    double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = H[i] + rec[(size_t)i * RW + (RW - 1)];
}

cudaError_t launch_bu1_band_top(cudaStream_t st, int n, const double* H_row, const double* rec_row,
                                double* out) {
  bu1_band_top_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, H_row, rec_row, out);
  return cudaGetLastError();
}

}  // namespace pxa
