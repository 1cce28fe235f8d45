// kernels_bu1_rk4.cu — serial RK4 of the nonlinear 1D Burgers direct problem on a
// thread-block cluster (Eq. seriesDirect), and the same sweep run per subinterval from
// boundary checkpoints (the recompute of Sec. 3.5).
//
// One time lane is split into contiguous chunks, one per CTA. Thread t works on local
// point p = t - 3, so the threads of one CTA cover its chunk plus 3 points on each side:
// the four RK4 stages are evaluated on shrinking ranges (+-3, +-2, +-1, 0) and a whole
// step needs the neighbours' 4 boundary values only once. After the last stage each
// CTA writes its 4 first and 4 last new values straight into the neighbours' shared
// memory with st.async; the receiver waits on its own mbarrier for those 64 bytes
// (no cluster-wide barrier).
//
// GB300 issues one FP64 warp instruction per 64 cycles on each SM sub-partition, so the
// step time is set by the FP64 instructions on a warp's path. Each stage here costs 5
// for k = N(y) + s(t) f, written as a (y_{i+1} + y_{i-1}) - y_i (b (y_{i+1} - y_{i-1}) +
// 2a) + c f with b = 1/(2h), a = nu/h^2, plus 1-2 for the stage state and the weighted
// sum: 27 per step. The objective's term (2 more) is issued after the halo sends, while
// the exchange is in flight.
#include <cooperative_groups.h>

#include "common.cuh"
#include "dsmem.cuh"
#include "kernels_1d.cuh"

namespace cg = cooperative_groups;

namespace pxa {

namespace {

constexpr int HX = 4;  // halo of one RK4 step (the stage ranges shrink by one point each)

// k = N(y) + c f at one point: a (yp + ym) - y0 (b (yp - ym) + 2a) + cf
__device__ __forceinline__ double stage_k(double b, double a, double a2, double ym, double y0,
                                          double yp, double cf) {
  const double s = yp + ym;
  const double d = yp - ym;
  const double t = fma(b, d, a2);
  const double r = fma(a, s, cf);
  return fma(-y0, t, r);
}

}  // namespace

// sc[3s + {0, 1, 2}] = s(t_s), s(t_s + dt/2), s(t_s + dt) with s(t) = sin(omega t).
__global__ void bu1_forcing_table_kernel(int64_t K, double dt, double omega, double* __restrict__ sc) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= K) return;
  const double t = (double)s * dt;
  sc[3 * s + 0] = sin(omega * t);
  sc[3 * s + 1] = sin(omega * (t + 0.5 * dt));
  sc[3 * s + 2] = sin(omega * (t + dt));
}

// Cluster l steps s = l*k .. l*k+k-1 from x0[l] (x0 == NULL: zero state). State rows
// go to out + (l*lane_rows + j)*n, j = 0..k (out may be NULL). With Jdev, J = (dt/T)
// sum_{j>=1} ||u_j - g||^2 (one lane only); with ckpt, every ck_every-th state goes to
// ckpt row s / ck_every. FORCED == false: s(t) = 1 (sc unused).
//
// Steps are taken in groups of Q: each CTA also steps the 4(Q-1) points on each side of
// its chunk (its neighbours' points, redundantly), so one exchange of 4Q boundary values
// per side serves Q steps. A group with parity x starts from state buffer A_x (halo
// received), alternates through B_x and writes its last step into A_{x^1}, whose halo the
// neighbours fill: a neighbour can run at most one group ahead and only ever writes the
// halo of the buffer the receiver reads next.
// Per-thread state of the RK4 sweep (one point per thread).
struct Rk4Thread {
  int p, cnt, n;
  int k;              // steps of this lane
  bool own;
  double fp, gp;      // forcing and target at the point
  double b, a, a2, h2, dt, dt6;
  double c1, c2, c4;  // s(t) at the stage times of the current step
  const double* scp;  // s(t) of the next step
  double* yap;
  double* ybp;
  double* orow;       // output row of the next state (own points)
  size_t n_stride;
  double* ckpt;
  int ck_left, ck_row, ck_every, start;
  double jp;
  bool with_j;
  bool to_left, to_right;
  uint32_t rl0, rl1, rr0, rr1, bl0, bl1, br0, br1;
};

// One RK4 step (index j, position m within its group of Q) on the points within
// 4(Q-1-m) + 3 of the chunk.
template <bool FORCED, int Q>
__device__ __forceinline__ void rk4_step(Rk4Thread& t, int j, int m, int m0, int x,
                                         const double*& in, double* A_x, double* B_x,
                                         double* A_next, bool exchange_after) {
  double* const outb = m == Q - 1 ? A_next : (((m - m0) & 1) ? A_x : B_x);
  const int w = 4 * (Q - 1 - m);  // the new state is valid on [-w, cnt + w)
  const int p = t.p;
  double n1 = 1.0, n2 = 1.0, n4 = 1.0;
  if (FORCED && j + 1 < t.k) {  // forcing factors of the next step, loaded a step ahead
    n1 = t.scp[0];
    n2 = t.scp[1];
    n4 = t.scp[2];
    t.scp += 3;
  }
  double cf1 = t.fp, cf2 = t.fp, cf4 = t.fp;
  if (FORCED) {
    cf1 = t.c1 * t.fp;
    cf2 = t.c2 * t.fp;
    cf4 = t.c4 * t.fp;
  }
  const double* Up = in + p;
  double u0 = 0.0, acc = 0.0;
  if (p >= -(w + 3) && p < t.cnt + w + 3) {
    u0 = Up[0];
    const double kk = stage_k(t.b, t.a, t.a2, Up[-1], u0, Up[1], cf1);
    t.yap[0] = fma(t.h2, kk, u0);
    acc = kk;
  }
  __syncthreads();
  if (p >= -(w + 2) && p < t.cnt + w + 2) {
    const double kk = stage_k(t.b, t.a, t.a2, t.yap[-1], t.yap[0], t.yap[1], cf2);
    t.ybp[0] = fma(t.h2, kk, u0);
    acc = fma(2.0, kk, acc);
  }
  __syncthreads();
  if (p >= -(w + 1) && p < t.cnt + w + 1) {
    const double kk = stage_k(t.b, t.a, t.a2, t.ybp[-1], t.ybp[0], t.ybp[1], cf2);
    t.yap[0] = fma(t.dt, kk, u0);
    acc = fma(2.0, kk, acc);
  }
  __syncthreads();
  if (p >= -w && p < t.cnt + w) {
    const double kk = stage_k(t.b, t.a, t.a2, t.yap[-1], t.yap[0], t.yap[1], cf4);
    const double un = fma(t.dt6, acc + kk, u0);
    outb[p] = un;
    if (m == Q - 1 && exchange_after) {
      if (t.to_left) st_async_f64(x ? t.rl0 : t.rl1, un, x ? t.bl0 : t.bl1);
      if (t.to_right) st_async_f64(x ? t.rr0 : t.rr1, un, x ? t.br0 : t.br1);
    }
    if (t.own) {
      if (t.with_j) {
        const double d = un - t.gp;
        t.jp = fma(d, d, t.jp);
      }
      if (t.orow) *t.orow = un;
      if (t.ckpt && t.ck_left == 1) t.ckpt[(size_t)t.ck_row * t.n + t.start + p] = un;
    }
  }
  if (t.orow) t.orow += t.n_stride;
  if (t.ckpt) {
    if (t.ck_left == 1) {
      t.ck_left = t.ck_every;
      ++t.ck_row;
    } else {
      --t.ck_left;
    }
  }
  if (FORCED) {
    t.c1 = n1;
    t.c2 = n2;
    t.c4 = n4;
  }
  in = outb;
  if (m < Q - 1) __syncthreads();
}

// Cluster l steps s = l*k .. l*k+k-1 from x0[l] (x0 == NULL: zero state). State rows
// go to out + (l*lane_rows + j)*n, j = 0..k (out may be NULL). With Jdev, J = (dt/T)
// sum_{j>=1} ||u_j - g||^2 (one lane only); with ckpt, every ck_every-th state goes to
// ckpt row s / ck_every. FORCED == false: s(t) = 1 (sc unused).
//
// Steps are taken in groups of Q: each CTA also steps the 4(Q-1) points on each side of
// its chunk (its neighbours' points, redundantly), so one exchange of 4Q boundary values
// per side serves Q steps. A group with parity x starts from state buffer A_x (halo
// received), alternates through B_x and writes its last step into A_{x^1}, whose halo the
// neighbours fill: a neighbour can run at most one group ahead and only ever writes the
// halo of the buffer the receiver reads next.
template <bool FORCED, int Q>
__global__ void bu1_rk4_sweep_kernel(int n, double b, double a, double dt, int k,
                                     const double* __restrict__ f, const double* __restrict__ sc,
                                     const double* __restrict__ x0, double* __restrict__ out,
                                     int lane_rows, const double* __restrict__ gt, double T,
                                     double* __restrict__ Jdev, double* __restrict__ ckpt,
                                     int ck_every, int* status) {
  constexpr int HQ = 4 * Q;      // halo of a group
  constexpr int EX = 4 * Q - 1;  // points stepped on each side beyond the chunk (stage 1)
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double sm[];
  __shared__ __align__(8) uint64_t bar[2];
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int nc = (n + C - 1) / C, start = rank * nc, cnt = min(nc, n - start);
  const int lane = (int)(blockIdx.x / C);
  const int s0 = lane * k;
  const int Wd = nc + 2 * HQ;
  double* const A0 = sm + HQ;
  double* const A1 = sm + Wd + HQ;
  double* const B0 = sm + 2 * Wd + HQ;
  double* const B1 = sm + 3 * Wd + HQ;
  double* const ya = sm + 4 * Wd + HQ;
  double* const yb = sm + 5 * Wd + HQ;
  double* const red = sm + 6 * Wd;  // 64 doubles
  const int tid = threadIdx.x;
  const bool multi = C > 1;
  const int left = (rank + C - 1) % C, right = (rank + 1) % C;
  const int cnt_left = min(nc, n - left * nc);
  Rk4Thread t;
  t.p = tid - EX;
  t.cnt = cnt;
  t.n = n;
  t.k = k;
  t.start = start;
  t.own = t.p >= 0 && t.p < cnt;
  const bool act = t.p >= -EX && t.p < cnt + EX;
  t.fp = act ? f[((start + t.p) % n + n) % n] : 0.0;
  t.gp = t.own && gt ? gt[start + t.p] : 0.0;
  t.b = b;
  t.a = a;
  t.a2 = 2.0 * a;
  t.h2 = 0.5 * dt;
  t.dt = dt;
  t.dt6 = dt / 6.0;
  t.with_j = Jdev != nullptr;
  t.jp = 0.0;
  if (multi && tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int q = tid - HQ; q < cnt + HQ; q += blockDim.x) {
    const int g = ((start + q) % n + n) % n;
    A0[q] = x0 ? x0[(size_t)lane * n + g] : 0.0;
  }
  __syncthreads();
  if (t.own) {
    if (out) out[((size_t)lane * lane_rows) * n + start + t.p] = A0[t.p];
    if (ckpt && s0 % ck_every == 0) ckpt[(size_t)(s0 / ck_every) * n + start + t.p] = A0[t.p];
  }
  t.ckpt = ckpt;
  t.ck_every = ck_every;
  t.ck_left = ckpt ? ck_every - (s0 % ck_every) : 0;  // steps until the next checkpoint
  t.ck_row = ckpt ? s0 / ck_every + 1 : 0;             // row of the next checkpoint
  t.c1 = t.c2 = t.c4 = 1.0;
  if (FORCED) {
    t.c1 = sc[3 * (size_t)s0];
    t.c2 = sc[3 * (size_t)s0 + 1];
    t.c4 = sc[3 * (size_t)s0 + 2];
  }
  t.scp = FORCED ? sc + 3 * ((size_t)s0 + 1) : nullptr;
  // remote halo slots (in A0 / A1) of my boundary points and their barriers
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
  t.yap = ya + t.p;
  t.ybp = yb + t.p;
  t.n_stride = (size_t)n;
  t.orow = (out && t.own) ? out + ((size_t)lane * lane_rows + 1) * n + start + t.p : nullptr;
  const int groups = (k + Q - 1) / Q;
  const int rem = k - (groups - 1) * Q;  // steps of the last group
  if (multi) {
    if (tid == 0 && groups > 1) mbar_arm(&bar[1], 2 * HQ * (int)sizeof(double));
    cl.sync();
  }
  uint32_t ph0 = 0u, ph1 = 0u;
  int j = 0;  // steps done
  for (int grp = 0; grp < groups; ++grp) {
    const int x = grp & 1;
    double* const Ax = x ? A1 : A0;
    double* const Bx = x ? B1 : B0;
    double* const An = x ? A0 : A1;
    const bool more = grp + 1 < groups;
    const double* in = Ax;
    if (more || rem == Q) {
#pragma unroll
      for (int m = 0; m < Q; ++m) rk4_step<FORCED, Q>(t, j + m, m, 0, x, in, Ax, Bx, An, more);
      j += Q;
    } else {
      for (int m = Q - rem; m < Q; ++m, ++j) rk4_step<FORCED, Q>(t, j, m, Q - rem, x, in, Ax, Bx, An, more);
    }
    if (more) {
      if (multi) {
        // arm the barrier of the exchange after the next group, then wait for this one
        if (tid == 0 && grp + 2 < groups) mbar_arm(x ? &bar[1] : &bar[0], 2 * HQ * (int)sizeof(double));
        mbar_wait_bounded(x ? &bar[0] : &bar[1], x ? ph0 : ph1, status);
        if (x) ph0 ^= 1u; else ph1 ^= 1u;
        __syncthreads();
      } else {
        __syncthreads();
        for (int q = tid; q < 2 * HQ; q += blockDim.x) {
          const int pp = q < HQ ? q - HQ : cnt + (q - HQ);
          An[pp] = An[((pp % n) + n) % n];
        }
        __syncthreads();
      }
    }
  }
  if (Jdev) {
    const double part = block_sum(t.jp, red + 16);
    if (multi) {
      double* r0 = cl.map_shared_rank(red, 0);
      if (tid == 0) r0[rank] = part;
      cl.sync();
    } else if (tid == 0) {
      red[0] = part;
    }
    if (rank == 0 && tid == 0) {
      double J = 0.0;
      for (int r = 0; r < C; ++r) J += red[r];
      J *= dt / T;
      *Jdev = J;
      if (!isfinite(J)) set_status(status, PXA_ERR_NONFINITE);
    }
  }
  if (multi) cl.sync();  // no CTA leaves while a neighbour could still address it
}

// ---- register wavefront form of the same sweep ---------------------------------------
// The lane's points live in registers, one per thread. Warp w of a CTA holds the 32
// consecutive local points p = base_w + lane, base_w = 24 w - 4Q, and keeps valid the
// 24 points of lanes 4..27: the four stages of one RK4 step shrink the valid range by
// one point per side and stage, so a stage takes its neighbours' values by warp
// shuffles, and each step ends at one block barrier where every warp passes its first
// and last 4 valid values to the adjacent warps through shared memory (double-buffered
// by step parity, so one barrier per step suffices). All four SM sub-partitions get one
// warp each at C2's size (64 points per CTA, Q = 4: 4 warps), where the shared-memory
// form runs 3 warps and four barriers per step. After a group of Q steps each CTA sends
// its first and last 4Q values to its cluster neighbours with st.async (double-buffered
// by group parity, completing on the receiver's mbarrier), exactly like
// bu1_rk4_sweep_kernel; a single CTA wraps its own values around the periodic grid.
constexpr int WF_OWN = 24;

template <bool FORCED, int Q>
__global__ void bu1_rk4_wave_kernel(int n, double b, double a, double dt, int k,
                                    const double* __restrict__ f, const double* __restrict__ sc,
                                    const double* __restrict__ x0, double* __restrict__ out,
                                    int lane_rows, const double* __restrict__ gt, double T,
                                    double* __restrict__ Jdev, double* __restrict__ ckpt,
                                    int ck_every, int* status) {
  constexpr int HQ = 4 * Q;  // halo of a group
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double sm[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ double red[56];  // [0, 16): the cluster's partial sums; [16, 56): block_sum scratch
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int nc = (n + C - 1) / C, start = rank * nc, cnt = min(nc, n - start);
  const int lane = (int)(blockIdx.x / C);
  const int s0 = lane * k;
  const int W = (int)(blockDim.x >> 5), warp = (int)(threadIdx.x >> 5), ln = (int)(threadIdx.x & 31);
  double* const xb = sm;           // [2 step parity][W][8]: first 4 and last 4 valid values
  double* const rb = sm + 16 * W;  // [2 group parity][2 side][HQ]: received halos
  const bool multi = C > 1;
  const int left = (rank + C - 1) % C, right = (rank + 1) % C;
  const int cnt_left = min(nc, n - left * nc);
  const int p = WF_OWN * warp - HQ + ln;  // local point of this thread
  const bool own = ln >= 4 && ln < 4 + WF_OWN && p >= 0 && p < cnt;
  const int gi = ((start + p) % n + n) % n;
  const double fp = f[gi];
  const double gp = (own && gt) ? gt[start + p] : 0.0;
  const double a2 = 2.0 * a, h2 = 0.5 * dt, dt6 = dt / 6.0;
  // halo slots this thread fills in the neighbours (own boundary points) and reads here
  const bool to_left = own && p < HQ, to_right = own && p >= cnt - HQ;
  const int in_left = p + HQ;   // 0 <= in_left < HQ: point p of the left halo
  const int in_right = p - cnt; // 0 <= in_right < HQ: point p of the right halo
  uint32_t rl0 = 0u, rl1 = 0u, rr0 = 0u, rr1 = 0u, bl0 = 0u, bl1 = 0u, br0 = 0u, br1 = 0u;
  if (multi && threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (multi && to_left) {  // my point p (< HQ) is point cnt_left + p of the left neighbour
    rl0 = map_rank(smem_u32(rb + 1 * HQ + p), left);
    rl1 = map_rank(smem_u32(rb + 3 * HQ + p), left);
    bl0 = map_rank(smem_u32(&bar[0]), left);
    bl1 = map_rank(smem_u32(&bar[1]), left);
  }
  if (multi && to_right) {  // my point p (>= cnt - HQ) is point p - cnt of the right neighbour
    rr0 = map_rank(smem_u32(rb + 0 * HQ + (p - (cnt - HQ))), right);
    rr1 = map_rank(smem_u32(rb + 2 * HQ + (p - (cnt - HQ))), right);
    br0 = map_rank(smem_u32(&bar[0]), right);
    br1 = map_rank(smem_u32(&bar[1]), right);
  }
  double u = x0 ? x0[(size_t)lane * n + gi] : 0.0;
  if (own) {
    if (out) out[((size_t)lane * lane_rows) * n + start + p] = u;
    if (ckpt && s0 % ck_every == 0) ckpt[(size_t)(s0 / ck_every) * n + start + p] = u;
  }
  int ck_left = ckpt ? ck_every - (s0 % ck_every) : 0;  // steps until the next checkpoint
  int ck_row = ckpt ? s0 / ck_every + 1 : 0;             // row of the next checkpoint
  double* orow = (out && own) ? out + ((size_t)lane * lane_rows + 1) * n + start + p : nullptr;
  const int groups = (k + Q - 1) / Q;
  if (multi) {
    if (threadIdx.x == 0) {
      if (groups > 1) mbar_arm(&bar[0], 2 * HQ * (int)sizeof(double));
      if (groups > 2) mbar_arm(&bar[1], 2 * HQ * (int)sizeof(double));
    }
    cl.sync();  // every CTA's barriers exist before any st.async targets them
  }
  // s(t) at the stage times of the current step; the next step's are loaded a step ahead
  double c1 = 1.0, c2 = 1.0, c4 = 1.0;
  if (FORCED) {
    c1 = sc[3 * (size_t)s0];
    c2 = sc[3 * (size_t)s0 + 1];
    c4 = sc[3 * (size_t)s0 + 2];
  }
  const double* scp = FORCED ? sc + 3 * ((size_t)s0 + 1) : nullptr;
  uint32_t ph0 = 0u, ph1 = 0u;
  double jp = 0.0;
  const unsigned FULL = 0xffffffffu;
  // per-thread constants of the step's exchanges, hoisted out of the loop
  const bool put_lo = ln >= 4 && ln < 8, put_hi = ln >= 24 && ln < 28;
  // (indices of lanes that do not access are set to 0: every address stays in bounds)
  const int put_at = put_lo ? warp * 8 + (ln - 4) : put_hi ? warp * 8 + 4 + (ln - 24) : 0;
  const bool get_lo = ln < 4 && warp > 0, get_hi = ln >= 28 && warp < W - 1;
  const int get_at = get_lo ? (warp - 1) * 8 + 4 + ln : get_hi ? (warp + 1) * 8 + (ln - 28) : 0;
  const bool halo_l = in_left >= 0 && in_left < HQ, halo_r = in_right >= 0 && in_right < HQ;
  const int halo_at = halo_l ? in_left : halo_r ? HQ + in_right : 0;  // within rb[2 gx .. 2 gx + 1]
  const bool with_j = Jdev != nullptr && own;
  const bool with_ck = ckpt != nullptr;
  int j = 0;  // steps done
  for (int grp = 0; grp < groups; ++grp) {
    const bool more = grp + 1 < groups;
    const int steps_here = min(Q, k - grp * Q);
    const int gx = grp & 1;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      if (m >= steps_here) break;  // the last group may be shorter (uniform)
      double n1 = 1.0, n2 = 1.0, n4 = 1.0;
      if (FORCED && j + 1 < k) {
        n1 = scp[0];
        n2 = scp[1];
        n4 = scp[2];
        scp += 3;
      }
      const double cf1 = FORCED ? c1 * fp : fp, cf2 = FORCED ? c2 * fp : fp, cf4 = FORCED ? c4 * fp : fp;
      // stage 1
      double ym = __shfl_up_sync(FULL, u, 1), yp = __shfl_down_sync(FULL, u, 1);
      double kk = stage_k(b, a, a2, ym, u, yp, cf1);
      double acc = kk;
      double y = fma(h2, kk, u);
      // stage 2
      ym = __shfl_up_sync(FULL, y, 1);
      yp = __shfl_down_sync(FULL, y, 1);
      kk = stage_k(b, a, a2, ym, y, yp, cf2);
      acc = fma(2.0, kk, acc);
      y = fma(h2, kk, u);
      // stage 3
      ym = __shfl_up_sync(FULL, y, 1);
      yp = __shfl_down_sync(FULL, y, 1);
      kk = stage_k(b, a, a2, ym, y, yp, cf2);
      acc = fma(2.0, kk, acc);
      y = fma(dt, kk, u);
      // stage 4
      ym = __shfl_up_sync(FULL, y, 1);
      yp = __shfl_down_sync(FULL, y, 1);
      kk = stage_k(b, a, a2, ym, y, yp, cf4);
      const double un = fma(dt6, acc + kk, u);
      if (FORCED) {
        c1 = n1;
        c2 = n2;
        c4 = n4;
      }
      const bool group_end = more && m == Q - 1;  // compile-time m; `more` uniform
      if (group_end) {
        if (multi) {
          if (to_left) st_async_f64(gx ? rl1 : rl0, un, gx ? bl1 : bl0);
          if (to_right) st_async_f64(gx ? rr1 : rr0, un, gx ? br1 : br0);
        } else {
          if (to_left) rb[(2 * gx + 1) * HQ + p] = un;
          if (to_right) rb[(2 * gx + 0) * HQ + (p - (cnt - HQ))] = un;
        }
      }
      // pass the first and last valid values to the adjacent warps (parity of step j)
      double* const xs = xb + (size_t)((Q % 2 == 0 ? m : grp * Q + m) & 1) * W * 8;
      if (put_lo || put_hi) xs[put_at] = un;
      if (with_j) {
        const double d = un - gp;
        jp = fma(d, d, jp);
      }
      if (orow) {
        *orow = un;
        orow += n;
      }
      if (with_ck) {
        if (own && ck_left == 1) ckpt[(size_t)ck_row * n + start + p] = un;
        if (ck_left == 1) {
          ck_left = ck_every;
          ++ck_row;
        } else {
          --ck_left;
        }
      }
      if (group_end && multi) {
        mbar_wait_bounded(&bar[gx], gx ? ph1 : ph0, status);
        if (gx) ph1 ^= 1u; else ph0 ^= 1u;
      }
      __syncthreads();
      u = (get_lo || get_hi) ? xs[get_at] : un;
      if (group_end) {
        if (halo_l || halo_r) u = rb[2 * gx * HQ + halo_at];
        // re-arm this parity's barrier for the exchange two groups on (every thread has
        // passed its wait of this phase: the block barrier above)
        if (multi && threadIdx.x == 0 && grp + 3 < groups) mbar_arm(&bar[gx], 2 * HQ * (int)sizeof(double));
      }
      ++j;
    }
  }
  if (Jdev) {
    const double part = block_sum(jp, red + 16);
    if (multi) {
      double* r0 = cl.map_shared_rank(red, 0);
      if (threadIdx.x == 0) r0[rank] = part;
      cl.sync();
    } else if (threadIdx.x == 0) {
      red[0] = part;
    }
    if (rank == 0 && threadIdx.x == 0) {
      double J = 0.0;
      for (int r = 0; r < C; ++r) J += red[r];
      J *= dt / T;
      *Jdev = J;
      if (!isfinite(J)) set_status(status, PXA_ERR_NONFINITE);
    }
  }
  if (multi) cl.sync();  // no CTA leaves while a neighbour could still address it
}

// Warps of the register wavefront for CTAs of nc points in clusters of C and groups of
// Q steps; 0 when the shared-memory form must run instead: more than 32 warps, or a
// single CTA whose grid is shorter than the 4Q-point halo (the halo would wrap around
// the periodic grid more than once).
static int wave_warps(int nc, int C, int q) {
  if (C == 1 && nc < 4 * q) return 0;
  const int w = (nc + 8 * (q - 1) + WF_OWN - 1) / WF_OWN;
  return w <= 32 ? w : 0;
}

// Steps per exchange Q in {1, 2, 4}: every CTA must own the 4Q-point halo its neighbours
// need and the threads (chunk + 2 (4Q - 1) points) must fit in one CTA; among those, the
// Q with the least estimated time per step (27 FP64 warp instructions per step at 64
// cycles on each of the 4 SM sub-partitions, ~600 cycles per exchange).
static bool rk4_group_ok(int n, int C, int q) {
  const int nc = (n + C - 1) / C, last = n - (C - 1) * nc;
  if (nc + 2 * (4 * q - 1) > 1024) return false;
  if (q > 1 && C > 1 && last < 4 * q) return false;
  if (q > 1 && C == 1 && n < 4 * q) return false;
  return true;
}

static int rk4_group(int n, int C, int want) {
  if (want == 4 || want == 2 || want == 1)
    for (int q = want; q >= 1; q /= 2)
      if (rk4_group_ok(n, C, q)) return q;
  const int nc = (n + C - 1) / C;
  int best = 1;
  double best_cost = 1e30;
  for (int q : {1, 2, 4}) {
    const int npts = nc + 2 * (4 * q - 1);
    if (!rk4_group_ok(n, C, q)) continue;
    const int ww = wave_warps(nc, C, q);
    const int warps = ww > 0 ? ww : (npts + 31) / 32;
    const double cost = (double)((warps + 3) / 4) * 27 * 64 + (C > 1 ? 600.0 : 100.0) / q;
    if (cost < best_cost) {
      best_cost = cost;
      best = q;
    }
  }
  return best;
}

bool bu1_rk4_valid_cluster(int n, int C) {
  if (C < 1 || C > 16) return false;
  const int nc = (n + C - 1) / C;
  if (nc + 6 > 1024) return false;
  if (C == 1) return true;
  return n - (C - 1) * nc >= HX;  // every CTA owns the 4 points a neighbour needs
}

// out = sum of parts[0..count) in order (one thread); NONFINITE status if not finite.
__global__ void sum_parts_kernel(int count, const double* __restrict__ parts, double* __restrict__ out,
                                 int* status) {
  double s = 0.0;
  for (int i = 0; i < count; ++i) s += parts[i];
  *out = s;
  if (!isfinite(s)) set_status(status, PXA_ERR_NONFINITE);
}

// The tracking objective from stored rows (Eq. cost, rectangle rule): one warp per row s
// in [s0, s1) writes Jrow[s] = sum_i (u_s,i - g_i)^2 (lane-strided sums, then a fixed
// shuffle tree: deterministic). With every row of the trajectory stored this takes the
// objective's two FP64 instructions per point and step off the serial direct's path.
__global__ void bu1_objective_rows_kernel(const double* __restrict__ traj, const double* __restrict__ g, int n,
                                          int64_t s0, int64_t s1, double* __restrict__ Jrow) {
  const int64_t s = s0 + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int ln = threadIdx.x & 31;
  if (s >= s1) return;
  const double* row = traj + (size_t)s * n;
  double acc = 0.0;
  for (int i = ln; i < n; i += 32) {
    const double d = row[i] - g[i];
    acc = fma(d, d, acc);
  }
  acc = warp_sum(acc);
  if (ln == 0) Jrow[s] = acc;
}

// J = scale * sum_{s=1..K} Jrow[s]: each thread sums a contiguous run of rows, then a
// fixed block tree (the order does not depend on how the rows were produced).
__global__ void bu1_objective_sum_kernel(const double* __restrict__ Jrow, int64_t K, double scale,
                                         double* __restrict__ Jdev, int* status) {
  __shared__ double red[40];
  const int64_t per = (K + blockDim.x - 1) / blockDim.x;
  const int64_t a = 1 + (int64_t)threadIdx.x * per, b = min(K + 1, a + per);
  double acc = 0.0;
  for (int64_t s = a; s < b; ++s) acc += Jrow[s];
  const double J = scale * block_sum(acc, red);
  if (threadIdx.x == 0) {
    *Jdev = J;
    if (!isfinite(J)) set_status(status, PXA_ERR_NONFINITE);
  }
}

cudaError_t launch_bu1_objective_rows(cudaStream_t st, const double* traj, const double* g, int n, int64_t s0,
                                      int64_t s1, double* Jrow, int priority) {
  if (s1 <= s0) return cudaSuccess;
  const int64_t blocks = (s1 - s0 + 7) / 8;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = priority;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bu1_objective_rows_kernel, traj, g, n, s0, s1, Jrow);
}

cudaError_t launch_bu1_objective_sum(cudaStream_t st, const double* Jrow, int64_t K, double scale, double* Jdev,
                                     int* status) {
  bu1_objective_sum_kernel<<<1, 256, 0, st>>>(Jrow, K, scale, Jdev, status);
  return cudaGetLastError();
}

// The failure path of the bounded waits, for tests: one thread block waits on an
// mbarrier that nothing completes (one expected arrival that never comes, no copy is
// issued, no peer exists), so the wait runs out after the context's wait limit and sets
// PXA_ERR_TIMEOUT. Nothing targets the block's shared memory, so it may leave then.
__global__ void wait_probe_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  mbar_wait_bounded(&bar, 0u, status);
}

cudaError_t launch_wait_probe(cudaStream_t st, int* status) {
  wait_probe_kernel<<<1, 32, 0, st>>>(status);
  return cudaGetLastError();
}

cudaError_t launch_sum_parts(cudaStream_t st, int count, const double* parts, double* out, int* status) {
  sum_parts_kernel<<<1, 1, 0, st>>>(count, parts, out, status);
  return cudaGetLastError();
}

cudaError_t launch_bu1_forcing_table(cudaStream_t st, int64_t K, double dt, double omega, double* sc) {
  const unsigned blocks = (unsigned)((K + 255) / 256);
  bu1_forcing_table_kernel<<<blocks, 256, 0, st>>>(K, dt, omega, sc);
  return cudaGetLastError();
}

template <bool FORCED, int Q>
static cudaError_t launch_rk4_q(cudaStream_t st, int C, int lanes, int nc, void** args,
                                int priority, size_t reserve) {
  const int W = wave_warps(nc, C, Q);
  size_t sh = W > 0 ? sizeof(double) * (16 * (size_t)W + 16 * Q)
                    : sizeof(double) * (6 * (size_t)(nc + 8 * Q) + 64);
  if (reserve > sh) sh = reserve;
  const void* fn = W > 0 ? (const void*)bu1_rk4_wave_kernel<FORCED, Q> : (const void*)bu1_rk4_sweep_kernel<FORCED, Q>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  const int npts = nc + 2 * (4 * Q - 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * lanes);
  cfg.blockDim = dim3(W > 0 ? 32 * W : ((npts + 31) / 32) * 32);
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

cudaError_t launch_bu1_rk4_sweep(cudaStream_t st, int C, int lanes, int n, double L, double nu,
                                 double dt, int64_t k, const double* f, const double* sc,
                                 const double* x0, double* out, int64_t lane_rows, const double* gt,
                                 double T, double* Jdev, double* ckpt, int64_t ck_every,
                                 int* status, int priority, size_t reserve_smem, int group) {
  const double h = L / n;
  double b = 1.0 / (2.0 * h), a = nu / (h * h);
  const int nc = (n + C - 1) / C;
  // step counts and row indices fit in int (K < 2^31); element offsets use size_t
  int ki = (int)k, lr = (int)lane_rows, ce = (int)ck_every;
  void* args[] = {&n, &b, &a, &dt, &ki, &f, &sc, &x0, &out, &lr, &gt, &T, &Jdev,
                  &ckpt, &ce, &status};
  const int q = rk4_group(n, C, group);
  if (sc) {
    if (q == 4) return launch_rk4_q<true, 4>(st, C, lanes, nc, args, priority, reserve_smem);
    if (q == 2) return launch_rk4_q<true, 2>(st, C, lanes, nc, args, priority, reserve_smem);
    return launch_rk4_q<true, 1>(st, C, lanes, nc, args, priority, reserve_smem);
  }
  if (q == 4) return launch_rk4_q<false, 4>(st, C, lanes, nc, args, priority, reserve_smem);
  if (q == 2) return launch_rk4_q<false, 2>(st, C, lanes, nc, args, priority, reserve_smem);
  return launch_rk4_q<false, 1>(st, C, lanes, nc, args, priority, reserve_smem);
}

}  // namespace pxa
