// kernels_ad2_roll.cu — 2D advection-diffusion RK4 steps (dq/dt = A q + s(t) f, FP32) for
// many lanes as a register wavefront: one warp per (lane, 64-column strip, row segment),
// with no block-level barrier.
//
// Thread t of a warp holds columns 2t, 2t+1 of its strip. The warp walks down the rows;
// when input row i arrives, stage 1 is evaluated on row i-1, stage 2 on row i-2,
// stage 3 on row i-3 and the final combination on row i-4, each from the previous
// stage's values on three consecutive rows held in registers (ring buffers indexed at
// compile time: the row loop is unrolled by 8) and from the horizontal neighbours,
// obtained by warp shuffles. Every stage invalidates one more column at each strip
// edge, so a strip of 64 input columns yields 56 output columns; segments overlap by 4
// rows on each side.
//
// Rows arrive through a per-warp shared-memory ring of blocks of AD2_ROLL_BR rows: one
// lane issues two TMA copies per block (cp.async.bulk.tensor: the state rows of its lane
// and the u, v, f rows) completing on the block's mbarrier, NB-1 blocks ahead, so DRAM
// latency is hidden without registers. The step then moves 8 bytes per point and step
// through HBM (state read + write); the coefficient fields are shared by all lanes and
// come from L2. This is the stencil of Eq. linInhomEqus / Eq. seriesDirect for the 2D
// problem of Sec. 4.2.
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels_ad2.cuh"

namespace pxa {

namespace {

constexpr int RS = 56;      // output columns per strip (64 input columns, 4 lost per side)
// one warp (one task) per block, 16 blocks per SM (124 registers, rings 144 KB): a block's
// resources free as soon as its task ends. Measured at 64 lanes x 2048^2: 3670 GB/s against
// 3083 (8 warps x 2 blocks), 3159 (2 x 8), 3307 (1 x 20, 96 registers) and 1987 (1 x 24)
constexpr int RWARPS = 1;   // warps (independent tasks) per CTA
constexpr int RBLOCKS_PER_SM = 16;
constexpr int BR = AD2_ROLL_BR;
constexpr int NB = 2;       // ring blocks per warp (one in flight while the other is read)
constexpr int BLOCK_FLOATS = 4 * BR * 64;  // state + u, v, f rows of one block
constexpr int RING_FLOATS = NB * BLOCK_FLOATS;
static_assert(8 % BR == 0, "blocks align with the 8-row unrolled body");

// Two FP32 values in one 64-bit register pair: the thread's points 2t (low) and 2t+1
// (high). Blackwell's packed FP32x2 instructions (fma/mul/add .rn.f32x2) round each half
// exactly as the scalar instruction would and halve the instruction count.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float lo_of(f2 v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return lo;
}
__device__ __forceinline__ float hi_of(f2 v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return hi;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

struct Coef2 {  // stencil coefficients of the thread's two points on one row
  f2 e, w, n, s, f;
};

// cE = d - a u, cW = d + a u, cN = d - a v, cS = d + a v (a = 1/(2h), d = nu/h^2)
__device__ __forceinline__ void make_coef(Coef2& c, f2 u, f2 v, f2 f, f2 A, f2 mA, f2 D) {
  c.e = fma2(u, mA, D);
  c.w = fma2(u, A, D);
  c.n = fma2(v, mA, D);
  c.s = fma2(v, A, D);
  c.f = f;
}

// k = (A x) + c f at the thread's two points of the centre row x (neighbours xs below,
// xn above, horizontal ones by shuffle).
__device__ __forceinline__ f2 stage_k2(const Coef2& c, f2 CC, f2 CS, f2 x, f2 xs, f2 xn) {
  const float x0 = lo_of(x), x1 = hi_of(x);
  const float w0 = __shfl_up_sync(0xffffffffu, x1, 1);    // column 2t-1
  const float e1 = __shfl_down_sync(0xffffffffu, x0, 1);  // column 2t+2
  f2 k = mul2(c.e, pk(x1, e1));
  k = fma2(c.w, pk(w0, x0), k);
  k = fma2(c.n, xn, k);
  k = fma2(c.s, xs, k);
  k = fma2(CC, x, k);
  return fma2(CS, c.f, k);
}

// Store a new value of domain point (x, y) and its periodic ghost copies.
__device__ __forceinline__ void put_point(float* dst, int Wp, int nx, int ny, int x, int y, float val) {
  const int X = x + G2, Y = y + G2;
  dst[(size_t)Y * Wp + X] = val;
  const bool xl = x < G2, xh = x >= nx - G2, yl = y < G2, yh = y >= ny - G2;
  if (!(xl | xh | yl | yh)) return;
  const int Xa = xl ? X + nx : X - nx;
  const int Ya = yl ? Y + ny : Y - ny;
  const bool hx = xl | xh, hy = yl | yh;
  if (hx) dst[(size_t)Y * Wp + Xa] = val;
  if (hy) dst[(size_t)Ya * Wp + X] = val;
  if (hx && hy) dst[(size_t)Ya * Wp + Xa] = val;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tma3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
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

struct RollTask {
  int X0, Y0, l, buf_in, lanes;
};

// Issue the copies of row block b (rows b*BR ..) into ring slot `slot` (lane 0 only).
__device__ __forceinline__ void issue_block(const CUtensorMap* qmap, const CUtensorMap* cmap,
                                            const RollTask& tk, float* ring, uint64_t* bars, int b,
                                            int slot) {
  float* dst = ring + slot * BLOCK_FLOATS;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bars[slot])),
               "r"((int)(BLOCK_FLOATS * sizeof(float)))
               : "memory");
  tma3d(dst, qmap, tk.X0, tk.Y0 + b * BR, tk.buf_in * tk.lanes + tk.l, &bars[slot]);
  tma3d(dst + BR * 64, cmap, tk.X0, tk.Y0 + b * BR, 0, &bars[slot]);
}

// The wavefront of one task. INNER: every output point is away from the periodic ghost
// layers (plain 8-byte stores).
template <bool INNER>
__device__ __forceinline__ void roll_task(const CUtensorMap* qmap, const CUtensorMap* cmap,
                                          const Ad2Params& p, const RollTask& tk, float* qo,
                                          float* ring, uint64_t* bars, int Hs, float c1, float c2,
                                          float c4, int* status) {
  const int t = threadIdx.x & 31;
  const float a = p.inv2h, d = p.nu * p.invh2;
  const f2 A = pk(a, a), mA = pk(-a, -a), D = pk(d, d), CC = pk(-4.0f * d, -4.0f * d);
  const f2 C1 = pk(c1, c1), C2 = pk(c2, c2), C4 = pk(c4, c4);
  const f2 DT = pk(p.dt, p.dt), HDT = pk(0.5f * p.dt, 0.5f * p.dt), SDT = pk(p.dt / 6.0f, p.dt / 6.0f);
  const f2 TWO = pk(2.0f, 2.0f);
  const bool out_col = t >= 2 && t < 30;  // strip columns 4 .. 59
  const int xd = tk.X0 - G2 + 2 * t;      // domain column of the thread's first point
  const int rows = Hs + 8, nblocks = rows / BR;
  f2 Q[8], Y1[4], Y2[4], Y3[4], ACC[4];
  Coef2 CF[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) Y1[j] = Y2[j] = Y3[j] = ACC[j] = 0ull;
  if (t == 0)
    for (int b = 0; b < NB - 1 && b < nblocks; ++b) issue_block(qmap, cmap, tk, ring, bars, b, b);
  // padded position of output row 0 (domain row Y0); the pointer walks down one row per
  // input row from row 8 on
  float* orow = qo + (size_t)(tk.Y0 + G2) * p.Wp + xd + G2;
  bool ok = true;
  for (int i0 = 0; i0 < rows; i0 += 8) {
#pragma unroll
    for (int I = 0; I < 8; ++I) {
      const int i = i0 + I;
      constexpr int slot_of_I[8] = {0, 0, 0, 0, 1, 1, 1, 1};  // (i / BR) % NB with BR = 4, NB = 2
      if (I % BR == 0) {
        // a new block: refill the slot of the block just finished, then wait for this one
        const int b = i / BR;
        __syncwarp();
        if (t == 0 && b + NB - 1 < nblocks) {
          // order the lanes' generic-proxy reads of that slot before the TMA overwrite
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue_block(qmap, cmap, tk, ring, bars, b + NB - 1, (b + NB - 1) % NB);
        }
        ok &= bar_wait(&bars[slot_of_I[I]], (uint32_t)((b / NB) & 1));
      }
      const float* src = ring + slot_of_I[I] * BLOCK_FLOATS + (I % BR) * 64 + 2 * t;
      Q[I] = *reinterpret_cast<const f2*>(src);
      const f2 un = *reinterpret_cast<const f2*>(src + BR * 64);
      const f2 vn = *reinterpret_cast<const f2*>(src + 2 * BR * 64);
      const f2 fn = *reinterpret_cast<const f2*>(src + 3 * BR * 64);
      // stage 1 on row i-1: neighbours q rows i-2, i
      {
        const f2 x = Q[(I + 7) & 7];
        const f2 k = stage_k2(CF[(I + 3) & 3], CC, C1, x, Q[(I + 6) & 7], Q[I]);
        Y1[(I + 3) & 3] = fma2(HDT, k, x);
        ACC[(I + 3) & 3] = k;
      }
      // stage 2 on row i-2
      {
        const f2 k = stage_k2(CF[(I + 2) & 3], CC, C2, Y1[(I + 2) & 3], Y1[(I + 1) & 3], Y1[(I + 3) & 3]);
        Y2[(I + 2) & 3] = fma2(HDT, k, Q[(I + 6) & 7]);
        ACC[(I + 2) & 3] = fma2(TWO, k, ACC[(I + 2) & 3]);
      }
      // stage 3 on row i-3
      {
        const f2 k = stage_k2(CF[(I + 1) & 3], CC, C2, Y2[(I + 1) & 3], Y2[I & 3], Y2[(I + 2) & 3]);
        Y3[(I + 1) & 3] = fma2(DT, k, Q[(I + 5) & 7]);
        ACC[(I + 1) & 3] = fma2(TWO, k, ACC[(I + 1) & 3]);
      }
      // stage 4 on row i-4: q_new = q + dt/6 (k1 + 2 k2 + 2 k3 + k4)
      {
        const f2 k = stage_k2(CF[I & 3], CC, C4, Y3[I & 3], Y3[(I + 3) & 3], Y3[(I + 1) & 3]);
        const f2 qn = fma2(SDT, add2(ACC[I & 3], k), Q[(I + 4) & 7]);
        if (i0 >= 8) {  // output row i - 8 of the segment
          if (out_col) {
            if (INNER) {
              *reinterpret_cast<f2*>(orow) = qn;
            } else {
              const int yd = tk.Y0 + i - 8;
              put_point(qo, p.Wp, p.nx, p.ny, xd, yd, lo_of(qn));
              put_point(qo, p.Wp, p.nx, p.ny, xd + 1, yd, hi_of(qn));
            }
          }
          orow += p.Wp;
        }
      }
      make_coef(CF[I & 3], un, vn, fn, A, mA, D);  // row i (slot of row i-4, used above for the last time)
    }
  }
  if (!ok) {
    if (t == 0) set_status(status, PXA_ERR_TIMEOUT);
    // a copy whose wait gave up may still be in flight: wait (bounded again) for the last
    // block issued to each ring slot before the warp's next task or the block's exit
    for (int s = 0; s < NB && s < nblocks; ++s) {
      const int last = s + NB * ((nblocks - 1 - s) / NB);  // the last block of slot s
      (void)bar_wait(&bars[s], (uint32_t)((last / NB) & 1));
    }
  }
}

// ---- reverse steps of the exact discrete adjoint for many lanes ----------------------
// One reverse step of the transposed RK4 map (the adjoint lanes of Eq. hybadjinhom):
// kbar4 = dt/6 lambda; Y3 = A^T kbar4, kbar3 = dt/3 lambda + dt Y3; Y2 = A^T kbar3,
// kbar2 = dt/3 lambda + dt/2 Y2; Y1 = A^T kbar2, kbar1 = dt/6 lambda + dt/2 Y1;
// lambda_new = lambda + Y3 + Y2 + Y1 + A^T kbar1 (+ the objective's source); the forcing
// gradient gains c4 kbar4 + c2 kbar3 + c2 kbar2 + c1 kbar1 (Eq. paramupdate), accumulated in
// FP32 over the lane's steps (FP32 stepping with FP32 accumulation; the lanes are summed in
// FP64 afterwards).
// The same wavefront as the forward step: stage A on row i-1, B on i-2, C on i-3, D on
// i-4, every A^T from the rows of the previous stage held in registers. A block of rows
// brings, by four TMA copies on one mbarrier, the lambda rows, the four A^T coefficient
// rows (tE, tW, tN, tS), and, eight rows behind (the rows that stage D finishes), the
// source rows of the lane's step and its FP64 gradient rows.

constexpr int TB_FLOATS = 7 * BR * 64;    // lambda, 4 coefficient planes, source, FP32 gradient
constexpr int TRING_FLOATS = NB * TB_FLOATS;
// one warp (one task) per block, 14 blocks per SM (their rings fill 215 KB of shared
// memory; 123 registers): 14 warps per SM where 4-warp blocks fit 3 (12 warps, 164
// registers), and a block's resources free as soon as its one task ends. Measured on C3's
// 64 lanes: 1.38 ms against 1.49 (4 x 3), 1.55 (2 x 8) and 1.63 ms (4 x 4)
constexpr int TWARPS = 1;
constexpr int TBLOCKS_PER_SM = 14;

struct CoefT2 {  // A^T coefficients of the thread's two points on one row
  f2 e, w, n, s;
};

// (A^T x) at the thread's two points of the centre row x (neighbours xs below, xn above).
__device__ __forceinline__ f2 stage_t2(const CoefT2& c, f2 CC, f2 x, f2 xs, f2 xn) {
  const float x0 = lo_of(x), x1 = hi_of(x);
  const float w0 = __shfl_up_sync(0xffffffffu, x1, 1);    // column 2t-1
  const float e1 = __shfl_down_sync(0xffffffffu, x0, 1);  // column 2t+2
  f2 k = mul2(c.e, pk(x1, e1));
  k = fma2(c.w, pk(w0, x0), k);
  k = fma2(c.n, xn, k);
  k = fma2(c.s, xs, k);
  return fma2(CC, x, k);
}

struct RollTTask {
  int X0, Y0, l, buf_in, lanes, zsrc, own_x0, own_y0;
};

__device__ __forceinline__ void issue_tblock(const CUtensorMap* qmap, const CUtensorMap* tmap,
                                             const CUtensorMap* smap, const CUtensorMap* gmap,
                                             const RollTTask& tk, float* ring, uint64_t* bars, int b,
                                             int slot) {
  float* dst = ring + slot * TB_FLOATS;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bars[slot])),
               "r"((int)(TB_FLOATS * sizeof(float)))
               : "memory");
  const int yrow = tk.Y0 + b * BR;
  tma3d(dst, qmap, tk.X0, yrow, tk.buf_in * tk.lanes + tk.l, &bars[slot]);
  tma3d(dst + BR * 64, tmap, tk.X0, yrow, 0, &bars[slot]);
  // domain coordinates of the rows stage D finishes in this block: padded row - 2 G2
  tma3d(dst + 5 * BR * 64, smap, tk.X0 - G2, yrow - 2 * G2, tk.zsrc, &bars[slot]);
  tma3d(dst + 6 * BR * 64, gmap, tk.X0 - G2, yrow - 2 * G2, tk.l, &bars[slot]);
}

template <bool INNER>
__device__ __forceinline__ void rollT_task(const CUtensorMap* qmap, const CUtensorMap* tmap,
                                           const CUtensorMap* smap, const CUtensorMap* gmap,
                                           const Ad2Params& p, const RollTTask& tk, float* qo,
                                           float* G, float* ring, uint64_t* bars, int Hs, float c1,
                                           float c2, float c4, float src_scale, bool add_src,
                                           int* status) {
  const int t = threadIdx.x & 31;
  const float d = p.nu * p.invh2, h = p.dt;
  const f2 CC = pk(-4.0f * d, -4.0f * d);
  const f2 H = pk(h, h), H2 = pk(0.5f * h, 0.5f * h), H3 = pk(h / 3.0f, h / 3.0f), H6 = pk(h / 6.0f, h / 6.0f);
  const f2 C1 = pk(c1, c1), C2 = pk(c2, c2), C4H6 = pk(c4 * (h / 6.0f), c4 * (h / 6.0f));
  const f2 SRC = pk(src_scale, src_scale);
  const bool out_col = t >= 2 && t < 30;  // strip columns 4 .. 59
  const int xd = tk.X0 - G2 + 2 * t;      // domain column of the thread's first point
  const bool own_col = out_col && xd >= tk.own_x0;  // gradient points this task updates
  const int rows = Hs + 8, nblocks = rows / BR;
  f2 Q[4], KB3[4], KB2[4], KB1[4], LN[4], GG[4];
  CoefT2 CT[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) Q[j] = KB3[j] = KB2[j] = KB1[j] = LN[j] = GG[j] = 0ull;
  if (t == 0)
    for (int b = 0; b < NB - 1 && b < nblocks; ++b) issue_tblock(qmap, tmap, smap, gmap, tk, ring, bars, b, b);
  float* orow = qo + (size_t)(tk.Y0 + G2) * p.Wp + xd + G2;
  float* grow = G + ((size_t)tk.l * p.ny + tk.Y0) * p.nx + xd;
  bool ok = true;
  // one block of BR = 4 rows per iteration (the row registers are 4-rings, so the body is
  // unrolled 4 times, not 8: half the code, fewer instruction-cache misses)
  static_assert(BR == 4, "one ring block per 4-row iteration");
  for (int i0 = 0; i0 < rows; i0 += BR) {
    const int b = i0 / BR, slot = b % NB;
    __syncwarp();
    if (t == 0 && b + NB - 1 < nblocks) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_tblock(qmap, tmap, smap, gmap, tk, ring, bars, b + NB - 1, (b + NB - 1) % NB);
    }
    ok &= bar_wait(&bars[slot], (uint32_t)((b / NB) & 1));
    const float* blk = ring + slot * TB_FLOATS + 2 * t;
#pragma unroll
    for (int I = 0; I < BR; ++I) {
      const int i = i0 + I;
      const float* src = blk + I * 64;
      Q[I & 3] = *reinterpret_cast<const f2*>(src);
      const f2 te = *reinterpret_cast<const f2*>(src + BR * 64);
      const f2 tw = *reinterpret_cast<const f2*>(src + 2 * BR * 64);
      const f2 tn = *reinterpret_cast<const f2*>(src + 3 * BR * 64);
      const f2 ts = *reinterpret_cast<const f2*>(src + 4 * BR * 64);
      const f2 sv = *reinterpret_cast<const f2*>(src + 5 * BR * 64);
      const f2 gold = *reinterpret_cast<const f2*>(src + 6 * BR * 64);
      // stage A on row i-1: Y3 = A^T (dt/6 lambda)
      {
        const f2 x = Q[(I + 3) & 3];
        const f2 y3 = mul2(H6, stage_t2(CT[(I + 3) & 3], CC, x, Q[(I + 2) & 3], Q[I & 3]));
        const f2 kb3 = fma2(H, y3, mul2(H3, x));
        KB3[(I + 3) & 3] = kb3;
        LN[(I + 3) & 3] = add2(x, y3);
        GG[(I + 3) & 3] = fma2(C2, kb3, mul2(C4H6, x));
      }
      // stage B on row i-2: Y2 = A^T kbar3
      {
        const f2 y2 = stage_t2(CT[(I + 2) & 3], CC, KB3[(I + 2) & 3], KB3[(I + 1) & 3], KB3[(I + 3) & 3]);
        const f2 kb2 = fma2(H2, y2, mul2(H3, Q[(I + 2) & 3]));
        KB2[(I + 2) & 3] = kb2;
        LN[(I + 2) & 3] = add2(LN[(I + 2) & 3], y2);
        GG[(I + 2) & 3] = fma2(C2, kb2, GG[(I + 2) & 3]);
      }
      // stage C on row i-3: Y1 = A^T kbar2
      {
        const f2 y1 = stage_t2(CT[(I + 1) & 3], CC, KB2[(I + 1) & 3], KB2[I & 3], KB2[(I + 2) & 3]);
        const f2 kb1 = fma2(H2, y1, mul2(H6, Q[(I + 1) & 3]));
        KB1[(I + 1) & 3] = kb1;
        LN[(I + 1) & 3] = add2(LN[(I + 1) & 3], y1);
        GG[(I + 1) & 3] = fma2(C1, kb1, GG[(I + 1) & 3]);
      }
      // stage D on row i-4: lambda_new = Ln + A^T kbar1 (+ source)
      {
        const f2 y0 = stage_t2(CT[I & 3], CC, KB1[I & 3], KB1[(I + 3) & 3], KB1[(I + 1) & 3]);
        f2 lam = add2(LN[I & 3], y0);
        if (add_src) lam = fma2(SRC, sv, lam);
        if (i0 >= 8) {  // output row i - 8 of the segment
          const int yd = tk.Y0 + i - 8;
          if (out_col) {
            if (INNER) {
              *reinterpret_cast<f2*>(orow) = lam;
            } else {
              put_point(qo, p.Wp, p.nx, p.ny, xd, yd, lo_of(lam));
              put_point(qo, p.Wp, p.nx, p.ny, xd + 1, yd, hi_of(lam));
            }
          }
          if (own_col && yd >= tk.own_y0) {
            *reinterpret_cast<f2*>(grow) = add2(gold, GG[I & 3]);
          }
          orow += p.Wp;
          grow += p.nx;
        }
      }
      CT[I & 3].e = te;  // row i (slot of row i-4, used above for the last time)
      CT[I & 3].w = tw;
      CT[I & 3].n = tn;
      CT[I & 3].s = ts;
    }
  }
  if (!ok) {
    if (t == 0) set_status(status, PXA_ERR_TIMEOUT);
    for (int s = 0; s < NB && s < nblocks; ++s) {
      const int last = s + NB * ((nblocks - 1 - s) / NB);
      (void)bar_wait(&bars[s], (uint32_t)((last / NB) & 1));
    }
  }
}

}  // namespace

// s(t) at the three stage times of steps s0 .. s0+count-1: sc[3j + {0,1,2}] (FP64 sin,
// stored as FP32 for the FP32 stepping).
__global__ void ad2_forcing_table_kernel(int64_t s0, int64_t count, double dt, double omega,
                                         float* __restrict__ sc) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const double t = (double)(s0 + j) * dt;
  sc[3 * j + 0] = omega == 0.0 ? 1.0f : (float)sin(omega * t);
  sc[3 * j + 1] = omega == 0.0 ? 1.0f : (float)sin(omega * (t + 0.5 * dt));
  sc[3 * j + 2] = omega == 0.0 ? 1.0f : (float)sin(omega * (t + dt));
}

// One RK4 step for `lanes` lanes: lane l reads buffer buf_in and writes the other; its
// forcing factors are sc[3*l*sc_stride + {0,1,2}]. Hs: output rows per segment (a
// multiple of 8).
__global__ void __launch_bounds__(32 * RWARPS, RBLOCKS_PER_SM) ad2_rk4_roll_kernel(
    const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap cmap, Ad2Params p,
    float* __restrict__ states, int lanes, int buf_in, int nstrips, int nsegs, int Hs,
    const float* __restrict__ sc, int sc_stride, int* status) {
  extern __shared__ __align__(1024) float rsm[];
  __shared__ __align__(8) uint64_t bars[RWARPS * NB];
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int task = blockIdx.x * RWARPS + warp;
  if (task >= lanes * nstrips * nsegs) return;  // whole warps only: no block barrier below
  uint64_t* wb = bars + warp * NB;
  if (t == 0) {
    for (int j = 0; j < NB; ++j)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&wb[j])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  RollTask tk;
  tk.l = task % lanes;
  const int rest = task / lanes;
  const int sx = rest % nstrips, sy = rest / nstrips;
  tk.X0 = min(sx * RS, p.nx - RS);  // first output column (domain) = first input column (padded)
  tk.Y0 = min(sy * Hs, p.ny - Hs);  // first output row (domain) = first input row (padded)
  tk.buf_in = buf_in;
  tk.lanes = lanes;
  const size_t plane = (size_t)p.Hp * p.Wp;
  float* qo = states + ((size_t)(1 - buf_in) * lanes + tk.l) * plane;
  const float* scl = sc + 3 * (size_t)tk.l * sc_stride;
  const float c1 = scl[0], c2 = scl[1], c4 = scl[2];
  float* ring = rsm + (size_t)warp * RING_FLOATS;
  const bool inner = tk.X0 >= G2 && tk.X0 + RS <= p.nx - G2 && tk.Y0 >= G2 && tk.Y0 + Hs <= p.ny - G2;
  if (inner)
    roll_task<true>(&qmap, &cmap, p, tk, qo, ring, wb, Hs, c1, c2, c4, status);
  else
    roll_task<false>(&qmap, &cmap, p, tk, qo, ring, wb, Hs, c1, c2, c4, status);
}

// One reverse step for lanes lane0 .. lane0 + count - 1 of `lanes`: lane l reads buffer
// buf_in and writes the other; it is at absolute step zsrc0 + l * z_stride (its source row
// in the trajectory, and its forcing factors sc[3 (zsrc0 + l * z_stride) + {0, 1, 2}]).
__global__ void __launch_bounds__(32 * TWARPS, TBLOCKS_PER_SM) ad2_rk4T_roll_kernel(
    const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap tmap,
    const __grid_constant__ CUtensorMap smap, const __grid_constant__ CUtensorMap gmap, Ad2Params p,
    float* __restrict__ states, float* __restrict__ G, int lanes, int lane0, int count, int buf_in,
    int nstrips, int nsegs, int Hs, const float* __restrict__ sc, int zsrc0, int z_stride, float src_scale,
    int add_src, int* status) {
  extern __shared__ __align__(1024) float rsm[];
  __shared__ __align__(8) uint64_t bars[TWARPS * NB];
  const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int task = blockIdx.x * TWARPS + warp;
  if (task >= count * nstrips * nsegs) return;  // whole warps only: no block barrier below
  uint64_t* wb = bars + warp * NB;
  if (t == 0) {
    for (int j = 0; j < NB; ++j)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&wb[j])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  RollTTask tk;
  tk.l = lane0 + task % count;
  const int rest = task / count;
  const int sx = rest % nstrips, sy = rest / nstrips;
  tk.X0 = min(sx * RS, p.nx - RS);
  tk.Y0 = min(sy * Hs, p.ny - Hs);
  tk.own_x0 = sx * RS;  // the last strip and segment overlap the previous ones: the points
  tk.own_y0 = sy * Hs;  // before these are that task's to update in G
  tk.buf_in = buf_in;
  tk.lanes = lanes;
  tk.zsrc = zsrc0 + tk.l * z_stride;
  const size_t plane = (size_t)p.Hp * p.Wp;
  float* qo = states + ((size_t)(1 - buf_in) * lanes + tk.l) * plane;
  const float* scl = sc + 3 * (size_t)tk.zsrc;
  const float c1 = scl[0], c2 = scl[1], c4 = scl[2];
  float* ring = rsm + (size_t)warp * TRING_FLOATS;
  const bool inner = tk.X0 >= G2 && tk.X0 + RS <= p.nx - G2 && tk.Y0 >= G2 && tk.Y0 + Hs <= p.ny - G2;
  if (inner)
    rollT_task<true>(&qmap, &tmap, &smap, &gmap, p, tk, qo, G, ring, wb, Hs, c1, c2, c4, src_scale,
                     add_src != 0, status);
  else
    rollT_task<false>(&qmap, &tmap, &smap, &gmap, p, tk, qo, G, ring, wb, Hs, c1, c2, c4, src_scale,
                      add_src != 0, status);
}

int ad2_roll_rows(int ny) {
  int hs = 128;
  while (hs > 8 && hs > ny) hs /= 2;
  return hs;
}

bool ad2_roll_ok(const Ad2Params& p) {
  // 56-column strips and 8-row segments inside the grid; 16-byte TMA x offsets
  return p.nx >= RS && p.ny >= 8 && (p.nx % 4) == 0 && ad2_roll_rows(p.ny) <= p.ny &&
         ad2_roll_rows(p.ny) % 8 == 0;
}

// Rows per segment for a launch of `lanes` lanes: among 128, 64, 32, 16 and 8 rows (at most
// ny), the one with the least estimated time, counted as whole waves of tasks (co-resident
// blocks x warps per block, one task per warp) times the rows one task steps (its segment
// and the 8 rows of overlap). A grid a little above one wave otherwise runs a second,
// mostly empty wave. `per_sm` caches the blocks per SM of the kernel (0: not known yet).
static int roll_rows_for(int nx, int ny, long long lanes, const void* fn, int warps, size_t smem, int& per_sm) {
  int dev = 0, sms = 0;
  if (per_sm == 0) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 32 * warps, smem) != cudaSuccess) {
      cudaGetLastError();
      return ad2_roll_rows(ny);
    }
    per_sm = per;
  }
  if (per_sm <= 0 || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return ad2_roll_rows(ny);
  }
  const long long cap = (long long)per_sm * sms * warps;
  const long long nstrips = (nx + RS - 1) / RS;
  int best = ad2_roll_rows(ny);
  long long best_cost = -1;
  for (int hs = 128; hs >= 8; hs /= 2) {
    if (hs > ny) continue;
    const long long tasks = lanes * nstrips * ((ny + hs - 1) / hs);
    const long long cost = ((tasks + cap - 1) / cap) * (hs + 8);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = hs;
    }
  }
  return best;
}

cudaError_t launch_ad2_forcing_table(cudaStream_t st, int64_t s0, int64_t count, double dt,
                                     double omega, float* sc) {
  if (count <= 0) return cudaSuccess;
  ad2_forcing_table_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(s0, count, dt, omega, sc);
  return cudaGetLastError();
}

cudaError_t launch_ad2_rk4_roll(cudaStream_t st, const CUtensorMap& qmap, const CUtensorMap& cmap,
                                const Ad2Params& p, float* states, int lanes, int buf_in,
                                const float* sc, int sc_stride, int* status) {
  const size_t sh = sizeof(float) * (size_t)RWARPS * RING_FLOATS;
  cudaError_t e = cudaFuncSetAttribute(ad2_rk4_roll_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(ad2_rk4_roll_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  static int per_sm = 0;
  const int Hs = roll_rows_for(p.nx, p.ny, lanes, (const void*)ad2_rk4_roll_kernel, RWARPS, sh, per_sm);
  const int nstrips = (p.nx + RS - 1) / RS, nsegs = (p.ny + Hs - 1) / Hs;
  const long long tasks = (long long)lanes * nstrips * nsegs;
  const unsigned blocks = (unsigned)((tasks + RWARPS - 1) / RWARPS);
  ad2_rk4_roll_kernel<<<blocks, 32 * RWARPS, sh, st>>>(qmap, cmap, p, states, lanes, buf_in, nstrips, nsegs,
                                                       Hs, sc, sc_stride, status);
  return cudaGetLastError();
}

cudaError_t launch_ad2_rk4T_roll(cudaStream_t st, const CUtensorMap& qmap, const CUtensorMap& tmap,
                                 const CUtensorMap& smap, const CUtensorMap& gmap, const Ad2Params& p,
                                 float* states, float* G, int lanes, int lane0, int count, int buf_in,
                                 const float* sc, int zsrc0, int z_stride, float src_scale, int add_src,
                                 int* status) {
  if (count <= 0 || lane0 < 0 || lane0 + count > lanes) return cudaErrorInvalidValue;
  const size_t sh = sizeof(float) * (size_t)TWARPS * TRING_FLOATS;
  cudaError_t e = cudaFuncSetAttribute(ad2_rk4T_roll_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  // the rings of all resident blocks: the largest shared-memory carveout
  e = cudaFuncSetAttribute(ad2_rk4T_roll_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  static int per_sm = 0;
  const int Hs = roll_rows_for(p.nx, p.ny, count, (const void*)ad2_rk4T_roll_kernel, TWARPS, sh, per_sm);
  const int nstrips = (p.nx + RS - 1) / RS, nsegs = (p.ny + Hs - 1) / Hs;
  const long long tasks = (long long)count * nstrips * nsegs;
  const unsigned blocks = (unsigned)((tasks + TWARPS - 1) / TWARPS);
  ad2_rk4T_roll_kernel<<<blocks, 32 * TWARPS, sh, st>>>(qmap, tmap, smap, gmap, p, states, G, lanes, lane0,
                                                         count, buf_in, nstrips, nsegs, Hs, sc, zsrc0, z_stride,
                                                         src_scale, add_src, status);
  return cudaGetLastError();
}

}  // namespace pxa
