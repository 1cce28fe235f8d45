// kernels_bu1_pair.cu — two-step banded adjoint chain for 1D Burgers.
//
// The serial adjoint chain (Eq. adjHomNormal with the stepper's own propagator, and the
// top subinterval with its source) is a recursion lambda_s = M_s^T lambda_{s+1} + r_s
// whose cost per step is dominated by the exchange of halo values between the CTAs of a
// cluster (~660 cycles), not by its 9 FMAs. Taking two steps at once with the product
// band P_s = M_s^T M_{s+1}^T (17 diagonals) and the combined source
// r_s + M_s^T r_{s+1} halves the exchanges:
//
//  - bu1_band_pair_kernel (parallel, run beside the direct solve): forms, for every
//    even row s, the record {P_s[i][i-8..i+8], r_s + (M_s^T r_{s+1})_i}.
//  - bu1_band_chain2_kernel (one cluster): follows a step plan built on the host. A pair
//    step is taken where nothing happens on the row in between (no lane value is added
//    there and the source is on for both rows or for neither); elsewhere a single step
//    with the one-step record. Every step exchanges 8 boundary values per side.
//  - bu1_band_fill_kernel (parallel): the rows skipped inside pair steps,
//    lambda_{s+1} = M_{s+1}^T lambda_{s+2} + r_{s+1}, for the gradient pass.
#include <cooperative_groups.h>

#include "common.cuh"
#include "dsmem.cuh"
#include "kernels_1d.cuh"

namespace cg = cooperative_groups;

namespace pxa {

namespace {

constexpr int RW = BU1_BAND_RECORD;   // one-step record: 9 taps + source
constexpr int PW = BU1_PAIR_RECORD;   // pair record: 17 taps + source
constexpr int HP = 8;                 // halo of a pair step
constexpr int PT2 = 128;              // points per tile of the parallel kernels

__device__ __forceinline__ int wrapn(int g, int n) {
  g %= n;
  return g < 0 ? g + n : g;
}

}  // namespace

// ---- pair records -------------------------------------------------------------------
// Grid (tiles, pair blocks); pair m combines rows 2m and 2m+1 for m in [m_lo, m_hi).
__global__ void __launch_bounds__(PT2) bu1_band_pair_kernel(int n, const double* __restrict__ rec,
                                                            int64_t m_lo, int64_t m_hi, int pairs_per_block,
                                                            double* __restrict__ rp) {
  __shared__ double nxt[(PT2 + 8) * RW];  // records of row 2m+1 on the tile +- 4
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * PT2;
  const int64_t mb = m_lo + (int64_t)blockIdx.y * pairs_per_block;
  int64_t me = mb + pairs_per_block;
  if (me > m_hi) me = m_hi;
  const int pt = i0 + tid;
  for (int64_t m = mb; m < me; ++m) {
    __syncthreads();
    const double* r1 = rec + (size_t)(2 * m + 1) * n * RW;
    for (int e = tid; e < (PT2 + 8) * RW; e += PT2) {
      const int q = e / RW, j = e % RW;
      nxt[e] = r1[(size_t)wrapn(i0 - 4 + q, n) * RW + j];
    }
    __syncthreads();
    if (pt >= n) continue;
    const double* a = rec + ((size_t)(2 * m) * n + pt) * RW;  // row i of M_s^T and r_s
    double ai[RW];
#pragma unroll
    for (int j = 0; j < RW; ++j) ai[j] = a[j];
    double out[PW];
#pragma unroll
    for (int o = 0; o < 17; ++o) out[o] = 0.0;
    double src = ai[RW - 1];
    // (M_s^T M_{s+1}^T)[i][i+o] = sum_e M_s^T[i][i+e] M_{s+1}^T[i+e][i+o]
#pragma unroll
    for (int e = -4; e <= 4; ++e) {
      const double* b = nxt + (tid + 4 + e) * RW;  // row i+e of M_{s+1}^T
      const double w = ai[e + 4];
#pragma unroll
      for (int f = -4; f <= 4; ++f) out[e + f + 8] = fma(w, b[f + 4], out[e + f + 8]);
      src = fma(w, b[RW - 1], src);
    }
    out[17] = src;
    double2* dst = reinterpret_cast<double2*>(rp + ((size_t)m * n + pt) * PW);
#pragma unroll
    for (int j = 0; j < PW / 2; ++j) dst[j] = make_double2(out[2 * j], out[2 * j + 1]);
  }
}

// ---- two-step chain ------------------------------------------------------------------
// plan[j] = {row produced, 1 (single) or 2 (pair), source on, lane index to add (0: none)}.
// lambda_{P k} = r_{P k} is the starting row; rows produced go to out_rows.
//
// Each point's taps are split over two warps on different SM sub-partitions (whose FP64
// units work in parallel): with G = ceil(chunk / 32) point groups, warp w serves group
// w % G and half w / G. Half 0 takes the taps -8..0 and the source, half 1 the taps
// 1..8 (pair steps only); half 1 hands its partial sum over through shared memory at a
// barrier of the two warps, and half 0 finishes, stores and sends the value.
template <int DEPTH>
__global__ void bu1_band_chain2_kernel(int n, const double* __restrict__ rec,
                                       const double* __restrict__ rp, const int4* __restrict__ plan,
                                       int nplan, int s_hi, const double* __restrict__ from_rows,
                                       const double* __restrict__ W, double* __restrict__ out_rows,
                                       int* status) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double smb[];
  __shared__ __align__(8) uint64_t bar[2];
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int nc = (n + C - 1) / C, start = rank * nc, cnt = min(nc, n - start);
  const int G = (nc + 31) / 32;
  const int Wd = nc + 2 * HP;
  double* const lam0 = smb + HP;
  double* const lam1 = smb + Wd + HP;
  double* const part = smb + 2 * Wd;         // [G * 32] partial sums of half 1
  double* const ring = part + G * 32;        // [DEPTH][2 * G * 32][PW]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lanei = tid & 31;
  const int g = warp % G, half = warp / G;
  const int p = g * 32 + lanei;              // this thread's point
  const bool act = p < cnt;
  const bool multi = C > 1;
  const int left = (rank + C - 1) % C, right = (rank + 1) % C;
  const int cnt_left = min(nc, n - left * nc);
  if (multi && tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // lambda_{s_hi}: row s_hi of from_rows (a chain continued from an earlier launch), or
  // the source of the last state, own points and halo
  for (int q = tid - HP; q < cnt + HP; q += nt) {
    const int gq = wrapn(start + q, n);
    const double v = from_rows ? from_rows[(size_t)s_hi * n + gq] : rec[((size_t)s_hi * n + gq) * RW + (RW - 1)];
    lam0[q] = v;
    if (!from_rows && q >= 0 && q < cnt) out_rows[(size_t)s_hi * n + start + q] = v;
  }
  const bool sender = multi && act && half == 0;
  const bool to_left = sender && p < HP, to_right = sender && p >= cnt - HP;
  uint32_t rl0 = 0, rl1 = 0, rr0 = 0, rr1 = 0, bl0 = 0, bl1 = 0, br0 = 0, br1 = 0;
  if (to_left) {
    rl0 = map_rank(smem_u32(lam0 + cnt_left + p), left);
    rl1 = map_rank(smem_u32(lam1 + cnt_left + p), left);
    bl0 = map_rank(smem_u32(&bar[0]), left);
    bl1 = map_rank(smem_u32(&bar[1]), left);
  }
  if (to_right) {
    rr0 = map_rank(smem_u32(lam0 + (p - cnt)), right);
    rr1 = map_rank(smem_u32(lam1 + (p - cnt)), right);
    br0 = map_rank(smem_u32(&bar[0]), right);
    br1 = map_rank(smem_u32(&bar[1]), right);
  }
  double* const my_ring = ring + (size_t)tid * PW;
  const int slot_stride = nt * PW;
  // plan entries of steps j .. j+3 in registers (e0 = step j); the entry of step j+4 is
  // loaded a step ahead of its use by the record prefetch
  const int4 none = make_int4(0, 0, 0, 0);
  int4 e0 = nplan > 0 ? plan[0] : none, e1 = nplan > 1 ? plan[1] : none,
       e2 = nplan > 2 ? plan[2] : none, e3 = nplan > 3 ? plan[3] : none;
  // the 16-byte chunks of a record this warp reads: half 0 the taps -8..0 (chunks 0..4)
  // and the source (chunk 8) of a pair record, or the whole one-step record; half 1 the
  // taps 1..8 (chunks 4..8) of a pair record
  auto prefetch = [&](const int4& e, bool valid, int slot) {
    if (act && valid) {
      double* d = my_ring + slot * slot_stride;
      if (e.y == 2) {
        const double* src = rp + ((size_t)(e.x / 2) * n + start + p) * PW;
        if (half == 0) {
#pragma unroll
          for (int q = 0; q < 5; ++q) cp_async16(d + 2 * q, src + 2 * q);
          cp_async16(d + 16, src + 16);
        } else {
#pragma unroll
          for (int q = 4; q < 9; ++q) cp_async16(d + 2 * q, src + 2 * q);
        }
      } else if (half == 0) {
        const double* src = rec + ((size_t)e.x * n + start + p) * RW;
#pragma unroll
        for (int q = 0; q < RW / 2; ++q) cp_async16(d + 2 * q, src + 2 * q);
      }
    }
    cp_async_commit();
  };
  static_assert(DEPTH == 4, "the plan queue holds DEPTH entries");
  prefetch(e0, nplan > 0, 0);
  prefetch(e1, nplan > 1, 1);
  prefetch(e2, nplan > 2, 2);
  if (multi) {
    if (tid == 0 && nplan > 1) mbar_arm(&bar[1], 2 * HP * (int)sizeof(double));
    cl.sync();
  } else {
    __syncthreads();
  }
  uint32_t ph0 = 0u, ph1 = 0u;
  for (int j = 0; j < nplan; ++j) {
    prefetch(e3, j + 3 < nplan, (j + 3) & (DEPTH - 1));
    cp_async_wait<DEPTH - 1>();
    const int4 e = e0;
    e0 = e1;
    e1 = e2;
    e2 = e3;
    e3 = j + 4 < nplan ? plan[j + 4] : none;
    const int b = (j + 1) & 1;  // buffer of lambda after step j (the start row is in lam0)
    double* const Ln = b ? lam1 : lam0;
    const double* const Lp = (b ? lam0 : lam1);
    const bool last = j + 1 == nplan;
    const double* r = my_ring + (j & (DEPTH - 1)) * slot_stride;
    const double* L = Lp + p;
    double acc = 0.0;
    if (act) {
      if (e.y == 2) {
        if (half == 0) {
          acc = e.z ? r[17] : 0.0;
#pragma unroll
          for (int o = -8; o <= 0; ++o) acc = fma(r[o + 8], L[o], acc);
        } else {
          acc = r[9] * L[1];
#pragma unroll
          for (int o = 2; o <= 8; ++o) acc = fma(r[o + 8], L[o], acc);
        }
      } else if (half == 0) {
        acc = e.z ? r[9] : 0.0;
#pragma unroll
        for (int o = -4; o <= 4; ++o) acc = fma(r[o + 4], L[o], acc);
      }
    }
    // hand half 1's partial sum to half 0 (barrier of the group's two warps)
    if (half == 1 && act) part[p] = acc;
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(64) : "memory");
    if (half == 0 && act) {
      if (e.y == 2) acc += part[p];
      if (e.w) acc += W[(size_t)e.w * n + start + p];
      Ln[p] = acc;
      if (!last) {
        if (to_left) st_async_f64(b ? rl1 : rl0, acc, b ? bl1 : bl0);
        if (to_right) st_async_f64(b ? rr1 : rr0, acc, b ? br1 : br0);
      }
      out_rows[(size_t)e.x * n + start + p] = acc;
    }
    if (!last) {
      if (multi) {
        if (tid == 0 && j + 2 < nplan) mbar_arm(b ? &bar[0] : &bar[1], 2 * HP * (int)sizeof(double));
        mbar_wait_bounded(b ? &bar[1] : &bar[0], b ? ph1 : ph0, status);
        if (b) ph1 ^= 1u; else ph0 ^= 1u;
        __syncthreads();
      } else {
        __syncthreads();
        for (int q = tid; q < 2 * HP; q += nt) {
          const int qq = q < HP ? q - HP : cnt + (q - HP);
          Ln[qq] = Ln[wrapn(qq, n)];
        }
        __syncthreads();
      }
    }
  }
  cp_async_wait<0>();
  if (multi) cl.sync();  // no CTA leaves while a neighbour could still address it
}

// ---- rows skipped by pair steps ---------------------------------------------------------
// Grid (tiles, plan blocks): for every two- or four-step entry {s, 2|4, src, w}, row
// s+1 = M_{s+1}^T row s+2 (+ r_{s+1} when the source is on); in a four-step entry row
// s+2 comes from bu1_band_fill4_kernel, run before.
__global__ void __launch_bounds__(PT2) bu1_band_fill_kernel(int n, const double* __restrict__ rec,
                                                            const int4* __restrict__ plan, int nplan,
                                                            int entries_per_block,
                                                            double* __restrict__ rows) {
  const int pt = blockIdx.x * PT2 + threadIdx.x;
  if (pt >= n) return;
  const int jb = blockIdx.y * entries_per_block;
  const int je = min(nplan, jb + entries_per_block);
  for (int j = jb; j < je; ++j) {
    const int4 e = plan[j];
    if (e.y < 2) continue;
    const int s1 = e.x + 1;
    const double* r = rec + ((size_t)s1 * n + pt) * RW;
    const double* up = rows + (size_t)(s1 + 1) * n;
    double acc = e.z ? r[9] : 0.0;
#pragma unroll
    for (int o = -4; o <= 4; ++o) acc = fma(r[o + 4], up[wrapn(pt + o, n)], acc);
    rows[(size_t)s1 * n + pt] = acc;
  }
}

// ---- host side ----------------------------------------------------------------------
// Step plan of the two-step chain from row P*k down to 0 (see the file comment).
int bu1_chain2_plan(int64_t K, int64_t k, int P, int4* out) { return bu1_chain_plan(K, k, P, 2, out); }

bool bu1_chain2_valid(int n, int C) {
  if (C < 1 || C > 16) return false;
  const int nc = (n + C - 1) / C;
  // two threads per point (groups of 32 points, at most 7 groups for the barrier ids and
  // the 4-deep ring of 144-byte records in 200 KB)
  if ((nc + 31) / 32 > 5) return false;
  if (C == 1) return true;
  return n - (C - 1) * nc >= HP;  // every CTA owns the 8 points a neighbour needs
}

cudaError_t launch_bu1_band_pair(cudaStream_t st, int n, const double* rec, int64_t m_lo,
                                 int64_t m_hi, double* rp, int priority) {
  if (m_hi <= m_lo) return cudaSuccess;
  const int tiles = (n + PT2 - 1) / PT2;
  int64_t ppb = ((m_hi - m_lo) * tiles + 1215) / 1216;
  if (ppb < 2) ppb = 2;
  int per = (int)ppb;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles, (unsigned)((m_hi - m_lo + per - 1) / per));
  cfg.blockDim = dim3(PT2);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = priority;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bu1_band_pair_kernel, n, rec, m_lo, m_hi, per, rp);
}

cudaError_t launch_bu1_band_chain2(cudaStream_t st, int C, int n, const double* rec, const double* rp,
                                   const int4* plan, int nplan, int s_hi, const double* from_rows,
                                   const double* W, double* out_rows, int* status, int priority,
                                   size_t reserve_smem) {
  if (nplan <= 0) return cudaSuccess;
  const int nc = (n + C - 1) / C;
  constexpr int DEPTH = 4;
  const int G = (nc + 31) / 32, nt = 64 * G;  // two warps (halves) per group of 32 points
  size_t sh = sizeof(double) * (2 * (size_t)(nc + 2 * HP) + (size_t)G * 32 + (size_t)DEPTH * nt * PW);
  if (reserve_smem > sh) sh = reserve_smem;  // no other CTA shares the SM
  const void* fn = (const void*)bu1_band_chain2_kernel<DEPTH>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {&n, &rec, &rp, &plan, &nplan, &s_hi, &from_rows, &W, &out_rows, &status};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(nt);
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

cudaError_t launch_bu1_band_fill(cudaStream_t st, int n, const double* rec, const int4* plan, int nplan,
                                 double* rows, int priority) {
  if (nplan <= 0) return cudaSuccess;
  const int tiles = (n + PT2 - 1) / PT2;
  int per = (int)(((int64_t)nplan * tiles + 1215) / 1216);
  if (per < 4) per = 4;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles, (unsigned)((nplan + per - 1) / per));
  cfg.blockDim = dim3(PT2);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = priority;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bu1_band_fill_kernel, n, rec, plan, nplan, per, rows);
}

}  // namespace pxa
