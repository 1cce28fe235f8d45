// kernels_bu1_quad.cu — four-step banded adjoint chain for 1D Burgers.
//
// The serial adjoint chain lambda_s = M_s^T lambda_{s+1} + r_s (Eq. adjHomNormal with the
// stepper's own propagator; the top subinterval with its source) costs about one halo
// exchange between the CTAs of a cluster per step taken, far more than its FMAs. Taking
// four steps at once with the product band Q_s = M_s^T M_{s+1}^T M_{s+2}^T M_{s+3}^T
// (33 diagonals) and the combined source of the four rows quarters the exchanges:
//
//  - bu1_band_quad_kernel (parallel, beside the direct solve): for every row s = 4q,
//    the record {Q_s[i][i-16..i+16], combined source} from the two-step records of
//    rows 4q and 4q+2: Q_s = P_s P_{s+2}, src = src_P(s) + P_s src_P(s+2).
//  - bu1_band_chain4_kernel (one cluster): follows a step plan of 4-, 2- and 1-step
//    entries (a longer step is taken where nothing happens on the rows it skips). Each
//    point's taps are split over four warps on the four SM sub-partitions; 16 boundary
//    values per side are exchanged.
//  - bu1_band_fill4_kernel (parallel): rows s+3 = M_{s+3}^T row s+4 (+ r) and
//    s+2 = P_{s+2} row s+4 (+ combined source) inside four-step entries; the two-step
//    fill then gives row s+1 from row s+2 for two- and four-step entries alike.
#include <cooperative_groups.h>

#include "common.cuh"
#include "dsmem.cuh"
#include "kernels_1d.cuh"

namespace cg = cooperative_groups;

namespace pxa {

namespace {

constexpr int RW = BU1_BAND_RECORD;   // one-step record: 9 taps + source
constexpr int PW = BU1_PAIR_RECORD;   // two-step record: 17 taps + source
constexpr int QW = BU1_QUAD_RECORD;   // four-step record: 33 taps + source
constexpr int HQ = 16;                // halo of a four-step entry
constexpr int QT = 128;               // points per tile of the parallel kernels

__device__ __forceinline__ int wrapq(int g, int n) {
  g %= n;
  return g < 0 ? g + n : g;
}

}  // namespace

// ---- four-step records -----------------------------------------------------------------
// Grid (tiles, quad blocks); quad q combines the two-step records 2q (rows 4q, 4q+1) and
// 2q+1 (rows 4q+2, 4q+3) for q in [q_lo, q_hi).
__global__ void __launch_bounds__(QT) bu1_band_quad_kernel(int n, const double* __restrict__ rp,
                                                           int64_t q_lo, int64_t q_hi, int quads_per_block,
                                                           double* __restrict__ rq) {
  __shared__ double nxt[(QT + 16) * PW];  // two-step records of row 4q+2 on the tile +- 8
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * QT;
  const int64_t qb = q_lo + (int64_t)blockIdx.y * quads_per_block;
  int64_t qe = qb + quads_per_block;
  if (qe > q_hi) qe = q_hi;
  const int pt = i0 + tid;
  for (int64_t q = qb; q < qe; ++q) {
    __syncthreads();
    const double* r1 = rp + (size_t)(2 * q + 1) * n * PW;
    for (int e = tid; e < (QT + 16) * PW; e += QT) {
      const int u = e / PW, j = e % PW;
      nxt[e] = r1[(size_t)wrapq(i0 - 8 + u, n) * PW + j];
    }
    __syncthreads();
    if (pt >= n) continue;
    const double* a = rp + ((size_t)(2 * q) * n + pt) * PW;  // row i of P_s and its source
    double ai[PW];
#pragma unroll
    for (int j = 0; j < PW; ++j) ai[j] = a[j];
    double out[QW];
#pragma unroll
    for (int o = 0; o < QW - 1; ++o) out[o] = 0.0;
    double src = ai[PW - 1];
    // Q_s[i][i+o] = sum_e P_s[i][i+e] P_{s+2}[i+e][i+o]
#pragma unroll
    for (int e = -8; e <= 8; ++e) {
      const double* b = nxt + (tid + 8 + e) * PW;  // row i+e of P_{s+2}
      const double w = ai[e + 8];
#pragma unroll
      for (int f = -8; f <= 8; ++f) out[e + f + 16] = fma(w, b[f + 8], out[e + f + 16]);
      src = fma(w, b[PW - 1], src);
    }
    out[QW - 1] = src;
    double2* dst = reinterpret_cast<double2*>(rq + ((size_t)q * n + pt) * QW);
#pragma unroll
    for (int j = 0; j < QW / 2; ++j) dst[j] = make_double2(out[2 * j], out[2 * j + 1]);
  }
}

// ---- four-step chain -----------------------------------------------------------------
// plan[j] = {row produced, steps (1, 2 or 4), source on, lane index to add (0: none)}.
// lambda_{s_hi} is row s_hi of from_rows (a chain continued from an earlier launch) or
// the source of the last state; rows produced go to out_rows.
//
// With G = ceil(chunk / 32) point groups, warp w serves group w / 4 and quarter w % 4.
// The quarters take consecutive runs of taps (four-step: -16..-9 with the source,
// -8..-1, 0..7, 8..16; two-step: -8..-5 with the source, -4..-1, 0..3, 4..8; one-step:
// quarter 0 alone). Quarters 1-3 hand their partial sums over through shared memory at a
// barrier of the group's four warps; quarter 0 finishes, stores and sends the value.
// The records of an entry for the CTA's points are contiguous in global memory (one row
// of the one-, two- or four-step records): one thread brings them into a DEPTH-deep ring
// in shared memory with a single bulk copy DEPTH-1 entries ahead, completing on the
// slot's mbarrier.

template <int DEPTH>
__global__ void bu1_band_chain4_kernel(int n, const double* __restrict__ rec,
                                       const double* __restrict__ rp, const double* __restrict__ rq,
                                       const int4* __restrict__ plan, int nplan, int s_hi,
                                       const double* __restrict__ from_rows,
                                       const double* __restrict__ W, double* __restrict__ out_rows,
                                       int* status) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) double smq[];
  __shared__ __align__(8) uint64_t bar[2];
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int nc = (n + C - 1) / C, start = rank * nc, cnt = min(nc, n - start);
  const int G = (nc + 31) / 32;
  const int Wd = nc + 2 * HQ;
  double* const lam0 = smq + HQ;
  double* const lam1 = smq + Wd + HQ;
  double* const part = smq + 2 * Wd;   // [3][G * 32] partial sums of quarters 1-3
  double* const ring = part + 3 * G * 32;  // [DEPTH][nc * QW]: the records of one entry per slot
  __shared__ __align__(8) uint64_t rbar[DEPTH];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lanei = tid & 31;
  // warp w = 4 g + qq: the four quarters of a group sit on the four SM sub-partitions
  // (w mod 4), and each sub-partition holds one warp of every group
  const int g = warp >> 2, qq = warp & 3;
  // The last group holds the 2 x HQ edge points, the only ones whose taps reach the
  // neighbours' values: it alone waits for the halo, while the other groups work through
  // the interior points [HQ, cnt - HQ) of the same entry.
  const bool edge = g == G - 1;
  const int p = edge ? (cnt >= 2 * HQ && lanei >= HQ ? cnt - 2 * HQ + lanei : lanei)
                     : HQ + g * 32 + lanei;  // this thread's point
  const bool act = edge ? p < cnt : p < cnt - HQ;
  const bool multi = C > 1;
  const int left = (rank + C - 1) % C, right = (rank + 1) % C;
  const int cnt_left = min(nc, n - left * nc);
  if (tid == 0) {
    if (multi) {
      mbar_init(&bar[0], 1);
      mbar_init(&bar[1], 1);
    }
    for (int s = 0; s < DEPTH; ++s) mbar_init(&rbar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int q = tid - HQ; q < cnt + HQ; q += nt) {
    const int gq = wrapq(start + q, n);
    const double v = from_rows ? from_rows[(size_t)s_hi * n + gq] : rec[((size_t)s_hi * n + gq) * RW + (RW - 1)];
    lam0[q] = v;
    if (!from_rows && q >= 0 && q < cnt) out_rows[(size_t)s_hi * n + start + q] = v;
  }
  const bool sender = multi && act && qq == 0;
  const bool to_left = sender && p < HQ, to_right = sender && p >= cnt - HQ;
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
  const int slot_stride = nc * QW;  // doubles per ring slot (a multiple of 2: 16-byte slots)
  const int4 none = make_int4(0, 0, 0, 0);
  int4 e0 = nplan > 0 ? plan[0] : none, e1 = nplan > 1 ? plan[1] : none,
       e2 = nplan > 2 ? plan[2] : none, e3 = nplan > 3 ? plan[3] : none;
  // records of entry e: row e.x of the one-step, e.x / 2 of the two-step or e.x / 4 of
  // the four-step records, W doubles per point (taps from offset -W/2 + 1 and the source)
  auto rec_width = [](const int4& e) { return e.y == 4 ? QW : e.y == 2 ? PW : RW; };
  auto prefetch = [&](const int4& e, bool valid, int slot) {
    if (tid != 0 || !valid) return;
    const double* src = e.y == 4   ? rq + ((size_t)(e.x / 4) * n + start) * QW
                        : e.y == 2 ? rp + ((size_t)(e.x / 2) * n + start) * PW
                                   : rec + ((size_t)e.x * n + start) * RW;
    const uint32_t bytes = (uint32_t)(cnt * rec_width(e) * sizeof(double));
    // the slot's previous entry was read before the block barrier that precedes this
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arm(&rbar[slot], (int)bytes);
    bulk_g2s(ring + (size_t)slot * slot_stride, src, bytes, &rbar[slot]);
  };
  static_assert(DEPTH == 4, "the plan queue holds DEPTH entries");
  prefetch(e0, nplan > 0, 0);
  prefetch(e1, nplan > 1, 1);
  prefetch(e2, nplan > 2, 2);
  // the halo of entry e (sent unless e is the last) lands in buffer (e + 1) & 1 and
  // completes on bar[(e + 1) & 1]; entries 0 and 1 are armed here, entry e + 1 by the
  // edge group right after its wait for entry e - 1 on the same barrier
  const bool armer = edge && qq == 0 && lanei == 0;
  if (multi) {
    if (tid == 0 && nplan > 1) mbar_arm(&bar[1], 2 * HQ * (int)sizeof(double));
    if (tid == 0 && nplan > 2) mbar_arm(&bar[0], 2 * HQ * (int)sizeof(double));
    cl.sync();
  } else {
    __syncthreads();
  }
  uint32_t ph0 = 0u, ph1 = 0u;
  for (int j = 0; j < nplan; ++j) {
    prefetch(e3, j + 3 < nplan, (j + 3) & (DEPTH - 1));
    if (multi && j > 0) {
      // buffer of lambda after entry j - 1 (read now): j & 1
      uint64_t* hb = (j & 1) ? &bar[1] : &bar[0];
      uint32_t& ph = (j & 1) ? ph1 : ph0;
      if (edge) {
        mbar_wait_bounded(hb, ph, status);
        if (armer && j + 2 < nplan) mbar_arm(hb, 2 * HQ * (int)sizeof(double));
      }
      ph ^= 1u;
    }
    mbar_wait_bounded(&rbar[j & (DEPTH - 1)], (uint32_t)((j / DEPTH) & 1), status);
    const int4 e = e0;
    e0 = e1;
    e1 = e2;
    e2 = e3;
    e3 = j + 4 < nplan ? plan[j + 4] : none;
    const int b = (j + 1) & 1;  // buffer of lambda after step j (the start row is in lam0)
    double* const Ln = b ? lam1 : lam0;
    const double* const Lp = b ? lam0 : lam1;
    const bool last = j + 1 == nplan;
    const int rw = rec_width(e);
    const double* rr = ring + (size_t)(j & (DEPTH - 1)) * slot_stride + (size_t)p * rw;
    // this quarter's run of taps: ntap taps from offset o0
    int ntap = 0, o0 = 0;
    if (e.y == 4) {
      ntap = qq == 3 ? 9 : 8;
      o0 = -16 + 8 * qq;
    } else if (e.y == 2) {
      ntap = qq == 3 ? 5 : 4;
      o0 = -8 + 4 * qq;
    } else if (qq == 0) {
      ntap = 9;
      o0 = -4;
    }
    double acc = 0.0;
    if (act) {
      // record index of tap offset o: o + rw / 2 - 1; the source is the last entry. All
      // nine loads are issued before the first FMA (the ones past the quarter's taps stay
      // inside the slot and the lambda buffer and are not used).
      const double* L = Lp + p + o0;
      const double* rt = rr + o0 + rw / 2 - 1;
      double cv[9], lv[9];
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        cv[t] = rt[t];
        lv[t] = L[t];
      }
      // one accumulator: the two warps that share an SM sub-partition's FP64 unit hide
      // each other's dependent-FMA latency, and merges of partial accumulators would
      // cost FP64 instructions of their own
      acc = (qq == 0 && e.z) ? rr[rw - 1] : 0.0;
#pragma unroll
      for (int t = 0; t < 9; ++t)
        if (t < ntap) acc = fma(cv[t], lv[t], acc);
    }
    // quarters 1-3 hand their partial sums to quarter 0 (barrier of the group's four warps)
    if (qq > 0 && act) part[(qq - 1) * G * 32 + p] = acc;
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(128) : "memory");
    if (qq == 0 && act) {
      acc = (acc + part[p]) + (part[G * 32 + p] + part[2 * G * 32 + p]);
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
        __syncthreads();
      } else {
        __syncthreads();
        for (int q = tid; q < 2 * HQ; q += nt) {
          const int qx = q < HQ ? q - HQ : cnt + (q - HQ);
          Ln[qx] = Ln[wrapq(qx, n)];
        }
        __syncthreads();
      }
    }
  }
  // every entry's copy was waited for above; after a wait that gave up, a copy may still
  // be in flight: let the last one of each slot land before the block leaves
  if (tid == 0 && *(volatile int*)status != 0)
    for (int s = 0; s < DEPTH && s < nplan; ++s)
      mbar_drain(&rbar[s], (uint32_t)(((s + DEPTH * ((nplan - 1 - s) / DEPTH)) / DEPTH) & 1));
  if (multi) cl.sync();  // no CTA leaves while a neighbour could still address it
  else __syncthreads();
}

// ---- rows skipped by four-step entries ----------------------------------------------
// Grid (tiles, plan blocks): for every entry {s, 4, src, w}: row s+3 = M_{s+3}^T row s+4
// (+ r_{s+3}) and row s+2 = P_{s+2} row s+4 (+ its combined source), both from row s+4.
__global__ void __launch_bounds__(QT) bu1_band_fill4_kernel(int n, const double* __restrict__ rec,
                                                            const double* __restrict__ rp,
                                                            const int4* __restrict__ plan, int nplan,
                                                            int entries_per_block, double* __restrict__ rows) {
  const int pt = blockIdx.x * QT + threadIdx.x;
  if (pt >= n) return;
  const int jb = blockIdx.y * entries_per_block;
  const int je = min(nplan, jb + entries_per_block);
  for (int j = jb; j < je; ++j) {
    const int4 e = plan[j];
    if (e.y != 4) continue;
    const int s = e.x;
    const double* up = rows + (size_t)(s + 4) * n;
    const double* r3 = rec + ((size_t)(s + 3) * n + pt) * RW;
    double a3 = e.z ? r3[RW - 1] : 0.0;
#pragma unroll
    for (int o = -4; o <= 4; ++o) a3 = fma(r3[o + 4], up[wrapq(pt + o, n)], a3);
    const double* r2 = rp + ((size_t)((s + 2) / 2) * n + pt) * PW;
    double a2 = e.z ? r2[PW - 1] : 0.0;
#pragma unroll
    for (int o = -8; o <= 8; ++o) a2 = fma(r2[o + 8], up[wrapq(pt + o, n)], a2);
    rows[(size_t)(s + 3) * n + pt] = a3;
    rows[(size_t)(s + 2) * n + pt] = a2;
  }
}

// ---- host side ----------------------------------------------------------------------
// Step plan of the chain from row s_hi down to s_lo with steps of up to max_len (1, 2 or
// 4) rows: a longer step is taken from row r where r is a multiple of its length (the
// pair and four-step records sit at rows 2j and 4j), it stays above s_lo, no lane value
// is added on the rows it skips and the source is on for all of its rows or for none.
// The source is on for rows above src_lo; the value of lane j (subintervals of k steps)
// is added at row j k for j in [lane_lo, lane_hi], j >= 1. Entries {row produced, steps,
// source on, lane added at that row}. Returns the number of entries; out must hold
// s_hi - s_lo entries.
int bu1_chain_plan_range(int64_t s_hi, int64_t s_lo, int64_t k, int64_t src_lo, int64_t lane_lo,
                         int64_t lane_hi, int max_len, int4* out) {
  auto inj = [&](int64_t r) {
    const int64_t j = r / k;
    return (r % k == 0 && j >= 1 && j >= lane_lo && j <= lane_hi) ? (int)j : 0;
  };
  auto src = [&](int64_t r) { return r > src_lo ? 1 : 0; };
  int cnt = 0;
  int64_t r = s_hi;
  while (r > s_lo) {
    int len = 1;
    for (int L = max_len; L >= 2; L /= 2) {
      if (r - L < s_lo || r % L != 0 || src(r - 1) != src(r - L)) continue;
      bool clear = true;
      for (int u = 1; u < L; ++u) clear = clear && inj(r - u) == 0;
      if (clear) {
        len = L;
        break;
      }
    }
    const int64_t ro = r - len;
    out[cnt++] = make_int4((int)ro, len, src(ro), inj(ro));
    r = ro;
  }
  return cnt;
}

// The plan of the whole chain: rows P k down to 0, the source on the top subinterval, the
// values of lanes 1 .. P-2 added at their bottom rows.
int bu1_chain_plan(int64_t K, int64_t k, int P, int max_len, int4* out) {
  return bu1_chain_plan_range(K, 0, k, (int64_t)(P - 1) * k, 1, P - 2, max_len, out);
}

bool bu1_chain4_valid(int n, int C) {
  if (C < 1 || C > 16) return false;
  const int nc = (n + C - 1) / C;
  // four threads per point: at most 4 groups of 32 points (512 threads; a 4-deep ring of
  // the entries' records, 4 x 128 x 272 B = 139 KB)
  if ((nc + 31) / 32 > 4) return false;
  if (C == 1) return n >= HQ;
  return n - (C - 1) * nc >= HQ;  // every CTA owns the 16 points a neighbour needs
}

cudaError_t launch_bu1_band_quad(cudaStream_t st, int n, const double* rp, int64_t q_lo, int64_t q_hi,
                                 double* rq, int priority) {
  if (q_hi <= q_lo) return cudaSuccess;
  const int tiles = (n + QT - 1) / QT;
  int64_t qpb = ((q_hi - q_lo) * tiles + 1215) / 1216;
  if (qpb < 1) qpb = 1;
  const int per = (int)qpb;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles, (unsigned)((q_hi - q_lo + per - 1) / per));
  cfg.blockDim = dim3(QT);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = priority;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bu1_band_quad_kernel, n, rp, q_lo, q_hi, per, rq);
}

cudaError_t launch_bu1_band_chain4(cudaStream_t st, int C, int n, const double* rec, const double* rp,
                                   const double* rq, const int4* plan, int nplan, int s_hi,
                                   const double* from_rows, const double* W, double* out_rows,
                                   int* status, int priority, size_t reserve_smem) {
  if (nplan <= 0) return cudaSuccess;
  const int nc = (n + C - 1) / C;
  constexpr int DEPTH = 4;
  const int G = (nc + 31) / 32, nt = 128 * G;  // four warps (quarters) per group of 32 points
  size_t sh = sizeof(double) * (2 * (size_t)(nc + 2 * HQ) + 3 * (size_t)G * 32 + (size_t)DEPTH * nc * QW);
  if (reserve_smem > sh) sh = reserve_smem;  // no other CTA shares the SM
  const void* fn = (const void*)bu1_band_chain4_kernel<DEPTH>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {&n, &rec, &rp, &rq, &plan, &nplan, &s_hi, &from_rows, &W, &out_rows, &status};
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

cudaError_t launch_bu1_band_fill4(cudaStream_t st, int n, const double* rec, const double* rp,
                                  const int4* plan, int nplan, double* rows, int priority) {
  if (nplan <= 0) return cudaSuccess;
  const int tiles = (n + QT - 1) / QT;
  int per = (int)(((int64_t)nplan * tiles + 1215) / 1216);
  if (per < 4) per = 4;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles, (unsigned)((nplan + per - 1) / per));
  cfg.blockDim = dim3(QT);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = priority;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, bu1_band_fill4_kernel, n, rec, rp, plan, nplan, per, rows);
}

}  // namespace pxa
