// kernels_ad2.cuh — constants, parameters and launch wrappers of the 2D kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pxa {

constexpr int G2 = 4;                // ghost layers of the padded 2D arrays
// tile interior (TX2 % 4 == 0 for 16-byte TMA x offsets). 18 rows: a 512 x 512 grid has
// 290 tiles, about two 8-warp blocks per SM, six rows per thread; measured on the C3
// gradient against 34, 26, 22, 14 and 10 rows (and 3 blocks per SM): the fastest
constexpr int TX2 = 56, TY2 = 18;
constexpr int BX2 = TX2 + 2 * G2;    // 64 floats = 256 bytes (a multiple of 16 for TMA)
constexpr int BY2 = TY2 + 2 * G2;    // 26 rows
constexpr int TILE2 = BX2 * BY2;     // 1664 floats = 6656 bytes (a multiple of 128)
constexpr int RG2 = (BY2 - 2) / 4;   // rows of the halo-3 region owned by one thread (6)
static_assert((BY2 - 2) % 4 == 0, "the halo-3 rows split evenly over the 4 row groups");
static_assert(BX2 - 2 <= 64, "one thread per halo-3 column");

struct Ad2Params {
  int nx, ny, Wp, Hp, tiles_x, tiles_y;
  float inv2h, invh2, nu, dt;
  double dtd, omega;
};

size_t ad2_smem_bytes();
bool ad2_make_map(CUtensorMap* map, float* base, const Ad2Params& p, int depth, int box_depth);
// 3D map over [depth][Hp][Wp] FP32 with a box of box_x x box_y x box_depth elements.
bool ad2_make_map_box(CUtensorMap* map, float* base, const Ad2Params& p, int depth, int box_x,
                      int box_y, int box_depth);
// Tile-kernel RK4 steps of a group of lanes; lane l is at absolute step l * lane_k + s_local
// (+ lane_off for the transposed step) and takes s(t) at its stage times from the table
// sc[3 step + {0, 1, 2}] (launch_ad2_forcing_table over every step used). pdl != 0 (the
// single-lane kernels): launched with programmatic dependent launch, so the coefficient
// tile and the table are read while the previous kernel in the stream finishes; allowed
// only when that kernel wrote neither of them (e.g. the previous step). The transposed step
// of one lane (lanes == map_lanes == 1) runs the register-layout kernel. The forcing-gradient
// accumulators G are double-float: [lanes][ny][nx] (hi, lo) FP32 pairs, summed in FP32
// arithmetic (two-sum; GB300's FP64 pipe issues one warp instruction per 64 cycles) and
// read out in FP64 by launch_ad2_sum_grad.
cudaError_t launch_ad2_rk4(cudaStream_t st, const CUtensorMap& qmap, const CUtensorMap& cmap,
                           const Ad2Params& p, float* states, int lanes, int map_lanes,
                           int lanes_per_cta, int buf_in, int64_t lane_k, int64_t s_local, const float* sc,
                           float* traj, int64_t traj_row, float* Jpart, int64_t jrow, int* status, int pdl);
cudaError_t launch_ad2_rk4T(cudaStream_t st, const CUtensorMap& qmap, const CUtensorMap& cmap,
                            const Ad2Params& p, float* states, int lanes, int map_lanes,
                            int lanes_per_cta, int buf_in, int64_t lane_k, int64_t lane_off, int64_t s_local,
                            int with_source, const float* traj, double src_scale, float2* G,
                            const float* sc, int* status, int pdl);
cudaError_t launch_ad2_pack_coef(cudaStream_t st, const Ad2Params& p, const double* u,
                                 const double* v, const double* f, const double* ft, float* coef);
cudaError_t launch_ad2_fill(cudaStream_t st, const Ad2Params& p, float* states, int lanes,
                            const float* traj, int64_t row0, int64_t row_step, double scale);
cudaError_t launch_ad2_add_padded(cudaStream_t st, size_t count, float* dst, const float* src);
// J = scale * the sum of the FP32 partials part[0 .. count) (double-float within blocks,
// FP64 across them), in two passes over at most AD2_REDUCE_J_BLOCKS blocks whose sums go
// to scratch (that many doubles).
constexpr int AD2_REDUCE_J_BLOCKS = 1024;
constexpr int AD2_J_WARPS = 8;  // objective partials per tile and step (one per warp)
cudaError_t launch_ad2_reduce_J(cudaStream_t st, const float* part, size_t count, double scale, double* scratch,
                                double* J, int* status);
// Register-wavefront RK4 step for many lanes (kernels_ad2_roll.cu); needs ad2_roll_ok.
bool ad2_roll_ok(const Ad2Params& p);
cudaError_t launch_ad2_forcing_table(cudaStream_t st, int64_t s0, int64_t count, double dt,
                                     double omega, float* sc);
// qmap: ad2_make_map_box over the state buffers (depth 2*lanes: z = buf*lanes + lane) with
// box {64, AD2_ROLL_BR, 1}; cmap: over the coefficient array (depth 3) with box
// {64, AD2_ROLL_BR, 3}. buf_in selects the input buffer; the output is the other one.
constexpr int AD2_ROLL_BR = 4;
cudaError_t launch_ad2_rk4_roll(cudaStream_t st, const CUtensorMap& qmap, const CUtensorMap& cmap,
                                const Ad2Params& p, float* states, int lanes, int buf_in,
                                const float* sc, int sc_stride, int* status);
// 3D map over [depth][ny][nx] unpadded planes of FP32 (elem_bytes 4) or FP64 (8), box
// {box_x, box_y, 1}.
bool ad2_make_map_plain(CUtensorMap* map, void* base, int elem_bytes, int nx, int ny, int depth, int box_x,
                        int box_y);
// tc = [4][Hp][Wp]: the coefficients of A^T (tE, tW, tN, tS) at every padded point.
cudaError_t launch_ad2_pack_coefT(cudaStream_t st, const Ad2Params& p, const double* u, const double* v,
                                  float* tc);
// One reverse step of the adjoint lanes as a register wavefront (kernels_ad2_roll.cu; needs
// ad2_roll_ok): qmap over the lane states (depth 2*lanes, box {64, AD2_ROLL_BR, 1}), tmap
// over tc (box {64, AD2_ROLL_BR, 4}), smap over the FP32 trajectory [K+1][ny][nx] and gmap
// over the FP32 lane gradients G [lanes][ny][nx] (both ad2_make_map_plain, box
// {64, AD2_ROLL_BR}). Steps lanes lane0 .. lane0 + count - 1 of `lanes`; lane l is at step
// zsrc0 + l z_stride: its source row and its forcing factors sc[3 step + {0, 1, 2}]; the
// source is added when add_src is set.
cudaError_t launch_ad2_rk4T_roll(cudaStream_t st, const CUtensorMap& qmap, const CUtensorMap& tmap,
                                 const CUtensorMap& smap, const CUtensorMap& gmap, const Ad2Params& p,
                                 float* states, float* G, int lanes, int lane0, int count, int buf_in,
                                 const float* sc, int zsrc0, int z_stride, float src_scale, int add_src,
                                 int* status);
// The chain's polynomial propagator (PXA_PROP_POLY): one launch forms the powers
// v_{i0+j} = (tau A^T)^j v_{i0}, j = 1..4, on every tile from plane buf_in of V (vmap: ad2_make_map
// over V with depth 2), writes v_{i0+4} to the other plane, and adds the interior's terms
// a_i v_i to H (padded plane; H = a_0 v_0 + ... when i0 == 0; skipped when want_h == 0) and
// b_i v_i to G (a double-float accumulator, [ny][nx] (hi, lo) FP32 pairs). ca and cb (FP32) hold the coefficients 0 .. i0 + 4.
// For i0 == 0 the input is v_0 = H + W: the tile of H (hmap, a map over the padded H
// plane) plus, when w_z >= 0, plane w_z of wmap (the lane value at the segment's top).
// pdl != 0: programmatic dependent launch (the coefficient tile and ca, cb are read before
// the wait for the previous kernel, which must not have written them).
cudaError_t launch_ad2_poly(cudaStream_t st, const CUtensorMap& vmap, const CUtensorMap& cmap, const CUtensorMap& hmap,
                            const CUtensorMap& wmap, int w_z, const Ad2Params& p, float tau, float* V, int buf_in,
                            int i0, const float* ca, const float* cb, float* H, int want_h, float2* G, int* status,
                            int pdl);
// The forcing-gradient coefficients b[s][0..m] of `segments` chain segments of kk steps
// from the omega-free families Q = [3][kk][m+1] (m < 256), summed in FP64, stored in FP32.
cudaError_t launch_ad2_poly_forcing(cudaStream_t st, int segments, int kk, int m, double dt, double omega,
                                    const double* Q, float* b);
// grad (FP64) = sum over `lanes` double-float accumulators G[l] and `flanes` FP32 ones Gf[l]
// (+ extra, a double-float accumulator, may be NULL).
cudaError_t launch_ad2_sum_grad(cudaStream_t st, size_t N, int lanes, const float2* G, int flanes, const float* Gf,
                                const float2* extra, double* grad, int* status);

}  // namespace pxa
