// kernels_1d.cuh — host-side launch wrappers of the 1D kernels (kernels_1d.cu).
#pragma once
#include <vector>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pxa {

struct Bu1Grid {
  int n;
  double inv2h, invh2, nu;
};

size_t krylov_smem_bytes(int n, int m, int extra_vecs, bool v_in_smem);
// FP32 CN band lanes with their states in global memory (kernels_ad1_stream.cu).
int ad1_stream_padded_taps(int r);
cudaError_t launch_ad1_stream_step(cudaStream_t st, int lanes, int n, int r, const float* taps_padded,
                                   const float* x, float* y);
cudaError_t launch_ad1_stream_fill(cudaStream_t st, int n, int lanes, const double* q0, float* x);
cudaError_t launch_ad1_stream_out(cudaStream_t st, size_t total, const float* x, double* out);
// Host: taps m_j (|j| <= r) of the circulant Crank-Nicolson map of the stencil (am, a0, ap).
void cn_band_taps(int n, double am, double a0, double ap, double dt, std::vector<double>& taps, int& r);
void cn_power_taps(int n, double am, double a0, double ap, double dt, int64_t steps, int cut_exp,
                   std::vector<double>& taps, int& r, bool expo = false);

cudaError_t launch_cn_lanes(cudaStream_t st, int lanes, int threads, int n, int r,
                            const double* taps, int transpose, int64_t steps, const double* x0,
                            const double* src, double* out);
cudaError_t launch_band_minus_identity(cudaStream_t st, int n, int r, const double* taps,
                                       int transpose, const double* x, double* y);
cudaError_t launch_ad1_apply(cudaStream_t st, int n, double am, double a0, double ap,
                             int transpose, const double* x, double* y);
cudaError_t launch_ad1_chain(cudaStream_t st, int threads, int n, double am, double a0, double ap,
                             int transpose, const double* E, int first, int stride, int count,
                             double* hout, double* Vglob, int m, int phi_mode, double hscale,
                             int64_t steps_per_sub, int nsub, double tol, int v_in_smem,
                             int* status, double* errmax);
// h = 0; for l < count: h += E[first + l stride]; h = B h (B^T when transpose) with B the
// circulant band taps[2r+1] of the subinterval propagator; hout = h. One block, FP64.
cudaError_t launch_ad1_band_chain(cudaStream_t st, int n, int r, const double* taps, int transpose,
                                  const double* E, int first, int stride, int count, double* hout);
cudaError_t launch_ad1_relpm_chain(cudaStream_t st, int threads, int n, double am, double a0, double ap,
                                   int transpose, const double* E, int first, int stride, int count,
                                   double* hout, const double* D, const double* z, int mmax, double ts,
                                   int nsub, int direct, double tol, int* status, double* errmax);
cudaError_t launch_ad1_relpm_expv(cudaStream_t st, int threads, int n, double am, double a0, double ap,
                                  int transpose, const double* x, double* y, const double* D, const double* z,
                                  int mmax, double ts, int nsub, int direct, double tol, int* status,
                                  double* errmax);
// Host: the real Leja points method for the propagator over a span t of the stencil
// (am, a0, ap): exp(t A) (steps == 0) or the CN power R(dt A)^steps; substeps, their
// length and the Newton nodes and divided differences (mmax + 1 each).
void relpm_setup_host(double t, double am, double a0, double ap, int mmax, int& nsub, double& ts,
                      std::vector<double>& z, std::vector<double>& D, int64_t steps);
cudaError_t launch_ad1_expv(cudaStream_t st, int threads, int n, double am, double a0, double ap,
                            int transpose, const double* x, double* y, double* Vglob, int m,
                            int phi_mode, double hscale, int64_t steps_per_sub, int nsub,
                            double tol, int v_in_smem, int* status, double* errmax);
cudaError_t launch_ad1_superpose_direct(cudaStream_t st, int threads, int n, int r,
                                        const double* taps, const double* q0, const double* elast,
                                        const double* hsum, const double* g, double* qT, double* srcT,
                                        double* J, int* status);
cudaError_t launch_ad1_superpose_adjoint(cudaStream_t st, int n, const double* lamK,
                                         const double* e0, const double* hsum, double* grad,
                                         int* status);
cudaError_t launch_bu1_magnus_chain(cudaStream_t st, int threads, Bu1Grid g, double dt, int64_t K,
                                    int P, int64_t k, int M, double omega, const double* traj,
                                    int64_t lane_k, const double* W, double* gH, double* Vglob, int m, double tol,
                                    int v_in_smem, int* status, double* errmax);
bool bu1c_valid_cluster(int n, int C);
cudaError_t launch_bu1c_adjoint_lanes(cudaStream_t st, int C, int lanes, int n, double L, double nu,
                                      double dt, double T, int64_t k, double omega, const double* f,
                                      const double* gt, const double* traj, const double* ckpt,
                                      double* scratch, double* wout, double* gout);
cudaError_t launch_bu1c_stepper_chain(cudaStream_t st, int C, int n, double L, double nu, double dt,
                                      double T, int64_t k, int P, double omega, const double* f,
                                      const double* gt, const double* rows, int64_t lane_k,
                                      const double* W, double* gH);
// Serial RK4 sweeps of the Burgers direct problem on clusters (kernels_bu1_rk4.cu).
bool bu1_rk4_valid_cluster(int n, int C);
// One iteration of Alg. 2 for 1D Burgers (kernels_bu1_nl.cu): Q -> Qn (every step), lanes
// into V, qbar [P][n]; change[0] = max_s ||Qn_s - Q_s||^2, change[1] = max_s ||Qn_s||^2,
// change[2] != 0 when non-finite. n <= 1024.
cudaError_t launch_nl_iteration(cudaStream_t st, int n, int64_t K, int P, double L, double nu, double dt,
                                const double* f, const double* sc, const double* Q, double* Qn, double* V,
                                double* qbar, double* change);
// The tracking objective from stored trajectory rows: Jrow[s] = ||u_s - g||^2 for s in
// [s0, s1), then J = scale * sum_{s=1..K} Jrow[s] in a fixed order.
cudaError_t launch_bu1_objective_rows(cudaStream_t st, const double* traj, const double* g, int n, int64_t s0,
                                      int64_t s1, double* Jrow, int priority);
cudaError_t launch_bu1_objective_sum(cudaStream_t st, const double* Jrow, int64_t K, double scale, double* Jdev,
                                     int* status);
// One block waiting on an mbarrier that nothing completes (the bounded wait's failure path).
cudaError_t launch_wait_probe(cudaStream_t st, int* status);
cudaError_t launch_bu1_forcing_table(cudaStream_t st, int64_t K, double dt, double omega, double* sc);
// reserve_smem > 0 requests that much dynamic shared memory per CTA, so that no other
// kernel's CTA fits beside the sweep on its SMs while it runs concurrently with them.
// group: steps per halo exchange (1, 2 or 4; 0 = chosen by a cost model; an invalid
// request falls back to the largest valid smaller one). The banded sweep takes the same.
cudaError_t launch_bu1_rk4_sweep(cudaStream_t st, int C, int lanes, int n, double L, double nu,
                                 double dt, int64_t k, const double* f, const double* sc,
                                 const double* x0, double* out, int64_t lane_rows, const double* gt,
                                 double T, double* Jdev, double* ckpt, int64_t ck_every,
                                 int* status, int priority, size_t reserve_smem, int group);
cudaError_t launch_sum_parts(cudaStream_t st, int count, const double* parts, double* out, int* status);

// Banded discrete adjoint of the Burgers RK4 map (kernels_bu1_band.cu). A record holds
// the 9 taps of row i of M_s^T and the objective's source dJ/du_s[i].
constexpr int BU1_BAND_RECORD = 10;
constexpr int BU1_PAIR_RECORD = 18;  // 17 taps of a row of M_s^T M_{s+1}^T + combined source
constexpr int BU1_QUAD_RECORD = 34;  // 33 taps of a row of M_s^T ... M_{s+3}^T + combined source
constexpr int BU1_BAND_MAX_CHUNK = 1024;  // points per CTA of the banded sweep
bool bu1_band_valid_cluster(int n, int C);
int bu1_band_grad_blocks(int64_t K, int n);
cudaError_t launch_bu1_band_prepass(cudaStream_t st, int n, double L, double nu, double dt, double T,
                                    double omega, const double* f, const double* gt,
                                    const double* rows, int64_t lane_k, int lanes, int64_t s_begin,
                                    int64_t s_end, int64_t K, double* rec, double* jt, int priority);
cudaError_t launch_bu1_band_sweep(cudaStream_t st, int C, int clusters, int lane0, int n,
                                  const double* rec, int64_t k, int P, int chain, const double* W,
                                  double* out_rows, double* wout, int* status, int priority,
                                  int group);
cudaError_t launch_bu1_band_grad(cudaStream_t st, int n, double dt, double omega, int64_t K,
                                 int64_t li_top, const double* LI, const double* H, const double* jt,
                                 double* partial, const double* extra, double* grad, int* status);
// The gradient in parts: step blocks [b_lo, b_hi) into their rows of partial, then the
// fixed-order sum over all blocks.
int bu1_band_steps_per_block(int64_t K, int n);
cudaError_t launch_bu1_band_grad_part(cudaStream_t st, int n, double dt, double omega, int64_t K,
                                      int64_t li_top, const double* LI, const double* H,
                                      const double* jt, double* partial, int b_lo, int b_hi,
                                      int priority);
cudaError_t launch_bu1_band_grad_reduce(cudaStream_t st, int n, int64_t K, const double* partial,
                                        const double* extra, double* grad, int* status);
// The gradient over steps [s_begin, s_end) in blocks of spb steps into partial rows
// block0, block0 + 1, ...; the fixed-order sum of the first `blocks` rows of partial.
cudaError_t launch_bu1_band_grad_range(cudaStream_t st, int n, double dt, double omega, int64_t s_begin,
                                       int64_t s_end, int spb, int64_t li_top, const double* LI,
                                       const double* H, const double* jt, double* partial, int block0,
                                       int priority);
cudaError_t launch_bu1_band_reduce_blocks(cudaStream_t st, int n, int blocks, const double* partial,
                                          double* grad, int* status);
// out = H_row + the source entries of rec_row (one row of n points).
cudaError_t launch_bu1_band_top(cudaStream_t st, int n, const double* H_row, const double* rec_row,
                                double* out);
// Two-step banded chain (kernels_bu1_pair.cu).
int bu1_chain2_plan(int64_t K, int64_t k, int P, int4* out);
bool bu1_chain2_valid(int n, int C);
cudaError_t launch_bu1_band_pair(cudaStream_t st, int n, const double* rec, int64_t m_lo,
                                 int64_t m_hi, double* rp, int priority);
cudaError_t launch_bu1_band_chain2(cudaStream_t st, int C, int n, const double* rec, const double* rp,
                                   const int4* plan, int nplan, int s_hi, const double* from_rows,
                                   const double* W, double* out_rows, int* status, int priority,
                                   size_t reserve_smem);
cudaError_t launch_bu1_band_fill(cudaStream_t st, int n, const double* rec, const int4* plan, int nplan,
                                 double* rows, int priority);
// Four-step banded chain (kernels_bu1_quad.cu).
int bu1_chain_plan(int64_t K, int64_t k, int P, int max_len, int4* out);
int bu1_chain_plan_range(int64_t s_hi, int64_t s_lo, int64_t k, int64_t src_lo, int64_t lane_lo,
                         int64_t lane_hi, int max_len, int4* out);
bool bu1_chain4_valid(int n, int C);
cudaError_t launch_bu1_band_quad(cudaStream_t st, int n, const double* rp, int64_t q_lo, int64_t q_hi,
                                 double* rq, int priority);
cudaError_t launch_bu1_band_chain4(cudaStream_t st, int C, int n, const double* rec, const double* rp,
                                   const double* rq, const int4* plan, int nplan, int s_hi,
                                   const double* from_rows, const double* W, double* out_rows,
                                   int* status, int priority, size_t reserve_smem);
cudaError_t launch_bu1_band_fill4(cudaStream_t st, int n, const double* rec, const double* rp,
                                  const int4* plan, int nplan, double* rows, int priority);
cudaError_t launch_sum_lanes(cudaStream_t st, int n, int lanes, const double* G, const double* extra,
                             double* grad, int* status);
cudaError_t launch_bu1_rhs(cudaStream_t st, Bu1Grid g, const double* u, double* y);
cudaError_t launch_bu1_jacT(cudaStream_t st, Bu1Grid g, const double* U, const double* x, double* y);

}  // namespace pxa
