// pxa_batch.cu — the C ABI of batches of independent 1D advection-diffusion problems
// (declared in include/pxa.h): set-up of the per-problem bands and work lists, the
// workspace, the gradient of every problem in one launch per phase, graph replay and the
// Krylov autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/pxa.h"
#include "common.cuh"
#include "kernels_1d.cuh"
#include "kernels_batch.cuh"

using namespace pxa;

struct pxa_batch {
  int device = 0;
  cudaStream_t stream = nullptr;      // the caller's stream (borrowed)
  cudaStream_t cap_stream = nullptr;  // library-owned stream used to capture graphs
  cudaStream_t side = nullptr;        // the Krylov chains, beside the stepped ones
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err;

  // problems
  int count = 0;
  std::vector<int> n;
  std::vector<double> nu;
  double c = 1.0, L = 0.0, T = 1.0;
  int64_t K = 0;
  int P = 1;
  int m = 30;
  double tol = 1e-8, reach = 0.04;
  double hom_ratio = 1.0;  // Krylov exponential where the cost model puts it <= ratio x the stepper's propagator
  bool power = true;       // the stepper's propagator over a subinterval as one band of M^(K/P)
  int lane_q_req = 0;      // CN steps per lane band application requested (0: automatic)
  int lane_q = 1;          // in use: the lanes and stepped chains apply the band of M^q
  bool use_graph = true;

  // set-up (host)
  bool ready = false;
  std::vector<BatchInst> hinst;
  std::vector<int64_t> off;
  int64_t total = 0;
  int nmax = 0, r32max = 0, r64max = 0, subs_max = 0, lanes_grid = 0;
  int rpmax = 0, pow_grid = 0;  // widest subinterval-propagator band; its chains' grid

  // workspace (device)
  std::vector<void*> allocs;
  BatchInst* inst = nullptr;
  float* taps32 = nullptr;
  double* taps64 = nullptr;
  int2* items_par = nullptr;
  int2* items_ser = nullptr;
  int2* items_step = nullptr;  // problems whose homogeneous parts are stepped
  int* kry_list = nullptr;     // problems whose homogeneous parts use the exponential
  int2* items_pow = nullptr;   // problems whose homogeneous parts apply the band of M^(K/P)
  int n_step = 0, n_kry = 0, n_pow = 0;
  std::vector<int> uses_krylov;  // per problem
  int* counter = nullptr;
  // one persistent launch with device-side dependencies (pxa_batch_set_schedule)
  int schedule = 1;          // requested: 1 = one launch when no problem uses Krylov, 0 = phases
  int4* items_flow = nullptr;
  int n_flow = 0, flow_grid = 0;
  int graph_kernels = 0;  // kernel nodes of the captured gradient graph
  int* flow_state = nullptr;  // [1 + 4 count]: queue counter, per-problem counters
  bool flow_last = false;     // the last gradient ran as one launch
  double *src = nullptr, *E = nullptr, *EA = nullptr, *h = nullptr, *hA = nullptr, *qT = nullptr,
         *srcT = nullptr, *V = nullptr, *errmax = nullptr;
  int* status = nullptr;
  int64_t bytes = 0;

  // graph cache
  cudaGraphExec_t gexec = nullptr;
  int g_mode = -1;
  const double* g_q0 = nullptr;
  const double* g_J = nullptr;
  const double* g_grad = nullptr;

  double err_last = 0.0;
  bool timing = false;
  cudaEvent_t ev[6] = {};
  float ms[5] = {};
};

namespace {

int bfail(pxa_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

#define BCUDA(b, expr, what)                                                                   \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) return bfail(b, PXA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void binvalidate(pxa_batch* b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  b->g_mode = -1;
}

void brelease(pxa_batch* b) {
  binvalidate(b);
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
  b->inst = nullptr;
  b->taps32 = nullptr;
  b->taps64 = nullptr;
  b->items_par = b->items_ser = b->items_step = b->items_pow = nullptr;
  b->kry_list = nullptr;
  b->n_step = b->n_kry = b->n_pow = 0;
  b->counter = b->status = nullptr;
  b->items_flow = nullptr;
  b->flow_state = nullptr;
  b->n_flow = b->flow_grid = 0;
  b->src = b->E = b->EA = b->h = b->hA = b->qT = b->srcT = b->V = b->errmax = nullptr;
  b->bytes = 0;
  b->ready = false;
}

template <typename T>
int balloc(pxa_batch* b, T** out, size_t count) {
  void* p = nullptr;
  const size_t bytes = sizeof(T) * (count ? count : 1);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, PXA_ERR_OOM, "batch workspace allocation of " + std::to_string(bytes) + " bytes failed");
  }
  b->allocs.push_back(p);
  b->bytes += (int64_t)bytes;
  *out = static_cast<T*>(p);
  return PXA_OK;
}

// Bands, substeps, work lists and workspace of the configured batch.
int bprepare(pxa_batch* b) {
  if (b->ready) return PXA_OK;
  if (b->count <= 0) return bfail(b, PXA_ERR_STATE, "pxa_batch_set first");
  BCUDA(b, cudaSetDevice(b->device), "cudaSetDevice");
  brelease(b);
  const int cnt = b->count, P = b->P;
  const double dt = b->T / (double)b->K, tau = b->T / (double)P;
  b->hinst.assign(cnt, BatchInst{});
  b->off.assign(cnt + 1, 0);
  std::vector<float> t32;
  std::vector<double> t64;
  b->nmax = b->r32max = b->r64max = b->subs_max = b->rpmax = 0;
  const int64_t kp = b->K / P;  // steps per subinterval
  // The lanes and the stepped chains apply the product band of M^q, the CN map taken q
  // times (q = 4, 2 or 1, dividing K/P): the same FMAs per CN step as q applications of
  // M, but one barrier and halo refresh per q steps and q times less zero padding of the
  // narrow bands; the FP64 band of M^q gives the sources (M^q - I) x. q = 1 keeps the
  // long-double band of M. The widest q whose FP32 bands fit the lanes is taken.
  auto stencil = [&](int i, BatchInst& I) {
    const double h = b->L / b->n[i];
    I.n = b->n[i];
    I.am = b->c / (2.0 * h) + b->nu[i] / (h * h);
    I.a0 = -2.0 * b->nu[i] / (h * h);
    I.ap = -b->c / (2.0 * h) + b->nu[i] / (h * h);
  };
  auto lane_band = [&](const BatchInst& I, int q, std::vector<double>& taps, int& r, int& r32) {
    if (q == 1)
      cn_band_taps(I.n, I.am, I.a0, I.ap, dt, taps, r);
    else
      cn_power_taps(I.n, I.am, I.a0, I.ap, dt, q, 50, taps, r);
    // the FP32 lanes keep the taps above 2^-40 of the largest (far below FP32 rounding)
    double big = 0.0;
    for (double v : taps) big = std::max(big, std::fabs(v));
    const double cut = std::ldexp(big, -40);
    r32 = 0;
    for (int j = 1; j <= r; ++j)
      if (std::fabs(taps[r + j]) >= cut || std::fabs(taps[r - j]) >= cut) r32 = j;
  };
  b->lane_q = 0;
  for (int q : {4, 2, 1}) {
    if ((b->lane_q_req != 0 && q != b->lane_q_req) || kp % q != 0) continue;
    bool fits = true;
    for (int i = 0; i < cnt && fits; ++i) {
      BatchInst I{};
      stencil(i, I);
      std::vector<double> taps;
      int r = 0, r32 = 0;
      lane_band(I, q, taps, r, r32);
      fits = r32 <= BATCH_MAX_R;
    }
    if (fits) {
      b->lane_q = q;
      break;
    }
  }
  if (b->lane_q == 0)
    return bfail(b, PXA_ERR_INVALID, b->lane_q_req != 0 && kp % b->lane_q_req != 0
                                         ? "the requested CN steps per lane band do not divide K/P"
                                         : "a problem's CN band is wider than the lanes hold");
  for (int i = 0; i < cnt; ++i) {
    const int n = b->n[i];
    BatchInst& I = b->hinst[i];
    stencil(i, I);
    std::vector<double> taps;
    int r = 0, r32 = 0;
    lane_band(I, b->lane_q, taps, r, r32);
    I.r64 = r;
    I.r32 = r32;
    I.t64 = (int64_t)t64.size();
    I.t32 = (int64_t)t32.size();
    t64.insert(t64.end(), taps.begin(), taps.end());
    for (int j = -r32; j <= r32; ++j) t32.push_back((float)taps[r + j]);
    // the subinterval propagator M^(K/P) as one band, kept to 2^-36 of its largest tap
    // (far below FP32 rounding); problems whose band is wider step instead
    I.rp = 0;
    I.tpw = 0;
    if (b->power && P > 1) {
      std::vector<double> pt;
      int rp = 0;
      cn_power_taps(n, I.am, I.a0, I.ap, dt, kp, 36, pt, rp);
      if (rp <= BATCH_MAX_RP) {
        I.rp = rp;
        I.tpw = (int64_t)t32.size();
        for (double v : pt) t32.push_back((float)v);
      }
    }
    I.off = b->off[i];
    b->off[i + 1] = b->off[i] + n;
    I.voff = (int64_t)(kMaxM + 1) * I.off;
    // Krylov substeps: each spans at most reach * m^2 / ||A||_inf
    const double anorm = std::fabs(I.am) + std::fabs(I.a0) + std::fabs(I.ap);
    const double span = b->reach * (double)b->m * (double)b->m / std::max(anorm, 1e-300);
    I.nsub = std::max(1, (int)std::ceil(tau / span - 1e-12));
    I.hsub = tau / I.nsub;
    b->nmax = std::max(b->nmax, n);
    b->r32max = std::max(b->r32max, r32);
    b->r64max = std::max(b->r64max, r);
    b->rpmax = std::max(b->rpmax, I.rp);
    b->subs_max = std::max(b->subs_max, I.nsub);
  }
  b->total = b->off[cnt];
  // work lists, largest lanes first
  std::vector<int> order(cnt);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const double cx = (double)b->hinst[x].n * (2 * b->hinst[x].r32 + 1);
    const double cy = (double)b->hinst[y].n * (2 * b->hinst[y].r32 + 1);
    return cx > cy;
  });
  std::vector<int2> ipar, iser;
  for (int p = 0; p < P; ++p)
    for (int i : order) ipar.push_back(make_int2(i, p));
  for (int i : order) iser.push_back(make_int2(i, 0));
  // P lanes of every problem, ordered by cost within each lane index: the problems'
  // largest lanes start first across the whole grid
  std::stable_sort(ipar.begin(), ipar.end(), [&](const int2& x, const int2& y) {
    const double cx = (double)b->hinst[x.x].n * (2 * b->hinst[x.x].r32 + 1);
    const double cy = (double)b->hinst[y.x].n * (2 * b->hinst[y.x].r32 + 1);
    return cx > cy;
  });
  // homogeneous propagation per problem: the Krylov exponential (FP64, one block per
  // problem: nsub substeps of an m-step Arnoldi with CGS2, ~2 m^2 n + 10 m n flop, at
  // one SM's FP64 rate) or the stepper's own propagator: one product with the band of
  // M^(K/P) per link where it exists, else k CN steps per link, in FP32 at one SM's FP32
  // rate but at least ~0.5 us per product (the latency of its barrier and band loads)
  const int64_t k = b->K / P;
  std::vector<int> kry;
  std::vector<int2> istep, ipow;
  for (int i : order) {
    const BatchInst& I = b->hinst[i];
    const double n = I.n, mm = b->m;
    const double t_kry = I.nsub * (2.0 * mm * mm * n + 10.0 * mm * n) / 8.2e9;
    const double t_step = I.rp > 0 ? std::max(2.0 * n * (2 * I.rp + 1) / 2.65e11, 5e-7)
                                   : (double)(k / b->lane_q) * std::max(2.0 * n * (2 * I.r32 + 1) / 2.65e11, 5e-7);
    if (P > 1 && t_kry <= b->hom_ratio * t_step)
      kry.push_back(i);
    else if (I.rp > 0)
      ipow.push_back(make_int2(i, 0));
    else
      istep.push_back(make_int2(i, 0));
  }
  std::stable_sort(ipow.begin(), ipow.end(), [&](const int2& x, const int2& y) {
    return (double)b->hinst[x.x].n * (2 * b->hinst[x.x].rp + 1) > (double)b->hinst[y.x].n * (2 * b->hinst[y.x].rp + 1);
  });
  b->uses_krylov.assign(cnt, 0);
  for (int i : kry) b->uses_krylov[i] = 1;
  b->n_kry = (int)kry.size();
  b->n_step = (int)istep.size();
  b->n_pow = (int)ipow.size();
  int rc;
  const size_t tot = (size_t)b->total;
  if ((rc = balloc(b, &b->inst, cnt))) return rc;
  if ((rc = balloc(b, &b->taps32, t32.size()))) return rc;
  if ((rc = balloc(b, &b->taps64, t64.size()))) return rc;
  if ((rc = balloc(b, &b->items_par, ipar.size()))) return rc;
  if ((rc = balloc(b, &b->items_ser, iser.size()))) return rc;
  if ((rc = balloc(b, &b->items_step, istep.size()))) return rc;
  if ((rc = balloc(b, &b->items_pow, ipow.size()))) return rc;
  if ((rc = balloc(b, &b->kry_list, kry.size()))) return rc;
  if ((rc = balloc(b, &b->counter, 1))) return rc;
  if ((rc = balloc(b, &b->status, 1))) return rc;
  // the queue of the one-launch schedule (Paraexp, no Krylov problems): sources; the
  // direct lanes in the order above, each problem's chain + superposition placed one
  // grid's worth of items after its last lane (so that its lanes are usually done when a
  // block takes it); then the adjoint lanes and each problem's adjoint chain + gradient
  // in the same way. Every item comes after the items it depends on.
  b->flow_grid = batch_flow_grid(b->device, b->nmax, b->r32max, b->rpmax);
  std::vector<int4> flow;
  if (P > 1 && kry.empty()) {
    for (int i : order) flow.push_back(make_int4(0, i, 0, 0));
    for (int phase = 0; phase < 2; ++phase) {
      std::vector<std::pair<double, int4>> keyed;
      std::vector<double> last(cnt, -1.0);
      for (size_t x = 0; x < ipar.size(); ++x) {
        keyed.push_back({(double)x, make_int4(phase ? 3 : 1, ipar[x].x, ipar[x].y, 0)});
        last[ipar[x].x] = (double)x;
      }
      for (int i = 0; i < cnt; ++i) keyed.push_back({last[i] + b->flow_grid + 0.5, make_int4(phase ? 4 : 2, i, 0, 0)});
      std::stable_sort(keyed.begin(), keyed.end(),
                       [](const std::pair<double, int4>& x, const std::pair<double, int4>& y) { return x.first < y.first; });
      for (auto& kv : keyed) flow.push_back(kv.second);
    }
  }
  b->n_flow = (int)flow.size();
  if (!flow.empty()) {
    if ((rc = balloc(b, &b->items_flow, flow.size()))) return rc;
    if ((rc = balloc(b, &b->flow_state, 1 + 4 * (size_t)cnt))) return rc;
    BCUDA(b, cudaMemcpy(b->items_flow, flow.data(), sizeof(int4) * flow.size(), cudaMemcpyHostToDevice), "copy queue");
  }
  if ((rc = balloc(b, &b->errmax, 1))) return rc;
  if ((rc = balloc(b, &b->src, tot))) return rc;
  if ((rc = balloc(b, &b->E, (size_t)P * tot))) return rc;
  if ((rc = balloc(b, &b->EA, (size_t)P * tot))) return rc;
  if ((rc = balloc(b, &b->h, tot))) return rc;
  if ((rc = balloc(b, &b->hA, tot))) return rc;
  if ((rc = balloc(b, &b->qT, tot))) return rc;
  if ((rc = balloc(b, &b->srcT, tot))) return rc;
  if (!kry.empty() && (rc = balloc(b, &b->V, (size_t)(kMaxM + 1) * tot))) return rc;
  BCUDA(b, cudaMemcpy(b->inst, b->hinst.data(), sizeof(BatchInst) * cnt, cudaMemcpyHostToDevice), "copy problems");
  BCUDA(b, cudaMemcpy(b->taps32, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice), "copy bands");
  BCUDA(b, cudaMemcpy(b->taps64, t64.data(), sizeof(double) * t64.size(), cudaMemcpyHostToDevice), "copy bands");
  BCUDA(b, cudaMemcpy(b->items_par, ipar.data(), sizeof(int2) * ipar.size(), cudaMemcpyHostToDevice), "copy lanes");
  BCUDA(b, cudaMemcpy(b->items_ser, iser.data(), sizeof(int2) * iser.size(), cudaMemcpyHostToDevice), "copy lanes");
  if (!istep.empty())
    BCUDA(b, cudaMemcpy(b->items_step, istep.data(), sizeof(int2) * istep.size(), cudaMemcpyHostToDevice),
          "copy chains");
  if (!ipow.empty())
    BCUDA(b, cudaMemcpy(b->items_pow, ipow.data(), sizeof(int2) * ipow.size(), cudaMemcpyHostToDevice),
          "copy chains");
  if (!kry.empty())
    BCUDA(b, cudaMemcpy(b->kry_list, kry.data(), sizeof(int) * kry.size(), cudaMemcpyHostToDevice), "copy chains");
  BCUDA(b, cudaMemset(b->status, 0, sizeof(int)), "reset status");
  if (!b->side) {
    BCUDA(b, cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking), "side stream");
    BCUDA(b, cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming), "event");
    BCUDA(b, cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming), "event");
  }
  b->lanes_grid = batch_lanes_grid(b->device, b->nmax, b->r32max);
  b->pow_grid = b->rpmax > 0 ? batch_lanes_grid(b->device, b->nmax, b->rpmax) : 1;
  BCUDA(b, cudaGetLastError(), "lane grid");
  b->ready = true;
  return PXA_OK;
}

// The whole gradient of every problem on stream st.
int benqueue(pxa_batch* b, cudaStream_t st, int mode, const double* q0, double* J, double* grad) {
  const int cnt = b->count, P = mode == PXA_SERIAL ? 1 : b->P;
  // band applications of M^q: K / q for a serial lane, K / (P q) per subinterval
  const int64_t K = b->K / b->lane_q, k = b->K / b->P / b->lane_q;
  auto mark = [&](int i) {
    if (b->timing && b->ev[i]) cudaEventRecord(b->ev[i], st);
  };
  mark(0);
  BCUDA(b, cudaMemsetAsync(b->errmax, 0, sizeof(double), st), "reset estimate");
  if (P == 1) {
    // plain serial stepping of every problem: K steps from q0, then K transposed steps
    BCUDA(b, launch_batch_cn_lanes(st, std::min(b->lanes_grid, cnt), b->inst, b->items_ser, cnt, b->counter, b->taps32, 0, K,
                                   q0, nullptr, b->E, 1, b->nmax, b->r32max), "serial lanes");
    mark(1);
    mark(2);
    BCUDA(b, launch_batch_superpose_direct(st, b->inst, cnt, b->nmax, b->taps64, nullptr, b->E, 1, 0, nullptr,
                                           b->qT, nullptr, J, b->status), "objective");
    BCUDA(b, launch_batch_cn_lanes(st, std::min(b->lanes_grid, cnt), b->inst, b->items_ser, cnt, b->counter, b->taps32, 1, K,
                                   b->qT, nullptr, b->EA, 1, b->nmax, b->r32max), "serial adjoint lanes");
    mark(3);
    mark(4);
    BCUDA(b, launch_batch_superpose_adjoint(st, b->inst, cnt, b->nmax, nullptr, b->EA, 1, nullptr, grad,
                                            b->status), "gradient");
    mark(5);
    return PXA_OK;
  }
  b->flow_last = b->schedule == 1 && b->n_flow > 0;
  if (b->flow_last) {
    // one persistent launch: every phase of every problem, ordered by device-side counters
    BCUDA(b, launch_batch_flow(st, b->flow_grid, b->inst, b->items_flow, b->n_flow, b->flow_state, cnt, P,
                               b->taps32, b->taps64, k, q0, b->src, b->E, b->qT, b->srcT, b->EA, J, grad,
                               b->status, b->nmax, b->r32max, b->rpmax), "one-launch gradient");
    mark(1);
    mark(2);
    mark(3);
    mark(4);
    mark(5);
    return PXA_OK;
  }
  // Eq. linzero: lanes of the shifted problem with the source (M - I) q0
  BCUDA(b, launch_batch_band_src(st, b->inst, cnt, b->nmax, b->taps64, 0, q0, b->src), "sources");
  BCUDA(b, launch_batch_cn_lanes(st, std::min(b->lanes_grid, cnt * P), b->inst, b->items_par, cnt * P, b->counter, b->taps32, 0, k,
                                 nullptr, b->src, b->E, P, b->nmax, b->r32max), "lanes");
  mark(1);
  // the Krylov chains (one block per problem, FP64) beside the stepped ones
  BCUDA(b, cudaEventRecord(b->ev_fork, st), "fork");
  BCUDA(b, cudaStreamWaitEvent(b->side, b->ev_fork, 0), "fork wait");
  BCUDA(b, launch_batch_chain(b->side, b->inst, b->kry_list, b->n_kry, b->nmax, b->m, 0, b->E, P, 0, 1, P - 1,
                              b->h, b->V, b->tol, b->status, b->errmax), "chains");
  BCUDA(b, cudaEventRecord(b->ev_join, b->side), "join");
  BCUDA(b, launch_batch_cn_chain(st, std::min(b->lanes_grid, std::max(b->n_step, 1)), b->inst, b->items_step, b->n_step, b->counter, b->taps32, 0, k,
                                 b->E, P, 0, 1, P - 1, b->h, b->nmax, b->r32max, 0), "stepped chains");
  BCUDA(b, launch_batch_cn_chain(st, std::min(b->pow_grid, std::max(b->n_pow, 1)), b->inst, b->items_pow, b->n_pow,
                                 b->counter, b->taps32, 0, k, b->E, P, 0, 1, P - 1, b->h, b->nmax, b->rpmax, 1),
        "propagator-band chains");
  BCUDA(b, cudaStreamWaitEvent(st, b->ev_join, 0), "join wait");
  mark(2);
  BCUDA(b, launch_batch_superpose_direct(st, b->inst, cnt, b->nmax, b->taps64, q0, b->E, P, P - 1, b->h, b->qT,
                                         b->srcT, J, b->status), "superposition");
  BCUDA(b, launch_batch_cn_lanes(st, std::min(b->lanes_grid, cnt * P), b->inst, b->items_par, cnt * P, b->counter, b->taps32, 1, k,
                                 nullptr, b->srcT, b->EA, P, b->nmax, b->r32max), "adjoint lanes");
  mark(3);
  BCUDA(b, cudaEventRecord(b->ev_fork, st), "fork");
  BCUDA(b, cudaStreamWaitEvent(b->side, b->ev_fork, 0), "fork wait");
  BCUDA(b, launch_batch_chain(b->side, b->inst, b->kry_list, b->n_kry, b->nmax, b->m, 1, b->EA, P, P - 1, -1,
                              P - 1, b->hA, b->V, b->tol, b->status, b->errmax), "adjoint chains");
  BCUDA(b, cudaEventRecord(b->ev_join, b->side), "join");
  BCUDA(b, launch_batch_cn_chain(st, std::min(b->lanes_grid, std::max(b->n_step, 1)), b->inst, b->items_step, b->n_step, b->counter, b->taps32, 1, k,
                                 b->EA, P, P - 1, -1, P - 1, b->hA, b->nmax, b->r32max, 0), "stepped adjoint chains");
  BCUDA(b, launch_batch_cn_chain(st, std::min(b->pow_grid, std::max(b->n_pow, 1)), b->inst, b->items_pow, b->n_pow,
                                 b->counter, b->taps32, 1, k, b->EA, P, P - 1, -1, P - 1, b->hA, b->nmax, b->rpmax, 1),
        "propagator-band adjoint chains");
  BCUDA(b, cudaStreamWaitEvent(st, b->ev_join, 0), "join wait");
  mark(4);
  BCUDA(b, launch_batch_superpose_adjoint(st, b->inst, cnt, b->nmax, b->qT, b->EA, P, b->hA, grad, b->status),
        "gradient");
  mark(5);
  return PXA_OK;
}

int bread_status(pxa_batch* b) {
  if (b->timing && b->ev[0]) {
    for (int i = 0; i < 4; ++i)
      if (cudaEventElapsedTime(&b->ms[i], b->ev[i], b->ev[i + 1]) != cudaSuccess) {
        cudaGetLastError();
        b->ms[i] = -1.f;
      }
    if (cudaEventElapsedTime(&b->ms[4], b->ev[0], b->ev[5]) != cudaSuccess) {
      cudaGetLastError();
      b->ms[4] = -1.f;
    }
  }
  int st = 0;
  BCUDA(b, cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  double e = 0.0;
  BCUDA(b, cudaMemcpy(&e, b->errmax, sizeof(double), cudaMemcpyDeviceToHost), "read estimate");
  b->err_last = e;
  if (st != 0) {
    BCUDA(b, cudaMemset(b->status, 0, sizeof(int)), "reset status");
    return bfail(b, st, st == PXA_ERR_NOT_CONVERGED ? "Krylov estimate above the tolerance"
                        : st == PXA_ERR_NONFINITE ? "non-finite objective or gradient"
                                                  : "device error");
  }
  return PXA_OK;
}

}  // namespace

extern "C" {

int pxa_batch_create(pxa_batch** out, int device, void* cuda_stream) {
  if (!out) return PXA_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return PXA_ERR_CUDA;
  }
  pxa_batch* b = new pxa_batch();
  b->device = device;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->L = 2.0 * 3.14159265358979323846;
  *out = b;
  return PXA_OK;
}

void pxa_batch_destroy(pxa_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  brelease(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  delete b;
}

const char* pxa_batch_last_error(const pxa_batch* b) { return b ? b->err.c_str() : "null batch"; }

int pxa_batch_set(pxa_batch* b, int count, const int* n, const double* nu, double c, double L, double T,
                  int64_t K, int P) {
  if (!b || count < 1 || !n || !nu) return PXA_ERR_INVALID;
  if (!(L > 0.0) || !(T > 0.0) || K < 1 || P < 1 || P > 64 || K % P != 0 || !std::isfinite(c))
    return bfail(b, PXA_ERR_INVALID, "need L > 0, T > 0, K % P == 0, 1 <= P <= 64");
  for (int i = 0; i < count; ++i)
    if (n[i] < 16 || n[i] > BATCH_MAX_N || !(nu[i] >= 0.0))
      return bfail(b, PXA_ERR_INVALID, "problem " + std::to_string(i) + ": need 16 <= n <= 4096 and nu >= 0");
  b->count = count;
  b->n.assign(n, n + count);
  b->nu.assign(nu, nu + count);
  b->c = c;
  b->L = L;
  b->T = T;
  b->K = K;
  b->P = P;
  brelease(b);
  return PXA_OK;
}

int pxa_batch_set_krylov(pxa_batch* b, int m, double tol, double reach) {
  if (!b || m < 2 || m > kMaxM || !(tol > 0.0) || !(reach > 0.0)) return PXA_ERR_INVALID;
  b->m = m;
  b->tol = tol;
  b->reach = reach;
  brelease(b);
  return PXA_OK;
}

int pxa_batch_set_homogeneous(pxa_batch* b, double ratio) {
  if (!b || !(ratio >= 0.0)) return PXA_ERR_INVALID;
  b->hom_ratio = ratio;
  brelease(b);
  return PXA_OK;
}

int pxa_batch_set_power(pxa_batch* b, int enable) {
  if (!b) return PXA_ERR_INVALID;
  b->power = enable != 0;
  brelease(b);
  return PXA_OK;
}

int pxa_batch_set_lane_steps(pxa_batch* b, int q) {
  if (!b || (q != 0 && q != 1 && q != 2 && q != 4)) return PXA_ERR_INVALID;
  b->lane_q_req = q;
  brelease(b);
  return PXA_OK;
}

int pxa_batch_set_timing(pxa_batch* b, int enable) {
  if (!b) return PXA_ERR_INVALID;
  BCUDA(b, cudaSetDevice(b->device), "cudaSetDevice");
  if (enable && !b->ev[0])
    for (auto& e : b->ev) BCUDA(b, cudaEventCreate(&e), "event");
  b->timing = enable != 0;
  return PXA_OK;
}

int pxa_batch_set_schedule(pxa_batch* b, int one_launch) {
  if (!b || (one_launch != 0 && one_launch != 1)) return PXA_ERR_INVALID;
  b->schedule = one_launch;
  binvalidate(b);
  return PXA_OK;
}

int pxa_batch_set_graph(pxa_batch* b, int enable) {
  if (!b) return PXA_ERR_INVALID;
  b->use_graph = enable != 0;
  binvalidate(b);
  return PXA_OK;
}

int pxa_batch_gradient(pxa_batch* b, int mode, const double* q0_dev, double* J_dev, double* grad_dev) {
  if (!b || !q0_dev || !J_dev || !grad_dev || (mode != PXA_SERIAL && mode != PXA_PARAEXP))
    return PXA_ERR_INVALID;
  BCUDA(b, cudaSetDevice(b->device), "cudaSetDevice");
  int rc = bprepare(b);
  if (rc) return rc;
  if (!b->use_graph || b->timing) return benqueue(b, b->stream, mode, q0_dev, J_dev, grad_dev);
  if (!b->gexec || b->g_mode != mode || b->g_q0 != q0_dev || b->g_J != J_dev || b->g_grad != grad_dev) {
    binvalidate(b);
    if (!b->cap_stream) BCUDA(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "capture stream");
    cudaGraph_t g;
    BCUDA(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
    const int erc = benqueue(b, b->cap_stream, mode, q0_dev, J_dev, grad_dev);
    const cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (erc) {
      if (e == cudaSuccess) cudaGraphDestroy(g);
      return erc;
    }
    BCUDA(b, e, "end capture");
    b->graph_kernels = graph_kernel_nodes(g);
    const cudaError_t ei = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    BCUDA(b, ei, "graph instantiate");
    b->g_mode = mode;
    b->g_q0 = q0_dev;
    b->g_J = J_dev;
    b->g_grad = grad_dev;
  }
  BCUDA(b, cudaGraphLaunch(b->gexec, b->stream), "graph launch");
  return PXA_OK;
}

int pxa_batch_sync(pxa_batch* b) {
  if (!b) return PXA_ERR_INVALID;
  if (!b->ready) return PXA_OK;
  BCUDA(b, cudaStreamSynchronize(b->stream), "stream sync");
  return bread_status(b);
}

int pxa_batch_autotune(pxa_batch* b, int mode, const double* q0_dev, double* J_dev, double* grad_dev,
                       double* best_ms_host) {
  if (!b || !q0_dev || !J_dev || !grad_dev) return PXA_ERR_INVALID;
  BCUDA(b, cudaSetDevice(b->device), "cudaSetDevice");
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0), "event");
  BCUDA(b, cudaEventCreate(&e1), "event");
  struct Cand { int m; double reach, ratio; };
  std::vector<Cand> cands;
  if (mode == PXA_PARAEXP && b->P > 1) {
    for (double q : {0.0, 0.25, 1.0, 4.0}) cands.push_back({32, 0.04, q});
    for (double r : {0.02, 0.04}) cands.push_back({32, r, 1e30});
    cands.push_back({40, 0.04, 1e30});
    cands.push_back({24, 0.04, 1.0});
  } else {
    cands.push_back({b->m, b->reach, b->hom_ratio});
  }
  const int m0 = b->m;
  const double r0 = b->hom_ratio, reach0 = b->reach;
  double best = 1e300;
  Cand bc{-1, 0.0, 0.0};
  for (const Cand& cd : cands) {
    b->m = cd.m;
    b->reach = cd.reach;
    b->hom_ratio = cd.ratio;
    brelease(b);
    int rc = pxa_batch_gradient(b, mode, q0_dev, J_dev, grad_dev);
    if (rc == PXA_OK) rc = pxa_batch_sync(b);
    if (rc) {
      if (rc == PXA_ERR_CUDA) break;
      continue;
    }
    double t = 1e300;
    for (int rep = 0; rep < 2 && rc == PXA_OK; ++rep) {
      BCUDA(b, cudaEventRecord(e0, b->stream), "record");
      rc = pxa_batch_gradient(b, mode, q0_dev, J_dev, grad_dev);
      BCUDA(b, cudaEventRecord(e1, b->stream), "record");
      BCUDA(b, cudaEventSynchronize(e1), "sync");
      if (rc == PXA_OK) rc = bread_status(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t = std::min(t, (double)ms);
    }
    if (rc) continue;
    if (t < best) {
      best = t;
      bc = cd;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (bc.m < 0) {
    b->m = m0;
    b->hom_ratio = r0;
    b->reach = reach0;
    brelease(b);
    return bfail(b, PXA_ERR_NOT_CONVERGED, "no autotuner candidate met the Krylov tolerance");
  }
  b->m = bc.m;
  b->reach = bc.reach;
  b->hom_ratio = bc.ratio;
  brelease(b);
  if (best_ms_host) *best_ms_host = best;
  return bprepare(b);
}

int pxa_batch_offsets(const pxa_batch* b, int64_t* offsets) {
  if (!b || !offsets || b->count <= 0) return PXA_ERR_INVALID;
  int64_t o = 0;
  for (int i = 0; i < b->count; ++i) {
    offsets[i] = o;
    o += b->n[i];
  }
  offsets[b->count] = o;
  return PXA_OK;
}

int pxa_batch_problem_info(const pxa_batch* b, int* taps32, int* taps64, int* krylov) {
  if (!b || !b->ready) return PXA_ERR_INVALID;
  for (int i = 0; i < b->count; ++i) {
    if (taps32) taps32[i] = 2 * b->hinst[i].r32 + 1;
    if (taps64) taps64[i] = 2 * b->hinst[i].r64 + 1;
    if (krylov) krylov[i] = b->uses_krylov[i];
  }
  return PXA_OK;
}

int pxa_batch_get_stats(const pxa_batch* b, pxa_batch_stats* out) {
  if (!b || !out) return PXA_ERR_INVALID;
  pxa_batch_stats s{};
  s.count = b->count;
  s.points = b->ready ? b->total : 0;
  s.krylov_m = b->m;
  s.krylov_reach = b->reach;
  s.substeps_max = b->subs_max;
  s.band32_max = 2 * b->r32max + 1;
  s.band64_max = 2 * b->r64max + 1;
  s.lanes_grid = b->lanes_grid;
  s.one_launch = b->flow_last ? 1 : 0;
  s.flow_grid = b->flow_grid;
  s.graph_kernels = b->graph_kernels;
  s.krylov_err_max = b->err_last;
  s.workspace_bytes = b->bytes;
  s.krylov_problems = b->n_kry;
  s.power_problems = b->n_pow;
  s.band_power_max = b->rpmax > 0 ? 2 * b->rpmax + 1 : 0;
  s.lane_steps = b->ready ? b->lane_q : 0;
  s.hom_ratio = b->hom_ratio;
  s.ms_lanes = b->ms[0];
  s.ms_chains = b->ms[1];
  s.ms_adjoint_lanes = b->ms[2];
  s.ms_adjoint_chains = b->ms[3];
  s.ms_total = b->ms[4];
  *out = s;
  return PXA_OK;
}

}  // extern "C"
