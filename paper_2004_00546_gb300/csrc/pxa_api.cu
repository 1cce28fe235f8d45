// pxa_api.cu — the C ABI of libpxa (declared in include/pxa.h): context, workspace,
// orchestration of the Paraexp direct-adjoint loop on one stream, CUDA-graph replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pxa.h"
#include "kernels_bu2.cuh"
#include "kernels_csr.cuh"
#include "kernels_1d.cuh"
#include "kernels_ad2.cuh"

using namespace pxa;

namespace pxa {

int graph_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  int k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

template <typename Real>
static void cn_band_taps_t(int n, double am, double a0, double ap, double dt, int cut_exp,
                           std::vector<double>& taps, int& r) {
  typedef std::complex<Real> C;
  const Real pi = (Real)3.141592653589793238462643383279502884L;
  std::vector<C> R(n), w(n);
  for (int k = 0; k < n; ++k) {
    Real ph = (Real)2 * pi * (Real)k / (Real)n;
    w[k] = C(std::cos(ph), std::sin(ph));
  }
  const Real th = (Real)0.5 * (Real)dt;
  for (int k = 0; k < n; ++k) {
    C lam = (Real)a0 + (Real)am * std::conj(w[k]) + (Real)ap * w[k];
    R[k] = ((Real)1 + th * lam) / ((Real)1 - th * lam);
  }
  auto tap = [&](int j) {
    C s = (Real)0;
    for (int k = 0; k < n; ++k) {
      long long idx = ((long long)k * (long long)(((j % n) + n) % n)) % n;
      s += R[k] * std::conj(w[idx]);
    }
    return (double)(s.real() / (Real)n);
  };
  std::vector<double> pos, neg;  // pos[j] = m_j, neg[j] = m_-j
  double m0 = tap(0);
  pos.push_back(m0);
  neg.push_back(m0);
  const double thr = std::ldexp(std::fabs(m0), -cut_exp);
  // widest band: every offset once; for even n the offset n/2 equals -n/2 and is
  // stored once (on the negative side)
  const int rmax = n / 2;
  r = 0;
  for (int j = 1; j <= rmax; ++j) {
    double mn = tap(-j);
    double mp = (2 * j == n) ? 0.0 : tap(j);
    pos.push_back(mp);
    neg.push_back(mn);
    r = j;
    if (std::fabs(mp) < thr && std::fabs(mn) < thr) break;  // the tail is below the cut
  }
  taps.assign(2 * r + 1, 0.0);
  for (int j = -r; j <= r; ++j) taps[r + j] = j >= 0 ? pos[j] : neg[-j];
}

// Taps m_j (|j| <= r) of the circulant Crank–Nicolson map
//   M = (I - dt/2 A)^{-1} (I + dt/2 A),  (M x)_i = sum_j m_j x_{i+j},
// from its eigenvalues R_k = (1 + dt/2 lam_k)/(1 - dt/2 lam_k), lam_k = a0 + am w^-k + ap w^k,
// by the inverse DFT m_j = (1/n) sum_k R_k w^{-kj}. The taps decay geometrically (the
// implicit matrix is diagonally dominant); the band stops where both |m_r| and |m_-r| fall
// below 2^-64 |m_0| (long double sums, n <= 65536), far under FP64 rounding of the step,
// or below 2^-50 |m_0| (double sums, longer grids, used by the FP32 lane kernels only);
// when they do not decay within n/2 the full circulant is used.
void cn_band_taps(int n, double am, double a0, double ap, double dt, std::vector<double>& taps, int& r) {
  if (n <= 65536)
    cn_band_taps_t<long double>(n, am, a0, ap, dt, 64, taps, r);
  else
    cn_band_taps_t<double>(n, am, a0, ap, dt, 50, taps, r);
}

// Taps m_j (|j| <= r) of the power M^steps of the circulant Crank-Nicolson map: the
// propagator of the stepper over `steps` steps, itself circulant with eigenvalues R_k^steps
// (R_k as in cn_band_taps; powers by repeated squaring, double sums); with expo, of
// exp(steps dt A) (eigenvalues exp(steps dt lam_k)). Advection shifts its
// peak by about (am - ap) steps dt points, so the band is cut relative to the largest tap:
// past the shift, once both |m_j| and |m_-j| stay below 2^-cut_exp max|m| for four
// consecutive offsets (or at n/2, the full circulant). The band is stored symmetric.
void cn_power_taps(int n, double am, double a0, double ap, double dt, int64_t steps, int cut_exp,
                   std::vector<double>& taps, int& r, bool expo) {
  typedef std::complex<double> C;
  const double pi = 3.141592653589793238462643383279502884;
  std::vector<C> Rp(n), w(n);
  for (int k = 0; k < n; ++k) {
    const double ph = 2.0 * pi * (double)k / (double)n;
    w[k] = C(std::cos(ph), std::sin(ph));
  }
  const double th = 0.5 * dt;
  for (int k = 0; k < n; ++k) {
    const C lam = a0 + am * std::conj(w[k]) + ap * w[k];
    if (expo) {  // exp(steps dt A) instead of the CN power
      Rp[k] = std::exp((double)steps * dt * lam);
      continue;
    }
    C base = (1.0 + th * lam) / (1.0 - th * lam), acc = 1.0;
    for (int64_t e = steps; e > 0; e >>= 1) {
      if (e & 1) acc *= base;
      base *= base;
    }
    Rp[k] = acc;
  }
  auto tap = [&](int j) {
    C s = 0.0;
    const long long jj = ((j % n) + n) % n;
    for (int k = 0; k < n; ++k) s += Rp[k] * std::conj(w[(size_t)(((long long)k * jj) % n)]);
    return s.real() / (double)n;
  };
  const double shift = std::fabs(am - ap) * (double)steps * dt;
  std::vector<double> pos, neg;  // pos[j] = m_j, neg[j] = m_-j
  const double m0 = tap(0);
  pos.push_back(m0);
  neg.push_back(m0);
  double big = std::fabs(m0);
  const int rmax = n / 2;
  int quiet = 0;
  r = 0;
  for (int j = 1; j <= rmax; ++j) {
    const double mn = tap(-j);
    const double mp = (2 * j == n) ? 0.0 : tap(j);
    pos.push_back(mp);
    neg.push_back(mn);
    r = j;
    big = std::max(big, std::max(std::fabs(mp), std::fabs(mn)));
    const double thr = std::ldexp(big, -cut_exp);
    quiet = (std::fabs(mp) < thr && std::fabs(mn) < thr) ? quiet + 1 : 0;
    if ((double)j > shift + 4.0 && quiet >= 4) break;
  }
  taps.assign(2 * r + 1, 0.0);
  for (int j = -r; j <= r; ++j) taps[r + j] = j >= 0 ? pos[j] : neg[-j];
}

// Real Leja points method (Sec. 4.1), host part. Leja points of [-2, 2]: 2 first, then
// each point maximises the sum of log distances to the earlier ones, searched on a
// uniform grid of 2^15 + 1 points.
static void leja_host(int m1, std::vector<double>& xi) {
  const int G = 32769;
  std::vector<double> acc(G, 0.0);
  std::vector<char> taken(G, 0);
  xi.assign(m1, 0.0);
  int g = G - 1;
  for (int j = 0; j < m1; ++j) {
    const double x = -2.0 + 4.0 * g / (G - 1);
    xi[j] = x;
    taken[g] = 1;
    int best = 0;
    double bv = -1e300;
    for (int q = 0; q < G; ++q) {
      if (taken[q]) continue;
      acc[q] += std::log(std::fabs(-2.0 + 4.0 * q / (G - 1) - x));
      if (acc[q] > bv) {
        bv = acc[q];
        best = q;
      }
    }
    g = best;
  }
}

// exp of a d x d row-major matrix in double: Taylor polynomial of degree 18 at norm <= 1/2
// (remainder below 1e-23), then repeated squaring.
static void expm_host(int d, std::vector<double> A, std::vector<double>& E) {
  double nrm = 0.0;
  for (int i = 0; i < d; ++i) {
    double r = 0.0;
    for (int j = 0; j < d; ++j) r += std::fabs(A[(size_t)i * d + j]);
    nrm = std::max(nrm, r);
  }
  int sq = 0;
  while (nrm > 0.5) {
    nrm *= 0.5;
    ++sq;
  }
  const double sc = std::ldexp(1.0, -sq);
  for (double& v : A) v *= sc;
  std::vector<double> term((size_t)d * d, 0.0), next((size_t)d * d);
  E.assign((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i) term[(size_t)i * d + i] = E[(size_t)i * d + i] = 1.0;
  for (int k = 1; k <= 18; ++k) {
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        double s = 0.0;
        for (int l = 0; l < d; ++l) s += term[(size_t)i * d + l] * A[(size_t)l * d + j];
        next[(size_t)i * d + j] = s / k;
      }
    term.swap(next);
    for (size_t e = 0; e < E.size(); ++e) E[e] += term[e];
  }
  for (int r = 0; r < sq; ++r) {
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        double s = 0.0;
        for (int l = 0; l < d; ++l) s += E[(size_t)i * d + l] * E[(size_t)l * d + j];
        next[(size_t)i * d + j] = s;
      }
    E.swap(next);
  }
}

// Substeps, nodes and Newton divided differences for the homogeneous propagator over a
// span t. steps == 0: exp(t A), interpolating phi(z) = (e^z - 1)/z (exp(B) = I + B phi(B));
// steps > 0: the Crank-Nicolson power R(dt A)^steps with dt = t / steps, interpolated
// directly as f(z) = R(z/m)^m on each substep of m steps (R(x) = (1 + x/2)/(1 - x/2)).
// The spectrum of A is the ellipse a0 + (am + ap) cos th + i (ap - am) sin th: centre
// a0, semi-axes |am + ap| (real) and |ap - am| (imaginary). Its confocal family with real
// foci a0 +- f, f^2 = max(|am+ap|^2 - |ap-am|^2, 0), gives the focal interval; substeps
// keep the capacity of the smallest such ellipse containing the spectrum <= 4 per
// substep (for the CN power, the smallest divisor of `steps` that does). Divided
// differences by Opitz's theorem: the first column of f(Z), Z lower bidiagonal (nodes on
// the diagonal, ones below); for phi read off exp([[Z, e_1], [0, 0]]).
void relpm_setup_host(double t, double am, double a0, double ap, int mmax, int& nsub, double& ts,
                      std::vector<double>& z, std::vector<double>& D, int64_t steps) {
  const double ra = std::fabs(am + ap), ib = std::fabs(ap - am);
  const double f = std::sqrt(std::max(ra * ra - ib * ib, 0.0));
  const double cap = 0.5 * (std::max(ra, std::sqrt(ib * ib + f * f)) + ib);
  nsub = std::max(1, (int)std::ceil(std::fabs(t) * cap / 4.0 - 1e-12));
  if (steps > 0) {
    while (nsub < steps && steps % nsub != 0) ++nsub;
    if (nsub > steps) nsub = (int)steps;
  }
  ts = t / nsub;
  std::vector<double> xi;
  leja_host(mmax + 1, xi);
  z.resize(mmax + 1);
  for (int j = 0; j <= mmax; ++j) z[j] = ts * a0 + 0.5 * ts * f * xi[j];
  D.resize(mmax + 1);
  if (steps == 0) {
    const int d = mmax + 2;
    std::vector<double> M((size_t)d * d, 0.0), E;
    for (int i = 0; i <= mmax; ++i) {
      M[(size_t)i * d + i] = z[i];
      if (i > 0) M[(size_t)i * d + i - 1] = 1.0;
    }
    M[(size_t)mmax + 1] = 1.0;  // row 0, column mmax + 1
    expm_host(d, M, E);
    for (int i = 0; i <= mmax; ++i) D[i] = E[(size_t)i * d + mmax + 1];
    return;
  }
  // R(Z/m) = (I - Z/(2m))^{-1} (I + Z/(2m)), lower triangular (forward substitution on
  // the lower bidiagonal I - Z/(2m)), then its m-th power by repeated squaring
  const int d = mmax + 1;
  const int64_t m = steps / nsub;
  const double hm = 0.5 / (double)m;
  std::vector<double> R((size_t)d * d, 0.0);
  for (int col = 0; col < d; ++col) {
    // column col of (I + Z/(2m)): 1 + z_col hm on the diagonal, hm below it
    for (int i = col; i < d; ++i) {
      double rhs = i == col ? 1.0 + z[i] * hm : (i == col + 1 ? hm : 0.0);
      if (i > col) rhs += hm * R[(size_t)(i - 1) * d + col];  // (I - Z hm) x = rhs: x_i (1 - z_i hm) - hm x_{i-1}
      R[(size_t)i * d + col] = rhs / (1.0 - z[i] * hm);
    }
  }
  auto mul = [&](const std::vector<double>& X, const std::vector<double>& Y) {
    std::vector<double> W((size_t)d * d, 0.0);
    for (int i = 0; i < d; ++i)
      for (int l = 0; l <= i; ++l) {
        const double x = X[(size_t)i * d + l];
        if (x == 0.0) continue;
        for (int j = 0; j <= l; ++j) W[(size_t)i * d + j] += x * Y[(size_t)l * d + j];
      }
    return W;
  };
  std::vector<double> F((size_t)d * d, 0.0), P = R;
  for (int i = 0; i < d; ++i) F[(size_t)i * d + i] = 1.0;
  for (int64_t e = m; e > 0; e >>= 1) {
    if (e & 1) F = mul(F, P);
    if (e > 1) P = mul(P, P);
  }
  for (int i = 0; i < d; ++i) D[i] = F[(size_t)i * d];
}


// The RK4 stepper's propagator over a chain segment of kk steps as a power series
// (PXA_PROP_POLY). With z = dt A and w = kk z = tau A (tau = kk dt, the segment's length),
// R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 and R(z)^kk = sum_i a_i w^i (degree 4kk; every
// a_i > 0 and a_i <= 1/i!, since R's coefficients do not exceed exp's). The forcing
// gradient that the homogeneous adjoint adds over the segment is sum_j g_j(dt A^T)
// lambda_{j+1} with g_j(z) = dt [s1 (1/6 + z/6 + z^2/12 + z^3/24) + s2 (2/3 + z/3 +
// z^2/12) + s4/6], the derivative of step j's map with respect to the forcing (s1, s2, s4:
// s(t) at its stage times), and lambda_{j+1} = R(dt A^T)^(kk-1-j) h: a polynomial in
// tau A^T applied to h, split into three omega-free families Q_w[j] = dt c_w(z)
// R(z)^(kk-1-j) (w = s1, s2, s4), whose s(t)-weighted sum the device forms per segment.
// Long double throughout; a_full is the whole series, Q is cut after degree m (products
// cut at degree m are exact below it).
void rk4_series_host(int kk, int m, double dt, std::vector<long double>& a_full, std::vector<double>& Q) {
  const long double s = 1.0L / (long double)kk;
  const long double R[5] = {1.0L, s, 0.5L * s * s, s * s * s / 6.0L, s * s * s * s / 24.0L};
  auto times_R = [&](const std::vector<long double>& x, int deg) {
    std::vector<long double> y((size_t)deg + 1, 0.0L);
    for (int i = 0; i < (int)x.size() && i <= deg; ++i)
      for (int r = 0; r < 5 && i + r <= deg; ++r) y[(size_t)i + r] += x[(size_t)i] * R[r];
    return y;
  };
  a_full.assign(1, 1.0L);
  for (int j = 1; j <= kk; ++j) a_full = times_R(a_full, 4 * j);
  // c_w(z) in powers of w = kk z
  const long double c1[4] = {1.0L / 6.0L, s / 6.0L, s * s / 12.0L, s * s * s / 24.0L};
  const long double c2[4] = {2.0L / 3.0L, s / 3.0L, s * s / 12.0L, 0.0L};
  const long double c4[4] = {1.0L / 6.0L, 0.0L, 0.0L, 0.0L};
  const long double* cw[3] = {c1, c2, c4};
  Q.assign((size_t)3 * kk * (m + 1), 0.0);
  std::vector<long double> pw(1, 1.0L);  // R^e cut at degree m, e = 0 first
  for (int e = 0; e < kk; ++e) {
    const int j = kk - 1 - e;
    for (int w = 0; w < 3; ++w)
      for (int i = 0; i <= m; ++i) {
        long double acc = 0.0L;
        for (int r = 0; r < 4 && r <= i; ++r)
          if (i - r < (int)pw.size()) acc += cw[w][r] * pw[(size_t)(i - r)];
        Q[((size_t)w * kk + j) * (m + 1) + i] = (double)((long double)dt * acc);
      }
    pw = times_R(pw, std::min(4 * (e + 1), m));
  }
}

// The plan of a PXA_PROP_POLY chain for k = K/P steps per subinterval: rho = ||dt B||_inf
// for the operator(s) B the chain applies. Segments of kk steps, kk the largest divisor of
// k with kk rho <= 4 (the series' partial sums then stay within e^4 of the result's scale);
// the degree m is the smallest multiple of 4 whose tail bound sum_{i>m} a_i (kk rho)^i is
// <= tol (m <= 4 kk, where the series is the whole polynomial). a_full: the whole series
// in powers of kk dt B.
struct PolyPlan {
  int sub = 1, kk = 1, m = 0;
  double tail = 0.0;
  std::vector<long double> a_full;
};

PolyPlan poly_plan(double rho, int64_t k, double dt, double tol) {
  PolyPlan pl;
  while (pl.sub < k && (k % pl.sub != 0 || (double)(k / pl.sub) * rho > 4.0)) ++pl.sub;
  pl.kk = (int)(k / pl.sub);
  const long double rs = (long double)pl.kk * rho;
  std::vector<double> Q;
  rk4_series_host(pl.kk, 0, dt, pl.a_full, Q);
  pl.m = 4 * pl.kk;
  for (int mm = 4; mm <= 4 * pl.kk; mm += 4) {
    long double t = 0.0L, pr = 1.0L;
    for (int i = 0; i <= 4 * pl.kk; ++i) {
      if (i > mm) t += pl.a_full[(size_t)i] * pr;
      pr *= rs;
    }
    if (t <= (long double)tol) {
      pl.m = mm;
      pl.tail = (double)t;
      break;
    }
  }
  return pl;
}

}  // namespace pxa

struct pxa_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;       // the caller's stream (borrowed)
  cudaStream_t cap_stream = nullptr;   // library-owned stream used to capture graphs
  std::string err;

  // configuration
  bool have_op = false, have_time = false;
  pxa_operator_desc op{};
  double T = 0.0;
  int64_t K = 0;
  int stepper = 0, P = 1;
  int kry_m = 30, kry_phi = PXA_PHI_STEPPER, kry_sub = 1;
  int prop = PXA_PROP_KRYLOV;  // homogeneous propagator method (ADVDIFF_1D)
  int relpm_mmax = 120;
  double* relpm_D = nullptr;   // Newton divided differences and nodes of the chain's substeps
  double* relpm_z = nullptr;
  int relpm_nsub = 1;
  double* band_p = nullptr;    // taps of the subinterval propagator as a circulant band
  int band_pr = 0;             // its half-width
  double relpm_ts = 0.0;
  // pxa_cn_lanes_1d: FP32 lane states in global memory and the padded FP32 band
  float* st1d = nullptr;
  int lanes1d = 0;
  float* taps1d = nullptr;
  int r1d = 0;
  double kry_tol = 1e-11;
  int magnus_M = 25;
  const double* control = nullptr;
  double omega = 0.0;
  const double* target = nullptr;
  int wait_limit_units = 0;    // bounded device waits give up after this many x 1024 cycles (0: 2^31 cycles)
  int obj_kind = 0;            // pxa_objective_kind in use (0: the operator's default)
  int step_prec = PXA_F64;     // pxa_precision of the time stepping
  pxa_batch* inner = nullptr;  // ADVDIFF_1D with FP32 stepping: a batch of one problem
  // PXA_CSR: A^T (library-owned, formed on the host from A) and the lanes' vectors
  int64_t* rpT = nullptr;
  int32_t* colT = nullptr;
  double* valT = nullptr;
  double* csr_work = nullptr;  // [P][4][n] lane vectors when they do not fit in shared memory
  // BURGERS_2D: the FP32 trajectory [(K+1)][2][n][n], the adjoint ping-pong, J partials
  float* b2traj = nullptr;
  float* b2lam = nullptr;  // [2][2][n][n]
  double* b2Jpart = nullptr;
  // Alg. 2 (pxa_nl_paraexp): the iterate, the next iterate, the lanes, qbar, the change
  double *nl_Q = nullptr, *nl_Qn = nullptr, *nl_V = nullptr, *nl_qbar = nullptr, *nl_change = nullptr;
  int memory = PXA_STORE_FULL;
  int band_req = 1;  // pxa_set_adjoint: 1 = banded adjoint when it fits, 0 = stage re-stepping
  bool use_graph = false, timing = false;
  // CTAs per thread-block cluster for the Burgers RK4 kernels (0 = choose automatically)
  int cl_req_direct = 0, cl_req_lanes = 0, cl_req_chain = 0;
  int cl_direct = 1, cl_lanes = 1, cl_chain = 1;

  // derived
  double am = 0, a0 = 0, ap = 0;  // advection-diffusion stencil
  int band_r = 0;
  // ADVDIFF_1D lanes: the band of M^q (q CN steps per application) and q
  double* taps_q = nullptr;
  int band_rq = 0, lane_q = 1, lane_q_req = 0;
  std::vector<double> band_host;

  // workspace (device)
  bool ready = false;
  std::vector<void*> allocs;
  int64_t ws_bytes = 0;
  double* taps = nullptr;     // 2r+1
  double* E = nullptr;        // [P][n] lane outputs (direct / Burgers W)
  double* EA = nullptr;       // [P][n] adjoint lane outputs (Burgers G)
  double* src = nullptr;      // n
  double* srcA = nullptr;     // n
  double* hsum = nullptr;     // n
  double* hsumA = nullptr;    // n
  double* qT = nullptr;       // n
  double* tmp = nullptr;      // n
  double* V = nullptr;        // Krylov basis (global fallback)
  double* traj = nullptr;     // Burgers direct trajectory (K+1)*n or checkpoints
  double* scratch = nullptr;  // Burgers recompute rows
  // banded discrete adjoint of the Burgers RK4 map (used when it fits in memory)
  bool band = false;
  int cl_band_lanes = 1, cl_band_chain = 1;
  int cl_rk4_direct = 1, cl_rk4_lanes = 1;  // cluster sizes of the RK4 sweeps (direct, recompute)
  double* sc = nullptr;       // [K][3] forcing factors s(t) at the stage times (omega != 0)
  // hybrid overlap: the direct runs in chunks on the caller's stream while a library-owned
  // low-priority stream builds the band records and runs the adjoint lanes of finished chunks
  bool overlap = true;
  int q_direct = 0, q_sweep = 0;  // steps per halo exchange of the RK4 / banded sweeps (0 = auto)
  cudaStream_t side = nullptr;
  cudaStream_t side2 = nullptr;  // adjoint lanes of the overlapped chunks
  cudaStream_t side3 = nullptr;  // re-step and records of the second interval buffer set
  static constexpr int kMaxChunks = 8;
  double part_r = 0.0;        // ratio of successive chunk lengths (0: equal chunks)
  cudaEvent_t ev_fork[kMaxChunks] = {};
  cudaEvent_t ev_prep[kMaxChunks] = {};
  cudaEvent_t ev_join = nullptr, ev_join2 = nullptr;
  double* Jparts = nullptr;   // [kMaxChunks] objective of each direct chunk
  double* Jrow = nullptr;     // [(K+1)] ||u_s - g||^2 per stored row (full storage)
  int prio_hi = 0, prio_lo = 0;
  size_t reserve_smem = 0;    // dynamic shared memory that makes a direct CTA own its SM
  double* rec = nullptr;      // [(K+1)][n][BU1_BAND_RECORD] rows of M_s^T and sources
  double* jt = nullptr;       // [K][n][BU1_BAND_RECORD] transposed stage rows (gradient)
  double* LI = nullptr;       // [(K+1)][n] adjoint lane rows
  double* Hrows = nullptr;    // [(K+1)][n] homogeneous chain rows
  double* gpart = nullptr;    // [blocks][n] gradient partial sums
  // two-step chain: pair records and the step plans of the Paraexp and serial chains
  int chain_len = 4;          // longest step of the chain (1, 2 or 4)
  double* rp = nullptr;       // [K/2][n][BU1_PAIR_RECORD]
  double* rq = nullptr;       // [K/4][n][BU1_QUAD_RECORD]
  // step plans of the chain: [Paraexp partition, serial][steps up to 2, up to 4]
  struct ChainPlan {
    int4* dev = nullptr;
    int count = 0;
    std::vector<int4> host;  // host copy (segment boundaries)
  };
  ChainPlan plans[2][2];
  // the chain runs in up to kMaxSeg launches; after each one the side stream fills the
  // skipped rows and sums the gradient over the finished rows
  static constexpr int kMaxSeg = 8;
  int chain_segments = 4;
  cudaEvent_t ev_seg[kMaxSeg] = {};
  // multi-checkpoint scheme (Sec. 3.5): C intervals of K/C steps, each re-stepped from its
  // checkpoint and solved by the Paraexp adjoint over its own P subintervals. Two interval
  // buffer sets alternate, so that one interval's re-step, records and lanes run on the
  // side streams while the chain of the other runs.
  int intervals = 0;  // C (0: off)
  struct IntervalSet {
    double* traj = nullptr;  // [(K/C+1)][n] direct states of the interval
    double* rec = nullptr;   // [(K/C+1)][n][BU1_BAND_RECORD]
    double* jt = nullptr;    // [(K/C)][n][BU1_BAND_RECORD]
    double* rp = nullptr;    // [(K/(2C)+1)][n][BU1_PAIR_RECORD]
    double* rq = nullptr;    // [(K/(4C)+1)][n][BU1_QUAD_RECORD]
    double* LI = nullptr;    // [(K/C+1)][n] adjoint lane rows
    double* H = nullptr;     // [(K/C+1)][n] chain rows
  };
  IntervalSet iv[2];
  double* ckpt = nullptr;     // [(C+1)][n] direct states at t = jT/C
  double* lamtop = nullptr;   // [n] adjoint value at the bottom row of the interval last done
  double* ivW = nullptr;      // [C*P][n] values of the adjoint lanes at their bottom rows
  // chain plans of all intervals: [Paraexp partition, serial][steps up to 2, up to 4]
  int4* iplan_dev[2][2] = {};
  std::vector<int> iplan_off[2][2];  // C+1 offsets into iplan_dev
  int iv_spb = 1, iv_blocks = 1;  // gradient steps per block and blocks per interval
  // per buffer set: records built, lanes done, chain done, buffers free
  cudaEvent_t ev_iv[4][2] = {};
  double* Jdev = nullptr;     // 1
  double* errmax = nullptr;   // 1
  int* status = nullptr;      // 1
  double* ctl_buf = nullptr;  // n (pxa_gradient_host)
  double* grad_buf = nullptr; // n (pxa_gradient_host)
  bool v_in_smem = false;

  int direct_mode = -1;  // mode of the last pxa_solve_direct whose state is still valid

  // 2D advection-diffusion workspace (FP32 padded states, TMA maps)
  Ad2Params p2{};
  float* coef2 = nullptr;   // [3][Hp][Wp]
  float* stD = nullptr;     // direct ping-pong [2][1][Hp][Wp]
  float* stA = nullptr;     // adjoint lanes ping-pong [2][P][Hp][Wp]
  float* stC = nullptr;     // homogeneous chain ping-pong [2][1][Hp][Wp]
  float* traj2 = nullptr;   // [(K+1)][ny*nx] FP32 direct trajectory
  float* Jpart = nullptr;   // [K][tiles][AD2_J_WARPS] warp partials of the objective
  double* Jred = nullptr;   // [AD2_REDUCE_J_BLOCKS] block sums of their reduction
  float2* G2buf = nullptr;  // [P][ny*nx] lane gradients, double-float (hi, lo) FP32 pairs
  float* G2f = nullptr;     // [P][ny*nx] FP32 gradients of the wavefront lanes (K/P steps each)
  float2* GC = nullptr;     // [ny*nx] chain gradient, double-float
  CUtensorMap mapD, mapA, mapC, mapCoef;
  CUtensorMap mapH;         // over hC (the series chain's carried value)
  // adjoint lanes as a register wavefront (P > 1, grids the wavefront covers)
  bool roll2 = false;
  float* tcoef2 = nullptr;  // [4][Hp][Wp] coefficients of A^T
  float* sc2 = nullptr;     // [K][3] s(t) at the stage times of every step
  CUtensorMap mapA4, mapT4, mapS4, mapG4;
  // chain by the power series of the stepper's propagator (PXA_PROP_POLY)
  float* polyA = nullptr;    // [m+1] coefficients of R(z)^kk cut at degree m (m % 4 == 0)
  double* polyAd = nullptr;  // the same in FP64 (CSR chains)
  double* polyQ = nullptr;   // [3][kk][m+1] omega-free forcing families
  float* polyB = nullptr;    // [segments][m+1] forcing-gradient coefficients of each segment (FP32)
  float* hC = nullptr;       // [Hp][Wp] the chain's carried value
  int poly_m = 0, poly_sub = 1, poly_kk = 0;
  double poly_tail = 0.0;
  float* stL = nullptr;     // pxa_rk4_lanes_2d states [2][lanesL][Hp][Wp]
  int lanesL = 0;
  float* scL = nullptr;     // pxa_rk4_lanes_2d forcing factors [lanes * steps][3]
  int64_t scL_count = 0;
  CUtensorMap mapL4, mapC4; // row-block maps of the lane states and coefficients (wavefront)
  CUtensorMap mapL;

  // graph cache
  cudaGraphExec_t gexec = nullptr;
  int g_mode = -1;
  const double* g_grad = nullptr;
  const double* g_J = nullptr;
  bool g_prep_marked = false;  // the captured gradient records ev[6]

  // statistics
  pxa_stats stats{};
  cudaEvent_t ev[7] = {};
  bool ev_ready = false;
  bool prep_marked = false;  // ev[6] marks the end of the adjoint preparation
  // timing events of the overlapped side-stream work, per direct chunk: on the records
  // stream [0] start, [1] after the band pre-pass, [2] after the pair records, [3] after
  // the four-step records; on the lanes stream [4] start and [5] end of the adjoint lanes
  cudaEvent_t ev_side[kMaxChunks][6] = {};
  int side_marked = 0, g_side_marked = 0;  // chunks whose side events were recorded
  bool side_lanes_marked[kMaxChunks] = {};
  bool g_side_lanes_marked[kMaxChunks] = {};
};

namespace {

int fail(pxa_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(pxa_ctx* c, cudaError_t e, const char* where) {
  return fail(c, PXA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PXA_CUDA(c, expr, where)               \
  do {                                          \
    cudaError_t _e = (expr);                    \
    if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
  } while (0)

void release_workspace(pxa_ctx* c) {
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  c->ws_bytes = 0;
  c->ready = false;
  c->taps = c->E = c->EA = c->src = c->srcA = c->hsum = c->hsumA = c->qT = c->tmp = nullptr;
  c->relpm_D = c->relpm_z = c->band_p = nullptr;
  c->band_pr = 0;
  c->st1d = c->taps1d = nullptr;
  c->taps_q = nullptr;
  c->band_rq = 0;
  c->lanes1d = 0;
  c->V = c->traj = c->scratch = c->Jdev = c->errmax = c->ctl_buf = c->grad_buf = nullptr;
  c->status = nullptr;
  c->coef2 = c->stD = c->stA = c->stC = c->traj2 = c->stL = c->tcoef2 = c->sc2 = nullptr;
  c->roll2 = false;
  c->lanesL = 0;
  c->rpT = nullptr;
  c->colT = nullptr;
  c->valT = c->csr_work = nullptr;
  c->nl_Q = c->nl_Qn = c->nl_V = c->nl_qbar = c->nl_change = nullptr;
  c->b2traj = c->b2lam = nullptr;
  c->b2Jpart = nullptr;
  if (c->inner) {
    pxa_batch_destroy(c->inner);
    c->inner = nullptr;
  }
  c->scL = nullptr;
  c->scL_count = 0;
  c->Jpart = nullptr;
  c->Jred = nullptr;
  c->G2buf = c->GC = nullptr;
  c->G2f = nullptr;
  c->rec = c->jt = c->LI = c->Hrows = c->gpart = c->sc = c->Jparts = c->rp = c->rq = nullptr;
  c->Jrow = nullptr;
  for (auto& row : c->plans)
    for (auto& pl : row) {
      pl.dev = nullptr;  // freed with the workspace
      pl.count = 0;
      pl.host.clear();
    }
  for (auto& e : c->ev_seg)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  for (auto& set : c->iv) set = pxa_ctx::IntervalSet{};
  c->ckpt = c->lamtop = c->ivW = nullptr;
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 2; ++q) {
      c->iplan_dev[s][q] = nullptr;
      c->iplan_off[s][q].clear();
    }
  for (auto& row : c->ev_iv)
    for (auto& e : row)
      if (e) {
        cudaEventDestroy(e);
        e = nullptr;
      }
  if (c->side) {
    cudaStreamDestroy(c->side);
    c->side = nullptr;
  }
  if (c->side3) {
    cudaStreamDestroy(c->side3);
    c->side3 = nullptr;
  }
  if (c->side2) {
    cudaStreamDestroy(c->side2);
    c->side2 = nullptr;
  }
  for (auto* arr : {c->ev_fork, c->ev_prep})
    for (int i = 0; i < pxa_ctx::kMaxChunks; ++i)
      if (arr[i]) {
        cudaEventDestroy(arr[i]);
        arr[i] = nullptr;
      }
  for (cudaEvent_t* e : {&c->ev_join, &c->ev_join2})
    if (*e) {
      cudaEventDestroy(*e);
      *e = nullptr;
    }
  c->band = false;
}

void invalidate(pxa_ctx* c) {
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->g_mode = -1;
  c->direct_mode = -1;
}

template <typename T>
int alloc(pxa_ctx* c, T** out, size_t count) {
  void* p = nullptr;
  size_t bytes = sizeof(T) * (count ? count : 1);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, PXA_ERR_OOM, std::string("workspace allocation of ") + std::to_string(bytes) +
                                    " bytes failed: " + cudaGetErrorString(e));
  }
  c->allocs.push_back(p);
  c->ws_bytes += (int64_t)bytes;
  *out = static_cast<T*>(p);
  return PXA_OK;
}

int threads_for(int n) {
  int t = ((n + 31) / 32) * 32;
  return t > 1024 ? 1024 : (t < 64 ? 64 : t);
}

int prepare(pxa_ctx* c) {
  if (c->ready) return PXA_OK;
  if (!c->have_op || !c->have_time) return fail(c, PXA_ERR_STATE, "set_operator and set_time first");
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  release_workspace(c);
  if (c->prop == PXA_PROP_POLY && c->op.kind != PXA_ADVDIFF_2D && c->op.kind != PXA_CSR)
    return fail(c, PXA_ERR_INVALID, "PXA_PROP_POLY is implemented for ADVDIFF_2D and CSR");
  const int n = c->op.n, P = c->P;
  int rc;
  if ((rc = alloc(c, &c->Jdev, 1))) return rc;
  if ((rc = alloc(c, &c->errmax, 1))) return rc;
  // [0] the status word, [1] the wait limit of the bounded device waits (units of 1024
  // cycles, 0: the default)
  if ((rc = alloc(c, &c->status, 2))) return rc;
  if ((rc = alloc(c, &c->ctl_buf, n))) return rc;
  if ((rc = alloc(c, &c->grad_buf, n))) return rc;
  const bool long1d = c->op.kind == PXA_ADVDIFF_1D && n > 4096;  // lanes in global memory only
  if (c->op.kind != PXA_ADVDIFF_2D && c->op.kind != PXA_BURGERS_2D && !long1d) {
    if ((rc = alloc(c, &c->E, (size_t)P * n))) return rc;
    if ((rc = alloc(c, &c->EA, (size_t)P * n))) return rc;
    if ((rc = alloc(c, &c->src, n))) return rc;
    if ((rc = alloc(c, &c->srcA, n))) return rc;
    if ((rc = alloc(c, &c->hsum, n))) return rc;
    if ((rc = alloc(c, &c->hsumA, n))) return rc;
    if ((rc = alloc(c, &c->qT, n))) return rc;
    if ((rc = alloc(c, &c->tmp, n))) return rc;
    // Krylov basis: in shared memory when it fits beside the dense scratch
    int extra = (c->op.kind == PXA_ADVDIFF_1D || c->op.kind == PXA_CSR) ? n : 5 * (n + 2) + n;
    size_t with_v = krylov_smem_bytes(n, c->kry_m, extra, true);
    c->v_in_smem = with_v <= 200 * 1024;
    if ((rc = alloc(c, &c->V, (size_t)(c->kry_m + 1) * n))) return rc;
  }
  if (c->op.kind == PXA_ADVDIFF_2D) {
    Ad2Params& a = c->p2;
    a.nx = c->op.nx;
    a.ny = c->op.ny;
    a.Wp = a.nx + 2 * G2;
    a.Hp = a.ny + 2 * G2;
    a.tiles_x = (a.nx + TX2 - 1) / TX2;
    a.tiles_y = (a.ny + TY2 - 1) / TY2;
    const double h = c->op.L / a.nx;
    a.inv2h = (float)(1.0 / (2.0 * h));
    a.invh2 = (float)(1.0 / (h * h));
    a.nu = (float)c->op.nu;
    a.dtd = c->T / (double)c->K;
    a.dt = (float)a.dtd;
    a.omega = 0.0;
    const size_t plane = (size_t)a.Hp * a.Wp, N = (size_t)a.nx * a.ny;
    if ((rc = alloc(c, &c->coef2, 3 * plane))) return rc;
    if ((rc = alloc(c, &c->stD, 2 * plane))) return rc;
    if ((rc = alloc(c, &c->stA, 2 * (size_t)P * plane))) return rc;
    if ((rc = alloc(c, &c->stC, 2 * plane))) return rc;
    if ((rc = alloc(c, &c->traj2, (size_t)(c->K + 1) * N))) return rc;
    if ((rc = alloc(c, &c->Jpart, (size_t)c->K * a.tiles_x * a.tiles_y * AD2_J_WARPS))) return rc;
    if ((rc = alloc(c, &c->Jred, (size_t)AD2_REDUCE_J_BLOCKS))) return rc;
    c->roll2 = P > 1 && ad2_roll_ok(a);
    // the halo-tile lanes' gradients: every lane's when they step the Paraexp lanes, else
    // only the serial adjoint's (the wavefront lanes have FP32 planes of their own)
    if ((rc = alloc(c, &c->G2buf, (size_t)(c->roll2 ? 1 : P) * N))) return rc;
    if ((rc = alloc(c, &c->GC, N))) return rc;
    PXA_CUDA(c, cudaMemset(c->coef2, 0, sizeof(float) * 3 * plane), "memset coef");
    PXA_CUDA(c, cudaMemset(c->stD, 0, sizeof(float) * 2 * plane), "memset");
    PXA_CUDA(c, cudaMemset(c->stA, 0, sizeof(float) * 2 * (size_t)P * plane), "memset");
    PXA_CUDA(c, cudaMemset(c->stC, 0, sizeof(float) * 2 * plane), "memset");
    if (!ad2_make_map(&c->mapD, c->stD, a, 2, 1) || !ad2_make_map(&c->mapA, c->stA, a, 2 * P, 1) ||
        !ad2_make_map(&c->mapC, c->stC, a, 2, 1) || !ad2_make_map(&c->mapCoef, c->coef2, a, 3, 3))
      return fail(c, PXA_ERR_CUDA, "cuTensorMapEncodeTiled failed for the 2D state arrays");
    if ((rc = alloc(c, &c->sc2, (size_t)3 * c->K))) return rc;
    if (c->roll2) {
      if ((rc = alloc(c, &c->tcoef2, 4 * plane))) return rc;
      if ((rc = alloc(c, &c->G2f, (size_t)P * N))) return rc;
      if (!ad2_make_map_box(&c->mapA4, c->stA, a, 2 * P, 64, AD2_ROLL_BR, 1) ||
          !ad2_make_map_box(&c->mapT4, c->tcoef2, a, 4, 64, AD2_ROLL_BR, 4) ||
          !ad2_make_map_plain(&c->mapS4, c->traj2, 4, a.nx, a.ny, (int)c->K + 1, 64, AD2_ROLL_BR) ||
          !ad2_make_map_plain(&c->mapG4, c->G2f, 4, a.nx, a.ny, P, 64, AD2_ROLL_BR))
        return fail(c, PXA_ERR_CUDA, "cuTensorMapEncodeTiled failed for the 2D adjoint lanes");
    }
    c->poly_m = 0;
    if (c->prop == PXA_PROP_POLY && P > 1) {
      // max-norm of dt A^T (largest absolute row sum of the transposed stencil), from the
      // velocity copied to the host once (set-up, not the solve path)
      std::vector<double> hu(N), hv(N);
      PXA_CUDA(c, cudaMemcpy(hu.data(), c->op.u_dev, sizeof(double) * N, cudaMemcpyDeviceToHost), "copy u");
      PXA_CUDA(c, cudaMemcpy(hv.data(), c->op.v_dev, sizeof(double) * N, cudaMemcpyDeviceToHost), "copy v");
      const double dd = c->op.nu / (h * h), ih = 1.0 / (2.0 * h);
      double rowmax = 0.0;
      for (int y = 0; y < a.ny; ++y)
        for (int x = 0; x < a.nx; ++x) {
          const size_t w = (size_t)y * a.nx + (x + a.nx - 1) % a.nx, e = (size_t)y * a.nx + (x + 1) % a.nx;
          const size_t sth = (size_t)((y + a.ny - 1) % a.ny) * a.nx + x, nth = (size_t)((y + 1) % a.ny) * a.nx + x;
          const double r = std::fabs(-hu[w] * ih + dd) + std::fabs(hu[e] * ih + dd) + std::fabs(-hv[sth] * ih + dd) +
                           std::fabs(hv[nth] * ih + dd) + 4.0 * dd;
          rowmax = std::max(rowmax, r);
        }
      const int64_t k = c->K / P;
      PolyPlan pl = poly_plan(a.dtd * rowmax, k, a.dtd, std::max(c->kry_tol, 1e-7));
      const int sub = pl.sub, kk = pl.kk, m = pl.m;
      const double tail = pl.tail;
      std::vector<long double>& afull = pl.a_full;
      std::vector<double> Q;
      if (m > c->relpm_mmax || m > 252)
        return fail(c, PXA_ERR_NOT_CONVERGED, "PXA_PROP_POLY: the series needs degree " + std::to_string(m) +
                                                  " for the tolerance, above the maximum degree");
      rk4_series_host(kk, m, a.dtd, afull, Q);
      std::vector<float> ah((size_t)m + 1);
      for (int i = 0; i <= m; ++i) ah[(size_t)i] = (float)afull[(size_t)i];
      const int segments = (P - 1) * sub;
      if ((rc = alloc(c, &c->polyA, (size_t)m + 1))) return rc;
      if ((rc = alloc(c, &c->polyQ, Q.size()))) return rc;
      if ((rc = alloc(c, &c->polyB, (size_t)segments * (m + 1)))) return rc;
      if ((rc = alloc(c, &c->hC, plane))) return rc;
      if (!ad2_make_map(&c->mapH, c->hC, a, 1, 1))
        return fail(c, PXA_ERR_CUDA, "cuTensorMapEncodeTiled failed for the series chain");
      PXA_CUDA(c, cudaMemcpy(c->polyA, ah.data(), sizeof(float) * ah.size(), cudaMemcpyHostToDevice), "copy");
      PXA_CUDA(c, cudaMemcpy(c->polyQ, Q.data(), sizeof(double) * Q.size(), cudaMemcpyHostToDevice), "copy");
      c->poly_m = m;
      c->poly_sub = sub;
      c->poly_kk = kk;
      c->poly_tail = tail;
    }
    c->stats.prop_degree = c->poly_m;
    c->stats.prop_substeps = c->poly_m ? c->poly_sub : 0;
    c->stats.prop_tail = c->poly_m ? c->poly_tail : 0.0;
  } else if (c->op.kind == PXA_ADVDIFF_1D) {
    double dt = c->T / (double)c->K;
    cn_band_taps(n, c->am, c->a0, c->ap, dt, c->band_host, c->band_r);
    if ((rc = alloc(c, &c->taps, c->band_host.size()))) return rc;
    PXA_CUDA(c, cudaMemcpy(c->taps, c->band_host.data(), sizeof(double) * c->band_host.size(),
                           cudaMemcpyHostToDevice), "copy taps");
    // The lanes take K/P CN steps as K/(P q) applications of the band of M^q (q = 4, 2
    // or 1, dividing K/P): M^q is circulant with taps from the eigenvalues R_k^q, and
    // since the implicit map's taps decay geometrically its band is barely wider than
    // M's, so q steps cost about one (FP64 taps kept to 2^-52 of the largest).
    c->lane_q = 0;
    for (int q : {4, 2, 1})
      if ((c->lane_q_req == 0 || q == c->lane_q_req) && (c->K / P) % q == 0 && (q == 1 || n <= 4096)) {
        c->lane_q = q;
        break;
      }
    if (c->lane_q == 0) return fail(c, PXA_ERR_INVALID, "the requested CN steps per lane band do not divide K/P");
    if (c->lane_q == 1) {
      c->taps_q = c->taps;
      c->band_rq = c->band_r;
    } else {
      std::vector<double> tq;
      cn_power_taps(n, c->am, c->a0, c->ap, dt, c->lane_q, 52, tq, c->band_rq);
      if ((rc = alloc(c, &c->taps_q, tq.size()))) return rc;
      PXA_CUDA(c, cudaMemcpy(c->taps_q, tq.data(), sizeof(double) * tq.size(), cudaMemcpyHostToDevice),
               "copy taps");
    }
    c->stats.lane_steps = c->lane_q;
    c->stats.lane_band_taps = 2 * c->band_rq + 1;
    if (c->prop == PXA_PROP_BAND) {
      // the subinterval propagator exp(tau A) or M^(K/P) as one circulant band
      std::vector<double> bt;
      cn_power_taps(n, c->am, c->a0, c->ap, dt, c->K / P, 50, bt, c->band_pr, c->kry_phi == PXA_PHI_EXP);
      c->stats.prop_band_taps = 2 * c->band_pr + 1;
      if ((rc = alloc(c, &c->band_p, bt.size()))) return rc;
      PXA_CUDA(c, cudaMemcpy(c->band_p, bt.data(), sizeof(double) * bt.size(), cudaMemcpyHostToDevice), "copy");
    }
    if (c->prop == PXA_PROP_RELPM) {
      // the chain's exponential over one subinterval tau = T / P
      std::vector<double> z, D;
      relpm_setup_host(c->T / P, c->am, c->a0, c->ap, c->relpm_mmax, c->relpm_nsub, c->relpm_ts, z, D,
                       c->kry_phi == PXA_PHI_STEPPER ? c->K / P : 0);
      if ((rc = alloc(c, &c->relpm_D, D.size()))) return rc;
      if ((rc = alloc(c, &c->relpm_z, z.size()))) return rc;
      PXA_CUDA(c, cudaMemcpy(c->relpm_D, D.data(), sizeof(double) * D.size(), cudaMemcpyHostToDevice), "copy");
      PXA_CUDA(c, cudaMemcpy(c->relpm_z, z.data(), sizeof(double) * z.size(), cudaMemcpyHostToDevice), "copy");
    }
  } else if (c->op.kind == PXA_BURGERS_2D) {
    const size_t plane2 = 2 * (size_t)c->op.nx * c->op.nx;
    const int tiles = (c->op.nx / BU2_TILE) * (c->op.nx / BU2_TILE);
    if ((rc = alloc(c, &c->b2traj, (size_t)(c->K + 1) * plane2))) return rc;
    if ((rc = alloc(c, &c->b2lam, 2 * plane2))) return rc;
    if ((rc = alloc(c, &c->b2Jpart, (size_t)tiles))) return rc;
  } else if (c->op.kind == PXA_CSR) {
    // A^T for the adjoint lanes and chain: A is copied to the host once and transposed
    // entry by entry (set-up, not the solve path)
    const int64_t* rp = c->op.row_ptr_dev;
    std::vector<int64_t> hrp((size_t)n + 1);
    PXA_CUDA(c, cudaMemcpy(hrp.data(), rp, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost), "copy A");
    const int64_t nnz = hrp[n];
    if (hrp[0] != 0 || nnz < 0 || nnz > (int64_t)INT32_MAX)
      return fail(c, PXA_ERR_INVALID, "CSR row pointers (row_ptr[0] == 0, nnz < 2^31)");
    for (int i = 0; i < n; ++i)
      if (hrp[i + 1] < hrp[i]) return fail(c, PXA_ERR_INVALID, "CSR row pointers must not decrease");
    std::vector<int32_t> hcol((size_t)(nnz > 0 ? nnz : 1));
    std::vector<double> hval((size_t)(nnz > 0 ? nnz : 1));
    if (nnz > 0) {
      PXA_CUDA(c, cudaMemcpy(hcol.data(), c->op.col_dev, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost), "copy A");
      PXA_CUDA(c, cudaMemcpy(hval.data(), c->op.val_dev, sizeof(double) * nnz, cudaMemcpyDeviceToHost), "copy A");
    }
    std::vector<int64_t> trp((size_t)n + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) {
      if (hcol[e] < 0 || hcol[e] >= n) return fail(c, PXA_ERR_INVALID, "CSR column index out of range");
      ++trp[(size_t)hcol[e] + 1];
    }
    for (int j = 0; j < n; ++j) trp[j + 1] += trp[j];
    std::vector<int64_t> fill(trp.begin(), trp.end() - 1);
    std::vector<int32_t> tcol((size_t)(nnz > 0 ? nnz : 1));
    std::vector<double> tval((size_t)(nnz > 0 ? nnz : 1));
    for (int i = 0; i < n; ++i)
      for (int64_t e = hrp[i]; e < hrp[i + 1]; ++e) {
        const int64_t d = fill[hcol[e]]++;
        tcol[d] = i;
        tval[d] = hval[e];
      }
    if ((rc = alloc(c, &c->rpT, (size_t)n + 1))) return rc;
    if ((rc = alloc(c, &c->colT, tcol.size()))) return rc;
    if ((rc = alloc(c, &c->valT, tval.size()))) return rc;
    PXA_CUDA(c, cudaMemcpy(c->rpT, trp.data(), sizeof(int64_t) * trp.size(), cudaMemcpyHostToDevice), "copy A^T");
    PXA_CUDA(c, cudaMemcpy(c->colT, tcol.data(), sizeof(int32_t) * tcol.size(), cudaMemcpyHostToDevice), "copy A^T");
    PXA_CUDA(c, cudaMemcpy(c->valT, tval.data(), sizeof(double) * tval.size(), cudaMemcpyHostToDevice), "copy A^T");
    if (!csr_lanes_fit_smem(n) && (rc = alloc(c, &c->csr_work, (size_t)4 * n * P))) return rc;
    c->poly_m = 0;
    if (c->prop == PXA_PROP_POLY && P > 1) {
      // the chains apply A (direct) and A^T (adjoint): rho = dt max(||A||_inf, ||A||_1)
      std::vector<double> rowsum((size_t)n, 0.0), colsum((size_t)n, 0.0);
      for (int i = 0; i < n; ++i)
        for (int64_t e = hrp[i]; e < hrp[i + 1]; ++e) {
          rowsum[(size_t)i] += std::fabs(hval[e]);
          colsum[(size_t)hcol[e]] += std::fabs(hval[e]);
        }
      double nrm = 0.0;
      for (int i = 0; i < n; ++i) nrm = std::max(nrm, std::max(rowsum[(size_t)i], colsum[(size_t)i]));
      const double dt = c->T / (double)c->K;
      PolyPlan pl = poly_plan(dt * nrm, c->K / P, dt, c->kry_tol);
      if (pl.m > c->relpm_mmax)
        return fail(c, PXA_ERR_NOT_CONVERGED, "PXA_PROP_POLY: the series needs degree " + std::to_string(pl.m) +
                                                  " for the tolerance, above the maximum degree");
      std::vector<double> ad((size_t)pl.m + 1);
      for (int i = 0; i <= pl.m; ++i) ad[(size_t)i] = (double)pl.a_full[(size_t)i];
      if ((rc = alloc(c, &c->polyAd, ad.size()))) return rc;
      PXA_CUDA(c, cudaMemcpy(c->polyAd, ad.data(), sizeof(double) * ad.size(), cudaMemcpyHostToDevice), "copy");
      c->poly_m = pl.m;
      c->poly_sub = pl.sub;
      c->poly_kk = pl.kk;
      c->poly_tail = pl.tail;
    }
    c->stats.prop_degree = c->poly_m;
    c->stats.prop_substeps = c->poly_m ? c->poly_sub : 0;
    c->stats.prop_tail = c->poly_m ? c->poly_tail : 0.0;
  } else {
    int64_t k = c->K / P;
    // the side streams, events and priorities of the banded adjoint
    auto band_streams = [&]() -> int {
      c->band = true;
      int least = 0, greatest = 0;
      PXA_CUDA(c, cudaDeviceGetStreamPriorityRange(&least, &greatest), "priority range");
      c->prio_lo = least;
      c->prio_hi = greatest;
      PXA_CUDA(c, cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, least), "side stream");
      PXA_CUDA(c, cudaStreamCreateWithPriority(&c->side2, cudaStreamNonBlocking, least), "side stream");
      for (auto& e : c->ev_fork) PXA_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
      for (auto& e : c->ev_prep) PXA_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
      for (auto& e : c->ev_seg) PXA_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
      PXA_CUDA(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "event");
      PXA_CUDA(c, cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming), "event");
      int optin = 0;
      PXA_CUDA(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device),
               "smem opt-in");
      // leave room for the kernel's static shared memory within the per-CTA limit
      c->reserve_smem = optin > 4096 ? (size_t)(optin - 2048) : 0;
      return PXA_OK;
    };
    if (c->intervals >= 2) {
      // multi-checkpoint scheme: C + 1 checkpoints and two interval buffer sets
      const int C = c->intervals;
      if (c->band_req == 0 || c->chain_len < 2)
        return fail(c, PXA_ERR_INVALID, "the multi-checkpoint scheme needs the banded adjoint with two- or "
                                        "four-step chain records (PXA_ADJ_BANDED or PXA_ADJ_BANDED_PAIR)");
      if (c->K % ((int64_t)C * P) != 0)
        return fail(c, PXA_ERR_INVALID, "the multi-checkpoint scheme needs K to be a multiple of C * P");
      const int64_t Kc = c->K / C;
      const size_t rows = (size_t)(Kc + 1) * n;
      c->iv_spb = bu1_band_steps_per_block(Kc, n);
      c->iv_blocks = (int)((Kc + c->iv_spb - 1) / c->iv_spb);
      if ((rc = alloc(c, &c->sc, (size_t)3 * c->K))) return rc;
      if ((rc = alloc(c, &c->ckpt, (size_t)(C + 1) * n))) return rc;
      if ((rc = alloc(c, &c->lamtop, n))) return rc;
      if ((rc = alloc(c, &c->Jparts, 2))) return rc;
      if ((rc = alloc(c, &c->ivW, (size_t)C * P * n))) return rc;
      if ((rc = alloc(c, &c->gpart, (size_t)C * c->iv_blocks * n))) return rc;
      for (auto& set : c->iv) {
        if ((rc = alloc(c, &set.traj, rows))) return rc;
        if ((rc = alloc(c, &set.rec, rows * BU1_BAND_RECORD))) return rc;
        if ((rc = alloc(c, &set.jt, (size_t)Kc * n * BU1_BAND_RECORD))) return rc;
        if ((rc = alloc(c, &set.rp, (size_t)(Kc / 2 + 1) * n * BU1_PAIR_RECORD))) return rc;
        if (c->chain_len >= 4 && (rc = alloc(c, &set.rq, (size_t)(Kc / 4 + 1) * n * BU1_QUAD_RECORD)))
          return rc;
        if ((rc = alloc(c, &set.LI, rows))) return rc;
        if ((rc = alloc(c, &set.H, rows))) return rc;
      }
      // chain plans of every interval, for the Paraexp partition (P subintervals of each
      // interval) and for serial stepping: rows (i+1)K/C down to iK/C, the source on the
      // interval's top subinterval, the lanes' values at the subinterval boundaries
      // including the interval's bottom row
      std::vector<int4> plan((size_t)c->K);
      for (int ser = 0; ser < 2; ++ser)
        for (int q4 = 0; q4 < (c->chain_len >= 4 ? 2 : 1); ++q4) {
          const int Pe = ser ? 1 : P;
          const int64_t kc = Kc / Pe;
          std::vector<int>& off = c->iplan_off[ser][q4];
          off.assign(1, 0);
          for (int ci = 0; ci < C; ++ci) {
            const int64_t a = ci * Kc;
            const int cnt = bu1_chain_plan_range(a + Kc, a, kc, a + (Pe - 1) * kc, (int64_t)ci * Pe,
                                                 (int64_t)ci * Pe + Pe - 2, q4 ? 4 : 2, plan.data() + off.back());
            off.push_back(off.back() + cnt);
          }
          if ((rc = alloc(c, &c->iplan_dev[ser][q4], (size_t)off.back()))) return rc;
          PXA_CUDA(c, cudaMemcpy(c->iplan_dev[ser][q4], plan.data(), sizeof(int4) * off.back(),
                                 cudaMemcpyHostToDevice), "copy plan");
        }
      if ((rc = band_streams())) return rc;
      PXA_CUDA(c, cudaStreamCreateWithPriority(&c->side3, cudaStreamNonBlocking, c->prio_lo), "side stream");
      for (auto& row : c->ev_iv)
        for (auto& e : row) PXA_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    } else {
      if (c->memory == PXA_STORE_FULL) {
        if ((rc = alloc(c, &c->traj, (size_t)(c->K + 1) * n))) return rc;
        if ((rc = alloc(c, &c->Jrow, (size_t)(c->K + 1)))) return rc;
      } else {
        if ((rc = alloc(c, &c->traj, (size_t)(P + 1) * n))) return rc;
        if ((rc = alloc(c, &c->scratch, (size_t)P * (size_t)(k + 1) * n))) return rc;
      }
      // The banded adjoint keeps two records per step and point plus two lambda
      // trajectories; it is used when that takes at most half of the free memory,
      // otherwise the adjoint re-steps the stages (kernels_bu1_cluster.cu).
      if ((rc = alloc(c, &c->sc, (size_t)3 * c->K))) return rc;
      const size_t rows1 = (size_t)(c->K + 1) * n;
      const size_t pair_doubles = c->chain_len >= 2 ? (size_t)(c->K / 2) * n * BU1_PAIR_RECORD : 0;
      const size_t quad_doubles = c->chain_len >= 4 ? (size_t)(c->K / 4) * n * BU1_QUAD_RECORD : 0;
      const size_t band_doubles = rows1 * BU1_BAND_RECORD + (size_t)c->K * n * BU1_BAND_RECORD +
                                  2 * rows1 + (size_t)bu1_band_grad_blocks(c->K, n) * n + pair_doubles +
                                  quad_doubles;
      size_t free_b = 0, total_b = 0;
      PXA_CUDA(c, cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
      if (c->band_req != 0 && band_doubles * sizeof(double) <= free_b / 2) {
        if ((rc = alloc(c, &c->rec, rows1 * BU1_BAND_RECORD))) return rc;
        if ((rc = alloc(c, &c->jt, (size_t)c->K * n * BU1_BAND_RECORD))) return rc;
        if ((rc = alloc(c, &c->LI, rows1))) return rc;
        if ((rc = alloc(c, &c->Hrows, rows1))) return rc;
        if ((rc = alloc(c, &c->gpart, (size_t)bu1_band_grad_blocks(c->K, n) * n))) return rc;
        if ((rc = alloc(c, &c->Jparts, pxa_ctx::kMaxChunks))) return rc;
        if (c->chain_len >= 2) {
          if ((rc = alloc(c, &c->rp, pair_doubles))) return rc;
          if (c->chain_len >= 4 && (rc = alloc(c, &c->rq, quad_doubles))) return rc;
          // step plans of the chain for the Paraexp partition and for serial stepping, with
          // steps of up to two and of up to four rows
          std::vector<int4> plan((size_t)c->K);
          for (int ser = 0; ser < 2; ++ser)
            for (int q4 = 0; q4 < (c->rq ? 2 : 1); ++q4) {
              pxa_ctx::ChainPlan& pl = c->plans[ser][q4];
              pl.count = bu1_chain_plan(c->K, ser ? c->K : k, ser ? 1 : P, q4 ? 4 : 2, plan.data());
              if ((rc = alloc(c, &pl.dev, (size_t)pl.count))) return rc;
              PXA_CUDA(c, cudaMemcpy(pl.dev, plan.data(), sizeof(int4) * pl.count, cudaMemcpyHostToDevice),
                       "copy plan");
              pl.host.assign(plan.begin(), plan.begin() + pl.count);
            }
        }
        if ((rc = band_streams())) return rc;
      }
    }
  }
  if (c->op.kind == PXA_BURGERS_1D) {
    // A serial lane gets the widest cluster that keeps >= 32 points per CTA; the P
    // concurrent adjoint lanes share the SMs (P * C <= number of SMs).
    int sms = 0;
    PXA_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device), "SM count");
    auto widest = [&](int limit) {
      int C = 16;
      while (C > 1 && (C > limit || n / C < 32 || !bu1c_valid_cluster(n, C))) C /= 2;
      return C;
    };
    c->cl_direct = c->cl_req_direct > 0 ? c->cl_req_direct : widest(16);
    c->cl_chain = c->cl_req_chain > 0 ? c->cl_req_chain : widest(16);
    c->cl_lanes = c->cl_req_lanes > 0 ? c->cl_req_lanes : widest(P > 0 ? sms / P : 1);
    for (int C : {c->cl_direct, c->cl_chain, c->cl_lanes})
      if (!bu1c_valid_cluster(n, C)) return fail(c, PXA_ERR_INVALID, "cluster size does not fit the grid");
    // the banded sweep needs >= 4 points per CTA (its halo) and <= 1024: the largest
    // size not above the requested one that satisfies both, else the smallest that does
    auto band_size = [&](int want) {
      for (int C = want; C >= 1; --C)
        if (bu1_band_valid_cluster(n, C)) return C;
      for (int C = want + 1; C <= 16; ++C)
        if (bu1_band_valid_cluster(n, C)) return C;
      return 0;
    };
    c->cl_band_lanes = band_size(c->cl_lanes);
    c->cl_band_chain = band_size(c->cl_chain);
    auto rk4_size = [&](int want) {
      for (int C = want; C >= 1; --C)
        if (bu1_rk4_valid_cluster(n, C)) return C;
      for (int C = want + 1; C <= 16; ++C)
        if (bu1_rk4_valid_cluster(n, C)) return C;
      return 0;
    };
    c->cl_rk4_direct = rk4_size(c->cl_direct);
    c->cl_rk4_lanes = rk4_size(c->cl_lanes);
    if (c->cl_rk4_direct == 0 || c->cl_rk4_lanes == 0)
      return fail(c, PXA_ERR_INVALID, "no cluster size fits the RK4 sweep");
    if (c->band && (c->cl_band_lanes == 0 || c->cl_band_chain == 0))
      return fail(c, PXA_ERR_INVALID, "no cluster size fits the banded adjoint sweep");
  }
  PXA_CUDA(c, cudaMemset(c->status, 0, sizeof(int)), "memset status");
  PXA_CUDA(c, cudaMemcpy(c->status + 1, &c->wait_limit_units, sizeof(int), cudaMemcpyHostToDevice), "wait limit");
  c->stats.workspace_bytes = c->ws_bytes;
  c->stats.band_taps = c->op.kind == PXA_ADVDIFF_1D ? 2 * c->band_r + 1 : 0;
  c->stats.cluster_direct = c->op.kind == PXA_BURGERS_1D ? c->cl_rk4_direct : c->cl_direct;
  c->stats.cluster_lanes = c->band ? c->cl_band_lanes : c->cl_lanes;
  c->stats.cluster_chain = c->band ? c->cl_band_chain : c->cl_chain;
  c->stats.adjoint_band = c->band ? 1 : 0;
  c->stats.group_direct = c->q_direct;
  c->stats.group_sweep = c->q_sweep;
  c->ready = true;
  return PXA_OK;
}

// Timing event `ev` on stream `s`; while a graph is being captured it becomes an
// external event-record node, which records the event like a stream would at replay.
void ev_record_on(pxa_ctx* c, cudaEvent_t ev, cudaStream_t s) {
  if (!(c->timing && c->ev_ready) || !ev) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  const cudaError_t e = cs == cudaStreamCaptureStatusActive
                            ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                            : cudaEventRecord(ev, s);
  if (e != cudaSuccess) cudaGetLastError();  // phase times then read as unavailable
}

// Phase event i on the context's stream.
void ev_record(pxa_ctx* c, int i) { ev_record_on(c, c->ev[i], c->stream); }

// The timing events (phases on the context's stream, side-stream work per chunk), created
// once per context.
int ensure_timing_events(pxa_ctx* c) {
  if (c->ev_ready) return PXA_OK;
  for (auto& e : c->ev) PXA_CUDA(c, cudaEventCreate(&e), "event create");
  for (auto& row : c->ev_side)
    for (auto& e : row) PXA_CUDA(c, cudaEventCreate(&e), "event create");
  c->ev_ready = true;
  return PXA_OK;
}

// ---- 1D advection-diffusion (IC control, terminal objective) ----------------
// parts: bit 0 = direct solve (J, q(T), adjoint source), bit 1 = adjoint solve (gradient)
int enqueue_ad1(pxa_ctx* c, int mode, int parts, double* Jdev, double* grad) {
  cudaStream_t st = c->stream;
  const bool do_d = parts & 1, do_a = parts & 2;
  // the lanes apply the band of M^q (taps_q, half-width r) K/q or K/(P q) times
  const int n = c->op.n, P = c->P, r = c->band_rq, th = threads_for(n);
  const double* taps = c->taps_q;
  const int64_t lq = c->lane_q;
  if (n > 4096)
    return fail(c, PXA_ERR_INVALID, "ADVDIFF_1D with n > 4096: the lanes and chains keep a lane in shared memory "
                                    "(pxa_cn_lanes_1d steps longer grids)");
  const int64_t K = c->K;
  const double dt = c->T / (double)K;
  const double* q0 = c->control;
  if (mode == PXA_SERIAL) {
    if (do_d) {
      ev_record(c, 0);
      PXA_CUDA(c, launch_cn_lanes(st, 1, th, n, r, taps, 0, K / lq, q0, nullptr, c->E), "cn serial");
      ev_record(c, 1);
      ev_record(c, 2);
      PXA_CUDA(c, launch_ad1_superpose_direct(st, th, n, r, taps, nullptr, c->E, nullptr, c->target, c->qT,
                                              nullptr, Jdev, c->status), "superpose");
    }
    if (do_a) {
      PXA_CUDA(c, launch_cn_lanes(st, 1, th, n, r, taps, 1, K / lq, c->qT, nullptr, c->EA), "cn serial T");
      ev_record(c, 3);
      ev_record(c, 4);
      PXA_CUDA(c, launch_ad1_superpose_adjoint(st, n, nullptr, c->EA, nullptr, grad, c->status), "grad");
      ev_record(c, 5);
    }
    return PXA_OK;
  }
  const int64_t k = K / P;
  const int nsub = c->kry_sub;
  const int64_t steps_sub = k / nsub;
  const double hscale = c->kry_phi == PXA_PHI_EXP ? dt * (double)steps_sub : dt;
  const int kth = 256;
  const bool relpm = c->prop == PXA_PROP_RELPM;
  const int relpm_direct = c->kry_phi == PXA_PHI_STEPPER ? 1 : 0;
  if (do_d) {
  PXA_CUDA(c, cudaMemsetAsync(c->errmax, 0, sizeof(double), st), "reset errmax");
  ev_record(c, 0);
  // Eq. linzero: the shifted problem has zero IC and source A q0; in CN form the
  // lane recursion is q~' = M q~ + (M - I) q0, and over q steps
  // q~'' = M^q q~ + (M^q - I) q0.
  PXA_CUDA(c, launch_band_minus_identity(st, n, r, taps, 0, q0, c->src), "src");
  PXA_CUDA(c, launch_cn_lanes(st, P, th, n, r, taps, 0, k / lq, nullptr, c->src, c->E), "lanes");
  ev_record(c, 1);
  if (P > 1 && c->prop == PXA_PROP_BAND) {
    PXA_CUDA(c, launch_ad1_band_chain(st, n, c->band_pr, c->band_p, 0, c->E, 0, 1, P - 1, c->hsum), "chain");
  } else if (P > 1 && relpm) {
    PXA_CUDA(c, launch_ad1_relpm_chain(st, kth, n, c->am, c->a0, c->ap, 0, c->E, 0, 1, P - 1, c->hsum,
                                       c->relpm_D, c->relpm_z, c->relpm_mmax, c->relpm_ts, c->relpm_nsub,
                                       relpm_direct, c->kry_tol, c->status, c->errmax), "chain");
  } else if (P > 1) {
    PXA_CUDA(c, launch_ad1_chain(st, kth, n, c->am, c->a0, c->ap, 0, c->E, 0, 1, P - 1, c->hsum,
                                 c->V, c->kry_m, c->kry_phi, hscale, steps_sub, nsub, c->kry_tol,
                                 c->v_in_smem, c->status, c->errmax), "chain");
  }
  ev_record(c, 2);
  PXA_CUDA(c, launch_ad1_superpose_direct(st, th, n, r, taps, q0, c->E + (size_t)(P - 1) * n,
                                          P > 1 ? c->hsum : nullptr, c->target, c->qT, c->srcA, Jdev,
                                          c->status), "superpose");
  }
  if (!do_a) return PXA_OK;
  PXA_CUDA(c, launch_cn_lanes(st, P, th, n, r, taps, 1, k / lq, nullptr, c->srcA, c->EA), "adj lanes");
  ev_record(c, 3);
  if (P > 1 && c->prop == PXA_PROP_BAND) {
    PXA_CUDA(c, launch_ad1_band_chain(st, n, c->band_pr, c->band_p, 1, c->EA, P - 1, -1, P - 1, c->hsumA),
             "adj chain");
  } else if (P > 1 && relpm) {
    PXA_CUDA(c, launch_ad1_relpm_chain(st, kth, n, c->am, c->a0, c->ap, 1, c->EA, P - 1, -1, P - 1, c->hsumA,
                                       c->relpm_D, c->relpm_z, c->relpm_mmax, c->relpm_ts, c->relpm_nsub,
                                       relpm_direct, c->kry_tol, c->status, c->errmax), "adj chain");
  } else if (P > 1) {
    PXA_CUDA(c, launch_ad1_chain(st, kth, n, c->am, c->a0, c->ap, 1, c->EA, P - 1, -1, P - 1,
                                 c->hsumA, c->V, c->kry_m, c->kry_phi, hscale, steps_sub, nsub,
                                 c->kry_tol, c->v_in_smem, c->status, c->errmax), "adj chain");
  }
  ev_record(c, 4);
  PXA_CUDA(c, launch_ad1_superpose_adjoint(st, n, c->qT, c->EA, P > 1 ? c->hsumA : nullptr, grad,
                                           c->status), "grad");
  ev_record(c, 5);
  return PXA_OK;
}

// Boundaries b[0..NC] (in steps) of the chunks of the overlapped direct solve: NC
// chunks of whole subintervals (P > 1) or of steps (P == 1). r == 0: equal lengths;
// 0 < r < 1: the geometric partition T_n = T (1 - r^n) / (1 - r^N) of Eq. nonEquiP,
// rounded to whole units with at least one unit per chunk. Returns NC.
int bu1_chunk_bounds(int64_t K, int P, double r, int max_chunks, int64_t* b) {
  const int64_t units = P > 1 ? P : K, unit = P > 1 ? K / P : 1;
  const int NC = (int)(units < max_chunks ? units : max_chunks);
  int64_t prev = 0;
  b[0] = 0;
  for (int i = 1; i <= NC; ++i) {
    double x;
    if (r > 0.0 && r < 1.0)
      x = (double)units * (1.0 - std::pow(r, i)) / (1.0 - std::pow(r, NC));
    else
      x = (double)units * i / NC;
    int64_t u = i == NC ? units : (int64_t)std::llround(x);
    if (u < prev + 1) u = prev + 1;
    if (u > units - (NC - i)) u = units - (NC - i);
    b[i] = u * unit;
    prev = u;
  }
  return NC;
}

// Base pointer of a buffer that holds rows first_row, first_row + 1, ... of row_len
// doubles each, such that base + row * row_len addresses row `row`: the kernels index
// their rows by absolute step and only touch the rows the buffer holds.
double* rows_from(double* buf, int64_t first_row, size_t row_len) {
  return reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(buf) -
                                   (uintptr_t)((size_t)first_row * row_len * sizeof(double)));
}

// ---- 1D Burgers, multi-checkpoint scheme (Sec. 3.5) ----------------------------------
// The direct keeps the states at t = iT/C and J (the rough pass). The adjoint takes the
// intervals [iK/C, (i+1)K/C] from the top; interval i is re-stepped from its checkpoint,
// its band (pair, four-step) records are built, the adjoint lanes of its lower P-1
// subintervals run, and the chain steps it from lambda at its top row (computed by the
// interval above; the objective's source at t = T for the top interval) down to its
// bottom row with the source of its top subinterval and the lanes' values at the
// subinterval boundaries. Then its skipped rows are filled and its gradient blocks
// summed. Two buffer sets alternate, each prepared on a stream of its own: while the
// chain runs on one interval, the next two intervals are being re-stepped and recorded.
int enqueue_bu1_iv(pxa_ctx* c, int mode, int parts, double* Jdev, double* grad, const double* sc) {
  cudaStream_t st = c->stream;
  const bool do_d = parts & 1, do_a = parts & 2;
  const int n = c->op.n, C = c->intervals;
  const int64_t K = c->K, Kc = K / C;
  const int P = mode == PXA_SERIAL ? 1 : c->P;
  const int64_t kc = Kc / P;
  const double dt = c->T / (double)K;
  if (P > 1 && c->kry_phi != PXA_PHI_STEPPER)
    return fail(c, PXA_ERR_INVALID, "the multi-checkpoint scheme uses the stepper propagator (PXA_PHI_STEPPER)");
  // with the adjoint in the same call, the rough pass keeps the top interval's states in
  // buffer set 0 (its last K/C steps in a launch of their own), which spares their re-step
  const bool keep_top = do_d && do_a;
  if (do_d) {
    ev_record(c, 0);
    if (keep_top) {
      PXA_CUDA(c, launch_bu1_rk4_sweep(st, c->cl_rk4_direct, 1, n, c->op.L, c->op.nu, dt, K - Kc, c->control, sc,
                                       nullptr, nullptr, 0, c->target, c->T, c->Jparts, c->ckpt, Kc, c->status, 0,
                                       0, c->q_direct), "rough direct");
      PXA_CUDA(c, launch_bu1_rk4_sweep(st, c->cl_rk4_direct, 1, n, c->op.L, c->op.nu, dt, Kc, c->control,
                                       sc ? sc + 3 * (K - Kc) : nullptr, c->ckpt + (size_t)(C - 1) * n,
                                       c->iv[0].traj, Kc + 1, c->target, c->T, c->Jparts + 1, nullptr, 1,
                                       c->status, 0, 0, c->q_direct), "rough direct, top interval");
      PXA_CUDA(c, launch_sum_parts(st, 2, c->Jparts, Jdev, c->status), "J");
    } else {
      PXA_CUDA(c, launch_bu1_rk4_sweep(st, c->cl_rk4_direct, 1, n, c->op.L, c->op.nu, dt, K, c->control, sc,
                                       nullptr, nullptr, 0, c->target, c->T, Jdev, c->ckpt, Kc, c->status, 0, 0,
                                       c->q_direct), "rough direct");
    }
    ev_record(c, 1);
  }
  if (!do_a) return PXA_OK;
  ev_record(c, 2);
  ev_record(c, 3);
  const bool four = c->chain_len >= 4 && bu1_chain4_valid(n, c->cl_band_chain);
  if (!four && !bu1_chain2_valid(n, c->cl_band_chain))
    return fail(c, PXA_ERR_INVALID, "no chain kernel fits the grid for the multi-checkpoint scheme");
  const int ser = P == 1 ? 1 : 0;
  const int4* plans = c->iplan_dev[ser][four ? 1 : 0];
  const std::vector<int>& off = c->iplan_off[ser][four ? 1 : 0];
  constexpr size_t RWd = BU1_BAND_RECORD, PWd = BU1_PAIR_RECORD, QWd = BU1_QUAD_RECORD;
  cudaEvent_t* const ev_rec = c->ev_iv[0];
  cudaEvent_t* const ev_chain = c->ev_iv[2];
  cudaEvent_t* const ev_free = c->ev_iv[3];
  // each buffer set has its own stream for the re-step, records and lanes, so that the
  // two sets are prepared at the same time; the fills and gradients go to side2
  cudaStream_t const prep_st[2] = {c->side, c->side3};
  PXA_CUDA(c, cudaEventRecord(c->ev_fork[0], st), "fork");
  for (cudaStream_t s2 : {c->side, c->side2, c->side3}) PXA_CUDA(c, cudaStreamWaitEvent(s2, c->ev_fork[0], 0), "fork wait");
  // re-step, records and lanes of interval number idx (from the top) into its buffer set
  auto prep = [&](int idx) -> int {
    const int ci = C - 1 - idx, set = idx & 1;
    const int64_t a = ci * Kc, b = a + Kc;
    const pxa_ctx::IntervalSet& B = c->iv[set];
    cudaStream_t ps = prep_st[set];
    if (idx >= 2) PXA_CUDA(c, cudaStreamWaitEvent(ps, ev_free[set], 0), "buffers free");
    if (!(idx == 0 && keep_top))
      PXA_CUDA(c, launch_bu1_rk4_sweep(ps, c->cl_rk4_direct, 1, n, c->op.L, c->op.nu, dt, Kc, c->control,
                                       sc ? sc + 3 * a : nullptr, c->ckpt + (size_t)ci * n, B.traj, Kc + 1,
                                       nullptr, c->T, nullptr, nullptr, 1, c->status, c->prio_lo, 0,
                                       c->q_direct), "interval re-step");
    double* rec = rows_from(B.rec, a, n * RWd);
    PXA_CUDA(c, launch_bu1_band_prepass(ps, n, c->op.L, c->op.nu, dt, c->T, c->omega, c->control,
                                        c->target, rows_from(B.traj, a, n), 0, 1, a, b == K ? b + 1 : b, K,
                                        rec, rows_from(B.jt, a, n * RWd), c->prio_lo), "band prepass");
    const int64_t m_lo = (a + 1) / 2, q_lo = (a + 3) / 4;
    PXA_CUDA(c, launch_bu1_band_pair(ps, n, rec, m_lo, b / 2, rows_from(B.rp, m_lo, n * PWd), c->prio_lo),
             "pair records");
    if (four)
      PXA_CUDA(c, launch_bu1_band_quad(ps, n, rows_from(B.rp, m_lo, n * PWd), q_lo, b / 4,
                                       rows_from(B.rq, q_lo, n * QWd), c->prio_lo), "four-step records");
    if (P > 1)
      PXA_CUDA(c, launch_bu1_band_sweep(ps, c->cl_band_lanes, P - 1, ci * P, n, rec, kc, P, 0, nullptr,
                                        rows_from(B.LI, a, n), c->ivW, c->status, c->prio_lo, c->q_sweep),
               "band lanes");
    PXA_CUDA(c, cudaEventRecord(ev_rec[set], ps), "interval ready");
    return PXA_OK;
  };
  int rc;
  if ((rc = prep(0))) return rc;
  if (C > 1 && (rc = prep(1))) return rc;
  for (int idx = 0; idx < C; ++idx) {
    const int ci = C - 1 - idx, set = idx & 1;
    const int64_t a = ci * Kc, b = a + Kc;
    const pxa_ctx::IntervalSet& B = c->iv[set];
    const double* rec = rows_from(B.rec, a, n * RWd);
    const double* rp = rows_from(B.rp, (a + 1) / 2, n * PWd);
    double* H = rows_from(B.H, a, n);
    PXA_CUDA(c, cudaStreamWaitEvent(st, ev_rec[set], 0), "interval wait");
    // lambda at the top row: the value the interval above left
    if (idx > 0)
      PXA_CUDA(c, cudaMemcpyAsync(B.H + (size_t)Kc * n, c->lamtop, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                  st), "interval top");
    const int4* pl = plans + off[ci];
    const int np = off[ci + 1] - off[ci];
    const double* from = idx > 0 ? H : nullptr;
    if (four)
      PXA_CUDA(c, launch_bu1_band_chain4(st, c->cl_band_chain, n, rec, rp, rows_from(B.rq, (a + 3) / 4, n * QWd),
                                         pl, np, (int)b, from, c->ivW, H, c->status, c->prio_hi,
                                         c->reserve_smem), "band chain");
    else
      PXA_CUDA(c, launch_bu1_band_chain2(st, c->cl_band_chain, n, rec, rp, pl, np, (int)b, from, c->ivW, H,
                                         c->status, c->prio_hi, c->reserve_smem), "band chain");
    if (ci > 0) PXA_CUDA(c, launch_bu1_band_top(st, n, B.H, B.rec, c->lamtop), "interval bottom");
    PXA_CUDA(c, cudaEventRecord(ev_chain[set], st), "chain done");
    // the rows skipped by the chain's steps, then the interval's gradient blocks
    PXA_CUDA(c, cudaStreamWaitEvent(c->side2, ev_chain[set], 0), "chain wait");
    if (four) PXA_CUDA(c, launch_bu1_band_fill4(c->side2, n, rec, rp, pl, np, H, c->prio_lo), "band fill");
    PXA_CUDA(c, launch_bu1_band_fill(c->side2, n, rec, pl, np, H, c->prio_lo), "band fill");
    PXA_CUDA(c, launch_bu1_band_grad_range(c->side2, n, dt, c->omega, a, b, c->iv_spb, a + (P - 1) * kc,
                                           P > 1 ? rows_from(B.LI, a, n) : nullptr, H,
                                           rows_from(B.jt, a, n * RWd), c->gpart, ci * c->iv_blocks,
                                           c->prio_lo), "band gradient");
    PXA_CUDA(c, cudaEventRecord(ev_free[set], c->side2), "buffers free");
    if (idx + 2 < C && (rc = prep(idx + 2))) return rc;
  }
  ev_record(c, 4);
  PXA_CUDA(c, cudaEventRecord(c->ev_join, c->side2), "join");
  PXA_CUDA(c, cudaStreamWaitEvent(st, c->ev_join, 0), "join wait");
  PXA_CUDA(c, launch_bu1_band_reduce_blocks(st, n, C * c->iv_blocks, c->gpart, grad, c->status), "gradient sum");
  ev_record(c, 5);
  return PXA_OK;
}

// ---- 1D Burgers (forcing control, tracking objective), hybrid scheme ----------
int enqueue_bu1(pxa_ctx* c, int mode, int parts, double* Jdev, double* grad) {
  cudaStream_t st = c->stream;
  const bool do_d = parts & 1, do_a = parts & 2;
  const int n = c->op.n;
  const int64_t K = c->K;
  const double dt = c->T / (double)K;
  const double h = c->op.L / n;
  Bu1Grid g{n, 1.0 / (2.0 * h), 1.0 / (h * h), c->op.nu};
  const int P = mode == PXA_SERIAL ? 1 : c->P;
  const int64_t k = K / P;
  const bool full = c->memory == PXA_STORE_FULL;
  PXA_CUDA(c, cudaMemsetAsync(c->errmax, 0, sizeof(double), st), "reset errmax");
  const double* sc = nullptr;
  if (c->omega != 0.0) {
    PXA_CUDA(c, launch_bu1_forcing_table(st, K, dt, c->omega, c->sc), "forcing table");
    sc = c->sc;
  }
  if (c->intervals >= 2) return enqueue_bu1_iv(c, mode, parts, Jdev, grad, sc);
  // Banded adjoint layout: the stepper chain covers the top subinterval itself (so lanes
  // 0..P-2 run separately); with exp(tA) (Magnus) all P lanes run and the chain uses W[P-1].
  const bool chain_top = c->band && (P == 1 || c->kry_phi == PXA_PHI_STEPPER);
  const int side_lanes = chain_top ? P - 1 : P;
  // With the overlap enabled the direct always runs in the same chunks (also for a direct
  // solve alone), so that J is summed in the same order whichever call computed it.
  const bool chunked = c->band && c->overlap && full && c->side;
  const bool overlap = chunked && do_d && do_a;
  // with the overlap, this stream waits for the last chunk's adjoint lanes only where the
  // chain first adds a lane value (the chain's top entries need the records alone)
  bool lanes_pending = false;
  if (do_d && chunked) {
    // Hybrid overlap (Sec. 3.3): the serial direct runs in chunks of whole subintervals on
    // this stream (high priority, each CTA owning its SM); after each chunk the side
    // stream builds the band records of its rows and runs the adjoint lanes whose
    // subintervals it completed, while the next chunk steps on.
    ev_record(c, 0);
    int64_t bounds[pxa_ctx::kMaxChunks + 1];
    const int NC = bu1_chunk_bounds(K, P, c->part_r, pxa_ctx::kMaxChunks, bounds);
    c->stats.chunks = NC;
    c->stats.partition_r = (float)c->part_r;
    int nch = 0;
    for (int ci = 0; ci < NC; ++ci) {
      const int64_t b0 = bounds[ci], b1 = bounds[ci + 1];
      // every row is stored: the objective is summed from the rows (off the serial path)
      PXA_CUDA(c, launch_bu1_rk4_sweep(st, c->cl_rk4_direct, 1, n, c->op.L, c->op.nu, dt, b1 - b0,
                                       c->control, sc ? sc + 3 * b0 : nullptr,
                                       ci == 0 ? nullptr : c->traj + (size_t)b0 * n,
                                       c->traj + (size_t)b0 * n, 0, nullptr, c->T, nullptr,
                                       nullptr, 1, c->status, c->prio_hi, c->reserve_smem,
                                       c->q_direct),
               "direct chunk");
      if (!overlap)
        PXA_CUDA(c, launch_bu1_objective_rows(st, c->traj, c->target, n, b0 + 1, b1 + 1, c->Jrow, 0), "objective");
      if (overlap) {
        PXA_CUDA(c, cudaEventRecord(c->ev_fork[ci], st), "fork");
        PXA_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_fork[ci], 0), "fork wait");
        PXA_CUDA(c, launch_bu1_objective_rows(c->side, c->traj, c->target, n, b0 + 1, b1 + 1, c->Jrow, c->prio_lo),
                 "objective");
        ev_record_on(c, c->ev_side[ci][0], c->side);
        PXA_CUDA(c, launch_bu1_band_prepass(c->side, n, c->op.L, c->op.nu, dt, c->T, c->omega,
                                            c->control, c->target, c->traj, 0, P, ci == 0 ? 0 : b0 + 1,
                                            b1 + 1, K, c->rec, c->jt, c->prio_lo), "band prepass");
        ev_record_on(c, c->ev_side[ci][1], c->side);
        // the adjoint lanes of the chunk (latency-bound, few SMs) on a second side stream,
        // beside the product records (throughput-bound) of the chain
        PXA_CUDA(c, cudaEventRecord(c->ev_prep[ci], c->side), "records ready");
        PXA_CUDA(c, cudaStreamWaitEvent(c->side2, c->ev_prep[ci], 0), "records wait");
        if (c->rp)
          PXA_CUDA(c, launch_bu1_band_pair(c->side, n, c->rec, (b0 + 1) / 2, (b1 + 1) / 2, c->rp,
                                           c->prio_lo), "pair records");
        ev_record_on(c, c->ev_side[ci][2], c->side);
        if (c->rq)
          PXA_CUDA(c, launch_bu1_band_quad(c->side, n, c->rp, (b0 + 1) / 4, (b1 + 1) / 4, c->rq, c->prio_lo),
                   "four-step records");
        ev_record_on(c, c->ev_side[ci][3], c->side);
        const int l0 = (int)(b0 / k), l1 = (int)(b1 / k) < side_lanes ? (int)(b1 / k) : side_lanes;
        // the lanes of the last chunk run with no direct solve beside them: a cluster as
        // wide as the chain's steps them about twice as fast as the narrow ones that share
        // the GPU with the direct
        const int cl = ci == NC - 1 && (l1 - l0) * c->cl_band_chain <= 128 ? c->cl_band_chain : c->cl_band_lanes;
        if (l1 > l0) {
          ev_record_on(c, c->ev_side[ci][4], c->side2);
          PXA_CUDA(c, launch_bu1_band_sweep(c->side2, cl, l1 - l0, l0, n, c->rec, k, P, 0,
                                            nullptr, c->LI, c->E, c->status, c->prio_lo, c->q_sweep),
                                            "band lanes");
          ev_record_on(c, c->ev_side[ci][5], c->side2);
        }
        if (c->timing && c->ev_ready) {
          c->side_marked = ci + 1;
          c->side_lanes_marked[ci] = l1 > l0;
        }
      }
      ++nch;
    }
    (void)nch;
    ev_record(c, 1);
    if (!overlap)
      PXA_CUDA(c, launch_bu1_objective_sum(st, c->Jrow, K, dt / c->T, Jdev, c->status), "J");
    if (overlap) {
      ev_record(c, 2);
      PXA_CUDA(c, cudaEventRecord(c->ev_join, c->side), "join");
      PXA_CUDA(c, cudaStreamWaitEvent(st, c->ev_join, 0), "join wait");
      PXA_CUDA(c, cudaEventRecord(c->ev_join2, c->side2), "join");
      // the fills and gradient segments on the side stream read the lanes' values
      PXA_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_join2, 0), "join wait");
      lanes_pending = true;
      PXA_CUDA(c, launch_bu1_objective_sum(st, c->Jrow, K, dt / c->T, Jdev, c->status), "J");
      if (c->timing && c->ev_ready) {
        ev_record(c, 6);
        c->prep_marked = true;
      }
      ev_record(c, 3);
    }
  } else if (do_d) {
    ev_record(c, 0);
    // direct (Eq. seriesDirect) on one cluster; every state (full storage) or the P+1
    // subinterval boundaries (checkpoints) are kept
    PXA_CUDA(c, launch_bu1_rk4_sweep(st, c->cl_rk4_direct, 1, n, c->op.L, c->op.nu, dt, K, c->control,
                                     sc, nullptr, full ? c->traj : nullptr, 0, full ? nullptr : c->target, c->T,
                                     full ? nullptr : Jdev, full ? nullptr : c->traj, k, c->status, 0, 0,
                                     c->q_direct), "direct");
    if (full) {  // the objective from the stored rows, in the same order as the chunked direct
      PXA_CUDA(c, launch_bu1_objective_rows(st, c->traj, c->target, n, 1, K + 1, c->Jrow, 0), "objective");
      PXA_CUDA(c, launch_bu1_objective_sum(st, c->Jrow, K, dt / c->T, Jdev, c->status), "J");
    }
    ev_record(c, 1);
  }
  if (!do_a) return PXA_OK;
  if (!overlap) ev_record(c, 2);
  if (c->band && !overlap) {
    // Banded discrete adjoint: stored (or recomputed) states -> rows of M_s^T (parallel),
    // P adjoint lanes + the homogeneous chain as 9-tap recursions, then the forcing
    // gradient over all steps (parallel).
    const double* rows = c->traj;
    int64_t lane_k = 0;
    if (!full) {
      PXA_CUDA(c, launch_bu1_rk4_sweep(st, P == 1 ? c->cl_rk4_direct : c->cl_rk4_lanes, P, n,
                                       c->op.L, c->op.nu, dt, k, c->control, sc, c->traj, c->scratch,
                                       k + 1, nullptr, c->T, nullptr, nullptr, 1, c->status, 0, 0,
                                       c->q_direct),
               "recompute");
      rows = c->scratch;
      lane_k = k;
    }
    PXA_CUDA(c, launch_bu1_band_prepass(st, n, c->op.L, c->op.nu, dt, c->T, c->omega, c->control,
                                        c->target, rows, lane_k, P, 0, K + 1, K, c->rec, c->jt, 0),
             "band prepass");
    if (c->rp) PXA_CUDA(c, launch_bu1_band_pair(st, n, c->rec, 0, K / 2, c->rp, 0), "pair records");
    if (c->rq) PXA_CUDA(c, launch_bu1_band_quad(st, n, c->rp, 0, K / 4, c->rq, 0), "four-step records");
    if (c->timing && c->ev_ready) {
      ev_record(c, 6);
      c->prep_marked = true;
    }
    PXA_CUDA(c, launch_bu1_band_sweep(st, c->cl_band_lanes, side_lanes, 0, n, c->rec, k, P, 0, nullptr,
                                      c->LI, c->E, c->status, 0, c->q_sweep), "band lanes");
    ev_record(c, 3);
  }
  auto join_lanes = [&]() -> int {
    if (lanes_pending) {
      PXA_CUDA(c, cudaStreamWaitEvent(st, c->ev_join2, 0), "join wait");
      lanes_pending = false;
    }
    return PXA_OK;
  };
  int rc_join = PXA_OK;
  if (c->band) {
    const double* rows = full ? c->traj : c->scratch;
    const int64_t lane_k = full ? 0 : k;
    const bool four = chain_top && c->rq && bu1_chain4_valid(n, c->cl_band_chain);
    if (four || (chain_top && c->rp && bu1_chain2_valid(n, c->cl_band_chain))) {
      // the top subinterval with its source, then the summed homogeneous problems, four
      // or two steps per exchange where the plan allows; then the rows skipped inside
      // those steps. With the overlap on, the chain runs in segments: after each one the
      // side stream fills its skipped rows and sums the gradient over the step blocks
      // whose rows are final, while the next segment runs (its CTAs own their SMs).
      const pxa_ctx::ChainPlan& pl = c->plans[P == 1 ? 1 : 0][four ? 1 : 0];
      const int np = pl.count;
      auto chain = [&](int j0, int j1, int s_hi, const double* from, int prio, size_t reserve) {
        return four ? launch_bu1_band_chain4(st, c->cl_band_chain, n, c->rec, c->rp, c->rq, pl.dev + j0, j1 - j0,
                                             s_hi, from, c->E, c->Hrows, c->status, prio, reserve)
                    : launch_bu1_band_chain2(st, c->cl_band_chain, n, c->rec, c->rp, pl.dev + j0, j1 - j0,
                                             s_hi, from, c->E, c->Hrows, c->status, prio, reserve);
      };
      auto fill = [&](cudaStream_t fs, int j0, int j1, int prio) -> cudaError_t {
        if (four) {
          cudaError_t e = launch_bu1_band_fill4(fs, n, c->rec, c->rp, pl.dev + j0, j1 - j0, c->Hrows, prio);
          if (e != cudaSuccess) return e;
        }
        return launch_bu1_band_fill(fs, n, c->rec, pl.dev + j0, j1 - j0, c->Hrows, prio);
      };
      int S = (c->overlap && c->side) ? c->chain_segments : 1;
      if (S > pxa_ctx::kMaxSeg) S = pxa_ctx::kMaxSeg;
      if (np < 64 * S) S = 1;
      if (S == 1) {
        if ((rc_join = join_lanes())) return rc_join;
        PXA_CUDA(c, chain(0, np, (int)K, nullptr, 0, 0), "band chain");
        PXA_CUDA(c, fill(st, 0, np, 0), "band fill");
      } else {
        const int spb = bu1_band_steps_per_block(K, n);
        const int64_t li_top = (int64_t)(P - 1) * k;
        int b_hi = bu1_band_grad_blocks(K, n);  // blocks [b_hi, end) are summed already
        // the first plan entry that adds a lane value
        int ja = 0;
        while (ja < np && pl.host[ja].w == 0) ++ja;
        for (int i = 0; i < S; ++i) {
          const int j0 = (int)((int64_t)np * i / S), j1 = (int)((int64_t)np * (i + 1) / S);
          const int s_hi = i == 0 ? (int)K : pl.host[j0 - 1].x;
          if (lanes_pending && ja > j0 && ja < j1) {
            // the entries above the first lane value run while the last lanes finish
            PXA_CUDA(c, chain(j0, ja, s_hi, i == 0 ? nullptr : c->Hrows, c->prio_hi, c->reserve_smem),
                     "band chain");
            if ((rc_join = join_lanes())) return rc_join;
            PXA_CUDA(c, chain(ja, j1, pl.host[ja - 1].x, c->Hrows, c->prio_hi, c->reserve_smem), "band chain");
          } else {
            if ((rc_join = join_lanes())) return rc_join;
            PXA_CUDA(c, chain(j0, j1, s_hi, i == 0 ? nullptr : c->Hrows, c->prio_hi, c->reserve_smem),
                     "band chain");
          }
          PXA_CUDA(c, cudaEventRecord(c->ev_seg[i], st), "segment");
          PXA_CUDA(c, cudaStreamWaitEvent(c->side, c->ev_seg[i], 0), "segment wait");
          PXA_CUDA(c, fill(c->side, j0, j1, c->prio_lo), "band fill");
          // rows >= low are final; block b reads rows b spb + 1 .. (b + 1) spb
          const int64_t low = pl.host[j1 - 1].x;
          const int b_lo = i == S - 1 ? 0 : (int)((low - 1 + spb - 1) / spb);
          PXA_CUDA(c, launch_bu1_band_grad_part(c->side, n, dt, c->omega, K, li_top,
                                                side_lanes > 0 ? c->LI : nullptr, c->Hrows, c->jt, c->gpart,
                                                b_lo, b_hi, c->prio_lo), "band gradient");
          b_hi = b_lo < b_hi ? b_lo : b_hi;
        }
        ev_record(c, 4);
        PXA_CUDA(c, cudaEventRecord(c->ev_join, c->side), "join");
        PXA_CUDA(c, cudaStreamWaitEvent(st, c->ev_join, 0), "join wait");
        PXA_CUDA(c, launch_bu1_band_grad_reduce(st, n, K, c->gpart, nullptr, grad, c->status), "gradient sum");
        ev_record(c, 5);
        return PXA_OK;
      }
    } else if (chain_top) {
      // the top subinterval with its source, then the summed homogeneous problems
      if ((rc_join = join_lanes())) return rc_join;
      PXA_CUDA(c, launch_bu1_band_sweep(st, c->cl_band_chain, 1, 0, n, c->rec, k, P, 1, c->E, c->Hrows,
                                        nullptr, c->status, 0, c->q_sweep), "band chain");
    } else {
      if ((rc_join = join_lanes())) return rc_join;
      PXA_CUDA(c, launch_bu1_magnus_chain(st, n > 2048 ? 1024 : 512, g, dt, K, P, k, c->magnus_M,
                                          c->omega, rows, lane_k, c->E, c->hsum, c->V, c->kry_m,
                                          c->kry_tol, c->v_in_smem, c->status, c->errmax),
               "magnus chain");
    }
    ev_record(c, 4);
    PXA_CUDA(c, launch_bu1_band_grad(st, n, dt, c->omega, K, chain_top ? (int64_t)(P - 1) * k : K,
                                     side_lanes > 0 ? c->LI : nullptr, chain_top ? c->Hrows : nullptr,
                                     c->jt, c->gpart, chain_top ? nullptr : c->hsum, grad, c->status),
             "band gradient");
    ev_record(c, 5);
    return PXA_OK;
  }
  if ((rc_join = join_lanes())) return rc_join;
  const int cl_lane = P == 1 ? c->cl_direct : c->cl_lanes;
  PXA_CUDA(c, launch_bu1c_adjoint_lanes(st, cl_lane, P, n, c->op.L, c->op.nu, dt, c->T, k, c->omega,
                                        c->control, c->target, full ? c->traj : nullptr,
                                        full ? nullptr : c->traj, c->scratch, c->E, c->EA),
           "adjoint lanes");
  ev_record(c, 3);
  if (P > 1 && c->kry_phi == PXA_PHI_STEPPER) {
    PXA_CUDA(c, launch_bu1c_stepper_chain(st, c->cl_chain, n, c->op.L, c->op.nu, dt, c->T, k, P,
                                          c->omega, c->control, c->target,
                                          full ? c->traj : c->scratch, full ? 0 : k, c->E, c->hsum),
             "stepper chain");
  } else if (P > 1) {
    PXA_CUDA(c, launch_bu1_magnus_chain(st, n > 2048 ? 1024 : 512, g, dt, K, P, k, c->magnus_M, c->omega,
                                        full ? c->traj : c->scratch, full ? 0 : k, c->E, c->hsum, c->V, c->kry_m, c->kry_tol, c->v_in_smem,
                                        c->status, c->errmax), "magnus chain");
  }
  ev_record(c, 4);
  PXA_CUDA(c, launch_sum_lanes(st, n, P, c->EA, P > 1 ? c->hsum : nullptr, grad, c->status), "sum");
  ev_record(c, 5);
  return PXA_OK;
}

// ---- 2D advection-diffusion (forcing control, tracking of the f_true trajectory) ----
int enqueue_ad2(pxa_ctx* c, int mode, int parts, double* Jdev, double* grad) {
  cudaStream_t st = c->stream;
  Ad2Params a = c->p2;
  a.omega = c->omega;
  const bool do_d = parts & 1, do_a = parts & 2;
  const int64_t K = c->K;
  const int P = mode == PXA_SERIAL ? 1 : c->P;
  const int64_t k = K / P;
  const size_t N = (size_t)a.nx * a.ny, plane = (size_t)a.Hp * a.Wp;
  const int tiles = a.tiles_x * a.tiles_y;
  const double src = 2.0 * a.dtd / c->T;
  if (mode == PXA_PARAEXP && c->kry_phi != PXA_PHI_STEPPER)
    return fail(c, PXA_ERR_INVALID, "ADVDIFF_2D Paraexp uses the stepper propagator (PXA_PHI_STEPPER)");
  PXA_CUDA(c, launch_ad2_pack_coef(st, a, c->op.u_dev, c->op.v_dev, c->control, c->target, c->coef2),
           "pack coefficients");
  PXA_CUDA(c, launch_ad2_forcing_table(st, 0, K, a.dtd, a.omega, c->sc2), "forcing table");
  if (do_d) {
    ev_record(c, 0);
    // Eq. seriesDirect: serial FP32 RK4 of the response to f - f_true, storing every state
    PXA_CUDA(c, cudaMemsetAsync(c->stD, 0, sizeof(float) * plane, st), "zero state");
    PXA_CUDA(c, cudaMemsetAsync(c->traj2, 0, sizeof(float) * N, st), "zero row 0");
    for (int64_t s = 0; s < K; ++s) {
      PXA_CUDA(c, launch_ad2_rk4(st, c->mapD, c->mapCoef, a, c->stD, 1, 1, 1, (int)(s & 1), 0, s, c->sc2,
                                 c->traj2, s + 1, c->Jpart, s, c->status, s > 0),
               "2d direct step");
    }
    PXA_CUDA(c, launch_ad2_reduce_J(st, c->Jpart, (size_t)K * tiles * AD2_J_WARPS, a.dtd / c->T, c->Jred, Jdev,
                                    c->status),
             "reduce J");
    ev_record(c, 1);
  }
  if (!do_a) return PXA_OK;
  ev_record(c, 2);
  // the lanes as a register wavefront where the grid allows it (FP32 gradients G2f), else on
  // halo tiles (double-float gradients G2buf): zero the one in use
  const bool roll = c->roll2 && P > 1;
  if (roll)
    PXA_CUDA(c, cudaMemsetAsync(c->G2f, 0, sizeof(float) * (size_t)P * N, st), "zero Gf");
  else
    PXA_CUDA(c, cudaMemsetAsync(c->G2buf, 0, sizeof(float2) * (size_t)P * N, st), "zero G");
  PXA_CUDA(c, cudaMemsetAsync(c->GC, 0, sizeof(float2) * N, st), "zero GC");
  // Eq. hybadjinhom: lane l starts from the objective's source at its top row (l+1) k
  PXA_CUDA(c, launch_ad2_fill(st, a, c->stA, P, c->traj2, k, k, src), "lane init");
  const int lpc = P >= 16 ? 16 : P;
  if (roll) {
    PXA_CUDA(c, launch_ad2_pack_coefT(st, a, c->op.u_dev, c->op.v_dev, c->tcoef2), "A^T coefficients");
  }
  for (int64_t j = 0; j < k; ++j) {
    const int64_t s_local = k - 1 - j;  // lane l at step l k + s_local
    if (roll)
      PXA_CUDA(c, launch_ad2_rk4T_roll(st, c->mapA4, c->mapT4, c->mapS4, c->mapG4, a, c->stA, c->G2f, P, 0, P,
                                       (int)(j & 1), c->sc2, (int)s_local, (int)k, (float)src, s_local > 0 ? 1 : 0,
                                       c->status),
               "2d adjoint lanes");
    else
      PXA_CUDA(c, launch_ad2_rk4T(st, c->mapA, c->mapCoef, a, c->stA, P, P, lpc, (int)(j & 1), k, 0, s_local, 1,
                                  c->traj2, src, c->G2buf, c->sc2, c->status, P == 1 && j > 0),
               "2d adjoint lanes");
  }
  ev_record(c, 3);
  if (P > 1 && c->poly_m > 0) {
    // Eq. adjHomNormal with the stepper's own propagator as its power series: the summed
    // homogeneous problems are carried down segment by segment (kk steps each, `sub` per
    // subinterval), h <- a(tau A^T)(h + w), and each segment's forcing gradient
    // b_s(tau A^T)(h + w) goes to GC; w is the lane value at the subinterval's top, added
    // at the first segment of each subinterval (a, b cut after degree m)
    const int m = c->poly_m, sub = c->poly_sub, kk = c->poly_kk;
    const int segments = (P - 1) * sub;
    const float tau = (float)((double)kk * a.dtd);
    PXA_CUDA(c, launch_ad2_poly_forcing(st, segments, kk, m, a.dtd, a.omega, c->polyQ, c->polyB), "poly forcing");
    PXA_CUDA(c, cudaMemsetAsync(c->hC, 0, sizeof(float) * plane, st), "zero chain");
    for (int sg = segments - 1; sg >= 0; --sg) {
      const bool top = (sg + 1) % sub == 0;  // the segment ends at a subinterval's top
      const int lane_above = (sg + 1) / sub;  // its lane value when it does
      // the first launch reads h + w itself: plane (k & 1) P + lane_above of the lane states
      const int w_z = top ? (int)((k & 1) * P + lane_above) : -1;
      const float* cb = c->polyB + (size_t)sg * (m + 1);
      for (int i0 = 0, buf = 0; i0 < m; i0 += 4, buf ^= 1)
        PXA_CUDA(c, launch_ad2_poly(st, c->mapC, c->mapCoef, c->mapH, c->mapA, w_z, a, tau, c->stC, buf, i0,
                                    c->polyA, cb, c->hC, sg > 0 ? 1 : 0, c->GC, c->status, i0 > 0),
                 "2d chain series");
    }
  } else if (P > 1) {
    // Eq. adjHomNormal with the stepper's own propagator: h = sum of the lane values
    // W_{l+1} carried down subinterval by subinterval, no source
    const float* Wbuf = c->stA + (size_t)(k & 1) * P * plane;
    PXA_CUDA(c, cudaMemsetAsync(c->stC, 0, sizeof(float) * plane, st), "zero chain");
    int bufc = 0;
    for (int lane = P - 2; lane >= 0; --lane) {
      PXA_CUDA(c, launch_ad2_add_padded(st, plane, c->stC + (size_t)bufc * plane,
                                        Wbuf + (size_t)(lane + 1) * plane), "chain add");
      for (int64_t j = 0; j < k; ++j) {
        PXA_CUDA(c, launch_ad2_rk4T(st, c->mapC, c->mapCoef, a, c->stC, 1, 1, 1, bufc, 0,
                                    (int64_t)lane * k, k - 1 - j, 0, nullptr, 0.0, c->GC, c->sc2, c->status,
                                    j > 0),
                 "2d chain step");
        bufc ^= 1;
      }
    }
  }
  ev_record(c, 4);
  PXA_CUDA(c, launch_ad2_sum_grad(st, N, roll ? 0 : P, c->G2buf, roll ? P : 0, c->G2f, P > 1 ? c->GC : nullptr, grad,
                                  c->status),
           "sum grad");
  ev_record(c, 5);
  return PXA_OK;
}

// ---- general sparse operator (CSR), classical RK4, IC control, terminal objective -----
// parts: bit 0 = direct solve (J, lambda(T), adjoint source), bit 1 = adjoint solve
int enqueue_csr(pxa_ctx* c, int mode, int parts, double* Jdev, double* grad) {
  cudaStream_t st = c->stream;
  const bool do_d = parts & 1, do_a = parts & 2;
  const int n = c->op.n;
  const int64_t* rp = c->op.row_ptr_dev;
  const int32_t* col = c->op.col_dev;
  const double* val = c->op.val_dev;
  const int64_t K = c->K;
  const double dt = c->T / (double)K;
  const double* q0 = c->control;
  if (mode == PXA_SERIAL) {
    // Eq. seriesDirect: one lane of K steps from q0; lambda(T) = q(T) - g; the adjoint
    // sweep of K transposed steps from lambda(T) gives lambda(0) = grad (Eq. initupdate)
    if (do_d) {
      ev_record(c, 0);
      PXA_CUDA(c, launch_csr_rk4_lanes(st, 1, n, rp, col, val, nullptr, dt, K, q0, c->E, c->csr_work), "serial");
      ev_record(c, 1);
      ev_record(c, 2);
      PXA_CUDA(c, launch_csr_superpose(st, n, nullptr, c->E, nullptr, c->target, c->qT, Jdev, c->status),
               "objective");
    }
    if (do_a) {
      PXA_CUDA(c, launch_csr_rk4_lanes(st, 1, n, c->rpT, c->colT, c->valT, nullptr, dt, K, c->qT, c->EA,
                                       c->csr_work), "serial adjoint");
      ev_record(c, 3);
      ev_record(c, 4);
      PXA_CUDA(c, launch_ad1_superpose_adjoint(st, n, nullptr, c->EA, nullptr, grad, c->status), "grad");
      ev_record(c, 5);
    }
    return PXA_OK;
  }
  const int P = c->P;
  const int64_t k = K / P;
  const int nsub = c->kry_sub;
  const int64_t steps_sub = k / nsub;
  const int phi_mode = c->kry_phi == PXA_PHI_EXP ? 0 : 2;  // exp(tau A) or the RK4 power
  const double hscale = c->kry_phi == PXA_PHI_EXP ? dt * (double)steps_sub : dt;
  if (do_d) {
    PXA_CUDA(c, cudaMemsetAsync(c->errmax, 0, sizeof(double), st), "reset errmax");
    ev_record(c, 0);
    // Eq. linzero / linInhomEqus: the shifted lanes start from zero with the source A q0
    PXA_CUDA(c, (pxa_spmv_csr(st, n, rp, col, val, q0, c->src) == PXA_OK ? cudaSuccess : cudaErrorLaunchFailure),
             "source");
    PXA_CUDA(c, launch_csr_rk4_lanes(st, P, n, rp, col, val, c->src, dt, k, nullptr, c->E, c->csr_work), "lanes");
    ev_record(c, 1);
    // Eq. hom: the summed homogeneous problems, h <- Phi (h + e_j), j = 0 .. P-2
    if (P > 1 && c->poly_m > 0)  // the stepper's propagator as its power series in kk dt A
      PXA_CUDA(c, launch_csr_series_chain(st, n, rp, col, val, c->E, 0, 1, P - 1, c->hsum, c->polyAd, c->poly_m,
                                          c->poly_sub, (double)c->poly_kk * dt, c->V),
               "chain");
    else if (P > 1)
      PXA_CUDA(c, launch_csr_chain(st, n, rp, col, val, c->E, 0, 1, P - 1, c->hsum, c->V, c->kry_m, phi_mode,
                                   hscale, steps_sub, nsub, c->kry_tol, c->v_in_smem, c->status, c->errmax),
               "chain");
    ev_record(c, 2);
    // Eq. fullsol0 at T, J and lambda(T) = q(T) - g; the adjoint lanes' source A^T lambda(T)
    PXA_CUDA(c, launch_csr_superpose(st, n, q0, c->E + (size_t)(P - 1) * n, P > 1 ? c->hsum : nullptr, c->target,
                                     c->qT, Jdev, c->status), "superpose");
    PXA_CUDA(c, (pxa_spmv_csr(st, n, c->rpT, c->colT, c->valT, c->qT, c->srcA) == PXA_OK ? cudaSuccess
                                                                                         : cudaErrorLaunchFailure),
             "adjoint source");
  }
  if (!do_a) return PXA_OK;
  // Eq. adjInhom: the shifted adjoint lanes from zero at T_{p+1} with A^T and A^T lambda(T)
  PXA_CUDA(c, launch_csr_rk4_lanes(st, P, n, c->rpT, c->colT, c->valT, c->srcA, dt, k, nullptr, c->EA,
                                   c->csr_work), "adjoint lanes");
  ev_record(c, 3);
  // Eq. adjHomNormal: carried down from the top with Phi^T
  if (P > 1 && c->poly_m > 0)
    PXA_CUDA(c, launch_csr_series_chain(st, n, c->rpT, c->colT, c->valT, c->EA, P - 1, -1, P - 1, c->hsumA,
                                        c->polyAd, c->poly_m, c->poly_sub, (double)c->poly_kk * dt, c->V),
             "adjoint chain");
  else if (P > 1)
    PXA_CUDA(c, launch_csr_chain(st, n, c->rpT, c->colT, c->valT, c->EA, P - 1, -1, P - 1, c->hsumA, c->V,
                                 c->kry_m, phi_mode, hscale, steps_sub, nsub, c->kry_tol, c->v_in_smem, c->status,
                                 c->errmax), "adjoint chain");
  ev_record(c, 4);
  // Eq. fulladjsol at 0, Eq. initupdate: grad = lambda(T) + e_0 + h
  PXA_CUDA(c, launch_ad1_superpose_adjoint(st, n, c->qT, c->EA, P > 1 ? c->hsumA : nullptr, grad, c->status),
           "grad");
  ev_record(c, 5);
  return PXA_OK;
}

// ---- 2D viscous Burgers (Sec. 4.3), IC control, terminal objective ----------------------
// The hybrid scheme (Sec. 3.3): the direct is stepped serially (FP32 RK4, every state kept);
// with a terminal objective the adjoint's inhomogeneous problems have no source, so they
// vanish, and the Paraexp adjoint is the one homogeneous problem carried from T by the
// stepper's own transposed step maps: the serial adjoint. Both modes run the same kernels.
int enqueue_bu2(pxa_ctx* c, int mode, int parts, double* Jdev, double* grad) {
  (void)mode;
  cudaStream_t st = c->stream;
  const int n = c->op.nx;
  const int64_t K = c->K;
  const double dt = c->T / (double)K;
  const size_t plane2 = 2 * (size_t)n * n;
  float* tr = c->b2traj;
  if (parts & 1) {
    ev_record(c, 0);
    PXA_CUDA(c, launch_bu2_convert(st, c->control, tr, plane2), "initial state");
    for (int64_t s = 0; s < K; ++s)
      PXA_CUDA(c, launch_bu2_step(st, tr + (size_t)s * plane2, tr + (size_t)(s + 1) * plane2, n, c->op.L, c->op.nu, dt),
               "direct step");
    ev_record(c, 1);
    ev_record(c, 2);
    PXA_CUDA(c, launch_bu2_terminal(st, tr + (size_t)K * plane2, c->target, n, c->b2lam, c->b2Jpart, Jdev, c->status),
             "objective");
  }
  if (!(parts & 2)) return PXA_OK;
  ev_record(c, 3);
  float* lam[2] = {c->b2lam, c->b2lam + plane2};
  int cur = 0;
  for (int64_t s = K - 1; s >= 0; --s) {
    PXA_CUDA(c, launch_bu2_adj_step(st, tr + (size_t)s * plane2, lam[cur], lam[cur ^ 1], n, c->op.L, c->op.nu, dt),
             "adjoint step");
    cur ^= 1;
  }
  ev_record(c, 4);
  PXA_CUDA(c, launch_bu2_convert_back(st, lam[cur], grad, plane2, c->status), "gradient");
  ev_record(c, 5);
  return PXA_OK;
}

// The objective kinds each operator supports (0: the operator's default).
bool objective_ok(int kind, int obj) {
  if (obj == 0) return true;
  if (kind == PXA_ADVDIFF_1D || kind == PXA_CSR || kind == PXA_BURGERS_2D) return obj == PXA_OBJ_TERMINAL_L2;
  return obj == PXA_OBJ_INTEGRAL_TRACKING;
}

int enqueue_parts(pxa_ctx* c, int mode, int parts, double* Jdev, double* grad) {
  if (mode != PXA_SERIAL && mode != PXA_PARAEXP) return fail(c, PXA_ERR_INVALID, "mode");
  if (!c->control) return fail(c, PXA_ERR_STATE, "set_control first");
  if (c->op.kind == PXA_BURGERS_1D && !c->target) return fail(c, PXA_ERR_STATE, "set_target first");
  if (c->op.kind == PXA_ADVDIFF_2D && !c->target) return fail(c, PXA_ERR_STATE, "set_target (f_true) first");
  if (!objective_ok(c->op.kind, c->obj_kind)) return fail(c, PXA_ERR_INVALID, "objective kind for this operator");
  if (c->op.kind == PXA_ADVDIFF_1D) return enqueue_ad1(c, mode, parts, Jdev, grad);
  if (c->op.kind == PXA_ADVDIFF_2D) return enqueue_ad2(c, mode, parts, Jdev, grad);
  if (c->op.kind == PXA_CSR) return enqueue_csr(c, mode, parts, Jdev, grad);
  if (c->op.kind == PXA_BURGERS_2D) {
    if (!c->target) return fail(c, PXA_ERR_STATE, "set_target (the target final state) first");
    return enqueue_bu2(c, mode, parts, Jdev, grad);
  }
  return enqueue_bu1(c, mode, parts, Jdev, grad);
}

int enqueue(pxa_ctx* c, int mode, double* Jdev, double* grad) {
  return enqueue_parts(c, mode, 3, Jdev, grad);
}

int read_status(pxa_ctx* c) {
  int st = 0;
  double em = 0.0;
  PXA_CUDA(c, cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  PXA_CUDA(c, cudaMemcpy(&em, c->errmax, sizeof(double), cudaMemcpyDeviceToHost), "read errmax");
  c->stats.krylov_err_max = em;
  if (st != 0) {
    PXA_CUDA(c, cudaMemset(c->status, 0, sizeof(int)), "reset status");
    if (st == PXA_ERR_NOT_CONVERGED)
      return fail(c, st, "Krylov error estimate above tolerance (increase m or substeps)");
    if (st == PXA_ERR_NONFINITE) return fail(c, st, "objective or gradient is not finite");
    return fail(c, st, "device error status " + std::to_string(st));
  }
  return PXA_OK;
}

}  // namespace

// ============================================================================
extern "C" {

int pxa_create(pxa_ctx** out, int device, void* cuda_stream) {
  if (!out) return PXA_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return PXA_ERR_CUDA;
  }
  pxa_ctx* c = new pxa_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = c;
  return PXA_OK;
}

void pxa_destroy(pxa_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  release_workspace(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& row : c->ev_side)
    for (auto& e : row)
      if (e) cudaEventDestroy(e);
  delete c;
}

const char* pxa_last_error(const pxa_ctx* c) { return c ? c->err.c_str() : "null context"; }

int pxa_set_operator(pxa_ctx* c, const pxa_operator_desc* op) {
  if (!c || !op) return PXA_ERR_INVALID;
  if (op->kind != PXA_ADVDIFF_1D && op->kind != PXA_BURGERS_1D && op->kind != PXA_ADVDIFF_2D &&
      op->kind != PXA_CSR && op->kind != PXA_BURGERS_2D)
    return fail(c, PXA_ERR_INVALID, "operator kind");
  c->obj_kind = 0;
  c->step_prec = (op->kind == PXA_ADVDIFF_2D || op->kind == PXA_BURGERS_2D) ? PXA_F32 : PXA_F64;
  if (op->kind == PXA_BURGERS_2D) {
    if (op->nx != op->ny || op->nx % BU2_TILE != 0 || op->nx < BU2_TILE || op->nx > 4096 || !(op->L > 0.0) ||
        !(op->nu >= 0.0))
      return fail(c, PXA_ERR_INVALID, "2D Burgers grid (nx == ny, nx % 16 == 0, 16 <= nx <= 4096, L > 0, nu >= 0)");
    c->op = *op;
    c->op.n = 2 * op->nx * op->ny;
    c->have_op = true;
    release_workspace(c);
    invalidate(c);
    return PXA_OK;
  }
  if (op->kind == PXA_CSR) {
    if (op->n < 1 || op->n > 16384 || !op->row_ptr_dev || !op->col_dev || !op->val_dev)
      return fail(c, PXA_ERR_INVALID, "CSR operator (1 <= n <= 16384, row_ptr, col, val)");
    c->op = *op;
    c->have_op = true;
    release_workspace(c);
    invalidate(c);
    return PXA_OK;
  }
  if (op->kind == PXA_ADVDIFF_2D) {
    if (op->nx != op->ny || op->nx % 4 != 0 || op->nx < 8 || op->nx > 8192 || !(op->L > 0.0) ||
        !(op->nu >= 0.0) || !op->u_dev || !op->v_dev)
      return fail(c, PXA_ERR_INVALID, "2D operator (nx == ny, nx % 4 == 0, 8 <= nx <= 8192, velocity)");
    c->op = *op;
    c->op.n = op->nx * op->ny;
    c->have_op = true;
    release_workspace(c);
    invalidate(c);
    return PXA_OK;
  }
  const int nmax = op->kind == PXA_ADVDIFF_1D ? (1 << 26) : 4096;
  if (op->n < 3 || op->n > nmax || !(op->L > 0.0) || !(op->nu >= 0.0))
    return fail(c, PXA_ERR_INVALID, "operator parameters (3 <= n <= 4096 (ADVDIFF_1D: 2^26), L > 0, nu >= 0)");
  c->op = *op;
  double h = op->L / op->n;
  c->am = op->c / (2.0 * h) + op->nu / (h * h);
  c->a0 = -2.0 * op->nu / (h * h);
  c->ap = -op->c / (2.0 * h) + op->nu / (h * h);
  c->have_op = true;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_time(pxa_ctx* c, double T, int64_t K, int stepper, int P) {
  if (!c) return PXA_ERR_INVALID;
  if (!(T > 0.0) || K < 1 || P < 1 || K % P != 0) return fail(c, PXA_ERR_INVALID, "T > 0, K >= 1, P >= 1, K % P == 0");
  if (!c->have_op) return fail(c, PXA_ERR_STATE, "set_operator first");
  if (c->op.kind == PXA_ADVDIFF_1D && stepper != PXA_CN) return fail(c, PXA_ERR_INVALID, "ADVDIFF_1D uses PXA_CN");
  if (c->op.kind == PXA_BURGERS_1D && stepper != PXA_RK4) return fail(c, PXA_ERR_INVALID, "BURGERS_1D uses PXA_RK4");
  if (c->op.kind == PXA_ADVDIFF_2D && stepper != PXA_RK4) return fail(c, PXA_ERR_INVALID, "ADVDIFF_2D uses PXA_RK4");
  if (c->op.kind == PXA_CSR && stepper != PXA_RK4) return fail(c, PXA_ERR_INVALID, "CSR uses PXA_RK4");
  if (c->op.kind == PXA_BURGERS_2D && stepper != PXA_RK4) return fail(c, PXA_ERR_INVALID, "BURGERS_2D uses PXA_RK4");
  if (c->op.kind == PXA_BURGERS_1D && K < 4) return fail(c, PXA_ERR_INVALID, "K >= 4 for time interpolation");
  c->T = T;
  c->K = K;
  c->stepper = stepper;
  c->P = P;
  c->have_time = true;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_krylov(pxa_ctx* c, int m, double tol, int phi, int substeps) {
  if (!c) return PXA_ERR_INVALID;
  if (m < 2 || m > 48 || !(tol > 0.0) || (phi != PXA_PHI_EXP && phi != PXA_PHI_STEPPER) || substeps < 1)
    return fail(c, PXA_ERR_INVALID, "krylov parameters (2 <= m <= 48, tol > 0, substeps >= 1)");
  if (c->have_time && (c->K / c->P) % substeps != 0)
    return fail(c, PXA_ERR_INVALID, "substeps must divide the steps of one subinterval");
  c->kry_m = m;
  c->kry_tol = tol;
  c->kry_phi = phi;
  c->kry_sub = substeps;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_magnus(pxa_ctx* c, int steps_per_magnus) {
  if (!c) return PXA_ERR_INVALID;
  if (steps_per_magnus < 1 || (c->have_time && (c->K / c->P) % steps_per_magnus != 0))
    return fail(c, PXA_ERR_INVALID, "steps_per_magnus must divide the steps of one subinterval");
  c->magnus_M = steps_per_magnus;
  invalidate(c);
  return PXA_OK;
}

int pxa_set_control(pxa_ctx* c, const double* control_dev, double omega) {
  if (!c || !control_dev) return PXA_ERR_INVALID;
  c->control = control_dev;
  c->omega = omega;
  invalidate(c);
  return PXA_OK;
}

int pxa_set_target(pxa_ctx* c, const double* target_dev) {
  if (!c || !target_dev) return PXA_ERR_INVALID;
  c->target = target_dev;
  invalidate(c);
  return PXA_OK;
}

int pxa_set_objective(pxa_ctx* c, const pxa_objective_desc* obj) {
  if (!c || !obj) return PXA_ERR_INVALID;
  if (obj->kind != PXA_OBJ_TERMINAL_L2 && obj->kind != PXA_OBJ_INTEGRAL_TRACKING)
    return fail(c, PXA_ERR_INVALID, "objective kind");
  if (!c->have_op) return fail(c, PXA_ERR_STATE, "set_operator first");
  if (!objective_ok(c->op.kind, obj->kind))
    return fail(c, PXA_ERR_INVALID, "this operator supports TERMINAL_L2 (ADVDIFF_1D, CSR) or INTEGRAL_TRACKING "
                                    "(BURGERS_1D, ADVDIFF_2D) only");
  if (obj->kind == PXA_OBJ_INTEGRAL_TRACKING && !obj->target_dev)
    return fail(c, PXA_ERR_INVALID, "INTEGRAL_TRACKING needs a target");
  c->obj_kind = obj->kind;
  c->target = obj->target_dev;
  if (c->inner) {  // the batch of one keeps J = 0.5 ||q(T)||^2: rebuilt at the next solve
    pxa_batch_destroy(c->inner);
    c->inner = nullptr;
  }
  invalidate(c);
  return PXA_OK;
}

int pxa_set_precision(pxa_ctx* c, int prec) {
  if (!c || (prec != PXA_F64 && prec != PXA_F32)) return PXA_ERR_INVALID;
  if (!c->have_op) return fail(c, PXA_ERR_STATE, "set_operator first");
  const int kind = c->op.kind;
  if ((kind == PXA_ADVDIFF_2D || kind == PXA_BURGERS_2D) && prec != PXA_F32)
    return fail(c, PXA_ERR_INVALID, "the 2D problems step in FP32 only");
  if ((kind == PXA_BURGERS_1D || kind == PXA_CSR) && prec != PXA_F64)
    return fail(c, PXA_ERR_INVALID, "BURGERS_1D and CSR step in FP64 only");
  if (kind == PXA_ADVDIFF_1D && prec == PXA_F32 && (c->op.n < 16 || c->op.n > 4096))
    return fail(c, PXA_ERR_INVALID, "FP32 stepping of ADVDIFF_1D needs 16 <= n <= 4096");
  c->step_prec = prec;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_memory(pxa_ctx* c, int policy) {
  if (!c || (policy != PXA_STORE_FULL && policy != PXA_STORE_CHECKPOINTS)) return PXA_ERR_INVALID;
  c->memory = policy;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_lane_steps(pxa_ctx* c, int q) {
  if (!c || (q != 0 && q != 1 && q != 2 && q != 4)) return PXA_ERR_INVALID;
  c->lane_q_req = q;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_checkpoints(pxa_ctx* c, int intervals) {
  if (!c || intervals < 0 || intervals > 65536) return PXA_ERR_INVALID;
  c->intervals = intervals >= 2 ? intervals : 0;
  c->stats.checkpoint_intervals = c->intervals;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_adjoint(pxa_ctx* c, int impl) {
  if (!c || (impl != PXA_ADJ_BANDED && impl != PXA_ADJ_RESTEP && impl != PXA_ADJ_BANDED_SINGLE &&
             impl != PXA_ADJ_BANDED_PAIR))
    return PXA_ERR_INVALID;
  c->band_req = impl == PXA_ADJ_RESTEP ? 0 : 1;
  c->chain_len = impl == PXA_ADJ_BANDED ? 4 : impl == PXA_ADJ_BANDED_PAIR ? 2 : 1;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_groups(pxa_ctx* c, int q_direct, int q_sweep) {
  if (!c) return PXA_ERR_INVALID;
  for (int q : {q_direct, q_sweep})
    if (q != 0 && q != 1 && q != 2 && q != 4) return fail(c, PXA_ERR_INVALID, "group sizes are 0, 1, 2 or 4");
  c->q_direct = q_direct;
  c->q_sweep = q_sweep;
  c->stats.group_direct = q_direct;
  c->stats.group_sweep = q_sweep;
  invalidate(c);
  return PXA_OK;
}

int pxa_set_overlap(pxa_ctx* c, int enable) {
  if (!c) return PXA_ERR_INVALID;
  c->overlap = enable != 0;
  invalidate(c);
  return PXA_OK;
}

int pxa_partition_bounds(int64_t K, int P, double r, int max_chunks, int64_t* bounds) {
  if (K < 1 || P < 1 || K % P != 0 || !(r >= 0.0 && r < 1.0) || max_chunks < 1 || max_chunks > 64 ||
      !bounds)
    return PXA_ERR_INVALID;
  return bu1_chunk_bounds(K, P, r, max_chunks, bounds);
}

int pxa_set_propagator(pxa_ctx* c, int method, int max_degree) {
  if (!c || (method != PXA_PROP_KRYLOV && method != PXA_PROP_RELPM && method != PXA_PROP_BAND &&
             method != PXA_PROP_POLY) ||
      max_degree < 2 || max_degree > 200)
    return PXA_ERR_INVALID;
  c->prop = method;
  c->relpm_mmax = max_degree;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_partition(pxa_ctx* c, double r) {
  if (!c) return PXA_ERR_INVALID;
  if (!(r >= 0.0 && r < 1.0)) return fail(c, PXA_ERR_INVALID, "partition ratio must be 0 (equal) or in (0, 1)");
  c->part_r = r;
  c->stats.partition_r = (float)r;
  invalidate(c);
  return PXA_OK;
}

int pxa_set_cluster(pxa_ctx* c, int direct, int lanes, int chain) {
  if (!c) return PXA_ERR_INVALID;
  for (int C : {direct, lanes, chain})
    if (C < 0 || C > 16) return fail(c, PXA_ERR_INVALID, "cluster sizes must be 0 (auto) or 1..16");
  c->cl_req_direct = direct;
  c->cl_req_lanes = lanes;
  c->cl_req_chain = chain;
  release_workspace(c);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_graph(pxa_ctx* c, int enable) {
  if (!c) return PXA_ERR_INVALID;
  c->use_graph = enable != 0;
  if (c->inner) pxa_batch_set_graph(c->inner, enable != 0);
  invalidate(c);
  return PXA_OK;
}

int pxa_set_timing(pxa_ctx* c, int enable) {
  if (!c) return PXA_ERR_INVALID;
  if (enable && !c->ev_ready) {
    PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
    if (int rc = ensure_timing_events(c)) return rc;
  }
  c->timing = enable != 0;
  invalidate(c);
  return PXA_OK;
}

// ADVDIFF_1D with FP32 stepping runs as a batch of one problem (FP32 lanes, FP64
// superposition and Krylov), built at the first solve after a set_* call.
static bool f32_path(const pxa_ctx* c) { return c->op.kind == PXA_ADVDIFF_1D && c->step_prec == PXA_F32; }

static int f32_ready(pxa_ctx* c) {
  if (c->inner) return PXA_OK;
  if (c->target) return fail(c, PXA_ERR_INVALID, "FP32 stepping of ADVDIFF_1D has J = 0.5 ||q(T)||^2 (no target)");
  pxa_batch* b = nullptr;
  int rc = pxa_batch_create(&b, c->device, c->stream);
  if (rc) return fail(c, rc, "FP32 stepping: batch context");
  c->inner = b;
  const int n = c->op.n;
  const double nu = c->op.nu;
  rc = pxa_batch_set(b, 1, &n, &nu, c->op.c, c->op.L, c->T, c->K, c->P);
  if (!rc) rc = pxa_batch_set_krylov(b, c->kry_m, c->kry_tol, 0.04);
  // the stepper's own propagator as one FP32 band per link, or FP64 Krylov exp(tau A)
  if (!rc) rc = pxa_batch_set_homogeneous(b, c->kry_phi == PXA_PHI_EXP ? 1e30 : 0.0);
  if (!rc) rc = pxa_batch_set_power(b, 1);
  if (!rc) rc = pxa_batch_set_graph(b, c->use_graph ? 1 : 0);
  if (!rc && c->lane_q_req) rc = pxa_batch_set_lane_steps(b, c->lane_q_req);
  if (rc) return fail(c, rc, std::string("FP32 stepping: ") + pxa_batch_last_error(b));
  return PXA_OK;
}

static int f32_sync(pxa_ctx* c) {
  if (!c->inner) return PXA_OK;
  const int rc = pxa_batch_sync(c->inner);
  if (rc) return fail(c, rc, std::string("FP32 stepping: ") + pxa_batch_last_error(c->inner));
  return PXA_OK;
}

int pxa_gradient_async(pxa_ctx* c, int mode, double* J_dev, double* grad_dev) {
  if (!c || !grad_dev) return PXA_ERR_INVALID;
  int rc = prepare(c);
  if (rc) return rc;
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  double* Jd = J_dev ? J_dev : c->Jdev;
  if (f32_path(c)) {
    if (mode != PXA_SERIAL && mode != PXA_PARAEXP) return fail(c, PXA_ERR_INVALID, "mode");
    if (!c->control) return fail(c, PXA_ERR_STATE, "set_control first");
    if ((rc = f32_ready(c))) return rc;
    rc = pxa_batch_gradient(c->inner, mode, c->control, Jd, grad_dev);
    if (rc) return fail(c, rc, std::string("FP32 stepping: ") + pxa_batch_last_error(c->inner));
    c->stats.lanes = mode == PXA_SERIAL ? 1 : c->P;
    return PXA_OK;
  }
  c->prep_marked = false;
  c->side_marked = 0;
  for (bool& b : c->side_lanes_marked) b = false;
  c->stats.lanes = mode == PXA_SERIAL ? 1 : c->P;
  c->stats.krylov_m = c->kry_m;
  c->stats.krylov_substeps = c->kry_sub;
  c->stats.magnus_steps = c->magnus_M;
  if (c->use_graph) {
    // (with timing on, the phase events are captured as event-record nodes of the graph)
    if (!c->gexec || c->g_mode != mode || c->g_grad != grad_dev || c->g_J != Jd) {
      invalidate(c);
      // Capture on a library-owned stream (the caller's may be the legacy default
      // stream, which cannot be captured); the graph is then launched on the caller's.
      if (!c->cap_stream)
        PXA_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
      cudaGraph_t graph;
      cudaStream_t user = c->stream;
      c->stream = c->cap_stream;
      cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) {
        c->stream = user;
        return cuda_fail(c, e, "begin capture");
      }
      int erc = enqueue(c, mode, Jd, grad_dev);
      e = cudaStreamEndCapture(c->stream, &graph);
      c->stream = user;
      if (erc) {
        if (e == cudaSuccess) cudaGraphDestroy(graph);
        return erc;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
      c->stats.graph_kernels = graph_kernel_nodes(graph);
      // kernel nodes keep their own priorities (the direct above the overlapped side work)
      e = cudaGraphInstantiateWithFlags(&c->gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
      c->g_mode = mode;
      c->g_grad = grad_dev;
      c->g_J = Jd;
      c->g_prep_marked = c->prep_marked;
      c->g_side_marked = c->side_marked;
      for (int i = 0; i < pxa_ctx::kMaxChunks; ++i) c->g_side_lanes_marked[i] = c->side_lanes_marked[i];
    }
    c->prep_marked = c->g_prep_marked;
    c->side_marked = c->g_side_marked;
    for (int i = 0; i < pxa_ctx::kMaxChunks; ++i) c->side_lanes_marked[i] = c->g_side_lanes_marked[i];
    PXA_CUDA(c, cudaGraphLaunch(c->gexec, c->stream), "graph launch");
    return PXA_OK;
  }
  return enqueue(c, mode, Jd, grad_dev);
}

static void collect_timing(pxa_ctx* c);

int pxa_sync(pxa_ctx* c) {
  if (!c) return PXA_ERR_INVALID;
  if (!c->ready) return PXA_OK;
  if (f32_path(c)) {
    int rc = f32_sync(c);
    if (rc) return rc;
  }
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  collect_timing(c);
  return read_status(c);
}

int pxa_gradient(pxa_ctx* c, int mode, double* J_host, double* grad_dev) {
  if (!c || !grad_dev) return PXA_ERR_INVALID;
  int rc = pxa_gradient_async(c, mode, nullptr, grad_dev);
  if (rc) return rc;
  if (f32_path(c) && (rc = f32_sync(c))) return rc;
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  double J = 0.0;
  PXA_CUDA(c, cudaMemcpy(&J, c->Jdev, sizeof(double), cudaMemcpyDeviceToHost), "read J");
  c->stats.J = J;
  if (J_host) *J_host = J;
  collect_timing(c);
  return read_status(c);
}

// Phase times of the last gradient from its CUDA events (timing on; stream synchronised).
static void collect_timing(pxa_ctx* c) {
  if (c->timing && c->ev_ready) {
    float a = 0, b = 0, d = 0, e = 0, t = 0;
    bool ok = true;
    auto el = [&](float* ms, int i, int j) {
      if (cudaEventElapsedTime(ms, c->ev[i], c->ev[j]) != cudaSuccess) {
        cudaGetLastError();  // not left for the caller's next call
        ok = false;
      }
    };
    el(&a, 0, 1);
    el(&b, 1, 2);
    float pr = 0;
    if (c->prep_marked) {
      el(&pr, 2, 6);
      el(&d, 6, 3);
    } else {
      el(&d, 2, 3);
    }
    el(&e, 3, 4);
    el(&t, 0, 5);
    if (!ok) a = b = pr = d = e = t = -1.f;  // phase times unavailable
    c->stats.ms_direct_inhom = a;
    c->stats.ms_direct_hom = b;
    c->stats.ms_adjoint_prep = pr;
    c->stats.ms_adjoint_inhom = d;
    c->stats.ms_adjoint_hom = e;
    c->stats.ms_total = t;
    // kernel time of the overlapped side-stream work, summed over the chunks
    float pre = 0.f, pair = 0.f, quad = 0.f, lanes = 0.f;
    bool sok = ok;
    for (int ci = 0; ci < c->side_marked && sok; ++ci) {
      float x = 0.f;
      auto side_el = [&](float* acc, cudaEvent_t a, cudaEvent_t b) {
        if (cudaEventElapsedTime(&x, a, b) != cudaSuccess) {
          cudaGetLastError();
          sok = false;
        } else {
          *acc += x;
        }
      };
      side_el(&pre, c->ev_side[ci][0], c->ev_side[ci][1]);
      side_el(&pair, c->ev_side[ci][1], c->ev_side[ci][2]);
      side_el(&quad, c->ev_side[ci][2], c->ev_side[ci][3]);
      if (c->side_lanes_marked[ci]) side_el(&lanes, c->ev_side[ci][4], c->ev_side[ci][5]);
    }
    if (!sok) pre = pair = quad = lanes = -1.f;
    c->stats.side_chunks = c->side_marked;
    c->stats.ms_side_prepass = c->side_marked ? pre : 0.f;
    c->stats.ms_side_pair = c->side_marked ? pair : 0.f;
    c->stats.ms_side_quad = c->side_marked ? quad : 0.f;
    c->stats.ms_side_lanes = c->side_marked ? lanes : 0.f;
  }
}

int pxa_solve_direct(pxa_ctx* c, int mode, double* J_host) {
  if (!c) return PXA_ERR_INVALID;
  if (f32_path(c)) return fail(c, PXA_ERR_INVALID, "FP32 stepping runs whole gradients (pxa_gradient)");
  int rc = prepare(c);
  if (rc) return rc;
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  rc = enqueue_parts(c, mode, 1, c->Jdev, nullptr);
  if (rc) return rc;
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  double J = 0.0;
  PXA_CUDA(c, cudaMemcpy(&J, c->Jdev, sizeof(double), cudaMemcpyDeviceToHost), "read J");
  c->stats.J = J;
  if (J_host) *J_host = J;
  rc = read_status(c);
  c->direct_mode = rc == PXA_OK ? mode : -1;
  return rc;
}

int pxa_solve_adjoint(pxa_ctx* c, int mode, double* grad_dev) {
  if (!c || !grad_dev) return PXA_ERR_INVALID;
  if (f32_path(c)) return fail(c, PXA_ERR_INVALID, "FP32 stepping runs whole gradients (pxa_gradient)");
  if (!c->ready || c->direct_mode != mode)
    return fail(c, PXA_ERR_STATE, "pxa_solve_adjoint needs a pxa_solve_direct of the same mode first");
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  int rc = enqueue_parts(c, mode, 2, c->Jdev, grad_dev);
  if (rc) return rc;
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  return read_status(c);
}

int pxa_gradient_host(pxa_ctx* c, int mode, const double* control_host, double* J_host,
                      double* grad_host) {
  if (!c || !control_host || !grad_host) return PXA_ERR_INVALID;
  int rc = prepare(c);
  if (rc) return rc;
  const int n = c->op.n;
  const double* saved = c->control;
  PXA_CUDA(c, cudaMemcpyAsync(c->ctl_buf, control_host, sizeof(double) * n, cudaMemcpyHostToDevice,
                              c->stream), "H2D control");
  if (saved != c->ctl_buf) {
    c->control = c->ctl_buf;
    invalidate(c);
  }
  rc = pxa_gradient(c, mode, J_host, c->grad_buf);
  if (rc) return rc;
  PXA_CUDA(c, cudaMemcpyAsync(grad_host, c->grad_buf, sizeof(double) * n, cudaMemcpyDeviceToHost,
                              c->stream), "D2H grad");
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  return PXA_OK;
}

// One configuration's time per gradient for the autotuner: a warm-up call (which also
// captures the graph when graphs are on), then the best of two timed calls through the
// same entry point the caller uses (graph replay or direct launches). Returns PXA_OK and
// *ms, or the error of the warm-up / timed calls.
static int tune_time(pxa_ctx* c, int mode, double* grad_dev, cudaEvent_t e0, cudaEvent_t e1, double* ms) {
  invalidate(c);
  int rc = pxa_gradient_async(c, mode, c->Jdev, grad_dev);
  if (rc == PXA_OK) rc = pxa_sync(c);
  if (rc) return rc;
  double best = 1e300;
  for (int rep = 0; rep < 2; ++rep) {
    PXA_CUDA(c, cudaEventRecord(e0, c->stream), "record");
    rc = pxa_gradient_async(c, mode, c->Jdev, grad_dev);
    PXA_CUDA(c, cudaEventRecord(e1, c->stream), "record");
    PXA_CUDA(c, cudaEventSynchronize(e1), "sync");
    if (rc == PXA_OK) rc = read_status(c);
    if (rc) return rc;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (t < best) best = t;
  }
  *ms = best;
  return PXA_OK;
}

int pxa_autotune(pxa_ctx* c, int mode, double* grad_dev, double* best_ms_host) {
  if (!c || !grad_dev) return PXA_ERR_INVALID;
  if (!c->have_op || !c->have_time || !c->control) return fail(c, PXA_ERR_STATE, "configure the problem first");
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (f32_path(c)) {  // the batch of one has its own autotuner
    int rc = prepare(c);
    if (!rc) rc = f32_ready(c);
    if (!rc) rc = pxa_batch_autotune(c->inner, mode, c->control, c->Jdev, grad_dev, best_ms_host);
    if (rc) return fail(c, rc, std::string("FP32 stepping: ") + pxa_batch_last_error(c->inner));
    return PXA_OK;
  }
  const bool timing = c->timing;
  c->timing = false;  // candidates are timed through the caller's path (graph replay when on)
  cudaEvent_t e0, e1;
  PXA_CUDA(c, cudaEventCreate(&e0), "event");
  PXA_CUDA(c, cudaEventCreate(&e1), "event");
  struct Cand { int a, b, cc; };
  std::vector<Cand> cands;
  const int64_t k = c->K / c->P;
  if (c->op.kind == PXA_ADVDIFF_1D) {
    for (int m : {16, 20, 24, 30, 36, 40})
      for (int sub : {1, 2, 4, 8})
        if (k % sub == 0 && m < c->op.n) cands.push_back({m, sub, 0});
  } else {
    int sms = 0;
    PXA_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device), "SM count");
    auto ok = [&](int C) {
      return bu1c_valid_cluster(c->op.n, C) && bu1_rk4_valid_cluster(c->op.n, C) &&
             (C == 1 || c->op.n / C >= 24);
    };
    for (int cd : {1, 2, 4, 8, 12, 16})
      for (int cl : {1, 2, 3, 4})
        if (ok(cd) && ok(cl) && cl * c->P <= (sms > 0 ? sms : 152)) cands.push_back({cd, cl, cd});
  }
  const int m0 = c->kry_m, s0 = c->kry_sub, rd = c->cl_req_direct, rl = c->cl_req_lanes, rc0 = c->cl_req_chain;
  double best = 1e300;
  Cand bestc{-1, -1, -1};
  for (const Cand& cd : cands) {
    if (c->op.kind == PXA_ADVDIFF_1D) {
      c->kry_m = cd.a;
      c->kry_sub = cd.b;
    } else {
      c->cl_req_direct = cd.a;
      c->cl_req_lanes = cd.b;
      c->cl_req_chain = cd.cc;
    }
    release_workspace(c);
    invalidate(c);
    if (prepare(c)) continue;
    double ms = 0.0;
    const int rc = tune_time(c, mode, grad_dev, e0, e1, &ms);
    if (rc) {
      // a candidate that does not converge or cannot be launched is skipped; a device
      // fault would be sticky and is reported
      const cudaError_t ce = cudaGetLastError();
      if (rc == PXA_ERR_CUDA && ce != cudaSuccess && ce != cudaErrorInvalidValue &&
          ce != cudaErrorInvalidConfiguration)
        break;
      continue;
    }
    if (ms < best) {
      best = ms;
      bestc = cd;
    }
  }
  c->timing = timing;
  if (bestc.a < 0) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->kry_m = m0;
    c->kry_sub = s0;
    c->cl_req_direct = rd;
    c->cl_req_lanes = rl;
    c->cl_req_chain = rc0;
    release_workspace(c);
    invalidate(c);
    return fail(c, PXA_ERR_NOT_CONVERGED, "no autotuner candidate met the Krylov tolerance");
  }
  if (c->op.kind == PXA_ADVDIFF_1D) {
    c->kry_m = bestc.a;
    c->kry_sub = bestc.b;
  } else {
    c->cl_req_direct = bestc.a;
    c->cl_req_lanes = bestc.b;
    c->cl_req_chain = bestc.cc;
  }
  release_workspace(c);
  invalidate(c);
  int rc = prepare(c);
  if (rc) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
  }
  if (c->op.kind == PXA_BURGERS_1D && c->band) {
    c->timing = false;
    // second pass at the chosen cluster sizes: steps per halo exchange of the direct
    // sweep and of the banded sweeps (no reallocation needed)
    int bqd = c->q_direct, bqs = c->q_sweep;
    for (int qd : {1, 2, 4})
      for (int qs : {1, 2, 4}) {
        c->q_direct = qd;
        c->q_sweep = qs;
        double ms = 0.0;
        if (tune_time(c, mode, grad_dev, e0, e1, &ms) != PXA_OK) continue;
        if (ms < best) {
          best = ms;
          bqd = qd;
          bqs = qs;
        }
      }
    c->q_direct = bqd;
    c->q_sweep = bqs;
    if (c->overlap && c->memory == PXA_STORE_FULL && c->side && c->intervals < 2) {
      // third pass: the chunk partition of the overlapped direct solve (Sec. 3.3).
      // k = tau_I_adj / tau_I comes from one run with the phases in sequence (direct;
      // band records and adjoint lanes); then equal chunks, r = k/(k+1) and r = k are
      // timed and the fastest is kept.
      if (int erc = ensure_timing_events(c)) return erc;
      const bool graph3 = c->use_graph;
      c->use_graph = false;
      c->overlap = false;
      c->timing = true;
      invalidate(c);
      double kr = 0.0;
      int mrc = enqueue(c, mode, c->Jdev, grad_dev);
      if (mrc == PXA_OK) mrc = enqueue(c, mode, c->Jdev, grad_dev);
      if (mrc == PXA_OK) {
        PXA_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
        float md = 0.f, ma = 0.f;
        cudaEventElapsedTime(&md, c->ev[0], c->ev[1]);
        cudaEventElapsedTime(&ma, c->ev[2], c->ev[3]);
        if (md > 0.f && read_status(c) == PXA_OK) kr = (double)ma / (double)md;
      }
      c->overlap = true;
      c->timing = false;
      c->use_graph = graph3;
      c->stats.tau_ratio = (float)kr;
      // besides the two ratios of the model, a few fixed ones: the adjoint work of a
      // chunk is not proportional to its length (the lanes take their subinterval's
      // length whatever the chunk), so the measured optimum can lie between
      std::vector<double> rs = {0.0};
      if (kr > 0.0) {
        rs.push_back(kr / (kr + 1.0));
        if (kr < 0.95) rs.push_back(kr);
      }
      for (double r : {0.6, 0.7, 0.8, 0.9}) {
        bool seen = false;
        for (double q : rs) seen = seen || std::fabs(q - r) < 0.02;
        if (!seen) rs.push_back(r);
      }
      double bms = 1e300, br = c->part_r;
      for (double r : rs) {
        c->part_r = r;
        double ms = 0.0;
        if (tune_time(c, mode, grad_dev, e0, e1, &ms) != PXA_OK) continue;
        if (ms < bms) {
          bms = ms;
          br = r;
        }
      }
      c->part_r = br;
      c->stats.partition_r = (float)br;
      if (bms < 1e299) best = bms;
    }
    c->timing = timing;
    invalidate(c);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->stats.krylov_m = c->kry_m;
  c->stats.krylov_substeps = c->kry_sub;
  c->stats.group_direct = c->q_direct;
  c->stats.group_sweep = c->q_sweep;
  if (best_ms_host) *best_ms_host = best;
  return PXA_OK;
}

int pxa_nl_paraexp(pxa_ctx* c, const double* guess_dev, double tol, int max_iter, double* traj_dev,
                   double* changes_host, int* iters_host) {
  if (!c || !traj_dev || max_iter < 1 || !(tol > 0.0)) return PXA_ERR_INVALID;
  if (!c->have_op || !c->have_time || c->op.kind != PXA_BURGERS_1D)
    return fail(c, PXA_ERR_STATE, "pxa_nl_paraexp needs a BURGERS_1D operator and set_time");
  if (c->op.n > 1024) return fail(c, PXA_ERR_INVALID, "pxa_nl_paraexp: n <= 1024 (one thread per grid point)");
  if (!c->control) return fail(c, PXA_ERR_STATE, "set_control (the forcing) first");
  int rc = prepare(c);
  if (rc) return rc;
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  const int n = c->op.n, P = c->P;
  const int64_t K = c->K;
  const double dt = c->T / (double)K;
  const size_t rows = (size_t)(K + 1) * n;
  if (!c->nl_Q) {
    if ((rc = alloc(c, &c->nl_Q, rows))) return rc;
    if ((rc = alloc(c, &c->nl_Qn, rows))) return rc;
    if ((rc = alloc(c, &c->nl_V, rows))) return rc;
    if ((rc = alloc(c, &c->nl_qbar, (size_t)P * n))) return rc;
    if ((rc = alloc(c, &c->nl_change, 3))) return rc;
    c->stats.workspace_bytes = c->ws_bytes;
  }
  cudaStream_t st = c->stream;
  const double* sc = nullptr;
  if (c->omega != 0.0) {
    PXA_CUDA(c, launch_bu1_forcing_table(st, K, dt, c->omega, c->sc), "forcing table");
    sc = c->sc;
  }
  // Alg. 2: the initial guess of the direct solution (q(t) = q0 = 0 when none is given)
  if (guess_dev)
    PXA_CUDA(c, cudaMemcpyAsync(c->nl_Q, guess_dev, sizeof(double) * rows, cudaMemcpyDeviceToDevice, st), "guess");
  else
    PXA_CUDA(c, cudaMemsetAsync(c->nl_Q, 0, sizeof(double) * rows, st), "guess");
  PXA_CUDA(c, cudaMemsetAsync(c->nl_V, 0, sizeof(double) * (size_t)n, st), "lane rows");
  double* Q = c->nl_Q;
  double* Qn = c->nl_Qn;
  int result = PXA_ERR_NOT_CONVERGED, it = 0;
  for (; it < max_iter;) {
    PXA_CUDA(c, launch_nl_iteration(st, n, K, P, c->op.L, c->op.nu, dt, c->control, sc, Q, Qn, c->nl_V, c->nl_qbar,
                                    c->nl_change), "iteration");
    double ch[3] = {0.0, 0.0, 0.0};
    PXA_CUDA(c, cudaMemcpyAsync(ch, c->nl_change, sizeof(ch), cudaMemcpyDeviceToHost, st), "read change");
    PXA_CUDA(c, cudaStreamSynchronize(st), "stream sync");
    std::swap(Q, Qn);  // q_i <- q_{i+1}
    ++it;
    const double err = ch[2] != 0.0 ? NAN : (ch[1] > 0.0 ? std::sqrt(ch[0] / ch[1]) : std::sqrt(ch[0]));
    if (changes_host) changes_host[it - 1] = err;
    if (!std::isfinite(err)) {
      result = PXA_ERR_NONFINITE;
      break;
    }
    if (err <= tol) {
      result = PXA_OK;
      break;
    }
  }
  if (iters_host) *iters_host = it;
  PXA_CUDA(c, cudaMemcpyAsync(traj_dev, Q, sizeof(double) * rows, cudaMemcpyDeviceToDevice, st), "trajectory");
  PXA_CUDA(c, cudaStreamSynchronize(st), "stream sync");
  if (result == PXA_ERR_NONFINITE) return fail(c, result, "the iteration diverged to non-finite values");
  if (result == PXA_ERR_NOT_CONVERGED)
    return fail(c, result, "the iteration's change stayed above the tolerance for max_iter iterations");
  return PXA_OK;
}

int pxa_direct_state(pxa_ctx* c, const double* ic_dev, double* state_dev) {
  if (!c || !ic_dev || !state_dev) return PXA_ERR_INVALID;
  if (!c->have_op || !c->have_time || c->op.kind != PXA_BURGERS_2D)
    return fail(c, PXA_ERR_STATE, "pxa_direct_state needs a BURGERS_2D operator and set_time");
  int rc = prepare(c);
  if (rc) return rc;
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  cudaStream_t st = c->stream;
  const int n = c->op.nx;
  const size_t plane2 = 2 * (size_t)n * n;
  const double dt = c->T / (double)c->K;
  float* tr = c->b2traj;
  PXA_CUDA(c, launch_bu2_convert(st, ic_dev, tr, plane2), "initial state");
  for (int64_t s = 0; s < c->K; ++s)
    PXA_CUDA(c, launch_bu2_step(st, tr + (size_t)s * plane2, tr + (size_t)(s + 1) * plane2, n, c->op.L, c->op.nu, dt),
             "direct step");
  PXA_CUDA(c, launch_bu2_convert_back(st, tr + (size_t)c->K * plane2, state_dev, plane2, c->status), "final state");
  invalidate(c);  // the stored trajectory no longer belongs to a solve of the control
  return pxa_sync(c);
}

int pxa_set_wait_limit(pxa_ctx* c, int64_t cycles) {
  if (!c || cycles < 0 || (cycles > 0 && (cycles < 1024 || cycles > ((int64_t)INT32_MAX << 10))))
    return PXA_ERR_INVALID;
  c->wait_limit_units = (int)(cycles >> 10);
  if (c->ready) {
    PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
    PXA_CUDA(c, cudaMemcpy(c->status + 1, &c->wait_limit_units, sizeof(int), cudaMemcpyHostToDevice),
             "wait limit");
  }
  return PXA_OK;
}

int pxa_wait_probe(pxa_ctx* c) {
  if (!c) return PXA_ERR_INVALID;
  int rc = prepare(c);
  if (rc) return rc;
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  PXA_CUDA(c, launch_wait_probe(c->stream, c->status), "wait probe");
  return pxa_sync(c);
}

int pxa_get_stats(const pxa_ctx* c, pxa_stats* out) {
  if (!c || !out) return PXA_ERR_INVALID;
  *out = c->stats;
  return PXA_OK;
}

// ---- building blocks ----------------------------------------------------------
int pxa_apply_operator(pxa_ctx* c, int transpose, const double* x_dev, double* y_dev) {
  if (!c || !x_dev || !y_dev) return PXA_ERR_INVALID;
  if (!c->have_op || c->op.kind != PXA_ADVDIFF_1D) return fail(c, PXA_ERR_STATE, "ADVDIFF_1D operator required");
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  PXA_CUDA(c, launch_ad1_apply(c->stream, c->op.n, c->am, c->a0, c->ap, transpose, x_dev, y_dev), "apply");
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
  return PXA_OK;
}

int pxa_step(pxa_ctx* c, int transpose, int64_t steps, const double* x_dev, double* y_dev) {
  if (!c || !x_dev || !y_dev || steps < 0) return PXA_ERR_INVALID;
  if (!c->have_op || c->op.kind != PXA_ADVDIFF_1D) return fail(c, PXA_ERR_STATE, "ADVDIFF_1D operator required");
  if (c->op.n > 4096) return fail(c, PXA_ERR_INVALID, "pxa_step needs n <= 4096 (one block holds the lane)");
  int rc = prepare(c);
  if (rc) return rc;
  const int n = c->op.n;
  PXA_CUDA(c, launch_cn_lanes(c->stream, 1, threads_for(n), n, c->band_r, c->taps, transpose, steps,
                              x_dev, nullptr, y_dev), "step");
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
  return PXA_OK;
}

int pxa_expv(pxa_ctx* c, int transpose, int64_t span_steps, int substeps, const double* x_dev,
             double* y_dev, double* err_host) {
  if (!c || !x_dev || !y_dev || span_steps < 1 || substeps < 1 || span_steps % substeps != 0)
    return PXA_ERR_INVALID;
  if (!c->have_op || c->op.kind != PXA_ADVDIFF_1D) return fail(c, PXA_ERR_STATE, "ADVDIFF_1D operator required");
  if (c->op.n > 4096) return fail(c, PXA_ERR_INVALID, "pxa_expv needs n <= 4096 (one block holds the vectors)");
  int rc = prepare(c);
  if (rc) return rc;
  const int n = c->op.n;
  const double dt = c->T / (double)c->K;
  const int64_t sps = span_steps / substeps;
  const double hscale = c->kry_phi == PXA_PHI_EXP ? dt * (double)sps : dt;
  PXA_CUDA(c, cudaMemsetAsync(c->errmax, 0, sizeof(double), c->stream), "reset errmax");
  if (c->prop == PXA_PROP_BAND) {
    // the propagator of the whole span as one circulant band (substeps not used)
    std::vector<double> bt;
    int br = 0;
    cn_power_taps(n, c->am, c->a0, c->ap, dt, span_steps, 50, bt, br, c->kry_phi == PXA_PHI_EXP);
    double* bd = nullptr;
    PXA_CUDA(c, cudaMalloc(&bd, sizeof(double) * bt.size()), "alloc");
    cudaError_t e = cudaMemcpy(bd, bt.data(), sizeof(double) * bt.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_ad1_band_chain(c->stream, n, br, bd, transpose, x_dev, 0, 0, 1, y_dev);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(bd);
    PXA_CUDA(c, e, "band expv");
  } else if (c->prop == PXA_PROP_RELPM) {
    // ReLPM picks its own substeps for the whole span
    std::vector<double> z, D;
    int ns = 1;
    double ts = 0.0;
    const bool stepper = c->kry_phi == PXA_PHI_STEPPER;
    relpm_setup_host(dt * (double)span_steps, c->am, c->a0, c->ap, c->relpm_mmax, ns, ts, z, D,
                     stepper ? span_steps : 0);
    double *Dd = nullptr, *zd = nullptr;
    PXA_CUDA(c, cudaMalloc(&Dd, sizeof(double) * D.size()), "alloc");
    PXA_CUDA(c, cudaMalloc(&zd, sizeof(double) * z.size()), "alloc");
    cudaMemcpy(Dd, D.data(), sizeof(double) * D.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(zd, z.data(), sizeof(double) * z.size(), cudaMemcpyHostToDevice);
    cudaError_t e = launch_ad1_relpm_expv(c->stream, 256, n, c->am, c->a0, c->ap, transpose, x_dev, y_dev, Dd, zd,
                                          c->relpm_mmax, ts, ns, stepper ? 1 : 0, c->kry_tol, c->status,
                                          c->errmax);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(Dd);
    cudaFree(zd);
    PXA_CUDA(c, e, "relpm expv");
  } else {
    PXA_CUDA(c, launch_ad1_expv(c->stream, 256, n, c->am, c->a0, c->ap, transpose, x_dev, y_dev, c->V,
                                c->kry_m, c->kry_phi, hscale, sps, substeps, c->kry_tol, c->v_in_smem,
                                c->status, c->errmax), "expv");
  }
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
  rc = read_status(c);
  if (err_host) *err_host = c->stats.krylov_err_max;
  return rc;
}

int pxa_cn_lanes_1d(pxa_ctx* c, int lanes, int64_t steps, double* out_dev, double* ms_host) {
  if (!c || lanes < 1 || steps < 1) return PXA_ERR_INVALID;
  if (!c->have_op || c->op.kind != PXA_ADVDIFF_1D) return fail(c, PXA_ERR_STATE, "ADVDIFF_1D operator required");
  if (!c->control) return fail(c, PXA_ERR_STATE, "set_control first (the lanes' initial state)");
  const int n = c->op.n;
  if (n % 4 != 0) return fail(c, PXA_ERR_INVALID, "pxa_cn_lanes_1d needs n % 4 == 0");
  int rc = prepare(c);
  if (rc) return rc;
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  if (!c->taps1d) {
    // FP32 band: the taps above 2^-40 of the centre one, zero-padded for the kernel
    const int r = c->band_r;
    const double cut = std::ldexp(std::fabs(c->band_host[r]), -40);
    int r32 = 0;
    for (int j = 1; j <= r; ++j)
      if (std::fabs(c->band_host[r + j]) >= cut || std::fabs(c->band_host[r - j]) >= cut) r32 = j;
    std::vector<float> t(ad1_stream_padded_taps(r32), 0.f);
    for (int j = -r32; j <= r32; ++j) t[r32 + j] = (float)c->band_host[r + j];
    if ((rc = alloc(c, &c->taps1d, t.size()))) return rc;
    PXA_CUDA(c, cudaMemcpy(c->taps1d, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice), "copy taps");
    c->r1d = r32;
  }
  if (c->lanes1d != lanes) {
    if ((rc = alloc(c, &c->st1d, 2 * (size_t)lanes * n))) return rc;
    c->lanes1d = lanes;
  }
  cudaStream_t st = c->stream;
  float* x = c->st1d;
  float* y = c->st1d + (size_t)lanes * n;
  PXA_CUDA(c, launch_ad1_stream_fill(st, n, lanes, c->control, x), "fill lanes");
  cudaEvent_t e0, e1;
  PXA_CUDA(c, cudaEventCreate(&e0), "event");
  PXA_CUDA(c, cudaEventCreate(&e1), "event");
  PXA_CUDA(c, cudaEventRecord(e0, st), "record");
  for (int64_t s = 0; s < steps; ++s) {
    cudaError_t e = launch_ad1_stream_step(st, lanes, n, c->r1d, c->taps1d, x, y);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(c, e, "1d lane step");
    }
    std::swap(x, y);
  }
  PXA_CUDA(c, cudaEventRecord(e1, st), "record");
  PXA_CUDA(c, cudaEventSynchronize(e1), "sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ms_host) *ms_host = ms;
  if (out_dev) {
    PXA_CUDA(c, launch_ad1_stream_out(st, (size_t)lanes * n, x, out_dev), "lanes out");
    PXA_CUDA(c, cudaStreamSynchronize(st), "sync");
  }
  return read_status(c);
}

int pxa_rk4_lanes_2d(pxa_ctx* c, int lanes, int64_t steps, double* out_dev, double* ms_host) {
  if (!c || lanes < 1 || steps < 1) return PXA_ERR_INVALID;
  if (!c->have_op || c->op.kind != PXA_ADVDIFF_2D) return fail(c, PXA_ERR_STATE, "ADVDIFF_2D operator required");
  if (!c->control || !c->target) return fail(c, PXA_ERR_STATE, "set_control and set_target first");
  int rc = prepare(c);
  if (rc) return rc;
  Ad2Params a = c->p2;
  a.omega = c->omega;
  const size_t plane = (size_t)a.Hp * a.Wp, N = (size_t)a.nx * a.ny;
  if (c->lanesL != lanes) {
    if ((rc = alloc(c, &c->stL, 2 * (size_t)lanes * plane))) return rc;
    if (!ad2_make_map(&c->mapL, c->stL, a, 2 * lanes, 1) ||
        !ad2_make_map_box(&c->mapL4, c->stL, a, 2 * lanes, 64, AD2_ROLL_BR, 1) ||
        !ad2_make_map_box(&c->mapC4, c->coef2, a, 3, 64, AD2_ROLL_BR, 3))
      return fail(c, PXA_ERR_CUDA, "cuTensorMapEncodeTiled failed for the lane states");
    c->lanesL = lanes;
  }
  cudaStream_t st = c->stream;
  PXA_CUDA(c, launch_ad2_pack_coef(st, a, c->op.u_dev, c->op.v_dev, c->control, c->target, c->coef2), "pack");
  PXA_CUDA(c, cudaMemsetAsync(c->stL, 0, sizeof(float) * (size_t)lanes * plane, st), "zero lanes");
  cudaEvent_t e0, e1;
  PXA_CUDA(c, cudaEventCreate(&e0), "event");
  PXA_CUDA(c, cudaEventCreate(&e1), "event");
  const int lpc = lanes >= 16 ? 16 : lanes;
  // lane l takes steps l*steps .. l*steps+steps-1 of one time axis
  const bool roll = ad2_roll_ok(a);
  if (c->scL_count < (int64_t)lanes * steps) {
    if ((rc = alloc(c, &c->scL, 3 * (size_t)lanes * steps))) return rc;
    c->scL_count = (int64_t)lanes * steps;
  }
  PXA_CUDA(c, launch_ad2_forcing_table(st, 0, (int64_t)lanes * steps, a.dtd, a.omega, c->scL), "table");
  PXA_CUDA(c, cudaEventRecord(e0, st), "record");
  for (int64_t s = 0; s < steps; ++s) {
    if (roll) {
      PXA_CUDA(c, launch_ad2_rk4_roll(st, c->mapL4, c->mapC4, a, c->stL, lanes, (int)(s & 1),
                                      c->scL + 3 * s, (int)steps, c->status), "lanes step");
    } else {
      PXA_CUDA(c, launch_ad2_rk4(st, c->mapL, c->mapCoef, a, c->stL, lanes, lanes, lpc, (int)(s & 1),
                                 steps, s, c->scL, nullptr, 0, nullptr, 0, c->status, 0), "lanes step");
    }
  }
  PXA_CUDA(c, cudaEventRecord(e1, st), "record");
  PXA_CUDA(c, cudaEventSynchronize(e1), "sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ms_host) *ms_host = ms;
  if (out_dev) {
    // copy the interiors of the final states (buffer steps & 1) out as FP64
    std::vector<float> tmp(plane);
    std::vector<double> row(N);
    const float* fin = c->stL + (size_t)(steps & 1) * lanes * plane;
    for (int l = 0; l < lanes; ++l) {
      PXA_CUDA(c, cudaMemcpy(tmp.data(), fin + (size_t)l * plane, sizeof(float) * plane, cudaMemcpyDeviceToHost), "copy");
      for (int y = 0; y < a.ny; ++y)
        for (int x = 0; x < a.nx; ++x) row[(size_t)y * a.nx + x] = tmp[(size_t)(y + G2) * a.Wp + x + G2];
      PXA_CUDA(c, cudaMemcpy(out_dev + (size_t)l * N, row.data(), sizeof(double) * N, cudaMemcpyHostToDevice), "copy");
    }
  }
  return read_status(c);
}

int pxa_burgers_rhs(pxa_ctx* c, const double* u_dev, double* y_dev) {
  if (!c || !u_dev || !y_dev) return PXA_ERR_INVALID;
  if (!c->have_op || c->op.kind != PXA_BURGERS_1D) return fail(c, PXA_ERR_STATE, "BURGERS_1D operator required");
  const int n = c->op.n;
  const double h = c->op.L / n;
  Bu1Grid g{n, 1.0 / (2.0 * h), 1.0 / (h * h), c->op.nu};
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  PXA_CUDA(c, launch_bu1_rhs(c->stream, g, u_dev, y_dev), "rhs");
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
  return PXA_OK;
}

int pxa_burgers_jac_T(pxa_ctx* c, const double* u_dev, const double* x_dev, double* y_dev) {
  if (!c || !u_dev || !x_dev || !y_dev) return PXA_ERR_INVALID;
  if (!c->have_op || c->op.kind != PXA_BURGERS_1D) return fail(c, PXA_ERR_STATE, "BURGERS_1D operator required");
  const int n = c->op.n;
  const double h = c->op.L / n;
  Bu1Grid g{n, 1.0 / (2.0 * h), 1.0 / (h * h), c->op.nu};
  PXA_CUDA(c, cudaSetDevice(c->device), "cudaSetDevice");
  PXA_CUDA(c, launch_bu1_jacT(c->stream, g, u_dev, x_dev, y_dev), "jacT");
  PXA_CUDA(c, cudaStreamSynchronize(c->stream), "sync");
  return PXA_OK;
}

}  // extern "C"
