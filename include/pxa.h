/*
 * pxa.h — C ABI of libpxa, Paraexp direct-adjoint gradients on one GB300 (sm_103a).
 *
 * Method: Skene, Eggl & Schmid, "A parallel-in-time approach for accelerating
 * direct-adjoint studies" (arXiv 2004.00546). The time window [0, T] is split into
 * P subintervals (Alg. 1, equal partition T_p = p T / P). The zero-initial-value
 * inhomogeneous subproblems of every subinterval (Eq. linInhomEqus, Eq. adjInhom,
 * Eq. hybadjinhom) are time-stepped concurrently, one "lane" per subinterval: a
 * thread-block cluster (1D problems: the lane's grid split over the cluster's CTAs,
 * halos exchanged through distributed shared memory), one thread block (batches,
 * CSR), or a set of thread blocks over the lane's tiles (2D). The homogeneous problems
 * (Eq. hom, Eq. adjHomNormal) are carried, by linearity, as their sum over the
 * problems active on one subinterval, by one of the propagators pxa_set_propagator
 * selects: Krylov matrix-exponential actions (Sec. 4.1, Saad 1992; the default), the
 * real Leja points method (Sec. 4.1), for periodic constant-coefficient 1D operators the
 * subinterval propagator itself as a circulant band (the fastest and the one the 1D
 * benchmarks use), and for the 2D operator the RK4 stepper's subinterval propagator as
 * its power series (operator applications only); the time-varying Burgers adjoint uses the stepper's own
 * transposed step maps (or 4th-order Magnus steps with Krylov exponentials). The full
 * solution is the superposition of Eq. fullsol0 / Eq. fulladjsol, and the gradient
 * follows from Eq. initupdate (initial-condition control) or Eq. paramupdate (forcing
 * control).
 *
 * Problems (Sec. 4.2, 4.3, restricted to what this library implements):
 *   PXA_ADVDIFF_1D: dq/dt = A q,  (A q)_i = -c (q_{i+1}-q_{i-1})/(2h)
 *                                  + nu (q_{i+1}-2 q_i+q_{i-1})/h^2,  periodic,
 *                   x_i = i h, h = L/n; Crank–Nicolson stepping; control = q(0);
 *                   objective J = 0.5 ||q(T)||^2.
 *   PXA_ADVDIFF_2D: dq/dt = A q + s(t) f, (A q) = -u q_x - v q_y + nu (q_xx + q_yy) by
 *                   central differences on a periodic nx x ny grid with a frozen
 *                   velocity (u, v); q(0) = 0; control = f; the target is the
 *                   trajectory driven by f_true (pxa_set_target), J = (1/T) sum_{j=1..K}
 *                   dt ||q_j(f) - q_j(f_true)||^2 (Eq. cost). RK4 stepping in FP32 on
 *                   TMA-staged halo tiles; J sums FP32 warp partials (double-float
 *                   within blocks, FP64 across them), the
 *                   gradient accumulates as double-float (hi, lo) FP32 pairs and is
 *                   returned in FP64. Serial direct + Paraexp adjoint (hybrid scheme,
 *                   Sec. 3.3) with the stepper's own propagator for the homogeneous
 *                   parts: its exact steps, or its power series (PXA_PROP_POLY).
 *   PXA_BURGERS_1D: du/dt = -u du/dx + nu d2u/dx2 + s(t) f(x), u(0) = 0, central
 *                   differences, periodic; classical RK4; control = f;
 *                   s(t) = sin(omega t) (omega != 0) or 1; objective
 *                   J = (1/T) sum_{j=1..K} dt ||u_j - g||^2 (rectangle rule of
 *                   Eq. cost). The direct problem is solved in series and the
 *                   adjoint in parallel (hybrid scheme, Sec. 3.3); its homogeneous
 *                   parts are carried by the exact transposed RK4 step maps (banded,
 *                   several steps per halo exchange; PXA_PHI_STEPPER, the default) or
 *                   by 4th-order Magnus steps with Krylov exponentials (PXA_PHI_EXP).
 *   PXA_BURGERS_2D: dq/dt = N(q), q = (u, v) on a periodic nx x nx grid,
 *                   N_u = -u u_x - v u_y + nu lap u, N_v = -u v_x - v v_y + nu lap v by
 *                   central differences (Sec. 4.3); classical RK4 in FP32; control = q(0)
 *                   (n = 2 nx nx values, u then v, each [ny][nx] row-major); objective
 *                   J = 0.5 ||q(T) - q_target||^2 (FP64), q_target from pxa_set_target
 *                   (the target final state, n values). Serial direct + the hybrid
 *                   adjoint (Sec. 3.3): with a terminal objective the adjoint's
 *                   inhomogeneous problems vanish and the Paraexp adjoint is the serial
 *                   adjoint (the exact transposed RK4 step maps), so both modes run the
 *                   same kernels.
 *   PXA_CSR:        dq/dt = A q for a constant sparse matrix A given in CSR form (any
 *                   discretised operator, Sec. 2), classical RK4; control = q(0);
 *                   objective J = 0.5 ||q(T) - g||^2 (g from pxa_set_objective or
 *                   pxa_set_target, 0 when none is set). Alg. 1 with Krylov
 *                   propagators: exp(tau A) (PXA_PHI_EXP) or the RK4 stepper's own
 *                   R(dt A)^(K/P), R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24
 *                   (PXA_PHI_STEPPER), evaluated on the Hessenberg matrix; or that
 *                   stepper propagator as its power series (PXA_PROP_POLY).
 *
 * Conventions:
 *   - Every call returns a pxa_status (0 = PXA_OK). No call aborts, traps or
 *     throws. Errors raised inside kernels are written to a device status word and
 *     reported by the next call that synchronises (pxa_gradient, pxa_sync).
 *   - Device pointers ("_dev") are caller-owned, borrowed for the duration of the
 *     call (or, for pxa_set_operator, pxa_set_control, pxa_set_target and
 *     pxa_set_objective, until the next call of the same setter or pxa_destroy) and
 *     never freed by the library. Host pointers ("_host") are
 *     read or written before the call returns.
 *   - All vectors are FP64, contiguous, n elements (the grid points in order).
 *   - The library owns its workspace. It is (re)allocated by the first solve after
 *     a set_* call; later solves allocate nothing.
 *   - All work is enqueued on the stream given to pxa_create (a cudaStream_t,
 *     borrowed; NULL = the legacy default stream).
 *   - Not thread-safe per context: one host thread at a time per pxa_ctx.
 */
#ifndef PXA_H
#define PXA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pxa_ctx pxa_ctx;

typedef enum {
  PXA_OK = 0,
  PXA_ERR_INVALID = -1,        /* bad argument or unsupported combination */
  PXA_ERR_CUDA = -2,           /* a CUDA runtime call failed (see pxa_last_error) */
  PXA_ERR_OOM = -3,            /* workspace allocation failed */
  PXA_ERR_NOT_CONVERGED = -4,  /* a Krylov error estimate exceeded the tolerance */
  PXA_ERR_TIMEOUT = -5,        /* a bounded device wait gave up */
  PXA_ERR_NONFINITE = -6,      /* J or the gradient is not finite */
  PXA_ERR_STATE = -7,          /* call made before the context was configured */
  PXA_ERR_TOO_LARGE = -8       /* request exceeds the fixed buffer of pxa_expv_static */
} pxa_status;

typedef enum { PXA_ADVDIFF_1D = 1, PXA_BURGERS_1D = 2, PXA_ADVDIFF_2D = 3, PXA_CSR = 4, PXA_BURGERS_2D = 5 } pxa_problem;
typedef enum { PXA_CN = 1, PXA_RK4 = 2 } pxa_stepper;
/* Homogeneous propagator. EXP: exp(t A) (the paper's choice). STEPPER: the stepper's
 * own amplification R(dt A)^k (R_CN(z) = (1+z/2)/(1-z/2)), which makes Paraexp
 * reproduce serial stepping up to the Krylov tolerance. */
typedef enum { PXA_PHI_EXP = 0, PXA_PHI_STEPPER = 1 } pxa_phi;
/* How the homogeneous propagations of ADVDIFF_1D are computed: Arnoldi/Krylov (default)
 * or the real Leja points method (Sec. 4.1: Newton interpolation of phi(z) = (e^z - 1)/z
 * at Leja points of the focal interval of the spectrum; exp(B) v = v + B phi(B) v; three
 * vectors of workspace instead of a Krylov basis; PXA_PHI_EXP only). PXA_PROP_POLY
 * (ADVDIFF_2D, CSR): the RK4 stepper's own propagator R(dt B)^kk (B = A or A^T) as its
 * power series in tau B (tau = kk dt), operator applications only, like ReLPM (see
 * pxa_set_propagator). */
typedef enum { PXA_PROP_KRYLOV = 0, PXA_PROP_RELPM = 1, PXA_PROP_BAND = 2, PXA_PROP_POLY = 3 } pxa_propagator;
/* SERIAL: one lane over [0, T] (plain serial stepping, same kernels).
 * PARAEXP: P lanes + homogeneous propagation + superposition. */
typedef enum { PXA_SERIAL = 0, PXA_PARAEXP = 1 } pxa_mode;
/* Direct-state storage for the time-varying adjoint (Sec. 3.5): FULL keeps every
 * step in HBM; CHECKPOINTS keeps the P+1 subinterval boundaries and recomputes each
 * subinterval inside its adjoint lane. */
typedef enum { PXA_STORE_FULL = 0, PXA_STORE_CHECKPOINTS = 1 } pxa_memory;
/* How the BURGERS_1D discrete adjoint (the transpose of the RK4 step map, Sec. 3.3) is
 * evaluated. BANDED (default): every step's exact transposed Jacobian M_s^T is formed
 * once as a 9-diagonal band by a parallel pass over the stored (or recomputed) states,
 * and the adjoint lanes and the homogeneous chain become 9-tap recursions; used when
 * its records (about 21 doubles per step and grid point) fit in half of the free
 * device memory; the serial chain then takes four (or two) steps per halo exchange
 * with the product bands M_s^T ... M_{s+3}^T (33 diagonals) or M_s^T M_{s+1}^T (17) where
 * no lane value is added on the rows skipped. BANDED_PAIR: the same with at most two steps
 * per exchange; BANDED_SINGLE: one step per exchange. RESTEP: every reverse step
 * re-evaluates the four stages and applies their transposed Jacobians in turn (no
 * per-step storage beyond the states). */
typedef enum {
  PXA_ADJ_BANDED = 0,
  PXA_ADJ_RESTEP = 1,
  PXA_ADJ_BANDED_SINGLE = 2,
  PXA_ADJ_BANDED_PAIR = 3
} pxa_adjoint;

typedef struct {
  int kind;   /* pxa_problem */
  int n;      /* 1D: grid points, 3 <= n <= 4096 (ADVDIFF_1D up to 2^26 for
                 pxa_cn_lanes_1d and pxa_apply_operator; the gradient needs <= 4096);
                 2D: ignored (set to nx * ny) */
  double L;   /* domain length (> 0), h = L / n (2D: L / nx on both axes) */
  double c;   /* advection speed (PXA_ADVDIFF_1D) */
  double nu;  /* diffusion coefficient (>= 0) */
  int nx, ny; /* PXA_ADVDIFF_2D: grid, nx == ny, nx % 4 == 0, 8 <= nx <= 8192;
                 PXA_BURGERS_2D: nx == ny, nx % 16 == 0, 16 <= nx <= 4096 */
  const double* u_dev; /* PXA_ADVDIFF_2D: velocity components (device, [ny][nx] row-major, */
  const double* v_dev; /*   x fastest), borrowed until the next set_operator */
  /* PXA_CSR: A with n rows (1 <= n <= 16384) in CSR form on the device, borrowed until
   * the next set_operator: row i holds entries row_ptr_dev[i] .. row_ptr_dev[i+1] - 1
   * (n + 1 int64 values, row_ptr_dev[0] == 0), col_dev (int32, 0 <= col < n) and val_dev
   * (FP64). The library copies A once to the host when it builds its workspace (first
   * solve after a set_* call) to form A^T for the adjoint; column indices out of range
   * make that solve fail with PXA_ERR_INVALID. L, c, nu, nx, ny, u_dev, v_dev unused. */
  const int64_t* row_ptr_dev;
  const int32_t* col_dev;
  const double* val_dev;
} pxa_operator_desc;

/* Objective (Sec. 2, Eq. cost and its terminal form). TERMINAL_L2:
 * J = 0.5 ||q(T) - g||^2 (ADVDIFF_1D, CSR: g = 0 when target_dev is NULL; BURGERS_2D:
 * target_dev required).
 * INTEGRAL_TRACKING: J = (1/T) sum_{j=1..K} dt ||q_j - g_j||^2, the rectangle rule of
 * Eq. cost, with a static target g (BURGERS_1D; target_dev required) or the trajectory
 * driven by the true forcing f_true = target_dev (ADVDIFF_2D; required). */
typedef enum { PXA_OBJ_TERMINAL_L2 = 1, PXA_OBJ_INTEGRAL_TRACKING = 2 } pxa_objective_kind;
typedef struct {
  int kind;                 /* pxa_objective_kind */
  const double* target_dev; /* device, n doubles, borrowed until the next pxa_set_objective or
                               pxa_set_target; may be NULL for TERMINAL_L2 */
} pxa_objective_desc;

/* Precision of the time stepping (the benchmark spec's split: Krylov, superposition and the
 * objective stay FP64). F64: FP64 stepping (ADVDIFF_1D, BURGERS_1D, CSR; the default for
 * them). F32: FP32 stepping with FP32 accumulation (ADVDIFF_2D, whose only mode it is,
 * and ADVDIFF_1D with 16 <= n <= 4096, run by the batched lanes as a batch of one). */
typedef enum { PXA_F64 = 0, PXA_F32 = 1 } pxa_precision;

typedef struct {
  double J;                 /* objective of the last gradient */
  double krylov_err_max;    /* largest a-posteriori Krylov error estimate (relative) */
  int krylov_m;             /* Krylov dimension in use */
  int krylov_substeps;      /* Krylov substeps per subinterval in use */
  int magnus_steps;         /* RK4 steps per Magnus step (Burgers) */
  int lanes;                /* lanes of the last solve */
  int64_t workspace_bytes;  /* device workspace owned by the context */
  float ms_direct_inhom;    /* phase times of the last pxa_gradient with timing on (-1:
                               the events could not be read) */
  float ms_direct_hom;
  float ms_adjoint_inhom;
  float ms_adjoint_hom;
  float ms_total;
  int band_taps;            /* taps of the circulant CN band (ADVDIFF_1D) */
  int cluster_direct;       /* CTAs per cluster in use (BURGERS_1D) */
  int cluster_lanes;
  int cluster_chain;
  float ms_adjoint_prep;    /* BURGERS_1D banded adjoint: recompute + band records */
  int adjoint_band;         /* 1 when the banded adjoint is in use */
  int group_direct;         /* requested steps per halo exchange (0 = cost model) */
  int group_sweep;
  int chunks;               /* chunks of the overlapped direct solve (last gradient) */
  float partition_r;        /* ratio of successive chunk lengths in use (0: equal chunks) */
  float tau_ratio;          /* k = adjoint-preparation time / direct time per step, as
                               last measured by the autotuner (0: not measured) */
  int checkpoint_intervals; /* C of the multi-checkpoint scheme in use (0: off) */
  int lane_steps;           /* ADVDIFF_1D: q, the lanes apply the band of M^q */
  int lane_band_taps;       /* ADVDIFF_1D: taps of that band */
  int prop_band_taps;       /* ADVDIFF_1D with PXA_PROP_BAND: taps of the subinterval propagator's band */
  /* BURGERS_1D with the hybrid overlap and timing on: kernel time of the work that ran on
   * the side streams beside the direct chunks, each summed over the chunks from events
   * recorded on its own stream (0 when nothing ran there; -1: the events could not be
   * read): the band pre-pass, the pair records, the four-step records and the adjoint
   * lanes. */
  int side_chunks;          /* chunks whose side-stream work was timed */
  float ms_side_prepass;
  float ms_side_pair;
  float ms_side_quad;
  float ms_side_lanes;
  int graph_kernels;        /* kernel nodes of the gradient's captured CUDA graph (the
                               kernels one graph replay launches; 0: no graph captured) */
  int prop_degree;          /* ADVDIFF_2D with PXA_PROP_POLY: degree m of the series in use
                               (0: the stepper chain) */
  int prop_substeps;        /* chain segments per subinterval of that series */
  double prop_tail;         /* its tail bound sum_{i>m} a_i ||tau A^T||_inf^i (relative) */
} pxa_stats;

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t
 * (borrowed; NULL = default stream). *out receives the context. */
int pxa_create(pxa_ctx** out, int device, void* cuda_stream);
/* Release the context and its workspace. NULL is ignored. */
void pxa_destroy(pxa_ctx* ctx);
/* Text of the last error raised on this context ("" if none). Never NULL. */
const char* pxa_last_error(const pxa_ctx* ctx);

/* Operator and grid (Sec. 2 state equation; Sec. 4.2 / 4.3 problems). Resets the
 * objective to the operator's default (TERMINAL_L2 for ADVDIFF_1D and CSR,
 * INTEGRAL_TRACKING otherwise) and the precision to its default. Invalidates the
 * workspace. */
int pxa_set_operator(pxa_ctx* ctx, const pxa_operator_desc* op);
/* Time window [0, T], K steps of `stepper` (PXA_CN for ADVDIFF_1D, PXA_RK4 for
 * BURGERS_1D, ADVDIFF_2D and CSR), P equal subintervals (Alg. 1: T_p = p T / P).
 * K % P == 0 is required. */
int pxa_set_time(pxa_ctx* ctx, double T, int64_t K, int stepper, int P);
/* Objective (pxa_objective_desc). A kind the operator does not support returns
 * PXA_ERR_INVALID (set the operator first: PXA_ERR_STATE otherwise). Same as
 * pxa_set_target for the target. Invalidates the stored direct state. */
int pxa_set_objective(pxa_ctx* ctx, const pxa_objective_desc* obj);
/* Stepping precision (pxa_precision). ADVDIFF_1D with PXA_F32 runs the whole gradient
 * through the batched FP32 lanes (pxa_batch_* with one problem: FP32 lanes, FP64
 * superposition; PXA_PHI_STEPPER carries the homogeneous parts by the stepper's own
 * propagator as an FP32 band, PXA_PHI_EXP by FP64 Krylov exponentials); with it,
 * pxa_gradient, pxa_gradient_async, pxa_sync and pxa_gradient_host are available and
 * the split solves return PXA_ERR_INVALID. FP32 stepping of K steps loses about
 * K * 2^-24 relative in J and the gradient. Unsupported combinations: PXA_ERR_INVALID.
 * Invalidates the workspace. */
int pxa_set_precision(pxa_ctx* ctx, int step_precision);
/* Krylov dimension m (2 <= m <= 48), tolerance on the a-posteriori estimate
 * (relative to ||v||), homogeneous propagator (pxa_phi) and the number of Krylov
 * substeps per subinterval (>= 1; each substep spans K/(P*substeps) steps, which
 * must be an integer). */
int pxa_set_krylov(pxa_ctx* ctx, int m, double tol, int phi, int substeps);
/* ADVDIFF_1D homogeneous propagator (pxa_propagator). With PXA_PROP_RELPM the Newton
 * series runs up to max_degree (2..200) terms per substep until its last two terms fall
 * below the tolerance of pxa_set_krylov times ||v|| (else PXA_ERR_NOT_CONVERGED); the
 * substeps keep the capacity of the spectral ellipse <= 4 each (automatic). With
 * PXA_PROP_BAND the subinterval propagator itself, exp(tau A) (PXA_PHI_EXP) or the CN
 * power M^(K/P) (PXA_PHI_STEPPER), is applied once per link as a circulant band: A is
 * circulant (periodic grid, constant coefficients), so the propagator's taps are the
 * inverse DFT of its eigenvalues, built on the host (FP64, kept to 2^-50 of the largest
 * tap; max_degree is not used). With PXA_PROP_POLY (ADVDIFF_2D and CSR, Paraexp; other
 * operators return PXA_ERR_INVALID at the first solve) the summed homogeneous problems are
 * carried by the RK4 stepper's own propagator over chain segments of kk steps,
 * R(dt B)^kk = sum_i a_i (tau B)^i with R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, tau = kk dt
 * and B = A^T (ADVDIFF_2D: the adjoint chain, Eq. adjHomNormal, whose forcing gradient over
 * each segment, Eq. paramupdate, is a second series in the same powers) or B = A and A^T
 * (CSR: the direct chain of Eq. hom and the adjoint chain). The series is cut after the
 * smallest degree m (a multiple of 4) whose tail bound sum_{i>m} a_i ||tau B||_inf^i is
 * below the tolerance of pxa_set_krylov (ADVDIFF_2D, FP32 stepping: at least 1e-7); kk is
 * the largest divisor of K/P with kk ||dt B||_inf <= 4. m above max_degree returns
 * PXA_ERR_NOT_CONVERGED at the first solve. The series needs only operator applications
 * (m per segment against 4 kk for stepping) and no inner products. Invalidates the
 * workspace. */
int pxa_set_propagator(pxa_ctx* ctx, int method, int max_degree);
/* Burgers: RK4 steps per Magnus step of the homogeneous adjoint (divides K/P). */
int pxa_set_magnus(pxa_ctx* ctx, int steps_per_magnus);
/* Control (Eq. initupdate / paramupdate): ADVDIFF_1D, CSR: q0_dev = initial condition.
 * BURGERS_1D: f_dev = forcing, s(t) = sin(omega t) or 1 when omega == 0. ADVDIFF_2D:
 * f_dev = forcing, s(t) = sin(omega t). */
int pxa_set_control(pxa_ctx* ctx, const double* control_dev, double omega);
/* The objective's target (see pxa_objective_desc): g (ADVDIFF_1D, CSR: terminal;
 * BURGERS_1D: tracking), or the true forcing f_true (ADVDIFF_2D). */
int pxa_set_target(pxa_ctx* ctx, const double* target_dev);
/* Direct-state storage policy (pxa_memory). */
int pxa_set_memory(pxa_ctx* ctx, int policy);
/* Multi-checkpoint scheme (Sec. 3.5), BURGERS_1D with the banded adjoint
 * (PXA_ADJ_BANDED or PXA_ADJ_BANDED_PAIR). With intervals = C >= 2 the direct solve is a
 * rough pass that keeps J and the C + 1 states at t = iT/C. The adjoint then takes the
 * intervals [iT/C, (i+1)T/C] from the top: each is re-stepped from its checkpoint and
 * solved by the Paraexp adjoint over its own P equal subintervals (K/(CP) steps each;
 * the placement of the checkpoints does not depend on the partition), starting from the
 * adjoint value at its top row that the interval above computed. Device memory for the
 * trajectory, the band records and the adjoint rows falls from K + 1 rows to
 * 2 (K/C + 1) rows: two interval buffer sets, so that the re-step, records and lanes of
 * one interval run beside the chain of the other. The gradient equals that of full
 * storage up to rounding order. Requires K % (C * P) == 0 (checked when the workspace is
 * built: PXA_ERR_INVALID) and, for Paraexp, PXA_PHI_STEPPER. The memory policy of
 * pxa_set_memory is not used while the scheme is on. intervals = 0 or 1: off (default).
 * intervals < 0 or > 65536: PXA_ERR_INVALID. Invalidates the workspace. */
int pxa_set_checkpoints(pxa_ctx* ctx, int intervals);
/* ADVDIFF_1D: CN steps per band application of the Paraexp and serial lanes, q = 1, 2
 * or 4 (the exact product band of M^q from the eigenvalues R_k^q, FP64 taps kept to
 * 2^-52 of the largest; the sources become (M^q - I) x), or 0 (default): the largest of
 * 4, 2, 1 that divides K/P. pxa_step keeps single steps. A q that does not divide K/P
 * makes the next solve fail with PXA_ERR_INVALID. Invalidates the workspace. */
int pxa_set_lane_steps(pxa_ctx* ctx, int q);
/* BURGERS_1D adjoint evaluation (pxa_adjoint). BANDED falls back to RESTEP when its
 * records do not fit; pxa_get_stats reports which one is in use. */
int pxa_set_adjoint(pxa_ctx* ctx, int impl);
/* BURGERS_1D with the banded adjoint and full storage: run the serial direct solve in
 * chunks of whole subintervals and, on a library-owned low-priority stream, build the
 * band records and run the adjoint lanes of each finished chunk while the next one is
 * stepped (1, default), or run the phases one after another (0). Results are the same
 * up to the summation order of J. */
int pxa_set_overlap(pxa_ctx* ctx, int enable);
/* BURGERS_1D overlapped direct solve: lengths of its chunks (at most 8). r == 0 (default):
 * equal chunks. 0 < r < 1: chunk lengths in geometric progression, Delta_{n+1} = r Delta_n,
 * i.e. boundaries T_n = T (1 - r^n) / (1 - r^N) (Eq. nonEquiP), each rounded to whole
 * subintervals (steps when P == 1) with at least one per chunk, so that the adjoint work
 * left after the last direct step shrinks. Sec. 3.3 takes r = k/(k+1) with
 * k = tau_I_adj / tau_I (processors that solve their adjoint parts side by side); for one
 * in-order stream of adjoint work the same equal-finish argument gives r = k. The
 * autotuner measures k and times both (and a few fixed ratios). Other r: PXA_ERR_INVALID. */
int pxa_set_partition(pxa_ctx* ctx, double r);
/* Host-only (no device work): the chunk boundaries, in steps, that the overlapped direct
 * solve uses for K steps and P subintervals (P == 1: chunks of steps) at ratio r, with at
 * most max_chunks chunks (1..64). Writes NC + 1 increasing values from 0 to K into
 * bounds (caller-owned, max_chunks + 1 entries) and returns NC >= 1; PXA_ERR_INVALID
 * for bad arguments (K < 1, P < 1, K % P != 0, r outside [0, 1), NULL bounds). */
int pxa_partition_bounds(int64_t K, int P, double r, int max_chunks, int64_t* bounds);
/* BURGERS_1D: steps per halo exchange of the serial RK4 sweep (q_direct) and of the
 * banded adjoint sweeps (q_sweep): 1, 2 or 4 (a CTA then also steps 4(q-1) of its
 * neighbours' points on each side, and needs at least 4q points of its own); 0 = chosen
 * by a cost model (default). The autotuner searches them. */
int pxa_set_groups(pxa_ctx* ctx, int q_direct, int q_sweep);
/* CTAs per thread-block cluster of the BURGERS_1D RK4 kernels: the serial direct
 * lane, each of the P concurrent adjoint lanes, and the homogeneous chain (1..16;
 * 0 = automatic: 16 for the serial lanes, SMs/P for the concurrent lanes, both capped
 * so that each CTA keeps >= 32 grid points). One lane is split into contiguous
 * chunks, one per CTA, exchanging halos through distributed shared memory. */
int pxa_set_cluster(pxa_ctx* ctx, int direct, int lanes, int chain);
/* Capture the whole gradient into a CUDA graph and replay it (1) or launch kernels
 * one by one (0, default). */
int pxa_set_graph(pxa_ctx* ctx, int enable);

/* One direct-adjoint loop (Sec. 2: state, adjoint, gradient; Alg. 1 in PXA_PARAEXP
 * mode, the hybrid scheme of Sec. 3.3 for BURGERS_1D and ADVDIFF_2D): J into *J_host
 * (may be NULL), dJ/d(control) into grad_dev (n doubles, caller-owned; Eq. initupdate
 * for an initial-condition control, Eq. paramupdate for a forcing). Synchronises the
 * stream; returns device-side errors (NOT_CONVERGED, NONFINITE, TIMEOUT). */
int pxa_gradient(pxa_ctx* ctx, int mode, double* J_host, double* grad_dev);
/* Same, asynchronous: J is written to J_dev (one double, device). Errors raised
 * inside kernels surface at the next pxa_sync. Graph-capturable once the workspace
 * exists (after one pxa_gradient). */
int pxa_gradient_async(pxa_ctx* ctx, int mode, double* J_dev, double* grad_dev);
/* The two halves of pxa_gradient, for a caller that differentiates through the
 * direct solve (e.g. an autograd function): pxa_solve_direct runs the direct problem
 * (Eq. seriesDirect serially; in PXA_PARAEXP mode Eq. linzero, linInhomEqus, hom and
 * fullsol0) and stores what the adjoint needs (q(T) and the adjoint source, or the
 * Burgers trajectory / checkpoints) in the context, returning J; pxa_solve_adjoint
 * then runs the adjoint problem of the same mode (Eq. adjInhom or hybadjinhom,
 * adjHomNormal, fulladjsol) and writes dJ/d(control) to grad_dev (Eq. initupdate /
 * paramupdate). Any set_* call in between invalidates the stored state
 * (PXA_ERR_STATE). Both synchronise the stream. */
int pxa_solve_direct(pxa_ctx* ctx, int mode, double* J_host);
int pxa_solve_adjoint(pxa_ctx* ctx, int mode, double* grad_dev);
/* Wait for the stream and report device-side errors (with timing on, also reads the
 * phase times of the last gradient into the statistics). */
int pxa_sync(pxa_ctx* ctx);
/* End-to-end call with host buffers: copies control_host (n doubles) to the device,
 * runs pxa_gradient and copies the gradient back into grad_host (n doubles). */
int pxa_gradient_host(pxa_ctx* ctx, int mode, const double* control_host, double* J_host,
                      double* grad_host);
/* BURGERS_2D building block: the final state q(T) (FP64, n values) of the direct
 * solve from the initial state ic_dev (n values), e.g. to make a tracking target from a
 * "true" initial state. Uses the context's trajectory buffer (a later pxa_solve_adjoint
 * needs a new pxa_solve_direct). Synchronous. */
int pxa_direct_state(pxa_ctx* ctx, const double* ic_dev, double* state_dev);
/* Iterative nonlinear Paraexp direct of Alg. 2 (Sec. 3.2, Eq. nonlinTrans, Jacobians,
 * nlHomIter, fullsolIter) for BURGERS_1D (n <= 1024, u(0) = 0, the forcing of
 * pxa_set_control): from the guess q_0(t) (guess_dev, (K+1) x n device rows, or NULL:
 * q_0(t) = 0), each iteration linearises about q_i with the Jacobian averaged over each
 * subinterval (dN/dq at the trapezoid-rule average of q_i there), steps the P linear
 * inhomogeneous problems from zero concurrently (one thread block each; their source at
 * each RK4 stage is N(Y) - J_p Y + s(t) f at the stage states Y of q_i's nonlinear RK4
 * step), carries their homogeneous problems from q0 with the stepper's own propagator of
 * (A + J_p) and sums them into q_{i+1} at every step. It stops when
 * max_s ||q_{i+1}(t_s) - q_i(t_s)|| / max_s ||q_{i+1}(t_s)|| <= tol or after max_iter
 * iterations. The fixed point is the serial RK4 trajectory. traj_dev ((K+1) x n,
 * caller-owned) receives the last iterate; changes_host (max_iter doubles, may be NULL)
 * the change of each iteration; *iters_host (may be NULL) their number. Allocates its
 * buffers (three trajectories) on the first call. Returns PXA_OK (converged),
 * PXA_ERR_NOT_CONVERGED (max_iter reached; traj_dev holds the last iterate),
 * PXA_ERR_NONFINITE (diverged), or a set-up error. Synchronous. */
int pxa_nl_paraexp(pxa_ctx* ctx, const double* guess_dev, double tol, int max_iter, double* traj_dev,
                   double* changes_host, int* iters_host);
/* Statistics of the last solve. */
int pxa_get_stats(const pxa_ctx* ctx, pxa_stats* out);
/* Limit of the context's bounded device waits (the mbarrier waits of the cluster halo
 * exchanges), in SM clock cycles: 0 = the default, 2^31 cycles (about 1 s at 2 GHz);
 * otherwise 1024 <= cycles <= 2^41 (rounded down to a multiple of 1024). A wait that
 * runs out sets PXA_ERR_TIMEOUT, which the next synchronising call returns; the kernel
 * then runs to its end (its results are not valid), the later waits of that launch give
 * up early, and the context stays usable. Other values: PXA_ERR_INVALID. */
int pxa_set_wait_limit(pxa_ctx* ctx, int64_t cycles);
/* Test of the failure path of the bounded waits (no counterpart in the paper): launches
 * one thread block that waits, with the context's wait limit, on an mbarrier that
 * nothing completes (no copy is issued, no peer exists), then synchronises like
 * pxa_sync. Returns PXA_ERR_TIMEOUT after the limit (the expected result), or an error
 * of the set-up. Builds the workspace if needed (the operator and time must be set). */
int pxa_wait_probe(pxa_ctx* ctx);
/* Per-phase CUDA-event timing inside pxa_gradient (0 = off, default); with graphs on,
 * the events are part of the captured graph. */
int pxa_set_timing(pxa_ctx* ctx, int enable);
/* Autotuner: times one gradient of `mode` for each candidate configuration on the
 * configured problem (control and target must be set) and keeps the fastest whose
 * Krylov error estimates stay within the tolerance. ADVDIFF_1D candidates: Krylov
 * dimension m and substeps per subinterval (m in {16, 20, 24, 30, 36, 40}, substeps in
 * {1, 2, 4, 8} dividing K/P). BURGERS_1D candidates: cluster sizes of the direct,
 * lane and chain kernels. grad_dev: n doubles of scratch for the trial gradients.
 * *best_ms_host (may be NULL) receives the best time. Allocates workspace while
 * tuning; returns PXA_ERR_NOT_CONVERGED if no candidate meets the tolerance. */
int pxa_autotune(pxa_ctx* ctx, int mode, double* grad_dev, double* best_ms_host);

/* ---- building blocks, exposed for kernel-level tests --------------------------
 * y = A x (transpose = 0) or A^T x (transpose = 1) for ADVDIFF_1D. */
int pxa_apply_operator(pxa_ctx* ctx, int transpose, const double* x_dev, double* y_dev);
/* y = M^steps x for the configured stepper (ADVDIFF_1D: the CN map
 * M = (I - dt/2 A)^{-1} (I + dt/2 A), dt = T/K), or (M^T)^steps x. One thread block. */
int pxa_step(pxa_ctx* ctx, int transpose, int64_t steps, const double* x_dev, double* y_dev);
/* y = phi(A) x over `substeps` Krylov substeps spanning `span_steps` time steps
 * (ADVDIFF_1D; phi from pxa_set_krylov). err_host (may be NULL) receives the
 * largest relative error estimate. */
int pxa_expv(pxa_ctx* ctx, int transpose, int64_t span_steps, int substeps,
             const double* x_dev, double* y_dev, double* err_host);
/* Burgers building blocks on the configured grid: y = N(u) (rhs, no forcing),
 * y = J(u)^T x (transposed Jacobian). */
int pxa_burgers_rhs(pxa_ctx* ctx, const double* u_dev, double* y_dev);
int pxa_burgers_jac_T(pxa_ctx* ctx, const double* u_dev, const double* x_dev, double* y_dev);

/* ADVDIFF_1D: `steps` FP32 Crank-Nicolson steps of `lanes` lanes whose states live in
 * global memory (n % 4 == 0; every lane starts from the configured control), one launch
 * per step over all lanes: the exact circulant CN band, FP32 arithmetic and accumulation.
 * Timed with CUDA events on the context's stream; allocates 2 * lanes * n floats on the
 * first call for a given lane count. *ms_host receives the elapsed time; out_dev
 * (optional, lanes * n doubles) the final states. */
int pxa_cn_lanes_1d(pxa_ctx* ctx, int lanes, int64_t steps, double* out_dev, double* ms_host);
/* ADVDIFF_2D: `steps` FP32 RK4 steps of `lanes` zero-initial-value inhomogeneous
 * lanes (Eq. linInhomEqus with the forcing s(t) f of the configured control; lane l
 * starts at step l * steps) on the TMA halo-tile kernel, timed with CUDA events on the
 * context's stream. Allocates its own lane states (2 * lanes padded FP32 arrays) on the
 * first call for a given lane count. *ms_host receives the elapsed time; out_dev
 * (optional, lanes * nx * ny doubles) receives the final lane states. */
int pxa_rk4_lanes_2d(pxa_ctx* ctx, int lanes, int64_t steps, double* out_dev, double* ms_host);

/* ---- allocation-free Krylov propagation ----------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that must
 * not allocate device memory: a plugin inside an application that owns every byte
 * of device memory, or a real-time loop that fixes its memory footprint at start-up
 * and cannot handle an allocation failure later. The context-based calls above
 * allocate their workspace on the first solve, so such callers cannot use them.
 *
 * Computes what pxa_expv computes for PXA_ADVDIFF_1D (stencil of pxa_operator_desc
 * with kind PXA_ADVDIFF_1D, time step dt = T/K): y = phi(A) x (or phi(A^T) x) over
 * `substeps` Krylov substeps spanning `span_steps` time steps, phi = exp (PXA_PHI_EXP)
 * or the Crank–Nicolson power (PXA_PHI_STEPPER); Krylov dimension m, tolerance tol
 * on the a-posteriori estimate. x_dev, y_dev: caller-owned device vectors of n doubles.
 * err_host (may be NULL) receives the largest relative error estimate.
 *
 * Memory: the Krylov basis, the status word and the error estimate live in one
 * fixed array of PXA_EXPV_STATIC_MAX_DOUBLES doubles (1 MiB) defined inside the
 * library; every GPU that loads the library holds it until the process exits. The
 * call allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Requests with n * (m + 1) > PXA_EXPV_STATIC_MAX_DOUBLES - 64 return
 * PXA_ERR_TOO_LARGE before touching the device.
 *
 * Set-up: the first call on a device looks up the array's device address (with that
 * device current) and caches it for the life of the process; make that first call
 * before any stream capture. The cached address does not survive a cudaDeviceReset
 * (or any other teardown of the device's primary context): do not call this entry
 * point on a device after it has been reset.
 * The call runs on `cuda_stream` of device `device` and synchronises that stream
 * before returning. Every call shares the one array, which keeps the last call's
 * contents: the status word and the error estimate are cleared by each call, the
 * basis is overwritten. Calls that overlap on the GPU (other streams, other host
 * threads) race on the array and must be serialised by the caller.
 * Returns PXA_OK, PXA_ERR_INVALID (bad arguments), PXA_ERR_TOO_LARGE,
 * PXA_ERR_NOT_CONVERGED (estimate above tol) or PXA_ERR_CUDA. */
#define PXA_EXPV_STATIC_MAX_DOUBLES 131072
int pxa_expv_static(int device, void* cuda_stream, const pxa_operator_desc* op, double T,
                    int64_t K, int m, double tol, int phi, int transpose, int64_t span_steps,
                    int substeps, const double* x_dev, double* y_dev, double* err_host);

/* ---- sparse building block -------------------------------------------------------
 * y = A x for A in CSR form: n rows (1 <= n <= 2^31 - 1), row_ptr[n + 1] (int64, row i
 * holds entries row_ptr[i] .. row_ptr[i+1] - 1), col[nnz] (int32, 0 <= col < n) and
 * val[nnz] (FP64); x[n], y[n] FP64. All device pointers, caller-owned; asynchronous on
 * `cuda_stream` (a cudaStream_t, NULL = the default stream); nothing is allocated. One
 * thread per row, suited to the short, uniform rows of discretised operators (Sec. 4).
 * Column indices are not checked; col and val must not be NULL even when A has no
 * entries. Returns PXA_ERR_INVALID for a null pointer or n out of range, PXA_ERR_CUDA
 * when the launch fails. */
int pxa_spmv_csr(void* cuda_stream, int64_t n, const int64_t* row_ptr, const int32_t* col,
                 const double* val, const double* x, double* y);

/* ---- batches of independent 1D advection-diffusion problems -----------------------
 * Alg. 1 for `count` independent ADVDIFF_1D problems with their own grid n[i] and
 * viscosity nu[i] (shared c, L, T, K, P): initial-condition control q0_i and the terminal
 * objective J_i = 0.5 ||q_i(T)||^2 (Eq. adjFinalTime, Eq. initupdate), all problems in one
 * launch per phase. The lanes (Eq. linInhomEqus / Eq. adjInhom: P per problem in Paraexp
 * mode, one serial lane of K steps per problem in serial mode) step the exact circulant
 * Crank-Nicolson band in FP32 with FP32 accumulation (q steps per band application,
 * pxa_batch_set_lane_steps), taken from a cost-sorted work list
 * by a persistent grid; the homogeneous propagations (Eq. hom / Eq. adjHomNormal) are
 * Krylov exponentials exp(tau A) in FP64 or the stepper's own propagator M^(K/P) in FP32
 * (pxa_batch_set_homogeneous, pxa_batch_set_power), and the superpositions are FP64.
 *
 * Packed layout: problem i owns points [off_i, off_i + n[i]) of every packed vector
 * (off_0 = 0, off_{i+1} = off_i + n[i]; pxa_batch_offsets returns them). */
typedef struct pxa_batch pxa_batch;
typedef struct {
  int count;                /* problems */
  int64_t points;           /* sum of n[i] */
  int krylov_m;             /* Krylov dimension in use */
  double krylov_reach;      /* substep rule: each substep spans at most reach * m^2 / ||A||_inf */
  int substeps_max;         /* Krylov substeps per subinterval of the stiffest problem */
  int band32_max;           /* widest FP32 lane band (taps) */
  int band64_max;           /* widest FP64 band (taps) */
  int lanes_grid;           /* thread blocks of the persistent lane launch */
  double krylov_err_max;    /* largest a-posteriori Krylov estimate of the last gradient */
  int64_t workspace_bytes;
  int krylov_problems;      /* problems whose homogeneous parts use the Krylov exponential */
  double hom_ratio;         /* cost-model threshold in use (see pxa_batch_set_homogeneous) */
  float ms_lanes;           /* phase times of the last gradient with timing on: direct lanes, */
  float ms_chains;          /*   direct homogeneous chains, */
  float ms_adjoint_lanes;   /*   adjoint lanes (with the superposition before them), */
  float ms_adjoint_chains;  /*   adjoint chains, */
  float ms_total;           /*   the whole gradient */
  int power_problems;       /* problems whose homogeneous parts apply the band of M^(K/P) */
  int band_power_max;       /* widest band of M^(K/P) in use (taps; 0: none) */
  int lane_steps;           /* q: the lanes apply the band of M^q, q CN steps at a time */
  int one_launch;           /* 1 when the last gradient ran as one persistent launch */
  int flow_grid;            /* thread blocks of that launch */
  int graph_kernels;        /* kernel nodes of the gradient's captured CUDA graph (0: none) */
} pxa_batch_stats;
/* Create / destroy a batch context on `device`; `cuda_stream` is borrowed (NULL = the
 * default stream). */
int pxa_batch_create(pxa_batch** out, int device, void* cuda_stream);
void pxa_batch_destroy(pxa_batch* b);
const char* pxa_batch_last_error(const pxa_batch* b);
/* The problems: count >= 1, n[i] in [16, 4096], nu[i] >= 0 (host arrays, copied);
 * c, L > 0, T > 0, K % P == 0, 1 <= P <= 64. Invalidates the workspace. */
int pxa_batch_set(pxa_batch* b, int count, const int* n, const double* nu, double c, double L, double T,
                  int64_t K, int P);
/* Krylov dimension m (2..48), tolerance of the a-posteriori estimate (relative) and the
 * substep rule reach > 0: each substep of exp(tau A) spans at most reach * m^2 / ||A||_inf
 * (default m = 30, tol = 1e-8, reach = 0.04; for a diffusion-dominated A the Krylov error
 * falls like exp(-m^2 / (5 rho)) with rho a quarter of the substep's spectral width, so
 * 1e-8 needs reach of a few hundredths). */
int pxa_batch_set_krylov(pxa_batch* b, int m, double tol, double reach);
/* Homogeneous propagation per problem (Paraexp mode): the Krylov exponential exp(tau A)
 * of Eq. hom (FP64), or the local chained form with the stepper's own propagator M^(K/P)
 * (FP32: the summed homogeneous problems carried subinterval by subinterval, which
 * reproduces serial stepping). A problem uses the exponential when a cost model puts it
 * at most `ratio` times the stepper's propagator (ratio >= 0; 0 = never, default 1; a
 * very large ratio = always the exponential). */
int pxa_batch_set_homogeneous(pxa_batch* b, double ratio);
/* How the stepper's propagator M^(K/P) is applied (Paraexp mode). enable = 1 (default):
 * M is circulant (periodic grid, constant coefficients), so M^(K/P) is the circulant band
 * whose taps are the inverse DFT of R_k^(K/P) (R_k the CN eigenvalues; taps kept to
 * 2^-36 of the largest), built on the host and applied once per link in FP32: a link
 * costs one band product instead of K/P CN steps. Problems whose band is wider than
 * 2 BATCH_MAX_RP + 1 = 2049 taps step instead. enable = 0: every link takes K/P CN steps.
 * Invalidates the workspace. */
int pxa_batch_set_power(pxa_batch* b, int enable);
/* CN steps per band application of the lanes and stepped chains: q = 1, 2 or 4 (the
 * lanes apply the exact product band of M^q, built on the host from the eigenvalues
 * R_k^q; FP32 taps kept to 2^-40 of the largest, FP64 taps of M^q for the sources
 * (M^q - I) x), or 0 (default): the largest of 4, 2, 1 that divides K/P and whose bands
 * fit the lanes (2 BATCH_MAX_R + 1 = 511 taps). A q that does not divide K/P makes the
 * next gradient fail with PXA_ERR_INVALID. Invalidates the workspace. */
int pxa_batch_set_lane_steps(pxa_batch* b, int q);
/* Capture the whole gradient into a CUDA graph and replay it (1, default) or launch the
 * kernels one by one (0). */
int pxa_batch_set_graph(pxa_batch* b, int enable);
/* Schedule of a Paraexp gradient. one_launch = 1 (default): when no problem uses the
 * Krylov exponential, the whole gradient of every problem is one persistent launch: a
 * grid of resident thread blocks takes (problem, subinterval, phase) items (the source,
 * each direct lane, the chain with the superposition, each adjoint lane, the adjoint
 * chain with the gradient) from a dependency-ordered queue through an atomic counter,
 * and an item starts once per-problem counters in device memory show its inputs done
 * (a bounded wait: PXA_ERR_TIMEOUT after about 2^31 cycles). A problem's chain thus
 * starts as soon as its own lanes are done instead of after every problem's. The
 * results are bit-identical to the phase schedule. one_launch = 0: one launch per phase
 * (seven). Serial stepping and batches with Krylov problems always use the phases.
 * Other values: PXA_ERR_INVALID. Invalidates the captured graph. */
int pxa_batch_set_schedule(pxa_batch* b, int one_launch);
/* Per-phase CUDA-event timing of the next gradients (launched one by one; 0 = off). */
int pxa_batch_set_timing(pxa_batch* b, int enable);
/* One direct-adjoint loop of every problem, asynchronous on the stream: q0_dev (packed,
 * caller-owned) -> J_dev[count] and grad_dev (packed) on the device. mode: PXA_SERIAL or
 * PXA_PARAEXP. Errors raised inside kernels surface at pxa_batch_sync. */
int pxa_batch_gradient(pxa_batch* b, int mode, const double* q0_dev, double* J_dev, double* grad_dev);
/* Wait for the stream; returns device-side errors (NOT_CONVERGED, NONFINITE). */
int pxa_batch_sync(pxa_batch* b);
/* Times one gradient of `mode` for each candidate Krylov dimension and cost-model
 * threshold (pxa_batch_set_homogeneous) and keeps the fastest whose estimates stay
 * within the tolerance; *best_ms_host (may be NULL) receives its time. */
int pxa_batch_autotune(pxa_batch* b, int mode, const double* q0_dev, double* J_dev, double* grad_dev,
                       double* best_ms_host);
/* Host: the count + 1 packed offsets (caller-owned array). */
int pxa_batch_offsets(const pxa_batch* b, int64_t* offsets);
/* Host: per problem, the taps (2 r + 1) of its FP32 lane band and of its FP64 band (both
 * of M^q, q = the lane_steps of pxa_batch_get_stats), and whether its homogeneous parts
 * use the Krylov exponential (1) or the stepper's own propagator (0) (count
 * entries each, caller-owned; any may be NULL); the workspace must exist (after a
 * gradient). */
int pxa_batch_problem_info(const pxa_batch* b, int* taps32, int* taps64, int* krylov);
int pxa_batch_get_stats(const pxa_batch* b, pxa_batch_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* PXA_H */
