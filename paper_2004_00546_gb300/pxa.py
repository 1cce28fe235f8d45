"""ctypes binding of libpxa (include/pxa.h): argument marshalling only.

Every numerical step runs inside libpxa's CUDA kernels; this module converts torch
tensors to device pointers, numpy arrays to host pointers, and pxa_status codes to
exceptions. It never computes anything itself and has no CPU fallback: if the
library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpxa.so")

OK, ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_NONFINITE, ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
ERR_TOO_LARGE = -8
EXPV_STATIC_MAX_DOUBLES = 131072
ADVDIFF_1D, BURGERS_1D, ADVDIFF_2D, CSR, BURGERS_2D = 1, 2, 3, 4, 5
OBJ_TERMINAL_L2, OBJ_INTEGRAL_TRACKING = 1, 2
F64, F32 = 0, 1
CN, RK4 = 1, 2
PHI_EXP, PHI_STEPPER = 0, 1
PROP_KRYLOV, PROP_RELPM, PROP_BAND, PROP_POLY = 0, 1, 2, 3
SERIAL, PARAEXP = 0, 1
STORE_FULL, STORE_CHECKPOINTS = 0, 1
ADJ_BANDED, ADJ_RESTEP, ADJ_BANDED_SINGLE, ADJ_BANDED_PAIR = 0, 1, 2, 3

_STATUS_NAMES = {ERR_INVALID: "INVALID", ERR_CUDA: "CUDA", ERR_OOM: "OOM",
                 ERR_NOT_CONVERGED: "NOT_CONVERGED", ERR_TIMEOUT: "TIMEOUT",
                 ERR_NONFINITE: "NONFINITE", ERR_STATE: "STATE", ERR_TOO_LARGE: "TOO_LARGE"}

EXPORTS = [
    "pxa_create", "pxa_destroy", "pxa_last_error", "pxa_set_operator", "pxa_set_time",
    "pxa_set_krylov", "pxa_set_magnus", "pxa_set_control", "pxa_set_target", "pxa_set_objective",
    "pxa_set_precision", "pxa_set_memory", "pxa_set_adjoint", "pxa_set_overlap", "pxa_set_partition", "pxa_set_checkpoints", "pxa_set_lane_steps", "pxa_partition_bounds", "pxa_set_propagator", "pxa_set_groups",
    "pxa_set_graph", "pxa_gradient", "pxa_gradient_async", "pxa_sync", "pxa_gradient_host",
    "pxa_get_stats", "pxa_set_timing", "pxa_set_wait_limit", "pxa_wait_probe", "pxa_nl_paraexp",
    "pxa_direct_state", "pxa_apply_operator", "pxa_step", "pxa_expv",
    "pxa_burgers_rhs", "pxa_burgers_jac_T", "pxa_expv_static", "pxa_set_cluster", "pxa_autotune", "pxa_solve_direct", "pxa_solve_adjoint",
    "pxa_rk4_lanes_2d", "pxa_cn_lanes_1d", "pxa_spmv_csr",
    "pxa_batch_create", "pxa_batch_destroy", "pxa_batch_last_error", "pxa_batch_set",
    "pxa_batch_set_homogeneous", "pxa_batch_set_power", "pxa_batch_set_lane_steps", "pxa_batch_set_timing",
    "pxa_batch_set_krylov", "pxa_batch_set_graph", "pxa_batch_set_schedule", "pxa_batch_gradient", "pxa_batch_sync",
    "pxa_batch_autotune", "pxa_batch_offsets", "pxa_batch_get_stats", "pxa_batch_problem_info",
]


class PxaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pxa status {_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class OperatorDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("L", ctypes.c_double),
                ("c", ctypes.c_double), ("nu", ctypes.c_double), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("u_dev", ctypes.c_void_p), ("v_dev", ctypes.c_void_p),
                ("row_ptr_dev", ctypes.c_void_p), ("col_dev", ctypes.c_void_p), ("val_dev", ctypes.c_void_p)]


class ObjectiveDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("target_dev", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("J", ctypes.c_double), ("krylov_err_max", ctypes.c_double),
                ("krylov_m", ctypes.c_int), ("krylov_substeps", ctypes.c_int),
                ("magnus_steps", ctypes.c_int), ("lanes", ctypes.c_int),
                ("workspace_bytes", ctypes.c_int64), ("ms_direct_inhom", ctypes.c_float),
                ("ms_direct_hom", ctypes.c_float), ("ms_adjoint_inhom", ctypes.c_float),
                ("ms_adjoint_hom", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("band_taps", ctypes.c_int), ("cluster_direct", ctypes.c_int),
                ("cluster_lanes", ctypes.c_int), ("cluster_chain", ctypes.c_int),
                ("ms_adjoint_prep", ctypes.c_float), ("adjoint_band", ctypes.c_int),
                ("group_direct", ctypes.c_int), ("group_sweep", ctypes.c_int),
                ("chunks", ctypes.c_int), ("partition_r", ctypes.c_float),
                ("tau_ratio", ctypes.c_float), ("checkpoint_intervals", ctypes.c_int),
                ("lane_steps", ctypes.c_int), ("lane_band_taps", ctypes.c_int),
                ("prop_band_taps", ctypes.c_int), ("side_chunks", ctypes.c_int),
                ("ms_side_prepass", ctypes.c_float), ("ms_side_pair", ctypes.c_float),
                ("ms_side_quad", ctypes.c_float), ("ms_side_lanes", ctypes.c_float),
                ("graph_kernels", ctypes.c_int), ("prop_degree", ctypes.c_int),
                ("prop_substeps", ctypes.c_int), ("prop_tail", ctypes.c_double)]


class BatchStats(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("points", ctypes.c_int64), ("krylov_m", ctypes.c_int),
                ("krylov_reach", ctypes.c_double), ("substeps_max", ctypes.c_int),
                ("band32_max", ctypes.c_int), ("band64_max", ctypes.c_int), ("lanes_grid", ctypes.c_int),
                ("krylov_err_max", ctypes.c_double), ("workspace_bytes", ctypes.c_int64),
                ("krylov_problems", ctypes.c_int), ("hom_ratio", ctypes.c_double),
                ("ms_lanes", ctypes.c_float), ("ms_chains", ctypes.c_float),
                ("ms_adjoint_lanes", ctypes.c_float), ("ms_adjoint_chains", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("power_problems", ctypes.c_int),
                ("band_power_max", ctypes.c_int), ("lane_steps", ctypes.c_int), ("one_launch", ctypes.c_int),
                ("flow_grid", ctypes.c_int), ("graph_kernels", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libpxa.so (built by ``paper_2004_00546_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libpxa.so not found at {path}: run paper_2004_00546_gb300.build.build()")
    L = ctypes.CDLL(path)
    p, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "pxa_create": [ctypes.POINTER(p), i, p],
        "pxa_destroy": [p],
        "pxa_last_error": [p],
        "pxa_set_operator": [p, ctypes.POINTER(OperatorDesc)],
        "pxa_set_time": [p, d, i64, i, i],
        "pxa_set_krylov": [p, i, d, i, i],
        "pxa_set_magnus": [p, i],
        "pxa_set_control": [p, p, d],
        "pxa_set_target": [p, p],
        "pxa_set_objective": [p, ctypes.POINTER(ObjectiveDesc)],
        "pxa_set_precision": [p, i],
        "pxa_set_memory": [p, i],
        "pxa_set_adjoint": [p, i],
        "pxa_set_overlap": [p, i],
        "pxa_set_partition": [p, d],
        "pxa_set_checkpoints": [p, i],
        "pxa_set_lane_steps": [p, i],
        "pxa_set_propagator": [p, i, i],
        "pxa_partition_bounds": [i64, i, d, i, ctypes.POINTER(i64)],
        "pxa_set_groups": [p, i, i],
        "pxa_set_graph": [p, i],
        "pxa_set_cluster": [p, i, i, i],
        "pxa_autotune": [p, i, p, p],
        "pxa_solve_direct": [p, i, p],
        "pxa_rk4_lanes_2d": [p, i, i64, p, p],
        "pxa_cn_lanes_1d": [p, i, i64, p, p],
        "pxa_spmv_csr": [p, i64, p, p, p, p, p],
        "pxa_solve_adjoint": [p, i, p],
        "pxa_set_timing": [p, i],
        "pxa_gradient": [p, i, p, p],
        "pxa_gradient_async": [p, i, p, p],
        "pxa_sync": [p],
        "pxa_gradient_host": [p, i, p, p, p],
        "pxa_get_stats": [p, ctypes.POINTER(Stats)],
        "pxa_set_wait_limit": [p, i64],
        "pxa_direct_state": [p, p, p],
        "pxa_nl_paraexp": [p, p, d, i, p, p, ctypes.POINTER(i)],
        "pxa_wait_probe": [p],
        "pxa_apply_operator": [p, i, p, p],
        "pxa_step": [p, i, i64, p, p],
        "pxa_expv": [p, i, i64, i, p, p, p],
        "pxa_burgers_rhs": [p, p, p],
        "pxa_burgers_jac_T": [p, p, p, p],
        "pxa_expv_static": [i, p, ctypes.POINTER(OperatorDesc), d, i64, i, d, i, i, i64, i, p, p, p],
        "pxa_batch_create": [ctypes.POINTER(p), i, p],
        "pxa_batch_destroy": [p],
        "pxa_batch_last_error": [p],
        "pxa_batch_set": [p, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(d), d, d, d, i64, i],
        "pxa_batch_set_krylov": [p, i, d, d],
        "pxa_batch_set_graph": [p, i],
        "pxa_batch_set_schedule": [p, i],
        "pxa_batch_set_homogeneous": [p, d],
        "pxa_batch_set_power": [p, i],
        "pxa_batch_set_lane_steps": [p, i],
        "pxa_batch_set_timing": [p, i],
        "pxa_batch_gradient": [p, i, p, p, p],
        "pxa_batch_sync": [p],
        "pxa_batch_autotune": [p, i, p, p, p, ctypes.POINTER(d)],
        "pxa_batch_offsets": [p, ctypes.POINTER(i64)],
        "pxa_batch_problem_info": [p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)],
        "pxa_batch_get_stats": [p, ctypes.POINTER(BatchStats)],
    }
    for name, argt in sig.items():
        fn = getattr(L, name)
        fn.argtypes = argt
        fn.restype = (None if name in ("pxa_destroy", "pxa_batch_destroy") else
                      ctypes.c_char_p if name in ("pxa_last_error", "pxa_batch_last_error") else i)
    _lib = L
    return L


def _dptr(t) -> ctypes.c_void_p:
    """Device pointer of a CUDA float64 contiguous torch tensor."""
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _tptr(t, dtype) -> ctypes.c_void_p:
    """Device pointer of a contiguous CUDA tensor of the given torch dtype."""
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous CUDA {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a) -> ctypes.c_void_p:
    import numpy as np

    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float64 numpy array")
    return a.ctypes.data_as(ctypes.c_void_p)


class Context:
    """One pxa_ctx on one device, bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self._L = load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._stream = stream
        h = ctypes.c_void_p()
        self._check(self._L.pxa_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream)),
                    ctx=None)
        self._h = h
        self._keep = {}

    # -- plumbing --------------------------------------------------------------------
    def _check(self, rc, ctx="self"):
        if rc != OK:
            msg = ""
            if ctx is not None and getattr(self, "_h", None):
                msg = self._L.pxa_last_error(self._h).decode()
            raise PxaError(rc, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._L.pxa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration ---------------------------------------------------------------
    def set_operator(self, kind, n, L=6.283185307179586, c=0.0, nu=0.0):
        desc = OperatorDesc(kind, n, L, c, nu, 0, 0, None, None, None, None, None)
        self._check(self._L.pxa_set_operator(self._h, ctypes.byref(desc)))
        self.n = n

    def set_operator_2d(self, nx, ny, u, v, nu, L=6.283185307179586):
        """2D advection-diffusion with a frozen velocity (u, v: CUDA float64 (ny, nx))."""
        self._keep["u"], self._keep["v"] = u, v
        desc = OperatorDesc(ADVDIFF_2D, nx * ny, L, 0.0, nu, nx, ny, _dptr(u).value, _dptr(v).value, None, None,
                            None)
        self._check(self._L.pxa_set_operator(self._h, ctypes.byref(desc)))
        self.n = nx * ny

    def set_operator_burgers_2d(self, n, nu, L=6.283185307179586):
        """2D viscous Burgers on an n x n periodic grid; control and gradient hold 2 n^2
        values (u then v)."""
        desc = OperatorDesc(BURGERS_2D, 2 * n * n, L, 0.0, nu, n, n, None, None, None, None, None)
        self._check(self._L.pxa_set_operator(self._h, ctypes.byref(desc)))
        self.n = 2 * n * n

    def direct_state(self, ic, out):
        """BURGERS_2D: q(T) of the direct solve from ic into out (CUDA float64, 2 n^2)."""
        self._check(self._L.pxa_direct_state(self._h, _dptr(ic), _dptr(out)))

    def set_operator_csr(self, row_ptr, col, val):
        """General sparse operator A (CSR on the device: int64 row_ptr[n + 1], int32 col,
        float64 val), borrowed until the next set_operator."""
        import torch

        n = int(row_ptr.numel()) - 1
        self._keep["csr"] = (row_ptr, col, val)
        desc = OperatorDesc(CSR, n, 0.0, 0.0, 0.0, 0, 0, None, None, _tptr(row_ptr, torch.int64).value,
                            _tptr(col, torch.int32).value, _dptr(val).value)
        self._check(self._L.pxa_set_operator(self._h, ctypes.byref(desc)))
        self.n = n

    def set_objective(self, kind, target=None):
        self._keep["target"] = target
        desc = ObjectiveDesc(kind, None if target is None else _dptr(target).value)
        self._check(self._L.pxa_set_objective(self._h, ctypes.byref(desc)))

    def set_precision(self, precision):
        self._check(self._L.pxa_set_precision(self._h, int(precision)))

    def set_time(self, T, K, stepper, P):
        self._check(self._L.pxa_set_time(self._h, T, int(K), stepper, int(P)))

    def set_krylov(self, m, tol, phi, substeps=1):
        self._check(self._L.pxa_set_krylov(self._h, int(m), tol, phi, int(substeps)))

    def set_magnus(self, steps_per_magnus):
        self._check(self._L.pxa_set_magnus(self._h, int(steps_per_magnus)))

    def set_control(self, control, omega=0.0):
        self._keep["control"] = control
        self._check(self._L.pxa_set_control(self._h, _dptr(control), omega))

    def set_target(self, target):
        self._keep["target"] = target
        self._check(self._L.pxa_set_target(self._h, _dptr(target)))

    def set_memory(self, policy):
        self._check(self._L.pxa_set_memory(self._h, policy))

    def set_adjoint(self, impl):
        self._check(self._L.pxa_set_adjoint(self._h, impl))

    def set_overlap(self, enable):
        self._check(self._L.pxa_set_overlap(self._h, 1 if enable else 0))

    def set_propagator(self, method, max_degree=120):
        self._check(self._L.pxa_set_propagator(self._h, method, max_degree))

    def set_partition(self, r):
        self._check(self._L.pxa_set_partition(self._h, float(r)))

    def set_lane_steps(self, q):
        """CN steps per lane band application (1D advection-diffusion): 1, 2, 4 or 0 (auto)."""
        self._check(self._L.pxa_set_lane_steps(self._h, int(q)))

    def set_checkpoints(self, intervals):
        """Multi-checkpoint scheme (Sec. 3.5) with `intervals` equal intervals (0: off)."""
        self._check(self._L.pxa_set_checkpoints(self._h, int(intervals)))

    def set_groups(self, q_direct=0, q_sweep=0):
        self._check(self._L.pxa_set_groups(self._h, q_direct, q_sweep))

    def set_cluster(self, direct=0, lanes=0, chain=0):
        self._check(self._L.pxa_set_cluster(self._h, int(direct), int(lanes), int(chain)))

    def set_graph(self, enable):
        self._check(self._L.pxa_set_graph(self._h, int(bool(enable))))

    def set_timing(self, enable):
        self._check(self._L.pxa_set_timing(self._h, int(bool(enable))))

    def set_wait_limit(self, cycles):
        """Limit of the bounded device waits in SM cycles (0: the default, 2^31)."""
        self._check(self._L.pxa_set_wait_limit(self._h, int(cycles)))

    def nl_paraexp(self, traj, guess=None, tol=1e-12, max_iter=50):
        """Alg. 2 for the configured Burgers problem: the last iterate into traj (CUDA
        float64 (K+1, n)); returns (changes per iteration, converged). Raises PxaError for
        a non-finite iterate or a set-up error."""
        import numpy as np

        ch = np.zeros(int(max_iter))
        it = ctypes.c_int(0)
        rc = self._L.pxa_nl_paraexp(self._h, None if guess is None else _dptr(guess), float(tol), int(max_iter),
                                    _dptr(traj), ch.ctypes.data_as(ctypes.c_void_p), ctypes.byref(it))
        if rc not in (OK, ERR_NOT_CONVERGED):
            self._check(rc)
        return ch[:it.value].copy(), rc == OK

    def wait_probe(self):
        """Runs the failure path of the bounded waits; raises PxaError(ERR_TIMEOUT)."""
        self._check(self._L.pxa_wait_probe(self._h))

    # -- solves ------------------------------------------------------------------------
    def gradient(self, mode, grad) -> float:
        J = ctypes.c_double()
        self._check(self._L.pxa_gradient(self._h, mode, ctypes.byref(J), _dptr(grad)))
        return J.value

    def solve_direct(self, mode) -> float:
        J = ctypes.c_double()
        self._check(self._L.pxa_solve_direct(self._h, mode, ctypes.byref(J)))
        return J.value

    def solve_adjoint(self, mode, grad):
        self._check(self._L.pxa_solve_adjoint(self._h, mode, _dptr(grad)))

    def gradient_async(self, mode, J_dev, grad):
        self._check(self._L.pxa_gradient_async(self._h, mode, _dptr(J_dev), _dptr(grad)))

    def sync(self):
        self._check(self._L.pxa_sync(self._h))

    def gradient_host(self, mode, control_host, grad_host) -> float:
        J = ctypes.c_double()
        self._check(self._L.pxa_gradient_host(self._h, mode, _hptr(control_host), ctypes.byref(J),
                                              _hptr(grad_host)))
        return J.value

    def autotune(self, mode, grad) -> float:
        ms = ctypes.c_double()
        self._check(self._L.pxa_autotune(self._h, mode, _dptr(grad), ctypes.byref(ms)))
        return ms.value

    def stats(self) -> dict:
        s = Stats()
        self._check(self._L.pxa_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def cluster_sizes(self):
        s = self.stats()
        return s["cluster_direct"], s["cluster_lanes"], s["cluster_chain"]

    # -- building blocks -----------------------------------------------------------------
    def apply_operator(self, x, y, transpose=False):
        self._check(self._L.pxa_apply_operator(self._h, int(transpose), _dptr(x), _dptr(y)))

    def step(self, x, y, steps, transpose=False):
        self._check(self._L.pxa_step(self._h, int(transpose), int(steps), _dptr(x), _dptr(y)))

    def expv(self, x, y, span_steps, substeps=1, transpose=False) -> float:
        err = ctypes.c_double()
        self._check(self._L.pxa_expv(self._h, int(transpose), int(span_steps), int(substeps),
                                     _dptr(x), _dptr(y), ctypes.byref(err)))
        return err.value

    def cn_lanes_1d(self, lanes, steps, out=None) -> float:
        ms = ctypes.c_double()
        self._check(self._L.pxa_cn_lanes_1d(self._h, lanes, int(steps), _dptr(out) if out is not None else None,
                                            ctypes.byref(ms)))
        return ms.value

    def rk4_lanes_2d(self, lanes, steps, out=None) -> float:
        ms = ctypes.c_double()
        self._check(self._L.pxa_rk4_lanes_2d(self._h, int(lanes), int(steps),
                                             None if out is None else _dptr(out), ctypes.byref(ms)))
        return ms.value

    def burgers_rhs(self, u, y):
        self._check(self._L.pxa_burgers_rhs(self._h, _dptr(u), _dptr(y)))

    def burgers_jac_T(self, u, x, y):
        self._check(self._L.pxa_burgers_jac_T(self._h, _dptr(u), _dptr(x), _dptr(y)))


def expv_static(x, y, n, c, nu, T, K, m, tol, phi, span_steps, substeps=1, transpose=False,
                L=6.283185307179586, device=0, stream=None) -> float:
    """pxa_expv_static: the Krylov propagation of Context.expv with the library's fixed
    device scratch array instead of an allocated workspace (see include/pxa.h)."""
    import torch

    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    desc = OperatorDesc(ADVDIFF_1D, n, L, c, nu)
    err = ctypes.c_double()
    rc = lib.pxa_expv_static(device, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(desc), T,
                             int(K), int(m), tol, phi, int(transpose), int(span_steps), int(substeps),
                             _dptr(x), _dptr(y), ctypes.byref(err))
    if rc != OK:
        raise PxaError(rc, "pxa_expv_static")
    return err.value


def spmv_csr(row_ptr, col, val, x, y, stream=None):
    """pxa_spmv_csr: y = A x for A in CSR form (int64 row_ptr, int32 col, float64 val and
    vectors, all CUDA tensors), asynchronous on the stream."""
    import torch

    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    rc = lib.pxa_spmv_csr(ctypes.c_void_p(stream.cuda_stream), int(row_ptr.numel() - 1),
                          _tptr(row_ptr, torch.int64), _tptr(col, torch.int32), _dptr(val), _dptr(x), _dptr(y))
    if rc != OK:
        raise PxaError(rc, "pxa_spmv_csr")


def partition_bounds(K, P, r, max_chunks=8):
    """pxa_partition_bounds: chunk boundaries (in steps) of the overlapped direct solve
    (host only, no device work)."""
    lib = load()
    out = (ctypes.c_int64 * (max_chunks + 1))()
    rc = lib.pxa_partition_bounds(int(K), int(P), float(r), int(max_chunks), out)
    if rc < 0:
        raise PxaError(rc, "pxa_partition_bounds")
    return [out[i] for i in range(rc + 1)]


class Batch:
    """Batches of independent 1D advection-diffusion problems (pxa_batch_* in
    include/pxa.h): argument marshalling only."""

    def __init__(self, device=0, stream=None):
        self._L = load()
        self._h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        rc = self._L.pxa_batch_create(ctypes.byref(self._h), device, s)
        if rc != OK:
            raise PxaError(rc, "pxa_batch_create")
        self.count = 0

    def _check(self, rc):
        if rc != OK:
            raise PxaError(rc, self._L.pxa_batch_last_error(self._h).decode())

    def close(self):
        if self._h:
            self._L.pxa_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set(self, n, nu, c=1.0, L=6.283185307179586, T=1.0, K=4096, P=16):
        import numpy as np

        n = np.ascontiguousarray(n, dtype=np.int32)
        nu = np.ascontiguousarray(nu, dtype=np.float64)
        self.count = len(n)
        self._check(self._L.pxa_batch_set(self._h, self.count,
                                          n.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                          nu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          c, L, T, int(K), int(P)))

    def set_krylov(self, m=30, tol=1e-8, reach=0.04):
        self._check(self._L.pxa_batch_set_krylov(self._h, m, tol, reach))

    def set_timing(self, enable):
        self._check(self._L.pxa_batch_set_timing(self._h, 1 if enable else 0))

    def set_homogeneous(self, ratio):
        self._check(self._L.pxa_batch_set_homogeneous(self._h, float(ratio)))

    def set_lane_steps(self, q):
        """CN steps per lane band application: 1, 2, 4, or 0 (automatic)."""
        self._check(self._L.pxa_batch_set_lane_steps(self._h, int(q)))

    def set_power(self, enable):
        """Apply the stepper's subinterval propagator as one band of M^(K/P) (1) or step it (0)."""
        self._check(self._L.pxa_batch_set_power(self._h, 1 if enable else 0))

    def set_graph(self, enable):
        self._check(self._L.pxa_batch_set_graph(self._h, 1 if enable else 0))

    def set_schedule(self, one_launch):
        """1: the whole Paraexp gradient as one persistent launch (default); 0: phases."""
        self._check(self._L.pxa_batch_set_schedule(self._h, 1 if one_launch else 0))

    def gradient_async(self, mode, q0, J, grad):
        self._check(self._L.pxa_batch_gradient(self._h, mode, _dptr(q0), _dptr(J), _dptr(grad)))

    def sync(self):
        self._check(self._L.pxa_batch_sync(self._h))

    def gradient(self, mode, q0, J, grad):
        self.gradient_async(mode, q0, J, grad)
        self.sync()

    def autotune(self, mode, q0, J, grad) -> float:
        ms = ctypes.c_double()
        self._check(self._L.pxa_batch_autotune(self._h, mode, _dptr(q0), _dptr(J), _dptr(grad),
                                               ctypes.byref(ms)))
        return ms.value

    def offsets(self):
        out = (ctypes.c_int64 * (self.count + 1))()
        self._check(self._L.pxa_batch_offsets(self._h, out))
        return [out[i] for i in range(self.count + 1)]

    def problem_info(self):
        """Per problem: FP32 lane band taps, FP64 band taps, Krylov (1) or stepped (0)."""
        a = (ctypes.c_int * self.count)()
        b = (ctypes.c_int * self.count)()
        k = (ctypes.c_int * self.count)()
        self._check(self._L.pxa_batch_problem_info(self._h, a, b, k))
        return list(a), list(b), list(k)

    def stats(self) -> dict:
        s = BatchStats()
        self._check(self._L.pxa_batch_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in BatchStats._fields_}
