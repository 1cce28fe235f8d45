"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the benchmark.

This module holds no arithmetic of the method: only a counter-based random number
generator and the recipes that turn its draws into fields shaped like the paper's
workloads (Sec. 4.2 and 4.3: periodic fields on [0, 2*pi) or [0, 2*pi)^2).

Generator: SplitMix64 (Steele, Lea & Flood, 2014) over a counter; the state for
draw ``i`` of stream ``seed`` is ``seed * 0x9E3779B97F4A7C15 + (i + 1) * gamma``
mixed by the SplitMix64 finaliser. Uniforms take the top 53 bits; normals use the
Box–Muller transform. Everything is computed in numpy uint64 / float64 so that
x86 and Arm hosts produce identical bits.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """A counter-based stream of uniform and normal draws."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def _u64(self, count: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + 1 + count, dtype=np.uint64)
        self.counter += count
        with np.errstate(over="ignore"):
            z = self.seed * _GAMMA + idx * _GAMMA
            return _mix(z)

    def uniform(self, count: int) -> np.ndarray:
        """Uniform draws in (0, 1): (top 53 bits + 0.5) / 2^53."""
        bits = self._u64(count) >> np.uint64(11)
        return (bits.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)

    def normal(self, count: int) -> np.ndarray:
        """Standard normal draws by Box–Muller (pairs of uniforms)."""
        m = (count + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)])
        return z[:count]


TWO_PI = 2.0 * math.pi


def grid1d(n: int, L: float = TWO_PI) -> np.ndarray:
    return np.arange(n, dtype=np.float64) * (L / n)


def grf_k2(n: int, seed: int) -> np.ndarray:
    """Gaussian random field with energy spectrum ~ k^-2 on a periodic 1D grid.

    Mode amplitudes |q_k| ~ 1/k for k = 1 .. n/2-1 with independent N(0,1) real and
    imaginary parts; the mean and the Nyquist mode are zero; the field is real
    (Hermitian spectrum) and scaled to unit RMS.
    """
    s = Stream(seed)
    kmax = n // 2 - 1
    re = s.normal(kmax)
    im = s.normal(kmax)
    spec = np.zeros(n // 2 + 1, dtype=np.complex128)
    k = np.arange(1, kmax + 1, dtype=np.float64)
    spec[1 : kmax + 1] = (re + 1j * im) / k
    q = np.fft.irfft(spec, n=n)
    q -= q.mean()
    return q / math.sqrt(np.mean(q * q))


def fourier1d(n: int, kmax: int, seed: int, L: float = TWO_PI) -> np.ndarray:
    """Random Fourier series sum_{k=1..kmax} (a_k cos kx + b_k sin kx) / (1 + k^2),
    a_k, b_k ~ N(0, 1), on the periodic grid x_i = i L / n (wavenumbers in units of
    2 pi / L)."""
    s = Stream(seed)
    x = grid1d(n, L) * (TWO_PI / L)
    out = np.zeros(n)
    ab = s.normal(2 * kmax)
    for k in range(1, kmax + 1):
        a, b = ab[2 * (k - 1)], ab[2 * (k - 1) + 1]
        out += (a * np.cos(k * x) + b * np.sin(k * x)) / (1.0 + k * k)
    return out


def fourier2d(nx: int, ny: int, kmax: int, seed: int, decay: float = 1.0) -> np.ndarray:
    """Random real 2D Fourier series with |k| <= kmax (k != 0), coefficient
    N(0,1) / (1 + |k|^2)^decay, returned as an (ny, nx) array (row = y)."""
    s = Stream(seed)
    x = grid1d(nx)
    y = grid1d(ny)
    X, Y = np.meshgrid(x, y)
    out = np.zeros((ny, nx))
    for kx in range(-kmax, kmax + 1):
        for ky in range(0, kmax + 1):
            if ky == 0 and kx <= 0:
                continue
            if kx * kx + ky * ky > kmax * kmax:
                continue
            a, b = s.normal(2)
            amp = 1.0 / (1.0 + kx * kx + ky * ky) ** decay
            ph = kx * X + ky * Y
            out += amp * (a * np.cos(ph) + b * np.sin(ph))
    return out


def streamfunction_velocity(nx: int, ny: int, kmax: int, seed: int):
    """Divergence-free velocity u = d(psi)/dy, v = -d(psi)/dx of a random
    streamfunction psi with |k| <= kmax, evaluated in closed form on the grid and
    scaled so that max(|u|, |v|) = 1. Returns (u, v) as (ny, nx) arrays."""
    s = Stream(seed)
    x = grid1d(nx)
    y = grid1d(ny)
    X, Y = np.meshgrid(x, y)
    u = np.zeros((ny, nx))
    v = np.zeros((ny, nx))
    for kx in range(-kmax, kmax + 1):
        for ky in range(0, kmax + 1):
            if ky == 0 and kx <= 0:
                continue
            if kx * kx + ky * ky > kmax * kmax:
                continue
            a, b = s.normal(2)
            amp = 1.0 / (1.0 + kx * kx + ky * ky)
            ph = kx * X + ky * Y
            # psi = amp (a cos ph + b sin ph); d/dy -> ky, d/dx -> kx
            dpsi = amp * (-a * np.sin(ph) + b * np.cos(ph))
            u += ky * dpsi
            v -= kx * dpsi
    scale = max(np.abs(u).max(), np.abs(v).max())
    return u / scale, v / scale


def batch_instances(count: int, seed: int, n_lo: int = 128, n_hi: int = 2048,
                    nu_lo: float = 1e-3, nu_hi: float = 1e-1):
    """Grid sizes n ~ U{n_lo..n_hi} and viscosities nu ~ log-uniform[nu_lo, nu_hi]."""
    s = Stream(seed)
    un = s.uniform(count)
    ns = (n_lo + np.floor(un * (n_hi - n_lo + 1))).astype(np.int64)
    ns = np.minimum(ns, n_hi)
    uv = s.uniform(count)
    nus = np.exp(np.log(nu_lo) + uv * (np.log(nu_hi) - np.log(nu_lo)))
    return ns, nus


# ---- named workloads ----------------------------------------------------------
# Seeds: 2004 + workload index.

def advdiff1d_problem(n: int = 256, seed: int = 2004):
    """1D linear advection-diffusion: c = 1, nu = 0.01, T = 1, IC control q0 ~ GRF k^-2."""
    return dict(n=n, c=1.0, nu=0.01, T=1.0, q0=grf_k2(n, seed))


def burgers1d_problem(n: int = 1024, seed: int = 2005):
    """1D viscous Burgers: nu = 0.005, T = 2, zero IC, forcing f and tracking target g
    drawn as random Fourier series with k <= 16."""
    return dict(n=n, nu=0.005, T=2.0, f=fourier1d(n, 16, seed), g=fourier1d(n, 16, seed + 1000))


def batch1d_problem(count: int = 256, seed: int = 2007, n_lo: int = 128, n_hi: int = 2048):
    """Independent 1D advection-diffusion problems: c = 1, T = 1, n ~ U{n_lo..n_hi},
    nu ~ log-uniform[1e-3, 1e-1], IC control q0_i ~ GRF k^-2 (seed 1000 * seed + i);
    q0 is packed (problem i at offsets[i] .. offsets[i + 1])."""
    ns, nus = batch_instances(count, seed, n_lo, n_hi)
    q0s = [grf_k2(int(n), 1000 * seed + i) for i, n in enumerate(ns)]
    offsets = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    return dict(n=ns, nu=nus, c=1.0, T=1.0, q0=np.concatenate(q0s), offsets=offsets)


def sparse_operator(n: int, per_row: int, seed: int, shift: float = 1.0):
    """A seeded sparse n x n matrix in CSR form (int64 row pointers, int32 columns, FP64
    values) with the structure of a discretised dissipative operator: every row holds its
    diagonal and `per_row` off-diagonal entries at distinct random columns, with values
    ~ N(0, 1); the diagonal is -(sum of the row's |off-diagonal| + shift), so every
    Gershgorin disc lies in the left half-plane (the operator is stable). Columns are
    sorted within each row."""
    s = Stream(seed)
    cols, vals = [], []
    rp = [0]
    for i in range(n):
        u = s.uniform(4 * per_row + 8)
        picked = []
        for x in u:
            j = int(x * n)
            if j != i and j not in picked:
                picked.append(j)
            if len(picked) == min(per_row, n - 1):
                break
        off = s.normal(len(picked))
        diag = -(float(np.abs(off).sum()) + shift)
        entries = sorted([(i, diag)] + list(zip(picked, off.tolist())))
        cols.extend(j for j, _ in entries)
        vals.extend(v for _, v in entries)
        rp.append(len(cols))
    return (np.asarray(rp, dtype=np.int64), np.asarray(cols, dtype=np.int32),
            np.asarray(vals, dtype=np.float64))


def burgers2d_problem(n: int = 256, seed: int = 2008, kmax: int = 12, amp: float = 0.15):
    """2D viscous Burgers initial states (Sec. 4.3 shape, periodic [0, 2 pi)^2): a "true"
    initial state (u, v), each a random Fourier series with |k| <= kmax (seeds
    1000 * seed + 1, + 2) scaled to max |.| = amp, whose final state is the tracking
    target, and a different seeded state of the same kind (seeds + 3, + 4) as a test
    point. The default amplitude keeps the cell Reynolds number max|u| h / nu below 2 on
    the 256^2 grid at nu = 2e-3 (0.15 x 0.0245 / 0.002 = 1.8), without which central
    differences let the steepening fronts oscillate and blow up before T = 1. Returned
    flattened as 2 n^2 values (u then v, each (n, n) row-major)."""
    def field(s):
        f = fourier2d(n, n, kmax, 1000 * seed + s)
        return amp * f / np.abs(f).max()

    true_ic = np.concatenate([field(1).ravel(), field(2).ravel()])
    other = np.concatenate([field(3).ravel(), field(4).ravel()])
    return {"true_ic": true_ic, "other_ic": other, "n": n}
