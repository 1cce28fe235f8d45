"""Parity of the CSR sparse matrix-vector product with the oracle's definition: random
matrices with uneven rows (empty ones included) and the 1D advection-diffusion stencil at
2^20 rows. The GPU sums with fused multiply-adds, the oracle with separate products and
sums: rows agree to a few units of FP64 rounding."""
import numpy as np
import pytest

import oracle as O
from paper_2004_00546_gb300 import inputs as I
from parity import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X(cuda_ok):
    from paper_2004_00546_gb300 import pxa

    return pxa


@pytest.fixture(scope="module")
def torch():
    import torch as t

    return t


def _run(X, torch, rp, col, val, x):
    d = lambda a: torch.as_tensor(a, device="cuda")
    y = torch.empty(rp.size - 1, dtype=torch.float64, device="cuda")
    X.spmv_csr(d(rp), d(col), d(val), d(x), y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("n,max_row", [(1, 3), (1000, 20), (100003, 9)])
def test_spmv_random_rows_match_the_oracle(X, torch, n, max_row):
    rng = np.random.default_rng(n)
    lens = rng.integers(1 if n == 1 else 0, max_row + 1, n)
    if n > 1:
        lens[rng.integers(0, n)] = 0  # an empty row
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = rng.integers(0, n, rp[-1]).astype(np.int32)
    val = rng.standard_normal(rp[-1])
    x = rng.standard_normal(n)
    y = _run(X, torch, rp, col, val, x)
    ref = O.spmv_csr(rp, col, val, x)
    scale = np.array([np.abs(val[rp[i]:rp[i + 1]]).sum() for i in range(n)]) * np.abs(x).max() + 1e-300
    assert np.all(np.abs(y - ref) <= 8e-16 * max_row * scale)


def test_spmv_stencil_at_a_million_rows(X, torch):
    n, c, nu = 1 << 20, 1.0, 0.01
    h = 2.0 * np.pi / n
    am, a0, ap = c / (2 * h) + nu / h ** 2, -2 * nu / h ** 2, -c / (2 * h) + nu / h ** 2
    i = np.arange(n)
    col = np.stack([(i - 1) % n, i, (i + 1) % n], 1).ravel().astype(np.int32)
    val = np.tile([am, a0, ap], n)
    rp = np.arange(0, 3 * n + 1, 3, dtype=np.int64)
    q = I.grf_k2(n, 11)
    y = _run(X, torch, rp, col, val, q)
    ref = O.spmv_csr(rp, col, val, q)
    assert rel(y, ref) < 1e-13
    with pytest.raises(X.PxaError):
        X.spmv_csr(torch.zeros(1, dtype=torch.int64, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"),
                   torch.zeros(0, dtype=torch.float64, device="cuda"), torch.zeros(1, dtype=torch.float64, device="cuda"),
                   torch.zeros(1, dtype=torch.float64, device="cuda"))
