"""pxa_expv_static: the allocation-free Krylov entry point.

Some callers cannot allocate device memory (a plugin inside an application that
owns all device memory, a real-time loop with a footprint fixed at start-up). For
them libpxa keeps the Krylov basis in one fixed device array and this entry point
takes only the caller's input and output vectors. The test calls it through the
C ABI twice in a row and checks each result against the context-based pxa_expv
on the same input, within the tolerance the other Krylov tests use (1e-10
relative); it also checks that oversized requests are refused before any device
work. The file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2004_00546_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_expv_static_matches_context_expv_twice(cuda_ok):
    import torch

    from paper_2004_00546_gb300 import pxa as X

    n, c, nu, T, K, m = 256, 1.0, 0.01, 1.0, 4096, 30
    for phi in (X.PHI_EXP, X.PHI_STEPPER):
        ctx = X.Context()
        ctx.set_operator(X.ADVDIFF_1D, n, c=c, nu=nu)
        ctx.set_time(T, K, X.CN, 8)
        ctx.set_krylov(m, 1e-10, phi, 1)
        for call, seed in enumerate((3, 4)):  # two calls in a row, different inputs
            x = torch.as_tensor(I.grf_k2(n, seed), device="cuda")
            y_ref = torch.empty_like(x)
            ctx.expv(x, y_ref, 512, substeps=2, transpose=bool(call))
            y = torch.full_like(x, float("nan"))
            err = X.expv_static(x, y, n, c, nu, T, K, m, 1e-10, phi, 512, substeps=2,
                                transpose=bool(call))
            a, b = y.cpu().numpy(), y_ref.cpu().numpy()
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10
            assert 0.0 <= err < 1e-10
        ctx.close()


def test_expv_static_rejects_oversized_requests(cuda_ok):
    import torch

    from paper_2004_00546_gb300 import pxa as X

    n, m = 4096, 40  # a basis of 4096 * 41 doubles does not fit in the fixed array
    assert n * (m + 1) > X.EXPV_STATIC_MAX_DOUBLES - 64
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(X.PxaError) as ei:
        X.expv_static(x, y, n, 1.0, 0.01, 1.0, 4096, m, 1e-10, X.PHI_EXP, 64)
    assert ei.value.code == X.ERR_TOO_LARGE
