"""pxa_expv_static: the allocation-free Krylov entry point.

Some callers cannot allocate device memory (a plugin inside an application that
owns all device memory, a real-time loop with a footprint fixed at start-up). For
them libpxa keeps the Krylov basis in one fixed device array and this entry point
takes only the caller's input and output vectors. The test calls it through the
C ABI twice in a row and checks each result against the context-based pxa_expv
on the same input and against the oracle's exact propagator (the naive-DFT
diagonalisation of the circulant operator), within the tolerance the other Krylov
tests use (1e-10, element-wise); that the device's free memory does not change
across the two calls; and that oversized requests are refused before any device
work. The file is named to be collected last.
"""
import numpy as np
import pytest

import oracle as O
from paper_2004_00546_gb300 import inputs as I
from parity import rel

pytestmark = pytest.mark.gpu


def test_expv_static_matches_context_expv_and_oracle_twice(cuda_ok):
    import torch

    from paper_2004_00546_gb300 import pxa as X

    n, c, nu, T, K, m, span = 256, 1.0, 0.01, 1.0, 4096, 30, 512
    for phi in (X.PHI_EXP, X.PHI_STEPPER):
        ctx = X.Context()
        ctx.set_operator(X.ADVDIFF_1D, n, c=c, nu=nu)
        ctx.set_time(T, K, X.CN, 8)
        ctx.set_krylov(m, 1e-10, phi, 1)
        xs = [torch.as_tensor(I.grf_k2(n, seed), device="cuda") for seed in (3, 4)]
        y_refs = [torch.empty_like(x) for x in xs]
        ys = [torch.full_like(x, float("nan")) for x in xs]
        for call, x in enumerate(xs):
            ctx.expv(x, y_refs[call], span, substeps=2, transpose=bool(call))
        # set-up call (looks up the fixed array's device address), then the two calls
        X.expv_static(xs[0], ys[0], n, c, nu, T, K, m, 1e-10, phi, span, substeps=2)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        errs = []
        for call, x in enumerate(xs):  # two calls in a row, different inputs
            errs.append(X.expv_static(x, ys[call], n, c, nu, T, K, m, 1e-10, phi, span, substeps=2,
                                      transpose=bool(call)))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        for call, x in enumerate(xs):
            a, b = ys[call].cpu().numpy(), y_refs[call].cpu().numpy()
            assert rel(a, b) < 1e-10
            v = x.cpu().numpy()
            if phi == X.PHI_EXP:
                exact = O.ad1_phi_dft(v, c, nu, O.PHI_EXP, t=span * T / K, transpose=bool(call))
            else:
                exact = O.ad1_phi_dft(v, c, nu, O.PHI_CN, dt=T / K, steps=span, transpose=bool(call))
            assert rel(a, exact) < 1e-10
            assert 0.0 <= errs[call] < 1e-10
        ctx.close()


def test_expv_static_rejects_oversized_requests(cuda_ok):
    import torch

    from paper_2004_00546_gb300 import pxa as X

    n, m = 4096, 40  # a basis of 4096 * 41 doubles does not fit in the fixed array
    assert n * (m + 1) > X.EXPV_STATIC_MAX_DOUBLES - 64
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.full_like(x, 7.0)
    torch.cuda.synchronize()
    with pytest.raises(X.PxaError) as ei:
        X.expv_static(x, y, n, 1.0, 0.01, 1.0, 4096, m, 1e-10, X.PHI_EXP, 64)
    assert ei.value.code == X.ERR_TOO_LARGE
    assert bool((y == 7.0).all())  # refused before any device work: the output is untouched
