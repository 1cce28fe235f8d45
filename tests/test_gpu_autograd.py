"""The autograd.Function: forward = direct solve, backward = Paraexp adjoint kernels.
Checked against the fused pxa_gradient, the oracle's gradient, central finite
differences on 16 random directions and torch.autograd.gradcheck."""
import numpy as np
import pytest

import oracle as O
from paper_2004_00546_gb300 import inputs as I
from parity import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(cuda_ok):
    import torch

    from paper_2004_00546_gb300 import autograd as A
    from paper_2004_00546_gb300 import pxa as X

    return torch, X, A


def ad_ctx(X, n, K, P, T=0.5, c=1.0, nu=0.02):
    ctx = X.Context()
    ctx.set_operator(X.ADVDIFF_1D, n, c=c, nu=nu)
    ctx.set_time(T, K, X.CN, P)
    ctx.set_krylov(30, 1e-11, X.PHI_STEPPER, 1)
    return ctx


def test_autograd_matches_fused_gradient_and_oracle(env):
    torch, X, A = env
    n, K, P = 128, 512, 4
    q0 = I.grf_k2(n, 31)
    ctx = ad_ctx(X, n, K, P)
    q = torch.as_tensor(q0, device="cuda").requires_grad_(True)
    J = A.objective(q, ctx)
    J.backward()
    g_auto = q.grad.detach().clone()
    g_fused = torch.empty_like(g_auto)
    J2 = ctx.gradient(X.PARAEXP, g_fused)
    assert float(J.detach()) == J2
    assert torch.equal(g_auto, g_fused)
    Jo, go, _ = O.ad1_cn_gradient_serial(q0, 1.0, 0.02, 0.5, K)
    assert abs(float(J.detach()) - Jo) / Jo < 1e-10
    assert rel(g_auto.cpu().numpy(), go) < 1e-10


def test_autograd_central_fd_16_directions_linear(env):
    """Linear dynamics with a quadratic objective: the central difference is exact for
    any step, so 16 directions must match <g, d> to rounding."""
    torch, X, A = env
    n, K, P = 256, 1024, 8
    ctx = ad_ctx(X, n, K, P, T=1.0, nu=0.01)
    q = torch.as_tensor(I.grf_k2(n, 41), device="cuda").requires_grad_(True)
    A.objective(q, ctx).backward()
    g = q.grad.detach()
    rng = np.random.default_rng(16)
    with torch.no_grad():
        for _ in range(16):
            d = torch.as_tensor(rng.standard_normal(n), device="cuda")
            Jp = float(A.objective(q + d, ctx))
            Jm = float(A.objective(q - d, ctx))
            fd = (Jp - Jm) / 2.0
            dd = float(torch.dot(g, d))
            assert abs(fd - dd) <= 1e-9 * max(abs(dd), 1e-3 * abs(Jp)), (fd, dd)


def test_autograd_burgers_fd_richardson(env):
    torch, X, A = env
    n, nu, T, K, P = 96, 0.02, 0.2, 400, 4
    ctx = X.Context()
    ctx.set_operator(X.BURGERS_1D, n, nu=nu)
    ctx.set_time(T, K, X.RK4, P)
    ctx.set_krylov(20, 1e-10, X.PHI_STEPPER, 1)
    tgt = torch.as_tensor(I.fourier1d(n, 6, 52), device="cuda")
    ctx.set_target(tgt)
    f = torch.as_tensor(2.0 * I.fourier1d(n, 6, 51), device="cuda").requires_grad_(True)
    A.objective(f, ctx).backward()
    g = f.grad.detach()
    rng = np.random.default_rng(7)
    with torch.no_grad():
        for _ in range(4):
            d = torch.as_tensor(rng.standard_normal(n), device="cuda")

            def cfd(eps):
                return (float(A.objective(f + eps * d, ctx)) - float(A.objective(f - eps * d, ctx))) / (2 * eps)

            rich = (4 * cfd(1e-3) - cfd(2e-3)) / 3
            dd = float(torch.dot(g, d))
            assert abs(rich - dd) < 1e-7 * abs(dd)


def test_autograd_recomputes_when_the_context_was_reused(env):
    torch, X, A = env
    n, K, P = 64, 256, 4
    ctx = ad_ctx(X, n, K, P)
    qa = torch.as_tensor(I.grf_k2(n, 1), device="cuda").requires_grad_(True)
    qb = torch.as_tensor(I.grf_k2(n, 2), device="cuda").requires_grad_(True)
    Ja = A.objective(qa, ctx)
    Jb = A.objective(qb, ctx)  # overwrites the context's direct state
    Ja.backward()
    Jb.backward()
    ga = torch.empty_like(qa)
    ctx.set_control(qa.detach())
    ctx.gradient(X.PARAEXP, ga)
    assert torch.allclose(qa.grad, ga, rtol=0, atol=1e-14 * float(ga.abs().max()))


def test_gradcheck_small(env):
    torch, X, A = env
    n, K, P = 16, 64, 2
    ctx = ad_ctx(X, n, K, P, T=0.25, nu=0.05)
    q = torch.as_tensor(I.grf_k2(n, 5), device="cuda").requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: A.objective(x, ctx), (q,), eps=1e-6, atol=1e-8, rtol=1e-6)
