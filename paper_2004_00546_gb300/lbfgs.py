"""L-BFGS driver for the direct-adjoint loop (Sec. 2: the gradient drives an iterative
optimisation of the control).

Two-loop recursion of limited-memory BFGS (Nocedal & Wright, Numerical Optimization,
2nd ed., Alg. 7.4) with an Armijo backtracking line search. The iterates, directions
and history stay on the device as torch tensors; each objective and gradient
evaluation is one call through the C ABI (pxa_solve_direct / pxa_gradient).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import pxa as X


@dataclass
class LbfgsResult:
    control: torch.Tensor
    J: list = field(default_factory=list)          # objective at each accepted iterate
    grad_norm: list = field(default_factory=list)  # ||grad|| at each accepted iterate
    evals: int = 0                                 # direct solves (objective evaluations)
    iterates: list = field(default_factory=list)   # copies of the accepted controls (if kept)


def _objective(ctx, control, mode):
    ctx.set_control(control, getattr(ctx, "_omega", 0.0))
    return ctx.solve_direct(mode)


def _gradient(ctx, control, mode, grad):
    ctx.set_control(control, getattr(ctx, "_omega", 0.0))
    return ctx.gradient(mode, grad)


def minimize(ctx, control0, iters=20, mode=X.PARAEXP, history=6, c1=1e-4, max_backtracks=30,
             keep_iterates=False, omega=0.0):
    """Minimise J(control) on a configured Context. Returns an LbfgsResult."""
    ctx._omega = omega
    x = control0.detach().clone().contiguous()
    g = torch.empty_like(x)
    J = _gradient(ctx, x, mode, g)
    res = LbfgsResult(control=x)
    res.J.append(J)
    res.grad_norm.append(float(torch.linalg.vector_norm(g)))
    res.evals = 1
    if keep_iterates:
        res.iterates.append(x.clone())
    S, Y, rho = [], [], []
    for _ in range(iters):
        # two-loop recursion: d = -H g
        q = g.clone()
        alpha = []
        for s, y, r in zip(reversed(S), reversed(Y), reversed(rho)):
            a = r * torch.dot(s, q)
            alpha.append(a)
            q -= a * y
        if S:
            gamma = torch.dot(S[-1], Y[-1]) / torch.dot(Y[-1], Y[-1])
            q *= gamma
        else:
            q *= 1.0 / max(float(torch.linalg.vector_norm(g)), 1e-300)
        for (s, y, r), a in zip(zip(S, Y, rho), reversed(alpha)):
            b = r * torch.dot(y, q)
            q += (a - b) * s
        d = -q
        slope = float(torch.dot(g, d))
        if slope >= 0.0:  # not a descent direction: restart from steepest descent
            S, Y, rho = [], [], []
            d = -g / max(float(torch.linalg.vector_norm(g)), 1e-300)
            slope = float(torch.dot(g, d))
        step = 1.0
        for _ in range(max_backtracks):
            xn = x + step * d
            Jn = _objective(ctx, xn, mode)
            res.evals += 1
            if Jn <= J + c1 * step * slope:
                break
            step *= 0.5
        else:
            break  # no sufficient decrease: stop
        gn = torch.empty_like(x)
        Jn = _gradient(ctx, xn, mode, gn)
        res.evals += 1
        s, y = xn - x, gn - g
        sy = float(torch.dot(s, y))
        if sy > 1e-300:
            S.append(s)
            Y.append(y)
            rho.append(1.0 / sy)
            if len(S) > history:
                S.pop(0)
                Y.pop(0)
                rho.pop(0)
        x, g, J = xn, gn, Jn
        res.J.append(J)
        res.grad_norm.append(float(torch.linalg.vector_norm(g)))
        if keep_iterates:
            res.iterates.append(x.clone())
    res.control = x
    return res
