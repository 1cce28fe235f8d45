"""Parity of the batched 1D advection-diffusion path (many problems of uneven size in one
launch per phase) with the CPU oracle, problem by problem.

Tolerances: the lanes step in FP32 (FP32 accumulation), so J and the gradient of each
problem are held to 1e-4 relative against the FP64 oracle: the oracle's serial CN for
serial stepping and for Paraexp problems whose homogeneous parts are stepped (the
stepper's own propagator reproduces serial stepping), the oracle's Paraexp with the
exact exponential of Eq. hom for problems that use the Krylov exponential (tolerance
1e-8). Problems are independent: a problem's result does not depend on the rest of the
batch, bit for bit.
"""
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


def dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def run(X, torch, prob, K, P, mode, m=30, reach=0.04, graph=True, ratio=1.0):
    b = X.Batch()
    b.set(prob["n"], prob["nu"], c=prob["c"], T=prob["T"], K=K, P=P)
    b.set_krylov(m, 1e-8, reach)
    b.set_homogeneous(ratio)
    b.set_graph(graph)
    q0 = dev(torch, prob["q0"])
    J = torch.empty(len(prob["n"]), dtype=torch.float64, device="cuda")
    g = torch.empty_like(q0)
    b.gradient(mode, q0, J, g)
    st = b.stats()
    st["krylov"] = b.problem_info()[2]
    off = b.offsets()
    b.close()
    return J.cpu().numpy(), g.cpu().numpy(), st, off


def reference(prob, off, i, K, P, krylov):
    """The oracle for problem i: serial CN, or Paraexp with the exact exponential when
    the problem's homogeneous parts use the Krylov exponential (stepped homogeneous
    parts reproduce serial stepping)."""
    q0 = prob["q0"][off[i]:off[i + 1]]
    if krylov:
        Jo, go, _ = O.ad1_cn_gradient_paraexp(q0, 1.0, prob["nu"][i], 1.0, K, P, O.PHI_EXP)
    else:
        Jo, go, _ = O.ad1_cn_gradient_serial(q0, 1.0, prob["nu"][i], 1.0, K)
    return Jo, go


@pytest.fixture(scope="module")
def small():
    # uneven grids from 16 points up, viscosities across two decades (stiff ones included)
    p = I.batch1d_problem(count=7, seed=77, n_lo=16, n_hi=320)
    p["n"][0] = 16
    p["nu"][0] = 0.1
    p["q0"] = np.concatenate([I.grf_k2(int(n), 500 + i) for i, n in enumerate(p["n"])])
    p["offsets"] = np.concatenate([[0], np.cumsum(p["n"])])
    return p


@pytest.mark.parametrize("mode,ratio", [("serial", 1.0), ("paraexp", 1e30), ("paraexp", 0.0),
                                        ("paraexp", 1.0)])
def test_batch_matches_oracle_problem_by_problem(X, torch, small, mode, ratio):
    """Serial stepping; Paraexp with every homogeneous part by the Krylov exponential, by
    stepping, and as the cost model chooses per problem."""
    K, P = 512, 8
    md = X.SERIAL if mode == "serial" else X.PARAEXP
    J, g, st, off = run(X, torch, small, K, P, md, ratio=ratio)
    assert off == list(small["offsets"])
    if mode == "paraexp" and ratio == 1e30:
        assert all(st["krylov"]) and st["krylov_problems"] == len(small["n"])
    if mode == "paraexp" and ratio == 0.0:
        assert not any(st["krylov"])
    errs = []
    for i, n in enumerate(small["n"]):
        Jo, go = reference(small, off, i, K, P, mode == "paraexp" and st["krylov"][i])
        eJ, eg = abs(J[i] - Jo) / Jo, rel(g[off[i]:off[i + 1]], go)
        errs.append((int(n), eJ, eg))
        assert eJ < 1e-4 and eg < 1e-4, errs
    if mode == "paraexp":
        assert 0.0 <= st["krylov_err_max"] <= 1e-8


def test_batch_problems_are_independent(X, torch, small):
    """The same problem alone, in the batch, and repeated gives the same bits; graph
    replay and direct launches agree bit for bit."""
    K, P = 256, 4
    Jb, gb, _, off = run(X, torch, small, K, P, X.PARAEXP)
    Je, ge, _, _ = run(X, torch, small, K, P, X.PARAEXP, graph=False)
    assert np.array_equal(Jb, Je) and np.array_equal(gb, ge)
    i = 3
    one = dict(n=small["n"][i:i + 1], nu=small["nu"][i:i + 1], c=1.0, T=1.0,
               q0=small["q0"][off[i]:off[i + 1]])
    J1, g1, _, _ = run(X, torch, one, K, P, X.PARAEXP)
    assert J1[0] == Jb[i] and np.array_equal(g1, gb[off[i]:off[i + 1]])
    three = dict(n=np.repeat(one["n"], 3), nu=np.repeat(one["nu"], 3), c=1.0, T=1.0,
                 q0=np.tile(one["q0"], 3))
    J3, g3, _, _ = run(X, torch, three, K, P, X.PARAEXP)
    assert np.all(J3 == J1[0])
    n = int(one["n"][0])
    for r in range(3):
        assert np.array_equal(g3[r * n:(r + 1) * n], g1)


def test_batch_autotune_keeps_the_tolerance(X, torch, small):
    K, P = 512, 8
    b = X.Batch()
    b.set(small["n"], small["nu"], K=K, P=P)
    q0 = dev(torch, small["q0"])
    J = torch.empty(len(small["n"]), dtype=torch.float64, device="cuda")
    g = torch.empty_like(q0)
    ms = b.autotune(X.PARAEXP, q0, J, g)
    st = b.stats()
    assert ms > 0 and st["krylov_m"] in (24, 32, 40)
    assert st["hom_ratio"] in (0.0, 0.25, 1.0, 4.0, 1e30) and st["krylov_reach"] in (0.02, 0.04)
    b.gradient(X.PARAEXP, q0, J, g)
    assert b.stats()["krylov_err_max"] <= 1e-8
    Jh, gh = J.cpu().numpy(), g.cpu().numpy()
    off = b.offsets()
    kry = b.problem_info()[2]
    for i in range(len(small["n"])):
        Jo, go = reference(small, off, i, K, P, kry[i])
        assert abs(Jh[i] - Jo) / Jo < 1e-4 and rel(gh[off[i]:off[i + 1]], go) < 1e-4
    b.close()


@pytest.mark.parametrize("K,P", [(512, 8), (1024, 16), (96, 2)])
def test_batch_propagator_band_equals_stepped_chain(X, torch, small, K, P):
    """The subinterval propagator M^(K/P) applied once per link as a circulant band (taps
    from the eigenvalues R_k^(K/P)) and the chains of K/P CN steps per link both match the
    oracle's serial stepping within the FP32-stepping tolerance, and each other. (The band
    rounds 15 times where the stepped chain rounds K/P times per link: at K = 1024, P = 16
    the band's J is 2e-6 from the oracle, the stepped chain's 4e-5.)"""
    q0 = dev(torch, small["q0"])
    nprob = len(small["n"])
    res = {}
    for power in (True, False):
        b = X.Batch()
        b.set(small["n"], small["nu"], c=small["c"], T=small["T"], K=K, P=P)
        b.set_homogeneous(0.0)
        b.set_power(power)
        J = torch.empty(nprob, dtype=torch.float64, device="cuda")
        g = torch.empty_like(q0)
        b.gradient(X.PARAEXP, q0, J, g)
        b.sync()
        st = b.stats()
        if power:
            assert st["power_problems"] == nprob and st["band_power_max"] >= 3
        else:
            assert st["power_problems"] == 0 and st["band_power_max"] == 0
        assert st["krylov_problems"] == 0
        res[power] = (J.cpu().numpy(), g.cpu().numpy(), b.offsets())
        b.close()
    off = res[True][2]
    for i in range(nprob):
        sl = slice(off[i], off[i + 1])
        Jo, go = reference(small, off, i, K, P, False)
        for power in (True, False):
            J, g, _ = res[power]
            assert abs(J[i] - Jo) / Jo < 1e-4 and rel(g[sl], go) < 1e-4, (i, power)
        assert abs(res[True][0][i] - res[False][0][i]) / Jo < 1e-4
        assert rel(res[True][1][sl], res[False][1][sl]) < 1e-4, i


@pytest.mark.parametrize("K,P", [(512, 8), (96, 16)])
def test_batch_lane_product_bands(X, torch, small, K, P):
    """Lanes that apply the band of M^q (q CN steps at a time, q = 1, 2, 4 or chosen) give
    the oracle's gradients within the FP32-stepping tolerance and agree with each other;
    q = 4 is refused when it does not divide K/P (96/16 = 6, where the choice is 2)."""
    q0 = dev(torch, small["q0"])
    nprob = len(small["n"])
    res = {}
    for q in (1, 2, 4, 0):
        b = X.Batch()
        b.set(small["n"], small["nu"], c=small["c"], T=small["T"], K=K, P=P)
        b.set_homogeneous(0.0)
        b.set_lane_steps(q)
        J = torch.empty(nprob, dtype=torch.float64, device="cuda")
        g = torch.empty_like(q0)
        if (K // P) % max(q, 1) != 0:
            with pytest.raises(X.PxaError):
                b.gradient(X.PARAEXP, q0, J, g)
            b.close()
            continue
        for mode in (X.PARAEXP, X.SERIAL):
            b.gradient(mode, q0, J, g)
            res[(q, mode)] = (J.cpu().numpy(), g.cpu().numpy())
        used = b.stats()["lane_steps"]
        assert used == (q if q else (4 if (K // P) % 4 == 0 else 2))
        off = b.offsets()
        b.close()
    for (q, mode), (J, g) in res.items():
        for i in range(nprob):
            sl = slice(off[i], off[i + 1])
            Jo, go = reference(small, off, i, K, P, False)
            assert abs(J[i] - Jo) / Jo < 1e-4 and rel(g[sl], go) < 1e-4, (q, mode, i)
            J1, g1 = res[(1, mode)]
            assert abs(J[i] - J1[i]) / Jo < 1e-4 and rel(g[sl], g1[sl]) < 1e-4, (q, mode, i)


def test_batch_rejects_bad_problems(X):
    b = X.Batch()
    with pytest.raises(X.PxaError):
        b.set([8, 64], [0.01, 0.01])  # n < 16
    with pytest.raises(X.PxaError):
        b.set([64], [0.01], K=100, P=16)  # K % P != 0
    with pytest.raises(X.PxaError):
        b.set_krylov(64, 1e-8, 0.04)  # m > 48
    b.close()


def test_batch_full_size_matches_oracle_on_a_stride(X, torch):
    """The benchmarked batch at full size (256 problems, n ~ U{128..2048}, CN K = 4096,
    P = 16, seed 2007) in the benchmark's launch configuration (the stepper's propagator
    as a band of M^(K/P), autotuned Paraexp; serial stepping), compared with the FP64
    oracle on every 16th problem, point by point. Tolerance from the arithmetic: FP32
    stepping rounds the state once per band application, so a contractive recursion of s
    steps loses at most about s u_32 (u_32 = 2^-24 = 6e-8): serial stepping's K = 4096
    steps give 2.4e-4, held to 2 K u_32 = 5e-4; Paraexp's lanes take K/P = 256 steps and
    its chains 15 band products, held to the small-case 1e-4."""
    prob = I.batch1d_problem(count=256, seed=2007)
    K, P, cnt = 4096, 16, 256
    q0 = dev(torch, prob["q0"])
    J = torch.empty(cnt, dtype=torch.float64, device="cuda")
    g = torch.empty_like(q0)
    off = prob["offsets"]
    stride = list(range(0, cnt, 16))
    oracle_serial = {}
    for i in stride:
        oracle_serial[i] = O.ad1_cn_gradient_serial(prob["q0"][off[i]:off[i + 1]], 1.0, prob["nu"][i], 1.0, K)[:2]
    for mode, tol in ((X.PARAEXP, 1e-4), (X.SERIAL, 2 * K * 2.0 ** -24)):
        b = X.Batch()
        b.set(prob["n"], prob["nu"], c=1.0, T=1.0, K=K, P=P)
        b.set_power(True)
        if mode == X.PARAEXP:
            b.autotune(mode, q0, J, g)
        b.gradient(mode, q0, J, g)
        b.sync()
        kry = b.problem_info()[2] if mode == X.PARAEXP else [0] * cnt
        assert list(b.offsets()) == list(off)
        Jh, gh = J.cpu().numpy(), g.cpu().numpy()
        b.close()
        assert np.all(np.isfinite(Jh)) and np.all(np.isfinite(gh))
        for i in stride:
            if kry[i]:
                Jo, go, _ = O.ad1_cn_gradient_paraexp(prob["q0"][off[i]:off[i + 1]], 1.0, prob["nu"][i], 1.0,
                                                      K, P, O.PHI_EXP)
            else:
                Jo, go = oracle_serial[i]
            eJ, eg = abs(Jh[i] - Jo) / Jo, rel(gh[off[i]:off[i + 1]], go)
            assert eJ < tol and eg < tol, (mode, i, int(prob["n"][i]), eJ, eg)


@pytest.mark.parametrize("K,P", [(512, 8), (96, 2), (4096, 16)])
def test_batch_one_launch_equals_the_phases(X, torch, small, K, P):
    """The one-launch schedule (a persistent grid taking dependency-ordered items: sources,
    lanes, chain + superposition, adjoint lanes, adjoint chain + gradient) gives the same
    bits as the seven-phase schedule, launched directly and as a graph replay, and the
    oracle's gradients within the FP32 tolerance."""
    q0 = dev(torch, small["q0"])
    nprob = len(small["n"])
    res, kernels = {}, {}
    for sched, graph in ((0, True), (1, True), (1, False)):
        b = X.Batch()
        b.set(small["n"], small["nu"], c=small["c"], T=small["T"], K=K, P=P)
        b.set_homogeneous(0.0)
        b.set_schedule(sched)
        b.set_graph(graph)
        J = torch.empty(nprob, dtype=torch.float64, device="cuda")
        g = torch.empty_like(q0)
        for _ in range(2):  # a second gradient reuses the queue and its counters
            b.gradient(X.PARAEXP, q0, J, g)
        b.sync()
        assert b.stats()["one_launch"] == sched
        kernels[(sched, graph)] = b.stats()["graph_kernels"]
        res[(sched, graph)] = (J.cpu().numpy(), g.cpu().numpy())
        off = b.offsets()
        b.close()
    for key in ((1, True), (1, False)):
        assert np.array_equal(res[key][0], res[(0, True)][0]) and np.array_equal(res[key][1], res[(0, True)][1])
    # the captured graphs' kernel nodes: one persistent launch against the phases' launches
    assert 1 <= kernels[(1, True)] < kernels[(0, True)]
    tol = 1e-4 if K <= 512 else 2 * K * 2.0 ** -24
    J, g = res[(1, True)]
    for i in range(nprob):
        Jo, go = reference(small, off, i, K, P, False)
        assert abs(J[i] - Jo) / Jo < tol and rel(g[off[i]:off[i + 1]], go) < tol, i
