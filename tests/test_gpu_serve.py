"""Serving: requests admitted continuously under an HBM budget.

Each result is the same whether the request ran alone or in a mix of
concurrent requests (relative L2 <= 1e-5 on T and J with the FP32 far field:
assembly sums quadrature contributions with shared-memory float atomics, so
two builds of one problem agree to FP32 rounding, not bitwise), and matches
the FP64 oracle's fixed point (T within 1e-5 for FP32, 1e-4 for the BF16
far field with high + low refinement sweeps).  The budget is never exceeded.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2306_05789_gb300 as rt
import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_05789_gb300 import build
    build.build()
    O.build()


def small_requests():
    """Six requests of differing sizes, frequency counts, kappa amplitudes and walls."""
    out = []
    for k, (n, F, amp, R0) in enumerate([(9, 2, 0.6, 0.7), (7, 1, 0.2, 0.0), (10, 3, 0.8, 0.9), (8, 2, 0.4, 0.5),
                                         (11, 1, 0.0, 0.3), (9, 3, 0.5, 0.9)]):
        out.append(W.cube_problem(n, W.sinprod_kappa(amp), W.midpoint_freqs(F, albedo=0.3, c_offset=0.5), R0=R0,
                                  name=f"req{k}"))
    return out


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def serve(probs, hp, slots, budget=120 * 10**9, one_by_one=False, **kw):
    srv = rt.Server(hp, hbm_budget=budget, slots=slots, tol=1e-7, **kw)
    res = []
    if one_by_one:
        for p in probs:
            res.append(srv.poll(srv.submit(p), wait_ms=-1))
    else:
        ids = [srv.submit(p) for p in probs]
        res = [srv.poll(i, wait_ms=-1) for i in ids]
    info = srv.info()
    srv.free()
    return res, info


def test_each_result_is_the_same_alone_and_in_the_mix():
    probs = small_requests()
    hp = rt.hparams(leaf=32)
    mix, imix = serve(probs, hp, slots=4)
    alone, ialone = serve(probs, hp, slots=1, one_by_one=True)
    assert imix["finished"] == len(probs) and imix["failed"] == 0
    assert imix["max_running"] >= 2          # the mix really overlapped on the device
    assert ialone["max_running"] == 1
    for (Jm, Tm, im), (Ja, Ta, ia) in zip(mix, alone):
        assert im["status"] == 0 and im["converged"] == 1
        assert rel_l2(Tm, Ta) <= 1e-5
        assert rel_l2(Jm, Ja) <= 1e-5
        assert abs(im["iters"] - ia["iters"]) <= 1
        assert im["t_submit"] <= im["t_admit"] <= im["t_built"] <= im["t_done"]
    for k in (0, 2):
        ref = O.fixed_point(probs[k], O.DenseOperator(probs[k]), tol=1e-10)
        assert rel_l2(mix[k][1], ref["T"]) <= 1e-5
        assert rel_l2(mix[k][0], ref["J"]) <= 1e-4


def test_budget_is_never_exceeded_and_queued_requests_wait():
    probs = small_requests()
    hp = rt.hparams(leaf=32)
    first, _ = serve(probs[:1], hp, slots=1)
    est = max(r[2]["est_bytes"] for r in first)
    # room for about one request at its assembly peak: the rest queue
    budget = int(est * 1.2)
    res, info = serve([probs[0]] * 4, hp, slots=4, budget=budget)
    assert info["finished"] == 4 and info["failed"] == 0
    assert info["peak_reserved_bytes"] <= budget
    assert info["reserved_bytes"] == 0 and info["running"] == 0 and info["queued"] == 0
    # a second copy fits only once the first has finished: one on the device at a time
    assert info["max_running"] == 1
    admits = sorted(r[2]["t_admit"] for r in res)
    dones = sorted(r[2]["t_done"] for r in res)
    assert all(admits[k] >= dones[k - 1] for k in range(1, 4))
    for r in res:
        assert r[2]["peak_bytes"] > 0 and r[2]["resident_bytes"] > 0
        assert rel_l2(r[1], res[0][1]) <= 1e-5


def test_bf16_far_field_with_refinement_matches_the_oracle():
    probs = small_requests()[:3]
    hp = rt.hparams(leaf=32, far_prec=rt.RT_PREC_BF16, refine=1)
    res, info = serve(probs, hp, slots=3, refine_tol=1e-3)
    assert info["failed"] == 0
    for p, (J, T, i) in zip(probs, res):
        ref = O.fixed_point(p, O.DenseOperator(p), tol=1e-10)
        assert rel_l2(T, ref["T"]) <= 1e-4
        assert rel_l2(J, ref["J"]) <= 1e-4


def test_request_errors_do_not_stop_the_server():
    srv = rt.Server(rt.hparams(leaf=32), hbm_budget=120 * 10**9, slots=2, tol=1e-7, max_iter=2)
    p = small_requests()[0]
    rid = srv.submit(p)
    J, T, info = srv.poll(rid, wait_ms=-1, raise_on_error=False)
    assert info["status"] == rt.RT_ENOCONV and info["iters"] == 2
    srv.free()
    res, _ = serve([p], rt.hparams(leaf=32), slots=1)
    assert res[0][2]["status"] == 0


def test_served_requests_with_walls_grids_and_opaque_boxes():
    """The server copies everything a request points to (further walls, the kappa
    grid, the opaque boxes) at submission: a mix of a Test-3 geometry request, a
    two-wall request with its corner path and a plain one, submitted from arrays
    that are released right after submission, gives the results of direct solves;
    the Test-3 request also matches the FP64 oracle's one-step residual."""
    koba = W.kobayashi_problem(0.05)
    walls = W.cube_problem(8, W.sinprod_kappa(0.5), W.midpoint_freqs(2, albedo=0.3), R0=0.5)
    walls.more_walls = (W.wall_y0(0.4),)
    walls.corner = True
    plain = small_requests()[0]
    probs = [koba, walls, plain]
    hp = rt.hparams(leaf=32)
    srv = rt.Server(hp, slots=3, tol=1e-7)
    ids = []
    for p in probs:
        ids.append(srv.submit(p))   # the marshalled arrays die with the call's temporaries
    res = [srv.poll(i, wait_ms=-1) for i in ids]
    srv.free()
    dev = torch.device("cuda:0")
    for p, (J, T, info) in zip(probs, res):
        op = rt.rt_build_operator(p, hp)
        Jd = torch.zeros(p.freqs.F, p.N, dtype=torch.float32, device=dev)
        Td = torch.zeros(p.N, dtype=torch.float64, device=dev)
        op.solve_fixed_point(Jd, Td, tol=1e-7, max_iter=400, check_every=4)
        op.free()
        assert rel_l2(T, Td.cpu().numpy()) < 1e-5, p.name
        assert rel_l2(J, Jd.cpu().numpy()) < 1e-5, p.name
    J, T, _ = res[0]
    rows = W.sample_rows(koba.N, 24, seed=61)
    r = O.one_step_residual(koba, rows, J.astype(np.float64), T)
    assert np.linalg.norm(r) / np.linalg.norm(J[:, rows]) < 1e-5
