"""Batches of independent instances: the persistent all-instance apply and the
batched fixed point agree with the single-instance paths and with the FP64
oracle.  The single-instance operators are rebuilt here, and assembly sums
quadrature contributions with shared-memory float atomics (not bitwise
reproducible, and ACA may then choose other pivots), so the comparison is at
the ACA tolerance class, not bitwise."""
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
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def batch():
    probs = W.batch_instances(count=10, seed=3, nmin=5, nmax=10, fmin=1, fmax=4)
    hp = rt.hparams(leaf=32)
    b = rt.rt_build_batch(probs, hp, threads=4, tune=True)
    yield probs, hp, b
    b.free()


def test_batch_apply_equals_single_instance_apply(batch):
    probs, hp, b = batch
    X = torch.tensor(W.rand_vectors(int(b.vec_off[-1]), seed=1), dtype=torch.float32, device=DEV)
    Y = torch.zeros_like(X)
    b.apply(X, Y)
    torch.cuda.synchronize()
    for k, p in enumerate(probs):
        op = rt.rt_build_operator(p, hp)
        lo, hi = int(b.vec_off[k]), int(b.vec_off[k + 1])
        x = X[lo:hi].reshape(p.freqs.F, p.N).contiguous()
        y = torch.zeros_like(x)
        op.apply(x, y)
        torch.cuda.synchronize()
        yb = Y[lo:hi].reshape(p.freqs.F, p.N).cpu().numpy()
        ys = y.cpu().numpy()
        assert np.abs(yb - ys).max() <= 2e-5 * np.abs(ys).max()
        op.free()
    info = b.info()
    assert info["count"] == len(probs) and info["n_works"] > 0


def test_batch_solve_equals_single_instance_solves_and_oracle(batch):
    probs, hp, b = batch
    J = torch.zeros(int(b.vec_off[-1]), dtype=torch.float32, device=DEV)
    T = torch.zeros(int(b.vert_off[-1]), dtype=torch.float64, device=DEV)
    iters, st = b.solve(J, T, tol=1e-6, max_iter=200, check_every=3)
    assert st["converged"] == 1
    for k, p in enumerate(probs):
        op = rt.rt_build_operator(p, hp)
        j = torch.zeros(p.freqs.F, p.N, dtype=torch.float32, device=DEV)
        t = torch.zeros(p.N, dtype=torch.float64, device=DEV)
        s1 = op.solve_fixed_point(j, t, tol=1e-6, max_iter=200, check_every=1)
        assert abs(int(iters[k]) - s1["iters"]) <= 1
        Tk = T[int(b.vert_off[k]):int(b.vert_off[k + 1])].cpu().numpy()
        np.testing.assert_allclose(Tk, t.cpu().numpy(), rtol=1e-5)
        op.free()
        if k < 3:
            ref = O.fixed_point(p, O.DenseOperator(p), tol=1e-10)
            assert np.linalg.norm(Tk - ref["T"]) / np.linalg.norm(ref["T"]) < 1e-5


def test_bounded_wait_gives_up_with_a_timeout_status_and_the_batch_stays_usable():
    """Failure detection on the device without a fault or a hang: every phase-2 wait of the
    persistent apply is made to target a completion count that no phase-1 item provides, with
    a short clock budget.  Each wait gives up, the solve reports RT_ETIMEOUT, the context stays
    usable, and with the normal wait restored the same batch solves and matches the oracle."""
    probs = W.batch_instances(count=3, seed=5, nmin=5, nmax=7, fmin=1, fmax=2)
    b = rt.rt_build_batch(probs, rt.hparams(leaf=32), threads=3, tune=False)
    try:
        nv, nt = int(b.vec_off[-1]), int(b.vert_off[-1])
        J = torch.zeros(nv, dtype=torch.float32, device=DEV)
        T = torch.zeros(nt, dtype=torch.float64, device=DEV)
        b.set_wait(20000, unreachable=True)   # ~10 microseconds per wait
        with pytest.raises(rt.RtError) as e:
            b.solve(J, T, tol=1e-6, max_iter=2, check_every=1, use_graph=False)
        assert e.value.code == rt.RT_ETIMEOUT
        torch.cuda.synchronize()   # the context is still usable
        b.set_wait(0, unreachable=False)
        iters, st = b.solve(J, T, tol=1e-6, max_iter=300, check_every=4)
        assert st["converged"] == 1
        Th = T.cpu().numpy()
        for k, p in enumerate(probs):
            ref = O.fixed_point(p, O.DenseOperator(p), tol=1e-10)
            t = Th[int(b.vert_off[k]):int(b.vert_off[k + 1])]
            assert np.linalg.norm(t - ref["T"]) / np.linalg.norm(ref["T"]) < 1e-5
    finally:
        b.free()
