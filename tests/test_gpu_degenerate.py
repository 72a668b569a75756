"""Degenerate cases of the method on the GPU, against the FP64 oracle:

* kappa = 0: the medium neither absorbs nor emits, G = 0, and the fixed point
  is the emitter source alone after one iteration (its view-factor limit is
  pinned in test_oracle_pins.py);
* no emitter: the source vanishes and so do J and T;
* pure scattering (albedo 1): the temperature balance has no weight (T = 0)
  and J solves the linear problem J = Sbar^E + G J.
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
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_05789_gb300 import build
    build.build()
    O.build()


def solve(p, hp, tol=1e-12, dt=torch.float64):
    op = rt.rt_build_operator(p, hp)
    try:
        J = torch.zeros(p.freqs.F, p.N, dtype=dt, device=DEV)
        T = torch.zeros(p.N, dtype=torch.float64, device=DEV)
        st = op.solve_fixed_point(J, T, tol=tol, max_iter=500, check_every=1)
        SE = torch.zeros(p.freqs.F, p.N, dtype=dt, device=DEV)
        op.source(SE)
        X = torch.tensor(W.rand_vectors((p.freqs.F, p.N), seed=71), dtype=dt, device=DEV)
        Y = torch.full_like(X, float("nan"))
        op.apply(X, Y)
        torch.cuda.synchronize()
        return st, J.double().cpu().numpy(), T.cpu().numpy(), SE.double().cpu().numpy(), Y.double().cpu().numpy()
    finally:
        op.free()


def test_zero_absorption_gives_the_source_alone():
    p = W.cube_problem(7, W.Kappa(W.KAPPA_CONST, 0.0, 0.0), W.midpoint_freqs(3, albedo=0.3), R0=0.5)
    st, J, T, SE, Y = solve(p, rt.hparams(mode=rt.RT_MODE_DENSE, prec=rt.RT_PREC_F64))
    assert (Y == 0).all()
    assert st["converged"] == 1
    ref = O.fixed_point(p, O.DenseOperator(p), tol=1e-12)
    np.testing.assert_allclose(J, ref["J"], rtol=1e-11, atol=1e-300)
    np.testing.assert_allclose(J, SE, rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(T, ref["T"], rtol=1e-11, atol=1e-300)


def test_no_emitter_gives_zero():
    p = W.cube_problem(8, W.sinprod_kappa(0.5), W.midpoint_freqs(2, albedo=0.3), R0=0.5)
    p.emit_tri = np.zeros((0, 3), dtype=np.int32)
    st, J, T, SE, Y = solve(p, rt.hparams(leaf=32), tol=1e-6, dt=torch.float32)
    assert st["converged"] == 1
    assert (SE == 0).all() and (J == 0).all() and (T == 0).all()
    assert np.isfinite(Y).all() and np.abs(Y).max() > 0      # the operator itself is there


def test_pure_scattering_solves_the_linear_problem_with_zero_temperature():
    p = W.cube_problem(7, W.sinprod_kappa(0.5), W.midpoint_freqs(2, albedo=1.0), R0=0.5)
    st, J, T, SE, Y = solve(p, rt.hparams(mode=rt.RT_MODE_DENSE, prec=rt.RT_PREC_F64))
    assert st["converged"] == 1
    ora = O.DenseOperator(p)
    ref = O.fixed_point(p, ora, tol=1e-12)
    assert (T == 0).all() and (ref["T"] == 0).all()
    np.testing.assert_allclose(J, ref["J"], rtol=1e-10)
    # J = Sbar^E + G J, checked through the oracle's operator
    np.testing.assert_allclose(J, ora.SE + ora.apply(J), rtol=1e-10)
