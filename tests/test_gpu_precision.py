"""Reduced-precision far field (BF16 / FP16 U,V with FP32 accumulation), the FP32
refinement sweeps, and the tcgen05 multi-right-hand-side apply.

Errors against the FP64 oracle are stated per precision: the FP32 path is held
to 1e-4; BF16 and FP16 storage have their own bounds (BF16 keeps 8 significant
bits per factor entry, FP16 11); refinement brings the solve back to 1e-4.
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def apply(op, X, dtype=torch.float32):
    Xd = torch.tensor(X, dtype=dtype, device=DEV)
    Y = torch.zeros_like(Xd)
    op.apply(Xd, Y)
    torch.cuda.synchronize()
    return Y.double().cpu().numpy()


@pytest.mark.parametrize("far,bound", [(rt.RT_PREC_BF16, 3e-3), (rt.RT_PREC_F16, 1e-4)])
def test_low_precision_far_field_apply_error(far, bound):
    p = W.cube_problem(12, W.sinprod_kappa(0.5), W.midpoint_freqs(4, albedo=0.3), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams(far_prec=far))
    X = W.rand_vectors((4, p.N), seed=2)
    err = rel_l2(apply(op, X), O.DenseOperator(p).apply(X))
    assert err < bound, err
    op.free()


@pytest.mark.parametrize("far", [rt.RT_PREC_BF16, rt.RT_PREC_F16])
def test_refined_low_precision_solve_reaches_fp32_accuracy(far):
    p = W.cube_problem(12, W.sinprod_kappa(0.5), W.midpoint_freqs(4, albedo=0.3), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams(far_prec=far, refine=1))
    J = torch.zeros(4, p.N, dtype=torch.float32, device=DEV)
    T = torch.zeros(p.N, dtype=torch.float64, device=DEV)
    st = op.solve_fixed_point(J, T, tol=1e-6, max_iter=300, check_every=2, refine_tol=1e-3)
    ref = O.fixed_point(p, O.DenseOperator(p), tol=1e-10)
    assert st["converged"] == 1
    assert rel_l2(T.cpu().numpy(), ref["T"]) < 1e-5
    assert rel_l2(J.cpu().numpy(), ref["J"]) < 1e-4
    op.free()


@pytest.mark.parametrize("far", [rt.RT_PREC_BF16, rt.RT_PREC_F16])
@pytest.mark.parametrize("n,F", [(12, 16), (16, 32)])
def test_tensor_core_apply_matches_cuda_core_apply(far, n, F):
    """One operator for all F frequencies (kappa_nu = kappa): the tcgen05 apply and the
    CUDA-core apply of the same BF16/FP16 operator agree (the right-hand sides keep ~16
    bits through the hi/lo split)."""
    p = W.cube_problem(n, W.sinprod_kappa(0.5), W.midpoint_freqs(F, albedo=0.3, c_offset=None), R0=0.5)
    X = W.rand_vectors((F, p.N), seed=3)
    op_tc = rt.rt_build_operator(p, rt.hparams(far_prec=far))
    op_cc = rt.rt_build_operator(p, rt.hparams(far_prec=far, tensor_cores=1))
    y_tc = apply(op_tc, X)
    y_cc = apply(op_cc, X)
    assert rel_l2(y_tc, y_cc) < 2e-4, rel_l2(y_tc, y_cc)
    # both against the FP64 oracle at the far-field precision
    ref = O.DenseOperator(p).apply(X)
    assert rel_l2(y_tc, ref) < (3e-3 if far == rt.RT_PREC_BF16 else 1e-4)
    op_tc.free()
    op_cc.free()


@pytest.mark.parametrize("far,bound", [(rt.RT_PREC_BF16, 3e-3), (rt.RT_PREC_F16, 2e-4)])
def test_tensor_core_apply_at_64_right_hand_sides_matches_the_oracle(far, bound):
    """The 64-right-hand-side tile width of the 64^3 workload on a 20^3 mesh (several
    column clusters per M = 128 tile, ragged leaves): the tcgen05 apply against dense FP64
    oracle rows at 200 sampled vertices, per far-field precision."""
    F = 64
    p = W.cube_problem(20, W.sinprod_kappa(0.5), W.midpoint_freqs(F, albedo=0.3, c_offset=None), R0=0.5)
    op = rt.rt_build_operator(p, rt.hparams(far_prec=far))
    assert op.info()["apply_tensor_cores"] == 1
    X = W.rand_vectors((F, p.N), seed=4)
    Y = apply(op, X)
    rows = W.sample_rows(p.N, 200, seed=5)
    R = O.G_rows(p, rows)[:, 0, :]          # one operator group: [rows, N]
    ref = (R @ X.T).T                        # [F, rows]
    err = rel_l2(Y[:, rows], ref)
    assert err < bound, err
    op.free()


@pytest.fixture(scope="module")
def cube64_golden():
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "cube64_F64s_apply_rows1000.npz"))
    return g["rows"], g["Y"]


@pytest.mark.parametrize("far,bound", [(rt.RT_PREC_BF16, 2e-4), (rt.RT_PREC_F16, 1e-4)])
def test_64cube_tensor_core_apply_on_1000_stored_oracle_rows(cube64_golden, far, bound):
    """The 64^3 workload (262144 vertices, one operator, 64 right-hand sides) on the streamed
    tcgen05 path against 1000 dense FP64 oracle rows stored by tests/golden/make_golden.py
    for X = rand_vectors((64, N), seed=0): BF16 and FP16 far fields, each with its bound."""
    rows, ref = cube64_golden
    p = W.shared_kappa_64()
    np.testing.assert_array_equal(rows, W.sample_rows(p.N, 1000, seed=0))
    op = rt.rt_build_operator(p, rt.hparams(far_prec=far))
    try:
        assert op.info()["apply_tensor_cores"] == 1
        Y = apply(op, W.rand_vectors((64, p.N), seed=0))
        err = rel_l2(Y[:, rows], ref)
        assert err < bound, err
    finally:
        op.free()
