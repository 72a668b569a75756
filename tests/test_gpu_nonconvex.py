"""A cellwise-constant kappa grid and opaque boxes (non-convex domains, Remark 1
after Lemma 1: kappa = +infinity in the convex hull outside the domain) on the
GPU, against the FP64 oracle, whose grid line integral and blocking are pinned
in test_oracle_pins.py (brute-force sampling, the opaque-slab identity, Lemma 1
row sums around an opaque cube).

Workloads: a cube with a random grid kappa; the unit box cut by an opaque slab;
the box-minus-cube geometry of the paper's Test 3 (three perfectly reflecting
planes through the origin, a low-absorption duct in the grid, the radiating
cube opaque).  Tolerances as in test_gpu_parity.py."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def entries(op, group, rows, cols):
    r = torch.tensor(np.asarray(rows, dtype=np.int32), device=DEV)
    c = torch.tensor(np.asarray(cols, dtype=np.int32), device=DEV)
    out = torch.zeros(r.numel(), dtype=torch.float64, device=DEV)
    op.eval_entries(group, r, c, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check_rows(op, p, rows, prec):
    R = O.G_rows(p, rows)
    for g in range(R.shape[1]):
        got = entries(op, g, np.repeat(rows, p.N), np.tile(np.arange(p.N), len(rows))).reshape(len(rows), p.N)
        ref = R[:, g, :]
        if prec == rt.RT_PREC_F64:
            np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-16)
        else:
            tol = 2e-5 * np.abs(ref) + 1e-6 * np.abs(ref).max(axis=1, keepdims=True)
            assert (np.abs(got - ref) <= tol).all(), np.abs(got - ref).max()
        assert ((got == 0) == (ref == 0)).all()      # the same paths are blocked


def grid_cube(n=6, F=2):
    rng = np.random.default_rng(51)
    grid = rng.uniform(0.2, 2.5, (5, 3, 4)).astype(np.float32)
    kap = W.Kappa(W.KAPPA_GRID, 0.0, 0.0, grid, (-0.05, 0.0, 0.1, 1.05, 1.0, 0.95))
    return W.cube_problem(n, kap, W.midpoint_freqs(F, albedo=0.3), R0=0.5)


def slab(opaque=True):
    xyz, tet = W.box_mesh((5, 5, 5), 0.2, hole=((2, 0, 0), (3, 5, 5)))
    emit = W.boundary_faces(xyz, tet, lambda cen: np.abs(cen[:, 0]) < 1e-9)
    obst = (W.Box((0.4, -0.1, -0.1), (0.6, 1.1, 1.1)),) if opaque else ()
    return W.Problem(xyz, tet, emit, W.Kappa(W.KAPPA_CONST, 0.9, 0.0), W.wall_z0(0.5),
                     W.midpoint_freqs(2, albedo=0.3), obstacles=obst)


@pytest.mark.parametrize("prec", [rt.RT_PREC_F64, rt.RT_PREC_F32])
def test_grid_kappa_entries_match_oracle(prec):
    p = grid_cube()
    op = rt.rt_build_operator(p, rt.hparams(mode=rt.RT_MODE_DENSE, prec=prec))
    try:
        check_rows(op, p, np.array([0, 3, 7, 50, 120, 171, 215], dtype=np.int32), prec)
    finally:
        op.free()


@pytest.mark.parametrize("prec", [rt.RT_PREC_F64, rt.RT_PREC_F32])
def test_opaque_slab_entries_and_source_match_oracle(prec):
    p = slab()
    op = rt.rt_build_operator(p, rt.hparams(mode=rt.RT_MODE_DENSE, prec=prec))
    try:
        rows = np.concatenate([W.sample_rows(p.N, 12, seed=52), [0, p.N - 1]]).astype(np.int32)
        check_rows(op, p, rows, prec)
        dt = torch.float64 if prec == rt.RT_PREC_F64 else torch.float32
        SE = torch.zeros(p.freqs.F, p.N, dtype=dt, device=DEV)
        op.source(SE)
        torch.cuda.synchronize()
        ref = O.DenseOperator(p).SE
        got = SE.double().cpu().numpy()
        if prec == rt.RT_PREC_F64:
            np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-16)
        else:
            np.testing.assert_allclose(got, ref, rtol=2e-5, atol=1e-6 * np.abs(ref).max())
        assert (got[:, p.xyz[:, 0] > 0.55] == 0).all()
    finally:
        op.free()


def test_grid_kappa_hmatrix_apply_matches_dense_oracle():
    """The admissible blocks go through ACA (at this size the kappa jumps make most of them
    fall back to dense storage, which still tests the ACA evaluations)."""
    p = grid_cube(n=10, F=3)
    op = rt.rt_build_operator(p, rt.hparams(leaf=32))
    try:
        info = op.info()
        assert info["n_far"] + info["n_dense_fallback"] > 0
        X = W.rand_vectors((3, p.N), seed=53)
        Xd = torch.tensor(X, dtype=torch.float32, device=DEV)
        Y = torch.zeros_like(Xd)
        op.apply(Xd, Y)
        torch.cuda.synchronize()
        assert rel_l2(Y.cpu().numpy(), O.DenseOperator(p).apply(X)) < 1e-4
    finally:
        op.free()


@pytest.fixture(scope="module")
def koba():
    return W.kobayashi_problem(0.05)


def test_kobayashi_entries_and_source_match_oracle(koba):
    """Box minus an opaque corner cube, three R0 = 1 planes with their corner paths, the
    duct in the kappa grid, the cube's three inner faces emitting: FP64 rows and source."""
    p = koba
    op = rt.rt_build_operator(p, rt.hparams(mode=rt.RT_MODE_DENSE, prec=rt.RT_PREC_F64))
    try:
        near_cube = np.where(np.linalg.norm(p.xyz - 0.1, axis=1) < 0.12)[0][::5]
        rows = np.unique(np.concatenate([W.sample_rows(p.N, 6, seed=54), near_cube[:6]])).astype(np.int32)
        check_rows(op, p, rows, rt.RT_PREC_F64)
        SE = torch.zeros(1, p.N, dtype=torch.float64, device=DEV)
        op.source(SE)
        torch.cuda.synchronize()
        srows = W.sample_rows(p.N, 400, seed=55)
        ref = O.source_geometric(p, srows)[:, 0] * O.emitter_intensity(p)[0]
        np.testing.assert_allclose(SE.cpu().numpy()[0, srows], ref, rtol=1e-11, atol=1e-16)
    finally:
        op.free()


def test_kobayashi_hmatrix_apply_and_solve(koba):
    """The compressed operator (visibility makes the kernel discontinuous across the cube's
    shadow) against oracle rows: the apply on 100 sampled rows and the grey fixed point's
    one-step residual on the same rows."""
    p = koba
    op = rt.rt_build_operator(p, rt.hparams())
    try:
        info = op.info()
        assert info["n_far"] + info["n_dense_fallback"] > 0
        rows = W.sample_rows(p.N, 100, seed=56)
        R = O.G_rows(p, rows)[:, 0, :]
        X = W.rand_vectors((1, p.N), seed=57)
        Xd = torch.tensor(X, dtype=torch.float32, device=DEV)
        Y = torch.zeros_like(Xd)
        op.apply(Xd, Y)
        torch.cuda.synchronize()
        assert rel_l2(Y.cpu().numpy()[0, rows], R @ X[0]) < 2e-4
        J = torch.zeros(1, p.N, dtype=torch.float32, device=DEV)
        T = torch.zeros(p.N, dtype=torch.float64, device=DEV)
        st = op.solve_fixed_point(J, T, tol=1e-7, max_iter=400, check_every=4)
        assert st["converged"] == 1
        Jh = J.double().cpu().numpy()
        res = O.one_step_residual(p, rows, Jh, T.cpu().numpy())
        print("kobayashi h=0.05:", info, "apply err", rel_l2(Y.cpu().numpy()[0, rows], R @ X[0]),
              "residual", np.linalg.norm(res) / np.linalg.norm(Jh[:, rows]))
        assert np.linalg.norm(res) / np.linalg.norm(Jh[:, rows]) < 1e-4
    finally:
        op.free()


def test_tetrahedron_inside_an_opaque_box_is_rejected():
    p = W.cube_problem(4, W.Kappa(W.KAPPA_CONST, 1.0, 0.0), W.grey_freqs(), grey=True)
    p.obstacles = (W.Box((0.3, 0.3, 0.3), (0.7, 0.7, 0.7)),)
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_operator(p, rt.hparams())
    assert e.value.code == rt.RT_EINVAL


def test_invalid_grid_is_rejected():
    p = grid_cube()
    p.kappa = W.Kappa(W.KAPPA_GRID, 0.0, 0.0, -np.ones((2, 2, 2), np.float32), (0, 0, 0, 1, 1, 1))
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_operator(p, rt.hparams())
    assert e.value.code == rt.RT_EINVAL
