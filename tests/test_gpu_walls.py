"""Several planar reflective walls on the GPU (Section 2: each wall adds one
reflected term, its mirror image of x with weight R0 and the broken path through
the reflection point; optional corner terms for perpendicular walls, the double
reflection), against the FP64 oracle, which is pinned for these terms by the
fourfold-domain identity and the unfolded-line optical depths in
test_oracle_pins.py.

Tolerances as in test_gpu_parity.py: FP64 entries and source 1e-11 relative;
FP32 entries 2e-5 relative plus 1e-6 of the row's largest entry; H-matrix apply
and solve 1e-4 / 1e-5 in relative L2 norm."""
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


def wall_y1(R0):
    """The plane y = 1, outward normal (0, 2, 0) (not unit: the library normalises)."""
    return W.Wall((0.0, 1.0, 0.0), (0.0, 2.0, 0.0), float(R0))


def walled(n, kap, freqs, first, more, corner, grey=False):
    p = W.cube_problem(n, kap, freqs, R0=0.0, grey=grey)
    p.wall = first
    p.more_walls = tuple(more)
    p.corner = corner
    return p


# (first wall, further walls, corner): two perpendicular walls with and without the
# corner path; a first wall with R0 = 0 (its term absent) before an active one; three
# walls, two of them parallel (corner paths only for the perpendicular pairs)
CASES = {
    "zy": (W.wall_z0(0.5), [W.wall_y0(0.4)], False),
    "zy_corner": (W.wall_z0(0.5), [W.wall_y0(0.4)], True),
    "z_off_y": (W.wall_z0(0.0), [W.wall_y0(0.6)], True),
    "zyy_corner": (W.wall_z0(0.7), [W.wall_y0(0.4), wall_y1(0.3)], True),
}


_DENSE = {}


def dense_oracle(case, p):
    """The oracle's dense operator of a 10^3 case, computed once per module."""
    if case not in _DENSE:
        _DENSE[case] = O.DenseOperator(p)
    return _DENSE[case]


def entries(op, group, rows, cols):
    r = torch.tensor(np.asarray(rows, dtype=np.int32), device=DEV)
    c = torch.tensor(np.asarray(cols, dtype=np.int32), device=DEV)
    out = torch.zeros(r.numel(), dtype=torch.float64, device=DEV)
    op.eval_entries(group, r, c, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [rt.RT_PREC_F64, rt.RT_PREC_F32])
def test_entries_match_oracle_rows(case, prec):
    first, more, corner = CASES[case]
    p = walled(6, W.sinprod_kappa(0.5), W.midpoint_freqs(2, albedo=0.3), first, more, corner)
    op = rt.rt_build_operator(p, rt.hparams(mode=rt.RT_MODE_DENSE, prec=prec))
    try:
        # a corner vertex on both walls, wall vertices, interior vertices
        rows = np.array([0, 3, 7, 50, 120, 171, 215], dtype=np.int32)
        R = O.G_rows(p, rows)
        for g in range(R.shape[1]):
            got = entries(op, g, np.repeat(rows, p.N), np.tile(np.arange(p.N), len(rows))).reshape(len(rows), p.N)
            ref = R[:, g, :]
            if prec == rt.RT_PREC_F64:
                np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-16)
            else:
                tol = 2e-5 * np.abs(ref) + 1e-6 * np.abs(ref).max(axis=1, keepdims=True)
                assert (np.abs(got - ref) <= tol).all(), np.abs(got - ref).max()
    finally:
        op.free()


def test_walls_change_the_entries():
    """The further terms carry weight: dropping the second wall or the corner path moves
    the oracle rows by far more than the tolerance, so the parity above is not vacuous."""
    first, more, _ = CASES["zy_corner"]
    rows = np.array([0, 50, 171], dtype=np.int32)
    base = O.G_rows(walled(6, W.sinprod_kappa(0.5), W.midpoint_freqs(2), first, more, True), rows)
    for alt in (walled(6, W.sinprod_kappa(0.5), W.midpoint_freqs(2), first, [], False),
                walled(6, W.sinprod_kappa(0.5), W.midpoint_freqs(2), first, more, False)):
        assert np.abs(O.G_rows(alt, rows) - base).max() > 1e-3 * np.abs(base).max()


@pytest.mark.parametrize("case", ["zy_corner", "zyy_corner"])
@pytest.mark.parametrize("grey", [False, True])
def test_source_matches_oracle(case, grey):
    """Emitter vertices on one or both walls take the limit value of every term whose
    source point is x itself."""
    first, more, corner = CASES[case]
    freqs = W.grey_freqs() if grey else W.midpoint_freqs(3, albedo=0.3)
    kap = W.Kappa(W.KAPPA_CONST, 0.8, 0.0) if grey else W.sinprod_kappa(0.5)
    p = walled(6, kap, freqs, first, more, corner, grey=grey)
    op = rt.rt_build_operator(p, rt.hparams(mode=rt.RT_MODE_DENSE, prec=rt.RT_PREC_F64))
    try:
        SE = torch.zeros(p.freqs.F, p.N, dtype=torch.float64, device=DEV)
        op.source(SE)
        torch.cuda.synchronize()
        np.testing.assert_allclose(SE.cpu().numpy(), O.DenseOperator(p).SE, rtol=1e-11, atol=1e-16)
    finally:
        op.free()


@pytest.mark.parametrize("case", ["zy_corner", "zyy_corner"])
def test_hmatrix_apply_matches_dense_oracle(case):
    """The ACA column kernel and the row-over-cluster kernel (near blocks and ACA rows)
    with the further terms: the compressed apply against the oracle's dense apply."""
    first, more, corner = CASES[case]
    p = walled(10, W.sinprod_kappa(0.5), W.midpoint_freqs(3, albedo=0.3), first, more, corner)
    op = rt.rt_build_operator(p, rt.hparams(leaf=32))
    try:
        assert op.info()["n_far"] > 0
        X = W.rand_vectors((3, p.N), seed=31)
        Xd = torch.tensor(X, dtype=torch.float32, device=DEV)
        Y = torch.zeros_like(Xd)
        op.apply(Xd, Y)
        torch.cuda.synchronize()
        assert rel_l2(Y.cpu().numpy(), dense_oracle(case, p).apply(X)) < 1e-4
    finally:
        op.free()


def test_hmatrix_fixed_point_with_two_walls_and_corner():
    first, more, corner = CASES["zy_corner"]
    p = walled(10, W.sinprod_kappa(0.5), W.midpoint_freqs(3, albedo=0.3), first, more, corner)
    op = rt.rt_build_operator(p, rt.hparams(leaf=32))
    try:
        J = torch.zeros(3, p.N, dtype=torch.float32, device=DEV)
        T = torch.zeros(p.N, dtype=torch.float64, device=DEV)
        st = op.solve_fixed_point(J, T, tol=1e-6, max_iter=200, check_every=4)
        ref = O.fixed_point(p, dense_oracle("zy_corner", p), tol=1e-10)
        assert st["converged"] == 1
        assert rel_l2(T.cpu().numpy(), ref["T"]) < 1e-5
        assert rel_l2(J.cpu().numpy(), ref["J"]) < 1e-4
    finally:
        op.free()


def test_surface_to_volume_operator_with_walls_and_corner():
    """The surface-to-volume matrix with the further terms: per-vertex emitter
    coefficients against the oracle's rows (the surface hat functions on every term)."""
    first, more, corner = CASES["zyy_corner"]
    F = 2
    p = walled(10, W.sinprod_kappa(0.5), W.midpoint_freqs(F, albedo=0.3), first, more, corner)
    op = rt.rt_build_operator(p, rt.hparams(leaf=32))
    sop = rt.rt_build_source_operator(op)
    try:
        L = sop.info()["L"]
        q = np.random.default_rng(32).uniform(0.2, 1.5, L)
        Q = torch.tensor(q, dtype=torch.float32, device=DEV)
        out = torch.zeros(F, p.N, dtype=torch.float32, device=DEV)
        sop.apply(Q, out)
        torch.cuda.synchronize()
        rows = np.unique(np.concatenate([W.sample_rows(p.N, 80, seed=33), O.emitter_vertices(p)[::5]]))
        rows = rows.astype(np.int32)
        H = O.source_hat_rows(p, rows)
        _, gidx = O.groups_of(p.freqs)
        Bv = O.emitter_intensity(p) / p.Q0
        ref = np.stack([Bv[f] * (H[:, gidx[f], :] @ q) for f in range(F)])
        assert rel_l2(out.double().cpu().numpy()[:, rows], ref) < 1e-4
    finally:
        sop.free()
        op.free()


def test_too_many_walls_are_rejected():
    p = walled(4, W.sinprod_kappa(0.5), W.midpoint_freqs(1), W.wall_z0(0.5),
               [W.wall_y0(0.5), wall_y1(0.5), W.Wall((1.0, 0.0, 0.0), (1.0, 0.0, 0.0), 0.5)], False)
    with pytest.raises(rt.RtError) as e:
        rt.rt_build_operator(p, rt.hparams())
    assert e.value.code == rt.RT_EINVAL
