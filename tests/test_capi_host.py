"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/rt.h declares, the host-side cluster/block tree (Section 2.1)
satisfies its invariants, and rt_build_operator rejects invalid walls, kappa
grids, opaque boxes and binning parameters on the host (RT_EINVAL) before any
device call."""
from __future__ import annotations

import os
import re

import numpy as np
import pytest

import paper_2306_05789_gb300 as rt
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2306_05789_gb300 import build
    build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = rt.lib()
    decl = declared_functions()
    assert set(decl) == set(rt.EXPORTS)
    for name in decl:
        assert hasattr(L, name), name


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(rt, "_lib", None)
    monkeypatch.setattr(rt, "LIB_PATH", "/nonexistent/librt.so")
    with pytest.raises(ImportError):
        rt.lib()


def _clusters(xyz, perm, start, size):
    p = xyz[perm[start:start + size]]
    c = p.mean(axis=0)
    return c, np.sqrt(((p - c) ** 2).sum(axis=1)).max()


@pytest.mark.parametrize("adm", [rt.RT_ADM_GAP, rt.RT_ADM_CENTER])
@pytest.mark.parametrize("n,leaf,eta", [(8, 16, 2.0), (12, 64, 2.0), (10, 32, 0.8)])
def test_block_tree_partitions_the_matrix_and_respects_admissibility(n, leaf, eta, adm):
    xyz, _ = W.cube_mesh(n)
    N = xyz.shape[0]
    perm, blocks, (nleaf, ndense, nfar) = rt.rt_plan(xyz, leaf, eta, adm)
    assert sorted(perm.tolist()) == list(range(N))
    assert blocks.shape[0] == ndense + nfar
    cover = np.zeros((N, N), dtype=np.int32)
    for r0, m, c0, nn, kind in blocks:
        cover[r0:r0 + m, c0:c0 + nn] += 1
        ct, Rt = _clusters(xyz, perm, r0, m)
        cs, Rs = _clusters(xyz, perm, c0, nn)
        d = np.linalg.norm(ct - cs) - (Rt + Rs if adm == rt.RT_ADM_GAP else 0.0)
        ok = d > 0 and max(Rt, Rs) < eta * d
        if kind == 1:
            assert ok
        else:
            assert not ok and m <= leaf and nn <= leaf
    assert (cover == 1).all()
    assert nleaf >= N // leaf


def test_literal_eta2_admits_every_sibling_pair_on_the_cube():
    """With max(R1,R2) < 2|c1-c2| taken literally, two distinct siblings are always
    admissible on the cube: only the diagonal leaf blocks stay dense."""
    xyz, _ = W.cube_mesh(16)
    perm, blocks, (nleaf, ndense, nfar) = rt.rt_plan(xyz, 64, 2.0, rt.RT_ADM_CENTER)
    assert ndense == nleaf
    dense = blocks[blocks[:, 4] == 0]
    assert (dense[:, 0] == dense[:, 2]).all()


def test_gap_admissibility_keeps_touching_clusters_dense():
    """With the cluster-gap reading, blocks of touching leaf clusters are dense and the
    dense part is a small fraction of the matrix that shrinks with N."""
    fr = []
    for n in (16, 32):
        xyz, _ = W.cube_mesh(n)
        N = xyz.shape[0]
        perm, blocks, (nleaf, ndense, nfar) = rt.rt_plan(xyz, 64, 2.0, rt.RT_ADM_GAP)
        dense = blocks[blocks[:, 4] == 0]
        assert ndense > nleaf
        fr.append((dense[:, 1].astype(np.int64) * dense[:, 3]).sum() / N ** 2)
    assert fr[1] < fr[0] < 0.25


@pytest.mark.parametrize("kind,leaf,adm", [("cube", 64, rt.RT_ADM_GAP), ("ties", 20, rt.RT_ADM_CENTER)])
def test_plan_is_the_same_on_one_and_on_many_host_threads(monkeypatch, kind, leaf, adm):
    """Point sets of >= 32768 points build the trees on several host threads; the
    permutation and every block must equal the one-thread build exactly (large random
    sets with repeated coordinates exercise the tie-breaking by vertex id)."""
    if kind == "cube":
        xyz = W.cube_mesh(40)[0]
    else:
        rng = np.random.default_rng(8)
        xyz = rng.uniform(0.0, 1.0, (50001, 3))
        xyz[:, 0] = np.floor(xyz[:, 0] * 20) / 20
        xyz[::5, 2] = 0.5
    plans = []
    for threads in ("1", "3", "16"):
        monkeypatch.setenv("RT_PLAN_THREADS", threads)
        plans.append(rt.rt_plan(xyz, leaf, 2.0, adm))
    for perm, blocks, counts in plans[1:]:
        np.testing.assert_array_equal(perm, plans[0][0])
        np.testing.assert_array_equal(blocks, plans[0][1])
        assert counts == plans[0][2]
    perm, blocks, _ = plans[0]
    assert sorted(perm.tolist()) == list(range(xyz.shape[0]))
    # the blocks tile the matrix: their areas add up to N^2
    assert int((blocks[:, 1].astype(np.int64) * blocks[:, 3]).sum()) == xyz.shape[0] ** 2


@pytest.mark.parametrize("n,leaf", [(1, 64), (2, 1), (300, 16), (40000, 64)])
def test_plan_of_coincident_points_is_all_dense(monkeypatch, n, leaf):
    """Degenerate point sets: one point, and many copies of one point (zero radius and
    zero distance: no pair is admissible, d > 0 fails).  Every block is a dense leaf
    block, the blocks tile the matrix once, leaves hold at most `leaf` points, and the
    large case plans the same on one and on many host threads."""
    xyz = np.tile(np.array([[0.3, 0.2, 0.9]]), (n, 1))
    monkeypatch.setenv("RT_PLAN_THREADS", "1")
    perm, blocks, (nleaf, ndense, nfar) = rt.rt_plan(xyz, leaf, 2.0)
    assert nfar == 0 and ndense == blocks.shape[0] == nleaf ** 2
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert (blocks[:, 4] == 0).all() and blocks[:, 1].max() <= leaf and blocks[:, 3].max() <= leaf
    assert int((blocks[:, 1].astype(np.int64) * blocks[:, 3]).sum()) == n * n
    if n >= 32768:
        monkeypatch.setenv("RT_PLAN_THREADS", "16")
        perm2, blocks2, _ = rt.rt_plan(xyz, leaf, 2.0)
        np.testing.assert_array_equal(perm2, perm)
        np.testing.assert_array_equal(blocks2, blocks)


def test_tree_order_keeps_leaves_spatially_compact():
    xyz, _ = W.cube_mesh(16)
    perm, blocks, _ = rt.rt_plan(xyz, 64, 2.0)
    dense = blocks[blocks[:, 4] == 0]
    for r0, m, _, _, _ in dense:
        p = xyz[perm[r0:r0 + m]]
        ext = p.max(axis=0) - p.min(axis=0)
        assert ext.max() <= 4.0 / 15 + 1e-12


# ---------------------------------------------------------------------------
# input validation runs on the host before any device call (rt_build_operator
# rejects a bad problem with RT_EINVAL and a message, GPU or not)
# ---------------------------------------------------------------------------
def _rejected(prob, hp=None, fix=None):
    import ctypes
    args = rt._ProblemArgs(prob)
    if fix is not None:
        fix(args.s)
    out = ctypes.c_void_p()
    hp = hp or rt.hparams()
    rc = rt.lib().rt_build_operator(ctypes.byref(args.s), ctypes.byref(hp), None, ctypes.byref(out))
    return rc, rt.lib().rt_last_error().decode()


def _cube():
    return W.cube_problem(4, W.sinprod_kappa(0.5), W.midpoint_freqs(2), R0=0.5)


def test_more_than_three_walls_are_rejected():
    p = _cube()
    p.more_walls = (W.wall_y0(0.5), W.Wall((0, 1, 0), (0, 1, 0), 0.5), W.Wall((1, 0, 0), (1, 0, 0), 0.5))
    rc, msg = _rejected(p)
    assert rc == rt.RT_EINVAL and "n_walls" in msg


@pytest.mark.parametrize("wall,what", [(W.Wall((0, 0, 0), (0, 0, 0), 0.5), "normal"),
                                       (W.Wall((0, 0, 0), (0, -1, 0), 1.5), "R0")])
def test_bad_walls_are_rejected(wall, what):
    p = _cube()
    p.more_walls = (wall,)
    rc, msg = _rejected(p)
    assert rc == rt.RT_EINVAL and what in msg


def test_corner_flag_must_be_zero_or_one():
    def bad(s):
        s.corner = 2
    rc, msg = _rejected(_cube(), fix=bad)
    assert rc == rt.RT_EINVAL and "corner" in msg


@pytest.mark.parametrize("grid,bbox,what", [
    (-np.ones((2, 2, 2)), (0, 0, 0, 1, 1, 1), "values"),
    (np.ones((2, 2, 2)), (0, 0, 0, 1, 0, 1), "box"),
    (np.ones((1, 1, 600)), (0, 0, 0, 1, 1, 1), "dims")])
def test_bad_kappa_grids_are_rejected(grid, bbox, what):
    p = _cube()
    p.kappa = W.Kappa(W.KAPPA_GRID, 0.0, 0.0, np.asarray(grid, dtype=np.float32), bbox)
    rc, msg = _rejected(p)
    assert rc == rt.RT_EINVAL and what in msg


def test_bad_opaque_boxes_are_rejected():
    p = _cube()
    p.obstacles = (W.Box((0.5, 0.5, 0.5), (0.4, 0.6, 0.6)),)
    rc, msg = _rejected(p)
    assert rc == rt.RT_EINVAL and "hi > lo" in msg
    p.obstacles = (W.Box((0.2, 0.2, 0.2), (0.8, 0.8, 0.8)),)   # the mesh fills it
    rc, msg = _rejected(p)
    assert rc == rt.RT_EINVAL and "inside an opaque box" in msg
    p.obstacles = tuple(W.Box((2.0 + k, 0, 0), (2.5 + k, 1, 1)) for k in range(5))
    rc, msg = _rejected(p)
    assert rc == rt.RT_EINVAL and "n_obstacles" in msg


def test_kappa_bins_out_of_range_are_rejected():
    rc, msg = _rejected(_cube(), hp=rt.hparams(kappa_bins=65))
    assert rc == rt.RT_EINVAL and "kappa_bins" in msg
