"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/rt.h declares, and the host-side cluster/block tree (Section 2.1)
satisfies its invariants."""
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


def test_tree_order_keeps_leaves_spatially_compact():
    xyz, _ = W.cube_mesh(16)
    perm, blocks, _ = rt.rt_plan(xyz, 64, 2.0)
    dense = blocks[blocks[:, 4] == 0]
    for r0, m, _, _, _ in dense:
        p = xyz[perm[r0:r0 + m]]
        ext = p.max(axis=0) - p.min(axis=0)
        assert ext.max() <= 4.0 / 15 + 1e-12
