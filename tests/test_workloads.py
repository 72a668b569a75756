"""The seeded input generators produce the geometry and draws their recipe states.

Inputs only (no GPU, no oracle): mesh volumes and closed boundaries (the
divergence theorem on the oriented boundary triangles), emitter position,
orientation and area, the box-minus-cube geometry of the paper's Test 3
(Section 4), the mirrored meshes used by the doubled- and fourfold-domain pins,
the frequency grid, and the ranges and determinism of the batch and serving
draws.
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W


def tet_volumes(xyz, tet):
    P = xyz[np.asarray(tet, dtype=np.int64)]
    e = P[:, 1:] - P[:, :1]
    return np.abs(np.linalg.det(e)) / 6.0


def tri_normals(xyz, tri):
    """Right-hand normal of each triangle, length = twice its area."""
    P = xyz[np.asarray(tri, dtype=np.int64)]
    return np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P.mean(axis=1)


def enclosed_volume(xyz, tri):
    """Divergence theorem with F(x) = x / 3 over outward-oriented boundary triangles."""
    nrm, cen = tri_normals(xyz, tri)
    return float(np.einsum("ij,ij->", cen, nrm) / 6.0)


@pytest.mark.parametrize("n", [2, 3, 6])
def test_cube_mesh_fills_the_unit_cube_and_has_a_closed_outward_boundary(n):
    xyz, tet = W.cube_mesh(n)
    assert (xyz.shape[0], tet.shape[0]) == W.kuhn_mesh_stats(n)
    assert xyz.min() == 0.0 and xyz.max() == 1.0
    vol = tet_volumes(xyz, tet)
    assert vol.min() > 0 and abs(vol.sum() - 1.0) < 1e-13
    # every vertex is used; vertex (i, j, k) h has index i + n j + n^2 k
    assert np.unique(tet).size == n ** 3
    h = 1.0 / (n - 1)
    idx = np.arange(n ** 3)
    np.testing.assert_allclose(xyz, np.stack([idx % n, (idx // n) % n, idx // (n * n)], axis=1) * h)
    bf = W.boundary_faces(xyz, tet)
    assert bf.shape[0] == 12 * (n - 1) ** 2
    nrm, _ = tri_normals(xyz, bf)
    np.testing.assert_allclose(nrm.sum(axis=0), 0.0, atol=1e-13)   # closed surface
    assert abs(enclosed_volume(xyz, bf) - 1.0) < 1e-13               # outward orientation


@pytest.mark.parametrize("n", [2, 5])
def test_emitter_face_is_x0_with_outward_normal_and_unit_area(n):
    xyz, _ = W.cube_mesh(n)
    tri = W.emitter_face_x0(n)
    assert tri.shape == (2 * (n - 1) ** 2, 3)
    assert (xyz[tri][:, :, 0] == 0.0).all()
    nrm, _ = tri_normals(xyz, tri)
    assert (nrm[:, 0] < 0).all() and np.allclose(nrm[:, 1:], 0.0)
    assert abs(0.5 * np.linalg.norm(nrm, axis=1).sum() - 1.0) < 1e-13
    # the same triangles, with the same orientation, as the mesh's own boundary on x = 0
    bf = W.boundary_faces(xyz, W.cube_mesh(n)[1], lambda c: np.abs(c[:, 0]) < 1e-12)
    key = lambda t: sorted(tuple(np.roll(r, -int(np.argmin(r)))) for r in t)   # rotation-invariant
    assert key(tri) == key(bf)


def test_cube_problem_defaults():
    p = W.cube_problem(4, W.sinprod_kappa(0.5), W.midpoint_freqs(3), R0=0.5)
    assert p.wall.R0 == 0.5 and p.wall.n == (0.0, 0.0, -1.0) and p.wall.p == (0.0, 0.0, 0.0)
    assert (p.kappa.kind, p.kappa.k0, p.kappa.amp) == (W.KAPPA_SINPROD, 1.0, 0.5)
    assert p.Q0 == 1.0 and p.T_emit == 1.0 and not p.grey
    assert W.cube_problem(4, W.sinprod_kappa(0.5), W.midpoint_freqs(3), R0=0.0).wall is None
    g = W.plain_grey_12()
    assert g.N == 12 ** 3 and g.grey and g.freqs.F == 1 and g.kappa.kind == W.KAPPA_CONST and g.kappa.k0 == 1.0


def test_midpoint_frequency_grid():
    fr = W.midpoint_freqs(16, albedo=0.3)
    d = 1.9 / 16
    np.testing.assert_allclose(fr.nu, 0.1 + (np.arange(16) + 0.5) * d, rtol=1e-15)
    np.testing.assert_allclose(fr.w, d)
    assert abs(fr.w.sum() - 1.9) < 1e-14
    np.testing.assert_allclose(fr.c, 0.5 + fr.nu)
    assert (fr.albedo == 0.3).all()
    s = W.midpoint_freqs(64, c_offset=None)
    assert (s.c == 1.0).all() and s.F == 64


def test_box_mesh_with_a_hole_is_the_box_minus_the_hole():
    xyz, tet = W.box_mesh((4, 3, 5), 0.25, hole=((1, 0, 2), (3, 2, 4)))
    vol = tet_volumes(xyz, tet)
    want = (4 * 3 * 5 - 2 * 2 * 2) * 0.25 ** 3
    assert vol.min() > 0 and abs(vol.sum() - want) < 1e-13
    assert np.unique(tet).size == xyz.shape[0]          # unused vertices dropped
    cen = xyz[tet].mean(axis=1)
    in_hole = ((cen[:, 0] > 0.25) & (cen[:, 0] < 0.75) & (cen[:, 2] > 0.5) & (cen[:, 2] < 1.0) &
               (cen[:, 1] < 0.5))
    assert not in_hole.any()
    bf = W.boundary_faces(xyz, tet)
    assert abs(enclosed_volume(xyz, bf) - want) < 1e-13


@pytest.mark.parametrize("h,nv", [(0.05, None), (1.0 / 30.0, 11164)])
def test_kobayashi_geometry(h, nv):
    p = W.kobayashi_problem(h)
    if nv is not None:
        assert p.N == nv
    vol = tet_volumes(p.xyz, p.tet)
    assert abs(vol.sum() - (0.6 * 1.0 * 0.6 - 0.1 ** 3)) < 1e-12
    lo, hi = p.xyz.min(axis=0), p.xyz.max(axis=0)
    np.testing.assert_allclose(lo, 0.0, atol=1e-15)
    np.testing.assert_allclose(hi, (0.6, 1.0, 0.6), rtol=1e-12)
    # no tetrahedron inside the radiating cube, which is the one opaque box
    cen = p.xyz[p.tet].mean(axis=1)
    assert not ((cen < 0.1 - 1e-12).all(axis=1)).any()
    assert len(p.obstacles) == 1 and p.obstacles[0].lo == (0.0, 0.0, 0.0) and p.obstacles[0].hi == (0.1, 0.1, 0.1)
    # the emitter is the cube's three faces inside the container: area 3 x 0.01, each
    # triangle's outward (domain) normal pointing into the cube
    nrm, tc = tri_normals(p.xyz, p.emit_tri)
    assert abs(0.5 * np.linalg.norm(nrm, axis=1).sum() - 0.03) < 1e-12
    assert (np.einsum("ij,ij->i", nrm, 0.05 - tc) > 0).all()
    assert (tc <= 0.1 + 1e-12).all() and (np.abs(tc - 0.1) < 1e-12).any(axis=1).all()
    # three R0 = 1 planes through the origin with outward normals -x, -y, -z; corner paths on
    walls = (p.wall,) + tuple(p.more_walls)
    assert [w.n for w in walls] == [(-1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, -1.0)]
    assert all(w.p == (0.0, 0.0, 0.0) and w.R0 == 1.0 for w in walls) and p.corner
    # kappa: 10 / m in 0.1 m cells, 0.01 / m in the duct (0, 0.1) x (0.1, 1) x (0, 0.1)
    g = p.kappa.grid
    assert p.kappa.kind == W.KAPPA_GRID and g.shape == (6, 10, 6) and g.dtype == np.float32
    assert tuple(p.kappa.bbox) == (0.0, 0.0, 0.0, 0.6, 1.0, 0.6)
    duct = np.zeros(g.shape, dtype=bool)
    duct[0, 1:, 0] = True
    assert (g[duct] == np.float32(0.01)).all() and (g[~duct] == 10.0).all()
    assert p.grey and p.Q0 == 0.1 and p.T_emit == 1.0


def test_doubled_and_quadrupled_meshes_are_mirror_images():
    n = 3
    xyz, tet = W.cube_mesh(n)
    dxyz, dtet, up, low = W.doubled_mesh(n)
    assert abs(tet_volumes(dxyz, dtet).sum() - 2.0) < 1e-13
    np.testing.assert_array_equal(dxyz[low], xyz * (1.0, 1.0, -1.0))
    assert abs(enclosed_volume(dxyz, W.boundary_faces(dxyz, dtet)) - 2.0) < 1e-13
    qxyz, qtet, img = W.quadrupled_mesh(n)
    assert abs(tet_volumes(qxyz, qtet).sum() - 4.0) < 1e-13
    for k in range(4):
        np.testing.assert_array_equal(qxyz[img[k]], xyz * (1.0, (-1.0) ** (k & 1), (-1.0) ** (k >> 1)))
    # the emitters of the mirrored meshes are the face x = 0 of the whole domain, outward
    for mxyz, tri, area in ((dxyz, W.doubled_emitter(n), 2.0), (qxyz, W.quadrupled_emitter(n), 4.0)):
        nrm, _ = tri_normals(mxyz, tri)
        assert (mxyz[tri][:, :, 0] == 0.0).all() and (nrm[:, 0] < 0).all()
        assert abs(0.5 * np.linalg.norm(nrm, axis=1).sum() - area) < 1e-13


def test_batch_draws_are_seeded_and_in_range():
    a = W.batch_instances(256, seed=0)
    b = W.batch_instances(256, seed=0)
    assert len(a) == 256
    ns = np.array([round(p.N ** (1 / 3)) for p in a])
    Fs = np.array([p.freqs.F for p in a])
    amps = np.array([p.kappa.amp for p in a])
    assert ns.min() >= 8 and ns.max() <= 24 and np.unique(ns).size > 10
    assert Fs.min() >= 1 and Fs.max() <= 8 and np.unique(Fs).size == 8
    assert amps.min() >= 0.0 and amps.max() <= 0.8 and amps.std() > 0.1
    assert all(p.N == q.N and p.freqs.F == q.freqs.F and p.kappa.amp == q.kappa.amp for p, q in zip(a, b))
    assert any(p.kappa.amp != q.kappa.amp for p, q in zip(a, W.batch_instances(256, seed=1)))
    assert all(p.wall.R0 == 0.5 and (p.freqs.albedo == 0.3).all() for p in a)


def test_serving_stream_is_poisson_at_the_stated_rate():
    reqs = W.serving_requests(400, rate_per_s=200.0, seed=0)
    t = np.array([r[0] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    # exponential gaps with mean 1/rate (400 draws: both within 3 standard errors)
    assert abs(gaps.mean() - 1 / 200) < 0.15 / 200
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.15             # coefficient of variation 1
    ns = np.array([round(p.N ** (1 / 3)) for _, p in reqs])
    Fs = np.array([p.freqs.F for _, p in reqs])
    R0 = np.array([p.wall.R0 if p.wall is not None else 0.0 for _, p in reqs])
    assert ns.min() >= 16 and ns.max() <= 48
    assert Fs.min() >= 1 and Fs.max() <= 32
    assert R0.min() >= 0.0 and R0.max() <= 0.9
    t2 = np.array([r[0] for r in W.serving_requests(50, seed=0)])
    np.testing.assert_array_equal(t2, t[:50])                     # seeded prefix


def test_random_vectors_and_sampled_rows():
    u = W.rand_vectors((4, 5000), seed=3)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    z = W.rand_vectors((4, 5000), seed=3, kind="normal")
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    np.testing.assert_array_equal(u, W.rand_vectors((4, 5000), seed=3))
    r = W.sample_rows(1000, 100, seed=5)
    assert r.dtype == np.int32 and r.size == 100 and np.unique(r).size == 100
    assert (np.diff(r) > 0).all() and r.min() >= 0 and r.max() < 1000
    assert W.sample_rows(10, 100).size == 10
