"""Seeded synthetic workloads shared by the tests, the smoke check and the benchmark.

This module holds inputs only -- geometry, coefficient fields, frequency grids,
random vectors and random instance draws.  It contains none of the method's
arithmetic (no kernel, quadrature, optical depth, Planck function or solver),
so both the FP64 oracle and the CUDA library can consume it.

Geometry follows the paper's FEM discretisation (Section 2: P1 elements on a
tetrahedral mesh of the domain, a triangulated boundary):

* ``cube_mesh(n)``: unit cube, n vertices per axis, vertex (i, j, k) at
  (i, j, k) * h with h = 1/(n-1), index i + n*j + n*n*k; each cell is split
  into 6 Kuhn tetrahedra, one per axis permutation pi:
  {c, c+e_pi0, c+e_pi0+e_pi1, c+(1,1,1)}.
* ``emitter_face_x0(n)``: the face x = 0 as triangles (the Kuhn face
  diagonals), ordered so that the right-hand normal is the outward (-x) one.
* ``wall_z0(R0)``: the reflective plane z = 0, outward normal (0, 0, -1).
* ``doubled_mesh(n)``: the cube and its mirror image in z = 0, i.e. the
  "symmetrised domain" of the academic test (Section 3.2), built by mirroring
  every tetrahedron so the lower half is the exact image of the upper half.
* ``box_mesh(dims, h, hole)``: the Kuhn mesh of a box of dims[0] x dims[1] x
  dims[2] cells of size h, with the cells of an index box removed (a
  non-convex domain, Remark 1 after Lemma 1), and ``boundary_faces`` to pick
  triangles of its boundary with the outward orientation.
* ``kobayashi_problem(h)``: the box-minus-cube geometry of the paper's Test 3
  (Section 4, after Kobayashi's test 1A): container (0, 0.6) x (0, 1) x
  (0, 0.6), radiating cube [0, 0.1]^3 opaque, its three inner faces emitting,
  three perfectly reflecting planes through the origin, a low-absorption duct
  prolonging the cube along y (lengths in metres, kappa per metre).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List

import numpy as np

KAPPA_CONST = 0
KAPPA_GRID = 2
KAPPA_SINPROD = 1

_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def cube_mesh(n: int):
    """Structured Kuhn mesh of [0,1]^3 with n vertices per axis.

    Returns (xyz float64 [N,3], tet int32 [6(n-1)^3, 4]).
    """
    if n < 2:
        raise ValueError("need at least 2 vertices per axis")
    h = 1.0 / (n - 1)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    xyz = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1).astype(np.float64)

    def vid(ii, jj, kk):
        return ii + n * jj + n * n * kk

    c = np.arange(n - 1)
    ck, cj, ci = np.meshgrid(c, c, c, indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    tets = []
    for p in _KUHN_PERMS:
        cur = [ci.copy(), cj.copy(), ck.copy()]
        v0 = vid(*cur)
        cur[p[0]] += 1
        v1 = vid(*cur)
        cur[p[1]] += 1
        v2 = vid(*cur)
        v3 = vid(ci + 1, cj + 1, ck + 1)
        tets.append(np.stack([v0, v1, v2, v3], axis=1))
    # interleave so that the 6 tetrahedra of one cell are adjacent
    tet = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return xyz, tet


def emitter_face_x0(n: int):
    """Triangles of the face x = 0, outward (-x) right-hand normal. int32 [2(n-1)^2, 3]."""
    c = np.arange(n - 1)
    kk, jj = np.meshgrid(c, c, indexing="ij")
    jj, kk = jj.ravel(), kk.ravel()

    def vid(j, k):
        return n * j + n * n * k

    a = vid(jj, kk)
    b = vid(jj + 1, kk)
    cc = vid(jj + 1, kk + 1)
    d = vid(jj, kk + 1)
    # (a, cc, b) and (a, d, cc) have normal -x
    t1 = np.stack([a, cc, b], axis=1)
    t2 = np.stack([a, d, cc], axis=1)
    return np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)


@dataclasses.dataclass
class Wall:
    """Planar reflective wall: point p, unit outward normal n, coefficient R0."""
    p: tuple = (0.0, 0.0, 0.0)
    n: tuple = (0.0, 0.0, -1.0)
    R0: float = 0.5


def wall_z0(R0: float = 0.5) -> Wall:
    return Wall((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), float(R0))


def wall_y0(R0: float = 0.5) -> Wall:
    """The reflective plane y = 0, outward normal (0, -1, 0)."""
    return Wall((0.0, 0.0, 0.0), (0.0, -1.0, 0.0), float(R0))


@dataclasses.dataclass
class Kappa:
    """kappa(x) = k0 (+ amp sin(2 pi x) sin(2 pi y) sin(2 pi z) when kind == SINPROD);
    kind == GRID: the value of the cell holding x of a grid of equal cells over
    bbox = (x0, y0, z0, x1, y1, z1), grid float32 [nz, ny, nx] (x fastest)."""
    kind: int = KAPPA_CONST
    k0: float = 1.0
    amp: float = 0.0
    grid: np.ndarray | None = None
    bbox: tuple | None = None


@dataclasses.dataclass
class Box:
    """Axis-aligned box [lo, hi]; as an obstacle it is opaque (kappa = +infinity inside)."""
    lo: tuple
    hi: tuple


@dataclasses.dataclass
class Freqs:
    """Frequency grid. kappa_nu = c[nu] * kappa(x); albedo a_nu; quadrature weight w_nu;
    optional caller-chosen operator group of each channel (None: chosen by the consumer)."""
    nu: np.ndarray
    w: np.ndarray
    c: np.ndarray
    albedo: np.ndarray
    group: np.ndarray | None = None

    @property
    def F(self) -> int:
        return int(self.nu.shape[0])


def midpoint_freqs(F: int, lo: float = 0.1, hi: float = 2.0, albedo: float = 0.3,
                   c_offset: float | None = 0.5) -> Freqs:
    """nu_k = lo + (k + 1/2) d, w_k = d, d = (hi - lo)/F.

    c_k = c_offset + nu_k (kappa_nu = kappa(x) (0.5 + nu)); c_offset=None gives
    a frequency-independent kappa_nu = kappa(x) (c_k = 1).
    """
    d = (hi - lo) / F
    nu = lo + (np.arange(F) + 0.5) * d
    w = np.full(F, d)
    c = np.ones(F) if c_offset is None else c_offset + nu
    return Freqs(nu.astype(np.float64), w.astype(np.float64), c.astype(np.float64),
                 np.full(F, float(albedo)))


def grey_freqs(albedo: float = 0.0) -> Freqs:
    """One 'grey' channel (Section 3, eq. (grey)); nu and w are unused there."""
    return Freqs(np.array([1.0]), np.array([1.0]), np.array([1.0]), np.array([float(albedo)]))


@dataclasses.dataclass
class Problem:
    """One radiative-transfer instance on a tetrahedral mesh."""
    xyz: np.ndarray
    tet: np.ndarray
    emit_tri: np.ndarray
    kappa: Kappa
    wall: Wall | None
    freqs: Freqs
    grey: bool = False
    Q0: float = 1.0
    T_emit: float = 1.0
    name: str = ""
    more_walls: tuple = ()   # further planar reflective walls (each one reflection, Section 2)
    corner: bool = False     # also the double reflections at perpendicular walls
    obstacles: tuple = ()    # opaque boxes inside the convex hull (non-convex domain)

    @property
    def N(self) -> int:
        return int(self.xyz.shape[0])


def cube_problem(n: int, kappa: Kappa, freqs: Freqs, R0: float = 0.5, grey: bool = False,
                 Q0: float = 1.0, T_emit: float = 1.0, name: str = "") -> Problem:
    """Unit cube, emitter on x = 0, reflective wall z = 0 (R0 = 0 keeps the wall off)."""
    xyz, tet = cube_mesh(n)
    return Problem(xyz, tet, emitter_face_x0(n), kappa, wall_z0(R0) if R0 > 0 else None,
                   freqs, grey, Q0, T_emit, name or f"cube{n}")


# ---------------------------------------------------------------------------
# The benchmark-shaped workloads
# ---------------------------------------------------------------------------
def plain_grey_12() -> Problem:
    """12^3 cube, kappa = 1, grey, emitter T=1 on x=0, wall z=0 with R0=0.5, dense."""
    return cube_problem(12, Kappa(KAPPA_CONST, 1.0, 0.0), grey_freqs(0.0), R0=0.5, grey=True,
                        name="cube12_grey_kappa1")


def sinprod_kappa(amp: float = 0.5) -> Kappa:
    return Kappa(KAPPA_SINPROD, 1.0, float(amp))


def multifreq_32(n: int = 32, F: int = 16) -> Problem:
    """32^3 cube, kappa = 1 + 0.5 sin sin sin, 16 midpoint frequencies in [0.1, 2],
    kappa_nu = kappa (0.5 + nu), albedo 0.3, wall z=0 with R0 = 0.5."""
    return cube_problem(n, sinprod_kappa(0.5), midpoint_freqs(F, albedo=0.3, c_offset=0.5), R0=0.5,
                        name=f"cube{n}_sinprod_F{F}")


def shared_kappa_64(n: int = 64, F: int = 64) -> Problem:
    """64^3 cube, same kappa field, 64 frequencies sharing kappa_nu = kappa(x)."""
    return cube_problem(n, sinprod_kappa(0.5), midpoint_freqs(F, albedo=0.3, c_offset=None), R0=0.5,
                        name=f"cube{n}_shared_F{F}")


def batch_instances(count: int = 256, seed: int = 0, nmin: int = 8, nmax: int = 24,
                    fmin: int = 1, fmax: int = 8, amax: float = 0.8) -> List[Problem]:
    """Independent instances: n ~ U{nmin..nmax}, F ~ U{fmin..fmax}, amplitude ~ U[0, amax],
    albedo 0.3, R0 0.5, kappa_nu = kappa (0.5 + nu)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        F = int(rng.integers(fmin, fmax + 1))
        a = float(rng.uniform(0.0, amax))
        out.append(cube_problem(n, sinprod_kappa(a), midpoint_freqs(F, albedo=0.3, c_offset=0.5),
                                R0=0.5, name=f"batch{b}_n{n}_F{F}"))
    return out


def serving_requests(count: int, rate_per_s: float = 200.0, seed: int = 0, nmin: int = 16,
                     nmax: int = 48, fmin: int = 1, fmax: int = 32, amax: float = 0.8,
                     rmax: float = 0.9):
    """Poisson arrivals (exponential gaps) of random instances.  Returns a list of
    (arrival_time_s, Problem)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        n = int(rng.integers(nmin, nmax + 1))
        F = int(rng.integers(fmin, fmax + 1))
        a = float(rng.uniform(0.0, amax))
        R0 = float(rng.uniform(0.0, rmax))
        out.append((t, cube_problem(n, sinprod_kappa(a), midpoint_freqs(F, albedo=0.3, c_offset=0.5),
                                    R0=R0, name=f"req{r}_n{n}_F{F}")))
    return out


# ---------------------------------------------------------------------------
# Test inputs
# ---------------------------------------------------------------------------
def quadrupled_mesh(n: int):
    """The cube mirrored in y = 0 and in z = 0: [0,1] x [-1,1] x [-1,1], four copies of
    every tetrahedron.  Returns (xyz [M,3], tet [4T,4], image [4][N]) with image[k][v]
    the id of vertex v mirrored by k = (flip y) + 2 (flip z); vertices on a mirror plane
    are shared."""
    xyz, tet = cube_mesh(n)
    N = xyz.shape[0]
    pts = [xyz]
    images = [np.arange(N)]
    nxt = N
    for k in (1, 2, 3):
        fy, fz = k & 1, k >> 1
        img = np.empty(N, dtype=np.int64)
        new = []
        for v in range(N):
            x = xyz[v].copy()
            if fy:
                x[1] = -x[1]
            if fz:
                x[2] = -x[2]
            # shared with an earlier copy when the flipped coordinates are zero
            same = None
            if (not fy or xyz[v, 1] == 0.0) and (not fz or xyz[v, 2] == 0.0):
                same = v
            elif fy and fz and xyz[v, 1] == 0.0:
                same = images[2][v]
            elif fy and fz and xyz[v, 2] == 0.0:
                same = images[1][v]
            if same is not None:
                img[v] = same
            else:
                img[v] = nxt
                new.append(x)
                nxt += 1
        images.append(img)
        if new:
            pts.append(np.array(new))
    qxyz = np.concatenate(pts, axis=0)
    qtet = np.concatenate([images[k][tet] for k in range(4)], axis=0).astype(np.int32)
    return qxyz, qtet, np.array(images)


def quadrupled_emitter(n: int):
    """Emitter face x = 0 of the quadrupled mesh (outward -x normal in every copy)."""
    tri = emitter_face_x0(n)
    _, _, img = quadrupled_mesh(n)
    out = [tri]
    for k in (1, 2, 3):
        t = img[k][tri]
        # one mirror flips the orientation, two restore it
        out.append(t[:, [0, 2, 1]] if k in (1, 2) else t)
    return np.concatenate(out, axis=0).astype(np.int32)


def doubled_mesh(n: int):
    """The cube [0,1]^3 together with its mirror image in z = 0 ([0,1]^2 x [-1,1]).

    Every tetrahedron of the cube is mirrored; vertices on z = 0 are shared.
    Returns (xyz [M,3], tet [2T,4], upper_index [N]) where upper_index maps the
    cube's vertex ids to ids in the doubled mesh, and mirror_index [N] gives
    the id of each vertex's mirror image."""
    xyz, tet = cube_mesh(n)
    N = xyz.shape[0]
    on_wall = xyz[:, 2] == 0.0
    low_ids = np.full(N, -1, dtype=np.int64)
    extra = np.nonzero(~on_wall)[0]
    low_ids[on_wall] = np.nonzero(on_wall)[0]
    low_ids[extra] = N + np.arange(extra.size)
    low_xyz = xyz[extra].copy()
    low_xyz[:, 2] = -low_xyz[:, 2]
    dxyz = np.concatenate([xyz, low_xyz], axis=0)
    dtet = np.concatenate([tet, low_ids[tet]], axis=0).astype(np.int32)
    return dxyz, dtet, np.arange(N), low_ids


def doubled_emitter(n: int):
    """Emitter face x = 0 of the doubled mesh (outward -x normal)."""
    tri = emitter_face_x0(n)
    _, _, _, low = doubled_mesh(n)
    # mirroring flips orientation: swap two vertices to keep the -x normal
    low_tri = low[tri][:, [0, 2, 1]]
    return np.concatenate([tri, low_tri], axis=0).astype(np.int32)


def rand_vectors(shape, seed: int = 0, kind: str = "uniform") -> np.ndarray:
    """Seeded test vectors: U[0,1] (positive, like a source) or N(0,1)."""
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.uniform(0.0, 1.0, size=shape)
    return rng.standard_normal(size=shape)


def sample_rows(N: int, count: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    count = min(count, N)
    return np.sort(rng.choice(N, size=count, replace=False)).astype(np.int32)


def kuhn_mesh_stats(n: int):
    """(N, T_e) of the cube mesh: N = n^3, T_e = 6 (n-1)^3."""
    return n ** 3, 6 * (n - 1) ** 3


# ---------------------------------------------------------------------------
# Non-convex domains: a box of Kuhn cells with a box of cells removed
# ---------------------------------------------------------------------------
def box_mesh(dims, h: float, hole=None):
    """Kuhn mesh of [0, dims[0] h] x [0, dims[1] h] x [0, dims[2] h] (dims = cells per
    axis); hole = ((i0, j0, k0), (i1, j1, k1)) removes the cells i0 <= i < i1, ... .
    Vertices that no tetrahedron uses are dropped; the rest keep the order
    i + (nx+1) (j + (ny+1) k).  Returns (xyz float64 [N, 3], tet int32 [T, 4])."""
    nx, ny, nz = (int(d) for d in dims)
    vx, vy = nx + 1, ny + 1
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    xyz = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1).astype(np.float64)

    def vid(ii, jj, kk):
        return ii + vx * (jj + vy * kk)

    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    if hole is not None:
        (i0, j0, k0), (i1, j1, k1) = hole
        keep = ~((ci >= i0) & (ci < i1) & (cj >= j0) & (cj < j1) & (ck >= k0) & (ck < k1))
        ci, cj, ck = ci[keep], cj[keep], ck[keep]
    tets = []
    for p in _KUHN_PERMS:
        cur = [ci.copy(), cj.copy(), ck.copy()]
        v0 = vid(*cur)
        cur[p[0]] += 1
        v1 = vid(*cur)
        cur[p[1]] += 1
        v2 = vid(*cur)
        v3 = vid(ci + 1, cj + 1, ck + 1)
        tets.append(np.stack([v0, v1, v2, v3], axis=1))
    tet = np.stack(tets, axis=1).reshape(-1, 4)
    used = np.zeros(xyz.shape[0], dtype=bool)
    used[tet.ravel()] = True
    new_id = np.cumsum(used) - 1
    return xyz[used].copy(), new_id[tet].astype(np.int32)


def boundary_faces(xyz, tet, select=None):
    """Boundary triangles of a tetrahedral mesh (faces of exactly one tetrahedron),
    ordered so that the right-hand normal points out of the domain.  select(centroids)
    -> bool mask keeps a subset.  int32 [K, 3]."""
    tet = np.asarray(tet, dtype=np.int64)
    faces, opp = [], []
    for a, b, c, d in ((0, 1, 2, 3), (0, 1, 3, 2), (0, 2, 3, 1), (1, 2, 3, 0)):
        faces.append(tet[:, [a, b, c]])
        opp.append(tet[:, d])
    faces = np.concatenate(faces)
    opp = np.concatenate(opp)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    inv = inv.ravel()
    once = cnt[inv] == 1
    faces, opp = faces[once], opp[once]
    P = xyz[faces]
    nrm = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    inward = np.einsum("ij,ij->i", nrm, xyz[opp] - P[:, 0]) > 0
    faces[inward] = faces[inward][:, [0, 2, 1]]
    if select is not None:
        faces = faces[np.asarray(select(xyz[faces].mean(axis=1)), dtype=bool)]
    return faces.astype(np.int32)


def kobayashi_problem(h: float = 0.05, freqs: Freqs | None = None, corner: bool = True) -> Problem:
    """Box-minus-cube geometry of the paper's Test 3 (Section 4, after Kobayashi's test 1A),
    lengths in metres: container D = (0, 0.6) x (0, 1) x (0, 0.6), opaque radiating cube
    C = [0, 0.1]^3 removed from the mesh (kappa = +infinity there), its three faces inside D
    emitting with Q0 = 0.1, perfectly reflecting planes x = 0, y = 0, z = 0 (R0 = 1, one
    reflection per wall, corner paths optional), kappa = 10 / m except 0.01 / m in the duct
    (0, 0.1) x (0.1, 1) x (0, 0.1) prolonging the cube, as a 6 x 10 x 6 grid of 0.1 m cells.
    h must divide 0.1."""
    m = int(round(0.1 / h))
    assert m >= 1 and abs(m * h - 0.1) < 1e-12
    xyz, tet = box_mesh((6 * m, 10 * m, 6 * m), h, hole=((0, 0, 0), (m, m, m)))
    eps = 1e-9

    def on_cube(cen):
        on_face = ((np.abs(cen[:, 0] - 0.1) < eps) | (np.abs(cen[:, 1] - 0.1) < eps) |
                   (np.abs(cen[:, 2] - 0.1) < eps))
        inside = (cen <= 0.1 + eps).all(axis=1)
        return on_face & inside

    emit = boundary_faces(xyz, tet, on_cube)
    grid = np.full((6, 10, 6), 10.0, dtype=np.float32)   # [z, y, x]
    grid[0, 1:, 0] = 0.01
    kap = Kappa(KAPPA_GRID, 0.0, 0.0, grid, (0.0, 0.0, 0.0, 0.6, 1.0, 0.6))
    walls = (Wall((0.0, 0.0, 0.0), (-1.0, 0.0, 0.0), 1.0), Wall((0.0, 0.0, 0.0), (0.0, -1.0, 0.0), 1.0),
             Wall((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), 1.0))
    fr = grey_freqs() if freqs is None else freqs
    return Problem(xyz, tet, emit, kap, walls[0], fr, grey=freqs is None, Q0=0.1, T_emit=1.0,
                   name=f"kobayashi_h{h:g}", more_walls=walls[1:], corner=corner,
                   obstacles=(Box((0.0, 0.0, 0.0), (0.1, 0.1, 0.1)),))
