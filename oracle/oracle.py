"""FP64 CPU oracle for the integral-form RTE with a reflective wall (arXiv 2306.05789).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``err_vs_oracle`` / ``--impl reference`` legs of
``bench.py``, never by the product package.  It shares no code with the CUDA library.

Layers:

* ``rt_oracle.c`` (built into ``liboracle.so`` by :func:`build`): optical depth
  by Gauss-Legendre, the direct and reflected volume kernels, dense rows of
  the P1 operator G, the emitter source (see that file's header).
* this module: the Planck function, the per-vertex temperature solve and the
  fixed-point iteration of Section 1.3 (equation (algo)), written with numpy.

Readings of the paper taken here:

* grey case (Section 3, eq. (grey)): B(T) = sigma T^4, sigma = pi^4/15, and the
  temperature update is kappa sigma T^4 = kappa J, i.e. T = (J/sigma)^(1/4).
* multi-frequency case: the Planck balance (RTb) discretised with the grid
  weights w_nu, kappa_nu = c_nu kappa(x) (kappa(x) cancels):
  sum_nu w_nu c_nu (1 - a_nu) (J_nu - B_nu(T)) = 0, solved per vertex by
  Newton's method safeguarded by bisection.
* residual: ||J^{k+1} - J^k||_2 / ||J^{k+1}||_2 over all vertices and frequencies.
* emitter intensity Q_nu = Q0 B_nu(T_emit) (Example of Section 1), grey:
  Q0 sigma T_emit^4.
* gridded kappa: the value of the grid cell holding the point (values pass
  through float32, as the library's C ABI takes them); its optical depth is the
  exact integral along the segment.
* non-convex domains (Remark 1 after Lemma 1): opaque boxes of the convex hull
  carry kappa = +infinity; a path crossing one has infinite optical depth.

Every function here is pinned (no part is "parity unpinned"): the header of
``rt_oracle.c`` and ``tests/test_oracle_pins.py`` name the pin of each one.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SIGMA = math.pi ** 4 / 15.0  # integral of the rescaled Planck function (Section 3, eq. (grey))


def build(force: bool = False) -> str:
    """Compile rt_oracle.c with gcc + OpenMP into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


MAX_OBST = 4
MAX_GRID_DIM = 512


class _Box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class _Kappa(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("k0", ctypes.c_double), ("amp", ctypes.c_double),
                ("grid", ctypes.c_void_p), ("dims", ctypes.c_int * 3), ("glo", ctypes.c_double * 3),
                ("ghi", ctypes.c_double * 3), ("n_obst", ctypes.c_int), ("obst", _Box * MAX_OBST)]


MAX_WALLS = 3


class _Plane(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double * 3), ("n", ctypes.c_double * 3), ("R0", ctypes.c_double)]


class _Wall(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("corner", ctypes.c_int), ("w", _Plane * MAX_WALLS)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i = ctypes.c_int
        _lib.or_G_rows.argtypes = [i, P, i, P, P, P, i, P, i, i, i, P, P, P]
        _lib.or_G_entry.argtypes = [i, P, i, P, P, P, i, P, i, i, i, P]
        _lib.or_source.argtypes = [i, P, i, P, P, P, i, P, i, i, i, P, P]
        _lib.or_gauss_legendre.argtypes = [i, P, P]
        _lib.or_tet_rule.argtypes = [i, P, P]
        _lib.or_tet_rule.restype = i
        _lib.or_tri_rule.argtypes = [i, P, P]
        _lib.or_tri_rule.restype = i
        _lib.or_kappa_at.argtypes = [P, P]
        _lib.or_kappa_at.restype = ctypes.c_double
        _lib.or_blocked.argtypes = [P, P, P]
        _lib.or_blocked.restype = i
        _lib.or_optical_depth.argtypes = [P, P, P, i]
        _lib.or_optical_depth.restype = ctypes.c_double
        _lib.or_kernel_point.argtypes = [P, P, P, P, i, P, i, P, P]
        _lib.or_source_hat.argtypes = [i, P, i, P, P, i, P, P, i, P, i, i, i, P, P]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _kappa_struct(kappa, obstacles=()) -> _Kappa:
    """kappa: kind, k0, amp and, for the grid kind, ``grid`` (cell values, array
    [nz, ny, nx], x fastest) and ``bbox`` (x0, y0, z0, x1, y1, z1).  obstacles:
    opaque boxes (each with lo, hi), kappa = +infinity inside."""
    k = _Kappa()
    k.kind = int(kappa.kind)
    k.k0 = float(kappa.k0)
    k.amp = float(kappa.amp)
    grid = getattr(kappa, "grid", None)
    if grid is not None:
        g = np.ascontiguousarray(np.asarray(grid, dtype=np.float32), dtype=np.float64)
        assert g.ndim == 3 and max(g.shape) <= MAX_GRID_DIM
        k._grid = g                                # keeps the array alive with the struct
        k.grid = g.ctypes.data
        nz, ny, nx = g.shape
        k.dims[0], k.dims[1], k.dims[2] = nx, ny, nz
        bb = kappa.bbox
        for d in range(3):
            k.glo[d] = float(bb[d])
            k.ghi[d] = float(bb[3 + d])
    obstacles = list(obstacles or ())
    assert len(obstacles) <= MAX_OBST
    k.n_obst = len(obstacles)
    for o, b in enumerate(obstacles):
        for d in range(3):
            k.obst[o].lo[d] = float(b.lo[d])
            k.obst[o].hi[d] = float(b.hi[d])
    return k


def _prob_kappa(prob) -> _Kappa:
    return _kappa_struct(prob.kappa, getattr(prob, "obstacles", ()))


def problem_walls(prob):
    """The problem's planar reflective walls (first wall, then any further ones)."""
    walls = [] if getattr(prob, "wall", None) is None else [prob.wall]
    return walls + list(getattr(prob, "more_walls", ()) or ())


def _wall_struct(walls, R0_override: Optional[float] = None, corner: bool = False) -> _Wall:
    """walls: None, one wall, or a list of walls (each with p, n, R0)."""
    w = _Wall()
    if walls is None:
        walls = []
    elif not isinstance(walls, (list, tuple)):
        walls = [walls]
    assert len(walls) <= MAX_WALLS
    w.n = len(walls)
    w.corner = 1 if corner else 0
    for k, wl in enumerate(walls):
        n = np.asarray(wl.n, dtype=np.float64)
        n = n / np.linalg.norm(n)
        for d in range(3):
            w.w[k].p[d] = float(wl.p[d])
            w.w[k].n[d] = float(n[d])
        w.w[k].R0 = float(wl.R0 if R0_override is None else R0_override)
    return w


def _prob_walls(prob, R0_override=None) -> _Wall:
    return _wall_struct(problem_walls(prob), R0_override, bool(getattr(prob, "corner", False)))


# ---------------------------------------------------------------------------
# Thin wrappers over the C functions
# ---------------------------------------------------------------------------
def gauss_legendre(n: int):
    t = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss_legendre(n, _ptr(t), _ptr(w))
    return t, w


def tet_rule(which: int):
    b = np.zeros((14, 4))
    w = np.zeros(14)
    q = lib().or_tet_rule(which, _ptr(b), _ptr(w))
    return b[:q].copy(), w[:q].copy()


def tri_rule(which: int):
    b = np.zeros((7, 3))
    w = np.zeros(7)
    q = lib().or_tri_rule(which, _ptr(b), _ptr(w))
    return b[:q].copy(), w[:q].copy()


def kappa_at(kappa, p) -> float:
    k = _kappa_struct(kappa)
    p = np.ascontiguousarray(p, dtype=np.float64)
    return lib().or_kappa_at(ctypes.byref(k), _ptr(p))


def optical_depth(kappa, a, b, ngauss: int = 16, obstacles=()) -> float:
    k = _kappa_struct(kappa, obstacles)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return lib().or_optical_depth(ctypes.byref(k), _ptr(a), _ptr(b), ngauss)


def blocked(obstacles, a, b) -> bool:
    """Does the open segment (a, b) cross the interior of one of the opaque boxes?"""
    from types import SimpleNamespace
    k = _kappa_struct(SimpleNamespace(kind=0, k0=0.0, amp=0.0), obstacles)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return bool(lib().or_blocked(ctypes.byref(k), _ptr(a), _ptr(b)))


def kernel_point(kappa, wall, x, y, c, ngauss: int = 16, corner: bool = False, obstacles=()):
    """(direct[G], reflected[G]) kernel values at the point pair (x, y); reflected = the sum
    of every wall's term (and the corner terms).  wall: None, a wall or a list of walls."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    k = _kappa_struct(kappa, obstacles)
    w = _wall_struct(wall, corner=corner)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    d = np.zeros(c.shape[0])
    r = np.zeros(c.shape[0])
    lib().or_kernel_point(ctypes.byref(k), ctypes.byref(w), _ptr(x), _ptr(y), c.shape[0], _ptr(c), ngauss,
                          _ptr(d), _ptr(r))
    return d, r


def groups_of(freqs, bins: int = 0):
    """Operator groups of the frequency channels (Remark of Section 2.1: one matrix per value
    of kappa_nu, a few values representing kappa_nu piecewise constantly; Section 4, Test 2).

    Returns (c_g per group, group index of each channel).
      * freqs.group given: the caller's map; c_g = (min + max)/2 of the member scales.
      * bins = K > 0: channels binned by c into K equal-width intervals of [min c, max c]
        (empty intervals dropped, groups in interval order); c_g as above.
      * otherwise: one group per distinct c (exact equality), in order of first appearance.
    """
    c = np.asarray(freqs.c, dtype=np.float64)
    grp = getattr(freqs, "group", None)
    if grp is not None or bins > 0:
        if grp is not None:
            gidx = np.asarray(grp, dtype=np.int64).copy()
        else:
            cmin, cmax = c.min(), c.max()
            if cmax > cmin:
                b = np.floor((c - cmin) / (cmax - cmin) * bins).astype(np.int64)
            else:
                b = np.zeros(c.shape[0], dtype=np.int64)
            b = np.clip(b, 0, bins - 1)
            used = np.unique(b)
            gidx = np.searchsorted(used, b)
        G = int(gidx.max()) + 1
        cg = np.array([0.5 * (c[gidx == g].min() + c[gidx == g].max()) for g in range(G)])
        return cg, gidx
    uniq = []
    gidx = np.zeros(c.shape[0], dtype=np.int64)
    for f, cv in enumerate(c):
        for g, u in enumerate(uniq):
            if u == cv:
                gidx[f] = g
                break
        else:
            gidx[f] = len(uniq)
            uniq.append(cv)
    return np.array(uniq, dtype=np.float64), gidx


def channel_scale(freqs, cg, gidx):
    """c_f / c_{g(f)}: channel f applies (c_f / c_g) G_g -- the kappa_nu(y) factor in front keeps
    the channel's own scale while the optical depths in the exponentials use the group's."""
    return np.asarray(freqs.c, dtype=np.float64) / np.asarray(cg)[np.asarray(gidx)]


def G_rows(prob, rows, c=None, ngauss: int = 16, refine: int = 0, R0=None, moments: bool = False):
    """Dense FP64 rows of G_g for each kappa group: array [len(rows), G, N] (and moments [.., G, 4])."""
    if c is None:
        c, _ = groups_of(prob.freqs)
    c = np.ascontiguousarray(c, dtype=np.float64)
    G = c.shape[0]
    assert G <= 64
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    xyz = np.ascontiguousarray(prob.xyz, dtype=np.float64)
    tet = np.ascontiguousarray(prob.tet, dtype=np.int32)
    N = xyz.shape[0]
    out = np.zeros((rows.shape[0], G, N))
    mom = np.zeros((rows.shape[0], G, 4)) if moments else None
    k = _prob_kappa(prob)
    w = _prob_walls(prob, R0)
    lib().or_G_rows(N, _ptr(xyz), tet.shape[0], _ptr(tet), ctypes.byref(k), ctypes.byref(w), G, _ptr(c),
                    ngauss, refine, rows.shape[0], _ptr(rows), _ptr(out),
                    _ptr(mom) if moments else None)
    return (out, mom) if moments else out


def G_entry(prob, i: int, j: int, c=None, ngauss: int = 16, R0=None):
    """One entry G_g^{ij} per group, by the literal sum over the tetrahedra around vertex j."""
    if c is None:
        c, _ = groups_of(prob.freqs)
    c = np.ascontiguousarray(c, dtype=np.float64)
    xyz = np.ascontiguousarray(prob.xyz, dtype=np.float64)
    tet = np.ascontiguousarray(prob.tet, dtype=np.int32)
    out = np.zeros(c.shape[0])
    k = _prob_kappa(prob)
    w = _prob_walls(prob, R0)
    lib().or_G_entry(xyz.shape[0], _ptr(xyz), tet.shape[0], _ptr(tet), ctypes.byref(k), ctypes.byref(w),
                     c.shape[0], _ptr(c), ngauss, int(i), int(j), _ptr(out))
    return out


def source_geometric(prob, rows=None, c=None, ngauss: int = 16, refine: int = 0, R0=None):
    """Shat_g(x_i) per group (emitter source without the intensity Q_nu): [len(rows), G]."""
    if c is None:
        c, _ = groups_of(prob.freqs)
    c = np.ascontiguousarray(c, dtype=np.float64)
    xyz = np.ascontiguousarray(prob.xyz, dtype=np.float64)
    tri = np.ascontiguousarray(prob.emit_tri, dtype=np.int32)
    N = xyz.shape[0]
    rows = np.arange(N, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros((rows.shape[0], c.shape[0]))
    k = _prob_kappa(prob)
    w = _prob_walls(prob, R0)
    lib().or_source(N, _ptr(xyz), tri.shape[0], _ptr(tri), ctypes.byref(k), ctypes.byref(w), c.shape[0],
                    _ptr(c), ngauss, refine, rows.shape[0], _ptr(rows), _ptr(out))
    return out


def emitter_vertices(prob):
    """The emitter-surface vertices (columns of the surface-to-volume matrix): the distinct
    vertex ids of the emitter triangles, ascending."""
    return np.unique(np.asarray(prob.emit_tri, dtype=np.int64).ravel()).astype(np.int32)


def source_hat_rows(prob, rows, c=None, ngauss: int = 16, refine: int = 0, R0=None):
    """Rows of the surface-to-volume matrix Sbar^E_{i,l} (Section 2: Q0 replaced by the P1 hat
    function of emitter vertex l), geometric part per group: [len(rows), G, L], columns in
    the order of emitter_vertices(prob)."""
    if c is None:
        c, _ = groups_of(prob.freqs)
    c = np.ascontiguousarray(c, dtype=np.float64)
    xyz = np.ascontiguousarray(prob.xyz, dtype=np.float64)
    tri = np.ascontiguousarray(prob.emit_tri, dtype=np.int32)
    sv = emitter_vertices(prob)
    col = np.full(xyz.shape[0], -1, dtype=np.int32)
    col[sv] = np.arange(sv.shape[0], dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    L = sv.shape[0]
    out = np.zeros((rows.shape[0], c.shape[0], L))
    k = _prob_kappa(prob)
    w = _prob_walls(prob, R0)
    lib().or_source_hat(xyz.shape[0], _ptr(xyz), tri.shape[0], _ptr(tri), _ptr(col), L, ctypes.byref(k),
                        ctypes.byref(w), c.shape[0], _ptr(c), ngauss, refine, rows.shape[0], _ptr(rows), _ptr(out))
    return out


# ---------------------------------------------------------------------------
# Planck function, emitter intensity, temperature solve (RTb)
# ---------------------------------------------------------------------------
def planck(nu, T):
    """B_nu(T) = nu^3 / (exp(nu/T) - 1) (rescaled Planck function, Section 1); B_nu(0) = 0."""
    nu = np.asarray(nu, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    nu_b, T_b = np.broadcast_arrays(nu, T)
    out = np.zeros(nu_b.shape)
    pos = T_b > 0
    with np.errstate(over="ignore"):
        out[pos] = nu_b[pos] ** 3 / np.expm1(nu_b[pos] / T_b[pos])
    return out


def planck_dT(nu, T):
    """dB_nu/dT = nu^3 e^{nu/T} (nu/T^2) / (e^{nu/T}-1)^2 (0 at T = 0)."""
    nu = np.asarray(nu, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    nu_b, T_b = np.broadcast_arrays(nu, T)
    out = np.zeros(nu_b.shape)
    pos = T_b > 0
    x = nu_b[pos] / T_b[pos]
    with np.errstate(over="ignore", invalid="ignore"):
        em = np.expm1(x)
        val = nu_b[pos] ** 3 * (x / T_b[pos]) * np.exp(x) / (em * em)
    val[~np.isfinite(val)] = 0.0
    out[pos] = val
    return out


def emitter_intensity(prob):
    """Q_nu = Q0 B_nu(T_emit); grey: Q0 sigma T_emit^4 (Example of Section 1)."""
    if prob.grey:
        return np.full(prob.freqs.F, prob.Q0 * SIGMA * prob.T_emit ** 4)
    return prob.Q0 * planck(prob.freqs.nu, prob.T_emit)


def temperature_grey(J):
    """kappa sigma T^4 = kappa J  =>  T = (J / sigma)^(1/4), J <= 0 -> 0 (Section 3, eq. (grey))."""
    J = np.asarray(J, dtype=np.float64)
    return np.where(J > 0, np.power(np.maximum(J, 0.0) / SIGMA, 0.25), 0.0)


def temperature_newton(J, freqs, T_init=None, rtol: float = 1e-14, max_iter: int = 200):
    """Per-vertex solve of sum_nu w c (1-a) (B_nu(T) - J_nu) = 0 for T >= 0.

    J: [F, N].  Newton's method on a bisection bracket [lo, hi]; a step that
    leaves the bracket is replaced by the midpoint.  Vertices whose weighted
    right-hand side is <= 0 get T = 0."""
    J = np.asarray(J, dtype=np.float64)
    F, N = J.shape
    wt = (np.asarray(freqs.w) * np.asarray(freqs.c) * (1.0 - np.asarray(freqs.albedo)))[:, None]
    nu = np.asarray(freqs.nu, dtype=np.float64)[:, None]
    rhs = (wt * J).sum(axis=0)
    T = np.zeros(N)
    act = rhs > 0
    if not act.any():
        return T
    r = rhs[act]
    lo = np.zeros(r.shape)
    hi = np.ones(r.shape)
    for _ in range(2000):
        g = (wt * planck(nu, hi[None, :])).sum(axis=0)
        grow = g < r
        if not grow.any():
            break
        lo = np.where(grow, hi, lo)
        hi = np.where(grow, hi * 2.0, hi)
    t = 0.5 * (lo + hi) if T_init is None else np.clip(np.asarray(T_init, dtype=np.float64)[act], lo, hi)
    t = np.where((t <= lo) | (t >= hi), 0.5 * (lo + hi), t)
    for _ in range(max_iter):
        f = (wt * planck(nu, t[None, :])).sum(axis=0) - r
        df = (wt * planck_dT(nu, t[None, :])).sum(axis=0)
        lo = np.where(f < 0, t, lo)
        hi = np.where(f > 0, t, hi)
        with np.errstate(divide="ignore", invalid="ignore"):
            tn = t - f / df
        bad = ~np.isfinite(tn) | (tn <= lo) | (tn >= hi)
        tn = np.where(bad, 0.5 * (lo + hi), tn)
        done = np.abs(tn - t) <= rtol * np.abs(tn)
        t = tn
        if done.all():
            break
    T[act] = t
    return T


def temperature_bisection(J, freqs, iters: int = 200):
    """Pure bisection for the same balance (used to pin the Newton solve)."""
    J = np.asarray(J, dtype=np.float64)
    wt = (np.asarray(freqs.w) * np.asarray(freqs.c) * (1.0 - np.asarray(freqs.albedo)))[:, None]
    nu = np.asarray(freqs.nu, dtype=np.float64)[:, None]
    rhs = (wt * J).sum(axis=0)
    lo = np.zeros(rhs.shape)
    hi = np.ones(rhs.shape)
    for _ in range(2000):
        grow = (wt * planck(nu, hi[None, :])).sum(axis=0) < rhs
        if not grow.any():
            break
        hi = np.where(grow, hi * 2, hi)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        f = (wt * planck(nu, mid[None, :])).sum(axis=0) - rhs
        lo = np.where(f < 0, mid, lo)
        hi = np.where(f >= 0, mid, hi)
    return np.where(rhs > 0, 0.5 * (lo + hi), 0.0)


# ---------------------------------------------------------------------------
# Dense operator and the fixed point (Section 1.3, equation (algo); Section 2)
# ---------------------------------------------------------------------------
class DenseOperator:
    """All rows of every group's G plus the emitter source, FP64, dense."""

    def __init__(self, prob, ngauss: int = 16, refine: int = 0, bins: int = 0):
        self.prob = prob
        self.c, self.gidx = groups_of(prob.freqs, bins)
        self.scale = channel_scale(prob.freqs, self.c, self.gidx)
        N = prob.N
        rows = np.arange(N, dtype=np.int32)
        R = G_rows(prob, rows, self.c, ngauss=ngauss, refine=refine)  # [N, G, N]
        self.G = np.ascontiguousarray(np.transpose(R, (1, 0, 2)))  # [G, N, N]
        shat = source_geometric(prob, rows, self.c, ngauss=ngauss, refine=refine)  # [N, G]
        Q = emitter_intensity(prob)
        self.SE = Q[:, None] * shat[:, self.gidx].T  # [F, N]

    def apply(self, X):
        """Y_nu = (c_nu / c_g) G_{g(nu)} X_nu for X [F, N] (the factor is 1 without binning)."""
        X = np.asarray(X, dtype=np.float64)
        return np.stack([self.scale[f] * (self.G[self.gidx[f]] @ X[f]) for f in range(X.shape[0])])


def source_update(prob, J, T):
    """S_nu = a_nu J_nu + (1 - a_nu) B_nu(T) (kappa is inside G); grey: B = sigma T^4."""
    fr = prob.freqs
    a = np.asarray(fr.albedo, dtype=np.float64)[:, None]
    if prob.grey:
        B = np.broadcast_to(SIGMA * np.asarray(T) ** 4, J.shape)
    else:
        B = planck(np.asarray(fr.nu)[:, None], np.asarray(T)[None, :])
    return a * J + (1.0 - a) * B


def temperature(prob, J, T_prev=None):
    if prob.grey:
        return temperature_grey(J[0])
    return temperature_newton(J, prob.freqs, T_init=T_prev)


def fixed_point(prob, op: DenseOperator, T0=0.0, J0=None, tol: float = 1e-10, max_iter: int = 500,
                history: bool = False):
    """Iterate S^k -> J^{k+1} = Sbar^E + G S^k -> T^{k+1} (eq. (algo)) until
    ||J^{k+1}-J^k||/||J^{k+1}|| <= tol.  Returns dict(J, T, iters, residual[, hist_T])."""
    F, N = prob.freqs.F, prob.N
    T = np.broadcast_to(np.asarray(T0, dtype=np.float64), (N,)).copy()
    J = np.zeros((F, N)) if J0 is None else np.array(J0, dtype=np.float64)
    hist = [T.copy()]
    res = np.inf
    k = 0
    for k in range(1, max_iter + 1):
        S = source_update(prob, J, T)
        Jn = op.SE + op.apply(S)
        T = temperature(prob, Jn, T)
        res = np.linalg.norm(Jn - J) / max(np.linalg.norm(Jn), 1e-300)
        J = Jn
        if history:
            hist.append(T.copy())
        if res <= tol:
            break
    out = dict(J=J, T=T, iters=k, residual=res)
    if history:
        out["hist_T"] = np.array(hist)
    return out


def one_step_residual(prob, rows, J, T, ngauss: int = 16, bins: int = 0):
    """F(J,T)_i = Sbar^E_i + (G S(J,T))_i - J_i at the sampled vertices `rows` (FP64 rows on the fly)."""
    c, gidx = groups_of(prob.freqs, bins)
    sc = channel_scale(prob.freqs, c, gidx)
    R = G_rows(prob, rows, c, ngauss=ngauss)  # [r, G, N]
    S = source_update(prob, np.asarray(J, dtype=np.float64), np.asarray(T, dtype=np.float64))
    shat = source_geometric(prob, rows, c, ngauss=ngauss)  # [r, G]
    Q = emitter_intensity(prob)
    out = np.zeros((prob.freqs.F, len(rows)))
    for f in range(prob.freqs.F):
        out[f] = Q[f] * shat[:, gidx[f]] + sc[f] * (R[:, gidx[f], :] @ S[f]) - np.asarray(J, dtype=np.float64)[f, rows]
    return out
