"""Independent continuous references for the oracle pins (test helper).

Everything here is written from the mathematics, not from the oracle: line
integrals of kappa in closed form, exit distances of rays from boxes, and the
solid-angle form of Lemma 1 (Section 1.1), which turns the row sum of the
volume operator into a sphere integral:

  sum_j G^{ij} -> (1/4pi) int_{S^2} (1 - e^{-c tau_exit(omega)}) d omega
               + R0 (1/4pi) int_{omega leaves through the wall}
                       (e^{-c tau_exit(omega)} - e^{-c tau_doubled(omega)}) d omega
"""
from __future__ import annotations

import math

import numpy as np


def sinprod_line_integral(x, w, s0, s1, k0, amp, zsign=1.0):
    """int_{s0}^{s1} k0 + amp sin(2pi X) sin(2pi Y) sin(2pi (zsign*Z)) ds along p(s) = x + s w.

    Exact (product-to-sum: sinA sinB sinC = 1/4[sin(A+B-C)+sin(B+C-A)+sin(C+A-B)-sin(A+B+C)]).
    Vectorised over leading dims of w, s0, s1."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    a = 2 * math.pi * x
    b = 2 * math.pi * w
    A0, B0, C0 = a[..., 0], a[..., 1], zsign * a[..., 2]
    A1, B1, C1 = b[..., 0], b[..., 1], zsign * b[..., 2]
    s0 = np.asarray(s0, dtype=np.float64)
    s1 = np.asarray(s1, dtype=np.float64)

    def isin(al, be):
        # int_{s0}^{s1} sin(al + be s) ds
        small = np.abs(be) < 1e-9
        be_safe = np.where(small, 1.0, be)
        exact = (np.cos(al + be * s0) - np.cos(al + be * s1)) / be_safe
        mid = np.sin(al + be * 0.5 * (s0 + s1)) * (s1 - s0)
        return np.where(small, mid, exact)

    tot = (isin(A0 + B0 - C0, A1 + B1 - C1) + isin(B0 + C0 - A0, B1 + C1 - A1)
           + isin(C0 + A0 - B0, C1 + A1 - B1) - isin(A0 + B0 + C0, A1 + B1 + C1))
    return k0 * (s1 - s0) + amp * 0.25 * tot


def sphere_rule(n_mu=256, n_phi=512):
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    M, P = np.meshgrid(mu, phi, indexing="ij")
    st = np.sqrt(1 - M ** 2)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), M], axis=-1).reshape(-1, 3)
    wts = (wmu[:, None] * np.full(n_phi, 2 * math.pi / n_phi)[None, :]).reshape(-1)
    return dirs, wts


def exit_distance(x, dirs, lo, hi):
    """Distance from x along each direction to the boundary of the box [lo, hi]; also the exit axis/side."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        tpos = np.where(dirs > 0, (np.asarray(hi) - x) / dirs, np.inf)
        tneg = np.where(dirs < 0, (np.asarray(lo) - x) / dirs, np.inf)
    t = np.minimum(tpos, tneg)
    L = t.min(axis=1)
    axis = t.argmin(axis=1)
    side_low = np.take_along_axis(tneg, axis[:, None], 1)[:, 0] <= np.take_along_axis(tpos, axis[:, None], 1)[:, 0]
    return np.maximum(L, 0.0), axis, side_low


def row_sum_reference(x, kappa_kind, k0, amp, c, R0, n_mu=256, n_phi=512):
    """Continuous row sum of c*G (direct + R0 mirror) at vertex x of the unit cube with wall z = 0."""
    dirs, wts = sphere_rule(n_mu, n_phi)
    L, axis, low = exit_distance(x, dirs, [0, 0, 0], [1, 1, 1])

    def tau(s0, s1, zsign=1.0):
        if kappa_kind == 0:
            return k0 * (s1 - s0)
        return sinprod_line_integral(np.broadcast_to(x, dirs.shape), dirs, s0, s1, k0, amp, zsign)

    tL = tau(np.zeros_like(L), L)
    direct = (wts * (1 - np.exp(-c * tL))).sum() / (4 * math.pi)
    if R0 == 0:
        return direct, direct
    through_wall = (axis == 2) & low
    LD, _, _ = exit_distance(x, dirs, [0, 0, -1], [1, 1, 1])
    # beyond the wall the evenly extended kappa is kappa(x, y, -z)
    t2 = tau(L, np.maximum(LD, L), zsign=-1.0)
    tD = tL + t2
    mirror = (wts * np.where(through_wall, np.exp(-c * tL) - np.exp(-c * tD), 0.0)).sum() / (4 * math.pi)
    return direct, direct + R0 * mirror


def rect_view(a, b, d):
    """int_0^a int_0^b d^2/(d^2+u^2+v^2)^2 du dv (point at height d above the corner (0,0))."""
    A, B = a / d, b / d
    return 0.5 * (A / math.sqrt(1 + A * A) * math.atan(B / math.sqrt(1 + A * A))
                  + B / math.sqrt(1 + B * B) * math.atan(A / math.sqrt(1 + B * B)))


def square_view(y0, z0, d, ylo=0.0, yhi=1.0, zlo=0.0, zhi=1.0):
    """int over the rectangle [ylo,yhi]x[zlo,zhi] of d^2/(d^2+(y-y0)^2+(z-z0)^2)^2, by superposing
    corner rectangles with signs (the foot point may lie outside the rectangle)."""
    def F(u, v):
        # signed integral over [0,u]x[0,v] in the frame of the foot point
        su, sv = math.copysign(1, u), math.copysign(1, v)
        if u == 0 or v == 0:
            return 0.0
        return su * sv * rect_view(abs(u), abs(v), d)
    return (F(yhi - y0, zhi - z0) - F(ylo - y0, zhi - z0) - F(yhi - y0, zlo - z0) + F(ylo - y0, zlo - z0))


def _composite_gauss_square(npan, nq):
    """Composite tensor Gauss-Legendre rule on [0,1]^2: points (s, t) and weights."""
    g, wg = np.polynomial.legendre.leggauss(nq)
    edges = np.linspace(0.0, 1.0, npan + 1)
    s = (0.5 * (edges[:-1, None] + edges[1:, None]) + 0.5 * (edges[1:, None] - edges[:-1, None]) * g[None, :]).ravel()
    ws = (0.5 * (edges[1:, None] - edges[:-1, None]) * wg[None, :]).ravel()
    S, T = np.meshgrid(s, s, indexing="ij")
    W2 = np.outer(ws, ws)
    return S.ravel(), T.ravel(), W2.ravel()


def emitter_source_reference(x, kappa_kind, k0, amp, c, R0, npan=24, nq=10, q0=None):
    """Emitter source (without the intensity Q) at an interior point x of the unit cube,
    emitter = the face x = 0, reflective wall z = 0 (Example of Section 1.2, squared-cosine form):

      (1/4pi) int_{[0,1]^2} d^2 e^{-c tau(x, y)} / |x - y|^4 dA(y)
      + R0 (1/4pi) int_{[0,1]^2} d^2 e^{-c tau_R(x, y)} / |xbar - y|^4 dA(y),

    d = x_1, xbar = (x_1, x_2, -x_3), and tau_R the optical depth along the broken
    path x -> x' -> y through the wall, i.e. the straight line from xbar to y in
    the doubled domain with kappa extended evenly in z.  Optical depths are exact
    line integrals (closed form), the face integral a composite tensor Gauss rule."""
    x = np.asarray(x, dtype=np.float64)
    S, T, Wq = _composite_gauss_square(npan, nq)
    Y = np.stack([np.zeros_like(S), S, T], axis=1)
    if q0 is not None:   # emitter coefficient Q0(y) on the face (weights the integrand)
        Wq = Wq * q0(Y)
    d = x[0]

    def line_tau(a, b, zsign=1.0):
        v = b - a
        L = np.linalg.norm(v, axis=-1)
        if kappa_kind == 0:
            return k0 * L
        return sinprod_line_integral(np.broadcast_to(a, v.shape), v / L[:, None], np.zeros_like(L), L, k0, amp, zsign)

    r2 = ((Y - x) ** 2).sum(axis=1)
    direct = (Wq * d * d * np.exp(-c * line_tau(x, Y)) / (r2 * r2)).sum() / (4 * math.pi)
    if R0 == 0:
        return direct
    xb = np.array([x[0], x[1], -x[2]])
    v = Y - xb
    rb2 = (v ** 2).sum(axis=1)
    # the crossing x' of z = 0 on [xbar, y]: below it kappa is taken at the mirror point
    sc = (-xb[2]) / v[:, 2]
    Xp = xb + sc[:, None] * v
    t_low = line_tau(np.broadcast_to(xb, Y.shape).copy(), Xp, zsign=-1.0) if kappa_kind else k0 * np.linalg.norm(Xp - xb, axis=1)
    t_up = line_tau(Xp, Y) if kappa_kind else k0 * np.linalg.norm(Y - Xp, axis=1)
    refl = (Wq * d * d * np.exp(-c * (t_low + t_up)) / (rb2 * rb2)).sum() / (4 * math.pi)
    return direct + R0 * refl


def entry_distance(x, dirs, lo, hi):
    """Distance from x (outside the box) along each direction to where the ray enters the
    open box (lo, hi); inf when it misses.  Slab clipping written out per axis."""
    x = np.asarray(x, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    t0 = np.zeros(dirs.shape[0])
    t1 = np.full(dirs.shape[0], np.inf)
    for d in range(3):
        v = dirs[:, d]
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (lo[d] - x[d]) / v
            tb = (hi[d] - x[d]) / v
        par = v == 0
        inside = (x[d] > lo[d]) & (x[d] < hi[d])
        ta = np.where(par, np.where(inside, -np.inf, np.inf), ta)
        tb = np.where(par, np.where(inside, np.inf, -np.inf), tb)
        t0 = np.maximum(t0, np.minimum(ta, tb))
        t1 = np.minimum(t1, np.maximum(ta, tb))
    return np.where(t1 > t0, t0, np.inf)


def row_sum_reference_obstacle(x, k0, c, box_lo, box_hi, obst_lo, obst_hi, n_mu=256, n_phi=512):
    """Lemma 1 with Remark 1 (kappa = +infinity inside an opaque box): the continuous row sum of
    c*G (constant kappa, no wall) at x is (1/4pi) int_S2 (1 - e^{-c k0 d(omega)}) with d the
    distance to the first of: leaving the container box, entering the opaque box."""
    dirs, wts = sphere_rule(n_mu, n_phi)
    L, _, _ = exit_distance(x, dirs, box_lo, box_hi)
    E = entry_distance(x, dirs, obst_lo, obst_hi)
    d = np.minimum(L, E)
    return (wts * (1 - np.exp(-c * k0 * d))).sum() / (4 * math.pi)
