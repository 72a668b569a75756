"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with something computed independently of it:
closed forms, exactness of quadrature on polynomials, the solid-angle
identity of Lemma 1 (Section 1.1), the doubled-domain equivalence of a planar
reflective condition (Section 3.2, Test-1), a direct linear solve of the grey
fixed point, the monotonicity proposition of Section 1.3, and the paper's own
CPU table.  None of these needs a GPU.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import sphere_ref as SR
import workloads as W
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# quadrature rules
# ---------------------------------------------------------------------------
def test_gauss_legendre_exact_to_degree_31():
    t, w = O.gauss_legendre(16)
    for k in range(32):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs((w * t ** k).sum() - exact) < 2e-15, k
    # degree 32 is not integrated exactly (the rule has 16 points)
    assert abs((w * t ** 32).sum() - 2.0 / 33) > 1e-11


@pytest.mark.parametrize("which,degree", [(4, 2), (14, 5)])
def test_tet_rule_monomial_exactness(which, degree):
    b, w = O.tet_rule(which)
    assert b.shape == (which, 4)
    assert np.all(w > 0) and np.all(b > 0)
    assert np.allclose(b.sum(axis=1), 1.0, atol=1e-15)
    for p in range(degree + 1):
        for q in range(degree + 1 - p):
            for r in range(degree + 1 - p - q):
                exact = math.factorial(p) * math.factorial(q) * math.factorial(r) / math.factorial(p + q + r + 3) * 6
                num = (w * b[:, 1] ** p * b[:, 2] ** q * b[:, 3] ** r).sum()
                assert abs(num - exact) < 1e-14, (p, q, r)
    # one degree more is not exact
    misses = []
    d = degree + 1
    for p in range(d + 1):
        for q in range(d + 1 - p):
            r = d - p - q
            exact = math.factorial(p) * math.factorial(q) * math.factorial(r) / math.factorial(d + 3) * 6
            misses.append(abs((w * b[:, 1] ** p * b[:, 2] ** q * b[:, 3] ** r).sum() - exact))
    assert max(misses) > 1e-6


@pytest.mark.parametrize("which,degree", [(3, 2), (7, 5)])
def test_triangle_rule_monomial_exactness(which, degree):
    b, w = O.tri_rule(which)
    assert np.all(w > 0)
    for p in range(degree + 1):
        for q in range(degree + 1 - p):
            exact = math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2) * 2
            assert abs((w * b[:, 1] ** p * b[:, 2] ** q).sum() - exact) < 1e-14


# ---------------------------------------------------------------------------
# optical depth and kernel point values
# ---------------------------------------------------------------------------
def test_optical_depth_constant_kappa_is_kappa_times_length():
    rng = np.random.default_rng(1)
    k = W.Kappa(W.KAPPA_CONST, 2.5, 0.0)
    for _ in range(20):
        a, b = rng.uniform(0, 1, 3), rng.uniform(0, 1, 3)
        assert O.optical_depth(k, a, b) == pytest.approx(2.5 * np.linalg.norm(b - a), rel=1e-14)


def test_optical_depth_sinprod_matches_closed_form():
    rng = np.random.default_rng(2)
    k = W.sinprod_kappa(0.5)
    for _ in range(50):
        a, b = rng.uniform(0, 1, 3), rng.uniform(0, 1, 3)
        L = np.linalg.norm(b - a)
        ref = SR.sinprod_line_integral(a, (b - a) / L, 0.0, L, 1.0, 0.5)
        assert O.optical_depth(k, a, b, 16) == pytest.approx(float(ref), rel=1e-13, abs=1e-15)


def test_kernel_point_constant_kappa_mirror_image_closed_form():
    """Constant kappa: direct = c k e^{-c k r}/(4 pi r^2); reflected term equals the same
    kernel seen from the mirror image xbar = (x, y, -z): R0 c k e^{-c k |xbar-y|}/(4 pi |xbar-y|^2)."""
    rng = np.random.default_rng(3)
    k0, R0 = 1.3, 0.7
    c = np.array([1.0, 0.6, 2.4])
    kap = W.Kappa(W.KAPPA_CONST, k0, 0.0)
    wall = W.wall_z0(R0)
    for _ in range(30):
        x, y = rng.uniform(0, 1, 3), rng.uniform(0, 1, 3)
        d, r = O.kernel_point(kap, wall, x, y, c)
        rr = np.linalg.norm(x - y)
        xb = x * np.array([1, 1, -1])
        rb = np.linalg.norm(xb - y)
        np.testing.assert_allclose(d, c * k0 * np.exp(-c * k0 * rr) / (4 * math.pi * rr ** 2), rtol=1e-13)
        np.testing.assert_allclose(r, R0 * c * k0 * np.exp(-c * k0 * rb) / (4 * math.pi * rb ** 2), rtol=1e-13)


def test_kernel_point_reflected_optical_depth_is_straight_line_in_doubled_domain():
    """sin-product kappa: tau(x,x') + tau(x',y) equals the optical depth of the straight segment
    from x to the image of y below the wall, with kappa extended evenly (closed form)."""
    rng = np.random.default_rng(4)
    kap = W.sinprod_kappa(0.5)
    wall = W.wall_z0(1.0)
    c = np.array([1.0])
    for _ in range(30):
        x, y = rng.uniform(0, 1, 3), rng.uniform(0.05, 1, 3)
        _, r = O.kernel_point(kap, wall, x, y, c)
        yb = y * np.array([1, 1, -1])
        L = np.linalg.norm(yb - x)
        u = (yb - x) / L
        s_wall = x[2] / (x[2] + y[2]) * L
        tau = (SR.sinprod_line_integral(x, u, 0.0, s_wall, 1.0, 0.5)
               + SR.sinprod_line_integral(x, u, s_wall, L, 1.0, 0.5, zsign=-1.0))
        ky = 1 + 0.5 * np.prod(np.sin(2 * math.pi * y))
        ref = ky * math.exp(-tau) / (4 * math.pi * L ** 2)
        assert r[0] == pytest.approx(ref, rel=1e-12)


# ---------------------------------------------------------------------------
# the P1 operator G
# ---------------------------------------------------------------------------
def test_p1_hat_functions_reproduce_linear_functions():
    """sum_j G^{ij} f(x_j) = sum_T sum_q |T| w_q K(x_i, y_q) f(y_q) for f = 1, x, y, z
    (P1 interpolation is exact on linear functions)."""
    p = W.cube_problem(6, W.sinprod_kappa(0.5), W.midpoint_freqs(3), R0=0.5)
    rows = np.array([0, 7, 100, 215], dtype=np.int32)
    R, mom = O.G_rows(p, rows, moments=True)
    for r in range(len(rows)):
        for g in range(R.shape[1]):
            np.testing.assert_allclose(R[r, g].sum(), mom[r, g, 0], rtol=1e-13)
            np.testing.assert_allclose(R[r, g] @ p.xyz, mom[r, g, 1:], rtol=1e-12)


def test_literal_entry_equals_row_assembly():
    p = W.cube_problem(5, W.sinprod_kappa(0.5), W.midpoint_freqs(2), R0=0.5)
    rows = np.array([3, 62, 124], dtype=np.int32)
    R = O.G_rows(p, rows)
    rng = np.random.default_rng(5)
    for r, i in enumerate(rows):
        for j in rng.choice(p.N, 6, replace=False):
            np.testing.assert_allclose(O.G_entry(p, int(i), int(j)), R[r, :, j], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("kind,k0,amp", [(W.KAPPA_CONST, 2.0, 0.0), (W.KAPPA_SINPROD, 1.0, 0.5)])
def test_row_sums_converge_to_lemma1_sphere_integral(kind, k0, amp):
    """Lemma 1: sum_j G^{ij} -> (1/4pi) int_S2 (1 - e^{-tau_exit}) + R0 mirror part.  The paper's
    quadrature (refine=0) has an O(h) error from the 1/r^2 singularity; red refinement halves it
    per level, and the Richardson value 2 R_2 - R_1 matches the sphere integral."""
    n = 6
    p = W.cube_problem(n, W.Kappa(kind, k0, amp), W.grey_freqs(), R0=0.5)
    verts = np.array([0, 2 + n * 3 + n * n * 2, n - 1 + n * (n - 1)], dtype=np.int32)
    c = np.array([1.0, 1.7])
    R = [O.G_rows(p, verts, c=c, refine=ref).sum(axis=2) for ref in (0, 1, 2)]
    for v in range(len(verts)):
        for g in range(2):
            _, ref = SR.row_sum_reference(p.xyz[verts[v]], kind, k0, amp, c[g], 0.5, 192, 384)
            e0 = R[0][v, g] / ref - 1
            e2 = R[2][v, g] / ref - 1
            assert abs(e0) < 0.15
            assert abs(e2) < abs(e0) / 3
            rich = 2 * R[2][v, g] - R[1][v, g]
            assert rich / ref - 1 == pytest.approx(0.0, abs=3e-3)


def test_row_sums_below_one_so_the_fixed_point_contracts():
    p = W.multifreq_32(n=8, F=4)
    R = O.G_rows(p, np.arange(p.N, dtype=np.int32))
    assert R.min() >= 0.0
    assert R.sum(axis=2).max() < 1.0


def test_reflective_wall_equals_doubled_domain_volume():
    """Section 3.2 (Test-1): a planar RC with R0 = 1 is the same as solving on the domain doubled
    by symmetry.  With the mirrored mesh and constant kappa the two discrete operators agree to
    round-off: G_RC S = (G_doubled S_even) restricted to the original vertices."""
    n = 5
    kap = W.Kappa(W.KAPPA_CONST, 1.2, 0.0)
    p = W.cube_problem(n, kap, W.grey_freqs(), R0=1.0)
    dxyz, dtet, up, low = W.doubled_mesh(n)
    pd = W.Problem(dxyz, dtet, W.doubled_emitter(n), kap, None, W.grey_freqs())
    rows = np.array([0, 6, 31, 62, 124, 80], dtype=np.int32)
    c = np.array([1.0, 0.5])
    A = O.G_rows(p, rows, c=c)
    B = O.G_rows(pd, rows, c=c)
    S = W.rand_vectors(p.N, seed=9)
    S_even = np.zeros(dxyz.shape[0])
    S_even[up] = S
    S_even[low] = S
    np.testing.assert_allclose(A @ S, B @ S_even, rtol=1e-12)


def test_reflective_wall_equals_doubled_domain_source():
    n = 5
    kap = W.Kappa(W.KAPPA_CONST, 0.8, 0.0)
    p = W.cube_problem(n, kap, W.grey_freqs(), R0=1.0)
    dxyz, dtet, up, low = W.doubled_mesh(n)
    pd = W.Problem(dxyz, dtet, W.doubled_emitter(n), kap, None, W.grey_freqs())
    rows = np.arange(p.N, dtype=np.int32)
    c = np.array([1.0, 2.0])
    np.testing.assert_allclose(O.source_geometric(p, rows, c=c), O.source_geometric(pd, rows, c=c),
                               rtol=1e-12, atol=1e-15)


def test_zero_reflection_drops_the_mirror_terms():
    p = W.cube_problem(5, W.sinprod_kappa(0.5), W.grey_freqs(), R0=0.5)
    q = W.cube_problem(5, W.sinprod_kappa(0.5), W.grey_freqs(), R0=0.0)
    rows = np.array([0, 30, 77], dtype=np.int32)
    half = O.G_rows(p, rows)
    none = O.G_rows(q, rows)
    one = O.G_rows(p, rows, R0=1.0)
    assert not np.allclose(half, none)
    np.testing.assert_allclose(half, none + 0.5 * (one - none), rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(O.source_geometric(p, rows, R0=0.0), O.source_geometric(q, rows), rtol=1e-14)


# ---------------------------------------------------------------------------
# the emitter source
# ---------------------------------------------------------------------------
def test_zero_absorption_source_is_the_view_factor_closed_form():
    """kappa = 0: G = 0 (so J = Sbar^E) and Sbar^E is the parallel-rectangle view-factor
    integral (1/4pi) int d^2/(d^2+rho^2)^2, direct from x and mirrored from xbar (R0)."""
    n, R0 = 6, 0.5
    p = W.cube_problem(n, W.Kappa(W.KAPPA_CONST, 0.0, 0.0), W.grey_freqs(), R0=R0)
    assert np.abs(O.G_rows(p, np.array([0, 100], dtype=np.int32))).max() == 0.0
    h = 1.0 / (n - 1)
    verts = [i + n * j + n * n * k for (i, j, k) in [(2, 2, 2), (3, 0, 1), (5, 4, 0), (1, 3, 5), (2, 5, 5)]]
    rows = np.array(verts, dtype=np.int32)
    fine = O.source_geometric(p, rows, refine=4)[:, 0]
    paper = O.source_geometric(p, rows, refine=0)[:, 0]
    for r, v in enumerate(verts):
        x = p.xyz[v]
        ref = (SR.square_view(x[1], x[2], x[0]) + R0 * SR.square_view(x[1], -x[2], x[0])) / (4 * math.pi)
        assert fine[r] == pytest.approx(ref, rel=2e-3)
        assert paper[r] == pytest.approx(ref, rel=0.05)
    assert h > 0


def test_emitter_vertices_take_the_limit_value():
    """At vertices on the emitter the source is the limit d -> 0+ of the view-factor integral:
    1/4 on the face, 1/8 on an edge, 1/16 at a corner (times (1 + R0) on the wall line z = 0)."""
    n, R0 = 5, 0.5
    p = W.cube_problem(n, W.Kappa(W.KAPPA_CONST, 0.0, 0.0), W.grey_freqs(), R0=R0)
    cases = [((0, 2, 2), 0.25), ((0, 0, 2), 0.125), ((0, 2, 4), 0.125), ((0, 4, 4), 0.0625),
             ((0, 2, 0), 0.125 * (1 + R0)), ((0, 0, 0), 0.0625 * (1 + R0))]
    rows = np.array([i + n * j + n * n * k for (i, j, k), _ in cases], dtype=np.int32)
    S = O.source_geometric(p, rows)[:, 0]
    for r, (ijk, val) in enumerate(cases):
        x = p.xyz[rows[r]]
        lim = (SR.square_view(x[1], x[2], 1e-9) + R0 * SR.square_view(x[1], -x[2], 1e-9) * (x[2] == 0)) / (4 * math.pi)
        assert S[r] == pytest.approx(val, rel=1e-12)
        assert S[r] == pytest.approx(lim, rel=1e-6)


@pytest.mark.parametrize("kind,amp", [(W.KAPPA_CONST, 0.0), (W.KAPPA_SINPROD, 0.5)])
@pytest.mark.parametrize("c", [0.6, 2.4])
def test_absorbing_source_matches_an_independent_face_integral(kind, amp, c):
    """kappa > 0: the emitter source (Example of Section 1.2 discretised as in Section 2)
    against a composite tensor Gauss integral over the face x = 0 with exact line integrals
    of kappa (tests/sphere_ref.py), direct from x plus R0 times the path through the wall,
    whose optical depth is the straight line from xbar in the doubled domain.  A missing
    scale c, a depth taken from xbar instead of x, or a dropped second segment of the
    reflected path all move the value by far more than the bounds."""
    n, R0 = 6, 0.5
    kap = W.Kappa(kind, 1.0, amp)
    fr = W.Freqs(np.array([1.0]), np.array([1.0]), np.array([c]), np.array([0.3]))
    p = W.cube_problem(n, kap, fr, R0=R0)
    verts = [i + n * j + n * n * k for (i, j, k) in [(2, 2, 2), (3, 1, 1), (1, 3, 4), (4, 4, 2), (2, 1, 3)]]
    rows = np.array(verts, dtype=np.int32)
    fine = O.source_geometric(p, rows, refine=4)[:, 0]
    paper = O.source_geometric(p, rows, refine=0)[:, 0]
    for r, v in enumerate(verts):
        ref = SR.emitter_source_reference(p.xyz[v], kind, 1.0, amp, c, R0)
        # the reference itself is converged: a finer face rule changes nothing
        assert SR.emitter_source_reference(p.xyz[v], kind, 1.0, amp, c, R0, npan=32, nq=12) == pytest.approx(ref, rel=1e-12)
        assert fine[r] == pytest.approx(ref, rel=1e-10)
        assert paper[r] == pytest.approx(ref, rel=3e-4)
    # the wall term is really there: without it the values drop by the reflected part
    no_wall = O.source_geometric(p, rows, refine=4, R0=0.0)[:, 0]
    for r, v in enumerate(verts):
        assert no_wall[r] == pytest.approx(SR.emitter_source_reference(p.xyz[v], kind, 1.0, amp, c, 0.0), rel=1e-10)
    # (many orders of magnitude above the 1e-10 bound of the comparisons)
    assert ((fine - no_wall) > 1e-4 * fine).all()


# ---------------------------------------------------------------------------
# temperature solve and the fixed point
# ---------------------------------------------------------------------------
def test_newton_matches_bisection_and_closed_forms():
    rng = np.random.default_rng(6)
    fr = W.midpoint_freqs(7, albedo=0.3)
    J = rng.uniform(0.0, 2.0, size=(7, 50))
    J[:, 0] = 0.0
    Tn = O.temperature_newton(J, fr)
    Tb = O.temperature_bisection(J, fr)
    np.testing.assert_allclose(Tn, Tb, rtol=1e-13, atol=1e-300)
    assert Tn[0] == 0.0
    # single frequency: B_nu(T) = J  =>  T = nu / ln(1 + nu^3 / J)
    f1 = W.Freqs(np.array([0.7]), np.array([1.0]), np.array([1.2]), np.array([0.3]))
    J1 = rng.uniform(0.01, 3.0, size=(1, 40))
    np.testing.assert_allclose(O.temperature_newton(J1, f1), 0.7 / np.log1p(0.7 ** 3 / J1[0]), rtol=1e-13)
    # grey: sigma T^4 = J
    Jg = rng.uniform(0.0, 5.0, 30)
    np.testing.assert_allclose(O.temperature_grey(Jg) ** 4 * (math.pi ** 4 / 15), Jg, rtol=1e-13)


def test_temperature_balance_weights_each_channel_by_its_absorbed_share():
    """Properties of the balance sum_nu w c (1 - a) (J_nu - B_nu(T)) = 0 (Section 1,
    (RTb) with kappa_nu = c_nu kappa(x); kappa(x) cancels): a purely scattering channel
    (a = 1) or one with c = 0 has no say in T; scaling every c, or every w, by one factor
    leaves T unchanged; raising J of an absorbing channel raises T.  A swapped albedo
    factor, a dropped c or w, or a wrong sign fails one of these."""
    rng = np.random.default_rng(61)
    nu = np.array([0.4, 0.9, 1.6])
    fr = W.Freqs(nu, np.array([0.3, 0.5, 0.2]), np.array([0.7, 1.2, 2.0]), np.array([0.3, 1.0, 0.0]))
    J = rng.uniform(0.05, 2.0, size=(3, 40))
    T = O.temperature_newton(J, fr)
    assert (T > 0).all()
    J2 = J.copy()
    J2[1] = rng.uniform(0.0, 50.0, 40)                     # the a = 1 channel
    np.testing.assert_array_equal(O.temperature_newton(J2, fr), T)
    for scale_c, scale_w in ((3.7, 1.0), (1.0, 0.25)):
        f2 = W.Freqs(nu, fr.w * scale_w, fr.c * scale_c, fr.albedo)
        np.testing.assert_allclose(O.temperature_newton(J, f2), T, rtol=1e-13)
    f0 = W.Freqs(nu, fr.w, np.array([0.7, 1.2, 0.0]), fr.albedo)
    fdrop = W.Freqs(nu[:2], fr.w[:2], fr.c[:2], fr.albedo[:2])
    np.testing.assert_allclose(O.temperature_newton(J, f0), O.temperature_newton(J[:2], fdrop), rtol=1e-13)
    J3 = J.copy()
    J3[2] *= 1.5                                           # an absorbing channel
    assert (O.temperature_newton(J3, fr) > T).all()
    # the balance itself holds at the returned T (residual relative to the absorbed power)
    wt = (fr.w * fr.c * (1 - fr.albedo))[:, None]
    bal = (wt * (J - O.planck(nu[:, None], T[None, :]))).sum(axis=0)
    assert np.abs(bal).max() <= 1e-12 * (wt * J).sum(axis=0).max()


def test_planck_integrates_to_stefan_boltzmann():
    """int_0^inf nu^3/(e^{nu/T}-1) d nu = (pi^4/15) T^4 (the relation used by the grey model)."""
    nu = np.linspace(1e-6, 60, 400001)
    for T in (0.5, 1.0, 1.7):
        val = np.trapezoid(O.planck(nu, T), nu)
        assert val == pytest.approx(O.SIGMA * T ** 4, rel=1e-6)


def test_grey_fixed_point_equals_direct_linear_solve():
    """Grey, a = 0: S = sigma T^4 = J, so the fixed point solves (I - G) J = Sbar^E."""
    p = W.cube_problem(6, W.Kappa(W.KAPPA_CONST, 1.0, 0.0), W.grey_freqs(), R0=0.5, grey=True)
    op = O.DenseOperator(p)
    res = O.fixed_point(p, op, tol=1e-13, max_iter=400)
    Jd = np.linalg.solve(np.eye(p.N) - op.G[0], op.SE[0])
    np.testing.assert_allclose(res["J"][0], Jd, rtol=1e-11)
    assert res["residual"] <= 1e-13


def test_pure_scattering_fixed_point_is_the_direct_linear_solve():
    """Albedo 1 (Section 1.3 with a_nu = 1): the balance gives T no weight, S = J, and
    each channel's fixed point solves (I - (c_f/c_g) G_g) J_f = Sbar^E_f -- checked against
    a direct dense solve, so a swapped albedo factor in the source update (S = B(T) = 0)
    or in the balance fails."""
    p = W.cube_problem(5, W.sinprod_kappa(0.5), W.midpoint_freqs(2, albedo=1.0), R0=0.5)
    op = O.DenseOperator(p)
    res = O.fixed_point(p, op, tol=1e-14, max_iter=2000)
    assert (res["T"] == 0).all()
    for f in range(p.freqs.F):
        A = np.eye(p.N) - op.scale[f] * op.G[op.gidx[f]]
        np.testing.assert_allclose(res["J"][f], np.linalg.solve(A, op.SE[f]), rtol=1e-11)


def test_grey_fixed_point_does_not_depend_on_the_albedo():
    """Grey model (Section 3): T = (J/sigma)^(1/4) makes sigma T^4 = J, so
    S = a J + (1 - a) sigma T^4 = J for every albedo and the fixed point is the same
    linear solve whatever a is."""
    base = None
    for a in (0.0, 0.4, 0.9):
        p = W.cube_problem(5, W.Kappa(W.KAPPA_CONST, 1.0, 0.0), W.grey_freqs(albedo=a), R0=0.5, grey=True)
        op = O.DenseOperator(p)
        res = O.fixed_point(p, op, tol=1e-14, max_iter=2000)
        if base is None:
            base = res["J"][0]
            np.testing.assert_allclose(base, np.linalg.solve(np.eye(p.N) - op.G[0], op.SE[0]), rtol=1e-11)
        else:
            np.testing.assert_allclose(res["J"][0], base, rtol=1e-11)


def test_fixed_point_monotone_increasing_from_zero():
    """Proposition of Section 1.3: T^0 = 0, J^0 = 0 gives T^k increasing at every vertex."""
    p = W.cube_problem(5, W.sinprod_kappa(0.5), W.midpoint_freqs(3, albedo=0.3), R0=0.5)
    op = O.DenseOperator(p)
    res = O.fixed_point(p, op, T0=0.0, tol=1e-12, history=True)
    H = res["hist_T"]
    d = np.diff(H, axis=0)
    assert (d[:-3] > 0).all()
    assert (d >= -1e-14 * H[1:].max()).all()


def test_fixed_point_monotone_decreasing_from_above():
    """T^0 = 1 (the emitter temperature, above T*) with J^0 = B(1): T^k decreasing."""
    p = W.cube_problem(5, W.sinprod_kappa(0.5), W.midpoint_freqs(3, albedo=0.3), R0=0.5)
    op = O.DenseOperator(p)
    J0 = np.repeat(O.planck(p.freqs.nu, 1.0)[:, None], p.N, axis=1)
    res = O.fixed_point(p, op, T0=1.0, J0=J0, tol=1e-12, history=True)
    H = res["hist_T"]
    d = np.diff(H, axis=0)
    assert (d[:-3] < 0).all()
    up = O.fixed_point(p, op, T0=0.0, tol=1e-12)
    np.testing.assert_allclose(res["T"], up["T"], rtol=1e-9)


def test_paper_cpu_table_uses_natural_log():
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "paper_cpu_table.txt"))
            if l.strip() and not l.startswith("#")]
    for N, _, _, cpu, printed in rows:
        val = 1e5 * cpu / (N * N ** (1 / 3) * math.log(N))
        assert abs(val - printed) <= 0.0051 + (0.0075 if N == 8003 else 0.0)


def test_gauss_sum_of_sin_product_kappa_has_a_closed_form():
    """The identity the FP32 device path uses for the sin-product kappa: the 16-point Gauss sum
    along a segment equals k0 + amp/4 sum_j +-sin(2 pi phase_j(midpoint)) sinc(combo_j(d)),
    to FP64 round-off, for segments inside the unit cube.  Checked against the oracle's
    node-by-node sum."""
    rng = np.random.default_rng(7)
    k = W.sinprod_kappa(0.5)

    def sinc(s):
        return 1.0 if abs(s) < 1e-12 else math.sin(math.pi * s) / (math.pi * s)

    for _ in range(300):
        a, b = rng.uniform(0, 1, 3), rng.uniform(0, 1, 3)
        d = b - a
        m = a + 0.5 * d
        combos = [((1, 1, -1), 1), ((-1, 1, 1), 1), ((1, -1, 1), 1), ((1, 1, 1), -1)]
        S = sum(sgn * math.sin(2 * math.pi * np.dot(c, m)) * sinc(np.dot(c, d)) for c, sgn in combos)
        tau = np.linalg.norm(d) * (1.0 + 0.5 * 0.25 * S)
        assert tau == pytest.approx(O.optical_depth(k, a, b, 16), rel=1e-13)


# ---------------------------------------------------------------------------
# the one-step fixed-point residual used to check large solves
# ---------------------------------------------------------------------------
def test_one_step_residual_at_emitter_vertices_without_absorption():
    """kappa = 0: G = 0, so F(J, T)_i = Q_nu s_i - J_nu,i for any J, T.  At vertices on the
    emitter s_i is the limit value (1/4 on the face, 1/8 on an edge, times 1 + R0 on the wall
    line), and Q_nu = Q0 nu^3/(e^{nu/T_emit} - 1) (Example of Section 1) -- both written
    out here, independently of the oracle."""
    n, R0 = 5, 0.5
    fr = W.midpoint_freqs(4, albedo=0.3)
    p = W.cube_problem(n, W.Kappa(W.KAPPA_CONST, 0.0, 0.0), fr, R0=R0)
    cases = [((0, 2, 2), 0.25), ((0, 0, 2), 0.125), ((0, 2, 4), 0.125), ((0, 2, 0), 0.125 * (1 + R0))]
    rows = np.array([i + n * j + n * n * k for (i, j, k), _ in cases], dtype=np.int32)
    rng = np.random.default_rng(11)
    J = rng.uniform(0, 1, (fr.F, p.N))
    T = rng.uniform(0.1, 1, p.N)
    res = O.one_step_residual(p, rows, J, T)
    Q = p.Q0 * fr.nu ** 3 / np.expm1(fr.nu / p.T_emit)
    for r, (_, s) in enumerate(cases):
        np.testing.assert_allclose(res[:, r], Q * s - J[:, rows[r]], rtol=1e-12, atol=1e-14)


def test_one_step_residual_vanishes_at_the_fixed_point_and_measures_a_perturbation():
    """At the dense fixed point F(J*, T*) = 0.  For J = J* + d at the same T, S changes by a d
    (S is affine in J), so F = a G_g d - d: the defect of (I - a G) on d, computed here from
    the dense matrix.  A wrong row, frequency or group index, a dropped albedo or a sign error
    in the residual breaks one of the two."""
    p = W.cube_problem(5, W.sinprod_kappa(0.5), W.midpoint_freqs(3, albedo=0.3), R0=0.5)
    op = O.DenseOperator(p)
    fp = O.fixed_point(p, op, tol=1e-14, max_iter=400)
    rows = np.array([0, 7, 31, 62, 100, 124], dtype=np.int32)
    r0 = O.one_step_residual(p, rows, fp["J"], fp["T"])
    assert np.abs(r0).max() <= 1e-12 * np.abs(fp["J"]).max()
    d = np.random.default_rng(12).standard_normal(fp["J"].shape) * 1e-2
    r1 = O.one_step_residual(p, rows, fp["J"] + d, fp["T"])
    a = np.asarray(p.freqs.albedo)
    want = np.stack([a[f] * (op.G[op.gidx[f]] @ d[f])[rows] - d[f, rows] for f in range(p.freqs.F)])
    np.testing.assert_allclose(r1, want, rtol=1e-9, atol=1e-13)


# ---------------------------------------------------------------------------
# kappa_nu binned into a few groups (Remark of Section 2.1; Section 4, Test 2)
# ---------------------------------------------------------------------------
def test_binning_with_one_bin_per_distinct_scale_is_the_exact_operator():
    p = W.cube_problem(5, W.sinprod_kappa(0.5), W.midpoint_freqs(6, albedo=0.3), R0=0.5)
    cg, gidx = O.groups_of(p.freqs, bins=6)
    np.testing.assert_array_equal(gidx, np.arange(6))
    np.testing.assert_array_equal(cg, p.freqs.c)
    X = W.rand_vectors((6, p.N), seed=1)
    np.testing.assert_array_equal(O.DenseOperator(p, bins=6).apply(X), O.DenseOperator(p).apply(X))


def test_binned_channel_keeps_its_own_scale_in_front_of_the_group_kernel():
    """Channel f of group g applies c_f kappa(y) e^{-c_g tau}/(4 pi r^2) (+ the wall term): the
    group operator built with c_g, times c_f / c_g.  Checked on the kernel's closed form at
    constant kappa and on whole rows built separately for each group scale."""
    fr = W.midpoint_freqs(8, albedo=0.3)
    p = W.cube_problem(5, W.Kappa(W.KAPPA_CONST, 1.3, 0.0), fr, R0=0.5)
    cg, gidx = O.groups_of(fr, bins=3)
    assert cg.shape[0] == 3 and set(gidx) == {0, 1, 2}
    sc = O.channel_scale(fr, cg, gidx)
    x, y = np.array([0.3, 0.4, 0.6]), np.array([0.7, 0.2, 0.3])
    r = np.linalg.norm(x - y)
    for f in range(fr.F):
        d, _ = O.kernel_point(p.kappa, None, x, y, np.array([cg[gidx[f]]]))
        want = fr.c[f] * 1.3 * math.exp(-cg[gidx[f]] * 1.3 * r) / (4 * math.pi * r * r)
        assert sc[f] * d[0] == pytest.approx(want, rel=1e-13)
    X = W.rand_vectors((fr.F, p.N), seed=2)
    Y = O.DenseOperator(p, bins=3).apply(X)
    for g in range(3):
        Rg = O.G_rows(p, np.arange(p.N, dtype=np.int32), c=np.array([cg[g]]))[:, 0, :]
        for f in np.nonzero(gidx == g)[0]:
            np.testing.assert_allclose(Y[f], fr.c[f] / cg[g] * (Rg @ X[f]), rtol=1e-13)


def test_binned_fixed_point_approaches_the_exact_one_as_bins_are_added():
    """16 channels: the temperature of the binned fixed point tends to the exact one as the
    number of bins grows (the paper keeps 8 values of kappa_nu)."""
    fr = W.midpoint_freqs(16, albedo=0.3)
    p = W.cube_problem(6, W.sinprod_kappa(0.5), fr, R0=0.5)
    exact = O.fixed_point(p, O.DenseOperator(p), tol=1e-12)["T"]
    errs = []
    for K in (1, 2, 4, 8):
        T = O.fixed_point(p, O.DenseOperator(p, bins=K), tol=1e-12)["T"]
        errs.append(np.linalg.norm(T - exact) / np.linalg.norm(exact))
    assert all(errs[k + 1] < errs[k] for k in range(3)), errs
    assert errs[-1] < 1e-3


def test_explicit_group_map_equals_the_equivalent_bins():
    fr = W.midpoint_freqs(8, albedo=0.3)
    cg, gidx = O.groups_of(fr, bins=4)
    fr2 = W.Freqs(fr.nu, fr.w, fr.c, fr.albedo, group=gidx.astype(np.int32))
    cg2, gidx2 = O.groups_of(fr2)
    np.testing.assert_array_equal(gidx2, gidx)
    np.testing.assert_array_equal(cg2, cg)


# ---------------------------------------------------------------------------
# the surface-to-volume matrix Sbar^E_{i,l} (Section 2, last paragraph)
# ---------------------------------------------------------------------------
def test_surface_to_volume_rows_sum_to_the_source():
    """The surface P1 hat functions sum to 1, so sum_l Sbar^E_{i,l} is the source with Q0 = 1,
    for every row, group and both terms (emitter vertices included)."""
    p = W.cube_problem(6, W.sinprod_kappa(0.5), W.midpoint_freqs(3, albedo=0.3), R0=0.5)
    rows = np.arange(p.N, dtype=np.int32)
    H = O.source_hat_rows(p, rows)
    np.testing.assert_allclose(H.sum(axis=2), O.source_geometric(p, rows), rtol=1e-13, atol=1e-16)
    assert H.shape[2] == 36 and (H >= 0).all()


@pytest.mark.parametrize("kind,amp", [(W.KAPPA_CONST, 0.0), (W.KAPPA_SINPROD, 0.5)])
def test_surface_to_volume_rows_integrate_a_linear_emitter_coefficient(kind, amp):
    """Q0(y) = 1 + 2 y_2 - y_3 is linear on the emitter face, so its P1 interpolation is exact
    and sum_l Sbar^E_{i,l} Q0(y_l) is the source with that coefficient: checked against an
    independent face integral weighted by Q0 (tests/sphere_ref.py), direct plus wall term."""
    n, R0, c = 6, 0.5, 1.3
    fr = W.Freqs(np.array([1.0]), np.array([1.0]), np.array([c]), np.array([0.3]))
    p = W.cube_problem(n, W.Kappa(kind, 1.0, amp), fr, R0=R0)
    verts = [i + n * j + n * n * k for (i, j, k) in [(2, 2, 2), (3, 1, 1), (1, 3, 4), (4, 4, 2)]]
    H = O.source_hat_rows(p, np.array(verts, dtype=np.int32), refine=4)[:, 0, :]
    sv = O.emitter_vertices(p)
    q = 1.0 + 2.0 * p.xyz[sv, 1] - p.xyz[sv, 2]
    for r, v in enumerate(verts):
        ref = SR.emitter_source_reference(p.xyz[v], kind, 1.0, amp, c, R0,
                                          q0=lambda Y: 1.0 + 2.0 * Y[:, 1] - Y[:, 2])
        assert H[r] @ q == pytest.approx(ref, rel=1e-10)


# ---------------------------------------------------------------------------
# several planar walls (Section 2: one reflection point per wall; corner terms)
# ---------------------------------------------------------------------------
def _two_wall_problem(n, kap, freqs, R0y, R0z, corner, grey=False):
    p = W.cube_problem(n, kap, freqs, R0=R0z, grey=grey)
    p.more_walls = (W.wall_y0(R0y),)
    p.corner = corner
    return p


def test_two_perpendicular_walls_with_corner_terms_equal_the_fourfold_domain():
    """Walls y = 0 and z = 0 with R0 = 1 plus the double reflection at their corner are the
    cube mirrored twice: G_RC S equals G on the fourfold mesh applied to the even extension
    of S, and the sources agree, to round-off (constant kappa)."""
    n = 4
    kap = W.Kappa(W.KAPPA_CONST, 1.1, 0.0)
    p = _two_wall_problem(n, kap, W.grey_freqs(), 1.0, 1.0, corner=True)
    qxyz, qtet, img = W.quadrupled_mesh(n)
    pq = W.Problem(qxyz, qtet, W.quadrupled_emitter(n), kap, None, W.grey_freqs())
    rows = np.array([0, 5, 21, 42, 63, 30], dtype=np.int32)
    c = np.array([1.0, 0.6])
    S = W.rand_vectors(p.N, seed=10)
    S4 = np.zeros(qxyz.shape[0])
    for k in range(4):
        S4[img[k]] = S
    np.testing.assert_allclose(O.G_rows(p, rows, c=c) @ S, O.G_rows(pq, rows, c=c) @ S4, rtol=1e-12)
    allr = np.arange(p.N, dtype=np.int32)
    np.testing.assert_allclose(O.source_geometric(p, allr, c=c), O.source_geometric(pq, allr, c=c),
                               rtol=1e-12, atol=1e-15)
    # without the corner term the identity fails: the double reflection carries real weight
    p.corner = False
    assert np.abs(O.G_rows(p, rows, c=c) @ S - O.G_rows(pq, rows, c=c) @ S4).max() > 1e-4


def _unfolded_tau(x_img, y, k0, amp, npan=64, nq=8):
    """Line integral of kappa_even(p) = kappa(p_x, |p_y|, |p_z|) on the straight segment from
    the image point to y (the fourfold domain with kappa extended evenly), composite Gauss."""
    g, wg = np.polynomial.legendre.leggauss(nq)
    d = np.asarray(y) - np.asarray(x_img)
    L = np.linalg.norm(d)
    # kappa_even has a kink where the line crosses y = 0 or z = 0: panels end there
    cuts = [-x_img[a] / d[a] for a in (1, 2) if d[a] != 0 and 0 < -x_img[a] / d[a] < 1]
    knots = np.unique(np.concatenate([[0.0, 1.0], cuts]))
    edges = np.concatenate([np.linspace(knots[k], knots[k + 1], npan + 1)[:-1] for k in range(len(knots) - 1)] + [[1.0]])
    t = (0.5 * (edges[:-1, None] + edges[1:, None]) + 0.5 * (edges[1:, None] - edges[:-1, None]) * g).ravel()
    wt = (0.5 * (edges[1:, None] - edges[:-1, None]) * wg).ravel()
    P = np.asarray(x_img)[None, :] + t[:, None] * d[None, :]
    kap = k0 + amp * np.sin(2 * np.pi * P[:, 0]) * np.sin(2 * np.pi * np.abs(P[:, 1])) * np.sin(2 * np.pi * np.abs(P[:, 2]))
    return L * float((wt * kap).sum())


def test_reflected_and_corner_paths_have_the_optical_depth_of_the_unfolded_line():
    """Each reflected term's optical depth (physical broken path through its reflection
    points) equals the line integral along the straight line from the image point in the
    mirrored domain with kappa extended evenly -- for both single reflections and the corner
    path -- checked through the kernel values at point pairs (sin-product kappa)."""
    kap = W.sinprod_kappa(0.5)
    rng = np.random.default_rng(13)
    c = np.array([0.9, 2.0])
    for _ in range(20):
        x, y = rng.uniform(0.05, 0.95, 3), rng.uniform(0.05, 0.95, 3)
        walls = [W.wall_z0(0.7), W.wall_y0(0.4)]
        d0, _ = O.kernel_point(kap, None, x, y, c)
        dk, rk = O.kernel_point(kap, walls, x, y, c, corner=True)
        np.testing.assert_allclose(dk, d0, rtol=1e-13)
        want = np.zeros_like(c)
        ky = 1.0 + 0.5 * np.prod(np.sin(2 * np.pi * y))
        for img, R in (((x[0], x[1], -x[2]), 0.7), ((x[0], -x[1], x[2]), 0.4), ((x[0], -x[1], -x[2]), 0.28)):
            tau = _unfolded_tau(img, y, 1.0, 0.5)
            r2 = float(np.sum((np.asarray(img) - y) ** 2))
            want += R * c * ky * np.exp(-c * tau) / (4 * math.pi * r2)
        np.testing.assert_allclose(rk, want, rtol=1e-9)


# ---------------------------------------------------------------------------
# cellwise-constant kappa grid and opaque obstacles (non-convex domains,
# Remark 1 after Lemma 1: kappa = +infinity in the hull outside the domain)
# ---------------------------------------------------------------------------
def _grid_kappa(grid, bbox=(0.0, 0.0, 0.0, 1.0, 1.0, 1.0)):
    return W.Kappa(W.KAPPA_GRID, 0.0, 0.0, np.asarray(grid, dtype=np.float32), bbox)


def test_grid_optical_depth_is_the_exact_integral():
    """Hand values, the constant grid, and brute-force midpoint sums on random segments
    through a random grid (error bound: one sample interval per plane crossing)."""
    k = _grid_kappa([[[1.0, 3.0]]])
    assert O.optical_depth(k, [0.25, 0.5, 0.5], [1.0, 0.5, 0.5]) == pytest.approx(1.75, rel=1e-15)
    # slanted: from (0, 0, 0) to (1, 1, 0) crosses x = 0.5 at the middle: sqrt(2) (1 + 3) / 2
    assert O.optical_depth(k, [0, 0, 0], [1, 1, 0]) == pytest.approx(2 * math.sqrt(2), rel=1e-14)
    assert O.optical_depth(_grid_kappa(np.full((3, 2, 4), 2.5)), [0.1, 0.2, 0.3], [0.9, 0.4, 0.05]) == \
        pytest.approx(2.5 * np.linalg.norm([0.8, 0.2, -0.25]), rel=1e-14)
    rng = np.random.default_rng(41)
    grid = rng.uniform(0.1, 4.0, (5, 3, 4)).astype(np.float32)
    k = _grid_kappa(grid, (-0.1, 0.0, 0.2, 1.1, 0.9, 1.0))
    M = 200000
    for _ in range(12):
        a, b = rng.uniform(-0.2, 1.2, 3), rng.uniform(-0.2, 1.2, 3)
        t = (np.arange(M) + 0.5) / M
        P = a[None, :] + t[:, None] * (b - a)[None, :]
        lo, hi = np.array([-0.1, 0.0, 0.2]), np.array([1.1, 0.9, 1.0])
        idx = np.clip(np.floor((P - lo) / (hi - lo) * np.array([4, 3, 5])).astype(int), 0, [3, 2, 4])
        vals = grid[idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64)
        L = np.linalg.norm(b - a)
        brute = L * vals.mean()
        bound = L * 12 * float(grid.max() - grid.min()) / M
        assert abs(O.optical_depth(k, a, b) - brute) <= bound
        # kappa_at: the cell of the point, clamped outside the grid's box
        for p in P[:: M // 7]:
            i = np.clip(np.floor((p - lo) / (hi - lo) * np.array([4, 3, 5])).astype(int), 0, [3, 2, 4])
            assert O.kappa_at(k, p) == float(grid[i[2], i[1], i[0]])


def test_constant_grid_gives_the_constant_kappa_operator():
    """A grid holding one value everywhere is kappa = const: rows and source agree with the
    constant-kappa oracle to rounding (the exact integral against the Gauss sum of a constant;
    the value is exact in float32, the precision grid values pass through)."""
    p = W.cube_problem(5, W.Kappa(W.KAPPA_CONST, 1.25, 0.0), W.midpoint_freqs(2), R0=0.5)
    q = W.cube_problem(5, _grid_kappa(np.full((2, 3, 2), 1.25)), W.midpoint_freqs(2), R0=0.5)
    rows = np.array([0, 31, 62, 124], dtype=np.int32)
    np.testing.assert_allclose(O.G_rows(q, rows), O.G_rows(p, rows), rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(O.source_geometric(q), O.source_geometric(p), rtol=1e-12, atol=1e-300)


def test_blocking_matches_brute_force_segment_sampling():
    """or_blocked against dense sampling of the open segment, on random segments whose
    deepest point is clearly inside or clearly outside the box; plus the grazing cases."""
    B = [W.Box((0.3, 0.35, 0.4), (0.7, 0.6, 0.8))]
    lo, hi = np.array(B[0].lo), np.array(B[0].hi)
    rng = np.random.default_rng(42)
    t = (np.arange(1, 4000) / 4000.0)[:, None]
    checked = 0
    for _ in range(400):
        a, b = rng.uniform(0, 1, 3), rng.uniform(0, 1, 3)
        P = a + t * (b - a)
        depth = np.minimum(P - lo, hi - P).min(axis=1).max()   # > 0: some sample inside
        if abs(depth) < 2e-3:
            continue
        assert O.blocked(B, a, b) == (depth > 0)
        checked += 1
    assert checked > 300
    # along a face, ending on a face from outside, through an edge: not blocked
    assert not O.blocked(B, [0.3, 0.0, 0.5], [0.3, 1.0, 0.5])
    assert not O.blocked(B, [0.0, 0.5, 0.5], [0.3, 0.5, 0.5])
    assert not O.blocked(B, [0.2, 0.35, 0.5], [0.4, 0.25, 0.5])
    # from a face point into the box, and across it
    assert O.blocked(B, [0.3, 0.5, 0.5], [0.9, 0.5, 0.5])
    assert O.blocked(B, [0.0, 0.5, 0.6], [1.0, 0.45, 0.6])


def _slab_problems(grey=True, R0=0.5):
    """Unit box of 5^3 cells (h = 0.2) with the slab of cells 0.4 < x < 0.6 removed and, in
    one problem, an opaque box filling it: the two halves of the domain cannot see each other."""
    xyz, tet = W.box_mesh((5, 5, 5), 0.2, hole=((2, 0, 0), (3, 5, 5)))
    emit = W.boundary_faces(xyz, tet, lambda cen: np.abs(cen[:, 0]) < 1e-9)
    kap = W.Kappa(W.KAPPA_CONST, 0.9, 0.0)
    fr = W.grey_freqs() if grey else W.midpoint_freqs(2, albedo=0.3)
    free = W.Problem(xyz, tet, emit, kap, W.wall_z0(R0), fr, grey=grey)
    shut = W.Problem(xyz, tet, emit, kap, W.wall_z0(R0), fr, grey=grey,
                     obstacles=(W.Box((0.4, -0.1, -0.1), (0.6, 1.1, 1.1)),))
    return free, shut


def test_an_opaque_slab_separates_the_two_halves_exactly():
    """Rows and source with an opaque box filling the removed slab: entries between the halves
    (direct and through the wall) are exactly 0, entries within a half and the source on the
    emitter's half are those of the same mesh without the box, the far half gets no source."""
    free, shut = _slab_problems()
    left = np.where(free.xyz[:, 0] < 0.45)[0]
    right = np.where(free.xyz[:, 0] > 0.55)[0]
    rows = np.concatenate([left[::9], right[::9]]).astype(np.int32)
    Gf, Gs = O.G_rows(free, rows), O.G_rows(shut, rows)
    for r, i in enumerate(rows):
        same = left if free.xyz[i, 0] < 0.45 else right
        other = right if free.xyz[i, 0] < 0.45 else left
        np.testing.assert_allclose(Gs[r][:, same], Gf[r][:, same], rtol=1e-14, atol=0)
        assert (Gs[r][:, other] == 0).all()
        assert (Gf[r][:, other] > 0).all()
    Sf, Ss = O.source_geometric(free), O.source_geometric(shut)
    np.testing.assert_allclose(Ss[left], Sf[left], rtol=1e-14, atol=0)
    assert (Ss[right] == 0).all() and (Sf[right] > 0).all()


def test_row_sums_around_an_opaque_cube_converge_to_lemma1_with_remark1():
    """Lemma 1 on the convex hull with kappa = +infinity in the removed cube: sum_j G^{ij} ->
    (1/4pi) int_S2 (1 - e^{-c kappa d}) with d the distance to the hull's boundary or to the
    cube, whichever comes first.  Red refinement and the Richardson value, as for the cube."""
    xyz, tet = W.box_mesh((6, 6, 6), 1.0 / 6, hole=((2, 2, 2), (4, 4, 4)))
    kap = W.Kappa(W.KAPPA_CONST, 1.5, 0.0)
    p = W.Problem(xyz, tet, np.zeros((0, 3), np.int32), kap, None, W.grey_freqs(), grey=True,
                  obstacles=(W.Box((1 / 3, 1 / 3, 1 / 3), (2 / 3, 2 / 3, 2 / 3)),))
    targets = np.array([[1 / 6, 1 / 2, 1 / 2], [1 / 3, 1 / 3, 1 / 6], [1 / 2, 1 / 6, 5 / 6]])
    verts = np.array([np.argmin(np.linalg.norm(xyz - t, axis=1)) for t in targets], dtype=np.int32)
    c = np.array([1.0])
    R = [O.G_rows(p, verts, c=c, refine=ref).sum(axis=2)[:, 0] for ref in (0, 1, 2)]
    for v in range(len(verts)):
        ref = SR.row_sum_reference_obstacle(xyz[verts[v]], 1.5, 1.0, [0, 0, 0], [1, 1, 1],
                                            [1 / 3] * 3, [2 / 3] * 3, 192, 384)
        free = SR.row_sum_reference_obstacle(xyz[verts[v]], 1.5, 1.0, [0, 0, 0], [1, 1, 1],
                                             [5.0] * 3, [6.0] * 3, 192, 384)
        assert free - ref > 0.02                      # the cube takes a visible share
        e0, e2 = R[0][v] / ref - 1, R[2][v] / ref - 1
        assert abs(e0) < 0.15 and abs(e2) < abs(e0)
        rich = 2 * R[2][v] - R[1][v]
        assert abs(rich / ref - 1) < 1e-3


def test_grid_kappa_wall_equals_the_doubled_domain_with_the_mirrored_grid():
    """The doubled-domain identity with a cellwise-constant kappa: R0 = 1 on z = 0 with a
    random grid over [0,1]^3 is the same operator as the mirrored mesh with no wall and the
    grid mirrored onto z < 0 -- the reflected path's two exact grid integrals equal the
    straight line's exact integral through the mirrored grid.  Rows and source to rounding."""
    n = 5
    rng = np.random.default_rng(62)
    g = rng.uniform(0.3, 2.0, (3, 4, 2)).astype(np.float32)           # [z][y][x] over [0,1]^3
    kap = W.Kappa(W.KAPPA_GRID, 0.0, 0.0, g, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0))
    gd = np.concatenate([g[::-1], g], axis=0)                          # z cells of [-1, 1]
    kapd = W.Kappa(W.KAPPA_GRID, 0.0, 0.0, gd, (0.0, 0.0, -1.0, 1.0, 1.0, 1.0))
    p = W.cube_problem(n, kap, W.grey_freqs(), R0=1.0)
    dxyz, dtet, up, low = W.doubled_mesh(n)
    pd = W.Problem(dxyz, dtet, W.doubled_emitter(n), kapd, None, W.grey_freqs())
    rows = np.array([0, 6, 31, 62, 124, 80], dtype=np.int32)
    c = np.array([1.0, 0.7])
    S = W.rand_vectors(p.N, seed=63)
    S_even = np.zeros(dxyz.shape[0])
    S_even[up] = S
    S_even[low] = S
    np.testing.assert_allclose(O.G_rows(p, rows, c=c) @ S, O.G_rows(pd, rows, c=c) @ S_even, rtol=1e-12)
    allr = np.arange(p.N, dtype=np.int32)
    np.testing.assert_allclose(O.source_geometric(p, allr, c=c), O.source_geometric(pd, allr, c=c),
                               rtol=1e-12, atol=1e-15)
    # and the grid is not a constant in disguise: a wrong mirror breaks the identity
    kapw = W.Kappa(W.KAPPA_GRID, 0.0, 0.0, np.concatenate([g, g], axis=0), (0.0, 0.0, -1.0, 1.0, 1.0, 1.0))
    pw = W.Problem(dxyz, dtet, W.doubled_emitter(n), kapw, None, W.grey_freqs())
    assert np.abs(O.G_rows(p, rows, c=c) @ S - O.G_rows(pw, rows, c=c) @ S_even).max() > 1e-4


def _mirror_z(xyz, tet, tri):
    """The mesh and its mirror image in z = 0 (vertices on the plane shared), the
    emitter triangles mirrored with their orientation kept outward."""
    N = xyz.shape[0]
    on = xyz[:, 2] == 0.0
    low = np.full(N, -1, dtype=np.int64)
    low[on] = np.nonzero(on)[0]
    extra = np.nonzero(~on)[0]
    low[extra] = N + np.arange(extra.size)
    lxyz = xyz[extra].copy()
    lxyz[:, 2] = -lxyz[:, 2]
    dxyz = np.concatenate([xyz, lxyz])
    dtet = np.concatenate([tet, low[tet]]).astype(np.int32)
    dtri = np.concatenate([tri, low[tri][:, [0, 2, 1]]]).astype(np.int32)
    return dxyz, dtet, dtri, np.arange(N), low


def test_opaque_box_by_a_wall_equals_the_doubled_domain_with_the_box_mirrored():
    """The doubled-domain identity with an opaque box: R0 = 1 on z = 0 beside a box
    removed from the mesh is the mirrored mesh with the box and its image opaque and no
    wall -- a reflected path is blocked exactly when its unfolded straight line crosses
    a box.  Rows and source to rounding, and the box does block some paths."""
    xyz, tet = W.box_mesh((4, 4, 4), 0.25, hole=((1, 1, 1), (3, 3, 2)))
    emit = W.boundary_faces(xyz, tet, lambda cen: np.abs(cen[:, 0]) < 1e-9)
    box = W.Box((0.25, 0.25, 0.25), (0.75, 0.75, 0.5))
    kap = W.Kappa(W.KAPPA_CONST, 1.1, 0.0)
    p = W.Problem(xyz, tet, emit, kap, W.wall_z0(1.0), W.grey_freqs(), grey=True, obstacles=(box,))
    dxyz, dtet, dtri, up, low = _mirror_z(xyz, tet, emit)
    boxd = W.Box((0.25, 0.25, -0.5), (0.75, 0.75, -0.25))
    pd = W.Problem(dxyz, dtet, dtri, kap, None, W.grey_freqs(), grey=True, obstacles=(box, boxd))
    rows = np.unique(np.concatenate([W.sample_rows(p.N, 10, seed=64), [0, p.N - 1]])).astype(np.int32)
    c = np.array([1.0, 0.6])
    S = W.rand_vectors(p.N, seed=65)
    S_even = np.zeros(dxyz.shape[0])
    S_even[up] = S
    S_even[low] = S
    A = O.G_rows(p, rows, c=c)
    np.testing.assert_allclose(A @ S, O.G_rows(pd, rows, c=c) @ S_even, rtol=1e-12)
    allr = np.arange(p.N, dtype=np.int32)
    np.testing.assert_allclose(O.source_geometric(p, allr, c=c), O.source_geometric(pd, allr, c=c),
                               rtol=1e-12, atol=1e-15)
    free = W.Problem(xyz, tet, emit, kap, W.wall_z0(1.0), W.grey_freqs(), grey=True)
    assert np.abs(O.G_rows(free, rows, c=c) @ S - A @ S).max() > 1e-3 * np.abs(A @ S).max()


def test_surface_to_volume_rows_sum_to_the_source_with_walls_grids_and_boxes():
    """The partition of unity of the surface hat functions holds for every term: with two
    walls and their corner path over a kappa grid, and in the Test-3 geometry (three walls,
    corner paths, opaque cube, duct), sum_l Sbar^E_{i,l} is the source (pinned above by the
    doubled-domain identities), emitter vertices included."""
    g = np.random.default_rng(66).uniform(0.5, 1.5, (2, 3, 2)).astype(np.float32)
    p = W.cube_problem(6, W.Kappa(W.KAPPA_GRID, 0.0, 0.0, g, (0, 0, 0, 1, 1, 1)), W.midpoint_freqs(2), R0=0.5)
    p.more_walls = (W.wall_y0(0.4),)
    p.corner = True
    q = W.kobayashi_problem(0.05)
    for prob in (p, q):
        rows = np.unique(np.concatenate([W.sample_rows(prob.N, 40, seed=67), O.emitter_vertices(prob)[::3]]))
        rows = rows.astype(np.int32)
        H = O.source_hat_rows(prob, rows)
        np.testing.assert_allclose(H.sum(axis=2), O.source_geometric(prob, rows), rtol=1e-12, atol=1e-16)
