/*
 * rt_oracle.c -- plain, slow FP64 CPU oracle for the integral-form radiative
 * transfer operator with planar reflective walls (Pironneau & Tournier,
 * "Reflective Conditions for Radiative Transfer in Integral Form with
 * H-Matrices", arXiv 2306.05789).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test suite, the smoke check and the oracle legs of
 * the benchmark (CPU baseline, sampled error, reference arm) do.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * What it computes (all in double precision, no blocking or compression):
 *   - kappa(x): constant, k0 + amp*sin(2 pi x) sin(2 pi y) sin(2 pi z), or a
 *     cellwise-constant grid (the value of the grid cell holding x).
 *   - optical depth  int_[a,b] kappa := |b-a| int_0^1 kappa(s b + (1-s) a) ds
 *     (definition under eq. (gen1), Section 1.1), by n-point Gauss-Legendre;
 *     for the grid, exactly: the sum over the pieces of [a,b] cut by the grid
 *     planes of (value of the piece's cell) x (piece length).
 *   - non-convex domains (Remark 1 after Lemma 1): opaque boxes in the convex
 *     hull carry kappa = +infinity, so a path whose open segment crosses the
 *     interior of a box has infinite optical depth and contributes nothing.
 *   - the volume kernel of the Corollary / Example of Section 1.2 with kappa
 *     folded in as in the FEM matrix G_kappa^{ij} of Section 2:
 *        direct    kappa(y) exp(-tau(x,y)) / (4 pi |x-y|^2)
 *        reflected R0 kappa(y) exp(-tau(x,x') - tau(x',y)) / (4 pi |xbar-y|^2)
 *     with xbar the mirror image of x in the wall and x' = [xbar,y] cut with
 *     the wall (Section 2, planar reflective boundaries; |x-x'|+|x'-y| =
 *     |xbar-y|, proof of Proposition 2).
 *   - rows of G^{ij} = sum_T sum_q |T| w_q K(x_i, y_q) lambda_j(y_q)
 *     (P1 hat function = barycentric coordinate on each tetrahedron,
 *     Section 2), quadrature rule of degree 5 (14 points) when the term's
 *     source point (x_i for the direct term, xbar_i for the reflected one) is
 *     within 2 diameters of the tetrahedron's centroid, degree 2 (4 points)
 *     otherwise (Section 2: "degree 5 when |x^i-y| is small").
 *   - the emitter source Sbar^E of the Example of Section 1.2 / Section 2,
 *     squared-cosine form, with the limit value at vertices lying on the
 *     emitter (the analytic formula the paper cites is not given).
 *
 * Frequencies enter only through kappa_nu = c_g * kappa(x): each "group" g
 * is one distinct scale c_g, and the oracle returns one matrix row per group.
 * The fixed point and the Newton temperature solve live in oracle.py.
 *
 * Pins (tests/test_oracle_pins.py; each compares with something other than
 * this file):
 *   or_gauss_legendre    exact on monomials to degree 31
 *   or_tet_rule          exact on monomials to degree 2 (4 points) and 5
 *                          (14 points), and not to one degree more
 *   or_tri_rule          exact to degree 2 (3 points) and 5 (7 points)
 *   or_optical_depth     kappa |b - a| for constant kappa; the closed form of
 *                          the sin-product integral; the grid's exact piecewise
 *                          sum against hand values and brute-force sampling
 *   or_kappa_at          a constant grid gives the constant-kappa operator
 *   or_blocked           dense segment sampling, grazing and corner cases; an
 *                          opaque slab separates the two halves exactly
 *   or_kernel_point      the mirror-image closed form (constant kappa); every
 *                          reflected and corner path has the optical depth of
 *                          the straight line through the unfolded domain
 *   or_G_rows,           P1 reproduction of linear functions; entry = row;
 *   or_G_entry             Lemma 1 row sums (with and without an opaque cube);
 *                          the doubled and fourfold domains for R0 = 1 walls,
 *                          also over a mirrored kappa grid and a mirrored box
 *   or_source            the kappa = 0 view factor in closed form; limit
 *                          values on the emitter; the absorbing source against
 *                          an independent face integral; the doubled and
 *                          fourfold domains
 *   or_source_hat        rows sum to or_source (partition of unity) and
 *                          integrate a linear emitter coefficient exactly
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

#define OR_MAX_OBST 4
#define OR_MAX_GRID_DIM 512
/* a path is blocked by a box when its open segment overlaps the open box on a
 * parameter interval longer than this (relative to the segment) */
#define OR_BLOCK_EPS 1e-6

typedef struct {
    double lo[3], hi[3];
} or_box;

typedef struct {
    int kind;          /* 0: kappa = k0; 1: k0 + amp*sin(2pi x)sin(2pi y)sin(2pi z); 2: grid */
    double k0, amp;
    /* kind 2: dims[0] x dims[1] x dims[2] equal cells of the box [glo, ghi];
     * cell (i, j, k) holds grid[i + dims[0] * (j + dims[1] * k)]; a point
     * outside the box takes the value of the nearest cell (clamped indices) */
    const double* grid;
    int dims[3];
    double glo[3], ghi[3];
    int n_obst;        /* opaque boxes (kappa = +infinity inside) */
    or_box obst[OR_MAX_OBST];
} or_kappa;

/* planar reflective walls: a point p of the plane, the unit OUTWARD normal n,
 * the reflection coefficient R0.  Each wall contributes the single-reflection
 * term of Section 2 (one reflection point per wall, Hypothesis H1); with
 * corner != 0 every pair of perpendicular walls also contributes the path that
 * reflects on both (the double image of x), which the identity with the
 * fourfold mirrored domain needs. */
#define OR_MAX_WALLS 3
typedef struct {
    double p[3];
    double n[3];
    double R0;
} or_plane;

typedef struct {
    int n;             /* walls (0 .. OR_MAX_WALLS) */
    int corner;        /* also the double reflections at perpendicular walls */
    or_plane w[OR_MAX_WALLS];
} or_wall;

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [-1,1] by Newton iteration on P_n.          */
/* ------------------------------------------------------------------ */
static void legendre_pair(int n, double x, double* pn, double* dpn)
{
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

void or_gauss_legendre(int n, double* t, double* w)
{
    for (int i = 0; i < n; ++i) {
        double x = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double p, dp;
        for (int it = 0; it < 200; ++it) {
            legendre_pair(n, x, &p, &dp);
            double dx = p / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        legendre_pair(n, x, &p, &dp);
        t[i] = x;
        w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

/* ------------------------------------------------------------------ */
/* Volume and surface quadrature rules (barycentric, weights sum to 1) */
/* ------------------------------------------------------------------ */
/* Degree-2 symmetric 4-point rule and the positive 14-point degree-5 rule
 * (orbits S31(a1), S31(a2), S22(b)); exactness is checked by the tests. */
int or_tet_rule(int which, double* bary, double* w)
{
    if (which == 4) {
        double al = (5.0 + 3.0 * sqrt(5.0)) / 20.0, be = (5.0 - sqrt(5.0)) / 20.0;
        for (int k = 0; k < 4; ++k) {
            for (int d = 0; d < 4; ++d) bary[4 * k + d] = (d == k) ? al : be;
            w[k] = 0.25;
        }
        return 4;
    }
    if (which == 14) {
        const double a[2] = {0.0927352503108912, 0.3108859192633006};
        const double wa[2] = {0.01224884051939366 * 6.0, 0.01878132095300264 * 6.0};
        const double b = 0.4544962958743504, wb = 0.007091003462846911 * 6.0;
        int q = 0;
        for (int o = 0; o < 2; ++o)
            for (int k = 0; k < 4; ++k, ++q) {
                for (int d = 0; d < 4; ++d) bary[4 * q + d] = (d == k) ? 1.0 - 3.0 * a[o] : a[o];
                w[q] = wa[o];
            }
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j, ++q) {
                for (int d = 0; d < 4; ++d) bary[4 * q + d] = (d == i || d == j) ? b : 0.5 - b;
                w[q] = wb;
            }
        return 14;
    }
    return 0;
}

/* Degree-2 3-point rule (2/3,1/6,1/6) and Radon's 7-point degree-5 rule. */
int or_tri_rule(int which, double* bary, double* w)
{
    if (which == 3) {
        for (int k = 0; k < 3; ++k) {
            for (int d = 0; d < 3; ++d) bary[3 * k + d] = (d == k) ? 2.0 / 3.0 : 1.0 / 6.0;
            w[k] = 1.0 / 3.0;
        }
        return 3;
    }
    if (which == 7) {
        double s = sqrt(15.0);
        double a[2] = {(6.0 - s) / 21.0, (6.0 + s) / 21.0};
        double wa[2] = {(155.0 - s) / 1200.0, (155.0 + s) / 1200.0};
        bary[0] = bary[1] = bary[2] = 1.0 / 3.0;
        w[0] = 9.0 / 40.0;
        int q = 1;
        for (int o = 0; o < 2; ++o)
            for (int k = 0; k < 3; ++k, ++q) {
                for (int d = 0; d < 3; ++d) bary[3 * q + d] = (d == k) ? 1.0 - 2.0 * a[o] : a[o];
                w[q] = wa[o];
            }
        return 7;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* kappa and the optical depth                                          */
/* ------------------------------------------------------------------ */
static int grid_cell(const or_kappa* k, int d, double x)
{
    double u = (x - k->glo[d]) / (k->ghi[d] - k->glo[d]) * k->dims[d];
    int c = (int)floor(u);
    if (c < 0) c = 0;
    if (c > k->dims[d] - 1) c = k->dims[d] - 1;
    return c;
}

double or_kappa_at(const or_kappa* k, const double* p)
{
    if (k->kind == 2) {
        int i = grid_cell(k, 0, p[0]), j = grid_cell(k, 1, p[1]), l = grid_cell(k, 2, p[2]);
        return k->grid[i + k->dims[0] * (j + k->dims[1] * l)];
    }
    double v = k->k0;
    if (k->kind == 1)
        v += k->amp * sin(2.0 * OR_PI * p[0]) * sin(2.0 * OR_PI * p[1]) * sin(2.0 * OR_PI * p[2]);
    return v;
}

/* does the open segment (a, b) cross the interior of one of the opaque boxes?
 * Slab clipping: the parameter interval of the segment inside each open slab
 * lo_d < x_d < hi_d, intersected over the three axes. */
int or_blocked(const or_kappa* k, const double* a, const double* b)
{
    for (int o = 0; o < k->n_obst; ++o) {
        const or_box* B = &k->obst[o];
        double t0 = 0.0, t1 = 1.0;
        int inside = 1;
        for (int d = 0; d < 3 && inside; ++d) {
            double dd = b[d] - a[d];
            if (dd == 0.0) {
                if (!(a[d] > B->lo[d] && a[d] < B->hi[d])) inside = 0;
                continue;
            }
            double ta = (B->lo[d] - a[d]) / dd, tb = (B->hi[d] - a[d]) / dd;
            if (ta > tb) {
                double tmp = ta;
                ta = tb;
                tb = tmp;
            }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        }
        if (inside && t1 - t0 > OR_BLOCK_EPS) return 1;
    }
    return 0;
}

static int cmp_double(const void* x, const void* y)
{
    double a = *(const double*)x, b = *(const double*)y;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* exact integral of the cellwise-constant grid over [a, b]: cut the segment at
 * every interior grid plane it crosses, take each piece's cell from the
 * piece's midpoint */
static double grid_depth(const or_kappa* k, const double* a, const double* b)
{
    double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double ts[3 * OR_MAX_GRID_DIM + 2];
    int nt = 0;
    ts[nt++] = 0.0;
    ts[nt++] = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
        if (d[ax] == 0.0) continue;
        double h = (k->ghi[ax] - k->glo[ax]) / k->dims[ax];
        for (int m = 1; m < k->dims[ax]; ++m) {
            double t = (k->glo[ax] + m * h - a[ax]) / d[ax];
            if (t > 0.0 && t < 1.0) ts[nt++] = t;
        }
    }
    qsort(ts, nt, sizeof(double), cmp_double);
    double s = 0.0;
    for (int q = 0; q + 1 < nt; ++q) {
        double tm = 0.5 * (ts[q] + ts[q + 1]);
        double p[3] = {a[0] + tm * d[0], a[1] + tm * d[1], a[2] + tm * d[2]};
        s += or_kappa_at(k, p) * (ts[q + 1] - ts[q]);
    }
    return L * s;
}

typedef struct {
    int n;
    double t[128], w[128];
} gauss_t;

/* int_[a,b] kappa = |b-a| * sum_g (w_g/2) kappa(a + (1+t_g)/2 (b-a)). */
static double optical_depth(const or_kappa* k, const double* a, const double* b, const gauss_t* g)
{
    if (k->n_obst > 0 && or_blocked(k, a, b)) return INFINITY;
    if (k->kind == 2) return grid_depth(k, a, b);
    double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (k->kind == 0) {
        /* constant kappa: the Gauss sum of a constant, written out */
        double s = 0.0;
        for (int i = 0; i < g->n; ++i) s += 0.5 * g->w[i] * k->k0;
        return L * s;
    }
    double s = 0.0;
    for (int i = 0; i < g->n; ++i) {
        double u = 0.5 * (1.0 + g->t[i]);
        double p[3] = {a[0] + u * d[0], a[1] + u * d[1], a[2] + u * d[2]};
        s += 0.5 * g->w[i] * or_kappa_at(k, p);
    }
    return L * s;
}

double or_optical_depth(const or_kappa* k, const double* a, const double* b, int ngauss)
{
    gauss_t g;
    g.n = ngauss;
    or_gauss_legendre(ngauss, g.t, g.w);
    return optical_depth(k, a, b, &g);
}

/* ------------------------------------------------------------------ */
/* Wall geometry: mirror image xbar and reflection point x'             */
/* ------------------------------------------------------------------ */
static void mirror(const or_plane* W, const double* x, double* xb)
{
    double s = (x[0] - W->p[0]) * W->n[0] + (x[1] - W->p[1]) * W->n[1] + (x[2] - W->p[2]) * W->n[2];
    for (int d = 0; d < 3; ++d) xb[d] = x[d] - 2.0 * s * W->n[d];
}

/* signed distance of a point from the plane (positive outside) */
static double side(const or_plane* W, const double* x)
{
    return (x[0] - W->p[0]) * W->n[0] + (x[1] - W->p[1]) * W->n[1] + (x[2] - W->p[2]) * W->n[2];
}

/* x' = the point where the segment [xbar, y] meets the wall plane. */
static void reflection_point(const or_plane* W, const double* xb, const double* y, double* xp)
{
    double sb = side(W, xb), sy = side(W, y);
    /* xbar lies on the outer side (sb >= 0), y on the inner side (sy < 0) */
    double den = sb - sy;
    double t = (den > 0.0) ? sb / den : 0.0;
    for (int d = 0; d < 3; ++d) xp[d] = xb[d] + t * (y[d] - xb[d]);
}

static double dist2(const double* a, const double* b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

/* The terms of the kernel at a source vertex x: 0 the direct path; then one
 * reflection on each wall with R0 != 0 (source point = the mirror image of x,
 * weight R0); then, with corner != 0, one path reflecting on both walls of
 * every perpendicular pair (source point = the double image, weight
 * R0_a R0_b).  Returns the number of terms. */
typedef struct {
    int kind, a, b;    /* 0 direct, 1 wall a, 2 walls a and b */
    double src[3];     /* source point of the term */
    double scale;      /* its weight */
} or_term;

static int or_terms(const or_wall* W, const double* x, or_term* T)
{
    int n = 0;
    T[n].kind = 0;
    T[n].a = T[n].b = -1;
    for (int d = 0; d < 3; ++d) T[n].src[d] = x[d];
    T[n].scale = 1.0;
    ++n;
    if (!W) return n;
    for (int a = 0; a < W->n; ++a) {
        if (W->w[a].R0 == 0.0) continue;
        T[n].kind = 1;
        T[n].a = a;
        T[n].b = -1;
        mirror(&W->w[a], x, T[n].src);
        T[n].scale = W->w[a].R0;
        ++n;
    }
    if (W->corner)
        for (int a = 0; a < W->n; ++a)
            for (int b = a + 1; b < W->n; ++b) {
                const or_plane *A = &W->w[a], *B = &W->w[b];
                double dot = A->n[0] * B->n[0] + A->n[1] * B->n[1] + A->n[2] * B->n[2];
                if (fabs(dot) > 1e-12 || A->R0 == 0.0 || B->R0 == 0.0) continue;
                double xa[3];
                mirror(A, x, xa);
                T[n].kind = 2;
                T[n].a = a;
                T[n].b = b;
                mirror(B, xa, T[n].src);
                T[n].scale = A->R0 * B->R0;
                ++n;
            }
    return n;
}

/* optical depth of the term's physical path from x to y */
static double term_tau(const or_kappa* k, const or_wall* W, const or_term* T, const double* x, const double* y,
                       const gauss_t* ga)
{
    if (T->kind == 0) return optical_depth(k, x, y, ga);
    if (T->kind == 1) {
        double xp[3];
        reflection_point(&W->w[T->a], T->src, y, xp);
        return optical_depth(k, x, xp, ga) + optical_depth(k, xp, y, ga);
    }
    /* two perpendicular walls: the straight line from y to the double image
     * crosses both planes; the plane crossed first (nearer y) holds the last
     * reflection point Q, and the crossing of the other plane, mirrored back in
     * the first one, is the first reflection point P: x -> P -> Q -> y */
    const or_plane *A = &W->w[T->a], *B = &W->w[T->b];
    const double* z = T->src;
    double sya = side(A, y), sza = side(A, z), syb = side(B, y), szb = side(B, z);
    double ta = sya / (sya - sza), tb = syb / (syb - szb);
    const or_plane *first = ta <= tb ? A : B, *second = ta <= tb ? B : A;
    double t1 = ta <= tb ? ta : tb, t2 = ta <= tb ? tb : ta;
    double Q[3], U[3], P[3];
    for (int d = 0; d < 3; ++d) {
        Q[d] = y[d] + t1 * (z[d] - y[d]);
        U[d] = y[d] + t2 * (z[d] - y[d]);
    }
    (void)second;
    mirror(first, U, P);
    return optical_depth(k, x, P, ga) + optical_depth(k, P, Q, ga) + optical_depth(k, Q, y, ga);
}

/* kernel value of one term at (x, y) per group:
 * scale c_g kappa(y) e^{-c_g tau} / (4 pi |src - y|^2) */
static void term_kernel(const or_kappa* k, const or_wall* W, const or_term* T, const double* x, const double* y,
                        const gauss_t* ga, int G, const double* c, double* out)
{
    double r2 = dist2(T->src, y);
    double tau = term_tau(k, W, T, x, y, ga);
    double ky = or_kappa_at(k, y);
    for (int g = 0; g < G; ++g) out[g] = T->scale * c[g] * ky * exp(-c[g] * tau) / (4.0 * OR_PI * r2);
}

/* ------------------------------------------------------------------ */
/* Tetrahedron helpers                                                  */
/* ------------------------------------------------------------------ */
static double tet_volume(const double* v0, const double* v1, const double* v2, const double* v3)
{
    double a[3], b[3], cc[3];
    for (int d = 0; d < 3; ++d) {
        a[d] = v1[d] - v0[d];
        b[d] = v2[d] - v0[d];
        cc[d] = v3[d] - v0[d];
    }
    double det = a[0] * (b[1] * cc[2] - b[2] * cc[1]) - a[1] * (b[0] * cc[2] - b[2] * cc[0]) +
                 a[2] * (b[0] * cc[1] - b[1] * cc[0]);
    return fabs(det) / 6.0;
}

static double tet_diam(const double* const* v)
{
    double m = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j) {
            double d = sqrt(dist2(v[i], v[j]));
            if (d > m) m = d;
        }
    return m;
}

/* Red refinement of a tetrahedron in barycentric coordinates: 8 children
 * of equal volume (4 corner tetrahedra + the inner octahedron split along
 * the diagonal joining the midpoints of edges 02 and 13).  Used only for
 * the brute-force quadrature reference (refine >= 1). */
static void red_children(const double* P /* [4][4] */, double* C /* [8][4][4] */)
{
    double M[4][4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int d = 0; d < 4; ++d) M[i][j][d] = 0.5 * (P[4 * i + d] + P[4 * j + d]);
    const double* tv[8][4] = {
        {&P[0], M[0][1], M[0][2], M[0][3]},
        {M[0][1], &P[4], M[1][2], M[1][3]},
        {M[0][2], M[1][2], &P[8], M[2][3]},
        {M[0][3], M[1][3], M[2][3], &P[12]},
        {M[0][2], M[1][3], M[0][1], M[0][3]},
        {M[0][2], M[1][3], M[0][3], M[2][3]},
        {M[0][2], M[1][3], M[2][3], M[1][2]},
        {M[0][2], M[1][3], M[1][2], M[0][1]},
    };
    for (int c = 0; c < 8; ++c)
        for (int k = 0; k < 4; ++k)
            for (int d = 0; d < 4; ++d) C[16 * c + 4 * k + d] = tv[c][k][d];
}

/* All sub-tetrahedra (barycentric vertex sets) of `refine` levels. */
static int subtets(int refine, double** out)
{
    int cnt = 1;
    double* cur = (double*)malloc(16 * sizeof(double));
    memset(cur, 0, 16 * sizeof(double));
    for (int k = 0; k < 4; ++k) cur[4 * k + k] = 1.0;
    for (int l = 0; l < refine; ++l) {
        double* nxt = (double*)malloc((size_t)cnt * 8 * 16 * sizeof(double));
        for (int s = 0; s < cnt; ++s) red_children(cur + 16 * s, nxt + 16 * 8 * s);
        free(cur);
        cur = nxt;
        cnt *= 8;
    }
    *out = cur;
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Rows of the volume operator G (Section 2)                            */
/* ------------------------------------------------------------------ */
/*
 * out[r][g][j] = G_g^{rows[r], j}, j = 0..nv-1, for each group g with scale c[g].
 *
 * refine = 0: the paper's rule (14 points near, 4 points far, per term).
 * refine = L >= 1: brute force -- every tetrahedron is red-refined L times
 * and the 14-point rule is used on every child; lambda_j stays the parent's
 * barycentric coordinate.  ngauss sets the Gauss points per segment.
 * mom (may be NULL): out moments mom[r][g][0..3] = sum_T sum_q |T| w_q K(x_i,y_q) * (1, y_q)
 * (no hat functions), for the P1-reproduction check.
 */
void or_G_rows(int nv, const double* xyz, int nt, const int* tet, const or_kappa* kap, const or_wall* wall,
               int G, const double* c, int ngauss, int refine, int nrows, const int* rows, double* out,
               double* mom)
{
    gauss_t ga;
    ga.n = ngauss;
    or_gauss_legendre(ngauss, ga.t, ga.w);
    double b4[16], w4[4], b14[56], w14[14];
    or_tet_rule(4, b4, w4);
    or_tet_rule(14, b14, w14);
    double* sub = NULL;
    int nsub = subtets(refine, &sub);

#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < nrows; ++r) {
        const double* xi = xyz + 3 * (size_t)rows[r];
        or_term terms[1 + OR_MAX_WALLS + 3];
        const int nterm = or_terms(wall, xi, terms);
        double* row = out + (size_t)r * G * nv;
        memset(row, 0, sizeof(double) * (size_t)G * nv);
        double* mrow = mom ? mom + (size_t)r * G * 4 : NULL;
        if (mrow) memset(mrow, 0, sizeof(double) * G * 4);
        double kv[64];
        for (int t = 0; t < nt; ++t) {
            const int* vt = tet + 4 * (size_t)t;
            const double* V[4] = {xyz + 3 * (size_t)vt[0], xyz + 3 * (size_t)vt[1], xyz + 3 * (size_t)vt[2],
                                  xyz + 3 * (size_t)vt[3]};
            double vol = tet_volume(V[0], V[1], V[2], V[3]);
            double cen[3];
            for (int d = 0; d < 3; ++d) cen[d] = 0.25 * (V[0][d] + V[1][d] + V[2][d] + V[3][d]);
            double diam = tet_diam(V);
            for (int term = 0; term < nterm; ++term) {
                const double* src = terms[term].src;
                for (int s = 0; s < nsub; ++s) {
                    const double* P = sub + 16 * s;
                    const double* qb;
                    const double* qw;
                    int nq;
                    if (refine == 0) {
                        int nearp = sqrt(dist2(src, cen)) < 2.0 * diam;
                        qb = nearp ? b14 : b4;
                        qw = nearp ? w14 : w4;
                        nq = nearp ? 14 : 4;
                    } else {
                        qb = b14;
                        qw = w14;
                        nq = 14;
                    }
                    double subvol = vol / (double)nsub;
                    for (int q = 0; q < nq; ++q) {
                        /* barycentric coordinates in the parent tetrahedron */
                        double lam[4] = {0, 0, 0, 0};
                        for (int k = 0; k < 4; ++k)
                            for (int d = 0; d < 4; ++d) lam[d] += qb[4 * q + k] * P[4 * k + d];
                        double y[3] = {0, 0, 0};
                        for (int d = 0; d < 4; ++d)
                            for (int e = 0; e < 3; ++e) y[e] += lam[d] * V[d][e];
                        term_kernel(kap, wall, &terms[term], xi, y, &ga, G, c, kv);
                        double wq = subvol * qw[q];
                        for (int g = 0; g < G; ++g) {
                            double val = wq * kv[g];
                            for (int d = 0; d < 4; ++d) row[(size_t)g * nv + vt[d]] += val * lam[d];
                            if (mrow) {
                                mrow[4 * g + 0] += val;
                                for (int e = 0; e < 3; ++e) mrow[4 * g + 1 + e] += val * y[e];
                            }
                        }
                    }
                }
            }
        }
    }
    free(sub);
}

/*
 * One entry G_g^{ij} written literally as the definition: the sum over the
 * tetrahedra T that contain vertex j (the support of the hat function) of
 * the quadrature of K(x_i, y) lambda_j(y) over T.  out[g].
 */
void or_G_entry(int nv, const double* xyz, int nt, const int* tet, const or_kappa* kap, const or_wall* wall,
                int G, const double* c, int ngauss, int i, int j, double* out)
{
    (void)nv;
    gauss_t ga;
    ga.n = ngauss;
    or_gauss_legendre(ngauss, ga.t, ga.w);
    double b4[16], w4[4], b14[56], w14[14];
    or_tet_rule(4, b4, w4);
    or_tet_rule(14, b14, w14);
    const double* xi = xyz + 3 * (size_t)i;
    or_term terms[1 + OR_MAX_WALLS + 3];
    const int nterm = or_terms(wall, xi, terms);
    for (int g = 0; g < G; ++g) out[g] = 0.0;
    double kv[64];
    for (int t = 0; t < nt; ++t) {
        const int* vt = tet + 4 * (size_t)t;
        int loc = -1;
        for (int d = 0; d < 4; ++d)
            if (vt[d] == j) loc = d;
        if (loc < 0) continue;
        const double* V[4] = {xyz + 3 * (size_t)vt[0], xyz + 3 * (size_t)vt[1], xyz + 3 * (size_t)vt[2],
                              xyz + 3 * (size_t)vt[3]};
        double vol = tet_volume(V[0], V[1], V[2], V[3]);
        double cen[3];
        for (int d = 0; d < 3; ++d) cen[d] = 0.25 * (V[0][d] + V[1][d] + V[2][d] + V[3][d]);
        double diam = tet_diam(V);
        /* every term: the direct one, then each reflection */
        for (int term = 0; term < nterm; ++term) {
            int nearp = sqrt(dist2(terms[term].src, cen)) < 2.0 * diam;
            const double* qb = nearp ? b14 : b4;
            const double* qw = nearp ? w14 : w4;
            int nq = nearp ? 14 : 4;
            for (int q = 0; q < nq; ++q) {
                double y[3] = {0, 0, 0};
                for (int d = 0; d < 4; ++d)
                    for (int e = 0; e < 3; ++e) y[e] += qb[4 * q + d] * V[d][e];
                term_kernel(kap, wall, &terms[term], xi, y, &ga, G, c, kv);
                for (int g = 0; g < G; ++g) out[g] += vol * qw[q] * kv[g] * qb[4 * q + loc];
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Emitter source Sbar^E (Example of Section 1.2; Section 2)            */
/* ------------------------------------------------------------------ */
static void cross3(const double* a, const double* b, double* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* interior angle of triangle (A,B,C) at vertex A */
static double angle_at(const double* A, const double* B, const double* C)
{
    double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double cu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double cv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double cs = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / (cu * cv);
    if (cs > 1.0) cs = 1.0;
    if (cs < -1.0) cs = -1.0;
    return acos(cs);
}

/*
 * Geometric source per group, out[r][g] = Shat_g(x_i), i = rows[r]:
 *   (1/4pi) int_{Gamma_Q} ([(x-y).n]_-)^2 e^{-c_g tau(x,y)} / |x-y|^4
 *   + R0 ([(xbar-y).n]_-)^2 e^{-c_g (tau(x,x')+tau(x',y))} / |xbar-y|^4  dGamma(y)
 * The physical source of frequency nu is Sbar^E_nu = Q_nu * Shat_{g(nu)}.
 * Emitter triangles are given as vertex triples whose right-hand normal is
 * the OUTWARD normal n of the domain.  Quadrature: 7-point degree-5 rule if
 * the term's source point is within 2 diameters of the triangle centroid,
 * 3-point degree-2 otherwise.  refine >= 1: every triangle is split into
 * 4^refine children with the 7-point rule on each.
 * Where the source point is a vertex of the triangle the integrand vanishes
 * on the triangle except at that point and the term is replaced by its limit
 * as the point approaches the plane from inside: (angle at the vertex)/(8 pi)
 * (times R0 for the reflected term).  Where it lies in the triangle's plane
 * elsewhere the term is 0.
 */
void or_source(int nv, const double* xyz, int ne, const int* tri, const or_kappa* kap, const or_wall* wall,
               int G, const double* c, int ngauss, int refine, int nrows, const int* rows, double* out)
{
    (void)nv;
    gauss_t ga;
    ga.n = ngauss;
    or_gauss_legendre(ngauss, ga.t, ga.w);
    double b3[9], w3[3], b7[21], w7[7];
    or_tri_rule(3, b3, w3);
    or_tri_rule(7, b7, w7);
    /* children of the reference triangle (barycentric), 4^refine of them */
    int nsub = 1;
    for (int l = 0; l < refine; ++l) nsub *= 4;
    double* sub = (double*)malloc((size_t)nsub * 9 * sizeof(double));
    {
        double* cur = (double*)malloc(9 * sizeof(double));
        memset(cur, 0, 9 * sizeof(double));
        cur[0] = cur[4] = cur[8] = 1.0;
        int cnt = 1;
        for (int l = 0; l < refine; ++l) {
            double* nxt = (double*)malloc((size_t)cnt * 4 * 9 * sizeof(double));
            for (int s = 0; s < cnt; ++s) {
                const double* P = cur + 9 * s;
                double M[3][3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        for (int d = 0; d < 3; ++d) M[i][j][d] = 0.5 * (P[3 * i + d] + P[3 * j + d]);
                const double* tv[4][3] = {{&P[0], M[0][1], M[0][2]},
                                          {M[0][1], &P[3], M[1][2]},
                                          {M[0][2], M[1][2], &P[6]},
                                          {M[1][2], M[0][2], M[0][1]}};
                for (int ch = 0; ch < 4; ++ch)
                    for (int k = 0; k < 3; ++k)
                        for (int d = 0; d < 3; ++d) nxt[9 * (4 * s + ch) + 3 * k + d] = tv[ch][k][d];
            }
            free(cur);
            cur = nxt;
            cnt *= 4;
        }
        memcpy(sub, cur, (size_t)nsub * 9 * sizeof(double));
        free(cur);
    }

#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < nrows; ++r) {
        int i = rows[r];
        const double* xi = xyz + 3 * (size_t)i;
        or_term terms[1 + OR_MAX_WALLS + 3];
        const int nterm = or_terms(wall, xi, terms);
        double* o = out + (size_t)r * G;
        for (int g = 0; g < G; ++g) o[g] = 0.0;
        for (int e = 0; e < ne; ++e) {
            const int* te = tri + 3 * (size_t)e;
            const double* V[3] = {xyz + 3 * (size_t)te[0], xyz + 3 * (size_t)te[1], xyz + 3 * (size_t)te[2]};
            double e1[3], e2[3], nn[3];
            for (int d = 0; d < 3; ++d) {
                e1[d] = V[1][d] - V[0][d];
                e2[d] = V[2][d] - V[0][d];
            }
            cross3(e1, e2, nn);
            double area2 = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            double area = 0.5 * area2;
            for (int d = 0; d < 3; ++d) nn[d] /= area2;
            double cen[3], diam = 0.0;
            for (int d = 0; d < 3; ++d) cen[d] = (V[0][d] + V[1][d] + V[2][d]) / 3.0;
            for (int a = 0; a < 3; ++a)
                for (int b = a + 1; b < 3; ++b) {
                    double dd = sqrt(dist2(V[a], V[b]));
                    if (dd > diam) diam = dd;
                }
            for (int term = 0; term < nterm; ++term) {
                const double* src = terms[term].src;
                double scale = terms[term].scale;
                /* is the source point a vertex of the triangle? */
                int vloc = -1;
                for (int k = 0; k < 3; ++k)
                    if (dist2(src, V[k]) <= 1e-24) vloc = k;
                if (vloc >= 0) {
                    double ang = angle_at(V[vloc], V[(vloc + 1) % 3], V[(vloc + 2) % 3]);
                    for (int g = 0; g < G; ++g) o[g] += scale * ang / (8.0 * OR_PI);
                    continue;
                }
                /* signed distance of the source point along the outward normal */
                double sd = (src[0] - V[0][0]) * nn[0] + (src[1] - V[0][1]) * nn[1] + (src[2] - V[0][2]) * nn[2];
                double cm = sd < 0.0 ? -sd : 0.0; /* [(x-y).n]_- , constant on the plane */
                if (cm <= 0.0) continue;
                for (int s = 0; s < nsub; ++s) {
                    const double* P = sub + 9 * s;
                    const double* qb;
                    const double* qw;
                    int nq;
                    if (refine == 0) {
                        int nearp = sqrt(dist2(src, cen)) < 2.0 * diam;
                        qb = nearp ? b7 : b3;
                        qw = nearp ? w7 : w3;
                        nq = nearp ? 7 : 3;
                    } else {
                        qb = b7;
                        qw = w7;
                        nq = 7;
                    }
                    for (int q = 0; q < nq; ++q) {
                        double lam[3] = {0, 0, 0};
                        for (int k = 0; k < 3; ++k)
                            for (int d = 0; d < 3; ++d) lam[d] += qb[3 * q + k] * P[3 * k + d];
                        double y[3] = {0, 0, 0};
                        for (int d = 0; d < 3; ++d)
                            for (int ee = 0; ee < 3; ++ee) y[ee] += lam[d] * V[d][ee];
                        double r2 = dist2(src, y);
                        double tau = term_tau(kap, wall, &terms[term], xi, y, &ga);
                        double geo = scale * area / (double)nsub * qw[q] * cm * cm / (r2 * r2) / (4.0 * OR_PI);
                        for (int g = 0; g < G; ++g) o[g] += geo * exp(-c[g] * tau);
                    }
                }
            }
        }
    }
    free(sub);
}

/* ------------------------------------------------------------------ */
/* Point values of the two kernel terms (for pinning)                   */
/* ------------------------------------------------------------------ */
/* out_direct[g] = c_g kappa(y) e^{-c_g tau(x,y)} / (4 pi |x-y|^2);
 * out_refl[g]   = R0 c_g kappa(y) e^{-c_g (tau(x,x')+tau(x',y))} / (4 pi |xbar-y|^2)
 * (0 without a wall). */
void or_kernel_point(const or_kappa* kap, const or_wall* wall, const double* x, const double* y, int G,
                     const double* c, int ngauss, double* out_direct, double* out_refl)
{
    gauss_t ga;
    ga.n = ngauss;
    or_gauss_legendre(ngauss, ga.t, ga.w);
    or_term terms[1 + OR_MAX_WALLS + 3];
    const int nterm = or_terms(wall, x, terms);
    double kv[64];
    term_kernel(kap, wall, &terms[0], x, y, &ga, G, c, out_direct);
    for (int g = 0; g < G; ++g) out_refl[g] = 0.0;
    for (int t = 1; t < nterm; ++t) {
        term_kernel(kap, wall, &terms[t], x, y, &ga, G, c, kv);
        for (int g = 0; g < G; ++g) out_refl[g] += kv[g];
    }
}

/* ------------------------------------------------------------------ */
/* Surface-to-volume matrix Sbar^E_{i,l} (Section 2, last paragraph)    */
/* ------------------------------------------------------------------ */
/*
 * The emitter source with Q0(y) replaced by the P1 hat function w_l(y) of
 * emitter-surface vertex l, so that Sbar^E_i = sum_l Sbar^E_{i,l} Q0_l when
 * Q0(y) = sum_l Q0_l w_l(y).  col[v] is the column of mesh vertex v (-1 if v
 * is not an emitter vertex); out[r][g][l] (L columns) receives the geometric
 * part per group, as or_source does, quadrature and limit rules unchanged:
 * each quadrature point's value is split over the triangle's three vertices
 * by its barycentric coordinates, and the limit value at a source point that
 * is a vertex of the triangle goes to that vertex's column (w_l(x_i) = 1).
 */
void or_source_hat(int nv, const double* xyz, int ne, const int* tri, const int* col, int L, const or_kappa* kap,
                   const or_wall* wall, int G, const double* c, int ngauss, int refine, int nrows, const int* rows,
                   double* out)
{
    (void)nv;
    gauss_t ga;
    ga.n = ngauss;
    or_gauss_legendre(ngauss, ga.t, ga.w);
    double b3[9], w3[3], b7[21], w7[7];
    or_tri_rule(3, b3, w3);
    or_tri_rule(7, b7, w7);
    int nsub = 1;
    for (int l = 0; l < refine; ++l) nsub *= 4;
    double* sub = (double*)malloc((size_t)nsub * 9 * sizeof(double));
    {
        double* cur = (double*)malloc(9 * sizeof(double));
        memset(cur, 0, 9 * sizeof(double));
        cur[0] = cur[4] = cur[8] = 1.0;
        int cnt = 1;
        for (int l = 0; l < refine; ++l) {
            double* nxt = (double*)malloc((size_t)cnt * 4 * 9 * sizeof(double));
            for (int s = 0; s < cnt; ++s) {
                const double* P = cur + 9 * s;
                double M[3][3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        for (int d = 0; d < 3; ++d) M[i][j][d] = 0.5 * (P[3 * i + d] + P[3 * j + d]);
                const double* tv[4][3] = {{&P[0], M[0][1], M[0][2]},
                                          {M[0][1], &P[3], M[1][2]},
                                          {M[0][2], M[1][2], &P[6]},
                                          {M[1][2], M[0][2], M[0][1]}};
                for (int ch = 0; ch < 4; ++ch)
                    for (int k = 0; k < 3; ++k)
                        for (int d = 0; d < 3; ++d) nxt[9 * (4 * s + ch) + 3 * k + d] = tv[ch][k][d];
            }
            free(cur);
            cur = nxt;
            cnt *= 4;
        }
        memcpy(sub, cur, (size_t)nsub * 9 * sizeof(double));
        free(cur);
    }

#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < nrows; ++r) {
        int i = rows[r];
        const double* xi = xyz + 3 * (size_t)i;
        or_term terms[1 + OR_MAX_WALLS + 3];
        const int nterm = or_terms(wall, xi, terms);
        double* o = out + (size_t)r * G * L;
        for (int k = 0; k < G * L; ++k) o[k] = 0.0;
        for (int e = 0; e < ne; ++e) {
            const int* te = tri + 3 * (size_t)e;
            const double* V[3] = {xyz + 3 * (size_t)te[0], xyz + 3 * (size_t)te[1], xyz + 3 * (size_t)te[2]};
            const int cl[3] = {col[te[0]], col[te[1]], col[te[2]]};
            double e1[3], e2[3], nn[3];
            for (int d = 0; d < 3; ++d) {
                e1[d] = V[1][d] - V[0][d];
                e2[d] = V[2][d] - V[0][d];
            }
            cross3(e1, e2, nn);
            double area2 = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            double area = 0.5 * area2;
            for (int d = 0; d < 3; ++d) nn[d] /= area2;
            double cen[3], diam = 0.0;
            for (int d = 0; d < 3; ++d) cen[d] = (V[0][d] + V[1][d] + V[2][d]) / 3.0;
            for (int a = 0; a < 3; ++a)
                for (int b = a + 1; b < 3; ++b) {
                    double dd = sqrt(dist2(V[a], V[b]));
                    if (dd > diam) diam = dd;
                }
            for (int term = 0; term < nterm; ++term) {
                const double* src = terms[term].src;
                double scale = terms[term].scale;
                int vloc = -1;
                for (int k = 0; k < 3; ++k)
                    if (dist2(src, V[k]) <= 1e-24) vloc = k;
                if (vloc >= 0) {
                    double ang = angle_at(V[vloc], V[(vloc + 1) % 3], V[(vloc + 2) % 3]);
                    for (int g = 0; g < G; ++g) o[g * L + cl[vloc]] += scale * ang / (8.0 * OR_PI);
                    continue;
                }
                double sd = (src[0] - V[0][0]) * nn[0] + (src[1] - V[0][1]) * nn[1] + (src[2] - V[0][2]) * nn[2];
                double cm = sd < 0.0 ? -sd : 0.0;
                if (cm <= 0.0) continue;
                for (int s = 0; s < nsub; ++s) {
                    const double* P = sub + 9 * s;
                    const double* qb;
                    const double* qw;
                    int nq;
                    if (refine == 0) {
                        int nearp = sqrt(dist2(src, cen)) < 2.0 * diam;
                        qb = nearp ? b7 : b3;
                        qw = nearp ? w7 : w3;
                        nq = nearp ? 7 : 3;
                    } else {
                        qb = b7;
                        qw = w7;
                        nq = 7;
                    }
                    for (int q = 0; q < nq; ++q) {
                        double lam[3] = {0, 0, 0};
                        for (int k = 0; k < 3; ++k)
                            for (int d = 0; d < 3; ++d) lam[d] += qb[3 * q + k] * P[3 * k + d];
                        double y[3] = {0, 0, 0};
                        for (int d = 0; d < 3; ++d)
                            for (int ee = 0; ee < 3; ++ee) y[ee] += lam[d] * V[d][ee];
                        double r2 = dist2(src, y);
                        double tau = term_tau(kap, wall, &terms[term], xi, y, &ga);
                        double geo = scale * area / (double)nsub * qw[q] * cm * cm / (r2 * r2) / (4.0 * OR_PI);
                        for (int g = 0; g < G; ++g) {
                            double v = geo * exp(-c[g] * tau);
                            for (int k = 0; k < 3; ++k) o[g * L + cl[k]] += v * lam[k];
                        }
                    }
                }
            }
        }
    }
    free(sub);
}
