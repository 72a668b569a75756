// rt_entry.cuh -- device evaluation of one matrix entry G_g^{ij} (Section 2).
//
//   G_g^{ij} = sum_{T containing x_j} sum_q |T| w_q lambda_j(y_q) K_g(x_i, y_q)
//   K_g(x, y) = c_g kappa(y) / (4 pi) [ e^{-c_g tau(x,y)} / |x-y|^2
//                                      + R0 e^{-c_g (tau(x,x') + tau(x',y))} / |xbar-y|^2 ]
// (Corollary and Example of Section 1.2 with kappa folded in as in the FEM
// matrix of Section 2; xbar = mirror image of x in the wall, x' = [xbar,y]
// cut with the wall plane; tau = line integral of kappa by n-point Gauss.)
// Quadrature per term: 14-point degree-5 rule when the term's source point
// (x_i for the direct term, xbar_i for the reflected one) lies within two
// diameters of the tetrahedron's centroid, 4-point degree-2 rule otherwise.
//
// Further reflected terms (the general instances, XT): each further wall adds
// its own single-reflection term (image of x in that plane, weight R0, broken
// path through the reflection point; Section 2 with one reflection per wall),
// and each pair of perpendicular walls the path reflecting on both (double
// image, weight R0_a R0_b).  tau may also be the exact integral of a
// cellwise-constant kappa grid, or +infinity when a path segment crosses an
// opaque box of a non-convex domain (Remark 1 after Lemma 1: kappa = +infinity
// in the convex hull outside the domain); such a term contributes nothing.
//
// One warp evaluates one entry: the (tetrahedron, quadrature point, term)
// items of the entry are distributed over the lanes through a warp prefix sum,
// each lane accumulates all groups, and a butterfly reduction leaves the sums
// in every lane.  tau is computed once per item and shared by all groups
// (kappa_nu = c_g kappa(x) => tau_g = c_g tau).
#pragma once

#include "rt_internal.h"

namespace rt {

// Tetrahedron and triangle rules as barycentric coordinates, set from the
// host once per device.  (The Gauss nodes live in KernelParams.)  This header
// is included by one translation unit only.
__constant__ double c_tet_b[18 * 4];  // rows 0..3: 4-point rule, rows 4..17: 14-point rule
__constant__ double c_tet_w[18];
__constant__ float c_tet_bf[18 * 4];
__constant__ float c_tet_wf[18];
__constant__ double c_tri_b[10 * 3];  // rows 0..2: 3-point rule, rows 3..9: 7-point rule
__constant__ double c_tri_w[10];

template <class R>
struct Vec3 {
    R x, y, z;
};

template <class R>
__device__ __forceinline__ R gauss_u(const KernelParams& P, int g);
template <>
__device__ __forceinline__ float gauss_u<float>(const KernelParams& P, int g) { return P.gu32[g]; }
template <>
__device__ __forceinline__ double gauss_u<double>(const KernelParams& P, int g) { return P.gu64[g]; }
template <class R>
__device__ __forceinline__ R gauss_w(const KernelParams& P, int g);
template <>
__device__ __forceinline__ float gauss_w<float>(const KernelParams& P, int g) { return P.gw32[g]; }
template <>
__device__ __forceinline__ double gauss_w<double>(const KernelParams& P, int g) { return P.gw64[g]; }

template <class R>
__device__ __forceinline__ R tet_b(int q, int k);
template <>
__device__ __forceinline__ float tet_b<float>(int q, int k) { return c_tet_bf[4 * q + k]; }
template <>
__device__ __forceinline__ double tet_b<double>(int q, int k) { return c_tet_b[4 * q + k]; }
template <class R>
__device__ __forceinline__ R tet_w(int q);
template <>
__device__ __forceinline__ float tet_w<float>(int q) { return c_tet_wf[q]; }
template <>
__device__ __forceinline__ double tet_w<double>(int q) { return c_tet_w[q]; }

// sin(2 pi x) in FP32 for the sin-product kappa: 2x = n + t with n = rint(2x)
// and t in [-1/2, 1/2], sin(pi (n + t)) = (-1)^n sin(pi t), and sin(pi t) by
// its Taylor series through t^11 (truncation below 6e-8 for |t| <= 1/2).
__device__ __forceinline__ float sin2pi(float x)
{
    constexpr double pi = kPi;
    constexpr float c1 = (float)pi;
    constexpr float c3 = (float)(-pi * pi * pi / 6.0);
    constexpr float c5 = (float)(pi * pi * pi * pi * pi / 120.0);
    constexpr float c7 = (float)(-pi * pi * pi * pi * pi * pi * pi / 5040.0);
    constexpr float c9 = (float)(pi * pi * pi * pi * pi * pi * pi * pi * pi / 362880.0);
    constexpr float c11 = (float)(-pi * pi * pi * pi * pi * pi * pi * pi * pi * pi * pi / 39916800.0);
    const float r = 2.0f * x;
    const float n = rintf(r);
    const float t = r - n;
    const float t2 = t * t;
    float p = fmaf(c11, t2, c9);
    p = fmaf(p, t2, c7);
    p = fmaf(p, t2, c5);
    p = fmaf(p, t2, c3);
    p = fmaf(p, t2, c1);
    const float v = p * t;
    return (((int)n) & 1) ? -v : v;
}
__device__ __forceinline__ double sin2pi(double x) { return sinpi(2.0 * x); }

// sin(2 pi x) on the special-function unit, for values that enter only through
// products of magnitude <= 1 (the sines of the sin-product kappa and of the
// midpoints in its line integral): sin has period 1 in x, so x - rint(x) in
// [-1/2, 1/2] keeps the argument of __sinf in [-pi, pi], where its absolute
// error stays below 4e-7.  The sinc quotients keep the polynomial sin2pi,
// whose relative accuracy near zero they need.
__device__ __forceinline__ float sin2pi_sfu(float x)
{
    const float t = x - rintf(x);
    return __sinf(6.28318530717958647692f * t);
}
__device__ __forceinline__ double sin2pi_sfu(double x) { return sin2pi(x); }
__device__ __forceinline__ float exp_r(float x) { return expf(x); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }
__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }

template <class R>
__device__ __forceinline__ R kp_k0(const KernelParams& P);
template <>
__device__ __forceinline__ float kp_k0<float>(const KernelParams& P) { return P.k0f; }
template <>
__device__ __forceinline__ double kp_k0<double>(const KernelParams& P) { return P.k0; }
template <class R>
__device__ __forceinline__ R kp_amp(const KernelParams& P);
template <>
__device__ __forceinline__ float kp_amp<float>(const KernelParams& P) { return P.ampf; }
template <>
__device__ __forceinline__ double kp_amp<double>(const KernelParams& P) { return P.amp; }
template <class R>
__device__ __forceinline__ R kp_c(const KernelParams& P, int g);
template <>
__device__ __forceinline__ float kp_c<float>(const KernelParams& P, int g) { return P.cf[g]; }
template <>
__device__ __forceinline__ double kp_c<double>(const KernelParams& P, int g) { return P.c[g]; }

template <class R>
__device__ __forceinline__ Vec3<R> load_xyz(const KernelParams& P, int v);
template <>
__device__ __forceinline__ Vec3<float> load_xyz<float>(const KernelParams& P, int v)
{
    float4 a = P.xyz32[v];
    return {a.x, a.y, a.z};
}
template <>
__device__ __forceinline__ Vec3<double> load_xyz<double>(const KernelParams& P, int v)
{
    return {P.xyz64[3 * (int64_t)v], P.xyz64[3 * (int64_t)v + 1], P.xyz64[3 * (int64_t)v + 2]};
}

template <class R>
__device__ __forceinline__ void load_tgeo(const KernelParams& P, int t, Vec3<R>& c, R& diam, R& vol);
template <>
__device__ __forceinline__ void load_tgeo<float>(const KernelParams& P, int t, Vec3<float>& c, float& diam,
                                                 float& vol)
{
    float4 g = P.tgeo32[t];
    c = {g.x, g.y, g.z};
    diam = g.w;
    vol = P.tvol32[t];
}
template <>
__device__ __forceinline__ void load_tgeo<double>(const KernelParams& P, int t, Vec3<double>& c, double& diam,
                                                  double& vol)
{
    dbl4 g = P.tgeo64[t];
    c = {g.x, g.y, g.z};
    diam = g.w;
    vol = P.tvol64[t];
}

template <class R>
__device__ __forceinline__ R dist2(const Vec3<R>& a, const Vec3<R>& b)
{
    R dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    return dx * dx + dy * dy + dz * dz;
}

// ---- cellwise-constant grid (RT_KAPPA_GRID), general instances only ---------
template <class R>
__device__ __forceinline__ R grid_value(const KernelParams& P, int idx);
template <>
__device__ __forceinline__ float grid_value<float>(const KernelParams& P, int idx) { return __ldg(P.kgrid32 + idx); }
template <>
__device__ __forceinline__ double grid_value<double>(const KernelParams& P, int idx) { return __ldg(P.kgrid64 + idx); }

// cell index along axis d of coordinate x, clamped to the grid
template <class R>
__device__ __forceinline__ int grid_cell(const KernelParams& P, int d, R x)
{
    R u = (x - R(P.glo[d])) / (R(P.ghi[d]) - R(P.glo[d])) * R(P.gdims[d]);
    u = u < R(0) ? R(0) : (u > R(P.gdims[d]) - R(0.5) ? R(P.gdims[d]) - R(0.5) : u);
    return (int)floor(u);
}

template <class R>
__device__ __forceinline__ R grid_kappa(const KernelParams& P, R x, R y, R z)
{
    const int i = grid_cell<R>(P, 0, x), j = grid_cell<R>(P, 1, y), k = grid_cell<R>(P, 2, z);
    return grid_value<R>(P, i + P.gdims[0] * (j + P.gdims[1] * k));
}

// XT: the general instances, which also know the grid
template <class R, bool XT = false>
__device__ __forceinline__ R kappa_at(const KernelParams& P, R x, R y, R z)
{
    if constexpr (XT) {
        if (P.kappa_kind == RT_KAPPA_GRID) return grid_kappa<R>(P, x, y, z);
    }
    R k = kp_k0<R>(P);
    if (P.kappa_kind == RT_KAPPA_SINPROD)
        k += kp_amp<R>(P) * sin2pi_sfu(x) * sin2pi_sfu(y) * sin2pi_sfu(z);
    return k;
}

// sin(pi s) / (pi s) in FP32, without a branch.  |s| < 1/4: the Taylor series
// of sin(p)/p, p = pi s, through p^8 (truncation below 3e-9, no division).
// Otherwise sin(pi s) from the special-function unit (absolute error below
// 4e-7) over pi s >= pi/4 with an approximate division: absolute error below
// 6e-7, which the bounded midpoint sines multiply.
__device__ __forceinline__ float sinc_pi(float s)
{
    const float ps = (float)kPi * s;
    const float p2 = ps * ps;
    const float series =
        fmaf(p2, fmaf(p2, fmaf(p2, fmaf(p2, 1.f / 362880.f, -1.f / 5040.f), 1.f / 120.f), -1.f / 6.f), 1.f);
    const float quot = __fdividef(sin2pi_sfu(0.5f * s), ps);
    return fabsf(s) < 0.25f ? series : quot;
}

// The Gauss sum sum_g w_g kappa(a + u_g d) for kappa = k0 + amp sin(2 pi x)
// sin(2 pi y) sin(2 pi z), evaluated exactly: sinA sinB sinC =
// 1/4 [sin(A+B-C) + sin(B+C-A) + sin(C+A-B) - sin(A+B+C)] turns the samples
// into four sinusoids sin(alpha + beta u) of the node u, and for a rule
// symmetric about 1/2, sum_g w_g sin(alpha + beta u_g) = sin(alpha + beta/2)
// C(beta) with C(beta) = sum_g w_g cos(beta (u_g - 1/2)).  C equals
// sin(beta/2)/(beta/2) up to the rule's error on cos, below 2e-14 for n >= 16
// nodes and |beta| <= 6 pi, i.e. |dx| + |dy| + |dz| <= 3.
__device__ __forceinline__ float gauss_sum_sinprod(const KernelParams& P, const Vec3<float>& a, float dx, float dy,
                                                   float dz)
{
    const float mx = a.x + 0.5f * dx, my = a.y + 0.5f * dy, mz = a.z + 0.5f * dz;
    const float S = sin2pi_sfu(mx + my - mz) * sinc_pi(dx + dy - dz) + sin2pi_sfu(-mx + my + mz) * sinc_pi(-dx + dy + dz) +
                    sin2pi_sfu(mx - my + mz) * sinc_pi(dx - dy + dz) - sin2pi_sfu(mx + my + mz) * sinc_pi(dx + dy + dz);
    return P.k0f + 0.25f * P.ampf * S;
}

// Exact int_[a,b] kappa for the cellwise-constant grid: walk the grid planes
// the segment crosses in order of the segment parameter t (one next crossing
// per axis, the smallest first); each piece [t0, t1] adds the value of its
// cell times its length.  Planes are x = glo + m h, m = 1 .. dims-1; a crossing
// counts when 0 < t < 1.  The cell of a piece is tracked by the walk itself
// (the cell ahead of a, then one step per plane crossed), which is the cell
// holding the piece's midpoint; a point outside the grid's box belongs to the
// nearest cell.
template <class R>
__device__ R grid_depth(const KernelParams& P, const Vec3<R>& a, const Vec3<R>& b)
{
    const R A[3] = {a.x, a.y, a.z};
    const R D[3] = {b.x - a.x, b.y - a.y, b.z - a.z};
    const R L = sqrt_r(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    R tn[3], h[3];
    int m[3], st[3], cell[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        h[d] = (R(P.ghi[d]) - R(P.glo[d])) / R(P.gdims[d]);
        st[d] = D[d] > R(0) ? 1 : -1;
        tn[d] = R(2);
        if (D[d] != R(0)) {
            const R u = (A[d] - R(P.glo[d])) / h[d];
            const R uc = u < R(-1) ? R(-1) : (u > R(P.gdims[d] + 1) ? R(P.gdims[d] + 1) : u);
            m[d] = D[d] > R(0) ? max((int)floor(uc) + 1, 1) : min((int)ceil(uc) - 1, P.gdims[d] - 1);
            // first plane strictly ahead of a (rounding may put the first guess behind)
            for (int it = 0; it < 3; ++it) {
                if (m[d] < 1 || m[d] > P.gdims[d] - 1) break;
                const R t = (R(P.glo[d]) + R(m[d]) * h[d] - A[d]) / D[d];
                if (t > R(0)) break;
                m[d] += st[d];
            }
            if (m[d] >= 1 && m[d] <= P.gdims[d] - 1) tn[d] = (R(P.glo[d]) + R(m[d]) * h[d] - A[d]) / D[d];
            // the cell between the last plane behind and the next one ahead
            const int c = D[d] > R(0) ? m[d] - 1 : m[d];
            cell[d] = c < 0 ? 0 : (c > P.gdims[d] - 1 ? P.gdims[d] - 1 : c);
        } else {
            m[d] = 0;
            cell[d] = grid_cell<R>(P, d, A[d]);
        }
    }
    R s = R(0), t0 = R(0);
    const int max_steps = P.gdims[0] + P.gdims[1] + P.gdims[2] + 4;
    for (int step = 0; step < max_steps; ++step) {
        R t1 = tn[0] < tn[1] ? tn[0] : tn[1];
        t1 = t1 < tn[2] ? t1 : tn[2];
        t1 = t1 < R(1) ? t1 : R(1);
        if (t1 > t0) {
            s += grid_value<R>(P, cell[0] + P.gdims[0] * (cell[1] + P.gdims[1] * cell[2])) * (t1 - t0);
            t0 = t1;
        }
        if (t1 >= R(1)) break;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (tn[d] == t1) {
                m[d] += st[d];
                cell[d] += st[d];
                tn[d] = (m[d] >= 1 && m[d] <= P.gdims[d] - 1) ? (R(P.glo[d]) + R(m[d]) * h[d] - A[d]) / D[d] : R(2);
            }
    }
    return L * s;
}

// Does the open segment (a, b) cross the interior of an opaque box?  Slab
// clipping of the parameter interval per axis; blocked when what is left is
// longer than 1e-6 (in units of the segment).
template <class R>
__device__ bool path_blocked(const KernelParams& P, const Vec3<R>& a, const Vec3<R>& b)
{
    const R A[3] = {a.x, a.y, a.z};
    const R D[3] = {b.x - a.x, b.y - a.y, b.z - a.z};
    for (int o = 0; o < P.n_obst; ++o) {
        R t0 = R(0), t1 = R(1);
        bool inside = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const R lo = R(P.olo[o][d]), hi = R(P.ohi[o][d]);
            if (D[d] == R(0)) {
                if (!(A[d] > lo && A[d] < hi)) inside = false;
                continue;
            }
            R ta = (lo - A[d]) / D[d], tb = (hi - A[d]) / D[d];
            if (ta > tb) {
                const R tmp = ta;
                ta = tb;
                tb = tmp;
            }
            t0 = ta > t0 ? ta : t0;
            t1 = tb < t1 ? tb : t1;
        }
        if (inside && t1 - t0 > R(1e-6)) return true;
    }
    return false;
}

// int_[a,b] kappa = |b-a| sum_g (w_g/2) kappa(a + u_g (b-a)).  For constant
// kappa the Gauss sum equals kappa |b-a| exactly (weights sum to 1).  The
// general instances (XT) also handle the opaque boxes (+infinity) and the
// grid (exact integral).
template <class R, bool XT = false>
__device__ __forceinline__ R optical_depth(const KernelParams& P, const Vec3<R>& a, const Vec3<R>& b)
{
    if constexpr (XT) {
        if (P.n_obst > 0 && path_blocked<R>(P, a, b)) return R(INFINITY);
        if (P.kappa_kind == RT_KAPPA_GRID) return grid_depth<R>(P, a, b);
    }
    R dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    R L = sqrt_r(dx * dx + dy * dy + dz * dz);
    if (P.kappa_kind != RT_KAPPA_SINPROD) return kp_k0<R>(P) * L;
    if constexpr (sizeof(R) == 4) {
        if (P.line_closed && fabsf(dx) + fabsf(dy) + fabsf(dz) <= 3.0f) return L * gauss_sum_sinprod(P, a, dx, dy, dz);
    }
    R s = R(0);
    for (int g = 0; g < P.ngauss; ++g) {
        R u = gauss_u<R>(P, g);
        s += gauss_w<R>(P, g) * kappa_at<R>(P, a.x + u * dx, a.y + u * dy, a.z + u * dz);
    }
    return L * s;
}

template <class R>
__device__ __forceinline__ Vec3<R> mirror_point(const KernelParams& P, const Vec3<R>& x)
{
    R s = (x.x - R(P.wp[0])) * R(P.wn[0]) + (x.y - R(P.wp[1])) * R(P.wn[1]) + (x.z - R(P.wp[2])) * R(P.wn[2]);
    return {x.x - R(2) * s * R(P.wn[0]), x.y - R(2) * s * R(P.wn[1]), x.z - R(2) * s * R(P.wn[2])};
}

// x' on the wall plane along [xbar, y]
template <class R>
__device__ __forceinline__ Vec3<R> wall_point(const KernelParams& P, const Vec3<R>& xb, const Vec3<R>& y)
{
    R sb = (xb.x - R(P.wp[0])) * R(P.wn[0]) + (xb.y - R(P.wp[1])) * R(P.wn[1]) + (xb.z - R(P.wp[2])) * R(P.wn[2]);
    R sy = (y.x - R(P.wp[0])) * R(P.wn[0]) + (y.y - R(P.wp[1])) * R(P.wn[1]) + (y.z - R(P.wp[2])) * R(P.wn[2]);
    R den = sb - sy;
    R t = den > R(0) ? sb / den : R(0);
    return {xb.x + t * (y.x - xb.x), xb.y + t * (y.y - xb.y), xb.z + t * (y.z - xb.z)};
}

// ---- further reflected terms (several walls, corner paths) -------------------
template <class R>
__device__ __forceinline__ R wall_side(const KernelParams& P, int w, const Vec3<R>& x)
{
    return (x.x - R(P.wps[w][0])) * R(P.wns[w][0]) + (x.y - R(P.wps[w][1])) * R(P.wns[w][1]) +
           (x.z - R(P.wps[w][2])) * R(P.wns[w][2]);
}

template <class R>
__device__ __forceinline__ Vec3<R> mirror_w(const KernelParams& P, int w, const Vec3<R>& x)
{
    const R s = wall_side<R>(P, w, x);
    return {x.x - R(2) * s * R(P.wns[w][0]), x.y - R(2) * s * R(P.wns[w][1]), x.z - R(2) * s * R(P.wns[w][2])};
}

// source point (the image of x) and weight of extra term k
template <class R>
__device__ __forceinline__ void extra_term(const KernelParams& P, int k, const Vec3<R>& x, Vec3<R>& src, R& scale)
{
    const int a = P.xa[k];
    src = mirror_w<R>(P, a, x);
    scale = R(P.wR[a]);
    if (P.xkind[k] == 2) {
        src = mirror_w<R>(P, P.xb[k], src);
        scale *= R(P.wR[P.xb[k]]);
    }
}

// optical depth of extra term k's physical path from x to y (src = its image of x):
// one wall: x -> x' -> y with x' on [src, y]; two perpendicular walls: the plane
// that the line from y to src crosses first holds the last reflection point Q, and
// the crossing of the other plane mirrored back in the first is the first one P
template <class R>
__device__ __forceinline__ R extra_tau(const KernelParams& P, int k, const Vec3<R>& x, const Vec3<R>& src,
                                       const Vec3<R>& y)
{
    const int a = P.xa[k];
    if (P.xkind[k] == 1) {
        const R sb = wall_side<R>(P, a, src), sy = wall_side<R>(P, a, y);
        const R den = sb - sy;
        const R t = den > R(0) ? sb / den : R(0);
        const Vec3<R> xp = {src.x + t * (y.x - src.x), src.y + t * (y.y - src.y), src.z + t * (y.z - src.z)};
        return optical_depth<R, true>(P, x, xp) + optical_depth<R, true>(P, xp, y);
    }
    const int b = P.xb[k];
    const R sya = wall_side<R>(P, a, y), sza = wall_side<R>(P, a, src);
    const R syb = wall_side<R>(P, b, y), szb = wall_side<R>(P, b, src);
    const R ta = sya / (sya - sza), tb = syb / (syb - szb);
    const bool afirst = ta <= tb;
    const R t1 = afirst ? ta : tb, t2 = afirst ? tb : ta;
    const Vec3<R> Q = {y.x + t1 * (src.x - y.x), y.y + t1 * (src.y - y.y), y.z + t1 * (src.z - y.z)};
    const Vec3<R> U = {y.x + t2 * (src.x - y.x), y.y + t2 * (src.y - y.y), y.z + t2 * (src.z - y.z)};
    const Vec3<R> Pp = mirror_w<R>(P, afirst ? a : b, U);
    return optical_depth<R, true>(P, x, Pp) + optical_depth<R, true>(P, Pp, Q) + optical_depth<R, true>(P, Q, y);
}

// Term t of the kernel at x, t < 2 + P.n_extra: 0 the direct path, 1 the first
// wall's image (present when P.has_wall), t >= 2 further term t - 2.  Source
// point and weight, and the optical depth of the term's path to y.
template <class R>
__device__ __forceinline__ void term_source(const KernelParams& P, int t, const Vec3<R>& xi, const Vec3<R>& xb,
                                            Vec3<R>& src, R& scale)
{
    if (t < 2) {
        src = t == 0 ? xi : xb;
        scale = t == 0 ? R(1) : R(P.R0);
    } else {
        extra_term<R>(P, t - 2, xi, src, scale);
    }
}

template <class R>
__device__ __forceinline__ R term_depth(const KernelParams& P, int t, const Vec3<R>& xi, const Vec3<R>& src,
                                        const Vec3<R>& y)
{
    if (t == 0) return optical_depth<R, true>(P, xi, y);
    if (t == 1) {
        const Vec3<R> xp = wall_point<R>(P, src, y);
        return optical_depth<R, true>(P, xi, xp) + optical_depth<R, true>(P, xp, y);
    }
    return extra_tau<R>(P, t - 2, xi, src, y);
}

// Evaluates G_g^{ij} for all groups g < P.G with the whole warp; every lane
// returns the sums in acc.  s_tet / s_cnt / s_pre: per-warp shared scratch of
// 32, 32 and 33 ints.
template <class R, int MG, bool XT = false>
__device__ void entry_warp(const KernelParams& P, int i, int j, R (&acc)[MG], int* s_tet, int* s_cnt, int* s_pre)
{
    const int lane = threadIdx.x & 31;
    const Vec3<R> xi = load_xyz<R>(P, i);
    Vec3<R> xb = xi;
    if (P.has_wall) xb = mirror_point<R>(P, xi);
#pragma unroll
    for (int g = 0; g < MG; ++g) acc[g] = R(0);
    const int t0 = P.vt_ptr[j], t1 = P.vt_ptr[j + 1];
    const R inv4pi = R(1.0 / (4.0 * kPi));
    for (int base = t0; base < t1; base += 32) {
        const int nt = min(32, t1 - base);
        int cnt = 0;
        if (lane < nt) {
            int packed = P.vt_idx[base + lane];
            Vec3<R> cen;
            R diam, vol;
            load_tgeo<R>(P, packed >> 2, cen, diam, vol);
            R lim = R(4) * diam * diam;
            int nd = dist2<R>(xi, cen) < lim ? 14 : 4;
            int nr = P.has_wall ? (dist2<R>(xb, cen) < lim ? 14 : 4) : 0;
            cnt = nd + nr;
            s_tet[lane] = packed;
            s_cnt[lane] = nd | (nr << 8);
        }
        int pre = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        const int total = __shfl_sync(0xffffffffu, pre, 31);
        s_pre[lane] = pre - cnt;
        __syncwarp();
        for (int k = lane; k < total; k += 32) {
            // locate the tetrahedron: last t with s_pre[t] <= k
            int lo = 0, hi = nt - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (s_pre[mid] <= k) lo = mid; else hi = mid - 1;
            }
            const int t = lo;
            const int q = k - s_pre[t];
            const int packed = s_tet[t];
            const int nd = s_cnt[t] & 0xff, nr = s_cnt[t] >> 8;
            const int tet = packed >> 2, loc = packed & 3;
            const bool refl = q >= nd;
            const int qq = refl ? q - nd : q;
            const int nq = refl ? nr : nd;
            const int row = (nq == 14 ? 4 : 0) + qq;
            const int4 tv = P.tet[tet];
            const Vec3<R> v0 = load_xyz<R>(P, tv.x), v1 = load_xyz<R>(P, tv.y), v2 = load_xyz<R>(P, tv.z),
                          v3 = load_xyz<R>(P, tv.w);
            const R b0 = tet_b<R>(row, 0), b1 = tet_b<R>(row, 1), b2 = tet_b<R>(row, 2), b3 = tet_b<R>(row, 3);
            Vec3<R> y;
            y.x = b0 * v0.x + b1 * v1.x + b2 * v2.x + b3 * v3.x;
            y.y = b0 * v0.y + b1 * v1.y + b2 * v2.y + b3 * v3.y;
            y.z = b0 * v0.z + b1 * v1.z + b2 * v2.z + b3 * v3.z;
            const R lam = loc == 0 ? b0 : (loc == 1 ? b1 : (loc == 2 ? b2 : b3));
            R vol;
            if constexpr (sizeof(R) == 4) vol = P.tvol32[tet]; else vol = P.tvol64[tet];
            R r2, tau;
            if (!refl) {
                r2 = dist2<R>(xi, y);
                tau = optical_depth<R, XT>(P, xi, y);
            } else {
                Vec3<R> xp = wall_point<R>(P, xb, y);
                r2 = dist2<R>(xb, y);
                tau = optical_depth<R, XT>(P, xi, xp) + optical_depth<R, XT>(P, xp, y);
            }
            if constexpr (XT) {
                if (!(tau < R(INFINITY))) continue;   // path through an opaque box
            }
            R w = vol * tet_w<R>(row) * lam * kappa_at<R, XT>(P, y.x, y.y, y.z) * inv4pi / r2;
            if (refl) w *= R(P.R0);
            bool done = false;
            if constexpr (sizeof(R) == 4) {
                if (P.c_arith) {
                    // exp(-c_g tau) = exp(-c_0 tau) exp(-dc tau)^g
                    float E = expf(-P.c0f * tau);
                    const float D = expf(-P.dcf * tau);
#pragma unroll
                    for (int g = 0; g < MG; ++g) {
                        if (g < P.G) acc[g] += w * P.cf[g] * E;
                        E *= D;
                    }
                    done = true;
                }
            }
            if (!done) {
#pragma unroll
                for (int g = 0; g < MG; ++g)
                    if (g < P.G) {
                        R cg = kp_c<R>(P, g);
                        acc[g] += w * cg * exp_r(-cg * tau);
                    }
            }
        }
        __syncwarp();
    }
    // further walls and corner paths (instances with XT): lanes over the
    // tetrahedra, points in series
    for (int k = 0; k < (XT ? P.n_extra : 0); ++k) {
        Vec3<R> src;
        R scale;
        extra_term<R>(P, k, xi, src, scale);
        for (int e = t0 + lane; e < t1; e += 32) {
            const int packed = P.vt_idx[e];
            const int tet = packed >> 2, loc = packed & 3;
            Vec3<R> cen;
            R diam, vol;
            load_tgeo<R>(P, tet, cen, diam, vol);
            const int nq = dist2<R>(src, cen) < R(4) * diam * diam ? 14 : 4;
            const int4 tv = P.tet[tet];
            const Vec3<R> v0 = load_xyz<R>(P, tv.x), v1 = load_xyz<R>(P, tv.y), v2 = load_xyz<R>(P, tv.z),
                          v3 = load_xyz<R>(P, tv.w);
            for (int q = 0; q < nq; ++q) {
                const int row = (nq == 14 ? 4 : 0) + q;
                const R b0 = tet_b<R>(row, 0), b1 = tet_b<R>(row, 1), b2 = tet_b<R>(row, 2), b3 = tet_b<R>(row, 3);
                const Vec3<R> y = {b0 * v0.x + b1 * v1.x + b2 * v2.x + b3 * v3.x, b0 * v0.y + b1 * v1.y + b2 * v2.y + b3 * v3.y,
                                   b0 * v0.z + b1 * v1.z + b2 * v2.z + b3 * v3.z};
                const R lam = loc == 0 ? b0 : (loc == 1 ? b1 : (loc == 2 ? b2 : b3));
                const R tau = extra_tau<R>(P, k, xi, src, y);
                const R w = scale * vol * tet_w<R>(row) * lam * kappa_at<R, true>(P, y.x, y.y, y.z) * inv4pi / dist2<R>(src, y);
#pragma unroll
                for (int g = 0; g < MG; ++g)
                    if (g < P.G) {
                        const R cg = kp_c<R>(P, g);
                        acc[g] += w * cg * exp_r(-cg * tau);
                    }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < MG; ++g) {
        R v = acc[g];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[g] = v;
    }
}

}  // namespace rt
