// rt_newton.cuh -- the per-vertex temperature solve of the fixed point
// (Section 1.3, the balance of Eq. (RTb) discretised over the frequency grid):
// sum_nu wt_nu B_nu(T) = rhs with B_nu(T) = nu^3 / expm1(nu / T), by
// safeguarded Newton iteration with a bisection bracket, to |dT| <= 1e-14 T
// in FP64.  The iteration first runs in FP32 (an FP64 operation costs dozens
// of FP32 ones on this part) and then polishes the FP32 root in FP64 inside
// the FP32 bracket; whenever FP32 cannot represent the problem, or the polish
// ends on a bracket end, the plain FP64 iteration runs from the previous T.
#pragma once

#include <cstdint>

namespace rt {

// temperature from the Planck balance: LPV lanes per vertex (the power of two
// >= F, at most 32; 32 / LPV vertices per warp), lanes over the frequencies;
// B_nu and dB_nu/dT share one expm1 per frequency and Newton step:
//   B = nu^3 / em,  dB/dT = B (x / T) (1 + 1/em),  em = expm1(x),  x = nu / T.
// Sums over a vertex's lanes use shuffles masked to its LPV lanes, so the
// vertices of a warp iterate independently.
template <int LPV>
__device__ __forceinline__ unsigned seg_mask(int lane)
{
    if constexpr (LPV == 32) return 0xffffffffu;
    return ((1u << LPV) - 1u) << (lane & ~(LPV - 1));
}

template <int LPV, class R>
__device__ __forceinline__ void planck_sum(const double* __restrict__ fq, int F, R t, int lane, R& g, R& dg)
{
    const int sl = lane & (LPV - 1);
    g = R(0);
    dg = R(0);
    if (t > R(0)) {
        for (int f = sl; f < F; f += LPV) {
            const R nu = (R)fq[4 * f], wt = (R)fq[4 * f + 1];
            const R x = nu / t;
            if constexpr (sizeof(R) == 8) {
                if (x < R(700)) {
                    const R em = expm1(x);
                    const R B = nu * nu * nu / em;
                    g += wt * B;
                    dg += wt * B * (x / t) * (R(1) + R(1) / em);
                }
            } else {
                if (x < R(80)) {
                    const R em = expm1f(x);
                    const R B = nu * nu * nu / em;
                    g += wt * B;
                    dg += wt * B * (x / t) * (R(1) + R(1) / em);
                }
            }
        }
    }
    const unsigned m = seg_mask<LPV>(lane);
#pragma unroll
    for (int o = LPV >> 1; o > 0; o >>= 1) {
        g += __shfl_xor_sync(m, g, o);
        dg += __shfl_xor_sync(m, dg, o);
    }
}

// Safeguarded Newton for sum_nu wt_nu B_nu(T) = rhs in FP64, started from t in
// the bracket [lo, hi] (g(lo) <= rhs <= g(hi)); stops when a step moves T by at
// most 1e-14 T.  Returns false after 100 steps without that.
template <int LPV>
__device__ bool newton64(const double* __restrict__ fq, int F, double rhs, int lane, double& t, double lo, double hi)
{
    double g, dg;
    for (int it = 0; it < 100; ++it) {
        planck_sum<LPV>(fq, F, t, lane, g, dg);
        const double fv = g - rhs;
        if (fv < 0.0) lo = t;
        if (fv > 0.0) hi = t;
        double tn = dg > 0.0 ? t - fv / dg : 0.5 * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        const bool done = fabs(tn - t) <= 1e-14 * fabs(tn);
        t = tn;
        if (done || fv == 0.0) return true;
    }
    return false;
}

// FP64 bracket [0, hi] by doubling from max(1, 2 tp), then Newton from tp
template <int LPV>
__device__ bool newton64_full(const double* __restrict__ fq, int F, double rhs, int lane, double tp, double& t)
{
    double lo = 0.0, hi = fmax(1.0, 2.0 * tp);
    double g, dg;
    planck_sum<LPV>(fq, F, hi, lane, g, dg);
    int guard = 0;
    while (g < rhs && guard < 200) {
        lo = hi;
        hi *= 2.0;
        planck_sum<LPV>(fq, F, hi, lane, g, dg);
        ++guard;
    }
    t = (tp > lo && tp < hi) ? tp : 0.5 * (lo + hi);
    return newton64<LPV>(fq, F, rhs, lane, t, lo, hi);
}

// The same safeguarded Newton iteration in FP32 (one FP64 step costs as much
// as dozens of FP32 steps on this part): returns the FP32 root and the last
// bracket, or false when FP32 cannot represent the problem (rhs out of the
// normal range, no bracket, no convergence).
template <int LPV>
__device__ bool newton32(const double* __restrict__ fq, int F, double rhs, int lane, double tp, float& t, float& lo,
                         float& hi)
{
    if (!(rhs > 1e-30 && rhs < 1e30)) return false;
    const float r = (float)rhs;
    float g, dg;
    lo = 0.f;
    hi = fmaxf(1.f, 2.f * (float)tp);
    planck_sum<LPV>(fq, F, hi, lane, g, dg);
    int guard = 0;
    while (g < r && guard < 100) {
        lo = hi;
        hi *= 2.f;
        planck_sum<LPV>(fq, F, hi, lane, g, dg);
        ++guard;
    }
    if (!(g >= r)) return false;
    const float tpf = (float)tp;
    t = (tpf > lo && tpf < hi) ? tpf : 0.5f * (lo + hi);
    for (int it = 0; it < 60; ++it) {
        planck_sum<LPV>(fq, F, t, lane, g, dg);
        const float fv = g - r;
        if (fv < 0.f) lo = t;
        if (fv > 0.f) hi = t;
        float tn = dg > 0.f ? t - fv / dg : 0.5f * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = 0.5f * (lo + hi);
        const bool done = fabsf(tn - t) <= 3e-6f * fabsf(tn);
        t = tn;
        if (done || fv == 0.f) return t > 0.f;
    }
    return false;
}

// T for one vertex (LPV lanes, all of them call): false when no iteration met
// the stopping rule within its step limit
template <int LPV>
__device__ bool solve_temperature(const double* __restrict__ fq, int F, double rhs, int lane, double tp, double& t)
{
    float t32, lo32, hi32;
    bool ok = false;
    if (newton32<LPV>(fq, F, rhs, lane, tp, t32, lo32, hi32)) {
        // polish in FP64 inside the FP32 bracket widened by 1e-4 (an FP32 sign
        // test can misjudge only points within FP32 rounding of the root)
        const double lo = (double)lo32 * (1.0 - 1e-4), hi = (double)hi32 * (1.0 + 1e-4);
        t = (double)t32;
        ok = newton64<LPV>(fq, F, rhs, lane, t, lo, hi);
        // a root pressed against a bracket end means the bracket was wrong
        if (ok && (fabs(t - lo) <= 1e-12 * t || fabs(t - hi) <= 1e-12 * t)) ok = false;
    }
    if (!ok) ok = newton64_full<LPV>(fq, F, rhs, lane, tp, t);
    return ok;
}

}  // namespace rt
