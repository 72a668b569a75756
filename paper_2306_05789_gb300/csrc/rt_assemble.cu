// rt_assemble.cu -- assembly of the operator on the GPU (Section 2, 2.1):
//   * constants: Gauss-Legendre nodes, tetrahedron and triangle rules
//   * entry kernels (warp per entry) for dense blocks, ACA rows/columns and
//     arbitrary entry lists
//   * the emitter source Sbar^E
//   * batched partially pivoted ACA with pivots shared by all kappa groups
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rt_entry.cuh"
#include "rt_internal.h"

namespace rt {


// ---------------------------------------------------------------------------
// host: quadrature tables
// ---------------------------------------------------------------------------
// Gauss-Legendre nodes: Newton iteration on P_n from the asymptotic guess
// cos(pi (4k + 3) / (4n + 2)); P_n and P_n' from the three-term recurrence.
void gauss_legendre_nodes(int n, std::vector<double>& t, std::vector<double>& w)
{
    t.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        double x = std::cos(kPi * (4.0 * k + 3.0) / (4.0 * n + 2.0));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1.0, p = x;
            for (int l = 1; l < n; ++l) {
                double pn = ((2.0 * l + 1.0) * x * p - l * pm) / (l + 1.0);
                pm = p;
                p = pn;
            }
            dp = n * (pm - x * p) / (1.0 - x * x);
            double step = p / dp;
            x -= step;
            if (std::fabs(step) <= 1e-16 * std::fabs(x) + 1e-300) break;
        }
        {
            double pm = 1.0, p = x;
            for (int l = 1; l < n; ++l) {
                double pn = ((2.0 * l + 1.0) * x * p - l * pm) / (l + 1.0);
                pm = p;
                p = pn;
            }
            dp = n * (pm - x * p) / (1.0 - x * x);
        }
        t[k] = x;
        w[k] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

// Tetrahedron rules in barycentric coordinates: the symmetric 4-point rule of
// degree 2 and the positive 14-point rule of degree 5 (two S31 orbits, one S22
// orbit); triangle rules: 3-point degree 2 and Radon's 7-point degree 5.
static void tet_rules(double* b, double* w)
{
    const double al = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, be = (5.0 - std::sqrt(5.0)) / 20.0;
    int r = 0;
    for (int k = 0; k < 4; ++k, ++r) {
        for (int d = 0; d < 4; ++d) b[4 * r + d] = d == k ? al : be;
        w[r] = 0.25;
    }
    const double s31[2][2] = {{0.0927352503108912, 0.07349304311636196}, {0.3108859192633006, 0.1126879257180159}};
    for (int o = 0; o < 2; ++o)
        for (int k = 0; k < 4; ++k, ++r) {
            for (int d = 0; d < 4; ++d) b[4 * r + d] = d == k ? 1.0 - 3.0 * s31[o][0] : s31[o][0];
            w[r] = s31[o][1];
        }
    const double s22 = 0.4544962958743504, ws22 = 0.04254602077708147;
    for (int a = 0; a < 4; ++a)
        for (int c = a + 1; c < 4; ++c, ++r) {
            for (int d = 0; d < 4; ++d) b[4 * r + d] = (d == a || d == c) ? s22 : 0.5 - s22;
            w[r] = ws22;
        }
}

static void tri_rules(double* b, double* w)
{
    int r = 0;
    for (int k = 0; k < 3; ++k, ++r) {
        for (int d = 0; d < 3; ++d) b[3 * r + d] = d == k ? 2.0 / 3.0 : 1.0 / 6.0;
        w[r] = 1.0 / 3.0;
    }
    b[3 * r] = b[3 * r + 1] = b[3 * r + 2] = 1.0 / 3.0;
    w[r++] = 0.225;
    const double q = std::sqrt(15.0);
    const double orb[2][2] = {{(6.0 - q) / 21.0, (155.0 - q) / 1200.0}, {(6.0 + q) / 21.0, (155.0 + q) / 1200.0}};
    for (int o = 0; o < 2; ++o)
        for (int k = 0; k < 3; ++k, ++r) {
            for (int d = 0; d < 3; ++d) b[3 * r + d] = d == k ? 1.0 - 2.0 * orb[o][0] : orb[o][0];
            w[r] = orb[o][1];
        }
}

int assemble_setup_constants(Operator& op, std::string& err)
{
    std::vector<double> t, w;
    gauss_legendre_nodes(op.ngauss, t, w);
    for (int g = 0; g < kMaxGauss; ++g) {
        const double u = g < op.ngauss ? 0.5 * (1.0 + t[g]) : 0.0, hw = g < op.ngauss ? 0.5 * w[g] : 0.0;
        op.kp.gu64[g] = u;
        op.kp.gw64[g] = hw;
        op.kp.gu32[g] = (float)u;
        op.kp.gw32[g] = (float)hw;
    }
    // fixed rule tables: uploaded once per device (serialised across host threads)
    static bool done[64] = {false};
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 64 && done[dev]) return RT_OK;
    double tb[18 * 4], tw[18];
    float tbf[18 * 4], twf[18];
    tet_rules(tb, tw);
    for (int k = 0; k < 72; ++k) tbf[k] = (float)tb[k];
    for (int k = 0; k < 18; ++k) twf[k] = (float)tw[k];
    double rb[30], rw[10];
    tri_rules(rb, rw);
    RT_CUDA_TRY(cudaMemcpyToSymbol(c_tet_b, tb, sizeof(tb)));
    RT_CUDA_TRY(cudaMemcpyToSymbol(c_tet_w, tw, sizeof(tw)));
    RT_CUDA_TRY(cudaMemcpyToSymbol(c_tet_bf, tbf, sizeof(tbf)));
    RT_CUDA_TRY(cudaMemcpyToSymbol(c_tet_wf, twf, sizeof(twf)));
    RT_CUDA_TRY(cudaMemcpyToSymbol(c_tri_b, rb, sizeof(rb)));
    RT_CUDA_TRY(cudaMemcpyToSymbol(c_tri_w, rw, sizeof(rw)));
    RT_CUDA_TRY(cudaDeviceSynchronize());
    if (dev < 64) done[dev] = true;
    return RT_OK;
}

// ---------------------------------------------------------------------------
// entry kernels
// ---------------------------------------------------------------------------
constexpr int kWarpsPerCta = 8;

__device__ __forceinline__ int find_span(const EntrySpan* sp, int ns, int64_t e)
{
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sp[mid].first <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class R, class OUT, int MG, bool XT = false>
__global__ void __launch_bounds__(32 * kWarpsPerCta) entries_span_kernel(KernelParams P, const EntrySpan* spans,
                                                                         int nspans, int64_t total, OUT* out)
{
    __shared__ int s_tet[kWarpsPerCta][32], s_cnt[kWarpsPerCta][32], s_pre[kWarpsPerCta][33];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerCta;
    for (int64_t e = (int64_t)blockIdx.x * kWarpsPerCta + wib; e < total; e += nw) {
        const int si = find_span(spans, nspans, e);
        const EntrySpan sp = spans[si];
        const int64_t loc = e - sp.first;
        const int ii = (int)(loc / sp.nj), jj = (int)(loc % sp.nj);
        R acc[MG];
        entry_warp<R, MG, XT>(P, sp.i0 + ii, sp.j0 + jj, acc, s_tet[wib], s_cnt[wib], s_pre[wib]);
#pragma unroll
        for (int g = 0; g < MG; ++g)
            if (g < P.G && lane == (g & 31)) out[sp.base + g * sp.gs + ii * sp.is + jj * sp.js] = (OUT)acc[g];
    }
}

// ACA rows (mode 0) / columns (mode 1) of the active far blocks.
struct AcaActive {
    int b;          // far block id
    int row0, m, col0, n;
    int64_t rbuf;   // offset of this block's [G][n] row buffer
    int64_t cbuf;   // offset of this block's [G][m] column buffer
    int64_t first_row, first_col;   // prefix of n (rows) and m (cols) over the active list
    int64_t uoff, voff;             // pool offsets of this step's u [G][m] and v [G][n]
    int64_t dot0;                   // first entry of this block's rank+1 dot products this step
    int64_t first_chunk;            // prefix of ceil(m / kColRows) over the active list
    int skip;       // set by the pivot kernel: zero row, no rank this step
};

__device__ __forceinline__ int find_active(const AcaActive* a, int na, int64_t e, int mode)
{
    int lo = 0, hi = na - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int64_t f = mode == 0 ? a[mid].first_row : (mode == 1 ? a[mid].first_col : a[mid].first_chunk);
        if (f <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ACA pivot columns: G_g[i, j*] for the rows i of an active block.  One CTA of
// kColRows threads per chunk of kColRows rows.  The quadrature points of the
// tetrahedra around the pivot vertex j* do not depend on the row, so each CTA
// tabulates them once per batch of 32 tetrahedra in shared memory (position,
// and vol * w_q * lambda_j(y) * kappa(y) / 4 pi for both rules) and every row
// walks the table -- the sums of entry_warp, with each point's position,
// kappa and hat-function weight computed once per chunk instead of per entry.
constexpr int kColRows = 64;
constexpr int kColTets = 32;

// acc[g] += w exp(-c_g tau) over the groups; the factor c_g of Eq. 5 (the
// group scale of the multi-frequency operator) multiplies the finished sums.
// exp recurrence when c_g is arithmetic.
template <int MG, bool XT = false>
__device__ __forceinline__ void row_accumulate(const KernelParams& P, float (&acc)[MG], float w, float tau)
{
    if constexpr (XT) {
        if (!(tau < INFINITY)) return;   // path through an opaque box
    }
    if (P.c_arith) {
        float E = expf(-P.c0f * tau);
        const float D = expf(-P.dcf * tau);
#pragma unroll
        for (int g = 0; g < MG; ++g) {
            if (g < P.G) acc[g] += w * E;
            E *= D;
        }
    } else {
#pragma unroll
        for (int g = 0; g < MG; ++g)
            if (g < P.G) acc[g] += w * expf(-P.cf[g] * tau);
    }
}

// add this thread's counts to the work counters (one atomic per warp and counter)
__device__ __forceinline__ void count_work(const KernelParams& P, unsigned terms, unsigned depths)
{
    if (!P.work) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        terms += __shfl_xor_sync(0xffffffffu, terms, o);
        depths += __shfl_xor_sync(0xffffffffu, depths, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(P.work, (unsigned long long)terms);
        atomicAdd(P.work + 1, (unsigned long long)depths);
    }
}

template <int MG, bool XT = false>
__global__ void __launch_bounds__(kColRows) aca_col_kernel(KernelParams P, const AcaActive* __restrict__ act, int na,
                                                           int64_t nchunks, const int* __restrict__ jstar,
                                                           float* __restrict__ buf)
{
    __shared__ float4 s_pt[kColTets][18];   // rule rows 0-3: 4-point rule, 4-17: 14-point rule
    __shared__ float4 s_cen[kColTets];      // centroid, 4 diam^2
    const float inv4pi = (float)(1.0 / (4.0 * kPi));
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int ai = find_active(act, na, c, 2);
        const AcaActive a = act[ai];
        if (a.skip) continue;   // CTA-uniform
        const int r0 = (int)(c - a.first_chunk) * kColRows;
        const int j = a.col0 + jstar[a.b];
        const int pos = r0 + threadIdx.x;
        const bool row_ok = pos < a.m;
        const int i = a.row0 + (row_ok ? pos : 0);
        const Vec3<float> xi = load_xyz<float>(P, i);
        Vec3<float> xb = xi;
        if (P.has_wall) xb = mirror_point<float>(P, xi);
        float acc[MG];
#pragma unroll
        for (int g = 0; g < MG; ++g) acc[g] = 0.f;
        const int t0 = P.vt_ptr[j], t1 = P.vt_ptr[j + 1];
        unsigned n_terms = 0, n_depths = 0;
        for (int b0 = t0; b0 < t1; b0 += kColTets) {
            const int nt = min(kColTets, t1 - b0);
            __syncthreads();   // the previous batch's table is no longer read
            for (int e = threadIdx.x; e < nt * 18; e += blockDim.x) {
                const int t = e / 18, q = e - t * 18;
                const int packed = P.vt_idx[b0 + t];
                const int tet = packed >> 2, loc = packed & 3;
                const int4 tv = P.tet[tet];
                const Vec3<float> v0 = load_xyz<float>(P, tv.x), v1 = load_xyz<float>(P, tv.y),
                                  v2 = load_xyz<float>(P, tv.z), v3 = load_xyz<float>(P, tv.w);
                const float b0w = tet_b<float>(q, 0), b1 = tet_b<float>(q, 1), b2 = tet_b<float>(q, 2),
                            b3 = tet_b<float>(q, 3);
                Vec3<float> y;
                y.x = b0w * v0.x + b1 * v1.x + b2 * v2.x + b3 * v3.x;
                y.y = b0w * v0.y + b1 * v1.y + b2 * v2.y + b3 * v3.y;
                y.z = b0w * v0.z + b1 * v1.z + b2 * v2.z + b3 * v3.z;
                const float lam = loc == 0 ? b0w : (loc == 1 ? b1 : (loc == 2 ? b2 : b3));
                const float w = P.tvol32[tet] * tet_w<float>(q) * lam * kappa_at<float, XT>(P, y.x, y.y, y.z) * inv4pi;
                s_pt[t][q] = make_float4(y.x, y.y, y.z, w);
                if (q == 0) {
                    Vec3<float> cen;
                    float diam, vol;
                    load_tgeo<float>(P, tet, cen, diam, vol);
                    s_cen[t] = make_float4(cen.x, cen.y, cen.z, 4.f * diam * diam);
                }
            }
            __syncthreads();
            if (row_ok) {
                for (int t = 0; t < nt; ++t) {
                    const float4 ce = s_cen[t];
                    const Vec3<float> cen = {ce.x, ce.y, ce.z};
                    const int nd = dist2<float>(xi, cen) < ce.w ? 14 : 4;
                    const int nr = P.has_wall ? (dist2<float>(xb, cen) < ce.w ? 14 : 4) : 0;
                    n_terms += nd + nr;
                    n_depths += nd + 2 * nr;
                    // direct points first, then the mirror-reflected ones: two
                    // loops, so that lanes whose rules differ never run the
                    // direct and the reflected branch at the same step
                    const float4* pd = s_pt[t] + (nd == 14 ? 4 : 0);
                    for (int q = 0; q < nd; ++q) {
                        const float4 pt = pd[q];
                        const Vec3<float> y = {pt.x, pt.y, pt.z};
                        row_accumulate<MG, XT>(P, acc, pt.w / dist2<float>(xi, y), optical_depth<float, XT>(P, xi, y));
                    }
                    const float4* pr = s_pt[t] + (nr == 14 ? 4 : 0);
                    for (int q = 0; q < nr; ++q) {
                        const float4 pt = pr[q];
                        const Vec3<float> y = {pt.x, pt.y, pt.z};
                        const Vec3<float> xp = wall_point<float>(P, xb, y);
                        const float tau = optical_depth<float, XT>(P, xi, xp) + optical_depth<float, XT>(P, xp, y);
                        row_accumulate<MG, XT>(P, acc, (float)P.R0 * pt.w / dist2<float>(xb, y), tau);
                    }
                    if constexpr (XT) {   // further walls, corner paths
                        for (int k = 0; k < P.n_extra; ++k) {
                            Vec3<float> src;
                            float sc;
                            extra_term<float>(P, k, xi, src, sc);
                            const int nx = dist2<float>(src, cen) < ce.w ? 14 : 4;
                            n_terms += nx;
                            n_depths += nx * (P.xkind[k] + 1);
                            const float4* px = s_pt[t] + (nx == 14 ? 4 : 0);
                            for (int q = 0; q < nx; ++q) {
                                const float4 pt = px[q];
                                const Vec3<float> y = {pt.x, pt.y, pt.z};
                                row_accumulate<MG, XT>(P, acc, sc * pt.w / dist2<float>(src, y),
                                                   extra_tau<float>(P, k, xi, src, y));
                            }
                        }
                    }
                }
            }
        }
        if (row_ok) {
#pragma unroll
            for (int g = 0; g < MG; ++g)
                if (g < P.G) buf[a.cbuf + (int64_t)g * a.m + pos] = acc[g] * P.cf[g];
        }
        count_work(P, n_terms, n_depths);
    }
}

// Arbitrary (row, col) pairs, internal vertex ids.
template <class R, int MG, bool XT = false>
__global__ void __launch_bounds__(32 * kWarpsPerCta) entries_pairs_kernel(KernelParams P, int group, int64_t count,
                                                                          const int32_t* rows, const int32_t* cols,
                                                                          const int* iperm, double* out)
{
    __shared__ int s_tet[kWarpsPerCta][32], s_cnt[kWarpsPerCta][32], s_pre[kWarpsPerCta][33];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarpsPerCta;
    for (int64_t e = (int64_t)blockIdx.x * kWarpsPerCta + wib; e < count; e += nw) {
        int i = rows[e], j = cols[e];
        if (iperm) {
            i = iperm[i];
            j = iperm[j];
        }
        R acc[MG];
        entry_warp<R, MG, XT>(P, i, j, acc, s_tet[wib], s_cnt[wib], s_pre[wib]);
        R v = R(0);
#pragma unroll
        for (int g = 0; g < MG; ++g)
            if (g == group) v = acc[g];
        if (lane == 0) out[e] = (double)v;
    }
}

static int grid_for(int64_t warps)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t ctas = (warps + kWarpsPerCta - 1) / kWarpsPerCta;
    int64_t cap = (int64_t)sms * 16;
    return (int)std::max<int64_t>(1, std::min(ctas, cap));
}

// Dispatch on the group count: the accumulator array is sized at compile time.
// general kernels (XT: further walls and corner terms, a kappa grid, opaque
// boxes): 16 or 64 group slots
#define RT_DISPATCH_MG_XT(G, MACRO) \
    do {                            \
        if ((G) <= 16) {            \
            MACRO(16, true);        \
        } else {                    \
            MACRO(64, true);        \
        }                           \
    } while (0)

#define RT_DISPATCH_MG(G, MACRO) \
    do {                         \
        if ((G) <= 1) {          \
            MACRO(1);            \
        } else if ((G) <= 4) {   \
            MACRO(4);            \
        } else if ((G) <= 8) {   \
            MACRO(8);            \
        } else if ((G) <= 16) {  \
            MACRO(16);           \
        } else if ((G) <= 32) {  \
            MACRO(32);           \
        } else {                 \
            MACRO(64);           \
        }                        \
    } while (0)

template <class R, class OUT>
static int launch_spans(Operator& op, const std::vector<EntrySpan>& spans_in, OUT* out, cudaStream_t s,
                        std::string& err)
{
    if (spans_in.empty()) return RT_OK;
    std::vector<EntrySpan> spans = spans_in;
    int64_t total = 0;
    for (auto& sp : spans) {
        sp.first = total;
        total += (int64_t)sp.ni * sp.nj;
    }
    EntrySpan* d_sp = nullptr;
    RT_CUDA_TRY(cudaMallocAsync((void**)&d_sp, spans.size() * sizeof(EntrySpan), s));
    RT_CUDA_TRY(cudaMemcpyAsync(d_sp, spans.data(), spans.size() * sizeof(EntrySpan), cudaMemcpyHostToDevice, s));
    int grid = grid_for(total);
    const int ns = (int)spans.size();
#define RT_LAUNCH_SPANS(MG, XT) \
    entries_span_kernel<R, OUT, MG, XT><<<grid, 32 * kWarpsPerCta, 0, s>>>(op.kp, d_sp, ns, total, out)
#define RT_LAUNCH_SPANS1(MG) RT_LAUNCH_SPANS(MG, false)
    if (op.kp.ext) RT_DISPATCH_MG_XT(op.G, RT_LAUNCH_SPANS);
    else RT_DISPATCH_MG(op.G, RT_LAUNCH_SPANS1);
#undef RT_LAUNCH_SPANS1
#undef RT_LAUNCH_SPANS
    RT_CUDA_TRY(cudaGetLastError());
    RT_CUDA_TRY(cudaFreeAsync(d_sp, s));
    op.info.entries_evaluated += total;
    return RT_OK;
}

// ---------------------------------------------------------------------------
// dense mode: the whole matrix [G][N][N] row-major
// ---------------------------------------------------------------------------
int assemble_dense(Operator& op, cudaStream_t s, std::string& err)
{
    const int64_t N = op.N;
    const size_t esz = op.prec == RT_PREC_F64 ? 8 : 4;
    int rc;
    if (op.prec == RT_PREC_F64) {
        double* d = nullptr;
        if ((rc = dev_alloc(op, &d, (size_t)op.G * N * N, err))) return rc;
        op.d_dense = d;
    } else {
        float* d = nullptr;
        if ((rc = dev_alloc(op, &d, (size_t)op.G * N * N, err))) return rc;
        op.d_dense = d;
    }
    // one span per row band keeps every span's entry count below 2^31
    std::vector<EntrySpan> spans;
    const int band = (int)std::max<int64_t>(1, std::min<int64_t>(N, (1 << 26) / std::max<int64_t>(N, 1)));
    for (int64_t r0 = 0; r0 < N; r0 += band) {
        EntrySpan sp{};
        sp.i0 = (int)r0;
        sp.ni = (int)std::min<int64_t>(band, N - r0);
        sp.j0 = 0;
        sp.nj = (int)N;
        sp.base = r0 * N;
        sp.gs = N * N;
        sp.is = N;
        sp.js = 1;
        spans.push_back(sp);
    }
    if (op.prec == RT_PREC_F64) rc = launch_spans<double, double>(op, spans, (double*)op.d_dense, s, err);
    else rc = launch_spans<float, float>(op, spans, (float*)op.d_dense, s, err);
    if (rc) return rc;
    op.info.stored_entries = N * N;
    op.info.apply_bytes = (int64_t)op.F * N * N * (int64_t)esz + 2 * (int64_t)op.F * N * (int64_t)esz;
    op.info.apply_flops = 2 * (int64_t)op.F * N * N;
    return RT_OK;
}

int eval_entries(Operator& op, int group, int64_t count, const int32_t* rows, const int32_t* cols, double* out,
                 cudaStream_t s, std::string& err)
{
    if (count <= 0) return RT_OK;
    int grid = grid_for(count);
    const int* ip = op.d_iperm;
    if (op.prec == RT_PREC_F64) {
#define RT_LAUNCH_PAIRS(MG, XT) \
    entries_pairs_kernel<double, MG, XT><<<grid, 32 * kWarpsPerCta, 0, s>>>(op.kp, group, count, rows, cols, ip, out)
#define RT_LAUNCH_PAIRS1(MG) RT_LAUNCH_PAIRS(MG, false)
        if (op.kp.ext) RT_DISPATCH_MG_XT(op.G, RT_LAUNCH_PAIRS);
        else RT_DISPATCH_MG(op.G, RT_LAUNCH_PAIRS1);
#undef RT_LAUNCH_PAIRS1
#undef RT_LAUNCH_PAIRS
    } else {
#define RT_LAUNCH_PAIRS(MG, XT) \
    entries_pairs_kernel<float, MG, XT><<<grid, 32 * kWarpsPerCta, 0, s>>>(op.kp, group, count, rows, cols, ip, out)
#define RT_LAUNCH_PAIRS1(MG) RT_LAUNCH_PAIRS(MG, false)
        if (op.kp.ext) RT_DISPATCH_MG_XT(op.G, RT_LAUNCH_PAIRS);
        else RT_DISPATCH_MG(op.G, RT_LAUNCH_PAIRS1);
#undef RT_LAUNCH_PAIRS1
#undef RT_LAUNCH_PAIRS
    }
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

// ---------------------------------------------------------------------------
// emitter source Sbar^E (Example of Section 1.2, Section 2)
// ---------------------------------------------------------------------------
// Shat_g(x_i) = (1/4pi) int_{Gamma_Q} ([(x-y).n]_-)^2 e^{-c_g tau(x,y)}/|x-y|^4
//             + R0 ([(xbar-y).n]_-)^2 e^{-c_g(tau(x,x')+tau(x',y))}/|xbar-y|^4 dGamma(y),
// 7-point rule within two diameters of the triangle centroid, 3-point rule
// otherwise; a source point that is a vertex of the triangle contributes the
// limit (angle at the vertex)/(8 pi) (times R0 for the image term).
// One warp per vertex; lanes over triangles.  out[f][i] = Q_f Shat_{g(f)}(x_i).
template <class R, int MG>
__global__ void __launch_bounds__(256) source_kernel(KernelParams P, int n_emit, const int4* emit, const int* fgroup,
                                                     const double* Q, int F, R* out)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const R inv4pi = R(1.0 / (4.0 * kPi));
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < P.N; i += nw) {
        const Vec3<R> xi = load_xyz<R>(P, (int)i);
        Vec3<R> xb = xi;
        bool on_wall = false;
        if (P.has_wall) {
            xb = mirror_point<R>(P, xi);
            on_wall = dist2<R>(xi, xb) <= R(1e-20);
        }
        R acc[MG];
#pragma unroll
        for (int g = 0; g < MG; ++g) acc[g] = R(0);
        for (int e = lane; e < n_emit; e += 32) {
            const int4 tv = emit[e];
            const Vec3<R> V0 = load_xyz<R>(P, tv.x), V1 = load_xyz<R>(P, tv.y), V2 = load_xyz<R>(P, tv.z);
            const Vec3<R> e1 = {V1.x - V0.x, V1.y - V0.y, V1.z - V0.z};
            const Vec3<R> e2 = {V2.x - V0.x, V2.y - V0.y, V2.z - V0.z};
            Vec3<R> nn = {e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x};
            const R a2 = sqrt_r(nn.x * nn.x + nn.y * nn.y + nn.z * nn.z);
            nn.x /= a2;
            nn.y /= a2;
            nn.z /= a2;
            const R area = R(0.5) * a2;
            const Vec3<R> cen = {(V0.x + V1.x + V2.x) / R(3), (V0.y + V1.y + V2.y) / R(3), (V0.z + V1.z + V2.z) / R(3)};
            R diam2 = dist2<R>(V0, V1);
            diam2 = fmax(diam2, dist2<R>(V0, V2));
            diam2 = fmax(diam2, dist2<R>(V1, V2));
            int vloc = tv.x == (int)i ? 0 : (tv.y == (int)i ? 1 : (tv.z == (int)i ? 2 : -1));
            for (int term = 0; term < 2 + P.n_extra; ++term) {
                if (term == 1 && !P.has_wall) continue;
                Vec3<R> src;
                R scale;
                term_source<R>(P, term, xi, xb, src, scale);
                // the source point is x itself: always for the direct term, for an
                // image when x lies on its wall(s)
                const bool at_x = term == 0 || (term == 1 ? on_wall : dist2<R>(xi, src) <= R(1e-20));
                if (vloc >= 0 && at_x) {
                    // limit at a vertex of the emitter: angle / (8 pi)
                    const Vec3<R> A = vloc == 0 ? V0 : (vloc == 1 ? V1 : V2);
                    const Vec3<R> B = vloc == 0 ? V1 : (vloc == 1 ? V2 : V0);
                    const Vec3<R> C = vloc == 0 ? V2 : (vloc == 1 ? V0 : V1);
                    const Vec3<R> u = {B.x - A.x, B.y - A.y, B.z - A.z}, v = {C.x - A.x, C.y - A.y, C.z - A.z};
                    R cs = (u.x * v.x + u.y * v.y + u.z * v.z) / sqrt_r((u.x * u.x + u.y * u.y + u.z * u.z) *
                                                                         (v.x * v.x + v.y * v.y + v.z * v.z));
                    cs = fmin(R(1), fmax(R(-1), cs));
                    const R lim = scale * acos(cs) * R(1.0 / (8.0 * kPi));
#pragma unroll
                    for (int g = 0; g < MG; ++g)
                        if (g < P.G) acc[g] += lim;
                    continue;
                }
                const R sd = (src.x - V0.x) * nn.x + (src.y - V0.y) * nn.y + (src.z - V0.z) * nn.z;
                if (!(sd < R(0))) continue;
                const R cm = -sd;
                const bool nearp = dist2<R>(src, cen) < R(4) * diam2;
                const int q0 = nearp ? 3 : 0, nq = nearp ? 7 : 3;
                for (int q = 0; q < nq; ++q) {
                    const R b0 = R(c_tri_b[3 * (q0 + q)]), b1 = R(c_tri_b[3 * (q0 + q) + 1]),
                            b2 = R(c_tri_b[3 * (q0 + q) + 2]);
                    const Vec3<R> y = {b0 * V0.x + b1 * V1.x + b2 * V2.x, b0 * V0.y + b1 * V1.y + b2 * V2.y,
                                       b0 * V0.z + b1 * V1.z + b2 * V2.z};
                    const R r2 = dist2<R>(src, y);
                    const R tau = term_depth<R>(P, term, xi, src, y);
                    const R geo = scale * area * R(c_tri_w[q0 + q]) * cm * cm / (r2 * r2) * inv4pi;
#pragma unroll
                    for (int g = 0; g < MG; ++g)
                        if (g < P.G) acc[g] += geo * exp_r(-kp_c<R>(P, g) * tau);
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
        if (lane == 0) {
            for (int f = 0; f < F; ++f) {
                R v = R(0);
#pragma unroll
                for (int g = 0; g < MG; ++g)
                    if (g == fgroup[f]) v = acc[g];
                out[(int64_t)f * P.N + i] = R(Q[f]) * v;
            }
        }
    }
}

int assemble_source(Operator& op, cudaStream_t s, std::string& err)
{
    int rc;
    int* d_fg = nullptr;
    double* d_Q = nullptr;
    RT_CUDA_TRY(cudaMallocAsync((void**)&d_fg, sizeof(int) * op.F, s));
    RT_CUDA_TRY(cudaMallocAsync((void**)&d_Q, sizeof(double) * op.F, s));
    RT_CUDA_TRY(cudaMemcpyAsync(d_fg, op.fgroup.data(), sizeof(int) * op.F, cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaMemcpyAsync(d_Q, op.Q.data(), sizeof(double) * op.F, cudaMemcpyHostToDevice, s));
    const int grid = grid_for(op.N);
    if (op.vec64) {
        double* d = nullptr;
        if ((rc = dev_alloc(op, &d, (size_t)op.F * op.N, err))) return rc;
        op.d_SE = d;
#define RT_LAUNCH_SRC(MG) \
    source_kernel<double, MG><<<grid, 256, 0, s>>>(op.kp, op.n_emit, op.d_emit, d_fg, d_Q, op.F, d)
        RT_DISPATCH_MG(op.G, RT_LAUNCH_SRC);
#undef RT_LAUNCH_SRC
    } else {
        float* d = nullptr;
        if ((rc = dev_alloc(op, &d, (size_t)op.F * op.N, err))) return rc;
        op.d_SE = d;
#define RT_LAUNCH_SRC(MG) \
    source_kernel<float, MG><<<grid, 256, 0, s>>>(op.kp, op.n_emit, op.d_emit, d_fg, d_Q, op.F, d)
        RT_DISPATCH_MG(op.G, RT_LAUNCH_SRC);
#undef RT_LAUNCH_SRC
    }
    RT_CUDA_TRY(cudaGetLastError());
    RT_CUDA_TRY(cudaFreeAsync(d_fg, s));
    RT_CUDA_TRY(cudaFreeAsync(d_Q, s));
    return RT_OK;
}

// ---------------------------------------------------------------------------
// Row evaluation over a column cluster: G_g[i, j] for every column j of a
// sub-cluster (at most kSubCols consecutive tree-order columns).  Each
// tetrahedron touching the sub-cluster is visited once: every quadrature
// point's kernel value feeds the (up to 4) hat functions of the tetrahedron's
// vertices that lie in the sub-cluster -- the same sums as entry_warp, in a
// different order, with each point evaluated once instead of once per vertex.
// One CTA per (row, sub-cluster); the row segment accumulates in shared
// memory [G][n] (float atomics, so the summation order is not fixed).
// ---------------------------------------------------------------------------
// threads of one row-over-cluster CTA: a (row, sub-cluster) item has a few
// hundred tetrahedra, so 128 threads keep each thread busy on several of them
// and let four CTAs per SM hide one another's end-of-item barrier
constexpr int kRowThreads = 128;

struct RowItem {
    int b;            // ACA block (row = i + istar[b]) or -1 (row = i)
    int i;
    int col0, n;      // sub-cluster columns
    int tet0, ntet;   // its tetrahedra in the sub-cluster tet list
    int64_t out;      // output offset of (column col0, group 0)
    int64_t gs, js;   // group and column strides of the output
};

// MG > 0: the four vertex sums of a tetrahedron accumulate in registers for
// all groups and are flushed once per tetrahedron; MG == 0 (more than 32
// groups): every point is added to shared memory directly.  Tetrahedra are
// handed out through a shared counter so that the few tetrahedra near x_i
// (14-point rules) do not hold up a fixed partition.
template <int MG, bool XT = false>
__global__ void __launch_bounds__(kRowThreads, MG <= 16 && !XT ? 4 : 2) row_cluster_kernel(KernelParams P, const RowItem* __restrict__ items,
                                                          const int* __restrict__ sub_tets,
                                                          const int* __restrict__ istar, float* __restrict__ out)
{
    extern __shared__ float acc[];   // [G][n]
    __shared__ int s_next;
    const RowItem it = items[blockIdx.x];
    const int i = it.b >= 0 ? it.i + istar[it.b] : it.i;
    const int G = P.G, n = it.n;
    for (int k = threadIdx.x; k < G * n; k += blockDim.x) acc[k] = 0.f;
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    const Vec3<float> xi = load_xyz<float>(P, i);
    Vec3<float> xb = xi;
    if (P.has_wall) xb = mirror_point<float>(P, xi);
    const float inv4pi = (float)(1.0 / (4.0 * kPi));
    unsigned n_terms = 0, n_depths = 0;
    for (;;) {
        const int t = atomicAdd(&s_next, 1);
        if (t >= it.ntet) break;
        const int tet = sub_tets[it.tet0 + t];
        const int4 tv = P.tet[tet];
        const int jj[4] = {tv.x - it.col0, tv.y - it.col0, tv.z - it.col0, tv.w - it.col0};
        const bool in0 = (unsigned)jj[0] < (unsigned)n, in1 = (unsigned)jj[1] < (unsigned)n,
                   in2 = (unsigned)jj[2] < (unsigned)n, in3 = (unsigned)jj[3] < (unsigned)n;
        const Vec3<float> v0 = load_xyz<float>(P, tv.x), v1 = load_xyz<float>(P, tv.y), v2 = load_xyz<float>(P, tv.z),
                          v3 = load_xyz<float>(P, tv.w);
        Vec3<float> cen;
        float diam, vol;
        load_tgeo<float>(P, tet, cen, diam, vol);
        const float lim = 4.f * diam * diam;
        const int nd = dist2<float>(xi, cen) < lim ? 14 : 4;
        const int nr = P.has_wall ? (dist2<float>(xb, cen) < lim ? 14 : 4) : 0;
        n_terms += nd + nr;
        n_depths += nd + 2 * nr;
        float a0[MG > 0 ? MG : 1], a1[MG > 0 ? MG : 1], a2[MG > 0 ? MG : 1], a3[MG > 0 ? MG : 1];
        if constexpr (MG > 0) {
#pragma unroll
            for (int g = 0; g < MG; ++g) a0[g] = a1[g] = a2[g] = a3[g] = 0.f;
        }
        // Pass 0 visits the direct rule's points; when the reflected rule is
        // the same one (nd == nr, the usual case away from the wall), the
        // point, its weight and kappa(y) serve both terms.  Pass 1 visits the
        // reflected rule's points only when the two rules differ.
        const bool share = nd == nr;
        for (int pass = 0; pass < 2; ++pass) {
            const int nq = pass == 0 ? nd : (share ? 0 : nr);
            const int base = (pass == 0 ? nd : nr) == 14 ? 4 : 0;
            for (int q = 0; q < nq; ++q) {
                const int row = base + q;
                const float b0 = tet_b<float>(row, 0), b1 = tet_b<float>(row, 1), b2 = tet_b<float>(row, 2),
                            b3 = tet_b<float>(row, 3);
                Vec3<float> y;
                y.x = b0 * v0.x + b1 * v1.x + b2 * v2.x + b3 * v3.x;
                y.y = b0 * v0.y + b1 * v1.y + b2 * v2.y + b3 * v3.y;
                y.z = b0 * v0.z + b1 * v1.z + b2 * v2.z + b3 * v3.z;
                const float wq = vol * tet_w<float>(row) * kappa_at<float, XT>(P, y.x, y.y, y.z) * inv4pi;
                auto accumulate = [&](float w, float tau) {
                    if constexpr (XT) {
                        if (!(tau < INFINITY)) return;   // path through an opaque box
                    }
                    if constexpr (MG > 0) {
                        // c_g multiplies the sums when they are flushed
                        const float w0 = w * b0, w1 = w * b1, w2 = w * b2, w3 = w * b3;
                        auto add = [&](int g, float eg) {
                            a0[g] += w0 * eg;
                            a1[g] += w1 * eg;
                            a2[g] += w2 * eg;
                            a3[g] += w3 * eg;
                        };
                        if (P.c_arith) {
                            // exp(-c_g tau) as exp(-c_0 tau) exp(-dc tau)^g: two SFU exponentials per point
                            float E = expf(-P.c0f * tau);
                            const float D = expf(-P.dcf * tau);
#pragma unroll
                            for (int g = 0; g < MG; ++g) {
                                if (g < G) add(g, E);
                                E *= D;
                            }
                        } else {
#pragma unroll
                            for (int g = 0; g < MG; ++g)
                                if (g < G) add(g, expf(-P.cf[g] * tau));
                        }
                    } else {
                        for (int g = 0; g < G; ++g) {
                            const float cg = P.cf[g];
                            const float val = w * cg * expf(-cg * tau);
                            float* a = acc + g * n;
                            if (in0) atomicAdd(a + jj[0], val * b0);
                            if (in1) atomicAdd(a + jj[1], val * b1);
                            if (in2) atomicAdd(a + jj[2], val * b2);
                            if (in3) atomicAdd(a + jj[3], val * b3);
                        }
                    }
                };
                if (pass == 0) accumulate(wq / dist2<float>(xi, y), optical_depth<float, XT>(P, xi, y));
                if (pass == 1 || share) {
                    const Vec3<float> xp = wall_point<float>(P, xb, y);
                    const float tau = optical_depth<float, XT>(P, xi, xp) + optical_depth<float, XT>(P, xp, y);
                    accumulate((float)P.R0 * wq / dist2<float>(xb, y), tau);
                }
            }
        }
        if constexpr (XT) {
            // further walls and corner paths, each with its own rule; the point
            // value is split over the vertices as above
            for (int k = 0; k < P.n_extra; ++k) {
                Vec3<float> src;
                float sc;
                extra_term<float>(P, k, xi, src, sc);
                const int nx = dist2<float>(src, cen) < lim ? 14 : 4;
                n_terms += nx;
                n_depths += nx * (P.xkind[k] + 1);
                for (int q = 0; q < nx; ++q) {
                    const int row = (nx == 14 ? 4 : 0) + q;
                    const float b0 = tet_b<float>(row, 0), b1 = tet_b<float>(row, 1), b2 = tet_b<float>(row, 2),
                                b3 = tet_b<float>(row, 3);
                    const Vec3<float> y = {b0 * v0.x + b1 * v1.x + b2 * v2.x + b3 * v3.x,
                                           b0 * v0.y + b1 * v1.y + b2 * v2.y + b3 * v3.y,
                                           b0 * v0.z + b1 * v1.z + b2 * v2.z + b3 * v3.z};
                    const float w = sc * vol * tet_w<float>(row) * kappa_at<float, XT>(P, y.x, y.y, y.z) * inv4pi /
                                    dist2<float>(src, y);
                    const float tau = extra_tau<float>(P, k, xi, src, y);
                    if constexpr (MG > 0) {
#pragma unroll
                        for (int g = 0; g < MG; ++g)
                            if (g < G) {
                                const float val = w * expf(-P.cf[g] * tau);   // c_g at the flush
                                a0[g] += val * b0;
                                a1[g] += val * b1;
                                a2[g] += val * b2;
                                a3[g] += val * b3;
                            }
                    } else {
                        for (int g = 0; g < G; ++g) {
                            const float val = w * P.cf[g] * expf(-P.cf[g] * tau);
                            float* a = acc + g * n;
                            if (in0) atomicAdd(a + jj[0], val * b0);
                            if (in1) atomicAdd(a + jj[1], val * b1);
                            if (in2) atomicAdd(a + jj[2], val * b2);
                            if (in3) atomicAdd(a + jj[3], val * b3);
                        }
                    }
                }
            }
        }
        if constexpr (MG > 0) {
#pragma unroll
            for (int g = 0; g < MG; ++g)
                if (g < G) {
                    float* a = acc + g * n;
                    const float cg = P.cf[g];
                    if (in0) atomicAdd(a + jj[0], a0[g] * cg);
                    if (in1) atomicAdd(a + jj[1], a1[g] * cg);
                    if (in2) atomicAdd(a + jj[2], a2[g] * cg);
                    if (in3) atomicAdd(a + jj[3], a3[g] * cg);
                }
        }
    }
    count_work(P, n_terms, n_depths);
    __syncthreads();
    for (int k = threadIdx.x; k < G * n; k += blockDim.x) {
        const int g = k / n, j = k - g * n;
        out[it.out + g * it.gs + j * it.js] = acc[k];
    }
}

// sub-clusters of every column cluster and the tetrahedra touching each
int prepare_row_eval(Operator& op, std::string& err)
{
    const Plan& P = op.plan;
    const int nc = (int)P.clusters.size();
    op.sub_of_cluster_ptr.assign(nc + 1, 0);
    op.sub_of_cluster.clear();
    op.sub_start.clear();
    op.sub_size.clear();
    op.sub_tet_ptr.assign(1, 0);
    std::vector<int> sub_id(nc, -1), tets, stamp(op.T, -1);
    std::vector<char> used(nc, 0);
    for (const FarBlock& b : P.far_blocks) used[b.sc] = 1;
    for (const FarBlock& b : P.near_blocks) used[b.sc] = 1;
    std::vector<std::vector<int>> subs(nc);
    for (int c = 0; c < nc; ++c) {
        if (!used[c]) continue;
        std::vector<int> stack = {c};
        while (!stack.empty()) {
            const int k = stack.back();
            stack.pop_back();
            const ClusterNode& C = P.clusters[k];
            if (C.size <= kSubCols || C.left < 0) {
                if (C.size > kSubCols) {
                    err = "cluster leaf larger than the row-evaluation width";
                    return RT_EINVAL;
                }
                subs[c].push_back(k);
            } else {
                stack.push_back(C.right);
                stack.push_back(C.left);
            }
        }
    }
    for (int c = 0; c < nc; ++c) {
        for (int k : subs[c]) {
            if (sub_id[k] < 0) {
                sub_id[k] = (int)op.sub_start.size();
                const ClusterNode& C = P.clusters[k];
                op.sub_start.push_back(C.start);
                op.sub_size.push_back(C.size);
                for (int v = C.start; v < C.start + C.size; ++v)
                    for (int e = op.h_vt_ptr[v]; e < op.h_vt_ptr[v + 1]; ++e) {
                        const int t = op.h_vt_idx[e] >> 2;
                        if (stamp[t] != sub_id[k]) {
                            stamp[t] = sub_id[k];
                            tets.push_back(t);
                        }
                    }
                op.sub_tet_ptr.push_back((int)tets.size());
            }
            op.sub_of_cluster.push_back(sub_id[k]);
        }
        op.sub_of_cluster_ptr[c + 1] = (int)op.sub_of_cluster.size();
    }
    int rc = dev_alloc(op, &op.d_sub_tets, tets.size(), err);
    if (rc) return rc;
    if ((rc = upload_async(op, op.d_sub_tets, tets.data(), tets.size(), err))) return rc;
    static bool attr_set[64] = {false};
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        const int bytes = (int)(kMaxGroups * kSubCols * sizeof(float));
        RT_CUDA_TRY(cudaFuncSetAttribute(row_cluster_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        RT_CUDA_TRY(cudaFuncSetAttribute(row_cluster_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        RT_CUDA_TRY(cudaFuncSetAttribute(row_cluster_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        RT_CUDA_TRY(cudaFuncSetAttribute(row_cluster_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        RT_CUDA_TRY(cudaFuncSetAttribute(row_cluster_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        RT_CUDA_TRY(cudaFuncSetAttribute(row_cluster_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        RT_CUDA_TRY(cudaFuncSetAttribute(row_cluster_kernel<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        RT_CUDA_TRY(cudaFuncSetAttribute(row_cluster_kernel<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        attr_set[dev] = true;
    }
    return RT_OK;
}

static int launch_rows(Operator& op, const std::vector<RowItem>& items, const int* istar, float* out, cudaStream_t s,
                       std::string& err)
{
    if (items.empty()) return RT_OK;
    RowItem* d = nullptr;
    RT_CUDA_TRY(cudaMallocAsync((void**)&d, sizeof(RowItem) * items.size(), s));
    RT_CUDA_TRY(cudaMemcpyAsync(d, items.data(), sizeof(RowItem) * items.size(), cudaMemcpyHostToDevice, s));
    int maxn = 0;
    for (const RowItem& it : items) maxn = std::max(maxn, it.n);
    const size_t smem = (size_t)op.G * maxn * sizeof(float);
    for (size_t k0 = 0; k0 < items.size(); k0 += (size_t)1 << 30) {
        const int cnt = (int)std::min<size_t>(items.size() - k0, (size_t)1 << 30);
        const int G = op.G;
        if (op.kp.ext) {   // further walls, corner paths, a kappa grid or opaque boxes
            if (G <= 16) row_cluster_kernel<16, true><<<cnt, kRowThreads, smem, s>>>(op.kp, d + k0, op.d_sub_tets, istar, out);
            else row_cluster_kernel<0, true><<<cnt, kRowThreads, smem, s>>>(op.kp, d + k0, op.d_sub_tets, istar, out);
        } else if (G <= 1) row_cluster_kernel<1><<<cnt, kRowThreads, smem, s>>>(op.kp, d + k0, op.d_sub_tets, istar, out);
        else if (G <= 4) row_cluster_kernel<4><<<cnt, kRowThreads, smem, s>>>(op.kp, d + k0, op.d_sub_tets, istar, out);
        else if (G <= 8) row_cluster_kernel<8><<<cnt, kRowThreads, smem, s>>>(op.kp, d + k0, op.d_sub_tets, istar, out);
        else if (G <= 16) row_cluster_kernel<16><<<cnt, kRowThreads, smem, s>>>(op.kp, d + k0, op.d_sub_tets, istar, out);
        else if (G <= 32) row_cluster_kernel<32><<<cnt, kRowThreads, smem, s>>>(op.kp, d + k0, op.d_sub_tets, istar, out);
        else row_cluster_kernel<0><<<cnt, kRowThreads, smem, s>>>(op.kp, d + k0, op.d_sub_tets, istar, out);
    }
    RT_CUDA_TRY(cudaGetLastError());
    RT_CUDA_TRY(cudaFreeAsync(d, s));
    return RT_OK;
}

// ---------------------------------------------------------------------------
// Batched partially pivoted ACA (Section 2.1), pivots shared by all groups.
//
// Every admissible block b (m x n) is approximated for all groups g at once:
//   step k: residual row  R_g = G_g[i*, :] - sum_{l<k} u_{g,l}[i*] v_{g,l}
//           pivot column  j*  = argmax_j sum_g |R_g[j]| / w_g   (first index on ties)
//           v_g = R_g / R_g[j*]           (skipped for a group whose pivot is 0)
//           u_g = G_g[:, j*] - sum_{l<k} u_{g,l} v_{g,l}[j*]
//           ||S_g||_F^2 += 2 sum_{l<k} (u_l.u)(v_l.v) + |u|^2 |v|^2      (FP64)
//           group g done when |u_g| |v_g| <= eps ||S_g||_F
//           next row i* = argmax over unused rows of sum_g |u_g[i]| / w_g
// w_g = ||S_g||_F (1 before the first term) puts the groups on one scale.
// A block stops when every group is done; when another term would make
// r (m + n) >= m n, or the rank limit is reached, it is stored dense.
// The first pivot row is the block's first row.
// ---------------------------------------------------------------------------
namespace {

enum { ACA_ACTIVE = 0, ACA_DONE = 1, ACA_DENSE = 2 };

__device__ __forceinline__ unsigned long long score_key(float s, int idx)
{
    if (!(s >= 0.0f) || isinf(s)) s = 0.0f;
    return ((unsigned long long)__float_as_uint(s) << 32) | (unsigned long long)(0xffffffffu - (unsigned)idx);
}

struct AcaDev {
    int G;
    int rmax;
    double eps;
    const FarBlock* blk;
    int* istar;
    int* jstar;
    int* rank;
    int* status;
    double* norm2;      // [nfar][G]
    float* wscale;      // [nfar][G]   score weights 1/w_g
    float* inv;         // [nfar][G]
    int64_t* uoff;      // [nfar][rmax]
    int64_t* voff;      // [nfar][rmax]
    unsigned char* used;   // [sum m]
    int64_t* used_off;  // [nfar]
    unsigned long long* key;   // [nfar]  row pivot key, then next-row key
    unsigned* rowmax;   // [nfar][G]  max |R_g| of the current row (float bits)
    double* dots;       // per step: [dot0 + l][G][2]  (u_l.u, v_l.v), l = rank -> (|u|^2, |v|^2)
    float* pool;
};

// residual row: R_g[jj] -= sum_l u_{g,l}[i*] v_{g,l}[jj]; row key = argmax score.
__global__ void aca_row_residual(AcaDev D, const AcaActive* act, int na, int64_t total, float* buf)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ai = find_active(act, na, e, 0);
        const AcaActive a = act[ai];
        const int jj = (int)(e - a.first_row);
        const int b = a.b, r = D.rank[b], is = D.istar[b];
        // lanes of this warp on the same block combine their row maxima first:
        // one atomic per block and group per warp instead of one per lane
        const unsigned peers = __match_any_sync(__activemask(), b);
        const bool leader = (threadIdx.x & 31) == __ffs(peers) - 1;
        float score = 0.0f;
        for (int g = 0; g < D.G; ++g) {
            float v = buf[a.rbuf + (int64_t)g * a.n + jj];
            for (int l = 0; l < r; ++l) {
                const float* U = D.pool + D.uoff[(int64_t)b * D.rmax + l] + (int64_t)g * a.m;
                const float* V = D.pool + D.voff[(int64_t)b * D.rmax + l] + (int64_t)g * a.n;
                v -= U[is] * V[jj];
            }
            buf[a.rbuf + (int64_t)g * a.n + jj] = v;
            score += fabsf(v) * D.wscale[(int64_t)b * D.G + g];
            const unsigned mx = __reduce_max_sync(peers, isfinite(v) ? __float_as_uint(fabsf(v)) : 0u);
            if (leader && mx) atomicMax(&D.rowmax[(int64_t)b * D.G + g], mx);
        }
        atomicMax(&D.key[b], score_key(score, jj));
    }
}

// pivot column j*, 1/delta per group; a zero row is skipped.
__global__ void aca_row_pivot(AcaDev D, AcaActive* act, int na, const float* buf)
{
    for (int ai = blockIdx.x * blockDim.x + threadIdx.x; ai < na; ai += gridDim.x * blockDim.x) {
        AcaActive& a = act[ai];
        const int b = a.b;
        const unsigned long long k = D.key[b];
        const float best = __uint_as_float((unsigned)(k >> 32));
        const int j = (int)(0xffffffffu - (unsigned)(k & 0xffffffffu));
        D.key[b] = 0ull;
        if (!(best > 0.0f)) {
            // exact zero row: mark it used and move to the next unused row
            a.skip = 1;
            D.used[D.used_off[b] + D.istar[b]] = 1;
            int nxt = -1;
            for (int i = 0; i < a.m; ++i)
                if (!D.used[D.used_off[b] + i]) {
                    nxt = i;
                    break;
                }
            if (nxt < 0) D.status[b] = ACA_DONE;
            else D.istar[b] = nxt;
            continue;
        }
        a.skip = 0;
        D.jstar[b] = j;
        for (int g = 0; g < D.G; ++g) {
            const float d = buf[a.rbuf + (int64_t)g * a.n + j];
            const float rmx = __uint_as_float(D.rowmax[(int64_t)b * D.G + g]);
            D.rowmax[(int64_t)b * D.G + g] = 0u;
            // a group whose value at the shared pivot is negligible skips this term
            D.inv[(int64_t)b * D.G + g] = (fabsf(d) > 1e-4f * rmx && fabsf(d) > 1e-37f) ? 1.0f / d : 0.0f;
        }
    }
}

// v_g = R_g * inv_g into the pool
__global__ void aca_store_v(AcaDev D, const AcaActive* act, int na, int64_t total, const float* buf)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ai = find_active(act, na, e, 0);
        const AcaActive a = act[ai];
        if (a.skip) continue;
        const int jj = (int)(e - a.first_row);
        for (int g = 0; g < D.G; ++g)
            D.pool[a.voff + (int64_t)g * a.n + jj] =
                buf[a.rbuf + (int64_t)g * a.n + jj] * D.inv[(int64_t)a.b * D.G + g];
    }
}

// u_g = C_g - sum_l u_{g,l} v_{g,l}[j*]; next-row key over unused rows.
__global__ void aca_col_residual(AcaDev D, const AcaActive* act, int na, int64_t total, const float* buf)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ai = find_active(act, na, e, 1);
        const AcaActive a = act[ai];
        if (a.skip) continue;
        const int ii = (int)(e - a.first_col);
        const int b = a.b, r = D.rank[b], js = D.jstar[b];
        float score = 0.0f;
        for (int g = 0; g < D.G; ++g) {
            float v = buf[a.cbuf + (int64_t)g * a.m + ii];
            for (int l = 0; l < r; ++l) {
                const float* U = D.pool + D.uoff[(int64_t)b * D.rmax + l] + (int64_t)g * a.m;
                const float* V = D.pool + D.voff[(int64_t)b * D.rmax + l] + (int64_t)g * a.n;
                v -= U[ii] * V[js];
            }
            if (D.inv[(int64_t)b * D.G + g] == 0.0f) v = 0.0f;
            D.pool[a.uoff + (int64_t)g * a.m + ii] = v;
            score += fabsf(v) * D.wscale[(int64_t)b * D.G + g];
        }
        if (ii != D.istar[b] && !D.used[D.used_off[b] + ii]) atomicMax(&D.key[b], score_key(score, ii));
    }
}

// dots (u_l.u, v_l.v) for l = 0..rank (l = rank: the new term itself); one CTA per (block, l).
struct DotItem {
    int ai;
    int l;
};

// one warp per (block, l).  The warp's lanes are split among the groups (gp
// groups at a time, gp a power of two <= 4, so L = 32 / gp >= 8 lanes per
// group and every load of a group still fills a whole 32-byte sector); each
// group's two dot products then need a reduction over only L lanes: FP32
// partial sums per lane (length / L terms), FP64 across lanes.
__global__ void __launch_bounds__(256) aca_dots(AcaDev D, const AcaActive* act, const DotItem* items, int nitems)
{
    const int lane = threadIdx.x & 31;
    int gp = 1;
    while (gp < D.G && gp < 4) gp <<= 1;
    const int L = 32 / gp;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < nitems; it += nw) {
        const DotItem di = items[it];
        const AcaActive a = act[di.ai];
        if (a.skip) continue;
        const int b = a.b;
        const int64_t ul = di.l == D.rank[b] ? a.uoff : D.uoff[(int64_t)b * D.rmax + di.l];
        const int64_t vl = di.l == D.rank[b] ? a.voff : D.voff[(int64_t)b * D.rmax + di.l];
        for (int g0 = 0; g0 < D.G; g0 += gp) {
            const int g = g0 + lane / L, sl = lane % L;
            float pu = 0.f, pv = 0.f;
            if (g < D.G) {
                const float* U0 = D.pool + ul + (int64_t)g * a.m;
                const float* U1 = D.pool + a.uoff + (int64_t)g * a.m;
                const float* V0 = D.pool + vl + (int64_t)g * a.n;
                const float* V1 = D.pool + a.voff + (int64_t)g * a.n;
                // unrolled so that several loads per lane are in flight
#pragma unroll 4
                for (int i = sl; i < a.m; i += L) pu += U0[i] * U1[i];
#pragma unroll 4
                for (int j = sl; j < a.n; j += L) pv += V0[j] * V1[j];
            }
            double su = pu, sv = pv;
            for (int o = L >> 1; o > 0; o >>= 1) {   // xor within aligned groups of L lanes
                su += __shfl_xor_sync(0xffffffffu, su, o);
                sv += __shfl_xor_sync(0xffffffffu, sv, o);
            }
            if (sl == 0 && g < D.G) {
                double* dst = D.dots + ((a.dot0 + di.l) * D.G + g) * 2;
                dst[0] = su;
                dst[1] = sv;
            }
        }
    }
}

__global__ void aca_finish(AcaDev D, const AcaActive* act, int na)
{
    for (int ai = blockIdx.x * blockDim.x + threadIdx.x; ai < na; ai += gridDim.x * blockDim.x) {
        const AcaActive a = act[ai];
        if (a.skip) continue;
        const int b = a.b, r = D.rank[b];
        bool all_done = true;
        for (int g = 0; g < D.G; ++g) {
            const double* dk = D.dots + ((a.dot0 + r) * D.G + g) * 2;
            const double uu = dk[0], vv = dk[1];
            double s = D.norm2[(int64_t)b * D.G + g];
            double cross = 0.0;
            for (int l = 0; l < r; ++l) {
                const double* dl = D.dots + ((a.dot0 + l) * D.G + g) * 2;
                cross += dl[0] * dl[1];
            }
            s += 2.0 * cross + uu * vv;
            if (s < 0.0) s = 0.0;
            D.norm2[(int64_t)b * D.G + g] = s;
            // a group that skipped this shared pivot (1/delta = 0) has learned nothing
            // from the term and is not declared converged by it
            const bool skipped = D.inv[(int64_t)b * D.G + g] == 0.0f;
            const bool done = !skipped && sqrt(uu * vv) <= D.eps * sqrt(s);
            all_done = all_done && done;
            D.wscale[(int64_t)b * D.G + g] = s > 0.0 ? (float)(1.0 / sqrt(s)) : 1.0f;
        }
        D.uoff[(int64_t)b * D.rmax + r] = a.uoff;
        D.voff[(int64_t)b * D.rmax + r] = a.voff;
        D.used[D.used_off[b] + D.istar[b]] = 1;
        const int nr = r + 1;
        D.rank[b] = nr;
        const unsigned long long k = D.key[b];
        D.key[b] = 0ull;
        const float best = __uint_as_float((unsigned)(k >> 32));
        if (all_done) {
            D.status[b] = ACA_DONE;
        } else if ((int64_t)(nr + 1) * (a.m + a.n) >= (int64_t)a.m * a.n || nr >= D.rmax) {
            D.status[b] = ACA_DENSE;
        } else if (k == 0ull || !(best > 0.0f)) {
            // no unused row with a nonzero residual: the approximation is exact on all rows seen
            D.status[b] = ACA_DONE;
        } else {
            D.istar[b] = (int)(0xffffffffu - (unsigned)(k & 0xffffffffu));
        }
    }
}

// repack converged blocks into V^T [G][r][n] and U^T [G][r][m] in the final storage type
template <class T>
__device__ __forceinline__ T to_store(float x);
template <>
__device__ __forceinline__ float to_store<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_store<__half>(float x) { return __float2half_rn(x); }

struct PackItem {
    int b;          // far block id (ACA numbering)
    int l;          // term
    int r, m, n, n8;
    int64_t voff_dst, uoff_dst;   // element offsets of the block's V^T and U^T in the final storage
    int c0, c1;     // chunk range [c0, c1) in the chunk array
};

// Each rank-1 term u v^T is stored as (s u)(v / s) with s chosen so that both
// factors have the same largest magnitude (s = 1 for FP32): the product is
// unchanged and 16-bit storage keeps both factors away from the subnormals.
// With `lo` set, each scaled value x is stored as the 16-bit high part
// h = round(x) in dst and the 16-bit remainder round(x - h) in lo.
template <class T>
__device__ __forceinline__ void store_split(T* dst, T* lo, int64_t i, float x)
{
    const T h = to_store<T>(x);
    dst[i] = h;
    if (lo) lo[i] = to_store<T>(x - (float)h);
}
template <class T>
__global__ void aca_pack(AcaDev D, const PackItem* items, int nitems, const Chunk* chunks, T* dst, T* lo)
{
    __shared__ float red[2][32];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const PackItem p = items[it];
        const int64_t us = D.uoff[(int64_t)p.b * D.rmax + p.l], vs = D.voff[(int64_t)p.b * D.rmax + p.l];
        for (int g = 0; g < D.G; ++g) {
            float su = 1.f;
            if (sizeof(T) == 2) {
                float mu = 0.f, mv = 0.f;
                for (int i = threadIdx.x; i < p.m; i += blockDim.x) mu = fmaxf(mu, fabsf(D.pool[us + (int64_t)g * p.m + i]));
                for (int j = threadIdx.x; j < p.n; j += blockDim.x) mv = fmaxf(mv, fabsf(D.pool[vs + (int64_t)g * p.n + j]));
                for (int o = 16; o > 0; o >>= 1) {
                    mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
                    mv = fmaxf(mv, __shfl_xor_sync(0xffffffffu, mv, o));
                }
                if ((threadIdx.x & 31) == 0) {
                    red[0][threadIdx.x >> 5] = mu;
                    red[1][threadIdx.x >> 5] = mv;
                }
                __syncthreads();
                mu = 0.f;
                mv = 0.f;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    mu = fmaxf(mu, red[0][w]);
                    mv = fmaxf(mv, red[1][w]);
                }
                __syncthreads();
                if (mu > 0.f && mv > 0.f) su = sqrtf(mv / mu);
            }
            const float sv = 1.f / su;
            for (int j = threadIdx.x; j < p.n; j += blockDim.x)
                store_split<T>(dst, lo, p.voff_dst + ((int64_t)g * p.r + p.l) * p.n8 + j,
                               sv * D.pool[vs + (int64_t)g * p.n + j]);
            for (int c = p.c0; c < p.c1; ++c) {
                const Chunk ch = chunks[c];
                for (int i = threadIdx.x; i < ch.m; i += blockDim.x)
                    store_split<T>(dst, lo, p.uoff_dst + ch.off + ((int64_t)g * p.r + p.l) * ch.m8 + i,
                                   su * D.pool[us + (int64_t)g * p.m + ch.rbeg + i]);
            }
        }
    }
}

}  // namespace

int assemble_hmatrix(Operator& op, cudaStream_t s, std::string& err)
{
    int rc;
    const int G = op.G;
    const std::vector<FarBlock>& farb = op.plan.far_blocks;
    const int nfar = (int)farb.size();
    const int rmax = op.rank_max;
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, s);

    std::vector<int> final_status(nfar, ACA_DENSE), final_rank(nfar, 0);
    int64_t aca_steps = 0;
    AcaDev D{};
    std::vector<void*> tmp;   // freed at the end
    int64_t scratch = 0;      // bytes of ACA scratch held now (tmp, pool, dot lists)
    auto note_peak = [&](int64_t extra) {
        op.info.peak_bytes = std::max<int64_t>(op.info.peak_bytes, op.info.device_bytes + scratch + extra);
    };
    auto talloc = [&](void** p, size_t bytes) -> int {
        cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 1, s);
        if (e != cudaSuccess) {
            err = std::string("cudaMalloc (ACA scratch): ") + cudaGetErrorString(e);
            return RT_ENOMEM;
        }
        tmp.push_back(*p);
        scratch += (int64_t)(bytes ? bytes : 1);
        note_peak(0);
        return RT_OK;
    };
    auto cleanup = [&]() {
        for (void* p : tmp) cudaFreeAsync(p, s);
        tmp.clear();
    };
    float* pool = nullptr;
    int64_t pool_cap = 0, pool_used = 0;
    float ms = 0.f, ms_pack = 0.f;
    const int esz = op.far_prec == RT_PREC_F32 ? 4 : 2;
    const bool split = op.refine && op.far_prec != RT_PREC_F32;

    // ---- waves: consecutive runs of far blocks whose ACA terms (estimated at
    // kWaveRank terms per block) take at most kWaveBytes of FP32 scratch.  Each
    // wave is approximated, packed into the far storage and its scratch freed
    // before the next starts, which bounds the assembly's memory peak.
    constexpr double kWaveRank = 24.0;
    const int64_t kWaveBytes = op.wave_bytes;
    std::vector<int> wave_start(1, 0);
    {
        double acc = 0.0;
        for (int b = 0; b < nfar; ++b) {
            const double est = 4.0 * G * (double)(farb[b].m + farb[b].n) * kWaveRank;
            if (acc > 0.0 && acc + est > (double)kWaveBytes) {
                wave_start.push_back(b);
                acc = 0.0;
            }
            acc += est;
        }
        wave_start.push_back(nfar);
    }
    const int nwaves = (int)wave_start.size() - 1;
    op.info.aca_waves = nfar > 0 ? nwaves : 0;
    int nw_max = 0;
    int64_t summ_max = 0, sumn_max = 0;
    for (int w = 0; w < nwaves; ++w) {
        int64_t sm = 0, sn = 0;
        for (int b = wave_start[w]; b < wave_start[w + 1]; ++b) {
            sm += farb[b].m;
            sn += farb[b].n;
        }
        nw_max = std::max(nw_max, wave_start[w + 1] - wave_start[w]);
        summ_max = std::max(summ_max, sm);
        sumn_max = std::max(sumn_max, sn);
    }

    // final far storage layout, filled wave by wave
    op.far_blocks.clear();
    op.dense_blocks = op.plan.near_blocks;
    op.rank.clear();
    op.far_v_off.clear();
    op.far_u_off.clear();
    op.far_chunks.clear();
    op.far_chunk_ptr.assign(1, 0);
    std::vector<int> far_src;   // ACA block id of each stored far block
    int64_t far_elems = 0;
    if (nwaves > 1) {
        // address range for the largest possible far field: every block at the
        // rank where dense storage becomes cheaper
        int64_t bound = 0;
        std::vector<Chunk> tmpc;
        for (int b = 0; b < nfar; ++b) {
            const FarBlock& fb = farb[b];
            const int64_t rcap = std::min<int64_t>(rmax, (int64_t)fb.m * fb.n / (fb.m + fb.n) + 1);
            tmpc.clear();
            bound += (int64_t)G * rcap * ((int64_t)round8(fb.n) + block_chunks(op.plan, fb.row0, fb.m, 1, tmpc));
        }
        if ((rc = growbuf_reserve(op.far_buf, (size_t)bound * esz, op.device, err))) return rc;
        if (split && (rc = growbuf_reserve(op.far_lo_buf, (size_t)bound * esz, op.device, err))) return rc;
    }
    if (nfar > 0) {
        D.G = G;
        D.rmax = rmax;
        D.eps = op.aca_eps;
#define TA(ptr, bytes)                                       \
    do {                                                     \
        if ((rc = talloc((void**)&(ptr), (bytes)))) {        \
            cleanup();                                       \
            return rc;                                       \
        }                                                    \
    } while (0)
        // per-block state, sized for the largest wave and indexed by the
        // block's position in its wave
        FarBlock* d_blk;
        TA(d_blk, sizeof(FarBlock) * nw_max);
        TA(D.istar, sizeof(int) * nw_max);
        TA(D.jstar, sizeof(int) * nw_max);
        TA(D.rank, sizeof(int) * nw_max);
        TA(D.status, sizeof(int) * nw_max);
        TA(D.norm2, sizeof(double) * nw_max * G);
        TA(D.wscale, sizeof(float) * nw_max * G);
        TA(D.inv, sizeof(float) * nw_max * G);
        TA(D.uoff, sizeof(int64_t) * nw_max * rmax);
        TA(D.voff, sizeof(int64_t) * nw_max * rmax);
        TA(D.used, summ_max);
        TA(D.used_off, sizeof(int64_t) * nw_max);
        TA(D.key, sizeof(unsigned long long) * nw_max);
        TA(D.rowmax, sizeof(unsigned) * nw_max * G);
        D.blk = d_blk;
        float *rowbuf, *colbuf;
        TA(rowbuf, sizeof(float) * (size_t)G * sumn_max);
        TA(colbuf, sizeof(float) * (size_t)G * summ_max);
        AcaActive* d_act;
        TA(d_act, sizeof(AcaActive) * nw_max);
        DotItem* d_dot = nullptr;
        double* d_dotv = nullptr;
        int64_t dot_cap = 0;
        std::vector<int> h_status_buf((size_t)nw_max * 2);
        int* h_status = h_status_buf.data();
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const std::vector<float> ones((size_t)nw_max * G, 1.0f);
        cudaEvent_t pk0, pk1;
        cudaEventCreate(&pk0);
        cudaEventCreate(&pk1);

        for (int w = 0; w < nwaves; ++w) {
            const int w0 = wave_start[w], nb = wave_start[w + 1] - w0;
            const FarBlock* fw = farb.data() + w0;
            std::vector<int64_t> used_off(nb);
            int64_t sum_m = 0;
            for (int b = 0; b < nb; ++b) {
                used_off[b] = sum_m;
                sum_m += fw[b].m;
            }
            RT_CUDA_TRY(cudaMemcpyAsync(d_blk, fw, sizeof(FarBlock) * nb, cudaMemcpyHostToDevice, s));
            RT_CUDA_TRY(cudaMemsetAsync(D.istar, 0, sizeof(int) * nb, s));
            RT_CUDA_TRY(cudaMemsetAsync(D.rank, 0, sizeof(int) * nb, s));
            RT_CUDA_TRY(cudaMemsetAsync(D.status, 0, sizeof(int) * nb, s));
            RT_CUDA_TRY(cudaMemsetAsync(D.norm2, 0, sizeof(double) * nb * G, s));
            RT_CUDA_TRY(cudaMemcpyAsync(D.wscale, ones.data(), sizeof(float) * nb * G, cudaMemcpyHostToDevice, s));
            RT_CUDA_TRY(cudaMemsetAsync(D.used, 0, sum_m, s));
            RT_CUDA_TRY(cudaMemcpyAsync(D.used_off, used_off.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
            RT_CUDA_TRY(cudaMemsetAsync(D.key, 0, sizeof(unsigned long long) * nb, s));
            RT_CUDA_TRY(cudaMemsetAsync(D.rowmax, 0, sizeof(unsigned) * nb * G, s));
            std::vector<int> h_rank(nb, 0), status(nb, ACA_ACTIVE);

            // term pool of this wave: kWaveRank terms per block, grown if needed
            pool_used = 0;
            pool_cap = 0;
            for (int b = 0; b < nb; ++b) pool_cap += (int64_t)G * (fw[b].m + fw[b].n) * (int64_t)kWaveRank;
            if (cudaMallocAsync((void**)&pool, sizeof(float) * pool_cap, s) != cudaSuccess) {
                cleanup();
                err = "cudaMalloc (ACA pool) failed";
                return RT_ENOMEM;
            }
            D.pool = pool;
            scratch += (int64_t)sizeof(float) * pool_cap;
            note_peak(0);

            std::vector<AcaActive> act;
            std::vector<DotItem> dots;
            for (int step = 0; step < rmax + 64; ++step) {
                act.clear();
                int64_t fr = 0, fc = 0, bufr = 0, bufc = 0, need = 0;
                for (int b = 0; b < nb; ++b)
                    if (status[b] == ACA_ACTIVE) need += (int64_t)G * (fw[b].m + fw[b].n);
                if (need == 0) break;
                if (pool_used + need > pool_cap) {
                    const int64_t ncap = std::max<int64_t>(pool_cap + pool_cap / 2, pool_used + need * 8);
                    float* np = nullptr;
                    if (cudaMallocAsync((void**)&np, sizeof(float) * ncap, s) != cudaSuccess) {
                        cudaFreeAsync(pool, s);
                        cleanup();
                        err = "cudaMalloc (ACA pool growth) failed";
                        return RT_ENOMEM;
                    }
                    RT_CUDA_TRY(cudaMemcpyAsync(np, pool, sizeof(float) * pool_used, cudaMemcpyDeviceToDevice, s));
                    note_peak((int64_t)sizeof(float) * ncap);   // old and new pool both live here
                    scratch += (int64_t)sizeof(float) * (ncap - pool_cap);
                    cudaFreeAsync(pool, s);
                    pool = np;
                    pool_cap = ncap;
                    D.pool = pool;
                }
                int64_t ndot = 0, nchunk = 0;
                for (int b = 0; b < nb; ++b) {
                    if (status[b] != ACA_ACTIVE) continue;
                    AcaActive a{};
                    a.b = b;
                    a.row0 = fw[b].row0;
                    a.m = fw[b].m;
                    a.col0 = fw[b].col0;
                    a.n = fw[b].n;
                    a.first_row = fr;
                    a.first_col = fc;
                    a.rbuf = bufr;
                    a.cbuf = bufc;
                    a.uoff = pool_used;
                    pool_used += (int64_t)G * a.m;
                    a.voff = pool_used;
                    pool_used += (int64_t)G * a.n;
                    a.dot0 = ndot;
                    ndot += h_rank[b] + 1;
                    a.first_chunk = nchunk;
                    nchunk += (a.m + kColRows - 1) / kColRows;
                    fr += a.n;
                    fc += a.m;
                    bufr += (int64_t)G * a.n;
                    bufc += (int64_t)G * a.m;
                    act.push_back(a);
                }
                const int na = (int)act.size();
                RT_CUDA_TRY(cudaMemcpyAsync(d_act, act.data(), sizeof(AcaActive) * na, cudaMemcpyHostToDevice, s));
                // 1. pivot rows: one CTA per (block, sub-cluster of its columns)
                {
                    std::vector<RowItem> ritems;
                    for (const AcaActive& a : act) {
                        const FarBlock& fb = fw[a.b];
                        for (int e = op.sub_of_cluster_ptr[fb.sc]; e < op.sub_of_cluster_ptr[fb.sc + 1]; ++e) {
                            const int sb = op.sub_of_cluster[e];
                            RowItem it{};
                            it.b = a.b;
                            it.i = fb.row0;
                            it.col0 = op.sub_start[sb];
                            it.n = op.sub_size[sb];
                            it.tet0 = op.sub_tet_ptr[sb];
                            it.ntet = op.sub_tet_ptr[sb + 1] - op.sub_tet_ptr[sb];
                            it.out = a.rbuf + (op.sub_start[sb] - fb.col0);
                            it.gs = fb.n;
                            it.js = 1;
                            ritems.push_back(it);
                        }
                    }
                    if ((rc = launch_rows(op, ritems, D.istar, rowbuf, s, err))) {
                        cleanup();
                        return rc;
                    }
                }
                const int eg_r = (int)std::min<int64_t>((fr + 255) / 256, (int64_t)sms * 32);
                aca_row_residual<<<std::max(1, eg_r), 256, 0, s>>>(D, d_act, na, fr, rowbuf);
                aca_row_pivot<<<(na + 127) / 128, 128, 0, s>>>(D, d_act, na, rowbuf);
                aca_store_v<<<std::max(1, eg_r), 256, 0, s>>>(D, d_act, na, fr, rowbuf);
                // 2. pivot columns: one CTA per 64-row chunk, the column's quadrature
                // points tabulated once per chunk
                {
                    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nchunk, (int64_t)sms * 32));
#define RT_LAUNCH_ACAC(MG, XT) \
    aca_col_kernel<MG, XT><<<grid, kColRows, 0, s>>>(op.kp, d_act, na, nchunk, D.jstar, colbuf)
#define RT_LAUNCH_ACAC1(MG) RT_LAUNCH_ACAC(MG, false)
                    if (op.kp.ext) RT_DISPATCH_MG_XT(G, RT_LAUNCH_ACAC);
                    else RT_DISPATCH_MG(G, RT_LAUNCH_ACAC1);
#undef RT_LAUNCH_ACAC1
#undef RT_LAUNCH_ACAC
                    RT_CUDA_TRY(cudaGetLastError());
                }
                const int eg_c = (int)std::min<int64_t>((fc + 255) / 256, (int64_t)sms * 32);
                aca_col_residual<<<std::max(1, eg_c), 256, 0, s>>>(D, d_act, na, fc, colbuf);
                // 3. dots with all previous terms and the new one (per-step scratch)
                dots.clear();
                for (int ai = 0; ai < na; ++ai)
                    for (int l = 0; l <= h_rank[act[ai].b]; ++l) dots.push_back({ai, l});
                if ((int64_t)dots.size() > dot_cap) {
                    if (d_dot) cudaFreeAsync(d_dot, s);
                    if (d_dotv) cudaFreeAsync(d_dotv, s);
                    scratch -= (int64_t)(sizeof(DotItem) + 2 * G * sizeof(double)) * dot_cap;
                    dot_cap = (int64_t)dots.size() * 2;
                    RT_CUDA_TRY(cudaMallocAsync((void**)&d_dot, sizeof(DotItem) * dot_cap, s));
                    RT_CUDA_TRY(cudaMallocAsync((void**)&d_dotv, sizeof(double) * 2 * G * dot_cap, s));
                    scratch += (int64_t)(sizeof(DotItem) + 2 * G * sizeof(double)) * dot_cap;
                    note_peak(0);
                }
                D.dots = d_dotv;
                RT_CUDA_TRY(cudaMemcpyAsync(d_dot, dots.data(), sizeof(DotItem) * dots.size(), cudaMemcpyHostToDevice, s));
                aca_dots<<<(int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)dots.size() + 7) / 8, (int64_t)sms * 32)),
                           256, 0, s>>>(D, d_act, d_dot, (int)dots.size());
                aca_finish<<<(na + 127) / 128, 128, 0, s>>>(D, d_act, na);
                RT_CUDA_TRY(cudaGetLastError());
                RT_CUDA_TRY(cudaMemcpyAsync(h_status, D.status, sizeof(int) * nb, cudaMemcpyDeviceToHost, s));
                RT_CUDA_TRY(cudaMemcpyAsync(h_status + nb, D.rank, sizeof(int) * nb, cudaMemcpyDeviceToHost, s));
                RT_CUDA_TRY(cudaStreamSynchronize(s));
                for (int b = 0; b < nb; ++b) {
                    status[b] = h_status[b];
                    h_rank[b] = h_status[nb + b];
                }
                ++aca_steps;
            }
            // ---- this wave's blocks: stored low rank, all-zero, or dense ------
            const int64_t elems0 = far_elems;
            const int k0 = (int)op.far_blocks.size();
            for (int b = 0; b < nb; ++b) {
                final_status[w0 + b] = status[b] == ACA_ACTIVE ? ACA_DENSE : status[b];
                final_rank[w0 + b] = h_rank[b];
                if (final_status[w0 + b] == ACA_DONE && h_rank[b] > 0) {
                    const FarBlock& fb = fw[b];
                    const int r = h_rank[b];
                    op.far_blocks.push_back(fb);
                    op.rank.push_back(r);
                    far_src.push_back(b);
                    op.far_v_off.push_back(far_elems);
                    far_elems += (int64_t)G * r * round8(fb.n);
                    op.far_u_off.push_back(far_elems);
                    far_elems += block_chunks(op.plan, fb.row0, fb.m, (int64_t)G * r, op.far_chunks);
                    op.far_chunk_ptr.push_back((int)op.far_chunks.size());
                } else if (final_status[w0 + b] == ACA_DONE) {
                    // an all-zero block: nothing to store
                } else {
                    op.dense_blocks.push_back(fw[b]);
                    op.n_fallback++;
                }
            }
            const int k1 = (int)op.far_blocks.size();
            // ---- storage for the new far blocks, then pack them -----------------
            if (nwaves == 1 && k1 > 0) {
                char *d = nullptr, *dl = nullptr;
                if ((rc = dev_alloc(op, &d, (size_t)far_elems * esz, err)) ||
                    (split && (rc = dev_alloc(op, &dl, (size_t)far_elems * esz, err)))) {
                    cudaFreeAsync(pool, s);
                    cleanup();
                    return rc;
                }
                op.d_far = d;
                op.d_far_lo = dl;
            } else if (nwaves > 1 && far_elems > elems0) {
                const size_t before = op.far_buf.mapped;
                if ((rc = growbuf_grow(op.far_buf, (size_t)far_elems * esz, err)) ||
                    (split && (rc = growbuf_grow(op.far_lo_buf, (size_t)far_elems * esz, err)))) {
                    cudaFreeAsync(pool, s);
                    cleanup();
                    return rc;
                }
                op.info.device_bytes += (int64_t)(op.far_buf.mapped - before) * (split ? 2 : 1);
                op.d_far = (void*)op.far_buf.base;
                op.d_far_lo = split ? (void*)op.far_lo_buf.base : nullptr;
            }
            if (k1 > k0) {
                char* base = (char*)op.d_far;
                char* base_lo = (char*)op.d_far_lo;
                RT_CUDA_TRY(cudaMemsetAsync(base + elems0 * esz, 0, (size_t)(far_elems - elems0) * esz, s));
                if (base_lo) RT_CUDA_TRY(cudaMemsetAsync(base_lo + elems0 * esz, 0, (size_t)(far_elems - elems0) * esz, s));
                note_peak(0);   // packed far field next to this wave's pool
                std::vector<PackItem> items;
                for (int k = k0; k < k1; ++k)
                    for (int l = 0; l < op.rank[k]; ++l)
                        items.push_back({far_src[k], l, op.rank[k], op.far_blocks[k].m, op.far_blocks[k].n,
                                         round8(op.far_blocks[k].n), op.far_v_off[k], op.far_u_off[k],
                                         op.far_chunk_ptr[k], op.far_chunk_ptr[k + 1]});
                PackItem* d_items = nullptr;
                Chunk* d_chunks = nullptr;
                const int c0 = op.far_chunk_ptr[k0], nc = op.far_chunk_ptr[k1] - c0;
                RT_CUDA_TRY(cudaMallocAsync((void**)&d_items, sizeof(PackItem) * items.size(), s));
                RT_CUDA_TRY(cudaMallocAsync((void**)&d_chunks, sizeof(Chunk) * op.far_chunks.size(), s));
                RT_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), sizeof(PackItem) * items.size(),
                                            cudaMemcpyHostToDevice, s));
                RT_CUDA_TRY(cudaMemcpyAsync(d_chunks + c0, op.far_chunks.data() + c0, sizeof(Chunk) * nc,
                                            cudaMemcpyHostToDevice, s));
                const int grid = (int)std::min<size_t>(items.size(), 152 * 64);
                const int ni = (int)items.size();
                cudaEventRecord(pk0, s);
                if (op.far_prec == RT_PREC_F32)
                    aca_pack<float><<<grid, 256, 0, s>>>(D, d_items, ni, d_chunks, (float*)base, nullptr);
                else if (op.far_prec == RT_PREC_BF16)
                    aca_pack<__nv_bfloat16><<<grid, 256, 0, s>>>(D, d_items, ni, d_chunks, (__nv_bfloat16*)base,
                                                                 (__nv_bfloat16*)base_lo);
                else aca_pack<__half><<<grid, 256, 0, s>>>(D, d_items, ni, d_chunks, (__half*)base, (__half*)base_lo);
                cudaEventRecord(pk1, s);
                RT_CUDA_TRY(cudaGetLastError());
                cudaFreeAsync(d_items, s);
                cudaFreeAsync(d_chunks, s);
                RT_CUDA_TRY(cudaEventSynchronize(pk1));
                float t = 0.f;
                cudaEventElapsedTime(&t, pk0, pk1);
                ms_pack += t;
            }
            cudaFreeAsync(pool, s);
            scratch -= (int64_t)sizeof(float) * pool_cap;
            pool = nullptr;
        }
        if (d_dot) cudaFreeAsync(d_dot, s);
        if (d_dotv) cudaFreeAsync(d_dotv, s);
        scratch -= (int64_t)(sizeof(DotItem) + 2 * G * sizeof(double)) * dot_cap;
        cudaEventDestroy(pk0);
        cudaEventDestroy(pk1);
#undef TA
    }
    cleanup();
    scratch = 0;
    op.n_far = (int)op.far_blocks.size();
    op.n_near = (int)op.dense_blocks.size();
    cudaEventRecord(ev1, s);
    cudaEventSynchronize(ev1);
    cudaEventElapsedTime(&ms, ev0, ev1);
    op.info.ms_aca = ms - ms_pack;
    op.info.ms_pack = ms_pack;
    op.info.aca_steps = aca_steps;

    // ---- dense blocks (near leaves and fallbacks): per leaf chunk A^T [G][n][m8]
    cudaEventRecord(ev0, s);
    int64_t near_elems = 0;
    op.dense_off.assign(op.n_near, 0);
    op.dense_chunks.clear();
    op.dense_chunk_ptr.assign(1, 0);
    for (int k = 0; k < op.n_near; ++k) {
        const FarBlock& fb = op.dense_blocks[k];
        op.dense_off[k] = near_elems;
        near_elems += block_chunks(op.plan, fb.row0, fb.m, (int64_t)G * fb.n, op.dense_chunks);
        op.dense_chunk_ptr.push_back((int)op.dense_chunks.size());
    }
    if (op.n_near > 0) {
        if ((rc = dev_alloc(op, &op.d_near, (size_t)near_elems, err))) return rc;
        RT_CUDA_TRY(cudaMemsetAsync(op.d_near, 0, sizeof(float) * (size_t)near_elems, s));
        std::vector<RowItem> ritems;
        for (int k = 0; k < op.n_near; ++k) {
            const FarBlock& fb = op.dense_blocks[k];
            for (int c = op.dense_chunk_ptr[k]; c < op.dense_chunk_ptr[k + 1]; ++c) {
                const Chunk& ch = op.dense_chunks[c];
                for (int ii = 0; ii < ch.m; ++ii)
                    for (int e = op.sub_of_cluster_ptr[fb.sc]; e < op.sub_of_cluster_ptr[fb.sc + 1]; ++e) {
                        const int sb = op.sub_of_cluster[e];
                        RowItem it{};
                        it.b = -1;
                        it.i = fb.row0 + ch.rbeg + ii;
                        it.col0 = op.sub_start[sb];
                        it.n = op.sub_size[sb];
                        it.tet0 = op.sub_tet_ptr[sb];
                        it.ntet = op.sub_tet_ptr[sb + 1] - op.sub_tet_ptr[sb];
                        it.out = op.dense_off[k] + ch.off + ii + (int64_t)(op.sub_start[sb] - fb.col0) * ch.m8;
                        it.gs = (int64_t)fb.n * ch.m8;
                        it.js = ch.m8;
                        ritems.push_back(it);
                    }
            }
        }
        if ((rc = launch_rows(op, ritems, nullptr, op.d_near, s, err))) return rc;
        for (int k = 0; k < op.n_near; ++k)
            op.info.entries_evaluated += (int64_t)op.dense_blocks[k].m * op.dense_blocks[k].n;
    }
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    cudaEventRecord(ev1, s);
    cudaEventSynchronize(ev1);
    cudaEventElapsedTime(&ms, ev0, ev1);
    op.info.ms_near = ms;
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);

    // ---- statistics ------------------------------------------------------------
    int64_t stored = 0, rsum = 0, rmin = INT64_MAX, rmx = 0;
    for (int k = 0; k < op.n_near; ++k) stored += (int64_t)op.dense_blocks[k].m * op.dense_blocks[k].n;
    for (int k = 0; k < op.n_far; ++k) {
        stored += (int64_t)op.rank[k] * (op.far_blocks[k].m + op.far_blocks[k].n);
        rsum += op.rank[k];
        rmin = std::min<int64_t>(rmin, op.rank[k]);
        rmx = std::max<int64_t>(rmx, op.rank[k]);
    }
    op.info.stored_entries = stored;
    op.info.rank_sum = rsum;
    op.info.rank_min = op.n_far ? rmin : 0;
    op.info.rank_max = rmx;
    for (int b = 0; b < nfar; ++b) op.info.entries_evaluated += (int64_t)final_rank[b] * (farb[b].m + farb[b].n);
    return RT_OK;
}


// ---------------------------------------------------------------------------
// Rows of the surface-to-volume matrix Sbar^E_{i,l} (Section 2, last
// paragraph): the emitter source with Q0 replaced by the P1 hat function of
// emitter vertex l.  Each quadrature value of a triangle is split over the
// triangle's three vertices by its barycentric weights; a source point that is
// a vertex of the triangle gives that vertex the limit (angle)/(8 pi).  One CTA
// per row, threads over the emitter triangles, the row [G][L] accumulated in
// shared memory (float atomics: the summation order is not fixed).
// col_of[v] = column (surface tree order) of tree vertex v, -1 off the emitter.
// out[g * gstride + (i - row0) * L + l], rows i in [row0, row0 + nrows).
// ---------------------------------------------------------------------------
template <int MG>
__global__ void __launch_bounds__(256) srcop_rows_kernel(KernelParams P, int n_emit, const int4* __restrict__ emit,
                                                         const int* __restrict__ col_of, int L, int row0, int nrows,
                                                         float* __restrict__ out, int64_t gstride)
{
    extern __shared__ float srow[];   // [G][L]
    const int G = P.G;
    const float inv4pi = (float)(1.0 / (4.0 * kPi));
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
        const int i = row0 + r;
        __syncthreads();
        for (int k = threadIdx.x; k < G * L; k += blockDim.x) srow[k] = 0.f;
        __syncthreads();
        const Vec3<float> xi = load_xyz<float>(P, i);
        Vec3<float> xb = xi;
        bool on_wall = false;
        if (P.has_wall) {
            xb = mirror_point<float>(P, xi);
            on_wall = dist2<float>(xi, xb) <= 1e-20f;
        }
        for (int e = threadIdx.x; e < n_emit; e += blockDim.x) {
            const int4 tv = emit[e];
            const int cl[3] = {col_of[tv.x], col_of[tv.y], col_of[tv.z]};
            const Vec3<float> V0 = load_xyz<float>(P, tv.x), V1 = load_xyz<float>(P, tv.y),
                              V2 = load_xyz<float>(P, tv.z);
            const Vec3<float> e1 = {V1.x - V0.x, V1.y - V0.y, V1.z - V0.z};
            const Vec3<float> e2 = {V2.x - V0.x, V2.y - V0.y, V2.z - V0.z};
            Vec3<float> nn = {e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x};
            const float a2 = sqrtf(nn.x * nn.x + nn.y * nn.y + nn.z * nn.z);
            nn.x /= a2;
            nn.y /= a2;
            nn.z /= a2;
            const float area = 0.5f * a2;
            const Vec3<float> cen = {(V0.x + V1.x + V2.x) / 3.f, (V0.y + V1.y + V2.y) / 3.f, (V0.z + V1.z + V2.z) / 3.f};
            float diam2 = fmaxf(fmaxf(dist2<float>(V0, V1), dist2<float>(V0, V2)), dist2<float>(V1, V2));
            const int vloc = tv.x == i ? 0 : (tv.y == i ? 1 : (tv.z == i ? 2 : -1));
            float a[3][MG];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int g = 0; g < MG; ++g) a[k][g] = 0.f;
            for (int term = 0; term < 2 + P.n_extra; ++term) {
                if (term == 1 && !P.has_wall) continue;
                Vec3<float> src;
                float scale;
                term_source<float>(P, term, xi, xb, src, scale);
                const bool at_x = term == 0 || (term == 1 ? on_wall : dist2<float>(xi, src) <= 1e-20f);
                if (vloc >= 0 && at_x) {
                    const Vec3<float> A = vloc == 0 ? V0 : (vloc == 1 ? V1 : V2);
                    const Vec3<float> B = vloc == 0 ? V1 : (vloc == 1 ? V2 : V0);
                    const Vec3<float> Cc = vloc == 0 ? V2 : (vloc == 1 ? V0 : V1);
                    const Vec3<float> u = {B.x - A.x, B.y - A.y, B.z - A.z}, v = {Cc.x - A.x, Cc.y - A.y, Cc.z - A.z};
                    float cs = (u.x * v.x + u.y * v.y + u.z * v.z) /
                               sqrtf((u.x * u.x + u.y * u.y + u.z * u.z) * (v.x * v.x + v.y * v.y + v.z * v.z));
                    cs = fminf(1.f, fmaxf(-1.f, cs));
                    const float lim = scale * acosf(cs) * (float)(1.0 / (8.0 * kPi));
#pragma unroll
                    for (int g = 0; g < MG; ++g) a[vloc][g] += lim;
                    continue;
                }
                const float sd = (src.x - V0.x) * nn.x + (src.y - V0.y) * nn.y + (src.z - V0.z) * nn.z;
                if (!(sd < 0.f)) continue;
                const float cm = -sd;
                const bool nearp = dist2<float>(src, cen) < 4.f * diam2;
                const int q0 = nearp ? 3 : 0, nq = nearp ? 7 : 3;
                for (int q = 0; q < nq; ++q) {
                    const float b[3] = {(float)c_tri_b[3 * (q0 + q)], (float)c_tri_b[3 * (q0 + q) + 1],
                                        (float)c_tri_b[3 * (q0 + q) + 2]};
                    const Vec3<float> y = {b[0] * V0.x + b[1] * V1.x + b[2] * V2.x, b[0] * V0.y + b[1] * V1.y + b[2] * V2.y,
                                           b[0] * V0.z + b[1] * V1.z + b[2] * V2.z};
                    const float r2 = dist2<float>(src, y);
                    const float tau = term_depth<float>(P, term, xi, src, y);
                    const float geo = scale * area * (float)c_tri_w[q0 + q] * cm * cm / (r2 * r2) * inv4pi;
#pragma unroll
                    for (int g = 0; g < MG; ++g) {
                        if (g < G) {
                            const float v = geo * expf(-P.cf[g] * tau);
#pragma unroll
                            for (int k = 0; k < 3; ++k) a[k][g] += v * b[k];
                        }
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < MG; ++g)
                if (g < G)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (cl[k] >= 0) atomicAdd(srow + g * L + cl[k], a[k][g]);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < G * L; k += blockDim.x) {
            const int g = k / L, l = k - g * L;
            out[g * gstride + (int64_t)r * L + l] = srow[k];
        }
    }
}

int srcop_eval_rows(Operator& op, const int* col_of, int L, int row0, int nrows, float* out, int64_t gstride,
                    cudaStream_t s, std::string& err)
{
    const size_t smem = sizeof(float) * (size_t)op.G * L;
    if (smem > 200 * 1024) {
        err = "surface-to-volume operator: G x L too large for one row in shared memory";
        return RT_EINVAL;
    }
    const int grid = std::max(1, std::min(nrows, 152 * 8));
#define RT_SRC_ROWS(MG)                                                                                        \
    do {                                                                                                       \
        RT_CUDA_TRY(cudaFuncSetAttribute(srcop_rows_kernel<MG>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                         (int)smem));                                                          \
        srcop_rows_kernel<MG><<<grid, 256, smem, s>>>(op.kp, op.n_emit, op.d_emit, col_of, L, row0, nrows, out, \
                                                      gstride);                                                \
    } while (0)
    if (op.G <= 1) RT_SRC_ROWS(1);
    else if (op.G <= 4) RT_SRC_ROWS(4);
    else if (op.G <= 8) RT_SRC_ROWS(8);
    else if (op.G <= 16) RT_SRC_ROWS(16);
    else {
        err = "surface-to-volume operator: at most 16 kappa groups";
        return RT_EINVAL;
    }
#undef RT_SRC_ROWS
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

// diagnostic: the library's FP32 sin(2 pi x) beside CUDA's sinpif(2x)
__global__ void sin2pi_probe(const float* __restrict__ x, float* __restrict__ lib, float* __restrict__ ref, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        lib[i] = sin2pi(x[i]);
        ref[i] = sinpif(2.0f * x[i]);
    }
}

int eval_sin2pi(const float* x, float* lib, float* ref, int64_t n, cudaStream_t s, std::string& err)
{
    if (n <= 0) return RT_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    sin2pi_probe<<<grid, 256, 0, s>>>(x, lib, ref, n);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

}  // namespace rt

