// rt_srcop.cu -- the surface-to-volume matrix Sbar^E_{i,l} as a compressed
// operator (Section 2, last paragraph; Section 2.1: "for each value of nu we
// have two large dense matrices", both compressed as H-matrices).
//
// Sbar^E_{i,l} is the emitter source with the emitter coefficient Q0 replaced
// by the P1 hat function of emitter-surface vertex l, so that for any
// per-vertex coefficients Q0_l,  Sbar^E_{nu,i} = sum_l Sbar^E_{i,l} Q0_l
// (times the intensity B_nu(T_emit)).  One N x L matrix per kappa group.
//
// Build:
//   * columns = the emitter vertices, clustered by the same median bisection
//     as the volume vertices; rows = the volume cluster tree of the operator;
//   * rectangular block tree: a (volume cluster, surface cluster) pair is
//     admissible under the operator's rule (max(R_t, R_s) < eta d(t, s));
//     otherwise the larger one is split; two leaves give a dense block;
//   * every entry is evaluated once on the GPU (rt_assemble.cu,
//     srcop_rows_kernel), in slabs of rows;
//   * each admissible block and group is compressed by partially pivoted ACA
//     on its stored entries (one CTA per block and group, FP64 norm update,
//     relative Frobenius tolerance eps); a block whose rank would reach the
//     cap stays dense.
// Apply (row-owned, deterministic): w = V^T q per far block, then per volume
// leaf y = sum U w + sum A q, then out_nu = B_nu(T_emit) y_{g(nu)} in the
// caller's vertex order.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "rt_internal.h"

namespace rt {

namespace so {
constexpr int kRankCap = 32;      // ACA terms per block before it is stored dense
constexpr int kThreads = 256;
}  // namespace so

struct SoBlock {
    int row0, m, col0, n;   // tree-order rows, surface-tree-order columns
    int far;                // 1 admissible (ACA), 0 dense
};

struct SoFarG {             // one far block and group after compression
    int64_t u;              // U [m][r] (row-major)
    int64_t v;              // V^T [r][n]
    int64_t w;              // w [r] offset in the apply scratch
    int r, b;
};

struct SoRec {              // one (block, group) piece of a volume leaf's rows
    int64_t a;              // far: U offset of the leaf's first row; dense: A offset of that row
    int64_t w;              // far: w offset; dense: -1
    int r_or_n;             // far: rank (U row length); dense: n (A row length)
    int col0;               // dense: first column
    int g;
};

// ---------------------------------------------------------------------------
// ACA on stored entries: one CTA per (far block, group)
// ---------------------------------------------------------------------------
struct SoAcaJob {
    int64_t d;       // entry (0, 0) of the block in the stored slab, row stride ld
    int64_t ld;
    int64_t u, v;    // scratch: U [m][cap], V [n][cap]
    int m, n;
};

__device__ __forceinline__ void so_argmax(float& val, int& idx, float* sv, int* si)
{
    // block-wide argmax of |val| (smallest index on ties)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, val, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (fabsf(ov) > fabsf(val) || (fabsf(ov) == fabsf(val) && oi < idx)) {
            val = ov;
            idx = oi;
        }
    }
    __syncthreads();
    if (lane == 0) {
        sv[warp] = val;
        si[warp] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (fabsf(sv[w]) > fabsf(sv[0]) || (fabsf(sv[w]) == fabsf(sv[0]) && si[w] < si[0])) {
                sv[0] = sv[w];
                si[0] = si[w];
            }
    }
    __syncthreads();
    val = sv[0];
    idx = si[0];
}

__device__ __forceinline__ double so_sum(double v, double* sd)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sd[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sd[w];
        sd[0] = t;
    }
    __syncthreads();
    return sd[0];
}

// ranks[job] = rank reached, or -1 when the block must stay dense.  `used`
// (scratch, one byte per row of every job) marks the rows already pivoted.
__global__ void __launch_bounds__(so::kThreads) so_aca_kernel(const SoAcaJob* __restrict__ jobs, int njobs,
                                                             const float* __restrict__ D, float* __restrict__ U,
                                                             float* __restrict__ V, unsigned char* __restrict__ used,
                                                             const int64_t* __restrict__ used_off, int* __restrict__ ranks,
                                                             float* __restrict__ rowbuf, const int64_t* __restrict__ row_off,
                                                             double eps)
{
    __shared__ float sv[so::kThreads / 32];
    __shared__ int si[so::kThreads / 32];
    __shared__ double sd[so::kThreads / 32];
    for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
        const SoAcaJob J = jobs[jb];
        const float* A = D + J.d;
        float* Uj = U + J.u;   // [m][cap]
        float* Vj = V + J.v;   // [n][cap]
        unsigned char* us = used + used_off[jb];
        float* rb = rowbuf + row_off[jb];   // residual row [n] then column [m]
        float* cb = rb + J.n;
        for (int i = threadIdx.x; i < J.m; i += blockDim.x) us[i] = 0;
        __syncthreads();
        int k = 0, istar = 0, nused = 0, result = -1;
        double norm2 = 0.0;
        const int cap = so::kRankCap;
        for (int guard = 0; guard < J.m + cap; ++guard) {
            // residual of row istar
            float best = 0.f;
            int bj = 0x7fffffff;
            for (int j = threadIdx.x; j < J.n; j += blockDim.x) {
                float r = A[(int64_t)istar * J.ld + j];
                for (int q = 0; q < k; ++q) r -= Uj[(int64_t)istar * cap + q] * Vj[(int64_t)j * cap + q];
                rb[j] = r;
                if (fabsf(r) > fabsf(best) || (fabsf(r) == fabsf(best) && j < bj)) {
                    best = r;
                    bj = j;
                }
            }
            so_argmax(best, bj, sv, si);
            if (threadIdx.x == 0) us[istar] = 1;
            ++nused;
            __syncthreads();
            if (!(fabsf(best) > 0.f)) {
                // a zero residual row: take the next row not yet used, or stop
                if (nused >= J.m) {
                    result = k;
                    break;
                }
                int nxt = -1;
                if (threadIdx.x == 0)
                    for (int i = 0; i < J.m; ++i)
                        if (!us[i]) {
                            nxt = i;
                            break;
                        }
                if (threadIdx.x == 0) si[0] = nxt;
                __syncthreads();
                istar = si[0];
                __syncthreads();
                continue;
            }
            if ((int64_t)(k + 1) * (J.m + J.n) >= (int64_t)J.m * J.n || k + 1 > cap) break;   // stays dense (-1)
            const float inv = 1.f / best;
            const int jstar = bj;
            double nv2 = 0.0, nu2 = 0.0;
            for (int j = threadIdx.x; j < J.n; j += blockDim.x) {
                const float v = rb[j] * inv;
                Vj[(int64_t)j * cap + k] = v;
                nv2 += (double)v * v;
            }
            // residual of column jstar
            float bu = 0.f;
            int bi = 0x7fffffff;
            for (int i = threadIdx.x; i < J.m; i += blockDim.x) {
                float u = A[(int64_t)i * J.ld + jstar];
                for (int q = 0; q < k; ++q) u -= Vj[(int64_t)jstar * cap + q] * Uj[(int64_t)i * cap + q];
                Uj[(int64_t)i * cap + k] = u;
                cb[i] = u;
                nu2 += (double)u * u;
                if (!us[i] && (fabsf(u) > fabsf(bu) || (fabsf(u) == fabsf(bu) && i < bi))) {
                    bu = u;
                    bi = i;
                }
            }
            __syncthreads();
            nv2 = so_sum(nv2, sd);
            nu2 = so_sum(nu2, sd);
            // |S_{k+1}|^2 = |S_k|^2 + 2 sum_q (U_q . u)(V_q . v) + |u|^2 |v|^2  (FP64)
            double cross = 0.0;
            for (int q = 0; q < k; ++q) {
                double du = 0.0, dv = 0.0;
                for (int i = threadIdx.x; i < J.m; i += blockDim.x) du += (double)Uj[(int64_t)i * cap + q] * cb[i];
                for (int j = threadIdx.x; j < J.n; j += blockDim.x)
                    dv += (double)Vj[(int64_t)j * cap + q] * Vj[(int64_t)j * cap + k];
                du = so_sum(du, sd);
                dv = so_sum(dv, sd);
                cross += du * dv;
            }
            norm2 += 2.0 * cross + nu2 * nv2;
            ++k;
            if (sqrt(nu2 * nv2) <= eps * sqrt(fmax(norm2, 0.0))) {
                result = k;
                break;
            }
            so_argmax(bu, bi, sv, si);
            if (bi == 0x7fffffff || nused >= J.m) {   // every row used: the block is exact at rank k
                result = k;
                break;
            }
            istar = bi;
        }
        if (threadIdx.x == 0) ranks[jb] = result;
        __syncthreads();
    }
}

// copy U (first r columns of the cap-wide scratch) and V^T into the packed storage
__global__ void so_pack_far(const SoAcaJob* __restrict__ jobs, const SoFarG* __restrict__ fg, int nf,
                            const int* __restrict__ job_of, const float* __restrict__ U, const float* __restrict__ V,
                            float* __restrict__ store)
{
    for (int f = blockIdx.x; f < nf; f += gridDim.x) {
        const SoFarG F = fg[f];
        const SoAcaJob J = jobs[job_of[f]];
        for (int e = threadIdx.x; e < J.m * F.r; e += blockDim.x) {
            const int i = e / F.r, q = e - i * F.r;
            store[F.u + e] = U[J.u + (int64_t)i * so::kRankCap + q];
        }
        for (int e = threadIdx.x; e < J.n * F.r; e += blockDim.x) {
            const int q = e / J.n, j = e - q * J.n;
            store[F.v + e] = V[J.v + (int64_t)j * so::kRankCap + q];
        }
    }
}

// dense blocks: copy the stored entries [m][n] (row stride ld) into the packed storage
struct SoDenseCopy {
    int64_t src, dst, ld;
    int m, n;
};
__global__ void so_pack_dense(const SoDenseCopy* __restrict__ cp, int nc, const float* __restrict__ D,
                              float* __restrict__ store)
{
    for (int c = blockIdx.x; c < nc; c += gridDim.x) {
        const SoDenseCopy C = cp[c];
        for (int e = threadIdx.x; e < C.m * C.n; e += blockDim.x) {
            const int i = e / C.n, j = e - i * C.n;
            store[C.dst + e] = D[C.src + (int64_t)i * C.ld + j];
        }
    }
}

// ---------------------------------------------------------------------------
// apply
// ---------------------------------------------------------------------------
// q (surface tree order) from the caller's per-vertex coefficients
__global__ void so_gather_q(const float* __restrict__ q_in, const int* __restrict__ perm, int L, float* __restrict__ q)
{
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x) q[l] = q_in[perm[l]];
}

// w[f.w + k] = sum_j V^T[k][j] q[col0 + j]: one warp per (far block, group, term)
__global__ void so_phase1(const SoFarG* __restrict__ fg, int nf, const SoBlock* __restrict__ blocks,
                          const float* __restrict__ store, const float* __restrict__ q, float* __restrict__ w,
                          const int64_t* __restrict__ term0)
{
    const int lane = threadIdx.x & 31;
    const int64_t nt = term0[nf];
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nt;
         t += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        int lo = 0, hi = nf - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (term0[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const SoFarG F = fg[lo];
        const int k = (int)(t - term0[lo]);
        const SoBlock B = blocks[F.b];
        const float* v = store + F.v + (int64_t)k * B.n;
        float s = 0.f;
        for (int j = lane; j < B.n; j += 32) s += v[j] * q[B.col0 + j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) w[F.w + k] = s;
    }
}

// per volume leaf (CTA) and group: y = sum_far U w + sum_dense A q over the leaf's
// records; then out[f][perm[row]] = scale[f] y_{g(f)}[row]
__global__ void __launch_bounds__(128) so_phase2(const int* __restrict__ leaf_row0, const int* __restrict__ leaf_m,
                                                 const int* __restrict__ rec_ptr, const SoRec* __restrict__ recs,
                                                 const float* __restrict__ store, const float* __restrict__ w,
                                                 const float* __restrict__ q, int G, int F,
                                                 const int* __restrict__ fgroup, const double* __restrict__ fscale,
                                                 const int* __restrict__ perm, int N, float* __restrict__ out)
{
    extern __shared__ float ys[];   // [G][64]
    const int l = blockIdx.x;
    const int row0 = leaf_row0[l], m = leaf_m[l];
    for (int k = threadIdx.x; k < G * 64; k += blockDim.x) ys[k] = 0.f;
    __syncthreads();
    // threads: 2 x 64 = rows x two halves of the record list
    const int i = threadIdx.x & 63, half = threadIdx.x >> 6;
    float acc[16];
#pragma unroll
    for (int g = 0; g < 16; ++g) acc[g] = 0.f;
    if (i < m) {
        for (int r = rec_ptr[l] + half; r < rec_ptr[l + 1]; r += 2) {
            const SoRec R = recs[r];
            float s = 0.f;
            if (R.w >= 0) {
                const float* u = store + R.a + (int64_t)i * R.r_or_n;
                for (int k = 0; k < R.r_or_n; ++k) s += u[k] * w[R.w + k];
            } else {
                const float* a = store + R.a + (int64_t)i * R.r_or_n;
                for (int j = 0; j < R.r_or_n; ++j) s += a[j] * q[R.col0 + j];
            }
#pragma unroll
            for (int g = 0; g < 16; ++g)
                if (g == R.g) acc[g] += s;
        }
    }
    for (int h = 0; h < 2; ++h) {
        if (half == h && i < m)
            for (int g = 0; g < G && g < 16; ++g) ys[g * 64 + i] += acc[g];
        __syncthreads();
    }
    for (int e = threadIdx.x; e < F * m; e += blockDim.x) {
        const int f = e / m, r = e - f * m;
        out[(int64_t)f * N + perm[row0 + r]] = (float)(fscale[f] * (double)ys[fgroup[f] * 64 + r]);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct SoNode {
    int start, size, left, right;
    double c[3], R;
};

// centroid and radius of every cluster node (points given in tree order)
static void so_geometry(const std::vector<ClusterNode>& cl, const std::vector<double>& pts, std::vector<SoNode>& out)
{
    out.resize(cl.size());
    for (size_t k = 0; k < cl.size(); ++k) {
        SoNode& o = out[k];
        o.start = cl[k].start;
        o.size = cl[k].size;
        o.left = cl[k].left;
        o.right = cl[k].right;
        o.c[0] = o.c[1] = o.c[2] = 0.0;
        for (int p = o.start; p < o.start + o.size; ++p)
            for (int d = 0; d < 3; ++d) o.c[d] += pts[3 * (size_t)p + d];
        for (int d = 0; d < 3; ++d) o.c[d] /= std::max(1, o.size);
        double R2 = 0.0;
        for (int p = o.start; p < o.start + o.size; ++p) {
            double r2 = 0.0;
            for (int d = 0; d < 3; ++d) r2 += (pts[3 * (size_t)p + d] - o.c[d]) * (pts[3 * (size_t)p + d] - o.c[d]);
            R2 = std::max(R2, r2);
        }
        o.R = std::sqrt(R2);
    }
}

static void so_blocks(const std::vector<SoNode>& T, int t, const std::vector<SoNode>& S, int s, double eta, int adm,
                      std::vector<SoBlock>& out)
{
    const SoNode &a = T[t], &b = S[s];
    double d = 0.0;
    for (int k = 0; k < 3; ++k) d += (a.c[k] - b.c[k]) * (a.c[k] - b.c[k]);
    d = std::sqrt(d);
    if (adm == RT_ADM_GAP) d -= a.R + b.R;
    if (std::max(a.R, b.R) < eta * d) {
        out.push_back({a.start, a.size, b.start, b.size, 1});
        return;
    }
    const bool lt = a.left < 0, ls = b.left < 0;
    if (lt && ls) {
        out.push_back({a.start, a.size, b.start, b.size, 0});
        return;
    }
    if (ls || (!lt && a.size >= b.size)) {
        so_blocks(T, a.left, S, s, eta, adm, out);
        so_blocks(T, a.right, S, s, eta, adm, out);
    } else {
        so_blocks(T, t, S, b.left, eta, adm, out);
        so_blocks(T, t, S, b.right, eta, adm, out);
    }
}

struct SourceOp {
    Operator* op = nullptr;
    int N = 0, L = 0, G = 0, F = 0;
    std::vector<int> sv_caller;   // column -> caller vertex id (ascending)
    std::vector<SoBlock> blocks;
    std::vector<SoFarG> far;
    int n_dense = 0;
    int64_t stored = 0, rank_sum = 0, rank_max = 0, apply_bytes = 0;
    double ms_eval = 0.0, ms_aca = 0.0;
    int64_t device_bytes = 0;
    // device
    float* store = nullptr;
    float* w = nullptr;
    float* q = nullptr;
    int* d_qperm = nullptr;       // surface tree position -> column (caller order)
    SoFarG* d_far = nullptr;
    int64_t* d_term0 = nullptr;
    SoBlock* d_blocks = nullptr;
    int *d_leaf_row0 = nullptr, *d_leaf_m = nullptr, *d_rec_ptr = nullptr;
    SoRec* d_recs = nullptr;
    double* d_fscale = nullptr;   // B_nu(T_emit) per channel (grey: sigma T_emit^4)
    std::vector<void*> allocs;
};

template <class T>
static int so_alloc(SourceOp& S, T** p, size_t count, cudaStream_t s, std::string& err)
{
    cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * std::max<size_t>(count, 1), s);
    if (e != cudaSuccess) {
        err = std::string("cudaMallocAsync (source operator): ") + cudaGetErrorString(e);
        *p = nullptr;
        return RT_ENOMEM;
    }
    S.allocs.push_back(*p);
    S.device_bytes += (int64_t)(sizeof(T) * std::max<size_t>(count, 1));
    return RT_OK;
}

void source_op_release(SourceOp& S, cudaStream_t s)
{
    for (void* p : S.allocs) cudaFreeAsync(p, s);
    S.allocs.clear();
}

int source_op_build(SourceOp& S, Operator& op, double eps, cudaStream_t s, std::string& err)
{
    if (op.mode != RT_MODE_HMATRIX) {
        err = "the surface-to-volume operator needs an H-matrix operator";
        return RT_EINVAL;
    }
    if (op.n_emit <= 0) {
        err = "the problem has no emitter";
        return RT_EINVAL;
    }
    for (int sz : op.plan.leaf_size)
        if (sz > 64) {
            err = "the surface-to-volume operator needs leaves of at most 64 rows";
            return RT_EINVAL;
        }
    int rc;
    S.op = &op;
    S.N = op.N;
    S.G = op.G;
    S.F = op.F;
    // ---- emitter vertices: columns in ascending caller order, then their cluster tree ----
    std::vector<int4> tri(op.n_emit);
    RT_CUDA_TRY(cudaMemcpyAsync(tri.data(), op.d_emit, sizeof(int4) * op.n_emit, cudaMemcpyDeviceToHost, s));
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int> tv;
    for (const int4& t : tri) {
        tv.push_back(t.x);
        tv.push_back(t.y);
        tv.push_back(t.z);
    }
    std::sort(tv.begin(), tv.end());
    tv.erase(std::unique(tv.begin(), tv.end()), tv.end());
    const int L = (int)tv.size();
    S.L = L;
    std::vector<int> caller(L);
    for (int l = 0; l < L; ++l) caller[l] = op.plan.perm[tv[l]];
    std::vector<int> ord(L);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return caller[a] < caller[b]; });
    S.sv_caller.resize(L);
    std::vector<int> col_tree(L);   // column (caller order) -> tree vertex
    for (int c = 0; c < L; ++c) {
        S.sv_caller[c] = caller[ord[c]];
        col_tree[c] = tv[ord[c]];
    }
    std::vector<double> xyz((size_t)op.N * 3);
    RT_CUDA_TRY(cudaMemcpyAsync(xyz.data(), op.d_xyz64, sizeof(double) * xyz.size(), cudaMemcpyDeviceToHost, s));
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<double> sxyz((size_t)L * 3);
    for (int c = 0; c < L; ++c)
        for (int d = 0; d < 3; ++d) sxyz[3 * (size_t)c + d] = xyz[3 * (size_t)col_tree[c] + d];
    Plan sp;
    if ((rc = plan_build(sxyz.data(), L, op.leaf, op.eta, op.adm, sp, err))) return rc;
    // surface tree position p holds column sp.perm[p]
    std::vector<double> spts((size_t)L * 3);
    for (int p = 0; p < L; ++p)
        for (int d = 0; d < 3; ++d) spts[3 * (size_t)p + d] = sxyz[3 * (size_t)sp.perm[p] + d];
    std::vector<int> col_of_tree(op.N, -1);   // tree vertex -> surface tree position
    for (int p = 0; p < L; ++p) col_of_tree[col_tree[sp.perm[p]]] = p;
    // ---- rectangular block tree ----
    std::vector<SoNode> Tn, Sn;
    so_geometry(op.plan.clusters, xyz, Tn);
    so_geometry(sp.clusters, spts, Sn);
    so_blocks(Tn, 0, Sn, 0, op.eta, op.adm, S.blocks);
    // ---- entries, a slab of rows at a time, then ACA / dense copies per slab ----
    int* d_col = nullptr;
    if ((rc = so_alloc(S, &d_col, op.N, s, err))) return rc;
    RT_CUDA_TRY(cudaMemcpyAsync(d_col, col_of_tree.data(), sizeof(int) * op.N, cudaMemcpyHostToDevice, s));
    // blocks sorted by row0 so that a slab of rows holds whole blocks
    std::stable_sort(S.blocks.begin(), S.blocks.end(), [](const SoBlock& a, const SoBlock& b) {
        return a.row0 != b.row0 ? a.row0 < b.row0 : a.col0 < b.col0;
    });
    const int G = S.G;
    // slab: consecutive blocks whose rows fit in about 1 GiB of entries
    const int64_t slab_entries = std::max<int64_t>((int64_t)1 << 28, (int64_t)L * 1024) / G;
    // every slab is packed into its own storage (sized after its compression); the
    // slab storages are concatenated at the end
    std::vector<SoFarG> far;
    std::vector<SoDenseCopy> dense_cp;
    int64_t store_len = 0;
    // final storage is filled per slab: grow a device buffer as needed
    float* D = nullptr;
    int64_t D_len = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    size_t b0 = 0;
    std::vector<float*> pieces;      // packed storage per slab (freed into S.store at the end)
    std::vector<int64_t> piece_len;
    while (b0 < S.blocks.size()) {
        // rows [r0, r1) of this slab hold whole blocks: a block that starts inside the
        // slab is always taken (and may extend it); one that starts at r1 or later is
        // taken while the slab stays within slab_entries per group
        const int r0 = S.blocks[b0].row0;
        int r1 = r0;
        size_t b1 = b0;
        while (b1 < S.blocks.size()) {
            const SoBlock& B = S.blocks[b1];
            if (b1 > b0 && B.row0 >= r1 && (int64_t)(std::max(r1, B.row0 + B.m) - r0) * L > slab_entries) break;
            r1 = std::max(r1, B.row0 + B.m);
            ++b1;
        }
        const int nrows = r1 - r0;
        const int64_t need = (int64_t)G * nrows * L;
        if (need > D_len) {
            if (D) cudaFreeAsync(D, s);
            RT_CUDA_TRY(cudaMallocAsync((void**)&D, sizeof(float) * need, s));
            D_len = need;
        }
        cudaEventRecord(e0, s);
        if ((rc = srcop_eval_rows(op, d_col, L, r0, nrows, D, (int64_t)nrows * L, s, err))) return rc;
        cudaEventRecord(e1, s);
        RT_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        S.ms_eval += ms;
        // ACA jobs of this slab's far blocks
        std::vector<SoAcaJob> jobs;
        std::vector<std::pair<int, int>> job_bg;
        std::vector<int64_t> uoff, roff;
        int64_t ulen = 0, vlen = 0, blen = 0, rlen = 0;
        for (size_t b = b0; b < b1; ++b) {
            const SoBlock& B = S.blocks[b];
            if (!B.far) continue;
            for (int g = 0; g < G; ++g) {
                SoAcaJob J;
                J.d = (int64_t)g * nrows * L + (int64_t)(B.row0 - r0) * L + B.col0;
                J.ld = L;
                J.u = ulen;
                J.v = vlen;
                J.m = B.m;
                J.n = B.n;
                ulen += (int64_t)B.m * so::kRankCap;
                vlen += (int64_t)B.n * so::kRankCap;
                uoff.push_back(blen);
                blen += B.m;
                roff.push_back(rlen);
                rlen += B.m + B.n;
                jobs.push_back(J);
                job_bg.push_back({(int)b, g});
            }
        }
        std::vector<int> ranks(jobs.size(), -1);
        float *dU = nullptr, *dV = nullptr, *drb = nullptr;
        unsigned char* dused = nullptr;
        SoAcaJob* djobs = nullptr;
        int64_t *duo = nullptr, *dro = nullptr;
        int* drk = nullptr;
        if (!jobs.empty()) {
            RT_CUDA_TRY(cudaMallocAsync((void**)&dU, sizeof(float) * ulen, s));
            RT_CUDA_TRY(cudaMallocAsync((void**)&dV, sizeof(float) * vlen, s));
            RT_CUDA_TRY(cudaMallocAsync((void**)&drb, sizeof(float) * rlen, s));
            RT_CUDA_TRY(cudaMallocAsync((void**)&dused, blen, s));
            RT_CUDA_TRY(cudaMallocAsync((void**)&djobs, sizeof(SoAcaJob) * jobs.size(), s));
            RT_CUDA_TRY(cudaMallocAsync((void**)&duo, sizeof(int64_t) * jobs.size(), s));
            RT_CUDA_TRY(cudaMallocAsync((void**)&dro, sizeof(int64_t) * jobs.size(), s));
            RT_CUDA_TRY(cudaMallocAsync((void**)&drk, sizeof(int) * jobs.size(), s));
            RT_CUDA_TRY(cudaMemcpyAsync(djobs, jobs.data(), sizeof(SoAcaJob) * jobs.size(), cudaMemcpyHostToDevice, s));
            RT_CUDA_TRY(cudaMemcpyAsync(duo, uoff.data(), sizeof(int64_t) * jobs.size(), cudaMemcpyHostToDevice, s));
            RT_CUDA_TRY(cudaMemcpyAsync(dro, roff.data(), sizeof(int64_t) * jobs.size(), cudaMemcpyHostToDevice, s));
            cudaEventRecord(e0, s);
            so_aca_kernel<<<(int)std::min<size_t>(jobs.size(), 152 * 8), so::kThreads, 0, s>>>(
                djobs, (int)jobs.size(), D, dU, dV, dused, duo, drk, drb, dro, op.aca_eps);
            RT_CUDA_TRY(cudaGetLastError());
            cudaEventRecord(e1, s);
            RT_CUDA_TRY(cudaMemcpyAsync(ranks.data(), drk, sizeof(int) * jobs.size(), cudaMemcpyDeviceToHost, s));
            RT_CUDA_TRY(cudaStreamSynchronize(s));
            cudaEventElapsedTime(&ms, e0, e1);
            S.ms_aca += ms;
        }
        // a far block stays compressed only if every group converged within the cap
        std::vector<int> block_ok(b1 - b0, 1);
        for (size_t k = 0; k < jobs.size(); ++k)
            if (ranks[k] < 0) block_ok[job_bg[k].first - b0] = 0;
        // packed layout of this slab
        std::vector<SoFarG> sfar;
        std::vector<int> sjob;
        std::vector<SoDenseCopy> sden;
        int64_t plen = 0;
        for (size_t k = 0; k < jobs.size(); ++k) {
            const int b = job_bg[k].first, g = job_bg[k].second;
            if (!block_ok[b - b0]) continue;
            const SoBlock& B = S.blocks[b];
            SoFarG F;
            F.r = ranks[k];
            F.b = b;
            F.u = plen;
            plen += (int64_t)B.m * F.r;
            F.v = plen;
            plen += (int64_t)F.r * B.n;
            F.w = 0;
            sfar.push_back(F);
            sjob.push_back((int)k);
        }
        for (size_t b = b0; b < b1; ++b) {
            SoBlock& B = S.blocks[b];
            if (B.far && block_ok[b - b0]) continue;
            B.far = 0;
            for (int g = 0; g < G; ++g) {
                SoDenseCopy C;
                C.src = (int64_t)g * nrows * L + (int64_t)(B.row0 - r0) * L + B.col0;
                C.ld = L;
                C.m = B.m;
                C.n = B.n;
                C.dst = plen;
                plen += (int64_t)B.m * B.n;
                sden.push_back(C);
            }
        }
        float* P = nullptr;
        RT_CUDA_TRY(cudaMallocAsync((void**)&P, sizeof(float) * std::max<int64_t>(plen, 1), s));
        if (!sfar.empty()) {
            SoFarG* dfg = nullptr;
            int* djo = nullptr;
            RT_CUDA_TRY(cudaMallocAsync((void**)&dfg, sizeof(SoFarG) * sfar.size(), s));
            RT_CUDA_TRY(cudaMallocAsync((void**)&djo, sizeof(int) * sjob.size(), s));
            RT_CUDA_TRY(cudaMemcpyAsync(dfg, sfar.data(), sizeof(SoFarG) * sfar.size(), cudaMemcpyHostToDevice, s));
            RT_CUDA_TRY(cudaMemcpyAsync(djo, sjob.data(), sizeof(int) * sjob.size(), cudaMemcpyHostToDevice, s));
            so_pack_far<<<(int)std::min<size_t>(sfar.size(), 152 * 8), 256, 0, s>>>(djobs, dfg, (int)sfar.size(), djo,
                                                                                   dU, dV, P);
            RT_CUDA_TRY(cudaGetLastError());
            cudaFreeAsync(dfg, s);
            cudaFreeAsync(djo, s);
        }
        if (!sden.empty()) {
            SoDenseCopy* dc = nullptr;
            RT_CUDA_TRY(cudaMallocAsync((void**)&dc, sizeof(SoDenseCopy) * sden.size(), s));
            RT_CUDA_TRY(cudaMemcpyAsync(dc, sden.data(), sizeof(SoDenseCopy) * sden.size(), cudaMemcpyHostToDevice, s));
            so_pack_dense<<<(int)std::min<size_t>(sden.size(), 152 * 8), 256, 0, s>>>(dc, (int)sden.size(), D, P);
            RT_CUDA_TRY(cudaGetLastError());
            cudaFreeAsync(dc, s);
        }
        for (void* p : {(void*)dU, (void*)dV, (void*)drb, (void*)dused, (void*)djobs, (void*)duo, (void*)dro, (void*)drk})
            if (p) cudaFreeAsync(p, s);
        // offsets become global once the slab storages are concatenated
        for (SoFarG& F : sfar) {
            F.u += store_len;
            F.v += store_len;
            far.push_back(F);
        }
        for (SoDenseCopy& C : sden) {
            C.dst += store_len;
            dense_cp.push_back(C);
        }
        pieces.push_back(P);
        piece_len.push_back(plen);
        store_len += plen;
        b0 = b1;
    }
    if (D) cudaFreeAsync(D, s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // one storage array
    if ((rc = so_alloc(S, &S.store, (size_t)std::max<int64_t>(store_len, 1), s, err))) return rc;
    {
        int64_t off = 0;
        for (size_t k = 0; k < pieces.size(); ++k) {
            if (piece_len[k] > 0)
                RT_CUDA_TRY(cudaMemcpyAsync(S.store + off, pieces[k], sizeof(float) * piece_len[k],
                                            cudaMemcpyDeviceToDevice, s));
            cudaFreeAsync(pieces[k], s);
            off += piece_len[k];
        }
    }
    // ---- apply structures ----
    int64_t wl = 0;
    std::vector<int64_t> term0(far.size() + 1, 0);
    for (size_t f = 0; f < far.size(); ++f) {
        far[f].w = wl;
        wl += far[f].r;
        term0[f + 1] = wl;
        S.rank_sum += far[f].r;
        S.rank_max = std::max<int64_t>(S.rank_max, far[f].r);
        S.stored += (int64_t)far[f].r * (S.blocks[far[f].b].m + S.blocks[far[f].b].n);
    }
    S.far = far;
    // per leaf: the (block, group) records over its rows
    const int nl = (int)op.plan.leaf_start.size();
    std::vector<std::vector<SoRec>> per(nl);
    auto leaf_of = [&](int row) {
        int lo = 0, hi = nl - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (op.plan.leaf_start[mid] <= row) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    // far entries of one block were stored group by group: the group is their index in the block
    {
        std::vector<int> seen(S.blocks.size(), 0);
        std::vector<int> gof(far.size());
        for (size_t f = 0; f < far.size(); ++f) gof[f] = seen[far[f].b]++;
        for (size_t f = 0; f < far.size(); ++f) {
            const SoFarG& F = far[f];
            const SoBlock& B = S.blocks[F.b];
            for (int l = leaf_of(B.row0); l < nl && op.plan.leaf_start[l] < B.row0 + B.m; ++l) {
                SoRec R;
                R.a = F.u + (int64_t)(op.plan.leaf_start[l] - B.row0) * F.r;
                R.w = F.w;
                R.r_or_n = F.r;
                R.col0 = B.col0;
                R.g = gof[f];
                per[l].push_back(R);
            }
        }
    }
    {   // dense copies were stored block by block, group by group
        size_t k = 0;
        for (size_t b = 0; b < S.blocks.size(); ++b) {
            const SoBlock& B = S.blocks[b];
            if (B.far) continue;
            ++S.n_dense;
            for (int g = 0; g < G; ++g, ++k) {
                const SoDenseCopy& C = dense_cp[k];
                S.stored += (int64_t)B.m * B.n;
                for (int l = leaf_of(B.row0); l < nl && op.plan.leaf_start[l] < B.row0 + B.m; ++l) {
                    SoRec R;
                    R.a = C.dst + (int64_t)(op.plan.leaf_start[l] - B.row0) * B.n;
                    R.w = -1;
                    R.r_or_n = B.n;
                    R.col0 = B.col0;
                    R.g = g;
                    per[l].push_back(R);
                }
            }
        }
    }
    std::vector<int> rec_ptr(nl + 1, 0);
    std::vector<SoRec> recs;
    for (int l = 0; l < nl; ++l) {
        rec_ptr[l] = (int)recs.size();
        recs.insert(recs.end(), per[l].begin(), per[l].end());
    }
    rec_ptr[nl] = (int)recs.size();
    std::vector<int> lm(nl);
    for (int l = 0; l < nl; ++l) lm[l] = op.plan.leaf_size[l];
    std::vector<int> qperm(L);   // surface tree position -> column
    for (int p = 0; p < L; ++p) qperm[p] = sp.perm[p];
    std::vector<double> fs(S.F);
    // the emitted intensity per unit Q0 (B_nu(T_emit); grey sigma T_emit^4); the kappa
    // scale of a binned channel enters the source only through the group's exponent
    for (int f = 0; f < S.F; ++f) fs[f] = op.q0 != 0.0 ? op.Q[f] / op.q0 : 0.0;
    if ((rc = so_alloc(S, &S.w, (size_t)std::max<int64_t>(wl, 1), s, err)) || (rc = so_alloc(S, &S.q, L, s, err)) ||
        (rc = so_alloc(S, &S.d_qperm, L, s, err)) || (rc = so_alloc(S, &S.d_far, far.size(), s, err)) ||
        (rc = so_alloc(S, &S.d_term0, term0.size(), s, err)) || (rc = so_alloc(S, &S.d_blocks, S.blocks.size(), s, err)) ||
        (rc = so_alloc(S, &S.d_leaf_row0, nl, s, err)) || (rc = so_alloc(S, &S.d_leaf_m, nl, s, err)) ||
        (rc = so_alloc(S, &S.d_rec_ptr, nl + 1, s, err)) || (rc = so_alloc(S, &S.d_recs, recs.size(), s, err)) ||
        (rc = so_alloc(S, &S.d_fscale, S.F, s, err)))
        return rc;
    RT_CUDA_TRY(cudaMemcpyAsync(S.d_qperm, qperm.data(), sizeof(int) * L, cudaMemcpyHostToDevice, s));
    if (!far.empty()) RT_CUDA_TRY(cudaMemcpyAsync(S.d_far, far.data(), sizeof(SoFarG) * far.size(), cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaMemcpyAsync(S.d_term0, term0.data(), sizeof(int64_t) * term0.size(), cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaMemcpyAsync(S.d_blocks, S.blocks.data(), sizeof(SoBlock) * S.blocks.size(), cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaMemcpyAsync(S.d_leaf_row0, op.plan.leaf_start.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaMemcpyAsync(S.d_leaf_m, lm.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaMemcpyAsync(S.d_rec_ptr, rec_ptr.data(), sizeof(int) * (nl + 1), cudaMemcpyHostToDevice, s));
    if (!recs.empty()) RT_CUDA_TRY(cudaMemcpyAsync(S.d_recs, recs.data(), sizeof(SoRec) * recs.size(), cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaMemcpyAsync(S.d_fscale, fs.data(), sizeof(double) * S.F, cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    RT_CUDA_TRY(cudaGetLastError());
    S.apply_bytes = 4 * S.stored + 4 * (int64_t)L + 4 * (int64_t)S.F * S.N;
    return RT_OK;
}

int source_op_apply(SourceOp& S, const float* Q0, float* out, cudaStream_t s, std::string& err)
{
    Operator& op = *S.op;
    so_gather_q<<<std::max(1, std::min((S.L + 255) / 256, 152)), 256, 0, s>>>(Q0, S.d_qperm, S.L, S.q);
    if (!S.far.empty()) {
        const int64_t nt = (int64_t)S.rank_sum;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nt + 7) / 8, 152 * 16));
        so_phase1<<<grid, 256, 0, s>>>(S.d_far, (int)S.far.size(), S.d_blocks, S.store, S.q, S.w, S.d_term0);
    }
    const int nl = (int)op.plan.leaf_start.size();
    so_phase2<<<nl, 128, sizeof(float) * 64 * std::max(1, S.G), s>>>(S.d_leaf_row0, S.d_leaf_m, S.d_rec_ptr, S.d_recs,
                                                                       S.store, S.w, S.q, S.G, S.F, op.d_fq_group,
                                                                       S.d_fscale, op.d_perm, S.N, out);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

}  // namespace rt

// ---- C ABI ------------------------------------------------------------------
struct rt_source_op {
    rt::SourceOp s;
};

extern "C" {

int rt_build_source_operator(rt_operator* op, void* stream, rt_source_op** out)
{
    if (!op || !out) {
        rt::set_last_error("null argument");
        return RT_EINVAL;
    }
    *out = nullptr;
    if (op->op.G > 16) {
        rt::set_last_error("the surface-to-volume operator supports at most 16 kappa groups");
        return RT_EINVAL;
    }
    rt_source_op* h = new (std::nothrow) rt_source_op;
    if (!h) {
        rt::set_last_error("host allocation failed");
        return RT_ENOMEM;
    }
    std::string err;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = rt::source_op_build(h->s, op->op, op->op.aca_eps, s, err);
    if (rc) {
        rt::source_op_release(h->s, s);
        cudaStreamSynchronize(s);
        delete h;
        rt::set_last_error(err);
        return rc;
    }
    *out = h;
    return RT_OK;
}

int rt_source_operator_info(const rt_source_op* h, rt_source_info* info, int32_t* vertices)
{
    if (!h || !info) {
        rt::set_last_error("null argument");
        return RT_EINVAL;
    }
    const rt::SourceOp& S = h->s;
    info->N = S.N;
    info->L = S.L;
    info->G = S.G;
    info->n_far = (int64_t)S.far.size();
    info->n_dense = S.n_dense;
    info->n_blocks = (int64_t)S.blocks.size();
    info->rank_sum = S.rank_sum;
    info->rank_max = S.rank_max;
    info->stored_entries = S.stored;
    info->compression = 1.0 - (double)S.stored / ((double)S.N * S.L * std::max(1, S.G));
    info->apply_bytes = S.apply_bytes;
    info->device_bytes = S.device_bytes;
    info->ms_eval = S.ms_eval;
    info->ms_aca = S.ms_aca;
    if (vertices)
        for (int l = 0; l < S.L; ++l) vertices[l] = S.sv_caller[l];
    return RT_OK;
}

int rt_apply_source(rt_source_op* h, const float* Q0, float* out, void* stream)
{
    if (!h || !Q0 || !out) {
        rt::set_last_error("null argument");
        return RT_EINVAL;
    }
    std::string err;
    int rc = rt::source_op_apply(h->s, Q0, out, (cudaStream_t)stream, err);
    if (rc) rt::set_last_error(err.empty() ? "kernel launch failed" : err);
    return rc;
}

void rt_source_free(rt_source_op* h)
{
    if (!h) return;
    rt::source_op_release(h->s, nullptr);
    cudaDeviceSynchronize();
    delete h;
}

}  // extern "C"
