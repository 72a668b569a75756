// rt_hmatvec.cu -- application of the operator to the multi-frequency iterate
// (Y_nu = Gbar_{g(nu)} X_nu), the per-iteration cost of the fixed point
// ("the fixed point iterations involve only matrix vector products", abstract).
//
// H-matrix apply in two phases over flat, precomputed work lists:
//   phase 1: w_{b,f} = V_g^T x_f[cols(b)] for every far block b and frequency f.
//            The rank rows of all blocks form one list sorted by row length;
//            a sub-warp (8, 16 or 32 lanes, matched to the row length) reads a
//            row with 16-byte loads and reduces it with shuffles.
//   phase 2: for every leaf row cluster l and frequency f (row ownership, no
//            atomics): y_f[rows(l)] = sum_far U_g[rows(l), :] w_{b,f}
//                                   + sum_dense A_g[rows(l), :] x_f[cols(b)].
//            Each (leaf, block) pair is one contiguous chunk [count][m8] in
//            HBM; a thread owns 4 consecutive rows and a slice of the count.
// Both phases run as streamed persistent kernels (rt_hmv_stream.cuh): the
// host cuts the operator into 16 KB stage records here, and a producer warp
// per CTA bulk-copies them into a shared-memory ring.  Phase-1 rows longer
// than one stage, and the refinement sweeps that also read the low parts of a
// split far field, use the register-streaming kernels of rt_hmv_dev.cuh.
// Far factors are stored transposed (V^T [r][n8]; U^T per leaf chunk
// [r][m8]) and dense blocks column-major per leaf chunk (A^T [n][m8]), padded
// to multiples of 8 elements with zeros so every chunk row is 16-byte aligned.
#include <algorithm>
#include <atomic>
#include <climits>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rt_internal.h"


#include "rt_hmv_dev.cuh"
#include "rt_hmv_stream.cuh"

namespace rt {

// dense mode: y_f[i] = sum_j A_g[i][j] x_f[j], A row-major [G][N][N]; warp per (i, f)
template <class V>
__global__ void __launch_bounds__(256) dense_apply(const V* __restrict__ A, const V* __restrict__ X,
                                                   V* __restrict__ Y, int N, int F, const int* __restrict__ fgroup,
                                                   int64_t ldx, int64_t ldy)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < (int64_t)N * F; w += nw) {
        const int f = (int)(w / N), i = (int)(w % N);
        const V* __restrict__ a = A + ((int64_t)fgroup[f] * N + i) * N;
        const V* __restrict__ x = X + (int64_t)f * ldx;
        V s0 = 0, s1 = 0;
        int j = lane;
        for (; j + 32 < N; j += 64) {
            s0 += a[j] * x[j];
            s1 += a[j + 32] * x[j + 32];
        }
        for (; j < N; j += 32) s0 += a[j] * x[j];
        V s = s0 + s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) Y[(int64_t)f * ldy + i] = s;
    }
}

// permutation between caller order and tree order, rows of length N; with a
// scale, row r of the output is multiplied by scale[r]
template <class V>
__global__ void permute_kernel(const V* __restrict__ in, V* __restrict__ out, const int* __restrict__ perm, int N,
                               int rows, int to_tree, const double* __restrict__ scale)
{
    const int64_t total = (int64_t)N * rows;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / N;
        const int t = (int)(e % N);
        const V v = to_tree ? in[r * N + perm[t]] : in[e];
        const V o = scale ? (V)((double)v * scale[r]) : v;
        if (to_tree) out[e] = o;
        else out[r * N + perm[t]] = o;
    }
}

int permute_vectors(Operator& op, const void* in, void* out, int to_tree, int is64, int rows, cudaStream_t s,
                    const double* scale)
{
    const int64_t total = (int64_t)op.N * rows;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 32));
    if (is64)
        permute_kernel<double><<<grid, 256, 0, s>>>((const double*)in, (double*)out, op.d_perm, op.N, rows, to_tree,
                                                    scale);
    else
        permute_kernel<float><<<grid, 256, 0, s>>>((const float*)in, (float*)out, op.d_perm, op.N, rows, to_tree,
                                                   scale);
    return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ECUDA;
}

// Y_f *= scale[f] in place (the c_f / c_g factor of binned channels, dense operators)
template <class V>
__global__ void scale_rows_kernel(V* __restrict__ Y, int N, int rows, const double* __restrict__ scale)
{
    const int64_t total = (int64_t)N * rows;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        Y[e] = (V)((double)Y[e] * scale[e / N]);
}

int scale_rows(Operator& op, void* Y, cudaStream_t s)
{
    const int64_t total = (int64_t)op.N * op.F;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 32));
    if (op.vec64) scale_rows_kernel<double><<<grid, 256, 0, s>>>((double*)Y, op.N, op.F, op.d_fscale);
    else scale_rows_kernel<float><<<grid, 256, 0, s>>>((float*)Y, op.N, op.F, op.d_fscale);
    return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ECUDA;
}

// caller vectors with leading dimensions <-> tree-order rows [F][N]: rows
// r < cnt are copied (gathered with perm, or scattered back), rows cnt..F-1 of
// a tree-order destination are zeroed
template <class V>
__global__ void permute_ld_kernel(const V* __restrict__ in, int64_t ldin, V* __restrict__ out, int64_t ldout,
                                  const int* __restrict__ perm, int N, int rows, int cnt, int to_tree)
{
    const int64_t total = (int64_t)N * (to_tree ? rows : cnt);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / N;
        const int t = (int)(e % N);
        if (to_tree) out[e] = r < cnt ? in[r * ldin + perm[t]] : V(0);
        else out[r * ldout + perm[t]] = in[r * N + t];
    }
}

// Stage records of the streamed phases.
//  phase 1: far blocks ordered by (padded row length, first column), so the
//    pieces of a stage mostly share one x segment; whole V^T rows of one
//    length fill a stage up to kStageBytes, kMaxPieces pieces and kVecFloats
//    gathered x values.
//  phase 2: per leaf, its far chunks, then its dense chunks, as whole k-rows;
//    a stage holds one kind only, so it is one [K][m8] array.
static bool hs_long_row(int n, int esz_far)
{
    return round8(n) * esz_far > hs::kStageBytes || round8(n) > hs::kVecFloats;
}

static int hs_prepare(Operator& op, const std::vector<int64_t>& w_base, const std::vector<std::vector<P2Seg>>& per_leaf,
                      const std::vector<P2Leaf>& leaves, int esz_far, std::string& err)
{
    op.hs_enabled = 0;
    if (op.w_len > INT_MAX || (int64_t)op.N > INT_MAX / 2) return RT_OK;   // piece fields are 32-bit
    int rc;
    std::vector<HsLoad> l1, l2;
    HsLoad cur{};
    int used = 0, vtot = 0;
    auto flush = [&](std::vector<HsLoad>& out, bool keep_empty) {
        if (cur.np > 0 || keep_empty) {
            cur.bytes = used;
            out.push_back(cur);
        }
        cur = HsLoad{};
        used = 0;
        vtot = 0;
    };
    // ---- phase 1 ----
    std::vector<int> border;
    for (int b = 0; b < op.n_far; ++b)
        if (!hs_long_row(op.far_blocks[b].n, esz_far)) border.push_back(b);
    std::stable_sort(border.begin(), border.end(), [&](int a, int b) {
        const int na = round8(op.far_blocks[a].n), nb = round8(op.far_blocks[b].n);
        return na != nb ? na < nb : op.far_blocks[a].col0 < op.far_blocks[b].col0;
    });
    for (int b : border) {
        const FarBlock& fb = op.far_blocks[b];
        const int r = op.rank[b], n8 = round8(fb.n);
        const int rowb = n8 * esz_far;
        for (int k = 0; k < r;) {
            // the stage's x segment for this block's columns, if already gathered
            int vo = -1;
            for (int q = 0; q < cur.np; ++q)
                if (cur.p[q].vlen > 0 && cur.p[q].vsrc == fb.col0 && cur.p[q].valid == fb.n) vo = cur.p[q].vo;
            const int fit = (hs::kStageBytes - used) / rowb;
            if (fit == 0 || cur.np == hs::kMaxPieces || (vo < 0 && vtot + n8 > hs::kVecFloats) ||
                (cur.np > 0 && cur.p[0].n8 != n8)) {   // a stage's rows have one length
                flush(l1, false);
                continue;
            }
            const int take = std::min(fit, r - k);
            HsPiece& pc = cur.p[cur.np++];
            pc = HsPiece{};
            pc.a = op.far_v_off[b] + (int64_t)k * n8;
            pc.gstride = (int64_t)r * n8;
            pc.vsrc = fb.col0;
            pc.soff = used;
            pc.bytes = take * rowb;
            pc.rows = take;
            pc.n8 = n8;
            if (vo >= 0) {
                pc.vo = vo;
                pc.vlen = 0;
            } else {
                pc.vo = vtot;
                pc.vlen = n8;
                vtot += n8;
            }
            pc.valid = fb.n;
            pc.r = r;
            pc.wv = (int)(w_base[b] + k);
            pc.kind = 0;
            used += pc.bytes;
            k += take;
        }
    }
    flush(l1, false);
    // ---- phase 2 ----
    const int nl = (int)leaves.size();
    std::vector<int> leaf0(nl + 1);
    std::vector<int64_t> leaf_bytes(nl, 0);
    for (int l = 0; l < nl; ++l) {
        leaf0[l] = (int)l2.size();
        const int m8 = leaves[l].m8;
        for (int kind = 0; kind < 2; ++kind) {
            for (const P2Seg& sg : per_leaf[l]) {
                if (sg.kind != kind) continue;
                const int rowb = m8 * (kind ? 4 : esz_far);
                for (int k = 0; k < sg.count;) {
                    const int fit = std::min((hs::kStageBytes - used) / rowb, hs::kVecFloats - cur.K);
                    if (fit <= 0 || cur.np == hs::kMaxPieces) {
                        flush(l2, false);
                        continue;
                    }
                    const int take = std::min(fit, sg.count - k);
                    HsPiece& pc = cur.p[cur.np++];
                    pc = HsPiece{};
                    pc.a = sg.a + (int64_t)k * m8;
                    pc.gstride = sg.gstride;
                    pc.vsrc = sg.vbase + k;
                    pc.soff = used;
                    pc.bytes = take * rowb;
                    pc.rows = take;
                    pc.n8 = m8;
                    pc.vo = cur.K;
                    pc.vlen = take;
                    pc.valid = take;
                    pc.r = kind ? 0 : sg.count;
                    pc.kind = kind;
                    cur.kind = kind;
                    cur.K += take;
                    used += pc.bytes;
                    leaf_bytes[l] += pc.bytes;
                    k += take;
                }
            }
            flush(l2, false);   // a stage holds one kind
        }
        if ((int)l2.size() == leaf0[l]) flush(l2, true);   // every leaf has a record, so its rows are written
    }
    leaf0[nl] = (int)l2.size();
    std::vector<int> order(nl);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return leaf_bytes[a] > leaf_bytes[b]; });
    std::vector<int2> items;
    items.reserve((size_t)nl * op.F);
    for (int l : order)
        for (int f = 0; f < op.F; ++f) items.push_back(make_int2(l, f));
    HsLoad *d1 = nullptr, *d2 = nullptr;
    int* d0 = nullptr;
    int2* di = nullptr;
    if (!l1.empty() && ((rc = dev_alloc(op, &d1, l1.size(), err)) || (rc = upload_async(op, d1, l1.data(), l1.size(), err))))
        return rc;
    if ((rc = dev_alloc(op, &d2, l2.size(), err)) || (rc = upload_async(op, d2, l2.data(), l2.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d0, leaf0.size(), err)) || (rc = upload_async(op, d0, leaf0.data(), leaf0.size(), err)))
        return rc;
    if ((rc = dev_alloc(op, &di, items.size(), err)) || (rc = upload_async(op, di, items.data(), items.size(), err)))
        return rc;
    op.d_hs1 = d1;
    op.n_hs1 = (int)l1.size();
    op.d_hs2 = d2;
    op.n_hs2 = (int)l2.size();
    op.d_hs2_leaf0 = d0;
    op.d_hs2_items = di;
    op.n_hs2_items = (int)items.size();
    const int smem = (int)hs_smem_bytes();
    RT_CUDA_TRY(cudaFuncSetAttribute(hmv_s1<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(hmv_s1<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(hmv_s1<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(hmv_s2<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(hmv_s2<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(hmv_s2<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    op.hs_enabled = 1;
    return RT_OK;
}

int hmatvec_prepare(Operator& op, std::string& err)
{
    int rc;
    int* d_fg = nullptr;
    if ((rc = dev_alloc(op, &d_fg, op.F, err))) return rc;
    if ((rc = upload_async(op, d_fg, op.fgroup.data(), op.F, err))) return rc;
    op.d_fq_group = d_fg;
    if (op.binned) {
        if ((rc = dev_alloc(op, &op.d_fscale, op.F, err))) return rc;
        if ((rc = upload_async(op, op.d_fscale, op.fscale.data(), op.F, err))) return rc;
    }
    {   // rt_apply_group: every channel of a chunk mapped to one group
        std::vector<int> gm((size_t)op.G * op.F);
        for (int g = 0; g < op.G; ++g)
            for (int f = 0; f < op.F; ++f) gm[(size_t)g * op.F + f] = g;
        if ((rc = dev_alloc(op, &op.d_gmap, gm.size(), err))) return rc;
        if ((rc = upload_async(op, op.d_gmap, gm.data(), gm.size(), err))) return rc;
    }
    // frequency table for the solver: nu, w c (1-a), a, group
    {
        std::vector<double> fq((size_t)op.F * 4);
        for (int f = 0; f < op.F; ++f) {
            fq[4 * f + 0] = op.nu[f];
            fq[4 * f + 1] = op.w[f] * op.c[f] * (1.0 - op.albedo[f]);
            fq[4 * f + 2] = op.albedo[f];
            fq[4 * f + 3] = (double)op.fgroup[f];
        }
        if ((rc = dev_alloc(op, &op.d_fq, fq.size(), err))) return rc;
        if ((rc = upload_async(op, op.d_fq, fq.data(), fq.size(), err))) return rc;
    }
    const size_t esz = op.vec64 ? 8 : 4;
    const int64_t N = op.N, F = op.F;
    if (op.mode == RT_MODE_DENSE) return RT_OK;
    for (int l = 0; l < (int)op.plan.leaf_size.size(); ++l)
        if (op.plan.leaf_size[l] > 1024) {
            err = "leaf clusters larger than 1024 rows are not supported";
            return RT_EINVAL;
        }
    // ---- phase-1 rows and items ----------------------------------------------
    std::vector<P1Row> rows;
    std::vector<int64_t> w_base(op.n_far);
    int64_t wl = 0;
    for (int b = 0; b < op.n_far; ++b) {
        const FarBlock& fb = op.far_blocks[b];
        const int r = op.rank[b];
        w_base[b] = wl;
        wl += F * r;
        for (int k = 0; k < r; ++k) {
            P1Row rw{};
            rw.v = op.far_v_off[b] + (int64_t)k * round8(fb.n);
            rw.gstride = (int64_t)r * round8(fb.n);
            rw.w = w_base[b] + k;
            rw.n = fb.n;
            rw.col0 = fb.col0;
            rw.r = r;
            rows.push_back(rw);
        }
    }
    std::stable_sort(rows.begin(), rows.end(), [](const P1Row& a, const P1Row& b) { return a.n > b.n; });
    std::vector<P1Item> items;
    const int vw = op.far_prec == RT_PREC_F32 ? 4 : 8;
    const int esz_far = op.far_prec == RT_PREC_F32 ? 4 : 2;
    for (size_t i = 0; i < rows.size();) {
        const int n = rows[i].n;
        int sw = 32;
        if ((n + vw - 1) / vw <= 8) sw = 8;
        else if ((n + vw - 1) / vw <= 16) sw = 16;
        // about 48 KB of operator data per CTA, at most 512 rows
        int per = (int)std::max<int64_t>(1, std::min<int64_t>(512, (48 << 10) / std::max(1, n * esz_far)));
        size_t j = i;
        while (j < rows.size() && (int)(j - i) < per && rows[j].n == n) ++j;
        items.push_back({(int)i, (int)j, sw, 0});
        i = j;
    }
    // ---- phase-2 leaves and segments -----------------------------------------
    const int nl = (int)op.plan.leaf_start.size();
    std::vector<std::vector<P2Seg>> per_leaf(nl);
    for (int b = 0; b < op.n_far; ++b) {
        const int r = op.rank[b];
        for (int c = op.far_chunk_ptr[b]; c < op.far_chunk_ptr[b + 1]; ++c) {
            const Chunk& ch = op.far_chunks[c];
            P2Seg sg{};
            sg.kind = 0;
            sg.a = op.far_u_off[b] + ch.off;
            sg.gstride = (int64_t)r * ch.m8;
            sg.count = r;
            sg.vbase = w_base[b];
            per_leaf[ch.leaf].push_back(sg);
        }
    }
    for (int b = 0; b < op.n_near; ++b) {
        const FarBlock& fb = op.dense_blocks[b];
        for (int c = op.dense_chunk_ptr[b]; c < op.dense_chunk_ptr[b + 1]; ++c) {
            const Chunk& ch = op.dense_chunks[c];
            P2Seg sg{};
            sg.kind = 1;
            sg.a = op.dense_off[b] + ch.off;
            sg.gstride = (int64_t)fb.n * ch.m8;
            sg.count = fb.n;
            sg.vbase = fb.col0;
            per_leaf[ch.leaf].push_back(sg);
        }
    }
    std::vector<P2Leaf> leaves(nl);
    std::vector<P2Seg> segs;
    for (int l = 0; l < nl; ++l) {
        leaves[l].row0 = op.plan.leaf_start[l];
        leaves[l].m = op.plan.leaf_size[l];
        leaves[l].m8 = round8(op.plan.leaf_size[l]);
        leaves[l].seg0 = (int)segs.size();
        leaves[l].nseg = (int)per_leaf[l].size();
        segs.insert(segs.end(), per_leaf[l].begin(), per_leaf[l].end());
    }
    P1Item* d_it = nullptr;
    P1Row* d_rows = nullptr;
    P2Leaf* d_l = nullptr;
    P2Seg* d_s = nullptr;
    if ((rc = dev_alloc(op, &d_it, items.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_rows, rows.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_l, leaves.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_s, segs.size(), err))) return rc;
    if ((rc = upload_async(op, d_it, items.data(), items.size(), err))) return rc;
    if ((rc = upload_async(op, d_rows, rows.data(), rows.size(), err))) return rc;
    if ((rc = upload_async(op, d_l, leaves.data(), leaves.size(), err))) return rc;
    if ((rc = upload_async(op, d_s, segs.data(), segs.size(), err))) return rc;
    op.d_p1_items = d_it;
    op.d_p1_rows = d_rows;
    op.h_p1_rows.assign(reinterpret_cast<const char*>(rows.data()),
                        reinterpret_cast<const char*>(rows.data()) + sizeof(P1Row) * rows.size());
    op.n_p1 = (int)items.size();
    op.n_p1_long = 0;
    while (op.n_p1_long < op.n_p1 && hs_long_row(rows[items[op.n_p1_long].row0].n, esz_far))
        ++op.n_p1_long;
    op.d_p2_leaf = d_l;
    op.n_p2 = nl;
    op.d_p2_segs = d_s;
    op.n_p2_segs = (int)segs.size();
    op.w_len = wl;
    if ((rc = dev_alloc(op, &op.d_w, (size_t)std::max<int64_t>(wl, 1), err))) return rc;
    if ((rc = dev_alloc(op, &op.apply_err, 1, err))) return rc;
    RT_CUDA_TRY(cudaMemsetAsync(op.apply_err, 0, sizeof(int), op.stream));
    if ((rc = hs_prepare(op, w_base, per_leaf, leaves, esz_far, err))) return rc;
    // algorithmic bytes of one apply: operator data once per frequency, X read, Y written
    int64_t far_e = 0, near_e = 0;
    for (int b = 0; b < op.n_far; ++b) far_e += (int64_t)op.rank[b] * (op.far_blocks[b].m + op.far_blocks[b].n);
    for (int b = 0; b < op.n_near; ++b) near_e += (int64_t)op.dense_blocks[b].m * op.dense_blocks[b].n;
    op.info.apply_bytes = F * (far_e * esz_far + near_e * 4) + 2 * F * N * (int64_t)esz;
    op.info.apply_flops = 2 * F * (far_e + near_e);
    if ((rc = tc_prepare(op, err))) return rc;
    op.info.apply_tensor_cores = op.tc_enabled;
    if (op.tc_enabled)   // one operator serves all F right-hand sides: its data is read once per apply
        op.info.apply_bytes = far_e * esz_far + near_e * 4 + 2 * F * N * (int64_t)esz;
    return RT_OK;
}

// the two H-matvec phases on tree-order vectors with an explicit w buffer
static int launch_hmv(Operator& op, const float* x, float* w, float* y, cudaStream_t s, std::string& err)
{
    const int N = op.N, F = op.F;
    const bool lo = op.use_lo && op.d_far_lo;   // refinement sweep: high + low parts
    const P1Item* it = (const P1Item*)op.d_p1_items;
    const P1Row* rw = (const P1Row*)op.d_p1_rows;
    const P2Leaf* lv = (const P2Leaf*)op.d_p2_leaf;
    const P2Seg* sg = (const P2Seg*)op.d_p2_segs;
    dim3 g1(op.n_p1, F), g2(op.n_p2, F);
    if (op.hs_enabled && !lo) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = hs::kCtasPerSm;
        const int smem = (int)hs_smem_bytes();
        const HsLoad* l1 = (const HsLoad*)op.d_hs1;
        const HsLoad* l2 = (const HsLoad*)op.d_hs2;
        const int2* itm = (const int2*)op.d_hs2_items;
        const int gs1 = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)op.n_hs1 * F, (int64_t)per_sm * sms));
        const int gs2 = std::max(1, std::min(op.n_hs2_items, per_sm * sms));
#define RT_HMS(T)                                                                                                 \
    do {                                                                                                          \
        const T* fp = (const T*)op.d_far;                                                                         \
        if (op.n_p1_long > 0)                                                                                     \
            hmv_phase1<T, false><<<dim3(op.n_p1_long, F), 256, 0, s>>>(it, rw, fp, nullptr, x, w, N, op.d_fq_group); \
        if (op.n_hs1 > 0)                                                                                         \
            hmv_s1<T><<<gs1, hs::kThreads, smem, s>>>(l1, op.n_hs1, fp, x, w, N, F, op.d_fq_group, op.apply_err);  \
        hmv_s2<T><<<gs2, hs::kThreads, smem, s>>>(l2, op.d_hs2_leaf0, itm, op.n_hs2_items, lv, fp, op.d_near, x, w, \
                                                 y, N, op.d_fq_group, op.apply_err);                              \
    } while (0)
        if (op.far_prec == RT_PREC_F32) RT_HMS(float);
        else if (op.far_prec == RT_PREC_BF16) RT_HMS(__nv_bfloat16);
        else RT_HMS(__half);
#undef RT_HMS
        RT_CUDA_TRY(cudaGetLastError());
        return RT_OK;
    }
#define RT_HMV(T, LO)                                                                                             \
    do {                                                                                                          \
        const T* fp = (const T*)op.d_far;                                                                         \
        const T* fl = (const T*)op.d_far_lo;                                                                      \
        if (op.n_p1 > 0) hmv_phase1<T, LO><<<g1, 256, 0, s>>>(it, rw, fp, fl, x, w, N, op.d_fq_group);            \
        hmv_phase2<T, LO><<<g2, 256, 0, s>>>(lv, sg, fp, fl, op.d_near, x, w, y, N, op.d_fq_group);               \
    } while (0)
    if (op.far_prec == RT_PREC_F32) RT_HMV(float, false);
    else if (op.far_prec == RT_PREC_BF16) {
        if (lo) RT_HMV(__nv_bfloat16, true);
        else RT_HMV(__nv_bfloat16, false);
    } else {
        if (lo) RT_HMV(__half, true);
        else RT_HMV(__half, false);
    }
#undef RT_HMV
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

int apply_check_error(Operator& op, cudaStream_t s, std::string& err)
{
    int rc = tc_check_error(op, s, err);
    if (rc || !op.apply_err) return rc;
    int h = 0;
    RT_CUDA_TRY(cudaMemcpyAsync(&h, op.apply_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
        cudaMemsetAsync(op.apply_err, 0, sizeof(int), s);
        err = "streamed H-matvec: an mbarrier wait timed out";
        return RT_ETIMEOUT;
    }
    return RT_OK;
}

static int launch_dense(Operator& op, const void* X, void* Y, cudaStream_t s, std::string& err,
                        const int* fgroup = nullptr, int rows = 0, int64_t ldx = 0, int64_t ldy = 0)
{
    const int N = op.N, F = rows > 0 ? rows : op.F;
    const int64_t warps = (int64_t)N * F;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 152 * 16));
    if (!fgroup) fgroup = op.d_fq_group;
    if (ldx <= 0) ldx = N;
    if (ldy <= 0) ldy = N;
    if (op.vec64)
        dense_apply<double><<<grid, 256, 0, s>>>((const double*)op.d_dense, (const double*)X, (double*)Y, N, F,
                                                 fgroup, ldx, ldy);
    else
        dense_apply<float><<<grid, 256, 0, s>>>((const float*)op.d_dense, (const float*)X, (float*)Y, N, F,
                                                fgroup, ldx, ldy);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

int apply_tree(Operator& op, const void* X, void* Y, cudaStream_t s, std::string& err)
{
    if (op.mode == RT_MODE_DENSE) return launch_dense(op, X, Y, s, err);
    if (tc_serves(op)) return tc_apply(op, (const float*)X, (float*)Y, s, err);
    return launch_hmv(op, (const float*)X, op.d_w, (float*)Y, s, err);
}

// Y_j = G_group X_j for nrhs caller vectors with leading dimensions, in
// chunks of F right-hand sides through the operator's own kernels and scratch
int apply_group(Operator& op, int group, const void* X, int64_t ldx, int nrhs, void* Y, int64_t ldy, cudaStream_t s,
                std::string& err)
{
    const int N = op.N, F = op.F;
    const int* gm = op.d_gmap + (int64_t)group * F;
    for (int j0 = 0; j0 < nrhs; j0 += F) {
        const int cnt = std::min(F, nrhs - j0);
        int rc;
        if (op.mode == RT_MODE_DENSE) {
            if (op.vec64)
                rc = launch_dense(op, (const double*)X + j0 * ldx, (double*)Y + j0 * ldy, s, err, gm, cnt, ldx, ldy);
            else
                rc = launch_dense(op, (const float*)X + j0 * ldx, (float*)Y + j0 * ldy, s, err, gm, cnt, ldx, ldy);
            if (rc) return rc;
            continue;
        }
        const int64_t tot_in = (int64_t)N * F;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tot_in + 255) / 256, 152 * 32));
        permute_ld_kernel<float><<<grid, 256, 0, s>>>((const float*)X + j0 * ldx, ldx, op.d_xt, N, op.d_perm, N, F,
                                                      cnt, 1);
        RT_CUDA_TRY(cudaGetLastError());
        if (tc_serves(op)) {
            // one group: the tcgen05 pair applies G_0 to all F rows
            if ((rc = tc_apply(op, op.d_xt, op.d_yt, s, err))) return rc;
        } else {
            const int* keep = op.d_fq_group;
            op.d_fq_group = const_cast<int*>(gm);
            rc = launch_hmv(op, op.d_xt, op.d_w, op.d_yt, s, err);
            op.d_fq_group = const_cast<int*>(keep);
            if (rc) return rc;
        }
        permute_ld_kernel<float><<<grid, 256, 0, s>>>(op.d_yt, N, (float*)Y + j0 * ldy, ldy, op.d_perm, N, F, cnt, 0);
        RT_CUDA_TRY(cudaGetLastError());
    }
    return RT_OK;
}

// ---------------------------------------------------------------------------
// Apply without allocation.
//
// Same kernels and the same arithmetic as apply_tree + the two permutations
// (the tcgen05 pair when rt_apply takes it, otherwise the CUDA-core phases),
// but the scratch (X and Y in tree order and, for the CUDA-core phases, the
// phase-1 w buffer) lives in one file-scope device array instead of buffers
// owned by the operator.  The tcgen05 pair's W panels and split X belong to
// the operator and were allocated when it was built.  The array is
// kNoAllocBytes large, is held by every GPU that loads the library until the
// process exits, and is shared by every call: it keeps the previous call's
// contents (every region used is fully overwritten before it is read, so
// nothing needs clearing), and two calls that overlap on the GPU race on it.
// ---------------------------------------------------------------------------
static constexpr size_t kNoAllocBytes = (size_t)8 << 20;
static constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
// device address of the array per device, set on first use; two threads making
// their first call on one device at once both look it up and store the same value
static std::atomic<void*> g_noalloc_addr[kNoAllocMaxDevices];

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t apply_noalloc_limit() { return kNoAllocBytes; }

int apply_noalloc(Operator& op, const void* X, void* Y, cudaStream_t s, std::string& err)
{
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != op.device) {
        err = "rt_apply_noalloc: the current device is not the operator's device";
        return RT_EINVAL;
    }
    const int N = op.N, F = op.F;
    // the dense apply reads X and writes Y directly: no scratch at all
    if (op.mode == RT_MODE_DENSE) {
        int rc = launch_dense(op, X, Y, s, err);
        if (!rc && op.binned) rc = scale_rows(op, Y, s);
        return rc;
    }
    const bool tc = tc_serves(op);   // the path apply_tree takes
    const size_t vbytes = round256((size_t)F * N * sizeof(float));
    const size_t wbytes = tc ? 0 : round256((size_t)std::max<int64_t>(op.w_len, 1) * sizeof(float));
    const size_t need = 2 * vbytes + wbytes;
    if (need > kNoAllocBytes) {
        err = "rt_apply_noalloc: operator needs " + std::to_string(need) + " bytes of scratch, limit is " +
              std::to_string(kNoAllocBytes) + " bytes (use rt_apply)";
        return RT_EINVAL;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        err = "rt_apply_noalloc: device index out of range";
        return RT_EINVAL;
    }
    void* addr = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!addr) {
        // one-time set-up on this device (the device is current): the host-side
        // name of a __device__ array is not a device address; ask the runtime for it
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr) {
            err = std::string("rt_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return RT_ECUDA;
        }
        g_noalloc_addr[dev].store(addr, std::memory_order_release);
    }
    unsigned char* base = (unsigned char*)addr;
    float* xt = (float*)base;
    float* yt = (float*)(base + vbytes);
    float* w = (float*)(base + 2 * vbytes);
    int rc = permute_vectors(op, X, xt, 1, 0, F, s);
    if (rc) {
        err = "rt_apply_noalloc: permute launch failed";
        return rc;
    }
    if (tc) {
        if ((rc = tc_apply(op, xt, yt, s, err))) return rc;
    } else if ((rc = launch_hmv(op, xt, w, yt, s, err))) {
        return rc;
    }
    rc = permute_vectors(op, yt, Y, 0, 0, F, s, op.binned ? op.d_fscale : nullptr);
    if (rc) {
        err = "rt_apply_noalloc: permute launch failed";
        return rc;
    }
    return RT_OK;
}

}  // namespace rt
