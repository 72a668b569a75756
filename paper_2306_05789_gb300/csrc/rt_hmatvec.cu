// rt_hmatvec.cu -- application of the operator to the multi-frequency iterate
// (Y_nu = Gbar_{g(nu)} X_nu), the per-iteration cost of the fixed point
// ("the fixed point iterations involve only matrix vector products", abstract).
//
// H-matrix apply in two phases, both over flat, precomputed work lists:
//   phase 1: for every far block b and frequency f:  w_{b,f} = V_g^T x_f[cols(b)]
//            (one warp per rank row k: a coalesced dot product of length n)
//   phase 2: for every leaf row cluster l and frequency f (row ownership, no
//            atomics): y_f[rows(l)] = sum_{far b over l} U_g[rows(l), :] w_{b,f}
//                                    + sum_{dense b in l} A_g[rows(l), :] x_f[cols(b)]
// Far factors are stored transposed (V^T [r][n], U^T [r][m]) and dense blocks
// column-major (A^T [n][m]) so that consecutive threads read consecutive rows.
#include <algorithm>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rt_internal.h"

namespace rt {

struct P1Item {
    int64_t v_off;   // element offset of the block's V^T [G][r][n]
    int64_t w_base;  // offset of the block's w [F][r]
    int n, col0, r, k0, nk, pad;
};

struct P2Leaf {
    int row0, m, seg0, nseg;
};

struct P2Seg {
    int64_t a_off;   // element offset of row (leaf start) of k = 0, group 0
    int64_t gstride; // elements between groups
    int64_t vbase;   // far: w_base of the block; dense: column offset col0
    int stride;      // elements between consecutive k (m of the block)
    int count;       // r (far) or n (dense)
    int kind;        // 0 far, 1 dense
    int pad;
};

template <class T>
__device__ __forceinline__ float ld_f(const T* p);
template <>
__device__ __forceinline__ float ld_f<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ld_f<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <>
__device__ __forceinline__ float ld_f<__half>(const __half* p) { return __half2float(*p); }

// phase 1: grid (items, F), 256 threads = 8 warps, warp per rank row
template <class T>
__global__ void __launch_bounds__(256) hmv_phase1(const P1Item* __restrict__ items, const T* __restrict__ far,
                                                  const float* __restrict__ X, float* __restrict__ W, int N,
                                                  const int* __restrict__ fgroup)
{
    const P1Item it = items[blockIdx.x];
    const int f = blockIdx.y;
    const int g = fgroup[f];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* __restrict__ x = X + (int64_t)f * N + it.col0;
    for (int k = it.k0 + warp; k < it.k0 + it.nk; k += 8) {
        const T* __restrict__ v = far + it.v_off + ((int64_t)g * it.r + k) * it.n;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int j = lane;
        for (; j + 96 < it.n; j += 128) {
            s0 += ld_f<T>(v + j) * __ldg(x + j);
            s1 += ld_f<T>(v + j + 32) * __ldg(x + j + 32);
            s2 += ld_f<T>(v + j + 64) * __ldg(x + j + 64);
            s3 += ld_f<T>(v + j + 96) * __ldg(x + j + 96);
        }
        for (; j < it.n; j += 32) s0 += ld_f<T>(v + j) * __ldg(x + j);
        float s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) W[it.w_base + (int64_t)f * it.r + k] = s;
    }
}

// phase 2: grid (leaves, F), 256 threads: row = t % 64, slice = t / 64
template <class T>
__global__ void __launch_bounds__(256) hmv_phase2(const P2Leaf* __restrict__ leaves, const P2Seg* __restrict__ segs,
                                                  const T* __restrict__ far, const float* __restrict__ nearp,
                                                  const float* __restrict__ X, const float* __restrict__ W,
                                                  float* __restrict__ Y, int N, const int* __restrict__ fgroup)
{
    __shared__ float red[4][64];
    const P2Leaf L = leaves[blockIdx.x];
    const int f = blockIdx.y;
    const int g = fgroup[f];
    const int t = threadIdx.x, rr = t & 63, slice = t >> 6;
    for (int rb = 0; rb < L.m; rb += 64) {
        const int row = rb + rr;
        const bool act = row < L.m;
        float a0 = 0.f, a1 = 0.f;
        for (int si = L.seg0; si < L.seg0 + L.nseg; ++si) {
            const P2Seg sg = segs[si];
            if (sg.kind == 0) {
                const T* __restrict__ a = far + sg.a_off + (int64_t)g * sg.gstride + row;
                const float* __restrict__ w = W + sg.vbase + (int64_t)f * sg.count;
                if (act) {
                    int k = slice;
                    for (; k + 4 < sg.count; k += 8) {
                        a0 += ld_f<T>(a + (int64_t)k * sg.stride) * __ldg(w + k);
                        a1 += ld_f<T>(a + (int64_t)(k + 4) * sg.stride) * __ldg(w + k + 4);
                    }
                    for (; k < sg.count; k += 4) a0 += ld_f<T>(a + (int64_t)k * sg.stride) * __ldg(w + k);
                }
            } else {
                const float* __restrict__ a = nearp + sg.a_off + (int64_t)g * sg.gstride + row;
                const float* __restrict__ x = X + (int64_t)f * N + sg.vbase;
                if (act) {
                    int k = slice;
                    for (; k + 4 < sg.count; k += 8) {
                        a0 += __ldg(a + (int64_t)k * sg.stride) * __ldg(x + k);
                        a1 += __ldg(a + (int64_t)(k + 4) * sg.stride) * __ldg(x + k + 4);
                    }
                    for (; k < sg.count; k += 4) a0 += __ldg(a + (int64_t)k * sg.stride) * __ldg(x + k);
                }
            }
        }
        red[slice][rr] = a0 + a1;
        __syncthreads();
        if (slice == 0 && act)
            Y[(int64_t)f * N + L.row0 + row] = (red[0][rr] + red[1][rr]) + (red[2][rr] + red[3][rr]);
        __syncthreads();
    }
}

// dense mode: y_f[i] = sum_j A_g[i][j] x_f[j], A row-major [G][N][N]; warp per (i, f)
template <class V>
__global__ void __launch_bounds__(256) dense_apply(const V* __restrict__ A, const V* __restrict__ X,
                                                   V* __restrict__ Y, int N, int F, const int* __restrict__ fgroup)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < (int64_t)N * F; w += nw) {
        const int f = (int)(w / N), i = (int)(w % N);
        const V* __restrict__ a = A + ((int64_t)fgroup[f] * N + i) * N;
        const V* __restrict__ x = X + (int64_t)f * N;
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
        if (lane == 0) Y[(int64_t)f * N + i] = s;
    }
}

// permutation between caller order and tree order, rows of length N
template <class V>
__global__ void permute_kernel(const V* __restrict__ in, V* __restrict__ out, const int* __restrict__ perm, int N,
                               int rows, int to_tree)
{
    const int64_t total = (int64_t)N * rows;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / N;
        const int t = (int)(e % N);
        if (to_tree) out[e] = in[r * N + perm[t]];
        else out[r * N + perm[t]] = in[e];
    }
}

int permute_vectors(Operator& op, const void* in, void* out, int to_tree, int is64, int rows, cudaStream_t s)
{
    const int64_t total = (int64_t)op.N * rows;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 32));
    if (is64)
        permute_kernel<double><<<grid, 256, 0, s>>>((const double*)in, (double*)out, op.d_perm, op.N, rows, to_tree);
    else
        permute_kernel<float><<<grid, 256, 0, s>>>((const float*)in, (float*)out, op.d_perm, op.N, rows, to_tree);
    return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ECUDA;
}

int hmatvec_prepare(Operator& op, std::string& err)
{
    int rc;
    int* d_fg = nullptr;
    if ((rc = dev_alloc(op, &d_fg, op.F, err))) return rc;
    RT_CUDA_TRY(cudaMemcpy(d_fg, op.fgroup.data(), sizeof(int) * op.F, cudaMemcpyHostToDevice));
    op.d_fq = nullptr;
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
        RT_CUDA_TRY(cudaMemcpy(op.d_fq, fq.data(), sizeof(double) * fq.size(), cudaMemcpyHostToDevice));
    }
    op.d_fq_group = d_fg;
    const size_t esz = op.vec64 ? 8 : 4;
    const int64_t N = op.N, F = op.F;
    if (op.mode == RT_MODE_DENSE) {
        return RT_OK;
    }
    // ---- phase-1 items -------------------------------------------------------
    std::vector<P1Item> p1;
    std::vector<int64_t> w_base(op.n_far);
    int64_t wl = 0;
    const int kchunk = 32;
    for (int b = 0; b < op.n_far; ++b) {
        const FarBlock& fb = op.far_blocks[b];
        const int r = op.rank[b];
        w_base[b] = wl;
        wl += F * r;
        for (int k0 = 0; k0 < r; k0 += kchunk) {
            P1Item it{};
            it.v_off = op.far_v_off[b];
            it.w_base = w_base[b];
            it.n = fb.n;
            it.col0 = fb.col0;
            it.r = r;
            it.k0 = k0;
            it.nk = std::min(kchunk, r - k0);
            p1.push_back(it);
        }
    }
    // longest first
    std::stable_sort(p1.begin(), p1.end(),
                     [](const P1Item& a, const P1Item& b) { return (int64_t)a.n * a.nk > (int64_t)b.n * b.nk; });
    // ---- phase-2 leaves and segments -----------------------------------------
    const int nl = (int)op.plan.leaf_start.size();
    std::vector<std::vector<P2Seg>> per_leaf(nl);
    auto leaf_of = [&](int row) {
        int lo = 0, hi = nl - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (op.plan.leaf_start[mid] <= row) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    for (int b = 0; b < op.n_far; ++b) {
        const FarBlock& fb = op.far_blocks[b];
        const int r = op.rank[b];
        for (int l = leaf_of(fb.row0); l < nl && op.plan.leaf_start[l] < fb.row0 + fb.m; ++l) {
            P2Seg sg{};
            sg.kind = 0;
            sg.a_off = op.far_u_off[b] + (op.plan.leaf_start[l] - fb.row0);
            sg.gstride = (int64_t)r * fb.m;
            sg.stride = fb.m;
            sg.count = r;
            sg.vbase = w_base[b];
            per_leaf[l].push_back(sg);
        }
    }
    for (int b = 0; b < op.n_near; ++b) {
        const FarBlock& fb = op.dense_blocks[b];
        for (int l = leaf_of(fb.row0); l < nl && op.plan.leaf_start[l] < fb.row0 + fb.m; ++l) {
            P2Seg sg{};
            sg.kind = 1;
            sg.a_off = op.dense_off[b] + (op.plan.leaf_start[l] - fb.row0);
            sg.gstride = (int64_t)fb.m * fb.n;
            sg.stride = fb.m;
            sg.count = fb.n;
            sg.vbase = fb.col0;
            per_leaf[l].push_back(sg);
        }
    }
    std::vector<P2Leaf> leaves(nl);
    std::vector<P2Seg> segs;
    for (int l = 0; l < nl; ++l) {
        leaves[l].row0 = op.plan.leaf_start[l];
        leaves[l].m = op.plan.leaf_size[l];
        leaves[l].seg0 = (int)segs.size();
        leaves[l].nseg = (int)per_leaf[l].size();
        segs.insert(segs.end(), per_leaf[l].begin(), per_leaf[l].end());
    }
    P1Item* d_p1 = nullptr;
    P2Leaf* d_l = nullptr;
    P2Seg* d_s = nullptr;
    if ((rc = dev_alloc(op, &d_p1, p1.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_l, leaves.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_s, segs.size(), err))) return rc;
    if (!p1.empty()) RT_CUDA_TRY(cudaMemcpy(d_p1, p1.data(), sizeof(P1Item) * p1.size(), cudaMemcpyHostToDevice));
    RT_CUDA_TRY(cudaMemcpy(d_l, leaves.data(), sizeof(P2Leaf) * leaves.size(), cudaMemcpyHostToDevice));
    if (!segs.empty()) RT_CUDA_TRY(cudaMemcpy(d_s, segs.data(), sizeof(P2Seg) * segs.size(), cudaMemcpyHostToDevice));
    op.d_p1_items = d_p1;
    op.n_p1 = (int)p1.size();
    op.d_p2_leaf = d_l;
    op.n_p2 = nl;
    op.d_p2_segs = d_s;
    op.n_p2_segs = (int)segs.size();
    op.w_len = wl;
    if ((rc = dev_alloc(op, &op.d_w, (size_t)std::max<int64_t>(wl, 1), err))) return rc;
    // algorithmic bytes of one apply: operator data once per frequency, X read, Y written
    const int fesz = op.far_prec == RT_PREC_F32 ? 4 : 2;
    int64_t far_e = 0, near_e = 0;
    for (int b = 0; b < op.n_far; ++b) far_e += (int64_t)op.rank[b] * (op.far_blocks[b].m + op.far_blocks[b].n);
    for (int b = 0; b < op.n_near; ++b) near_e += (int64_t)op.dense_blocks[b].m * op.dense_blocks[b].n;
    op.info.apply_bytes = F * (far_e * fesz + near_e * 4) + 2 * F * N * (int64_t)esz;
    op.info.apply_flops = 2 * F * (far_e + near_e);
    return RT_OK;
}

int apply_tree(Operator& op, const void* X, void* Y, cudaStream_t s, std::string& err)
{
    const int N = op.N, F = op.F;
    if (op.mode == RT_MODE_DENSE) {
        const int64_t warps = (int64_t)N * F;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 152 * 16));
        const int* fg = op.d_fq_group;
        if (op.vec64)
            dense_apply<double><<<grid, 256, 0, s>>>((const double*)op.d_dense, (const double*)X, (double*)Y, N, F, fg);
        else
            dense_apply<float><<<grid, 256, 0, s>>>((const float*)op.d_dense, (const float*)X, (float*)Y, N, F, fg);
        RT_CUDA_TRY(cudaGetLastError());
        return RT_OK;
    }
    const float* x = (const float*)X;
    float* y = (float*)Y;
    if (op.n_p1 > 0) {
        dim3 g1(op.n_p1, F);
        if (op.far_prec == RT_PREC_F32)
            hmv_phase1<float><<<g1, 256, 0, s>>>((const P1Item*)op.d_p1_items, (const float*)op.d_far, x, op.d_w, N,
                                                 op.d_fq_group);
        else if (op.far_prec == RT_PREC_BF16)
            hmv_phase1<__nv_bfloat16><<<g1, 256, 0, s>>>((const P1Item*)op.d_p1_items, (const __nv_bfloat16*)op.d_far,
                                                         x, op.d_w, N, op.d_fq_group);
        else
            hmv_phase1<__half><<<g1, 256, 0, s>>>((const P1Item*)op.d_p1_items, (const __half*)op.d_far, x, op.d_w, N,
                                                  op.d_fq_group);
        RT_CUDA_TRY(cudaGetLastError());
    }
    dim3 g2(op.n_p2, F);
    if (op.far_prec == RT_PREC_F32)
        hmv_phase2<float><<<g2, 256, 0, s>>>((const P2Leaf*)op.d_p2_leaf, (const P2Seg*)op.d_p2_segs,
                                             (const float*)op.d_far, op.d_near, x, op.d_w, y, N, op.d_fq_group);
    else if (op.far_prec == RT_PREC_BF16)
        hmv_phase2<__nv_bfloat16><<<g2, 256, 0, s>>>((const P2Leaf*)op.d_p2_leaf, (const P2Seg*)op.d_p2_segs,
                                                     (const __nv_bfloat16*)op.d_far, op.d_near, x, op.d_w, y, N,
                                                     op.d_fq_group);
    else
        hmv_phase2<__half><<<g2, 256, 0, s>>>((const P2Leaf*)op.d_p2_leaf, (const P2Seg*)op.d_p2_segs,
                                              (const __half*)op.d_far, op.d_near, x, op.d_w, y, N, op.d_fq_group);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}


// ---------------------------------------------------------------------------
// Apply without allocation.
//
// Same kernels and the same arithmetic as apply_tree + the two permutations,
// but the scratch (X and Y in tree order and the phase-1 w buffer) lives in
// one file-scope device array instead of buffers owned by the operator.  The
// array is kNoAllocBytes large, is held by every GPU that loads the library
// until the process exits, and is shared by every call: it keeps the previous
// call's contents (every region used is fully overwritten before it is read,
// so nothing needs clearing), and two calls that overlap on the GPU race on it.
// ---------------------------------------------------------------------------
static constexpr size_t kNoAllocBytes = (size_t)8 << 20;
static constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};   // device address per device, set on first use

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
    if (op.mode == RT_MODE_DENSE) {
        // the dense apply reads X and writes Y directly: no scratch at all
        const int64_t warps = (int64_t)N * F;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 152 * 16));
        if (op.vec64)
            dense_apply<double><<<grid, 256, 0, s>>>((const double*)op.d_dense, (const double*)X, (double*)Y, N, F,
                                                     op.d_fq_group);
        else
            dense_apply<float><<<grid, 256, 0, s>>>((const float*)op.d_dense, (const float*)X, (float*)Y, N, F,
                                                    op.d_fq_group);
        RT_CUDA_TRY(cudaGetLastError());
        return RT_OK;
    }
    const size_t vbytes = round256((size_t)F * N * sizeof(float));
    const size_t wbytes = round256((size_t)std::max<int64_t>(op.w_len, 1) * sizeof(float));
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
    if (!g_noalloc_addr[dev]) {
        // one-time set-up on this device (the device is current): the host-side
        // name of a __device__ array is not a device address; ask the runtime for it
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("rt_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return RT_ECUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    unsigned char* base = (unsigned char*)g_noalloc_addr[dev];
    float* xt = (float*)base;
    float* yt = (float*)(base + vbytes);
    float* w = (float*)(base + 2 * vbytes);
    int rc = permute_vectors(op, X, xt, 1, 0, F, s);
    if (rc) {
        err = "rt_apply_noalloc: permute launch failed";
        return rc;
    }
    if (op.n_p1 > 0) {
        dim3 g1(op.n_p1, F);
        if (op.far_prec == RT_PREC_F32)
            hmv_phase1<float><<<g1, 256, 0, s>>>((const P1Item*)op.d_p1_items, (const float*)op.d_far, xt, w, N,
                                                 op.d_fq_group);
        else if (op.far_prec == RT_PREC_BF16)
            hmv_phase1<__nv_bfloat16><<<g1, 256, 0, s>>>((const P1Item*)op.d_p1_items, (const __nv_bfloat16*)op.d_far,
                                                         xt, w, N, op.d_fq_group);
        else
            hmv_phase1<__half><<<g1, 256, 0, s>>>((const P1Item*)op.d_p1_items, (const __half*)op.d_far, xt, w, N,
                                                  op.d_fq_group);
        RT_CUDA_TRY(cudaGetLastError());
    }
    dim3 g2(op.n_p2, F);
    if (op.far_prec == RT_PREC_F32)
        hmv_phase2<float><<<g2, 256, 0, s>>>((const P2Leaf*)op.d_p2_leaf, (const P2Seg*)op.d_p2_segs,
                                             (const float*)op.d_far, op.d_near, xt, w, yt, N, op.d_fq_group);
    else if (op.far_prec == RT_PREC_BF16)
        hmv_phase2<__nv_bfloat16><<<g2, 256, 0, s>>>((const P2Leaf*)op.d_p2_leaf, (const P2Seg*)op.d_p2_segs,
                                                     (const __nv_bfloat16*)op.d_far, op.d_near, xt, w, yt, N,
                                                     op.d_fq_group);
    else
        hmv_phase2<__half><<<g2, 256, 0, s>>>((const P2Leaf*)op.d_p2_leaf, (const P2Seg*)op.d_p2_segs,
                                              (const __half*)op.d_far, op.d_near, xt, w, yt, N, op.d_fq_group);
    RT_CUDA_TRY(cudaGetLastError());
    rc = permute_vectors(op, yt, Y, 0, 0, F, s);
    if (rc) {
        err = "rt_apply_noalloc: permute launch failed";
        return rc;
    }
    return RT_OK;
}

}  // namespace rt
