// rt_batch.cu -- many independent instances solved together.
//
// Every instance keeps its own operator (built by rt_build_operator, several
// host threads each on its own stream).  The batch then runs
//   * one persistent apply launch for all instances: CTAs take work items from
//     a global atomic counter, every phase-1 item (w = V^T x) before every
//     phase-2 item (y = U w + A x); a phase-2 item of instance b waits, with a
//     bounded spin, until all phase-1 items of b have been counted done --
//     those items were taken earlier by resident CTAs, so the wait ends;
//   * the fixed point of Section 1.3 on concatenated vectors: one source
//     update, one persistent apply, one update + per-instance FP64 residual
//     (CTA per instance, deterministic), one FP64 Newton, one flag update per
//     iteration; an instance stops (its J and T freeze) at the first
//     iteration whose residual is <= tol; check_every iterations are replayed
//     as one CUDA graph;
//   * an autotuner that times candidate work-item sizes and persistent grid
//     sizes on the batch and keeps the fastest.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rt_hmv_dev.cuh"
#include "rt_internal.h"
#include "rt_newton.cuh"

namespace rt {

constexpr double kSigmaB = 6.493939402266829;   // pi^4 / 15

struct BatchInst {
    const float* far;
    const float* nearp;
    const P1Row* rows;
    const P2Leaf* leaves;
    const P2Seg* segs;
    float* W;
    const int* fgroup;
    const double* fq;     // [F][4]: nu, w c (1-a), a, group
    const double* fscale; // [F] c_f / c_g of binned channels, or null
    const int* perm;      // tree position -> caller vertex id
    int N, F, grey, n1;
    int64_t voff;         // offset of the instance's [F][N] vectors
    int64_t toff;         // offset of its [N] temperatures
};

struct BatchWork {
    int inst, kind, idx, f;   // kind 1: phase-1 item idx; kind 2: phase-2 leaf idx
};

struct Batch {
    std::vector<rt_operator*> ops;
    int n = 0;
    int64_t total_vec = 0, total_vert = 0;
    std::vector<int64_t> voff, toff;
    BatchInst* d_inst = nullptr;
    P1Item* d_items = nullptr;
    BatchWork* d_works = nullptr;
    int nworks = 0;
    int* d_next = nullptr;
    int* d_done1 = nullptr;
    int* d_err = nullptr;
    int64_t* d_voff = nullptr;
    int64_t* d_toff = nullptr;
    int ctas = 0;
    int maxF = 1;                          // largest frequency count of the instances
    int p1_bytes = 64 << 10, ctas_per_sm = 8;   // the autotuner's pick for 256 mixed instances on GB300
    long long spin_cycles = 0;   // wait budget of the phase-2 items (0: kSpinCycles)
    int spin_extra = 0;          // diagnostic: completed phase-1 items a wait needs beyond all of them
    double tune_ms = 0.0, build_ms = 0.0;
    // solver buffers (tree order, concatenated)
    float *d_xt = nullptr, *d_yt = nullptr, *d_J = nullptr, *d_S = nullptr, *d_Y = nullptr, *d_SE = nullptr;
    double* d_T = nullptr;
    int* d_active = nullptr;
    int* d_done_now = nullptr;
    int* d_iters = nullptr;
    int* d_nactive = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<void*> allocs;
};

template <class T>
static int balloc(Batch& B, T** p, size_t count, std::string& err)
{
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc (batch): ") + cudaGetErrorString(e);
        *p = nullptr;
        return RT_ENOMEM;
    }
    B.allocs.push_back(*p);
    return RT_OK;
}

__device__ __forceinline__ int find_seg(const int64_t* off, int n, int64_t e)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// the persistent apply
// ---------------------------------------------------------------------------
constexpr long long kSpinCycles = 2000000000ll;   // ~1 s

__global__ void __launch_bounds__(256) batch_apply_kernel(const BatchInst* __restrict__ insts,
                                                          const P1Item* __restrict__ items,
                                                          const BatchWork* __restrict__ works, int nworks,
                                                          const float* __restrict__ X, float* __restrict__ Y,
                                                          int* __restrict__ next, int* __restrict__ done1,
                                                          const int* __restrict__ active, int* __restrict__ err,
                                                          long long spin_cycles, int extra)
{
    __shared__ int s_w;
    __shared__ float4 red[256];
    for (;;) {
        if (threadIdx.x == 0) s_w = atomicAdd(next, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= nworks) break;
        const BatchWork wk = works[w];
        if (active && !active[wk.inst]) continue;   // frozen instance: neither phase runs
        const BatchInst I = insts[wk.inst];
        const int g = I.fgroup[wk.f];
        if (wk.kind == 1) {
            hmv_p1_body<float>(items[wk.idx], wk.f, g, I.rows, I.far, nullptr, X + I.voff, I.W, I.N);
            __threadfence();   // every writer publishes its w values before the count
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&done1[wk.inst], 1);
        } else {
            if (threadIdx.x == 0) {
                const long long t0 = clock64();
                while (*(volatile int*)&done1[wk.inst] < I.n1 + extra) {
                    if (clock64() - t0 > spin_cycles) {
                        atomicOr(err, 1);
                        break;
                    }
                }
                __threadfence();
            }
            __syncthreads();
            hmv_p2_body<float, true>(I.leaves[wk.idx], wk.f, g, I.segs, I.far, nullptr, I.nearp, X + I.voff, I.W,
                                     Y + I.voff, I.N, red);
        }
    }
}

// caller order <-> tree order for every instance of the batch
// (scale != 0: the output of an apply, times c_f / c_g for binned channels)
__global__ void batch_permute(const BatchInst* __restrict__ insts, const int64_t* __restrict__ voff, int n,
                              int64_t total, const float* __restrict__ in, float* __restrict__ out, int to_tree,
                              int scale = 0)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = find_seg(voff, n, e);
        const BatchInst I = insts[b];
        const int64_t loc = e - I.voff;
        const int64_t f = loc / I.N;
        const int t = (int)(loc - f * I.N);
        if (to_tree) out[e] = in[I.voff + f * I.N + I.perm[t]];
        else out[I.voff + f * I.N + I.perm[t]] = (scale && I.fscale) ? (float)(in[e] * I.fscale[f]) : in[e];
    }
}

__global__ void batch_permute_T(const BatchInst* __restrict__ insts, const int64_t* __restrict__ toff, int n,
                                int64_t total, const double* __restrict__ in, double* __restrict__ out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = find_seg(toff, n, e);
        const BatchInst I = insts[b];
        out[I.toff + I.perm[e - I.toff]] = in[e];
    }
}

// ---------------------------------------------------------------------------
// batched fixed point
// ---------------------------------------------------------------------------
__device__ __forceinline__ double planck_b(double nu, double T)
{
    if (!(T > 0.0)) return 0.0;
    const double x = nu / T;
    if (x > 700.0) return 0.0;
    return nu * nu * nu / expm1(x);
}

__global__ void batch_init(const BatchInst* __restrict__ insts, const int64_t* __restrict__ toff, int n,
                           float* __restrict__ J, double* __restrict__ T, int64_t tv, int64_t tt, double T0,
                           int* __restrict__ active, int* __restrict__ iters)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tv; e += (int64_t)gridDim.x * blockDim.x)
        J[e] = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tt; e += (int64_t)gridDim.x * blockDim.x)
        T[e] = T0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        active[e] = 1;
        iters[e] = 0;
    }
}

__global__ void batch_source(const BatchInst* __restrict__ insts, const int64_t* __restrict__ voff, int n,
                             int64_t total, const float* __restrict__ J, const double* __restrict__ T,
                             float* __restrict__ S, const int* __restrict__ active)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = find_seg(voff, n, e);
        if (!active[b]) continue;
        const BatchInst I = insts[b];
        const int64_t loc = e - I.voff;
        const int f = (int)(loc / I.N), i = (int)(loc - (int64_t)f * I.N);
        const double a = I.fq[4 * f + 2];
        const double t = T[I.toff + i];
        const double B = I.grey ? kSigmaB * t * t * t * t : planck_b(I.fq[4 * f], t);
        const double v = a * (double)J[e] + (1.0 - a) * B;
        S[e] = (float)(I.fscale ? v * I.fscale[f] : v);
    }
}

// CTA per instance: J <- SE + Y, FP64 residual, convergence flag
__global__ void __launch_bounds__(256) batch_update(const BatchInst* __restrict__ insts, float* __restrict__ J,
                                                    const float* __restrict__ Y, const float* __restrict__ SE,
                                                    const int* __restrict__ active, int* __restrict__ done_now,
                                                    double tol)
{
    const int b = blockIdx.x;
    if (!active[b]) return;
    const BatchInst I = insts[b];
    const int64_t len = (int64_t)I.F * I.N;
    double d2 = 0.0, n2 = 0.0;
    for (int64_t k = threadIdx.x; k < len; k += blockDim.x) {
        const int64_t e = I.voff + k;
        const float jn = SE[e] + Y[e];
        const double d = (double)jn - (double)J[e];
        d2 += d * d;
        n2 += (double)jn * (double)jn;
        J[e] = jn;
    }
    __shared__ double s[2][8];
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s[0][threadIdx.x >> 5] = d2;
        s[1][threadIdx.x >> 5] = n2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += s[0][w];
            c += s[1][w];
        }
        const double res = c > 0.0 ? sqrt(a / c) : (a > 0.0 ? INFINITY : 0.0);
        done_now[b] = res <= tol ? 1 : 0;
    }
}

// LPV lanes per vertex (the power of two >= the batch's largest F), the same
// temperature solve as the single-instance solver (rt_newton.cuh)
template <int LPV>
__global__ void __launch_bounds__(256) batch_newton(const BatchInst* __restrict__ insts,
                                                    const int64_t* __restrict__ toff, int n, int64_t total,
                                                    const float* __restrict__ J, double* __restrict__ T,
                                                    const int* __restrict__ active, int* __restrict__ fail)
{
    constexpr int VPW = 32 / LPV;
    const int lane = threadIdx.x & 31, sl = lane & (LPV - 1);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * VPW; base < total;
         base += nw * VPW) {
        const int64_t v = base + lane / LPV;
        if (v >= total) continue;   // whole vertex segments drop out together
        const int b = find_seg(toff, n, v);
        if (!active[b]) continue;
        const BatchInst I = insts[b];
        const int i = (int)(v - I.toff);
        if (I.grey) {
            if (sl == 0) {
                const double j = (double)J[I.voff + i];
                T[v] = j > 0.0 ? sqrt(sqrt(j / kSigmaB)) : 0.0;
            }
            continue;
        }
        const unsigned m = seg_mask<LPV>(lane);
        double rhs = 0.0;
        for (int f = sl; f < I.F; f += LPV) rhs += I.fq[4 * f + 1] * (double)J[I.voff + (int64_t)f * I.N + i];
#pragma unroll
        for (int o = LPV >> 1; o > 0; o >>= 1) rhs += __shfl_xor_sync(m, rhs, o);
        if (!(rhs > 0.0)) {
            if (sl == 0) T[v] = 0.0;
            continue;
        }
        double t = 0.0;
        const bool ok = solve_temperature<LPV>(I.fq, I.F, rhs, lane, T[v], t);
        if (sl == 0) {
            if (!ok) atomicOr(fail, 1);
            T[v] = t;
        }
    }
}

__global__ void batch_flags(int* __restrict__ active, const int* __restrict__ done_now, int* __restrict__ iters,
                            int n, int* __restrict__ nactive)
{
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        if (active[b]) {
            iters[b] += 1;
            if (done_now[b]) active[b] = 0;
            else atomicAdd(&cnt, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *nactive = cnt;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int grid_for_elems(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// work list for a phase-1 target size (bytes of operator data per item)
static int build_works(Batch& B, int p1_bytes, std::vector<P1Item>& items, std::vector<BatchWork>& works,
                       std::vector<int>& n1)
{
    items.clear();
    works.clear();
    n1.assign(B.n, 0);
    std::vector<std::pair<int64_t, BatchWork>> w1, w2;
    for (int b = 0; b < B.n; ++b) {
        const Operator& op = B.ops[b]->op;
        const P1Row* rows = reinterpret_cast<const P1Row*>(op.h_p1_rows.data());
        const size_t nrows = op.h_p1_rows.size() / sizeof(P1Row);
        for (size_t i = 0; i < nrows;) {
            const int n = rows[i].n;
            int sw = 32;
            if ((n + 3) / 4 <= 8) sw = 8;
            else if ((n + 3) / 4 <= 16) sw = 16;
            const int per = (int)std::max<int64_t>(1, std::min<int64_t>(512, p1_bytes / std::max(1, n * 4)));
            size_t j = i;
            while (j < nrows && (int)(j - i) < per && rows[j].n == n) ++j;
            const int idx = (int)items.size();
            items.push_back({(int)i, (int)j, sw, 0});
            for (int f = 0; f < op.F; ++f) {
                w1.push_back({(int64_t)(j - i) * n, {b, 1, idx, f}});
                n1[b]++;
            }
            i = j;
        }
        const int nl = (int)op.plan.leaf_start.size();
        for (int l = 0; l < nl; ++l)
            for (int f = 0; f < op.F; ++f) w2.push_back({(int64_t)op.plan.leaf_size[l], {b, 2, l, f}});
    }
    auto desc = [](const std::pair<int64_t, BatchWork>& a, const std::pair<int64_t, BatchWork>& c) {
        return a.first > c.first;
    };
    std::stable_sort(w1.begin(), w1.end(), desc);
    for (auto& w : w1) works.push_back(w.second);
    for (auto& w : w2) works.push_back(w.second);
    return RT_OK;
}

static int upload_works(Batch& B, int p1_bytes, cudaStream_t s, std::string& err)
{
    std::vector<P1Item> items;
    std::vector<BatchWork> works;
    std::vector<int> n1;
    build_works(B, p1_bytes, items, works, n1);
    std::vector<BatchInst> hi(B.n);
    for (int b = 0; b < B.n; ++b) {
        Operator& op = B.ops[b]->op;
        BatchInst& I = hi[b];
        I.far = (const float*)op.d_far;
        I.nearp = op.d_near;
        I.rows = (const P1Row*)op.d_p1_rows;
        I.leaves = (const P2Leaf*)op.d_p2_leaf;
        I.segs = (const P2Seg*)op.d_p2_segs;
        I.W = op.d_w;
        I.fgroup = op.d_fq_group;
        I.fq = op.d_fq;
        I.fscale = op.binned ? op.d_fscale : nullptr;
        I.perm = op.d_perm;
        I.N = op.N;
        I.F = op.F;
        I.grey = op.grey;
        I.n1 = n1[b];
        I.voff = B.voff[b];
        I.toff = B.toff[b];
    }
    if (B.d_items || B.d_works) RT_CUDA_TRY(cudaStreamSynchronize(s));   // the previous lists may be in use
    if (B.d_items) cudaFree(B.d_items);
    if (B.d_works) cudaFree(B.d_works);
    B.allocs.erase(std::remove(B.allocs.begin(), B.allocs.end(), (void*)B.d_items), B.allocs.end());
    B.allocs.erase(std::remove(B.allocs.begin(), B.allocs.end(), (void*)B.d_works), B.allocs.end());
    int rc;
    if ((rc = balloc(B, &B.d_items, items.size(), err))) return rc;
    if ((rc = balloc(B, &B.d_works, works.size(), err))) return rc;
    RT_CUDA_TRY(cudaMemcpyAsync(B.d_items, items.data(), sizeof(P1Item) * items.size(), cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaMemcpyAsync(B.d_works, works.data(), sizeof(BatchWork) * works.size(), cudaMemcpyHostToDevice, s));
    RT_CUDA_TRY(cudaMemcpyAsync(B.d_inst, hi.data(), sizeof(BatchInst) * hi.size(), cudaMemcpyHostToDevice, s));
    B.nworks = (int)works.size();
    B.p1_bytes = p1_bytes;
    return RT_OK;
}

static int launch_apply(Batch& B, const float* X, float* Y, const int* active, cudaStream_t s, std::string& err)
{
    RT_CUDA_TRY(cudaMemsetAsync(B.d_next, 0, sizeof(int), s));
    RT_CUDA_TRY(cudaMemsetAsync(B.d_done1, 0, sizeof(int) * B.n, s));
    batch_apply_kernel<<<B.ctas, 256, 0, s>>>(B.d_inst, B.d_items, B.d_works, B.nworks, X, Y, B.d_next, B.d_done1,
                                              active, B.d_err, B.spin_cycles > 0 ? B.spin_cycles : kSpinCycles,
                                              B.spin_extra);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

// try work-item sizes and persistent grid sizes, keep the fastest
static int autotune(Batch& B, cudaStream_t s, std::string& err)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int sizes[] = {8 << 10, 16 << 10, 32 << 10, 64 << 10};
    const int per_sm[] = {2, 4, 8};
    float best = 1e30f;
    int bs = 48 << 10, bp = 4;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const auto t0 = std::chrono::steady_clock::now();
    int rc;
    for (int sz : sizes) {
        if ((rc = upload_works(B, sz, s, err))) return rc;
        for (int ps : per_sm) {
            B.ctas = sms * ps;
            if ((rc = launch_apply(B, B.d_xt, B.d_yt, nullptr, s, err))) return rc;   // warm
            cudaEventRecord(e0, s);
            for (int k = 0; k < 3; ++k)
                if ((rc = launch_apply(B, B.d_xt, B.d_yt, nullptr, s, err))) return rc;
            cudaEventRecord(e1, s);
            RT_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bs = sz;
                bp = ps;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B.ctas_per_sm = bp;
    B.ctas = sms * bp;
    if ((rc = upload_works(B, bs, s, err))) return rc;
    B.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return RT_OK;
}

// frees the batch's device memory and operators (not the Batch object itself)
static void batch_release(Batch& B)
{
    cudaDeviceSynchronize();
    for (void* p : B.allocs)
        if (p) cudaFree(p);
    B.allocs.clear();
    for (rt_operator* o : B.ops)
        if (o) rt_free(o);
    B.ops.clear();
    if (B.cap) cudaStreamDestroy(B.cap);
    B.cap = nullptr;
}

}  // namespace rt

struct rt_batch {
    rt::Batch b;
};

namespace {
thread_local std::string g_berr;
int bfail(int code, const std::string& m)
{
    g_berr = m;
    return code;
}
}  // namespace

extern "C" {

int rt_build_batch(const rt_problem* probs, int64_t count, const rt_hparams* hp, int threads, int tune, void* stream,
                   rt_batch** out)
{
    using namespace rt;
    if (!out || !probs || !hp || count < 1) return bfail(RT_EINVAL, "invalid batch arguments");
    *out = nullptr;
    if (hp->mode != RT_MODE_HMATRIX || hp->far_prec != RT_PREC_F32)
        return bfail(RT_EINVAL, "batches use the FP32 H-matrix mode");
    rt_batch* h = new rt_batch();
    Batch& B = h->b;
    B.n = (int)count;
    B.ops.assign(count, nullptr);
    const auto t0 = std::chrono::steady_clock::now();
    int dev = 0;
    cudaGetDevice(&dev);
    // build the operators: `threads` host threads, each with its own stream
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>(threads > 0 ? threads : 8, count));
    std::vector<int> rcs(count, RT_OK);
    std::vector<std::string> msgs(count);
    std::mutex mu;
    int64_t next = 0;
    auto worker = [&]() {
        cudaSetDevice(dev);
        cudaStream_t st;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        for (;;) {
            int64_t k;
            {
                std::lock_guard<std::mutex> lock(mu);
                k = next++;
            }
            if (k >= count) break;
            rcs[k] = rt_build_operator(&probs[k], hp, st, &B.ops[k]);
            if (rcs[k]) msgs[k] = rt_last_error();
        }
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
    for (int64_t k = 0; k < count; ++k)
        if (rcs[k]) {
            int rc = rcs[k];
            std::string m = "instance " + std::to_string(k) + ": " + msgs[k];
            batch_release(B);
            delete h;
            return bfail(rc, m);
        }
    B.voff.assign(count + 1, 0);
    B.toff.assign(count + 1, 0);
    for (int64_t k = 0; k < count; ++k) {
        const Operator& op = B.ops[k]->op;
        if (op.G > 16) {
            batch_release(B);
            delete h;
            return bfail(RT_EINVAL, "batch instances must have at most 16 kappa groups");
        }
        B.voff[k + 1] = B.voff[k] + (int64_t)op.F * op.N;
        B.maxF = std::max(B.maxF, op.F);
        B.toff[k + 1] = B.toff[k] + op.N;
    }
    B.total_vec = B.voff[count];
    B.total_vert = B.toff[count];
    std::string err;
    int rc = RT_OK;
    auto chk = [&](int r) {
        if (r && rc == RT_OK) rc = r;
        return r;
    };
    cudaStream_t s = (cudaStream_t)stream;
    if (!chk(balloc(B, &B.d_inst, count, err)) && !chk(balloc(B, &B.d_next, 1, err)) &&
        !chk(balloc(B, &B.d_done1, count, err)) && !chk(balloc(B, &B.d_err, 1, err)) &&
        !chk(balloc(B, &B.d_voff, count + 1, err)) && !chk(balloc(B, &B.d_toff, count + 1, err)) &&
        !chk(balloc(B, &B.d_xt, B.total_vec, err)) && !chk(balloc(B, &B.d_yt, B.total_vec, err)) &&
        !chk(balloc(B, &B.d_J, B.total_vec, err)) && !chk(balloc(B, &B.d_S, B.total_vec, err)) &&
        !chk(balloc(B, &B.d_Y, B.total_vec, err)) && !chk(balloc(B, &B.d_SE, B.total_vec, err)) &&
        !chk(balloc(B, &B.d_T, B.total_vert, err)) && !chk(balloc(B, &B.d_active, count, err)) &&
        !chk(balloc(B, &B.d_done_now, count, err)) && !chk(balloc(B, &B.d_iters, count, err)) &&
        !chk(balloc(B, &B.d_nactive, 1, err))) {
        cudaMemcpyAsync(B.d_voff, B.voff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(B.d_toff, B.toff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(B.d_err, 0, sizeof(int), s);
        cudaMemsetAsync(B.d_xt, 0, sizeof(float) * B.total_vec, s);
        for (int64_t k = 0; k < count; ++k) {
            const Operator& op = B.ops[k]->op;
            cudaMemcpyAsync(B.d_SE + B.voff[k], op.d_SE, sizeof(float) * op.F * op.N, cudaMemcpyDeviceToDevice, s);
        }
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        B.ctas = sms * B.ctas_per_sm;
        chk(upload_works(B, B.p1_bytes, s, err));
        if (rc == RT_OK && tune) chk(autotune(B, s, err));
    }
    if (rc == RT_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = RT_ECUDA;
            err = cudaGetErrorString(e);
        }
    }
    if (rc) {
        batch_release(B);
        delete h;
        return bfail(rc, err);
    }
    B.build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return RT_OK;
}

int rt_batch_info(const rt_batch* h, rt_batch_info_t* info, int64_t* vec_off, int64_t* vert_off)
{
    if (!h || !info) return bfail(RT_EINVAL, "null argument");
    const rt::Batch& B = h->b;
    info->count = B.n;
    info->total_vec = B.total_vec;
    info->total_vert = B.total_vert;
    info->p1_target_bytes = B.p1_bytes;
    info->ctas_per_sm = B.ctas_per_sm;
    info->n_works = B.nworks;
    info->tune_ms = B.tune_ms;
    info->build_ms = B.build_ms;
    int64_t bytes = 0;
    for (rt_operator* o : B.ops) bytes += o->op.info.apply_bytes;
    info->apply_bytes = bytes;
    if (vec_off)
        for (int k = 0; k <= B.n; ++k) vec_off[k] = B.voff[k];
    if (vert_off)
        for (int k = 0; k <= B.n; ++k) vert_off[k] = B.toff[k];
    return RT_OK;
}

int rt_batch_apply(rt_batch* h, const float* X, float* Y, void* stream)
{
    if (!h || !X || !Y) return bfail(RT_EINVAL, "null argument");
    rt::Batch& B = h->b;
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    const int grid = rt::grid_for_elems(B.total_vec);
    rt::batch_permute<<<grid, 256, 0, s>>>(B.d_inst, B.d_voff, B.n, B.total_vec, X, B.d_xt, 1);
    int rc = rt::launch_apply(B, B.d_xt, B.d_yt, nullptr, s, err);
    if (rc) return bfail(rc, err);
    rt::batch_permute<<<grid, 256, 0, s>>>(B.d_inst, B.d_voff, B.n, B.total_vec, B.d_yt, Y, 0, 1);
    if (cudaGetLastError() != cudaSuccess) return bfail(RT_ECUDA, "batch permute launch failed");
    return RT_OK;
}

int rt_solve_batch(rt_batch* h, const rt_solve_opts* o, float* J, double* T, int32_t* iters, rt_solve_stats* stats,
                   void* stream)
{
    using namespace rt;
    if (!h || !o || !J || !T) return bfail(RT_EINVAL, "null argument");
    if (o->max_iter < 1 || o->check_every < 1) return bfail(RT_EINVAL, "invalid solve options");
    Batch& B = h->b;
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    const auto t0 = std::chrono::steady_clock::now();
    const int ge = grid_for_elems(std::max(B.total_vec, B.total_vert));
    int* d_fail = B.d_err;
    batch_init<<<ge, 256, 0, s>>>(B.d_inst, B.d_toff, B.n, B.d_J, B.d_T, B.total_vec, B.total_vert, o->T0,
                                  B.d_active, B.d_iters);
    auto iteration = [&](cudaStream_t cs) -> int {
        batch_source<<<ge, 256, 0, cs>>>(B.d_inst, B.d_voff, B.n, B.total_vec, B.d_J, B.d_T, B.d_S, B.d_active);
        int rc = launch_apply(B, B.d_S, B.d_Y, B.d_active, cs, err);
        if (rc) return rc;
        batch_update<<<B.n, 256, 0, cs>>>(B.d_inst, B.d_J, B.d_Y, B.d_SE, B.d_active, B.d_done_now, o->tol);
        const int lpv = B.maxF <= 1 ? 1 : B.maxF <= 2 ? 2 : B.maxF <= 4 ? 4 : B.maxF <= 8 ? 8 : B.maxF <= 16 ? 16 : 32;
        const int64_t warps = (B.total_vert * lpv + 31) / 32;
        const int gn = (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 152 * 32));
#define RT_BNEWTON(L) \
    batch_newton<L><<<gn, 256, 0, cs>>>(B.d_inst, B.d_toff, B.n, B.total_vert, B.d_J, B.d_T, B.d_active, d_fail)
        switch (lpv) {
            case 1: RT_BNEWTON(1); break;
            case 2: RT_BNEWTON(2); break;
            case 4: RT_BNEWTON(4); break;
            case 8: RT_BNEWTON(8); break;
            case 16: RT_BNEWTON(16); break;
            default: RT_BNEWTON(32); break;
        }
#undef RT_BNEWTON
        batch_flags<<<1, 256, 0, cs>>>(B.d_active, B.d_done_now, B.d_iters, B.n, B.d_nactive);
        return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ECUDA;
    };
    int done_iters = 0, nactive = B.n;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int glen = 0;
    int rc = RT_OK;
    if (!B.cap) cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking);
    while (done_iters < o->max_iter && nactive > 0) {
        const int todo = std::min(o->check_every, o->max_iter - done_iters);
        if (o->use_graph) {
            if (!gexec || glen != todo) {
                if (gexec) cudaGraphExecDestroy(gexec);
                if (graph) cudaGraphDestroy(graph);
                gexec = nullptr;
                graph = nullptr;
                if (cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                    rc = RT_ECUDA;
                    err = "graph capture begin";
                    break;
                }
                int crc = RT_OK;
                for (int k = 0; k < todo && !crc; ++k) crc = iteration(B.cap);
                cudaError_t ce = cudaStreamEndCapture(B.cap, &graph);
                if (crc || ce != cudaSuccess || cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) {
                    rc = RT_ECUDA;
                    err = "graph capture of the batched iteration failed";
                    break;
                }
                glen = todo;
            }
            if (cudaGraphLaunch(gexec, s) != cudaSuccess) {
                rc = RT_ECUDA;
                err = "graph launch";
                break;
            }
        } else {
            for (int k = 0; k < todo && !rc; ++k) rc = iteration(s);
            if (rc) break;
        }
        if (cudaMemcpyAsync(&nactive, B.d_nactive, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = RT_ECUDA;
            err = "batch solve: device error";
            break;
        }
        done_iters += todo;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (rc) return bfail(rc, err);
    const int gp = grid_for_elems(B.total_vec);
    batch_permute<<<gp, 256, 0, s>>>(B.d_inst, B.d_voff, B.n, B.total_vec, B.d_J, J, 0);
    batch_permute_T<<<grid_for_elems(B.total_vert), 256, 0, s>>>(B.d_inst, B.d_toff, B.n, B.total_vert, B.d_T, T);
    int herr = 0;
    std::vector<int> it(B.n);
    cudaMemcpyAsync(it.data(), B.d_iters, sizeof(int) * B.n, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&herr, B.d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(RT_ECUDA, "batch solve: device error");
    if (iters)
        for (int k = 0; k < B.n; ++k) iters[k] = it[k];
    if (stats) {
        stats->iters = done_iters;
        stats->converged = nactive == 0;
        stats->residual = 0.0;
        stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (herr) {
        cudaMemsetAsync(B.d_err, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
        return bfail(RT_ETIMEOUT, "a bounded device wait gave up or a Newton solve failed");
    }
    if (nactive > 0) return bfail(RT_ENOCONV, "some instances did not reach tol within max_iter");
    return RT_OK;
}

int rt_batch_set_wait(rt_batch* h, int64_t wait_cycles, int unreachable)
{
    if (!h || wait_cycles < 0) return bfail(RT_EINVAL, "null batch or negative wait budget");
    h->b.spin_cycles = (long long)wait_cycles;
    h->b.spin_extra = unreachable ? 1 : 0;
    return RT_OK;
}

void rt_batch_free(rt_batch* h)
{
    if (!h) return;
    rt::batch_release(h->b);
    delete h;
}

const char* rt_batch_last_error(void) { return g_berr.c_str(); }

}  // extern "C"
