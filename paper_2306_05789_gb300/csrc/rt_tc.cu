// rt_tc.cu -- multi-right-hand-side H-matvec on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators) for one operator applied to F frequencies
// at once (kappa_nu = kappa(x) for every nu: one operator, F right-hand sides).
//
//   phase 1: W_b [r x F] = V_b^T X_c            (far blocks; K = n, the block width)
//   phase 2: Y_l [m x F] = sum_b U_{b,l} W_b    (far blocks over leaf l; K = r)
//   near   : Y_l += sum_dense A_{b,l} X_c       (FP32 CUDA cores, all F at once)
// The far factors are stored in BF16 or FP16.  The other operand (X, or W)
// is split into a 16-bit high part and a 16-bit remainder, and both products
// accumulate into the same FP32 TMEM tile, so the right-hand sides keep ~16
// significant bits.  Tiles are staged through registers into the canonical
// no-swizzle K-major shared-memory layout (8-row x 16-byte core matrices);
// one elected thread issues tcgen05.mma and commits to an mbarrier; every
// wait on that barrier is bounded and reports a timeout through a flag.
#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rt_internal.h"

namespace rt {

namespace tc {

constexpr int kM = 128;          // MMA rows (TMEM lanes)
constexpr int kKT = 64;          // K elements per staged tile (4 MMAs of K = 16)
constexpr int kThreads = 128;    // one warpgroup: warp q reads TMEM lanes 32q..32q+31
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz

// ---- PTX wrappers --------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: start, leading (K) and stride
// (M/N) byte offsets in 16-byte units, descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16 (bf16 = 1) or F16,
// both K-major, N and M dimensions
__device__ __forceinline__ uint32_t idesc_f16(int bf16, int M, int N)
{
    uint32_t d = 0;
    d |= 1u << 4;
    d |= (uint32_t)bf16 << 7;
    d |= (uint32_t)bf16 << 10;
    d |= (uint32_t)(N >> 3) << 17;
    d |= (uint32_t)(M >> 4) << 24;
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
}

// wait for the given phase parity with a clock budget (non-blocking probes);
// returns false on timeout
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done = 0;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// byte offset of element (row, k) in a K-major no-swizzle tile of kKT columns
__device__ __forceinline__ uint32_t tile_off(int row, int k)
{
    return (uint32_t)((row >> 3) * (kKT / 8 * 128) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <class T>
__device__ __forceinline__ T to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }
__device__ __forceinline__ float from16(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float from16(__half x) { return __half2float(x); }

template <class T>
__device__ __forceinline__ void st16(unsigned char* tile, int row, int k, T v)
{
    *reinterpret_cast<T*>(tile + tile_off(row, k)) = v;
}

// Copy rows [0, nrows) x 16-byte chunks [0, 8) of a K-major tile from global
// memory (row r, chunk c at src + r * ld + 8 c elements; zero where the
// predicate fails).  A warp handles 8 rows x 4 chunks per step, so each group
// of 8 consecutive lanes stores 8 different rows of one chunk: 8 distinct
// 16-byte bank groups in the no-swizzle layout (no conflicts), while every
// row contributes a 64-byte contiguous run to the global load.
template <class T, class Pred>
__device__ __forceinline__ void stage_rows(unsigned char* tile, int nrows, const T* __restrict__ src, int64_t ld,
                                           Pred valid)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int r_in = lane & 7, c_in = lane >> 3;
    const int steps = (nrows >> 3) * 2;   // (8-row group, chunk half) pairs
    for (int st = warp; st < steps; st += nw) {
        const int row = (st >> 1) * 8 + r_in;
        const int c = (st & 1) * 4 + c_in;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (valid(row, c)) v = __ldg(reinterpret_cast<const uint4*>(src + (int64_t)row * ld + 8 * c));
        *reinterpret_cast<uint4*>(tile + tile_off(row, 8 * c)) = v;
    }
}

}  // namespace tc

// X (FP32, tree order, [F][N]) -> high and low 16-bit parts
template <class T>
__global__ void tc_split_kernel(const float* __restrict__ X, T* __restrict__ hi, T* __restrict__ lo, int64_t total)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const float x = X[e];
        const T h = tc::to16<T>(x);
        hi[e] = h;
        lo[e] = tc::to16<T>(x - tc::from16(h));
    }
}

struct TcBlock {
    int64_t v;      // element offset of V^T [r][n8]
    int64_t w;      // offset of the block's W16 [F][r16] (hi and lo arrays)
    int n, n8, col0, r, r16, pad;
};

// phase 1: persistent CTAs walk the far blocks; one block = ceil(r/128) M tiles.
// W_b = V_b^T X_c is written as 16-bit high and low parts, [F][r16] per block.
template <class T>
__global__ void __launch_bounds__(tc::kThreads) tc_phase1(const TcBlock* __restrict__ blocks, int nblocks,
                                                          const T* __restrict__ far, const T* __restrict__ xhi,
                                                          const T* __restrict__ xlo, T* __restrict__ whi,
                                                          T* __restrict__ wlo, int N, int F, int xaligned,
                                                          int* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // [A: 128 x 64 | B_hi: F x 64 | B_lo: F x 64]
    unsigned char* sA = smem;
    unsigned char* sBh = smem + tc::kM * tc::kKT * 2;
    unsigned char* sBl = sBh + F * tc::kKT * 2;
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = F <= 32 ? 32 : (F <= 64 ? 64 : (F <= 128 ? 128 : 256));
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(&s_tmem), ncols);
    if (tid == 0) {
        tc::bar_init(tc::smem_addr(&bar));
        tc::fence_async_smem();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t bar_a = tc::smem_addr(&bar);
    const uint32_t idesc = tc::idesc_f16(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, tc::kM, F);
    const uint32_t lbo = 128, sbo = tc::kKT / 8 * 128;
    uint32_t phase = 0;
    bool ok = true;
    for (int bi = blockIdx.x; bi < nblocks && ok; bi += gridDim.x) {
        const TcBlock B = blocks[bi];
        for (int m0 = 0; m0 < B.r && ok; m0 += tc::kM) {
            const int mr = min(tc::kM, B.r - m0);
            int first = 1;
            for (int k0 = 0; k0 < B.n && ok; k0 += tc::kKT) {
                // A: rows m0.. of V^T, columns k0..k0+63 (V rows are zero-padded to n8)
                tc::stage_rows<T>(sA, tc::kM, far + B.v + (int64_t)m0 * B.n8 + k0, B.n8,
                                  [&](int row, int c) { return row < mr && k0 + 8 * c < B.n8; });
                // B: right-hand side f, columns k0..k0+63 of the block (zero beyond n)
                if (xaligned && (B.col0 & 7) == 0) {   // 16-byte loads need 8-element aligned row starts
                    const T* bh = xhi + B.col0 + k0;
                    const T* bl = xlo + B.col0 + k0;
                    const int full = (B.n - k0) >> 3;   // whole 8-element chunks inside the block
                    tc::stage_rows<T>(sBh, F, bh, N, [&](int, int c) { return c < full; });
                    tc::stage_rows<T>(sBl, F, bl, N, [&](int, int c) { return c < full; });
                    // a partial last chunk (n not a multiple of 8): element-wise, after the
                    // zero fill of that chunk above
                    if (((B.n - k0) & 7) && full < 8) {
                        __syncthreads();
                        for (int e = tid; e < F * 8; e += tc::kThreads) {
                            const int f = e >> 3, j = e & 7, col = k0 + 8 * full + j;
                            T h = tc::to16<T>(0.f), l = tc::to16<T>(0.f);
                            if (col < B.n) {
                                h = xhi[(int64_t)f * N + B.col0 + col];
                                l = xlo[(int64_t)f * N + B.col0 + col];
                            }
                            tc::st16<T>(sBh, f, 8 * full + j, h);
                            tc::st16<T>(sBl, f, 8 * full + j, l);
                        }
                    }
                } else {
                    for (int e = tid; e < F * tc::kKT; e += tc::kThreads) {
                        const int f = e % F, c = e / F, col = k0 + c;
                        T h = tc::to16<T>(0.f), l = tc::to16<T>(0.f);
                        if (col < B.n) {
                            const int64_t idx = (int64_t)f * N + B.col0 + col;
                            h = xhi[idx];
                            l = xlo[idx];
                        }
                        tc::st16<T>(sBh, f, c, h);
                        tc::st16<T>(sBl, f, c, l);
                    }
                }
                tc::fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_addr(sA), bh0 = tc::smem_addr(sBh), bl0 = tc::smem_addr(sBl);
                    const int nks = (min(tc::kKT, B.n - k0) + 15) / 16;
                    for (int ks = 0; ks < nks; ++ks) {
                        const uint64_t da = tc::sdesc(a0 + ks * 2 * lbo, lbo, sbo);
                        tc::mma_f16(tmem, da, tc::sdesc(bh0 + ks * 2 * lbo, lbo, sbo), idesc, first ? 0u : 1u);
                        first = 0;
                        tc::mma_f16(tmem, da, tc::sdesc(bl0 + ks * 2 * lbo, lbo, sbo), idesc, 1u);
                    }
                    tc::mma_commit(bar_a);
                }
                first = 0;
                const bool waited = tc::bar_wait(bar_a, phase);
                phase ^= 1u;
                tc::tc_fence_after();
                if (__syncthreads_or(!waited)) {   // CTA-uniform decision
                    ok = false;
                    if (tid == 0) atomicOr(err, 1);
                }
            }
            if (!ok) break;
            // epilogue: thread of warp q holds TMEM lane (row k) 32q + lane; write W as hi + lo
            const int row = warp * 32 + lane;
            for (int c0 = 0; c0 < F; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
                if (row < mr) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const T h = tc::to16<T>(v[k]);
                        const int64_t idx = B.w + (int64_t)(c0 + k) * B.r16 + m0 + row;
                        whi[idx] = h;
                        wlo[idx] = tc::to16<T>(v[k] - tc::from16(h));
                    }
                }
            }
            tc::tc_fence_before();
            __syncthreads();
        }
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

struct TcSeg {
    int64_t u;      // element offset of the chunk U^T [r][m8]
    int64_t w;      // offset of the block's W16 [F][r16]
    int r, r16;
};

struct TcLeaf {
    int row0, m, m8, seg0, nseg, pad;
};

// phase 2 (far part): CTA per leaf, Y_l = sum_b U_{b,l} W_b, overwrites Y
template <class T>
__global__ void __launch_bounds__(tc::kThreads) tc_phase2(const TcLeaf* __restrict__ leaves,
                                                          const TcSeg* __restrict__ segs, const T* __restrict__ far,
                                                          const T* __restrict__ whi, const T* __restrict__ wlo,
                                                          float* __restrict__ Y, int N, int F, int* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sBh = smem + tc::kM * tc::kKT * 2;
    unsigned char* sBl = sBh + F * tc::kKT * 2;
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = F <= 32 ? 32 : (F <= 64 ? 64 : (F <= 128 ? 128 : 256));
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(&s_tmem), ncols);
    if (tid == 0) {
        tc::bar_init(tc::smem_addr(&bar));
        tc::fence_async_smem();
    }
    // rows beyond the leaf stay zero for the whole kernel
    for (int e = tid; e < tc::kM * tc::kKT * 2 / 16; e += tc::kThreads)
        reinterpret_cast<uint4*>(sA)[e] = make_uint4(0, 0, 0, 0);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t bar_a = tc::smem_addr(&bar);
    const uint32_t idesc = tc::idesc_f16(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, tc::kM, F);
    const uint32_t lbo = 128, sbo = tc::kKT / 8 * 128;
    uint32_t phase = 0;
    bool ok = true;
    const TcLeaf L = leaves[blockIdx.x];
    int first = 1;
    for (int si = L.seg0; si < L.seg0 + L.nseg && ok; ++si) {
        const TcSeg S = segs[si];
        for (int k0 = 0; k0 < S.r && ok; k0 += tc::kKT) {
            const int kc = min(tc::kKT, S.r - k0), kc16 = (kc + 15) & ~15;
            // A: (row i, k) = U^T[k0 + k][i], transposed into K-major; 8 rows i per 16-byte load
            for (int e = tid; e < kc16 * (L.m8 >> 3); e += tc::kThreads) {
                const int k = e % kc16, ic = e / kc16;
                if (k < kc) {
                    const uint4 v = __ldg(reinterpret_cast<const uint4*>(far + S.u + (int64_t)(k0 + k) * L.m8 + 8 * ic));
                    const T* pv = reinterpret_cast<const T*>(&v);
#pragma unroll
                    for (int j = 0; j < 8; ++j) tc::st16<T>(sA, 8 * ic + j, k, pv[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) tc::st16<T>(sA, 8 * ic + j, k, tc::to16<T>(0.f));
                }
            }
            // B: (f, k) = W_b[f][k0 + k], hi and lo parts (zero-padded to r16)
            tc::stage_rows<T>(sBh, F, whi + S.w + k0, S.r16, [&](int, int c) { return 8 * c < kc16; });
            tc::stage_rows<T>(sBl, F, wlo + S.w + k0, S.r16, [&](int, int c) { return 8 * c < kc16; });
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after();
                const uint32_t a0 = tc::smem_addr(sA), bh0 = tc::smem_addr(sBh), bl0 = tc::smem_addr(sBl);
                for (int ks = 0; ks < kc16 / 16; ++ks) {
                    const uint64_t da = tc::sdesc(a0 + ks * 2 * lbo, lbo, sbo);
                    tc::mma_f16(tmem, da, tc::sdesc(bh0 + ks * 2 * lbo, lbo, sbo), idesc, first ? 0u : 1u);
                    first = 0;
                    tc::mma_f16(tmem, da, tc::sdesc(bl0 + ks * 2 * lbo, lbo, sbo), idesc, 1u);
                }
                tc::mma_commit(bar_a);
            }
            first = 0;
            const bool waited = tc::bar_wait(bar_a, phase);
            phase ^= 1u;
            tc::tc_fence_after();
            if (__syncthreads_or(!waited)) {   // CTA-uniform decision
                ok = false;
                if (tid == 0) atomicOr(err, 1);
            }
        }
    }
    if (ok) {
        const int row = warp * 32 + lane;
        for (int c0 = 0; c0 < F; c0 += 16) {
            float v[16];
            if (first) {
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = 0.f;   // no far segment: the far part is zero
            } else {
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            }
            if (row < L.m) {
#pragma unroll
                for (int k = 0; k < 16; ++k) Y[(int64_t)(c0 + k) * N + L.row0 + row] = v[k];
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

struct NearSeg {
    int64_t a;      // element offset of the chunk A^T [n][m8]
    int col0, n;
};

// near field, FP32 CUDA cores, all F right-hand sides per read of A:
// CTA per leaf, thread owns 4 rows x 4 right-hand sides; Y += A X
__global__ void __launch_bounds__(256) near_mrhs(const TcLeaf* __restrict__ leaves, const NearSeg* __restrict__ segs,
                                                 const float* __restrict__ A, const float* __restrict__ X,
                                                 float* __restrict__ Y, int N, int F)
{
    extern __shared__ float sx[];   // [64][F] staged X columns of one segment (k major)
    const TcLeaf L = leaves[blockIdx.x];
    const int tid = threadIdx.x;
    const int nr4 = L.m8 >> 2;                 // row quads
    const int nf4 = F >> 2;                    // rhs quads
    for (int base = 0; base < nr4 * nf4; base += blockDim.x) {
        const int t = base + tid;
        const bool act = t < nr4 * nf4;
        const int rq = act ? t % nr4 : 0, fq = act ? t / nr4 : 0;
        float acc[4][4] = {};
        for (int si = L.seg0; si < L.seg0 + L.nseg; ++si) {
            const NearSeg S = segs[si];
            for (int k0 = 0; k0 < S.n; k0 += 64) {
                const int kc = min(64, S.n - k0);
                __syncthreads();
                for (int e = tid; e < kc * F; e += blockDim.x) {
                    const int f = e / kc, k = e % kc;
                    sx[k * F + f] = X[(int64_t)f * N + S.col0 + k0 + k];
                }
                __syncthreads();
                if (act) {
#pragma unroll 4
                    for (int k = 0; k < kc; ++k) {
                        const float4 a = __ldg(reinterpret_cast<const float4*>(A + S.a + (int64_t)(k0 + k) * L.m8 + 4 * rq));
                        const float4 x = *reinterpret_cast<const float4*>(sx + k * F + 4 * fq);
                        const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * xv[j];
                    }
                }
            }
        }
        if (act) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = 4 * rq + i;
                if (row < L.m)
#pragma unroll
                    for (int j = 0; j < 4; ++j) Y[(int64_t)(4 * fq + j) * N + L.row0 + row] += acc[i][j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
int tc_prepare(Operator& op, std::string& err)
{
    op.tc_enabled = 0;
    if (op.tc_off) return RT_OK;
    if (op.mode != RT_MODE_HMATRIX || op.G != 1 || op.F % 16 != 0 || op.F < 16 || op.F > 256) return RT_OK;
    if (op.far_prec != RT_PREC_BF16 && op.far_prec != RT_PREC_F16) return RT_OK;
    for (int l = 0; l < (int)op.plan.leaf_size.size(); ++l)
        if (op.plan.leaf_size[l] > tc::kM) return RT_OK;
    int rc;
    std::vector<TcBlock> blocks;
    std::vector<int64_t> w_base(op.n_far);
    int64_t wl = 0;
    for (int b = 0; b < op.n_far; ++b) {
        const int r16 = (op.rank[b] + 15) & ~15;
        w_base[b] = wl;
        wl += (int64_t)op.F * r16;
        const FarBlock& fb = op.far_blocks[b];
        blocks.push_back({op.far_v_off[b], w_base[b], fb.n, round8(fb.n), fb.col0, op.rank[b], r16, 0});
    }
    std::stable_sort(blocks.begin(), blocks.end(),
                     [](const TcBlock& a, const TcBlock& b) { return (int64_t)a.n * a.r > (int64_t)b.n * b.r; });
    const int nl = (int)op.plan.leaf_start.size();
    std::vector<std::vector<TcSeg>> fl(nl);
    std::vector<std::vector<NearSeg>> nlst(nl);
    for (int b = 0; b < op.n_far; ++b)
        for (int c = op.far_chunk_ptr[b]; c < op.far_chunk_ptr[b + 1]; ++c) {
            const Chunk& ch = op.far_chunks[c];
            fl[ch.leaf].push_back({op.far_u_off[b] + ch.off, w_base[b], op.rank[b], (op.rank[b] + 15) & ~15});
        }
    for (int b = 0; b < op.n_near; ++b)
        for (int c = op.dense_chunk_ptr[b]; c < op.dense_chunk_ptr[b + 1]; ++c) {
            const Chunk& ch = op.dense_chunks[c];
            nlst[ch.leaf].push_back({op.dense_off[b] + ch.off, op.dense_blocks[b].col0, op.dense_blocks[b].n});
        }
    std::vector<TcLeaf> lf(nl), ln(nl);
    std::vector<TcSeg> fs;
    std::vector<NearSeg> ns;
    for (int l = 0; l < nl; ++l) {
        const int m = op.plan.leaf_size[l];
        lf[l] = {op.plan.leaf_start[l], m, round8(m), (int)fs.size(), (int)fl[l].size(), 0};
        ln[l] = {op.plan.leaf_start[l], m, round8(m), (int)ns.size(), (int)nlst[l].size(), 0};
        fs.insert(fs.end(), fl[l].begin(), fl[l].end());
        ns.insert(ns.end(), nlst[l].begin(), nlst[l].end());
    }
    TcBlock* d_b;
    TcLeaf *d_lf, *d_ln;
    TcSeg* d_fs;
    NearSeg* d_ns;
    if ((rc = dev_alloc(op, &d_b, blocks.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_lf, lf.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_ln, ln.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_fs, fs.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_ns, ns.size(), err))) return rc;
    if ((rc = upload_async(op, d_b, blocks.data(), blocks.size(), err))) return rc;
    if ((rc = upload_async(op, d_lf, lf.data(), lf.size(), err))) return rc;
    if ((rc = upload_async(op, d_ln, ln.data(), ln.size(), err))) return rc;
    if ((rc = upload_async(op, d_fs, fs.data(), fs.size(), err))) return rc;
    if ((rc = upload_async(op, d_ns, ns.data(), ns.size(), err))) return rc;
    op.tc_blocks = d_b;
    op.tc_nblocks = (int)blocks.size();
    op.tc_leaf_far = d_lf;
    op.tc_leaf_near = d_ln;
    op.tc_segs_far = d_fs;
    op.tc_segs_near = d_ns;
    op.tc_wlen = wl;
    void* p = nullptr;
    if ((rc = dev_alloc(op, (char**)&p, (size_t)2 * 2 * op.F * op.N, err))) return rc;
    op.tc_xsplit = p;
    // W as 16-bit hi and lo parts, [F][r16] per block; the padding stays zero
    if ((rc = dev_alloc(op, (char**)&p, (size_t)2 * 2 * std::max<int64_t>(wl, 1), err))) return rc;
    op.tc_w = (float*)p;
    RT_CUDA_TRY(cudaMemsetAsync(p, 0, (size_t)2 * 2 * std::max<int64_t>(wl, 1), op.stream));
    if ((rc = dev_alloc(op, &op.tc_err, 1, err))) return rc;
    RT_CUDA_TRY(cudaMemsetAsync(op.tc_err, 0, sizeof(int), op.stream));
    const int smem = tc::kM * tc::kKT * 2 + 2 * op.F * tc::kKT * 2;
    RT_CUDA_TRY(cudaFuncSetAttribute(tc_phase1<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(tc_phase1<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(tc_phase2<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(tc_phase2<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    op.tc_enabled = 1;
    return RT_OK;
}

// Y = Gbar X for all F right-hand sides (tree order), tensor-core far field
int tc_apply(Operator& op, const float* X, float* Y, cudaStream_t s, std::string& err)
{
    const int N = op.N, F = op.F;
    const int64_t total = (int64_t)F * N;
    const int smem = tc::kM * tc::kKT * 2 + 2 * F * tc::kKT * 2;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g1 = (int)std::max<int64_t>(1, std::min<int64_t>(op.tc_nblocks, (int64_t)sms * 4));
    const int nl = (int)op.plan.leaf_start.size();
    const int xal = ((int64_t)N % 8 == 0) ? 1 : 0;   // 16-byte X loads need every row start aligned
    if (op.far_prec == RT_PREC_BF16) {
        using T = __nv_bfloat16;
        T* hi = (T*)op.tc_xsplit;
        T* lo = hi + total;
        T* whi = (T*)op.tc_w;
        T* wlo = whi + std::max<int64_t>(op.tc_wlen, 1);
        tc_split_kernel<T><<<(int)std::min<int64_t>((total + 255) / 256, sms * 16), 256, 0, s>>>(X, hi, lo, total);
        if (op.tc_nblocks > 0)
            tc_phase1<T><<<g1, tc::kThreads, smem, s>>>((const TcBlock*)op.tc_blocks, op.tc_nblocks, (const T*)op.d_far,
                                                        hi, lo, whi, wlo, N, F, xal, op.tc_err);
        tc_phase2<T><<<nl, tc::kThreads, smem, s>>>((const TcLeaf*)op.tc_leaf_far, (const TcSeg*)op.tc_segs_far,
                                                    (const T*)op.d_far, whi, wlo, Y, N, F, op.tc_err);
    } else {
        using T = __half;
        T* hi = (T*)op.tc_xsplit;
        T* lo = hi + total;
        T* whi = (T*)op.tc_w;
        T* wlo = whi + std::max<int64_t>(op.tc_wlen, 1);
        tc_split_kernel<T><<<(int)std::min<int64_t>((total + 255) / 256, sms * 16), 256, 0, s>>>(X, hi, lo, total);
        if (op.tc_nblocks > 0)
            tc_phase1<T><<<g1, tc::kThreads, smem, s>>>((const TcBlock*)op.tc_blocks, op.tc_nblocks, (const T*)op.d_far,
                                                        hi, lo, whi, wlo, N, F, xal, op.tc_err);
        tc_phase2<T><<<nl, tc::kThreads, smem, s>>>((const TcLeaf*)op.tc_leaf_far, (const TcSeg*)op.tc_segs_far,
                                                    (const T*)op.d_far, whi, wlo, Y, N, F, op.tc_err);
    }
    RT_CUDA_TRY(cudaGetLastError());
    near_mrhs<<<nl, 256, (size_t)64 * F * sizeof(float), s>>>((const TcLeaf*)op.tc_leaf_near,
                                                             (const NearSeg*)op.tc_segs_near, op.d_near, X, Y, N, F);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

int tc_check_error(Operator& op, std::string& err)
{
    if (!op.tc_enabled) return RT_OK;
    int h = 0;
    RT_CUDA_TRY(cudaMemcpyAsync(&h, op.tc_err, sizeof(int), cudaMemcpyDeviceToHost, op.stream));
    RT_CUDA_TRY(cudaStreamSynchronize(op.stream));
    if (h) {
        err = "tensor-core apply: an mbarrier wait timed out";
        return RT_ETIMEOUT;
    }
    return RT_OK;
}

}  // namespace rt
