// rt_tc.cu -- multi-right-hand-side H-matvec on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators) for one operator applied to F frequencies
// at once (kappa_nu = kappa(x) for every nu: one operator, F right-hand sides).
//
//   phase 1: W_b [r x F] = V_b^T X_c           far blocks stacked by column
//            cluster c: one M = 128 tile holds the V^T rows of several blocks
//            that share X_c, so each staged X_c tile serves 128 real rows
//   phase 2: Y_l [m x F] = sum_b U_{b,l} W_b + sum_near A_{b,l} X_c
//            one M = 64 TMEM tile per leaf l (m <= 64), the far and near
//            contributions accumulated in the same tile, Y written once
//
// Operands: the far factors U, V are stored in BF16 or FP16.  X, W and the
// FP32 near blocks are split into a 16-bit high part and a 16-bit remainder;
// the products high*high + high*low (+ low*high for the near blocks)
// accumulate in FP32, so the right-hand sides and the near field keep about 16
// significant bits.  Near-field products always use BF16 (its exponent range
// covers the entries); far products use the storage type.
//
// Shared-memory tiles use the canonical no-swizzle layouts (8-row x 16-byte
// core matrices).  A descriptor's leading byte offset is the distance between
// core matrices adjacent along K and its stride byte offset the distance along
// M/N, for K-major and MN-major operands alike.  U and the near blocks are
// stored with the row index contiguous ([k][i]), so they enter as MN-major A
// operands (instruction-descriptor bit 15).  An M = 64 accumulator holds row
// i in TMEM lane 32 (i / 16) + i % 16.
//
// Tiles stream through a three-stage shared-memory ring: 16-byte cp.async
// copies (zero-filled where a row or K index lies outside the data) or, for
// operands that are split on the fly, register loads; one elected thread
// issues the MMAs of a stage and commits them to that stage's mbarrier, which
// frees the stage for the copies two steps later.  Every mbarrier wait is
// bounded by a clock budget and reports a timeout through a flag.
#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rt_internal.h"

namespace rt {

namespace tc {

constexpr int kThreads = 256;    // 8 warps
constexpr int kKT = 64;          // K elements per stage
constexpr int kStages = 3;
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
// A MN-major when mn_a, B K-major, N and M dimensions
__device__ __forceinline__ uint32_t idesc_f16(int bf16, int mn_a, int M, int N)
{
    uint32_t d = 0;
    d |= 1u << 4;
    d |= (uint32_t)bf16 << 7;
    d |= (uint32_t)bf16 << 10;
    d |= (uint32_t)mn_a << 15;
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

// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// byte offset of (row, k) in a K-major tile of kKT columns (core matrix = 8 rows x 8 k)
__device__ __forceinline__ uint32_t kmaj(int row, int k)
{
    return (uint32_t)((row >> 3) * (kKT / 8 * 128) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
// byte offset of (i, k) in an MN-major tile of 64 rows (core matrix = 8 i x 8 k)
__device__ __forceinline__ uint32_t mnmaj64(int i, int k)
{
    return (uint32_t)((i >> 3) * 128 + (k >> 3) * 1024 + (k & 7) * 16 + (i & 7) * 2);
}

template <class T>
__device__ __forceinline__ T to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }
__device__ __forceinline__ float from16(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float from16(__half x) { return __half2float(x); }

// eight FP32 values -> 16-bit high parts and remainders, packed 16 bytes each
template <class T>
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo)
{
    T h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        h[j] = to16<T>(v[j]);
        l[j] = to16<T>(v[j] - from16(h[j]));
    }
    hi = *reinterpret_cast<const uint4*>(h);
    lo = *reinterpret_cast<const uint4*>(l);
}

// B operand from X: rows f < F, columns col0 + k0 + k (k < kvalid), zero
// beyond; K16 = kvalid rounded up to 16.  X rows are not 16-byte aligned at an
// arbitrary column, so each thread reads 8 scalars and writes 16 bytes.
template <class T>
__device__ __forceinline__ void stage_x(unsigned char* sBh, unsigned char* sBl, const float* __restrict__ X, int N,
                                        int F, int col, int kvalid, int K16)
{
    const int units = F * (K16 >> 3);
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
        const int f = u / (K16 >> 3), c = u - f * (K16 >> 3);
        const float* __restrict__ x = X + (int64_t)f * N + col + 8 * c;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 8 * c + j < kvalid ? __ldg(x + j) : 0.f;
        uint4 hi, lo;
        split8<T>(v, hi, lo);
        *reinterpret_cast<uint4*>(sBh + kmaj(f, 8 * c)) = hi;
        *reinterpret_cast<uint4*>(sBl + kmaj(f, 8 * c)) = lo;
    }
}

// B operand rows f < F from X already split into 16-bit parts, when every
// chunk start is 16-byte aligned (N and the cluster's first column multiples
// of 8): asynchronous copies, the part of a chunk beyond kvalid zero-filled
template <class T>
__device__ __forceinline__ void copy_x(unsigned char* sBh, unsigned char* sBl, const T* __restrict__ xh,
                                       const T* __restrict__ xl, int N, int F, int col, int kvalid, int K16)
{
    const int nc = K16 >> 3;
    for (int e = threadIdx.x; e < F * nc; e += blockDim.x) {
        const int f = e / nc, c = e - f * nc, k = 8 * c;
        const uint32_t nb = (uint32_t)(2 * max(0, min(8, kvalid - k)));
        const int64_t o = (int64_t)f * N + col + k;
        cp_async16(smem_addr(sBh + kmaj(f, k)), nb ? (const void*)(xh + o) : (const void*)xh, nb);
        cp_async16(smem_addr(sBl + kmaj(f, k)), nb ? (const void*)(xl + o) : (const void*)xl, nb);
    }
}

// per-stage mbarrier bookkeeping: commits and completed waits per stage
struct Ring {
    uint32_t bar0;                 // shared address of bar[0] (8 bytes apart)
    uint32_t committed[kStages];
    uint32_t waited[kStages];
    __device__ __forceinline__ uint32_t bar(int s) const { return bar0 + 8u * (uint32_t)s; }
    // wait until every commit on stage s has completed; false on timeout
    __device__ __forceinline__ bool drain(int s)
    {
        while (waited[s] < committed[s]) {
            if (!bar_wait(bar(s), waited[s] & 1u)) return false;
            ++waited[s];
        }
        return true;
    }
};

}  // namespace tc

// X (FP32, tree order, [F][N]) -> 16-bit high parts and remainders, same layout
template <class T>
__global__ void tc_split_x(const float* __restrict__ X, T* __restrict__ hi, T* __restrict__ lo, int64_t total)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const float x = X[e];
        const T h = tc::to16<T>(x);
        hi[e] = h;
        lo[e] = tc::to16<T>(x - tc::from16(h));
    }
}

// ---------------------------------------------------------------------------
// phase 1: W_b = V_b^T X_c, M = 128 tiles of V^T rows stacked by column cluster
// ---------------------------------------------------------------------------
struct TcRow {
    int64_t v;      // element offset of this V^T row in the far storage
    int64_t w;      // W index of (f = 0, this row); frequency f adds f * r8
    int r8, pad;    // W row length of the row's block (rank rounded up to 8)
};

struct TcTile {
    int col0, n, n8;    // the column cluster: first column, width, V^T row length
    int row0, nrows;    // rows [row0, row0 + nrows) of the row table
    int pad;
};

template <class T>
__global__ void __launch_bounds__(tc::kThreads) tc_phase1(const TcTile* __restrict__ tiles, int ntiles,
                                                          const TcRow* __restrict__ rows, const T* __restrict__ far,
                                                          const float* __restrict__ X, const T* __restrict__ xh,
                                                          const T* __restrict__ xl, T* __restrict__ whi,
                                                          T* __restrict__ wlo, int N, int F, int* __restrict__ err)
{
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int stage_bytes = 128 * kKT * 2 + 2 * F * kKT * 2;   // A (128 rows) | B high | B low
    __shared__ __align__(8) unsigned long long bars[kStages];
    __shared__ uint32_t s_tmem;
    __shared__ TcTile s_tile[3];
    __shared__ TcRow s_rows[3][128];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = F <= 32 ? 32 : (F <= 64 ? 64 : 128);
    if (warp == 0) tmem_alloc(smem_addr(&s_tmem), ncols);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) bar_init(smem_addr(&bars[s]));
        fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    Ring R{smem_addr(&bars[0]), {0, 0, 0}, {0, 0, 0}};
    const uint32_t idesc = idesc_f16(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, 0, 128, F);
    // this CTA's tiles: blockIdx.x + j gridDim.x; one stream of K steps runs
    // through all of them, the copies two steps ahead of the MMAs
    const int nitems = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    auto nsteps_of = [&](const TcTile& t) { return (t.n + kKT - 1) / kKT; };
    int lj = 0, lt = 0, gl = 0;   // copy cursor: item, step in item, global step
    int mj = 0, mt = 0, gm = 0;   // MMA cursor
    auto issue = [&]() {
        if (lj >= nitems) return;
        const int slot = lj % 3;
        if (lt == 0) {
            // the slot's previous tile (lj - 3) finished its epilogue: the copies run at most
            // two steps ahead of the MMAs and every tile has at least one step
            const TcTile t = tiles[blockIdx.x + lj * gridDim.x];
            for (int r = tid; r < 128; r += blockDim.x) s_rows[slot][r] = r < t.nrows ? rows[t.row0 + r] : TcRow{-1, 0, 0, 0};
            if (tid == 0) s_tile[slot] = t;
            __syncthreads();
        }
        const TcTile& Tl = s_tile[slot];
        unsigned char* sA = smem + (gl % kStages) * stage_bytes;
        unsigned char* sBh = sA + 128 * kKT * 2;
        unsigned char* sBl = sBh + F * kKT * 2;
        const int k0 = lt * kKT, kvalid = min(kKT, Tl.n - k0), K16 = (kvalid + 15) & ~15, nc = K16 >> 3;
        // V^T rows are zero-padded to n8; zeros beyond n8, for padding rows (v < 0) and
        // below the tile's rows
        for (int e = tid; e < 128 * nc; e += blockDim.x) {
            const int row = e / nc, c = e - row * nc, k = k0 + 8 * c;
            const int64_t v = s_rows[slot][row].v;
            const bool in = k < Tl.n8 && v >= 0;
            cp_async16(smem_addr(sA + kmaj(row, 8 * c)), in ? (const void*)(far + v + k) : (const void*)far, in ? 16u : 0u);
        }
        if (xh) copy_x<T>(sBh, sBl, xh, xl, N, F, Tl.col0 + k0, kvalid, K16);
        cp_async_commit();
        if (!xh) stage_x<T>(sBh, sBl, X, N, F, Tl.col0 + k0, kvalid, K16);
        ++gl;
        if (++lt == nsteps_of(Tl)) {
            ++lj;
            lt = 0;
        }
    };
    bool ok = true;
    issue();
    issue();
    while (mj < nitems) {
        const int s = gm % kStages;
        if (gl - gm - 1 >= 1) cp_async_wait<1>();
        else cp_async_wait<0>();
        fence_async_smem();
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        const TcTile& Tl = s_tile[mj % 3];
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_addr(smem + s * stage_bytes);
            const uint32_t bh0 = a0 + 128 * kKT * 2, bl0 = bh0 + F * kKT * 2;
            const int nks = (min(kKT, Tl.n - mt * kKT) + 15) >> 4;
            for (int ks = 0; ks < nks; ++ks) {
                const uint64_t da = sdesc(a0 + ks * 256, 128, 1024);
                mma_f16(tmem, da, sdesc(bh0 + ks * 256, 128, 1024), idesc, (mt > 0 || ks > 0) ? 1u : 0u);
                mma_f16(tmem, da, sdesc(bl0 + ks * 256, 128, 1024), idesc, 1u);
            }
            mma_commit(R.bar(s));
        }
        R.committed[s]++;
        const bool last = mt + 1 == nsteps_of(Tl);
        // copies of step gm + 2 into the stage that step gm - 1 used
        const bool more = gl == gm + 2 && lj < nitems;
        bool fail = more && !R.drain(gl % kStages);
        if (__syncthreads_or(fail)) {
            ok = false;
            break;
        }
        if (more) issue();
        if (last) {
            fail = !R.drain(s);   // this tile's last MMAs are done
            tc_fence_after();
        }
        if (__syncthreads_or(fail)) {
            ok = false;
            break;
        }
        if (last) {
            // epilogue: warp w reads TMEM lanes 32 (w % 4) + lane = tile rows; column chunks
            // alternate between the two warps of a lane quarter; W as high and low parts
            const int row = (warp & 3) * 32 + lane;
            const TcRow rw = s_rows[mj % 3][row];
            for (int c0 = (warp >> 2) * 16; c0 < F; c0 += 32) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
                if (row < Tl.nrows) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const T h = to16<T>(v[k]);
                        const int64_t idx = rw.w + (int64_t)(c0 + k) * rw.r8;
                        whi[idx] = h;
                        wlo[idx] = to16<T>(v[k] - from16(h));
                    }
                }
            }
            tc_fence_before();
            __syncthreads();   // TMEM read before the next tile's first MMA overwrites it
            ++mj;
            mt = 0;
        } else {
            ++mt;
        }
        ++gm;
    }
    cp_async_wait<0>();
    bool bad = !ok;
    for (int s = 0; s < kStages; ++s) bad = bad || !R.drain(s);
    if (bad && tid == 0) atomicOr(err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// phase 2: per leaf, Y_l = sum_far U_{b,l} W_b + sum_near A_{b,l} X_c (M = 64)
// ---------------------------------------------------------------------------
struct TcSeg {
    int64_t a;      // far: element offset of the leaf chunk U^T [r][m8]; near: of A^T [n][m8] (FP32)
    int64_t w;      // far: W offset of the block ([F][r8], high and low arrays)
    int count;      // far: r; near: n (block columns)
    int kind;       // 0 far, 1 near
    int col0;       // near: first column of the block
    int r8;         // far: W row length
};

struct TcLeaf {
    int row0, m, m8, seg0, nseg, nsteps;
};

template <class T>
__global__ void __launch_bounds__(tc::kThreads) tc_phase2(const TcLeaf* __restrict__ leaves, int nleaves,
                                                          const TcSeg* __restrict__ segs, const T* __restrict__ far,
                                                          const float* __restrict__ nearp, const T* __restrict__ whi,
                                                          const T* __restrict__ wlo, const float* __restrict__ X,
                                                          const __nv_bfloat16* __restrict__ xh,
                                                          const __nv_bfloat16* __restrict__ xl, float* __restrict__ Y,
                                                          int N, int F, int* __restrict__ err)
{
    using namespace tc;
    using B16 = __nv_bfloat16;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int stage_bytes = 2 * 64 * kKT * 2 + 2 * F * kKT * 2;   // A high | A low | B high | B low
    __shared__ __align__(8) unsigned long long bars[kStages];
    __shared__ uint32_t s_tmem;
    __shared__ TcLeaf s_leaf[3];
    __shared__ int s_kind[kStages], s_k16[kStages];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = F <= 32 ? 32 : (F <= 64 ? 64 : 128);
    if (warp == 0) tmem_alloc(smem_addr(&s_tmem), ncols);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) bar_init(smem_addr(&bars[s]));
        fence_async_smem();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    Ring R{smem_addr(&bars[0]), {0, 0, 0}, {0, 0, 0}};
    const uint32_t idesc_far = idesc_f16(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, 1, 64, F);
    const uint32_t idesc_near = idesc_f16(1, 1, 64, F);
    // this CTA's leaves: blockIdx.x + j gridDim.x (tree order, every leaf has >= 1 step);
    // one stream of steps runs through all of them, the copies two steps ahead
    const int nitems = blockIdx.x < nleaves ? (nleaves - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    int lj = 0, lt = 0, gl = 0, cs = 0, ck = 0;   // copy cursor: item, step, global step, segment, K offset
    int mj = 0, mt = 0, gm = 0;                   // MMA cursor
    auto issue = [&]() {
        if (lj >= nitems) return;
        const int slot = lj % 3;
        if (lt == 0) {
            if (tid == 0) s_leaf[slot] = leaves[blockIdx.x + lj * gridDim.x];
            cs = 0;
            ck = 0;
            __syncthreads();
        }
        const TcLeaf& L = s_leaf[slot];
        const int st = gl % kStages;
        unsigned char* sAh = smem + st * stage_bytes;
        unsigned char* sBh = sAh + 2 * 64 * kKT * 2;
        unsigned char* sBl = sBh + F * kKT * 2;
        const TcSeg S = segs[L.seg0 + cs];
        const int k0 = ck;
        int K16;
        if (S.kind == 0) {
            const int r16 = (S.count + 15) & ~15;
            K16 = min(kKT, r16 - k0);
            // A = U^T rows k (8 leaf rows per 16 bytes) -> MN-major; zeros beyond r
            const int ng = L.m8 >> 3;
            for (int e = tid; e < K16 * 8; e += blockDim.x) {
                const int kk = e >> 3, g = e & 7, k = k0 + kk;
                const bool in = g < ng && k < S.count;
                cp_async16(smem_addr(sAh + mnmaj64(8 * g, kk)),
                           in ? (const void*)(far + S.a + (int64_t)k * L.m8 + 8 * g) : (const void*)far, in ? 16u : 0u);
            }
            // B = W_b rows f (K-major), zero-padded from r8 on
            const int nc = K16 >> 3;
            for (int e = tid; e < F * nc; e += blockDim.x) {
                const int f = e / nc, c = e - f * nc, k = k0 + 8 * c;
                const bool in = k < S.r8;
                const int64_t o = S.w + (int64_t)f * S.r8 + k;
                cp_async16(smem_addr(sBh + kmaj(f, 8 * c)), in ? (const void*)(whi + o) : (const void*)whi, in ? 16u : 0u);
                cp_async16(smem_addr(sBl + kmaj(f, 8 * c)), in ? (const void*)(wlo + o) : (const void*)wlo, in ? 16u : 0u);
            }
            if (k0 + kKT >= r16) {
                ++cs;
                ck = 0;
            } else {
                ck += kKT;
            }
            cp_async_commit();
        } else {
            const int kvalid = min(kKT, S.count - k0);
            K16 = (kvalid + 15) & ~15;
            // A = near block rows k (FP32 [k][m8]) copied raw into the A area as [kk][64]
            // floats; split into BF16 parts in place just before the MMAs
            for (int e = tid; e < K16 * 16; e += blockDim.x) {
                const int kk = e >> 4, q = e & 15;
                const bool in = kk < kvalid && 4 * q < L.m8;
                cp_async16(smem_addr(sAh + kk * 256 + q * 16),
                           in ? (const void*)(nearp + S.a + (int64_t)(k0 + kk) * L.m8 + 4 * q) : (const void*)nearp,
                           in ? 16u : 0u);
            }
            if (xh) copy_x<B16>(sBh, sBl, xh, xl, N, F, S.col0 + k0, kvalid, K16);
            cp_async_commit();
            if (!xh) stage_x<B16>(sBh, sBl, X, N, F, S.col0 + k0, kvalid, K16);
            if (k0 + kKT >= S.count) {
                ++cs;
                ck = 0;
            } else {
                ck += kKT;
            }
        }
        if (tid == 0) {
            s_kind[st] = S.kind;
            s_k16[st] = K16;
        }
        ++gl;
        if (++lt == L.nsteps) {
            ++lj;
            lt = 0;
        }
    };
    bool ok = true;
    issue();
    issue();
    bool started = false;
    while (mj < nitems) {
        const int s = gm % kStages;
        if (gl - gm - 1 >= 1) cp_async_wait<1>();
        else cp_async_wait<0>();
        fence_async_smem();
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        if (s_kind[s] == 1) {
            // near step: raw FP32 [kk][64] -> BF16 high / low MN-major tiles, in place
            unsigned char* sA = smem + s * stage_bytes;
            const int K16 = s_k16[s];
            float v[2][8];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int e = tid + j * (int)blockDim.x;
                if (e < K16 * 8) {
                    const float* src = reinterpret_cast<const float*>(sA + (e >> 3) * 256 + (e & 7) * 32);
                    const float4 a = *reinterpret_cast<const float4*>(src);
                    const float4 b = *reinterpret_cast<const float4*>(src + 4);
                    v[j][0] = a.x; v[j][1] = a.y; v[j][2] = a.z; v[j][3] = a.w;
                    v[j][4] = b.x; v[j][5] = b.y; v[j][6] = b.z; v[j][7] = b.w;
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int e = tid + j * (int)blockDim.x;
                if (e < K16 * 8) {
                    uint4 hi, lo;
                    split8<B16>(v[j], hi, lo);
                    *reinterpret_cast<uint4*>(sA + mnmaj64(8 * (e & 7), e >> 3)) = hi;
                    *reinterpret_cast<uint4*>(sA + 64 * kKT * 2 + mnmaj64(8 * (e & 7), e >> 3)) = lo;
                }
            }
            fence_async_smem();
            __syncthreads();
        }
        const TcLeaf& L = s_leaf[mj % 3];
        if (tid == 0) {
            tc_fence_after();
            const uint32_t ah = smem_addr(smem + s * stage_bytes), al = ah + 64 * kKT * 2;
            const uint32_t bh = al + 64 * kKT * 2, bl = bh + F * kKT * 2;
            const int nks = s_k16[s] >> 4;
            for (int ks = 0; ks < nks; ++ks) {
                const uint64_t dah = sdesc(ah + ks * 2048, 1024, 128);
                const uint64_t dbh = sdesc(bh + ks * 256, 128, 1024), dbl = sdesc(bl + ks * 256, 128, 1024);
                if (s_kind[s] == 0) {
                    mma_f16(tmem, dah, dbh, idesc_far, started ? 1u : 0u);
                    mma_f16(tmem, dah, dbl, idesc_far, 1u);
                } else {
                    mma_f16(tmem, dah, dbh, idesc_near, started ? 1u : 0u);
                    mma_f16(tmem, dah, dbl, idesc_near, 1u);
                    mma_f16(tmem, sdesc(al + ks * 2048, 1024, 128), dbh, idesc_near, 1u);
                }
                started = true;
            }
            mma_commit(R.bar(s));
        }
        R.committed[s]++;
        const bool last = mt + 1 == L.nsteps;
        const bool more = gl == gm + 2 && lj < nitems;
        bool fail = more && !R.drain(gl % kStages);
        if (__syncthreads_or(fail)) {
            ok = false;
            break;
        }
        if (more) issue();
        if (last) {
            fail = !R.drain(s);   // this leaf's last MMAs are done
            tc_fence_after();
        }
        if (__syncthreads_or(fail)) {
            ok = false;
            break;
        }
        if (last) {
            // leaf row i sits in TMEM lane 32 (i / 16) + i % 16; warp w reads its lane quarter
            // (rows 16 (w % 4) .. +15 in lanes 0..15); column chunks alternate between warps w, w + 4
            const int row = (warp & 3) * 16 + lane;
            for (int c0 = (warp >> 2) * 16; c0 < F; c0 += 32) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
                if (lane < 16 && row < L.m) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) Y[(int64_t)(c0 + k) * N + L.row0 + row] = v[k];
                }
            }
            tc_fence_before();
            __syncthreads();   // TMEM read before the next leaf's first MMA overwrites it
            if (tid == 0) started = false;
            ++mj;
            mt = 0;
        } else {
            ++mt;
        }
        ++gm;
    }
    cp_async_wait<0>();
    bool bad = !ok;
    for (int s = 0; s < kStages; ++s) bad = bad || !R.drain(s);
    if (bad && tid == 0) atomicOr(err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int tc_prepare(Operator& op, std::string& err)
{
    op.tc_enabled = 0;
    if (op.tc_off) return RT_OK;
    int rc0 = tc2_prepare(op, err);   // the streamed form, when it applies (F = 64)
    if (rc0 || op.tc2) return rc0;
    if (op.mode != RT_MODE_HMATRIX || op.G != 1 || op.F % 16 != 0 || op.F < 16 || op.F > 128) return RT_OK;
    if (op.far_prec != RT_PREC_BF16 && op.far_prec != RT_PREC_F16) return RT_OK;
    for (int l = 0; l < (int)op.plan.leaf_size.size(); ++l)
        if (op.plan.leaf_size[l] > 64) return RT_OK;
    int rc;
    const int F = op.F;
    // W layout: block b at w_base[b], [F][r8]
    std::vector<int64_t> w_base(op.n_far);
    int64_t wl = 0;
    for (int b = 0; b < op.n_far; ++b) {
        w_base[b] = wl;
        wl += (int64_t)F * round8(op.rank[b]);
    }
    // phase 1: rows of the blocks of each column cluster, stacked into tiles of 128
    const int nc = (int)op.plan.clusters.size();
    std::vector<std::vector<int>> by_col(nc);
    for (int b = 0; b < op.n_far; ++b) by_col[op.far_blocks[b].sc].push_back(b);
    std::vector<TcRow> rows;
    std::vector<TcTile> tiles;
    for (int c = 0; c < nc; ++c) {
        if (by_col[c].empty()) continue;
        const FarBlock& f0 = op.far_blocks[by_col[c][0]];
        const int first = (int)rows.size();
        for (int b : by_col[c]) {
            const FarBlock& fb = op.far_blocks[b];
            // r8 rows per block: the padding rows (v = -1) produce zeros, so every W element
            // is written and no partly written sector is read back
            for (int k = 0; k < round8(op.rank[b]); ++k)
                rows.push_back({k < op.rank[b] ? op.far_v_off[b] + (int64_t)k * round8(fb.n) : -1, w_base[b] + k,
                                round8(op.rank[b]), 0});
        }
        for (int r0 = first; r0 < (int)rows.size(); r0 += 128)
            tiles.push_back({f0.col0, f0.n, round8(f0.n), r0, std::min(128, (int)rows.size() - r0), 0});
    }
    std::stable_sort(tiles.begin(), tiles.end(), [](const TcTile& a, const TcTile& b) { return a.n > b.n; });
    // phase 2: per leaf, the far chunks and near chunks over its rows
    const int nl = (int)op.plan.leaf_start.size();
    std::vector<std::vector<TcSeg>> per(nl);
    for (int b = 0; b < op.n_far; ++b)
        for (int c = op.far_chunk_ptr[b]; c < op.far_chunk_ptr[b + 1]; ++c) {
            const Chunk& ch = op.far_chunks[c];
            per[ch.leaf].push_back({op.far_u_off[b] + ch.off, w_base[b], op.rank[b], 0, 0, round8(op.rank[b])});
        }
    for (int b = 0; b < op.n_near; ++b)
        for (int c = op.dense_chunk_ptr[b]; c < op.dense_chunk_ptr[b + 1]; ++c) {
            const Chunk& ch = op.dense_chunks[c];
            per[ch.leaf].push_back({op.dense_off[b] + ch.off, 0, op.dense_blocks[b].n, 1, op.dense_blocks[b].col0, 0});
        }
    std::vector<TcLeaf> leaves(nl);
    std::vector<TcSeg> segs;
    for (int l = 0; l < nl; ++l) {
        int steps = 0;
        for (const TcSeg& s : per[l])
            steps += s.kind == 0 ? ((s.count + 15) / 16 * 16 + tc::kKT - 1) / tc::kKT : (s.count + tc::kKT - 1) / tc::kKT;
        if (steps == 0) return RT_OK;   // a leaf without blocks: keep the CUDA-core apply
        const int m = op.plan.leaf_size[l];
        leaves[l] = {op.plan.leaf_start[l], m, round8(m), (int)segs.size(), (int)per[l].size(), steps};
        segs.insert(segs.end(), per[l].begin(), per[l].end());
    }
    // leaves stay in tree order: neighbouring leaves share most far blocks, so the W
    // panels they read are still in L2
    TcTile* d_t;
    TcRow* d_r;
    TcLeaf* d_l;
    TcSeg* d_s;
    if ((rc = dev_alloc(op, &d_t, tiles.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_r, rows.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_l, leaves.size(), err))) return rc;
    if ((rc = dev_alloc(op, &d_s, segs.size(), err))) return rc;
    if ((rc = upload_async(op, d_t, tiles.data(), tiles.size(), err))) return rc;
    if ((rc = upload_async(op, d_r, rows.data(), rows.size(), err))) return rc;
    if ((rc = upload_async(op, d_l, leaves.data(), leaves.size(), err))) return rc;
    if ((rc = upload_async(op, d_s, segs.data(), segs.size(), err))) return rc;
    op.tc_tiles = d_t;
    op.tc_rows = d_r;
    op.tc_leaves = d_l;
    op.tc_segs = d_s;
    op.tc_ntiles = (int)tiles.size();
    op.tc_nleaves = nl;
    op.tc_wlen = std::max<int64_t>(wl, 8);
    char* w = nullptr;
    if ((rc = dev_alloc(op, &w, (size_t)2 * 2 * op.tc_wlen, err))) return rc;
    RT_CUDA_TRY(cudaMemsetAsync(w, 0, (size_t)2 * 2 * op.tc_wlen, op.stream));   // padding stays zero
    op.tc_w = w;
    // X split once per apply into 16-bit parts when every cluster starts on a
    // 16-byte boundary (then B tiles are plain asynchronous copies)
    op.tc_xal = op.N % 8 == 0;
    for (int l = 0; l < nl && op.tc_xal; ++l) op.tc_xal = op.plan.leaf_start[l] % 8 == 0;
    if (op.tc_xal) {
        const int nparts = op.far_prec == RT_PREC_F16 ? 4 : 2;   // BF16 (near) and, for FP16 far, FP16 parts
        char* xs = nullptr;
        if ((rc = dev_alloc(op, &xs, (size_t)nparts * 2 * F * op.N, err))) return rc;
        op.tc_xsplit = xs;
    }
    if ((rc = dev_alloc(op, &op.tc_err, 1, err))) return rc;
    RT_CUDA_TRY(cudaMemsetAsync(op.tc_err, 0, sizeof(int), op.stream));
    const int st = tc::kStages;
    const int smem1 = st * (128 * tc::kKT * 2 + 2 * F * tc::kKT * 2);
    const int smem2 = st * (2 * 64 * tc::kKT * 2 + 2 * F * tc::kKT * 2);
    RT_CUDA_TRY(cudaFuncSetAttribute(tc_phase1<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1));
    RT_CUDA_TRY(cudaFuncSetAttribute(tc_phase1<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1));
    RT_CUDA_TRY(cudaFuncSetAttribute(tc_phase2<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    RT_CUDA_TRY(cudaFuncSetAttribute(tc_phase2<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    op.tc_enabled = 1;
    return RT_OK;
}

template <class T>
static int tc_launch(Operator& op, const float* X, float* Y, cudaStream_t s, std::string& err)
{
    const int N = op.N, F = op.F;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int st = tc::kStages;
    const int smem1 = st * (128 * tc::kKT * 2 + 2 * F * tc::kKT * 2);
    const int smem2 = st * (2 * 64 * tc::kKT * 2 + 2 * F * tc::kKT * 2);
    const int per_sm = F <= 64 ? 2 : 1;
    T* whi = (T*)op.tc_w;
    T* wlo = whi + op.tc_wlen;
    const int64_t total = (int64_t)F * N;
    const __nv_bfloat16 *bh = nullptr, *bl = nullptr;
    const T *th = nullptr, *tl = nullptr;
    if (op.tc_xal) {
        __nv_bfloat16* b = (__nv_bfloat16*)op.tc_xsplit;
        const int gs = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 16);
        tc_split_x<__nv_bfloat16><<<gs, 256, 0, s>>>(X, b, b + total, total);
        bh = b;
        bl = b + total;
        if (std::is_same<T, __half>::value) {
            __half* h = (__half*)(b + 2 * total);
            tc_split_x<__half><<<gs, 256, 0, s>>>(X, h, h + total, total);
            th = (const T*)h;
            tl = (const T*)(h + total);
        } else {
            th = (const T*)bh;
            tl = (const T*)bl;
        }
        RT_CUDA_TRY(cudaGetLastError());
    }
    if (op.tc_ntiles > 0) {
        const int g1 = std::max(1, std::min(op.tc_ntiles, per_sm * sms));
        tc_phase1<T><<<g1, tc::kThreads, smem1, s>>>((const TcTile*)op.tc_tiles, op.tc_ntiles, (const TcRow*)op.tc_rows,
                                                   (const T*)op.d_far, X, th, tl, whi, wlo, N, F, op.tc_err);
        RT_CUDA_TRY(cudaGetLastError());
    }
    const int g2 = std::max(1, std::min(op.tc_nleaves, per_sm * sms));
    tc_phase2<T><<<g2, tc::kThreads, smem2, s>>>((const TcLeaf*)op.tc_leaves, op.tc_nleaves, (const TcSeg*)op.tc_segs,
                                               (const T*)op.d_far, op.d_near, whi, wlo, X, bh, bl, Y, N, F,
                                               op.tc_err);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

// Y = Gbar X for all F right-hand sides (tree order), tensor cores
int tc_apply(Operator& op, const float* X, float* Y, cudaStream_t s, std::string& err)
{
    if (op.tc2) return tc2_apply(op, X, Y, s, err);
    if (op.far_prec == RT_PREC_BF16) return tc_launch<__nv_bfloat16>(op, X, Y, s, err);
    return tc_launch<__half>(op, X, Y, s, err);
}

int tc_check_error(Operator& op, cudaStream_t s, std::string& err)
{
    if (!op.tc_enabled) return RT_OK;
    int h = 0;
    RT_CUDA_TRY(cudaMemcpyAsync(&h, op.tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
        err = "tensor-core apply: an mbarrier wait timed out";
        return RT_ETIMEOUT;
    }
    return RT_OK;
}

}  // namespace rt
