// rt_tc2.cu -- streamed tcgen05 apply of one operator to 64 right-hand sides
// (kappa_nu = kappa(x) for every channel: one operator group, F = 64).
//
//   phase 1: W = V^T X per column cluster c.  The V^T rows of every far block
//            with column cluster c are stacked into M = 128 tiles; K runs over
//            c's columns in steps of 64; N = 64 right-hand sides.
//   phase 2: per leaf l (M = 64 rows): Y_l = sum_b U_{b,l} W_b + sum_near A X_c
//            as one K sequence: the rank terms of every far block over l, then
//            the columns of every near block; Y_l is written once (row
//            ownership, no atomics).
//
// Operands never need re-arranging on the SM.  At build time every operator
// row is written to an image in the exact byte order of a 128-byte-swizzled
// shared-memory tile (a 64-element row of 128 bytes, its 16-byte chunks
// permuted by the row's position mod 8), and phase 1 writes W the same way.
// Each pipeline stage is then a handful of cp.async.bulk copies of whole rows:
//   phase 1: the tile's V^T rows for this 64-column window (K-major A) and the
//            64 rows of X^T of that window (MN-major B);
//   phase 2: runs of U^T rows (MN-major A, i contiguous) with the matching W
//            rows (MN-major B, frequency contiguous), or near-block rows
//            (BF16 high and low parts) with the matching X^T rows.
// A swizzled row can only land on a shared-memory row of the same phase, so
// each far block starts in its leaf's K sequence at a position congruent to
// its first W row mod 8 (near blocks: to their first column).  Blocks are
// ordered greedily to match; the few remaining gap rows, and the rows between
// the last used one and the step's MMA extent, are zero-filled in A by copies
// from a zero buffer (the B rows there may hold stale finite data).
//
// X enters scaled by a power of two s with max|X s| in [0.5, 1), split into
// 16-bit high and low parts (X^T, [row][64]); W is stored as the far type's
// high part (and low part for BF16, or during refinement sweeps); Y = D / s.
// Products accumulate in FP32 in TMEM (two accumulators per CTA, so the
// epilogue of one tile or leaf overlaps the MMAs of the next).
//
// Warp roles (two persistent CTAs per SM): warps 0 .. P-1 produce, one ring
// slot each (bulk copies into the slot, completion on its "full" mbarrier; the
// record of the slot's next stage is read one stage ahead), warp P issues the
// MMAs (one lane) and commits them to the stage's "empty" mbarrier and, at the
// end of a tile or leaf, to the accumulator's "full" mbarrier, and the last
// warps are the epilogue (TMEM -> registers -> W or Y).  With stages of 64 K
// rows and N = 64, the single issuing thread, not the tensor pipe, bounds a
// CTA, hence two CTAs per SM; phase 2 also rotates consecutive K slices over
// several accumulators, summed in the epilogue.  Every wait is bounded; a wait
// that gives up raises a shared abort flag that ends every role's loop, sets
// *err, and the CTA drains its copies and MMAs (bounded) before it frees TMEM.
#include <algorithm>
#include <climits>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rt_bulk.cuh"
#include "rt_internal.h"
#include "rt_tcgen05.cuh"

namespace rt {

namespace t2 {
constexpr int kF = 64;               // right-hand sides
constexpr int kRowB = 128;           // bytes of one 64-element 16-bit row
constexpr int kRingBytes = 196608;   // shared memory for the stage ring
constexpr int kMaxStages = 8;
constexpr int kCtasPerSm = 2;        // phase-1 TMEM: 4 x 64 columns per CTA; phase 2: 2 x (4 / kCtasPerSm) x 64
constexpr int kZeroBytes = 8192;
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz
}  // namespace t2

struct T2Tile {       // phase-1 tile
    int64_t vimg;     // byte offset of step 0's rows in the V^T image (steps follow, R rows each)
    int64_t wrow0;    // W row of tile row 0
    int R, steps;     // rows (1..128), 64-column windows
    int xrow0, pad;   // X^T row of window 0's first column
};

struct T2Leaf {
    int row0, m, step0, nsteps;
    int nslices;     // 16-row K slices of the leaf (they rotate over the accumulators)
    int pad[3];
};

struct T2Step {
    int piece0, np, k16, kind;   // kind 0: far (U W), 1: near (A X)
};

struct T2Piece {      // one bulk copy into a stage
    int64_t src;      // byte offset in array `arr`
    int dst;          // byte offset in the stage
    uint32_t info;    // bytes | arr << 24 | flags << 29
};

enum { T2_UHI = 0, T2_ULO, T2_NHI, T2_NLO, T2_WHI, T2_WLO, T2_XHI, T2_XLO, T2_ZERO, T2_NARR };
constexpr uint32_t kT2FlagLo = 1;   // copied only in refinement sweeps (U low parts)
constexpr uint32_t kT2FlagW2 = 2;   // copied only when W has a low part

struct T2Arrays {
    const unsigned char* a[T2_NARR];
};

// phase-2 stage layout: A high | A low | B high | B low, 8 KB each
constexpr int kT2A = 0, kT2AL = 8192, kT2B = 16384, kT2BL = 24576, kT2Stage2 = 32768;

// ---- small device helpers ---------------------------------------------------
struct T2Ctl {
    uint64_t full[t2::kMaxStages], empty[t2::kMaxStages];
    uint64_t accf[4], acce[4];
    uint64_t drain;
    int meta_k16[t2::kMaxStages], meta_kind[t2::kMaxStages];
    uint32_t tmem;
    uint32_t hint;      // suspend-time hint (ns) of the pipeline waits
    volatile int abort;
};

// bounded wait that also gives up when another role raised the abort flag
__device__ __forceinline__ bool t2_wait(uint32_t bar, uint32_t parity, T2Ctl& C, uint32_t hint)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done = 0;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(hint)
            : "memory");
        if (done) return true;
        if (C.abort) return false;
        if (clock64() - t0 > t2::kWaitCycles) {
            C.abort = 1;
            return false;
        }
    }
}

__device__ __forceinline__ unsigned char* t2_ring()
{
    extern __shared__ unsigned char t2_dyn[];
    const uint32_t a = t5::smem_u32(t2_dyn);
    return t2_dyn + (((a + 1023u) & ~1023u) - a);
}

template <class T>
__device__ __forceinline__ T t2_to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 t2_to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half t2_to16<__half>(float x) { return __float2half_rn(x); }
__device__ __forceinline__ float t2_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float t2_f(__half x) { return __half2float(x); }

// eight values -> 16-bit high parts (and remainders), 16 bytes each
template <class T>
__device__ __forceinline__ void t2_split8(const float* v, uint4& hi, uint4& lo)
{
    T h[8], l[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        h[j] = t2_to16<T>(v[j]);
        l[j] = t2_to16<T>(v[j] - t2_f(h[j]));
    }
    hi = *reinterpret_cast<const uint4*>(h);
    lo = *reinterpret_cast<const uint4*>(l);
}

// Warp layout of both kernels: warps 0 .. P-1 produce (warp p fills ring slot p
// for stages p, p + P, p + 2P, ... of the CTA, so the latency of reading a
// stage's record and issuing its copies is spread over P warps), warp P issues
// the MMAs, warps P+1 .. P+4 are the epilogue (any four consecutive warps cover
// the four TMEM lane quarters).
__device__ __forceinline__ int t2_mma_warp(int nst) { return nst; }

// common set-up: barriers, zeroed ring, TMEM (the MMA warp allocates)
__device__ __forceinline__ void t2_setup(T2Ctl& C, int nst, int ring_bytes, int ncols, uint32_t hint)
{
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            bulk::bar_init(t5::smem_u32(&C.full[s]), 1);
            bulk::bar_init(t5::smem_u32(&C.empty[s]), 1);
        }
        C.hint = hint;
        for (int b = 0; b < 4; ++b) {
            bulk::bar_init(t5::smem_u32(&C.accf[b]), 1);
            bulk::bar_init(t5::smem_u32(&C.acce[b]), 4);
        }
        bulk::bar_init(t5::smem_u32(&C.drain), 1);
        C.abort = 0;
        bulk::fence_init();
    }
    // stale rows of a stage are multiplied by zeros: keep them finite from the start
    uint4* r = reinterpret_cast<uint4*>(t2_ring());
    for (int k = threadIdx.x; k < ring_bytes / 16; k += blockDim.x) r[k] = make_uint4(0, 0, 0, 0);
    t5::fence_async_smem();
    if (warp == t2_mma_warp(nst)) t5::tmem_alloc(t5::smem_u32(&C.tmem), (uint32_t)ncols);
    t5::fence_before();
    __syncthreads();
    t5::fence_after();
}

// end of a kernel: every role has left its loop.  The MMA lane waits (bounded)
// for its last MMAs, each producer for the copies of its slot's last use; then
// TMEM is freed.  `issued` = stages this producer warp filled.
__device__ __forceinline__ void t2_teardown(T2Ctl& C, int nst, uint32_t issued, int ncols, int* err)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == t2_mma_warp(nst) && lane == 0) {
        t5::commit(t5::smem_u32(&C.drain));
        const long long t0 = clock64();
        for (;;) {
            uint32_t done = 0;
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(t5::smem_u32(&C.drain)), "r"(0u), "r"(bulk::kSuspendNs)
                : "memory");
            if (done || clock64() - t0 > t2::kWaitCycles) break;
        }
    }
    if (warp < nst && lane == 0 && issued > 0)   // a wait on an already completed phase returns at once
        bulk::wait(t5::smem_u32(&C.full[warp]), (issued - 1) & 1u);
    t5::fence_before();
    __syncthreads();
    if (C.abort && threadIdx.x == 0) atomicExch(err, 1);
    if (warp == t2_mma_warp(nst)) t5::tmem_dealloc(C.tmem, (uint32_t)ncols);
}

// ---------------------------------------------------------------------------
// X -> scale s and the split X^T rows (both 16-bit types as needed)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) t2_xmax(const float* __restrict__ X, int64_t total, unsigned* __restrict__ mx)
{
    __shared__ unsigned red[8];
    unsigned m = 0;
    const int64_t n4 = total >> 2;
    const float4* X4 = reinterpret_cast<const float4*>(X);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = X4[e];
        m = max(max(m, __float_as_uint(fabsf(v.x))), max(__float_as_uint(fabsf(v.y)), __float_as_uint(fabsf(v.z))));
        m = max(m, __float_as_uint(fabsf(v.w)));
    }
    for (int64_t e = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(X[e])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
        atomicMax(mx, m);
    }
}

// thread (column j, chunk c): frequencies 8c..8c+7 of column j -> 16 bytes of
// row j of X^T (chunk position c ^ (j mod 8)), high and low parts
template <class T>
__global__ void t2_xsplit(const float* __restrict__ X, int N, const unsigned* __restrict__ mx,
                          float* __restrict__ scale, unsigned char* __restrict__ hi, unsigned char* __restrict__ lo)
{
    const float m = __uint_as_float(*mx);
    const float s = (m > 0.f && isfinite(m)) ? exp2f((float)(-ilogbf(m) - 1)) : 1.f;
    if (blockIdx.x == 0 && threadIdx.x == 0 && scale) {
        scale[0] = s;
        scale[1] = 1.f / s;
    }
    const int64_t total = (int64_t)N * 8;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / N), j = (int)(e % N);
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = X[(int64_t)(8 * c + q) * N + j] * s;
        uint4 h, l;
        t2_split8<T>(v, h, l);
        const int64_t o = (int64_t)j * t2::kRowB + ((c ^ (j & 7)) << 4);
        *reinterpret_cast<uint4*>(hi + o) = h;
        *reinterpret_cast<uint4*>(lo + o) = l;
    }
}

// ---------------------------------------------------------------------------
// images built once per operator
// ---------------------------------------------------------------------------
struct T2VSeg {       // rows of one block in one phase-1 tile
    int64_t src;      // element offset of the segment's first V^T row
    int64_t img;      // byte offset of the tile's window 0
    int n8, n, delta; // V^T row stride, valid columns, window shift (col0 mod 8)
    int rows, trow0;  // rows, first tile row
    int R, steps;     // tile rows, windows
};

template <class T>
__global__ void t2_build_v(const T2VSeg* __restrict__ segs, int nseg, const T* __restrict__ far,
                           unsigned char* __restrict__ img)
{
    for (int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const T2VSeg S = segs[sg];
        const int units = S.rows * S.steps * 8;
        for (int u = threadIdx.x; u < units; u += blockDim.x) {
            const int c = u & 7, rs = u >> 3, t = rs % S.rows, w = rs / S.rows;
            const T* row = far + S.src + (int64_t)t * S.n8;
            T v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = 64 * w + 8 * c + q - S.delta;
                v[q] = (j >= 0 && j < S.n) ? row[j] : t2_to16<T>(0.f);
            }
            const int tr = S.trow0 + t;
            const int64_t o = S.img + ((int64_t)w * S.R + tr) * t2::kRowB + ((c ^ (tr & 7)) << 4);
            *reinterpret_cast<uint4*>(img + o) = *reinterpret_cast<const uint4*>(v);
        }
    }
}

struct T2USeg {       // rows of one U^T leaf chunk (far) or A^T leaf chunk (near) in a leaf's image
    int64_t src;      // element offset of the first row
    int64_t img_row;  // image row of the first row
    int m8, m;        // row stride, valid entries (leaf rows)
    int rows, pos0;   // rows, K position of the first row (swizzle phase = position mod 8)
};

template <class T>
__global__ void t2_build_u(const T2USeg* __restrict__ segs, int nseg, const T* __restrict__ far,
                           unsigned char* __restrict__ img)
{
    for (int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const T2USeg S = segs[sg];
        for (int u = threadIdx.x; u < S.rows * 8; u += blockDim.x) {
            const int c = u & 7, t = u >> 3;
            const T* row = far + S.src + (int64_t)t * S.m8;
            T v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = 8 * c + q < S.m ? row[8 * c + q] : t2_to16<T>(0.f);
            const int ph = (S.pos0 + t) & 7;
            *reinterpret_cast<uint4*>(img + (S.img_row + t) * t2::kRowB + ((c ^ ph) << 4)) =
                *reinterpret_cast<const uint4*>(v);
        }
    }
}

// near rows: FP32 -> BF16 high and low parts
__global__ void t2_build_n(const T2USeg* __restrict__ segs, int nseg, const float* __restrict__ nearp,
                           unsigned char* __restrict__ hi, unsigned char* __restrict__ lo)
{
    for (int sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const T2USeg S = segs[sg];
        for (int u = threadIdx.x; u < S.rows * 8; u += blockDim.x) {
            const int c = u & 7, t = u >> 3;
            const float* row = nearp + S.src + (int64_t)t * S.m8;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = 8 * c + q < S.m ? row[8 * c + q] : 0.f;
            uint4 h, l;
            t2_split8<__nv_bfloat16>(v, h, l);
            const int64_t o = (S.img_row + t) * t2::kRowB + ((c ^ ((S.pos0 + t) & 7)) << 4);
            *reinterpret_cast<uint4*>(hi + o) = h;
            *reinterpret_cast<uint4*>(lo + o) = l;
        }
    }
}

// ---------------------------------------------------------------------------
// phase 1: W = V^T X (M = 128 stacked V^T rows, N = 64, K = 64-column windows)
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(32 * (t2::kMaxStages + 9), 1)
    t2_phase1(const T2Tile* __restrict__ tiles, int ntiles, const unsigned char* __restrict__ vhi,
              const unsigned char* __restrict__ vlo, const unsigned char* __restrict__ xhi,
              const unsigned char* __restrict__ xlo, unsigned char* __restrict__ whi, unsigned char* __restrict__ wlo,
              int use_lo, int w2, int nst, uint32_t hint, int* __restrict__ err)
{
    // four accumulators and two epilogue groups of four warps: tile j uses
    // accumulator j mod 4 and epilogue group j mod 2 (most tiles are one
    // 64-column window deep, so the epilogue, not the copies, would set the pace)
    __shared__ T2Ctl C;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int abytes = 128 * t2::kRowB;                      // 16 KB per A part
    const int sbytes = (use_lo ? 2 : 1) * abytes + 2 * 8192; // A high [| A low] | B high | B low
    const int boff = (use_lo ? 2 : 1) * abytes;
    t2_setup(C, nst, nst * sbytes, 256, hint);
    unsigned char* ring = t2_ring();
    const int mw = t2_mma_warp(nst);
    uint32_t issued = 0;
    if (warp < nst) {
        // ---- producer of slot `warp`: stages warp, warp + nst, ... of (tile, window) ----
        int t = blockIdx.x, w = 0;
        T2Tile tl{};
        if (t < ntiles) tl = tiles[t];
        auto next = [&]() {
            if (++w < tl.steps) return;
            w = 0;
            t += gridDim.x;
            if (t < ntiles) tl = tiles[t];
        };
        for (int k = 0; k < warp && t < ntiles; ++k) next();
        const int s = warp;
        const uint32_t fb = t5::smem_u32(&C.full[s]);
        unsigned char* st = ring + (size_t)s * sbytes;
        for (uint32_t use = 0; t < ntiles && !C.abort; ++use) {
            if (use > 0 && !t2_wait(t5::smem_u32(&C.empty[s]), (use - 1) & 1u, C, C.hint)) break;
            const uint32_t ab = (uint32_t)tl.R * t2::kRowB;
            if (lane == 0) bulk::arrive_expect(fb, ab * (use_lo ? 2u : 1u) + 2u * 8192u);
            __syncwarp();
            const int64_t va = tl.vimg + (int64_t)w * ab;
            const int64_t xa = (int64_t)(tl.xrow0 + 64 * w) * t2::kRowB;
            if (lane == 0) bulk::copy(t5::smem_u32(st), vhi + va, ab, fb);
            if (lane == 1 && use_lo) bulk::copy(t5::smem_u32(st + abytes), vlo + va, ab, fb);
            if (lane == 2) bulk::copy(t5::smem_u32(st + boff), xhi + xa, 8192, fb);
            if (lane == 3) bulk::copy(t5::smem_u32(st + boff + 8192), xlo + xa, 8192, fb);
            issued = use + 1;
            for (int k = 0; k < nst && t < ntiles; ++k) next();
        }
    } else if (warp == mw) {
        // ---- MMA issue (one lane) ----
        if (lane == 0) {
            const uint32_t id = t5::idesc(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, 0, 1, 128, t2::kF);
            uint32_t g = 0;
            int j = 0;
            for (int t = blockIdx.x; t < ntiles && !C.abort; t += gridDim.x, ++j) {
                const int b = j & 3;
                const uint32_t ub = (uint32_t)(j >> 2);
                if (ub > 0 && !t2_wait(t5::smem_u32(&C.acce[b]), (ub - 1) & 1u, C, C.hint)) break;
                t5::fence_after();
                const uint32_t acc = C.tmem + (uint32_t)(b * t2::kF);
                const int steps = tiles[t].steps;
                bool ok = true;
                for (int w = 0; w < steps; ++w, ++g) {
                    const int s = (int)(g % (uint32_t)nst);
                    if (!t2_wait(t5::smem_u32(&C.full[s]), (g / (uint32_t)nst) & 1u, C, C.hint)) {
                        ok = false;
                        break;
                    }
                    t5::fence_after();
                    const uint32_t a0 = t5::smem_u32(ring + (size_t)s * sbytes);
                    const uint32_t b0 = a0 + boff;
                    // K slice ks: +32 ks bytes along the K-major A rows (+2 in the descriptor's
                    // start-address field), +2048 ks bytes down the MN-major B rows (+128)
                    const uint64_t da0 = t5::desc_sw128(a0, 16, 1024), dl0 = t5::desc_sw128(a0 + abytes, 16, 1024);
                    const uint64_t db0 = t5::desc_sw128(b0, 1024, 1024), dbl0 = t5::desc_sw128(b0 + 8192, 1024, 1024);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t da = da0 + (uint64_t)(2 * ks), db = db0 + (uint64_t)(128 * ks);
                        t5::mma(acc, da, db, id, (w > 0 || ks > 0) ? 1u : 0u);
                        t5::mma(acc, da, dbl0 + (uint64_t)(128 * ks), id, 1u);
                        if (use_lo) t5::mma(acc, dl0 + (uint64_t)(2 * ks), db, id, 1u);
                    }
                    t5::commit(t5::smem_u32(&C.empty[s]));
                }
                if (!ok) break;
                t5::commit(t5::smem_u32(&C.accf[b]));
            }
        }
        __syncwarp();
    } else if (warp <= mw + 8) {
        // ---- epilogue group e (warps mw+1+4e .. mw+4+4e): TMEM lanes 32 q .. 32 q + 31
        // are tile rows; each thread writes its W row (128 bytes per part, the 16-byte
        // chunks in the row's swizzled order) ----
        const int q = warp & 3, e = (warp - mw - 1) >> 2;
        int j = e;
        for (int t = blockIdx.x + e * gridDim.x; t < ntiles; t += 2 * gridDim.x, j += 2) {
            const int b = j & 3;
            if (!__all_sync(0xffffffffu, t2_wait(t5::smem_u32(&C.accf[b]), (uint32_t)(j >> 2) & 1u, C, 20000u)))
                break;
            t5::fence_after();
            const T2Tile tl = tiles[t];
            const int row = 32 * q + lane;
            const int64_t wr = tl.wrow0 + row;
            const uint32_t ta = C.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * t2::kF);
            float v[4][16];
#pragma unroll
            for (int c16 = 0; c16 < 4; ++c16) t5::tmem_ld16(ta + 16 * c16, v[c16]);
            t5::fence_before();
            __syncwarp();
            if (lane == 0) bulk::arrive(t5::smem_u32(&C.acce[b]));   // the accumulator is free again
            if (row < tl.R) {
                unsigned char* ph = whi + wr * t2::kRowB;
                unsigned char* pl = wlo + wr * t2::kRowB;
                const int sw = (int)(wr & 7);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    uint4 hv, lv;
                    t2_split8<T>(&v[c >> 1][8 * (c & 1)], hv, lv);
                    *reinterpret_cast<uint4*>(ph + ((c ^ sw) << 4)) = hv;
                    if (w2) *reinterpret_cast<uint4*>(pl + ((c ^ sw) << 4)) = lv;
                }
            }
        }
    }
    t2_teardown(C, nst, issued, 256, err);
}

// ---------------------------------------------------------------------------
// phase 2: Y_l = sum U W + sum A X (M = 64 leaf rows, N = 64, K = the leaf's sequence)
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(32 * (t2::kMaxStages + 9), 1)
    t2_phase2(const T2Leaf* __restrict__ leaves, int nleaves, const T2Step* __restrict__ steps,
              const T2Piece* __restrict__ pieces, T2Arrays arrs, const float* __restrict__ scale,
              float* __restrict__ Y, int N, int use_lo, int w2, int nst, int nacc, uint32_t hint,
              int* __restrict__ err)
{
    __shared__ T2Ctl C;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    t2_setup(C, nst, nst * kT2Stage2, 2 * nacc * t2::kF, hint);
    unsigned char* ring = t2_ring();
    const int mw = t2_mma_warp(nst);
    uint32_t issued = 0;
    const uint32_t enabled = (use_lo ? kT2FlagLo : 0u) | (w2 ? kT2FlagW2 : 0u);
    if (warp < nst) {
        // ---- producer of slot `warp`: stages warp, warp + nst, ... of (leaf, step); the
        // record of its next stage (header, piece `lane`) is read one stage ahead ----
        int l = blockIdx.x, st = 0, nsteps = 0, step0 = 0;
        if (l < nleaves) {
            const T2Leaf L = leaves[l];
            nsteps = L.nsteps;
            step0 = L.step0;
        }
        auto next = [&]() {
            if (++st < nsteps) return;
            st = 0;
            l += gridDim.x;
            if (l < nleaves) {
                const T2Leaf L = leaves[l];
                nsteps = L.nsteps;
                step0 = L.step0;
            }
        };
        for (int k = 0; k < warp && l < nleaves; ++k) next();
        int4 hdr = make_int4(0, 0, 0, 0);
        T2Piece pc{};
        auto fetch = [&]() {
            if (l >= nleaves) return;
            hdr = *reinterpret_cast<const int4*>(steps + step0 + st);
            if (lane < hdr.y) pc = pieces[hdr.x + lane];
        };
        fetch();
        const int s = warp;
        const uint32_t fb = t5::smem_u32(&C.full[s]);
        unsigned char* sp = ring + (size_t)s * kT2Stage2;
        for (uint32_t use = 0; l < nleaves && !C.abort; ++use) {
            const int4 H = hdr;
            const T2Piece P = pc;
            for (int k = 0; k < nst && l < nleaves; ++k) next();
            fetch();   // in flight while this stage waits for its slot
            const bool on = lane < H.y && ((P.info >> 29) & ~enabled) == 0;
            uint32_t bytes = on ? (P.info & 0xFFFFFFu) : 0u;
            for (int p = 32 + lane; p < H.y; p += 32) {
                const uint32_t info = pieces[H.x + p].info;
                if (((info >> 29) & ~enabled) == 0) bytes += info & 0xFFFFFFu;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            if (use > 0 && !t2_wait(t5::smem_u32(&C.empty[s]), (use - 1) & 1u, C, C.hint)) break;
            if (lane == 0) {
                C.meta_k16[s] = H.z;
                C.meta_kind[s] = H.w;
                bulk::arrive_expect(fb, bytes);
            }
            __syncwarp();
            if (on) bulk::copy(t5::smem_u32(sp + P.dst), arrs.a[(P.info >> 24) & 31u] + P.src, P.info & 0xFFFFFFu, fb);
            for (int p = 32 + lane; p < H.y; p += 32) {
                const T2Piece Q = pieces[H.x + p];
                if (((Q.info >> 29) & ~enabled) == 0)
                    bulk::copy(t5::smem_u32(sp + Q.dst), arrs.a[(Q.info >> 24) & 31u] + Q.src, Q.info & 0xFFFFFFu, fb);
            }
            issued = use + 1;
        }
    } else if (warp == mw) {
        if (lane == 0) {
            const uint32_t idf = t5::idesc(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, 1, 1, 64, t2::kF);
            const uint32_t idn = t5::idesc(1, 1, 1, 64, t2::kF);
            uint32_t g = 0;
            int j = 0;
            for (int l = blockIdx.x; l < nleaves && !C.abort; l += gridDim.x, ++j) {
                const int b = j & 1;
                const uint32_t ub = (uint32_t)(j >> 1);
                if (ub > 0 && !t2_wait(t5::smem_u32(&C.acce[b]), (ub - 1) & 1u, C, C.hint)) break;
                t5::fence_after();
                // slice q accumulates into accumulator q mod 4 of buffer b: consecutive MMAs
                // write different accumulators, so they do not wait on one another
                const uint32_t acc0 = C.tmem + (uint32_t)(b * nacc * t2::kF);
                const int nsteps = leaves[l].nsteps;
                bool ok = true;
                int q = 0;
                for (int st = 0; st < nsteps; ++st, ++g) {
                    const int s = (int)(g % (uint32_t)nst);
                    if (!t2_wait(t5::smem_u32(&C.full[s]), (g / (uint32_t)nst) & 1u, C, C.hint)) {
                        ok = false;
                        break;
                    }
                    t5::fence_after();
                    const uint32_t a0 = t5::smem_u32(ring + (size_t)s * kT2Stage2);
                    const int nks = C.meta_k16[s] >> 4;
                    const bool nearst = C.meta_kind[s] == 1;
                    // descriptors of the stage's first 16-row slice; slice ks starts 2048 ks bytes
                    // later, i.e. 128 ks in the descriptor's start-address field (16-byte units)
                    const uint64_t ah0 = t5::desc_sw128(a0 + kT2A, 1024, 1024);
                    const uint64_t al0 = t5::desc_sw128(a0 + kT2AL, 1024, 1024);
                    const uint64_t bh0 = t5::desc_sw128(a0 + kT2B, 1024, 1024);
                    const uint64_t bl0 = t5::desc_sw128(a0 + kT2BL, 1024, 1024);
                    for (int ks = 0; ks < nks; ++ks, ++q) {
                        const uint64_t o = (uint64_t)(128 * ks);
                        const uint64_t ah = ah0 + o, al = al0 + o, bh = bh0 + o, bl = bl0 + o;
                        const uint32_t acc = acc0 + (uint32_t)((q & (nacc - 1)) * t2::kF);
                        const uint32_t accum = q < nacc ? 0u : 1u;   // the accumulator's first slice overwrites it
                        if (nearst) {
                            t5::mma(acc, ah, bh, idn, accum);
                            t5::mma(acc, ah, bl, idn, 1u);
                            t5::mma(acc, al, bh, idn, 1u);
                        } else {
                            t5::mma(acc, ah, bh, idf, accum);
                            if (w2) t5::mma(acc, ah, bl, idf, 1u);
                            if (use_lo) t5::mma(acc, al, bh, idf, 1u);
                        }
                    }
                    t5::commit(t5::smem_u32(&C.empty[s]));
                }
                if (!ok) break;
                t5::commit(t5::smem_u32(&C.accf[b]));
            }
        }
        __syncwarp();
    } else if (warp <= mw + 4) {
        // ---- epilogue: an M = 64 accumulator keeps row i in TMEM lane 32 (i / 16) + i % 16 ----
        const int q = warp & 3;
        const float inv = scale[1];
        int j = 0;
        for (int l = blockIdx.x; l < nleaves; l += gridDim.x, ++j) {
            const int b = j & 1;
            if (!__all_sync(0xffffffffu, t2_wait(t5::smem_u32(&C.accf[b]), (uint32_t)(j >> 1) & 1u, C, 20000u))) break;
            t5::fence_after();
            const T2Leaf L = leaves[l];
            const int row = 16 * q + lane;
            const uint32_t ta = C.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * nacc * t2::kF);
            float v[4][16];
#pragma unroll
            for (int c16 = 0; c16 < 4; ++c16) t5::tmem_ld16(ta + 16 * c16, v[c16]);
            const int na = min(L.nslices, nacc);
            for (int a = 1; a < na; ++a) {
#pragma unroll
                for (int c16 = 0; c16 < 4; ++c16) {
                    float u[16];
                    t5::tmem_ld16(ta + (uint32_t)(a * t2::kF) + 16 * c16, u);
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[c16][k] += u[k];
                }
            }
            t5::fence_before();
            __syncwarp();
            if (lane == 0) bulk::arrive(t5::smem_u32(&C.acce[b]));   // the accumulator is free again
            if (lane < 16 && row < L.m) {
#pragma unroll
                for (int c16 = 0; c16 < 4; ++c16)
#pragma unroll
                    for (int k = 0; k < 16; ++k) Y[(int64_t)(16 * c16 + k) * N + L.row0 + row] = v[c16][k] * inv;
            }
        }
    }
    t2_teardown(C, nst, issued, 2 * nacc * t2::kF, err);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int t2_grid(int items, int per_sm)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, std::min(items, per_sm * sms));
}

int tc2_prepare(Operator& op, std::string& err)
{
    op.tc2 = 0;
    if (op.tc_off || op.mode != RT_MODE_HMATRIX || op.G != 1 || op.F != t2::kF) return RT_OK;
    if (op.far_prec != RT_PREC_BF16 && op.far_prec != RT_PREC_F16) return RT_OK;
    const int nl = (int)op.plan.leaf_start.size();
    for (int l = 0; l < nl; ++l)
        if (op.plan.leaf_size[l] > 64) return RT_OK;
    if ((int64_t)op.N + 256 > INT_MAX / 2) return RT_OK;
    int rc;
    // ---- phase-1 tiles: V^T rows of the blocks of each column cluster, stacked ----
    const int ncl = (int)op.plan.clusters.size();
    std::vector<std::vector<int>> by_col(ncl);
    for (int b = 0; b < op.n_far; ++b) by_col[op.far_blocks[b].sc].push_back(b);
    std::vector<int64_t> wfirst(op.n_far, 0);   // W row of each block's rank term 0
    struct PTile {
        int R, steps, xrow0, col0, n, delta;
        int64_t wrow0;
        std::vector<T2VSeg> segs;
    };
    std::vector<PTile> pt;
    int64_t wrows = 0;
    for (int c = 0; c < ncl; ++c) {
        if (by_col[c].empty()) continue;
        const FarBlock& f0 = op.far_blocks[by_col[c][0]];
        const int col0 = f0.col0, n = f0.n, delta = col0 & 7;
        const int steps = (delta + n + 63) / 64;
        PTile cur{0, steps, col0 - delta, col0, n, delta, wrows, {}};
        for (int b : by_col[c]) {
            const int r = op.rank[b];
            wfirst[b] = wrows;
            for (int k = 0; k < r;) {
                if (cur.R == 128) {
                    pt.push_back(std::move(cur));
                    cur = PTile{0, steps, col0 - delta, col0, n, delta, wrows, {}};
                }
                const int take = std::min(r - k, 128 - cur.R);
                T2VSeg sg{};
                sg.src = op.far_v_off[b] + (int64_t)k * round8(n);
                sg.n8 = round8(n);
                sg.n = n;
                sg.delta = delta;
                sg.rows = take;
                sg.trow0 = cur.R;
                sg.steps = steps;
                cur.segs.push_back(sg);
                cur.R += take;
                k += take;
                wrows += take;
            }
        }
        if (cur.R > 0) pt.push_back(std::move(cur));
    }
    std::stable_sort(pt.begin(), pt.end(), [](const PTile& a, const PTile& b) { return a.steps > b.steps; });
    std::vector<T2Tile> tiles;
    std::vector<T2VSeg> vsegs;
    int64_t vbytes = 0;
    for (PTile& p : pt) {
        T2Tile t{};
        t.vimg = vbytes;
        t.wrow0 = p.wrow0;
        t.R = p.R;
        t.steps = p.steps;
        t.xrow0 = p.xrow0;
        for (T2VSeg s : p.segs) {
            s.img = vbytes;
            s.R = p.R;
            vsegs.push_back(s);
        }
        vbytes += (int64_t)p.R * p.steps * t2::kRowB;
        tiles.push_back(t);
    }
    // ---- phase-2 leaves: K sequence of far rank terms, then near columns ----
    std::vector<std::vector<int>> far_of(nl), near_of(nl);   // chunk ids per leaf
    for (int b = 0; b < op.n_far; ++b)
        for (int c = op.far_chunk_ptr[b]; c < op.far_chunk_ptr[b + 1]; ++c) far_of[op.far_chunks[c].leaf].push_back(c);
    std::vector<int> far_block_of((size_t)op.far_chunks.size()), near_block_of((size_t)op.dense_chunks.size());
    for (int b = 0; b < op.n_far; ++b)
        for (int c = op.far_chunk_ptr[b]; c < op.far_chunk_ptr[b + 1]; ++c) far_block_of[c] = b;
    for (int b = 0; b < op.n_near; ++b)
        for (int c = op.dense_chunk_ptr[b]; c < op.dense_chunk_ptr[b + 1]; ++c) {
            near_block_of[c] = b;
            near_of[op.dense_chunks[c].leaf].push_back(c);
        }
    std::vector<T2Leaf> leaves(nl);
    std::vector<T2Step> stepv;
    std::vector<T2Piece> pcs;
    std::vector<T2USeg> usegs, nsegs;
    int64_t urows = 0, nrows = 0;
    auto mk = [](int64_t src, int dst, int bytes, int arr, uint32_t flags) {
        T2Piece p;
        p.src = src;
        p.dst = dst;
        p.info = (uint32_t)bytes | ((uint32_t)arr << 24) | (flags << 29);
        return p;
    };
    struct Item {      // one block in the sequence
        int64_t a_row; // first image row
        int64_t b_row; // first B row (W row or X^T row)
        int pos, rows;
        int kind;
    };
    for (int l = 0; l < nl; ++l) {
        std::vector<Item> items;
        // far: greedy order so that each block's position is congruent to its W row mod 8
        std::vector<std::vector<int>> bucket(8);
        for (int c : far_of[l]) bucket[(int)(wfirst[far_block_of[c]] & 7)].push_back(c);
        int pos = 0;
        size_t left = far_of[l].size();
        while (left > 0) {
            int pick = -1;
            for (int d = 0; d < 8 && pick < 0; ++d)
                if (!bucket[(pos + d) & 7].empty()) pick = (pos + d) & 7;
            const int c = bucket[pick].back();
            bucket[pick].pop_back();
            --left;
            const int b = far_block_of[c];
            const Chunk& ch = op.far_chunks[c];
            const int r = op.rank[b];
            const int start = pos + ((pick - pos) & 7);
            T2USeg sg{};
            sg.src = op.far_u_off[b] + ch.off;
            sg.img_row = urows;
            sg.m8 = ch.m8;
            sg.m = ch.m;
            sg.rows = r;
            sg.pos0 = start;
            usegs.push_back(sg);
            items.push_back({urows, wfirst[b], start, r, 0});
            urows += r;
            pos = start + r;
        }
        const int kfar = pos;
        pos = (pos + 63) / 64 * 64;   // near steps start on a fresh stage
        for (int c : near_of[l]) {
            const int b = near_block_of[c];
            const Chunk& ch = op.dense_chunks[c];
            const int col0 = op.dense_blocks[b].col0, n = op.dense_blocks[b].n;
            const int start = pos + ((col0 - pos) & 7);
            T2USeg sg{};
            sg.src = op.dense_off[b] + ch.off;
            sg.img_row = nrows;
            sg.m8 = ch.m8;
            sg.m = ch.m;
            sg.rows = n;
            sg.pos0 = start;
            nsegs.push_back(sg);
            items.push_back({nrows, col0, start, n, 1});
            nrows += n;
            pos = start + n;
        }
        (void)kfar;
        // cut the sequence into 64-row stages
        leaves[l].row0 = op.plan.leaf_start[l];
        leaves[l].m = op.plan.leaf_size[l];
        leaves[l].step0 = (int)stepv.size();
        leaves[l].nslices = 0;
        const int nstage = (pos + 63) / 64;
        size_t it0 = 0;
        for (int sgi = 0; sgi < nstage; ++sgi) {
            const int lo = 64 * sgi, hi = lo + 64;
            while (it0 < items.size() && items[it0].pos + items[it0].rows <= lo) ++it0;
            T2Step S{};
            S.piece0 = (int)pcs.size();
            S.kind = -1;
            int last = lo;   // first row not yet covered
            auto zero_rows = [&](int from, int to) {
                if (to <= from) return;
                pcs.push_back(mk(0, kT2A + (from - lo) * t2::kRowB, (to - from) * t2::kRowB, T2_ZERO, 0));
                pcs.push_back(mk(0, kT2AL + (from - lo) * t2::kRowB, (to - from) * t2::kRowB, T2_ZERO, 0));
            };
            int run_a0 = -1, run_p0 = 0, run_n = 0;
            int64_t run_src = 0;
            int run_kind = 0;
            auto flush_a = [&]() {
                if (run_a0 < 0) return;
                const int dst = (run_p0 - lo) * t2::kRowB, bytes = run_n * t2::kRowB;
                if (run_kind == 0) {
                    pcs.push_back(mk(run_src * t2::kRowB, kT2A + dst, bytes, T2_UHI, 0));
                    if (op.d_far_lo) pcs.push_back(mk(run_src * t2::kRowB, kT2AL + dst, bytes, T2_ULO, kT2FlagLo));
                } else {
                    pcs.push_back(mk(run_src * t2::kRowB, kT2A + dst, bytes, T2_NHI, 0));
                    pcs.push_back(mk(run_src * t2::kRowB, kT2AL + dst, bytes, T2_NLO, 0));
                }
                run_a0 = -1;
            };
            for (size_t it = it0; it < items.size() && items[it].pos < hi; ++it) {
                const Item& I = items[it];
                const int p0 = std::max(I.pos, lo), p1 = std::min(I.pos + I.rows, hi);
                if (p1 <= p0) continue;
                if (S.kind < 0) S.kind = I.kind;
                const int64_t arow = I.a_row + (p0 - I.pos);
                // A: extend the current run when both the rows and the positions continue it
                if (run_a0 >= 0 && run_kind == I.kind && run_src + run_n == arow && run_p0 + run_n == p0) {
                    run_n += p1 - p0;
                } else {
                    flush_a();
                    zero_rows(last, p0);
                    run_a0 = 1;
                    run_src = arow;
                    run_p0 = p0;
                    run_n = p1 - p0;
                    run_kind = I.kind;
                }
                // B: W rows (far) or X^T rows (near) of the same positions
                const int64_t brow = I.b_row + (p0 - I.pos);
                const int dst = (p0 - lo) * t2::kRowB, bytes = (p1 - p0) * t2::kRowB;
                if (I.kind == 0) {
                    pcs.push_back(mk(brow * t2::kRowB, kT2B + dst, bytes, T2_WHI, 0));
                    pcs.push_back(mk(brow * t2::kRowB, kT2BL + dst, bytes, T2_WLO, kT2FlagW2));
                } else {
                    pcs.push_back(mk(brow * t2::kRowB, kT2B + dst, bytes, T2_XHI, 0));
                    pcs.push_back(mk(brow * t2::kRowB, kT2BL + dst, bytes, T2_XLO, 0));
                }
                last = p1;
            }
            flush_a();
            if (S.kind < 0) {   // an empty stage cannot occur: every stage holds at least one row
                err = "tc2: empty stage";
                return RT_EINVAL;
            }
            const int used = last - lo;
            S.k16 = (used + 15) & ~15;
            zero_rows(last, lo + S.k16);
            S.np = (int)pcs.size() - S.piece0;
            stepv.push_back(S);
            leaves[l].nslices += S.k16 / 16;
        }
        leaves[l].nsteps = (int)stepv.size() - leaves[l].step0;
    }
    // ---- every copy stays inside its source array and its stage region ----
    const int parts = op.far_prec == RT_PREC_F16 ? 4 : 2;   // X^T BF16 high/low (+ FP16 high/low)
    const int64_t xrows = (int64_t)op.N + 256;
    {
        const int64_t lim[T2_NARR] = {urows * t2::kRowB, urows * t2::kRowB, nrows * t2::kRowB, nrows * t2::kRowB,
                                      wrows * t2::kRowB, wrows * t2::kRowB, xrows * t2::kRowB, xrows * t2::kRowB,
                                      t2::kZeroBytes};
        for (const T2Piece& P : pcs) {
            const int arr = (int)((P.info >> 24) & 31u), bytes = (int)(P.info & 0xFFFFFFu);
            const int reg = P.dst / 8192;
            if (arr >= T2_NARR || bytes <= 0 || (bytes & 15) || (P.src & 15) || (P.dst & 15) || P.src < 0 ||
                P.src + bytes > lim[arr] || P.dst < 0 || reg > 3 || P.dst + bytes > 8192 * (reg + 1)) {
                err = "tc2: a copy piece falls outside its array or stage region";
                return RT_EINVAL;
            }
        }
        for (const T2Step& S : stepv)
            if (S.k16 < 16 || S.k16 > 64 || (S.k16 & 15) || S.np <= 0) {
                err = "tc2: malformed stage";
                return RT_EINVAL;
            }
        for (const T2Tile& t : tiles)
            if (t.R < 1 || t.R > 128 || t.vimg + (int64_t)t.steps * t.R * t2::kRowB > vbytes || t.xrow0 < 0 ||
                t.xrow0 + 64LL * t.steps > xrows || t.wrow0 + t.R > wrows) {
                err = "tc2: malformed phase-1 tile";
                return RT_EINVAL;
            }
    }
    // ---- device buffers and images ----
    unsigned char *vhi = nullptr, *vlo = nullptr, *uhi = nullptr, *ulo = nullptr, *nhi = nullptr, *nlo = nullptr;
    unsigned char *whi = nullptr, *wlo = nullptr, *xs = nullptr, *zero = nullptr;
    const bool lo_parts = op.d_far_lo != nullptr;
    if ((rc = dev_alloc(op, &vhi, (size_t)std::max<int64_t>(vbytes, 16), err))) return rc;
    if (lo_parts && (rc = dev_alloc(op, &vlo, (size_t)std::max<int64_t>(vbytes, 16), err))) return rc;
    if ((rc = dev_alloc(op, &uhi, (size_t)std::max<int64_t>(urows, 1) * t2::kRowB, err))) return rc;
    if (lo_parts && (rc = dev_alloc(op, &ulo, (size_t)std::max<int64_t>(urows, 1) * t2::kRowB, err))) return rc;
    if ((rc = dev_alloc(op, &nhi, (size_t)std::max<int64_t>(nrows, 1) * t2::kRowB, err))) return rc;
    if ((rc = dev_alloc(op, &nlo, (size_t)std::max<int64_t>(nrows, 1) * t2::kRowB, err))) return rc;
    if ((rc = dev_alloc(op, &whi, (size_t)std::max<int64_t>(wrows, 1) * t2::kRowB, err))) return rc;
    if ((rc = dev_alloc(op, &wlo, (size_t)std::max<int64_t>(wrows, 1) * t2::kRowB, err))) return rc;
    if ((rc = dev_alloc(op, &xs, (size_t)parts * xrows * t2::kRowB, err))) return rc;
    if ((rc = dev_alloc(op, &zero, (size_t)t2::kZeroBytes, err))) return rc;
    RT_CUDA_TRY(cudaMemsetAsync(xs, 0, (size_t)parts * xrows * t2::kRowB, op.stream));   // rows >= N stay zero
    RT_CUDA_TRY(cudaMemsetAsync(zero, 0, (size_t)t2::kZeroBytes, op.stream));
    T2Tile* d_tiles = nullptr;
    T2Leaf* d_leaves = nullptr;
    T2Step* d_steps = nullptr;
    T2Piece* d_pcs = nullptr;
    T2VSeg* d_vs = nullptr;
    T2USeg *d_us = nullptr, *d_ns = nullptr;
    if ((rc = dev_alloc(op, &d_tiles, tiles.size(), err)) || (rc = upload_async(op, d_tiles, tiles.data(), tiles.size(), err)))
        return rc;
    if ((rc = dev_alloc(op, &d_leaves, leaves.size(), err)) ||
        (rc = upload_async(op, d_leaves, leaves.data(), leaves.size(), err)))
        return rc;
    if ((rc = dev_alloc(op, &d_steps, stepv.size(), err)) || (rc = upload_async(op, d_steps, stepv.data(), stepv.size(), err)))
        return rc;
    if ((rc = dev_alloc(op, &d_pcs, pcs.size(), err)) || (rc = upload_async(op, d_pcs, pcs.data(), pcs.size(), err)))
        return rc;
    // segment lists are needed only while the images are built
    if ((rc = dev_alloc(op, &d_vs, vsegs.size(), err)) || (rc = upload_async(op, d_vs, vsegs.data(), vsegs.size(), err)))
        return rc;
    if ((rc = dev_alloc(op, &d_us, usegs.size(), err)) || (rc = upload_async(op, d_us, usegs.data(), usegs.size(), err)))
        return rc;
    if ((rc = dev_alloc(op, &d_ns, nsegs.size(), err)) || (rc = upload_async(op, d_ns, nsegs.data(), nsegs.size(), err)))
        return rc;
    const int gb = t2_grid(1 << 20, 8);
    if (op.far_prec == RT_PREC_BF16) {
        using B = __nv_bfloat16;
        if (!vsegs.empty()) t2_build_v<B><<<gb, 256, 0, op.stream>>>(d_vs, (int)vsegs.size(), (const B*)op.d_far, vhi);
        if (!vsegs.empty() && lo_parts) t2_build_v<B><<<gb, 256, 0, op.stream>>>(d_vs, (int)vsegs.size(), (const B*)op.d_far_lo, vlo);
        if (!usegs.empty()) t2_build_u<B><<<gb, 256, 0, op.stream>>>(d_us, (int)usegs.size(), (const B*)op.d_far, uhi);
        if (!usegs.empty() && lo_parts) t2_build_u<B><<<gb, 256, 0, op.stream>>>(d_us, (int)usegs.size(), (const B*)op.d_far_lo, ulo);
    } else {
        using H = __half;
        if (!vsegs.empty()) t2_build_v<H><<<gb, 256, 0, op.stream>>>(d_vs, (int)vsegs.size(), (const H*)op.d_far, vhi);
        if (!vsegs.empty() && lo_parts) t2_build_v<H><<<gb, 256, 0, op.stream>>>(d_vs, (int)vsegs.size(), (const H*)op.d_far_lo, vlo);
        if (!usegs.empty()) t2_build_u<H><<<gb, 256, 0, op.stream>>>(d_us, (int)usegs.size(), (const H*)op.d_far, uhi);
        if (!usegs.empty() && lo_parts) t2_build_u<H><<<gb, 256, 0, op.stream>>>(d_us, (int)usegs.size(), (const H*)op.d_far_lo, ulo);
    }
    if (!nsegs.empty()) t2_build_n<<<gb, 256, 0, op.stream>>>(d_ns, (int)nsegs.size(), op.d_near, nhi, nlo);
    RT_CUDA_TRY(cudaGetLastError());
    op.t2_tiles = d_tiles;
    op.t2_ntiles = (int)tiles.size();
    op.t2_leaves = d_leaves;
    op.t2_nleaves = nl;
    op.t2_steps = d_steps;
    op.t2_pieces = d_pcs;
    op.t2_vhi = vhi;
    op.t2_vlo = vlo;
    op.t2_uhi = uhi;
    op.t2_ulo = ulo;
    op.t2_nhi = nhi;
    op.t2_nlo = nlo;
    op.t2_whi = whi;
    op.t2_wlo = wlo;
    op.t2_xs = xs;
    op.t2_xrows = xrows;
    op.t2_zero = zero;
    op.t2_wrows = wrows;
    op.t2_stats[0] = (int64_t)stepv.size();
    op.t2_stats[1] = (int64_t)pcs.size();
    op.t2_stats[2] = urows;
    op.t2_stats[3] = nrows;
    if (!op.t2_scale) {
        float* sc = nullptr;
        if ((rc = dev_alloc(op, &sc, 4, err))) return rc;
        op.t2_scale = sc;
    }
    if (!op.tc_err) {
        if ((rc = dev_alloc(op, &op.tc_err, 1, err))) return rc;
        RT_CUDA_TRY(cudaMemsetAsync(op.tc_err, 0, sizeof(int), op.stream));
    }
    const int smem = t2::kRingBytes + 1024;
    RT_CUDA_TRY(cudaFuncSetAttribute(t2_phase1<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(t2_phase1<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(t2_phase2<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RT_CUDA_TRY(cudaFuncSetAttribute(t2_phase2<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    op.tc2 = 1;
    op.tc_enabled = 1;
    return RT_OK;
}

template <class T>
static int tc2_launch(Operator& op, const float* X, float* Y, cudaStream_t s, std::string& err)
{
    const int N = op.N;
    const int use_lo = op.use_lo && op.d_far_lo ? 1 : 0;
    const int w2 = (std::is_same<T, __nv_bfloat16>::value || use_lo) ? 1 : 0;
    unsigned char* xs = (unsigned char*)op.t2_xs;
    const int64_t part = op.t2_xrows * t2::kRowB;
    unsigned char *xb_hi = xs, *xb_lo = xs + part;                     // BF16 (near blocks; BF16 far)
    unsigned char *xf_hi = xb_hi, *xf_lo = xb_lo;                      // far type (phase 1)
    float* sc = (float*)op.t2_scale;
    unsigned* mx = (unsigned*)(sc + 2);
    const int64_t total = (int64_t)op.F * N;
    const int ge = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 8));
    RT_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned), s));
    t2_xmax<<<ge, 256, 0, s>>>(X, total, mx);
    const int gs = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)N * 8 + 255) / 256, 152 * 8));
    t2_xsplit<__nv_bfloat16><<<gs, 256, 0, s>>>(X, N, mx, sc, xb_hi, xb_lo);
    if (std::is_same<T, __half>::value) {
        xf_hi = xs + 2 * part;
        xf_lo = xs + 3 * part;
        t2_xsplit<__half><<<gs, 256, 0, s>>>(X, N, mx, nullptr, xf_hi, xf_lo);
    }
    RT_CUDA_TRY(cudaGetLastError());
    // two CTAs per SM, each with half the ring and half of TMEM: one MMA-issuing thread
    // per CTA, and with stages of 64 K rows the issue path, not the tensor pipe, sets the
    // pace of a CTA (measured on the 32^3 and 64^3 operators: one CTA per SM 2.78 ms,
    // two 2.17 ms, three 2.58 ms at 64^3)
    const int per_sm = t2::kCtasPerSm;
    const int ring = t2::kRingBytes / per_sm;
    const int smem = ring + 1024;
    const uint32_t hint = bulk::kSuspendNs;
    if (op.t2_ntiles > 0) {
        const int sb = (use_lo ? 2 : 1) * 128 * t2::kRowB + 2 * 8192;
        const int nst = std::max(2, std::min(t2::kMaxStages, ring / sb));
        t2_phase1<T><<<t2_grid(op.t2_ntiles, per_sm), 32 * (nst + 9), smem, s>>>(
            (const T2Tile*)op.t2_tiles, op.t2_ntiles, (const unsigned char*)op.t2_vhi, (const unsigned char*)op.t2_vlo,
            xf_hi, xf_lo, (unsigned char*)op.t2_whi, (unsigned char*)op.t2_wlo, use_lo, w2, nst, hint, op.tc_err);
        RT_CUDA_TRY(cudaGetLastError());
    }
    T2Arrays A{};
    A.a[T2_UHI] = (const unsigned char*)op.t2_uhi;
    A.a[T2_ULO] = (const unsigned char*)op.t2_ulo;
    A.a[T2_NHI] = (const unsigned char*)op.t2_nhi;
    A.a[T2_NLO] = (const unsigned char*)op.t2_nlo;
    A.a[T2_WHI] = (const unsigned char*)op.t2_whi;
    A.a[T2_WLO] = (const unsigned char*)op.t2_wlo;
    A.a[T2_XHI] = xb_hi;
    A.a[T2_XLO] = xb_lo;
    A.a[T2_ZERO] = (const unsigned char*)op.t2_zero;
    const int nst2 = std::max(2, std::min(t2::kMaxStages, ring / kT2Stage2));
    const int nacc = 4 / per_sm;   // 2 nacc 64-column accumulators per CTA: all of TMEM per SM
    t2_phase2<T><<<t2_grid(op.t2_nleaves, per_sm), 32 * (nst2 + 5), smem, s>>>(
        (const T2Leaf*)op.t2_leaves, op.t2_nleaves, (const T2Step*)op.t2_steps, (const T2Piece*)op.t2_pieces, A, sc, Y,
        N, use_lo, w2, nst2, nacc, hint, op.tc_err);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

int tc2_apply(Operator& op, const float* X, float* Y, cudaStream_t s, std::string& err)
{
    if (op.far_prec == RT_PREC_BF16) return tc2_launch<__nv_bfloat16>(op, X, Y, s, err);
    return tc2_launch<__half>(op, X, Y, s, err);
}

}  // namespace rt
