// rt_hmv_stream.cuh -- the two H-matvec phases as streamed, warp-specialised
// persistent kernels.  The arithmetic is that of rt_hmv_dev.cuh; only the way
// operator data reaches the SM differs:
//
//   * the host cuts the operator into stage records: each record lists up to
//     kMaxPieces contiguous pieces (runs of V^T rows in phase 1; k-ranges of a
//     leaf's U^T / A^T chunks in phase 2) that together fill at most one
//     kStageBytes stage;
//   * every stage slot of a CTA has its own producer warp.  It reads the
//     record (one 64-byte piece per lane), raises the slot's "full" mbarrier
//     by the record's byte count, and each lane issues one cp.async.bulk for
//     its piece.  The warp then gathers the vector values the stage multiplies
//     (x columns in phase 1; w or x entries in phase 2) into the slot's vector
//     area with ordinary loads, and arrives on "full";
//   * eight consumer warps wait for "full", compute from shared memory only,
//     and release the slot on its "empty" mbarrier.
//
// So every SM keeps several 16 KB copies in flight whatever the block sizes,
// and the consumers never wait on a global load: the latency of the record
// and vector reads is spread over kStages independent producer warps.  All
// waits are bounded (rt_bulk.cuh); a wait that gives up sets *err and the
// kernel returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rt_bulk.cuh"
#include "rt_internal.h"

namespace rt {

namespace hs {
constexpr int kStages = 5;        // stage slots = producer warps
constexpr int kStageBytes = 16384;
constexpr int kVecFloats = 1024;  // gathered vector values per stage
constexpr int kMaxPieces = 15;
constexpr int kConsumerWarps = 8;
constexpr int kConsumers = 32 * kConsumerWarps;
constexpr int kThreads = kConsumers + 32 * kStages;
constexpr int kCtasPerSm = 2;
}  // namespace hs

struct HsPiece {      // one contiguous copy into a stage (64 bytes)
    int64_t a;        // element offset for group 0 (far array; near array for a dense piece)
    int64_t gstride;  // elements between groups
    int64_t vsrc;     // first vector entry for f = 0: phase 1 the block's first column;
                      // phase 2 the w index (far) or x column (dense) of the first k
    int soff;         // byte offset in the stage (multiple of 16)
    int bytes;        // bytes copied (multiple of 16)
    int rows;         // phase 1: V^T rows; phase 2: k count
    int n8;           // row length in elements (phase 1: padded columns; phase 2: leaf m8)
    int vo;           // float offset of the piece's values in the stage's vector area
    int vlen;         // values gathered there (0: an earlier piece's values at vo are used)
    int valid;        // gathered values at positions >= valid are zero (padding columns)
    int r;            // rank of the block: w stride between frequencies
    int wv;           // phase 1: w index of the first row for f = 0
    int kind;         // 0 far (element type T), 1 dense (float)
};

struct HsLoad {       // one stage's record (976 bytes)
    int np;           // pieces
    int bytes;        // bytes copied into the stage
    int K;            // phase 2: k rows of the stage ([K][m8], one kind)
    int kind;         // phase 2: 0 far, 1 dense
    HsPiece p[hs::kMaxPieces];
};

constexpr size_t hs_smem_bytes()
{
    return (size_t)hs::kStages * (hs::kStageBytes + 4 * hs::kVecFloats + sizeof(HsLoad) + 16) +
           sizeof(float4) * hs::kConsumers;
}

// ---- shared-memory element loads (converted to float) ----------------------
__device__ __forceinline__ void lds16(const float* p, float* v)
{
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}
template <class H>
__device__ __forceinline__ void lds16h(const H* p, float* v)
{
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    const unsigned u[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const H* h = reinterpret_cast<const H*>(&u[k]);
        v[2 * k] = to_f(h[0]);
        v[2 * k + 1] = to_f(h[1]);
    }
}
__device__ __forceinline__ void lds16(const __nv_bfloat16* p, float* v) { lds16h(p, v); }
__device__ __forceinline__ void lds16(const __half* p, float* v) { lds16h(p, v); }

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
template <class H>
__device__ __forceinline__ float4 lds4h(const H* p)
{
    const uint2 a = *reinterpret_cast<const uint2*>(p);
    const H* h0 = reinterpret_cast<const H*>(&a.x);
    const H* h1 = reinterpret_cast<const H*>(&a.y);
    return make_float4(to_f(h0[0]), to_f(h0[1]), to_f(h1[0]), to_f(h1[1]));
}
__device__ __forceinline__ float4 lds4(const __nv_bfloat16* p) { return lds4h(p); }
__device__ __forceinline__ float4 lds4(const __half* p) { return lds4h(p); }

__device__ __forceinline__ void fma4(float4& acc, const float4 a, float w)
{
    acc.x += a.x * w;
    acc.y += a.y * w;
    acc.z += a.z * w;
    acc.w += a.w * w;
}

// ---- the ring --------------------------------------------------------------
struct HsRing {
    unsigned char* stage;   // [kStages][kStageBytes]
    float* vec;             // [kStages][kVecFloats]
    HsLoad* meta;           // [kStages]
    uint64_t* bars;         // full[kStages], empty[kStages]
    float4* red;            // [kConsumers]
    __device__ __forceinline__ uint32_t full(int s) const { return bulk::saddr(bars + s); }
    __device__ __forceinline__ uint32_t empty(int s) const { return bulk::saddr(bars + hs::kStages + s); }
};

__device__ __forceinline__ HsRing hs_ring_init()
{
    extern __shared__ __align__(128) unsigned char hs_smem[];
    HsRing R;
    R.stage = hs_smem;
    R.vec = reinterpret_cast<float*>(hs_smem + (size_t)hs::kStages * hs::kStageBytes);
    R.meta = reinterpret_cast<HsLoad*>(R.vec + hs::kStages * hs::kVecFloats);
    R.bars = reinterpret_cast<uint64_t*>(R.meta + hs::kStages);
    R.red = reinterpret_cast<float4*>(R.bars + 2 * hs::kStages);
    if (threadIdx.x == 0) {
        for (int s = 0; s < hs::kStages; ++s) {
            bulk::bar_init(R.full(s), 1);
            bulk::bar_init(R.empty(s), hs::kConsumerWarps);
        }
        bulk::fence_init();
    }
    __syncthreads();
    return R;
}

// A stage record as the producer warp holds it: the header (every lane) and
// piece `lane`.  Records are fixed-size, so every lane < kMaxPieces may read
// its slot whatever the piece count: header and pieces arrive in one round
// trip, and the producer loads the next stage's record while it fills the
// current one.
struct HsRec {
    int4 hdr;     // np, bytes, K, kind
    HsPiece pc;   // piece `lane` (meaningful for lane < np)
    int f, g;     // frequency and its kappa group
};

__device__ __forceinline__ void hs_fetch(HsRec& c, const HsLoad* __restrict__ rec, int f,
                                         const int* __restrict__ fgroup)
{
    const int lane = threadIdx.x & 31;
    c.hdr = *reinterpret_cast<const int4*>(rec);
    if (lane < hs::kMaxPieces) c.pc = rec->p[lane];
    c.f = f;
    c.g = fgroup[f];
}

// Fill stage slot s for its use u (the whole producer warp): wait until the
// slot is free (u > 0), copy the record's pieces in, gather the vector values,
// arrive.  Vector values come from X (phase 1; dense pieces) or W (far pieces
// of phase 2).  Returns false on timeout.
template <class T>
__device__ __forceinline__ bool hs_fill(const HsRing& R, int s, uint32_t u, const HsRec& c, const T* __restrict__ far,
                                        const float* __restrict__ nearp, const float* __restrict__ X,
                                        const float* __restrict__ W, int N, bool phase2)
{
    const int lane = threadIdx.x & 31;
    // every lane observes the phase it depends on (its writes overwrite the slot)
    if (u > 0 && !__all_sync(0xffffffffu, bulk::wait(R.empty(s), (u - 1) & 1u))) return false;
    const int np = c.hdr.x;
    const HsPiece& pc = c.pc;
    const float* vb = nullptr;   // vector values of this lane's piece
    if (lane < np) {
        R.meta[s].p[lane] = pc;
        vb = (!phase2 || pc.kind == 1) ? X + (int64_t)c.f * N + pc.vsrc : W + pc.vsrc + (int64_t)c.f * pc.r;
    }
    if (lane == 0) {
        *reinterpret_cast<int4*>(&R.meta[s]) = c.hdr;
        bulk::expect_tx(R.full(s), (uint32_t)c.hdr.y);
    }
    __syncwarp();
    if (lane < np) {
        const void* src = pc.kind == 1 ? (const void*)(nearp + pc.a + (int64_t)c.g * pc.gstride)
                                       : (const void*)(far + pc.a + (int64_t)c.g * pc.gstride);
        bulk::copy(bulk::saddr(R.stage + (size_t)s * hs::kStageBytes + pc.soff), src, (uint32_t)pc.bytes, R.full(s));
    }
    float* sv = R.vec + s * hs::kVecFloats;
    for (int p = 0; p < np; ++p) {
        const int vlen = __shfl_sync(0xffffffffu, pc.vlen, p);
        if (vlen == 0) continue;
        const int vo = __shfl_sync(0xffffffffu, pc.vo, p), valid = __shfl_sync(0xffffffffu, pc.valid, p);
        const float* b = reinterpret_cast<const float*>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(vb), p));
        for (int t = lane; t < vlen; t += 128) {
            float v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = t + 32 * k < valid ? __ldg(b + t + 32 * k) : 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (t + 32 * k < vlen) sv[vo + t + 32 * k] = v[k];
        }
    }
    __syncwarp();
    if (lane == 0) bulk::arrive(R.full(s));
    return true;
}

// wait (bounded) for the slot's last copies, so that none is in flight when
// the CTA exits: when a producer leaves normally, and after its own timeout (a
// consumer that gives up can then leave at once)
__device__ __forceinline__ void hs_drain(const HsRing& R, int s, uint32_t uses)
{
    if ((threadIdx.x & 31) == 0 && uses > 0) bulk::wait(R.full(s), (uses - 1) & 1u);
}

// ---------------------------------------------------------------------------
// phase 1, w_{b,f} = V_g^T x_f[cols(b)]: stage records x frequencies, record
// major (the F frequencies of a record run on neighbouring CTAs, so the record
// is read from L2 after its first use)
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(hs::kThreads) hmv_s1(const HsLoad* __restrict__ loads, int nloads,
                                                       const T* __restrict__ far, const float* __restrict__ X,
                                                       float* __restrict__ W, int N, int F,
                                                       const int* __restrict__ fgroup, int* err)
{
    const HsRing R = hs_ring_init();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t total = (int64_t)nloads * F;
    if (warp >= hs::kConsumerWarps) {
        const int s = warp - hs::kConsumerWarps;
        const int64_t step = (int64_t)hs::kStages * gridDim.x;
        int64_t j = blockIdx.x + (int64_t)s * gridDim.x;
        HsRec nxt;
        if (j < total) hs_fetch(nxt, loads + j / F, (int)(j % F), fgroup);
        uint32_t u = 0;
        for (; j < total; j += step, ++u) {
            const HsRec cur = nxt;
            if (j + step < total) hs_fetch(nxt, loads + (j + step) / F, (int)((j + step) % F), fgroup);
            if (!hs_fill<T>(R, s, u, cur, far, nullptr, X, nullptr, N, false)) {
                if (lane == 0) atomicExch(err, 1);
                hs_drain(R, s, u);
                return;
            }
        }
        hs_drain(R, s, u);   // the last copies have landed before this warp leaves
        return;
    }
    constexpr int VW = VecW<T>::n;
    int64_t i = 0;
    for (int64_t j = blockIdx.x; j < total; j += gridDim.x, ++i) {
        const int s = (int)(i % hs::kStages);
        if (!__all_sync(0xffffffffu, bulk::wait(R.full(s), (uint32_t)((i / hs::kStages) & 1)))) {
            if (lane == 0) atomicExch(err, 1);
            return;
        }
        const int f = (int)(j % F);
        const unsigned char* st = R.stage + (size_t)s * hs::kStageBytes;
        const float* sv = R.vec + s * hs::kVecFloats;
        // The stage is one [Rt][n8] row matrix (its pieces are whole rows of
        // one length, back to back).  Lane p holds piece p: its first row
        // (prefix sum of the row counts), x offset, w index and rank.
        const int np = R.meta[s].np;
        int rows = 0, vo = 0, wv = 0, r = 0;
        if (lane < np) {
            const HsPiece& pm = R.meta[s].p[lane];
            rows = pm.rows;
            vo = pm.vo;
            wv = pm.wv;
            r = pm.r;
        }
        int rend = rows;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, rend, o);
            if (lane >= o) rend += t;
        }
        const int rs = rend - rows;
        const int Rt = __shfl_sync(0xffffffffu, rend, 31);
        const int n8 = R.meta[s].p[0].n8;
        // lanes per row: at least four 16-byte quads per lane (few shuffle
        // levels), at least 4 lanes; when a row's lanes span less than 128
        // bytes, the rows of a unit visit their quads in rotated order so
        // that they fall on different banks
        const int nq = n8 / VW;
        const int lg = nq <= 16 ? 2 : (nq <= 32 ? 3 : (nq <= 64 ? 4 : 5));
        const int sw = 1 << lg, sl = lane & (sw - 1), sub = lane >> lg;
        const int per = 32 >> lg;
        const int nql = nq >> lg;                 // quads per lane when sw divides nq
        const bool rot = (nql << lg) == nq;
        const T* V0 = reinterpret_cast<const T*>(st);
        // the loop bound is warp-uniform, so every lane reaches the shuffles
        for (int u = warp; u * per < Rt; u += hs::kConsumerWarps) {
            const int row = u * per + sub;
            // piece of each sub-warp's row: the last lane whose first row is <= it.
            // Usually one piece holds all rows of the unit: two ballots decide it.
            const unsigned m0 = __ballot_sync(0xffffffffu, lane < np && rs <= u * per);
            const unsigned m1 = __ballot_sync(0xffffffffu, lane < np && rs <= u * per + per - 1);
            int pp = 31 - __clz(m0);
            if (m0 != m1) {
                for (int k = 1; k < per; ++k) {
                    const unsigned m = __ballot_sync(0xffffffffu, lane < np && rs <= u * per + k);
                    if (k == sub) pp = 31 - __clz(m);
                }
            }
            const int pvo = __shfl_sync(0xffffffffu, vo, pp), pwv = __shfl_sync(0xffffffffu, wv, pp);
            const int pr = __shfl_sync(0xffffffffu, r, pp), prs = __shfl_sync(0xffffffffu, rs, pp);
            const bool rok = row < Rt;
            float acc = 0.f, acc2 = 0.f;
            if (rok) {
                const T* vr = V0 + row * n8;
                const float* xs = sv + pvo;
                if (rot && nql == 4) {
                    // exactly four quads per lane, visited from quad (sub mod 4)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int q = sl + (((sub + k) & 3) << lg);
                        float v[VW], x[VW];
                        lds16(vr + q * VW, v);
#pragma unroll
                        for (int e = 0; e < VW; e += 4) lds16(xs + q * VW + e, x + e);
#pragma unroll
                        for (int e = 0; e < VW; e += 2) {
                            acc += v[e] * x[e];
                            acc2 += v[e + 1] * x[e + 1];
                        }
                    }
                } else if (rot) {
                    int t = sub % nql;
                    for (int k = 0; k < nql; ++k) {
                        const int q = sl + (t << lg);
                        float v[VW], x[VW];
                        lds16(vr + q * VW, v);
#pragma unroll
                        for (int e = 0; e < VW; e += 4) lds16(xs + q * VW + e, x + e);
#pragma unroll
                        for (int e = 0; e < VW; e += 2) {
                            acc += v[e] * x[e];
                            acc2 += v[e + 1] * x[e + 1];
                        }
                        t = t + 1 == nql ? 0 : t + 1;
                    }
                } else {
                    for (int q = sl; q < nq; q += sw) {
                        float v[VW], x[VW];
                        lds16(vr + q * VW, v);
#pragma unroll
                        for (int e = 0; e < VW; e += 4) lds16(xs + q * VW + e, x + e);
#pragma unroll
                        for (int e = 0; e < VW; e += 2) {
                            acc += v[e] * x[e];
                            acc2 += v[e + 1] * x[e + 1];
                        }
                    }
                }
                acc += acc2;
            }
            for (int o = sw >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, sw);
            if (rok && sl == 0) W[(int64_t)pwv + (row - prs) + (int64_t)f * pr] = acc;
        }
        __syncwarp();
        if (lane == 0) bulk::arrive(R.empty(s));
    }
}

// ---------------------------------------------------------------------------
// phase 2, y_f[rows(l)] = sum_far U_g w_{b,f} + sum_dense A_g x_f[cols(b)]:
// items (leaf, f) in the host's order (largest leaves first, the F
// frequencies of a leaf together).  A leaf's records are consecutive and each
// holds k-rows of one kind only, so a stage is one [K][m8] array with its K
// vector values beside it.
// ---------------------------------------------------------------------------
template <class E>
__device__ __forceinline__ void hs_p2_rows(const E* A, const float* sv, int K, int m8, int k0, int nslice, float4& acc0,
                                           float4& acc1)
{
    int k = k0;
    for (; k + nslice < K; k += 2 * nslice) {
        fma4(acc0, lds4(A + k * m8), sv[k]);
        fma4(acc1, lds4(A + (k + nslice) * m8), sv[k + nslice]);
    }
    if (k < K) fma4(acc0, lds4(A + k * m8), sv[k]);
}

template <class T>
__global__ void __launch_bounds__(hs::kThreads) hmv_s2(const HsLoad* __restrict__ loads,
                                                       const int* __restrict__ leaf_load0,
                                                       const int2* __restrict__ items, int nitems,
                                                       const P2Leaf* __restrict__ leaves, const T* __restrict__ far,
                                                       const float* __restrict__ nearp, const float* __restrict__ X,
                                                       const float* __restrict__ W, float* __restrict__ Y, int N,
                                                       const int* __restrict__ fgroup, int* err)
{
    const HsRing R = hs_ring_init();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= hs::kConsumerWarps) {
        const int s = warp - hs::kConsumerWarps;
        // cursor over this CTA's stage sequence: item j, its records [ld, ld1)
        int j = blockIdx.x, ld = 0, ld1 = 0;
        int2 it = make_int2(0, 0);
        auto enter = [&]() {   // first record of item j or a later item
            for (; j < nitems; j += gridDim.x) {
                it = items[j];
                ld = leaf_load0[it.x];
                ld1 = leaf_load0[it.x + 1];
                if (ld < ld1) return;
            }
        };
        auto next = [&]() {    // the stage after the cursor's
            if (++ld < ld1) return;
            j += gridDim.x;
            enter();
        };
        enter();
        for (int k = 0; k < s && j < nitems; ++k) next();
        HsRec nxt;
        if (j < nitems) hs_fetch(nxt, loads + ld, it.y, fgroup);
        uint32_t u = 0;
        for (; j < nitems; ++u) {
            const HsRec cur = nxt;
            for (int k = 0; k < hs::kStages && j < nitems; ++k) next();
            if (j < nitems) hs_fetch(nxt, loads + ld, it.y, fgroup);
            if (!hs_fill<T>(R, s, u, cur, far, nearp, X, W, N, true)) {
                if (lane == 0) atomicExch(err, 1);
                hs_drain(R, s, u);
                return;
            }
        }
        hs_drain(R, s, u);   // the last copies have landed before this warp leaves
        return;
    }
    const int tid = threadIdx.x;   // consumer thread 0 .. kConsumers - 1
    int64_t i = 0;
    for (int j = blockIdx.x; j < nitems; j += gridDim.x) {
        const int2 it = items[j];
        const P2Leaf L = leaves[it.x];
        const int f = it.y;
        const int ncol = L.m8 >> 2;   // float4 columns (<= 256)
        const int nslice = hs::kConsumers / ncol;
        const int c = tid % ncol, slice = tid / ncol;
        const bool act = slice < nslice;
        float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
        int kbase = 0;   // k rows of the leaf's earlier stages: slices take rows round robin
        const int ld0 = leaf_load0[it.x], ld1 = leaf_load0[it.x + 1];
        for (int ld = ld0; ld < ld1; ++ld, ++i) {
            const int s = (int)(i % hs::kStages);
            const bool ok = bulk::wait(R.full(s), (uint32_t)((i / hs::kStages) & 1));
            // every consumer warp leaves together, so none is left at a barrier
            if (bulk::bar_or(2, hs::kConsumers, !ok)) {
                if (tid == 0) atomicExch(err, 1);
                return;
            }
            const int K = R.meta[s].K;
            if (act) {
                const unsigned char* st = R.stage + (size_t)s * hs::kStageBytes;
                const float* sv = R.vec + s * hs::kVecFloats;
                const int k0 = (slice - kbase % nslice + nslice) % nslice;
                if (R.meta[s].kind == 0)
                    hs_p2_rows(reinterpret_cast<const T*>(st) + 4 * c, sv, K, L.m8, k0, nslice, acc0, acc1);
                else
                    hs_p2_rows(reinterpret_cast<const float*>(st) + 4 * c, sv, K, L.m8, k0, nslice, acc0, acc1);
            }
            kbase += K;
            __syncwarp();
            if (lane == 0) bulk::arrive(R.empty(s));
        }
        // the leaf's rows: sum the slices (row ownership, no atomics)
        R.red[tid] = make_float4(acc0.x + acc1.x, acc0.y + acc1.y, acc0.z + acc1.z, acc0.w + acc1.w);
        bulk::bar_sync(1, hs::kConsumers);
        if (tid < ncol) {
            float4 t = R.red[tid];
            for (int sl = 1; sl < nslice; ++sl) {
                const float4 u = R.red[sl * ncol + tid];
                t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
            }
            const int r0 = 4 * tid;
            float* __restrict__ y = Y + (int64_t)f * N + L.row0;
            if (r0 < L.m) y[r0] = t.x;
            if (r0 + 1 < L.m) y[r0 + 1] = t.y;
            if (r0 + 2 < L.m) y[r0 + 2] = t.z;
            if (r0 + 3 < L.m) y[r0 + 3] = t.w;
        }
        // the slice sums are read before the next leaf writes red again
        bulk::bar_sync(1, hs::kConsumers);
    }
}

}  // namespace rt
