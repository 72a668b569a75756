// rt_hmv_dev.cuh -- device bodies of the two H-matvec phases (see
// rt_hmatvec.cu for the data layout); shared by the per-operator kernels and
// the persistent batched kernel so that both perform the same arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rt_internal.h"

namespace rt {

struct P1Row {
    int64_t v;        // element offset of row k of V^T for group 0
    int64_t gstride;  // elements between groups (r * n8)
    int64_t w;        // w index for f = 0 (w_base + k); frequency f adds f * r
    int n, col0, r, pad;
};

struct P1Item {
    int row0, row1;   // range of the row list
    int sw;           // sub-warp width (8, 16 or 32)
    int pad;
};

struct P2Leaf {
    int row0, m, m8, seg0, nseg, pad;
};

struct P2Seg {
    int64_t a;        // element offset of the chunk for group 0
    int64_t gstride;  // elements between groups (count * m8)
    int64_t vbase;    // far: w_base of the block; dense: column offset col0
    int count;        // r (far) or n (dense)
    int kind;         // 0 far, 1 dense
};

// ---- element loads ---------------------------------------------------------
template <class T>
struct VecW;
template <>
struct VecW<float> {
    static constexpr int n = 4;
};
template <>
struct VecW<__nv_bfloat16> {
    static constexpr int n = 8;
};
template <>
struct VecW<__half> {
    static constexpr int n = 8;
};

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }

// 16-byte load of VecW<T>::n elements, converted to float
__device__ __forceinline__ void load16(const float* p, float* v)
{
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}
__device__ __forceinline__ void load16(const __nv_bfloat16* p, float* v)
{
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    const unsigned u[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[k]));
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}
__device__ __forceinline__ void load16(const __half* p, float* v)
{
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    const unsigned u[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u[k]));
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}

// 4 consecutive elements (16 bytes for float, 8 for 16-bit types), converted
__device__ __forceinline__ float4 load4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 load4(const __nv_bfloat16* p)
{
    const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&a.x));
    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&a.y));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ float4 load4(const __half* p)
{
    const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&a.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&a.y));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// add the low 16-bit parts of a split far field (kLo) to values just loaded
template <bool kLo, class T, int n>
__device__ __forceinline__ void add_lo16(const T* __restrict__ lo, float* v)
{
    if constexpr (kLo) {
        float l[n];
        load16(lo, l);
#pragma unroll
        for (int e = 0; e < n; ++e) v[e] += l[e];
    }
}
template <bool kLo, class T>
__device__ __forceinline__ float4 add_lo4(const T* __restrict__ lo, float4 v)
{
    if constexpr (kLo) {
        const float4 l = load4(lo);
        v.x += l.x; v.y += l.y; v.z += l.z; v.w += l.w;
    }
    return v;
}

// phase 1 body: one item (a run of rank rows) for frequency f of group g, 256 threads.
// kLo: the far field is stored as 16-bit high parts `far` plus 16-bit
// remainders `far_lo` at the same offsets (refinement sweeps read both).
template <class T, bool kLo = false>
__device__ __forceinline__ void hmv_p1_body(const P1Item it, int f, int g, const P1Row* __restrict__ rows,
                                            const T* __restrict__ far, const T* __restrict__ far_lo,
                                            const float* __restrict__ X, float* __restrict__ W, int N)
{
    constexpr int VW = VecW<T>::n;
    const int sw = it.sw;
    const int lane = threadIdx.x & 31;
    const int sl = lane & (sw - 1);                 // lane within the sub-warp
    const int per_warp = 32 / sw;                   // rows handled by one warp at a time
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const float* __restrict__ xf = X + (int64_t)f * N;
    // the loop bound is warp-uniform, so every lane reaches the shuffles below
    for (int rb = it.row0 + warp * per_warp; rb < it.row1; rb += nwarps * per_warp) {
        const int ri = rb + lane / sw;
        const bool ok = ri < it.row1;
        float s = 0.f;
        P1Row rw{};
        if (ok) {
            rw = rows[ri];
            const int64_t vo = rw.v + (int64_t)g * rw.gstride;
            const T* __restrict__ v = far + vo;
            const T* __restrict__ vl = kLo ? far_lo + vo : nullptr;
            const float* __restrict__ x = xf + rw.col0;
            const int nv = rw.n - rw.n % VW;
            float s0 = 0.f, s1 = 0.f;
            int j = sl * VW;
            for (; j + sw * VW < nv; j += 2 * sw * VW) {
                float a[VW], b[VW];
                load16(v + j, a);
                load16(v + j + sw * VW, b);
                add_lo16<kLo, T, VW>(vl + j, a);
                add_lo16<kLo, T, VW>(vl + j + sw * VW, b);
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    s0 += a[e] * __ldg(x + j + e);
                    s1 += b[e] * __ldg(x + j + sw * VW + e);
                }
            }
            for (; j < nv; j += sw * VW) {
                float a[VW];
                load16(v + j, a);
                add_lo16<kLo, T, VW>(vl + j, a);
#pragma unroll
                for (int e = 0; e < VW; ++e) s0 += a[e] * __ldg(x + j + e);
            }
            for (int t = nv + sl; t < rw.n; t += sw) s0 += (to_f(v[t]) + (kLo ? to_f(vl[t]) : 0.f)) * __ldg(x + t);
            s = s0 + s1;
        }
        for (int o = sw >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, sw);
        if (ok && sl == 0) W[rw.w + (int64_t)f * rw.r] = s;
    }
}

// phase 1: grid (items, F), 256 threads
template <class T, bool kLo>
__global__ void __launch_bounds__(256) hmv_phase1(const P1Item* __restrict__ items, const P1Row* __restrict__ rows,
                                                  const T* __restrict__ far, const T* __restrict__ far_lo,
                                                  const float* __restrict__ X, float* __restrict__ W, int N,
                                                  const int* __restrict__ fgroup)
{
    const int f = blockIdx.y;
    hmv_p1_body<T, kLo>(items[blockIdx.x], f, fgroup[f], rows, far, far_lo, X, W, N);
}

// phase-2 reads of w: through the read-only path, or L2-coherent when w is
// produced by other CTAs of the same (persistent) launch
template <bool kCoherentW>
__device__ __forceinline__ float ld_w(const float* p)
{
    if constexpr (kCoherentW) return __ldcg(p);
    else return __ldg(p);
}

// phase 2 body: one leaf for frequency f of group g, 256 threads;
// thread owns rows 4c..4c+3 and a slice of each segment's count
template <class T, bool kCoherentW, bool kLo = false>
__device__ __forceinline__ void hmv_p2_body(const P2Leaf L, int f, int g, const P2Seg* __restrict__ segs,
                                            const T* __restrict__ far, const T* __restrict__ far_lo,
                                            const float* __restrict__ nearp,
                                            const float* __restrict__ X, const float* __restrict__ W,
                                            float* __restrict__ Y, int N, float4* red)
{
    const int ncol = L.m8 >> 2;                     // float4 columns (<= 256)
    const int nslice = blockDim.x / ncol;
    const int c = threadIdx.x % ncol, slice = threadIdx.x / ncol;
    const bool act = slice < nslice;
    float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
    if (act) {
        for (int si = L.seg0; si < L.seg0 + L.nseg; ++si) {
            const P2Seg sg = segs[si];
            if (sg.kind == 0) {
                const int64_t ao = sg.a + (int64_t)g * sg.gstride + 4 * c;
                const T* __restrict__ a = far + ao;
                const T* __restrict__ al = kLo ? far_lo + ao : nullptr;
                const float* __restrict__ w = W + sg.vbase + (int64_t)f * sg.count;
                int k = slice;
                for (; k + nslice < sg.count; k += 2 * nslice) {
                    const float4 p = add_lo4<kLo>(al + (int64_t)k * L.m8, load4(a + (int64_t)k * L.m8));
                    const float4 q = add_lo4<kLo>(al + (int64_t)(k + nslice) * L.m8, load4(a + (int64_t)(k + nslice) * L.m8));
                    const float wp = ld_w<kCoherentW>(w + k), wq = ld_w<kCoherentW>(w + k + nslice);
                    acc0.x += p.x * wp; acc0.y += p.y * wp; acc0.z += p.z * wp; acc0.w += p.w * wp;
                    acc1.x += q.x * wq; acc1.y += q.y * wq; acc1.z += q.z * wq; acc1.w += q.w * wq;
                }
                for (; k < sg.count; k += nslice) {
                    const float4 p = add_lo4<kLo>(al + (int64_t)k * L.m8, load4(a + (int64_t)k * L.m8));
                    const float wp = ld_w<kCoherentW>(w + k);
                    acc0.x += p.x * wp; acc0.y += p.y * wp; acc0.z += p.z * wp; acc0.w += p.w * wp;
                }
            } else {
                const float* __restrict__ a = nearp + sg.a + (int64_t)g * sg.gstride + 4 * c;
                const float* __restrict__ x = X + (int64_t)f * N + sg.vbase;
                int k = slice;
                for (; k + nslice < sg.count; k += 2 * nslice) {
                    const float4 p = load4(a + (int64_t)k * L.m8);
                    const float4 q = load4(a + (int64_t)(k + nslice) * L.m8);
                    const float xp = __ldg(x + k), xq = __ldg(x + k + nslice);
                    acc0.x += p.x * xp; acc0.y += p.y * xp; acc0.z += p.z * xp; acc0.w += p.w * xp;
                    acc1.x += q.x * xq; acc1.y += q.y * xq; acc1.z += q.z * xq; acc1.w += q.w * xq;
                }
                for (; k < sg.count; k += nslice) {
                    const float4 p = load4(a + (int64_t)k * L.m8);
                    const float xp = __ldg(x + k);
                    acc0.x += p.x * xp; acc0.y += p.y * xp; acc0.z += p.z * xp; acc0.w += p.w * xp;
                }
            }
        }
    }
    red[threadIdx.x] = make_float4(acc0.x + acc1.x, acc0.y + acc1.y, acc0.z + acc1.z, acc0.w + acc1.w);
    __syncthreads();
    if (threadIdx.x < ncol) {
        float4 t = red[threadIdx.x];
        for (int sl = 1; sl < nslice; ++sl) {
            const float4 u = red[sl * ncol + threadIdx.x];
            t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
        }
        const int r0 = 4 * threadIdx.x;
        float* __restrict__ y = Y + (int64_t)f * N + L.row0;
        if (r0 < L.m) y[r0] = t.x;
        if (r0 + 1 < L.m) y[r0 + 1] = t.y;
        if (r0 + 2 < L.m) y[r0 + 2] = t.z;
        if (r0 + 3 < L.m) y[r0 + 3] = t.w;
    }
}

// phase 2: grid (leaves, F), 256 threads
template <class T, bool kLo>
__global__ void __launch_bounds__(256) hmv_phase2(const P2Leaf* __restrict__ leaves, const P2Seg* __restrict__ segs,
                                                  const T* __restrict__ far, const T* __restrict__ far_lo,
                                                  const float* __restrict__ nearp, const float* __restrict__ X,
                                                  const float* __restrict__ W, float* __restrict__ Y, int N,
                                                  const int* __restrict__ fgroup)
{
    __shared__ float4 red[256];
    const int f = blockIdx.y;
    hmv_p2_body<T, false, kLo>(leaves[blockIdx.x], f, fgroup[f], segs, far, far_lo, nearp, X, W, Y, N, red);
}


}  // namespace rt
