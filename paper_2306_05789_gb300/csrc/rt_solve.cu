// rt_solve.cu -- the monotone fixed point of Section 1.3 (eq. (algo)) on the GPU:
//   S^k_nu  = a_nu J^k_nu + (1 - a_nu) B_nu(T^k)            (kappa is inside G)
//   J^{k+1} = Sbar^E + Gbar S^k
//   T^{k+1}: sum_nu w_nu c_nu (1 - a_nu) (J^{k+1}_nu - B_nu(T)) = 0 per vertex
//            (FP64 Newton safeguarded by bisection; grey: T = (J/sigma)^{1/4},
//             eq. (grey) of Section 3)
//   residual ||J^{k+1} - J^k||_2 / ||J^{k+1}||_2 in FP64, deterministic two-pass reduction.
// The loop runs in tree order; check_every iterations are captured in one CUDA
// graph and replayed; the host reads the residual history between replays.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "rt_internal.h"
#include "rt_newton.cuh"

namespace rt {

constexpr double kSigma = 6.493939402266829;   // pi^4 / 15
constexpr int kRedThreads = 256;

__device__ __forceinline__ double planck(double nu, double T)
{
    if (!(T > 0.0)) return 0.0;
    const double x = nu / T;
    if (x > 700.0) return 0.0;
    return nu * nu * nu / expm1(x);
}

template <class V>
__global__ void fp_init(V* J, double* T, int64_t nJ, int N, double T0, int keepJ)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nJ; e += (int64_t)gridDim.x * blockDim.x) {
        if (!keepJ) J[e] = V(0);
        if (e < N) T[e] = T0;
    }
}

// S = a J + (1-a) B(T)
// S = a J + (1-a) B(T), times c_f / c_g for binned channels (fscale non-null),
// so that the group operator G_g applied to S gives the channel's c_f kappa(y)
// prefactor
template <class V>
__global__ void fp_source(const V* __restrict__ J, const double* __restrict__ T, V* __restrict__ S,
                          const double* __restrict__ fq, int N, int F, int grey, const double* __restrict__ fscale)
{
    const int64_t total = (int64_t)N * F;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(e / N), i = (int)(e % N);
        const double a = fq[4 * f + 2];
        const double t = T[i];
        const double B = grey ? kSigma * t * t * t * t : planck(fq[4 * f + 0], t);
        const double v = a * (double)J[e] + (1.0 - a) * B;
        S[e] = (V)(fscale ? v * fscale[f] : v);
    }
}

// J <- SE + Y, per-CTA partial sums of (Jnew - Jold)^2 and Jnew^2
template <class V>
__global__ void __launch_bounds__(kRedThreads) fp_update(V* __restrict__ J, const V* __restrict__ Y,
                                                         const V* __restrict__ SE, int64_t total,
                                                         double* __restrict__ part)
{
    double d2 = 0.0, n2 = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const V jn = SE[e] + Y[e];
        const double d = (double)jn - (double)J[e];
        d2 += d * d;
        n2 += (double)jn * (double)jn;
        J[e] = jn;
    }
    __shared__ double s[2][kRedThreads / 32];
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
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) {
            a += s[0][w];
            b += s[1][w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// res[iter] = sqrt(sum d2 / sum n2); iter = *counter (then incremented)
__global__ void fp_reduce(const double* __restrict__ part, int nparts, double* res, int* counter, int cap)
{
    __shared__ double s[2][32];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s[0][threadIdx.x >> 5] = a;
        s[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ta += s[0][w];
            tb += s[1][w];
        }
        const int it = *counter;
        if (it < cap) res[it] = tb > 0.0 ? sqrt(ta / tb) : (ta > 0.0 ? INFINITY : 0.0);
        *counter = it + 1;
    }
}

template <class V, int LPV>
__global__ void __launch_bounds__(256) fp_newton(const V* __restrict__ J, double* __restrict__ T,
                                                 const double* __restrict__ fq, int N, int F, int grey,
                                                 int* __restrict__ fail)
{
    constexpr int VPW = 32 / LPV;
    const int lane = threadIdx.x & 31, sl = lane & (LPV - 1);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * VPW; base < N;
         base += nw * VPW) {
        const int64_t i = base + lane / LPV;
        if (i >= N) continue;   // whole vertex segments drop out together
        if (grey) {
            if (sl == 0) {
                const double j = (double)J[i];
                T[i] = j > 0.0 ? sqrt(sqrt(j / kSigma)) : 0.0;
            }
            continue;
        }
        const unsigned m = seg_mask<LPV>(lane);
        double rhs = 0.0;
        for (int f = sl; f < F; f += LPV) rhs += fq[4 * f + 1] * (double)J[(int64_t)f * N + i];
#pragma unroll
        for (int o = LPV >> 1; o > 0; o >>= 1) rhs += __shfl_xor_sync(m, rhs, o);
        if (!(rhs > 0.0)) {
            if (sl == 0) T[i] = 0.0;
            continue;
        }
        double t = 0.0;
        const bool ok = solve_temperature<LPV>(fq, F, rhs, lane, T[i], t);
        if (sl == 0) {
            if (!ok) atomicOr(fail, 1);
            T[i] = t;
        }
    }
}

static int grid_elem(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}

template <class V>
static int one_iteration(Operator& op, cudaStream_t s, int grey, int* d_counter, int* d_fail, int cap,
                         std::string& err)
{
    const int N = op.N, F = op.F;
    const int64_t tot = (int64_t)N * F;
    fp_source<V><<<grid_elem(tot), 256, 0, s>>>((const V*)op.d_J, op.d_T, (V*)op.d_S, op.d_fq, N, F, grey,
                                                  op.binned ? op.d_fscale : nullptr);
    RT_CUDA_TRY(cudaGetLastError());
    int rc = apply_tree(op, op.d_S, op.d_Y, s, err);
    if (rc) return rc;
    fp_update<V><<<op.n_part, kRedThreads, 0, s>>>((V*)op.d_J, (const V*)op.d_Y, (const V*)op.d_SE, tot, op.d_part);
    fp_reduce<<<1, 256, 0, s>>>(op.d_part, op.n_part, op.d_res, d_counter, cap);
    // LPV lanes per vertex: the power of two >= F (1 for the grey closed form)
    const int lpv = grey ? 1 : (F <= 1 ? 1 : F <= 2 ? 2 : F <= 4 ? 4 : F <= 8 ? 8 : F <= 16 ? 16 : 32);
    const int64_t warps = ((int64_t)N * lpv + 31) / 32;
    const int gn = (int)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 152 * 32));
#define RT_NEWTON(L) \
    fp_newton<V, L><<<gn, 256, 0, s>>>((const V*)op.d_J, op.d_T, op.d_fq, N, F, grey, d_fail)
    switch (lpv) {
        case 1: RT_NEWTON(1); break;
        case 2: RT_NEWTON(2); break;
        case 4: RT_NEWTON(4); break;
        case 8: RT_NEWTON(8); break;
        case 16: RT_NEWTON(16); break;
        default: RT_NEWTON(32); break;
    }
#undef RT_NEWTON
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

template <class V>
static int solve_impl(Operator& op, const rt_solve_opts& o, void* J_out, double* T_out, rt_solve_stats& st,
                      cudaStream_t s, std::string& err)
{
    int rc;
    const int N = op.N, F = op.F;
    const int64_t tot = (int64_t)N * F;
    const int cap = std::max(1, o.max_iter);
    const int every = std::max(1, o.check_every);
    if (!op.d_J) {
        op.stream = s;
        V *J, *S, *Y;
        if ((rc = dev_alloc(op, &J, tot, err))) return rc;
        if ((rc = dev_alloc(op, &S, tot, err))) return rc;
        if ((rc = dev_alloc(op, &Y, tot, err))) return rc;
        op.d_J = J;
        op.d_S = S;
        op.d_Y = Y;
        if ((rc = dev_alloc(op, &op.d_T, N, err))) return rc;
        op.n_part = (int)std::max<int64_t>(1, std::min<int64_t>((tot + kRedThreads - 1) / kRedThreads, 152 * 8));
        if ((rc = dev_alloc(op, &op.d_part, 2 * (size_t)op.n_part, err))) return rc;
    }
    double* d_res = nullptr;
    int* d_ctr = nullptr;
    RT_CUDA_TRY(cudaMallocAsync((void**)&d_res, sizeof(double) * cap, s));
    RT_CUDA_TRY(cudaMallocAsync((void**)&d_ctr, sizeof(int) * 2, s));
    RT_CUDA_TRY(cudaMemsetAsync(d_ctr, 0, sizeof(int) * 2, s));
    op.d_res = d_res;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    // initial state (J0 from the caller when requested)
    if (o.use_J0) {
        if ((rc = permute_vectors(op, J_out, op.d_J, 1, sizeof(V) == 8, F, s))) {
            err = "permute failed";
            return rc;
        }
    }
    fp_init<V><<<grid_elem(tot), 256, 0, s>>>((V*)op.d_J, op.d_T, tot, N, o.T0, o.use_J0);
    RT_CUDA_TRY(cudaGetLastError());

    std::vector<double> hres(cap);
    int iters = 0;
    bool converged = false;
    double last = INFINITY;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    int graph_len = 0, graph_lo = -1;
    // operators with split (high + low) far fields start on the high parts
    // alone and switch to both once the residual reaches refine_tol
    op.use_lo = (op.d_far_lo && !(o.refine_tol > 0.0)) ? 1 : 0;
    while (iters < cap && !converged) {
        const int todo = std::min(every, cap - iters);
        if (o.use_graph) {
            if (!gexec || graph_len != todo || graph_lo != op.use_lo) {
                if (gexec) cudaGraphExecDestroy(gexec);
                if (graph) cudaGraphDestroy(graph);
                gexec = nullptr;
                graph = nullptr;
                // capture on a library-owned stream (the caller's stream may be the
                // legacy default stream, which cannot be captured); replay on `s`
                if (!op.cap_stream) RT_CUDA_TRY(cudaStreamCreateWithFlags(&op.cap_stream, cudaStreamNonBlocking));
                RT_CUDA_TRY(cudaStreamBeginCapture(op.cap_stream, cudaStreamCaptureModeThreadLocal));
                int crc = RT_OK;
                for (int k = 0; k < todo && crc == RT_OK; ++k)
                    crc = one_iteration<V>(op, op.cap_stream, op.grey, d_ctr, d_ctr + 1, cap, err);
                cudaError_t ce = cudaStreamEndCapture(op.cap_stream, &graph);
                if (crc) return crc;
                if (ce != cudaSuccess) {
                    err = std::string("graph capture: ") + cudaGetErrorString(ce);
                    return RT_ECUDA;
                }
                RT_CUDA_TRY(cudaGraphInstantiate(&gexec, graph, 0));
                graph_len = todo;
                graph_lo = op.use_lo;
            }
            RT_CUDA_TRY(cudaGraphLaunch(gexec, s));
        } else {
            for (int k = 0; k < todo; ++k)
                if ((rc = one_iteration<V>(op, s, op.grey, d_ctr, d_ctr + 1, cap, err))) return rc;
        }
        RT_CUDA_TRY(cudaMemcpyAsync(hres.data() + iters, d_res + iters, sizeof(double) * todo, cudaMemcpyDeviceToHost, s));
        RT_CUDA_TRY(cudaStreamSynchronize(s));
        for (int k = 0; k < todo; ++k) {
            last = hres[iters + k];
            if (last <= o.tol && (!op.d_far_lo || op.use_lo)) converged = true;
        }
        iters += todo;
        if (op.d_far_lo && !op.use_lo && last <= std::max(o.refine_tol, o.tol)) op.use_lo = 1;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    op.use_lo = 0;
    if ((rc = apply_check_error(op, s, err))) return rc;   // a bounded apply wait gave up
    int fail = 0;
    RT_CUDA_TRY(cudaMemcpyAsync(&fail, d_ctr + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    // results back to caller order
    if ((rc = permute_vectors(op, op.d_J, J_out, 0, sizeof(V) == 8, F, s))) {
        err = "permute failed";
        return rc;
    }
    if ((rc = permute_vectors(op, op.d_T, T_out, 0, 1, 1, s))) {
        err = "permute failed";
        return rc;
    }
    cudaEventRecord(e1, s);
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(d_res, s);
    cudaFreeAsync(d_ctr, s);
    op.d_res = nullptr;
    st.iters = iters;
    st.converged = converged ? 1 : 0;
    st.residual = last;
    st.ms_total = ms;
    if (fail) {
        err = "temperature Newton solve did not converge at some vertex";
        return RT_ENOCONV;
    }
    if (!converged) {
        err = "fixed point did not reach tol within max_iter";
        return RT_ENOCONV;
    }
    return RT_OK;
}

int solve_fixed_point(Operator& op, const rt_solve_opts& o, void* J, double* T, rt_solve_stats& st, cudaStream_t s,
                      std::string& err)
{
    if (op.vec64) return solve_impl<double>(op, o, J, T, st, s, err);
    return solve_impl<float>(op, o, J, T, st, s, err);
}

}  // namespace rt
