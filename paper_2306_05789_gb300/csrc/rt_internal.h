// rt_internal.h -- internal structures of the radiative-transfer library.
//
// Layout conventions (all device arrays, tree order of vertices):
//   xyz      : float4 [N] (x, y, z, 0) and double [N][3]
//   tet      : int4 [T] vertex ids in tree order
//   tgeo     : float4/dbl4 [T] (centroid x, y, z, diameter); tvol [T]
//   vt_ptr   : int [N+1], vt_idx: int [nnz] packed (tet << 2) | local vertex slot
//   vectors  : [F][N] frequency-major
//   rows of every block are split into leaf chunks (the leaves of the cluster
//   tree that the block's row cluster contains); padded sizes are multiples of 8
//   far block b, group g : V^T [r][n8] at far_v_off[b] + g*r*n8;
//                          chunk c: U^T [r][m8_c] at far_u_off[b] + off_c + g*r*m8_c
//   dense block b, chunk c, group g: A^T [n][m8_c] at dense_off[b] + off_c + g*n*m8_c
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rt.h"

namespace rt {

constexpr int kMaxGroups = 64;
constexpr int kMaxWalls = 3;     // planar reflective walls per problem
constexpr int kMaxXTerms = 5;    // reflected terms beyond the first wall's: 2 walls + 3 corners
constexpr int kMaxObst = 4;      // opaque boxes per problem
constexpr int kMaxGauss = 32;
constexpr int kSubCols = 256;   // columns per sub-cluster in row evaluations
constexpr double kPi = 3.14159265358979323846;

struct alignas(16) dbl4 {
    double x, y, z, w;
};
inline dbl4 make_dbl4(double x, double y, double z, double w) { return dbl4{x, y, z, w}; }

// Kernel parameters of one instance (passed by value to kernels).
struct KernelParams {
    int N;              // vertices
    int T;              // tetrahedra
    int kappa_kind;
    float k0f, ampf;
    double k0, amp;
    int has_wall;       // R0 != 0 and a wall is present
    double wp[3], wn[3];
    double R0;
    // further reflected terms (walls beyond the first with R0 != 0, then the corner
    // paths of perpendicular pairs): kind 1 = one reflection on wall xa, kind 2 =
    // reflections on walls xa and xb; walls indexed in wps / wns / wR
    int n_extra;
    int xkind[kMaxXTerms], xa[kMaxXTerms], xb[kMaxXTerms];
    double wps[kMaxWalls][3], wns[kMaxWalls][3], wR[kMaxWalls];
    // cellwise-constant kappa (kappa_kind == RT_KAPPA_GRID): gdims cells of the
    // box [glo, ghi], values in kgrid32 / kgrid64
    const float* kgrid32;
    const double* kgrid64;
    int gdims[3];
    double glo[3], ghi[3];
    // opaque boxes (kappa = +infinity inside)
    int n_obst;
    double olo[kMaxObst][3], ohi[kMaxObst][3];
    // the instance needs the general kernels (further walls, grid or obstacles)
    int ext;
    int G;              // groups
    double c[kMaxGroups];
    float cf[kMaxGroups];
    // group scales in arithmetic progression c_g = c_0 + g dc: the FP32 paths
    // get exp(-c_g tau) = exp(-c_0 tau) exp(-dc tau)^g by repeated products
    int c_arith;
    float c0f, dcf;
    int ngauss;
    int line_closed;    // closed-form Gauss sums for the sin-product kappa (FP32 paths)
    // Gauss-Legendre nodes mapped to [0,1] (u = (1+t)/2) and half weights
    float gu32[kMaxGauss], gw32[kMaxGauss];
    double gu64[kMaxGauss], gw64[kMaxGauss];
    // device geometry (tree order)
    const float4* xyz32;
    const double* xyz64;
    const int4* tet;
    const float4* tgeo32;
    const dbl4* tgeo64;
    const float* tvol32;
    const double* tvol64;
    const int* vt_ptr;
    const int* vt_idx;
    // assembly work counters (may be null): [0] kernel terms evaluated (one direct or
    // one reflected value e^{-c tau} / r^2 at a point pair), [1] optical depths
    unsigned long long* work;
};

// A rectangular set of entries G_g[i0 + ii][j0 + jj], ii < ni, jj < nj, written
// to out[base + g*gs + ii*is + jj*js] (float or double, per launch).
struct EntrySpan {
    int i0, ni, j0, nj;
    int64_t base, gs, is, js;
    int64_t first;   // prefix: index of this span's first entry in the launch
};

// One far (admissible) block in tree order.
struct FarBlock {
    int row0, m, col0, n;
    int tc, sc;   // row and column cluster ids in Plan::clusters
};

// Node of the cluster tree: points [start, start + size) in tree order.
struct ClusterNode {
    int start, size, left, right;
};

inline int round8(int x) { return (x + 7) & ~7; }

// Leaf chunk of a block's rows: rows [rbeg, rbeg + m) of the block (local),
// padded to m8 = round8(m), stored at offset off from the block's base.
struct Chunk {
    int leaf, rbeg, m, m8;
    int64_t off;
};

// Host-side plan of one instance.
struct Plan {
    int N = 0;
    int leaf = 64;
    std::vector<int> perm;      // tree position -> original vertex id
    std::vector<int> iperm;     // original vertex id -> tree position
    std::vector<int> leaf_start, leaf_size;   // leaves in tree order
    std::vector<ClusterNode> clusters;        // every node of the cluster tree (0 = root)
    std::vector<FarBlock> near_blocks;        // dense leaf blocks
    std::vector<FarBlock> far_blocks;         // admissible blocks
};

int plan_build(const double* xyz, int64_t n, int leaf, double eta, int adm, Plan& out, std::string& err);

// Leaf chunks of rows [row0, row0 + m); per_row = elements stored per padded
// row (G*r for far U, G*n for dense blocks).  Returns the total element count.
inline int64_t block_chunks(const Plan& P, int row0, int m, int64_t per_row, std::vector<Chunk>& out)
{
    const int nl = (int)P.leaf_start.size();
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (P.leaf_start[mid] <= row0) lo = mid; else hi = mid - 1;
    }
    int64_t off = 0;
    for (int l = lo; l < nl && P.leaf_start[l] < row0 + m; ++l) {
        Chunk c;
        c.leaf = l;
        c.rbeg = P.leaf_start[l] - row0;
        c.m = P.leaf_size[l];
        c.m8 = round8(c.m);
        c.off = off;
        off += per_row * c.m8;
        out.push_back(c);
    }
    return off;
}

// Device buffer that grows in place: a reserved virtual address range whose
// physical memory is mapped chunk by chunk as it grows, so that data already
// written never moves (rt_vmm.cu).
struct GrowBuf {
    unsigned long long base = 0;   // device address of byte 0
    size_t reserved = 0, mapped = 0, gran = 0;
    int device = 0;
    std::vector<unsigned long long> handles;   // physical allocations, in address order
    std::vector<size_t> sizes;
};
int growbuf_reserve(GrowBuf& b, size_t bytes, int device, std::string& err);
int growbuf_grow(GrowBuf& b, size_t bytes, std::string& err);   // mapped >= bytes afterwards
void growbuf_release(GrowBuf& b);   // no work may still use the buffer

// Operator (one instance).
struct Operator {
    int device = 0;
    int mode = RT_MODE_HMATRIX, prec = RT_PREC_F32, far_prec = RT_PREC_F32;
    int N = 0, F = 0, G = 0, T = 0;
    int grey = 0;
    double aca_eps = 1e-4, eta = 2.0;
    int adm = RT_ADM_GAP;
    int leaf = 64, ngauss = 16, rank_max = 512;
    int64_t wave_bytes = (int64_t)8 << 30;   // ACA scratch bound per wave
    KernelParams kp{};
    // frequencies (host copies) and the group of each frequency
    std::vector<double> nu, w, c, albedo, Q;
    double q0 = 0.0;            // the problem's emitter coefficient Q0 (Q[f] = q0 B_nu(T_emit))
    std::vector<int> fgroup;
    std::vector<double> gc;     // group scales
    std::vector<double> fscale; // per channel c_f / c_{g(f)} (1 unless channels are binned)
    int binned = 0;             // some fscale != 1
    double* d_fscale = nullptr; // device copy [F] when binned
    int* d_gmap = nullptr;      // [G][F]: row g has every entry g (rt_apply_group)
    Plan plan;
    // device geometry
    float4* d_xyz32 = nullptr;
    double* d_xyz64 = nullptr;
    int4* d_tet = nullptr;
    float4* d_tgeo32 = nullptr;
    dbl4* d_tgeo64 = nullptr;
    float* d_tvol32 = nullptr;
    double* d_tvol64 = nullptr;
    int* d_vt_ptr = nullptr;
    int* d_vt_idx = nullptr;
    int* d_perm = nullptr;      // tree -> original
    int* d_iperm = nullptr;     // original -> tree
    // emitter
    int n_emit = 0;
    int4* d_emit = nullptr;     // tree-order vertex ids of each triangle (w unused)
    double* d_emit_lim = nullptr; // per vertex: sum of (angle / 8 pi) over emitter triangles at the vertex
    // source (tree order), vector element type = vec64 ? double : float
    int vec64 = 0;
    void* d_SE = nullptr;       // [F][N]
    // dense mode
    void* d_dense = nullptr;    // [G][N][N] row-major (double or float)
    // H-matrix mode
    int n_near = 0, n_far = 0, n_fallback = 0;
    std::vector<int> rank;      // per far block (final; -1 = stored dense)
    std::vector<FarBlock> far_blocks, dense_blocks;   // final split
    float* d_near = nullptr;    // dense blocks' A^T
    std::vector<int64_t> dense_off;
    std::vector<int> dense_chunk_ptr, far_chunk_ptr;   // CSR over the chunk arrays
    std::vector<Chunk> dense_chunks, far_chunks;
    void* d_far = nullptr;      // far U/V (float, bf16 or f16)
    void* d_far_lo = nullptr;   // refinement: 16-bit remainders (value - high part) of a BF16/FP16
                                // far field, same layout as d_far
    int refine = 0;
    int use_lo = 0;             // apply with high + low parts (set by the solver)
    std::vector<int64_t> far_v_off, far_u_off;
    GrowBuf far_buf, far_lo_buf;   // backing of d_far / d_far_lo when ACA ran in several waves
    // matvec work lists (device)
    void* d_p1_items = nullptr; int n_p1 = 0;
    void* d_p1_rows = nullptr;
    std::vector<char> h_p1_rows;   // host copy of the (length-sorted) phase-1 row list
    void* d_p2_leaf = nullptr;  int n_p2 = 0;
    void* d_p2_segs = nullptr;  int n_p2_segs = 0;
    float* d_w = nullptr;       int64_t w_len = 0;   // phase-1 scratch [sum r][F]
    // streamed form of the two phases (bulk copies into a shared-memory ring):
    // stage records of phase 1 and phase 2, the first record of every leaf,
    // the (leaf, frequency) items in launch order, and the number of phase-1
    // items (a prefix of d_p1_items) whose rows are too long for one stage
    int hs_enabled = 0;
    void* d_hs1 = nullptr;      int n_hs1 = 0;
    void* d_hs2 = nullptr;      int n_hs2 = 0;
    int* d_hs2_leaf0 = nullptr;
    void* d_hs2_items = nullptr; int n_hs2_items = 0;
    int n_p1_long = 0;
    int* apply_err = nullptr;   // set by a bounded wait of an apply kernel that gave up
    float* d_xt = nullptr;      // permuted input scratch [F][N]
    float* d_yt = nullptr;      // permuted output scratch [F][N]
    // solver scratch
    void* d_J = nullptr; void* d_S = nullptr; void* d_Y = nullptr;
    double* d_T = nullptr;
    double* d_part = nullptr; int n_part = 0;
    double* d_res = nullptr;
    double* h_res = nullptr;    // pinned
    cudaStream_t cap_stream = nullptr;   // library-owned stream used for graph capture
    // frequency tables on device
    double* d_fq = nullptr;     // [F][4]: nu, w*c*(1-a), a, group
    int* d_fq_group = nullptr;  // [F] group of each frequency
    // row evaluation over column clusters: sub-clusters of at most kSubCols
    // columns, each with the list of tetrahedra touching its vertices (CSR)
    std::vector<int> sub_of_cluster_ptr, sub_of_cluster;   // per cluster: its sub-clusters
    std::vector<int> sub_start, sub_size, sub_tet_ptr;     // per sub-cluster
    int* d_sub_tets = nullptr;
    std::vector<int> h_vt_ptr, h_vt_idx;                   // host copy of the vertex -> tetrahedra CSR
    // tensor-core multi-right-hand-side apply (one operator group, F % 16 == 0)
    int tc_enabled = 0;
    int tc_off = 0;     // tensor cores disabled by the caller
    void *tc_tiles = nullptr, *tc_rows = nullptr, *tc_leaves = nullptr, *tc_segs = nullptr;
    int tc_ntiles = 0, tc_nleaves = 0;
    int64_t tc_wlen = 0;
    void* tc_w = nullptr;       // W high parts [tc_wlen], then low parts [tc_wlen]
    int tc_xal = 0;             // X columns of every cluster 16-byte aligned: X split once per apply
    void* tc_xsplit = nullptr;  // X high / low parts (BF16; then FP16 for an FP16 far field)
    int* tc_err = nullptr;
    unsigned long long* d_work = nullptr;   // assembly work counters (KernelParams::work)
    // streamed tcgen05 apply (rt_tc2.cu; F = 64): swizzled operator images,
    // phase-1 tiles, phase-2 leaves with their stages and copy pieces
    int tc2 = 0;
    void *t2_tiles = nullptr, *t2_leaves = nullptr, *t2_steps = nullptr, *t2_pieces = nullptr;
    int t2_ntiles = 0, t2_nleaves = 0;
    void *t2_vhi = nullptr, *t2_vlo = nullptr, *t2_uhi = nullptr, *t2_ulo = nullptr;
    void *t2_nhi = nullptr, *t2_nlo = nullptr, *t2_whi = nullptr, *t2_wlo = nullptr;
    void *t2_xs = nullptr, *t2_zero = nullptr;
    int64_t t2_xrows = 0, t2_wrows = 0;
    float* t2_scale = nullptr;   // [s, 1/s, max|X| bits, -]
    int64_t t2_stats[4] = {0, 0, 0, 0};   // stages, pieces, U image rows, near image rows
    // stats
    rt_info info{};
    std::vector<void*> allocations;
    // stream that orders the operator's allocations and host uploads (the
    // build stream; the solve stream while a solve allocates its vectors)
    cudaStream_t stream = nullptr;
};

// ---- kernels / drivers implemented in the .cu files -----------------------
int assemble_setup_constants(Operator& op, std::string& err);
void gauss_legendre_nodes(int n, std::vector<double>& t, std::vector<double>& w);
int assemble_dense(Operator& op, cudaStream_t s, std::string& err);
int assemble_source(Operator& op, cudaStream_t s, std::string& err);
int assemble_hmatrix(Operator& op, cudaStream_t s, std::string& err);
int prepare_row_eval(Operator& op, std::string& err);
int eval_entries(Operator& op, int group, int64_t count, const int32_t* rows, const int32_t* cols, double* out,
                 cudaStream_t s, std::string& err);
int hmatvec_prepare(Operator& op, std::string& err);
// X, Y in tree order, [F][N], element type float (H-matrix / dense F32) or double (dense F64)
int apply_tree(Operator& op, const void* X, void* Y, cudaStream_t s, std::string& err);
int permute_vectors(Operator& op, const void* in, void* out, int to_tree, int is64, int rows, cudaStream_t s,
                    const double* scale = nullptr);
int scale_rows(Operator& op, void* Y, cudaStream_t s);   // Y_f *= fscale[f] (binned channels)
int apply_group(Operator& op, int group, const void* X, int64_t ldx, int nrhs, void* Y, int64_t ldy, cudaStream_t s,
                std::string& err);
// rt_apply with its scratch in a file-scope device array (no allocation)
int apply_noalloc(Operator& op, const void* X, void* Y, cudaStream_t s, std::string& err);
size_t apply_noalloc_limit();
int tc_prepare(Operator& op, std::string& err);
int eval_sin2pi(const float* x, float* lib, float* ref, int64_t n, cudaStream_t s, std::string& err);
// rows [row0, row0 + nrows) (tree order) of the surface-to-volume matrix, [G][nrows][L] at out (gstride per group)
int srcop_eval_rows(Operator& op, const int* col_of, int L, int row0, int nrows, float* out, int64_t gstride,
                    cudaStream_t s, std::string& err);
int tc_apply(Operator& op, const float* X, float* Y, cudaStream_t s, std::string& err);
int tc2_prepare(Operator& op, std::string& err);
int tc2_apply(Operator& op, const float* X, float* Y, cudaStream_t s, std::string& err);
// the tcgen05 path serves this apply (the streamed one also serves refinement sweeps)
inline bool tc_serves(const Operator& op) { return op.tc_enabled && (!op.use_lo || op.tc2); }
int tc_check_error(Operator& op, cudaStream_t s, std::string& err);
// RT_ETIMEOUT if a bounded wait of an apply kernel (tensor-core or streamed) gave up
int apply_check_error(Operator& op, cudaStream_t s, std::string& err);
int solve_fixed_point(Operator& op, const rt_solve_opts& o, void* J, double* T, rt_solve_stats& st,
                      cudaStream_t s, std::string& err);

// error helpers
#define RT_CUDA_TRY(expr)                                                            \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            err = std::string(#expr) + ": " + cudaGetErrorString(e_);               \
            return RT_ECUDA;                                                         \
        }                                                                            \
    } while (0)

template <class T>
int dev_alloc(Operator& op, T** p, size_t count, std::string& err)
{
    *p = nullptr;
    if (count == 0) count = 1;
    // stream-ordered: no device-wide synchronisation, so builds on other
    // streams keep running
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), op.stream);
    if (e != cudaSuccess) {
        err = std::string("cudaMallocAsync(") + std::to_string(count * sizeof(T)) + " bytes): " + cudaGetErrorString(e);
        *p = nullptr;
        return RT_ENOMEM;
    }
    op.allocations.push_back((void*)*p);
    op.info.device_bytes += (int64_t)(count * sizeof(T));
    return RT_OK;
}

// host -> device copy ordered on the operator's stream (the source is staged
// before the call returns, so it may be a temporary)
template <class T>
int upload_async(Operator& op, T* dst, const T* src, size_t count, std::string& err)
{
    if (count == 0) return RT_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, op.stream);
    if (e != cudaSuccess) {
        err = std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e);
        return RT_ECUDA;
    }
    return RT_OK;
}

// free every device allocation of the operator, ordered on stream s
void operator_release(Operator& op, cudaStream_t s);
// checks and the build behind rt_build_operator (pre: a plan computed for the
// same mesh and hparams, moved into the operator; may be null)
int validate_problem(const rt_problem* P, const rt_hparams* H, std::string& err);
int build_operator(Operator& op, const rt_problem* P, const rt_hparams* H, cudaStream_t s, std::string& err,
                   Plan* pre);
void set_last_error(const std::string& msg);

}  // namespace rt

// the opaque handle of the C ABI
struct rt_operator {
    rt::Operator op;
};
