/*
 * rt.h -- C ABI of the GB300 (sm_103a) integral-form radiative-transfer
 * library: assembly of the compressed operator Gbar (dense near-field blocks
 * plus rank-r U V^T far-field blocks from partially pivoted ACA), its
 * application to the multi-frequency iterate, and the monotone fixed point.
 *
 * Method: Pironneau & Tournier, "Reflective Conditions for Radiative
 * Transfer in Integral Form with H-Matrices" (arXiv 2306.05789).
 *   - kernel and reflected-path terms: Corollary and Example of Section 1.2
 *   - P1 FEM matrix G_kappa^{ij} and source Sbar^E_i: Section 2
 *   - H-matrix compression, admissibility max(R1,R2) < eta |x1-x2|, ACA with a
 *     relative Frobenius tolerance: Section 2.1
 *   - fixed-point algorithm, eq. (algo): Section 1.3; grey variant eq. (grey): Section 3
 *
 * Conventions for every entry point
 *   - Return value: RT_OK (0) or a negative RT_E* code.  Nothing throws or
 *     aborts across the ABI; rt_last_error() returns a thread-local message
 *     describing the last failure on the calling thread.
 *   - Host inputs (meshes, coefficient arrays) are owned by the caller and
 *     copied during the call; they may be freed on return.
 *   - Device pointers (X, Y, J, T, out) are owned by the caller, must hold the
 *     stated number of elements, and are used in stream order on `stream`
 *     (a cudaStream_t passed as void*, NULL = legacy default stream).
 *   - Vectors over vertices and frequencies are laid out [F][N] (frequency
 *     major, vertex index contiguous) in the caller's vertex order.
 *   - The operator is owned by the library, resident on the device that was
 *     current at build time, and released by rt_free().
 *   - Results are deterministic for a given operator (no floating-point
 *     atomics in the apply or solve paths).
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RT_OK 0
#define RT_EINVAL (-1)   /* invalid argument or malformed input */
#define RT_ENOMEM (-2)   /* device or host allocation failed */
#define RT_ECUDA (-3)    /* a CUDA call failed */
#define RT_ENOCONV (-4)  /* fixed point did not reach tol within max_iter */
#define RT_ETIMEOUT (-5) /* a bounded device-side wait gave up */
#define RT_EAGAIN (-6)   /* rt_poll: the request has not finished yet */

/* kappa(x) descriptors (kappa_nu = c_nu * kappa(x)) */
#define RT_KAPPA_CONST 0   /* kappa = k0 */
#define RT_KAPPA_SINPROD 1 /* kappa = k0 + amp sin(2 pi x) sin(2 pi y) sin(2 pi z) */
#define RT_KAPPA_GRID 2    /* cellwise-constant grid, see rt_kappa */
#define RT_MAX_GRID_DIM 512
#define RT_MAX_OBSTACLES 4

/* operator storage modes and precisions */
#define RT_MODE_DENSE 0   /* every entry of G stored (FP64 or FP32) */
#define RT_MODE_HMATRIX 1 /* H-matrix: dense leaves + ACA far blocks */
#define RT_PREC_F64 0
#define RT_PREC_F32 1
#define RT_PREC_BF16 2
#define RT_PREC_F16 3

/* evaluation of the n-point Gauss sum along a segment (n >= 16) for the
 * sin-product kappa: RT_LINE_CLOSED uses the exact trigonometric identity
 * (product-to-sum; the Gauss sum of a sinusoid is its midpoint value times
 * sum_g w_g cos(beta (u_g - 1/2)) = sinc(beta/2) within the Gauss truncation
 * error, below 2e-14 for segments with |dx|+|dy|+|dz| <= 3); RT_LINE_NODES
 * sums the kappa samples node by node.  Both compute the same sum. */
#define RT_LINE_CLOSED 0
#define RT_LINE_NODES 1

/* admissibility readings of max(R1,R2) < eta |x1 - x2| (Section 2.1) */
#define RT_ADM_GAP 0    /* |x1 - x2| = distance between the clusters' bounding spheres (|c1-c2| - R1 - R2) */
#define RT_ADM_CENTER 1 /* |x1 - x2| = distance between the cluster centroids (literal) */

/* Tetrahedral P1 mesh of the domain (Section 2).  xyz: [n_vert][3] doubles;
 * tet: [n_tet][4] vertex ids (0-based). */
typedef struct {
    int64_t n_vert;
    const double* xyz;
    int64_t n_tet;
    const int32_t* tet;
} rt_mesh;

/* Absorption kappa(x) (kappa_nu = c_nu kappa(x), Section 1.1).  RT_KAPPA_GRID:
 * dims[0] x dims[1] x dims[2] equal cells of the box bbox = (x0, y0, z0, x1,
 * y1, z1); cell (i, j, k) holds grid[i + dims[0] (j + dims[1] k)] >= 0 (host
 * array, copied during the build); a point outside the box takes the value of
 * the nearest cell.  The optical depth int_[a,b] kappa of a grid is computed
 * exactly (the segment cut at the grid planes, each piece times its cell's
 * value); the analytic kinds use the Gauss-Legendre rule of rt_hparams. */
typedef struct {
    int kind;  /* RT_KAPPA_* */
    double k0; /* constant part */
    double amp;
    const float* grid;  /* RT_KAPPA_GRID only, else NULL */
    int dims[3];        /* cells per axis, 1 .. RT_MAX_GRID_DIM */
    double bbox[6];
} rt_kappa;

/* Opaque axis-aligned box [lo, hi] inside the convex hull of a non-convex
 * domain (Remark 1 after Lemma 1: kappa = +infinity in the hull outside the
 * domain).  A path whose open segment overlaps the open box on a parameter
 * interval longer than 1e-6 of the segment has infinite optical depth and
 * contributes nothing.  No tetrahedron may lie inside a box (RT_EINVAL). */
typedef struct {
    double lo[3];
    double hi[3];
} rt_box;

/* Planar reflective wall (Section 2, planar reflective boundaries): a point
 * p of the plane, the OUTWARD normal n (any length, normalised by the
 * library), reflection coefficient R0 in [0, 1].  The plane's intersection
 * with the (convex) domain is taken as the reflecting face.  Up to
 * RT_MAX_WALLS walls per problem, each adding one reflected term (its mirror
 * image of x, weight R0; Hypothesis 1 with one reflection per wall). */
#define RT_MAX_WALLS 3
typedef struct {
    double p[3];
    double n[3];
    double R0;
} rt_wall;

/* Frequency grid: F channels with quadrature weight w, absorption scale c
 * (kappa_nu = c * kappa(x)) and albedo a.  Operators are built per group of
 * channels (Remark of Section 2.1: one matrix pair per value of kappa_nu, and
 * fewer than ten values usually represent kappa_nu piecewise constantly;
 * Section 4, Test 2: 583 frequencies, 8 values of kappa_nu in the
 * exponentials).
 *   - group == NULL and rt_hparams.kappa_bins == 0: channels with equal c share
 *     one group (exact, no approximation).
 *   - group == NULL and kappa_bins = K > 0: the channels are binned by c into K
 *     equal-width intervals of [min c, max c] (empty intervals dropped).
 *   - group != NULL: group[f] in [0, G) is the caller's group of channel f;
 *     every index in [0, G) must be used.
 * A group's scale c_g is the midpoint (min c + max c) / 2 of its channels'
 * scales.  The optical depths in the exponentials use c_g; the kappa_nu(y)
 * factor in front keeps the channel's own c, so channel f applies
 * (c_f / c_g) G_g (G_g built with c_g in both places; the factor is 1
 * without binning).  The temperature balance uses every channel's own c. */
typedef struct {
    int F;
    const double* nu;
    const double* w;
    const double* c;
    const double* albedo;
    const int32_t* group;   /* [F] or NULL */
} rt_freqs;

/* One problem instance.  Emitting boundary: n_emit triangles (vertex ids of
 * the mesh, right-hand normal = outward normal) radiating
 * Q_nu = Q0 [omega.n]_- B_nu(T_emit) (Example of Section 1), grey:
 * Q0 sigma T_emit^4.  grey != 0 selects the grey formulation (eq. (grey),
 * Section 3; F must be 1).
 * Walls: n_walls in [0, RT_MAX_WALLS] planes in walls[].  corner != 0 adds,
 * for every pair of perpendicular walls (|n_a . n_b| <= 1e-12 |n_a| |n_b|)
 * with R0_a, R0_b > 0, the path that reflects on both (source point the
 * double image of x, weight R0_a R0_b): the second-order term of Section 2's
 * series of images, which Hypothesis 1 leaves out (corner = 0 is the paper's
 * model). */
typedef struct {
    rt_mesh mesh;
    rt_kappa kappa;
    int n_walls;           /* 0 .. RT_MAX_WALLS */
    const rt_wall* walls;  /* [n_walls] or NULL when n_walls == 0 */
    int64_t n_emit;
    const int32_t* emit_tri;
    double Q0;
    double T_emit;
    int grey;
    rt_freqs freqs;
    int corner;            /* 0 or 1, see above */
    int n_obstacles;       /* 0 .. RT_MAX_OBSTACLES opaque boxes */
    const rt_box* obstacles;
} rt_problem;

/* Assembly parameters (Section 2 and 2.1). */
typedef struct {
    int mode;        /* RT_MODE_DENSE or RT_MODE_HMATRIX */
    int prec;        /* dense: RT_PREC_F64 or RT_PREC_F32; H-matrix: RT_PREC_F32 (near field, vectors) */
    int far_prec;    /* H-matrix far-field U/V storage: RT_PREC_F32, RT_PREC_BF16 or RT_PREC_F16 */
    double aca_eps;  /* ACA relative Frobenius tolerance (e.g. 1e-4) */
    int leaf;        /* cluster-tree leaf size (e.g. 64) */
    double eta;      /* admissibility max(R1,R2) < eta |c1 - c2| (e.g. 2) */
    int gauss_pts;   /* Gauss-Legendre points per line integral (1..32, e.g. 16) */
    int rank_max;    /* ACA rank limit before a block is stored dense (0 = 512) */
    int adm;         /* RT_ADM_GAP (default) or RT_ADM_CENTER */
    int line_eval;   /* RT_LINE_CLOSED (default) or RT_LINE_NODES (FP32 paths) */
    int refine;      /* with a BF16/FP16 far field: also store each value's 16-bit remainder
                        (value - high part, same layout) for refinement sweeps, so that the
                        far field takes 4 bytes per entry in all, like FP32 storage */
    int tensor_cores; /* 0: use the tcgen05 apply when eligible (one operator group, F a multiple
                         of 16 up to 256, BF16/FP16 far field, leaves <= 128); 1: CUDA cores only */
    int64_t wave_bytes; /* ACA runs over consecutive waves of admissible blocks whose FP32 term
                           scratch (estimated at 24 terms per block) stays below this many bytes;
                           each wave is packed and its scratch freed before the next (0 = 8 GiB) */
    int kappa_bins;  /* 0: one operator group per distinct c; K > 0: bin the channels by c into at
                        most K groups (see rt_freqs); ignored when the problem gives a group map */
} rt_hparams;

typedef struct rt_operator rt_operator;

/* Operator statistics (filled by rt_operator_info). */
typedef struct {
    int64_t N, F, G;             /* vertices, frequencies, operator groups */
    int mode, prec, far_prec;
    int64_t n_leaves, n_near, n_far, n_dense_fallback;
    int64_t stored_entries;      /* per group: sum m*n (dense) + sum r*(m+n) (far) */
    double compression;          /* 1 - stored_entries / N^2 (per group) */
    int64_t rank_min, rank_max, rank_sum;
    int64_t aca_steps;           /* ACA sweeps until every block finished */
    int64_t entries_evaluated;   /* kernel entries evaluated during assembly (all groups count once) */
    int64_t apply_bytes;         /* algorithmic bytes moved by one rt_apply (all groups): stored operator
                                    entries x element size (once per frequency, or once in all for the
                                    tcgen05 apply) + X read + Y written */
    int64_t apply_flops;
    int64_t device_bytes;        /* device memory held by the operator */
    double ms_tree, ms_near, ms_aca, ms_pack, ms_source; /* assembly phase times */
    int64_t peak_bytes;          /* largest device footprint during assembly (operator + ACA scratch) */
    int64_t aca_waves;           /* waves of admissible blocks the ACA ran in */
    int64_t apply_tensor_cores;  /* 1 if rt_apply runs on the tcgen05 multi-right-hand-side path */
    int64_t assembly_terms;      /* H-matrix assembly: kernel terms evaluated (one direct or one reflected
                                    value of the kernel at a point pair, all groups at once) */
    int64_t assembly_depths;     /* H-matrix assembly: optical depths evaluated (one per direct term,
                                    two per reflected term) */
} rt_info;

/* Fixed-point options (Section 1.3).  The iteration starts from T = T0 at
 * every vertex and J = 0 (or J = J_dev on entry if use_J0 != 0). */
typedef struct {
    double tol;      /* stop when ||J^{k+1}-J^k||_2 / ||J^{k+1}||_2 <= tol */
    int max_iter;
    int check_every; /* iterations between host convergence checks (>= 1) */
    double T0;
    int use_J0;
    int use_graph;   /* capture check_every iterations in a CUDA graph */
    double refine_tol; /* operator built with refine: iterate on the 16-bit high parts of the far
                          field until the residual is <= refine_tol, then on high + low parts down
                          to tol (0: high + low parts from the start) */
} rt_solve_opts;

typedef struct {
    int iters;
    int converged;
    double residual;
    double ms_total;
} rt_solve_stats;

/* Build the operator for one problem (Section 2, 2.1).  Host inputs are
 * copied; assembly runs on `stream`; returns when the operator is complete.
 * Errors: RT_EINVAL for malformed meshes/parameters, RT_ENOMEM, RT_ECUDA. */
int rt_build_operator(const rt_problem* prob, const rt_hparams* hp, void* stream, rt_operator** out);

/* Statistics of a built operator. */
int rt_operator_info(const rt_operator* op, rt_info* info);

/* Y = Gbar X per frequency, Y_nu = G_{g(nu)} X_nu: the matrix-vector product
 * that is the whole per-iteration cost of the fixed point (abstract; the
 * discrete operator J_i = Sbar^E_i + sum_j G^{ij} S_j of Section 2, applied in
 * its compressed form of Section 2.1: dense near blocks plus U V^T far blocks).
 * X and Y are device arrays [F][N] in the caller's vertex order; element type
 * double for a dense FP64 operator, float otherwise.  X and Y must not
 * overlap.  Asynchronous on `stream`: it returns once the kernels are queued.
 * The H-matrix kernels' device-side waits are bounded (about 2 s); a wait
 * that gives up leaves Y unspecified and sets a flag that the operator's next
 * rt_solve_fixed_point returns as RT_ETIMEOUT.  Errors: RT_EINVAL (null
 * operator or vectors), RT_ECUDA (a launch failed). */
int rt_apply(rt_operator* op, const void* X, void* Y, void* stream);

/* Y_j = G_group X_j for nrhs vectors of one operator group (Section 2.1:
 * one matrix per value of kappa_nu), without the per-channel factor
 * c_f / c_g of a binned grid.  X_j = X + j * ldx and Y_j = Y + j * ldy
 * (j < nrhs, ldx, ldy >= N) are device vectors of N elements in the caller's
 * vertex order, element type as in rt_apply; X and Y must not overlap.  The
 * right-hand sides run in chunks of F (the operator's channel count) through
 * rt_apply's kernels and scratch, so calls on one operator must be ordered.
 * Asynchronous on `stream`.  RT_EINVAL for a group outside [0, G), nrhs < 0,
 * ld < N or null vectors; RT_ECUDA if a launch fails. */
int rt_apply_group(rt_operator* op, int group, const void* X, int64_t ldx, int nrhs, void* Y, int64_t ldy,
                   void* stream);

/* Y = Gbar X with the same kernels and arithmetic as rt_apply (its tcgen05
 * pair where rt_apply takes it, its CUDA-core phases otherwise), for callers
 * that cannot allocate device memory while they run: for example an
 * application whose device memory is entirely handed out by its own pool
 * allocator, or a host loop with a fixed time budget that cannot afford the
 * synchronisation a cudaMalloc or cudaFree may imply.
 * (The paper has no counterpart: this is a deployment convenience.)
 * The scratch rt_apply keeps in the operator -- X and Y in the internal vertex
 * order and, on CUDA cores, one FP32 value per (far-block rank term,
 * frequency) -- is taken from a static 8 MiB device array instead
 * (2 * 4 F N bytes, plus 4 F sum(rank) bytes on CUDA cores, each rounded up to
 * 256, must fit; larger operators get RT_EINVAL).  The tcgen05 path's other
 * buffers belong to the operator and were allocated when it was built.
 * The array exists once per GPU that loads the library and stays allocated
 * until the process exits.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it.  All calls share the
 * array: calls whose work overlaps on the GPU (different streams or threads
 * without ordering) race on it.  Nothing needs clearing between calls (each
 * region is overwritten before it is read).  The current device must be the
 * operator's device.  Dense operators need no scratch and are applied
 * directly.  Allocates nothing: no cudaMalloc, cudaFree or allocating library
 * call. */
int rt_apply_noalloc(rt_operator* op, const void* X, void* Y, void* stream);

/* Sbar^E_nu (Proposition 2 / Example of Section 1.2, discretised as in
 * Section 2) into out [F][N] (vector element type as in rt_apply). */
int rt_source(rt_operator* op, void* out, void* stream);

/* Evaluate `count` individual entries G_g^{ij} with the library's entry
 * evaluator (same arithmetic as assembly): rows/cols are device int32 arrays
 * of vertex ids (caller order), out is a device double array [count]. */
int rt_eval_entries(rt_operator* op, int group, int64_t count, const int32_t* rows, const int32_t* cols,
                    double* out, void* stream);

/* ---- the surface-to-volume matrix (Section 2, last paragraph; Section 2.1) --
 * Sbar^E_{i,l} is the emitter source of Section 2 with the emitter coefficient
 * Q0(y) replaced by the P1 hat function of emitter-surface vertex l (the
 * distinct vertices of the problem's emitter triangles, in ascending vertex
 * id).  For per-vertex coefficients Q0_l, Q0(y) = sum_l Q0_l w_l(y) and
 * Sbar^E_{nu,i} = sum_l Sbar^E_{i,l} Q0_l, times the intensity B_nu(T_emit)
 * (grey: sigma T_emit^4); with every Q0_l equal to the problem's Q0 this is
 * rt_source.  One N x L matrix per kappa group (the optical depths use the
 * group's scale), compressed like Gbar: a rectangular block tree of the
 * operator's volume clusters against clusters of the emitter vertices, the
 * operator's admissibility rule, partially pivoted ACA with the operator's
 * tolerance on admissible blocks (a block that would need more than 32 terms
 * stays dense), dense blocks elsewhere.  Every entry is evaluated once on the
 * device during the build (FP32, the quadrature and limit rules of the
 * source).  Needs an H-matrix operator with at most 16 groups and leaves of at
 * most 64 rows. */
typedef struct rt_source_op rt_source_op;

typedef struct {
    int64_t N, L, G;             /* rows, emitter vertices, kappa groups */
    int64_t n_blocks, n_far, n_dense; /* blocks; far (block, group) pieces; dense blocks */
    int64_t rank_sum, rank_max;
    int64_t stored_entries;      /* all groups: sum r (m + n) + sum m n */
    double compression;          /* 1 - stored_entries / (N L G) */
    int64_t apply_bytes;         /* algorithmic bytes of one rt_apply_source */
    int64_t device_bytes;
    double ms_eval, ms_aca;      /* entry evaluation and compression times */
} rt_source_info;

/* Build the surface-to-volume operator of a built operator `op` (which must
 * outlive it) on `stream`.  RT_EINVAL: dense operator, no emitter, more than
 * 16 groups, leaves over 64 rows or G x L over the row buffer (200 KB of
 * FP32); RT_ENOMEM; RT_ECUDA. */
int rt_build_source_operator(rt_operator* op, void* stream, rt_source_op** out);

/* Sizes and statistics; vertices (may be NULL): [L] vertex ids of the columns. */
int rt_source_operator_info(const rt_source_op* s, rt_source_info* info, int32_t* vertices);

/* out [F][N] (device floats, caller vertex order) = B_nu(T_emit) sum_l
 * Sbar^E_{g(nu)}[i, l] Q0[l] for device coefficients Q0 [L] in the column
 * order of rt_source_operator_info.  Asynchronous on `stream`; calls on one
 * operator must be ordered (they share its scratch).  RT_EINVAL for null
 * arguments, RT_ECUDA if a launch fails. */
int rt_apply_source(rt_source_op* s, const float* Q0, float* out, void* stream);

/* Release the surface-to-volume operator (synchronises the device). */
void rt_source_free(rt_source_op* s);

/* Diagnostic (no paper counterpart): the library's FP32 sin(2 pi x), used by
 * the sin-product kappa on the FP32 paths, for n device values x: lib_out[i]
 * receives it and ref_out[i] CUDA's sinpif(2 x[i]) for comparison.  All three
 * are caller-owned device float arrays of n elements.  Asynchronous on
 * `stream`.  RT_EINVAL for n < 0 or null arrays, RT_ECUDA if the launch
 * fails. */
int rt_eval_sin2pi(const float* x, float* lib_out, float* ref_out, int64_t n, void* stream);

/* Fixed point of Section 1.3 (eq. (algo)) on the device: S = a J + (1-a)
 * B_nu(T), J <- Sbar^E + Gbar S, T <- Planck balance per vertex (FP64
 * Newton, or (J/sigma)^(1/4) for grey).  J_dev [F][N] (vector element type),
 * T_dev [N] doubles; both receive the final iterate.  Returns RT_ENOCONV
 * (with J, T and stats filled) if tol is not reached within max_iter, and
 * RT_ETIMEOUT if a bounded device-side wait of an apply (this solve's or an
 * earlier rt_apply's) gave up. */
int rt_solve_fixed_point(rt_operator* op, const rt_solve_opts* opts, void* J_dev, double* T_dev,
                         rt_solve_stats* stats, void* stream);

/* Release the operator and its device memory. */
void rt_free(rt_operator* op);

/* ---- batches of independent instances ------------------------------------
 * A batch holds one operator per problem (same hparams, H-matrix mode with
 * an FP32 far field, at most 16 kappa groups per problem) and applies or
 * solves all of them together: one persistent launch applies every
 * operator, and the fixed point runs on concatenated vectors, each instance
 * stopping at its own first iteration with residual <= tol.  Vectors of a
 * batch are the instances' [F_b][N_b] vectors (caller vertex order)
 * concatenated in problem order; temperatures the [N_b] arrays likewise. */
typedef struct rt_batch rt_batch;

typedef struct {
    int64_t count;          /* instances */
    int64_t total_vec;      /* sum F_b N_b */
    int64_t total_vert;     /* sum N_b */
    int p1_target_bytes;    /* operator bytes per phase-1 work item (chosen by the autotuner) */
    int ctas_per_sm;        /* persistent grid size per SM (chosen by the autotuner) */
    int n_works;            /* work items of one apply */
    int64_t apply_bytes;    /* algorithmic bytes of one apply of every operator */
    double tune_ms, build_ms;
} rt_batch_info_t;

/* Build the operators of `count` problems with `threads` host threads (each
 * on its own stream; 0 = 8), then, if tune != 0, time candidate work-item
 * sizes and persistent grid sizes on the batch and keep the fastest. */
int rt_build_batch(const rt_problem* probs, int64_t count, const rt_hparams* hp, int threads, int tune, void* stream,
                   rt_batch** out);

/* Sizes and tuner choices; vec_off / vert_off (may be NULL) receive count+1
 * offsets of each instance's vectors and temperatures. */
int rt_batch_info(const rt_batch* b, rt_batch_info_t* info, int64_t* vec_off, int64_t* vert_off);

/* Y = Gbar X for every instance, X and Y device arrays [total_vec]. */
int rt_batch_apply(rt_batch* b, const float* X, float* Y, void* stream);

/* Fixed point of every instance from T = T0, J = 0 (use_J0 and refine_tol are
 * ignored): J_dev [total_vec], T_dev [total_vert] (device), iters (host,
 * may be NULL) [count] = iterations each instance took.  RT_ENOCONV if some
 * instance did not reach tol; RT_ETIMEOUT if a bounded device wait gave up. */
int rt_solve_batch(rt_batch* b, const rt_solve_opts* opts, float* J_dev, double* T_dev, int32_t* iters,
                   rt_solve_stats* stats, void* stream);

/* Diagnostic (no paper counterpart): the clock budget, in SM clock cycles, of
 * the wait with which a phase-2 item of the batch apply waits for its
 * instance's phase-1 items (0 restores the default of about 1 s).  With
 * unreachable != 0 every such wait targets one more completed phase-1 item
 * than exist, so every wait runs out: the apply then finishes with Y
 * unspecified and rt_solve_batch returns RT_ETIMEOUT.  This drives the
 * timeout path without faulting or hanging the GPU.  RT_EINVAL for a null
 * batch or a negative budget. */
int rt_batch_set_wait(rt_batch* b, int64_t wait_cycles, int unreachable);

void rt_batch_free(rt_batch* b);

/* Thread-local text of the last batch error. */
const char* rt_batch_last_error(void);

/* Thread-local text of the last error on the calling thread ("" if none). */
const char* rt_last_error(void);

/* ---- host-only planning (no GPU needed) --------------------------------
 * Cluster tree by recursive bisection at the median along the longest box
 * axis down to `leaf` points, and the block tree with the admissibility rule
 * of Section 2.1, max(R_t, R_s) < eta d(t, s) with R = max distance from the
 * centroid and d = |c_t - c_s| - R_t - R_s (adm = RT_ADM_GAP) or
 * d = |c_t - c_s| (adm = RT_ADM_CENTER).  perm (may be NULL): [n] tree order -> vertex id.  blocks (may
 * be NULL): [cap][5] rows (row0, m, col0, n, kind: 0 dense leaf, 1
 * admissible) in tree order.  counts: [0] = leaves, [1] = dense blocks,
 * [2] = admissible blocks.
 * Point sets of at least 32768 points are planned on several host threads
 * (environment variable RT_PLAN_THREADS, default the hardware threads, at
 * most 16); the plan does not depend on the thread count, bit for bit.  The
 * operator builds and rt_submit plan the same way. */
int rt_plan(const double* xyz, int64_t n, int leaf, double eta, int adm, int32_t* perm, int32_t* blocks,
            int64_t cap, int64_t* counts);

/* ---- serving: continuous admission of independent solve requests --------
 * (The paper solves one problem at a time; this is the deployment form.)
 * A server owns `slots` worker threads, each with its own CUDA stream on the
 * device current at rt_server_create.  A submitted request (a problem as for
 * rt_build_operator) waits in a queue until a slot is free and its estimated
 * device footprint fits in what the budget has left; it is then assembled
 * (Section 2, 2.1) and iterated to the fixed point (Section 1.3) on that
 * slot's stream, so the work of several requests overlaps on the device.
 * Each request's operator and iterates stay on the device until its result
 * has been copied to host memory; then they are freed and the next request
 * is admitted.  Admission is first come, first served, except that a request
 * that fits may start ahead of one that does not, at most `max_bypass` times
 * per waiting request.  The estimate (cluster and block tree plus an assumed
 * far-block rank) is replaced by the operator's measured size once it is
 * built.  Results do not depend on what else is in flight. */
typedef struct rt_server rt_server;

typedef struct {
    int64_t hbm_budget;      /* bytes of device memory the admitted requests may hold (> 0) */
    int slots;               /* requests on the device at once (1..64) */
    int max_bypass;          /* times a waiting request may be overtaken (>= 0) */
    rt_hparams hp;           /* assembly parameters of every request (H-matrix mode) */
    rt_solve_opts opts;      /* fixed-point options of every request (T0, tol, ...) */
} rt_server_opts;

typedef struct {
    int status;              /* RT_OK or the request's error code */
    int iters, converged;
    double residual;
    int64_t N, F;
    int64_t est_bytes;       /* footprint estimate used for admission */
    int64_t peak_bytes;      /* measured peak during assembly (operator + ACA scratch) */
    int64_t resident_bytes;  /* operator + iterates while the fixed point ran */
    double t_submit, t_admit, t_built, t_done;   /* seconds since rt_server_create */
    double ms_build, ms_solve;
} rt_request_info;

typedef struct {
    int64_t submitted, finished, failed, queued, running;
    int64_t reserved_bytes;      /* budget held by admitted requests now */
    int64_t peak_reserved_bytes; /* largest value it reached */
    int64_t max_running;         /* most requests on the device at once */
} rt_server_info_t;

/* Start a server.  RT_EINVAL for bad options. */
int rt_server_create(const rt_server_opts* opts, rt_server** out);

/* Queue one request; its inputs are copied.  *id receives its handle.
 * RT_EINVAL for a malformed problem, RT_ENOMEM if its estimated footprint
 * alone exceeds the budget. */
int rt_submit(rt_server* s, const rt_problem* prob, int64_t* id);

/* Wait up to wait_ms milliseconds (< 0: no limit) for request `id`.  Returns
 * RT_EAGAIN if it is still queued or running (nothing is copied).  Otherwise
 * the request is retired: J_host [F][N] floats and T_host [N] doubles (each
 * may be NULL) receive the final iterate in the caller's vertex order, info
 * (may be NULL) its record, and the return value is the request's status.
 * RT_EINVAL for an unknown (or already retired) id. */
int rt_poll(rt_server* s, int64_t id, int wait_ms, float* J_host, double* T_host, rt_request_info* info);

/* Counters of the server. */
int rt_server_info(rt_server* s, rt_server_info_t* info);

/* Finish the requests on the device, drop the queued ones, free everything. */
void rt_server_free(rt_server* s);

#ifdef __cplusplus
}
#endif
#endif /* RT_H */
