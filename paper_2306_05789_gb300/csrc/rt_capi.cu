// rt_capi.cu -- the C ABI (include/rt.h): validation, host geometry
// preparation, operator lifetime and error reporting.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rt_internal.h"


namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}


double planck_host(double nu, double T)
{
    if (!(T > 0.0)) return 0.0;
    return nu * nu * nu / std::expm1(nu / T);
}

int validate(const rt_problem* P, const rt_hparams* H)
{
    if (!P || !H) return fail(RT_EINVAL, "null problem or hparams");
    const rt_mesh& M = P->mesh;
    if (M.n_vert <= 3 || !M.xyz) return fail(RT_EINVAL, "mesh: need at least 4 vertices and xyz");
    if (M.n_vert > (int64_t)1 << 28) return fail(RT_EINVAL, "mesh: too many vertices");
    if (M.n_tet <= 0 || !M.tet) return fail(RT_EINVAL, "mesh: no tetrahedra");
    if (M.n_tet > (int64_t)1 << 29) return fail(RT_EINVAL, "mesh: too many tetrahedra");
    for (int64_t k = 0; k < 4 * M.n_tet; ++k)
        if (M.tet[k] < 0 || M.tet[k] >= M.n_vert) return fail(RT_EINVAL, "mesh: tetrahedron vertex id out of range");
    for (int64_t k = 0; k < 3 * M.n_vert; ++k)
        if (!std::isfinite(M.xyz[k])) return fail(RT_EINVAL, "mesh: non-finite coordinate");
    if (P->n_emit < 0 || (P->n_emit > 0 && !P->emit_tri)) return fail(RT_EINVAL, "emitter triangles missing");
    for (int64_t k = 0; k < 3 * P->n_emit; ++k)
        if (P->emit_tri[k] < 0 || P->emit_tri[k] >= M.n_vert) return fail(RT_EINVAL, "emitter vertex id out of range");
    if (P->n_walls < 0 || P->n_walls > RT_MAX_WALLS) return fail(RT_EINVAL, "n_walls must lie in [0, RT_MAX_WALLS]");
    if (P->n_walls > 0 && !P->walls) return fail(RT_EINVAL, "walls pointer missing");
    for (int w = 0; w < P->n_walls; ++w) {
        const double* n = P->walls[w].n;
        const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0.0) || !std::isfinite(nn)) return fail(RT_EINVAL, "wall normal must be nonzero");
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(P->walls[w].p[d])) return fail(RT_EINVAL, "wall point must be finite");
        if (!(P->walls[w].R0 >= 0.0 && P->walls[w].R0 <= 1.0)) return fail(RT_EINVAL, "R0 must lie in [0, 1]");
    }
    if (P->corner != 0 && P->corner != 1) return fail(RT_EINVAL, "corner must be 0 or 1");
    const rt_kappa& K = P->kappa;
    if (K.kind != RT_KAPPA_CONST && K.kind != RT_KAPPA_SINPROD && K.kind != RT_KAPPA_GRID)
        return fail(RT_EINVAL, "kappa kind");
    if (K.kind == RT_KAPPA_GRID) {
        if (!K.grid) return fail(RT_EINVAL, "kappa grid values missing");
        int64_t cells = 1;
        for (int d = 0; d < 3; ++d) {
            if (K.dims[d] < 1 || K.dims[d] > RT_MAX_GRID_DIM) return fail(RT_EINVAL, "kappa grid dims must lie in [1, 512]");
            if (!std::isfinite(K.bbox[d]) || !std::isfinite(K.bbox[3 + d]) || !(K.bbox[3 + d] > K.bbox[d]))
                return fail(RT_EINVAL, "kappa grid box must be finite with x1 > x0");
            cells *= K.dims[d];
        }
        for (int64_t c = 0; c < cells; ++c)
            if (!(K.grid[c] >= 0.0f) || !std::isfinite(K.grid[c])) return fail(RT_EINVAL, "kappa grid values must be finite and >= 0");
    } else {
        if (!(K.k0 >= 0.0) || !std::isfinite(K.k0)) return fail(RT_EINVAL, "kappa: k0 must be >= 0");
        if (K.kind == RT_KAPPA_SINPROD && !(std::fabs(K.amp) <= K.k0))
            return fail(RT_EINVAL, "kappa must stay nonnegative (|amp| <= k0)");
    }
    if (P->n_obstacles < 0 || P->n_obstacles > RT_MAX_OBSTACLES) return fail(RT_EINVAL, "n_obstacles must lie in [0, 4]");
    if (P->n_obstacles > 0 && !P->obstacles) return fail(RT_EINVAL, "obstacles pointer missing");
    for (int o = 0; o < P->n_obstacles; ++o)
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(P->obstacles[o].lo[d]) || !std::isfinite(P->obstacles[o].hi[d]) ||
                !(P->obstacles[o].hi[d] > P->obstacles[o].lo[d]))
                return fail(RT_EINVAL, "obstacle box must be finite with hi > lo");
    if (P->n_obstacles > 0) {
        // Remark 1: the boxes are the hull's part outside the domain, so no
        // tetrahedron may lie inside one (its centroid is a strict interior point)
        for (int64_t t = 0; t < M.n_tet; ++t) {
            double c[3] = {0, 0, 0};
            for (int k = 0; k < 4; ++k)
                for (int d = 0; d < 3; ++d) c[d] += 0.25 * M.xyz[3 * (int64_t)M.tet[4 * t + k] + d];
            for (int o = 0; o < P->n_obstacles; ++o) {
                const rt_box& B = P->obstacles[o];
                if (c[0] > B.lo[0] && c[0] < B.hi[0] && c[1] > B.lo[1] && c[1] < B.hi[1] && c[2] > B.lo[2] &&
                    c[2] < B.hi[2])
                    return fail(RT_EINVAL, "a tetrahedron lies inside an opaque box");
            }
        }
    }
    const rt_freqs& Fq = P->freqs;
    if (Fq.F < 1 || Fq.F > 4096) return fail(RT_EINVAL, "frequency count must be in [1, 4096]");
    if (!Fq.nu || !Fq.w || !Fq.c || !Fq.albedo) return fail(RT_EINVAL, "frequency arrays missing");
    for (int f = 0; f < Fq.F; ++f) {
        if (!(Fq.c[f] > 0.0) || !std::isfinite(Fq.c[f])) return fail(RT_EINVAL, "c must be > 0");
        if (!(Fq.albedo[f] >= 0.0 && Fq.albedo[f] <= 1.0)) return fail(RT_EINVAL, "albedo must lie in [0, 1]");
        if (!P->grey && !(Fq.nu[f] > 0.0)) return fail(RT_EINVAL, "nu must be > 0");
    }
    if (P->grey && Fq.F != 1) return fail(RT_EINVAL, "grey formulation needs F == 1");
    if (H->mode != RT_MODE_DENSE && H->mode != RT_MODE_HMATRIX) return fail(RT_EINVAL, "mode");
    if (H->mode == RT_MODE_DENSE && H->prec != RT_PREC_F64 && H->prec != RT_PREC_F32)
        return fail(RT_EINVAL, "dense mode needs prec F64 or F32");
    if (H->mode == RT_MODE_HMATRIX) {
        if (H->prec != RT_PREC_F32) return fail(RT_EINVAL, "H-matrix mode computes in F32 (prec = RT_PREC_F32)");
        if (H->far_prec != RT_PREC_F32 && H->far_prec != RT_PREC_BF16 && H->far_prec != RT_PREC_F16)
            return fail(RT_EINVAL, "far_prec must be F32, BF16 or F16");
        if (!(H->aca_eps > 0.0 && H->aca_eps < 1.0)) return fail(RT_EINVAL, "aca_eps must lie in (0, 1)");
        if (H->leaf < 1) return fail(RT_EINVAL, "leaf must be >= 1");
        if (!(H->eta > 0.0)) return fail(RT_EINVAL, "eta must be > 0");
        if (H->rank_max < 0 || H->rank_max > 8192) return fail(RT_EINVAL, "rank_max must be in [0, 8192]");
        if (H->adm != RT_ADM_GAP && H->adm != RT_ADM_CENTER) return fail(RT_EINVAL, "adm must be RT_ADM_GAP or RT_ADM_CENTER");
        if (H->wave_bytes < 0) return fail(RT_EINVAL, "wave_bytes must be >= 0");
    }
    if (H->kappa_bins < 0 || H->kappa_bins > rt::kMaxGroups) return fail(RT_EINVAL, "kappa_bins must be in [0, 64]");
    if (H->gauss_pts < 1 || H->gauss_pts > rt::kMaxGauss) return fail(RT_EINVAL, "gauss_pts must be in [1, 32]");
    if (H->line_eval != RT_LINE_CLOSED && H->line_eval != RT_LINE_NODES) return fail(RT_EINVAL, "line_eval");
    if (M.n_vert * (int64_t)M.n_vert * Fq.F > ((int64_t)1 << 40) && H->mode == RT_MODE_DENSE)
        return fail(RT_EINVAL, "dense operator too large");
    return RT_OK;
}

template <class T>
int upload(rt::Operator& op, T** dst, const std::vector<T>& src, std::string& err)
{
    int rc = rt::dev_alloc(op, dst, src.size(), err);
    if (rc) return rc;
    return rt::upload_async(op, *dst, src.data(), src.size(), err);
}

// Operator groups of the frequency channels (Remark of Section 2.1): exact
// equality of c, K equal-width bins of [min c, max c], or the caller's map.
// A group's scale is the midpoint of its channels' scales; channel f applies
// (c_f / c_g) G_g.
int group_channels(rt::Operator& op, const rt_freqs& Fq, int bins, std::string& err)
{
    using namespace rt;
    const int F = Fq.F;
    op.fgroup.assign(F, 0);
    op.gc.clear();
    if (Fq.group) {
        int G = 0;
        for (int f = 0; f < F; ++f) {
            if (Fq.group[f] < 0 || Fq.group[f] >= kMaxGroups) {
                err = "group map entries must lie in [0, 64)";
                return RT_EINVAL;
            }
            G = std::max(G, Fq.group[f] + 1);
            op.fgroup[f] = Fq.group[f];
        }
        std::vector<int> used(G, 0);
        for (int f = 0; f < F; ++f) used[op.fgroup[f]] = 1;
        for (int g = 0; g < G; ++g)
            if (!used[g]) {
                err = "group map leaves group " + std::to_string(g) + " empty";
                return RT_EINVAL;
            }
        std::vector<double> lo(G, 1e300), hi(G, -1e300);
        for (int f = 0; f < F; ++f) {
            lo[op.fgroup[f]] = std::min(lo[op.fgroup[f]], Fq.c[f]);
            hi[op.fgroup[f]] = std::max(hi[op.fgroup[f]], Fq.c[f]);
        }
        for (int g = 0; g < G; ++g) op.gc.push_back(lo[g] == hi[g] ? lo[g] : 0.5 * (lo[g] + hi[g]));
    } else if (bins > 0) {
        double cmin = Fq.c[0], cmax = Fq.c[0];
        for (int f = 1; f < F; ++f) {
            cmin = std::min(cmin, Fq.c[f]);
            cmax = std::max(cmax, Fq.c[f]);
        }
        std::vector<int> bin(F);
        std::vector<double> lo(bins, 1e300), hi(bins, -1e300);
        for (int f = 0; f < F; ++f) {
            int b = cmax > cmin ? (int)std::floor((Fq.c[f] - cmin) / (cmax - cmin) * bins) : 0;
            b = std::min(std::max(b, 0), bins - 1);
            bin[f] = b;
            lo[b] = std::min(lo[b], Fq.c[f]);
            hi[b] = std::max(hi[b], Fq.c[f]);
        }
        std::vector<int> gid(bins, -1);
        for (int b = 0; b < bins; ++b)
            if (lo[b] <= hi[b]) {
                gid[b] = (int)op.gc.size();
                op.gc.push_back(lo[b] == hi[b] ? lo[b] : 0.5 * (lo[b] + hi[b]));
            }
        if ((int)op.gc.size() > kMaxGroups) {
            err = "more than 64 kappa groups";
            return RT_EINVAL;
        }
        for (int f = 0; f < F; ++f) op.fgroup[f] = gid[bin[f]];
    } else {
        for (int f = 0; f < F; ++f) {
            int g = -1;
            for (int k = 0; k < (int)op.gc.size(); ++k)
                if (op.gc[k] == Fq.c[f]) g = k;
            if (g < 0) {
                if ((int)op.gc.size() >= kMaxGroups) {
                    err = "more than 64 distinct kappa scales c";
                    return RT_EINVAL;
                }
                g = (int)op.gc.size();
                op.gc.push_back(Fq.c[f]);
            }
            op.fgroup[f] = g;
        }
    }
    op.G = (int)op.gc.size();
    op.fscale.assign(F, 1.0);
    op.binned = 0;
    for (int f = 0; f < F; ++f) {
        op.fscale[f] = Fq.c[f] / op.gc[op.fgroup[f]];
        if (op.fscale[f] != 1.0) op.binned = 1;
    }
    return RT_OK;
}

int build(rt::Operator& op, const rt_problem* P, const rt_hparams* H, cudaStream_t s, std::string& err,
          rt::Plan* pre)
{
    using namespace rt;
    int rc;
    cudaEvent_t e0, e1;
    RT_CUDA_TRY(cudaGetDevice(&op.device));
    op.stream = s;
    const int64_t N = P->mesh.n_vert, T = P->mesh.n_tet;
    op.N = (int)N;
    op.T = (int)T;
    op.mode = H->mode;
    op.prec = H->mode == RT_MODE_DENSE ? H->prec : RT_PREC_F32;
    op.far_prec = H->mode == RT_MODE_DENSE ? op.prec : H->far_prec;
    op.vec64 = op.mode == RT_MODE_DENSE && op.prec == RT_PREC_F64;
    op.aca_eps = H->aca_eps;
    op.leaf = H->leaf;
    op.eta = H->eta;
    op.adm = H->adm;
    op.tc_off = H->tensor_cores == 1;
    op.refine = H->mode == RT_MODE_HMATRIX && H->refine && H->far_prec != RT_PREC_F32;
    op.ngauss = H->gauss_pts;
    op.rank_max = H->rank_max > 0 ? H->rank_max : 512;
    op.wave_bytes = H->wave_bytes > 0 ? H->wave_bytes : ((int64_t)8 << 30);
    op.grey = P->grey ? 1 : 0;
    const rt_freqs& Fq = P->freqs;
    op.F = Fq.F;
    op.nu.assign(Fq.nu, Fq.nu + Fq.F);
    op.w.assign(Fq.w, Fq.w + Fq.F);
    op.c.assign(Fq.c, Fq.c + Fq.F);
    op.albedo.assign(Fq.albedo, Fq.albedo + Fq.F);
    if ((rc = group_channels(op, Fq, H->kappa_bins, err))) return rc;
    op.q0 = P->Q0;
    op.Q.assign(Fq.F, 0.0);
    for (int f = 0; f < Fq.F; ++f)
        op.Q[f] = P->grey ? P->Q0 * 6.493939402266829 * std::pow(P->T_emit, 4.0) : P->Q0 * planck_host(Fq.nu[f], P->T_emit);

    // ---- vertex order: cluster tree (H-matrix) or caller order (dense) -------
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    if (op.mode == RT_MODE_HMATRIX) {
        if (pre) op.plan = std::move(*pre);   // computed earlier for the same mesh and parameters
        else if ((rc = plan_build(P->mesh.xyz, N, op.leaf, op.eta, op.adm, op.plan, err))) return rc;
    } else {
        op.plan = Plan();
        op.plan.N = (int)N;
        op.plan.perm.resize(N);
        op.plan.iperm.resize(N);
        for (int64_t k = 0; k < N; ++k) op.plan.perm[k] = op.plan.iperm[k] = (int)k;
        op.plan.leaf_start.push_back(0);
        op.plan.leaf_size.push_back((int)N);
        op.plan.clusters.push_back({0, (int)N, -1, -1});
    }
    const std::vector<int>& perm = op.plan.perm;
    const std::vector<int>& iperm = op.plan.iperm;
    std::vector<double> xyz64(3 * N);
    std::vector<float4> xyz32(N);
    for (int64_t t = 0; t < N; ++t) {
        const double* p = P->mesh.xyz + 3 * (int64_t)perm[t];
        for (int d = 0; d < 3; ++d) xyz64[3 * t + d] = p[d];
        xyz32[t] = make_float4((float)p[0], (float)p[1], (float)p[2], 0.f);
    }
    std::vector<int4> tet(T);
    std::vector<dbl4> tg64(T);
    std::vector<float4> tg32(T);
    std::vector<double> tv64(T);
    std::vector<float> tv32(T);
    std::vector<int> cnt(N + 1, 0);
    for (int64_t k = 0; k < T; ++k) {
        const int32_t* v = P->mesh.tet + 4 * k;
        int a[4] = {iperm[v[0]], iperm[v[1]], iperm[v[2]], iperm[v[3]]};
        tet[k] = make_int4(a[0], a[1], a[2], a[3]);
        const double* X[4];
        for (int d = 0; d < 4; ++d) X[d] = &xyz64[3 * (int64_t)a[d]];
        double e[3][3];
        for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) e[r][d] = X[r + 1][d] - X[0][d];
        const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                           e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        const double vol = std::fabs(det) / 6.0;
        if (!(vol > 0.0)) {
            err = "mesh: degenerate tetrahedron " + std::to_string(k);
            return RT_EINVAL;
        }
        double cen[3], dm = 0.0;
        for (int d = 0; d < 3; ++d) cen[d] = 0.25 * (X[0][d] + X[1][d] + X[2][d] + X[3][d]);
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j) {
                double s2 = 0.0;
                for (int d = 0; d < 3; ++d) s2 += (X[i][d] - X[j][d]) * (X[i][d] - X[j][d]);
                dm = std::max(dm, std::sqrt(s2));
            }
        tg64[k] = make_dbl4(cen[0], cen[1], cen[2], dm);
        tg32[k] = make_float4((float)cen[0], (float)cen[1], (float)cen[2], (float)dm);
        tv64[k] = vol;
        tv32[k] = (float)vol;
        for (int d = 0; d < 4; ++d) cnt[a[d] + 1]++;
    }
    for (int64_t v = 0; v < N; ++v) cnt[v + 1] += cnt[v];
    std::vector<int> vt_idx(cnt[N]);
    {
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t k = 0; k < T; ++k) {
            const int a[4] = {tet[k].x, tet[k].y, tet[k].z, tet[k].w};
            for (int d = 0; d < 4; ++d) vt_idx[fill[a[d]]++] = (int)(k << 2) | d;
        }
    }
    for (int64_t v = 0; v < N; ++v)
        if (cnt[v + 1] == cnt[v]) {
            err = "mesh: vertex " + std::to_string(perm[v]) + " belongs to no tetrahedron";
            return RT_EINVAL;
        }
    std::vector<int4> emit(std::max<int64_t>(P->n_emit, 1));
    for (int64_t k = 0; k < P->n_emit; ++k)
        emit[k] = make_int4(iperm[P->emit_tri[3 * k]], iperm[P->emit_tri[3 * k + 1]], iperm[P->emit_tri[3 * k + 2]], 0);
    op.n_emit = (int)P->n_emit;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    op.info.ms_tree = ms;

    if ((rc = upload(op, &op.d_xyz64, xyz64, err))) return rc;
    if ((rc = upload(op, &op.d_xyz32, xyz32, err))) return rc;
    if ((rc = upload(op, &op.d_tet, tet, err))) return rc;
    if ((rc = upload(op, &op.d_tgeo64, tg64, err))) return rc;
    if ((rc = upload(op, &op.d_tgeo32, tg32, err))) return rc;
    if ((rc = upload(op, &op.d_tvol64, tv64, err))) return rc;
    if ((rc = upload(op, &op.d_tvol32, tv32, err))) return rc;
    if ((rc = upload(op, &op.d_vt_ptr, cnt, err))) return rc;
    if ((rc = upload(op, &op.d_vt_idx, vt_idx, err))) return rc;
    op.h_vt_ptr = std::move(cnt);
    op.h_vt_idx = std::move(vt_idx);
    if ((rc = upload(op, &op.d_perm, perm, err))) return rc;
    if ((rc = upload(op, &op.d_iperm, iperm, err))) return rc;
    if ((rc = upload(op, &op.d_emit, emit, err))) return rc;

    KernelParams& kp = op.kp;
    kp.N = (int)N;
    kp.T = (int)T;
    kp.kappa_kind = P->kappa.kind;
    kp.k0 = P->kappa.k0;
    kp.amp = P->kappa.kind == RT_KAPPA_SINPROD ? P->kappa.amp : 0.0;
    if (P->kappa.kind == RT_KAPPA_GRID) {
        kp.k0 = kp.amp = 0.0;
        const int64_t cells = (int64_t)P->kappa.dims[0] * P->kappa.dims[1] * P->kappa.dims[2];
        std::vector<float> g32(P->kappa.grid, P->kappa.grid + cells);
        std::vector<double> g64(g32.begin(), g32.end());
        float* d32 = nullptr;
        double* d64 = nullptr;
        if ((rc = upload(op, &d32, g32, err))) return rc;
        if ((rc = upload(op, &d64, g64, err))) return rc;
        kp.kgrid32 = d32;
        kp.kgrid64 = d64;
        for (int d = 0; d < 3; ++d) {
            kp.gdims[d] = P->kappa.dims[d];
            kp.glo[d] = P->kappa.bbox[d];
            kp.ghi[d] = P->kappa.bbox[3 + d];
        }
    }
    kp.n_obst = P->n_obstacles;
    for (int o = 0; o < P->n_obstacles; ++o)
        for (int d = 0; d < 3; ++d) {
            kp.olo[o][d] = P->obstacles[o].lo[d];
            kp.ohi[o][d] = P->obstacles[o].hi[d];
        }
    kp.k0f = (float)kp.k0;
    kp.ampf = (float)kp.amp;
    // the first wall keeps its own fields (the one-wall kernels' path); the
    // further walls and the corner paths go to the extra-term list
    kp.has_wall = (P->n_walls >= 1 && P->walls[0].R0 > 0.0) ? 1 : 0;
    for (int w = 0; w < P->n_walls; ++w) {
        const double* n = P->walls[w].n;
        const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int d = 0; d < 3; ++d) {
            kp.wps[w][d] = P->walls[w].p[d];
            kp.wns[w][d] = n[d] / nn;
        }
        kp.wR[w] = P->walls[w].R0;
    }
    if (P->n_walls >= 1) {
        for (int d = 0; d < 3; ++d) {
            kp.wp[d] = kp.wps[0][d];
            kp.wn[d] = kp.wns[0][d];
        }
        kp.R0 = kp.wR[0];
    }
    kp.n_extra = 0;
    for (int w = 1; w < P->n_walls; ++w)
        if (kp.wR[w] > 0.0) {
            kp.xkind[kp.n_extra] = 1;
            kp.xa[kp.n_extra] = w;
            kp.xb[kp.n_extra] = -1;
            ++kp.n_extra;
        }
    if (P->corner)
        for (int a = 0; a < P->n_walls; ++a)
            for (int b = a + 1; b < P->n_walls; ++b) {
                const double dot = kp.wns[a][0] * kp.wns[b][0] + kp.wns[a][1] * kp.wns[b][1] + kp.wns[a][2] * kp.wns[b][2];
                if (std::fabs(dot) > 1e-12 || !(kp.wR[a] > 0.0) || !(kp.wR[b] > 0.0)) continue;
                kp.xkind[kp.n_extra] = 2;
                kp.xa[kp.n_extra] = a;
                kp.xb[kp.n_extra] = b;
                ++kp.n_extra;
            }
    kp.ext = (kp.n_extra > 0 || kp.n_obst > 0 || kp.kappa_kind == RT_KAPPA_GRID) ? 1 : 0;
    kp.G = op.G;
    for (int g = 0; g < op.G; ++g) {
        kp.c[g] = op.gc[g];
        kp.cf[g] = (float)op.gc[g];
    }
    kp.c_arith = 0;
    if (op.G >= 3) {
        const double dc = op.gc[1] - op.gc[0];
        bool arith = dc != 0.0;
        for (int g = 2; g < op.G && arith; ++g)
            arith = std::fabs(op.gc[g] - (op.gc[0] + g * dc)) <= 1e-12 * std::max(1.0, std::fabs(op.gc[g]));
        if (arith) {
            kp.c_arith = 1;
            kp.c0f = (float)op.gc[0];
            kp.dcf = (float)dc;
        }
    }
    kp.ngauss = op.ngauss;
    kp.line_closed = (H->line_eval == RT_LINE_CLOSED && op.ngauss >= 16) ? 1 : 0;
    kp.xyz32 = op.d_xyz32;
    kp.xyz64 = op.d_xyz64;
    kp.tet = op.d_tet;
    kp.tgeo32 = op.d_tgeo32;
    kp.tgeo64 = op.d_tgeo64;
    kp.tvol32 = op.d_tvol32;
    kp.tvol64 = op.d_tvol64;
    kp.vt_ptr = op.d_vt_ptr;
    kp.vt_idx = op.d_vt_idx;
    if ((rc = dev_alloc(op, &op.d_work, 2, err))) return rc;
    RT_CUDA_TRY(cudaMemsetAsync(op.d_work, 0, 2 * sizeof(unsigned long long), s));
    kp.work = op.d_work;
    if ((rc = assemble_setup_constants(op, err))) return rc;

    cudaEventRecord(e0, s);
    if ((rc = assemble_source(op, s, err))) return rc;
    cudaEventRecord(e1, s);
    RT_CUDA_TRY(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    op.info.ms_source = ms;
    if (op.mode == RT_MODE_DENSE) {
        cudaEventRecord(e0, s);
        if ((rc = assemble_dense(op, s, err))) return rc;
        cudaEventRecord(e1, s);
        RT_CUDA_TRY(cudaEventSynchronize(e1));
        cudaEventElapsedTime(&ms, e0, e1);
        op.info.ms_near = ms;
        op.n_near = 1;
    } else {
        if ((rc = prepare_row_eval(op, err))) return rc;
        if ((rc = assemble_hmatrix(op, s, err))) return rc;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((rc = hmatvec_prepare(op, err))) return rc;
    const size_t esz = op.vec64 ? 8 : 4;
    {
        char *a = nullptr, *b = nullptr;
        if ((rc = dev_alloc(op, &a, (size_t)op.F * N * esz, err))) return rc;
        if ((rc = dev_alloc(op, &b, (size_t)op.F * N * esz, err))) return rc;
        op.d_xt = (float*)a;
        op.d_yt = (float*)b;
    }
    RT_CUDA_TRY(cudaStreamSynchronize(s));
    RT_CUDA_TRY(cudaGetLastError());
    // statistics
    rt_info& I = op.info;
    {
        unsigned long long w[2] = {0, 0};
        RT_CUDA_TRY(cudaMemcpy(w, op.d_work, sizeof(w), cudaMemcpyDeviceToHost));
        I.assembly_terms = (int64_t)w[0];
        I.assembly_depths = (int64_t)w[1];
    }
    I.N = N;
    I.F = op.F;
    I.G = op.G;
    I.mode = op.mode;
    I.prec = op.prec;
    I.far_prec = op.far_prec;
    I.n_leaves = (int64_t)op.plan.leaf_start.size();
    I.n_near = op.mode == RT_MODE_DENSE ? 1 : (int64_t)op.plan.near_blocks.size();
    I.n_far = op.n_far;
    I.n_dense_fallback = op.n_fallback;
    I.compression = 1.0 - (double)I.stored_entries / ((double)N * (double)N);
    I.peak_bytes = std::max(I.peak_bytes, I.device_bytes);
    return RT_OK;
}

}  // namespace

namespace rt {
int validate_problem(const rt_problem* P, const rt_hparams* H, std::string& err)
{
    const int rc = validate(P, H);
    if (rc) err = g_err;
    return rc;
}

int build_operator(Operator& op, const rt_problem* P, const rt_hparams* H, cudaStream_t s, std::string& err,
                   Plan* pre)
{
    try {
        return build(op, P, H, s, err, pre);
    } catch (const std::bad_alloc&) {
        err = "host allocation failed";
        return RT_ENOMEM;
    } catch (...) {
        err = "unexpected exception during build";
        return RT_EINVAL;
    }
}

void set_last_error(const std::string& msg) { g_err = msg; }

void operator_release(Operator& op, cudaStream_t s)
{
    for (void* p : op.allocations)
        if (p) cudaFreeAsync(p, s);
    op.allocations.clear();
    if (op.far_buf.base || op.far_lo_buf.base) {
        // unmapping is not stream ordered: wait for the work queued on s
        cudaStreamSynchronize(s);
        growbuf_release(op.far_buf);
        growbuf_release(op.far_lo_buf);
    }
    if (op.cap_stream) cudaStreamDestroy(op.cap_stream);
    op.cap_stream = nullptr;
}
}  // namespace rt

extern "C" {

int rt_build_operator(const rt_problem* prob, const rt_hparams* hp, void* stream, rt_operator** out)
{
    if (!out) return fail(RT_EINVAL, "out is null");
    *out = nullptr;
    int rc = validate(prob, hp);
    if (rc) return rc;
    rt_operator* h = new (std::nothrow) rt_operator();
    if (!h) return fail(RT_ENOMEM, "host allocation failed");
    std::string err;
    rc = rt::build_operator(h->op, prob, hp, (cudaStream_t)stream, err, nullptr);
    if (rc) {
        rt::operator_release(h->op, (cudaStream_t)stream);
        cudaStreamSynchronize((cudaStream_t)stream);
        delete h;
        return fail(rc, err);
    }
    *out = h;
    g_err.clear();
    return RT_OK;
}

int rt_operator_info(const rt_operator* op, rt_info* info)
{
    if (!op || !info) return fail(RT_EINVAL, "null argument");
    *info = op->op.info;
    return RT_OK;
}

int rt_apply(rt_operator* h, const void* X, void* Y, void* stream)
{
    if (!h || !X || !Y) return fail(RT_EINVAL, "null argument");
    rt::Operator& op = h->op;
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    int rc;
    if (op.mode == RT_MODE_DENSE) {
        rc = rt::apply_tree(op, X, Y, s, err);
        if (!rc && op.binned) rc = rt::scale_rows(op, Y, s);
    } else {
        rc = rt::permute_vectors(op, X, op.d_xt, 1, op.vec64, op.F, s);
        if (!rc) rc = rt::apply_tree(op, op.d_xt, op.d_yt, s, err);
        if (!rc) rc = rt::permute_vectors(op, op.d_yt, Y, 0, op.vec64, op.F, s, op.binned ? op.d_fscale : nullptr);
    }
    if (rc && err.empty()) err = "kernel launch failed";
    if (rc) return fail(rc, err);
    return RT_OK;
}

int rt_apply_group(rt_operator* h, int group, const void* X, int64_t ldx, int nrhs, void* Y, int64_t ldy,
                   void* stream)
{
    if (!h || (nrhs > 0 && (!X || !Y))) return fail(RT_EINVAL, "null argument");
    rt::Operator& op = h->op;
    if (group < 0 || group >= op.G) return fail(RT_EINVAL, "group out of range");
    if (nrhs < 0 || ldx < op.N || ldy < op.N) return fail(RT_EINVAL, "nrhs < 0 or leading dimension < N");
    std::string err;
    int rc = rt::apply_group(op, group, X, ldx, nrhs, Y, ldy, (cudaStream_t)stream, err);
    if (rc && err.empty()) err = "kernel launch failed";
    if (rc) return fail(rc, err);
    return RT_OK;
}

int rt_apply_noalloc(rt_operator* h, const void* X, void* Y, void* stream)
{
    if (!h || !X || !Y) return fail(RT_EINVAL, "null argument");
    std::string err;
    int rc = rt::apply_noalloc(h->op, X, Y, (cudaStream_t)stream, err);
    if (rc) return fail(rc, err);
    return RT_OK;
}

int rt_eval_sin2pi(const float* x, float* lib_out, float* ref_out, int64_t n, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !lib_out || !ref_out))) return fail(RT_EINVAL, "null argument");
    std::string err;
    int rc = rt::eval_sin2pi(x, lib_out, ref_out, n, (cudaStream_t)stream, err);
    if (rc) return fail(rc, err);
    return RT_OK;
}

int rt_source(rt_operator* h, void* out, void* stream)
{
    if (!h || !out) return fail(RT_EINVAL, "null argument");
    rt::Operator& op = h->op;
    int rc = rt::permute_vectors(op, op.d_SE, out, 0, op.vec64, op.F, (cudaStream_t)stream);
    if (rc) return fail(rc, "permute failed");
    return RT_OK;
}

int rt_eval_entries(rt_operator* h, int group, int64_t count, const int32_t* rows, const int32_t* cols, double* out,
                    void* stream)
{
    if (!h || (count > 0 && (!rows || !cols || !out))) return fail(RT_EINVAL, "null argument");
    if (group < 0 || group >= h->op.G) return fail(RT_EINVAL, "group out of range");
    std::string err;
    int rc = rt::eval_entries(h->op, group, count, rows, cols, out, (cudaStream_t)stream, err);
    if (rc) return fail(rc, err);
    return RT_OK;
}

int rt_solve_fixed_point(rt_operator* h, const rt_solve_opts* opts, void* J_dev, double* T_dev, rt_solve_stats* stats,
                         void* stream)
{
    if (!h || !opts || !J_dev || !T_dev) return fail(RT_EINVAL, "null argument");
    if (opts->max_iter < 1 || opts->check_every < 1 || !(opts->tol >= 0.0) || !(opts->T0 >= 0.0))
        return fail(RT_EINVAL, "invalid solve options");
    rt_solve_stats st{};
    std::string err;
    int rc = rt::solve_fixed_point(h->op, *opts, J_dev, T_dev, st, (cudaStream_t)stream, err);
    if (stats) *stats = st;
    if (rc) return fail(rc, err);
    return RT_OK;
}

void rt_free(rt_operator* h)
{
    if (!h) return;
    // the operator may still be read by work the caller queued on any stream
    cudaDeviceSynchronize();
    rt::operator_release(h->op, nullptr);
    cudaStreamSynchronize(nullptr);
    delete h;
}

const char* rt_last_error(void) { return g_err.c_str(); }

int rt_plan(const double* xyz, int64_t n, int leaf, double eta, int adm, int32_t* perm, int32_t* blocks,
            int64_t cap, int64_t* counts)
{
    if (!xyz || !counts) return fail(RT_EINVAL, "null argument");
    rt::Plan P;
    std::string err;
    int rc;
    try {
        rc = rt::plan_build(xyz, n, leaf, eta, adm, P, err);
    } catch (...) {
        rc = RT_ENOMEM;
        err = "host allocation failed";
    }
    if (rc) return fail(rc, err);
    counts[0] = (int64_t)P.leaf_start.size();
    counts[1] = (int64_t)P.near_blocks.size();
    counts[2] = (int64_t)P.far_blocks.size();
    if (perm)
        for (int64_t k = 0; k < n; ++k) perm[k] = P.perm[k];
    if (blocks) {
        int64_t k = 0;
        for (const auto& b : P.near_blocks) {
            if (k >= cap) break;
            int32_t* o = blocks + 5 * k++;
            o[0] = b.row0; o[1] = b.m; o[2] = b.col0; o[3] = b.n; o[4] = 0;
        }
        for (const auto& b : P.far_blocks) {
            if (k >= cap) break;
            int32_t* o = blocks + 5 * k++;
            o[0] = b.row0; o[1] = b.m; o[2] = b.col0; o[3] = b.n; o[4] = 1;
        }
    }
    return RT_OK;
}

}  // extern "C"
