// rt_plan.cpp -- host cluster tree and block tree (Section 2.1).
//
// Cluster tree: recursive bisection of the point set along the longest axis
// of its bounding box, at the median point (ties broken by vertex id), down
// to clusters of at most `leaf` points.  Each cluster carries its centroid
// and radius (largest distance from the centroid).
//
// Block tree: recursion from (root, root); a pair (t, s) is admissible when
// max(R_t, R_s) < eta d(t, s) (the paper's geometric criterion) and then
// becomes one far block compressed by ACA; otherwise the non-leaf side(s) are
// split; two leaves give a dense block.  d(t, s) is the distance between the
// clusters' bounding spheres, |c_t - c_s| - R_t - R_s (RT_ADM_GAP), or the
// distance between the centroids, |c_t - c_s| (RT_ADM_CENTER, the literal
// reading, under which touching clusters are admissible).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "rt_internal.h"

namespace rt {
namespace {

struct Cluster {
    int start, size;
    double c[3];
    double R;
    int left = -1, right = -1;
};

struct Builder {
    const double* xyz;
    int leaf;
    std::vector<int> idx;   // tree order -> vertex id (being permuted)
    std::vector<Cluster> cl;

    int build(int start, int size)
    {
        Cluster C;
        C.start = start;
        C.size = size;
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        double s[3] = {0, 0, 0};
        for (int k = start; k < start + size; ++k) {
            const double* p = xyz + 3 * (int64_t)idx[k];
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], p[d]);
                hi[d] = std::max(hi[d], p[d]);
                s[d] += p[d];
            }
        }
        for (int d = 0; d < 3; ++d) C.c[d] = s[d] / size;
        double R2 = 0.0;
        for (int k = start; k < start + size; ++k) {
            const double* p = xyz + 3 * (int64_t)idx[k];
            double r2 = 0.0;
            for (int d = 0; d < 3; ++d) r2 += (p[d] - C.c[d]) * (p[d] - C.c[d]);
            R2 = std::max(R2, r2);
        }
        C.R = std::sqrt(R2);
        int id = (int)cl.size();
        cl.push_back(C);
        if (size > leaf) {
            int ax = 0;
            for (int d = 1; d < 3; ++d)
                if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
            auto b = idx.begin() + start, e = idx.begin() + start + size;
            const double* X = xyz;
            std::stable_sort(b, e, [X, ax](int a, int bb) {
                double pa = X[3 * (int64_t)a + ax], pb = X[3 * (int64_t)bb + ax];
                if (pa != pb) return pa < pb;
                return a < bb;
            });
            int half = size / 2;
            int l = build(start, half);
            int r = build(start + half, size - half);
            cl[id].left = l;
            cl[id].right = r;
        }
        return id;
    }
};

void block_recursion(const std::vector<Cluster>& cl, double eta, int adm, int t, int s,
                     std::vector<FarBlock>& nearb, std::vector<FarBlock>& farb)
{
    const Cluster& T = cl[t];
    const Cluster& S = cl[s];
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) d2 += (T.c[k] - S.c[k]) * (T.c[k] - S.c[k]);
    double d = std::sqrt(d2);
    if (adm == RT_ADM_GAP) d -= T.R + S.R;
    const bool admissible = d > 0.0 && std::max(T.R, S.R) < eta * d;
    if (admissible) {
        farb.push_back({T.start, T.size, S.start, S.size, t, s});
        return;
    }
    bool tl = T.left < 0, sl = S.left < 0;
    if (tl && sl) {
        nearb.push_back({T.start, T.size, S.start, S.size, t, s});
        return;
    }
    if (tl) {
        block_recursion(cl, eta, adm, t, S.left, nearb, farb);
        block_recursion(cl, eta, adm, t, S.right, nearb, farb);
    } else if (sl) {
        block_recursion(cl, eta, adm, T.left, s, nearb, farb);
        block_recursion(cl, eta, adm, T.right, s, nearb, farb);
    } else {
        block_recursion(cl, eta, adm, T.left, S.left, nearb, farb);
        block_recursion(cl, eta, adm, T.left, S.right, nearb, farb);
        block_recursion(cl, eta, adm, T.right, S.left, nearb, farb);
        block_recursion(cl, eta, adm, T.right, S.right, nearb, farb);
    }
}

}  // namespace

int plan_build(const double* xyz, int64_t n, int leaf, double eta, int adm, Plan& out, std::string& err)
{
    if (n <= 0 || n > (int64_t)1 << 30) {
        err = "plan: vertex count out of range";
        return RT_EINVAL;
    }
    if (leaf < 1) {
        err = "plan: leaf size must be >= 1";
        return RT_EINVAL;
    }
    if (adm != RT_ADM_GAP && adm != RT_ADM_CENTER) {
        err = "plan: unknown admissibility reading";
        return RT_EINVAL;
    }
    if (!(eta > 0.0)) {
        err = "plan: eta must be > 0";
        return RT_EINVAL;
    }
    Builder B;
    B.xyz = xyz;
    B.leaf = leaf;
    B.idx.resize(n);
    std::iota(B.idx.begin(), B.idx.end(), 0);
    B.cl.reserve(4 * (size_t)(n / leaf + 1));
    B.build(0, (int)n);
    out = Plan();
    out.N = (int)n;
    out.leaf = leaf;
    out.perm = B.idx;
    out.iperm.assign(n, 0);
    for (int64_t k = 0; k < n; ++k) out.iperm[out.perm[k]] = (int)k;
    out.clusters.reserve(B.cl.size());
    for (const Cluster& C : B.cl) out.clusters.push_back({C.start, C.size, C.left, C.right});
    for (const Cluster& C : B.cl)
        if (C.left < 0) {
            out.leaf_start.push_back(C.start);
            out.leaf_size.push_back(C.size);
        }
    // leaves are produced in tree order by the depth-first build
    block_recursion(B.cl, eta, adm, 0, 0, out.near_blocks, out.far_blocks);
    auto key = [](const FarBlock& a, const FarBlock& b) {
        if (a.row0 != b.row0) return a.row0 < b.row0;
        return a.col0 < b.col0;
    };
    std::sort(out.near_blocks.begin(), out.near_blocks.end(), key);
    std::sort(out.far_blocks.begin(), out.far_blocks.end(), key);
    return RT_OK;
}

}  // namespace rt
