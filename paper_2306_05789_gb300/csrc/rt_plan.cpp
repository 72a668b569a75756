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
//
// Host threads.  Large point sets (>= kParMin points) build the two trees on
// several host threads (RT_PLAN_THREADS in the environment, default: the
// hardware threads, at most 16; 1 = one thread).  The result is identical to
// the one-thread build, bit for bit:
//   - a cluster's id is its position in depth-first pre-order, known before
//     its subtree is built (the size of a subtree depends only on its point
//     count), so the subtrees of a split are built concurrently into disjoint
//     parts of the index array and of the cluster array, each with exactly
//     the arithmetic of the sequential recursion;
//   - the block recursion is split at its first levels into independent pair
//     recursions whose lists are concatenated in the sequential order;
//   - the blocks are then sorted by (row0, col0), which identifies a block of
//     the partition uniquely, so the order does not depend on the threads.
#include <algorithm>
#include <system_error>
#include <cmath>
#include <cstdlib>
#include <exception>
#include <functional>
#include <map>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "rt_internal.h"

namespace rt {
namespace {

constexpr int64_t kParMin = 32768;   // fewer points: one thread
constexpr int kMaxPlanThreads = 16;

struct Cluster {
    int start, size;
    double c[3];
    double R;
    int left = -1, right = -1;
};

// Runs f(k) for k = 0 .. count-1, each on its own thread when threads > 1
// (the last one on the calling thread); an exception in any of them is
// rethrown on the calling thread after all have finished.
void run_all(int count, bool threads, const std::function<void(int)>& f)
{
    if (!threads || count < 2) {
        for (int k = 0; k < count; ++k) f(k);
        return;
    }
    std::vector<std::exception_ptr> errs(count);
    std::vector<std::thread> th;
    auto guarded = [&](int k) {
        try {
            f(k);
        } catch (...) {
            errs[k] = std::current_exception();
        }
    };
    for (int k = 0; k + 1 < count; ++k) {
        try {
            th.emplace_back(guarded, k);
        } catch (const std::system_error&) {
            guarded(k);   // no thread available: run it here
        }
    }
    guarded(count - 1);
    for (auto& t : th) t.join();
    for (auto& e : errs)
        if (e) std::rethrow_exception(e);
}

struct Builder {
    const double* xyz;
    int leaf;
    int par_depth = 0;               // split levels that run on separate threads
    std::vector<int> idx;            // tree order -> vertex id (being permuted)
    std::vector<Cluster> cl;         // pre-order, sized before the build
    std::map<int, int> count_memo;   // subtree cluster count by point count (read-only while building)

    int count(int size)
    {
        if (size <= leaf) return 1;
        auto it = count_memo.find(size);
        if (it != count_memo.end()) return it->second;
        const int c = 1 + count(size / 2) + count(size - size / 2);
        count_memo.emplace(size, c);
        return c;
    }

    int count_const(int size) const
    {
        return size <= leaf ? 1 : count_memo.at(size);
    }

    // cluster `id` holds points [start, start + size) of idx
    void build(int start, int size, int id, int depth)
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
            const int half = size / 2;
            C.left = id + 1;
            C.right = id + 1 + count_const(half);
            cl[id] = C;
            run_all(2, depth < par_depth, [&](int k) {
                if (k == 0) build(start, half, C.left, depth + 1);
                else build(start + half, size - half, C.right, depth + 1);
            });
        } else {
            cl[id] = C;
        }
    }
};

struct BlockLists {
    std::vector<FarBlock> nearb, farb;
};

// The pairs a non-admissible, non-leaf pair (t, s) splits into, in the order
// of the sequential recursion.
int split_pairs(const Cluster& T, const Cluster& S, int t, int s, int (*out)[2])
{
    const bool tl = T.left < 0, sl = S.left < 0;
    if (tl) {
        out[0][0] = t, out[0][1] = S.left;
        out[1][0] = t, out[1][1] = S.right;
        return 2;
    }
    if (sl) {
        out[0][0] = T.left, out[0][1] = s;
        out[1][0] = T.right, out[1][1] = s;
        return 2;
    }
    out[0][0] = T.left, out[0][1] = S.left;
    out[1][0] = T.left, out[1][1] = S.right;
    out[2][0] = T.right, out[2][1] = S.left;
    out[3][0] = T.right, out[3][1] = S.right;
    return 4;
}

// Admissible (far) or leaf-leaf (near) pairs end the recursion: returns true
// after recording the block.
bool leaf_pair(const std::vector<Cluster>& cl, double eta, int adm, int t, int s, BlockLists& out)
{
    const Cluster& T = cl[t];
    const Cluster& S = cl[s];
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) d2 += (T.c[k] - S.c[k]) * (T.c[k] - S.c[k]);
    double d = std::sqrt(d2);
    if (adm == RT_ADM_GAP) d -= T.R + S.R;
    const bool admissible = d > 0.0 && std::max(T.R, S.R) < eta * d;
    if (admissible) {
        out.farb.push_back({T.start, T.size, S.start, S.size, t, s});
        return true;
    }
    if (T.left < 0 && S.left < 0) {
        out.nearb.push_back({T.start, T.size, S.start, S.size, t, s});
        return true;
    }
    return false;
}

void block_recursion(const std::vector<Cluster>& cl, double eta, int adm, int t, int s, BlockLists& out)
{
    if (leaf_pair(cl, eta, adm, t, s, out)) return;
    int pr[4][2];
    const int np = split_pairs(cl[t], cl[s], t, s, pr);
    for (int k = 0; k < np; ++k) block_recursion(cl, eta, adm, pr[k][0], pr[k][1], out);
}

// The same recursion with its first `depth` levels of splits on separate
// threads; the lists of the sub-recursions are appended in the sequential order.
void block_recursion_par(const std::vector<Cluster>& cl, double eta, int adm, int t, int s, int depth,
                         BlockLists& out)
{
    if (depth <= 0) {
        block_recursion(cl, eta, adm, t, s, out);
        return;
    }
    if (leaf_pair(cl, eta, adm, t, s, out)) return;
    int pr[4][2];
    const int np = split_pairs(cl[t], cl[s], t, s, pr);
    std::vector<BlockLists> part(np);
    run_all(np, true, [&](int k) { block_recursion_par(cl, eta, adm, pr[k][0], pr[k][1], depth - 1, part[k]); });
    for (int k = 0; k < np; ++k) {
        out.nearb.insert(out.nearb.end(), part[k].nearb.begin(), part[k].nearb.end());
        out.farb.insert(out.farb.end(), part[k].farb.begin(), part[k].farb.end());
    }
}

bool block_before(const FarBlock& a, const FarBlock& b)
{
    if (a.row0 != b.row0) return a.row0 < b.row0;
    return a.col0 < b.col0;
}

// Sort by (row0, col0) -- unique per block, so any correct sort gives the same
// order: `parts` chunks sorted concurrently, then merged pairwise.
void sort_blocks(std::vector<FarBlock>& v, int parts)
{
    const size_t n = v.size();
    if (parts < 2 || n < 4096) {
        std::sort(v.begin(), v.end(), block_before);
        return;
    }
    std::vector<size_t> cut(parts + 1);
    for (int k = 0; k <= parts; ++k) cut[k] = n * (size_t)k / (size_t)parts;
    run_all(parts, true, [&](int k) { std::sort(v.begin() + cut[k], v.begin() + cut[k + 1], block_before); });
    for (int w = 1; w < parts; w *= 2) {
        const int nm = (parts + 2 * w - 1) / (2 * w);
        run_all(nm, true, [&](int m) {
            const int a = 2 * m * w, b = std::min(a + w, parts), c = std::min(a + 2 * w, parts);
            if (b < c)
                std::inplace_merge(v.begin() + cut[a], v.begin() + cut[b], v.begin() + cut[c], block_before);
        });
    }
}

int plan_threads(int64_t n)
{
    if (n < kParMin) return 1;
    int t = (int)std::thread::hardware_concurrency();
    if (const char* e = std::getenv("RT_PLAN_THREADS")) {
        const int v = std::atoi(e);
        if (v >= 1) t = v;
    }
    return std::max(1, std::min(t, kMaxPlanThreads));
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
    const int threads = plan_threads(n);
    // split levels on separate threads: 2^levels >= threads (cluster tree),
    // 4^levels >= threads (block tree)
    int cl_levels = 0, bl_levels = 0;
    while (threads > 1 && (1 << cl_levels) < threads) ++cl_levels;
    while (threads > 1 && (1 << (2 * bl_levels)) < threads) ++bl_levels;
    Builder B;
    B.xyz = xyz;
    B.leaf = leaf;
    B.par_depth = cl_levels;
    B.idx.resize(n);
    std::iota(B.idx.begin(), B.idx.end(), 0);
    B.cl.resize((size_t)B.count((int)n));
    B.build(0, (int)n, 0, 0);
    out = Plan();
    out.N = (int)n;
    out.leaf = leaf;
    out.perm = B.idx;
    out.iperm.assign(n, 0);
    for (int64_t k = 0; k < n; ++k) out.iperm[out.perm[k]] = (int)k;
    out.clusters.reserve(B.cl.size());
    for (const Cluster& C : B.cl) out.clusters.push_back({C.start, C.size, C.left, C.right});
    // pre-order ids: the leaves come out in tree order
    for (const Cluster& C : B.cl)
        if (C.left < 0) {
            out.leaf_start.push_back(C.start);
            out.leaf_size.push_back(C.size);
        }
    BlockLists bl;
    block_recursion_par(B.cl, eta, adm, 0, 0, bl_levels, bl);
    out.near_blocks = std::move(bl.nearb);
    out.far_blocks = std::move(bl.farb);
    run_all(2, threads > 1, [&](int k) {
        if (k == 0) sort_blocks(out.far_blocks, std::max(1, threads - 1));
        else sort_blocks(out.near_blocks, 1);
    });
    return RT_OK;
}

}  // namespace rt
