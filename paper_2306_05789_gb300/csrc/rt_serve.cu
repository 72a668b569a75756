// rt_serve.cu -- continuous admission of independent solve requests (the
// rt_server_* / rt_submit / rt_poll part of include/rt.h).
//
// Each request is one problem of Section 2 solved by the fixed point of
// Section 1.3.  A fixed set of worker slots, each owning a CUDA stream, takes
// requests from a queue as soon as a slot is free and the request's estimated
// device footprint fits into what the HBM budget has left.  The operator and
// the iterates of a request stay on the device until its result has been
// copied out; then everything of it is freed in stream order and the budget
// it held is returned, which may admit the next request.  Builds and solves of
// different slots run concurrently on the device: the host waits in the
// assembly (one per ACA sweep) and in the fixed point (one per convergence
// check) block only their own slot.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rt_internal.h"

namespace rt {

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2 };

// A request owns deep copies of every host array of its problem.
struct Request {
    int64_t id = 0;
    rt_problem prob{};
    std::vector<double> xyz;
    std::vector<int32_t> tet, emit;
    std::vector<rt_wall> walls;
    std::vector<float> kgrid;
    std::vector<rt_box> obstacles;
    std::vector<double> nu, w, c, albedo;
    std::vector<int32_t> group;
    Plan plan;
    int64_t est_peak = 0, est_resident = 0;
    int64_t held = 0;            // budget this request holds now
    int bypassed = 0;            // times a later request was admitted first
    int state = REQ_QUEUED;
    int status = RT_OK;
    std::string msg;
    std::vector<float> J;
    std::vector<double> T;
    rt_request_info info{};
};

}  // namespace

// Estimated device footprint of one request: the peak during assembly and the
// size while the fixed point runs.  Exact for the near field and the vectors;
// the far field assumes every admissible block reaches rank r_hat, a little
// above the mean rank that ACA reaches at the given tolerance (about 19 at
// 1e-4 on the cube workloads).  The ACA term scratch lives one wave at a time
// (at most hp.wave_bytes of 24-term pools, grown by half once at worst) and
// is gone before the near field is allocated.
struct Footprint {
    int64_t peak = 0, resident = 0;
};

static Footprint estimate_footprint(const Plan& P, int64_t N, int64_t T, int F, int G, const rt_hparams& hp)
{
    const double r_hat = std::max(8.0, 6.0 * std::log10(1.0 / hp.aca_eps));
    const int esz = hp.far_prec == RT_PREC_F32 ? 4 : (hp.refine ? 4 : 2);
    std::vector<Chunk> tmp;
    int64_t near = 0, far_elems = 0, pool = 0, bufs = 0;
    for (const FarBlock& b : P.near_blocks) {
        tmp.clear();
        near += block_chunks(P, b.row0, b.m, (int64_t)G * b.n, tmp);
    }
    for (const FarBlock& b : P.far_blocks) {
        tmp.clear();
        const int64_t mpad = block_chunks(P, b.row0, b.m, 1, tmp);
        far_elems += (int64_t)std::ceil(G * r_hat) * ((int64_t)round8(b.n) + mpad);
        pool += (int64_t)G * 24 * (b.m + b.n);
        bufs += (int64_t)G * (b.m + b.n);
    }
    const int64_t wave = hp.wave_bytes > 0 ? hp.wave_bytes : ((int64_t)8 << 30);
    const int64_t aca = (int64_t)(1.5 * (double)std::min<int64_t>(4 * pool, wave)) +
                        std::min<int64_t>(4 * bufs, wave / 24 + ((int64_t)64 << 20));
    const int64_t geo = N * 64 + T * 120 + (int64_t)F * N * 4;
    const int64_t vec = (int64_t)F * N * 4 * 6 + N * 16 + (int64_t)F * (int64_t)P.far_blocks.size() * (int64_t)r_hat * 4;
    Footprint f;
    f.resident = geo + 4 * near + (int64_t)esz * far_elems + vec;
    f.peak = geo + (int64_t)esz * far_elems + std::max<int64_t>(aca, 4 * near + vec);
    return f;
}

struct Server {
    rt_server_opts o{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work;   // workers: a request may have become admissible
    std::condition_variable cv_done;   // pollers: a request finished
    std::deque<Request*> queue;
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
    rt_server_info_t stats{};

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    // first-come-first-served with bounded overtaking; called with mu held
    Request* pick()
    {
        const int64_t left = o.hbm_budget - stats.reserved_bytes;
        for (size_t k = 0; k < queue.size(); ++k) {
            Request* r = queue[k];
            if (r->est_peak <= left) {
                for (size_t j = 0; j < k; ++j)
                    if (queue[j]->bypassed >= o.max_bypass) return nullptr;   // nobody may pass it again
                for (size_t j = 0; j < k; ++j) queue[j]->bypassed++;
                queue.erase(queue.begin() + (std::ptrdiff_t)k);
                return r;
            }
        }
        return nullptr;
    }

    void run_one(Request* r, cudaStream_t st);
    void worker();
};

void Server::run_one(Request* r, cudaStream_t st)
{
    std::string err;
    Operator op;
    float* dJ = nullptr;
    double* dT = nullptr;
    int rc = RT_OK;
    const auto tb = Clock::now();
    rc = build_operator(op, &r->prob, &o.hp, st, err, &r->plan);
    const double ms_build = std::chrono::duration<double, std::milli>(Clock::now() - tb).count();
    const int64_t N = r->prob.mesh.n_vert, F = r->prob.freqs.F;
    if (rc == RT_OK) {
        // the assembly peak is over: hold only what stays resident
        const int64_t resident = op.info.device_bytes + F * N * 4 * 3 + N * 16;
        std::lock_guard<std::mutex> lk(mu);
        stats.reserved_bytes += resident - r->held;
        r->held = resident;
        r->info.t_built = now();
        r->info.resident_bytes = resident;
        r->info.peak_bytes = op.info.peak_bytes;
        cv_work.notify_all();
    }
    rt_solve_stats ss{};
    if (rc == RT_OK) {
        if (cudaMallocAsync((void**)&dJ, sizeof(float) * F * N, st) != cudaSuccess ||
            cudaMallocAsync((void**)&dT, sizeof(double) * N, st) != cudaSuccess) {
            rc = RT_ENOMEM;
            err = "cudaMallocAsync (request iterates) failed";
        }
    }
    if (rc == RT_OK) rc = solve_fixed_point(op, o.opts, dJ, dT, ss, st, err);
    if (rc == RT_OK || rc == RT_ENOCONV) {
        r->J.resize((size_t)F * N);
        r->T.resize((size_t)N);
        // device -> pageable host copies return once the data has arrived
        if (cudaMemcpyAsync(r->J.data(), dJ, sizeof(float) * F * N, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(r->T.data(), dT, sizeof(double) * N, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            rc = RT_ECUDA;
            err = "copy of the result to the host failed";
        }
    }
    if (dJ) cudaFreeAsync(dJ, st);
    if (dT) cudaFreeAsync(dT, st);
    operator_release(op, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == RT_OK) {
        rc = RT_ECUDA;
        err = "device error in the request's stream";
    }
    r->status = rc;
    r->msg = err;
    r->info.status = rc;
    r->info.iters = ss.iters;
    r->info.converged = ss.converged;
    r->info.residual = ss.residual;
    r->info.ms_build = ms_build;
    r->info.ms_solve = ss.ms_total;
}

void Server::worker()
{
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || (r = pick()) != nullptr; });
            if (!r) break;   // stopping with nothing admissible for this slot
            r->state = REQ_RUNNING;
            r->held = r->est_peak;
            stats.reserved_bytes += r->held;
            stats.peak_reserved_bytes = std::max(stats.peak_reserved_bytes, stats.reserved_bytes);
            stats.queued--;
            stats.running++;
            stats.max_running = std::max(stats.max_running, stats.running);
            r->info.t_admit = now();
        }
        run_one(r, st);
        {
            std::lock_guard<std::mutex> lk(mu);
            stats.reserved_bytes -= r->held;
            r->held = 0;
            stats.running--;
            stats.finished++;
            if (r->status != RT_OK) stats.failed++;
            r->info.t_done = now();
            r->state = REQ_DONE;
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
    cudaStreamDestroy(st);
}

}  // namespace rt

struct rt_server {
    rt::Server s;
};

using rt::Request;

extern "C" {

int rt_server_create(const rt_server_opts* opts, rt_server** out)
{
    if (!opts || !out) {
        rt::set_last_error("null argument");
        return RT_EINVAL;
    }
    *out = nullptr;
    if (!(opts->hbm_budget > 0) || opts->slots < 1 || opts->slots > 64 || opts->max_bypass < 0) {
        rt::set_last_error("server options: need hbm_budget > 0, 1 <= slots <= 64, max_bypass >= 0");
        return RT_EINVAL;
    }
    if (opts->hp.mode != RT_MODE_HMATRIX) {
        rt::set_last_error("the server assembles H-matrix operators (hp.mode = RT_MODE_HMATRIX)");
        return RT_EINVAL;
    }
    if (opts->opts.max_iter < 1 || opts->opts.check_every < 1 || !(opts->opts.tol >= 0.0) || !(opts->opts.T0 >= 0.0)) {
        rt::set_last_error("invalid solve options");
        return RT_EINVAL;
    }
    rt_server* h = new (std::nothrow) rt_server();
    if (!h) {
        rt::set_last_error("host allocation failed");
        return RT_ENOMEM;
    }
    rt::Server& S = h->s;
    S.o = *opts;
    S.o.opts.use_J0 = 0;
    S.t0 = rt::Clock::now();
    cudaGetDevice(&S.device);
    for (int k = 0; k < opts->slots; ++k) S.workers.emplace_back([&S] { S.worker(); });
    *out = h;
    return RT_OK;
}

int rt_submit(rt_server* h, const rt_problem* P, int64_t* id)
{
    if (!h || !P || !id) {
        rt::set_last_error("null argument");
        return RT_EINVAL;
    }
    rt::Server& S = h->s;
    const double t_sub = S.now();
    std::string err;
    int rc = rt::validate_problem(P, &S.o.hp, err);
    if (rc) {
        rt::set_last_error(err);
        return rc;
    }
    auto r = std::make_unique<Request>();
    try {
        const int64_t N = P->mesh.n_vert, T = P->mesh.n_tet, F = P->freqs.F;
        r->xyz.assign(P->mesh.xyz, P->mesh.xyz + 3 * N);
        r->tet.assign(P->mesh.tet, P->mesh.tet + 4 * T);
        if (P->n_emit > 0) r->emit.assign(P->emit_tri, P->emit_tri + 3 * P->n_emit);
        if (P->n_walls > 0) r->walls.assign(P->walls, P->walls + P->n_walls);
        if (P->kappa.kind == RT_KAPPA_GRID)
            r->kgrid.assign(P->kappa.grid, P->kappa.grid + (int64_t)P->kappa.dims[0] * P->kappa.dims[1] * P->kappa.dims[2]);
        if (P->n_obstacles > 0) r->obstacles.assign(P->obstacles, P->obstacles + P->n_obstacles);
        r->nu.assign(P->freqs.nu, P->freqs.nu + F);
        r->w.assign(P->freqs.w, P->freqs.w + F);
        r->c.assign(P->freqs.c, P->freqs.c + F);
        r->albedo.assign(P->freqs.albedo, P->freqs.albedo + F);
        if (P->freqs.group) r->group.assign(P->freqs.group, P->freqs.group + F);
        r->prob = *P;
        r->prob.mesh.xyz = r->xyz.data();
        r->prob.mesh.tet = r->tet.data();
        r->prob.emit_tri = r->emit.empty() ? nullptr : r->emit.data();
        r->prob.walls = r->walls.empty() ? nullptr : r->walls.data();
        r->prob.kappa.grid = r->kgrid.empty() ? nullptr : r->kgrid.data();
        r->prob.obstacles = r->obstacles.empty() ? nullptr : r->obstacles.data();
        r->prob.freqs.nu = r->nu.data();
        r->prob.freqs.w = r->w.data();
        r->prob.freqs.c = r->c.data();
        r->prob.freqs.albedo = r->albedo.data();
        r->prob.freqs.group = r->group.empty() ? nullptr : r->group.data();   // the estimate below
        // counts distinct c, an upper bound on the groups of a binned grid
        rc = rt::plan_build(r->xyz.data(), N, S.o.hp.leaf, S.o.hp.eta, S.o.hp.adm, r->plan, err);
        if (rc) {
            rt::set_last_error(err);
            return rc;
        }
        std::vector<double> cs;
        for (int64_t f = 0; f < F; ++f)
            if (std::find(cs.begin(), cs.end(), r->c[f]) == cs.end()) cs.push_back(r->c[f]);
        const rt::Footprint fp = rt::estimate_footprint(r->plan, N, T, (int)F, (int)cs.size(), S.o.hp);
        r->est_peak = fp.peak;
        r->est_resident = fp.resident;
        r->info.N = N;
        r->info.F = F;
        r->info.est_bytes = fp.peak;
        r->info.t_submit = t_sub;
    } catch (const std::bad_alloc&) {
        rt::set_last_error("host allocation failed");
        return RT_ENOMEM;
    }
    if (r->est_peak > S.o.hbm_budget) {
        rt::set_last_error("request needs an estimated " + std::to_string(r->est_peak) + " bytes, more than the budget of " +
                           std::to_string(S.o.hbm_budget));
        return RT_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(S.mu);
        r->id = S.next_id++;
        *id = r->id;
        S.queue.push_back(r.get());
        S.reqs.emplace(r->id, std::move(r));
        S.stats.submitted++;
        S.stats.queued++;
    }
    S.cv_work.notify_all();
    return RT_OK;
}

int rt_poll(rt_server* h, int64_t id, int wait_ms, float* J_host, double* T_host, rt_request_info* info)
{
    if (!h) {
        rt::set_last_error("null argument");
        return RT_EINVAL;
    }
    rt::Server& S = h->s;
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.reqs.find(id);
    if (it == S.reqs.end()) {
        rt::set_last_error("unknown or retired request id");
        return RT_EINVAL;
    }
    Request* r = it->second.get();
    auto done = [&] { return r->state == rt::REQ_DONE; };
    if (wait_ms < 0) S.cv_done.wait(lk, done);
    else S.cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), done);
    if (!done()) return RT_EAGAIN;
    if (J_host && !r->J.empty()) std::copy(r->J.begin(), r->J.end(), J_host);
    if (T_host && !r->T.empty()) std::copy(r->T.begin(), r->T.end(), T_host);
    if (info) *info = r->info;
    const int st = r->status;
    if (st != RT_OK) rt::set_last_error(r->msg);
    S.reqs.erase(it);
    return st;
}

int rt_server_info(rt_server* h, rt_server_info_t* info)
{
    if (!h || !info) {
        rt::set_last_error("null argument");
        return RT_EINVAL;
    }
    std::lock_guard<std::mutex> lk(h->s.mu);
    *info = h->s.stats;
    return RT_OK;
}

void rt_server_free(rt_server* h)
{
    if (!h) return;
    rt::Server& S = h->s;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop = true;
        S.stats.queued -= (int64_t)S.queue.size();
        S.queue.clear();
    }
    S.cv_work.notify_all();
    for (auto& t : S.workers) t.join();
    delete h;
}

}  // extern "C"
