// Continuous-batching solve server: requests of different size arrive at any
// time; each is admitted as soon as a worker slot, its device-memory need and
// its share of resident CTAs are free, then runs the paper's pipeline (ALNS
// first, BRKGA warm-started from the ALNS incumbent, Section 4) on its own
// non-blocking stream, so the work of all admitted requests overlaps on the
// device.  Every random draw is counter-based and every kernel is
// deterministic, so a request's answer does not depend on what else runs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <string>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace vrp {
size_t alns_device_bytes(int n, int m, int qmax, const vrprpd_alns_params* P, int iterations);
int alns_blocks_per_sm(int n, int m);
}  // namespace vrp

struct vrprpd_server {
    struct Req {
        int64_t id = 0;
        vrprpd_request r{};
        std::vector<int32_t> coords, p;
        size_t need = 0;
        int ctas = 0;
        double sm_share = 0;   // SMs' worth of resident ALNS CTAs this request holds: ctas / (CTAs per SM at its n)
        double t_submit = 0, t_start = 0, t_end = 0;
        int done = 0;
        int rc = VRPRPD_OK;
        int32_t z_alns = 0, z_brkga = 0, z_best = 0;
        int64_t brkga_fitness = 0;
        std::vector<int32_t> best_ops, best_off;
        double device_ms = 0;
        std::string message;
    };
    int device = 0;
    size_t budget = 0, in_use = 0, peak_use = 0;
    int max_active = 1, active = 0, peak_active = 0;
    int sms = 0;
    double sm_in_use = 0;      // sum of the running requests' sm_share, at most sms
    int64_t next_id = 1;
    bool stopping = false;
    std::deque<int64_t> pending;
    std::map<int64_t, Req> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    std::chrono::steady_clock::time_point t0;
    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace vrp {

static size_t request_bytes(const vrprpd_request& r) {
    const size_t N1 = static_cast<size_t>(r.n) + 1;
    const size_t inst = N1 * N1 * 6 + N1 * 12 + 4096;
    int qmax = std::max(4, static_cast<int>(static_cast<long long>(r.n) * 5 / 100));
    if (r.alns.q_max > 0) qmax = r.alns.q_max;
    qmax = std::min(qmax, r.n);
    const size_t alns = r.alns.iterations > 0 ? alns_device_bytes(r.n, r.m, qmax, &r.alns, r.alns.iterations) : 0;
    const size_t L = r.brkga.layout == VRPRPD_LAYOUT_HINTS ? 4ull * r.n : 2ull * r.n + r.m;
    const size_t pop = static_cast<size_t>(std::max(r.brkga.pop, 0));
    const size_t brkga = r.brkga.generations > 0
                             ? pop * L * 8 + pop * (2ull * r.n + r.m + 1) * 4 + pop * 48 + L * 4 +
                                   static_cast<size_t>(r.brkga.generations) * 8 + 8192
                             : 0;
    return inst + alns + brkga;
}

static void serve_one(vrprpd_server* S, vrprpd_server::Req& q, cudaStream_t stream) {
    const vrprpd_request& r = q.r;
    vrprpd_instance* I = nullptr;
    int rc = vrprpd_instance_create(q.coords.data(), q.p.data(), r.n, r.m, r.R, r.Q, r.flags, &I);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, stream);
    std::vector<int32_t> ops(2 * r.n), off(r.m + 1), bops(2 * r.n), boff(r.m + 1);
    vrprpd_solution init{ops.data(), off.data(), 0, 0};
    // the start: the paper's three-phase constructor and its refinement on this
    // request's share of the CTAs, or the plain sweep
    if (rc == VRPRPD_OK)
        rc = r.alns.init_mode == 1 ? initial_solution_paper_tb(I, r.alns.init_refine_rounds, &init, stream, q.ctas)
                                   : vrprpd_initial_solution(I, &init);
    int32_t z_alns = 0;
    if (rc == VRPRPD_OK) {
        vrprpd_alns_params P = r.alns;
        P.team_blocks = q.ctas;
        vrprpd_solution best{bops.data(), boff.data(), 0, 0};
        rc = vrprpd_alns_run(I, &init, &P, r.seed, &best, nullptr, nullptr, nullptr, stream);
        if (rc == VRPRPD_OK) {
            ops = bops;
            off = boff;
            z_alns = best.makespan;
        }
    }
    int32_t z_brkga = 0;
    int64_t fit = 0;
    std::vector<int32_t> gops(2 * r.n), goff(r.m + 1);
    if (rc == VRPRPD_OK && r.brkga.generations > 0) {
        vrprpd_solution warm{ops.data(), off.data(), 0, 0};
        vrprpd_solution best{gops.data(), goff.data(), 0, 0};
        rc = vrprpd_brkga_run(I, &r.brkga, &warm, r.seed, &best, &fit, nullptr, nullptr, stream);
        z_brkga = best.makespan;
    }
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (I) vrprpd_instance_destroy(I);
    const std::string msg = rc ? std::string(vrprpd_last_error()) : std::string();
    std::lock_guard<std::mutex> lock(S->mu);
    q.rc = rc;
    q.message = msg;
    q.z_alns = z_alns;
    q.z_brkga = z_brkga;
    q.brkga_fitness = fit;
    // the pipeline's answer: the better of the ALNS incumbent and the BRKGA best
    const bool brkga_better = r.brkga.generations > 0 && fit < 1000000 && z_brkga < z_alns;
    q.z_best = brkga_better ? z_brkga : z_alns;
    q.best_ops = brkga_better ? gops : ops;
    q.best_off = brkga_better ? goff : off;
    q.device_ms = ms;
}

static void worker_main(vrprpd_server* S) {
    cudaSetDevice(S->device);
    cudaStream_t stream;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    for (;;) {
        int64_t id = 0;
        vrprpd_server::Req* qp = nullptr;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            // FIFO admission: the head request starts once memory and CTAs allow
            S->cv_work.wait(lock, [&] {
                if (S->stopping && S->pending.empty()) return true;
                if (S->pending.empty()) return false;
                const auto& q = S->reqs[S->pending.front()];
                return S->in_use + q.need <= S->budget && S->sm_in_use + q.sm_share <= S->sms + 1e-9;
            });
            if (S->pending.empty()) break;
            id = S->pending.front();
            S->pending.pop_front();
            qp = &S->reqs.at(id);
            auto& q = *qp;
            S->in_use += q.need;
            S->sm_in_use += q.sm_share;
            S->active += 1;
            S->peak_active = std::max(S->peak_active, S->active);
            S->peak_use = std::max(S->peak_use, S->in_use);
            q.t_start = S->now_ms();
        }
        S->cv_work.notify_all();
        auto& q = *qp;               // map nodes stay put while others are inserted
        serve_one(S, q, stream);
        {
            std::lock_guard<std::mutex> lock(S->mu);
            q.t_end = S->now_ms();
            q.done = 1;
            S->in_use -= q.need;
            S->sm_in_use -= q.sm_share;
            S->active -= 1;
        }
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    cudaStreamDestroy(stream);
}

}  // namespace vrp

using namespace vrp;

extern "C" int vrprpd_server_create(size_t mem_budget, int32_t max_active, vrprpd_server** out) {
    VRP_CHECK(out && mem_budget > 0 && max_active >= 1 && max_active <= 256, VRPRPD_EINVAL, "bad server arguments");
    vrprpd_server* S = new vrprpd_server();
    VRP_CUDA(cudaGetDevice(&S->device));
    int sms = 0;
    VRP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device));
    S->sms = sms;
    S->budget = mem_budget;
    S->max_active = max_active;
    S->t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < max_active; ++i) S->workers.emplace_back(worker_main, S);
    *out = S;
    return VRPRPD_OK;
}

extern "C" int vrprpd_server_submit(vrprpd_server* S, const vrprpd_request* r, int64_t* id) {
    VRP_CHECK(S && r && id && r->coords && r->p, VRPRPD_EINVAL, "NULL argument");
    VRP_CHECK(r->n >= 1 && r->m >= 1 && r->m <= 32 && 2 * r->n + r->m <= 4096, VRPRPD_EINVAL,
              "request sizes outside the searches' limits (n=%d m=%d)", r->n, r->m);
    VRP_CHECK(r->alns.iterations >= 1 && r->brkga.generations >= 0, VRPRPD_EINVAL,
              "a request runs at least one ALNS iteration");
    vrprpd_server::Req q;
    q.r = *r;
    q.coords.assign(r->coords, r->coords + 2 * (r->n + 1));
    q.p.assign(r->p, r->p + r->n);
    q.r.coords = nullptr;
    q.r.p = nullptr;
    q.need = request_bytes(*r);
    // ALNS team size: what the instance would take alone, capped by a fair
    // share of the GPU's resident ALNS CTAs at this n (every CTA of a team is
    // resident at once: a cooperative launch)
    const long long G = 2ll * r->n + r->m;
    const long long tiles = ((G + 31) / 32) * ((G + 63) / 64);
    const int occ = alns_blocks_per_sm(r->n, r->m);
    VRP_CHECK(occ >= 1, VRPRPD_EINVAL, "an ALNS block of n=%d does not fit on an SM", r->n);
    const int share = std::max(1, occ * S->sms / S->max_active);
    q.ctas = (G < 64) ? 1 : static_cast<int>(std::max<long long>(1, std::min<long long>(tiles, share)));
    q.sm_share = static_cast<double>(q.ctas) / occ;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stopping) { set_error("server is shutting down"); return VRPRPD_EBUSY; }
        if (q.need > S->budget) {
            set_error("request needs %zu bytes of device memory; the server budget is %zu", q.need, S->budget);
            return VRPRPD_EBUSY;
        }
        q.id = S->next_id++;
        q.t_submit = S->now_ms();
        *id = q.id;
        S->reqs[q.id] = std::move(q);
        S->pending.push_back(*id);
    }
    S->cv_work.notify_all();
    return VRPRPD_OK;
}

static int fill_result(vrprpd_server::Req& q, vrprpd_result* out, int32_t* ops, int32_t* off) {
    out->id = q.id;
    out->status = q.rc;
    out->z_alns = q.z_alns;
    out->z_brkga = q.z_brkga;
    out->z_best = q.z_best;
    out->t_submit_ms = q.t_submit;
    out->t_start_ms = q.t_start;
    out->t_end_ms = q.t_end;
    out->device_ms = q.device_ms;
    out->n = q.r.n;
    out->m = q.r.m;
    std::snprintf(out->message, sizeof(out->message), "%s", q.message.c_str());
    if (q.rc == VRPRPD_OK) {
        if (ops) std::copy(q.best_ops.begin(), q.best_ops.end(), ops);
        if (off) std::copy(q.best_off.begin(), q.best_off.end(), off);
    }
    return VRPRPD_OK;
}

extern "C" int vrprpd_server_poll(vrprpd_server* S, int64_t id, vrprpd_result* out, int32_t* ops, int32_t* off) {
    VRP_CHECK(S && out, VRPRPD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(id);
    VRP_CHECK(it != S->reqs.end(), VRPRPD_EINVAL, "unknown request %lld", static_cast<long long>(id));
    if (!it->second.done) return VRPRPD_ENOTREADY;
    return fill_result(it->second, out, ops, off);
}

extern "C" int vrprpd_server_wait(vrprpd_server* S, int64_t id, vrprpd_result* out, int32_t* ops, int32_t* off) {
    VRP_CHECK(S && out, VRPRPD_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->reqs.find(id);
    VRP_CHECK(it != S->reqs.end(), VRPRPD_EINVAL, "unknown request %lld", static_cast<long long>(id));
    S->cv_done.wait(lock, [&] { return it->second.done != 0; });
    return fill_result(it->second, out, ops, off);
}

extern "C" int vrprpd_server_get_stats(vrprpd_server* S, vrprpd_server_stats* out) {
    VRP_CHECK(S && out, VRPRPD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    int done = 0;
    std::vector<double> lat;
    for (auto& kv : S->reqs)
        if (kv.second.done == 1) {
            ++done;
            lat.push_back(kv.second.t_end - kv.second.t_submit);
        }
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
        if (lat.empty()) return 0.0;
        size_t k = static_cast<size_t>(std::ceil(q * lat.size())) - 1;
        return lat[std::min(k, lat.size() - 1)];
    };
    out->submitted = static_cast<int32_t>(S->reqs.size());
    out->completed = done;
    out->pending = static_cast<int32_t>(S->pending.size());
    out->active = S->active;
    out->peak_active = S->peak_active;
    out->bytes_in_use = S->in_use;
    out->peak_bytes = S->peak_use;
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    return VRPRPD_OK;
}

extern "C" int vrprpd_server_cancel_pending(vrprpd_server* S, int32_t* withdrawn) {
    VRP_CHECK(S, VRPRPD_EINVAL, "NULL server");
    int32_t k = 0;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        const double t = S->now_ms();
        for (const int64_t id : S->pending) {
            auto& q = S->reqs.at(id);
            q.rc = VRPRPD_EBUSY;
            q.message = "withdrawn before admission";
            q.t_start = q.t_end = t;
            q.done = 2;                        // finished without running: no latency sample
            ++k;
        }
        S->pending.clear();
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    if (withdrawn) *withdrawn = k;
    return VRPRPD_OK;
}

extern "C" void vrprpd_server_destroy(vrprpd_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
}
