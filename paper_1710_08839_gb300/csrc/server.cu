// Serving runtime: several lanes of the batched solve engine, one per class
// of lattice size, each with its own CUDA stream, engine and host worker
// thread. A lane steps its own requests as fast as their size allows, so a
// request on a small lattice does not wait for the steps of large ones (in
// one lockstep engine every step of every request lasts as long as the step
// of the largest). Requests are submitted and polled from any thread; the
// worker of a lane is the only thread that touches its engine. The paper
// solves one system at a time; this is a serving design of this library.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "qxd_internal.cuh"
#include "solver.cuh"

namespace qxd {
namespace {

struct Req {
    long long id;
    qxd_lattice* op;
    void* x;
    const void* b;
    qxd_solver_params P;
};

struct Record {
    int lane = 0;
    bool done = false;
    qxd_solve_info info{};
};

struct Lane {
    long long max_sites = 0;  // lattices of fewer simulated sites (the last lane: any)
    size_t budget = 0;
    cudaStream_t st = nullptr;
    qxd_engine* eng = nullptr;
    std::thread worker;
    std::mutex mu;  // guards inbox
    std::condition_variable cv;
    std::deque<Req> inbox;
    std::vector<std::pair<long long, long long>> live;  // (request id, engine id); worker only
    std::atomic<long long> submitted{0}, completed{0}, steps{0};
    int err = QXD_OK;  // first engine failure of the lane; later requests fail with it
};

}  // namespace
}  // namespace qxd

struct qxd_server {
    std::vector<std::unique_ptr<qxd::Lane>> lanes;
    int device = 0;
    std::atomic<long long> next_id{1};
    std::atomic<bool> stop{false};
    std::mutex rec_mu;  // guards records
    std::map<long long, qxd::Record> records;

    void finish(long long id, int status, const qxd_solve_info* info) {
        std::lock_guard<std::mutex> lock(rec_mu);
        qxd::Record& r = records[id];
        if (info) r.info = *info;
        r.info.status = status;
        r.done = true;
    }

    // worker of lane L: take new requests into the engine, step it while it
    // has work, record finished requests; sleep while idle
    void run(qxd::Lane* L) {
        cudaSetDevice(device);
        for (;;) {
            std::deque<qxd::Req> fresh;
            {
                std::unique_lock<std::mutex> lock(L->mu);
                L->cv.wait(lock, [&] { return stop.load() || !L->inbox.empty() || !L->live.empty(); });
                fresh.swap(L->inbox);
                if (fresh.empty() && L->live.empty() && stop.load()) return;
            }
            for (qxd::Req& r : fresh) {
                long long eid = 0;
                const int rc = L->err ? L->err : qxd_engine_submit(L->eng, r.op, r.x, r.b, &r.P, &eid);
                if (rc) finish(r.id, rc, nullptr);
                else L->live.emplace_back(r.id, eid);
            }
            if (L->live.empty()) continue;
            int na = 0, np = 0, nd = 0;
            const int rc = qxd_engine_step(L->eng, &na, &np, &nd);
            ++L->steps;
            if (rc) {  // the engine could not complete the step: its requests fail
                L->err = rc;
                for (auto& lv : L->live) finish(lv.first, rc, nullptr);
                L->live.clear();
                continue;
            }
            if (nd == 0) continue;
            for (size_t i = 0; i < L->live.size();) {
                qxd_solve_info info{};
                int done = 0;
                qxd_engine_poll(L->eng, L->live[i].second, &info, &done);
                if (done) {
                    qxd_engine_forget(L->eng, L->live[i].second);
                    finish(L->live[i].first, info.status, &info);
                    ++L->completed;
                    L->live[i] = L->live.back();
                    L->live.pop_back();
                } else {
                    ++i;
                }
            }
        }
    }

    void shutdown() {
        stop = true;
        for (auto& L : lanes) {
            {
                std::lock_guard<std::mutex> lock(L->mu);
            }
            L->cv.notify_all();
        }
        for (auto& L : lanes)
            if (L->worker.joinable()) L->worker.join();
        for (auto& L : lanes) {
            if (L->eng) qxd_engine_destroy(L->eng);
            if (L->st) cudaStreamDestroy(L->st);
            L->eng = nullptr;
            L->st = nullptr;
        }
    }
};

using namespace qxd;

extern "C" {

int qxd_server_create(qxd_server** out, int nlanes, const long long* lane_sites, const size_t* lane_budget,
                      int max_active) {
    if (!out || nlanes < 1 || !lane_budget || (nlanes > 1 && !lane_sites) || max_active < 1)
        return fail(QXD_ERR_ARG, "qxd_server_create: NULL argument, nlanes < 1 or max_active < 1");
    for (int i = 0; i + 1 < nlanes; ++i)
        if (lane_sites[i] < 1 || (i > 0 && lane_sites[i] <= lane_sites[i - 1]))
            return fail(QXD_ERR_ARG, "qxd_server_create: lane_sites must be positive and increasing");
    std::unique_ptr<qxd_server> s(new (std::nothrow) qxd_server());
    if (!s) return fail(QXD_ERR_OOM, "qxd_server_create: host allocation failed");
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) return cuda_fail(e, "qxd_server_create: cudaGetDevice");
    // stream priorities: the lane of the smallest lattices on the highest, so
    // that the thread blocks of short requests are scheduled as soon as blocks
    // of the large lattices' kernels retire, instead of after those kernels
    int least = 0, greatest = 0;
    if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess)
        return cuda_fail(e, "qxd_server_create: cudaDeviceGetStreamPriorityRange");
    for (int i = 0; i < nlanes; ++i) {
        std::unique_ptr<Lane> L(new (std::nothrow) Lane());
        if (!L) {
            s->shutdown();
            return fail(QXD_ERR_OOM, "qxd_server_create: host allocation failed");
        }
        L->max_sites = i + 1 < nlanes ? lane_sites[i] : -1;
        L->budget = lane_budget[i];
        const int prio = std::max(greatest, least - (nlanes - 1 - i));  // greatest is numerically lowest
        if ((e = cudaStreamCreateWithPriority(&L->st, cudaStreamNonBlocking, prio)) != cudaSuccess) {
            s->shutdown();
            return cuda_fail(e, "qxd_server_create: cudaStreamCreate");
        }
        int rc = qxd_engine_create(&L->eng, L->budget, max_active, L->st);
        if (rc) {
            cudaStreamDestroy(L->st);
            s->shutdown();
            return rc;
        }
        s->lanes.push_back(std::move(L));
    }
    for (auto& L : s->lanes) {
        Lane* lp = L.get();
        qxd_server* sp = s.get();
        L->worker = std::thread([sp, lp] { sp->run(lp); });
    }
    *out = s.release();
    return QXD_OK;
}

int qxd_server_destroy(qxd_server* s) {
    if (!s) return QXD_OK;
    s->shutdown();
    delete s;
    return QXD_OK;
}

int qxd_server_submit(qxd_server* s, qxd_lattice* op, void* x, const void* b, const qxd_solver_params* p,
                      long long* id) {
    if (!s || !id) return fail(QXD_ERR_ARG, "qxd_server_submit: NULL argument");
    int rc = engine_check_request(op, x, b, p, "qxd_server_submit");
    if (rc) return rc;
    if (s->stop.load()) return fail(QXD_ERR_STATE, "qxd_server_submit: the server is shutting down");
    int lane = 0;
    while (lane + 1 < (int)s->lanes.size() && (long long)op->g.V >= s->lanes[lane]->max_sites) ++lane;
    const long long rid = s->next_id++;
    {
        std::lock_guard<std::mutex> lock(s->rec_mu);
        Record& r = s->records[rid];
        r.lane = lane;
        r.info.status = QXD_ERR_STATE;  // pending
    }
    Lane* L = s->lanes[lane].get();
    {
        std::lock_guard<std::mutex> lock(L->mu);
        L->inbox.push_back(Req{rid, op, x, b, *p});
    }
    ++L->submitted;
    L->cv.notify_one();
    *id = rid;
    return QXD_OK;
}

int qxd_server_poll(qxd_server* s, long long id, qxd_solve_info* info, int* done) {
    if (!s) return fail(QXD_ERR_ARG, "qxd_server_poll: NULL server");
    std::lock_guard<std::mutex> lock(s->rec_mu);
    auto it = s->records.find(id);
    if (it == s->records.end()) return fail(QXD_ERR_ARG, "qxd_server_poll: unknown request id");
    if (info) *info = it->second.info;
    if (done) *done = it->second.done ? 1 : 0;
    return QXD_OK;
}

int qxd_server_forget(qxd_server* s, long long id) {
    if (!s) return fail(QXD_ERR_ARG, "qxd_server_forget: NULL server");
    std::lock_guard<std::mutex> lock(s->rec_mu);
    auto it = s->records.find(id);
    if (it == s->records.end()) return fail(QXD_ERR_ARG, "qxd_server_forget: unknown request id");
    if (!it->second.done) return fail(QXD_ERR_STATE, "qxd_server_forget: request not finished");
    s->records.erase(it);
    return QXD_OK;
}

int qxd_server_stats(const qxd_server* s, int lane, long long* submitted, long long* completed, long long* steps) {
    if (!s || lane < 0 || lane >= (int)s->lanes.size()) return fail(QXD_ERR_ARG, "qxd_server_stats: bad server or lane");
    const Lane& L = *s->lanes[lane];
    if (submitted) *submitted = L.submitted.load();
    if (completed) *completed = L.completed.load();
    if (steps) *steps = L.steps.load();
    return QXD_OK;
}

}  // extern "C"
