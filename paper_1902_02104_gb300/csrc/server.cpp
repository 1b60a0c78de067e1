// server.cpp -- continuous-batching server for independent A^t A requests
// (ata_server_*, ata_submit, ata_poll).
//
// A host scheduler thread admits queued requests in arrival order whenever a
// stream slot is free, the device-memory budget can hold the request's plan,
// and the device has that much memory free (cudaMemGetInfo, plus a reserve).  Plans stay resident per shape (m, n, lda) and are reused; a second
// instance of a shape's plan is created when the first is busy (a plan runs
// one execution at a time); idle plans are evicted least recently used when
// the budget is needed.  Each admitted request runs its plan's graph on one of
// `max_inflight` non-blocking streams, so requests overlap on the device, and
// its completion is seen through a CUDA event.  Results do not depend on the
// mix: every request runs the same kernels on its own workspace.
//
// Executions are launched directly on the slot's stream, without a CUDA
// graph: capturing a graph on this thread would race with device-wide
// synchronisation that the application's other threads may issue at any
// time, which breaks the capture.  The application must still not free or
// overwrite a request's A or C before its ticket completes, and must have
// finished writing A before it submits it: the server's streams do not wait
// for the application's streams.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <string>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "runtime.h"

using namespace ata;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    ata_ticket id;
    int64_t m, n, lda;
    const void* A;
    double* C;
    Clock::time_point t_submit;
};

struct PlanEntry {
    ata_plan plan = nullptr;
    size_t bytes = 0;
    bool busy = false;
    Clock::time_point last_use;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    ata_ticket ticket = 0;
    PlanEntry* entry = nullptr;
    Clock::time_point t_submit;
};

enum TicketState : int { T_QUEUED = 0, T_RUNNING = 1, T_DONE = 2 };

struct TicketInfo {
    int state = T_QUEUED;
    ata_status result = ATA_OK;
    std::string msg;
};

}  // namespace

// Device memory kept free beyond a new plan's bytes when the server admits
// it (graph instantiation, tables, other users of the device).
constexpr size_t kFreeReserve = size_t(256) << 20;

struct ata_server_s {
    size_t budget = 0, used = 0;
    ata_dtype dtype = ATA_F32_BF16X3;
    int device = 0;
    std::vector<Slot> slots;
    std::map<std::tuple<int64_t, int64_t, int64_t>, std::list<std::unique_ptr<PlanEntry>>> plans;
    std::deque<Request> queue;
    std::unordered_map<ata_ticket, TicketInfo> tickets;
    std::vector<double> latencies_us;
    int64_t kernels = 0;  // kernel launches of the executions queued since the last reset
    ata_ticket next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    bool check_status = false;  // read each plan's self-check word after completion
    std::thread thread;

    // Finds an idle plan for the request's shape, creating one if the budget
    // allows (evicting idle plans of any shape, least recently used first).
    // Returns nullptr when nothing can be admitted now.  Caller holds mu.
    PlanEntry* acquire_plan(const Request& r, ata_status* err) {
        auto key = std::make_tuple(r.m, r.n, r.lda);
        auto& lst = plans[key];
        for (auto& e : lst)
            if (!e->busy) return e.get();
        // need a new instance: size it with the planner first (no allocation)
        ata_plan_info info;
        ata_status st = ata_plan_query(r.m, r.n, dtype, 0, &info);
        if (st != ATA_OK) {
            *err = st;
            return nullptr;
        }
        const size_t bytes = (size_t)info.workspace_bytes + (size_t)info.n_leaf_tiles * 16 +
                             (size_t)info.n_leaf_products * 512 +
                             (size_t)(info.n_sum_tasks + info.n_combine_tasks) * 128 + (1u << 20);
        if (bytes > budget) {
            *err = ATA_EBUSY;
            return nullptr;
        }
        // Free device memory as the driver reports it (other plans, other
        // users of the device): a new plan needs its bytes plus a reserve,
        // else it waits like a request over the budget.
        size_t dev_free = 0, dev_total = 0;
        const bool mem_ok = cudaMemGetInfo(&dev_free, &dev_total) != cudaSuccess ||
                            dev_free >= bytes + kFreeReserve;
        if (!mem_ok && (used == 0 || bytes + kFreeReserve > dev_total)) {
            *err = ATA_EBUSY;  // nothing of ours to evict, or it could never fit
            return nullptr;
        }
        if (used + bytes > budget || !mem_ok) {
            // Memory is reclaimed only while no request is in flight, so that a
            // plan is never freed while the device runs other work.
            for (const Slot& s : slots)
                if (s.busy) return nullptr;  // retry once running requests complete
            auto fits = [&]() {
                size_t f = 0, tt = 0;
                const bool dev_ok = cudaMemGetInfo(&f, &tt) != cudaSuccess || f >= bytes + kFreeReserve;
                return used + bytes <= budget && dev_ok;
            };
            while (!fits()) {
                // evict the least recently used plan (all are idle here)
                PlanEntry* victim = nullptr;
                std::list<std::unique_ptr<PlanEntry>>* vlist = nullptr;
                for (auto& kv : plans)
                    for (auto& e : kv.second)
                        if (!e->busy && (!victim || e->last_use < victim->last_use)) {
                            victim = e.get();
                            vlist = &kv.second;
                        }
                if (!victim) break;
                used -= victim->bytes;
                ata_plan_destroy(victim->plan);
                vlist->remove_if([&](const std::unique_ptr<PlanEntry>& e) { return e.get() == victim; });
            }
            if (!fits()) {
                *err = ATA_EBUSY;  // cannot fit even with every other plan evicted
                return nullptr;
            }
        }
        ata_plan p = nullptr;
        cudaSetDevice(device);
        st = ata_plan_create(&p, r.m, r.n, dtype, 0);
        if (st != ATA_OK) {
            *err = st;
            return nullptr;
        }
        std::unique_ptr<PlanEntry> e(new PlanEntry());
        e->plan = p;
        e->bytes = bytes;
        used += bytes;
        lst.push_back(std::move(e));
        return lst.back().get();
    }

    void complete(Slot& s, ata_status st, const std::string& msg = std::string()) {
        TicketInfo& ti = tickets[s.ticket];
        ti.state = T_DONE;
        ti.result = st;
        ti.msg = msg;
        const double us =
            std::chrono::duration<double, std::micro>(Clock::now() - s.t_submit).count();
        latencies_us.push_back(us);
        s.entry->busy = false;
        s.entry->last_use = Clock::now();
        s.busy = false;
        s.entry = nullptr;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            // 1. completions
            bool any_busy = false;
            for (Slot& s : slots) {
                if (!s.busy) continue;
                const cudaError_t q = cudaEventQuery(s.done);
                if (q == cudaSuccess) {
                    int code = 0;
                    if (check_status) ata_plan_device_status(s.entry->plan, &code);
                    if (code != 0)
                        complete(s, ATA_ECUDA, "kernel self-check code " + std::to_string(code));
                    else
                        complete(s, ATA_OK);
                } else if (q != cudaErrorNotReady) {
                    complete(s, ATA_ECUDA, std::string("device error: ") + cudaGetErrorString(q));
                } else {
                    any_busy = true;
                }
            }
            cv_done.notify_all();
            // 2. admissions, in arrival order
            while (!queue.empty()) {
                Slot* free_slot = nullptr;
                for (Slot& s : slots)
                    if (!s.busy) {
                        free_slot = &s;
                        break;
                    }
                if (!free_slot) break;
                Request r = queue.front();
                ata_status err = ATA_OK;
                PlanEntry* e = acquire_plan(r, &err);
                if (!e) {
                    if (err != ATA_OK) {  // cannot ever run: fail the request
                        queue.pop_front();
                        TicketInfo& ti = tickets[r.id];
                        ti.state = T_DONE;
                        ti.result = err;
                        ti.msg = g_last_error;
                        cv_done.notify_all();
                        continue;
                    }
                    break;  // wait for memory
                }
                queue.pop_front();
                e->busy = true;
                int nk = 0;
                ata_status st = execute_direct(e->plan, r.A, r.lda, r.C, free_slot->stream, &nk);
                std::string emsg = st == ATA_OK ? std::string() : g_last_error;
                kernels += nk;
                if (st == ATA_OK && cudaEventRecord(free_slot->done, free_slot->stream) != cudaSuccess) {
                    st = ATA_ECUDA;
                    emsg = "cudaEventRecord failed";
                }
                free_slot->busy = true;
                free_slot->ticket = r.id;
                free_slot->entry = e;
                free_slot->t_submit = r.t_submit;
                tickets[r.id].state = T_RUNNING;
                if (st != ATA_OK) complete(*free_slot, st, emsg);
                any_busy = true;
            }
            if (stop && queue.empty() && !any_busy) break;
            if (any_busy) {
                // work in flight: poll its events again shortly
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else if (queue.empty()) {
                cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            } else {
                cv_work.wait_for(lk, std::chrono::microseconds(200));
            }
        }
    }
};

extern "C" {

ata_status ata_server_create(ata_server* out, size_t budget, ata_dtype dtype, int max_inflight) {
    if (!out) return fail(ATA_EINVAL, "out is NULL");
    *out = nullptr;
    if (budget == 0) return fail(ATA_EINVAL, "budget must be > 0");
    if (max_inflight < 1 || max_inflight > 64) return fail(ATA_EINVAL, "max_inflight must be in [1, 64]");
    if ((int)dtype < ATA_F64 || (int)dtype > ATA_F64_OZAKI) return fail(ATA_EINVAL, "unknown dtype");
    std::unique_ptr<ata_server_s> s(new ata_server_s());
    s->budget = budget;
    s->dtype = dtype;
    if (cudaGetDevice(&s->device) != cudaSuccess) return fail(ATA_ECUDA, "cudaGetDevice failed");
    {
        const char* chk = getenv("ATA_CHECK_BOUNDS");
        s->check_status = chk && chk[0] == '1';
    }
    s->slots.resize(max_inflight);
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
            return fail(ATA_ECUDA, "stream/event creation failed");
    }
    ata_server_s* raw = s.get();
    s->thread = std::thread([raw] { raw->run(); });
    *out = s.release();
    return ATA_OK;
}

ata_status ata_submit(ata_server srv, int64_t m, int64_t n, const void* A, int64_t lda, double* C_packed,
                      ata_ticket* ticket) {
    if (!srv || !ticket) return fail(ATA_EINVAL, "NULL argument");
    if (m < 0 || n < 0 || lda < n || lda < 1) return fail(ATA_EINVAL, "bad sizes");
    if (m > 0 && n > 0 && !A) return fail(ATA_EINVAL, "A is NULL");
    if (n > 0 && !C_packed) return fail(ATA_EINVAL, "C_packed is NULL");
    Request r;
    r.m = m;
    r.n = n;
    r.lda = lda;
    r.A = A;
    r.C = C_packed;
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return fail(ATA_EINVAL, "server is stopping");
        r.id = srv->next_ticket++;
        srv->tickets[r.id] = TicketInfo();
        srv->queue.push_back(r);
    }
    srv->cv_work.notify_one();
    *ticket = r.id;
    return ATA_OK;
}

ata_status ata_poll(ata_server srv, ata_ticket ticket, int timeout_us) {
    if (!srv) return fail(ATA_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) return fail(ATA_EINVAL, "unknown ticket");
    if (it->second.state != T_DONE && timeout_us > 0) {
        srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] {
            auto jt = srv->tickets.find(ticket);
            return jt == srv->tickets.end() || jt->second.state == T_DONE;
        });
        it = srv->tickets.find(ticket);
        if (it == srv->tickets.end()) return fail(ATA_EINVAL, "unknown ticket");
    }
    if (it->second.state != T_DONE) return timeout_us > 0 ? ATA_ETIMEOUT : ATA_PENDING;
    const ata_status r = it->second.result;
    const std::string msg = it->second.msg;
    srv->tickets.erase(it);
    if (r != ATA_OK) return fail(r, "request failed: " + msg);
    return ATA_OK;
}

ata_status ata_server_stats(ata_server srv, double* p50_us, double* p99_us, int64_t* completed) {
    if (!srv || !p50_us || !p99_us || !completed) return fail(ATA_EINVAL, "NULL argument");
    std::vector<double> v;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        v = srv->latencies_us;
    }
    *completed = (int64_t)v.size();
    *p50_us = *p99_us = 0.0;
    if (v.empty()) return ATA_OK;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        const size_t i = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
        return v[i];
    };
    *p50_us = pct(0.50);
    *p99_us = pct(0.99);
    return ATA_OK;
}

ata_status ata_server_reset_stats(ata_server srv) {
    if (!srv) return fail(ATA_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->latencies_us.clear();
    srv->kernels = 0;
    return ATA_OK;
}

ata_status ata_server_kernels(ata_server srv, int64_t* kernels) {
    if (!srv || !kernels) return fail(ATA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *kernels = srv->kernels;
    return ATA_OK;
}

void ata_server_destroy(ata_server srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->thread.joinable()) srv->thread.join();
    for (Slot& s : srv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    for (auto& kv : srv->plans)
        for (auto& e : kv.second) ata_plan_destroy(e->plan);
    delete srv;
}

}  // extern "C"
