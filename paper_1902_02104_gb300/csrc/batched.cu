// batched.cu -- many independent products in one queued batch.  The task
// tables of all instances are merged level by level, so the whole batch is
// one split launch per level, one persistent leaf launch whose tiles (all
// instances) run heaviest first, and one combine launch per level, captured
// once as a CUDA graph.  The kernels read the instances' bindings from a
// device array, so a batch has no limit on its instance count.
//
// Two entry points share this machinery: ata_execute_batched takes pointer
// arrays on every call (tables found by the set of plans), and a prepared
// ata_batch binds its plans once to one packed input buffer and one packed
// output buffer, so that a call passes two base pointers and costs the host
// a few microseconds.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <vector>

#include "runtime.h"

namespace ata {
namespace {

struct BatchEntry {
    DeviceTables tables;
    GraphCache graph;
    std::vector<uint64_t> ids;
    std::shared_ptr<OrderEvent> order_ev;  // recorded after each launch
    ~BatchEntry() {
        graph.release();
        tables.free_all();
    }
};

std::mutex g_batch_mu;

// Batched executions launch the batch's graph and may upload bindings from a
// host staging buffer: neither can be recorded into a caller's capture.
constexpr const char* kBatchCaptureRefused =
    "the stream is capturing: batched executions cannot be recorded; capture ata_execute per plan instead";
std::map<std::vector<int64_t>, std::unique_ptr<BatchEntry>> g_batches;

// Checks the plans and leading dimensions of a batch; fills the cache key
// (plan id, lda per instance) and the dtype family.
ata_status check_batch(const ata_plan* plans, int count, const int64_t* lda, LeafKind* leaf,
                       std::vector<int64_t>* key) {
    key->clear();
    std::vector<uint64_t> ids;
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return fail(ATA_EINVAL, "NULL plan in batch");
        const Plan& P = plan_of(plans[i]);
        if (P.gemm) return fail(ATA_EINVAL, "general-product plans run through ata_gemm_tn");
        if (i == 0) *leaf = P.leaf;
        if (P.leaf != *leaf) return fail(ATA_EINVAL, "plans of one batch must share the dtype family");
        if (lda[i] < P.n || lda[i] < 1) return fail(ATA_EINVAL, "lda[i] must be >= max(n_i, 1)");
        key->push_back((int64_t)plan_id(plans[i]));
        key->push_back(lda[i]);
        ids.push_back(plan_id(plans[i]));
    }
    std::sort(ids.begin(), ids.end());
    if (std::adjacent_find(ids.begin(), ids.end()) != ids.end())
        return fail(ATA_EINVAL, "a plan appears twice in one batch");
    return ATA_OK;
}

// Merged tables of instances [g0, g1).
ata_status build_entry(const ata_plan* plans, const int64_t* lda, int g0, int g1, LeafKind leaf,
                       std::unique_ptr<BatchEntry>* out) {
    std::unique_ptr<BatchEntry> e(new BatchEntry());
    HostTables h;
    h.leaf = leaf;
    size_t ns = 0, nc = 0;
    for (int i = g0; i < g1; ++i) {
        ns = std::max(ns, plan_of(plans[i]).split_levels.size());
        nc = std::max(nc, plan_of(plans[i]).combine_levels.size());
    }
    h.split_pending.resize(ns);
    h.comb_pending.resize(nc);
    int8_t in_dt = DT_F64, sum_dt = DT_F64;
    for (int i = g0; i < g1; ++i) {
        const Plan& P = plan_of(plans[i]);
        append_plan_tables(P, i - g0, lda[i], &h);
        e->ids.push_back(plan_id(plans[i]));
        in_dt = P.in_dt;
        sum_dt = P.sum_dt;
    }
    finalize_tables(&h, in_dt, sum_dt);
    ata_status st = upload_tables(h, &e->tables);
    if (st != ATA_OK) return st;
    if (leaf != LEAF_F64 && !h.prods.empty()) {
        std::vector<char*> ws;
        for (int i = g0; i < g1; ++i) ws.push_back(plan_workspace(plans[i]));
        st = build_tc_tables(h, ws, &e->tables);
        if (st != ATA_OK) return st;
    }
    *out = std::move(e);
    return ATA_OK;
}

}  // namespace
}  // namespace ata

using namespace ata;

// A prepared batch: the plans, their packed layout, and their merged tables
// and graph.
struct ata_batch_s {
    std::vector<ata_plan> plans;
    std::vector<int64_t> lda, a_off, c_off;
    std::vector<uint64_t> ids;
    std::unique_ptr<BatchEntry> entry;
    std::vector<Bind> binds;  // of the most recent call
    const void* last_A = nullptr;
    double* last_C = nullptr;
    int elem = 8;         // bytes per input element
    bool dead = false;    // a plan of the batch was destroyed
};

namespace ata {
namespace {
std::set<ata_batch_s*> g_prepared;
}

void forget_plan_in_batches(uint64_t id) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto it = g_batches.begin(); it != g_batches.end();) {
        bool hit = false;
        for (uint64_t x : it->second->ids) hit |= (x == id);
        if (hit)
            it = g_batches.erase(it);
        else
            ++it;
    }
    for (ata_batch_s* b : g_prepared)
        if (!b->dead && std::binary_search(b->ids.begin(), b->ids.end(), id)) {
            b->dead = true;
            b->entry.reset();  // its tables and graph refer to the plan's workspace
        }
}

}  // namespace ata

extern "C" ata_status ata_execute_batched(const ata_plan* plans, int count, const void* const* A, const int64_t* lda,
                                          double* const* C_packed, void* stream) {
    NvtxRange nv("ata_execute_batched");
    if (count < 0) return fail(ATA_EINVAL, "count must be >= 0");
    if (count == 0) return ATA_OK;
    if (!plans || !A || !lda || !C_packed) return fail(ATA_EINVAL, "NULL array argument");
    LeafKind leaf = LEAF_F64;
    std::vector<int64_t> key;
    ata_status st = check_batch(plans, count, lda, &leaf, &key);
    if (st != ATA_OK) return st;
    for (int i = 0; i < count; ++i) {
        const Plan& P = plan_of(plans[i]);
        if (P.m > 0 && P.n > 0 && !A[i]) return fail(ATA_EINVAL, "A[i] is NULL");
        if (P.n > 0 && !C_packed[i]) return fail(ATA_EINVAL, "C_packed[i] is NULL");
        const int es = P.in_dt == DT_F64 ? 8 : 4;
        if (reinterpret_cast<uintptr_t>(A[i]) % es || reinterpret_cast<uintptr_t>(C_packed[i]) % 8)
            return fail(ATA_EINVAL, "A[i] or C_packed[i] is misaligned");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (stream_capturing(s)) return fail(ATA_EINVAL, kBatchCaptureRefused);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_batches.find(key);
    if (it == g_batches.end()) {
        std::unique_ptr<BatchEntry> e;
        st = build_entry(plans, lda, 0, count, leaf, &e);
        if (st != ATA_OK) return st;
        it = g_batches.emplace(key, std::move(e)).first;
    }
    std::vector<Bind> binds;
    binds.reserve(count);
    for (int i = 0; i < count; ++i) binds.push_back(make_bind(plans[i], A[i], lda[i], C_packed[i]));
    st = order_wait(plans, count, s);
    if (st != ATA_OK) return st;
    st = launch_via_graph(it->second->tables, binds.data(), count, &it->second->graph, s);
    if (st != ATA_OK) return st;
    return order_record(plans, count, s, &it->second->order_ev);
}

extern "C" ata_status ata_batched_graph_kernels(const ata_plan* plans, int count, const int64_t* lda,
                                               int32_t* kernels) {
    if (!kernels || count < 0 || (count > 0 && (!plans || !lda))) return fail(ATA_EINVAL, "NULL or invalid argument");
    *kernels = 0;
    std::vector<int64_t> key;
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return fail(ATA_EINVAL, "NULL plan in batch");
        key.push_back((int64_t)plan_id(plans[i]));
        key.push_back(lda[i]);
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (count == 0) return ATA_OK;
    auto it = g_batches.find(key);
    if (it == g_batches.end() || !it->second->graph.exec) return fail(ATA_EINVAL, "this batch has not been executed yet");
    *kernels = it->second->graph.kernels;
    return ATA_OK;
}

extern "C" ata_status ata_batch_create(ata_batch* out, const ata_plan* plans, int count, const int64_t* lda,
                                       const int64_t* a_off, const int64_t* c_off) {
    if (!out) return fail(ATA_EINVAL, "NULL output handle");
    *out = nullptr;
    if (count < 0) return fail(ATA_EINVAL, "count must be >= 0");
    if (count > 0 && (!plans || !lda || !a_off || !c_off)) return fail(ATA_EINVAL, "NULL array argument");
    LeafKind leaf = LEAF_F64;
    std::vector<int64_t> key;
    ata_status st = check_batch(plans, count, lda, &leaf, &key);
    if (st != ATA_OK) return st;
    std::unique_ptr<ata_batch_s> b(new ata_batch_s());
    for (int i = 0; i < count; ++i) {
        if (a_off[i] < 0 || c_off[i] < 0) return fail(ATA_EINVAL, "offsets must be >= 0");
        b->elem = plan_of(plans[i]).in_dt == DT_F64 ? 8 : 4;
    }
    b->plans.assign(plans, plans + count);
    b->lda.assign(lda, lda + count);
    b->a_off.assign(a_off, a_off + count);
    b->c_off.assign(c_off, c_off + count);
    for (int i = 0; i < count; ++i) b->ids.push_back(plan_id(plans[i]));
    std::sort(b->ids.begin(), b->ids.end());
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (count > 0) {
        st = build_entry(plans, lda, 0, count, leaf, &b->entry);
        if (st != ATA_OK) return st;
    }
    g_prepared.insert(b.get());
    *out = b.release();
    return ATA_OK;
}

extern "C" ata_status ata_batch_execute(ata_batch b, const void* A, double* C, void* stream) {
    NvtxRange nv("ata_batch_execute");
    if (!b) return fail(ATA_EINVAL, "NULL batch");
    const int count = (int)b->plans.size();
    if (count == 0) return ATA_OK;
    if (!A || !C) return fail(ATA_EINVAL, "NULL A or C");
    if (reinterpret_cast<uintptr_t>(A) % b->elem || reinterpret_cast<uintptr_t>(C) % 8)
        return fail(ATA_EINVAL, "A or C is misaligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (stream_capturing(s)) return fail(ATA_EINVAL, kBatchCaptureRefused);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (b->dead) return fail(ATA_EINVAL, "a plan of this batch has been destroyed");
    if (A != b->last_A || C != b->last_C) {
        b->binds.clear();
        for (int i = 0; i < count; ++i)
            b->binds.push_back(make_bind(b->plans[i], static_cast<const char*>(A) + b->a_off[i] * b->elem,
                                         b->lda[i], C + b->c_off[i]));
        b->last_A = A;
        b->last_C = C;
    }
    ata_status st = order_wait(b->plans.data(), count, s);
    if (st != ATA_OK) return st;
    st = launch_via_graph(b->entry->tables, b->binds.data(), count, &b->entry->graph, s);
    if (st != ATA_OK) {
        b->last_A = nullptr;  // rebuild the bindings on the next call
        return st;
    }
    return order_record(b->plans.data(), count, s, &b->entry->order_ev);
}

extern "C" ata_status ata_batch_graph_kernels(ata_batch b, int32_t* kernels) {
    if (!b || !kernels) return fail(ATA_EINVAL, "NULL argument");
    *kernels = 0;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (b->dead) return fail(ATA_EINVAL, "a plan of this batch has been destroyed");
    if (b->plans.empty()) return ATA_OK;
    if (!b->entry || !b->entry->graph.exec) return fail(ATA_EINVAL, "this batch has not been executed yet");
    *kernels = b->entry->graph.kernels;
    return ATA_OK;
}

extern "C" void ata_batch_destroy(ata_batch b) {
    if (!b) return;
    if (b->entry) cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_prepared.erase(b);
    delete b;
}
