// batched.cu -- ata_execute_batched: many independent products in one queued
// batch.  The task tables of all instances are merged level by level, so the
// whole batch is one split launch per level, one persistent leaf launch whose
// tiles (all instances) run heaviest first, and one combine launch per level,
// captured once as a CUDA graph per distinct set of plans.
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "runtime.h"

namespace ata {
namespace {

struct BatchEntry {
    DeviceTables tables;
    GraphCache graph;
    std::vector<uint64_t> ids;
    ~BatchEntry() {
        graph.release();
        tables.free_all();
    }
};

std::mutex g_batch_mu;
std::map<std::vector<int64_t>, std::unique_ptr<BatchEntry>> g_batches;

}  // namespace

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
}

}  // namespace ata

using namespace ata;

extern "C" ata_status ata_execute_batched(const ata_plan* plans, int count, const void* const* A, const int64_t* lda,
                                          double* const* C_packed, void* stream) {
    if (count < 0) return fail(ATA_EINVAL, "count must be >= 0");
    if (count == 0) return ATA_OK;
    if (!plans || !A || !lda || !C_packed) return fail(ATA_EINVAL, "NULL array argument");
    const LeafKind leaf = plans[0] ? plan_of(plans[0]).leaf : LEAF_F64;
    std::vector<int64_t> key;
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return fail(ATA_EINVAL, "NULL plan in batch");
        const Plan& P = plan_of(plans[i]);
        if (P.gemm) return fail(ATA_EINVAL, "general-product plans run through ata_gemm_tn");
        if (P.leaf != leaf) return fail(ATA_EINVAL, "plans of one batch must share the dtype family");
        if (lda[i] < P.n || lda[i] < 1) return fail(ATA_EINVAL, "lda[i] must be >= max(n_i, 1)");
        if (P.m > 0 && P.n > 0 && !A[i]) return fail(ATA_EINVAL, "A[i] is NULL");
        if (P.n > 0 && !C_packed[i]) return fail(ATA_EINVAL, "C_packed[i] is NULL");
        const int es = P.in_dt == DT_F64 ? 8 : 4;
        if (reinterpret_cast<uintptr_t>(A[i]) % es || reinterpret_cast<uintptr_t>(C_packed[i]) % 8)
            return fail(ATA_EINVAL, "A[i] or C_packed[i] is misaligned");
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return fail(ATA_EINVAL, "a plan appears twice in one batch");
        key.push_back((int64_t)plan_id(plans[i]));
        key.push_back(lda[i]);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    // groups of at most kMaxBatchBind instances, each one merged table set
    for (int g0 = 0; g0 < count; g0 += kMaxBatchBind) {
        const int g1 = std::min(count, g0 + kMaxBatchBind);
        std::vector<int64_t> gkey(key.begin() + 2 * g0, key.begin() + 2 * g1);
        auto it = g_batches.find(gkey);
        if (it == g_batches.end()) {
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
            it = g_batches.emplace(gkey, std::move(e)).first;
        }
        std::vector<Bind> binds;
        for (int i = g0; i < g1; ++i) {
            const Plan& P = plan_of(plans[i]);
            binds.push_back(make_bind(plans[i], A[i], lda[i], C_packed[i]));
        }
        ata_status st = launch_via_graph(it->second->tables, binds.data(), (int)binds.size(), &it->second->graph, s);
        if (st != ATA_OK) return st;
    }
    return ATA_OK;
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
    int32_t total = 0;
    for (int g0 = 0; g0 < count; g0 += kMaxBatchBind) {
        const int g1 = std::min(count, g0 + kMaxBatchBind);
        auto it = g_batches.find(std::vector<int64_t>(key.begin() + 2 * g0, key.begin() + 2 * g1));
        if (it == g_batches.end() || !it->second->graph.exec)
            return fail(ATA_EINVAL, "this batch has not been executed yet");
        total += it->second->graph.kernels;
    }
    *kernels = total;
    return ATA_OK;
}
