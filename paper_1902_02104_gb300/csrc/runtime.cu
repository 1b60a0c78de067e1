// runtime.cu -- plans, device task tables, CUDA-graph execution and the C ABI
// declared in include/ata.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ata.h"
#include "kernels.h"
#include "plan.h"
#include "runtime.h"

namespace ata {

thread_local std::string g_last_error;

ata_status fail(ata_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

ata_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return ATA_ECUDA;
}

#define ATA_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

static std::atomic<uint64_t> g_plan_ids{1};

// ---------------------------------------------------------------------------
// Device allocations: bytes held, and host-side allocation-failure injection.

namespace {
std::mutex g_alloc_mu;
std::map<void*, size_t> g_alloc_live;
int64_t g_alloc_bytes = 0;
std::string g_fault_spec;   // last value of ATA_FAULT seen
int64_t g_fault_at = 0;     // allocation to fail (1-based), 0 = none
int64_t g_alloc_calls = 0;  // allocations since ATA_FAULT took its value
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
    *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        const char* f = getenv("ATA_FAULT");
        const std::string spec = f ? f : "";
        if (spec != g_fault_spec) {
            g_fault_spec = spec;
            g_alloc_calls = 0;
            g_fault_at = 0;
            if (spec.rfind("alloc@", 0) == 0) g_fault_at = std::atoll(spec.c_str() + 6);
        }
        if (g_fault_at > 0 && ++g_alloc_calls == g_fault_at) return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc_live[*p] = bytes;
    g_alloc_bytes += (int64_t)bytes;
    return cudaSuccess;
}

void dev_free(void* p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        auto it = g_alloc_live.find(p);
        if (it != g_alloc_live.end()) {
            g_alloc_bytes -= (int64_t)it->second;
            g_alloc_live.erase(it);
        }
    }
    cudaFree(p);
}

// ---------------------------------------------------------------------------
// Host tables -> one device blob.

static int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Row chunks of an elementwise task (split or combine), one block each: about
// 2048 elements (8 per thread of a 256-thread block), so that a level's
// launch has several blocks per SM even when it holds a single Strassen node
// (a 1125 x 1125 combine: 563 blocks; with 16384-element chunks it had 75
// and reached 8% of HBM bandwidth).
void build_chunks(int64_t rows, int64_t cols, int32_t task, std::vector<Chunk>* out) {
    if (rows <= 0 || cols <= 0) return;
    const int64_t per = std::max<int64_t>(1, (2048 + cols - 1) / cols);
    for (int64_t r0 = 0; r0 < rows; r0 += per) {
        Chunk c;
        c.task = task;
        c.row0 = (int32_t)r0;
        c.nrows = (int32_t)std::min<int64_t>(per, rows - r0);
        out->push_back(c);
    }
}

ata_status upload_tables(const HostTables& h, DeviceTables* d) {
    d->free_all();
    int64_t off = 0;
    auto place = [&](int64_t bytes) {
        int64_t o = off;
        off = align_up(off + std::max<int64_t>(bytes, 0), 256);
        return o;
    };
    const int64_t o_terms = place(h.terms.size() * sizeof(Term));
    const int64_t o_prods = place(h.prods.size() * sizeof(LeafProduct));
    const int64_t o_tiles = place(h.tiles.size() * sizeof(LeafTile));
    const int64_t o_cnt = place(64);
    const int64_t o_split = place(h.split.size() * sizeof(SplitTask));
    const int64_t o_schunk = place(h.split_chunks.size() * sizeof(Chunk));
    const int64_t o_comb = place(h.comb.size() * sizeof(CombineTask));
    const int64_t o_cchunk = place(h.comb_chunks.size() * sizeof(Chunk));
    const int64_t o_psum = place(h.partial_sums.size() * sizeof(PartialSum));
    const int64_t total = std::max<int64_t>(off, 256);
    char* blob = nullptr;
    cudaError_t e = dev_malloc(&blob, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ATA_ENOMEM, "task tables: cudaMalloc failed");
    }
    std::vector<char> hb(total, 0);
    auto put = [&](int64_t o, const void* src, size_t bytes) {
        if (bytes) std::memcpy(hb.data() + o, src, bytes);
    };
    put(o_terms, h.terms.data(), h.terms.size() * sizeof(Term));
    put(o_prods, h.prods.data(), h.prods.size() * sizeof(LeafProduct));
    put(o_tiles, h.tiles.data(), h.tiles.size() * sizeof(LeafTile));
    put(o_split, h.split.data(), h.split.size() * sizeof(SplitTask));
    put(o_schunk, h.split_chunks.data(), h.split_chunks.size() * sizeof(Chunk));
    put(o_comb, h.comb.data(), h.comb.size() * sizeof(CombineTask));
    put(o_cchunk, h.comb_chunks.data(), h.comb_chunks.size() * sizeof(Chunk));
    put(o_psum, h.partial_sums.data(), h.partial_sums.size() * sizeof(PartialSum));
    e = cudaMemcpy(blob, hb.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dev_free(blob);
        return cuda_fail(e, "task tables: upload");
    }
    d->blob = blob;
    d->terms = reinterpret_cast<Term*>(blob + o_terms);
    d->prods = reinterpret_cast<LeafProduct*>(blob + o_prods);
    d->tiles = reinterpret_cast<LeafTile*>(blob + o_tiles);
    d->counter = reinterpret_cast<int*>(blob + o_cnt);
    d->split = reinterpret_cast<SplitTask*>(blob + o_split);
    d->split_chunks = reinterpret_cast<Chunk*>(blob + o_schunk);
    d->comb = reinterpret_cast<CombineTask*>(blob + o_comb);
    d->comb_chunks = reinterpret_cast<Chunk*>(blob + o_cchunk);
    d->partial_sums = reinterpret_cast<PartialSum*>(blob + o_psum);
    d->npartial_sums = (int)h.partial_sums.size();
    d->ntiles = (int)h.tiles.size();
    d->split_lv = h.split_lv;
    d->comb_lv = h.comb_lv;
    d->leaf = h.leaf;
    d->tc_pair = h.leaf != LEAF_F64 && h.tile_rows == kTcPairRows;
    return ATA_OK;
}

// Appends plan `P` (instance `inst`, A leading dimension `lda`) to host tables.
// Tables of several plans concatenate level by level (batched execution).
void append_plan_tables(const Plan& P, int inst, int64_t lda, HostTables* h, int64_t ldb, int64_t ldc) {
    const int32_t t_base = (int32_t)h->terms.size();
    const int32_t p_base = (int32_t)h->prods.size();
    // offsets planned for dense A (ld n), Y (ld r) and C (ld r) move to the
    // caller's leading dimensions
    auto rebase = [](int64_t off, int64_t planned_ld, int64_t ld) {
        return planned_ld > 0 ? off / planned_ld * ld + off % planned_ld : off;
    };
    auto fix_term = [&](Term t) {
        t.inst = inst;
        if (t.buf == BUF_A && P.n > 0) {
            t.off = rebase(t.off, P.n, lda);
            t.ld = lda;
        } else if (t.buf == BUF_B && P.r > 0) {
            t.off = rebase(t.off, P.r, ldb);
            t.ld = ldb;
        }
        return t;
    };
    for (const Term& t : P.terms) h->terms.push_back(fix_term(t));
    for (LeafProduct lp : P.products) {
        lp.x0 += t_base;
        lp.y0 += t_base;
        lp.inst = inst;
        if (lp.out_kind == OUT_CDENSE) {
            lp.out_off = rebase(lp.out_off, P.r, ldc);
            lp.out_ld = (int32_t)ldc;
        }
        h->prods.push_back(lp);
    }
    for (size_t i = 0; i < P.products.size(); ++i) {
        const LeafProduct& lp = P.products[i];
        const int tm = P.leaf == LEAF_F64 ? kF64Tile : h->tile_rows;
        const int tn = P.leaf == LEAF_F64 ? kF64Tile : tc_cols_for(P.leaf, tm);
        const int64_t a = (lp.out_rows + tm - 1) / tm, b = (lp.out_cols + tn - 1) / tn;
        // FP64 tiles cut along K: kparts ranges of whole 16-value slabs
        const int parts = P.leaf == LEAF_F64 && lp.kparts > 1 ? lp.kparts : 1;
        const int kc = parts > 1 ? (lp.K + parts * 16 - 1) / (parts * 16) * 16 : lp.K;
        int32_t tile_index = 0;
        for (int64_t ti = 0; ti < a; ++ti)
            for (int64_t tj = (lp.out_kind == OUT_SYRK ? ti * tm / tn : 0); tj < b; ++tj, ++tile_index) {
                LeafTile t;
                t.prod = p_base + (int32_t)i;
                t.ti = (int32_t)ti;
                t.tj = (int32_t)tj;
                if (parts <= 1) {
                    t.k0 = 0;
                    t.k1 = lp.K;
                    t.part = -1;
                    h->tiles.push_back(t);
                    continue;
                }
                for (int q = 0; q < parts; ++q) {
                    t.k0 = std::min(lp.K, q * kc);
                    t.k1 = std::min(lp.K, (q + 1) * kc);
                    t.part = tile_index * parts + q;
                    h->tiles.push_back(t);
                }
                h->partial_sums.push_back(PartialSum{t.prod, t.ti, t.tj, tile_index * parts});
            }
    }
    // split / combine levels, merged level by level
    if (h->split_lv.size() < P.split_levels.size()) h->split_lv.resize(P.split_levels.size());
    if (h->comb_lv.size() < P.combine_levels.size()) h->comb_lv.resize(P.combine_levels.size());
    for (size_t l = 0; l < P.split_levels.size(); ++l)
        for (SplitTask st : P.split_levels[l]) {
            st.src = fix_term(st.src);
            st.inst = inst;
            h->split_pending[l].push_back(st);
        }
    for (size_t l = 0; l < P.combine_levels.size(); ++l)
        for (CombineTask ct : P.combine_levels[l]) {
            ct.inst = inst;
            if (ct.dst_kind == OUT_CDENSE) {
                ct.dst_off = rebase(ct.dst_off, P.r, ldc);
                ct.dst_ld = (int32_t)ldc;
            }
            h->comb_pending[l].push_back(ct);
        }
}

// Orders leaf tiles heaviest first and lays out split/combine tasks and chunks
// contiguously per level.
void finalize_tables(HostTables* h, int8_t in_dt, int8_t sum_dt) {
    std::stable_sort(h->tiles.begin(), h->tiles.end(),
                     [](const LeafTile& a, const LeafTile& b) { return a.k1 - a.k0 > b.k1 - b.k0; });
    for (size_t l = 0; l < h->split_lv.size(); ++l) {
        LevelRange& lr = h->split_lv[l];
        lr.chunk0 = (int32_t)h->split_chunks.size();
        lr.src_dt = l == 0 ? in_dt : sum_dt;
        lr.dst_dt = sum_dt;
        for (const SplitTask& st : h->split_pending[l]) {
            const int32_t tid = (int32_t)h->split.size();
            h->split.push_back(st);
            build_chunks(st.K1, st.c1, tid, &h->split_chunks);
        }
        lr.nchunks = (int32_t)h->split_chunks.size() - lr.chunk0;
    }
    for (size_t l = 0; l < h->comb_lv.size(); ++l) {
        LevelRange& lr = h->comb_lv[l];
        lr.chunk0 = (int32_t)h->comb_chunks.size();
        for (const CombineTask& ct : h->comb_pending[l]) {
            const int32_t tid = (int32_t)h->comb.size();
            h->comb.push_back(ct);
            build_chunks(ct.p1, ct.r1, tid, &h->comb_chunks);
        }
        lr.nchunks = (int32_t)h->comb_chunks.size() - lr.chunk0;
    }
    h->split_pending.clear();
    h->comb_pending.clear();
}


void DeviceTables::free_all() {
    dev_free(blob);
    dev_free(tc_blob);
    blob = nullptr;
    tc_blob = nullptr;
    partial_sums = nullptr;
    npartial_sums = 0;
    tcp = nullptr;
    prep = nullptr;
    colmax = nullptr;
    term_mx = mx_list = atom_mx = nullptr;
    scale = nullptr;
    col_e = nullptr;
    atom_terms = nullptr;
    term_max = nullptr;
    status = nullptr;
    sched = nullptr;
    wfirst = nullptr;
    nworkers = 0;
}

// Queues one execution of `t` with bindings `binds` on `s` (no graph).
// SM count and resident leaf blocks per SM of the current device (queried
// outside any stream capture, once per process).
static void device_params(int* sms, int* per_sm) {
    static int s_sms = -1, s_per = -1;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (s_sms < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&s_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s_sms <= 0)
            s_sms = 1;
        s_per = leaf_f64_blocks_per_sm();
    }
    *sms = s_sms;
    *per_sm = s_per;
}

ata_status enqueue_tables(const DeviceTables& t, const Bind* binds, int nb, cudaStream_t s, const cudaEvent_t* ev) {
    int sms = 1, per_sm = 1;
    device_params(&sms, &per_sm);
    int* fstatus = t.counter + 1;  // status word of the FP64 / split / combine kernels
    if (ev) ATA_CUDA(cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal));
    for (size_t l = 0; l < t.split_lv.size(); ++l) {
        const LevelRange& lr = t.split_lv[l];
        ATA_CUDA(launch_split(fstatus, binds, nb, t.split, t.split_chunks + lr.chunk0, lr.nchunks, lr.src_dt,
                              lr.dst_dt, s));
    }
    if (t.ntiles > 0) ATA_CUDA(cudaMemsetAsync(t.counter, 0, sizeof(int), s));
    if (ev) ATA_CUDA(cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal));
    if (t.ntiles > 0) {
        if (t.leaf == LEAF_F64) {
            if (ev) ATA_CUDA(cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal));
            const int grid = std::max(1, std::min(t.ntiles, sms * per_sm));
            ATA_CUDA(launch_leaf_f64(fstatus, binds, nb, t.prods, t.terms, t.tiles, t.ntiles, t.counter, grid, s));
            if (t.npartial_sums > 0)
                ATA_CUDA(launch_partial_sums(fstatus, binds, nb, t.prods, t.partial_sums, t.npartial_sums, s));
        } else {
            ata_status st = launch_leaf_tc(t, binds, nb, s, ev ? ev[2] : nullptr);
            if (st != ATA_OK) return st;
        }
    }
    if (ev && t.ntiles == 0) ATA_CUDA(cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal));
    if (ev) ATA_CUDA(cudaEventRecordWithFlags(ev[3], s, cudaEventRecordExternal));
    for (int l = (int)t.comb_lv.size() - 1; l >= 0; --l) {
        const LevelRange& lr = t.comb_lv[l];
        ATA_CUDA(launch_combine(fstatus, binds, nb, t.comb, t.comb_chunks + lr.chunk0, lr.nchunks, s));
    }
    if (ev) ATA_CUDA(cudaEventRecordWithFlags(ev[4], s, cudaEventRecordExternal));
    return ATA_OK;
}

// Captures the launches of `t` into a graph and instantiates (or updates) `g`.
ata_status capture_graph(const DeviceTables& t, const Bind* binds, int nb, GraphCache* g) {
    if (!g->cap_stream) ATA_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    if (g->timing && !g->ev[0])
        for (int i = 0; i < 5; ++i) ATA_CUDA(cudaEventCreate(&g->ev[i]));
    {
        int sms, per_sm;
        device_params(&sms, &per_sm);  // before capture: attribute queries are not captured work
    }
    ATA_CUDA(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
    ata_status st = enqueue_tables(t, binds, nb, g->cap_stream, g->timing ? g->ev : nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
    if (st != ATA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    {
        // kernel nodes of the captured work (the launches one replay makes)
        size_t nn = 0;
        if (cudaGraphGetNodes(graph, nullptr, &nn) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_fail(cudaGetLastError(), "cudaGraphGetNodes");
        }
        std::vector<cudaGraphNode_t> nodes(nn);
        int kernels = 0;
        if (nn > 0 && cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess) {
            for (size_t i = 0; i < nn; ++i) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
            }
        }
        g->kernels = kernels;
    }
    if (g->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(g->exec, graph, &info) == cudaSuccess) {
            cudaGraphDestroy(graph);
            return ATA_OK;
        }
        cudaGetLastError();
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    return ATA_OK;
}

void GraphCache::release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (int i = 0; i < 5; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    for (int i = 0; i < 5; ++i) ev[i] = nullptr;
    exec = nullptr;
    cap_stream = nullptr;
    if (launched) cudaEventSynchronize(launched);
    dev_free(dev_binds);
    if (stage_binds) cudaFreeHost(stage_binds);
    for (cudaEvent_t* e : {&uploaded, &launched}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
    }
    dev_binds = nullptr;
    stage_binds = nullptr;
    dev_count = 0;
    binds.clear();
    kernels = 0;
    timed_run = false;
}

bool same_binds(const std::vector<Bind>& a, const Bind* b, int nb) {
    if ((int)a.size() != nb) return false;
    for (int i = 0; i < nb; ++i)
        if (a[i].A != b[i].A || a[i].B != b[i].B || a[i].C != b[i].C || a[i].W != b[i].W || a[i].n != b[i].n)
            return false;
    return true;
}

// Launches the tables through the cached graph (captured on first use or
// when the bindings change).
ata_status launch_via_graph(const DeviceTables& t, const Bind* binds, int nb, GraphCache* g, cudaStream_t s) {
    if (nb <= 1) {
        if (!g->exec || !same_binds(g->binds, binds, nb)) {
            ata_status st = capture_graph(t, binds, nb, g);
            if (st != ATA_OK) return st;
            g->binds.assign(binds, binds + nb);
        }
        ATA_CUDA(cudaGraphLaunch(g->exec, s));
        g->timed_run = g->timing;
        return ATA_OK;
    }
    // Several instances: the kernels read the bindings from a device array
    // that the graph refers to, so buffers that move need an upload of the
    // array, not a new capture.
    const size_t bytes = (size_t)nb * sizeof(Bind);
    if (!g->exec || g->dev_count != nb) {
        if (g->exec || g->dev_binds) g->release();
        ATA_CUDA(dev_malloc(&g->dev_binds, bytes));
        ATA_CUDA(cudaMallocHost(&g->stage_binds, bytes));
        ATA_CUDA(cudaEventCreateWithFlags(&g->uploaded, cudaEventDisableTiming));
        ATA_CUDA(cudaEventCreateWithFlags(&g->launched, cudaEventDisableTiming));
        g->dev_count = nb;
        std::memcpy(g->stage_binds, binds, bytes);
        ATA_CUDA(cudaMemcpy(g->dev_binds, g->stage_binds, bytes, cudaMemcpyHostToDevice));
        ata_status st = capture_graph(t, g->dev_binds, nb, g);
        if (st != ATA_OK) return st;
        g->binds.assign(binds, binds + nb);
    } else if (!same_binds(g->binds, binds, nb)) {
        // after every earlier launch of the graph (on any stream), and once
        // the previous upload has left the staging buffer
        ATA_CUDA(cudaStreamWaitEvent(s, g->launched, 0));
        ATA_CUDA(cudaEventSynchronize(g->uploaded));
        std::memcpy(g->stage_binds, binds, bytes);
        ATA_CUDA(cudaMemcpyAsync(g->dev_binds, g->stage_binds, bytes, cudaMemcpyHostToDevice, s));
        ATA_CUDA(cudaEventRecord(g->uploaded, s));
        g->binds.assign(binds, binds + nb);
    }
    ATA_CUDA(cudaGraphLaunch(g->exec, s));
    ATA_CUDA(cudaEventRecord(g->launched, s));
    g->timed_run = g->timing;
    return ATA_OK;
}

}  // namespace ata

// ===========================================================================
// C ABI
// ===========================================================================
using namespace ata;

// Pipelined host execution (ata_execute_host_async): two device staging sets
// used alternately, the copy-in, execution and copy-out of a call on three
// streams ordered by events, and one graph per staging set.
struct HostPipe {
    bool ready = false;
    cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
    cudaEvent_t a_ready[2] = {nullptr, nullptr};    // staging A[b] holds the call's input
    cudaEvent_t comp_done[2] = {nullptr, nullptr};  // the execution on set b has finished
    cudaEvent_t c_read[2] = {nullptr, nullptr};     // C[b] has been copied out
    void* A[2] = {nullptr, nullptr};
    double* C[2] = {nullptr, nullptr};
    GraphCache graph[2];
    uint64_t calls = 0;
    void sync() const {
        for (cudaStream_t s : {h2d, comp, d2h})
            if (s) cudaStreamSynchronize(s);
    }
    void release() {
        sync();
        for (int b = 0; b < 2; ++b) {
            graph[b].release();
            for (cudaEvent_t* e : {&a_ready[b], &comp_done[b], &c_read[b]}) {
                if (*e) cudaEventDestroy(*e);
                *e = nullptr;
            }
            dev_free(A[b]);
            dev_free(C[b]);
            A[b] = nullptr;
            C[b] = nullptr;
        }
        for (cudaStream_t* s : {&h2d, &comp, &d2h}) {
            if (*s) cudaStreamDestroy(*s);
            *s = nullptr;
        }
        ready = false;
        calls = 0;
    }
};

struct ata_plan_s {
    uint64_t id = 0;
    Plan plan;
    ata_dtype dtype = ATA_F64;
    int device = 0;
    char* ws = nullptr;
    int64_t lda = -1;           // leading dimensions the device tables are built for
    int64_t ldb = -1, ldc = -1; // (Y and C: general products only)
    DeviceTables tables;
    GraphCache graph;
    std::mutex mu;
    int64_t check = 0;          // self-checked kernels (ATA_CHECK_BOUNDS=1 at creation)
    // canary guard bands around the workspace (ATA_CANARY=1 at creation):
    // ws_base = ws - guard; guard bytes of kCanaryByte before and after
    char* ws_base = nullptr;
    int64_t guard = 0;
    uint64_t wait_ns = 0;       // tensor-core leaves: pipeline wait limit (0 = default)
    // staging for ata_execute_host
    void* stage_A = nullptr;
    double* stage_C = nullptr;
    HostPipe pipe;  // ata_execute_host_async
    // the latest execution: its event and stream (guarded by g_order_mu)
    std::shared_ptr<OrderEvent> own_ev, last_ev;
    cudaStream_t last_stream = nullptr;
    ~ata_plan_s() {
        pipe.release();
        graph.release();
        tables.free_all();
        dev_free(ws_base ? ws_base : ws);
        dev_free(stage_A);
        dev_free(stage_C);
    }
};

namespace {

int elem_bytes(ata_dtype d) { return (d == ATA_F64 || d == ATA_F64_OZAKI) ? 8 : 4; }

bool valid_dtype(int d) { return d >= ATA_F64 && d <= ATA_F64_OZAKI; }

LeafKind leaf_of(ata_dtype d) {
    switch (d) {
        case ATA_F32_BF16X3: return LEAF_BF16X3;
        case ATA_F32_TF32: return LEAF_TF32;
        case ATA_F64_OZAKI: return LEAF_OZAKI;
        default: return LEAF_F64;
    }
}

ata_status make_options(int64_t m, int64_t n, ata_dtype dtype, const ata_plan_options& u, PlanOptions* o) {
    if (m < 0 || n < 0) return fail(ATA_EINVAL, "m and n must be >= 0");
    if (!valid_dtype(dtype)) return fail(ATA_EINVAL, "unknown dtype");
    const int cutoff = u.cutoff;
    if (cutoff != 0 && (cutoff < 16 || cutoff > 4096)) return fail(ATA_EINVAL, "cutoff must be 0 or in [16, 4096]");
    const int variant = u.variant < 0 ? ATA_STRASSEN : u.variant;
    if (variant != ATA_STRASSEN && variant != ATA_WINOGRAD) return fail(ATA_EINVAL, "unknown variant");
    if (u.fuse_levels < -1 || u.fuse_levels > 16) return fail(ATA_EINVAL, "fuse_levels must be -1 or in [0, 16]");
    if (u.max_strassen_levels < -1 || u.max_strassen_levels > 64)
        return fail(ATA_EINVAL, "max_strassen_levels must be -1 or in [0, 64]");
    if (u.cta_pair < -1 || u.cta_pair > 1) return fail(ATA_EINVAL, "cta_pair must be -1, 0 or 1");
    if (u.wait_limit_us < -1 || u.wait_limit_us > 1000000)
        return fail(ATA_EINVAL, "wait_limit_us must be -1, 0 or in [1, 1000000]");
    o->wait_ns = u.wait_limit_us > 0 ? (uint64_t)u.wait_limit_us * 1000u : 0;
    o->leaf = leaf_of(dtype);
    o->variant = variant;
    o->cutoff = cutoff != 0 ? cutoff : default_cutoff(m, n, dtype);
    o->fuse_levels = u.fuse_levels >= 0 ? u.fuse_levels : default_fuse_levels(dtype, variant);
    o->max_levels = u.max_strassen_levels >= 0 ? u.max_strassen_levels : kFreeLevels;
    // CTA pairs by default for TF32, whose leaf is bound by L2 reads (a pair
    // stages half of B per SM); single CTAs for the others
    o->cta_pair = u.cta_pair == 1 || (u.cta_pair < 0 && dtype == ATA_F32_TF32);
    return ATA_OK;
}

ata_plan_options default_opts(int cutoff, int variant) {
    ata_plan_options u;
    u.cutoff = cutoff;
    u.variant = variant;
    u.fuse_levels = -1;
    u.max_strassen_levels = -1;
    u.cta_pair = -1;
    u.wait_limit_us = -1;
    return u;
}

void fill_info(const Plan& P, ata_dtype dtype, ata_plan_info* out) {
    std::memset(out, 0, sizeof(*out));
    out->m = P.m;
    out->n = P.n;
    out->dtype = dtype;
    out->cutoff = P.cutoff;
    out->depth = P.stats.depth;
    out->n_diag_leaves = P.stats.n_diag_leaves;
    out->n_nodes = P.stats.n_nodes;
    out->max_strassen_levels = P.stats.max_strassen_levels;
    out->n_leaf_products = (int32_t)P.products.size();
    int64_t tiles = 0;
    const int tm = P.leaf == LEAF_F64 ? kF64Tile : P.tc_tile_rows;  // planned tile shape
    const int tn = P.leaf == LEAF_F64 ? kF64Tile : tc_cols_for(P.leaf, tm);
    for (const LeafProduct& lp : P.products) tiles += leaf_tiles(lp, tm, tn);
    out->n_leaf_tiles = (int32_t)tiles;
    int64_t ns = 0, nc = 0;
    for (auto& v : P.split_levels) ns += v.size();
    for (auto& v : P.combine_levels) nc += v.size();
    out->n_sum_tasks = (int32_t)ns;
    out->n_combine_tasks = (int32_t)nc;
    // kernels one execution launches: a split and a combine kernel per level,
    // then the leaf kernel, preceded for tensor-core leaves by the operand
    // preparation (and the column maxima of the sliced modes, and the column
    // scales of the FP64 emulation), and followed by the partial sums of FP64
    // tiles cut along K
    bool cut = false;
    for (const LeafProduct& lp : P.products) cut = cut || (P.leaf == LEAF_F64 && lp.kparts > 1);
    const int leaf_kernels = P.products.empty()    ? 0
                             : P.leaf == LEAF_F64   ? (cut ? 2 : 1)
                             : P.leaf == LEAF_TF32  ? 2
                             : P.leaf == LEAF_OZAKI ? 4
                                                    : 3;
    out->n_launches = (int32_t)(P.split_levels.size() + P.combine_levels.size() + leaf_kernels);
    out->mults = P.stats.mults;
    out->classical_mults = P.m * P.n * (P.n + 1) / 2;  // A^t A: the upper triangle
    out->adds = P.stats.adds;
    out->workspace_bytes = P.ws_bytes;
    out->leaf_tile_rows = tm;
    out->leaf_tile_cols = tn;
    if (P.gemm) {
        out->r = P.r;
        out->classical_mults = P.m * P.n * P.r;
    }
}

ata_status check_terms(const Plan& P) {
    for (const LeafProduct& lp : P.products)
        if (lp.nx > kMaxTerms || lp.ny > kMaxTerms)
            return fail(ATA_EUNSUPPORTED, "a leaf operand has more fused terms than the kernels accept");
    return ATA_OK;
}

ata_status rebuild_tables(ata_plan plan, int64_t lda, int64_t ldb = 0, int64_t ldc = 0) {
    HostTables h;
    h.leaf = plan->plan.leaf;
    if (h.leaf != LEAF_F64) h.tile_rows = tc_rows_for(plan->plan);
    h.split_pending.resize(plan->plan.split_levels.size());
    h.comb_pending.resize(plan->plan.combine_levels.size());
    append_plan_tables(plan->plan, 0, lda, &h, ldb, ldc);
    finalize_tables(&h, plan->plan.in_dt, plan->plan.sum_dt);
    ata_status st = upload_tables(h, &plan->tables);
    if (st != ATA_OK) return st;
    if (plan->plan.leaf != LEAF_F64 && !h.prods.empty()) {
        st = build_tc_tables(h, std::vector<char*>{plan->ws}, &plan->tables);
        if (st != ATA_OK) return st;
    }
    plan->tables.wait_ns = plan->wait_ns;
    plan->lda = lda;
    plan->ldb = ldb;
    plan->ldc = ldc;
    plan->graph.release();
    plan->pipe.graph[0].release();
    plan->pipe.graph[1].release();
    return ATA_OK;
}

// Host rows of A into a dense device staging buffer: one linear copy when
// the rows are contiguous (lda == n), a pitched copy otherwise.
cudaError_t copy_rows_in(void* dst, const void* A_host, int64_t m, int64_t n, int64_t lda, int es, cudaStream_t s) {
    if (lda == n) return cudaMemcpyAsync(dst, A_host, (size_t)m * n * es, cudaMemcpyHostToDevice, s);
    return cudaMemcpy2DAsync(dst, (size_t)n * es, A_host, (size_t)lda * es, (size_t)n * es, (size_t)m,
                             cudaMemcpyHostToDevice, s);
}

ata_status check_ptr(const void* p, int align, const char* what) {
    if (reinterpret_cast<uintptr_t>(p) % align != 0)
        return fail(ATA_EINVAL, std::string(what) + " is not aligned to its element size");
    return ATA_OK;
}

bool capturing(cudaStream_t s) { return stream_capturing(s); }

// Inside a stream capture the plan's kernels are enqueued themselves (a
// graph launch cannot be captured), with its current tables: a leading
// dimension that needs new tables is refused there.
ata_status capture_tables_refused() {
    return fail(ATA_EINVAL,
                "the stream is capturing and the plan's tables are for another leading dimension: run the "
                "plan once outside the capture with these leading dimensions first");
}

// One execution of an A^t A plan on `s` through graph cache g (arguments
// checked by the caller).
ata_status execute_on(ata_plan plan, const void* A, int64_t lda, double* C_packed, cudaStream_t s, GraphCache* g) {
    std::lock_guard<std::mutex> lk(plan->mu);
    if (capturing(s)) {
        if (lda != plan->lda) return capture_tables_refused();
        Bind b = make_bind(plan, A, lda, C_packed);
        return enqueue_tables(plan->tables, &b, 1, s);
    }
    if (lda != plan->lda) {
        // the streams may still run the previous tables
        ATA_CUDA(cudaStreamSynchronize(s));
        plan->pipe.sync();
        ata_status st = order_sync(plan);  // the latest execution, on any stream
        if (st == ATA_OK) st = rebuild_tables(plan, lda);
        if (st != ATA_OK) return st;
    }
    Bind b = make_bind(plan, A, lda, C_packed);
    ata_status st = order_wait(&plan, 1, s);
    if (st != ATA_OK) return st;
    st = launch_via_graph(plan->tables, &b, 1, g, s);
    if (st != ATA_OK) return st;
    return order_record(&plan, 1, s, &plan->own_ev);
}

}  // namespace

// One execution of an A^t A plan launched directly on `s`, without a CUDA
// graph.  The serving layer uses it: a stream capture on its scheduler
// thread would be broken by device-wide synchronisation that other threads
// of the process may issue at any time (cudaDeviceSynchronize, or an
// allocation that synchronises), so its executions make no capture.  The
// kernels and their parameters are those a graph replay runs, so the
// results are the same bits.  Returns the number of kernels launched.
ata_status ata::execute_direct(ata_plan plan, const void* A, int64_t lda, double* C_packed, cudaStream_t s,
                               int* kernels) {
    NvtxRange nv("ata_server: execute");
    *kernels = 0;
    if (plan->plan.gemm) return fail(ATA_EINVAL, "a general-product plan");
    const int64_t n = plan->plan.n;
    if (lda < n || lda < 1) return fail(ATA_EINVAL, "lda must be >= max(n, 1)");
    if (n == 0) return ATA_OK;
    std::lock_guard<std::mutex> lk(plan->mu);
    if (lda != plan->lda) {
        ATA_CUDA(cudaStreamSynchronize(s));
        plan->pipe.sync();
        ata_status st = order_sync(plan);  // the latest execution, on any stream
        if (st == ATA_OK) st = rebuild_tables(plan, lda);
        if (st != ATA_OK) return st;
    }
    Bind b = make_bind(plan, A, lda, C_packed);
    ata_status st = order_wait(&plan, 1, s);
    if (st != ATA_OK) return st;
    st = enqueue_tables(plan->tables, &b, 1, s);
    if (st != ATA_OK) return st;
    st = order_record(&plan, 1, s, &plan->own_ev);
    if (st != ATA_OK) return st;
    ata_plan_info info;
    fill_info(plan->plan, plan->dtype, &info);
    *kernels = info.n_launches;
    return ATA_OK;
}

extern "C" {

const char* ata_status_string(ata_status s) {
    switch (s) {
        case ATA_OK: return "ATA_OK";
        case ATA_EINVAL: return "ATA_EINVAL";
        case ATA_ENOMEM: return "ATA_ENOMEM";
        case ATA_EUNSUPPORTED: return "ATA_EUNSUPPORTED";
        case ATA_ECUDA: return "ATA_ECUDA";
        case ATA_PENDING: return "ATA_PENDING";
        case ATA_ETIMEOUT: return "ATA_ETIMEOUT";
        case ATA_EBUSY: return "ATA_EBUSY";
    }
    return "ATA_UNKNOWN";
}

const char* ata_last_error_message(void) { return g_last_error.c_str(); }

int64_t ata_device_bytes_held(void) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc_bytes;
}

ata_status ata_plan_query(int64_t m, int64_t n, ata_dtype dtype, int cutoff, ata_plan_info* out) {
    const ata_plan_options u = default_opts(cutoff, ATA_STRASSEN);
    return ata_plan_query_opts(m, n, dtype, &u, out);
}

ata_status ata_plan_query_opts(int64_t m, int64_t n, ata_dtype dtype, const ata_plan_options* opts,
                               ata_plan_info* out) {
    if (!out || !opts) return fail(ATA_EINVAL, "NULL argument");
    PlanOptions o;
    ata_status st = make_options(m, n, dtype, *opts, &o);
    if (st != ATA_OK) return st;
    if (opts->cutoff == 0) {
        st = autotune_cutoff(m, n, dtype, o.variant, &o);
        if (st != ATA_OK) return st;
    }
    Plan P;
    std::string err;
    if (!build_plan(m, n, o, &P, &err)) return fail(ATA_EINVAL, err);
    fill_info(P, dtype, out);
    return ATA_OK;
}

}  // extern "C"

namespace {

// Host check of a built plan's tables: every term inside its buffer, every
// workspace range inside the workspace, and every output entry written
// exactly once (packed upper C of A^t A, or dense p x r C of a general
// product; the coverage check runs up to 2^24 entries).
ata_status check_plan_tables(const Plan& P) {
    const int64_t ws = P.ws_bytes;
    const int64_t n = P.n;
    char msg[256];
    auto term_ok = [&](const Term& t, const char* what) -> bool {
        if (t.rows <= 0 || t.cols <= 0) return true;
        if (t.buf == BUF_A || t.buf == BUF_B) {
            const int64_t w = t.buf == BUF_A ? P.n : P.r;
            const int64_t r0 = w ? t.off / w : 0, c0 = w ? t.off % w : 0;
            if ((t.buf == BUF_B && !P.gemm) || t.ld != w || r0 + t.rows > P.m || c0 + t.cols > w) {
                snprintf(msg, sizeof msg, "%s: input term rows %lld+%d cols %lld+%d outside %lldx%lld", what,
                         (long long)r0, t.rows, (long long)c0, t.cols, (long long)P.m, (long long)w);
                return false;
            }
        } else {
            const int es = t.dt == DT_F64 ? 8 : 4;
            const int64_t end = (t.off + (int64_t)(t.rows - 1) * t.ld + t.cols) * es;
            if (t.off < 0 || t.cols > t.ld || end > ws) {
                snprintf(msg, sizeof msg, "%s: W term ends at byte %lld of %lld", what, (long long)end,
                         (long long)ws);
                return false;
            }
        }
        return true;
    };
    const int64_t n_out = P.gemm ? P.n * P.r : n * (n + 1) / 2;
    const bool cover = n_out <= (int64_t(1) << 24);
    std::vector<uint8_t> hits(cover ? (size_t)n_out : 0, 0);
    auto mark = [&](int64_t i, int64_t j) -> bool {
        int64_t k;
        if (P.gemm) {
            if (i < 0 || j < 0 || i >= P.n || j >= P.r) return false;
            k = i * P.r + j;
        } else {
            if (i < 0 || j < i || j >= n) return false;
            k = i * n - i * (i - 1) / 2 + (j - i);
        }
        if (cover) {
            uint8_t& h = hits[(size_t)k];
            if (h) return false;
            h = 1;
        }
        return true;
    };
    auto kind_ok = [&](int8_t kind) {
        return P.gemm ? (kind == OUT_DENSE || kind == OUT_CDENSE) : (kind != OUT_CDENSE);
    };
    // FP64 tiles cut along K: each product's partial tiles inside W, the
    // regions of different products disjoint
    {
        std::vector<std::pair<int64_t, int64_t>> regions;
        for (const LeafProduct& lp : P.products) {
            if (P.leaf != LEAF_F64 || lp.kparts <= 1) continue;
            const int64_t bytes = leaf_tiles(lp, kF64Tile, kF64Tile) * lp.kparts * (int64_t)kF64Tile * kF64Tile * 8;
            if (lp.part_off < 0 || lp.part_off * 8 + bytes > ws)
                return fail(ATA_EINVAL, "partial tiles beyond the workspace");
            regions.push_back({lp.part_off * 8, lp.part_off * 8 + bytes});
        }
        std::sort(regions.begin(), regions.end());
        for (size_t i = 1; i < regions.size(); ++i)
            if (regions[i].first < regions[i - 1].second) return fail(ATA_EINVAL, "partial tile regions overlap");
    }
    for (const LeafProduct& lp : P.products) {
        for (int t = 0; t < lp.nx; ++t)
            if (!term_ok(P.terms[lp.x0 + t], "leaf X")) return fail(ATA_EINVAL, msg);
        for (int t = 0; t < lp.ny; ++t)
            if (!term_ok(P.terms[lp.y0 + t], "leaf Y")) return fail(ATA_EINVAL, msg);
        if (lp.nx > kMaxTerms || lp.ny > kMaxTerms) return fail(ATA_EINVAL, "too many fused terms");
        if (lp.out_rows > lp.p || lp.out_cols > lp.r) return fail(ATA_EINVAL, "leaf extent beyond its product");
        if (!kind_ok(lp.out_kind)) return fail(ATA_EINVAL, "leaf output kind does not match the plan");
        if (lp.out_kind == OUT_CDENSE) {
            // planned with ld r and offset i0 * r + j0
            const int64_t i0 = lp.out_off / P.r, j0 = lp.out_off % P.r;
            if (lp.out_ld != P.r) return fail(ATA_EINVAL, "leaf C output with a wrong leading dimension");
            for (int64_t i = 0; i < lp.out_rows; ++i)
                for (int64_t j = 0; j < lp.out_cols; ++j)
                    if (!mark(i0 + i, j0 + j)) return fail(ATA_EINVAL, "leaf writes C outside or twice");
        } else if (lp.out_kind == OUT_DENSE) {
            const int64_t end = (lp.out_off + (int64_t)(lp.out_rows - 1) * lp.out_ld + lp.out_cols) * 8;
            if (lp.out_cols > lp.out_ld || end > ws) return fail(ATA_EINVAL, "leaf dense output beyond workspace");
        } else {
            for (int64_t i = 0; i < lp.out_rows; ++i)
                for (int64_t j = (lp.out_kind == OUT_SYRK ? i : 0); j < lp.out_cols; ++j)
                    if (!mark(lp.ci0 + i, lp.cj0 + j)) {
                        snprintf(msg, sizeof msg, "leaf writes C(%lld,%lld) outside or twice", (long long)(lp.ci0 + i),
                                 (long long)(lp.cj0 + j));
                        return fail(ATA_EINVAL, msg);
                    }
        }
        if (P.leaf != LEAF_F64) {
            const TcGeom g = tc_geom(P.leaf);
            if ((lp.tc_x_off + (int64_t)g.parts * lp.p_pad * lp.K_pad * g.elem) > ws ||
                (lp.tc_y_off + (int64_t)g.parts * lp.r_pad * lp.K_pad * g.elem) > ws ||
                lp.K_pad % 64 || lp.p_pad % kTcTile || lp.r_pad % kTcTile || lp.K_pad < lp.K)
                return fail(ATA_EINVAL, "tensor-core part buffers outside the workspace");
            // the planned tile grid: a tile stages X rows [ti tm, (ti + 1) tm) and Y
            // rows [tj tn, (tj + 1) tn) of every part.  X rows stay inside the
            // padded parts; Y rows may pass the padding only where the operand
            // has one part (nothing follows it in the tensor map, and the TMA
            // box reads zeros there) and by at most the odd CTA's half of a tile
            const int tm = P.tc_tile_rows > 0 ? P.tc_tile_rows : kTcTile, tn = tc_cols_for(P.leaf, tm);
            const int64_t a = (lp.out_rows + tm - 1) / tm, b = (lp.out_cols + tn - 1) / tn;
            if (tm == kTcPairRows && lp.p_pad % kTcPairRows)
                return fail(ATA_EINVAL, "CTA-pair tiles need X parts padded to whole 256-row tiles");
            if (a * tm > lp.p_pad) return fail(ATA_EINVAL, "leaf tiles read X rows past the padded parts");
            if (b * tn > lp.r_pad && !(g.parts == 1 && b * tn - lp.r_pad <= tn / 2))
                return fail(ATA_EINVAL, "leaf tiles read Y rows past the padded parts");
        }
    }
    for (auto& lv : P.split_levels)
        for (const SplitTask& stk : lv) {
            if (!term_ok(stk.src, "split source")) return fail(ATA_EINVAL, msg);
            const int es = stk.dst_dt == DT_F64 ? 8 : 4;
            for (int k = 0; k < stk.nout; ++k)
                if ((stk.out_off[k] + (int64_t)stk.K1 * stk.c1) * es > ws)
                    return fail(ATA_EINVAL, "split output beyond workspace");
        }
    for (auto& lv : P.combine_levels)
        for (const CombineTask& ct : lv) {
            if ((ct.m_off + 7LL * ct.p1 * ct.r1) * 8 > ws) return fail(ATA_EINVAL, "combine sources beyond workspace");
            if (!kind_ok(ct.dst_kind)) return fail(ATA_EINVAL, "combine output kind does not match the plan");
            if (ct.dst_kind == OUT_CDENSE) {
                const int64_t i0 = ct.dst_off / P.r, j0 = ct.dst_off % P.r;
                if (ct.dst_ld != P.r) return fail(ATA_EINVAL, "combine C output with a wrong leading dimension");
                for (int64_t i = 0; i < ct.p; ++i)
                    for (int64_t j = 0; j < ct.r; ++j)
                        if (!mark(i0 + i, j0 + j)) return fail(ATA_EINVAL, "combine writes C outside or twice");
            } else if (ct.dst_kind == OUT_DENSE) {
                if ((ct.dst_off + (int64_t)(ct.p - 1) * ct.dst_ld + ct.r) * 8 > ws || ct.r > ct.dst_ld)
                    return fail(ATA_EINVAL, "combine output beyond workspace");
            } else {
                for (int64_t i = 0; i < ct.p; ++i)
                    for (int64_t j = 0; j < ct.r; ++j)
                        if (!mark(ct.ci0 + i, ct.cj0 + j)) {
                            snprintf(msg, sizeof msg, "combine writes C(%lld,%lld) outside or twice",
                                     (long long)(ct.ci0 + i), (long long)(ct.cj0 + j));
                            return fail(ATA_EINVAL, msg);
                        }
            }
        }
    if (cover)
        for (size_t k = 0; k < hits.size(); ++k)
            if (!hits[k]) return fail(ATA_EINVAL, "an entry of C is never written");
    return ATA_OK;
}

// Options (opts may be NULL for the defaults), then the autotuned cutoff.
ata_status resolve_options(int64_t m, int64_t n, int64_t r, ata_dtype dtype, const ata_plan_options* opts,
                           PlanOptions* o) {
    const ata_plan_options u = opts ? *opts : default_opts(0, ATA_STRASSEN);
    ata_status st = make_options(m, n, dtype, u, o);
    if (st != ATA_OK) return st;
    if (u.cutoff == 0) return autotune_cutoff(m, n, dtype, o->variant, o, r);
    return ATA_OK;
}

// Allocates the workspace and tables of a built plan.
constexpr int64_t kCanaryBytes = 65536;  // keeps the workspace 256-byte aligned
constexpr int kCanaryByte = 0xA5;

ata_status finish_create(std::unique_ptr<ata_plan_s>& p, ata_dtype dtype) {
    ata_status st = check_terms(p->plan);
    if (st != ATA_OK) return st;
    if (!leaf_supported(p->plan.leaf)) return fail(ATA_EUNSUPPORTED, "leaf kind not built into this library");
    p->id = g_plan_ids.fetch_add(1);
    p->dtype = dtype;
    {
        const char* chk = getenv("ATA_CHECK_BOUNDS");
        p->check = (chk && chk[0] == '1') ? 1 : 0;
    }
    ATA_CUDA(cudaGetDevice(&p->device));
    {
        const char* cn = getenv("ATA_CANARY");
        p->guard = (cn && cn[0] == '1' && p->plan.ws_bytes > 0) ? kCanaryBytes : 0;
    }
    if (p->plan.ws_bytes > 0) {
        cudaError_t e = dev_malloc(&p->ws_base, p->plan.ws_bytes + 2 * p->guard);
        if (e == cudaSuccess && p->guard > 0) {
            e = cudaMemset(p->ws_base, kCanaryByte, p->guard);
            if (e == cudaSuccess) e = cudaMemset(p->ws_base + p->guard + p->plan.ws_bytes, kCanaryByte, p->guard);
        }
        p->ws = p->ws_base ? p->ws_base + p->guard : nullptr;
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ATA_ENOMEM, "workspace: cudaMalloc of " + std::to_string(p->plan.ws_bytes) + " bytes failed");
        }
    }
    return p->plan.gemm ? rebuild_tables(p.get(), p->plan.n, p->plan.r, p->plan.r) : rebuild_tables(p.get(), p->plan.n);
}

}  // namespace

extern "C" {

ata_status ata_plan_check(int64_t m, int64_t n, ata_dtype dtype, const ata_plan_options* opts) {
    if (!opts) return fail(ATA_EINVAL, "NULL argument");
    PlanOptions o;
    ata_status st = resolve_options(m, n, -1, dtype, opts, &o);
    if (st != ATA_OK) return st;
    Plan P;
    std::string err;
    if (!build_plan(m, n, o, &P, &err)) return fail(ATA_EINVAL, err);
    return check_plan_tables(P);
}

ata_status ata_gemm_plan_check(int64_t m, int64_t p, int64_t r, ata_dtype dtype, const ata_plan_options* opts) {
    if (r < 0) return fail(ATA_EINVAL, "r must be >= 0");
    PlanOptions o;
    ata_status st = resolve_options(m, p, r, dtype, opts, &o);
    if (st != ATA_OK) return st;
    Plan P;
    std::string err;
    if (!build_gemm_plan(m, p, r, o, &P, &err)) return fail(ATA_EINVAL, err);
    return check_plan_tables(P);
}

ata_status ata_gemm_query(int64_t m, int64_t p, int64_t r, ata_dtype dtype, const ata_plan_options* opts,
                          ata_plan_info* out) {
    if (!out) return fail(ATA_EINVAL, "NULL argument");
    if (r < 0) return fail(ATA_EINVAL, "r must be >= 0");
    PlanOptions o;
    ata_status st = resolve_options(m, p, r, dtype, opts, &o);
    if (st != ATA_OK) return st;
    Plan P;
    std::string err;
    if (!build_gemm_plan(m, p, r, o, &P, &err)) return fail(ATA_EINVAL, err);
    fill_info(P, dtype, out);
    return ATA_OK;
}

ata_status ata_gemm_plan_create(ata_plan* out, int64_t m, int64_t p, int64_t r, ata_dtype dtype,
                                const ata_plan_options* opts) {
    NvtxRange nv("ata_gemm_plan_create");
    if (!out) return fail(ATA_EINVAL, "NULL argument");
    *out = nullptr;
    if (r < 0) return fail(ATA_EINVAL, "r must be >= 0");
    PlanOptions o;
    ata_status st = resolve_options(m, p, r, dtype, opts, &o);
    if (st != ATA_OK) return st;
    std::unique_ptr<ata_plan_s> pl(new ata_plan_s());
    std::string err;
    if (!build_gemm_plan(m, p, r, o, &pl->plan, &err)) return fail(ATA_EINVAL, err);
    pl->wait_ns = o.wait_ns;
    st = finish_create(pl, dtype);
    if (st != ATA_OK) return st;
    *out = pl.release();
    return ATA_OK;
}

ata_status ata_gemm_tn(ata_plan plan, const void* X, int64_t ldx, const void* Y, int64_t ldy, double* C,
                       int64_t ldc, void* stream) {
    NvtxRange nv("ata_gemm_tn");
    if (!plan) return fail(ATA_EINVAL, "plan is NULL");
    if (!plan->plan.gemm) return fail(ATA_EINVAL, "an A^t A plan: use ata_execute");
    const int64_t m = plan->plan.m, p = plan->plan.n, r = plan->plan.r;
    if (ldx < p || ldx < 1) return fail(ATA_EINVAL, "ldx must be >= max(p, 1)");
    if (ldy < r || ldy < 1) return fail(ATA_EINVAL, "ldy must be >= max(r, 1)");
    if (ldc < r || ldc < 1) return fail(ATA_EINVAL, "ldc must be >= max(r, 1)");
    if (m > 0 && p > 0 && r > 0 && (!X || !Y)) return fail(ATA_EINVAL, "X or Y is NULL");
    if (p > 0 && r > 0 && !C) return fail(ATA_EINVAL, "C is NULL");
    ata_status st = check_ptr(X, elem_bytes(plan->dtype), "X");
    if (st == ATA_OK) st = check_ptr(Y, elem_bytes(plan->dtype), "Y");
    if (st == ATA_OK) st = check_ptr(C, 8, "C");
    if (st != ATA_OK) return st;
    if (p == 0 || r == 0) return ATA_OK;
    std::lock_guard<std::mutex> lk(plan->mu);
    const bool cap = capturing(static_cast<cudaStream_t>(stream));
    if (cap && (ldx != plan->lda || ldy != plan->ldb || ldc != plan->ldc)) return capture_tables_refused();
    if (ldx != plan->lda || ldy != plan->ldb || ldc != plan->ldc) {
        ATA_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
        st = order_sync(plan);  // the latest execution, on any stream
        if (st == ATA_OK) st = rebuild_tables(plan, ldx, ldy, ldc);
        if (st != ATA_OK) return st;
    }
    Bind b = make_bind(plan, X, ldx, C);
    b.B = Y;
    b.b_elems = m > 0 ? (m - 1) * ldy + r : 0;
    b.c_elems = (p - 1) * ldc + r;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cap) return enqueue_tables(plan->tables, &b, 1, s);
    st = order_wait(&plan, 1, s);
    if (st != ATA_OK) return st;
    st = launch_via_graph(plan->tables, &b, 1, &plan->graph, s);
    if (st != ATA_OK) return st;
    return order_record(&plan, 1, s, &plan->own_ev);
}


ata_status ata_plan_create_opts(ata_plan* out, int64_t m, int64_t n, ata_dtype dtype, const ata_plan_options* opts) {
    NvtxRange nv("ata_plan_create");
    if (!out || !opts) return fail(ATA_EINVAL, "NULL argument");
    *out = nullptr;
    PlanOptions o;
    ata_status st = resolve_options(m, n, -1, dtype, opts, &o);
    if (st != ATA_OK) return st;
    std::unique_ptr<ata_plan_s> p(new ata_plan_s());
    std::string err;
    if (!build_plan(m, n, o, &p->plan, &err)) return fail(ATA_EINVAL, err);
    p->wait_ns = o.wait_ns;
    st = finish_create(p, dtype);
    if (st != ATA_OK) return st;
    *out = p.release();
    return ATA_OK;
}

ata_status ata_plan_create(ata_plan* out, int64_t m, int64_t n, ata_dtype dtype, int cutoff) {
    const ata_plan_options u = default_opts(cutoff, ATA_STRASSEN);
    return ata_plan_create_opts(out, m, n, dtype, &u);
}

ata_status ata_plan_get_info(ata_plan plan, ata_plan_info* out) {
    if (!plan || !out) return fail(ATA_EINVAL, "NULL argument");
    fill_info(plan->plan, plan->dtype, out);
    if (plan->plan.leaf != LEAF_F64) {
        // the tile shape that runs on this device (the CTA-pair kernel may be
        // unavailable), and the tile count for it
        const int tm = tc_rows_for(plan->plan), tn = tc_cols_for(plan->plan.leaf, tm);
        int64_t tiles = 0;
        for (const LeafProduct& lp : plan->plan.products) tiles += leaf_tiles(lp, tm, tn);
        out->n_leaf_tiles = (int32_t)tiles;
        out->leaf_tile_rows = tm;
        out->leaf_tile_cols = tn;
    }
    return ATA_OK;
}

ata_status ata_plan_workspace_size(ata_plan plan, size_t* bytes) {
    if (!plan || !bytes) return fail(ATA_EINVAL, "NULL argument");
    *bytes = (size_t)plan->plan.ws_bytes;
    return ATA_OK;
}

ata_status ata_execute(ata_plan plan, const void* A, int64_t lda, double* C_packed, void* stream) {
    NvtxRange nv("ata_execute");
    if (!plan) return fail(ATA_EINVAL, "plan is NULL");
    if (plan->plan.gemm) return fail(ATA_EINVAL, "a general-product plan: use ata_gemm_tn");
    const int64_t m = plan->plan.m, n = plan->plan.n;
    if (lda < n || lda < 1) return fail(ATA_EINVAL, "lda must be >= max(n, 1)");
    if (m > 0 && n > 0 && !A) return fail(ATA_EINVAL, "A is NULL");
    if (n > 0 && !C_packed) return fail(ATA_EINVAL, "C_packed is NULL");
    ata_status st = check_ptr(A, elem_bytes(plan->dtype), "A");
    if (st != ATA_OK) return st;
    st = check_ptr(C_packed, 8, "C_packed");
    if (st != ATA_OK) return st;
    if (n == 0) return ATA_OK;
    return execute_on(plan, A, lda, C_packed, static_cast<cudaStream_t>(stream), &plan->graph);
}

ata_status ata_execute_host(ata_plan plan, const void* A_host, int64_t lda, double* C_host, void* stream) {
    NvtxRange nv("ata_execute_host");
    if (!plan) return fail(ATA_EINVAL, "plan is NULL");
    if (plan->plan.gemm) return fail(ATA_EINVAL, "a general-product plan: use ata_gemm_tn");
    const int64_t m = plan->plan.m, n = plan->plan.n;
    const int es = elem_bytes(plan->dtype);
    if (lda < n || lda < 1) return fail(ATA_EINVAL, "lda must be >= max(n, 1)");
    if (m > 0 && n > 0 && !A_host) return fail(ATA_EINVAL, "A is NULL");
    if (n > 0 && !C_host) return fail(ATA_EINVAL, "C_packed is NULL");
    if (n == 0) return ATA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (stream_capturing(s))
        return fail(ATA_EINVAL, "the stream is capturing: host-buffer executions copy from host memory and cannot be "
                                "recorded; capture ata_execute on device buffers instead");
    {
        std::lock_guard<std::mutex> lk(plan->mu);
        if (!plan->stage_A && m > 0) {
            if (dev_malloc(&plan->stage_A, (size_t)m * n * es) != cudaSuccess) {
                cudaGetLastError();
                plan->stage_A = nullptr;
                return fail(ATA_ENOMEM, "staging buffer for A");
            }
        }
        if (!plan->stage_C) {
            if (dev_malloc(&plan->stage_C, (size_t)(n * (n + 1) / 2) * 8) != cudaSuccess) {
                cudaGetLastError();
                plan->stage_C = nullptr;
                return fail(ATA_ENOMEM, "staging buffer for C");
            }
        }
    }
    if (m > 0) ATA_CUDA(copy_rows_in(plan->stage_A, A_host, m, n, lda, es, s));
    ata_status st = ata_execute(plan, plan->stage_A ? plan->stage_A : (const void*)plan->stage_C, n, plan->stage_C, stream);
    if (st != ATA_OK) return st;
    ATA_CUDA(cudaMemcpyAsync(C_host, plan->stage_C, (size_t)(n * (n + 1) / 2) * 8, cudaMemcpyDeviceToHost, s));
    ATA_CUDA(cudaStreamSynchronize(s));
    return ATA_OK;
}

ata_status ata_execute_host_async(ata_plan plan, const void* A_host, int64_t lda, double* C_host) {
    NvtxRange nv("ata_execute_host_async");
    if (!plan) return fail(ATA_EINVAL, "plan is NULL");
    if (plan->plan.gemm) return fail(ATA_EINVAL, "a general-product plan: use ata_gemm_tn");
    const int64_t m = plan->plan.m, n = plan->plan.n;
    const int es = elem_bytes(plan->dtype);
    if (lda < n || lda < 1) return fail(ATA_EINVAL, "lda must be >= max(n, 1)");
    if (m > 0 && n > 0 && !A_host) return fail(ATA_EINVAL, "A is NULL");
    if (n > 0 && !C_host) return fail(ATA_EINVAL, "C_packed is NULL");
    if (n == 0) return ATA_OK;
    HostPipe& P = plan->pipe;
    const size_t a_bytes = (size_t)m * n * es, c_bytes = (size_t)(n * (n + 1) / 2) * 8;
    int b;
    {
        std::lock_guard<std::mutex> lk(plan->mu);
        if (!P.ready) {
            bool ok = true;
            for (cudaStream_t* st : {&P.h2d, &P.comp, &P.d2h})
                ok = ok && cudaStreamCreateWithFlags(st, cudaStreamNonBlocking) == cudaSuccess;
            for (int i = 0; i < 2 && ok; ++i) {
                for (cudaEvent_t* e : {&P.a_ready[i], &P.comp_done[i], &P.c_read[i]})
                    ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
                ok = ok && (m == 0 || dev_malloc(&P.A[i], a_bytes) == cudaSuccess);
                ok = ok && dev_malloc(&P.C[i], c_bytes) == cudaSuccess;
            }
            if (!ok) {
                cudaGetLastError();
                P.release();
                return fail(ATA_ENOMEM, "pipelined host execution: streams, events or staging buffers");
            }
            P.ready = true;
        }
        b = (int)(P.calls++ & 1);
    }
    // copy-in, once the execution that last read staging set b has finished
    ATA_CUDA(cudaStreamWaitEvent(P.h2d, P.comp_done[b], 0));
    if (m > 0) ATA_CUDA(copy_rows_in(P.A[b], A_host, m, n, lda, es, P.h2d));
    ATA_CUDA(cudaEventRecord(P.a_ready[b], P.h2d));
    // execution, once the input has arrived and the copy-out that last read
    // C[b] has finished
    ATA_CUDA(cudaStreamWaitEvent(P.comp, P.a_ready[b], 0));
    ATA_CUDA(cudaStreamWaitEvent(P.comp, P.c_read[b], 0));
    ata_status st = execute_on(plan, P.A[b] ? P.A[b] : (const void*)P.C[b], n, P.C[b], P.comp, &P.graph[b]);
    if (st != ATA_OK) return st;
    ATA_CUDA(cudaEventRecord(P.comp_done[b], P.comp));
    // copy-out
    ATA_CUDA(cudaStreamWaitEvent(P.d2h, P.comp_done[b], 0));
    ATA_CUDA(cudaMemcpyAsync(C_host, P.C[b], c_bytes, cudaMemcpyDeviceToHost, P.d2h));
    ATA_CUDA(cudaEventRecord(P.c_read[b], P.d2h));
    return ATA_OK;
}

ata_status ata_plan_wait(ata_plan plan) {
    if (!plan) return fail(ATA_EINVAL, "plan is NULL");
    const HostPipe& P = plan->pipe;
    if (!P.ready) return ATA_OK;
    for (cudaStream_t s : {P.h2d, P.comp, P.d2h}) ATA_CUDA(cudaStreamSynchronize(s));
    return ATA_OK;
}

ata_status ata_plan_enable_stage_timing(ata_plan plan, int enable) {
    if (!plan) return fail(ATA_EINVAL, "plan is NULL");
    std::lock_guard<std::mutex> lk(plan->mu);
    const bool want = enable != 0;
    if (want != plan->graph.timing) {
        plan->graph.release();
        plan->graph.timing = want;
    }
    return ATA_OK;
}

ata_status ata_plan_stage_times(ata_plan plan, float* ms) {
    if (!plan || !ms) return fail(ATA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(plan->mu);
    if (!plan->graph.timing || !plan->graph.timed_run || !plan->graph.ev[0])
        return fail(ATA_EINVAL, "stage timing is not enabled or nothing has run");
    for (int i = 0; i < 4; ++i) ATA_CUDA(cudaEventElapsedTime(&ms[i], plan->graph.ev[i], plan->graph.ev[i + 1]));
    return ATA_OK;
}

ata_status ata_plan_graph_kernels(ata_plan plan, int32_t* kernels) {
    if (!plan || !kernels) return fail(ATA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(plan->mu);
    if (!plan->graph.exec) return fail(ATA_EINVAL, "the plan has not been executed yet");
    *kernels = plan->graph.kernels;
    return ATA_OK;
}

ata_status ata_plan_device_status(ata_plan plan, int* code) {
    if (!plan || !code) return fail(ATA_EINVAL, "NULL argument");
    *code = 0;
    if (plan->tables.status) ATA_CUDA(cudaMemcpy(code, plan->tables.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (*code == 0 && plan->tables.counter)
        ATA_CUDA(cudaMemcpy(code, plan->tables.counter + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (*code == 0 && plan->guard > 0) {
        // canary guard bands: any byte changed means a write outside the workspace
        std::vector<unsigned char> g((size_t)plan->guard);
        for (int side = 0; side < 2 && *code == 0; ++side) {
            const char* src = side == 0 ? plan->ws_base : plan->ws + plan->plan.ws_bytes;
            ATA_CUDA(cudaMemcpy(g.data(), src, g.size(), cudaMemcpyDeviceToHost));
            for (unsigned char b : g)
                if (b != (unsigned char)kCanaryByte) {
                    *code = side == 0 ? 90 : 91;
                    break;
                }
        }
    }
    return ATA_OK;
}

void ata_plan_destroy(ata_plan plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    forget_plan_in_batches(plan->id);
    delete plan;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Accessors used by the batched and serving layers.
namespace ata {
Bind make_bind(ata_plan p, const void* A, int64_t lda, double* C) {
    Bind b{};
    b.A = A;
    b.C = C;
    b.W = p->ws;
    b.n = p->plan.n;
    b.a_elems = p->plan.m > 0 ? (p->plan.m - 1) * lda + p->plan.n : 0;
    b.w_bytes = p->plan.ws_bytes;
    b.c_elems = p->plan.n * (p->plan.n + 1) / 2;
    b.check = p->check;
    return b;
}
namespace {
std::mutex g_order_mu;  // the plans' latest-execution fields
}  // namespace

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

OrderEvent::~OrderEvent() {
    if (e) cudaEventDestroy(e);
}

ata_status order_wait(const ata_plan* plans, int count, cudaStream_t s) {
    if (capturing(s)) return ATA_OK;
    std::lock_guard<std::mutex> lk(g_order_mu);
    std::vector<const OrderEvent*> waited;  // each distinct event once
    for (int i = 0; i < count; ++i) {
        const ata_plan p = plans[i];
        if (!p->last_ev || p->last_stream == s) continue;
        const OrderEvent* e = p->last_ev.get();
        if (std::find(waited.begin(), waited.end(), e) != waited.end()) continue;
        ATA_CUDA(cudaStreamWaitEvent(s, e->e, 0));
        waited.push_back(e);
    }
    return ATA_OK;
}

ata_status order_record(const ata_plan* plans, int count, cudaStream_t s, std::shared_ptr<OrderEvent>* ev) {
    if (capturing(s)) return ATA_OK;
    std::lock_guard<std::mutex> lk(g_order_mu);
    if (!*ev) {
        auto made = std::make_shared<OrderEvent>();
        ATA_CUDA(cudaEventCreateWithFlags(&made->e, cudaEventDisableTiming));
        *ev = std::move(made);
    }
    ATA_CUDA(cudaEventRecord((*ev)->e, s));
    for (int i = 0; i < count; ++i) {
        plans[i]->last_ev = *ev;
        plans[i]->last_stream = s;
    }
    return ATA_OK;
}

ata_status order_sync(ata_plan p) {
    std::shared_ptr<OrderEvent> ev;
    {
        std::lock_guard<std::mutex> lk(g_order_mu);
        ev = p->last_ev;
    }
    if (ev) ATA_CUDA(cudaEventSynchronize(ev->e));
    return ATA_OK;
}

const Plan& plan_of(ata_plan p) { return p->plan; }
uint64_t plan_id(ata_plan p) { return p->id; }
char* plan_workspace(ata_plan p) { return p->ws; }
ata_dtype plan_dtype(ata_plan p) { return p->dtype; }
}  // namespace ata
