// runtime.h -- internal runtime types shared by the C-ABI translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <map>
#include <string>
#include <memory>
#include <vector>

#include "../../include/ata.h"
#include "kernels.h"
#include "plan.h"

namespace ata {

// Chunks of one split or combine level.
struct LevelRange {
    int32_t chunk0 = 0, nchunks = 0;
    int8_t src_dt = DT_F64, dst_dt = DT_F64;
};

// Tensor-core leaf product as the GEMM kernel sees it: TMA maps of the split
// parts of both operands (parts stacked along rows) and the output target.
// Aligned as CUtensorMap is (the TMA maps must sit on their alignment).
struct TcProd {
    CUtensorMap tmx;
    CUtensorMap tmy;
    int32_t p_pad, r_pad, K_pad, inst;
    int32_t out_rows, out_cols, out_kind, out_ld;
    int64_t out_off;
    int32_t ci0, cj0;
    uint64_t* ex;      // FP64 emulation: max |x| per row of X (bit patterns)
    uint64_t* ey;      // ... per row of Y
    int64_t ex_index, ey_index;
};

// A 64-column strip of a leaf operand for the preparation kernels: rows
// [k0, k1) of columns [c0, c0 + 64) (one 64 x 64 tile for the slicing
// kernel, up to kColSpan rows for the column-maximum kernel).
struct PrepTask {
    int32_t prod;
    int8_t side, pad_[3];
    int32_t c0, k0, k1;
};
constexpr int kColSpan = 1024;

// Task tables on the host, ready to upload (one plan or a merged batch).
struct HostTables {
    LeafKind leaf = LEAF_F64;
    int tile_rows = kTcTile;  // tensor-core leaves: kTcPairRows selects the CTA-pair kernel
    std::vector<Term> terms;
    std::vector<LeafProduct> prods;
    std::vector<LeafTile> tiles;
    std::vector<SplitTask> split;
    std::vector<Chunk> split_chunks;
    std::vector<LevelRange> split_lv;
    std::vector<CombineTask> comb;
    std::vector<Chunk> comb_chunks;
    std::vector<LevelRange> comb_lv;
    std::vector<std::vector<SplitTask>> split_pending;
    std::vector<std::vector<CombineTask>> comb_pending;
    std::vector<PartialSum> partial_sums;  // FP64 tiles cut along K
};

// The same tables in device memory (one allocation).
struct DeviceTables {
    LeafKind leaf = LEAF_F64;
    bool tc_pair = false;  // tensor-core leaves run as CTA pairs (256-row tiles)
    char* blob = nullptr;
    Term* terms = nullptr;
    LeafProduct* prods = nullptr;
    LeafTile* tiles = nullptr;
    int ntiles = 0;
    int* counter = nullptr;
    SplitTask* split = nullptr;
    Chunk* split_chunks = nullptr;
    std::vector<LevelRange> split_lv;
    CombineTask* comb = nullptr;
    Chunk* comb_chunks = nullptr;
    PartialSum* partial_sums = nullptr;
    int npartial_sums = 0;
    std::vector<LevelRange> comb_lv;
    // tensor-core leaves
    char* tc_blob = nullptr;
    TcProd* tcp = nullptr;
    PrepTask* prep = nullptr;
    int nprep = 0;
    PrepTask* colmax = nullptr;  // column-maximum strips (sliced modes; FP64 emulation: per distinct block)
    int ncolmax = 0;
    int64_t* term_mx = nullptr;              // FP64 emulation: per term, the start of its list in mx_list
    int64_t* mx_list = nullptr;              // ... maxima offsets of the row segments of a block, -1 ended
    Term* atom_terms = nullptr;              // ... the row segments (disjoint blocks of the buffers)
    int64_t* atom_mx = nullptr;              // ... per segment, its maxima offset in term_max
    unsigned long long* term_max = nullptr;  // ... the segments' column maxima (bit patterns)
    PrepTask* scale = nullptr;               // ... column-scale strips (one per 64 columns of an operand)
    int nscale = 0;
    int* col_e = nullptr;                    // ... column scales E(c), indexed like the column maxima
    int* status = nullptr;     // device error word of the tensor-core kernels
    char* tc_ex = nullptr;     // FP64 emulation: column maxima (zeroed per run)
    size_t tc_ex_bytes = 0;
    uint64_t wait_ns = 0;      // limit of the leaf kernel's pipeline waits (0 = its default)
    // leaf tile schedule: worker w (a CTA or a CTA pair) runs sched[wfirst[w] .. wfirst[w+1])
    LeafTile* sched = nullptr;
    int32_t* wfirst = nullptr;
    int nworkers = 0;
    void free_all();
};

// An instantiated CUDA graph of one table set and the bindings it was
// captured with.
struct GraphCache {
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<Bind> binds;
    int kernels = 0;            // kernel nodes of the captured graph
    bool timing = false;        // graph records ev[] around its stages
    bool timed_run = false;     // an execution with timing has been queued
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // batched graphs (more than one instance): the device array of bindings
    // the kernels read, its pinned staging buffer, and events that order an
    // upload after the graph's earlier launches and before the staging
    // buffer's next refill
    Bind* dev_binds = nullptr;
    Bind* stage_binds = nullptr;
    int dev_count = 0;
    cudaEvent_t uploaded = nullptr, launched = nullptr;
    void release();
};

// Device allocations of the library's own buffers (workspaces, tables,
// staging).  dev_malloc counts the bytes held (ata_device_bytes_held) and
// honours the host-side fault injection ATA_FAULT=alloc@N: the N-th
// allocation after the variable takes a new value fails as if the device
// were out of memory (nothing is allocated).  dev_free(nullptr) is a no-op.
cudaError_t dev_malloc(void** p, size_t bytes);
void dev_free(void* p);
template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) {
    void* v = nullptr;
    cudaError_t e = dev_malloc(&v, bytes);
    *p = static_cast<T*>(v);
    return e;
}

// NVTX range over a host call of the C ABI (plan creation, execution,
// batches, tuning): a profiler attached to the process shows where each call
// spent its host time and which launches it queued.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

extern thread_local std::string g_last_error;
ata_status fail(ata_status s, const std::string& msg);
ata_status cuda_fail(cudaError_t e, const char* what);

// lda: leading dimension of A (X of a general product); ldb, ldc: of Y and of
// the dense C of a general product (unused for A^t A plans).
void append_plan_tables(const Plan& P, int inst, int64_t lda, HostTables* h, int64_t ldb = 0, int64_t ldc = 0);
void finalize_tables(HostTables* h, int8_t in_dt, int8_t sum_dt);
ata_status upload_tables(const HostTables& h, DeviceTables* d);
ata_status enqueue_tables(const DeviceTables& t, const Bind* binds, int nb, cudaStream_t s,
                          const cudaEvent_t* ev = nullptr);
ata_status launch_via_graph(const DeviceTables& t, const Bind* binds, int nb, GraphCache* g, cudaStream_t s);

// Tensor-core leaf launch (bf16x3 / TF32 / FP64 emulation).
ata_status launch_leaf_tc(const DeviceTables& t, const Bind* binds, int nb, cudaStream_t s,
                          cudaEvent_t before_gemm = nullptr);
ata_status build_tc_tables(const HostTables& h, const std::vector<char*>& ws, DeviceTables* d);
bool leaf_supported(LeafKind k);
// Row tile of the tensor-core kernel that runs plan P on this device.
int tc_rows_for(const Plan& P);

// Planner defaults and the autotuner.
int default_cutoff(int64_t m, int64_t n, ata_dtype dtype);
int default_fuse_levels(ata_dtype dtype, int variant);
// r >= 0 tunes the general product X^t Y (X: m x n, Y: m x r) instead.
ata_status autotune_cutoff(int64_t m, int64_t n, ata_dtype dtype, int variant, PlanOptions* o, int64_t r = -1);
// The cost model's cutoff candidates for plan options o, fastest first,
// among the plans whose workspace fits the cap.
std::vector<std::pair<double, int>> rank_cutoffs(int64_t m, int64_t n, ata_dtype dtype, const PlanOptions& o,
                                                 int64_t r);
// The same for an automatic plan shape: fewer Strassen levels where the
// depth is free and no cutoff fits the cap, else the smallest workspace;
// *max_levels receives the level cap of the ranked plans.
std::vector<std::pair<double, int>> rank_plans(int64_t m, int64_t n, ata_dtype dtype, const PlanOptions& o,
                                               int64_t r, int* max_levels);

// Executions of a plan run one at a time, whatever streams they are queued
// on: they share its workspace, leaf tile counter and status word.  Before
// an execution, order_wait makes its stream wait for the latest earlier
// execution of every plan it uses that ran on another stream; after it,
// order_record records `ev` (the plan's own event, or a batch's) on the
// stream as their latest.  Both do nothing on a capturing stream.
struct OrderEvent {
    cudaEvent_t e = nullptr;
    ~OrderEvent();
};
ata_status order_wait(const ata_plan* plans, int count, cudaStream_t s);
ata_status order_record(const ata_plan* plans, int count, cudaStream_t s, std::shared_ptr<OrderEvent>* ev);
// Waits on the host until the plan's latest execution has finished.
ata_status order_sync(ata_plan p);
// True when s is capturing a CUDA graph.
bool stream_capturing(cudaStream_t s);

// Plan accessors (runtime.cu) and batch-cache maintenance (batched.cu).
const Plan& plan_of(ata_plan p);
Bind make_bind(ata_plan p, const void* A, int64_t lda, double* C);
// An execution launched directly on s (no graph capture; see runtime.cu).
ata_status execute_direct(ata_plan plan, const void* A, int64_t lda, double* C_packed, cudaStream_t s,
                          int* kernels);
uint64_t plan_id(ata_plan p);
char* plan_workspace(ata_plan p);
ata_dtype plan_dtype(ata_plan p);
void forget_plan_in_batches(uint64_t id);

}  // namespace ata
