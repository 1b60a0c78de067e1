// noalloc.cu -- ata_execute_static_scratch: the FP64 path with its scratch
// memory taken from a fixed array compiled into this library.
//
// Some callers must not allocate device memory while they run: code that is
// about to capture work into a CUDA graph, services that fix their memory
// footprint at start-up and treat any later cudaMalloc as a fault, and hosts
// whose device memory belongs to another allocator (a framework's caching
// pool) that this library must not bypass.  For them this entry point runs
// the same split -> leaf -> combine kernels as ata_execute, but the task
// tables, the leaf tile counter and the Strassen workspace all live in
// g_ata_scratch below, a file-scope device array of kScratchBytes that every
// GPU loading the library holds until the process exits.  The caller still
// passes A and C.  Nothing here calls cudaMalloc, cudaFree, a graph API or
// any other allocating routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.h"

namespace ata {
namespace {

constexpr int64_t kScratchBytes = int64_t(64) << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) char g_ata_scratch[kScratchBytes];

std::mutex g_setup_mu;
char* g_scratch_addr[kMaxDevices] = {};

// Device address of g_ata_scratch on the current device.  In host code the
// symbol itself is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.
ata_status scratch_address(char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(ATA_EUNSUPPORTED, "device ordinal beyond the scratch table");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ata_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_ata_scratch)");
        g_scratch_addr[dev] = static_cast<char*>(p);
    }
    *out = g_scratch_addr[dev];
    return ATA_OK;
}

int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace ata

using namespace ata;

extern "C" ata_status ata_execute_static_scratch(int64_t m, int64_t n, const double* A, int64_t lda,
                                                 double* C_packed, int cutoff, void* stream) {
    if (m < 0 || n < 0) return fail(ATA_EINVAL, "m and n must be >= 0");
    if (lda < n || lda < 1) return fail(ATA_EINVAL, "lda must be >= max(n, 1)");
    if (cutoff < 16 || cutoff > 4096) return fail(ATA_EINVAL, "cutoff must be in [16, 4096]");
    if (m > 0 && n > 0 && !A) return fail(ATA_EINVAL, "A is NULL");
    if (n > 0 && !C_packed) return fail(ATA_EINVAL, "C_packed is NULL");
    if (reinterpret_cast<uintptr_t>(A) % 8 || reinterpret_cast<uintptr_t>(C_packed) % 8)
        return fail(ATA_EINVAL, "A and C_packed must be 8-byte aligned");
    if (n == 0) return ATA_OK;
    {
        // The task tables are copied from a host buffer that lives only for
        // this call; a copy recorded into a graph under capture would read it
        // after it is gone.
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
        if (cs != cudaStreamCaptureStatusNone)
            return fail(ATA_EINVAL, "the stream is capturing: this call copies its tables from a temporary host "
                                    "buffer and cannot be recorded");
    }

    char* scratch = nullptr;
    ata_status st = scratch_address(&scratch);
    if (st != ATA_OK) return st;

    PlanOptions o;
    o.cutoff = cutoff;
    o.variant = 0;
    o.leaf = LEAF_F64;
    o.fuse_levels = 0;
    Plan P;
    std::string err;
    if (!build_plan(m, n, o, &P, &err)) return fail(ATA_EINVAL, err);

    HostTables h;
    h.leaf = LEAF_F64;
    h.split_pending.resize(P.split_levels.size());
    h.comb_pending.resize(P.combine_levels.size());
    append_plan_tables(P, 0, lda, &h);
    finalize_tables(&h, P.in_dt, P.sum_dt);

    // scratch layout: [tables | tile counter | Strassen workspace]
    int64_t off = 0;
    auto place = [&](int64_t bytes) {
        const int64_t o2 = off;
        off = align256(off + bytes);
        return o2;
    };
    const int64_t o_terms = place(h.terms.size() * sizeof(Term));
    const int64_t o_prods = place(h.prods.size() * sizeof(LeafProduct));
    const int64_t o_tiles = place(h.tiles.size() * sizeof(LeafTile));
    const int64_t o_cnt = place(256);
    const int64_t o_split = place(h.split.size() * sizeof(SplitTask));
    const int64_t o_schunk = place(h.split_chunks.size() * sizeof(Chunk));
    const int64_t o_comb = place(h.comb.size() * sizeof(CombineTask));
    const int64_t o_cchunk = place(h.comb_chunks.size() * sizeof(Chunk));
    const int64_t o_psum = place(h.partial_sums.size() * sizeof(PartialSum));
    const int64_t tables_bytes = off;
    const int64_t o_ws = place(P.ws_bytes);
    if (off > kScratchBytes)
        return fail(ATA_EINVAL, "problem needs " + std::to_string(off) + " bytes of scratch; the static scratch holds " +
                                    std::to_string(kScratchBytes) + " bytes (use ata_execute, or a larger cutoff)");

    std::vector<char> hb(tables_bytes, 0);
    auto put = [&](int64_t o2, const void* src, size_t bytes) {
        if (bytes) std::memcpy(hb.data() + o2, src, bytes);
    };
    put(o_terms, h.terms.data(), h.terms.size() * sizeof(Term));
    put(o_prods, h.prods.data(), h.prods.size() * sizeof(LeafProduct));
    put(o_tiles, h.tiles.data(), h.tiles.size() * sizeof(LeafTile));
    put(o_split, h.split.data(), h.split.size() * sizeof(SplitTask));
    put(o_schunk, h.split_chunks.data(), h.split_chunks.size() * sizeof(Chunk));
    put(o_comb, h.comb.data(), h.comb.size() * sizeof(CombineTask));
    put(o_cchunk, h.comb_chunks.data(), h.comb_chunks.size() * sizeof(Chunk));
    put(o_psum, h.partial_sums.data(), h.partial_sums.size() * sizeof(PartialSum));

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The tables overwrite whatever the previous call left in the array; the
    // tile counter (zeroed by the copy of hb) must start at zero.
    cudaError_t e = cudaMemcpyAsync(scratch, hb.data(), tables_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(tables -> static scratch)");

    DeviceTables t;
    t.leaf = LEAF_F64;
    t.blob = nullptr;  // not owned: nothing to free
    t.terms = reinterpret_cast<Term*>(scratch + o_terms);
    t.prods = reinterpret_cast<LeafProduct*>(scratch + o_prods);
    t.tiles = reinterpret_cast<LeafTile*>(scratch + o_tiles);
    t.counter = reinterpret_cast<int*>(scratch + o_cnt);
    t.split = reinterpret_cast<SplitTask*>(scratch + o_split);
    t.split_chunks = reinterpret_cast<Chunk*>(scratch + o_schunk);
    t.comb = reinterpret_cast<CombineTask*>(scratch + o_comb);
    t.comb_chunks = reinterpret_cast<Chunk*>(scratch + o_cchunk);
    t.partial_sums = reinterpret_cast<PartialSum*>(scratch + o_psum);
    t.npartial_sums = (int)h.partial_sums.size();
    t.ntiles = (int)h.tiles.size();
    t.split_lv = h.split_lv;
    t.comb_lv = h.comb_lv;
    Bind b{};
    b.A = A;
    b.C = C_packed;
    b.W = scratch + o_ws;
    b.n = n;
    return enqueue_tables(t, &b, 1, s);
}
