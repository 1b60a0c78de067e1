// tune.cu -- planner defaults and cutoff selection.
//
// The cutoff replaces the paper's fixed base-case size of 32 (Algorithm 1).
// Selection is by a cost model of the plan the planner actually builds:
//   time = leaf multiply-adds / leaf rate + Strassen additions / add rate
//          + workspace traffic / HBM rate,
// with the rates of this part (FP64: 1.2 TFLOP/s DFMA, 0.5 Gop/s... per
// second DADD; tensor-core modes: the MMA rate of the leaf arithmetic),
// subject to a workspace cap.  Candidates whose trees would exceed a task
// budget are skipped.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <set>
#include <tuple>

#include "runtime.h"

namespace ata {
namespace {

struct Rates {
    double leaf_fma;   // leaf multiply-adds per second (of the A^t A scalar product)
    double add;        // Strassen sum / combine additions per second
    double hbm;        // bytes per second
};

// Rates measured on GB300: DFMA leaves at ~90% of 1.26 TFLOP/s; tensor-core
// leaves at the measured fraction of the 1.89 PFLOP/s bf16 (0.93 tf32) peak
// (0.75 FP64 emulation, 0.68 bf16x3, 0.53 TF32) divided by the part
// products per scalar product (21, 6, 1); Strassen sums/combines on the
// FP64 (0.5 Gop/s) or FP32 pipe.
Rates rates_for(ata_dtype d) {
    switch (d) {
        case ATA_F64: return {0.57e12, 0.50e12, 6.0e12};
        case ATA_F32_BF16X3: return {1.89e15 * 0.68 / 2 / 6, 35e12, 6.0e12};
        case ATA_F32_TF32: return {0.93e15 * 0.53 / 2, 35e12, 6.0e12};
        case ATA_F64_OZAKI: return {1.89e15 * 0.75 / 2 / 21, 0.5e12, 6.0e12};
    }
    return {0.6e12, 0.5e12, 6e12};
}

// Bytes the operand preparation of the tensor-core leaves moves: every
// distinct leaf operand (operands with equal terms share one part buffer)
// reads its terms twice (column maxima, slicing) and writes its parts.
double prep_bytes(const Plan& P) {
    if (P.leaf == LEAF_F64) return 0.0;
    const TcGeom g = tc_geom(P.leaf);
    const double in = P.in_dt == DT_F64 ? 8.0 : 4.0;
    // a fused operand sum reads each of its nt terms in both passes
    double bytes = 0;
    std::set<int64_t> seen;
    for (const LeafProduct& lp : P.products) {
        if (seen.insert(lp.tc_x_off).second)
            bytes += (double)lp.K_pad * lp.p_pad * (2.0 * in * lp.nx + g.parts * g.elem);
        if (lp.out_kind != OUT_SYRK && seen.insert(lp.tc_y_off).second)
            bytes += (double)lp.K_pad * lp.r_pad * (2.0 * in * lp.ny + g.parts * g.elem);
    }
    return bytes;
}

constexpr int64_t kWorkspaceCap = int64_t(48) << 30;  // bytes
constexpr int64_t kMaxLeafProducts = 400000;

double model_time(const Plan& P, ata_dtype d) {
    const Rates r = rates_for(d);
    // tensor-core leaves compute on whole tiles (128 x 128, or 256 x 128 for
    // CTA pairs)
    // FP64 leaves skip padding in 16 x 32 warp blocks (upper blocks only on
    // diagonal leaves), so they pay for whole blocks
    double leaf = 0;
    if (P.leaf == LEAF_F64) {
        for (const LeafProduct& lp : P.products) {
            const double rb = std::ceil(lp.out_rows / 16.0), cb = std::ceil(lp.out_cols / 32.0);
            const double blocks = lp.out_kind == OUT_SYRK ? rb * cb / 2 + std::min(rb, cb) / 2 : rb * cb;
            leaf += blocks * 16.0 * 32.0 * lp.K;
        }
    } else {
        leaf = 0;
        const int tm = P.tc_tile_rows > 0 ? P.tc_tile_rows : kTcTile, tn = tc_cols_for(P.leaf, tm);
        for (const LeafProduct& lp : P.products)
            leaf += (double)leaf_tiles(lp, tm, tn) * tm * tn * lp.K_pad;
    }
    return leaf / r.leaf_fma + (double)P.stats.adds / r.add + 2.0 * (double)P.ws_bytes / r.hbm +
           prep_bytes(P) / (0.5 * r.hbm) + 2e-6 * (double)(P.split_levels.size() + P.combine_levels.size() + 1);
}

// Leaf products a cutoff would create, estimated without building the plan:
// every off-diagonal block at depth d has 7^s leaves (s <= max_levels).
double estimate_products(int64_t m, int64_t n, int cutoff, int max_levels) {
    double total = 0;
    int64_t w = n, md = m;
    for (int d = 0; d < 40 && std::min(md, w) > cutoff; ++d) {
        int64_t p = (w + 1) / 2, q = (md + 1) / 2, r = w / 2;
        int s = 0;
        while (s < max_levels && std::min(p, std::min(q, r)) > cutoff) {
            p = (p + 1) / 2;
            q = (q + 1) / 2;
            r = (r + 1) / 2;
            ++s;
        }
        total += std::pow(2.0, d) * std::pow(7.0, s);
        w = (w + 1) / 2;
        md = (md + 1) / 2;
    }
    return total;
}

std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int64_t, int64_t, int, int, int, int, int>, std::pair<int, int>> g_tuned;

}  // namespace

int default_fuse_levels(ata_dtype dtype, int variant) {
    // FP64: additions run on the same FP64 pipe as the leaf DFMAs, so sums
    // recomputed per tile cost more than materialising them once.
    if (dtype == ATA_F64) return 0;
    // The FP64 emulation forms the bottom level's operand sums in fixed point
    // while slicing them.  Their scale is bounded from the blocks' maxima, one
    // bit above the largest for a two-term Strassen sum; Winograd's chained
    // sums (up to four terms) would lose two of the 48 bits, so its sums stay
    // materialised in FP64 and sliced at their exact scale.
    if (dtype == ATA_F64_OZAKI) return variant == ATA_WINOGRAD ? 0 : 1;
    return 1;
}

int default_cutoff(int64_t m, int64_t n, ata_dtype dtype) {
    (void)m;
    (void)n;
    switch (dtype) {
        case ATA_F64: return 256;
        default: return 1024;
    }
}

namespace {

constexpr int kCutoffs[] = {64, 96, 128, 160, 192, 256, 320, 384, 512, 768, 1024, 1536, 2048, 3072, 4096};

// Builds the plan of cutoff c under options o into *P; false when the
// leaf kernels would not accept it (product count, fused terms per operand).
bool candidate_plan(int64_t m, int64_t n, ata_dtype dtype, const PlanOptions& o, int64_t r, int c, Plan* P) {
    if (r < 0 && estimate_products(m, n, c, o.max_levels) > kMaxLeafProducts) return false;
    if (dtype != ATA_F64 && c < 256) return false;  // tensor-core tiles are 128 x 128
    PlanOptions t = o;
    t.cutoff = c;
    std::string err;
    if (!(r < 0 ? build_plan(m, n, t, P, &err) : build_gemm_plan(m, n, r, t, P, &err))) return false;
    if ((int64_t)P->products.size() > kMaxLeafProducts) return false;
    for (const LeafProduct& lp : P->products)
        if (lp.nx > kMaxTerms || lp.ny > kMaxTerms) return false;
    return true;
}

}  // namespace

// Cutoff candidates ranked by the cost model (fastest first), among the
// plans whose workspace fits kWorkspaceCap.
std::vector<std::pair<double, int>> rank_cutoffs(int64_t m, int64_t n, ata_dtype dtype, const PlanOptions& o,
                                                 int64_t r) {
    std::vector<std::pair<double, int>> out;
    for (int c : kCutoffs) {
        Plan P;
        if (!candidate_plan(m, n, dtype, o, r, c, &P) || P.ws_bytes > kWorkspaceCap) continue;
        out.push_back({model_time(P, dtype), c});
    }
    std::stable_sort(out.begin(), out.end(),
                     [](const std::pair<double, int>& a, const std::pair<double, int>& b) { return a.first < b.first; });
    return out;
}

// Ranked cutoffs for an automatic plan shape.  Every Strassen level
// materialises the operand sums and outputs of all its products at once, so
// a large product may fit the workspace cap only with fewer levels: when no
// cutoff fits and the caller left the depth free (max_levels >= kFreeLevels),
// the level cap is lowered until one does.  When none fits even without
// Strassen levels, the cutoff with the smallest workspace is the one
// candidate (creating the plan then succeeds wherever the device holds it).
// *max_levels receives the level cap the ranking used.
std::vector<std::pair<double, int>> rank_plans(int64_t m, int64_t n, ata_dtype dtype, const PlanOptions& o,
                                               int64_t r, int* max_levels) {
    *max_levels = o.max_levels;
    auto ranked = rank_cutoffs(m, n, dtype, o, r);
    if (!ranked.empty()) return ranked;
    PlanOptions t = o;
    if (o.max_levels >= kFreeLevels) {
        for (int lv = 3; lv >= 0 && ranked.empty(); --lv) {
            t.max_levels = lv;
            ranked = rank_cutoffs(m, n, dtype, t, r);
            if (!ranked.empty()) *max_levels = lv;
        }
        if (!ranked.empty()) return ranked;
        t.max_levels = 0;
    }
    int64_t best_ws = -1;
    int best_c = 0;
    for (int c : kCutoffs) {
        Plan P;
        if (!candidate_plan(m, n, dtype, t, r, c, &P)) continue;
        if (best_ws < 0 || P.ws_bytes < best_ws) {
            best_ws = P.ws_bytes;
            best_c = c;
        }
    }
    if (best_ws >= 0) {
        ranked.push_back({0.0, best_c});
        *max_levels = t.max_levels;
    }
    return ranked;
}

ata_status autotune_cutoff(int64_t m, int64_t n, ata_dtype dtype, int variant, PlanOptions* o, int64_t r) {
    const auto key = std::make_tuple(m, n, r, (int)dtype, variant, o->fuse_levels, o->max_levels, (int)o->cta_pair);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            o->cutoff = it->second.first;
            o->max_levels = it->second.second;
            return ATA_OK;
        }
    }
    int levels = o->max_levels;
    const auto ranked = rank_plans(m, n, dtype, *o, r, &levels);
    if (!ranked.empty()) {
        o->cutoff = ranked.front().second;
        o->max_levels = levels;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = {o->cutoff, o->max_levels};
    return ATA_OK;
}

}  // namespace ata

// ---------------------------------------------------------------------------
// Measured tuning (ata_tune): the cost model ranks the cutoffs; the best few,
// and single-CTA against CTA-pair tiles in the tensor-core modes, are timed
// on this device with CUDA events on a synthetic input of the exact shape,
// and the fastest wins.  Results are cached per (shape, dtype, options).

namespace ata {
namespace {

// Deterministic fill of the tuning input: values in [-1, 1) from a 64-bit
// integer hash of the index (timing does not depend on them, but they
// exercise every slice and every column scale).
__global__ void tune_fill_kernel(void* A, int64_t count, int f64) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull;
        h ^= h >> 31;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 29;
        const double v = (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0;
        if (f64)
            static_cast<double*>(A)[i] = v;
        else
            static_cast<float*>(A)[i] = (float)v;
    }
}

struct TuneKey {
    int device;
    int64_t m, n;
    int dtype, variant, fuse, max_levels, cta_pair;
    bool operator<(const TuneKey& o) const {
        return std::tie(device, m, n, dtype, variant, fuse, max_levels, cta_pair) <
               std::tie(o.device, o.m, o.n, o.dtype, o.variant, o.fuse, o.max_levels, o.cta_pair);
    }
};
std::map<TuneKey, std::pair<ata_plan_options, float>> g_measured;

}  // namespace
}  // namespace ata

extern "C" ata_status ata_tune(int64_t m, int64_t n, ata_dtype dtype, const ata_plan_options* base, int candidates,
                               ata_plan_options* out, float* best_ms) {
    using namespace ata;
    NvtxRange nv("ata_tune");
    if (!out) return fail(ATA_EINVAL, "out is NULL");
    if (candidates < 1 || candidates > 8) return fail(ATA_EINVAL, "candidates must be in [1, 8]");
    ata_plan_options u;
    if (base) {
        u = *base;
    } else {
        u.cutoff = 0;
        u.variant = -1;
        u.fuse_levels = -1;
        u.max_strassen_levels = -1;
        u.cta_pair = -1;
        u.wait_limit_us = -1;
    }
    u.cutoff = 0;
    const bool tune_pair = u.cta_pair < 0;
    ata_plan_info info;
    ata_status st = ata_plan_query_opts(m, n, dtype, &u, &info);  // validates the arguments
    if (st != ATA_OK) return st;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    const TuneKey key{device, m, n, (int)dtype, u.variant, u.fuse_levels, u.max_strassen_levels, u.cta_pair};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_measured.find(key);
        if (it != g_measured.end()) {
            *out = it->second.first;
            if (best_ms) *best_ms = it->second.second;
            return ATA_OK;
        }
    }
    // candidate cutoffs: the model's best `candidates` (with the options as
    // the plan would resolve them)
    PlanOptions o;
    o.leaf = dtype == ATA_F64 ? LEAF_F64 : dtype == ATA_F32_BF16X3 ? LEAF_BF16X3 : dtype == ATA_F32_TF32 ? LEAF_TF32 : LEAF_OZAKI;
    o.variant = u.variant < 0 ? ATA_STRASSEN : u.variant;
    o.fuse_levels = u.fuse_levels >= 0 ? u.fuse_levels : default_fuse_levels(dtype, o.variant);
    o.max_levels = u.max_strassen_levels >= 0 ? u.max_strassen_levels : kFreeLevels;
    o.cta_pair = u.cta_pair == 1 || (u.cta_pair < 0 && dtype == ATA_F32_TF32);
    int levels = o.max_levels;
    auto ranked = rank_plans(m, n, dtype, o, -1, &levels);
    if (ranked.empty()) ranked.push_back({0.0, info.cutoff});
    if ((int)ranked.size() > candidates) ranked.resize(candidates);
    std::vector<ata_plan_options> cands;
    for (const auto& rc : ranked) {
        ata_plan_options c = u;
        c.cutoff = rc.second;
        if (levels < kFreeLevels) c.max_strassen_levels = levels;
        if (dtype == ATA_F64 || !tune_pair) {
            cands.push_back(c);
        } else {
            c.cta_pair = 0;
            cands.push_back(c);
            c.cta_pair = 1;
            cands.push_back(c);
        }
    }
    // synthetic input of the exact shape and an output buffer
    const int es = (dtype == ATA_F64 || dtype == ATA_F64_OZAKI) ? 8 : 4;
    void* A = nullptr;
    double* C = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (s) cudaStreamSynchronize(s);
        dev_free(A);
        dev_free(C);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    };
    const int64_t a_elems = std::max<int64_t>(m * n, 1), c_elems = std::max<int64_t>(n * (n + 1) / 2, 1);
    if (dev_malloc(&A, (size_t)a_elems * es) != cudaSuccess || dev_malloc(&C, (size_t)c_elems * 8) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(ATA_ENOMEM, "tuning buffers");
    }
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return cuda_fail(cudaGetLastError(), "tuning stream/events");
    }
    tune_fill_kernel<<<1024, 256, 0, s>>>(A, a_elems, es == 8);
    float best = 1e30f;
    ata_plan_options best_o = cands.front();
    st = ATA_OK;
    for (const ata_plan_options& c : cands) {
        ata_plan p = nullptr;
        ata_status cs = ata_plan_create_opts(&p, m, n, dtype, &c);
        if (cs == ATA_ENOMEM) continue;  // a candidate that does not fit is skipped
        if (cs != ATA_OK) {
            st = cs;
            break;
        }
        float times[3];
        for (int rep = 0; rep < 4 && cs == ATA_OK; ++rep) {
            if (rep > 0 && cudaEventRecord(e0, s) != cudaSuccess) cs = ATA_ECUDA;
            if (cs == ATA_OK) cs = ata_execute(p, A, n, C, s);
            if (cs == ATA_OK && rep > 0) {
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&times[rep - 1], e0, e1) != cudaSuccess)
                    cs = ATA_ECUDA;
            }
        }
        ata_plan_destroy(p);
        if (cs != ATA_OK) {
            st = cs;
            break;
        }
        std::sort(times, times + 3);
        if (times[1] < best) {
            best = times[1];
            best_o = c;
        }
    }
    cleanup();
    if (st != ATA_OK) return st;
    if (best >= 1e30f) return fail(ATA_ENOMEM, "no tuning candidate fits on the device");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_measured[key] = {best_o, best};
    }
    *out = best_o;
    if (best_ms) *best_ms = best;
    return ATA_OK;
}
