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
#include <tuple>

#include "runtime.h"

namespace ata {
namespace {

struct Rates {
    double leaf_fma;   // leaf multiply-adds per second (of the A^t A scalar product)
    double add;        // Strassen sum / combine additions per second
    double hbm;        // bytes per second
};

Rates rates_for(ata_dtype d) {
    switch (d) {
        case ATA_F64: return {0.60e12, 0.50e12, 6.0e12};
        case ATA_F32_BF16X3: return {1.9e15 / 2 / 6, 35e12, 6.0e12};
        case ATA_F32_TF32: return {1.0e15 / 2, 35e12, 6.0e12};
        case ATA_F64_OZAKI: return {1.9e15 / 2 / 15, 0.5e12, 6.0e12};
    }
    return {0.6e12, 0.5e12, 6e12};
}

constexpr int64_t kWorkspaceCap = int64_t(48) << 30;  // bytes
constexpr int64_t kMaxLeafProducts = 400000;

double model_time(const Plan& P, ata_dtype d) {
    const Rates r = rates_for(d);
    return (double)P.stats.mults / r.leaf_fma + (double)P.stats.adds / r.add + 2.0 * (double)P.ws_bytes / r.hbm +
           2e-6 * (double)(P.split_levels.size() + P.combine_levels.size() + 1);
}

// Leaf products a cutoff would create, estimated without building the plan:
// every off-diagonal block at depth d has 7^s leaves.
double estimate_products(int64_t m, int64_t n, int cutoff) {
    double total = 0;
    int64_t w = n, md = m;
    for (int d = 0; d < 40 && std::min(md, w) > cutoff; ++d) {
        int64_t p = (w + 1) / 2, q = (md + 1) / 2, r = w / 2;
        int s = 0;
        while (std::min(p, std::min(q, r)) > cutoff) {
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
std::map<std::tuple<int64_t, int64_t, int, int>, int> g_tuned;

}  // namespace

int default_fuse_levels(ata_dtype dtype, int variant) {
    (void)variant;
    // FP64: additions run on the same FP64 pipe as the leaf DFMAs, so sums
    // recomputed per tile cost more than materialising them once.
    if (dtype == ATA_F64 || dtype == ATA_F64_OZAKI) return 0;
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

ata_status autotune_cutoff(int64_t m, int64_t n, ata_dtype dtype, int variant, PlanOptions* o) {
    const auto key = std::make_tuple(m, n, (int)dtype, variant);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            o->cutoff = it->second;
            return ATA_OK;
        }
    }
    static const int cands[] = {64, 96, 128, 160, 192, 256, 320, 384, 512, 768, 1024, 1536, 2048};
    double best = 1e300;
    int best_c = o->cutoff;
    for (int c : cands) {
        if (estimate_products(m, n, c) > kMaxLeafProducts) continue;
        PlanOptions t = *o;
        t.cutoff = c;
        Plan P;
        std::string err;
        if (!build_plan(m, n, t, &P, &err)) continue;
        if (P.ws_bytes > kWorkspaceCap) continue;
        const double tm = model_time(P, dtype);
        if (tm < best) {
            best = tm;
            best_c = c;
        }
    }
    o->cutoff = best_c;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best_c;
    return ATA_OK;
}

}  // namespace ata
