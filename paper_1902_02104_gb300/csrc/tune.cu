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
std::map<std::tuple<int64_t, int64_t, int64_t, int, int, int, int, int>, int> g_tuned;

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

ata_status autotune_cutoff(int64_t m, int64_t n, ata_dtype dtype, int variant, PlanOptions* o, int64_t r) {
    const auto key = std::make_tuple(m, n, r, (int)dtype, variant, o->fuse_levels, o->max_levels, (int)o->cta_pair);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            o->cutoff = it->second;
            return ATA_OK;
        }
    }
    static const int cands[] = {64, 96, 128, 160, 192, 256, 320, 384, 512, 768, 1024, 1536, 2048, 3072, 4096};
    double best = 1e300;
    int best_c = o->cutoff;
    for (int c : cands) {
        if (r < 0 && estimate_products(m, n, c) > kMaxLeafProducts) continue;
        if (dtype != ATA_F64 && c < 256) continue;  // tensor-core tiles are 128 x 128
        PlanOptions t = *o;
        t.cutoff = c;
        Plan P;
        std::string err;
        if (!(r < 0 ? build_plan(m, n, t, &P, &err) : build_gemm_plan(m, n, r, t, &P, &err))) continue;
        if ((int64_t)P.products.size() > kMaxLeafProducts) continue;
        if (P.ws_bytes > kWorkspaceCap) continue;
        bool terms_ok = true;
        for (const LeafProduct& lp : P.products) terms_ok = terms_ok && lp.nx <= kMaxTerms && lp.ny <= kMaxTerms;
        if (!terms_ok) continue;
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
