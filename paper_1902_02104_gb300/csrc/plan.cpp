// plan.cpp -- host recursion planner (see plan.h).
#include "plan.h"

#include <algorithm>
#include <map>
#include <cstring>

namespace ata {
namespace {

constexpr int64_t kAlign = 256;  // bytes; every workspace buffer starts on this boundary

// Block-coefficient tables of the seven products (Section 4.2.2, with M1 and
// M7 in Strassen's own form; Winograd's variant as S1..S4 / T1..T4).
// Blocks of a K x c operand are indexed b = 2*kb + cb (kb: K half, cb:
// column half).  The left factor of a product is X^t, so its block (a, b)
// is X's block (b, a)^t.  coef[variant][side][product][block].
const int8_t kCoef[2][2][7][4] = {
    {   // Strassen
        {   // side X (left factor X^t): L11=B0, L12=B2, L21=B1, L22=B3
            {1, 0, 0, 1},    // M1: L11 + L22
            {0, 1, 0, 1},    // M2: L21 + L22
            {1, 0, 0, 0},    // M3: L11
            {0, 0, 0, 1},    // M4: L22
            {1, 0, 1, 0},    // M5: L11 + L12
            {-1, 1, 0, 0},   // M6: L21 - L11
            {0, 0, 1, -1},   // M7: L12 - L22
        },
        {   // side Y (right factor): R11=B0, R12=B1, R21=B2, R22=B3
            {1, 0, 0, 1},    // M1: R11 + R22
            {1, 0, 0, 0},    // M2: R11
            {0, 1, 0, -1},   // M3: R12 - R22
            {-1, 0, 1, 0},   // M4: R21 - R11
            {0, 0, 0, 1},    // M5: R22
            {1, 1, 0, 0},    // M6: R11 + R12
            {0, 0, 1, 1},    // M7: R21 + R22
        },
    },
    {   // Winograd
        {   // side X: S1 = L21 + L22, S2 = S1 - L11, S3 = L11 - L21, S4 = L12 - S2
            {1, 0, 0, 0},    // M1: L11
            {0, 0, 1, 0},    // M2: L12
            {1, -1, 1, -1},  // M3: S4 = L12 - L21 - L22 + L11
            {0, 0, 0, 1},    // M4: L22
            {0, 1, 0, 1},    // M5: S1
            {-1, 1, 0, 1},   // M6: S2
            {1, -1, 0, 0},   // M7: S3
        },
        {   // side Y: T1 = R12 - R11, T2 = R22 - T1, T3 = R22 - R12, T4 = T2 - R21
            {1, 0, 0, 0},    // M1: R11
            {0, 0, 1, 0},    // M2: R21
            {0, 0, 0, 1},    // M3: R22
            {1, -1, -1, 1},  // M4: T4 = R22 - R12 + R11 - R21
            {-1, 1, 0, 0},   // M5: T1
            {1, -1, 0, 1},   // M6: T2
            {0, -1, 0, 1},   // M7: T3
        },
    },
};

// Products whose operand on `side` is a sum (materialised by a split task),
// in the order the split kernel writes them.
//   Strassen X: M1 M2 M5 M6 M7   Strassen Y: M1 M3 M4 M6 M7
//   Winograd X: M5(S1) M6(S2) M7(S3) M3(S4)   Winograd Y: M5(T1) M6(T2) M7(T3) M4(T4)
const int kSumProducts[2][2][5] = {
    {{0, 1, 4, 5, 6}, {0, 2, 3, 5, 6}},
    {{4, 5, 6, 2, -1}, {4, 5, 6, 3, -1}},
};
const int kNumSums[2] = {5, 4};

struct Target {
    int8_t kind;        // OUT_DENSE or OUT_PACKED
    int64_t off;        // dense: FP64 element offset in W
    int32_t ld;         // dense
    int32_t ci0, cj0;   // packed
};

struct Ctx {
    Plan* P;
    const PlanOptions* opt;
    int64_t ws = 0;
    // tensor-core part buffers by operand: equal operands (the same signed
    // terms, K and padding) share one buffer, prepared once
    std::map<std::vector<int64_t>, int64_t> parts;
    int64_t alloc(int64_t bytes) {
        int64_t off = ws;
        ws += (bytes + kAlign - 1) / kAlign * kAlign;
        return off;
    }
    int64_t parts_buffer(const std::vector<Term>& ts, int64_t K, int32_t rows_pad, int32_t K_pad, int8_t dt,
                         int64_t bytes) {
        std::vector<int64_t> key{K, rows_pad, K_pad, dt};
        for (const Term& t : ts) {
            key.push_back(t.off);
            key.push_back(t.ld);
            key.push_back(((int64_t)t.rows << 32) | (uint32_t)t.cols);
            key.push_back(t.buf * 16 + t.dt * 4 + t.neg);
        }
        auto it = parts.find(key);
        if (it != parts.end()) return it->second;
        const int64_t off = alloc(bytes);
        parts.emplace(std::move(key), off);
        return off;
    }
};

int elem_size(int8_t dt) { return dt == DT_F64 ? 8 : 4; }

std::vector<Term> sub_block(const std::vector<Term>& ts, int64_t kb, int64_t cb, int64_t K1, int64_t c1) {
    std::vector<Term> out;
    for (const Term& t : ts) {
        const int64_t r0 = kb * K1, col0 = cb * c1;
        const int64_t rows = std::min<int64_t>(std::max<int64_t>(t.rows - r0, 0), K1);
        const int64_t cols = std::min<int64_t>(std::max<int64_t>(t.cols - col0, 0), c1);
        if (rows <= 0 || cols <= 0) continue;  // an all-zero (padding) block adds nothing
        Term u = t;
        u.off = t.off + r0 * t.ld + col0;
        u.rows = (int32_t)rows;
        u.cols = (int32_t)cols;
        out.push_back(u);
    }
    return out;
}

void append_signed(std::vector<Term>* dst, const std::vector<Term>& src, int sign) {
    for (Term t : src) {
        if (sign < 0) t.neg ^= 1;
        dst->push_back(t);
    }
}

int strassen_levels(int64_t p, int64_t q, int64_t r, int cutoff, int max_levels) {
    int s = 0;
    while (s < max_levels && std::min(p, std::min(q, r)) > cutoff) {
        p = ceil_half(p);
        q = ceil_half(q);
        r = ceil_half(r);
        ++s;
    }
    return s;
}

void emit_leaf(Ctx& c, const std::vector<Term>& X, const std::vector<Term>& Y, int64_t p, int64_t r,
               int64_t K, const Target& out, int64_t out_rows, int64_t out_cols, bool syrk, int8_t x_dt,
               int8_t y_dt) {
    Plan& P = *c.P;
    LeafProduct lp{};
    lp.p = (int32_t)p;
    lp.r = (int32_t)r;
    lp.K = (int32_t)K;
    lp.x0 = (int32_t)P.terms.size();
    lp.nx = (int32_t)X.size();
    P.terms.insert(P.terms.end(), X.begin(), X.end());
    lp.y0 = (int32_t)P.terms.size();
    lp.ny = (int32_t)Y.size();
    P.terms.insert(P.terms.end(), Y.begin(), Y.end());
    lp.out_rows = (int32_t)out_rows;
    lp.out_cols = (int32_t)out_cols;
    lp.x_dt = x_dt;
    lp.y_dt = y_dt;
    if (P.leaf != LEAF_F64) {
        // split parts of both operands, K-major, zero padded to whole tiles
        const TcGeom g = tc_geom(P.leaf);
        // X rows of a leaf above one tile are padded to whole CTA-pair tiles
        // (256 rows); a SYRK leaf reads the same buffer as Y
        const int64_t xr = c.opt->cta_pair && p > kTcTile ? kTcPairRows : kTcTile;
        lp.p_pad = (int32_t)((p + xr - 1) / xr * xr);
        lp.r_pad = syrk ? lp.p_pad : (int32_t)((r + kTcTile - 1) / kTcTile * kTcTile);
        lp.K_pad = (int32_t)std::max<int64_t>((K + g.k_align - 1) / g.k_align * g.k_align, g.k_align);
        lp.tc_x_off = c.parts_buffer(X, K, lp.p_pad, lp.K_pad, x_dt, (int64_t)g.parts * lp.p_pad * lp.K_pad * g.elem);
        lp.tc_y_off = syrk ? lp.tc_x_off
                           : c.parts_buffer(Y, K, lp.r_pad, lp.K_pad, y_dt,
                                            (int64_t)g.parts * lp.r_pad * lp.K_pad * g.elem);
    }
    if (syrk) {
        lp.out_kind = OUT_SYRK;
        lp.ci0 = out.ci0;
        lp.cj0 = out.cj0;
        lp.work = K * p * (p + 1) / 2;
    } else {
        lp.out_kind = out.kind;
        lp.out_off = out.off;
        lp.out_ld = out.ld;
        lp.ci0 = out.ci0;
        lp.cj0 = out.cj0;
        lp.work = p * r * K;
    }
    P.stats.mults += lp.work;
    if (P.leaf == LEAF_F64) {
        // operand sums recomputed per tile by fused loads (64-wide tiles)
        const int64_t tiles_r = (r + 63) / 64, tiles_p = (p + 63) / 64;
        if (lp.nx > 1) P.stats.adds += (int64_t)(lp.nx - 1) * K * p * tiles_r;
        if (lp.ny > 1) P.stats.adds += (int64_t)(lp.ny - 1) * K * r * tiles_p;
    } else {
        // fused sums are formed once per element by the operand preparation
        if (lp.nx > 1) P.stats.adds += (int64_t)(lp.nx - 1) * K * p;
        if (lp.ny > 1) P.stats.adds += (int64_t)(lp.ny - 1) * K * r;
    }
    P.products.push_back(lp);
}

// Strassen expansion of out(p x r) = X^t Y (X: K x p, Y: K x r) at `level`
// of a tree with `s_total` levels.
void expand(Ctx& c, const std::vector<Term>& X, const std::vector<Term>& Y, int64_t p, int64_t q, int64_t r,
            int64_t K, int level, int s_total, const Target& out, int8_t x_dt, int8_t y_dt) {
    Plan& P = *c.P;
    if (level == s_total) {
        emit_leaf(c, X, Y, p, r, K, out, p, r, false, x_dt, y_dt);
        return;
    }
    const int v = P.variant;
    const int64_t p1 = ceil_half(p), r1 = ceil_half(r), K1 = ceil_half(K), q1 = ceil_half(q);
    std::vector<Term> Xb[4], Yb[4];
    for (int kb = 0; kb < 2; ++kb)
        for (int cb = 0; cb < 2; ++cb) {
            Xb[2 * kb + cb] = sub_block(X, kb, cb, K1, p1);
            Yb[2 * kb + cb] = sub_block(Y, kb, cb, K1, r1);
        }
    const bool mat = (level + 1) <= s_total - P.fuse_levels;
    std::vector<Term> childX[7], childY[7];
    int8_t cdt[2][7];
    for (int side = 0; side < 2; ++side) {
        const std::vector<Term>* blocks = side == 0 ? Xb : Yb;
        const std::vector<Term>& parent = side == 0 ? X : Y;
        const int64_t c1 = side == 0 ? p1 : r1;
        std::vector<Term>* child = side == 0 ? childX : childY;
        const int8_t parent_dt = side == 0 ? x_dt : y_dt;
        int sum_slot[7];
        for (int i = 0; i < 7; ++i) sum_slot[i] = -1;
        if (mat && parent.empty()) {
            // an all-padding operand: every child operand is zero as well
            for (int i = 0; i < 7; ++i) cdt[side][i] = parent_dt;
        } else if (mat) {
            // the parent operand is a single term here (a block of A or a
            // materialised buffer); one split task writes every sum
            SplitTask st{};
            st.src = parent.at(0);
            st.K1 = (int32_t)K1;
            st.c1 = (int32_t)c1;
            st.side = (int8_t)side;
            st.variant = (int8_t)v;
            st.dst_dt = P.sum_dt;
            st.nout = (int8_t)kNumSums[v];
            const int64_t bytes = K1 * c1 * elem_size(P.sum_dt);
            for (int s = 0; s < kNumSums[v]; ++s) {
                st.out_off[s] = c.alloc(bytes) / elem_size(P.sum_dt);
                sum_slot[kSumProducts[v][side][s]] = s;
            }
            if ((int)P.split_levels.size() <= level) P.split_levels.resize(level + 1);
            P.split_levels[level].push_back(st);
            P.stats.adds += (int64_t)kNumSums[v] * K1 * c1;
            for (int i = 0; i < 7; ++i) {
                if (sum_slot[i] >= 0) {
                    Term t{};
                    t.off = st.out_off[sum_slot[i]];
                    t.ld = c1;
                    t.rows = (int32_t)K1;
                    t.cols = (int32_t)c1;
                    t.buf = BUF_W;
                    t.dt = P.sum_dt;
                    child[i].push_back(t);
                    cdt[side][i] = P.sum_dt;
                } else {
                    for (int b = 0; b < 4; ++b)
                        if (kCoef[v][side][i][b] != 0) append_signed(&child[i], blocks[b], kCoef[v][side][i][b]);
                    cdt[side][i] = parent_dt;
                }
            }
        } else {
            for (int i = 0; i < 7; ++i) {
                for (int b = 0; b < 4; ++b)
                    if (kCoef[v][side][i][b] != 0) append_signed(&child[i], blocks[b], kCoef[v][side][i][b]);
                cdt[side][i] = parent_dt;
            }
        }
    }
    // seven child results, contiguous FP64 p1 x r1 buffers
    const int64_t msz = p1 * r1;
    const int64_t m_off = c.alloc(7 * msz * 8) / 8;
    CombineTask ct{};
    ct.m_off = m_off;
    ct.p = (int32_t)p;
    ct.r = (int32_t)r;
    ct.p1 = (int32_t)p1;
    ct.r1 = (int32_t)r1;
    ct.dst_kind = out.kind;
    ct.variant = (int8_t)v;
    ct.dst_ld = out.ld;
    ct.dst_off = out.off;
    ct.ci0 = out.ci0;
    ct.cj0 = out.cj0;
    if ((int)P.combine_levels.size() <= level) P.combine_levels.resize(level + 1);
    P.combine_levels[level].push_back(ct);
    P.stats.adds += (v == 0 ? 8 : 7) * msz;
    for (int i = 0; i < 7; ++i) {
        Target t{};
        t.kind = OUT_DENSE;
        t.off = m_off + i * msz;
        t.ld = (int32_t)r1;
        expand(c, childX[i], childY[i], p1, q1, r1, K1, level + 1, s_total, t, cdt[0][i], cdt[1][i]);
    }
}

Term a_block(const Plan& P, int64_t c0, int64_t w) {
    Term t{};
    t.off = c0;
    t.ld = P.n;  // planned for a dense A; the runtime rebases to the caller's lda
    t.rows = (int32_t)P.m;
    t.cols = (int32_t)w;
    t.buf = BUF_A;
    t.dt = P.in_dt;
    return t;
}

void recurse_columns(Ctx& c, int64_t c0, int64_t w, int depth) {
    Plan& P = *c.P;
    int64_t m_d = P.m;
    for (int i = 0; i < depth; ++i) m_d = ceil_half(m_d);
    P.stats.depth = std::max(P.stats.depth, depth);
    if (std::min(m_d, w) <= P.cutoff) {
        // base case of Algorithm 1: the classical product on the diagonal block
        std::vector<Term> X{a_block(P, c0, w)};
        Target t{};
        t.kind = OUT_PACKED;
        t.ci0 = (int32_t)c0;
        t.cj0 = (int32_t)c0;
        emit_leaf(c, X, X, w, w, P.m, t, w, w, true, P.in_dt, P.in_dt);
        P.stats.n_diag_leaves++;
        return;
    }
    const int64_t n1 = ceil_half(w), n2 = w / 2;
    // off-diagonal block C_12 = A_L^t A_R over all m rows
    const int64_t q = ceil_half(m_d);
    const int s = strassen_levels(n1, q, n2, P.cutoff, P.max_levels);
    P.stats.max_strassen_levels = std::max(P.stats.max_strassen_levels, s);
    P.stats.n_nodes++;
    Target t{};
    t.kind = OUT_PACKED;
    t.ci0 = (int32_t)c0;
    t.cj0 = (int32_t)(c0 + n1);
    std::vector<Term> X{a_block(P, c0, n1)}, Y{a_block(P, c0 + n1, n2)};
    expand(c, X, Y, n1, q, n2, P.m, 0, s, t, P.in_dt, P.in_dt);
    recurse_columns(c, c0, n1, depth + 1);
    recurse_columns(c, c0 + n1, n2, depth + 1);
}

}  // namespace

TcGeom tc_geom(LeafKind k) {
    switch (k) {
        case LEAF_BF16X3: return {3, 2, 64};
        case LEAF_TF32: return {1, 4, 64};
        case LEAF_OZAKI: return {6, 2, 64};
        default: return {0, 8, 1};
    }
}

int64_t leaf_tiles(const LeafProduct& p, int tm, int tn) {
    const int64_t a = (p.out_rows + tm - 1) / tm, b = (p.out_cols + tn - 1) / tn;
    if (p.out_kind == OUT_SYRK) {
        // tiles that hold an upper entry: tile column tj from (ti * tm) / tn on
        int64_t cnt = 0;
        for (int64_t ti = 0; ti < a; ++ti) cnt += std::max<int64_t>(0, b - ti * tm / tn);
        return cnt;
    }
    return a * b;
}

namespace {

bool check_options(const PlanOptions& opt, std::string* err) {
    if (opt.cutoff < 16 || opt.cutoff > 4096) {
        *err = "cutoff must be in [16, 4096]";
        return false;
    }
    if (opt.variant != 0 && opt.variant != 1) {
        *err = "variant must be 0 (Strassen) or 1 (Winograd)";
        return false;
    }
    return true;
}

void start_plan(Plan& P, int64_t m, int64_t n, const PlanOptions& opt) {
    P = Plan();
    P.m = m;
    P.n = n;
    P.cutoff = opt.cutoff;
    P.variant = opt.variant;
    P.leaf = opt.leaf;
    P.in_dt = (opt.leaf == LEAF_F64 || opt.leaf == LEAF_OZAKI) ? DT_F64 : DT_F32;
    P.sum_dt = P.in_dt;
    P.fuse_levels = std::max(0, opt.fuse_levels);
    P.max_levels = std::max(0, opt.max_levels);
}

void finish_plan(Plan& P, const Ctx& c, const PlanOptions& opt) {
    P.ws_bytes = c.ws;
    if (P.leaf == LEAF_F64) {
        // A plan with fewer 64 x 64 FP64 tiles than two per SM leaves most SMs
        // idle while the longest tile's K loop runs (GB300 issues 2-3 DFMA per
        // clock per SM).  Each tile of a product is then cut into kparts equal
        // K ranges, each computed by its own block into an FP64 partial tile
        // in W after everything else there, and one more kernel adds a tile's
        // partials in part order: deterministic, and part of the plan, so
        // single, batched and static-scratch executions cut alike.
        int64_t tiles = 0;
        for (const LeafProduct& lp : P.products) tiles += leaf_tiles(lp, kF64Tile, kF64Tile);
        if (tiles > 0 && tiles < kSplitKTiles) {
            const int want = (int)std::min<int64_t>(kSplitKMaxParts, (kSplitKTiles + tiles - 1) / tiles);
            int64_t ws = (P.ws_bytes + 255) / 256 * 256;
            for (LeafProduct& lp : P.products) {
                const int parts = std::min(want, std::max(1, lp.K / kSplitKMinK));
                if (parts <= 1) continue;
                lp.kparts = parts;
                lp.part_off = ws / 8;
                ws += leaf_tiles(lp, kF64Tile, kF64Tile) * parts * (int64_t)kF64Tile * kF64Tile * 8;
                ws = (ws + 255) / 256 * 256;
            }
            P.ws_bytes = ws;
        }
    }
    if (P.leaf != LEAF_F64) {
        // CTA-pair tiles when every X operand is padded to them and they add
        // at most 1/8 to the tile area of 128 x 128 tiles
        bool all = !P.products.empty();
        double a1 = 0, a2 = 0;
        const int pc = tc_cols_for(P.leaf, kTcPairRows);
        for (const LeafProduct& lp : P.products) {
            all = all && lp.p_pad % kTcPairRows == 0;
            a1 += (double)leaf_tiles(lp, kTcTile, kTcTile) * kTcTile * kTcTile;
            a2 += (double)leaf_tiles(lp, kTcPairRows, pc) * kTcPairRows * pc;
        }
        P.tc_tile_rows = opt.cta_pair && all && a2 <= 1.125 * a1 ? kTcPairRows : kTcTile;
    }
}

}  // namespace

bool build_plan(int64_t m, int64_t n, const PlanOptions& opt, Plan* out, std::string* err) {
    if (m < 0 || n < 0) {
        *err = "m and n must be >= 0";
        return false;
    }
    if (m > INT32_MAX || n > INT32_MAX) {
        *err = "m and n must be < 2^31";
        return false;
    }
    if (!check_options(opt, err)) return false;
    Plan& P = *out;
    start_plan(P, m, n, opt);
    Ctx c;
    c.P = &P;
    c.opt = &opt;
    if (n > 0) recurse_columns(c, 0, n, 0);
    finish_plan(P, c, opt);
    return true;
}

bool build_gemm_plan(int64_t m, int64_t p, int64_t r, const PlanOptions& opt, Plan* out, std::string* err) {
    if (m < 0 || p < 0 || r < 0) {
        *err = "m, p and r must be >= 0";
        return false;
    }
    if (m > INT32_MAX || p > INT32_MAX || r > INT32_MAX) {
        *err = "m, p and r must be < 2^31";
        return false;
    }
    if (!check_options(opt, err)) return false;
    Plan& P = *out;
    start_plan(P, m, p, opt);
    P.gemm = true;
    P.r = r;
    Ctx c;
    c.P = &P;
    c.opt = &opt;
    if (p > 0 && r > 0) {
        // X and Y as whole operands (planned with dense leading dimensions p
        // and r; the runtime rebases them to the caller's ldx, ldy), the
        // output a dense p x r block of C (planned ld r, rebased to ldc)
        Term x{}, y{};
        x.off = 0;
        x.ld = p;
        x.rows = (int32_t)m;
        x.cols = (int32_t)p;
        x.buf = BUF_A;
        x.dt = P.in_dt;
        y = x;
        y.ld = r;
        y.cols = (int32_t)r;
        y.buf = BUF_B;
        std::vector<Term> X, Y;
        if (m > 0) {
            X.push_back(x);
            Y.push_back(y);
        }
        Target t{};
        t.kind = OUT_CDENSE;
        t.off = 0;
        t.ld = (int32_t)r;
        const int s = strassen_levels(p, m, r, P.cutoff, P.max_levels);
        P.stats.max_strassen_levels = s;
        P.stats.n_nodes = 1;
        expand(c, X, Y, p, m, r, m, 0, s, t, P.in_dt, P.in_dt);
    }
    finish_plan(P, c, opt);
    return true;
}

}  // namespace ata
