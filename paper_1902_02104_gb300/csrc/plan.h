// plan.h -- host recursion planner for C = A^t A (no CUDA calls here).
//
// The planner turns (m, n, cutoff) into three flat task tables:
//
//   * split tasks  (Section 4.2.2, operand sums of the seven Strassen
//                   products): one task per (Strassen node, operand side)
//                   that reads the four blocks of a parent operand once and
//                   writes the sums its children need;
//   * leaf products: every product the recursion bottoms out in -- the base
//                   case "mult" of Algorithm 1 on each diagonal block (upper
//                   tiles only) and the leaf products of every Strassen tree;
//   * combine tasks (Section 4.2.2, D11..D22 from M1..M7): one task per
//                   Strassen node, writing the four quadrants of its output.
//
// Column recursion (Algorithm 1, Eq. "Cij"): a node owns columns
// [c0, c0 + w) of A and all m rows.  It is a base case when
// min(m_d, w) <= cutoff, where m_d = ceil^d(m) is the row count the
// paper's sub-matrix has at depth d.  Otherwise w splits into n1 = ceil(w/2)
// and n2 = floor(w/2); the two diagonal blocks recurse and the off-diagonal
// block C_12 = A_L^t A_R (L = first n1 columns, R = the other n2) is one
// product with reduction length m.  The paper's row split only makes the two
// addends of each block (S1 + S2, S3 + S4, S5 + S6); summing them inside one
// product over all m rows gives the same C.
//
// A product out = X^t Y is stored as two "K x cols" row-major operands
// (X: K x p, Y: K x r), both blocks of A: X = A[:, L], Y = A[:, R].  Its
// Strassen recursion stops when min(p, q, r) <= cutoff, q being the paper's
// HASA reduction length ceil(m_d / 2) (halved with p, r and K at each level).
// Odd sizes split into ceil/floor halves with implicit zero padding.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace ata {

// A Strassen level cap at or above this leaves the depth free (to the
// cutoff, or to what fits the workspace when the cutoff is automatic).
constexpr int kFreeLevels = 64;

// Buffers a term or an output refers to: the caller's A (or X of a general
// product), the plan workspace W, the caller's C, and Y of a general product.
enum BufId : int8_t { BUF_A = 0, BUF_W = 1, BUF_C = 2, BUF_B = 3 };
enum ElemType : int8_t { DT_F64 = 0, DT_F32 = 1 };

// Leaf arithmetic family of a plan.
enum LeafKind : int8_t { LEAF_F64 = 0, LEAF_BF16X3 = 1, LEAF_TF32 = 2, LEAF_OZAKI = 3 };

// One signed term of an operand: a row-major block of `rows x cols` valid
// elements (reads outside the valid extent are zero).  Offsets and leading
// dimensions count elements of the term's own type.
struct Term {
    int64_t off;
    int64_t ld;
    int32_t rows, cols;
    int8_t buf, dt, neg, pad_;
    int32_t inst;             // instance of a batched execution (0 for one plan)
};
static_assert(sizeof(Term) == 32, "Term layout");

// Output of a leaf or combine: a dense block of W, a block of packed C, the
// upper part of a diagonal block of packed C, or a dense block of the
// caller's C (general product; leading dimension ldc after rebasing).
enum OutKind : int8_t { OUT_DENSE = 0, OUT_PACKED = 1, OUT_SYRK = 2, OUT_CDENSE = 3 };

// Leaf product: out(p x r) = X^t Y, X and Y sums of terms (K rows each).
struct LeafProduct {
    int32_t p, r, K;          // padded sizes
    int32_t x0, nx, y0, ny;   // term ranges in Plan::terms
    int32_t out_rows, out_cols;  // extent written (<= p, r)
    int8_t out_kind, x_dt, y_dt, pad_;
    int32_t out_ld;           // OUT_DENSE: leading dimension (FP64 elements)
    int64_t out_off;          // OUT_DENSE: FP64 element offset in W
    int32_t ci0, cj0;         // OUT_PACKED / OUT_SYRK: global (row, col) of the block
    int64_t work;             // scalar multiplications (for ordering and stats)
    int32_t inst;             // instance of a batched execution (0 for one plan)
    int32_t kparts;           // FP64 leaves: K ranges each tile is cut into (<= 1: none)
    int64_t part_off;         // ... and the FP64 element offset in W of its partial tiles
    // tensor-core leaves: split operand parts, K-major, in W (byte offsets)
    int64_t tc_x_off, tc_y_off;   // parts x rows_pad x K_pad elements each
    int32_t p_pad, r_pad, K_pad;  // rows of X / Y parts (multiples of 128), K padded
    int32_t pad3_;
};

// Split task: one operand block (K x c, single term `src`) -> child sums.
// The four blocks are B[kb][cb] (kb: K half, cb: column half), each
// K1 x c1 with zero padding.  out_off[s] is the element offset in W of the
// s-th sum buffer (K1 x c1, leading dimension c1, type dst_dt).
struct SplitTask {
    Term src;
    int32_t K1, c1;
    int8_t side;              // 0: left operand (X, transposed in the product), 1: right (Y)
    int8_t variant;           // 0 Strassen, 1 Winograd
    int8_t dst_dt, nout;
    int32_t inst;
    int64_t out_off[5];
};

// Combine task: seven child results M1..M7 (each p1 x r1 FP64, dense in W at
// m_off + i * p1 * r1, leading dimension r1) -> the four quadrants of the
// parent output (p x r), dense in W or a block of packed C.
struct CombineTask {
    int64_t m_off;
    int32_t p, r, p1, r1;
    int8_t dst_kind, variant, pad_[2];
    int32_t dst_ld;
    int64_t dst_off;          // OUT_DENSE
    int32_t ci0, cj0;         // OUT_PACKED
    int32_t inst;
    int32_t pad2_;
};

struct PlanStats {
    int32_t depth = 0, n_diag_leaves = 0, n_nodes = 0, max_strassen_levels = 0;
    int64_t mults = 0, adds = 0;
};

struct Plan {
    int64_t m = 0, n = 0;
    // general product C = X^t Y (X: m x n, Y: m x r), the HASA entry point;
    // false: C = A^t A (A: m x n)
    bool gemm = false;
    int64_t r = 0;
    int cutoff = 0;
    int variant = 0;
    LeafKind leaf = LEAF_F64;
    int8_t in_dt = DT_F64;    // element type of A
    int8_t sum_dt = DT_F64;   // element type of materialised operand sums
    int fuse_levels = 1;      // bottom Strassen levels whose sums are fused into leaf loads
    int max_levels = kFreeLevels;  // cap on Strassen levels per product

    std::vector<Term> terms;
    std::vector<LeafProduct> products;
    std::vector<std::vector<SplitTask>> split_levels;    // [l] builds level l+1 operands
    std::vector<std::vector<CombineTask>> combine_levels; // [l] children at level l+1 -> level l
    int64_t ws_bytes = 0;
    int tc_tile_rows = 0;     // tensor-core leaves: 256 when every X operand is padded to
                              // whole 256-row tiles (the CTA-pair kernel applies), else 128;
                              // the tile's columns are tc_cols_for(leaf, tc_tile_rows)
    PlanStats stats;
};

// Tensor-core leaf geometry per leaf kind.
struct TcGeom {
    int parts;       // split parts per operand
    int elem;        // bytes per part element (2: bf16, 4: tf32 as fp32)
    int k_align;     // K padding of part buffers (elements)
};
TcGeom tc_geom(LeafKind k);
constexpr int kF64Tile = 64;      // FP64 leaf tile (rows and columns)
// FP64 leaves of a plan with fewer tiles than this are cut along K (see
// finish_plan): two resident blocks on each of GB300's 152 SMs.
constexpr int64_t kSplitKTiles = 304;
constexpr int kSplitKMaxParts = 8;
constexpr int kSplitKMinK = 128;  // K values per part at least
constexpr int kTcTile = 128;      // tensor-core leaf tile (rows and columns)
constexpr int kTcPairRows = 256;  // rows of the CTA-pair tile
constexpr int kTcWideCols = 256;  // columns of the TF32 CTA-pair tile
// Columns of the tensor-core leaf tile with `tile_rows` rows: the TF32 pair
// kernel computes 256 x 256 tiles (N = 256), every other one 128 columns.
inline int tc_cols_for(LeafKind k, int tile_rows) {
    return k == LEAF_TF32 && tile_rows == kTcPairRows ? kTcWideCols : kTcTile;
}

struct PlanOptions {
    int cutoff = 64;
    int variant = 0;
    LeafKind leaf = LEAF_F64;
    int fuse_levels = 1;
    int max_levels = kFreeLevels;
    bool cta_pair = false;  // tensor-core leaves on 256 x 128 CTA-pair tiles where eligible
    uint64_t wait_ns = 0;   // tensor-core leaves: pipeline wait limit (0 = the kernel's default)
};

// Builds the plan.  Returns false and sets *err on invalid input.
bool build_plan(int64_t m, int64_t n, const PlanOptions& opt, Plan* out, std::string* err);

// Builds the plan of the general product C = X^t Y, X: m x p, Y: m x r, C:
// p x r dense (Section 4.2.2's HASA on two operands): Strassen levels while
// min(p, m, r) > cutoff (halving all three), leaf products below.
bool build_gemm_plan(int64_t m, int64_t p, int64_t r, const PlanOptions& opt, Plan* out, std::string* err);

// Number of output tiles of `p` for a leaf tile of tm x tn (upper tiles only for SYRK).
int64_t leaf_tiles(const LeafProduct& p, int tm, int tn);

inline int64_t ceil_half(int64_t x) { return (x + 1) / 2; }
inline int64_t packed_row_start(int64_t i, int64_t n) { return i * n - i * (i - 1) / 2; }

}  // namespace ata
