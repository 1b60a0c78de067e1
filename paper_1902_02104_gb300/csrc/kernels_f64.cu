// kernels_f64.cu -- FP64 leaf products, Strassen operand splits and output
// combines.
//
// On GB300 the FP64 pipe issues about two DFMA per clock per SM (measured
// 1.20 TFLOP/s on 152 SMs; DMMA is slower, 1.05 TFLOP/s), so the FP64 leaf
// is a SIMT DFMA kernel and is bound by that pipe: a 64 x 64 tile with a K
// slab of 16 takes ~32k clocks of DFMA per block while its 16 KB of operand
// loads take a few hundred.  What matters is that the pipe runs only useful
// DFMAs: no FP64 additions in the operand loads, and no DFMA issued on
// padding (work is skipped in 16 x 32 warp blocks outside the valid extent
// and below the diagonal of symmetric (SYRK) tiles).
#include <cstdint>

#include "kernels.h"

namespace ata {
namespace {

__device__ __forceinline__ int64_t packed_start(int64_t i, int64_t n) { return i * n - i * (i - 1) / 2; }

template <typename T>
__device__ __forceinline__ const T* term_ptr(const Bind& b, const Term& t) {
    // b is the instance of the term (t.inst)
    return term_base<T>(b, t.buf) + t.off;
}

// Value of a fused operand (sum of signed terms) at (k, c); zero outside
// each term's valid extent (implicit zero padding of uneven blocks).  A
// single term (every materialised operand) needs no FP64 addition: its sign
// is applied to the bit pattern, so the FP64 pipe only runs the leaf DFMAs.
// Self-check of a global access (only when the binding asks for it): the
// element index must lie inside its buffer; otherwise the access is skipped
// and `code` is recorded in *status.
__device__ __forceinline__ bool in_bounds(const Bind& b, int8_t buf, int64_t idx, int es, int* status, int code) {
    if (!b.check) return true;
    const int64_t lim = buf == BUF_A   ? b.a_elems
                        : buf == BUF_B ? b.b_elems
                        : buf == BUF_W ? b.w_bytes / es
                                       : b.c_elems;
    if (idx >= 0 && idx < lim) return true;
    atomicCAS(status, 0, code);
    return false;
}

// One entry (i, j) of a leaf product's output (i, j relative to the
// product): a dense workspace block, a dense block of C, a block of packed C,
// or the upper part of a diagonal block.  Entries outside the extent, and
// below the diagonal of a symmetric block, are not written.
__device__ __forceinline__ void store_leaf_entry(const LeafProduct& sp, const Bind& bind, int i, int j, double v,
                                                 int* status) {
    if (i >= sp.out_rows || j >= sp.out_cols) return;
    if (sp.out_kind == OUT_DENSE) {
        const int64_t idx = sp.out_off + (int64_t)i * sp.out_ld + j;
        if (in_bounds(bind, BUF_W, idx, 8, status, 12)) reinterpret_cast<double*>(bind.W)[idx] = v;
    } else if (sp.out_kind == OUT_CDENSE) {
        const int64_t idx = sp.out_off + (int64_t)i * sp.out_ld + j;
        if (in_bounds(bind, BUF_C, idx, 8, status, 12)) bind.C[idx] = v;
    } else {
        const int64_t gi = (int64_t)sp.ci0 + i, gj = (int64_t)sp.cj0 + j;
        if (sp.out_kind == OUT_SYRK && gj < gi) return;
        const int64_t idx = packed_start(gi, bind.n) + (gj - gi);
        if (in_bounds(bind, BUF_C, idx, 8, status, 12)) bind.C[idx] = v;
    }
}

template <int NB>
__device__ __forceinline__ double operand_at(const BindSet<NB>& bs, const Term* ts, int nt, int k, int c,
                                             int* status) {
    if (nt == 1) {
        const Term& tm = ts[0];
        if (k >= tm.rows || c >= tm.cols) return 0.0;
        const int64_t idx = tm.off + (int64_t)k * tm.ld + c;
        if (!in_bounds(bs.b[tm.inst], tm.buf, idx, 8, status, 11)) return 0.0;
        const double x = __ldg(term_ptr<double>(bs.b[tm.inst], tm) + (int64_t)k * tm.ld + c);
        return __longlong_as_double(__double_as_longlong(x) ^ ((long long)tm.neg << 63));
    }
    double v = 0.0;
    for (int t = 0; t < nt; ++t) {
        const Term& tm = ts[t];
        if (k < tm.rows && c < tm.cols) {
            const int64_t idx = tm.off + (int64_t)k * tm.ld + c;
            if (!in_bounds(bs.b[tm.inst], tm.buf, idx, 8, status, 11)) continue;
            const double x = __ldg(term_ptr<double>(bs.b[tm.inst], tm) + (int64_t)k * tm.ld + c);
            v = tm.neg ? v - x : v + x;
        }
    }
    return v;
}

constexpr int TILE = kF64Tile;  // 64
constexpr int BK = 16;
constexpr int NTHREADS = 256;
constexpr int LOADS = (BK * TILE) / NTHREADS;  // operand elements per thread per slab and side

// Persistent leaf kernel: blocks pull tiles (heaviest first) from a counter.
// out(p x r) = X^t Y where X (K x p) and Y (K x r) are term sums.
//
// Warp w owns the 16 x 32 block (rows 16*(w/2).., cols 32*(w%2)..) of the
// 64 x 64 tile; lane (lr, lc) owns rows 4lr..4lr+3 of it and columns
// lc + 8b, b = 0..3.  Raggedness is therefore warp-uniform: a warp whose
// block lies outside the valid extent (or strictly below the diagonal of a
// symmetric tile) skips the whole slab with a branch, and active warps run
// unpredicated DFMAs -- a predicated-off DFMA still occupies the FP64 pipe.
// K is staged in slabs of 16, double-buffered through registers.
// Accumulation runs k ascending per entry over the tile's K range; a tile cut
// along K (part >= 0) writes its partial 64 x 64 tile to its slot in W, and
// partial_sum_kernel adds the parts in order.
template <int NB>
__global__ void __launch_bounds__(NTHREADS) leaf_f64_kernel(const __grid_constant__ BindSet<NB> bs,
                                                            const LeafProduct* __restrict__ prods,
                                                            const Term* __restrict__ terms,
                                                            const LeafTile* __restrict__ tiles, int ntiles,
                                                            int* __restrict__ counter, int* __restrict__ status) {
    __shared__ __align__(16) double Xs[2][BK][TILE];
    __shared__ __align__(16) double Ys[2][BK][TILE];
    __shared__ Term sx[kMaxTerms], sy[kMaxTerms];
    __shared__ int s_tile;
    __shared__ LeafProduct sp;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int lr = lane >> 3, lc = lane & 7;
    const int row0 = 16 * (warp >> 1) + 4 * lr;  // first of this lane's 4 rows
    const int col0 = 32 * (warp & 1) + lc;       // first of this lane's 4 columns (stride 8)

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const LeafTile lt = tiles[t];
        if (tid == 0) sp = prods[lt.prod];
        __syncthreads();
        const int nx = sp.nx, ny = sp.ny;
        if (tid < nx) sx[tid] = terms[sp.x0 + tid];
        if (tid >= 64 && tid - 64 < ny) sy[tid - 64] = terms[sp.y0 + tid - 64];
        const int i0 = lt.ti * TILE, j0 = lt.tj * TILE;
        const int rows_v = min(TILE, sp.out_rows - i0);
        const int cols_v = min(TILE, sp.out_cols - j0);
        const bool diag = sp.out_kind == OUT_SYRK && lt.ti == lt.tj;
        const int kbeg = lt.k0, kend = min(lt.k1, sp.K);
        __syncthreads();

        // warp-uniform activity: some valid row, some valid column, and not
        // entirely below the diagonal of a symmetric tile
        const int wr = 16 * (warp >> 1), wc = 32 * (warp & 1);
        const bool active = wr < rows_v && wc < cols_v && (!diag || wc + 31 >= wr);

        double acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

        double px[LOADS], py[LOADS];
        auto fetch = [&](int k0) {
#pragma unroll
            for (int e = 0; e < LOADS; ++e) {
                const int idx = tid + e * NTHREADS;
                const int kk = idx / TILE, c = idx % TILE;
                const int k = k0 + kk;
                px[e] = (k < kend) ? operand_at(bs, sx, nx, k, i0 + c, status) : 0.0;
                py[e] = (k < kend) ? operand_at(bs, sy, ny, k, j0 + c, status) : 0.0;
            }
        };
        auto stash = [&](int buf) {
#pragma unroll
            for (int e = 0; e < LOADS; ++e) {
                const int idx = tid + e * NTHREADS;
                const int kk = idx / TILE, c = idx % TILE;
                Xs[buf][kk][c] = px[e];
                Ys[buf][kk][c] = py[e];
            }
        };

        int buf = 0;
        if (kbeg < kend) {
            fetch(kbeg);
            stash(0);
        }
        __syncthreads();
        for (int k0 = kbeg; k0 < kend; k0 += BK) {
            const bool more = k0 + BK < kend;
            if (more) fetch(k0 + BK);  // global loads in flight during the slab's DFMAs
            if (active) {
                const int kmax = min(BK, kend - k0);
                for (int kk = 0; kk < kmax; ++kk) {
                    const double2 xa = *reinterpret_cast<const double2*>(&Xs[buf][kk][row0]);
                    const double2 xb = *reinterpret_cast<const double2*>(&Xs[buf][kk][row0 + 2]);
                    const double x[4] = {xa.x, xa.y, xb.x, xb.y};
                    double y[4];
#pragma unroll
                    for (int b = 0; b < 4; ++b) y[b] = Ys[buf][kk][col0 + 8 * b];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
                }
            }
            if (more) stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }

        // epilogue: the output (dense workspace block, block of packed C, or
        // upper part of a diagonal block), or this K range's partial tile
        const Bind& bind = bs.b[sp.inst];
        if (active) {
            if (lt.part >= 0) {
                const int64_t slot = sp.part_off + (int64_t)lt.part * TILE * TILE;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int64_t idx = slot + (row0 + a) * TILE + col0 + 8 * b;
                        if (in_bounds(bind, BUF_W, idx, 8, status, 13)) reinterpret_cast<double*>(bind.W)[idx] = acc[a][b];
                    }
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        store_leaf_entry(sp, bind, i0 + row0 + a, j0 + col0 + 8 * b, acc[a][b], status);
            }
        }
        __syncthreads();
    }
}

// Partial tiles of FP64 tiles cut along K, added in part order (k ascending
// across the parts) and stored like the leaf's own output.  One block per
// cut tile; entries outside the product's extent, or below the diagonal of a
// symmetric block, were never written by the leaf and are not read.
template <int NB>
__global__ void __launch_bounds__(NTHREADS) partial_sum_kernel(const __grid_constant__ BindSet<NB> bs,
                                                               const LeafProduct* __restrict__ prods,
                                                               const PartialSum* __restrict__ tasks,
                                                               int* __restrict__ status) {
    const PartialSum ps = tasks[blockIdx.x];
    const LeafProduct sp = prods[ps.prod];
    const Bind& bind = bs.b[sp.inst];
    const double* W = reinterpret_cast<const double*>(bind.W);
    for (int e = threadIdx.x; e < TILE * TILE; e += NTHREADS) {
        const int i = ps.ti * TILE + e / TILE, j = ps.tj * TILE + e % TILE;
        if (i >= sp.out_rows || j >= sp.out_cols) continue;
        if (sp.out_kind == OUT_SYRK && (int64_t)sp.cj0 + j < (int64_t)sp.ci0 + i) continue;
        double v = 0.0;
        for (int q = 0; q < sp.kparts; ++q) {
            const int64_t idx = sp.part_off + (int64_t)(ps.slot0 + q) * TILE * TILE + e;
            if (in_bounds(bind, BUF_W, idx, 8, status, 14)) v += W[idx];
        }
        store_leaf_entry(sp, bind, i, j, v, status);
    }
}

// ---------------------------------------------------------------------------
// Operand split (Section 4.2.2 sums).  Each thread handles one (k, c) of the
// K1 x c1 child block: it reads the four parent blocks once and writes every
// sum of this side.  Output slot order matches the planner's table.
template <int NB, typename TS, typename TD>
__global__ void __launch_bounds__(256) split_kernel(const __grid_constant__ BindSet<NB> bs,
                                                    const SplitTask* __restrict__ tasks,
                                                    const Chunk* __restrict__ chunks, int* __restrict__ status) {
    const Chunk ch = chunks[blockIdx.x];
    const SplitTask& st = tasks[ch.task];
    const Bind& bind = bs.b[st.inst];
    const int c1 = st.c1, K1 = st.K1;
    const TS* src = term_ptr<TS>(bind, st.src);
    const int64_t ld = st.src.ld;
    const int srows = st.src.rows, scols = st.src.cols;
    const bool neg = st.src.neg;
    TD* W = reinterpret_cast<TD*>(bind.W);
    const int total = ch.nrows * c1;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int k = ch.row0 + e / c1, c = e % c1;
        TD B[4];
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
#pragma unroll
            for (int cb = 0; cb < 2; ++cb) {
                const int rr = kb * K1 + k, cc = cb * c1 + c;
                TD v = 0;
                if (rr < srows && cc < scols &&
                    in_bounds(bind, st.src.buf, st.src.off + (int64_t)rr * ld + cc, sizeof(TS), status, 21))
                    v = (TD)src[(int64_t)rr * ld + cc];
                B[2 * kb + cb] = neg ? -v : v;
            }
        const int64_t o = (int64_t)k * c1 + c;
        if (bind.check) {
            bool ok = true;
            for (int q = 0; q < st.nout; ++q)
                ok &= in_bounds(bind, BUF_W, st.out_off[q] + o, sizeof(TD), status, 22);
            if (!ok) continue;
        }
        if (st.variant == 0) {
            if (st.side == 0) {  // left factor X^t: M1 M2 M5 M6 M7
                W[st.out_off[0] + o] = B[0] + B[3];
                W[st.out_off[1] + o] = B[1] + B[3];
                W[st.out_off[2] + o] = B[0] + B[2];
                W[st.out_off[3] + o] = B[1] - B[0];
                W[st.out_off[4] + o] = B[2] - B[3];
            } else {             // right factor Y: M1 M3 M4 M6 M7
                W[st.out_off[0] + o] = B[0] + B[3];
                W[st.out_off[1] + o] = B[1] - B[3];
                W[st.out_off[2] + o] = B[2] - B[0];
                W[st.out_off[3] + o] = B[0] + B[1];
                W[st.out_off[4] + o] = B[2] + B[3];
            }
        } else {
            if (st.side == 0) {  // S1 S2 S3 S4 (Winograd, chained)
                const TD s1 = B[1] + B[3];
                const TD s2 = s1 - B[0];
                W[st.out_off[0] + o] = s1;
                W[st.out_off[1] + o] = s2;
                W[st.out_off[2] + o] = B[0] - B[1];
                W[st.out_off[3] + o] = B[2] - s2;
            } else {             // T1 T2 T3 T4
                const TD t1 = B[1] - B[0];
                const TD t2 = B[3] - t1;
                W[st.out_off[0] + o] = t1;
                W[st.out_off[1] + o] = t2;
                W[st.out_off[2] + o] = B[3] - B[1];
                W[st.out_off[3] + o] = t2 - B[2];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Output combine (Section 4.2.2: D11..D22 from M1..M7, additions in the
// printed order; Winograd's U-chain for the variant).  Each thread handles
// one (i, j) of the p1 x r1 child grid and writes up to four quadrants.
template <int NB>
__global__ void __launch_bounds__(256) combine_kernel(const __grid_constant__ BindSet<NB> bs,
                                                      const CombineTask* __restrict__ tasks,
                                                      const Chunk* __restrict__ chunks, int* __restrict__ status) {
    const Chunk ch = chunks[blockIdx.x];
    const CombineTask& ct = tasks[ch.task];
    const Bind& bind = bs.b[ct.inst];
    const int p = ct.p, r = ct.r, p1 = ct.p1, r1 = ct.r1;
    const double* M = reinterpret_cast<const double*>(bind.W) + ct.m_off;
    const int64_t msz = (int64_t)p1 * r1;
    const int total = ch.nrows * r1;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = ch.row0 + e / r1, j = e % r1;
        const int64_t o = (int64_t)i * r1 + j;
        double m[7];
#pragma unroll
        for (int t = 0; t < 7; ++t)
            m[t] = in_bounds(bind, BUF_W, ct.m_off + t * msz + o, 8, status, 31) ? M[t * msz + o] : 0.0;
        double d[4];
        if (ct.variant == 0) {
            d[0] = m[0] - m[4] + m[6] + m[3];  // D11 = M1 - M5 + M7 + M4
            d[1] = m[2] + m[4];                // D12 = M3 + M5
            d[2] = m[1] + m[3];                // D21 = M2 + M4
            d[3] = m[2] + m[5] - m[1] + m[0];  // D22 = M3 + M6 - M2 + M1
        } else {
            const double u2 = m[0] + m[5];     // U2 = M1 + M6
            const double u3 = u2 + m[6];       // U3 = U2 + M7
            d[0] = m[0] + m[1];                // D11 = M1 + M2
            d[1] = (u2 + m[4]) + m[2];         // D12 = U4 + M3, U4 = U2 + M5
            d[2] = u3 - m[3];                  // D21 = U3 - M4
            d[3] = u3 + m[4];                  // D22 = U3 + M5
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ii = (q >> 1) * p1 + i, jj = (q & 1) * r1 + j;
            if (ii >= p || jj >= r) continue;
            if (ct.dst_kind == OUT_DENSE) {
                const int64_t idx = ct.dst_off + (int64_t)ii * ct.dst_ld + jj;
                if (in_bounds(bind, BUF_W, idx, 8, status, 32)) reinterpret_cast<double*>(bind.W)[idx] = d[q];
            } else if (ct.dst_kind == OUT_CDENSE) {
                const int64_t idx = ct.dst_off + (int64_t)ii * ct.dst_ld + jj;
                if (in_bounds(bind, BUF_C, idx, 8, status, 32)) bind.C[idx] = d[q];
            } else {
                const int64_t gi = (int64_t)ct.ci0 + ii, gj = (int64_t)ct.cj0 + jj;
                const int64_t idx = packed_start(gi, bind.n) + (gj - gi);
                if (in_bounds(bind, BUF_C, idx, 8, status, 32)) bind.C[idx] = d[q];
            }
        }
    }
}

template <int NB>
BindSet<NB> make_set(const Bind* binds, int nb) {
    BindSet<NB> s{};
    if constexpr (NB == kDevBinds)
        s.b = binds;  // device array
    else
        for (int i = 0; i < nb && i < NB; ++i) s.b[i] = binds[i];
    return s;
}

}  // namespace

cudaError_t launch_leaf_f64(int* status, const Bind* binds, int nb, const LeafProduct* prods, const Term* terms,
                            const LeafTile* tiles, int ntiles, int* counter, int grid, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (nb <= 1)
        leaf_f64_kernel<1><<<grid, NTHREADS, 0, s>>>(make_set<1>(binds, nb), prods, terms, tiles, ntiles, counter,
                                                     status);
    else
        leaf_f64_kernel<kDevBinds><<<grid, NTHREADS, 0, s>>>(make_set<kDevBinds>(binds, nb), prods, terms, tiles,
                                                             ntiles, counter, status);
    return cudaGetLastError();
}

cudaError_t launch_partial_sums(int* status, const Bind* binds, int nb, const LeafProduct* prods,
                                const PartialSum* tasks, int ntasks, cudaStream_t s) {
    if (ntasks <= 0) return cudaSuccess;
    if (nb <= 1)
        partial_sum_kernel<1><<<ntasks, NTHREADS, 0, s>>>(make_set<1>(binds, nb), prods, tasks, status);
    else
        partial_sum_kernel<kDevBinds><<<ntasks, NTHREADS, 0, s>>>(make_set<kDevBinds>(binds, nb), prods, tasks, status);
    return cudaGetLastError();
}

int leaf_f64_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, leaf_f64_kernel<1>, NTHREADS, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

template <int NB>
static cudaError_t split_dispatch(int* status, const BindSet<NB>& bs, const SplitTask* tasks, const Chunk* chunks,
                                  int nchunks, int8_t src_dt, int8_t dst_dt, cudaStream_t s) {
    if (src_dt == DT_F64 && dst_dt == DT_F64)
        split_kernel<NB, double, double><<<nchunks, 256, 0, s>>>(bs, tasks, chunks, status);
    else if (src_dt == DT_F32 && dst_dt == DT_F32)
        split_kernel<NB, float, float><<<nchunks, 256, 0, s>>>(bs, tasks, chunks, status);
    else if (src_dt == DT_F32 && dst_dt == DT_F64)
        split_kernel<NB, float, double><<<nchunks, 256, 0, s>>>(bs, tasks, chunks, status);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_split(int* status, const Bind* binds, int nb, const SplitTask* tasks, const Chunk* chunks,
                         int nchunks, int8_t src_dt, int8_t dst_dt, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    if (nb <= 1) return split_dispatch<1>(status, make_set<1>(binds, nb), tasks, chunks, nchunks, src_dt, dst_dt, s);
    return split_dispatch<kDevBinds>(status, make_set<kDevBinds>(binds, nb), tasks, chunks, nchunks, src_dt, dst_dt,
                                     s);
}

cudaError_t launch_combine(int* status, const Bind* binds, int nb, const CombineTask* tasks, const Chunk* chunks,
                           int nchunks, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    if (nb <= 1)
        combine_kernel<1><<<nchunks, 256, 0, s>>>(make_set<1>(binds, nb), tasks, chunks, status);
    else
        combine_kernel<kDevBinds><<<nchunks, 256, 0, s>>>(make_set<kDevBinds>(binds, nb), tasks, chunks, status);
    return cudaGetLastError();
}

}  // namespace ata
