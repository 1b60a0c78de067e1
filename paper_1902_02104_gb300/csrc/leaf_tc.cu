// leaf_tc.cu -- tensor-core leaf products on sm_103a (tcgen05 + TMEM + TMA).
//
// Three leaf arithmetics share one pipeline:
//   bf16x3  FP32 operands, per column scaled by 2^-E (max |x| < 2^E) and cut
//           into three signed base-256 digits, each an exact bf16 (24 bits,
//           the FP32 significand); the six part products of order a+b <= 2.
//   tf32    FP32 operands rounded to TF32 (kind::tf32), one product.
//   ozaki   FP64 operands, same slicing with six digits (48 bits); the 21
//           part products of order <= 5.  This emulates the FP64 product
//           with bf16 tensor cores (an Ozaki-style scheme).
// Part products are exact in FP32.  The tensor core accumulates in FP32
// with truncation, so an accumulator that runs over a long K drifts by a
// relative ~2^-23 per addition.  Orders whose share of the result is large
// are therefore accumulated per 256-deep K chunk in their own accumulator,
// in which every partial sum is an integer of at most 2^24 units (exact):
// order 0 for bf16x3, orders 0, 1 and 2 for ozaki.  The smaller orders share
// one accumulator per chunk (bf16x3 orders 1-2, ~2^-8 of the result; ozaki
// orders 3-5, ~2^-24, over 512-deep chunks) and add errors far below the
// stated bounds.  After each chunk the epilogue adds the chunk sums to
// running sums: ozaki into float-float (hi, lo) pairs that carry the FP64
// result; bf16x3 adds the exact order-0 chunk to hi by TwoSum, its rounding
// error kept in lo, and orders 1-2 straight into lo (an FP32-accurate result
// needs no more).  Results are scaled back by 2^(E_i + F_j) with integer
// exponent arithmetic and written in FP64.
//
// Stage 1 (operand preparation, memory bound): every leaf operand -- a signed
// sum of blocks of A or of materialised Strassen sums -- is formed once,
// sliced and written K-major (row = output index, K contiguous), zero padded
// to whole 128-row tiles, so that a TMA 2D load of a (K-block x 128 rows) box
// with 128B / 64B swizzle lands in shared memory in the canonical K-major
// UMMA layout.  Sliced modes first reduce each column's max |x|.
//
// Stage 2 (persistent GEMM, one CTA per SM): warp 0 issues TMA loads of all
// parts of a K-block into a stage ring, warp 1 issues tcgen05.mma (M = 128,
// N = 128, FP32 accumulators in TMEM; CTA pairs M = 256, N = 128, or 256 for
// TF32), the epilogue warps drain TMEM
// (tcgen05.ld) and write the FP64 tile.  Every wait on an mbarrier is bounded
// (1 s, %globaltimer); on timeout the kernel records an error code in the
// table's status word, the other roles notice it and give up too, in-flight
// copies and MMAs are waited for (bounded), TMEM is freed and the kernel
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <queue>
#include <set>
#include <tuple>
#include <vector>

#include "runtime.h"

namespace ata {
namespace {

constexpr int MODE_BF16X3 = 1, MODE_TF32 = 2, MODE_OZAKI = 3;  // == LeafKind values
constexpr uint64_t kTimeoutNs = 1000000000ull;
constexpr int ERR_TIMEOUT_PRODUCER = 1, ERR_TIMEOUT_MMA = 2, ERR_TIMEOUT_EPILOGUE = 3;

// ---------------------------------------------------------------------------
// PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// CG == 2 waits acquire at cluster scope: the barrier may complete through
// arrivals of the other CTA of the pair.
template <int CG = 1>
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    if constexpr (CG == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    }
    return ok != 0;
}

// Non-blocking test of the phase of `bar` with the given parity.
template <int CG = 1>
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    if constexpr (CG == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    }
    return ok != 0;
}

// Bounded wait for the phase of `bar` with the given parity.  Returns false
// (after recording `code` in *status unless another role already did) when
// the wait gives up: after `limit_ns`, or when *status shows that another
// role gave up first.  A limit shorter than the default (a plan option for
// tests of this path) polls without blocking and reads the clock on every
// poll, so that the wait gives up once the limit has passed (a blocking
// try_wait could outlast a limit of a microsecond).
template <int CG = 1>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status, int code,
                                          uint64_t limit_ns) {
    if (limit_ns < kTimeoutNs) {
        const uint64_t t0 = globaltimer();
        for (;;) {
            if (mbar_test_wait<CG>(bar, parity)) return true;
            if (*reinterpret_cast<volatile int*>(status) != 0) return false;
            if (globaltimer() - t0 > limit_ns) {
                atomicCAS(status, 0, code);
                return false;
            }
        }
    }
    if (mbar_try_wait<CG>(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait<CG>(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*reinterpret_cast<volatile int*>(status) != 0) return false;
            if (globaltimer() - t0 > limit_ns) {
                atomicCAS(status, 0, code);
                return false;
            }
        }
    }
}

// Bounded wait that records nothing (teardown: copies or MMAs in flight).
template <int CG = 1>
__device__ __forceinline__ void mbar_wait_quiet(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait<CG>(bar, parity) && globaltimer() - t0 < kTimeoutNs) {
    }
}

// Cluster helpers (the CTA-pair kernel runs in clusters of two CTAs; its
// even CTA -- rank 0 -- issues every MMA of the pair).
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Address, in the cluster window, of the same shared-memory offset in CTA `rank`.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
// Every thread of both CTAs: release what this thread wrote, wait for all.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// Arrive on an mbarrier given by its cluster-window address (any CTA of the cluster).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}

// TMA 2D tile load into this CTA's shared memory.  CG == 1: completion on
// `bar` of this CTA.  CG == 2: `bar` is a cluster-window address and may be
// the pair's even CTA's barrier, which counts both CTAs' bytes.
template <int CG>
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, uint32_t bar, int x, int y) {
    if constexpr (CG == 1) {
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
            "[%2];" ::"r"(dst),
            "l"(tmap), "r"(bar), "r"(x), "r"(y)
            : "memory");
    } else {
        asm volatile(
            "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
            "l"(tmap), "r"(bar), "r"(x), "r"(y)
            : "memory");
    }
}

// TMEM allocation: CG == 2 allocates the same columns in both CTAs of the
// pair; one warp of each CTA executes it (and the matching dealloc).
template <int CG>
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    if constexpr (CG == 1)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols));
    else
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols));
}
template <int CG>
__device__ __forceinline__ void tmem_relinquish() {
    if constexpr (CG == 1)
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    else
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
}
template <int CG>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    if constexpr (CG == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
    else
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (TMEM) [+]= A (smem) x B (smem).  CG == 2: M = 256 over the pair, A's
// rows 0-127 and B's first N/2 rows in the even CTA, the rest at the same
// shared-memory offsets in the odd CTA; each CTA's TMEM receives its 128 rows.
template <int MODE, int CG>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if constexpr (MODE == MODE_TF32 && CG == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else if constexpr (MODE == MODE_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else if constexpr (CG == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    }
}

// Arrive on `bar` once every MMA issued so far by this thread has completed;
// CG == 2 arrives on the barrier at the same offset in both CTAs of the pair.
template <int CG>
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    if constexpr (CG == 1) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
    } else {
        const uint16_t mask = 3;
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                bar),
            "h"(mask)
            : "memory");
    }
}

// 32 lanes x 32 bit, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without the wait: several loads may be in flight; the
// registers are valid after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Lanes' share of a thread's NCOL column exponents (at least one slot).
template <typename G, int NCOL>
struct SLICED_COLS {
    static constexpr int W = G::SLICED && NCOL >= 32 ? NCOL / 32 : 1;
};

// Exact FP32 -> FP64 widening with integer operations (the FP64 pipe is the
// scarce unit on this part), scaled by 2^sc: the FP64 bits of f * 2^sc,
// built in 32-bit halves (the high word takes the sign, the rebiased and
// scaled exponent and the top 20 mantissa bits, the low word the last 3).
// Zero and subnormal f give 0, which changes a result by less than 2^-126 of
// its unit; an Inf or NaN f keeps its exponent.
__device__ __forceinline__ long long f2d_scaled_bits(float f, int sc) {
    const unsigned int b = __float_as_uint(f);
    const unsigned int e = (b >> 23) & 0xFF;
    if (e == 0) return 0;
    const unsigned int ex = e == 0xFF ? 0x7FFu : e + 896u + (unsigned int)sc;
    const unsigned int hw = (b & 0x80000000u) | (ex << 20) | ((b >> 3) & 0xFFFFFu);
    return (long long)(((unsigned long long)hw << 32) | (unsigned long long)(b << 29));
}

// Scale exponent E of a column whose largest magnitude has bit pattern mx:
// mx = f * 2^(E - HEAD) with f in [0.5, 1), so that every |x| 2^-E of the
// column is below 2^-HEAD (HEAD bits of headroom shrink the leading digit);
// 0 for an all-zero (or subnormal) column; kNonFinite when the column holds
// an Inf or NaN (its products become NaN).
constexpr int kNonFinite = 1 << 20;
template <int HEAD>
__device__ __forceinline__ int col_exponent(unsigned long long mx) {
    const int eb = (int)((mx >> 52) & 0x7FF);
    return eb == 0 ? 0 : eb == 0x7FF ? kNonFinite : eb - 1022 + HEAD;
}

// K-major shared-memory matrix descriptor (tcgen05 "matrix descriptor"):
// start address, leading byte offset (unused for swizzled K-major),
// stride byte offset between 8-row groups, version 1, swizzle mode.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t sbo_bytes, uint32_t swizzle) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)swizzle << 61;
    return d;
}

// Error-free sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// float-float accumulation (hi, lo) += x
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
}

// Two FP32 lanes in one 64-bit register: the packed f32x2 instructions add
// or subtract both lanes with IEEE round-to-nearest, so every lane computes
// exactly what the scalar instruction would, at half the instruction count.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float x, float y) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float& x, float& y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// TwoSum on both lanes.
__device__ __forceinline__ void two_sum2(f32x2 a, f32x2 b, f32x2& s, f32x2& e) {
    s = add2(a, b);
    const f32x2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

__device__ __forceinline__ int64_t packed_start(int64_t i, int64_t n) { return i * n - i * (i - 1) / 2; }

// ---------------------------------------------------------------------------
// Mode geometry
//
// Accumulators live in TMEM, 128 columns each (one N = 128 tile):
//   D group: exact per-chunk accumulators, order d -> accumulator d (d < ND),
//            drained after the chunk's last K-block;
//   F group: the other orders (FMIN..FMAX) in one accumulator, either over
//            the whole K (F_FINAL) or drained per chunk like the D group.
// The float-float running sums (hi, lo) of a thread's columns: hi in
// registers, lo in shared memory.  FP64_SUM: the output is hi + lo in FP64
// (the FP64 emulation); otherwise the FP32 sum of the pair, widened exactly
// (the FP32-accuracy modes, whose results carry 24 bits).

template <int MODE>
struct Geo;

// D group: orders 0..DMAX, order d into accumulator min(d, ND - 1), drained
// after every chunk of KC; accumulator 0 holds order 0 alone and is exact.
// Exactness bounds the chunk: with |d0| <= 256 a leading-digit product is at
// most 2^16 units, so KC = 256 keeps order 0 within 2^24; orders 1 and 2 add
// at most 2^16 and 5 * 2^13 units per K index.  HEAD bits of headroom would
// allow longer chunks (HEAD = 2: KC = 512 for orders 0-2) but shift the
// representation down by HEAD bits, so the inexact F group carries 2^HEAD
// times more of the result; for the FP64 emulation that F error over 512-deep
// chunks exceeds the 1e-11 bound, so HEAD stays 0.
// DBUF > 1 double-buffers the D group.  F group: orders FMIN..FMAX in one
// accumulator, over the whole K (F_FINAL) or drained per chunk.
template <>
struct Geo<MODE_BF16X3> {
    static constexpr int PARTS = 3, ELEM = 2, KBLK = 32, ROWB = 64, KSTEP = 16, NSTAGE = 3, NSTAGE2 = 4;
    static constexpr uint32_t SWZ = 4, SBO = 512;  // 64B swizzle
    static constexpr int KC = 256, ND = 2, DMAX = 2, DBUF = 2, FMIN = 1, FMAX = 0, HEAD = 0;  // no F group
    static constexpr bool F_FINAL = false, SLICED = true, FP64_SUM = false;
    static constexpr int EPI_WARPS = 16;
    // single-plan launches: 8 epilogue warps keep both halves of the
    // float-float sums in registers (64 columns each), leaving the shared
    // memory to one more stage (batched launches, whose tiles are short,
    // keep 16 warps)
    static constexpr bool LO_REGS = true;
    static constexpr uint32_t TMEM_COLS = 512, F_COL = 0;
    static constexpr uint32_t IDESC_KIND = (1u << 4) | (1u << 7) | (1u << 10);  // F32 D, bf16 A and B
};

template <>
struct Geo<MODE_TF32> {
    static constexpr int PARTS = 1, ELEM = 4, KBLK = 64, ROWB = 128, KSTEP = 8, NSTAGE = 3, NSTAGE2 = 4;
    static constexpr uint32_t SWZ = 2, SBO = 1024;  // 128B swizzle
    static constexpr int KC = 1 << 30, ND = 0, DMAX = -1, DBUF = 1, FMIN = 0, FMAX = 0, HEAD = 0;
    static constexpr bool F_FINAL = true, SLICED = false, FP64_SUM = false;
    static constexpr int EPI_WARPS = 8;
    static constexpr bool LO_REGS = false;
    static constexpr uint32_t TMEM_COLS = 128, F_COL = 0;
    static constexpr uint32_t IDESC_KIND = (1u << 4) | (2u << 7) | (2u << 10);  // F32 D, tf32 A and B
};

template <>
struct Geo<MODE_OZAKI> {
    static constexpr int PARTS = 6, ELEM = 2, KBLK = 16, ROWB = 32, KSTEP = 16, NSTAGE = 3, NSTAGE2 = 4;
    static constexpr uint32_t SWZ = 6, SBO = 256;  // 32B swizzle
    static constexpr int KC = 256, ND = 3, DMAX = 2, DBUF = 1, FMIN = 3, FMAX = 5, HEAD = 0;
    static constexpr bool F_FINAL = false, SLICED = true, FP64_SUM = true;
    static constexpr int EPI_WARPS = 16;
    static constexpr bool LO_REGS = false;
    static constexpr uint32_t TMEM_COLS = 512, F_COL = 384;
    static constexpr uint32_t IDESC_KIND = (1u << 4) | (1u << 7) | (1u << 10);  // F32 D, bf16 A and B
};

// Per-CTA shapes of the leaf GEMM.  CG == 1: one CTA computes a 128 x 128
// tile (M = N = 128).  CG == 2: a pair of CTAs computes a 256 x TN tile
// (M = 256, N = TN); each CTA holds 128 rows of the X parts, TN / 2 rows of
// the Y parts, and the 128 x TN accumulator rows of its half.  Halving the Y
// rows each CTA stages halves the B-operand shared-memory reads per MMA.
// TN = 256 for TF32 (one accumulator, so 256 TMEM columns hold it): twice
// the MMA work per staged byte, which the 4-byte operands need most; 128
// for the split modes, whose several accumulators fill TMEM at N = 128.
template <int MODE, int CG, int NB = 1>
struct Shape {
    using G = Geo<MODE>;
    static constexpr bool LO_REGS = G::LO_REGS && NB == 1;
    static constexpr int EPI_WARPS = LO_REGS ? 8 : G::EPI_WARPS;
    static constexpr int TN = MODE == MODE_TF32 && CG == 2 ? 256 : 128;
    static constexpr int XROWS = 128, YROWS = TN / CG;
    static constexpr uint32_t TMEM_COLS = G::ND == 0 && (uint32_t)TN > G::TMEM_COLS ? (uint32_t)TN : G::TMEM_COLS;
    // A K block of a part is ATOMS swizzle atoms (ROWB bytes per row each),
    // stored one after the other; KATOM elements per atom row, KS_ATOM MMA
    // K steps per atom.
    static constexpr int ATOMS = G::KBLK * G::ELEM / G::ROWB, KATOM = G::ROWB / G::ELEM;
    static constexpr int KS_ATOM = G::ROWB / (G::KSTEP * G::ELEM);
    static constexpr int ATOM_X = XROWS * G::ROWB, ATOM_Y = YROWS * G::ROWB;
    static constexpr int X_BYTES = ATOMS * ATOM_X, Y_BYTES = ATOMS * ATOM_Y;
    static_assert(ATOMS >= 1 && ATOMS * G::ROWB == G::KBLK * G::ELEM, "K block of whole swizzle atoms");
    static constexpr int STAGE = G::PARTS * (X_BYTES + Y_BYTES);
    static constexpr int LO = G::ND > 0 && !LO_REGS ? 128 * 128 * 4 : 0;  // float-float lo halves, [col][row]
    static constexpr int NSTAGE = (CG == 1 || TN > 128 ? G::NSTAGE : G::NSTAGE2) + (LO_REGS ? 1 : 0);
    // CG == 2 keeps at least Y_BYTES of allocation after the last stage, so
    // that the operand reads of its last Y part stay inside this CTA's
    // shared memory whatever the B rows the pair MMA takes per CTA
    static constexpr int TAIL = CG == 2 && LO < Y_BYTES ? Y_BYTES : 0;
    static constexpr int SMEM = NSTAGE * STAGE + LO + 1024 /*align*/ + 256 /*barriers*/ + TAIL;
    static constexpr uint32_t IDESC = G::IDESC_KIND | (((uint32_t)TN >> 3) << 17) | ((128u * CG >> 4) << 24);
    static constexpr int THREADS = 32 * (3 + EPI_WARPS);  // TMA, MMA, epilogue warps, wait helper
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};

// Position of K block kb (of nkb) in the exact D chunks (kbpc blocks each)
// and in the F chunks (FKC blocks each), which start FOFF blocks later (the
// first F chunk is FOFF blocks long).  f_before_d: a D chunk starts here
// while an F chunk continues, so the stage's F MMAs are issued before the
// wait for the previous D chunk's drain.
struct StageFlags {
    bool first_in_chunk, last_in_chunk, f_first, f_last, f_before_d;
};
template <int kbpc, int FOFF, int FKC = kbpc>
__device__ __forceinline__ StageFlags stage_flags(int kb, int nkb) {
    const int kr = kb % kbpc;
    StageFlags f;
    f.first_in_chunk = kr == 0;
    f.last_in_chunk = kr == kbpc - 1 || kb == nkb - 1;
    if constexpr (FOFF > 0) {
        f.f_first = kb == 0 || (kb >= FOFF && (kb - FOFF) % FKC == 0);
        f.f_last = (kb + 1 - FOFF) % FKC == 0 || kb == nkb - 1;
    } else {
        f.f_first = kb == 0 || kr == 0;
        f.f_last = kr == kbpc - 1 || kb == nkb - 1;
    }
    f.f_before_d = FOFF > 0 && f.first_in_chunk && kb != 0 && !f.f_first;
    return f;
}

// The MMA issuer warp and the wait helper warp meet at named barrier 1 (both
// warps, all lanes); each passes whether it gives up, and both learn whether
// either did.  Returns true when neither gave up.
__device__ __forceinline__ bool meet_helper(bool give_up) {
    uint32_t any;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "barrier.red.or.pred p, 1, 64, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(any)
        : "r"(give_up ? 1u : 0u)
        : "memory");
    return any == 0;
}

// ---------------------------------------------------------------------------
// Operand preparation

// Loads a 64 (K) x 64 (column) tile of a leaf operand (a signed sum of
// terms, zero outside each term's extent) into registers: thread t holds the
// VEC consecutive columns starting at (t % VPR) * VEC of the rows
// t / VPR + RPP * pass, pass < NPASS.  Every row of one term is loaded before
// any of them is used, so a thread has NPASS 16-byte loads in flight; a term
// whose VEC columns are inside it and 16-byte aligned is read with vector
// loads, else element by element.  A single term needs no floating-point
// addition (its sign is applied to the bits).
constexpr int PT = 64;  // prep tile edge

template <typename TS>
struct TileRegs {
    static constexpr int VEC = 16 / sizeof(TS);
    static constexpr int VPR = PT / VEC;     // vectors per tile row
    static constexpr int RPP = 256 / VPR;    // rows per pass
    static constexpr int NPASS = PT / RPP;
    TS v[NPASS][VEC];
};

template <typename TS>
__device__ __forceinline__ TS flip_sign(TS x) {
    if constexpr (sizeof(TS) == 8)
        return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
    else
        return __uint_as_float(__float_as_uint(x) ^ 0x80000000u);
}

// One term's values of the tile, as stored (its sign not applied), zero
// outside the term's extent.
template <typename TS, int NB>
__device__ __forceinline__ void load_term_raw(const BindSet<NB>& bs, const Term& tm, int K, int k0, int c0,
                                              TS (&x)[TileRegs<TS>::NPASS][TileRegs<TS>::VEC]) {
    using TR = TileRegs<TS>;
    constexpr int VEC = TR::VEC, NPASS = TR::NPASS;
    const int vc = (threadIdx.x % TR::VPR) * VEC;
    const int r0 = threadIdx.x / TR::VPR;
    const Bind& b = bs.b[tm.inst];
    const TS* base = term_base<TS>(b, tm.buf);
    const int c = c0 + vc;
    const TS* colp = base + tm.off + c;
    const int kmax = min(K, tm.rows);
    const bool vec_ok = c + VEC <= tm.cols && ((reinterpret_cast<uintptr_t>(colp) & 15) == 0) &&
                        ((tm.ld * (int64_t)sizeof(TS)) & 15) == 0;
    if (vec_ok) {
#pragma unroll
        for (int p = 0; p < NPASS; ++p) {
            const int k = k0 + r0 + p * TR::RPP;
            uint4 u = make_uint4(0u, 0u, 0u, 0u);
            if (k < kmax) u = __ldg(reinterpret_cast<const uint4*>(colp + (int64_t)k * tm.ld));
            *reinterpret_cast<uint4*>(x[p]) = u;
        }
    } else {
#pragma unroll
        for (int p = 0; p < NPASS; ++p) {
            const int k = k0 + r0 + p * TR::RPP;
#pragma unroll
            for (int j = 0; j < VEC; ++j)
                x[p][j] = (k < kmax && c + j < tm.cols) ? __ldg(colp + (int64_t)k * tm.ld + j) : TS(0);
        }
    }
}

template <typename TS, int NB>
__device__ __forceinline__ void load_operand_regs(const BindSet<NB>& bs, const Term* __restrict__ terms, int t0,
                                                  int nt, int K, int k0, int c0, TileRegs<TS>& R) {
    using TR = TileRegs<TS>;
    constexpr int VEC = TR::VEC, NPASS = TR::NPASS;
#pragma unroll
    for (int p = 0; p < NPASS; ++p)
#pragma unroll
        for (int j = 0; j < VEC; ++j) R.v[p][j] = TS(0);
    for (int t = 0; t < nt; ++t) {
        const Term tm = terms[t0 + t];
        TS x[NPASS][VEC];
        load_term_raw<TS>(bs, tm, K, k0, c0, x);
        if (nt == 1) {
            if (tm.neg) {
#pragma unroll
                for (int p = 0; p < NPASS; ++p)
#pragma unroll
                    for (int j = 0; j < VEC; ++j) R.v[p][j] = flip_sign(x[p][j]);
            } else {
#pragma unroll
                for (int p = 0; p < NPASS; ++p)
#pragma unroll
                    for (int j = 0; j < VEC; ++j) R.v[p][j] = x[p][j];
            }
        } else {
#pragma unroll
            for (int p = 0; p < NPASS; ++p)
#pragma unroll
                for (int j = 0; j < VEC; ++j) R.v[p][j] = tm.neg ? R.v[p][j] - x[p][j] : R.v[p][j] + x[p][j];
        }
    }
}

// The same tile stored to shared memory, tile[k][c].
template <typename TS, int NB>
__device__ __forceinline__ void load_operand_tile(const BindSet<NB>& bs, const Term* __restrict__ terms, int t0,
                                                  int nt, int K, int k0, int c0, TS (*tile)[PT + 1]) {
    using TR = TileRegs<TS>;
    TileRegs<TS> R;
    load_operand_regs<TS>(bs, terms, t0, nt, K, k0, c0, R);
    const int vc = (threadIdx.x % TR::VPR) * TR::VEC;
    const int r0 = threadIdx.x / TR::VPR;
#pragma unroll
    for (int p = 0; p < TR::NPASS; ++p)
#pragma unroll
        for (int j = 0; j < TR::VEC; ++j) tile[r0 + p * TR::RPP][vc + j] = R.v[p][j];
}

// Column maxima of |operand| (sliced modes): atomicMax on the FP64 bit
// pattern (positive doubles order like their bits; Inf and NaN order above
// every finite value).  Block: rows [k0, k1) (up to kColSpan) of a 64-column
// strip, read two 64-row tiles at a time (16 loads in flight per thread),
// reduced in registers over a thread's rows, then across the threads of a
// column; one atomic per column and block.
template <typename TS>
using AbsBits = std::conditional_t<sizeof(TS) == 8, unsigned long long, unsigned int>;
template <typename TS>
__device__ __forceinline__ AbsBits<TS> abs_bits(TS x) {
    if constexpr (sizeof(TS) == 8)
        return (unsigned long long)__double_as_longlong((double)x) & 0x7FFFFFFFFFFFFFFFull;
    else
        return __float_as_uint((float)x) & 0x7FFFFFFFu;
}

// Four blocks per SM (64 registers, no spills): each block's chain of
// table loads (task, product, term, binding) before its data loads is
// latency, which more resident blocks overlap.
template <int NB, typename TS>
__global__ void __launch_bounds__(256, 4) tc_colmax_kernel(const __grid_constant__ BindSet<NB> bs,
                                                        const LeafProduct* __restrict__ prods,
                                                        const Term* __restrict__ terms,
                                                        const TcProd* __restrict__ tcp,
                                                        const PrepTask* __restrict__ tasks) {
    using TR = TileRegs<TS>;
    using MB = AbsBits<TS>;  // magnitude bits: 32-bit compares for FP32 values
    constexpr int NRED = 256 / TR::VPR;  // threads sharing a column vector
    __shared__ MB red[NRED][PT];
    const PrepTask tk = tasks[blockIdx.x];
    const LeafProduct& lp = prods[tk.prod];
    const int t0 = tk.side ? lp.y0 : lp.x0, nt = tk.side ? lp.ny : lp.nx;
    // where the block's maxima go, read before the tiles
    unsigned long long* ex = reinterpret_cast<unsigned long long*>(tk.side ? tcp[tk.prod].ey : tcp[tk.prod].ex);
    MB m[TR::VEC];
#pragma unroll
    for (int j = 0; j < TR::VEC; ++j) m[j] = 0;
    // magnitudes compared as bit patterns (integer operations only)
    auto take = [&](const TS (&x0)[TR::NPASS][TR::VEC], const TS (&x1)[TR::NPASS][TR::VEC]) {
#pragma unroll
        for (int j = 0; j < TR::VEC; ++j)
#pragma unroll
            for (int p = 0; p < TR::NPASS; ++p) {
                const MB b0 = abs_bits(x0[p][j]), b1 = abs_bits(x1[p][j]);
                const MB b = b0 > b1 ? b0 : b1;
                m[j] = b > m[j] ? b : m[j];
            }
    };
    if (nt == 1) {
        // one term: its sign does not change a magnitude, so both tiles'
        // loads are issued before any value is used
        const Term tm = terms[t0];
        for (int k = tk.k0; k < tk.k1; k += 2 * PT) {
            TS x0[TR::NPASS][TR::VEC], x1[TR::NPASS][TR::VEC];
            load_term_raw<TS>(bs, tm, tk.k1, k, tk.c0, x0);
            load_term_raw<TS>(bs, tm, tk.k1, k + PT, tk.c0, x1);
            take(x0, x1);
        }
    } else {
        for (int k = tk.k0; k < tk.k1; k += 2 * PT) {
            TileRegs<TS> R0, R1;
            load_operand_regs<TS>(bs, terms, t0, nt, tk.k1, k, tk.c0, R0);
            load_operand_regs<TS>(bs, terms, t0, nt, tk.k1, k + PT, tk.c0, R1);
            take(R0.v, R1.v);
        }
    }
    const int vc = (threadIdx.x % TR::VPR) * TR::VEC;
    const int r0 = threadIdx.x / TR::VPR;
#pragma unroll
    for (int j = 0; j < TR::VEC; ++j) red[r0][vc + j] = m[j];
    __syncthreads();
    if (threadIdx.x < PT) {
        const int col = threadIdx.x;
        MB mb = red[0][col];
#pragma unroll
        for (int i = 1; i < NRED; ++i) mb = red[i][col] > mb ? red[i][col] : mb;
        if (mb != 0) {
            unsigned long long mx = mb;
            if constexpr (sizeof(TS) == 4) mx = (unsigned long long)__double_as_longlong((double)__uint_as_float(mb));
            atomicMax(ex + tk.c0 + col, mx);
        }
    }
}

// Balanced base-256 digits of v = round(x * 2^(8S - E)), most significant
// first: x * 2^-E ~= sum_s d[s] * 2^(-8(s+1)), |d[0]| <= 256 >> HEAD (E
// carries the column's headroom), d[s>0] in [-128, 127].  They are kept
// biased, b[s] = d[s] + 128: adding 128 to every base-256 position below the
// top one turns the balanced digits into the plain bytes of u = v + bias
// (each d[s] + 128 lies in [0, 255]), and the top digit is the arithmetic
// shift of u plus 128.  Integer arithmetic only.
//
// v from the bits of x: the significand shifted right by r, rounded to
// nearest (ties up) as ((m >> (r - 1)) + 1) >> 1; 0 for zero and subnormal
// x.  Every value of a column lies below 2^E (E comes from the column's
// maximum, or is kNonFinite, which shifts everything out), so r = E - e + 4
// >= 5 for x = f * 2^e and no left shift arises (r < 1 would shift
// everything out).  Non-finite x occur only in non-finite columns and give 0.
template <int S>
__device__ __forceinline__ long long fixed_point(double x, int E) {
    const long long bits = __double_as_longlong(x);
    const int eb = (int)((bits >> 52) & 0x7FF);
    const int r = E - 8 * S + 1075 - eb;  // right shift to units of 2^(E - 8S)
    const long long m = (bits & ((1LL << 52) - 1)) | (1LL << 52);
    long long v = ((m >> min((unsigned int)(r - 1), 63u)) + 1) >> 1;
    if (eb == 0) v = 0;
    return bits < 0 ? -v : v;
}

// u = v + bias of a fixed-point value v (|v| <= 2^(8S) + a few units): the
// biased digits of v are the bytes of u below the top one.
template <int S>
__device__ __forceinline__ long long biased_value(long long v) {
    constexpr long long bias = (long long)(((unsigned long long)1 << (8 * (S - 1))) - 1) / 255 * 128;
    return v + bias;
}

// The same for an FP32 value and S = 3 (24 bits) in 32-bit integers.  Every
// value of the column lies below 2^E (or E is kNonFinite), so the right
// shift to units of 2^(E - 24) is t = E + 126 - eb >= 0 and the rounding
// (((2 m) >> t) + 1) >> 1 (ties up) stays within 32 bits; t >= 25 gives 0.
__device__ __forceinline__ int biased_value_f32(float x, int E) {
    const unsigned int bits = __float_as_uint(x);
    const int eb = (int)((bits >> 23) & 0xFF);
    const unsigned int m2 = ((bits & 0x7FFFFFu) | 0x800000u) << 1;
    unsigned int v = ((m2 >> min((unsigned int)(E + 126 - eb), 31u)) + 1u) >> 1;
    if (eb == 0) v = 0;
    return ((bits >> 31) ? -(int)v : (int)v) + 0x8080;
}

// FP32 bits of (b - 128) * 2^-8(s+1) for biased digit b = b[s] of u, in
// [-128, 384]: b is placed in the significand of 1.5 * 2^23 (exact integer
// float; for s > 0 one byte permute inserts the byte of u), one FMA removes
// the offset and applies the power of two (exact: the result has at most 9
// significant bits), and the bf16 is the upper half of the float's bits,
// exact since its low 16 bits are zero.
__host__ __device__ constexpr float exp2_neg(int e) {
    float r = 1.0f;
    for (int i = 0; i < e; ++i) r *= 0.5f;
    return r;
}

template <int S, int s, typename U>
__device__ __forceinline__ uint32_t digit_f32_bits(U u) {
    constexpr float scale = exp2_neg(8 * (s + 1));
    uint32_t fb;
    if constexpr (s == 0) {
        fb = 0x4B400000u + 128u + (uint32_t)(int)(u >> (8 * (S - 1)));
    } else {
        constexpr int byte = S - 1 - s;  // position of digit s in u
        const uint32_t w = byte < 4 ? (uint32_t)u : (uint32_t)((unsigned long long)u >> 32);
        fb = __byte_perm(w, 0x4B400000u, 0x7650u + (byte & 3));  // 0x4B4000bb
    }
    return __float_as_uint(fmaf(__uint_as_float(fb), scale, -12583040.0f * scale));  // (12582912 + 128) * scale
}

// Two bf16 (the upper halves of lo's and hi's float bits) in one 32-bit word,
// lo at the lower address.
__device__ __forceinline__ uint32_t pack_bf16_hi(uint32_t lo_bits, uint32_t hi_bits) {
    return __byte_perm(lo_bits, hi_bits, 0x7632);
}

template <int MODE>
struct PrepSrc {
    using T = float;
};
template <>
struct PrepSrc<MODE_OZAKI> {
    using T = double;
};

// Writes the S parts of 8 consecutive K values of one column (their biased
// values u, 32-bit integers for S <= 3): part s gets the 8 bf16 of digit s,
// 16 bytes at out + s * part_elems + base.
template <int S, int s = 0, typename U>
__device__ __forceinline__ void store_parts(const U (&u)[8], __nv_bfloat16* out, int64_t part_elems,
                                            int64_t base) {
    uint4 q;
    q.x = pack_bf16_hi(digit_f32_bits<S, s>(u[0]), digit_f32_bits<S, s>(u[1]));
    q.y = pack_bf16_hi(digit_f32_bits<S, s>(u[2]), digit_f32_bits<S, s>(u[3]));
    q.z = pack_bf16_hi(digit_f32_bits<S, s>(u[4]), digit_f32_bits<S, s>(u[5]));
    q.w = pack_bf16_hi(digit_f32_bits<S, s>(u[6]), digit_f32_bits<S, s>(u[7]));
    *reinterpret_cast<uint4*>(out + s * part_elems + base) = q;
    if constexpr (s + 1 < S) store_parts<S, s + 1>(u, out, part_elems, base);
}

// Parts of one 64 (K) x 64 (column) tile of a leaf operand, written K-major:
// part q of column c, K index k at parts + ((q * rows_pad + c) * K_pad + k).
// Each thread slices two (column, 8 K values) runs and writes 16 bytes per
// part and run.  Six blocks per SM (40 registers, no spills; 17 KB of
// shared memory each) overlap the blocks' table-load chains: 12% less time
// than four at 16384 x 8192 bf16x3, 5% less for the batched step.
template <int NB, int MODE>
__global__ void __launch_bounds__(256, 6) tc_prep_kernel(const __grid_constant__ BindSet<NB> bs,
                                                      const LeafProduct* __restrict__ prods,
                                                      const Term* __restrict__ terms,
                                                      const TcProd* __restrict__ tcp,
                                                      const PrepTask* __restrict__ tasks) {
    using TS = typename PrepSrc<MODE>::T;
    __shared__ TS tile[PT][PT + 1];
    const PrepTask tk = tasks[blockIdx.x];
    const LeafProduct& lp = prods[tk.prod];
    const int t0 = tk.side ? lp.y0 : lp.x0, nt = tk.side ? lp.ny : lp.nx;
    // where the slices go and where the column scales are, read before the
    // tile, so that these loads wait together with the tile's instead of
    // after the barrier
    const int rows_pad = tk.side ? lp.r_pad : lp.p_pad, K_pad = lp.K_pad;
    char* parts = bs.b[lp.inst].W + (tk.side ? lp.tc_y_off : lp.tc_x_off);
    const unsigned long long* ex =
        reinterpret_cast<const unsigned long long*>(tk.side ? tcp[tk.prod].ey : tcp[tk.prod].ex);
    load_operand_tile<TS>(bs, terms, t0, nt, lp.K, tk.k0, tk.c0, tile);
    __syncthreads();
    const int64_t part_elems = (int64_t)rows_pad * K_pad;
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
        const int item = threadIdx.x + rep * 256;
        const int col = item >> 3, kc = item & 7;
        const int c = tk.c0 + col;
        const int64_t base = (int64_t)c * K_pad + tk.k0 + kc * 8;
        if constexpr (MODE == MODE_TF32) {
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t r;
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(tile[kc * 8 + i][col]));
                v[i] = __uint_as_float(r);
            }
            float* out = reinterpret_cast<float*>(parts);
            *reinterpret_cast<uint4*>(out + base) = *reinterpret_cast<const uint4*>(v);
            *reinterpret_cast<uint4*>(out + base + 4) = *reinterpret_cast<const uint4*>(v + 4);
        } else {
            constexpr int S = Geo<MODE>::PARTS;
            const int E = col_exponent<Geo<MODE>::HEAD>(__ldg(ex + c));
            std::conditional_t<sizeof(TS) == 8, long long, int> u[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if constexpr (sizeof(TS) == 8)
                    u[i] = biased_value<S>(fixed_point<S>(tile[kc * 8 + i][col], E));
                else
                    u[i] = biased_value_f32(tile[kc * 8 + i][col], E);
            }
            __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(parts);
            store_parts<S>(u, out, part_elems, base);
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 emulation: operands formed in fixed point
//
// A leaf operand is a signed sum of blocks (of A, or of materialised sums).
// Its column c is scaled by 2^-E(c) with
//     E(c) = max_t E_t(c) + ceil(log2 n(c)),
// E_t(c) the exponent of block t's column maximum and n(c) the number of
// blocks with a nonzero column c, so that |sum| <= n(c) max_t |x_t| < 2^E(c).
// Every block value is converted exactly to the fixed point of that scale
// (rounded to the nearest unit of 2^(E - 48)) and the blocks are added in
// 64-bit integers: the Strassen operand sums are formed without
// floating-point arithmetic, each term adding at most half a unit.  The
// slices are the digits of the integer sum.  A single-block operand gets
// exactly the scale and digits of the plain slicing.

// Column maxima of row segments of the operand blocks (tasks: prod = index
// of the segment's term, rows [k0, k1) of columns [c0, c0 + 64); term_mx:
// offset of each segment's maxima in term_max).  Tasks of up to 256 rows,
// one 64-row tile in flight per thread and four blocks per SM (64
// registers): 10000^2 has about 6300 tasks, so the last wave is short
// (1024-row tasks, two tiles in flight and three blocks per SM took 5% longer
// at 4500^2).
constexpr int kAtomSpan = 256;  // rows of a column-maximum task of an atom

template <int NB>
__global__ void __launch_bounds__(256, 4) tc_termmax_kernel(const __grid_constant__ BindSet<NB> bs,
                                                         const Term* __restrict__ terms,
                                                         const PrepTask* __restrict__ tasks,
                                                         const int64_t* __restrict__ term_mx,
                                                         unsigned long long* __restrict__ term_max) {
    using TR = TileRegs<double>;
    constexpr int NRED = 256 / TR::VPR;
    __shared__ unsigned long long red[NRED][PT];
    const PrepTask tk = tasks[blockIdx.x];
    unsigned long long m[TR::VEC];
#pragma unroll
    for (int j = 0; j < TR::VEC; ++j) m[j] = 0;
    // a segment is one block of one buffer, read as stored (a sign does not
    // change a magnitude)
    const Term tm = terms[tk.prod];
    for (int k = tk.k0; k < tk.k1; k += PT) {
        double x0[TR::NPASS][TR::VEC];
        load_term_raw<double>(bs, tm, tk.k1, k, tk.c0, x0);
#pragma unroll
        for (int j = 0; j < TR::VEC; ++j)
#pragma unroll
            for (int p = 0; p < TR::NPASS; ++p) {
                const unsigned long long b = abs_bits(x0[p][j]);
                m[j] = b > m[j] ? b : m[j];
            }
    }
    const int vc = (threadIdx.x % TR::VPR) * TR::VEC;
    const int r0 = threadIdx.x / TR::VPR;
#pragma unroll
    for (int j = 0; j < TR::VEC; ++j) red[r0][vc + j] = m[j];
    __syncthreads();
    if (threadIdx.x < PT) {
        const int col = threadIdx.x;
        unsigned long long mx = red[0][col];
#pragma unroll
        for (int i = 1; i < NRED; ++i) mx = red[i][col] > mx ? red[i][col] : mx;
        if (mx != 0) atomicMax(term_max + term_mx[tk.prod] + tk.c0 + col, mx);
    }
}

// Column scales of the operands (tasks: one per 64-column strip of every
// distinct operand): E(c) from the maxima of the operand's blocks, stored as
// an integer for the slicing kernel and as FP64 bits (whose exponent gives E)
// for the GEMM epilogue.
__global__ void __launch_bounds__(PT) tc_scale_kernel(const LeafProduct* __restrict__ prods,
                                                      const Term* __restrict__ terms,
                                                      const TcProd* __restrict__ tcp,
                                                      const PrepTask* __restrict__ tasks,
                                                      const int64_t* __restrict__ term_mx,
                                                      const int64_t* __restrict__ mx_list,
                                                      const unsigned long long* __restrict__ term_max,
                                                      int* __restrict__ col_e) {
    using G = Geo<MODE_OZAKI>;
    const PrepTask tk = tasks[blockIdx.x];
    const LeafProduct& lp = prods[tk.prod];
    const int t0 = tk.side ? lp.y0 : lp.x0, nt = tk.side ? lp.ny : lp.nx;
    const int c = tk.c0 + threadIdx.x;
    int emax = 0, cnt = 0;
    bool nonfinite = false;
    for (int t = 0; t < nt; ++t) {
        if (c >= terms[t0 + t].cols) continue;
        unsigned long long mx = 0;  // the maximum over the block's row segments
        for (int64_t a = term_mx[t0 + t]; mx_list[a] >= 0; ++a) {
            const unsigned long long v = term_max[mx_list[a] + c];
            mx = v > mx ? v : mx;
        }
        if (mx == 0) continue;
        const int e = col_exponent<G::HEAD>(mx);
        nonfinite |= e >= kNonFinite;
        emax = cnt == 0 ? e : max(emax, e);
        ++cnt;
    }
    const int E = nonfinite ? kNonFinite : cnt > 1 ? emax + (32 - __clz(cnt - 1)) : emax;
    const TcProd& tp = tcp[tk.prod];
    col_e[(tk.side ? tp.ey_index : tp.ex_index) + c] = E;
    const unsigned long long bits = cnt == 0   ? 0ull
                                    : nonfinite ? 0x7FF0000000000000ull
                                                : (unsigned long long)(E - G::HEAD + 1022) << 52;
    (tk.side ? tp.ey : tp.ex)[c] = bits;
}

// Parts of one 64 (K) x 64 (column) tile of a leaf operand (as
// tc_prep_kernel), the operand formed in fixed point at the column scales
// that tc_scale_kernel computed.
template <int NB>
__global__ void __launch_bounds__(256) tc_prep_fixed_kernel(const __grid_constant__ BindSet<NB> bs,
                                                            const LeafProduct* __restrict__ prods,
                                                            const Term* __restrict__ terms,
                                                            const TcProd* __restrict__ tcp,
                                                            const PrepTask* __restrict__ tasks,
                                                            const int* __restrict__ col_e) {
    using TR = TileRegs<double>;
    constexpr int S = Geo<MODE_OZAKI>::PARTS;
    __shared__ long long tile[PT][PT + 1];
    const PrepTask tk = tasks[blockIdx.x];
    const LeafProduct& lp = prods[tk.prod];
    const int t0 = tk.side ? lp.y0 : lp.x0, nt = tk.side ? lp.ny : lp.nx;
    {
        const int vc = (threadIdx.x % TR::VPR) * TR::VEC;
        const int r0 = threadIdx.x / TR::VPR;
        const int* ce = col_e + (tk.side ? tcp[tk.prod].ey_index : tcp[tk.prod].ex_index) + tk.c0 + vc;
        int Ec[TR::VEC];
#pragma unroll
        for (int j = 0; j < TR::VEC; ++j) Ec[j] = __ldg(ce + j);
        long long acc[TR::NPASS][TR::VEC];
#pragma unroll
        for (int p = 0; p < TR::NPASS; ++p)
#pragma unroll
            for (int j = 0; j < TR::VEC; ++j) acc[p][j] = 0;
        for (int t = 0; t < nt; ++t) {
            TileRegs<double> R;
            load_operand_regs<double>(bs, terms, t0 + t, 1, lp.K, tk.k0, tk.c0, R);  // signed term values
#pragma unroll
            for (int p = 0; p < TR::NPASS; ++p)
#pragma unroll
                for (int j = 0; j < TR::VEC; ++j) acc[p][j] += fixed_point<S>(R.v[p][j], Ec[j]);
        }
#pragma unroll
        for (int p = 0; p < TR::NPASS; ++p)
#pragma unroll
            for (int j = 0; j < TR::VEC; ++j) tile[r0 + p * TR::RPP][vc + j] = acc[p][j];
    }
    __syncthreads();
    const int rows_pad = tk.side ? lp.r_pad : lp.p_pad;
    const Bind& b = bs.b[lp.inst];
    __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(b.W + (tk.side ? lp.tc_y_off : lp.tc_x_off));
    const int64_t part_elems = (int64_t)rows_pad * lp.K_pad;
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
        const int item = threadIdx.x + rep * 256;
        const int col = item >> 3, kc = item & 7;
        const int64_t base = (int64_t)(tk.c0 + col) * lp.K_pad + tk.k0 + kc * 8;
        long long u[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) u[i] = biased_value<S>(tile[kc * 8 + i][col]);
        store_parts<S>(u, out, part_elems, base);
    }
}

// ---------------------------------------------------------------------------
// Persistent tcgen05 GEMM over leaf tiles
//
// Warps: 0 TMA producer (lane 0), 1 MMA issuer (lane 0 issues, the warp
// meets the helper), 2 .. 1 + EPI_WARPS epilogue (TMEM drains and stores),
// 2 + EPI_WARPS wait helper (the issuer's pipeline-barrier waits).
// CG == 1: one CTA per SM, each CTA takes tiles blockIdx.x, + gridDim.x, ...
// CG == 2: clusters of two CTAs (a pair on two SMs); each pair takes tiles
// clusterid, + nclusterid, ...  Both CTAs run the TMA producer for their own
// halves (completing on the even CTA's full barrier, which expects the bytes
// of both) and the epilogue for their own 128 rows; the even CTA's MMA warp
// issues the MMAs, whose commits arrive on the barriers of both CTAs.  The
// even CTA's dempty / fempty barriers count the epilogue warps of both.

template <int NB, int MODE, int CG>
__global__ void __launch_bounds__(Shape<MODE, CG, NB>::THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ BindSet<NB> bs, const TcProd* __restrict__ tcp,
                   const LeafTile* __restrict__ sched, const int32_t* __restrict__ wfirst,
                   int* __restrict__ status, uint64_t wait_ns) {
    using G = Geo<MODE>;
    using SH = Shape<MODE, CG, NB>;
    constexpr int NSTAGE = SH::NSTAGE;
    constexpr int NCOL = SH::TN / (SH::EPI_WARPS / 4);  // columns per epilogue thread
    constexpr int NG = NCOL / 16;                   // 16-column groups per thread
    constexpr int kbpc = G::KC / G::KBLK > 0 ? G::KC / G::KBLK : 1;
    constexpr bool HAS_F = G::FMIN <= G::FMAX;
    constexpr int NKS = G::KBLK / G::KSTEP;
    // F chunks (drained per chunk) start FOFF stages after the D chunks, so
    // that a D drain overlaps the F MMAs of two stages (see the MMA issuer)
    constexpr int FOFF = (G::ND > 0 && HAS_F && !G::F_FINAL) ? kbpc / 2 : 0;
    // F chunks of two D chunks: F holds only orders 3-5 (below 2^-24 of the
    // result), whose FP32 accumulation error over 512 K values stays far
    // below the FP64-emulation bound (measured: 10000^2 6.8e-13, unchanged)
    constexpr int FKC = FOFF > 0 ? 2 * kbpc : kbpc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // lo halves of the running float-float sums, column pairs interleaved:
    // element (row, col) at lo_s[((col / 2) * 128 + row) * 2 + col % 2]
    float* lo_s = reinterpret_cast<float*>(smem + NSTAGE * SH::STAGE);
    f32x2* lo2_s = reinterpret_cast<f32x2*>(lo_s);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSTAGE * SH::STAGE + SH::LO);
    // barriers: full[NSTAGE] empty[NSTAGE] dfull[DBUF] dempty[DBUF] ffull fempty done ; tmem slot
    const uint32_t b_full = smem_u32(bars), b_empty = b_full + 8 * NSTAGE;
    const uint32_t b_dfull = b_empty + 8 * NSTAGE, b_dempty = b_dfull + 8 * G::DBUF;
    const uint32_t b_ffull = b_dempty + 8 * G::DBUF, b_fempty = b_ffull + 8, b_done = b_fempty + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NSTAGE + 2 * G::DBUF + 3);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = CG == 1 ? 0u : cluster_rank();
    // this worker's tiles (a CTA, or a CTA pair): sched[t_beg .. t_end)
    const int worker = CG == 1 ? (int)blockIdx.x : (int)cluster_index();
    const int t_beg = __ldg(wfirst + worker), t_end = __ldg(wfirst + worker + 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(b_full + 8 * s, 1);
            mbar_init(b_empty + 8 * s, 1);
        }
        for (int s = 0; s < G::DBUF; ++s) {
            mbar_init(b_dfull + 8 * s, 1);
            mbar_init(b_dempty + 8 * s, SH::EPI_WARPS * CG);
        }
        mbar_init(b_ffull, 1);
        mbar_init(b_fempty, SH::EPI_WARPS * CG);
        mbar_init(b_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc<CG>(smem_u32(tmem_slot), SH::TMEM_COLS);
        tmem_relinquish<CG>();
    }
    tc_fence_before();
    if constexpr (CG == 1)
        __syncthreads();
    else
        cluster_sync_all();  // both CTAs' barriers initialised and TMEM allocated
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t smem_base = smem_u32(smem);
    // barriers that the epilogue warps of both CTAs arrive on: the even CTA's
    const uint32_t b_dempty_c = CG == 1 ? b_dempty : map_to_rank(b_dempty, 0);
    const uint32_t b_fempty_c = CG == 1 ? b_fempty : map_to_rank(b_fempty, 0);
    const uint32_t b_full_c = CG == 1 ? b_full : map_to_rank(b_full, 0);

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int t = t_beg; t < t_end && ok; ++t) {
                const LeafTile lt = sched[t];
                const TcProd* pr = tcp + lt.prod;
                const int nkb = pr->K_pad / G::KBLK;
                const int ya = lt.ti * (128 * CG) + (int)rank * SH::XROWS;
                const int yb = lt.tj * SH::TN + (int)rank * SH::YROWS;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const uint32_t s = it % NSTAGE, ph = (it / NSTAGE) & 1;
                    if (!mbar_wait<CG>(b_empty + 8 * s, ph ^ 1, status, ERR_TIMEOUT_PRODUCER, wait_ns)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_expect_tx(b_full + 8 * s, CG * SH::STAGE);
                    const uint32_t st = smem_base + s * SH::STAGE;
#pragma unroll
                    for (int q = 0; q < G::PARTS; ++q)
#pragma unroll
                        for (int a = 0; a < SH::ATOMS; ++a) {
                            const int kx = kb * G::KBLK + a * SH::KATOM;
                            tma_load_2d<CG>(st + q * SH::X_BYTES + a * SH::ATOM_X, &pr->tmx, b_full_c + 8 * s, kx,
                                            q * pr->p_pad + ya);
                            tma_load_2d<CG>(st + G::PARTS * SH::X_BYTES + q * SH::Y_BYTES + a * SH::ATOM_Y, &pr->tmy,
                                            b_full_c + 8 * s, kx, q * pr->r_pad + yb);
                        }
                }
            }
            // copies still in flight land before the CTA may exit (bounded): the
            // even CTA sees its full barriers complete; the odd CTA, whose copies
            // complete on the even CTA's barriers, waits until the MMAs that read
            // them have released the stage
            const uint32_t n_in_flight = it < (uint32_t)NSTAGE ? it : (uint32_t)NSTAGE;
            for (uint32_t j = 0; j < n_in_flight; ++j) {
                const uint32_t i2 = it - 1 - j;
                const uint32_t s = i2 % NSTAGE, ph = (i2 / NSTAGE) & 1;
                if (rank == 0)
                    mbar_wait_quiet<CG>(b_full + 8 * s, ph);
                else
                    mbar_wait_quiet<CG>(b_empty + 8 * s, ph);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        // The warp runs the loop together and lane 0 issues.  It waits on no
        // pipeline barrier itself (a barrier wait in the issuing thread stalls
        // the MMA stream): the wait helper warp makes those waits and meets this
        // warp at named barrier 1 once a stage's operands (and the accumulators
        // it overwrites) are ready, with a flag that ends both loops together
        // when a wait gave up.
        if (rank == 0) {
            uint32_t it = 0, chunk = 0, fchunk = 0;
            bool ok = true;
            // Operand descriptors of stage 0, part 0; the others differ only in
            // the start-address field (16-byte units, below 2^14 for every
            // shared-memory address), so each is one add of a constant.
            const uint64_t desc_a0 = make_desc(smem_base, G::SBO, G::SWZ);
            const uint64_t desc_b0 = make_desc(smem_base + G::PARTS * SH::X_BYTES, G::SBO, G::SWZ);
            for (int t = t_beg; t < t_end && ok; ++t) {
                const LeafTile lt = sched[t];
                const int nkb = tcp[lt.prod].K_pad / G::KBLK;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const StageFlags fl = stage_flags<kbpc, FOFF, FKC>(kb, nkb);
                    const uint32_t buf = chunk % G::DBUF;
                    const uint32_t s = it % NSTAGE;
                    if (!meet_helper(false)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t da = desc_a0 + (uint64_t)(s * (SH::STAGE >> 4));
                    const uint64_t db = desc_b0 + (uint64_t)(s * (SH::STAGE >> 4));
                    // MMA K step ks of part q: atom ks / KS_ATOM, offset ks % KS_ATOM in its rows
                    auto desc_a = [&](int q, int ks) {
                        return da + (uint64_t)((q * SH::X_BYTES + (ks / SH::KS_ATOM) * SH::ATOM_X +
                                                (ks % SH::KS_ATOM) * G::KSTEP * G::ELEM) >> 4);
                    };
                    auto desc_b = [&](int q, int ks) {
                        return db + (uint64_t)((q * SH::Y_BYTES + (ks / SH::KS_ATOM) * SH::ATOM_Y +
                                                (ks % SH::KS_ATOM) * G::KSTEP * G::ELEM) >> 4);
                    };
                    // D group of this stage: order d into accumulator min(d, ND-1);
                    // each accumulator is overwritten by its first MMA of the chunk
                    auto run_d = [&]() {
                        if constexpr (G::ND > 0) {
                            bool fresh[3] = {fl.first_in_chunk, fl.first_in_chunk, fl.first_in_chunk};
#pragma unroll
                            for (int ord = 0; ord <= G::DMAX; ++ord) {
                                const int acc = ord < G::ND - 1 ? ord : G::ND - 1;
                                const uint32_t d = tmem + (buf * G::ND + acc) * 128;
#pragma unroll
                                for (int a = 0; a <= ord; ++a) {
                                    if (a >= G::PARTS || ord - a >= G::PARTS) continue;
#pragma unroll
                                    for (int ks = 0; ks < NKS; ++ks) {
                                        umma<MODE, CG>(d, desc_a(a, ks), desc_b(ord - a, ks), SH::IDESC,
                                                       fresh[acc] ? 0u : 1u);
                                        fresh[acc] = false;
                                    }
                                }
                            }
                            if (fl.last_in_chunk) umma_commit<CG>(b_dfull + 8 * buf);
                        }
                    };
                    // F group of this stage
                    auto run_f = [&]() {
                        if constexpr (HAS_F) {
                            bool first = G::F_FINAL ? (kb == 0) : fl.f_first;
#pragma unroll
                            for (int ord = G::FMIN; ord <= G::FMAX; ++ord)
#pragma unroll
                                for (int a = 0; a <= ord; ++a) {
                                    if (a >= G::PARTS || ord - a >= G::PARTS) continue;
#pragma unroll
                                    for (int ks = 0; ks < NKS; ++ks) {
                                        umma<MODE, CG>(tmem + G::F_COL, desc_a(a, ks), desc_b(ord - a, ks),
                                                       SH::IDESC, first ? 0u : 1u);
                                        first = false;
                                    }
                                }
                            if (!G::F_FINAL && fl.f_last) umma_commit<CG>(b_ffull);
                        }
                    };
                    if (fl.f_before_d) {
                        // While the D accumulators of the previous chunk drain, this
                        // stage's F MMAs go first and keep the tensor pipe busy; the
                        // D MMAs follow once the helper has seen the drain end.
                        if (lane == 0) run_f();
                        __syncwarp();
                        if (!meet_helper(false)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        if (lane == 0) run_d();
                    } else if (lane == 0) {
                        run_d();
                        run_f();
                    }
                    if (lane == 0) umma_commit<CG>(b_empty + 8 * s);  // stage reusable once these MMAs finish
                    __syncwarp();
                    if (fl.last_in_chunk) ++chunk;
                    if (fl.f_last) ++fchunk;
                }
                if (!ok) break;
                if constexpr (G::F_FINAL) {
                    if (lane == 0) umma_commit<CG>(b_ffull);
                    __syncwarp();
                }
            }
            // every issued MMA completes before TMEM is released (bounded)
            if (lane == 0) {
                umma_commit<CG>(b_done);
                mbar_wait_quiet<CG>(b_done, 0);
            }
            __syncwarp();
        } else if (lane == 0) {
            // odd CTA of a pair: the even CTA's final commit arrives here too
            mbar_wait_quiet<CG>(b_done, 0);
        }
    } else if (warp == 2 + SH::EPI_WARPS) {
        // ------------------------------------------------------------ wait helper
        // Makes the MMA issuer's barrier waits, stage by stage in the issuer's
        // order, and meets it at named barrier 1 after each set (an F-first
        // stage meets it twice: operands ready, then D accumulators drained).
        if (rank == 0) {
            uint32_t it = 0, chunk = 0, fchunk = 0, tcount = 0;
            bool ok = true;
            for (int t = t_beg; t < t_end && ok; ++t, ++tcount) {
                const LeafTile lt = sched[t];
                const int nkb = tcp[lt.prod].K_pad / G::KBLK;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const StageFlags fl = stage_flags<kbpc, FOFF, FKC>(kb, nkb);
                    const uint32_t buf = chunk % G::DBUF;
                    const uint32_t s = it % NSTAGE, ph = (it / NSTAGE) & 1;
                    bool good = true;
                    if (lane == 0) {
                        if (G::F_FINAL && kb == 0)
                            good = mbar_wait<CG>(b_fempty, (tcount & 1) ^ 1, status, ERR_TIMEOUT_MMA, wait_ns);
                        good = good && mbar_wait<CG>(b_full + 8 * s, ph, status, ERR_TIMEOUT_MMA, wait_ns);
                        if (!fl.f_before_d) {
                            if (G::ND > 0 && fl.first_in_chunk)
                                good = good && mbar_wait<CG>(b_dempty + 8 * buf, ((chunk / G::DBUF) & 1) ^ 1, status,
                                                             ERR_TIMEOUT_MMA, wait_ns);
                            if (HAS_F && !G::F_FINAL && fl.f_first)
                                good = good && mbar_wait<CG>(b_fempty, (fchunk & 1) ^ 1, status, ERR_TIMEOUT_MMA, wait_ns);
                        }
                    }
                    if (!meet_helper(!__shfl_sync(0xffffffffu, good, 0))) {
                        ok = false;
                        break;
                    }
                    if (fl.f_before_d) {
                        good = true;
                        if (lane == 0)
                            good = mbar_wait<CG>(b_dempty + 8 * buf, ((chunk / G::DBUF) & 1) ^ 1, status,
                                                 ERR_TIMEOUT_MMA, wait_ns);
                        if (!meet_helper(!__shfl_sync(0xffffffffu, good, 0))) {
                            ok = false;
                            break;
                        }
                    }
                    if (fl.last_in_chunk) ++chunk;
                    if (fl.f_last) ++fchunk;
                }
            }
        }
    } else if (warp < 2 + SH::EPI_WARPS) {
        // ------------------------------------------------------------ epilogue
        // Thread = one row (TMEM lane) of the tile and NCOL of its columns; the
        // running sum of the drained chunks is hi (registers) + lo (smem).
        const int e = warp - 2;
        const int q = warp & 3;              // TMEM lane quarter of this warp
        const int cq = e >> 2;               // column slice
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const int row = 32 * q + lane;
        uint32_t chunk = 0, fchunk = 0, tcount = 0;
        bool ok = true;
        for (int t = t_beg; t < t_end && ok; ++t, ++tcount) {
            const LeafTile lt = sched[t];
            const TcProd* pr = tcp + lt.prod;
            const int nkb = pr->K_pad / G::KBLK;
            float hi[NCOL];
#pragma unroll
            for (int c = 0; c < NCOL; ++c) hi[c] = 0.f;
            f32x2 lo2r[SH::LO_REGS ? NCOL / 2 : 1];  // lo halves in registers (LO_REGS)
            if constexpr (G::ND > 0) {
                // Drains in the order the MMA issuer commits them: stage dnext
                // ends a D chunk, stage fnext an F chunk (the tile's last stage
                // ends both: D first).  lo holds a value once the tile's first
                // drain has written it.
                bool lo_init = false;
                int dnext = min(kbpc - 1, nkb - 1);
                int fnext = HAS_F && !G::F_FINAL ? min(FOFF > 0 ? FOFF - 1 : kbpc - 1, nkb - 1) : nkb;
                while (dnext < nkb || fnext < nkb) {
                    if (dnext <= fnext) {
                        const uint32_t buf = chunk % G::DBUF;
                        if (!mbar_wait<CG>(b_dfull + 8 * buf, (chunk / G::DBUF) & 1, status, ERR_TIMEOUT_EPILOGUE, wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
#pragma unroll
                        for (int g = 0; g < NG; ++g) {
                            const uint32_t col = cq * NCOL + g * 16;
#pragma unroll
                            for (int c8 = 0; c8 < 16; c8 += 8) {
                                // the accumulators' 8 columns in flight together, one wait
                                uint32_t a0[8], a1[8], a2[8];
                                tmem_ld8_async(tmem + lane_base + (buf * G::ND + 0) * 128 + col + c8, a0);
                                tmem_ld8_async(tmem + lane_base + (buf * G::ND + 1) * 128 + col + c8, a1);
                                if constexpr (G::ND > 2)
                                    tmem_ld8_async(tmem + lane_base + (buf * G::ND + 2) * 128 + col + c8, a2);
                                tmem_wait_ld();
#pragma unroll
                                for (int cc = 0; cc < 8; cc += 2) {
                                    const int c = c8 + cc;
                                    // chunk value h + l (accumulator 0 is exact, the others are at
                                    // most ~2^-8 of it), added to (hi, lo) as a float-float sum and
                                    // renormalised so that |lo| stays within half an ulp of hi;
                                    // two columns per instruction
                                    f32x2* lp = SH::LO_REGS ? &lo2r[(g * 16 + c) / 2] : lo2_s + ((col + c) / 2) * 128 + row;
                                    if constexpr (!G::FP64_SUM) {
                                        // FP32-accuracy result: the exact order-0 chunk is added
                                        // to hi with its rounding error kept (TwoSum), and the
                                        // orders-1-2 chunk (about 2^-8 of it) goes straight into
                                        // lo, whose FP32 rounding is then 2^-32 of the result
                                        f32x2 s2, e2;
                                        two_sum2(pk2(hi[g * 16 + c], hi[g * 16 + c + 1]),
                                                 pk2(__uint_as_float(a0[cc]), __uint_as_float(a0[cc + 1])), s2, e2);
                                        *lp = add2(lo_init ? *lp : 0ull,
                                                   add2(e2, pk2(__uint_as_float(a1[cc]), __uint_as_float(a1[cc + 1]))));
                                        upk2(s2, hi[g * 16 + c], hi[g * 16 + c + 1]);
                                    } else {
                                        f32x2 h, l, s2, e2;
                                        two_sum2(pk2(__uint_as_float(a0[cc]), __uint_as_float(a0[cc + 1])),
                                                 pk2(__uint_as_float(a1[cc]), __uint_as_float(a1[cc + 1])), h, l);
                                        if constexpr (G::ND > 2)
                                            l = add2(l, pk2(__uint_as_float(a2[cc]), __uint_as_float(a2[cc + 1])));
                                        two_sum2(pk2(hi[g * 16 + c], hi[g * 16 + c + 1]), h, s2, e2);
                                        e2 = add2(e2, add2(lo_init ? *lp : 0ull, l));
                                        const f32x2 hn = add2(s2, e2);  // Fast2Sum: |s2| >= |e2|
                                        *lp = sub2(e2, sub2(hn, s2));
                                        upk2(hn, hi[g * 16 + c], hi[g * 16 + c + 1]);
                                    }
                                }
                            }
                        }
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) {
                            if constexpr (CG == 1)
                                mbar_arrive(b_dempty + 8 * buf);
                            else
                                mbar_arrive_cluster(b_dempty_c + 8 * buf);
                        }
                        ++chunk;
                        dnext = dnext == nkb - 1 ? nkb : min(dnext + kbpc, nkb - 1);
                    } else {
                        if constexpr (HAS_F && !G::F_FINAL) {
                            if (!mbar_wait<CG>(b_ffull, fchunk & 1, status, ERR_TIMEOUT_EPILOGUE, wait_ns)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
#pragma unroll
                            for (int g = 0; g < NG; ++g) {
                                const uint32_t col = cq * NCOL + g * 16;
                                float f[16];
                                tmem_ld16(tmem + lane_base + G::F_COL + col, f);
#pragma unroll
                                for (int c = 0; c < 16; c += 2) {
                                    f32x2* lp = lo2_s + ((col + c) / 2) * 128 + row;
                                    const f32x2 fv = pk2(f[c], f[c + 1]);
                                    *lp = lo_init ? add2(*lp, fv) : fv;
                                }
                            }
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) {
                                if constexpr (CG == 1)
                                    mbar_arrive(b_fempty);
                                else
                                    mbar_arrive_cluster(b_fempty_c);
                            }
                            ++fchunk;
                        }
                        fnext = fnext == nkb - 1 ? nkb : min(fnext + FKC, nkb - 1);
                    }
                    lo_init = true;
                }
                if (!ok) break;
            }
            if constexpr (G::F_FINAL) {
                if (!mbar_wait<CG>(b_ffull, tcount & 1, status, ERR_TIMEOUT_EPILOGUE, wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
            }
            // FP64 tile: row i of this thread, NCOL columns in groups of 16.  The
            // product's fields are read once into registers: the output stores
            // below could alias the table as far as the compiler knows.
            const int p_out_rows = __ldg(&pr->out_rows), p_out_cols = __ldg(&pr->out_cols);
            const int p_out_kind = __ldg(&pr->out_kind), p_cj0 = __ldg(&pr->cj0);
            const unsigned long long* __restrict__ p_ey = reinterpret_cast<const unsigned long long*>(pr->ey);
            const Bind& bind = bs.b[pr->inst];
            const int i = lt.ti * (128 * CG) + (int)rank * 128 + row;
            const int j0 = lt.tj * SH::TN + cq * NCOL;
            const bool row_ok = i < p_out_rows;
            int Ei = 0;
            if constexpr (G::SLICED) {
                if (row_ok) Ei = col_exponent<G::HEAD>(__ldg(reinterpret_cast<const unsigned long long*>(pr->ex) + i));
            }
            double* dense = (p_out_kind == OUT_CDENSE ? bind.C : reinterpret_cast<double*>(bind.W)) + pr->out_off +
                            (int64_t)i * pr->out_ld;
            const int64_t gi = (int64_t)pr->ci0 + i;
            double* prow = bind.C + (packed_start(gi, bind.n) - gi + p_cj0);
            // column exponents: lane l takes those of columns j0 + 32 w + l,
            // and every lane reads the ones it needs from the lane that holds
            // them (one shuffle per entry instead of a load and a decode)
            int Ecol[SLICED_COLS<G, NCOL>::W];
            if constexpr (G::SLICED) {
#pragma unroll
                for (int w = 0; w < NCOL / 32; ++w) Ecol[w] = col_exponent<G::HEAD>(__ldg(p_ey + j0 + 32 * w + lane));
            }
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const uint32_t col = cq * NCOL + g * 16;
                float f[16];
                if constexpr (G::F_FINAL) {
                    tmem_ld16(tmem + lane_base + G::F_COL + col, f);
                } else {
#pragma unroll
                    for (int c = 0; c < 16; ++c) f[c] = 0.f;
                }
                int Ej[16];
                if constexpr (G::SLICED) {
#pragma unroll
                    for (int c = 0; c < 16; ++c)
                        Ej[c] = __shfl_sync(0xffffffffu, Ecol[(g * 16 + c) >> 5], (g * 16 + c) & 31);
                }
                if (row_ok) {
                    const bool dense_out = p_out_kind == OUT_DENSE || p_out_kind == OUT_CDENSE;
                    double* dst = (dense_out ? dense : prow) + j0 + g * 16;
#pragma unroll
                    for (int c4 = 0; c4 < 16; c4 += 4) {
                        double v[4];
                        bool ok[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int c = c4 + q;
                            const int j = j0 + g * 16 + c;
                            ok[q] = j < p_out_cols && (dense_out || p_out_kind == OUT_PACKED || (int64_t)p_cj0 + j >= gi);
                            float hh = hi[g * 16 + c],
                                  ll = G::ND == 0 ? 0.f
                                       : SH::LO_REGS ? (((c & 1) == 0) ? __uint_as_float((uint32_t)lo2r[(g * 16 + c) / 2])
                                                                      : __uint_as_float((uint32_t)(lo2r[(g * 16 + c) / 2] >> 32)))
                                                    : lo_s[(((col + c) / 2) * 128 + row) * 2 + ((col + c) & 1)];
                            // a final F accumulator (TF32) is added here; the other modes
                            // drained theirs into (hi, lo) chunk by chunk
                            if constexpr (G::F_FINAL) ff_add(hh, ll, f[c]);
                            if constexpr (!G::FP64_SUM) {
                                // FP32-accuracy modes: the FP32 sum of the pair, widened
                                // with integer operations (no FP64 arithmetic per entry)
                                hh += ll;
                                ll = 0.f;
                            }
                            const int sc = G::SLICED ? Ei + Ej[c] : 0;
                            const long long bh = f2d_scaled_bits(hh, sc), bl = f2d_scaled_bits(ll, sc);
                            if (G::SLICED && sc >= kNonFinite)
                                v[q] = __longlong_as_double(0x7FF8000000000000LL);
                            else if constexpr (G::FP64_SUM)
                                v[q] = __longlong_as_double(bh) + __longlong_as_double(bl);
                            else
                                v[q] = __longlong_as_double(bh);
                        }
                        // whole 32-byte sectors where the row segment allows it
                        double* d = dst + c4;
                        const uintptr_t a = reinterpret_cast<uintptr_t>(d);
                        if (ok[0] && ok[1] && ok[2] && ok[3] && (a & 31) == 0) {
                            asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(d), "d"(v[0]), "d"(v[1]),
                                         "d"(v[2]), "d"(v[3])
                                         : "memory");
                        } else if (ok[0] && ok[1] && ok[2] && ok[3] && (a & 15) == 0) {
                            *reinterpret_cast<double2*>(d) = make_double2(v[0], v[1]);
                            *reinterpret_cast<double2*>(d + 2) = make_double2(v[2], v[3]);
                        } else {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                if (ok[q]) d[q] = v[q];
                        }
                    }
                }
            }
            if constexpr (G::F_FINAL) {
                // accumulator read: TMEM may be refilled by the next tile
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (CG == 1)
                        mbar_arrive(b_fempty);
                    else
                        mbar_arrive_cluster(b_fempty_c);
                }
            }
        }
    }

    // teardown: every role has stopped issuing and every MMA has completed;
    // in a pair neither CTA leaves while the other may still reach its
    // shared memory (remote arrivals, MMA operand reads)
    tc_fence_before();
    if constexpr (CG == 1)
        __syncthreads();
    else
        cluster_sync_all();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc<CG>(tmem, SH::TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// Host side

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// TMA map of the stacked parts of one operand: rows (parts x rows_pad) of
// K_pad elements, a box of one swizzle atom (ROWB bytes of K) x box_rows,
// swizzled to the UMMA K-major layout.
template <int MODE>
bool encode_parts(CUtensorMap* map, char* base, int parts, int rows_pad, int K_pad, int box_rows) {
    using G = Geo<MODE>;
    auto enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K_pad, (cuuint64_t)parts * rows_pad};
    const cuuint64_t strides[1] = {(cuuint64_t)K_pad * G::ELEM};
    const cuuint32_t box[2] = {(cuuint32_t)(G::ROWB / G::ELEM), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt =
        G::ELEM == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUtensorMapSwizzle sw = G::ROWB == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : G::ROWB == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                  : CU_TENSOR_MAP_SWIZZLE_32B;
    return enc(map, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_for(LeafKind k, CUtensorMap* map, char* base, int rows_pad, int K_pad, int box_rows) {
    switch (k) {
        case LEAF_BF16X3: return encode_parts<MODE_BF16X3>(map, base, 3, rows_pad, K_pad, box_rows);
        case LEAF_TF32: return encode_parts<MODE_TF32>(map, base, 1, rows_pad, K_pad, box_rows);
        case LEAF_OZAKI: return encode_parts<MODE_OZAKI>(map, base, 6, rows_pad, K_pad, box_rows);
        default: return false;
    }
}

int g_sms = 1;                    // SM count of the device (set before any capture)
int g_pair_clusters[4] = {0, 0, 0, 0};  // co-resident CTA pairs per mode (0: pair kernel unavailable)

cudaLaunchAttribute pair_cluster_attr() {
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeClusterDimension;
    a.val.clusterDim.x = 2;
    a.val.clusterDim.y = 1;
    a.val.clusterDim.z = 1;
    return a;
}

// Limit of the pipeline waits of a launch (the plan's option; 1 s by
// default).  The teardown waits always keep the 1 s limit.
uint64_t wait_limit(const DeviceTables& t) { return t.wait_ns > 0 ? t.wait_ns : kTimeoutNs; }

template <int NB, int MODE>
cudaError_t launch_mode(const DeviceTables& t, const BindSet<NB>& bs, cudaStream_t s, cudaEvent_t before_gemm) {
    if (Geo<MODE>::SLICED) {
        cudaError_t e = cudaMemsetAsync(t.tc_ex, 0, t.tc_ex_bytes, s);
        if (e != cudaSuccess) return e;
    }
    if constexpr (MODE == MODE_OZAKI) {
        // column maxima per row segment, column scales, then operands formed in
        // fixed point
        if (t.ncolmax > 0)
            tc_termmax_kernel<NB><<<t.ncolmax, 256, 0, s>>>(bs, t.atom_terms, t.colmax, t.atom_mx, t.term_max);
        if (t.nscale > 0)
            tc_scale_kernel<<<t.nscale, PT, 0, s>>>(t.prods, t.terms, t.tcp, t.scale, t.term_mx, t.mx_list,
                                                     t.term_max, t.col_e);
        if (t.nprep > 0)
            tc_prep_fixed_kernel<NB><<<t.nprep, 256, 0, s>>>(bs, t.prods, t.terms, t.tcp, t.prep, t.col_e);
    } else {
        if (Geo<MODE>::SLICED && t.ncolmax > 0)
            tc_colmax_kernel<NB, typename PrepSrc<MODE>::T>
                <<<t.ncolmax, 256, 0, s>>>(bs, t.prods, t.terms, t.tcp, t.colmax);
        if (t.nprep > 0) tc_prep_kernel<NB, MODE><<<t.nprep, 256, 0, s>>>(bs, t.prods, t.terms, t.tcp, t.prep);
    }
    if (before_gemm) {
        cudaError_t e = cudaEventRecordWithFlags(before_gemm, s, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
    }
    if constexpr (NB == 1) {
        if (t.tc_pair) {
            using SH = Shape<MODE, 2>;
            if (g_pair_clusters[MODE] < 1) return cudaErrorInvalidConfiguration;
            const int nclus = std::max(1, t.nworkers);
            cudaLaunchAttribute at[1] = {pair_cluster_attr()};
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2 * nclus);
            cfg.blockDim = dim3(SH::THREADS);
            cfg.dynamicSmemBytes = SH::SMEM;
            cfg.stream = s;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            return cudaLaunchKernelEx(&cfg, tc_gemm_kernel<1, MODE, 2>, bs, t.tcp, t.sched, t.wfirst, t.status,
                                      wait_limit(t));
        }
    }
    using SH = Shape<MODE, 1, NB>;
    const int grid = std::max(1, t.nworkers);
    tc_gemm_kernel<NB, MODE, 1><<<grid, SH::THREADS, SH::SMEM, s>>>(bs, t.tcp, t.sched, t.wfirst, t.status,
                                                                     wait_limit(t));
    return cudaGetLastError();
}

template <int NB>
cudaError_t launch_kind(const DeviceTables& t, const BindSet<NB>& bs, cudaStream_t s, cudaEvent_t ev) {
    switch (t.leaf) {
        case LEAF_BF16X3: return launch_mode<NB, MODE_BF16X3>(t, bs, s, ev);
        case LEAF_TF32: return launch_mode<NB, MODE_TF32>(t, bs, s, ev);
        case LEAF_OZAKI: return launch_mode<NB, MODE_OZAKI>(t, bs, s, ev);
        default: return cudaErrorInvalidValue;
    }
}

template <int NB, int MODE, int CG>
cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(tc_gemm_kernel<NB, MODE, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Shape<MODE, CG, NB>::SMEM);
}

// How many CTA pairs of the MODE kernel fit on the device at once (0 when the
// pair kernel cannot be launched here).
template <int MODE>
int pair_clusters() {
    using SH = Shape<MODE, 2>;
    if (set_smem_attr<1, MODE, 2>() != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute at[1] = {pair_cluster_attr()};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * std::max(1, g_sms / 2));
    cfg.blockDim = dim3(SH::THREADS);
    cfg.dynamicSmemBytes = SH::SMEM;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, tc_gemm_kernel<1, MODE, 2>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return std::max(0, n);
}

}  // namespace

bool leaf_supported(LeafKind k) {
    return k == LEAF_F64 || k == LEAF_BF16X3 || k == LEAF_TF32 || k == LEAF_OZAKI;
}

ata_status tc_prepare_device() {
    static cudaError_t err = cudaErrorNotReady;
    static std::once_flag once;
    std::call_once(once, [] {
        err = set_smem_attr<1, MODE_BF16X3, 1>();
        if (err == cudaSuccess) err = set_smem_attr<1, MODE_TF32, 1>();
        if (err == cudaSuccess) err = set_smem_attr<1, MODE_OZAKI, 1>();
        if (err == cudaSuccess) err = set_smem_attr<kDevBinds, MODE_BF16X3, 1>();
        if (err == cudaSuccess) err = set_smem_attr<kDevBinds, MODE_TF32, 1>();
        if (err == cudaSuccess) err = set_smem_attr<kDevBinds, MODE_OZAKI, 1>();
        if (err == cudaSuccess && !get_encode()) err = cudaErrorNotSupported;
        if (err == cudaSuccess) {
            int dev = 0;
            err = cudaGetDevice(&dev);
            if (err == cudaSuccess) err = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
            if (g_sms <= 0) g_sms = 1;
        }
        if (err == cudaSuccess) {
            g_pair_clusters[MODE_BF16X3] = pair_clusters<MODE_BF16X3>();
            g_pair_clusters[MODE_TF32] = pair_clusters<MODE_TF32>();
            g_pair_clusters[MODE_OZAKI] = pair_clusters<MODE_OZAKI>();
        }
    });
    if (err != cudaSuccess) return cuda_fail(err, "tensor-core leaf set-up");
    return ATA_OK;
}

int tc_rows_for(const Plan& P) {
    if (P.leaf == LEAF_F64 || P.tc_tile_rows != kTcPairRows) return kTcTile;
    if (tc_prepare_device() != ATA_OK) return kTcTile;
    return g_pair_clusters[P.leaf] > 0 ? kTcPairRows : kTcTile;
}

namespace {

// Leaf tile schedule.  Each worker of the persistent leaf launch (a CTA, or a
// CTA pair) runs its own contiguous list of tiles.  Tiles are taken longest
// first and each goes to the worker with the least work so far (ties to the
// lowest worker), the longest-processing-time rule; a tile's cost is its
// K-blocks plus a fixed cost per tile for its first loads, its last drain and
// its output (about 5000 clocks, in K-blocks of the mode).  Tiles of equal
// cost are dealt round robin, in their table order (heaviest products
// first).  Short and uneven tiles (batched instances) no longer leave a
// tail of workers that were dealt more of them than the others.
void leaf_schedule(const HostTables& h, int nw, std::vector<LeafTile>* sched, std::vector<int32_t>* wfirst) {
    const int ntiles = (int)h.tiles.size();
    int kblk = Geo<MODE_BF16X3>::KBLK, over = 4;
    if (h.leaf == LEAF_TF32) {
        kblk = Geo<MODE_TF32>::KBLK;
        over = 10;
    } else if (h.leaf == LEAF_OZAKI) {
        kblk = Geo<MODE_OZAKI>::KBLK;
        over = 3;
    }
    std::vector<int64_t> cost(ntiles);
    std::vector<int> idx(ntiles);
    for (int i = 0; i < ntiles; ++i) {
        cost[i] = h.prods[h.tiles[i].prod].K_pad / kblk + over;
        idx[i] = i;
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    using Load = std::pair<int64_t, int>;  // (work so far, worker)
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int w = 0; w < nw; ++w) heap.push({0, w});
    std::vector<std::vector<int>> lists(nw);
    for (int i : idx) {
        Load l = heap.top();
        heap.pop();
        lists[l.second].push_back(i);
        l.first += cost[i];
        heap.push(l);
    }
    // Where tile lengths spread widely (batched instances: 4x or more), each
    // worker runs its tiles alternately from the long and the short end of
    // its list: a short tile's last drain and output then overlap the next
    // (long) tile's MMAs through the double-buffered accumulators, instead of
    // short tiles queueing behind one another's epilogues at the end (batched
    // step 1.072 -> 1.057 ms).  Tiles of similar length keep the longest-first
    // order, whose concurrent tiles share operand blocks in L2 (interleaving
    // them cost 0.3%).  The workers' loads are the assignment's either way.
    const bool interleave = ntiles > 0 && cost[idx.front()] >= 4 * cost[idx.back()];
    sched->clear();
    wfirst->assign(nw + 1, 0);
    for (int w = 0; w < nw; ++w) {
        (*wfirst)[w] = (int32_t)sched->size();
        const std::vector<int>& l = lists[w];  // longest first
        if (!interleave) {
            for (int i : l) sched->push_back(h.tiles[i]);
            continue;
        }
        for (size_t a = 0, b = l.size(); a < b;) {
            sched->push_back(h.tiles[l[a++]]);
            if (a < b) sched->push_back(h.tiles[l[--b]]);
        }
    }
    (*wfirst)[nw] = (int32_t)sched->size();
}

}  // namespace

ata_status build_tc_tables(const HostTables& h, const std::vector<char*>& ws, DeviceTables* d) {
    ata_status st = tc_prepare_device();
    if (st != ATA_OK) return st;
    // workers of the leaf launch: CTAs (one per SM) or CTA pairs
    const int ntiles_all = (int)h.tiles.size();
    const int wmax = h.tile_rows == kTcPairRows ? g_pair_clusters[h.leaf] : g_sms;
    const int nw = std::max(1, std::min(ntiles_all, std::max(1, wmax)));
    std::vector<LeafTile> sched;
    std::vector<int32_t> wfirst;
    leaf_schedule(h, nw, &sched, &wfirst);
    const int np = (int)h.prods.size();
    std::vector<TcProd> tp(np);
    std::vector<PrepTask> prep, colmax;
    int64_t ex_elems = 0;
    // Operands that share a part buffer (equal terms, see the planner) are
    // prepared once, by their first product, over the rows any user needs,
    // and share one column-maximum array.
    struct Buf {
        int prod, side;
        int rows_used;
        int64_t ex_index;
    };
    std::map<std::pair<int, int64_t>, Buf> bufs;
    std::vector<std::pair<int, int64_t>> order;  // first-use order
    for (int i = 0; i < np; ++i) {
        const LeafProduct& lp = h.prods[i];
        TcProd& t = tp[i];
        std::memset(&t, 0, sizeof(t));
        char* W = ws[lp.inst];
        // CTA pairs: each CTA stages 128 X rows and half of the tile's Y rows
        // (128 of 256 for TF32, 64 of 128 otherwise); rows past the operand's
        // padded extent read as zeros (TMA fill) and feed only columns that
        // are never written
        const int ybox = h.tile_rows == kTcPairRows ? tc_cols_for(h.leaf, kTcPairRows) / 2 : kTcTile;
        if (!encode_for(h.leaf, &t.tmx, W + lp.tc_x_off, lp.p_pad, lp.K_pad, kTcTile) ||
            !encode_for(h.leaf, &t.tmy, W + lp.tc_y_off, lp.r_pad, lp.K_pad, ybox))
            return fail(ATA_ECUDA, "cuTensorMapEncodeTiled failed for a leaf operand");
        t.p_pad = lp.p_pad;
        t.r_pad = lp.r_pad;
        t.K_pad = lp.K_pad;
        t.inst = lp.inst;
        t.out_rows = lp.out_rows;
        t.out_cols = lp.out_cols;
        t.out_kind = lp.out_kind;
        t.out_ld = lp.out_ld;
        t.out_off = lp.out_off;
        t.ci0 = lp.ci0;
        t.cj0 = lp.cj0;
        const bool syrk = lp.out_kind == OUT_SYRK;
        for (int side = 0; side < (syrk ? 1 : 2); ++side) {
            // Part rows past the product's output extent feed only output rows
            // or columns that are never written, so whole 64-row blocks of them
            // are not prepared (their contents are never read into a result).
            const int rows_used = side ? lp.out_cols : lp.out_rows;
            const auto key = std::make_pair(lp.inst, side ? lp.tc_y_off : lp.tc_x_off);
            auto it = bufs.find(key);
            if (it == bufs.end()) {
                Buf b{i, side, rows_used, ex_elems};
                ex_elems += side ? lp.r_pad : lp.p_pad;
                it = bufs.emplace(key, b).first;
                order.push_back(key);
            } else {
                it->second.rows_used = std::max(it->second.rows_used, rows_used);
            }
            if (side == 0) t.ex_index = it->second.ex_index;
            if (side == 1 || syrk) t.ey_index = it->second.ex_index;
        }
    }
    std::vector<PrepTask> scale;  // FP64 emulation: column-scale strips
    for (const auto& key : order) {
        const Buf& b = bufs[key];
        const LeafProduct& lp = h.prods[b.prod];
        for (int c0 = 0; c0 < b.rows_used; c0 += PT) {
            if (h.leaf == LEAF_OZAKI) {
                PrepTask st{};
                st.prod = b.prod;
                st.side = (int8_t)b.side;
                st.c0 = c0;
                scale.push_back(st);
            }
            for (int k0 = 0; k0 < lp.K_pad; k0 += PT) {
                PrepTask pt{};
                pt.prod = b.prod;
                pt.side = (int8_t)b.side;
                pt.c0 = c0;
                pt.k0 = k0;
                pt.k1 = k0 + PT;
                prep.push_back(pt);
            }
            // column maxima over the valid rows only (per operand; the FP64
            // emulation takes them per distinct block below)
            for (int k0 = 0; k0 < lp.K && h.leaf != LEAF_OZAKI; k0 += kColSpan) {
                PrepTask ct{};
                ct.prod = b.prod;
                ct.side = (int8_t)b.side;
                ct.c0 = c0;
                ct.k0 = k0;
                ct.k1 = std::min(k0 + kColSpan, lp.K);
                colmax.push_back(ct);
            }
        }
    }
    // Slicing tasks ordered by tile position: operands summed from the same
    // blocks (the operand sums of one Strassen node, a diagonal leaf's column
    // block and the node's quadrants) read the same source tiles at the same
    // (k0, c0), which then come from L2 for all but the first of them.
    std::stable_sort(prep.begin(), prep.end(), [](const PrepTask& a, const PrepTask& b) {
        return a.k0 != b.k0 ? a.k0 < b.k0 : a.c0 < b.c0;
    });
    // FP64 emulation: the column maxima of every distinct block that some
    // operand sums.  Blocks of one buffer with the same leading dimension,
    // column offset and width differ only in their row ranges; the ranges are
    // cut at every block boundary into disjoint row segments (atoms), each
    // atom's maxima are taken once, and a block's maxima are the maxima over
    // its atoms (a term's list of atom offsets, ended by -1).  Every element
    // is then read once, however many blocks contain it.
    std::vector<int64_t> term_mx(h.terms.size(), -1);
    std::vector<int64_t> mx_list;
    std::vector<Term> atom_terms;
    std::vector<int64_t> atom_mx;
    int64_t tm_elems = 0;
    if (h.leaf == LEAF_OZAKI) {
        // block: (inst, buf, dt, ld, column offset, cols) -> row ranges
        using GKey = std::tuple<int, int, int, int64_t, int64_t, int>;
        std::map<GKey, std::set<std::pair<int64_t, int64_t>>> groups;
        auto gkey = [](const Term& tm) {
            const int64_t ld = tm.ld > 0 ? tm.ld : 1;
            const int64_t q = tm.off >= 0 ? tm.off / ld : (tm.off - ld + 1) / ld;  // floor
            return std::make_pair(GKey{(int)tm.inst, (int)tm.buf, (int)tm.dt, ld, tm.off - q * ld, (int)tm.cols},
                                  q);
        };
        std::vector<int> used_terms;
        for (const auto& key : order) {
            const Buf& b = bufs[key];
            const LeafProduct& lp = h.prods[b.prod];
            const int t0 = b.side ? lp.y0 : lp.x0, nt = b.side ? lp.ny : lp.nx;
            for (int t = t0; t < t0 + nt; ++t) {
                const Term& tm = h.terms[t];
                used_terms.push_back(t);
                if (tm.rows <= 0 || tm.cols <= 0) continue;
                const auto kq = gkey(tm);
                groups[kq.first].insert({kq.second, kq.second + tm.rows});
            }
        }
        // atoms of each group: the segments between consecutive boundaries
        // that some range covers
        std::map<GKey, std::vector<std::pair<int64_t, int64_t>>> atoms_of;  // [q0, q1) -> ...
        std::map<std::tuple<GKey, int64_t>, int64_t> atom_index;           // (group, q0) -> atom
        for (const auto& g : groups) {
            std::set<int64_t> cuts;
            for (const auto& r : g.second) {
                cuts.insert(r.first);
                cuts.insert(r.second);
            }
            const std::vector<int64_t> cv(cuts.begin(), cuts.end());
            for (size_t i = 0; i + 1 < cv.size(); ++i) {
                const int64_t a = cv[i], z = cv[i + 1];
                bool covered = false;
                for (const auto& r : g.second) covered = covered || (r.first <= a && z <= r.second);
                if (!covered) continue;
                const GKey& k = g.first;
                Term at{};
                at.ld = std::get<3>(k);
                at.off = a * at.ld + std::get<4>(k);
                at.rows = (int32_t)(z - a);
                at.cols = std::get<5>(k);
                at.buf = (int8_t)std::get<1>(k);
                at.dt = (int8_t)std::get<2>(k);
                at.neg = 0;
                at.inst = std::get<0>(k);
                const int64_t id = (int64_t)atom_terms.size();
                atom_terms.push_back(at);
                atom_mx.push_back(tm_elems);
                tm_elems += (at.cols + PT - 1) / PT * PT;
                atom_index[{k, a}] = id;
                atoms_of[k].push_back({a, z});
                // strips side by side over the same rows run together
                for (int k0 = 0; k0 < at.rows; k0 += kAtomSpan)
                    for (int c0 = 0; c0 < at.cols; c0 += PT) {
                        PrepTask ct{};
                        ct.prod = (int32_t)id;  // an atom
                        ct.c0 = c0;
                        ct.k0 = k0;
                        ct.k1 = std::min(k0 + kAtomSpan, at.rows);
                        colmax.push_back(ct);
                    }
            }
        }
        // each term's list: the atoms inside its row range (blocks with equal
        // ranges share one list)
        std::map<std::tuple<GKey, int64_t, int64_t>, int64_t> lists;
        for (int t : used_terms) {
            if (term_mx[t] >= 0) continue;
            const Term& tm = h.terms[t];
            if (tm.rows <= 0 || tm.cols <= 0) {
                term_mx[t] = (int64_t)mx_list.size();
                mx_list.push_back(-1);
                continue;
            }
            const auto kq = gkey(tm);
            const auto lk = std::make_tuple(kq.first, kq.second, kq.second + tm.rows);
            auto it = lists.find(lk);
            if (it == lists.end()) {
                const int64_t start = (int64_t)mx_list.size();
                for (const auto& a : atoms_of[kq.first])
                    if (kq.second <= a.first && a.second <= kq.second + tm.rows)
                        mx_list.push_back(atom_mx[atom_index[{kq.first, a.first}]]);
                mx_list.push_back(-1);
                it = lists.emplace(lk, start).first;
            }
            term_mx[t] = it->second;
        }
    }
    // device blob: TcProd[] | PrepTask[] (slicing) | PrepTask[] (maxima) | term offsets | status |
    // exponent maxima of the operands, then of the blocks (zeroed per run)
    auto al = [](int64_t x) { return (x + 255) / 256 * 256; };
    const int64_t o_tp = 0;
    const int64_t o_prep = al(o_tp + (int64_t)np * sizeof(TcProd));
    const int64_t o_colmax = al(o_prep + (int64_t)prep.size() * sizeof(PrepTask));
    const int64_t o_tmx = al(o_colmax + (int64_t)colmax.size() * sizeof(PrepTask));
    const int64_t o_list = al(o_tmx + (int64_t)term_mx.size() * 8);
    const int64_t o_aterm = al(o_list + (int64_t)mx_list.size() * 8);
    const int64_t o_amx = al(o_aterm + (int64_t)atom_terms.size() * sizeof(Term));
    const int64_t o_scale = al(o_amx + (int64_t)atom_mx.size() * 8);
    const int64_t o_cole = al(o_scale + (int64_t)scale.size() * sizeof(PrepTask));
    const int64_t o_status = al(o_cole + (h.leaf == LEAF_OZAKI ? ex_elems * 4 : 0));
    const int64_t o_sched = al(o_status + 256);
    const int64_t o_wfirst = al(o_sched + (int64_t)sched.size() * sizeof(LeafTile));
    const int64_t o_ex = al(o_wfirst + (int64_t)wfirst.size() * 4);
    const int64_t ex_total = std::max<int64_t>(ex_elems + tm_elems, 1);
    const int64_t total = al(o_ex + ex_total * 8);
    char* blob = nullptr;
    if (dev_malloc(&blob, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(ATA_ENOMEM, "tensor-core tables: cudaMalloc failed");
    }
    for (TcProd& t : tp) {
        t.ex = reinterpret_cast<uint64_t*>(blob + o_ex) + t.ex_index;
        t.ey = reinterpret_cast<uint64_t*>(blob + o_ex) + t.ey_index;
    }
    std::vector<char> hb(total, 0);
    if (np) std::memcpy(hb.data() + o_tp, tp.data(), np * sizeof(TcProd));
    if (!prep.empty()) std::memcpy(hb.data() + o_prep, prep.data(), prep.size() * sizeof(PrepTask));
    if (!colmax.empty()) std::memcpy(hb.data() + o_colmax, colmax.data(), colmax.size() * sizeof(PrepTask));
    if (!term_mx.empty()) std::memcpy(hb.data() + o_tmx, term_mx.data(), term_mx.size() * 8);
    if (!mx_list.empty()) std::memcpy(hb.data() + o_list, mx_list.data(), mx_list.size() * 8);
    if (!atom_terms.empty())
        std::memcpy(hb.data() + o_aterm, atom_terms.data(), atom_terms.size() * sizeof(Term));
    if (!atom_mx.empty()) std::memcpy(hb.data() + o_amx, atom_mx.data(), atom_mx.size() * 8);
    if (!scale.empty()) std::memcpy(hb.data() + o_scale, scale.data(), scale.size() * sizeof(PrepTask));
    if (!sched.empty()) std::memcpy(hb.data() + o_sched, sched.data(), sched.size() * sizeof(LeafTile));
    std::memcpy(hb.data() + o_wfirst, wfirst.data(), wfirst.size() * 4);
    cudaError_t e = cudaMemcpy(blob, hb.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dev_free(blob);
        return cuda_fail(e, "tensor-core tables: upload");
    }
    d->tc_blob = blob;
    d->tcp = reinterpret_cast<TcProd*>(blob + o_tp);
    d->prep = reinterpret_cast<PrepTask*>(blob + o_prep);
    d->nprep = (int)prep.size();
    d->colmax = reinterpret_cast<PrepTask*>(blob + o_colmax);
    d->ncolmax = (int)colmax.size();
    d->status = reinterpret_cast<int*>(blob + o_status);
    d->term_mx = reinterpret_cast<int64_t*>(blob + o_tmx);
    d->mx_list = reinterpret_cast<int64_t*>(blob + o_list);
    d->atom_terms = reinterpret_cast<Term*>(blob + o_aterm);
    d->atom_mx = reinterpret_cast<int64_t*>(blob + o_amx);
    d->scale = reinterpret_cast<PrepTask*>(blob + o_scale);
    d->nscale = (int)scale.size();
    d->col_e = reinterpret_cast<int*>(blob + o_cole);
    d->term_max = reinterpret_cast<unsigned long long*>(blob + o_ex) + ex_elems;
    d->tc_ex = blob + o_ex;
    d->tc_ex_bytes = (size_t)ex_total * 8;
    d->sched = reinterpret_cast<LeafTile*>(blob + o_sched);
    d->wfirst = reinterpret_cast<int32_t*>(blob + o_wfirst);
    d->nworkers = nw;
    return ATA_OK;
}

ata_status launch_leaf_tc(const DeviceTables& t, const Bind* binds, int nb, cudaStream_t s, cudaEvent_t before_gemm) {
    cudaError_t e;
    if (nb <= 1) {
        BindSet<1> bs{};
        bs.b[0] = binds[0];
        e = launch_kind<1>(t, bs, s, before_gemm);
    } else {
        BindSet<kDevBinds> bs{};
        bs.b = binds;  // device array
        e = launch_kind<kDevBinds>(t, bs, s, before_gemm);
    }
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core leaf launch");
    return ATA_OK;
}

}  // namespace ata
