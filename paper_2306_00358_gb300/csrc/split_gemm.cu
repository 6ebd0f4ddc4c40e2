// Split-precision FP64 GEMM on the tcgen05 tensor cores (TRG_SPLIT_BF16).
//
// Each FP64 operand row (A) / column (B) gets a power-of-two scale 2^e with
// |x| < 2^e over the row, and is written as a fixed-point integer
//     X = rint(x * 2^(F - e)),   F = 7 + 8 (S - 1),
// cut into S signed digits, X = sum_p d_p 2^(8 (S-1-p)), |d_0| <= 128,
// d_p in [-128, 127] (an Ozaki-type error-free splitting; Ozaki, Ogita,
// Oishi, Rump, Numer. Algorithms 59 (2012) 95).  Slice p is stored in BF16
// as d_p 2^(-8p), exact (at most 8 significant bits), so
//     x = 2^(e - 7) sum_p slice_p   and
//     sum_k a_k b_k ~= 2^(ea + eb - 14) sum_{p + q < S} (A_p B_q^T).
// Products of BF16 values are exact in FP32.  With |d_0 e_0| <= 2^14 and
// |d_0 e_1| + |d_1 e_0| <= 2^15, runs of 512 K sum exactly in FP32 (|sum| <=
// 2^24), so the tensor cores accumulate
//   ACC0 = (0,0)            and  ACC1 = (0,1) + (1,0)   exactly over 512-K chunks,
//   R, R2 = the products with 2 <= p+q < S               in FP32 over the whole K
// (these carry weight <= 2^-16 relative to ACC0, so their FP32 rounding stays
// below the truncation error).  After every chunk the epilogue warps move
// ACC0 and ACC1 into an int64 per column; at the end of a tile the sum
//   V = I0 2^22 + I1 2^14 + rint(R 2^22) + rint(R2 2^22)      (int64, exact)
// is turned into the FP64 result V 2^(ea + eb - 36) with integer operations,
// keeping the FP64 pipe (1/64 of the FP32 rate on this part) out of the loop.
//
// Kernel layout: persistent, one CTA per SM, 128 x 128 output tiles, BF16
// operand tiles of 128 x 32 staged by TMA (64-byte swizzle) through an
// mbarrier pipeline; warp 0 issues TMA, warp 1 owns TMEM and issues
// tcgen05.mma (one thread), 16 epilogue warps drain TMEM (four per 32-lane
// quadrant, 32 columns each).  The single issuing thread, not the tensor
// pipe, limits a stream of 128 x 128 x 16 MMAs, so products that share an A
// slice and land in adjacent accumulators are issued as one N = 256 MMA
// (see ins_of: 6 instructions for the 10 products of four slices).  The
// remainder products are issued while the epilogue drains a finished chunk,
// so the tensor pipe keeps working across the drain.  Waiting threads are
// suspended in mbarrier.try_wait rather than spinning (spinning costs
// shared-memory cycles that the MMA operand reads need).  Every wait is
// bounded: on expiry the kernel records ST_TIMEOUT and leaves its loops.
//
// A second instance runs each 256 x 128 tile on a CTA pair (cta_group::2)
// with the same product table at M = 256: a wide entry A_p [B_b | B_b+1]
// takes B_b from the even CTA and B_b+1 from the odd one (each CTA stages one
// slice of every wide pair), a narrow entry A_p B_q takes 64 of B_q's columns
// from each CTA (half-height tiles).  Every instruction then drives both SMs,
// so the issuing thread (the even CTA's) needs half the instructions per
// product, and each SM reads less operand data from shared memory; the even
// CTA's barriers collect the loads and TMEM drains of the pair.  Enabled by
// mma_pairs.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace trg {

namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 32;                        // K per stage: 64 bytes of BF16
constexpr int TILE_BYTES = BM * BK * 2;       // 8 KB per 128 x 32 BF16 tile
constexpr int CHUNK_STAGES = 512 / BK;        // exact-accumulation run (512 K)
constexpr int EPI_WARPS = 16;
constexpr int THREADS = 64 + 32 * EPI_WARPS;  // TMA warp + MMA warp + epilogue
constexpr uint32_t TMEM_COLS = 512;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bounded mbarrier waits: 2 s

constexpr int CPT = 32;                        // accumulator columns per epilogue thread
constexpr int STAGING_BYTES = EPI_WARPS * 32 * 8 * 8;    // epilogue store staging, 32 KB
constexpr int SMEM_LIMIT = 232448;             // opt-in shared memory per block
constexpr int BAR_BYTES = 512;                 // mbarriers, TMEM address, flags, row maxima

// CG = CTAs per MMA (1, or a pair with cta_group::2).  A CTA stages its own
// 128 rows of A (all S slices) per stage, and B as follows.  One CTA: all S
// 128-row B slice tiles.  A pair issues the single-CTA product table (ins_of)
// with M = 256: a wide entry A_p [B_b | B_b+1] (b even) takes its first 128
// columns from the even CTA and the other 128 from the odd one, so each CTA
// holds one slice of every wide pair (the even CTA B0, B2, the odd one B1,
// B3: pair_wide_tiles); a narrow entry A_p B_q (q even, N = 128) takes 64 of
// B_q's 128 columns from each CTA, staged as half-height tiles
// (pair_half_tiles).  Both CTAs' accumulators then receive exactly the
// single-CTA products of their own rows.
constexpr int HALF_TILE_BYTES = TILE_BYTES / 2;  // 64 x 32 BF16
__host__ __device__ constexpr int pair_wide_tiles(int S) { return S >= 4 ? 2 : 1; }
__host__ __device__ constexpr int pair_half_tiles(int S) { return S == 2 ? 1 : S == 5 ? 3 : 2; }
__host__ __device__ constexpr int stage_bytes_for(int S, int CG) {
    return CG == 1 ? 2 * S * TILE_BYTES : (S + pair_wide_tiles(S)) * TILE_BYTES + pair_half_tiles(S) * HALF_TILE_BYTES;
}
// Only the staged epilogue uses the store staging tile; the other two leave
// its 32 KB to the operand pipeline, which a pair turns into one more stage.
__host__ __device__ constexpr int staging_bytes_for(int MODE) { return MODE == 0 ? STAGING_BYTES : 0; }
__host__ __device__ constexpr int stages_for(int S, int CG, int MODE) {
    return CG == 1 ? (S <= 4 ? 3 : 2)
                   : ((SMEM_LIMIT - 1024 - BAR_BYTES - staging_bytes_for(MODE)) / stage_bytes_for(S, CG) > 6
                          ? 6
                          : (SMEM_LIMIT - 1024 - BAR_BYTES - staging_bytes_for(MODE)) / stage_bytes_for(S, CG));
}
__host__ __device__ constexpr int smem_bytes_for(int S, int CG, int MODE) {
    // at least 120 KB so that a second CTA (and its 512 TMEM columns) never shares the SM
    return (stages_for(S, CG, MODE) * stage_bytes_for(S, CG) + 1024 + BAR_BYTES + staging_bytes_for(MODE)) > 120 * 1024
               ? stages_for(S, CG, MODE) * stage_bytes_for(S, CG) + 1024 /*align*/ + BAR_BYTES + staging_bytes_for(MODE)
               : 120 * 1024;
}
constexpr bool smem_fits() {
    for (int S = 2; S <= 5; ++S)
        for (int CG = 1; CG <= 2; ++CG)
            for (int MODE = 0; MODE <= 3; ++MODE)
                if (smem_bytes_for(S, CG, MODE) > SMEM_LIMIT || stages_for(S, CG, MODE) < 2) return false;
    return true;
}
static_assert(smem_fits(), "split MMA shared memory");

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// As mbar_try, but the thread is suspended until the phase completes or
// about `hint_ns` pass, instead of spinning on shared memory (a spinning
// waiter takes shared-memory cycles that the MMA operand reads need).
__device__ __forceinline__ bool mbar_try_suspend(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// Bounded wait; returns false (and flags the status word) on expiry or when
// another role of the CTA has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* status, unsigned long long limit_ns = WAIT_NS) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_suspend(bar, parity, 2000u)) {
        if (*abort_flag) return false;
        if (global_ns() - t0 > limit_ns) {
            *abort_flag = 1;
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// CTA pairs: rank in the cluster, peer addresses, remote arrive, cluster barrier
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Pair form: the load lands in this CTA's shared memory and completes its
// bytes on the mbarrier at a cluster address (the leader CTA's barrier).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major BF16 tile, 64-byte rows,
// 64-byte swizzle; 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                         // descriptor version
    d |= (uint64_t)4 << 61;                         // swizzle: 64 bytes
    return d;
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
template <int CG>
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (CG == 1)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// Arrive on this CTA's barrier once the MMAs issued so far have completed.
template <int CG>
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    if constexpr (CG == 1)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(bar)) : "memory");
    else
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(bar)) : "memory");
}
// ... on the barrier at the same offset in every CTA of the pair.
template <int CG>
__device__ __forceinline__ void mma_commit_all(uint64_t* bar) {
    if constexpr (CG == 1)
        mma_commit<1>(bar);
    else
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
            ::"r"(smem_u32(bar)), "h"((unsigned short)3) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// rint(x) as int64 for |x| < 2^46 with 32-bit conversions only (the 64-bit
// conversion runs on the FP64 pipe, 1/64 of the FP32 rate on this part):
// hf = rint(x 2^-16) and the remainder x - hf 2^16 are both exact in FP32,
// and rint(x) = hf 2^16 + rint(remainder) since hf 2^16 is an even integer.
__device__ __forceinline__ long long rint_f32_to_i64(float x) {
    const float hf = rintf(x * (1.0f / 65536.0f));
    const int lo = __float2int_rn(fmaf(-hf, 65536.0f, x));
    return ((long long)__float2int_rn(hf) << 16) + lo;
}

// Exact int64 -> FP64 bits times 2^e2, round-to-nearest-even, integer
// operations only.  Results below the normal range (|value| < 2^-1022, far
// under any entry that matters next to a normalised tensor) flush to zero.
__device__ __forceinline__ double scaled_i64_to_double(long long v, int e2) {
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int top = 63 - __clzll((long long)a);      // position of the leading one
    unsigned long long mant;
    int ex = top + e2;                                // unbiased exponent of the result
    if (top <= 52) {
        mant = a << (52 - top);
    } else {
        const int sh = top - 52;
        const unsigned long long half = 1ull << (sh - 1);
        const unsigned long long rem = a & ((1ull << sh) - 1);
        mant = a >> sh;
        if (rem > half || (rem == half && (mant & 1))) {
            ++mant;
            if (mant >> 53) { mant >>= 1; ++ex; }
        }
    }
    if (ex < -1022) return __longlong_as_double((long long)sign);
    if (ex > 1023) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
    const unsigned long long bits = sign | ((unsigned long long)(ex + 1023) << 52) | (mant & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

// The same for |v| < 2^53 (the value is exact: no rounding step).
__device__ __forceinline__ double scaled_i64_to_double_exact(long long v, int e2) {
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int top = 63 - __clzll((long long)a);
    const int ex = top + e2;
    if (ex < -1022) return __longlong_as_double((long long)sign);
    if (ex > 1023) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
    const unsigned long long mant = a << (52 - top);
    return __longlong_as_double((long long)(sign | ((unsigned long long)(ex + 1023) << 52) | (mant & ((1ull << 52) - 1))));
}

// |v| rounded to 53 significant bits (half to even), as the FP64 value of v
// has it, and the position of its leading one afterwards.
__device__ __forceinline__ unsigned long long round53(unsigned long long a, int& top) {
    top = 63 - __clzll((long long)a);
    if (top <= 52) return a;
    const int sh = top - 52;
    const unsigned long long half = 1ull << (sh - 1);
    const unsigned long long rem = a & ((1ull << sh) - 1);
    unsigned long long mant = a >> sh;
    if (rem > half || (rem == half && (mant & 1))) {
        ++mant;
        if (mant >> 53) { mant >>= 1; ++top; }
    }
    return mant << (top - 52);
}
// Biased exponent field of the FP64 value v 2^e2 (0 when v = 0 or the value
// flushes to zero, as in scaled_i64_to_double).
__device__ __forceinline__ int fp64_exponent_field(long long v, int e2) {
    if (v == 0) return 0;
    int top;
    round53(v < 0 ? (unsigned long long)(-v) : (unsigned long long)v, top);
    const int ex = top + e2 + 1023;
    return ex < 1 ? 0 : (ex > 2046 ? 2047 : ex);
}
// The fixed-point integer X = rint(x 2^(F - e_row)) (halves away from zero)
// that slicing the FP64 value x = v 2^e2 produces, computed from v: with
// V53 = |v| rounded to 53 bits and r = e_row - e2 - F, X = V53 / 2^r rounded
// (r > 0) or V53 2^-r (r <= 0).
// The same two for |v| < 2^53, where the FP64 value holds v exactly.
__device__ __forceinline__ int fp64_exponent_field_exact(long long v, int e2) {
    if (v == 0) return 0;
    const int top = 63 - __clzll(v < 0 ? -v : v);
    const int ex = top + e2 + 1023;
    return ex < 1 ? 0 : (ex > 2046 ? 2047 : ex);
}
template <int S>
__device__ __forceinline__ long long fused_fixed_point_exact(long long v, int e2, int e_row) {
    constexpr int F = 7 + 8 * (S - 1);
    if (v == 0) return 0;
    const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
    if (63 - __clzll((long long)a) + e2 + 1023 < 1) return 0;   // the FP64 value flushes to zero
    const int r = e_row - e2 - F;
    const long long X = r >= 63 ? 0 : r > 0 ? (long long)((a + (1ull << (r - 1))) >> r) : (long long)(a << (-r));
    return v < 0 ? -X : X;
}
template <int S>
__device__ __forceinline__ long long fused_fixed_point(long long v, int e2, int e_row) {
    constexpr int F = 7 + 8 * (S - 1);
    if (v == 0) return 0;
    int top;
    const unsigned long long a = round53(v < 0 ? (unsigned long long)(-v) : (unsigned long long)v, top);
    if (top + e2 + 1023 < 1) return 0;           // the FP64 value flushes to zero
    const int r = e_row - e2 - F;
    long long X;
    if (r >= 63) X = 0;
    else if (r > 0) X = (long long)((a + (1ull << (r - 1))) >> r);
    else X = (long long)(a << (-r));
    return v < 0 ? -X : X;
}

struct MmaArgs {
    int M, N, Kp;                  // logical rows / cols, padded K (multiple of BK)
    int Mp, Np;                    // padded rows of the A / B slice arrays
    int S;                         // slices
    const int* ea;                 // per-row exponents of A
    const int* eb;                 // per-col exponents of B
    double* C;
    const int64_t* c_m;
    const int64_t* c_n;
    int* status;
    int* cons_ef;              // optional: exponent fields of the consumer's rows
    const int64_t* cons_m;
    const int64_t* cons_n;
    int group_n;               // tile order: column blocks per group (see tile_coords)
    // optional fused hand-over: the consumer's A slices instead of C
    uint16_t* cs_out;
    int64_t cs_plane;          // Mp * Kp of the consumer's slice arrays
    int64_t cs_kp;
    int* cs_e;
    const int64_t* ck_m;
    const int64_t* ck_n;
    int rows_per_crow, cols_per_crow;
    int64_t ck_stride;         // fused: consumer-column step between adjacent producer columns
    int v_exact53;             // fused: every V is below 2^53 in magnitude (K <= 8192)
    int c_rows_fast;           // C's rows are adjacent: store without staging ...
    int64_t c_col_stride;      // ... with c_n[n + j] = c_n[n] + j c_col_stride in a 32-column group
    // limit of the epilogue's wait for a finished accumulator chunk (the
    // other waits keep WAIT_NS); a short one lets tests reach the timeout path
    unsigned long long acc_wait_ns;
    // split K (EPI_KSPLIT): a unit of work is (tile, part), part p
    // covering k blocks [p kb_per, (p + 1) kb_per) (kb_per a multiple of the
    // 512-deep chunk); each unit stores its exact fixed-point sums V in
    // kpart[(p N + n) M + m] and k_ksplit_reduce forms C.  ksplit = 1,
    // kb_per >= Kp / BK: one unit per tile.
    int ksplit, kb_per;
    long long* kpart;
    // optional list of the tiles to compute (mb << 32 | nb), in order; with
    // sym, C is symmetric and the list holds the tiles that reach the
    // diagonal or above: elements above the diagonal are written at (m, n)
    // and at (n, m), those below it not at all (their mirrors are)
    const long long* tile_list;
    int n_list;
    int sym;
};

// Tile order: column blocks in groups of group_n; inside a group the tiles run
// row block by row block.  The CTAs of one wave then share about
// grid / group_n row blocks of A and group_n column blocks of B, a working
// set the host sizes to stay in L2 (a plain row-major order over many column
// blocks streams all of B through L2 once per wave).
__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int group_n, int& mb, int& nb);
// Row and column block of the tile-th tile of a launch (a listed tile, or
// the tile order of tile_coords).
__device__ __forceinline__ void unit_tile(const MmaArgs& g, int tile, int tiles_m, int tiles_n, int& mb, int& nb) {
    if (g.tile_list) {
        const long long v = g.tile_list[tile];
        mb = (int)(v >> 32);
        nb = (int)(v & 0xffffffffll);
    } else {
        tile_coords(tile, tiles_m, tiles_n, g.group_n, mb, nb);
    }
}
__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int group_n, int& mb, int& nb) {
    const int per_group = tiles_m * group_n;
    const int group = tile / per_group;
    const int first_n = group * group_n;
    const int width = min(group_n, tiles_n - first_n);
    const int local = tile - group * per_group;
    mb = local / width;
    nb = first_n + local % width;
}

// The slice products of one 16-wide K step, as tcgen05.mma instructions.
// TMEM holds four 128-column accumulators, ACC0 | ACC1 | R | R2:
//   ACC0 = A0 B0 and ACC1 = A0 B1 + A1 B0, exact over 512-K chunks and drained
//   into int64 after each chunk; R and R2 = FP32 sums of the remaining
//   products (2 <= p + q < S) over the whole tile.
// Slices are stored with their weights (slice p = d_p 2^-8p), so a remainder
// product may go to either of R and R2; the assignment below lets one N = 256
// instruction cover A_p [B_q | B_q+1] (adjacent smem tiles) when its two
// results land in adjacent accumulators, which cuts the instruction count the
// single issuing thread has to sustain (S = 4: 6 instructions for 10 products).
// flag: 0 = reset at a chunk start, 1 = reset at a tile start, 2 = accumulate.
// Group 1 (touches ACC0 / ACC1, or initialises R) precedes group 2 except at a
// chunk start inside a tile, where group 2 runs while the epilogue drains.
struct SliceIns { int a, b, wide, col, flag, group; };
__host__ __device__ constexpr int ins_count(int S) { return S == 2 ? 2 : S == 3 ? 4 : S == 4 ? 6 : 9; }
__host__ __device__ constexpr SliceIns ins_of(int S, int t) {
    // common head: A0 [B0|B1] -> ACC0|ACC1, then (S >= 3) R initialised by A2 B0
    // (with A2 B1 into R2 when S >= 4), then A1 [B0|B1] -> ACC1|R
    return S == 2 ? (t == 0 ? SliceIns{0, 0, 1, 0, 0, 1} : SliceIns{1, 0, 0, 128, 2, 1})
         : S == 3 ? (t == 0 ? SliceIns{0, 0, 1, 0, 0, 1}
                   : t == 1 ? SliceIns{2, 0, 0, 256, 1, 1}
                   : t == 2 ? SliceIns{1, 0, 1, 128, 2, 1}
                            : SliceIns{0, 2, 0, 256, 2, 2})
         : S == 4 ? (t == 0 ? SliceIns{0, 0, 1, 0, 0, 1}
                   : t == 1 ? SliceIns{2, 0, 1, 256, 1, 1}
                   : t == 2 ? SliceIns{1, 0, 1, 128, 2, 1}
                   : t == 3 ? SliceIns{0, 2, 1, 256, 2, 2}
                   : t == 4 ? SliceIns{1, 2, 0, 384, 2, 2}
                            : SliceIns{3, 0, 0, 384, 2, 2})
                  : (t == 0 ? SliceIns{0, 0, 1, 0, 0, 1}
                   : t == 1 ? SliceIns{2, 0, 1, 256, 1, 1}
                   : t == 2 ? SliceIns{1, 0, 1, 128, 2, 1}
                   : t == 3 ? SliceIns{0, 2, 1, 256, 2, 2}
                   : t == 4 ? SliceIns{1, 2, 1, 256, 2, 2}
                   : t == 5 ? SliceIns{3, 0, 1, 256, 2, 2}
                   : t == 6 ? SliceIns{2, 2, 0, 384, 2, 2}
                   : t == 7 ? SliceIns{0, 4, 0, 384, 2, 2}
                            : SliceIns{4, 0, 0, 384, 2, 2});
}
// Every product p + q < S exactly once, and no other (checked at compile time).
__host__ __device__ constexpr bool ins_cover_ok(int S) {
    int seen[5][5] = {};
    for (int t = 0; t < ins_count(S); ++t) {
        const SliceIns in = ins_of(S, t);
        seen[in.a][in.b] += 1;
        if (in.wide) {
            if (in.b + 1 >= S) return false;
            seen[in.a][in.b + 1] += 1;
        }
    }
    for (int p = 0; p < 5; ++p)
        for (int q = 0; q < 5; ++q)
            if (seen[p][q] != ((p < S && q < S && p + q < S) ? 1 : 0)) return false;
    return true;
}
static_assert(ins_cover_ok(2) && ins_cover_ok(3) && ins_cover_ok(4) && ins_cover_ok(5), "slice product table");

// A pair issues the same table: every wide entry starts at an even B slice
// whose pair a CTA stages (b / 2 < pair_wide_tiles), every narrow entry reads
// an even B slice staged as half tiles (q / 2 < pair_half_tiles).
__host__ __device__ constexpr bool pair_table_ok(int S) {
    for (int t = 0; t < ins_count(S); ++t) {
        const SliceIns in = ins_of(S, t);
        if (in.b % 2 != 0) return false;
        if (in.wide && (in.b / 2 >= pair_wide_tiles(S) || in.b + 1 >= S)) return false;
        if (!in.wide && in.b / 2 >= pair_half_tiles(S)) return false;
    }
    return true;
}
static_assert(pair_table_ok(2) && pair_table_ok(3) && pair_table_ok(4) && pair_table_ok(5), "pair staging");

// Epilogue kinds: FP64 results stored through a staging tile (columns
// adjacent in C), stored directly (rows adjacent in C), or the consumer's
// slices (fused hand-over).  One kernel instance each keeps the register
// allocation of each epilogue to itself.
enum EpiMode { EPI_STAGED = 0, EPI_DIRECT = 1, EPI_FUSED = 2, EPI_KSPLIT = 3 };

template <int S, int CG, int MODE>
__global__ void __launch_bounds__(THREADS, 1)
k_split_mma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const __grid_constant__ CUtensorMap tmBh, const MmaArgs g) {
    constexpr int STAGES = stages_for(S, CG, MODE);
    constexpr int STAGE_BYTES = stage_bytes_for(S, CG);
    constexpr int B_TILE = TILE_BYTES;
    constexpr int PW = pair_wide_tiles(S), PH = pair_half_tiles(S);   // pair staging (CG = 2)
    constexpr int TILE_M = BM * CG;                // output rows per tile (per CTA pair)
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* mma_done = acc_empty + 1;
    uint64_t* cs_bar = mma_done + 1;             // epilogue warps: consumer-row maxima are complete
    uint32_t* tmem_slot = (uint32_t*)(cs_bar + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    unsigned* cs_slot = (unsigned*)(tmem_slot + 4);   // 2 x 16 consumer-row maxima, tagged by tile
    double* staging = (double*)(smem + STAGES * STAGE_BYTES + BAR_BYTES);   // EPI_WARPS x 32 x 8 doubles

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int tiles_m = (g.M + TILE_M - 1) / TILE_M;
    const int tiles_n = (g.N + BN - 1) / BN;
    const int num_tiles = g.tile_list ? g.n_list : tiles_m * tiles_n;
    const int num_kb = g.Kp / BK;
    const int num_units = num_tiles * g.ksplit;
    // a pair shares every tile: the leader (rank 0) issues the MMAs for both,
    // and its barriers collect the loads and the drains of both CTAs
    const uint32_t rank = CG == 2 ? cluster_rank() : 0u;
    const int first_tile = (int)blockIdx.x / CG, tile_step = (int)gridDim.x / CG;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, EPI_WARPS * CG);
        mbar_init(mma_done, 1);
        mbar_init(cs_bar, EPI_WARPS);
        *abort_flag = 0;
        for (int i = 0; i < 32; ++i) cs_slot[i] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        if constexpr (CG == 1) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        } else {
            // one warp of each CTA of the pair takes part
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                         ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
        }
    }
    tc_fence_before();
    if constexpr (CG == 2)
        cluster_sync_all();     // the peer's barriers are initialised before any remote arrive
    else
        __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t leader_full0 = CG == 2 ? map_to_rank(smem_u32(full), 0) : smem_u32(full);
    const uint32_t leader_acc_empty = CG == 2 ? map_to_rank(smem_u32(acc_empty), 0) : smem_u32(acc_empty);

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued[STAGES];          // parity of the last load issued per stage, -1 = none
#pragma unroll
            for (int s = 0; s < STAGES; ++s) issued[s] = -1;
            bool ok = true;
            for (int unit = first_tile; unit < num_units && ok; unit += tile_step) {
                const int tile = unit / g.ksplit;
                const int kb0 = (unit - tile * g.ksplit) * g.kb_per;
                const int kb1 = min(num_kb, kb0 + g.kb_per);
                int mb, nb;
                unit_tile(g, tile, tiles_m, tiles_n, mb, nb);
                const int arow = mb * TILE_M + (int)rank * BM, brow = nb * BN;
                for (int kb = kb0; kb < kb1 && ok; ++kb) {
                    ok = mbar_wait(&empty[stage], phase ^ 1, abort_flag, g.status);
                    if (!ok) break;
                    uint8_t* st = smem + stage * STAGE_BYTES;
                    if (rank == 0) mbar_expect_tx(&full[stage], CG * STAGE_BYTES);   // both CTAs' bytes
                    if constexpr (CG == 1) {
                        for (int p = 0; p < S; ++p) {
                            tma_load_2d(st + p * TILE_BYTES, &tmA, kb * BK, p * g.Mp + arow, &full[stage]);
                            tma_load_2d(st + S * TILE_BYTES + p * B_TILE, &tmB, kb * BK, p * g.Np + brow,
                                        &full[stage]);
                        }
                    } else {
                        const uint32_t bar = leader_full0 + (uint32_t)(stage * sizeof(uint64_t));
                        for (int p = 0; p < S; ++p)
                            tma_load_2d_pair(st + p * TILE_BYTES, &tmA, kb * BK, p * g.Mp + arow, bar);
                        // wide pairs: this CTA's slice 2w + rank of the pair (2w, 2w + 1)
                        for (int w = 0; w < PW; ++w)
                            tma_load_2d_pair(st + S * TILE_BYTES + w * B_TILE, &tmB, kb * BK,
                                             (2 * w + (int)rank) * g.Np + brow, bar);
                        // narrow products: this CTA's 64 columns of slice 2h
                        for (int h = 0; h < PH; ++h)
                            tma_load_2d_pair(st + (S + PW) * TILE_BYTES + h * HALF_TILE_BYTES, &tmBh, kb * BK,
                                             2 * h * g.Np + brow + (int)rank * (BN / 2), bar);
                    }
#pragma unroll
                    for (int s = 0; s < STAGES; ++s)
                        if (s == stage) issued[s] = (int)phase;
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
            }
            // every load issued has landed before the CTA may exit (bounded,
            // and done even after an abort); the leader's barriers count the
            // bytes of both CTAs of a pair
            volatile int never = 0;
            if (rank == 0) {
#pragma unroll
                for (int s = 0; s < STAGES; ++s)
                    if (issued[s] >= 0) mbar_wait(&full[s], (uint32_t)issued[s], &never, g.status);
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0 && rank == 0) {
            constexpr uint32_t IDESC = idesc_bf16(TILE_M, BN);
            constexpr uint32_t IDESC_N256 = idesc_bf16(TILE_M, 2 * BN);
            int stage = 0;
            uint32_t phase = 0;
            uint32_t chunk_no = 0;      // chunks issued so far (all tiles)
            bool ok = true;
            for (int unit = first_tile; unit < num_units && ok; unit += tile_step) {
                // k blocks of this unit, counted from its first (a chunk boundary)
                const int kb0 = (unit % g.ksplit) * g.kb_per;
                const int nkb = min(num_kb, kb0 + g.kb_per) - kb0;
                for (int kb = 0; kb < nkb && ok; ++kb) {
                    const bool chunk_start = (kb % CHUNK_STAGES) == 0;
                    const bool tile_end = kb + 1 == nkb;
                    const bool chunk_end = ((kb + 1) % CHUNK_STAGES) == 0 || tile_end;
                    ok = mbar_wait(&full[stage], phase, abort_flag, g.status);
                    if (!ok) break;
                    tc_fence_after();
                    // descriptors of this stage: one base, compile-time offsets
                    // (start address in 16-byte units in the low 14 bits)
                    const uint64_t dbase = smem_desc(smem_u32(smem + stage * STAGE_BYTES));
                    // the instructions of one group for both 16-wide K steps
                    auto issue = [&](int group) {
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
                            for (int t = 0; t < ins_count(S); ++t) {
                                const SliceIns in = ins_of(S, t);
                                if (in.group != group) continue;
                                uint32_t acc = 1u;
                                if (in.flag == 0) acc = (chunk_start && kk == 0) ? 0u : 1u;
                                if (in.flag == 1) acc = (kb == 0 && kk == 0) ? 0u : 1u;
                                const uint64_t da = dbase + (uint64_t)((in.a * TILE_BYTES + kk * 32) >> 4);
                                // one CTA: B_q and B_q+1 are adjacent 128-row tiles, so a wide entry is
                                // one N = 256 product.  A pair: a wide entry reads the pair's tile b / 2
                                // (B_b in the even CTA, B_b+1 in the odd one), a narrow one the half
                                // tiles of B_b (64 columns in each CTA)
                                const int boff = CG == 1 ? S * TILE_BYTES + in.b * B_TILE
                                               : in.wide ? (S + in.b / 2) * TILE_BYTES
                                                         : (S + PW) * TILE_BYTES + (in.b / 2) * HALF_TILE_BYTES;
                                const uint64_t db = dbase + (uint64_t)((boff + kk * 32) >> 4);
                                mma_bf16<CG>(tmem + in.col, da, db, in.wide ? IDESC_N256 : IDESC, acc);
                            }
                        }
                    };
                    if (chunk_start && kb > 0) {
                        // a drain of the exact accumulators inside this tile is
                        // pending: keep the tensor pipe busy on R / R2 meanwhile
                        issue(2);
                        ok = mbar_wait(acc_empty, (chunk_no - 1) & 1, abort_flag, g.status);
                        if (!ok) break;
                        tc_fence_after();
                        issue(1);
                    } else {
                        if (chunk_start && chunk_no > 0) {
                            // the previous tile's results (R and R2 included) have been read
                            ok = mbar_wait(acc_empty, (chunk_no - 1) & 1, abort_flag, g.status);
                            if (!ok) break;
                            tc_fence_after();
                        }
                        issue(1);
                        if (chunk_end && !tile_end) {
                            mma_commit_all<CG>(acc_full);    // tracks group 1 (ACC0, ACC1) only
                            ++chunk_no;
                        }
                        issue(2);
                    }
                    mma_commit_all<CG>(&empty[stage]);
                    if (tile_end) {
                        mma_commit_all<CG>(acc_full);
                        ++chunk_no;
                    }
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
            }
            // every MMA issued has completed (also after an abort) ...
            mma_commit<CG>(mma_done);
            volatile int never = 0;
            mbar_wait(mma_done, 0, &never, g.status);
            // ... and the last chunk has been drained before TMEM is released
            if (ok && chunk_no > 0) mbar_wait(acc_empty, (chunk_no - 1) & 1, abort_flag, g.status);
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - 2;                  // 0..15
        const int quad = warp & 3;                // TMEM lane quadrant this warp may access
        const int colh = ew >> 2;                 // which 32-column quarter
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        const int row_in_tile = quad * 32 + lane;
        uint32_t chunk_no = 0;
        uint32_t tile_iter = 0;                   // tiles done by this CTA (tags the row maxima)
        bool ok = true;
        for (int unit = first_tile; unit < num_units && ok; unit += tile_step) {
            const int tile = unit / g.ksplit;
            const int part = unit - tile * g.ksplit;
            const int kb0 = part * g.kb_per;
            const int nchunks = (min(num_kb, kb0 + g.kb_per) - kb0 + CHUNK_STAGES - 1) / CHUNK_STAGES;
            int mb, nb;
            unit_tile(g, tile, tiles_m, tiles_n, mb, nb);
            ++tile_iter;
            const int row0 = mb * TILE_M + (int)rank * BM;   // this CTA's rows of the tile
            // J = I0 2^8 + I1: the exact ACC0 and ACC1 sums of this tile's
            // columns in one int64 each; at the end J becomes
            // V = J 2^14 + rint(R 2^22) + rint(R2 2^22) and then, in place, the FP64 bits
            long long J[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) J[j] = 0;
            for (int c = 0; c < nchunks && ok; ++c) {
                // one lane waits, the warp follows (the TMEM loads are warp-collective)
                int w_ok = 1;
                if (lane == 0) w_ok = mbar_wait(acc_full, chunk_no & 1, abort_flag, g.status, g.acc_wait_ns) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
                if (!ok) break;
                tc_fence_after();
                const bool last = (c == nchunks - 1);
                const int m = row0 + row_in_tile;
                const bool row_ok = m < g.M;
                const int ea = (last && row_ok) ? g.ea[m] : 0;
#pragma unroll
                for (int h = 0; h < CPT / 8; ++h) {           // 8 columns at a time
                    const uint32_t col = (uint32_t)(colh * CPT + h * 8);
                    uint32_t r[8];
                    tmem_ld8(tmem + lane_base + col, r);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; ++j) J[h * 8 + j] += (long long)__float2int_rn(__uint_as_float(r[j])) << 8;
                    tmem_ld8(tmem + lane_base + 128 + col, r);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; ++j) J[h * 8 + j] += __float2int_rn(__uint_as_float(r[j]) * 256.0f);
                    if (last) {
                        // fold in R and R2: J becomes V = J 2^14 + rint(R 2^22) + rint(R2 2^22)
                        // (with two slices no product lands in R, with three none in R2:
                        // their columns are never written and read as zero here)
                        long long rr[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) rr[j] = 0;
                        if (S >= 3) {
                            tmem_ld8(tmem + lane_base + 256 + col, r);
                            tmem_wait_ld();
#pragma unroll
                            for (int j = 0; j < 8; ++j) rr[j] = rint_f32_to_i64(__uint_as_float(r[j]) * 4194304.0f);
                        }
                        if (S >= 4) {
                            tmem_ld8(tmem + lane_base + 384 + col, r);
                            tmem_wait_ld();
#pragma unroll
                            for (int j = 0; j < 8; ++j) rr[j] += rint_f32_to_i64(__uint_as_float(r[j]) * 4194304.0f);
                        }
#pragma unroll
                        for (int j = 0; j < 8; ++j) J[h * 8 + j] = (J[h * 8 + j] << 14) + rr[j];
                    }
                }
                // TMEM is free for the next tile before the FP64 results are
                // formed and stored
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (CG == 1)
                        mbar_arrive(acc_empty);
                    else
                        mbar_arrive_cluster(leader_acc_empty);
                }
                ++chunk_no;
                if (last) {
                    const int nt = nb * BN + colh * CPT;
                    if constexpr (MODE == EPI_DIRECT) {
                        // rows adjacent in C: form, record and store each result in one
                        // pass (the lanes, adjacent rows, write 256 contiguous bytes).
                        // The warp's 32 columns are the same for every lane: lane j
                        // loads column j's exponent and consumer-row offset once and
                        // the loop takes them by shuffle, so no global load waits
                        // inside it.
                        const bool col_in = nt + lane < g.N;
                        const int eb_l = col_in ? g.eb[nt + lane] - 36 : 0;
                        const long long cn_l = (g.cons_ef && col_in) ? (long long)g.cons_n[nt + lane] : 0;
                        double* cp = g.C + (row_ok ? g.c_m[m] + g.c_n[nt] : 0);
                        const int64_t step = g.c_col_stride;
                        const int64_t cm0 = (g.cons_ef && row_ok) ? g.cons_m[m] : 0;
                        int64_t cur = -1;
                        int cur_max = 0;
#pragma unroll
                        for (int j = 0; j < CPT; ++j) {
                            const int e2 = ea + __shfl_sync(0xffffffffu, eb_l, j);
                            const long long cn = __shfl_sync(0xffffffffu, cn_l, j);
                            if (row_ok && nt + j < g.N) {
                                const double v = g.v_exact53 ? scaled_i64_to_double_exact(J[j], e2)
                                                             : scaled_i64_to_double(J[j], e2);
                                *cp = v;
                                if (g.cons_ef) {
                                    const int64_t crow = cm0 + cn;
                                    const int ef = (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF);
                                    if (crow != cur) {
                                        if (cur >= 0 && cur_max) atomicMax(&g.cons_ef[cur], cur_max);
                                        cur = crow;
                                        cur_max = ef;
                                    } else {
                                        cur_max = max(cur_max, ef);
                                    }
                                }
                            }
                            cp += step;
                        }
                        if (cur >= 0 && cur_max) atomicMax(&g.cons_ef[cur], cur_max);
                        continue;
                    }
                    if constexpr (MODE == EPI_KSPLIT) {
                        // split K: this part's exact sums, rows adjacent (a warp
                        // writes 256 contiguous bytes per column); k_ksplit_reduce
                        // forms the FP64 results
                        if (row_ok) {
                            long long* dst = g.kpart + ((int64_t)part * g.N + nt) * g.M + m;
#pragma unroll
                            for (int j = 0; j < CPT; ++j)
                                if (nt + j < g.N) dst[(int64_t)j * g.M] = J[j];
                        }
                        continue;
                    }
                    if constexpr (MODE == EPI_STAGED) {
                        // the FP64 results, in place
#pragma unroll
                        for (int j = 0; j < CPT; ++j) {
                            const int n = nt + j;
                            double v = 0.0;
                            if (row_ok && n < g.N) v = scaled_i64_to_double(J[j], ea + g.eb[n] - 36);
                            J[j] = __double_as_longlong(v);
                        }
                    }
                    if constexpr (MODE == EPI_FUSED) {
                        // fused hand-over: the consumer's rows lie in this tile; a
                        // warp's lanes and a thread's columns share one of them.  The
                        // slices follow from V directly, equal to slicing the FP64
                        // value V 2^(ea + eb - 36) (see fused_fixed_point).
                        // |V| < 2^53 (K <= 8192) needs no rounding to 53 bits
                        const bool exact53 = g.v_exact53 != 0;
                        unsigned tmax = 0;
#pragma unroll
                        for (int j = 0; j < CPT; ++j)
                            if (row_ok && nt + j < g.N)
                                tmax = max(tmax, (unsigned)(exact53 ? fp64_exponent_field_exact(J[j], ea + g.eb[nt + j] - 36)
                                                                    : fp64_exponent_field(J[j], ea + g.eb[nt + j] - 36)));
                        const unsigned wmax = __reduce_max_sync(0xffffffffu, tmax);
                        // double-buffered by tile parity: a warp may run one tile ahead
                        const int slot = (int)(tile_iter & 1) * 16 + (row_in_tile / g.rows_per_crow) * (BN / g.cols_per_crow) +
                                         (colh * CPT) / g.cols_per_crow;
                        int w_ok = 1;
                        if (lane == 0) {
                            atomicMax(&cs_slot[slot], (tile_iter << 11) | wmax);
                            mbar_arrive(cs_bar);    // release: the maximum above is visible after the wait
                            w_ok = mbar_wait(cs_bar, (tile_iter - 1) & 1, abort_flag, g.status) ? 1 : 0;
                        }
                        ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
                        if (!ok) break;
                        const unsigned sv = cs_slot[slot];
                        const int ef = ((sv >> 11) == (tile_iter & 0x1FFFFFu)) ? (int)(sv & 0x7FFu) : 0;
                        const int e_row = ef ? ef - 1022 : -1022;           // |x| < 2^e_row over the row
                        if (row_ok && nt < g.N) {
                            const int64_t crow = g.cons_m[m] + g.cons_n[nt];
                            if (lane == 0) g.cs_e[crow] = e_row;
                            // consumer column of this thread's column j: ck_m[m] + ck_n[nt] +
                            // j ck_stride, with ck_m[m] = the lane's row offset (adjacent
                            // lanes, adjacent columns): each store writes 64 contiguous bytes
                            uint16_t* dst = g.cs_out + crow * g.cs_kp + g.ck_m[m] + g.ck_n[nt];
                            const int64_t step = g.ck_stride, plane = g.cs_plane;
#pragma unroll
                            for (int j = 0; j < CPT; ++j) {
                                const int e2 = ea + g.eb[nt + j] - 36;
                                long long X = exact53 ? fused_fixed_point_exact<S>(J[j], e2, e_row)
                                                      : fused_fixed_point<S>(J[j], e2, e_row);
                                int d[S];
                                // signed base-256 digits; |X| <= 2^F, so after S - 3 digits
                                // (S >= 4) the rest fits in 32 bits
#pragma unroll
                                for (int p = S - 1; p >= 1; --p) {
                                    const int lo8 = (int)(((unsigned)X + 128u) & 255u) - 128;   // low bits only
                                    d[p] = lo8;
                                    if (p > 2) X = (X - lo8) >> 8;
                                    else X = ((int)X - lo8) >> 8;
                                }
                                d[0] = (int)X;
#pragma unroll
                                for (int p = 0; p < S; ++p) {
                                    // small integer -> FP32 exactly, times 2^-8p; the top half is the BF16
                                    float f = __int_as_float(0x4B400000 + d[p]) - 12582912.0f;
                                    if (p > 0) f *= __int_as_float((127 - 8 * p) << 23);
                                    dst[p * plane] = (uint16_t)(__float_as_uint(f) >> 16);
                                }
                                dst += step;
                            }
                        }
                    }
                    if (MODE == EPI_STAGED && g.cons_ef && row_ok) {
                        // exponent fields of the consumer's rows: run-length maxima
                        // over this thread's columns, one atomic per run
                        const int64_t cm0 = g.cons_m[m];
                        int64_t cur = -1;
                        int cur_max = 0;
#pragma unroll
                        for (int j = 0; j < CPT; ++j) {
                            const int n = nt + j;
                            if (n < g.N) {
                                const int64_t crow = cm0 + g.cons_n[n];
                                const int ef = (int)(((unsigned long long)J[j] >> 52) & 0x7FF);
                                if (crow != cur) {
                                    if (cur >= 0 && cur_max) atomicMax(&g.cons_ef[cur], cur_max);
                                    cur = crow;
                                    cur_max = ef;
                                } else {
                                    cur_max = max(cur_max, ef);
                                }
                            }
                        }
                        if (cur >= 0 && cur_max) atomicMax(&g.cons_ef[cur], cur_max);
                    }
                    if (MODE == EPI_FUSED) continue;
                    if (MODE == EPI_STAGED && g.sym && row_ok) {
                        // symmetric C: the mirror (n, m) of each element above the
                        // diagonal (adjacent lanes, adjacent rows m: contiguous in
                        // a row of C)
                        const int64_t cm_mirror = g.c_n[m];
#pragma unroll
                        for (int j = 0; j < CPT; ++j) {
                            const int n = nt + j;
                            if (n < g.N && n > m) g.C[g.c_m[n] + cm_mirror] = __longlong_as_double(J[j]);
                        }
                    }
                    // stores through the warp's 32 x 8 staging tile: lanes of a
                    // quarter-warp then write 8 adjacent columns (64 B) of one row
                    double* stg = staging + ew * (32 * 8);
                    const int quarter = lane >> 3, cl = lane & 7;
#pragma unroll
                    for (int pass = 0; pass < CPT / 8; ++pass) {
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj)
                            stg[lane * 8 + (jj ^ ((lane >> 1) & 7))] = __longlong_as_double(J[pass * 8 + jj]);
                        __syncwarp();
                        const int n = nb * BN + colh * CPT + pass * 8 + cl;
                        const int64_t cn = (n < g.N) ? g.c_n[n] : 0;
#pragma unroll 4
                        for (int q = 0; q < 8; ++q) {
                            const int rr = 4 * q + quarter;
                            const int mr = row0 + quad * 32 + rr;
                            if (mr < g.M && n < g.N && (!g.sym || n >= mr))
                                g.C[g.c_m[mr] + cn] = stg[rr * 8 + (cl ^ ((rr >> 1) & 7))];
                        }
                        __syncwarp();
                    }
                }
            }
        }
    }

    // no MMA of the pair is in flight and both CTAs have drained their TMEM
    tc_fence_before();
    if constexpr (CG == 2)
        cluster_sync_all();
    else
        __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        if constexpr (CG == 1)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
        else
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// ------------------------------------------------------------- slicing ----
// Per-row maximum of the biased FP64 exponent field (0 for an all-zero row).
// Source element (r, k) at src[off_r[r] + off_c[k]].
constexpr int SL_R = 32, SL_K = 64;

__global__ void __launch_bounds__(256) k_row_exponent(const double* __restrict__ src, const int64_t* __restrict__ off_r,
                                                      const int64_t* __restrict__ off_c, int R, int K, int k_fast,
                                                      int* __restrict__ ef_out) {
    __shared__ int rmax[SL_R];
    const int k0 = blockIdx.x * SL_K;
    const int nby = (R + SL_R - 1) / SL_R;   // row blocks, strided over grid.y (at most 65535)
    for (int by = blockIdx.y; by < nby; by += gridDim.y) {
        const int r0 = by * SL_R;
        if (threadIdx.x < SL_R) rmax[threadIdx.x] = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < SL_R * SL_K; e += 256) {
            int rr, kk;
            if (k_fast) { kk = e % SL_K; rr = e / SL_K; } else { rr = e % SL_R; kk = e / SL_R; }
            const int r = r0 + rr, k = k0 + kk;
            if (r < R && k < K) {
                const unsigned long long b = (unsigned long long)__double_as_longlong(src[off_r[r] + off_c[k]]);
                const int ef = (int)((b >> 52) & 0x7FF);
                if (ef) atomicMax(&rmax[rr], ef);
            }
        }
        __syncthreads();
        if (threadIdx.x < SL_R && r0 + (int)threadIdx.x < R && rmax[threadIdx.x])
            atomicMax(&ef_out[r0 + threadIdx.x], rmax[threadIdx.x]);
        __syncthreads();
    }
}

// Split K: C(m, n) = the sum over the parts, in part order, of their exact
// fixed-point sums V (kpart[(p N + n) M + m]), scaled by 2^(ea_m + eb_n - 36)
// as the staged epilogue scales an unsplit V.
__global__ void __launch_bounds__(256) k_ksplit_reduce(const long long* __restrict__ part, int ksplit, int M, int N,
                                                       const int* __restrict__ ea, const int* __restrict__ eb,
                                                       double* C, const int64_t* __restrict__ c_m,
                                                       const int64_t* __restrict__ c_n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * N) return;
    const int n = (int)(i / M), m = (int)(i - (int64_t)n * M);
    long long v = 0;
    for (int p = 0; p < ksplit; ++p) v += part[((int64_t)p * N + n) * M + m];
    C[c_m[m] + c_n[n]] = scaled_i64_to_double(v, ea[m] + eb[n] - 36);
}

// Convert the raw exponent fields to scale exponents e (|x| < 2^e).
__global__ void k_exponent_finish(int* ef, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) ef[r] = ef[r] ? ef[r] - 1022 : -1022;
}

// Slices: out[p][r][k] (BF16 bits), r < Rp, k < Kp, zero in the padding.
template <int S>
__global__ void __launch_bounds__(256) k_slice(const double* __restrict__ src, const int64_t* __restrict__ off_r,
                                               const int64_t* __restrict__ off_c, int R, int K, int Rp, int Kp,
                                               int k_fast, const int* __restrict__ e_row,
                                               uint16_t* __restrict__ out) {
    __shared__ double tile[SL_R][SL_K + 1];
    const int k0 = blockIdx.x * SL_K;
    const int nby = (Rp + SL_R - 1) / SL_R;   // row blocks, strided over grid.y (at most 65535)
    for (int by = blockIdx.y; by < nby; by += gridDim.y) {
        const int r0 = by * SL_R;
        __syncthreads();   // the previous block's tile has been read
        for (int e = threadIdx.x; e < SL_R * SL_K; e += 256) {
            int rr, kk;
            if (k_fast) { kk = e % SL_K; rr = e / SL_K; } else { rr = e % SL_R; kk = e / SL_R; }
            const int r = r0 + rr, k = k0 + kk;
            tile[rr][kk] = (r < R && k < K) ? src[off_r[r] + off_c[k]] : 0.0;
        }
        __syncthreads();
        constexpr int F = 7 + 8 * (S - 1);
        for (int e = threadIdx.x; e < SL_R * SL_K; e += 256) {
            const int kk = e % SL_K, rr = e / SL_K;
            const int r = r0 + rr, k = k0 + kk;
            if (r >= Rp || k >= Kp) continue;
            long long X = 0;
            if (r < R) {
                const unsigned long long b = (unsigned long long)__double_as_longlong(tile[rr][kk]);
                const int ex = (int)((b >> 52) & 0x7FF);
                if (ex) {
                    const int ea = e_row[r];                       // |x| < 2^ea
                    const int shift = 52 + 1023 + ea - ex - F;     // >= 53 - F > 0
                    if (shift < 63) {
                        const unsigned long long m53 = (b & ((1ull << 52) - 1)) | (1ull << 52);
                        X = (long long)((m53 + (1ull << (shift - 1))) >> shift);
                        if (b >> 63) X = -X;
                    }
                }
            }
            int d[S];
#pragma unroll
            for (int p = S - 1; p >= 1; --p) {
                const int lo = (int)(((X + 128) & 255) - 128);
                d[p] = lo;
                X = (X - lo) >> 8;
            }
            d[0] = (int)X;
            const size_t plane = (size_t)Rp * Kp;
#pragma unroll
            for (int p = 0; p < S; ++p) {
                // small integer -> FP32 exactly (|d| < 2^22), times 2^-8p, top 16 bits = BF16
                const float f = (__int_as_float(0x4B400000 + d[p]) - 12582912.0f) * __int_as_float((127 - 8 * p) << 23);
                out[p * plane + (size_t)r * Kp + k] = (uint16_t)(__float_as_uint(f) >> 16);
            }
        }
    }
}

// Slices of an operand whose rows are contiguous runs (src + off_r[r] + k):
// a warp per row, four columns per lane per pass with 16-byte loads and
// 8-byte stores of four BF16 per slice.  Same arithmetic as k_slice (the
// slices are bit-identical), without the tile transpose through shared memory.
template <int S>
__global__ void __launch_bounds__(256) k_slice_contig(const double* __restrict__ src, const int64_t* __restrict__ off_r,
                                                      int R, int K, int Rp, int Kp, const int* __restrict__ e_row,
                                                      uint16_t* __restrict__ out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * 8 + warp;
    if (r >= Rp) return;
    const size_t plane = (size_t)Rp * Kp;
    uint16_t* orow = out + (size_t)r * Kp;
    constexpr int F = 7 + 8 * (S - 1);
    const bool real = r < R;
    const double* row = real ? src + off_r[r] : nullptr;
    const bool vec = real && ((reinterpret_cast<uintptr_t>(row) & 15) == 0);
    const int ea = real ? e_row[r] : 0;
    for (int k0 = lane * 4; k0 < Kp; k0 += 128) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (real) {
            if (vec && k0 + 3 < K) {
                const double2 a = *reinterpret_cast<const double2*>(row + k0);
                const double2 b = *reinterpret_cast<const double2*>(row + k0 + 2);
                v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (k0 + j < K) v[j] = row[k0 + j];
            }
        }
        uint32_t pk[S][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(v[j]);
            const int ex = (int)((b >> 52) & 0x7FF);
            long long X = 0;
            if (ex) {
                const int shift = 52 + 1023 + ea - ex - F;     // >= 53 - F > 0
                if (shift < 63) {
                    const unsigned long long m53 = (b & ((1ull << 52) - 1)) | (1ull << 52);
                    X = (long long)((m53 + (1ull << (shift - 1))) >> shift);
                    if (b >> 63) X = -X;
                }
            }
            int d[S];
#pragma unroll
            for (int p = S - 1; p >= 1; --p) {
                const int lo = (int)(((X + 128) & 255) - 128);
                d[p] = lo;
                X = (X - lo) >> 8;
            }
            d[0] = (int)X;
#pragma unroll
            for (int p = 0; p < S; ++p) {
                const float f = (__int_as_float(0x4B400000 + d[p]) - 12582912.0f) * __int_as_float((127 - 8 * p) << 23);
                const uint32_t hb = __float_as_uint(f) >> 16;
                if (j & 1) pk[p][j >> 1] |= hb << 16;
                else pk[p][j >> 1] = hb;
            }
        }
#pragma unroll
        for (int p = 0; p < S; ++p) *reinterpret_cast<uint2*>(orow + p * plane + k0) = make_uint2(pk[p][0], pk[p][1]);
    }
}

// The S BF16 slices (bits) of x in a row with |x| < 2^ea: the fixed-point
// value X = rint(x 2^(F - ea)) (halves away from zero), F = 7 + 8 (S - 1),
// as S signed base-256 digits, each exact in BF16.  The arithmetic of
// k_slice and k_slice_contig, element for element.
template <int S>
__device__ __forceinline__ void slice_bits(double x, int ea, uint16_t (&h)[S]) {
    constexpr int F = 7 + 8 * (S - 1);
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    long long X = 0;
    if (ex) {
        const int shift = 52 + 1023 + ea - ex - F;     // >= 53 - F > 0
        if (shift < 63) {
            const unsigned long long m53 = (b & ((1ull << 52) - 1)) | (1ull << 52);
            X = (long long)((m53 + (1ull << (shift - 1))) >> shift);
            if (b >> 63) X = -X;
        }
    }
    int d[S];
#pragma unroll
    for (int p = S - 1; p >= 1; --p) {
        const int lo = (int)(((X + 128) & 255) - 128);
        d[p] = lo;
        X = (X - lo) >> 8;
    }
    d[0] = (int)X;
#pragma unroll
    for (int p = 0; p < S; ++p) {
        const float f = (__int_as_float(0x4B400000 + d[p]) - 12582912.0f) * __int_as_float((127 - 8 * p) << 23);
        h[p] = (uint16_t)(__float_as_uint(f) >> 16);
    }
}

// Exponents and slices of a few rows in one launch (the n x m blocks the
// isometry multiplies by M: m rows of n as a B operand): a CTA per row r < Rp
// takes the largest exponent field of its row (e_row[r] = field - 1022,
// -1022 for a zero row, as row_exponents gives it), then writes the row's
// slices, reading the row a second time through L1 / L2.  Bit-identical to
// row_exponents followed by k_slice.
template <int S>
__global__ void __launch_bounds__(256) k_slice_rows(const double* __restrict__ src, const int64_t* __restrict__ off_r,
                                                    const int64_t* __restrict__ off_c, int R, int K, int Rp, int Kp,
                                                    int* __restrict__ e_row, uint16_t* __restrict__ out) {
    __shared__ int wmax[8];
    const int r = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool real = r < R;
    const double* row = real ? src + off_r[r] : src;
    unsigned ef = 0;
    if (real)
        for (int k = threadIdx.x; k < K; k += 256)
            ef = max(ef, (unsigned)(((unsigned long long)__double_as_longlong(row[off_c[k]]) >> 52) & 0x7FF));
    ef = __reduce_max_sync(0xffffffffu, ef);
    if (lane == 0) wmax[warp] = (int)ef;
    __syncthreads();
    int mx = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) mx = max(mx, wmax[w]);
    const int ea = mx ? mx - 1022 : -1022;
    if (real && threadIdx.x == 0) e_row[r] = ea;
    const size_t plane = (size_t)Rp * Kp;
    for (int k = threadIdx.x; k < Kp; k += 256) {
        uint16_t h[S];
        slice_bits<S>((real && k < K) ? row[off_c[k]] : 0.0, ea, h);
#pragma unroll
        for (int p = 0; p < S; ++p) out[p * plane + (size_t)r * Kp + k] = h[p];
    }
}

// ------------------------------------------------------------- host side ---
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    static int err = 0;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            err = 1;
        else
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    if (err || !fn) fail(TRG_ENOTSUP, "cuTensorMapEncodeTiled not available");
    return fn;
}

CUtensorMap make_map(const void* base, int rows, int kp, int box_rows = BM) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(TRG_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return m;
}

// Column blocks per tile group.  The CTAs of a wave walk K in near lockstep,
// so a row block of A is read once by the group_n CTAs that share it and
// then streams on; the column blocks of B are re-read by every wave of the
// group and stay in L2 only if group_n of them fit.  Pick the group width
// with the fewest operand bytes read from DRAM under that model.
// tile_coords on the host (the symmetric products' tile lists)
static void tile_coords_host(int tile, int tiles_m, int tiles_n, int group_n, int& mb, int& nb) {
    const int per_group = tiles_m * group_n;
    const int group = tile / per_group;
    const int first_n = group * group_n;
    const int width = std::min(group_n, tiles_n - first_n);
    const int local = tile - group * per_group;
    mb = local / width;
    nb = first_n + local % width;
}

int choose_group_n(int tiles_m, int tiles_n, int grid, int kp, int S) {
    const double block = (double)BM * kp * S * 2;            // bytes of one 128-row slice block
    const double budget = 80.0 * (1 << 20);
    int best = tiles_n;
    double best_cost = 1e300;
    int prev = -1;
    for (int parts = 1; parts <= tiles_n; ++parts) {
        const int g = (tiles_n + parts - 1) / parts;
        if (g == prev) continue;
        prev = g;
        const int groups = (tiles_n + g - 1) / g;
        const double waves_per_group = std::ceil((double)tiles_m * g / grid);
        const double b_reads = (g * block <= budget) ? 1.0 : waves_per_group;
        const double cost = groups * tiles_m * block + b_reads * tiles_n * block;
        if (cost < best_cost) { best_cost = cost; best = g; }
    }
    return std::max(1, best);
}

template <int S, int CG, int MODE>
void launch_mma_k(Ctx& ctx, const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tbh,
                  const MmaArgs& a0) {
    MmaArgs a = a0;
    static std::once_flag once;
    static int max_clusters = 0;
    std::call_once(once, [&ctx] {
        TRG_CUDA(cudaFuncSetAttribute(k_split_mma<S, CG, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      smem_bytes_for(S, CG, MODE)));
        if (CG == 2) {
            // pairs that can be resident at once (a persistent grid must not exceed it)
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3((unsigned)(ctx.sm_count & ~1));
            cfg.blockDim = dim3(THREADS);
            cfg.dynamicSmemBytes = smem_bytes_for(S, CG, MODE);
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            TRG_CUDA(cudaOccupancyMaxActiveClusters(&max_clusters, k_split_mma<S, CG, MODE>, &cfg));
        }
    });
    const int tiles_m = (a.M + BM * CG - 1) / (BM * CG), tiles_n = (a.N + BN - 1) / BN;
    const int tiles = (a.tile_list ? a.n_list : tiles_m * tiles_n) * a.ksplit;   // units of work
    const int ctas = CG == 1 ? std::max(1, std::min(tiles, ctx.sm_count)) : 2 * std::max(1, std::min(tiles, max_clusters));
    if (a.group_n <= 0) a.group_n = choose_group_n(tiles_m * CG, tiles_n, ctas, a.Kp, S);
    cudaError_t e;
    if (CG == 1) {
        const int grid = ctas;
        k_split_mma<S, CG, MODE><<<grid, THREADS, smem_bytes_for(S, CG, MODE), ctx.stream>>>(ta, tb, tbh, a);
        e = cudaGetLastError();
    } else {
        if (max_clusters < 1) fail(TRG_ENOTSUP, "split MMA: no CTA pair fits on this device");
        const int pairs = std::max(1, std::min(tiles, max_clusters));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(2 * pairs));
        cfg.blockDim = dim3(THREADS);
        cfg.dynamicSmemBytes = smem_bytes_for(S, CG, MODE);
        cfg.stream = ctx.stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_split_mma<S, CG, MODE>, ta, tb, tbh, a);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    ctx.launches++;
    if (e != cudaSuccess) {
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, k_split_mma<S, CG, MODE>);
        fail(TRG_ECUDA, std::string("split MMA launch: ") + cudaGetErrorString(e) + " (regs " +
                            std::to_string(fa.numRegs) + ", max threads " + std::to_string(fa.maxThreadsPerBlock) +
                            ", dyn smem " + std::to_string(smem_bytes_for(S, CG, MODE)) + " / " +
                            std::to_string(fa.maxDynamicSharedSizeBytes) + ", local " +
                            std::to_string(fa.localSizeBytes) + ")");
    }
}

template <int S, int CG>
void launch_mma(Ctx& ctx, const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tbh, const MmaArgs& a) {
    if (a.cs_out) launch_mma_k<S, CG, EPI_FUSED>(ctx, ta, tb, tbh, a);
    else if (a.c_rows_fast) launch_mma_k<S, CG, EPI_DIRECT>(ctx, ta, tb, tbh, a);
    else if (a.ksplit > 1) launch_mma_k<S, CG, EPI_KSPLIT>(ctx, ta, tb, tbh, a);
    else launch_mma_k<S, CG, EPI_STAGED>(ctx, ta, tb, tbh, a);
}

template <int S>
void launch_slice(Ctx& ctx, const Gather& g, int R, int K, int Rp, int Kp, const int* e, uint16_t* out) {
    if (g.c_identity) {
        k_slice_contig<S><<<(unsigned)((Rp + 7) / 8), 256, 0, ctx.stream>>>(g.base, g.off_r, R, K, Rp, Kp, e, out);
        TRG_LAUNCHED(ctx);
        return;
    }
    dim3 grid((unsigned)((Kp + SL_K - 1) / SL_K), (unsigned)std::min<int64_t>((Rp + SL_R - 1) / SL_R, 65535));
    k_slice<S><<<grid, 256, 0, ctx.stream>>>(g.base, g.off_r, g.off_c, R, K, Rp, Kp, g.c_fast ? 1 : 0, e, out);
    TRG_LAUNCHED(ctx);
}

void row_exponents(Ctx& ctx, const Gather& g, int R, int K, int* e);

// Exponents and slices of an operand (rows r < R of length K, padded to Rp x
// Kp): one launch for at most SLICE_ROWS_MAX rows, else the two passes.
constexpr int SLICE_ROWS_MAX = 256;
template <int S>
void exponents_and_slices(Ctx& ctx, const Gather& g, int R, int K, int Rp, int Kp, int* e, uint16_t* out) {
    if (Rp <= SLICE_ROWS_MAX) {
        k_slice_rows<S><<<(unsigned)Rp, 256, 0, ctx.stream>>>(g.base, g.off_r, g.off_c, R, K, Rp, Kp, e, out);
        TRG_LAUNCHED(ctx);
        return;
    }
    row_exponents(ctx, g, R, K, e);
    launch_slice<S>(ctx, g, R, K, Rp, Kp, e, out);
}

void row_exponents(Ctx& ctx, const Gather& g, int R, int K, int* e) {
    TRG_CUDA(cudaMemsetAsync(e, 0, (size_t)R * sizeof(int), ctx.stream));
    dim3 grid((unsigned)((K + SL_K - 1) / SL_K), (unsigned)std::min<int64_t>((R + SL_R - 1) / SL_R, 65535));
    k_row_exponent<<<grid, 256, 0, ctx.stream>>>(g.base, g.off_r, g.off_c, R, K, g.c_fast ? 1 : 0, e);
    TRG_LAUNCHED(ctx);
    k_exponent_finish<<<(unsigned)((R + 255) / 256), 256, 0, ctx.stream>>>(e, R);
    TRG_LAUNCHED(ctx);
}

}  // namespace

// B operand as (n, k): swap the roles of its two tables.
static Gather transpose_gather(const Gather& b, const int64_t* off_k, const int64_t* off_n) {
    Gather t = b;
    t.off_r = off_n;
    t.off_c = off_k;
    t.c_fast = false;
    t.c_identity = false;
    return t;
}

// Exponents and BF16 slices of an A operand in the layout a split product
// reads (rows padded per split_rows_padded, K per split_k_padded), for a
// caller that reuses one A across several products.
void split_slice_operand(Ctx& ctx, const Gather& A, int64_t M, int64_t K, uint16_t* slices, int* e) {
    const int S = slices_now(ctx);
    const int Mi = (int)M, Ki = (int)std::max<int64_t>(K, 1);
    const int Mp = (int)split_rows_padded(ctx, M), Kp = (int)split_k_padded(K);
    row_exponents(ctx, A, Mi, Ki, e);
    switch (S) {
        case 2: launch_slice<2>(ctx, A, Mi, Ki, Mp, Kp, e, slices); break;
        case 3: launch_slice<3>(ctx, A, Mi, Ki, Mp, Kp, e, slices); break;
        case 4: launch_slice<4>(ctx, A, Mi, Ki, Mp, Kp, e, slices); break;
        case 5: launch_slice<5>(ctx, A, Mi, Ki, Mp, Kp, e, slices); break;
        default: fail(TRG_EINVAL, "split_slices must be 2..5");
    }
}

// Exponents and BF16 slices of a B operand (K x N) as a split product reads
// it: rows n of B^T, padded to the 128-column tile.
void split_slice_b(Ctx& ctx, const Gather& B, int64_t K, int64_t N, uint16_t* slices, int* e) {
    const int S = slices_now(ctx);
    const int Ni = (int)N, Ki = (int)std::max<int64_t>(K, 1);
    const int Np = (int)split_cols_padded(N), Kp = (int)split_k_padded(K);
    const Gather bt = transpose_gather(B, B.off_r, B.off_c);
    row_exponents(ctx, bt, Ni, Ki, e);
    switch (S) {
        case 2: launch_slice<2>(ctx, bt, Ni, Ki, Np, Kp, e, slices); break;
        case 3: launch_slice<3>(ctx, bt, Ni, Ki, Np, Kp, e, slices); break;
        case 4: launch_slice<4>(ctx, bt, Ni, Ki, Np, Kp, e, slices); break;
        case 5: launch_slice<5>(ctx, bt, Ni, Ki, Np, Kp, e, slices); break;
        default: fail(TRG_EINVAL, "split_slices must be 2..5");
    }
}
int64_t split_cols_padded(int64_t N) { return (N + BN - 1) / BN * BN; }

int64_t split_rows_padded(const Ctx& ctx, int64_t M) {
    const int64_t tile = (ctx.cfg.mma_pairs && M > BM) ? 2 * BM : BM;
    return (M + tile - 1) / tile * tile;
}
int64_t split_k_padded(int64_t K) { return (std::max<int64_t>(K, 1) + BK - 1) / BK * BK; }

// Measured launch choice of a split product (the tile autotuner): one CTA or
// a CTA pair per tile, and the width of the tile groups (tile_coords).  Every
// choice gives identical bits (the pair issues the same product table, and
// the tile order changes no sum), so the choice is a pure speed decision and
// results never depend on it.  On the first product of a shape (M, N, K, S,
// epilogue kind) worth tuning, each candidate is launched twice and timed
// with events on the context's stream; the fastest is kept in a table shared
// by every context of the process.  Smaller products, and contexts with
// autotune off, take the model choice (pairs as configured, choose_group_n).
struct TuneChoice { int cg, group_n; };
struct TuneKey {
    int M, N, Kp, S, mode, cg_max;
    bool operator<(const TuneKey& o) const {
        return std::tie(M, N, Kp, S, mode, cg_max) < std::tie(o.M, o.N, o.Kp, o.S, o.mode, o.cg_max);
    }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneChoice> g_tune;
constexpr double TUNE_MIN_MACS = 1.0 * (1 << 30);   // products below ~1 G multiply-adds keep the model choice

template <class Launch>
static TuneChoice tuned_choice(Ctx& ctx, int M, int N, int Kp, int S, int mode, int cg_max, Launch&& launch) {
    const int tiles_n = (N + BN - 1) / BN;
    auto model_group = [&](int cg) {
        const int tiles_m = (M + BM * cg - 1) / (BM * cg);
        const int ctas = std::max(1, std::min(tiles_m * tiles_n * cg, ctx.sm_count & ~(cg - 1)));
        return choose_group_n(tiles_m * cg, tiles_n, ctas, Kp, S);
    };
    const TuneChoice model{cg_max, model_group(cg_max)};
    if (!ctx.cfg.autotune || (double)M * N * Kp < TUNE_MIN_MACS) return model;
    const TuneKey key{M, N, Kp, S, mode, cg_max};
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    std::vector<TuneChoice> cand;
    for (int cg = cg_max; cg >= 1; --cg) {
        const int g = model_group(cg);
        for (int gn : {g, std::max(1, g / 2), std::min(tiles_n, 2 * g)}) {
            bool seen = false;
            for (auto& c : cand) seen = seen || (c.cg == cg && c.group_n == gn);
            if (!seen) cand.push_back({cg, gn});
        }
    }
    cudaEvent_t e0 = ctx.get_event(), e1 = ctx.get_event();
    TuneChoice best = model;
    float best_ms = 1e30f;
    for (const TuneChoice& c : cand) {
        launch(c.cg, c.group_n);     // warm (the output is the same every time)
        TRG_CUDA(cudaEventRecord(e0, ctx.stream));
        launch(c.cg, c.group_n);
        TRG_CUDA(cudaEventRecord(e1, ctx.stream));
        TRG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TRG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) { best_ms = ms; best = c; }
    }
    ctx.event_pool.push_back(e0);
    ctx.event_pool.push_back(e1);
    ctx.counters[6] += 1;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.emplace(key, best);
    return g_tune[key];
}

void gemm_split(Ctx& ctx, const GemmDesc& d) {
    if (d.M <= 0 || d.N <= 0) return;
    if (d.beta != 0.0) fail(TRG_EINVAL, "split GEMM overwrites its output (beta must be 0)");
    if (d.M > (1ll << 30) || d.N > (1ll << 30) || d.K > (1 << 17)) fail(TRG_EINVAL, "split GEMM: size out of range");
    const int S = slices_now(ctx);
    const int M = (int)d.M, N = (int)d.N, K = (int)std::max<int64_t>(d.K, 1);
    // CTA pairs (256-row tiles) once A has more than one 128-row block
    const int CG = (ctx.cfg.mma_pairs && M > BM) ? 2 : 1;
    const int Mp = (int)split_rows_padded(ctx, M), Np = (N + BN - 1) / BN * BN, Kp = (int)split_k_padded(K);
    const bool pre_a = d.a_slices != nullptr;    // A arrives sliced from its producer
    if (d.gram && (M != N || d.b_slices || pre_a || d.cs_out || d.cons_ef || d.c_rows_fast))
        fail(TRG_EINVAL, "split GEMM: a Gram product takes a square C and plain operands");
    // a Gram product reads A's slices for B too (same rows, same padding)
    const bool gram_b = d.gram && Mp == Np;
    const bool pre_b = d.b_slices != nullptr || gram_b;   // B arrives sliced (shared by several products)

    // scratch: exponents + slices of A and B (unless given)
    const size_t bytes_e = (size_t)(Mp + Np) * sizeof(int);
    const size_t bytes_a = pre_a ? 0 : (size_t)S * Mp * Kp * 2, bytes_b = pre_b ? 0 : (size_t)S * Np * Kp * 2;
    ctx.ensure(ctx.split_ws, bytes_e + bytes_a + bytes_b + 1024);
    uint8_t* base = ctx.split_ws.as<uint8_t>();
    int* ea = pre_a ? const_cast<int*>(d.a_e) : (int*)base;
    int* eb = gram_b ? ea : pre_b ? const_cast<int*>(d.b_e) : (int*)base + Mp;
    uint16_t* sa = pre_a ? const_cast<uint16_t*>(d.a_slices) : (uint16_t*)(base + ((bytes_e + 255) & ~(size_t)255));
    uint16_t* sb = gram_b ? sa
                 : pre_b ? const_cast<uint16_t*>(d.b_slices)
                         : (uint16_t*)(base + ((bytes_e + 255) & ~(size_t)255)) + (pre_a ? 0 : (size_t)S * Mp * Kp);

    // B as rows n, columns k: element (n, k) at B[b_k[k] + b_n[n]]
    const Gather bt = transpose_gather(d.B, d.B.off_r, d.B.off_c);
    Gather bt2 = bt;
    bt2.c_fast = false;
    // contiguous along k in memory?  (the k-table of B is B.off_r)
    if (pre_a) {
        // slices and exponents of A were written by the producing product
    } else if (d.a_ef) {
        // the producing product already recorded A's exponent fields
        TRG_CUDA(cudaMemcpyAsync(ea, d.a_ef, (size_t)M * sizeof(int), cudaMemcpyDeviceToDevice, ctx.stream));
        k_exponent_finish<<<(unsigned)((M + 255) / 256), 256, 0, ctx.stream>>>(ea, M);
        TRG_LAUNCHED(ctx);
    } else {
        row_exponents(ctx, d.A, M, K, ea);
    }
    switch (S) {
        case 2: if (!pre_a) launch_slice<2>(ctx, d.A, M, K, Mp, Kp, ea, sa);
                if (!pre_b) exponents_and_slices<2>(ctx, bt2, N, K, Np, Kp, eb, sb); break;
        case 3: if (!pre_a) launch_slice<3>(ctx, d.A, M, K, Mp, Kp, ea, sa);
                if (!pre_b) exponents_and_slices<3>(ctx, bt2, N, K, Np, Kp, eb, sb); break;
        case 4: if (!pre_a) launch_slice<4>(ctx, d.A, M, K, Mp, Kp, ea, sa);
                if (!pre_b) exponents_and_slices<4>(ctx, bt2, N, K, Np, Kp, eb, sb); break;
        case 5: if (!pre_a) launch_slice<5>(ctx, d.A, M, K, Mp, Kp, ea, sa);
                if (!pre_b) exponents_and_slices<5>(ctx, bt2, N, K, Np, Kp, eb, sb); break;
        default: fail(TRG_EINVAL, "split_slices must be 2..5");
    }
    const CUtensorMap ta = make_map(sa, S * Mp, Kp);
    const CUtensorMap tb = make_map(sb, S * Np, Kp);
    // a pair also reads B as 64-row half tiles (its narrow products)
    const CUtensorMap tbh = CG == 2 ? make_map(sb, S * Np, Kp, BN / 2) : tb;
    MmaArgs a;
    a.M = M; a.N = N; a.Kp = Kp; a.Mp = Mp; a.Np = Np; a.S = S;
    a.ea = ea; a.eb = eb; a.C = d.C; a.c_m = d.c_m; a.c_n = d.c_n;
    a.status = ctx.status.as<int>();
    a.acc_wait_ns = ctx.acc_wait_ns ? ctx.acc_wait_ns : WAIT_NS;
    a.cons_ef = d.cons_ef; a.cons_m = d.cons_m; a.cons_n = d.cons_n;
    a.cs_out = d.cs_out; a.cs_plane = d.cs_mp * d.cs_kp; a.cs_kp = d.cs_kp; a.cs_e = d.cs_e;
    a.ck_m = d.ck_m; a.ck_n = d.ck_n; a.rows_per_crow = d.rows_per_crow; a.cols_per_crow = d.cols_per_crow;
    a.ck_stride = d.ck_stride; a.c_rows_fast = d.c_rows_fast ? 1 : 0; a.c_col_stride = d.c_col_stride;
    // |V| <= (K / 512) (2^32 + 2^24) 2^14 + 2 K 2^20 < 2^53 for K <= 8192
    a.v_exact53 = Kp <= 8192 ? 1 : 0;
    // split K where the tiles leave most SMs idle: a function of the shape
    // and the SM count only (not of the CTA grouping), so every launch
    // choice still gives the same bits
    a.ksplit = 1; a.kb_per = Kp / BK; a.kpart = nullptr;
    a.tile_list = nullptr; a.n_list = 0; a.sym = d.gram ? 1 : 0;
    if (d.allow_ksplit && !d.cs_out && !d.c_rows_fast && !d.cons_ef && !d.gram) {
        const int chunks = (Kp / BK + CHUNK_STAGES - 1) / CHUNK_STAGES;
        const int tiles128 = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
        if (2 * tiles128 <= ctx.sm_count && chunks >= 2) {
            const int want = std::min(chunks, ctx.sm_count / tiles128);
            const int per = (chunks + want - 1) / want;          // chunks per part
            a.kb_per = per * CHUNK_STAGES;
            a.ksplit = (chunks + per - 1) / per;
            if (a.ksplit > 1) {
                ctx.ensure(ctx.ksplit_ws, (size_t)a.ksplit * N * M * sizeof(long long));
                a.kpart = ctx.ksplit_ws.as<long long>();
            } else {
                a.kb_per = Kp / BK;
            }
        }
    }
    if (d.cs_out) {
        // a consumer row = rows_per_crow consecutive rows (32, 64 or 128, so a
        // warp's lanes and the CTA's 128-row tile hold whole groups) times
        // cols_per_crow consecutive columns (so a thread's 32 hold one group)
        auto pow2_32_128 = [](int v) { return v == 32 || v == 64 || v == 128; };
        const bool shape_ok = pow2_32_128(d.rows_per_crow) && pow2_32_128(d.cols_per_crow) &&
                              M % d.rows_per_crow == 0 && N % d.cols_per_crow == 0 && d.cs_kp % 8 == 0 &&
                              d.cons_m && d.cons_n && d.ck_m && d.ck_n && d.cs_e;
        if (!shape_ok) fail(TRG_EINVAL, "fused slice hand-over: consumer rows do not tile");
    }
    auto launch = [&](int cg, int group_n) {
        MmaArgs b = a;
        b.group_n = group_n;
        if (d.gram) {
            // the tiles that reach the diagonal or above, in tile_coords order
            const int tile_m = BM * cg, tiles_m = (M + tile_m - 1) / tile_m, tiles_n = (N + BN - 1) / BN;
            const int gn = group_n > 0 ? group_n : tiles_n;
            b.group_n = gn;
            const std::string key = "sym:" + std::to_string(tiles_m) + ":" + std::to_string(tiles_n) + ":" +
                                    std::to_string(gn) + ":" + std::to_string(tile_m);
            auto it = ctx.tables.find(key);
            if (it == ctx.tables.end()) {
                std::vector<long long> h;
                for (int t = 0; t < tiles_m * tiles_n; ++t) {
                    int mb, nb;
                    tile_coords_host(t, tiles_m, tiles_n, gn, mb, nb);
                    if ((int64_t)nb * BN + BN - 1 >= (int64_t)mb * tile_m) h.push_back(((long long)mb << 32) | nb);
                }
                Buf buf;
                ctx.ensure(buf, h.size() * sizeof(long long));
                TRG_CUDA(cudaMemcpyAsync(buf.p, h.data(), h.size() * sizeof(long long), cudaMemcpyHostToDevice,
                                         ctx.stream));
                TRG_CUDA(cudaStreamSynchronize(ctx.stream));   // h dies here
                it = ctx.tables.emplace(key, buf).first;
                ctx.list_len[key] = (int)h.size();
            }
            b.tile_list = it->second.as<long long>();
            b.n_list = ctx.list_len[key];
        }
        switch (S * 2 + cg - 1) {
            case 4: launch_mma<2, 1>(ctx, ta, tb, tbh, b); break;
            case 5: launch_mma<2, 2>(ctx, ta, tb, tbh, b); break;
            case 6: launch_mma<3, 1>(ctx, ta, tb, tbh, b); break;
            case 7: launch_mma<3, 2>(ctx, ta, tb, tbh, b); break;
            case 8: launch_mma<4, 1>(ctx, ta, tb, tbh, b); break;
            case 9: launch_mma<4, 2>(ctx, ta, tb, tbh, b); break;
            case 10: launch_mma<5, 1>(ctx, ta, tb, tbh, b); break;
            case 11: launch_mma<5, 2>(ctx, ta, tb, tbh, b); break;
        }
    };
    const int mode = d.cs_out ? 2 : (d.c_rows_fast ? 1 : (a.ksplit > 1 ? 3 : (d.gram ? 4 : 0)));
    const TuneChoice ch = tuned_choice(ctx, M, N, Kp, S, mode, CG, launch);
    const int tok = ctx.region_begin(TRG_PHASE_MMA);
    const int tok_x2 = ctx.phase == TRG_PHASE_X2 ? ctx.region_begin(TRG_PHASE_MMA_X2) : -1;
    launch(ch.cg, ch.group_n);
    if (a.ksplit > 1) {
        const int64_t tot = (int64_t)M * N;
        k_ksplit_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, ctx.stream>>>(a.kpart, a.ksplit, M, N, ea, eb, d.C,
                                                                             d.c_m, d.c_n);
        TRG_LAUNCHED(ctx);
    }
    const double products = (double)S * (S + 1) / 2;
    ctx.region_end(tok_x2, 2.0 * (double)M * N * K, products * 2.0 * (double)M * N * Kp);
    ctx.region_end(tok, 2.0 * (double)M * N * K, products * 2.0 * (double)M * N * Kp);
}

// ----------------------------------------------------------------------------
// Allocation-free variant of the split GEMM (trg_gemm_noalloc).
//
// For callers that must not allocate device memory while they run: code that
// has already handed all device memory to its own pool (a serving process
// that sized its arena at start-up), code running where a cudaMalloc would
// synchronise the device or is not permitted, and code that cannot own a
// context object.  Its scratch -- offset tables, scale exponents, BF16 slices
// and the status word -- lives in one file-scope device array of fixed size,
// which every GPU that loads the library holds until the process exits.
// ----------------------------------------------------------------------------
namespace {

constexpr size_t NOALLOC_BYTES = (size_t)64 << 20;   // 64 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// The array's name is a host-side stand-in in host code; the device address
// comes from cudaGetSymbolAddress, once per device, with that device current.
constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[MAX_DEVICES] = {};
int g_noalloc_sms[MAX_DEVICES] = {};

__global__ void k_affine_table(int64_t* t, int64_t n, int64_t stride) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) t[i] = i * stride;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

}  // namespace trg

extern "C" int trg_gemm_noalloc(int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                                double* C, int ldc, int slices, void* stream_ptr) {
    using namespace trg;
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < N || ldc < N) return TRG_EINVAL;
    if (slices < 2 || slices > 5 || K > (1 << 17)) return TRG_EINVAL;
    // the padded sizes below are ints: bound M and N first (as trg_gemm does)
    if (M > (1 << 30) || N > (1 << 30)) return TRG_EINVAL;
    const int S = slices;
    const int Mp = (M + BM - 1) / BM * BM, Np = (N + BN - 1) / BN * BN, Kp = (K + BK - 1) / BK * BK;
    // layout of the scratch array
    const size_t o_am = 0;
    const size_t o_ak = o_am + round256((size_t)M * 8);
    const size_t o_bk = o_ak + round256((size_t)K * 8);
    const size_t o_bn = o_bk + round256((size_t)K * 8);
    const size_t o_cm = o_bn + round256((size_t)N * 8);
    const size_t o_cn = o_cm + round256((size_t)M * 8);
    const size_t o_st = o_cn + round256((size_t)N * 8);
    const size_t o_ea = o_st + 256;
    const size_t o_eb = o_ea + round256((size_t)Mp * 4);
    const size_t o_sa = o_eb + round256((size_t)Np * 4);
    const size_t o_sb = o_sa + round256((size_t)S * Mp * Kp * 2);
    const size_t total = o_sb + round256((size_t)S * Np * Kp * 2);
    if (total > NOALLOC_BYTES) return TRG_EINVAL;   // beyond the fixed scratch: use trg_gemm

    cudaStream_t stream = (cudaStream_t)stream_ptr;
    try {
        int dev = 0;
        TRG_CUDA(cudaGetDevice(&dev));
        if (dev < 0 || dev >= MAX_DEVICES) return TRG_ENOTSUP;
        unsigned char* base;
        int sms;
        {
            std::lock_guard<std::mutex> lock(g_noalloc_mu);
            if (!g_noalloc_ptr[dev]) {
                cudaDeviceProp prop;
                TRG_CUDA(cudaGetDeviceProperties(&prop, dev));
                if (prop.major != 10 || prop.minor != 3) return TRG_ENOTSUP;
                void* p = nullptr;
                const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
                if (e != cudaSuccess || !p) return TRG_ECUDA;
                g_noalloc_sms[dev] = prop.multiProcessorCount;
                g_noalloc_ptr[dev] = p;
            }
            base = (unsigned char*)g_noalloc_ptr[dev];
            sms = g_noalloc_sms[dev];
        }
        int64_t* am = (int64_t*)(base + o_am);
        int64_t* ak = (int64_t*)(base + o_ak);
        int64_t* bk = (int64_t*)(base + o_bk);
        int64_t* bn = (int64_t*)(base + o_bn);
        int64_t* cm = (int64_t*)(base + o_cm);
        int64_t* cn = (int64_t*)(base + o_cn);
        int* status = (int*)(base + o_st);
        int* ea = (int*)(base + o_ea);
        int* eb = (int*)(base + o_eb);
        uint16_t* sa = (uint16_t*)(base + o_sa);
        uint16_t* sb = (uint16_t*)(base + o_sb);

        // the array keeps the previous call's contents: rebuild the tables,
        // clear the status word and the exponents (maxima start from zero)
        const struct { int64_t* t; int64_t n, s; } tabs[6] = {
            {am, M, lda}, {ak, K, 1}, {bk, K, ldb}, {bn, N, 1}, {cm, M, ldc}, {cn, N, 1}};
        for (const auto& tb : tabs) {
            k_affine_table<<<(unsigned)((tb.n + 255) / 256), 256, 0, stream>>>(tb.t, tb.n, tb.s);
            TRG_CUDA(cudaGetLastError());
        }
        TRG_CUDA(cudaMemsetAsync(status, 0, sizeof(int), stream));
        TRG_CUDA(cudaMemsetAsync(ea, 0, (size_t)M * sizeof(int), stream));
        TRG_CUDA(cudaMemsetAsync(eb, 0, (size_t)N * sizeof(int), stream));

        // row exponents and slices of A (rows m, k contiguous) and of B as (n, k)
        {
            dim3 ga((unsigned)((K + SL_K - 1) / SL_K), (unsigned)std::min<int64_t>((M + SL_R - 1) / SL_R, 65535));
            k_row_exponent<<<ga, 256, 0, stream>>>(A, am, ak, M, K, 1, ea);
            dim3 gb((unsigned)((K + SL_K - 1) / SL_K), (unsigned)std::min<int64_t>((N + SL_R - 1) / SL_R, 65535));
            k_row_exponent<<<gb, 256, 0, stream>>>(B, bn, bk, N, K, 0, eb);
            k_exponent_finish<<<(unsigned)((M + 255) / 256), 256, 0, stream>>>(ea, M);
            k_exponent_finish<<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(eb, N);
            TRG_CUDA(cudaGetLastError());
            dim3 sa_grid((unsigned)((Kp + SL_K - 1) / SL_K), (unsigned)std::min<int64_t>(Mp / SL_R, 65535));
            dim3 sb_grid((unsigned)((Kp + SL_K - 1) / SL_K), (unsigned)std::min<int64_t>(Np / SL_R, 65535));
            switch (S) {
                case 2: k_slice<2><<<sa_grid, 256, 0, stream>>>(A, am, ak, M, K, Mp, Kp, 1, ea, sa);
                        k_slice<2><<<sb_grid, 256, 0, stream>>>(B, bn, bk, N, K, Np, Kp, 0, eb, sb); break;
                case 3: k_slice<3><<<sa_grid, 256, 0, stream>>>(A, am, ak, M, K, Mp, Kp, 1, ea, sa);
                        k_slice<3><<<sb_grid, 256, 0, stream>>>(B, bn, bk, N, K, Np, Kp, 0, eb, sb); break;
                case 4: k_slice<4><<<sa_grid, 256, 0, stream>>>(A, am, ak, M, K, Mp, Kp, 1, ea, sa);
                        k_slice<4><<<sb_grid, 256, 0, stream>>>(B, bn, bk, N, K, Np, Kp, 0, eb, sb); break;
                default: k_slice<5><<<sa_grid, 256, 0, stream>>>(A, am, ak, M, K, Mp, Kp, 1, ea, sa);
                         k_slice<5><<<sb_grid, 256, 0, stream>>>(B, bn, bk, N, K, Np, Kp, 0, eb, sb); break;
            }
            TRG_CUDA(cudaGetLastError());
        }
        const CUtensorMap ta = make_map(sa, S * Mp, Kp);
        const CUtensorMap tbm = make_map(sb, S * Np, Kp);
        MmaArgs a;
        a.M = M; a.N = N; a.Kp = Kp; a.Mp = Mp; a.Np = Np; a.S = S;
        a.ea = ea; a.eb = eb; a.C = C; a.c_m = cm; a.c_n = cn; a.status = status;
        a.cons_ef = nullptr; a.cons_m = nullptr; a.cons_n = nullptr;
        a.cs_out = nullptr; a.cs_plane = 0; a.cs_kp = 0; a.cs_e = nullptr; a.ck_m = nullptr; a.ck_n = nullptr;
        a.rows_per_crow = a.cols_per_crow = 0;
        a.ck_stride = 0; a.c_rows_fast = 0; a.c_col_stride = 0; a.v_exact53 = 0;
        a.acc_wait_ns = WAIT_NS;
        a.ksplit = 1; a.kb_per = Kp / BK; a.kpart = nullptr;
        a.tile_list = nullptr; a.n_list = 0; a.sym = 0;
        const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
        const int grid = std::max(1, std::min(tiles, sms));
        a.group_n = choose_group_n((M + BM - 1) / BM, (N + BN - 1) / BN, grid, Kp, S);
        switch (S) {
#define TRG_NOALLOC_MMA(SS)                                                                                  \
    TRG_CUDA(cudaFuncSetAttribute(k_split_mma<SS, 1, EPI_STAGED>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                  smem_bytes_for(SS, 1, EPI_STAGED)));                                                   \
    k_split_mma<SS, 1, EPI_STAGED><<<grid, THREADS, smem_bytes_for(SS, 1, EPI_STAGED), stream>>>(ta, tbm, tbm, a);                        \
    break;
            case 2: TRG_NOALLOC_MMA(2)
            case 3: TRG_NOALLOC_MMA(3)
            case 4: TRG_NOALLOC_MMA(4)
            default: TRG_NOALLOC_MMA(5)
#undef TRG_NOALLOC_MMA
        }
        TRG_CUDA(cudaGetLastError());
        int st = 0;
        TRG_CUDA(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, stream));
        TRG_CUDA(cudaStreamSynchronize(stream));
        if (st & ST_TIMEOUT) return TRG_ETIMEOUT;
        return TRG_OK;
    } catch (const Error& e) {
        return e.status;
    }
}
