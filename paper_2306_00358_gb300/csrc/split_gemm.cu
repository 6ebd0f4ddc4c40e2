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
// Products of BF16 values are exact in FP32, and with |d_0 e_0|, |d_0 e_1|,
// |d_1 e_0| <= 2^14 a run of 1024 of them sums exactly in an FP32
// accumulator (|sum| <= 2^24).  The tensor cores therefore accumulate
//   ACC0  = (0,0),  ACC01 = (0,1),  ACC10 = (1,0)   exactly over 1024-K chunks,
//   ACCR  = all (p,q) with 2 <= p+q < S             in FP32 over the whole K
// (ACCR carries weight <= 2^-16 relative to ACC0, so its FP32 rounding stays
// below the truncation error).  After every chunk the epilogue warps move
// ACC0 and ACC01 + ACC10 into int32 registers; at the end of a tile the sum
//   V = I0 2^22 + I1 2^14 + rint(ACCR 2^22)      (int64, exact)
// is turned into the FP64 result V 2^(ea + eb - 36) with integer operations,
// keeping the FP64 pipe (1/64 of the FP32 rate on this part) out of the loop.
//
// Kernel layout: persistent, one CTA per SM, 128 x 128 output tiles, BF16
// operand tiles of 128 x 32 staged by TMA (64-byte swizzle) through an
// mbarrier pipeline; warp 0 issues TMA, warp 1 owns TMEM and issues
// tcgen05.mma (one thread), warps 2..9 drain TMEM (two warps per 32-lane
// quadrant, 64 columns each).  Every wait is bounded: on expiry the kernel
// records ST_TIMEOUT and leaves its loops.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace trg {

namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 32;                        // K per stage: 64 bytes of BF16
constexpr int TILE_BYTES = BM * BK * 2;       // 8 KB per 128 x 32 BF16 tile
constexpr int CHUNK_STAGES = 1024 / BK;       // exact-accumulation run (1024 K)
constexpr int EPI_WARPS = 16;
constexpr int THREADS = 64 + 32 * EPI_WARPS;  // TMA warp + MMA warp + epilogue
constexpr uint32_t TMEM_COLS = 512;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bounded mbarrier waits: 2 s

__host__ __device__ constexpr int stages_for(int S) { return S <= 4 ? 3 : 2; }
constexpr int CPT = 32;                        // accumulator columns per epilogue thread
constexpr int STAGING_BYTES = EPI_WARPS * 32 * 8 * 8;    // epilogue store staging, 32 KB
__host__ __device__ constexpr int smem_bytes_for(int S) {
    // at least 120 KB so that a second CTA (and its 512 TMEM columns) never shares the SM
    return (stages_for(S) * 2 * S * TILE_BYTES + 1024 + 256 + STAGING_BYTES) > 120 * 1024
               ? stages_for(S) * 2 * S * TILE_BYTES + 1024 /*align*/ + 256 /*barriers*/ + STAGING_BYTES
               : 120 * 1024;
}

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
// Bounded wait; returns false (and flags the status word) on expiry or when
// another role of the CTA has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* status) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    unsigned n = 0;
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if ((++n & 255u) == 0 && global_ns() - t0 > WAIT_NS) {
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
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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
};

template <int S>
__global__ void __launch_bounds__(THREADS, 1)
k_split_mma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const MmaArgs g) {
    constexpr int STAGES = stages_for(S);
    constexpr int STAGE_BYTES = 2 * S * TILE_BYTES;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* mma_done = acc_empty + 1;
    uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    double* staging = (double*)(smem + STAGES * STAGE_BYTES + 256);   // EPI_WARPS x 32 x 8 doubles

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int tiles_m = (g.M + BM - 1) / BM;
    const int tiles_n = (g.N + BN - 1) / BN;
    const int num_tiles = tiles_m * tiles_n;
    const int num_kb = g.Kp / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, EPI_WARPS);
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued[STAGES];          // parity of the last load issued per stage, -1 = none
#pragma unroll
            for (int s = 0; s < STAGES; ++s) issued[s] = -1;
            bool ok = true;
            for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
                const int mb = tile / tiles_n, nb = tile % tiles_n;
                for (int kb = 0; kb < num_kb && ok; ++kb) {
                    ok = mbar_wait(&empty[stage], phase ^ 1, abort_flag, g.status);
                    if (!ok) break;
                    uint8_t* st = smem + stage * STAGE_BYTES;
                    mbar_expect_tx(&full[stage], STAGE_BYTES);
                    for (int p = 0; p < S; ++p) {
                        tma_load_2d(st + p * TILE_BYTES, &tmA, kb * BK, p * g.Mp + mb * BM, &full[stage]);
                        tma_load_2d(st + (S + p) * TILE_BYTES, &tmB, kb * BK, p * g.Np + nb * BN, &full[stage]);
                    }
#pragma unroll
                    for (int s = 0; s < STAGES; ++s)
                        if (s == stage) issued[s] = (int)phase;
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
            }
            // every load this thread issued has landed before the CTA may exit
            // (bounded, and done even after an abort)
            volatile int never = 0;
#pragma unroll
            for (int s = 0; s < STAGES; ++s)
                if (issued[s] >= 0) mbar_wait(&full[s], (uint32_t)issued[s], &never, g.status);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16(BM, BN);
            const uint32_t acc0 = tmem, acc01 = tmem + 128, acc10 = tmem + 256, accr = tmem + 384;
            int stage = 0;
            uint32_t phase = 0;
            uint32_t chunk_no = 0;      // chunks issued so far (all tiles)
            bool ok = true;
            for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
                bool accr_started = false;
                for (int kb = 0; kb < num_kb && ok; ++kb) {
                    const bool chunk_start = (kb % CHUNK_STAGES) == 0;
                    if (chunk_start && chunk_no > 0) {
                        // the epilogue must have drained the previous chunk
                        ok = mbar_wait(acc_empty, (chunk_no - 1) & 1, abort_flag, g.status);
                        if (!ok) break;
                        tc_fence_after();
                    }
                    ok = mbar_wait(&full[stage], phase, abort_flag, g.status);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const bool first_in_chunk = chunk_start && kk == 0;
#pragma unroll
                        for (int p = 0; p < S; ++p) {
#pragma unroll
                            for (int q = 0; q + p < S; ++q) {
                                const uint64_t da = smem_desc(base + p * TILE_BYTES + kk * 32);
                                const uint64_t db = smem_desc(base + (S + q) * TILE_BYTES + kk * 32);
                                uint32_t d;
                                uint32_t accum;
                                if (p + q == 0) { d = acc0; accum = first_in_chunk ? 0u : 1u; }
                                else if (p == 0 && q == 1) { d = acc01; accum = first_in_chunk ? 0u : 1u; }
                                else if (p == 1 && q == 0) { d = acc10; accum = first_in_chunk ? 0u : 1u; }
                                else { d = accr; accum = accr_started ? 1u : 0u; accr_started = true; }
                                mma_bf16(d, da, db, IDESC, accum);
                            }
                        }
                    }
                    mma_commit(&empty[stage]);
                    const bool chunk_end = ((kb + 1) % CHUNK_STAGES) == 0 || kb + 1 == num_kb;
                    if (chunk_end) {
                        mma_commit(acc_full);
                        ++chunk_no;
                    }
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
            }
            // every MMA issued has completed (also after an abort) ...
            mma_commit(mma_done);
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
        const int nchunks = (num_kb + CHUNK_STAGES - 1) / CHUNK_STAGES;
        uint32_t chunk_no = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
            const int mb = tile / tiles_n, nb = tile % tiles_n;
            // J = I0 2^8 + I1: the exact ACC0 and ACC01 + ACC10 sums of this
            // tile's columns in one int64 each; at the end J becomes
            // V = J 2^14 + rint(ACCR 2^22) and then, in place, the FP64 bits
            long long J[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) J[j] = 0;
            for (int c = 0; c < nchunks && ok; ++c) {
                // one lane waits, the warp follows (the TMEM loads are warp-collective)
                int w_ok = 1;
                if (lane == 0) w_ok = mbar_wait(acc_full, chunk_no & 1, abort_flag, g.status) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
                if (!ok) break;
                tc_fence_after();
                const bool last = (c == nchunks - 1);
                const int m = mb * BM + row_in_tile;
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
                    tmem_ld8(tmem + lane_base + 256 + col, r);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; ++j) J[h * 8 + j] += __float2int_rn(__uint_as_float(r[j]) * 256.0f);
                    if (last) {
                        // fold in ACCR and form these columns' FP64 results in place
                        if (S >= 3) {
                            tmem_ld8(tmem + lane_base + 384 + col, r);
                            tmem_wait_ld();
                        } else {
                            // two slices: no product lands in ACCR, whose columns are never written
#pragma unroll
                            for (int j = 0; j < 8; ++j) r[j] = 0u;
                        }
                        const int n0 = nb * BN + (int)col;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int n = n0 + j;
                            double v = 0.0;
                            if (row_ok && n < g.N) {
                                const long long iv = (J[h * 8 + j] << 14) +
                                                     __float2ll_rn(__uint_as_float(r[j]) * 4194304.0f);
                                v = scaled_i64_to_double(iv, ea + g.eb[n] - 36);
                            }
                            J[h * 8 + j] = __double_as_longlong(v);
                        }
                    }
                }
                if (last && g.cons_ef && row_ok) {
                    // exponent fields of the consumer's rows: run-length maxima
                    // over this thread's columns, one atomic per run
                    const int64_t cm0 = g.cons_m[m];
                    int64_t cur = -1;
                    int cur_max = 0;
#pragma unroll
                    for (int j = 0; j < CPT; ++j) {
                        const int n = nb * BN + colh * CPT + j;
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
                // TMEM is free for the next tile before the stores go out
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
                ++chunk_no;
                if (last) {
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
                            const int mr = mb * BM + quad * 32 + rr;
                            if (mr < g.M && n < g.N) g.C[g.c_m[mr] + cn] = stg[rr * 8 + (cl ^ ((rr >> 1) & 7))];
                        }
                        __syncwarp();
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
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
    const int r0 = blockIdx.y * SL_R, k0 = blockIdx.x * SL_K;
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
    const int r0 = blockIdx.y * SL_R, k0 = blockIdx.x * SL_K;
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

CUtensorMap make_map(const void* base, int rows, int kp) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(TRG_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return m;
}

template <int S>
void launch_mma(Ctx& ctx, const CUtensorMap& ta, const CUtensorMap& tb, const MmaArgs& a) {
    static std::once_flag once;
    std::call_once(once, [] {
        TRG_CUDA(cudaFuncSetAttribute(k_split_mma<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes_for(S)));
    });
    const int tiles = ((a.M + BM - 1) / BM) * ((a.N + BN - 1) / BN);
    const int grid = std::max(1, std::min(tiles, ctx.sm_count));
    k_split_mma<S><<<grid, THREADS, smem_bytes_for(S), ctx.stream>>>(ta, tb, a);
    ctx.launches++;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, k_split_mma<S>);
        fail(TRG_ECUDA, std::string("split MMA launch: ") + cudaGetErrorString(e) + " (regs " +
                            std::to_string(fa.numRegs) + ", max threads " + std::to_string(fa.maxThreadsPerBlock) +
                            ", dyn smem " + std::to_string(smem_bytes_for(S)) + " / " +
                            std::to_string(fa.maxDynamicSharedSizeBytes) + ", local " +
                            std::to_string(fa.localSizeBytes) + ")");
    }
}

template <int S>
void launch_slice(Ctx& ctx, const Gather& g, int R, int K, int Rp, int Kp, const int* e, uint16_t* out) {
    dim3 grid((unsigned)((Kp + SL_K - 1) / SL_K), (unsigned)((Rp + SL_R - 1) / SL_R));
    k_slice<S><<<grid, 256, 0, ctx.stream>>>(g.base, g.off_r, g.off_c, R, K, Rp, Kp, g.c_fast ? 1 : 0, e, out);
    TRG_LAUNCHED(ctx);
}

void row_exponents(Ctx& ctx, const Gather& g, int R, int K, int* e) {
    TRG_CUDA(cudaMemsetAsync(e, 0, (size_t)R * sizeof(int), ctx.stream));
    dim3 grid((unsigned)((K + SL_K - 1) / SL_K), (unsigned)((R + SL_R - 1) / SL_R));
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
    return t;
}

void gemm_split(Ctx& ctx, const GemmDesc& d) {
    if (d.M <= 0 || d.N <= 0) return;
    if (d.beta != 0.0) fail(TRG_EINVAL, "split GEMM overwrites its output (beta must be 0)");
    if (d.M > (1ll << 30) || d.N > (1ll << 30) || d.K > (1 << 17)) fail(TRG_EINVAL, "split GEMM: size out of range");
    const int S = ctx.cfg.split_slices;
    const int M = (int)d.M, N = (int)d.N, K = (int)std::max<int64_t>(d.K, 1);
    const int Mp = (M + BM - 1) / BM * BM, Np = (N + BN - 1) / BN * BN, Kp = (K + BK - 1) / BK * BK;

    // scratch: exponents + slices of A and B
    const size_t bytes_e = (size_t)(Mp + Np) * sizeof(int);
    const size_t bytes_a = (size_t)S * Mp * Kp * 2, bytes_b = (size_t)S * Np * Kp * 2;
    ctx.ensure(ctx.split_ws, bytes_e + bytes_a + bytes_b + 1024);
    uint8_t* base = ctx.split_ws.as<uint8_t>();
    int* ea = (int*)base;
    int* eb = ea + Mp;
    uint16_t* sa = (uint16_t*)(base + ((bytes_e + 255) & ~(size_t)255));
    uint16_t* sb = sa + (size_t)S * Mp * Kp;

    // B as rows n, columns k: element (n, k) at B[b_k[k] + b_n[n]]
    const Gather bt = transpose_gather(d.B, d.B.off_r, d.B.off_c);
    Gather bt2 = bt;
    bt2.c_fast = false;
    // contiguous along k in memory?  (the k-table of B is B.off_r)
    if (d.a_ef) {
        // the producing product already recorded A's exponent fields
        TRG_CUDA(cudaMemcpyAsync(ea, d.a_ef, (size_t)M * sizeof(int), cudaMemcpyDeviceToDevice, ctx.stream));
        k_exponent_finish<<<(unsigned)((M + 255) / 256), 256, 0, ctx.stream>>>(ea, M);
        TRG_LAUNCHED(ctx);
    } else {
        row_exponents(ctx, d.A, M, K, ea);
    }
    row_exponents(ctx, bt2, N, K, eb);
    switch (S) {
        case 2: launch_slice<2>(ctx, d.A, M, K, Mp, Kp, ea, sa); launch_slice<2>(ctx, bt2, N, K, Np, Kp, eb, sb); break;
        case 3: launch_slice<3>(ctx, d.A, M, K, Mp, Kp, ea, sa); launch_slice<3>(ctx, bt2, N, K, Np, Kp, eb, sb); break;
        case 4: launch_slice<4>(ctx, d.A, M, K, Mp, Kp, ea, sa); launch_slice<4>(ctx, bt2, N, K, Np, Kp, eb, sb); break;
        case 5: launch_slice<5>(ctx, d.A, M, K, Mp, Kp, ea, sa); launch_slice<5>(ctx, bt2, N, K, Np, Kp, eb, sb); break;
        default: fail(TRG_EINVAL, "split_slices must be 2..5");
    }
    const CUtensorMap ta = make_map(sa, S * Mp, Kp);
    const CUtensorMap tb = make_map(sb, S * Np, Kp);
    MmaArgs a;
    a.M = M; a.N = N; a.Kp = Kp; a.Mp = Mp; a.Np = Np; a.S = S;
    a.ea = ea; a.eb = eb; a.C = d.C; a.c_m = d.c_m; a.c_n = d.c_n;
    a.status = ctx.status.as<int>();
    a.cons_ef = d.cons_ef; a.cons_m = d.cons_m; a.cons_n = d.cons_n;
    const int tok = ctx.region_begin(TRG_PHASE_MMA);
    switch (S) {
        case 2: launch_mma<2>(ctx, ta, tb, a); break;
        case 3: launch_mma<3>(ctx, ta, tb, a); break;
        case 4: launch_mma<4>(ctx, ta, tb, a); break;
        case 5: launch_mma<5>(ctx, ta, tb, a); break;
    }
    const double products = (double)S * (S + 1) / 2;
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
            dim3 ga((unsigned)((K + SL_K - 1) / SL_K), (unsigned)((M + SL_R - 1) / SL_R));
            k_row_exponent<<<ga, 256, 0, stream>>>(A, am, ak, M, K, 1, ea);
            dim3 gb((unsigned)((K + SL_K - 1) / SL_K), (unsigned)((N + SL_R - 1) / SL_R));
            k_row_exponent<<<gb, 256, 0, stream>>>(B, bn, bk, N, K, 0, eb);
            k_exponent_finish<<<(unsigned)((M + 255) / 256), 256, 0, stream>>>(ea, M);
            k_exponent_finish<<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(eb, N);
            TRG_CUDA(cudaGetLastError());
            dim3 sa_grid((unsigned)((Kp + SL_K - 1) / SL_K), (unsigned)(Mp / SL_R));
            dim3 sb_grid((unsigned)((Kp + SL_K - 1) / SL_K), (unsigned)(Np / SL_R));
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
        const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
        const int grid = std::max(1, std::min(tiles, sms));
        switch (S) {
#define TRG_NOALLOC_MMA(SS)                                                                                  \
    TRG_CUDA(cudaFuncSetAttribute(k_split_mma<SS>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                  smem_bytes_for(SS)));                                                      \
    k_split_mma<SS><<<grid, THREADS, smem_bytes_for(SS), stream>>>(ta, tbm, a);                              \
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
