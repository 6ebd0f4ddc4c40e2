// Plain FP64 gathered GEMM on the CUDA cores (the TRG_FP64 precision mode).
//
// Every contraction of the HOTRG step (environment, U.T.T.U, M.Q products of
// the subspace iteration) is a matrix product once its multi-indices are
// flattened; offset tables do the flattening, so permuted and rotated views
// (the y half-step) cost nothing extra.  64x64 output tile per 256-thread
// block, K in steps of 16 through shared memory, 4x4 outputs per thread.
#include <algorithm>

#include "internal.h"

namespace trg {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

struct GemmArgs {
    int64_t M, N, K;
    int64_t kper;          // split-K: K range of blockIdx.z is [z*kper, min(K, (z+1)*kper))
    double* partial;       // split-K: dense M x N partial sums per z (else nullptr)
    const double* A; const int64_t* a_m; const int64_t* a_k; int a_kfast;
    const double* B; const int64_t* b_k; const int64_t* b_n; int b_nfast;
    double* C; const int64_t* c_m; const int64_t* c_n;
    double beta;
};

__global__ void __launch_bounds__(NT) k_gemm_f64(const GemmArgs g) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t m0 = (int64_t)blockIdx.y * BM;
    const int64_t n0 = (int64_t)blockIdx.x * BN;

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    const int64_t kbeg = (int64_t)blockIdx.z * g.kper;
    const int64_t kend = min(g.K, kbeg + g.kper);
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int e = tid; e < BM * BK; e += NT) {
            int r, kk;
            if (g.a_kfast) { kk = e % BK; r = e / BK; } else { r = e % BM; kk = e / BM; }
            const int64_t m = m0 + r, k = k0 + kk;
            double v = 0.0;
            if (m < g.M && k < kend) v = g.A[g.a_m[m] + g.a_k[k]];
            As[kk][r] = v;
        }
#pragma unroll
        for (int e = tid; e < BN * BK; e += NT) {
            int c, kk;
            if (g.b_nfast) { c = e % BN; kk = e / BN; } else { kk = e % BK; c = e / BK; }
            const int64_t n = n0 + c, k = k0 + kk;
            double v = 0.0;
            if (n < g.N && k < kend) v = g.B[g.b_k[k] + g.b_n[n]];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    if (g.partial) {
        double* P = g.partial + (int64_t)blockIdx.z * g.M * g.N;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t m = m0 + ty + 16 * i;
            if (m >= g.M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t n = n0 + tx + 16 * j;
                if (n < g.N) P[m * g.N + n] = acc[i][j];
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
        const int64_t cm = g.c_m[m];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t n = n0 + tx + 16 * j;
            if (n >= g.N) continue;
            double* dst = g.C + cm + g.c_n[n];
            *dst = (g.beta != 0.0) ? fma(g.beta, *dst, acc[i][j]) : acc[i][j];
        }
    }
}

// C = beta C + sum_z P[z], summed in z order (deterministic).
__global__ void k_reduce_partials(const double* __restrict__ P, int nz, int64_t M, int64_t N, double* C,
                                  const int64_t* c_m, const int64_t* c_n, double beta) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += P[(int64_t)z * M * N + e];
    const int64_t m = e / N, n = e % N;
    double* dst = C + c_m[m] + c_n[n];
    *dst = (beta != 0.0) ? fma(beta, *dst, s) : s;
}

}  // namespace

void gemm_f64(Ctx& ctx, const GemmDesc& d) {
    if (d.M <= 0 || d.N <= 0) return;
    GemmArgs g;
    g.M = d.M; g.N = d.N; g.K = d.K;
    g.kper = std::max<int64_t>(d.K, 1);
    g.partial = nullptr;
    g.A = d.A.base; g.a_m = d.A.off_r; g.a_k = d.A.off_c; g.a_kfast = d.A.c_fast ? 1 : 0;
    g.B = d.B.base; g.b_k = d.B.off_r; g.b_n = d.B.off_c; g.b_nfast = d.B.c_fast ? 1 : 0;
    g.C = d.C; g.c_m = d.c_m; g.c_n = d.c_n; g.beta = d.beta;
    const int64_t gx = (d.N + BN - 1) / BN, gy = (d.M + BM - 1) / BM;
    if (gy > 65535) fail(TRG_EINVAL, "gemm_f64: too many row tiles");
    // few output tiles and a long K (Gram and Rayleigh-Ritz products of the
    // subspace iteration): split K over the SMs, then reduce in a fixed order
    int64_t nz = 1;
    if (gx * gy * 4 <= ctx.sm_count && d.K >= 1024) {
        nz = std::min<int64_t>(d.K / 256, (2 * ctx.sm_count + gx * gy - 1) / (gx * gy));
        nz = std::max<int64_t>(nz, 1);
    }
    if (nz > 1) {
        g.kper = ((d.K + nz - 1) / nz + BK - 1) / BK * BK;
        nz = (d.K + g.kper - 1) / g.kper;
        ctx.ensure(ctx.f64_partial, (size_t)(nz * d.M * d.N) * sizeof(double));
        g.partial = ctx.f64_partial.as<double>();
    }
    dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)nz);
    k_gemm_f64<<<grid, NT, 0, ctx.stream>>>(g);
    TRG_LAUNCHED(ctx);
    if (nz > 1) {
        const int64_t tot = d.M * d.N;
        k_reduce_partials<<<(unsigned)((tot + 255) / 256), 256, 0, ctx.stream>>>(g.partial, (int)nz, d.M, d.N, d.C,
                                                                              d.c_m, d.c_n, d.beta);
        TRG_LAUNCHED(ctx);
    }
}

}  // namespace trg
