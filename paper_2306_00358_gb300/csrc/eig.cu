// Isometry of the HOTRG step: leading eigenvectors of the environment M.
//
// The paper (Sec. 2, SVD helper of the coarse-graining listing) keeps the
// leading min(n, Dcut) left singular vectors of M; M is a Gram matrix
// (symmetric PSD), so these are its leading eigenvectors.  Here they come from
// block subspace iteration:
//   Y = M Q                                  (GEMM, the context's precision)
//   H = Q^T Y, H = W diag(theta) W^T         (Rayleigh-Ritz, FP64 Jacobi)
//   residual |Y w_i - theta_i Q w_i| <= tol * theta_1 for i < Dn  -> done
//   Q <- orth(Y W)                           (FP64 Cholesky-QR, two passes)
// Cholesky-QR works on column-normalised blocks; a column whose Cholesky
// pivot shows it is numerically dependent on the earlier ones is replaced by
// a fresh seeded random column (this happens when M's spectrum falls below
// rounding, e.g. in the ordered phase).  All blocks are column-major (n x m).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.h"

namespace trg {

namespace {

constexpr int MAX_M = 112;   // largest block (Dcut + oversampling) held in shared memory

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Seeded uniform(-1, 1) entries; only columns with flags[c] != 0 when flags is given.
__global__ void k_rand_cols(double* Y, int64_t n, int m, const int* flags, uint64_t seed, uint64_t salt) {
    const int c = blockIdx.y;
    if (c >= m || (flags && !flags[c])) return;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        uint64_t h = splitmix64(seed ^ splitmix64(salt * 0x100000001B3ull + (uint64_t)c * 0x9E3779B1ull + (uint64_t)r));
        Y[(int64_t)c * n + r] = 2.0 * ((double)(h >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
}

template <int NT>
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < NT / 32) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) red[0] = s;
    }
    __syncthreads();
    return red[0];
}

// Scale every column to unit 2-norm; flag columns that are zero or not finite.
__global__ void __launch_bounds__(256) k_col_normalize(double* Y, int64_t n, int* flags) {
    __shared__ double red[32];
    const int c = blockIdx.x;
    double* y = Y + (int64_t)c * n;
    double mx = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += 256) mx = fmax(mx, fabs(y[r]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int i = 0; i < 8; ++i) v = fmax(v, red[i]);
        red[8] = v;
    }
    __syncthreads();
    mx = red[8];
    __syncthreads();
    if (!(mx > 0.0) || !isfinite(mx)) {
        if (threadIdx.x == 0) flags[c] = 1;
        return;
    }
    const double inv = 1.0 / mx;   // scale first so the squares cannot under/overflow
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += 256) { const double v = y[r] * inv; s = fma(v, v, s); }
    s = block_sum<256>(s, red);
    const double scale = inv / sqrt(s);
    for (int64_t r = threadIdx.x; r < n; r += 256) y[r] *= scale;
}

// Right-looking Cholesky G = L L^T of an m x m Gram matrix of unit columns.
// Per column: warp 0 takes the pivot and scales the column (also into a
// broadcast copy), then all threads update the trailing triangle.
// A pivot d_j <= tau * G_jj marks column j as dependent (flags[j] = 1,
// *nbad += 1); the pivot is then replaced by G_jj so the factorisation can
// continue.
// The trailing update of column j touches the elements (i, k), j < k <= i.
// They are listed once, by k descending (k = m-1 first), so those of column
// j are the first (m-1-j)(m-j)/2 entries: every thread takes a share and a
// warp's FP64 instructions run on all 32 lanes (the FP64 pipe, not the
// lanes, is what a lane-per-column layout of short rows wastes).
__host__ __device__ constexpr int chol_table_entries(int m) { return m * (m - 1) / 2; }
__global__ void __launch_bounds__(256) k_chol_flag(const double* G, double* Lout, int m, double tau,
                                                   int* flags, int* nbad, double* pivmin_out) {
    // m rows of ld = m + 1 (an odd stride: the rows of one column fall in
    // different banks), m of the original diagonal, m of column j, then the
    // trailing-element list (i << 7 | k, 16 bits each)
    extern __shared__ double L[];
    const int ld = m + 1;
    double* gd = L + m * ld;
    double* colj = gd + m;
    uint16_t* tab = (uint16_t*)(colj + m);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) L[(e / m) * ld + e % m] = G[e];
    for (int i = threadIdx.x; i < m; i += blockDim.x) gd[i] = G[(int64_t)i * m + i];
    for (int e = threadIdx.x; e < chol_table_entries(m); e += blockDim.x) {
        // group gidx = m-1-k holds the gidx+1 elements (k..m-1, k) from offset gidx(gidx+1)/2
        int gidx = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (gidx * (gidx + 1) / 2 > e) --gidx;
        while ((gidx + 1) * (gidx + 2) / 2 <= e) ++gidx;
        const int k = m - 1 - gidx, i = k + (e - gidx * (gidx + 1) / 2);
        tab[e] = (uint16_t)((i << 7) | k);
    }
    __syncthreads();
    double pivmin = 1.0;    // smallest d_j / G_jj (thread 0): 1 / pivmin bounds cond(Y)^2 from below
    for (int j = 0; j < m; ++j) {
        if (warp == 0) {
            double d = L[j * ld + j];
            if (lane == 0) {
                const double gjj = gd[j];
                pivmin = fmin(pivmin, (gjj > 0.0 && isfinite(d)) ? d / gjj : 0.0);
                if (!(d > tau * gjj) || !isfinite(d)) {
                    flags[j] = 1;
                    atomicAdd(nbad, 1);
                    d = (gjj > 0.0 && isfinite(gjj)) ? gjj : 1.0;
                }
            }
            d = __shfl_sync(0xffffffffu, d, 0);
            const double il = rsqrt(d);
            if (lane == 0) L[j * ld + j] = d * il;
            for (int i = j + 1 + lane; i < m; i += 32) {
                const double v = L[i * ld + j] * il;
                L[i * ld + j] = v;
                colj[i] = v;
            }
        }
        __syncthreads();
        const int cnt = (m - 1 - j) * (m - j) / 2;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const unsigned t = tab[e];
            const int i = (int)(t >> 7), k = (int)(t & 127u);
            L[i * ld + k] = fma(-colj[i], colj[k], L[i * ld + k]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x)
        Lout[e] = ((e % m) <= (e / m)) ? L[(e / m) * ld + e % m] : 0.0;
    if (threadIdx.x == 0 && pivmin_out) *pivmin_out = pivmin;
}

// Q = Y L^{-T} row by row, in place allowed: 32 rows per block, a lane per
// row, the solution in shared memory.  Right-looking: after x_j is known,
// every later column k subtracts L[k][j] x_j.  Column k belongs to warp
// k % 8, so the eight warps (two per FP64 pipe, which hides the latency of
// each one's load-FMA-store chain) share the updates and x_j needs no
// reduction, one block barrier per column.
constexpr int TRSM_ROWS = 32;
constexpr int TRSM_THREADS = 256;
constexpr int TRSM_WARPS = TRSM_THREADS / 32;
__global__ void __launch_bounds__(TRSM_THREADS) k_trsm_rows(double* Y, const double* Lg, int64_t n, int m) {
    extern __shared__ double L[];   // m*m, m inverse diagonals, TRSM_ROWS rows of m + 1, 2 x TRSM_ROWS x_j
    double* dinv = L + m * m;
    double* rows = dinv + m;
    double* xb = rows + TRSM_ROWS * (m + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) L[e] = Lg[e];
    for (int i = threadIdx.x; i < m; i += blockDim.x) dinv[i] = 1.0 / Lg[(int64_t)i * m + i];
    const int64_t r0 = (int64_t)blockIdx.x * TRSM_ROWS;
    for (int e = threadIdx.x; e < m * TRSM_ROWS; e += blockDim.x) {
        const int j = e / TRSM_ROWS, t = e % TRSM_ROWS;
        rows[t * (m + 1) + j] = (r0 + t < n) ? Y[(int64_t)j * n + r0 + t] : 0.0;
    }
    __syncthreads();
    double* y = rows + lane * (m + 1);
    for (int j = 0; j < m; ++j) {
        double* xs = xb + (j & 1) * TRSM_ROWS;
        if (warp == (j & (TRSM_WARPS - 1))) {
            const double x = y[j] * dinv[j];
            y[j] = x;
            xs[lane] = x;
        }
        __syncthreads();
        const double x = xs[lane];
        int k = j + 1 + ((warp - (j + 1)) & (TRSM_WARPS - 1));   // first column > j owned by this warp
        for (; k < m; k += TRSM_WARPS) y[k] = fma(-L[k * m + j], x, y[k]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * TRSM_ROWS; e += blockDim.x) {
        const int j = e / TRSM_ROWS, t = e % TRSM_ROWS;
        if (r0 + t < n) Y[(int64_t)j * n + r0 + t] = rows[t * (m + 1) + j];
    }
}

// Tall-skinny G = A^T B for column-major n x m blocks A, B: each CTA sums a
// slab of rows into its own m x m partial (rows staged in shared memory);
// k_gram_reduce adds the partials in slab order (deterministic).
__global__ void __launch_bounds__(256) k_gram_partial(const double* A, const double* B, int64_t n, int m,
                                                      int64_t rows_per_cta, double* part, int sym) {
    extern __shared__ double sh[];   // rows_per_cta x m for A, then for B
    const int64_t r0 = blockIdx.x * rows_per_cta;
    const int64_t nr = max((int64_t)0, min(rows_per_cta, n - r0));
    double* As = sh;
    double* Bs = sh + rows_per_cta * m;
    for (int64_t e = threadIdx.x; e < nr * m; e += 256) {
        const int64_t c = e / nr, r = e % nr;
        As[r * m + c] = A[c * n + r0 + r];
        Bs[r * m + c] = B[c * n + r0 + r];
    }
    __syncthreads();
    double* P = part + (int64_t)blockIdx.x * m * m;
    // A = B: the partial is symmetric and the products of (j, i) are those
    // of (i, j), so the upper triangle is mirrored (identical bits)
    const int ne = sym ? m * (m + 1) / 2 : m * m;
    for (int e0 = threadIdx.x; e0 < ne; e0 += 256) {
        int i, j;
        if (sym) {
            // e0 -> (i, j), i <= j, row-major over the upper triangle
            i = (int)(((2.0f * m + 1.0f) - sqrtf((2.0f * m + 1.0f) * (2.0f * m + 1.0f) - 8.0f * (float)e0)) * 0.5f);
            while (i > 0 && i * m - i * (i - 1) / 2 > e0) --i;
            while ((i + 1) * m - (i + 1) * i / 2 <= e0) ++i;
            j = i + (e0 - (i * m - i * (i - 1) / 2));
        } else {
            i = e0 / m;
            j = e0 % m;
        }
        const int e = i * m + j;
        double s0 = 0.0, s1 = 0.0;
        int64_t r = 0;
        for (; r + 1 < nr; r += 2) {
            s0 = fma(As[r * m + i], Bs[r * m + j], s0);
            s1 = fma(As[(r + 1) * m + i], Bs[(r + 1) * m + j], s1);
        }
        if (r < nr) s0 = fma(As[r * m + i], Bs[r * m + j], s0);
        P[e] = s0 + s1;
        if (sym && i != j) P[j * m + i] = s0 + s1;
    }
}

__global__ void __launch_bounds__(64) k_gram_reduce(const double* part, int nparts, int m, double* G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    double s = 0.0;
#pragma unroll 8
    for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * m * m + e];
    G[e] = s;
}

// Cyclic Jacobi sweeps with parallel (round-robin) ordering on a symmetric
// m x m matrix H (row-major, shared memory), accumulating W <- W J (W
// column-major).  Rotation (p,q): tau = (h_qq - h_pp)/(2 h_pq),
// t = sign(tau)/(|tau| + sqrt(1+tau^2)), c = 1/sqrt(1+t^2), s = t c;
// H <- J^T H J.  Rotations with |h_pq| <= tol sqrt(|h_pp h_qq|) are skipped
// (relative-accuracy threshold for graded matrices); the loop ends when no
// pair is above the threshold.  Returns the number of sweeps that rotated
// (max_sweeps + 1 if the limit was hit).  All threads of the block call it.
__device__ __forceinline__ void rr_pair(int r, int i, int mp, int& p, int& q) {
    if (i == 0) { p = mp - 1; q = r; }
    else { p = (r + i) % (mp - 1); q = (r - i + (mp - 1)) % (mp - 1); }
    if (p > q) { const int x = p; p = q; q = x; }
}

template <typename T>
__device__ __forceinline__ bool jacobi_rotates(T hpq, T hpp, T hqq, T tol) {
    return fabs(hpq) > tol * sqrt(fabs(hpp * hqq)) && fabs(hpq) > (T)1e-300;
}

template <typename T>
__device__ int jacobi_sweeps(T* H, int ld, T* W, int m, T tol, int max_sweeps, T* cs, int* rot, int* pq) {
    const int mp = m + (m & 1);            // even player count (dummy index m when odd)
    const int npair = mp / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        // A sweep rotates nothing exactly when no pair of the current H is
        // above the threshold (H only changes by rotations), so one scan of
        // the pairs stands in for that last, confirming sweep.
        if (threadIdx.x == 0) *rot = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int p = e / m, q = e % m;
            if (p < q && jacobi_rotates<T>(H[p * ld + q], H[p * ld + p], H[q * ld + q], tol)) *(volatile int*)rot = 1;
        }
        __syncthreads();
        if (*rot == 0) return sweep;
        __syncthreads();
        for (int r = 0; r < mp - 1; ++r) {
            for (int i = threadIdx.x; i < npair; i += blockDim.x) {
                int p, q;
                rr_pair(r, i, mp, p, q);
                T c = 1, s = 0;
                if (q < m) {
                    const T hpq = H[p * ld + q], hpp = H[p * ld + p], hqq = H[q * ld + q];
                    if (jacobi_rotates<T>(hpq, hpp, hqq, tol)) {
                        const T tau = (hqq - hpp) / (2 * hpq);
                        const T t = (tau >= 0) ? 1 / (tau + sqrt(1 + tau * tau)) : -1 / (-tau + sqrt(1 + tau * tau));
                        c = 1 / sqrt(1 + t * t);
                        s = t * c;
                    }
                }
                cs[2 * i] = c;
                cs[2 * i + 1] = s;
                pq[2 * i] = p;
                pq[2 * i + 1] = q;
            }
            __syncthreads();
            // columns: H <- H J, W <- W J (a warp per rotation, a lane per row)
            for (int i = warp; i < npair; i += nwarps) {
                const T s = cs[2 * i + 1];
                if (s == 0) continue;
                const T c = cs[2 * i];
                const int p = pq[2 * i], q = pq[2 * i + 1];
                T* wp = W + (int64_t)p * m;
                T* wq = W + (int64_t)q * m;
                for (int k = lane; k < m; k += 32) {
                    const T hkp = H[k * ld + p], hkq = H[k * ld + q];
                    H[k * ld + p] = c * hkp - s * hkq;
                    H[k * ld + q] = s * hkp + c * hkq;
                    const T vp = wp[k], vq = wq[k];
                    wp[k] = c * vp - s * vq;
                    wq[k] = s * vp + c * vq;
                }
            }
            __syncthreads();
            // rows: H <- J^T H, then the annihilated pair is exactly zero
            for (int i = warp; i < npair; i += nwarps) {
                const T s = cs[2 * i + 1];
                if (s == 0) continue;
                const T c = cs[2 * i];
                const int p = pq[2 * i], q = pq[2 * i + 1];
                T* hp = H + p * ld;
                T* hq = H + q * ld;
                for (int k = lane; k < m; k += 32) {
                    const T hpk = hp[k], hqk = hq[k];
                    hp[k] = c * hpk - s * hqk;
                    hq[k] = s * hpk + c * hqk;
                }
                __syncwarp();
                if (lane == 0) { hp[q] = 0; hq[p] = 0; }
            }
            __syncthreads();
        }
    }
    return max_sweeps + 1;
}

// Rayleigh-Ritz eigensolve of the symmetric m x m matrix Hg (global), in
// two precisions:
//  1. FP32 Jacobi on H / max|H| to a relative threshold of 1e-6 (the FP32
//     pipe is ~60x the FP64 pipe on this part); rotations accumulate in W32
//     (k_rr_fp32, one CTA);
//  2. W = W32 in FP64, refined by two Ogita-Aishima steps and a Lowdin
//     step (k_oa_step, k_lowdin): m x m FP64 products on many SMs
//     (k_small_nn, k_small_tn, k_small_apply) that leave W orthonormal to
//     rounding and the couplings of the separated pairs of H' = W^T H W
//     squared twice (at beta_c, Dcut 24, none is left above the FP64
//     threshold; off critical a graded tail of a few hundred pairs is);
//  3. FP64 Jacobi sweeps on H' (k_rr_fp64, one CTA): they find only the
//     pairs step 2 left coupled (near-degenerate ones), W <- W J.
// A rough Rayleigh-Ritz far from convergence (no FP64 sweeps) instead
// re-orthonormalises W32 by Cholesky-QR and takes theta = diag(W^T H W).
// Output: theta sorted descending, W (column-major, global) in that order.
// Shared memory of the one-CTA kernels: H (m rows of ld = m + 1 doubles: the
// odd stride puts the rows of one column in different banks, so the column
// updates are conflict-free) + m*ld doubles of scratch + small arrays.
__global__ void __launch_bounds__(512) k_rr_fp32(const double* Hg, int m, double* Hsym, double* Wout,
                                                 int* sweeps_out) {
    extern __shared__ double sm[];
    const int mp = m + (m & 1);
    const int ld = m + 1;
    float* H32 = (float*)sm;                   // m*ld floats
    float* W32 = H32 + m * ld;                 // m*m floats
    float* cs32 = W32 + m * m;                 // mp
    int* rot = (int*)(cs32 + mp + (mp & 1));   // 1
    int* pq = rot + 2;                         // mp: the pairs of the current round
    __shared__ double hmax_s;
    if (threadIdx.x == 0) hmax_s = 0.0;
    __syncthreads();
    double lmax = 0.0;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        const double v = 0.5 * (Hg[(int64_t)i * m + j] + Hg[(int64_t)j * m + i]);
        Hsym[e] = v;
        lmax = fmax(lmax, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long*)&hmax_s, (unsigned long long)__double_as_longlong(lmax));
    __syncthreads();
    const double hscale = hmax_s > 0.0 ? 1.0 / hmax_s : 1.0;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        H32[i * ld + j] = (float)(0.5 * (Hg[(int64_t)i * m + j] + Hg[(int64_t)j * m + i]) * hscale);
        W32[e] = (i == j) ? 1.0f : 0.0f;
    }
    __syncthreads();
    const int s32 = jacobi_sweeps<float>(H32, ld, W32, m, 1e-6f, 40, cs32, rot, pq);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) Wout[e] = (double)W32[e];
    if (threadIdx.x == 0 && sweeps_out) atomicAdd(sweeps_out, s32);
}

// C[i][j] = sum_r A[i*m + r] B[j*m + r] (the columns of two column-major m x
// m blocks): a CTA per row i, a thread per column j, the sum in order of r.
__global__ void __launch_bounds__(128) k_small_tn(const double* A, const double* B, int m, double* C) {
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double a = 0.0;
        for (int r = 0; r < m; ++r) a = fma(A[(int64_t)i * m + r], B[(int64_t)j * m + r], a);
        C[(int64_t)i * m + j] = a;
    }
}

// (H W)[r][j] = sum_k H[r*m + k] W[j*m + k] (row-major H, column-major W),
// stored column-major: C[j*m + r].
__global__ void __launch_bounds__(128) k_small_nn(const double* H, const double* W, int m, double* C) {
    const int r = blockIdx.x;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double a = 0.0;
        for (int k = 0; k < m; ++k) a = fma(H[(int64_t)r * m + k], W[(int64_t)j * m + k], a);
        C[(int64_t)j * m + r] = a;
    }
}

// Xout = X (I + E) = X + X E for a column-major m x m X and a row-major E:
// a CTA per column j, a thread per row r, the sum in order of k.
__global__ void __launch_bounds__(128) k_small_apply(const double* X, const double* E, int m, double* Xout) {
    const int j = blockIdx.x;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        double a = 0.0;
        for (int k = 0; k < m; ++k) a = fma(X[(int64_t)k * m + r], E[(int64_t)k * m + j], a);
        Xout[(int64_t)j * m + r] = X[(int64_t)j * m + r] + a;
    }
}

// One refinement step of an approximate eigenbasis X of the symmetric H
// after Ogita and Aishima (Iterative refinement for symmetric eigenvalue
// decomposition, Japan J. Indust. Appl. Math. 35, 2018).  With S = X^T H X
// (symmetrised here) and P = X^T X = I - R:
//   lambda_i = s_ii / p_ii,
//   E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)   for a separated pair,
//   E_ij = r_ij / 2                                         otherwise and for i = j,
// and X <- X (I + E) (k_small_apply): to first order that makes X^T X = I
// (E + E^T = R) and zeroes the separated couplings, so both shrink
// quadratically from step to step.  Where the published step separates
// pairs by one global gap bound, this one takes a pair as separated when
// |lambda_j - lambda_i| > OA_SEP (|s_ij| + max(|lambda_i|, |lambda_j|) |r_ij|),
// i.e. |E_ij| < 1 / OA_SEP: a symmetric test, so E + E^T = R holds exactly,
// and a strict one, so that the second-order terms (X^T X - I after a step
// is about E^T E) stay small even where the FP32 vectors of a graded tail
// are poor.  Pairs it leaves coupled (near-degenerate ones, the tail) are
// left to FP64 Jacobi.
// One CTA.
constexpr double OA_SEP = 256.0;
constexpr int OA_STEPS = 2;
__global__ void __launch_bounds__(256) k_oa_step(const double* S, const double* P, int m, double* E) {
    __shared__ double lam[MAX_M];
    for (int i = threadIdx.x; i < m; i += blockDim.x) lam[i] = S[(int64_t)i * m + i] / P[(int64_t)i * m + i];
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        const double r = (i == j ? 1.0 : 0.0) - P[e];
        double v = 0.5 * r;
        if (i != j) {
            const double sij = 0.5 * (S[e] + S[(int64_t)j * m + i]);
            const double gap = lam[j] - lam[i];
            const double bound = OA_SEP * (fabs(sij) + fmax(fabs(lam[i]), fabs(lam[j])) * fabs(r));
            if (fabs(gap) > bound) v = (sij + lam[j] * r) / gap;
        }
        E[e] = v;
    }
}

// Second-order Lowdin (symmetric) orthonormalisation: for X^T X = P = I - R
// with R small, X (I + F) with F = R / 2 + 3 R^2 / 8 (the series of
// (I - R)^(-1/2)) has (I + F)^T P (I + F) = I + O(R^3).  PP = P P gives
// R^2 = PP - 2 P + I.  F is row-major (P, PP symmetric).
__global__ void __launch_bounds__(256) k_lowdin(const double* P, const double* PP, int m, double* F) {
    for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < m * m; e += blockDim.x * gridDim.x) {
        const int i = e / m, j = e % m;
        const double id = (i == j) ? 1.0 : 0.0;
        const double r = id - P[e];
        const double r2 = PP[e] - 2.0 * P[e] + id;
        F[e] = 0.5 * r + 0.375 * r2;
    }
}

// Step 3 of the Rayleigh-Ritz solve: H = (G + G^T) / 2, FP64 sweeps from
// W = Win (accumulated in shared memory), then theta and W sorted by
// descending theta (ties keep index order) into Wout (may alias Win).
__global__ void __launch_bounds__(512) k_rr_fp64(const double* G, int m, double tol, int max_sweeps,
                                                 double* theta, const double* Win, double* Wout, int* status,
                                                 int* sweeps_out, int fp64_sweeps) {
    extern __shared__ double sm[];
    const int mp = m + (m & 1);
    const int ld = m + 1;
    double* H = sm;                            // m*ld
    double* Ws = H + m * ld;                   // m*m (W, accumulated)
    double* cs64 = Ws + m * ld;                // mp
    int* rot = (int*)(cs64 + mp);              // 1
    int* perm = rot + 2;                       // m
    int* pq = perm + m + (m & 1);              // mp
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        H[i * ld + j] = 0.5 * (G[(int64_t)i * m + j] + G[(int64_t)j * m + i]);
        Ws[e] = Win[e];
    }
    __syncthreads();
    // (skipped for a rough Rayleigh-Ritz far from convergence: then theta is
    // the diagonal of H' and W the re-orthonormalised W32)
    const int s64 = fp64_sweeps ? jacobi_sweeps<double>(H, ld, Ws, m, tol, max_sweeps, cs64, rot, pq) : 0;
    // rank of each diagonal value, descending; ties by index
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double hi = H[i * ld + i];
        int r = 0;
        for (int j = 0; j < m; ++j) {
            const double hj = H[j * ld + j];
            r += (hj > hi || (hj == hi && j < i)) ? 1 : 0;
        }
        perm[r] = i;
    }
    if (threadIdx.x == 0) {
        if (s64 > max_sweeps) atomicOr(status, ST_EIG_NOCONV);
        if (sweeps_out) atomicAdd(sweeps_out + 1, s64);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) theta[i] = H[perm[i] * ld + perm[i]];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int col = e / m, row = e % m;
        Wout[e] = Ws[perm[col] * m + row];
    }
}

// max_i<dn |Z_i - theta_i QW_i| / theta_0, as bits of a non-negative double.
__global__ void __launch_bounds__(256) k_residual(const double* Z, const double* QW, const double* theta,
                                                  int64_t n, unsigned long long* out_bits) {
    __shared__ double red[33];
    const int c = blockIdx.x;
    const double th = theta[c];
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += 256) {
        const double d = Z[(int64_t)c * n + r] - th * QW[(int64_t)c * n + r];
        s = fma(d, d, s);
    }
    s = block_sum<256>(s, red);
    if (threadIdx.x == 0) {
        double rel = sqrt(s) / fabs(theta[0]);
        if (!isfinite(rel)) rel = INFINITY;
        atomicMax(out_bits, (unsigned long long)__double_as_longlong(rel));
    }
}

// Y <- Y - sigma Q (the shift of a power step)
__global__ void k_shift(double* Y, const double* Q, double sigma, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        Y[i] = fma(-sigma, Q[i], Y[i]);
}

// U[r*dn + i] = QW[i*n + r]
__global__ void k_to_isometry(const double* QW, int64_t n, int dn, double* U) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * dn) return;
    const int64_t r = e / dn, i = e % dn;
    U[e] = QW[i * n + r];
}

}  // namespace

static size_t rr32_smem(int m) {
    const int mp = m + (m & 1);
    return (size_t)m * (m + 1) * 4 + (size_t)m * m * 4 + (size_t)(mp + 2) * 4 + (size_t)(mp + 4) * 4 + 64;
}

static size_t rr64_smem(int m) {
    const int mp = m + (m & 1);
    return (size_t)2 * m * (m + 1) * 8 + (size_t)mp * 8 + (size_t)(m + 4) * 4 + (size_t)mp * 4 + 64;
}

static size_t chol_smem(int m) {
    return (size_t)m * (m + 1) * 8 + (size_t)m * 16 + (size_t)chol_table_entries(m) * 2 + 16;
}

static size_t trsm_smem(int m) {
    return (size_t)m * m * 8 + (size_t)m * 8 + (size_t)TRSM_ROWS * (m + 1) * 8 + 2 * TRSM_ROWS * 8;
}

static void set_smem(const void* fn, size_t bytes) {
    TRG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// Column-major n x m "A^T B" (m x m result, row-major) and "A W" products.
static void gram(Ctx& ctx, const double* A, const double* B, int64_t n, int m, double* G, int precision) {
    (void)precision;   // the Gram / Rayleigh-Ritz products are FP64 in every mode
    const int64_t rows = std::max<int64_t>(8, (n + ctx.sm_count - 1) / ctx.sm_count);
    const int64_t rows_c = std::min<int64_t>(rows, (int64_t)(96 * 1024 / (16 * m)));   // <= 96 KB staged
    const int nparts = (int)((n + rows_c - 1) / rows_c);
    ctx.ensure(ctx.f64_partial, (size_t)nparts * m * m * sizeof(double));
    const size_t smem = (size_t)rows_c * m * 2 * sizeof(double);
    static std::once_flag once;
    std::call_once(once, [] {
        TRG_CUDA(cudaFuncSetAttribute((const void*)k_gram_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      100 * 1024));
    });
    k_gram_partial<<<nparts, 256, smem, ctx.stream>>>(A, B, n, m, rows_c, ctx.f64_partial.as<double>(), A == B ? 1 : 0);
    TRG_LAUNCHED(ctx);
    k_gram_reduce<<<(m * m + 63) / 64, 64, 0, ctx.stream>>>(ctx.f64_partial.as<double>(), nparts, m, G);
    TRG_LAUNCHED(ctx);
}
static void times_small(Ctx& ctx, const double* A, const double* W, int64_t n, int m, double* C) {
    GemmDesc g;
    g.M = n; g.N = m; g.K = m;
    g.A.base = A; g.A.off_r = ctx.table({{n, 1}}); g.A.off_c = ctx.table({{m, n}}); g.A.c_fast = false;
    g.B.base = W; g.B.off_r = ctx.table({{m, 1}}); g.B.off_c = ctx.table({{m, m}}); g.B.c_fast = false;
    g.C = C; g.c_m = ctx.table({{n, 1}}); g.c_n = ctx.table({{m, n}}); g.beta = 0.0;
    gemm(ctx, g, TRG_FP64);
}

// Orthonormalise the columns of Y in place (two Cholesky-QR passes).  After
// one pass Q^T Q = I to about eps / min_j(d_j / G_jj) (the pivots of the
// column-normalised Gram matrix bound its conditioning); when the next step
// is another power step rather than a Rayleigh-Ritz step (`power_next`),
// which needs only a well-conditioned basis, a clean first pass with
// pivots above PASS2_PIVMIN is enough and the second pass is skipped.
constexpr double PASS2_PIVMIN = 1e-3;
static void orthonormalise(Ctx& ctx, double* Y, int64_t n, int m, double* G, double* L, int* flags,
                           int* nbad, uint64_t seed, uint64_t& salt, bool power_next = false) {
    double* pivmin = ctx.scal.as<double>() + SC_PIVMIN;
    double pm = 0.0;
    bool first_clean = true;    // the first pass needed no column repair
    for (int pass = 0; pass < 2; ++pass) {
        int attempt = 0;
        for (;; ++attempt) {
            TRG_CUDA(cudaMemsetAsync(flags, 0, (size_t)(m + 1) * sizeof(int), ctx.stream));
            k_col_normalize<<<m, 256, 0, ctx.stream>>>(Y, n, flags);
            TRG_LAUNCHED(ctx);
            gram(ctx, Y, Y, n, m, G, TRG_FP64);
            k_chol_flag<<<1, 256, chol_smem(m), ctx.stream>>>(G, L, m, pass == 0 ? 1e-8 : 1e-12, flags,
                                                                     nbad, pivmin);
            TRG_LAUNCHED(ctx);
            int hb = 0;
            TRG_CUDA(cudaMemcpyAsync(&hb, nbad, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
            TRG_CUDA(cudaMemcpyAsync(&pm, pivmin, sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
            TRG_CUDA(cudaStreamSynchronize(ctx.stream));
            if (hb == 0) break;
            if (pass == 0) first_clean = false;
            ctx.counters[4] += (uint64_t)hb;
            if (attempt >= 16) fail(TRG_ENUMERIC, "Cholesky-QR: could not complete a basis");
            dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)m);
            k_rand_cols<<<grid, 256, 0, ctx.stream>>>(Y, n, m, flags, seed, ++salt);
            TRG_LAUNCHED(ctx);
        }
        k_trsm_rows<<<(unsigned)((n + TRSM_ROWS - 1) / TRSM_ROWS), TRSM_THREADS, trsm_smem(m), ctx.stream>>>(Y, L, n,
                                                                                                          m);
        TRG_LAUNCHED(ctx);
        if (pass == 0 && power_next && first_clean && pm >= PASS2_PIVMIN) {
            ctx.counters[5] += 1;
            return;
        }
    }
}

int isometry(Ctx& ctx, const double* M, int64_t n, int dcut, double* U, std::vector<double>& lam,
             int step, int precision) {
    const int dn_paper = (int)std::min<int64_t>(n, dcut);
    // block of dn + p columns, at most the shared-memory block of the small
    // kernels (p shrinks there: Dcut 96 runs with p = 16)
    if (dn_paper >= MAX_M && dn_paper < n)
        fail(TRG_ENOTSUP, "isometry: Dcut above the supported block (111 kept vectors)");
    const int m = (int)std::min<int64_t>({n, (int64_t)dn_paper + std::max(1, ctx.cfg.oversample), (int64_t)MAX_M});
    static std::once_flag once;
    std::call_once(once, [] {
        set_smem((const void*)k_chol_flag, chol_smem(MAX_M));
        set_smem((const void*)k_trsm_rows, trsm_smem(MAX_M));
        set_smem((const void*)k_rr_fp32, rr32_smem(MAX_M));
        set_smem((const void*)k_rr_fp64, rr64_smem(MAX_M));
    });
    // buffers: Q, Y, Z, QW (n x m each); G, L, W (m x m); theta (m)
    ctx.ensure(ctx.eig, (size_t)(4 * n * m) * sizeof(double));
    ctx.ensure(ctx.eig_small, (size_t)(9 * m * m + 2 * m + 8) * sizeof(double));
    ctx.ensure(ctx.flags, (size_t)(m + 8) * sizeof(int));
    double* Q = ctx.eig.as<double>();
    double* Y = Q + n * m;
    double* Z = Y + n * m;
    double* QW = Z + n * m;
    double* G = ctx.eig_small.as<double>();
    double* L = G + m * m;
    double* W = L + m * m;
    double* theta = W + m * m;
    double* Hs = theta + 2 * m + 8;    // Rayleigh-Ritz scratch: symmetrised H, H W, Gram matrices
    double* T1 = Hs + m * m;
    double* G2 = T1 + m * m;
    double* Pm = G2 + m * m;           // X^T X of the refinement
    double* E = Pm + m * m;            // its correction
    double* Xb = E + m * m;            // a second basis buffer
    int* flags = ctx.flags.as<int>();
    int* nbad = flags + m;
    int* sweeps = flags + m + 2;   // [0] FP32 sweeps, [1] FP64 sweeps of the last Rayleigh-Ritz

    int* status = ctx.status.as<int>();
    double* res_slot = ctx.scal.as<double>() + SC_RES;
    const uint64_t seed = ctx.cfg.seed ^ (0xA24BAED4963EE407ull * (uint64_t)step);
    uint64_t salt = 0;

    {
        dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 64), (unsigned)m);
        k_rand_cols<<<grid, 256, 0, ctx.stream>>>(Q, n, m, nullptr, seed, salt);
        TRG_LAUNCHED(ctx);
    }
    // Y = M Q.  In split mode M is sliced once for all the products of this
    // solve (each product then slices only the n x m block Q).
    Gather gm;
    gm.base = M; gm.off_r = ctx.table({{n, n}}); gm.off_c = ctx.table({{n, 1}}); gm.c_fast = true;
    gm.c_identity = true;
    const uint16_t* m_slices = nullptr;
    const int* m_e = nullptr;
    if (precision == TRG_SPLIT_BF16) {
        const size_t sl = (size_t)slices_now(ctx) * split_rows_padded(ctx, n) * split_k_padded(n) * 2;
        const size_t eb = (size_t)split_rows_padded(ctx, n) * sizeof(int);
        ctx.ensure(ctx.eig_slices, sl + eb + 256);
        uint16_t* sp = ctx.eig_slices.as<uint16_t>();
        int* ep = (int*)(ctx.eig_slices.as<uint8_t>() + ((sl + 255) & ~(size_t)255));
        split_slice_operand(ctx, gm, n, n, sp, ep);
        m_slices = sp;
        m_e = ep;
    }
    auto apply_m = [&](double shift) {
        GemmDesc g;
        g.M = n; g.N = m; g.K = n;
        g.A = gm;
        g.a_slices = m_slices;
        g.a_e = m_e;
        g.B.base = Q; g.B.off_r = ctx.table({{n, 1}}); g.B.off_c = ctx.table({{m, n}}); g.B.c_fast = false;
        g.C = Y; g.c_m = ctx.table({{n, 1}}); g.c_n = ctx.table({{m, n}}); g.beta = 0.0;
        g.allow_ksplit = true;    // n / 128 tiles of 128 x m: K is split over the idle SMs
        gemm(ctx, g, precision);
        if (shift > 0.0) {
            const int64_t cnt = n * m;
            k_shift<<<(unsigned)std::min<int64_t>((cnt + 255) / 256, 4 * ctx.sm_count), 256, 0, ctx.stream>>>(
                Y, Q, shift, cnt);
            TRG_LAUNCHED(ctx);
        }
    };
    // Power steps apply M - sigma I with sigma = theta_m / 2 (a degree-one
    // Chebyshev filter of the unwanted interval [0, theta_m]): the
    // components outside the block shrink by (theta_m / 2) / (theta_dn -
    // theta_m / 2) a step instead of theta_m / theta_dn, at the cost of one
    // axpy.  theta_m comes from the last Rayleigh-Ritz step, or from the
    // previous solve of this direction before the first; a Rayleigh-Ritz
    // product is never shifted.
    auto shifted_rate = [](double th_m, double th_dn) {
        if (!(th_m > 0.0) || !(th_dn > th_m)) return 0.98;
        return std::min(std::max(0.5 * th_m / (th_dn - 0.5 * th_m), 0.05), 0.98);
    };
    // The number of products that reached the tolerance in the previous solve
    // of this direction (same sizes) is the plan: the spectra of successive
    // same-direction environments are close, and a random start needs about
    // as many products each time.  Without one, two plain power steps precede
    // a first, FP32-only Rayleigh-Ritz that measures the convergence rate.
    Ctx::EigHint& hint = ctx.eig_hint[step & 1];
    const bool have_hint = hint.n == n && hint.m == m && hint.precision == precision && hint.products > 0;
    double sigma = (have_hint && hint.theta_m > 0.0) ? 0.5 * hint.theta_m : 0.0;
    // the start block is followed by power steps unless the first step is a
    // Rayleigh-Ritz step (no plan and m = n)
    orthonormalise(ctx, Q, n, m, G, L, flags, nbad, seed, salt, have_hint || m < n);
    int applied = 0;                 // products of M in the span of Q
    if (!have_hint) {
        for (int pre = 0; pre < 2 && m < n; ++pre) {
            apply_m(0.0);
            std::swap(Q, Y);
            orthonormalise(ctx, Q, n, m, G, L, flags, nbad, seed, salt, pre == 0);
            ++applied;
        }
    }

    // Split products carry ~2^-(8S-1) relative error, which floors the Ritz
    // residual; f is insensitive to residuals far above that floor (1e-6
    // moves f by ~1e-12 on the Ising workloads), so stop at 2^-(8S-10).
    double tol = ctx.cfg.eig_tol;
    const int S_env = slices_now(ctx);   // the slices of this solve's M.Q products
    if (precision == TRG_SPLIT_BF16) tol = std::max(tol, std::ldexp(1.0, -(8 * S_env - 10)));
    std::vector<double> th((size_t)m);
    const int max_it = std::max(1, ctx.cfg.eig_max_iter);
    // Rayleigh-Ritz is the costly part (a one-SM Jacobi solve), so it is not
    // done after every product: the first one, in FP32 only, measures the
    // residual and the convergence rate rho ~ theta_m / theta_dn; the power
    // steps needed to reach the tolerance follow from rho and run without a
    // Rayleigh-Ritz; the next (full FP64) one normally converges.
    int pending = have_hint ? std::min(hint.products, 60) : 0;   // planned plain power steps
    int rr_done = have_hint ? 1 : 0;
    double prev_res = 0.0;
    int since_rr = 0;                // products applied since the previous Rayleigh-Ritz
    for (int it = 1; it <= max_it; ++it) {
        if (pending > 0) {
            apply_m(sigma);
            std::swap(Q, Y);
            orthonormalise(ctx, Q, n, m, G, L, flags, nbad, seed, salt, pending > 1);
            --pending;
            ++since_rr;
            ++applied;
            ctx.counters[0] += 1;
            continue;
        }
        // Y = M Q
        apply_m(0.0);
        // Rayleigh-Ritz
        gram(ctx, Q, Y, n, m, G, TRG_FP64);
        TRG_CUDA(cudaMemsetAsync(sweeps, 0, 2 * sizeof(int), ctx.stream));
        const int full = (rr_done > 0 || m == n) ? 1 : 0;
        // FP64 rotations stop at |h_pq| <= jtol sqrt(h_pp h_qq).  An unrotated
        // pair leaves at most m jtol theta_1 in a Ritz residual, so jtol =
        // 1e-3 tol keeps that far below the tolerance; with FP64 products
        // (tol 1e-12) it is 1e-13 (eigenvalues exact to ~1e-26 relative, the
        // vectors of pairs with a relative gap g to ~1e-13 / g), with split
        // products (tol 2^-(8S-10)) 2.4e-10 at S = 4.
        const double jtol = std::max(1e-13, 1e-3 * tol);
        {
            // the Rayleigh-Ritz solve of G = Q^T M Q into theta, W: FP32
            // Jacobi, then (see k_rr_fp32) FP64 products and FP64 Jacobi
            k_rr_fp32<<<1, 512, rr32_smem(m), ctx.stream>>>(G, m, Hs, W, sweeps);
            TRG_LAUNCHED(ctx);
            const double* Wj = W;    // the basis the FP64 sweeps start from
            if (full) {
                // Refine the FP32 eigenbasis in FP64 on many SMs: OA_STEPS
                // Ogita-Aishima steps (k_oa_step), then a Lowdin step; the
                // sweeps are left the pairs the steps could not separate.
                double* X = W;
                double* Xn = Xb;
                auto small = [&](auto kern, const double* a, const double* b, double* c) {
                    kern<<<m, 128, 0, ctx.stream>>>(a, b, m, c);
                    TRG_LAUNCHED(ctx);
                };
                for (int st = 0; st < OA_STEPS; ++st) {
                    small(k_small_nn, Hs, X, T1);      // H X
                    small(k_small_tn, X, T1, G2);      // S = X^T H X
                    small(k_small_tn, X, X, Pm);       // P = X^T X
                    k_oa_step<<<1, 256, 0, ctx.stream>>>(G2, Pm, m, E);
                    TRG_LAUNCHED(ctx);
                    small(k_small_apply, X, E, Xn);
                    std::swap(X, Xn);
                }
                small(k_small_tn, X, X, Pm);
                small(k_small_tn, Pm, Pm, T1);          // P P (P symmetric)
                k_lowdin<<<(m * m + 255) / 256, 256, 0, ctx.stream>>>(Pm, T1, m, E);
                TRG_LAUNCHED(ctx);
                small(k_small_apply, X, E, Xn);
                std::swap(X, Xn);
                small(k_small_nn, Hs, X, T1);
                small(k_small_tn, X, T1, G2);          // H' = X^T H X
                Wj = X;
            } else {
                // a rough Rayleigh-Ritz (no FP64 sweeps): W re-orthonormalised
                // by Cholesky-QR, theta the diagonal of H' = W^T H W
                k_small_tn<<<m, 128, 0, ctx.stream>>>(W, W, m, G2);
                TRG_LAUNCHED(ctx);
                k_chol_flag<<<1, 256, chol_smem(m), ctx.stream>>>(G2, L, m, 0.0, flags, nbad, nullptr);
                TRG_LAUNCHED(ctx);
                k_trsm_rows<<<(unsigned)((m + TRSM_ROWS - 1) / TRSM_ROWS), TRSM_THREADS, trsm_smem(m),
                              ctx.stream>>>(W, L, m, m);
                TRG_LAUNCHED(ctx);
                k_small_nn<<<m, 128, 0, ctx.stream>>>(Hs, W, m, T1);
                TRG_LAUNCHED(ctx);
                k_small_tn<<<m, 128, 0, ctx.stream>>>(W, T1, m, G2);
                TRG_LAUNCHED(ctx);
            }
            k_rr_fp64<<<1, 512, rr64_smem(m), ctx.stream>>>(G2, m, jtol, 60, theta, Wj, W, status, sweeps, full);
            TRG_LAUNCHED(ctx);
        }
        times_small(ctx, Y, W, n, m, Z);
        times_small(ctx, Q, W, n, m, QW);
        TRG_CUDA(cudaMemsetAsync(res_slot, 0, sizeof(double), ctx.stream));
        k_residual<<<dn_paper, 256, 0, ctx.stream>>>(Z, QW, theta, n, (unsigned long long*)res_slot);
        TRG_LAUNCHED(ctx);
        double res = 0.0;
        int hsw[2] = {0, 0};
        TRG_CUDA(cudaMemcpyAsync(th.data(), theta, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
        TRG_CUDA(cudaMemcpyAsync(&res, res_slot, sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
        TRG_CUDA(cudaMemcpyAsync(hsw, sweeps, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
        TRG_CUDA(cudaStreamSynchronize(ctx.stream));
        ctx.counters[0] += 1;
        ctx.counters[1] += 1;
        ctx.counters[2] += (uint64_t)hsw[0];
        ctx.counters[3] += (uint64_t)hsw[1];
        if (read_status(ctx) & ST_EIG_NOCONV) fail(TRG_ENUMERIC, "Rayleigh-Ritz Jacobi did not converge");
        if (!(th[0] > 0.0) || !std::isfinite(th[0])) fail(TRG_ENUMERIC, "environment has no positive eigenvalue");
        if ((res <= tol && full) || m == n) {
            {
                // The next plan is this solve's product count less the
                // products beyond what the tolerance needed (at the rate
                // theta_m / theta_dn), two kept spare: a plan that falls short
                // costs a second Rayleigh-Ritz, several times a product.
                const double r = sigma > 0.0
                                     ? shifted_rate(th[(size_t)m - 1], th[(size_t)dn_paper - 1])
                                     : std::min(std::max(th[(size_t)m - 1] / th[(size_t)dn_paper - 1], 0.05), 0.98);
                const int slack = (res > 0.0 && res < tol) ? (int)std::floor(std::log(tol / res) / -std::log(r)) : 0;
                hint.n = n; hint.m = m; hint.precision = precision;
                hint.products = std::max(1, applied - std::max(0, slack - 2));
                hint.theta_m = m < n ? th[(size_t)m - 1] : 0.0;
            }
            int dn = dn_paper;
            if (ctx.cfg.trunc == TRG_TRUNC_MULTIPLET && dn < n) {
                // split products separate exactly degenerate eigenvalues by up
                // to ~2^-(8S-12) lambda_1: treat smaller gaps as degenerate
                double gtol = ctx.cfg.gap_tol;
                if (precision == TRG_SPLIT_BF16)
                    gtol = std::max(gtol, std::ldexp(1.0, -(8 * S_env - 12)));
                while (dn > 1 && (th[(size_t)dn - 1] - th[(size_t)dn]) < gtol * th[0]) --dn;
            }
            lam.assign(th.begin(), th.begin() + dn);
            const int64_t tot = n * dn;
            k_to_isometry<<<(unsigned)((tot + 255) / 256), 256, 0, ctx.stream>>>(QW, n, dn, U);
            TRG_LAUNCHED(ctx);
            return dn;
        }
        // plan the power steps to the next Rayleigh-Ritz (shifted by the
        // fresh theta_m)
        sigma = (m < n && th[(size_t)m - 1] > 0.0) ? 0.5 * th[(size_t)m - 1] : 0.0;
        double rho = sigma > 0.0 ? shifted_rate(th[(size_t)m - 1], th[(size_t)dn_paper - 1])
                                 : th[(size_t)m - 1] / th[(size_t)dn_paper - 1];
        if (rr_done > 0 && prev_res > 0.0 && res > 0.0 && since_rr > 0)
            rho = std::max(rho, std::pow(res / prev_res, 1.0 / since_rr));
        rho = std::min(std::max(rho, 0.05), 0.98);
        int k = (res > tol) ? (int)std::ceil(std::log(tol / res) / std::log(rho)) : 0;
        pending = std::min(std::max(k, 0), 40);   // k - 1 needed after the product below, plus one spare
        ++rr_done;
        prev_res = res;
        since_rr = 1;
        // next block: orth(Y W) = orth(M Q W), same span as M Q
        ++applied;
        std::swap(Q, Z);
        orthonormalise(ctx, Q, n, m, G, L, flags, nbad, seed, salt, pending > 0);
    }
    fail(TRG_ENUMERIC, "subspace iteration did not converge");
}

}  // namespace trg
