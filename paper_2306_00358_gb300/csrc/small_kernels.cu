// Small kernels of the path: initial tensors, max-abs normalisation with the
// FP64 log-norm accumulation, the periodic trace, identity isometry, strided
// copies.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace trg {

namespace {

// I_n(x) = sum_k (x/2)^(2k+n) / (k! (k+n)!), integer n (I_{-n} = I_n).
__device__ double bessel_i_series(int n, double x) {
    n = n < 0 ? -n : n;
    if (x == 0.0) return n == 0 ? 1.0 : 0.0;
    const double half = 0.5 * x;
    double term = 1.0;
    for (int i = 1; i <= n; ++i) term *= half / i;   // (x/2)^n / n!
    double total = term;
    for (int k = 1; k < 400; ++k) {
        term *= half * half / ((double)k * (double)(k + n));
        total += term;
        if (term < 1e-18 * total) break;
    }
    return total;
}

// Ising: T[i,j,k,l] = sum_s e^{beta h s} W[s,i] W[s,j] W[s,k] W[s,l],
// W = B^(1/2), B = [[e^b, e^-b], [e^-b, e^b]] (s = +1, -1), from B's
// eigenpairs 2cosh(b) on (1,1)/sqrt2 and 2sinh(b) on (1,-1)/sqrt2.
// impure: the spin s inserted at the site (factor s in the sum).
__global__ void k_init_ising(double* T, double beta, double h, int impure) {
    const int e = threadIdx.x;
    if (e >= 16) return;
    const int i = (e >> 3) & 1, j = (e >> 2) & 1, k = (e >> 1) & 1, l = e & 1;
    const double a = sqrt(2.0 * cosh(beta));
    const double b = beta > 0.0 ? sqrt(2.0 * sinh(beta)) : 0.0;
    const double w[2][2] = {{0.5 * (a + b), 0.5 * (a - b)}, {0.5 * (a - b), 0.5 * (a + b)}};
    double t = 0.0;
    for (int s = 0; s < 2; ++s) {
        const double spin = s == 0 ? 1.0 : -1.0;
        t += (impure ? spin : 1.0) * exp(beta * h * spin) * w[s][i] * w[s][j] * w[s][k] * w[s][l];
    }
    T[e] = t;
}

// Cubic-lattice Ising: T[x,x',y,y',z,z'] = sum_s e^{beta h s} W[s,x] W[s,x']
// W[s,y] W[s,y'] W[s,z] W[s,z'] (the 2D construction with two more legs).
__global__ void k_init_ising3d(double* T, double beta, double h) {
    const int e = threadIdx.x;
    if (e >= 64) return;
    const double a = sqrt(2.0 * cosh(beta));
    const double b = beta > 0.0 ? sqrt(2.0 * sinh(beta)) : 0.0;
    const double w[2][2] = {{0.5 * (a + b), 0.5 * (a - b)}, {0.5 * (a - b), 0.5 * (a + b)}};
    double t = 0.0;
    for (int s = 0; s < 2; ++s) {
        const double spin = s == 0 ? 1.0 : -1.0;
        double p = exp(beta * h * spin);
        for (int leg = 0; leg < 6; ++leg) p *= w[s][(e >> (5 - leg)) & 1];
        t += p;
    }
    T[e] = t;
}

// Tr T = sum_{x,y,z} T[x,x,y,y,z,z] of a strided rank-6 view (dims n, strides s)
__global__ void __launch_bounds__(256) k_trace3(const double* T, int64_t nx, int64_t ny, int64_t nz, int64_t sx,
                                                int64_t sy, int64_t sz, double* out, int* status) {
    double acc = 0.0;
    for (int64_t e = threadIdx.x; e < nx * ny * nz; e += 256) {
        const int64_t z = e % nz, y = (e / nz) % ny, x = e / nz / ny;
        acc += T[x * sx + y * sy + z * sz];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        *out = t;
        if (!(t > 0.0) || !isfinite(t)) atomicOr(status, ST_BAD_TRACE);
    }
}

// XY (character expansion, |n| <= nmax, index = n + nmax):
// T[nl,nu,nr,nd] = prod sqrt(I_n(beta)) * I_{nl+nu-nr-nd}(beta h)
// impure: cos(theta) inserted; cos = (e^{i theta} + e^{-i theta}) / 2 turns the
// site factor into (I_{div-1}(beta h) + I_{div+1}(beta h)) / 2.
__global__ void k_init_xy(double* T, int d0, double beta, double h, int impure) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)d0 * d0 * d0 * d0;
    if (e >= tot) return;
    const int nmax = d0 / 2;
    const int id = (int)(e % d0), ir = (int)((e / d0) % d0), iu = (int)((e / d0 / d0) % d0),
              il = (int)(e / d0 / d0 / d0);
    const int nl = il - nmax, nu = iu - nmax, nr = ir - nmax, nd = id - nmax;
    const double legs = sqrt(bessel_i_series(nl, beta)) * sqrt(bessel_i_series(nu, beta)) *
                        sqrt(bessel_i_series(nr, beta)) * sqrt(bessel_i_series(nd, beta));
    const int div = nl + nu - nr - nd;
    const double site = impure ? 0.5 * (bessel_i_series(div - 1, beta * h) + bessel_i_series(div + 1, beta * h))
                               : bessel_i_series(div, beta * h);
    T[e] = legs * site;
}

// q-state Potts (q <= 8): W = L L^T with W_ss' = e^beta (s = s'), 1 otherwise;
// T[i,j,k,l] = sum_s e^{beta h [s=0]} L[s,i] L[s,j] L[s,k] L[s,l].
// Each thread factors the small W itself (plain Cholesky, row by row).
// impure: [s = 0] inserted (only the s = 0 term).
__global__ void k_init_potts(double* T, int q, double beta, double h, int impure) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)q * q * q * q;
    if (e >= tot) return;
    double L[8][8];
    const double eb = exp(beta);
    for (int i = 0; i < q; ++i) {
        for (int j = 0; j <= i; ++j) {
            double a = (i == j) ? eb : 1.0;
            for (int k = 0; k < j; ++k) a -= L[i][k] * L[j][k];
            L[i][j] = (i == j) ? sqrt(a) : a / L[j][j];
        }
        for (int j = i + 1; j < q; ++j) L[i][j] = 0.0;
    }
    const int l = (int)(e % q), k = (int)((e / q) % q), j = (int)((e / q / q) % q), i = (int)(e / q / q / q);
    double t = 0.0;
    for (int s = 0; s < (impure ? 1 : q); ++s) {
        const double w = (s == 0) ? exp(beta * h) : 1.0;
        t += w * L[s][i] * L[s][j] * L[s][k] * L[s][l];
    }
    T[e] = t;
}

__global__ void __launch_bounds__(256) k_maxabs(const double* __restrict__ x, int64_t n,
                                                unsigned long long* out_bits) {
    double mx = 0.0;
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // 2-wide vector loads where aligned
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        const double2* x2 = reinterpret_cast<const double2*>(x);
        const int64_t n2 = n / 2;
        for (int64_t q = i; q < n2; q += stride) {
            const double2 v = x2[q];
            bad |= !(v.x == v.x) || !(v.y == v.y);
            mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
        }
        if (i == 0 && (n & 1)) { const double v = x[n - 1]; bad |= !(v == v); mx = fmax(mx, fabs(v)); }
    } else {
        for (int64_t q = i; q < n; q += stride) { const double v = x[q]; bad |= !(v == v); mx = fmax(mx, fabs(v)); }
    }
    if (bad) mx = NAN;   // NaN bits compare above +inf: the maximum carries it
    unsigned long long b = bad ? 0x7FF8000000000000ull : (unsigned long long)__double_as_longlong(mx);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, b, o);
        b = v > b ? v : b;
    }
    __shared__ unsigned long long red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) b = red[w] > b ? red[w] : b;
        atomicMax(out_bits, b);
    }
}

// x *= 1 / n, n read from the device slot.
__global__ void __launch_bounds__(256) k_scale_by_norm(double* __restrict__ x, int64_t n,
                                                       const unsigned long long* norm_bits) {
    const double nk = __longlong_as_double((long long)*norm_bits);
    if (!(nk > 0.0) || !isfinite(nk)) return;
    const double inv = 1.0 / nk;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride) x[q] *= inv;
}

// x *= exp(-v), v read from a device slot.
__global__ void __launch_bounds__(256) k_scale_by_exp_neg(double* __restrict__ x, int64_t n, const double* v) {
    const double f = exp(-*v);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride) x[q] *= f;
}

__global__ void __launch_bounds__(256) k_mean2(double* __restrict__ y, const double* __restrict__ z, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += stride) y[q] = 0.5 * (y[q] + z[q]);
}

// lognorm += 2^-k ln n_k   (k = 0: ln n0 slot instead)
__global__ void k_lognorm(double* scal, int k, int* status) {
    const double nk = __longlong_as_double((long long)*(const unsigned long long*)(scal + SC_NORM));
    if (!(nk > 0.0) || !isfinite(nk)) { atomicOr(status, ST_BAD_NORM); return; }
    if (k == 0) scal[SC_LN_N0] = log(nk);
    else scal[SC_LOGNORM] += ldexp(log(nk), -k);
}

// Tr T = sum_{i,j} T[i, j, i, j]
__global__ void __launch_bounds__(256) k_trace(const double* T, int64_t Dx, int64_t Dy, double* out, int* status,
                                               int check) {
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < Dx * Dy; e += 256) {
        const int64_t i = e / Dy, j = e % Dy;
        s += T[((i * Dy + j) * Dx + i) * Dy + j];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        *out = t;
        if (check && (!(t > 0.0) || !isfinite(t))) atomicOr(status, ST_BAD_TRACE);
    }
}

__global__ void k_identity(double* U, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n * n) U[e] = (e / n == e % n) ? 1.0 : 0.0;
}

__global__ void k_fill(double* x, int64_t n, double v) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) x[e] = v;
}

__global__ void k_copy4(View4 src, View4 dst) {
    const int64_t tot = src.n[0] * src.n[1] * src.n[2] * src.n[3];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e;
        const int64_t i3 = r % src.n[3]; r /= src.n[3];
        const int64_t i2 = r % src.n[2]; r /= src.n[2];
        const int64_t i1 = r % src.n[1]; r /= src.n[1];
        const int64_t i0 = r;
        dst.p[i0 * dst.s[0] + i1 * dst.s[1] + i2 * dst.s[2] + i3 * dst.s[3]] =
            src.p[i0 * src.s[0] + i1 * src.s[1] + i2 * src.s[2] + i3 * src.s[3]];
    }
}

unsigned grid_for(const Ctx& ctx, int64_t n, int threads) {
    const int64_t want = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)ctx.sm_count * 8;
    return (unsigned)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace

void launch_init_ising(Ctx& ctx, double* T, double beta, double h, int impure) {
    k_init_ising<<<1, 32, 0, ctx.stream>>>(T, beta, h, impure);
    TRG_LAUNCHED(ctx);
}

void launch_init_xy(Ctx& ctx, double* T, int d0, double beta, double h, int impure) {
    const int64_t tot = (int64_t)d0 * d0 * d0 * d0;
    k_init_xy<<<(unsigned)((tot + 127) / 128), 128, 0, ctx.stream>>>(T, d0, beta, h, impure);
    TRG_LAUNCHED(ctx);
}

void launch_init_potts(Ctx& ctx, double* T, int q, double beta, double h, int impure) {
    const int64_t tot = (int64_t)q * q * q * q;
    k_init_potts<<<(unsigned)((tot + 127) / 128), 128, 0, ctx.stream>>>(T, q, beta, h, impure);
    TRG_LAUNCHED(ctx);
}

void launch_maxabs(Ctx& ctx, const double* x, int64_t n, double* slot_bits) {
    TRG_CUDA(cudaMemsetAsync(slot_bits, 0, sizeof(double), ctx.stream));
    k_maxabs<<<grid_for(ctx, n / 2 + 1, 256), 256, 0, ctx.stream>>>(x, n, (unsigned long long*)slot_bits);
    TRG_LAUNCHED(ctx);
}

// T /= max|T|; accumulate the log-norm with weight 2^-k (k = 0: ln n0).
void launch_normalise(Ctx& ctx, double* x, int64_t n, int k, bool initial) {
    double* scal = ctx.scal.as<double>();
    launch_maxabs(ctx, x, n, scal + SC_NORM);
    k_scale_by_norm<<<grid_for(ctx, n, 256), 256, 0, ctx.stream>>>(x, n, (const unsigned long long*)(scal + SC_NORM));
    TRG_LAUNCHED(ctx);
    k_lognorm<<<1, 1, 0, ctx.stream>>>(scal, initial ? 0 : k, ctx.status.as<int>());
    TRG_LAUNCHED(ctx);
}

void launch_init_ising3d(Ctx& ctx, double* T, double beta, double h) {
    k_init_ising3d<<<1, 64, 0, ctx.stream>>>(T, beta, h);
    TRG_LAUNCHED(ctx);
}

void launch_trace3(Ctx& ctx, const View6& t, double* slot) {
    k_trace3<<<1, 256, 0, ctx.stream>>>(t.p, t.n[0], t.n[2], t.n[4], t.s[0] + t.s[1], t.s[2] + t.s[3],
                                        t.s[4] + t.s[5], slot, ctx.status.as<int>());
    TRG_LAUNCHED(ctx);
}

void launch_trace(Ctx& ctx, const double* T, int64_t Dx, int64_t Dy, double* slot) {
    k_trace<<<1, 256, 0, ctx.stream>>>(T, Dx, Dy, slot, ctx.status.as<int>(), 1);
    TRG_LAUNCHED(ctx);
}

void launch_trace_signed(Ctx& ctx, const double* T, int64_t Dx, int64_t Dy, double* slot) {
    k_trace<<<1, 256, 0, ctx.stream>>>(T, Dx, Dy, slot, ctx.status.as<int>(), 0);
    TRG_LAUNCHED(ctx);
}

void launch_scale_by_exp_neg(Ctx& ctx, double* x, int64_t n, const double* slot) {
    k_scale_by_exp_neg<<<grid_for(ctx, n, 256), 256, 0, ctx.stream>>>(x, n, slot);
    TRG_LAUNCHED(ctx);
}

void launch_scale_by_last_norm(Ctx& ctx, double* x, int64_t n) {
    k_scale_by_norm<<<grid_for(ctx, n, 256), 256, 0, ctx.stream>>>(
        x, n, (const unsigned long long*)(ctx.scal.as<double>() + SC_NORM));
    TRG_LAUNCHED(ctx);
}

void launch_mean2(Ctx& ctx, double* y, const double* z, int64_t n) {
    k_mean2<<<grid_for(ctx, n, 256), 256, 0, ctx.stream>>>(y, z, n);
    TRG_LAUNCHED(ctx);
}

void launch_identity(Ctx& ctx, double* U, int64_t n) {
    k_identity<<<(unsigned)((n * n + 255) / 256), 256, 0, ctx.stream>>>(U, n);
    TRG_LAUNCHED(ctx);
}

void launch_fill(Ctx& ctx, double* x, int64_t n, double v) {
    if (n <= 0) return;
    k_fill<<<(unsigned)((n + 255) / 256), 256, 0, ctx.stream>>>(x, n, v);
    TRG_LAUNCHED(ctx);
}

void launch_copy_strided(Ctx& ctx, const View4& src, const View4& dst) {
    const int64_t tot = src.n[0] * src.n[1] * src.n[2] * src.n[3];
    if (tot <= 0) return;
    k_copy4<<<grid_for(ctx, tot, 256), 256, 0, ctx.stream>>>(src, dst);
    TRG_LAUNCHED(ctx);
}

int read_status(Ctx& ctx) {
    int st = 0;
    TRG_CUDA(cudaMemcpyAsync(&st, ctx.status.p, sizeof(int), cudaMemcpyDeviceToHost, ctx.stream));
    TRG_CUDA(cudaStreamSynchronize(ctx.stream));
    return st;
}

}  // namespace trg
