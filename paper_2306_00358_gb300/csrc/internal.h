// Internal declarations of libtrg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "trg.h"

namespace trg {

// ------------------------------------------------------------ errors ----
struct Error {
    int status;
    std::string msg;
};

[[noreturn]] void fail(int status, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define TRG_CUDA(call) ::trg::check_cuda((call), #call, __FILE__, __LINE__)
// After every launch: catch configuration errors immediately.
#define TRG_LAUNCHED(ctx) do { (ctx).launches++; ::trg::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__); } while (0)

// Device status word bits (written by kernels, read by the host at sync points).
enum : int {
    ST_BAD_NORM = 1,       // norm <= 0, NaN or inf
    ST_BAD_TRACE = 2,      // trace <= 0 or NaN
    ST_EIG_NOCONV = 4,     // Jacobi sweeps exhausted
    ST_CHOL_BREAK = 8,     // Cholesky pivot could not be repaired
    ST_TIMEOUT = 16,       // a bounded device wait ran out
    ST_BOUNDS = 32         // a checked index fell outside its buffer (skipped)
};

// ------------------------------------------------------- device memory ----
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// A rank-4 strided view of FP64 device memory (element strides).
struct View4 {
    double* p;
    int64_t n[4];
    int64_t s[4];
};

// A rank-6 strided view (the cubic-lattice tensor t[x, x', y, y', z, z']).
struct View6 {
    double* p;
    int64_t n[6];
    int64_t s[6];
};

// A half-step between its isometry and its contraction: step k (odd = x,
// even = y), the tensor the x formulas see (T itself, or its rotation for a
// y step), the kept dimension and eigenvalues.
struct HalfPlan {
    int k = 0;
    bool xdir = true;
    int precision = 0;
    View4 r{};
    int64_t dn = 0;
    std::vector<double> lam;   // empty when U = I
};

struct Ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    trg_config cfg{};
    trg_alloc_fn alloc_fn = nullptr;
    trg_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    std::string last_error;
    uint64_t launches = 0;
    // split products: limit of the epilogue's wait for a finished accumulator
    // chunk in ns (0 = the kernel's default of 2 s); see trg_set_wait_limit
    unsigned long long acc_wait_ns = 0;

    // ---- solve state
    bool have_tensor = false;
    int Dx = 0, Dy = 0;
    int steps = 0;
    double beta = 0.0;
    Buf T, Tnext;          // current / next site tensor
    // a half-step split over ranks (trg_shard_begin .. trg_shard_finish)
    bool shard_pending = false;
    HalfPlan shard;
    // impure tensor (an observable inserted at one site), blocked alongside T
    bool have_impure = false;
    int model = -1, d0 = 0;    // model of the last trg_init_tensor (-1 after a raw init)
    double h_field = 0.0;
    Buf Timp, Timp_next, Timp_tmp;
    Buf M;                 // environment
    Buf U;                 // isometry (n x Dn row-major)
    Buf scal;              // device scalars, see SC_* below
    Buf status;            // device status word (int)
    std::vector<std::vector<double>> spectra;

    // ---- scratch
    Buf ws;                // contraction workspace (X1, X2 slices)
    Buf envP, envQ;        // environment intermediates
    Buf eig;               // subspace-iteration buffers
    Buf eig_small;         // m x m buffers
    Buf flags;             // per-column flags (int)
    Buf split_ws;          // split GEMM: exponents and BF16 slices of both operands
    Buf f64_partial;       // FP64 GEMM: split-K partial sums
    Buf ksplit_ws;         // split GEMM: split-K partial fixed-point sums
    Buf bslices;           // contraction: the D^7 product's B slices, shared by its j-blocks
    Buf cons_ef;           // exponent fields recorded by a producing product (two halves)
    Buf eig_slices;        // split mode: M sliced once per isometry solve
    Buf s3[10];            // cubic-lattice step: P1, P2, Ux, Uy, Mx, My, then A, W, C, D of the contraction
    std::map<std::string, Buf> tables;  // cached offset tables (and tile lists)
    std::map<std::string, int> list_len;   // entries of the cached tile lists

    // ---- phase timing
    bool prof = false;
    int phase = TRG_PHASE_ENV;
    struct PhaseAcc {
        double ms = 0.0, flops = 0.0, mma_flops = 0.0;
        uint64_t calls = 0;
        std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    } ph[TRG_PHASE_COUNT];
    std::vector<cudaEvent_t> event_pool;
    // diagnostics: subspace iterations, Rayleigh-Ritz solves, FP32 / FP64
    // Jacobi sweeps, Cholesky-QR column repairs
    uint64_t counters[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // Subspace iteration: power steps that reached the tolerance in the last
    // solve of each direction (x / y half-steps), used as the next plan.
    // plan of the next isometry of one direction: the products its
    // predecessor needed and that solve's smallest Ritz value theta_m
    struct EigHint { int64_t n = -1; int m = -1; int precision = -1; int products = 0; double theta_m = 0.0; };
    EigHint eig_hint[2];
    cudaEvent_t get_event();
    // Record the start of a timed region of phase p (no-op unless profiling).
    int region_begin(int p);
    void region_end(int token, double flops, double mma_flops);
    void collect_timings();

    void* raw_alloc(size_t bytes);
    void raw_free(void* p, size_t bytes);
    void ensure(Buf& b, size_t bytes);
    void release(Buf& b);
    const int64_t* table(const std::vector<std::pair<int64_t, int64_t>>& modes);
};

// Device scalar slots (doubles) in Ctx::scal.
enum : int {
    SC_LOGNORM = 0,   // sum_k 2^-k ln n_k
    SC_LN_N0 = 1,     // ln n0
    SC_NORM = 2,      // last max|T| (as the bits of a non-negative double)
    SC_TRACE = 3,     // last trace
    SC_RES = 4,       // max Ritz residual / lambda_1 (subspace iteration)
    SC_TRACE_IMP = 5, // last trace of the impure tensor
    SC_PIVMIN = 6,    // smallest pivot ratio d_j / G_jj of the last Cholesky-QR pass
    SC_COUNT = 8
};

// ------------------------------------------------------------ GEMM ----
// C[c_m[m] + c_n[n]] = sum_k A[a_m[m] + a_k[k]] * B[b_k[k] + b_n[n]]  (+ beta*C)
// Offset tables (int64, elements) make any strided multi-index layout a
// plain matrix for the kernels.
struct Gather {
    const double* base;
    const int64_t* off_r;   // row offsets   (A: m, B: k, C: m)
    const int64_t* off_c;   // col offsets   (A: k, B: n, C: n)
    bool c_fast;            // consecutive columns are adjacent in memory
    bool c_identity = false;   // off_c[k] == k: every row is one contiguous run
};
struct GemmDesc {
    int64_t M, N, K;
    Gather A, B;
    double* C;
    const int64_t* c_m;
    const int64_t* c_n;
    double beta = 0.0;      // 0: overwrite, 1: accumulate
    // Split mode, FP64 output through staging only: the product may split K
    // over several CTAs per tile when its tiles cannot fill the SMs (the
    // n x m products of the isometry); exact partial sums, deterministic.
    bool allow_ksplit = false;
    // The split epilogue may store without staging when consecutive rows are
    // adjacent in C and c_n[n + j] = c_n[n] + j c_col_stride inside each
    // aligned group of 32 columns.
    bool c_rows_fast = false;
    int64_t c_col_stride = 0;
    // Split mode only.  Producer side: record, for the product that will
    // consume C as its A operand, the largest FP64 exponent field of each of
    // its rows (row of element (m, n) = cons_m[m] + cons_n[n]) into cons_ef
    // (zeroed beforehand).  Consumer side: a_ef holds those fields for this
    // product's A rows, so the exponent pass over A is skipped.
    int* cons_ef = nullptr;
    const int64_t* cons_m = nullptr;
    const int64_t* cons_n = nullptr;
    const int* a_ef = nullptr;
    // Split mode, fused hand-over: instead of C, the producer writes the
    // consumer's BF16 A slices ([S][Mp][Kp], element (m, n) at consumer row
    // cons_m[m] + cons_n[n], column ck_m[m] + ck_n[n]) and their row
    // exponents (cs_e).  Valid when every consumer row lies in one 128 x 128
    // tile as rows_per_crow consecutive rows (a multiple of 32) times
    // cols_per_crow consecutive columns (32, 64 or 128); the consumer then
    // takes a_slices / a_e and skips slicing A.  Bit-identical to slicing C.
    uint16_t* cs_out = nullptr;
    int64_t cs_mp = 0, cs_kp = 0;
    int* cs_e = nullptr;
    const int64_t* ck_m = nullptr;
    const int64_t* ck_n = nullptr;
    int rows_per_crow = 0, cols_per_crow = 0;
    int64_t ck_stride = 0;  // consumer column of producer column n + 1 minus that of n, inside a row group
    const uint16_t* a_slices = nullptr;
    const int* a_e = nullptr;
    // C = A A^T (a Gram product): B is A read the other way (B(k, n) =
    // A(n, k)), M = N, and c_m, c_n address C for either index.  Split mode
    // slices A once for both operands (when their padded sizes agree),
    // computes only the tiles that reach the diagonal or above it, and
    // writes each element above the diagonal also at its mirror position,
    // so C is exactly symmetric; FP64 mode computes all of C.
    bool gram = false;
    // Split mode: B arrives sliced (split_slice_b), for a B that several
    // products share; the product then skips B's exponent and slicing passes.
    const uint16_t* b_slices = nullptr;
    const int* b_e = nullptr;
};
// Rows and columns of the padded slice arrays a split product of M rows and
// K columns reads for its A operand (the fused hand-over writes this layout).
int64_t split_rows_padded(const Ctx& ctx, int64_t M);
int64_t split_k_padded(int64_t K);
// Slice an A operand once for several split products (GemmDesc::a_slices / a_e).
void split_slice_operand(Ctx& ctx, const Gather& A, int64_t M, int64_t K, uint16_t* slices, int* e);
// Exponents (per column n) and BF16 slices of a K x N B operand in the layout
// a split product reads: [S][split_cols_padded(N)][split_k_padded(K)].
void split_slice_b(Ctx& ctx, const Gather& B, int64_t K, int64_t N, uint16_t* slices, int* e);
int64_t split_cols_padded(int64_t N);
void gemm(Ctx& ctx, const GemmDesc& g, int precision);
void gemm_f64(Ctx& ctx, const GemmDesc& g);

// Table helpers: enumerate all index tuples of `modes` (size, stride),
// first mode slowest, and return the device table of offsets.
std::vector<int64_t> build_table(const std::vector<std::pair<int64_t, int64_t>>& modes);

// ------------------------------------------------------ path pieces ----
// Arithmetic of half-step `step` on a tensor whose leg dimensions multiply to
// dd (Dx Dy; Dx Dy Dz on the cubic lattice).
int precision_for_step(const Ctx& ctx, int step, int64_t dd);
// BF16 slices of the split products issued now: env_slices during the
// environment and the isometry (when set), split_slices otherwise.
int slices_now(const Ctx& ctx);
void environment(Ctx& ctx, const View4& t, double* M, int precision);
// Tx = U . top . bottom . U (the upper tensor of the blocked pair is `top`,
// the lower one `bottom`; both the same tensor for the pure half-step).
// Only the output rows j in [j_begin, j_end) are computed (j_end < 0: all);
// `out` starts at j = j_out0 (its element (i, j, k, l) is at
// (j - j_out0) s[1] + ...), so a slab of j can be written on its own.
void contract(Ctx& ctx, const View4& top, const View4& bottom, const double* U, int64_t Dn, const View4& out,
              int precision, int64_t j_begin = 0, int64_t j_end = -1, int64_t j_out0 = 0);
// Returns Dn actually kept; lam (host) gets the kept eigenvalues.
int isometry(Ctx& ctx, const double* M, int64_t n, int dcut, double* U, std::vector<double>& lam,
             int step, int precision);

// Small kernels (small_kernels.cu)
// impure = 1: the observable inserted (Ising s, XY cos(theta), Potts [s = 0])
void launch_init_ising(Ctx& ctx, double* T, double beta, double h, int impure = 0);
void launch_init_xy(Ctx& ctx, double* T, int d0, double beta, double h, int impure = 0);
void launch_init_potts(Ctx& ctx, double* T, int q, double beta, double h, int impure = 0);
// x *= exp(-scal[slot]) (the impure tensor takes the pure tensor's ln n0)
void launch_scale_by_exp_neg(Ctx& ctx, double* x, int64_t n, const double* slot);
// x *= 1 / (the norm in scal[SC_NORM]), the pure tensor's last n_k
void launch_scale_by_last_norm(Ctx& ctx, double* x, int64_t n);
// y = (y + z) / 2
void launch_mean2(Ctx& ctx, double* y, const double* z, int64_t n);
// Tr T into a slot without the positivity check (an observable's trace may be <= 0)
void launch_trace_signed(Ctx& ctx, const double* T, int64_t Dx, int64_t Dy, double* slot);
void launch_maxabs(Ctx& ctx, const double* x, int64_t n, double* slot_bits);
void launch_normalise(Ctx& ctx, double* x, int64_t n, int step_weight_exp, bool initial);
void launch_trace(Ctx& ctx, const double* T, int64_t Dx, int64_t Dy, double* slot);
void launch_identity(Ctx& ctx, double* U, int64_t n);
void launch_fill(Ctx& ctx, double* x, int64_t n, double v);
void launch_copy_strided(Ctx& ctx, const View4& src, const View4& dst);

// Cubic lattice (path3d.cu, small_kernels.cu)
void launch_init_ising3d(Ctx& ctx, double* T, double beta, double h);
void launch_trace3(Ctx& ctx, const View6& t, double* slot);
// One z step of the view t into out (contiguous [X][X'][Y][Y'][z][z']);
// returns (Nx, Ny) and appends the kept eigenvalues of both isometries.
std::pair<int64_t, int64_t> step3(Ctx& ctx, const View6& t, int dcut, int step, double* out, int precision,
                                  std::vector<double>& lam_x, std::vector<double>& lam_y);

int read_status(Ctx& ctx);  // synchronises the stream
void trim_buffers(Ctx& ctx);  // free every solve buffer (engine.cu)

}  // namespace trg

struct trg_ctx : public trg::Ctx {};
