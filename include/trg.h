/*
 * trg.h -- C ABI of the GB300-native HOTRG coarse-graining library (libtrg).
 *
 * The library computes the free energy of 2D classical spin models with the
 * higher-order tensor renormalisation group step of arXiv:2306.00358
 * ("GPU-Acceleration of Tensor Renormalization with PyTorch using CUDA"),
 * Sec. 2: the coarse-graining listing (environment einsum, SVD isometry,
 * U.T.T.U contraction, normalisation) and Fig. 1 (two directional blockings
 * per iteration, periodic trace after N iterations).  Every step runs in the
 * library's own CUDA kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions
 *  - Every function returns a trg_status (0 = TRG_OK).  On failure the
 *    context keeps its previous state where possible and trg_last_error()
 *    gives a one-line reason.
 *  - Site tensors are FP64, row-major, legs (left, up, right, down) with
 *    shape (Dx, Dy, Dx, Dy): element T[l][u][r][d] sits at
 *    ((l*Dy + u)*Dx + r)*Dy + d.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory on the context's device.  The library never takes
 *    ownership of caller buffers; it copies what it keeps.
 *  - All device work of a context is ordered on one CUDA stream (the
 *    default stream unless trg_set_stream is called).  Calls on one context
 *    are not thread-safe; different contexts are independent.
 *  - Device memory the context needs is allocated through the allocator
 *    hook (cudaMalloc by default) and freed by trg_destroy.
 */
#ifndef TRG_H
#define TRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- status ----- */
typedef enum trg_status {
    TRG_OK = 0,
    TRG_EINVAL = 1,    /* bad argument (NULL, out-of-range size, non-finite beta, ...) */
    TRG_ESTATE = 2,    /* call out of order (e.g. coarse-grain before init) */
    TRG_ENOMEM = 3,    /* allocation failed or exceeds the configured budget */
    TRG_ENUMERIC = 4,  /* non-positive / NaN norm or trace, eigensolver not converged */
    TRG_ETIMEOUT = 5,  /* a bounded device-side wait ran out */
    TRG_ECUDA = 6,     /* a CUDA runtime call failed (see trg_last_error) */
    TRG_ENOTSUP = 7,   /* feature not available on this device / build */
    TRG_EAGAIN = 8,    /* serving: the request has not finished yet */
    TRG_ECANCELED = 9  /* serving: the request was cancelled before it started */
} trg_status;

typedef enum trg_model { TRG_ISING = 0, TRG_XY = 1, TRG_POTTS = 2 } trg_model;

/* Arithmetic of the contractions (environment, U.T.T.U, M.Q products).
 * Cholesky-QR, the Rayleigh-Ritz eigensolve, normalisation and the log-norm
 * accumulation are FP64 in every mode. */
typedef enum trg_precision {
    TRG_FP64 = 0,        /* plain FP64 on the CUDA cores */
    TRG_SPLIT_BF16 = 1   /* FP64 operands cut into BF16 slices, exact FP32
                            partial sums on tcgen05 tensor cores, summed wide */
} trg_precision;

typedef enum trg_trunc {
    TRG_TRUNC_PAPER = 0,     /* keep min(Dx^2, Dcut) vectors, as the SVD helper does */
    TRG_TRUNC_MULTIPLET = 1  /* lower Dn so the cut never splits a degenerate multiplet */
} trg_trunc;

typedef struct trg_config {
    int precision;           /* trg_precision (default TRG_FP64) */
    int split_slices;        /* BF16 slices per operand in TRG_SPLIT_BF16, 2..5 (default 4);
                                the contraction products use it (see env_slices) */
    int split_from_step;     /* in TRG_SPLIT_BF16 the half-steps k <= split_from_step run in FP64
                                (default 0) */
    int trunc;               /* trg_trunc (default TRG_TRUNC_PAPER) */
    double gap_tol;          /* multiplet gap, relative to lambda_1 (default 1e-6; in
                                TRG_SPLIT_BF16 at least 2^-(8*S-12), S = the env slices) */
    int oversample;          /* subspace-iteration oversampling p (default 24; at most 112 - Dcut) */
    double eig_tol;          /* Ritz residual tolerance relative to lambda_1 (default 1e-12; in
                                TRG_SPLIT_BF16 at least 2^-(8*S-10), S = the env slices) */
    int eig_max_iter;        /* subspace iterations before TRG_ENUMERIC (default 300) */
    uint64_t seed;           /* seed of the start block of the subspace iteration */
    size_t workspace_bytes;  /* bound on the contraction workspace (0 = 4 GiB) */
    int mma_pairs;           /* TRG_SPLIT_BF16: 1 (default) runs products with more than 128
                                rows on CTA pairs (256-row tiles, cta_group::2: every
                                tensor-core instruction drives two SMs, each staging half
                                of B); 0 keeps one CTA per 128 x 128 tile.  Results are
                                identical either way. */
    int fused_slices;        /* TRG_SPLIT_BF16, bond dimensions 32, 64 or 128: 1 (default)
                                lets the D^7 contraction product write the last product's
                                BF16 operand slices directly (no FP64 intermediate, no
                                slicing pass); 2 also hands the first product over as
                                slices; 0 always goes through FP64.  Results are identical
                                in all three. */
    int fp64_max_dd;         /* TRG_SPLIT_BF16: half-steps on a tensor with Dx*Dy <= fp64_max_dd
                                (Dx*Dy*Dz on the cubic lattice) run in FP64 (default 16: the
                                first three half-steps of a model's solve, bond dimensions 2
                                to 4, whose norms weigh 1/2, 1/4 and 1/8 in ln Z / V; in
                                FP64 they cost nothing and keep the split path's error in f
                                several times lower) */
    int env_slices;          /* TRG_SPLIT_BF16: BF16 slices of the environment products and of
                                the isometry's M.Q products, 2..5; 0 (default) = split_slices.
                                The isometry's tolerances above then follow env_slices. */
    int autotune;            /* TRG_SPLIT_BF16: 1 (default) times the launch choices (one CTA or
                                a CTA pair per tile, tile-group width) on the first product of
                                each shape above ~1e9 multiply-adds and keeps the fastest in a
                                process-wide table; 0 takes the model choice.  Every choice
                                gives identical bits. */
} trg_config;

typedef struct trg_ctx trg_ctx;

/* Allocator hook: alloc returns device memory of `bytes` usable on `stream`
 * (NULL on failure); free releases it.  `user` is passed back unchanged. */
typedef void* (*trg_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*trg_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Fill *cfg with the defaults listed above. */
int trg_config_default(trg_config* cfg);

/* Create a context on CUDA device `device`: the state of one free-energy
 * solve of Sec. 2 (the site tensor, its norms and the coarse-graining
 * settings; the paper keeps the same state in Python variables between the
 * calls of its coarse-graining listing).  cfg may be NULL (defaults).
 * *out receives the handle (NULL on failure).  Returns TRG_EINVAL for a bad
 * device index or config, TRG_ENOTSUP if the device is not sm_103 (GB300),
 * TRG_ENOMEM / TRG_ECUDA if its two small device buffers cannot be made. */
int trg_create(trg_ctx** out, int device, const trg_config* cfg);

/* Destroy a context and free all device memory it allocated. NULL is a no-op. */
int trg_destroy(trg_ctx* ctx);

/* Order all later device work of ctx on `stream` (a cudaStream_t). */
int trg_set_stream(trg_ctx* ctx, void* stream);

/* Route the context's device allocations through alloc/free.  Must be
 * called before the first allocation (right after trg_create). */
int trg_set_allocator(trg_ctx* ctx, trg_alloc_fn alloc, trg_free_fn free_fn, void* user);

/* Limit, in ns, of one bounded device wait of the split products: the
 * epilogue's wait for a finished accumulator chunk (0 = the default, 2 s).
 * Every other wait keeps its 2 s limit.  When a wait runs out, the kernel
 * records a timeout, stops issuing, waits (bounded) for its own copies and
 * tensor-core work in flight, frees its tensor memory and returns; the call
 * that launched it returns TRG_ETIMEOUT (trg_gemm clears the flag at its
 * next call).  A limit below the time of one 512-deep chunk of products
 * (microseconds) makes that path run; it exists for tests of it. */
int trg_set_wait_limit(trg_ctx* ctx, uint64_t acc_wait_ns);

/* Change the precision mode for later half-steps (see trg_config).  The
 * paper does not state the arithmetic of its contractions (PyTorch float64
 * tensors, Sec. 3 and the appendix); TRG_FP64 is that reading, and
 * TRG_SPLIT_BF16 with split_slices BF16 slices per operand is this library's
 * tensor-core form of the same products.  split_from_step keeps the
 * half-steps k <= split_from_step in FP64.  Invalid values: TRG_EINVAL and
 * the context keeps its settings. */
int trg_set_precision(trg_ctx* ctx, int precision, int split_slices, int split_from_step);

/* -------------------------------------------------------- full solve ---- */
/*
 * Build the initial site tensor T0 on the device and reset the solve.
 *   TRG_ISING: D0 must be 2.  T[i,j,k,l] = sum_s e^{beta h s} W_si W_sj W_sk W_sl
 *              with W the symmetric square root of B_ss' = e^{beta s s'}
 *              (H = -sum s s' - h sum s).
 *   TRG_XY:    D0 odd (charges |n| <= (D0-1)/2);
 *              T = prod_legs sqrt(I_n(beta)) * I_{n_l+n_u-n_r-n_d}(beta h).
 *   TRG_POTTS: D0 = q (2..8) states (Sec. 3.3): W_ss' = e^beta if s = s' else 1,
 *              W = L L^T (Cholesky), T = sum_s e^{beta h [s=0]} L_si L_sj L_sk L_sl.
 * beta must be > 0 and finite, h finite.  T0 is divided by n0 = max|T0|.
 */
int trg_init_tensor(trg_ctx* ctx, int model, double beta, double h, int D0);

/* Same, from a caller tensor (host, shape (Dx,Dy,Dx,Dy), copied). */
int trg_init_tensor_raw(trg_ctx* ctx, const double* T_host, int Dx, int Dy, double beta);

/*
 * Impure tensor: the initial tensor with an observable O inserted at its
 * site, coarse-grained alongside T so that an expectation value can be read
 * at the end (the magnetization study of Sec. 3.1 inserts one to measure M
 * of the XY model).  Every half-step blocks it with the pure tensor in both
 * places of the pair with the pure tensor's isometry, takes the mean of the
 * two, and divides it by the pure tensor's n_k; after N half-steps
 * Tr T_imp / Tr T is the mean of <O> over the 2^N sites.  It triples the
 * contraction work of a half-step.
 *
 * trg_init_impure: the model's own observable, after trg_init_tensor and
 *   before the first half-step (else TRG_ESTATE): Ising O = s; XY O =
 *   cos(theta) (site factor (I_{div-1}(beta h) + I_{div+1}(beta h)) / 2);
 *   Potts O = [s = 0].
 * trg_init_impure_raw: any impure tensor (host, same shape as the initial
 *   tensor, copied before return); it is divided by the same n0 as T.
 * A later trg_init_tensor / _raw drops the impure tensor.
 */
int trg_init_impure(trg_ctx* ctx);
int trg_init_impure_raw(trg_ctx* ctx, const double* Timp_host);

/* <O> = Tr T_imp / Tr T of the current tensors (TRG_ESTATE without an impure
 * tensor, TRG_ENUMERIC if Tr T <= 0). */
int trg_expectation(trg_ctx* ctx, double* value_out);

/*
 * Run `nsteps` directional blockings (half-steps), continuing the x/y
 * alternation of earlier calls (x first).  Each half-step: environment M of
 * two stacked tensors, isometry U = leading min(Dx^2, Dcut) eigenvectors of M,
 * Tx = U.T.T.U, then T /= n_k = max|T| and lognorm += 2^-k ln n_k.
 * Dcut >= 1.  Returns TRG_ENUMERIC on a non-positive or NaN norm, or if the
 * eigensolver does not converge.
 */
int trg_coarse_grain(trg_ctx* ctx, int Dcut, int nsteps);

/*
 * Close the current tensor with periodic boundary conditions and return
 * f = -(ln Z / V) / beta and (if lnz_per_site != NULL) ln Z / V, where
 * ln Z / V = ln n0 + sum_k 2^-k ln n_k + 2^-N ln Tr T_N, Tr T = sum_ij T[i,j,i,j]
 * (Sec. 2 and Fig. 1 for the trace, Sec. 3.2 for f = -T ln Z).
 */
int trg_free_energy(trg_ctx* ctx, double* f_out, double* lnz_per_site);

/* ------------------------------------------- one half-step over ranks */
/*
 * A half-step whose contraction is split over several processes (one GPU
 * each).  The paper runs its contractions on one or two GPUs and reports the
 * two-GPU speed-up (Sec. 3.1, Sec. 4) without the partition; here the
 * contraction of Sec. 2 (Tx[i,j,k,l] = sum U[a,b,i] t[b,j,d,c] t[a,c,e,l]
 * U[e,d,k]) is split over its free index j, the up leg of the upper tensor,
 * whose slices are independent.  Every rank holds the same tensor and runs
 * the environment and the isometry itself (same inputs and kernels, so the
 * same U on every rank), computes the output rows j in [j_begin, j_end), and
 * the caller exchanges the slabs (an all-gather) before trg_shard_finish.
 * For a y half-step the formulas see the rotated tensor (as in
 * trg_coarse_grain), so j is then its left leg.
 *
 * trg_shard_extent: *nj_out = the extent of j for the next half-step (Dy for
 *   an x step, Dx for a y step).
 * trg_shard_begin: environment, isometry (*dn_out = Dn), and the output rows
 *   j_begin <= j < j_end written to slab_dev (device, caller-owned, capacity
 *   slab_cap doubles >= (j_end - j_begin) * Dn * Dn * nj) as
 *   S[jj][i][k][l] = O[i, j_begin + jj, k, l], O of shape (Dn, nj, Dn, nj).
 *   An empty range (j_begin == j_end) only runs the first two parts.  Size
 *   the slab for Dn <= min(Dx^2, Dcut) (Dx the extent of the blocked legs);
 *   a slab that proves too small gives TRG_EINVAL.  TRG_ESTATE before
 *   init or while a split half-step is open; TRG_ENOTSUP with an impure
 *   tensor.
 * trg_shard_finish: gathered_dev (device) holds G[j][i][k][l] = O[i,j,k,l]
 *   for j < nj in rows of Dn * Dn * nj doubles (j_rows >= nj rows; rows past
 *   nj are ignored padding): the slabs of all ranks in j order.  It places O
 *   as the coarse tensor, normalises it and closes the half-step exactly as
 *   trg_coarse_grain would; the result is identical to an unsplit half-step.
 * Between the two calls the context's tensor must not change (no other call
 * that advances or resets the solve).
 */
int trg_shard_extent(trg_ctx* ctx, int* nj_out);
int trg_shard_begin(trg_ctx* ctx, int Dcut, int j_begin, int j_end, double* slab_dev, size_t slab_cap,
                    int* dn_out);
int trg_shard_finish(trg_ctx* ctx, const double* gathered_dev, int j_rows);

/* ------------------------------------------------------- cubic lattice */
/*
 * A whole solve of the Ising model on the cubic lattice, the direction the
 * paper leaves to future work (Sec. 1, Sec. 4), blocked as the 2D variant of
 * Sec. 2 with a third pair of legs.  The site tensor is
 *   T[x,x',y,y',z,z'] = sum_s e^{beta h s} W[s,x] W[s,x'] W[s,y] W[s,y'] W[s,z] W[s,z'],
 * W the symmetric square root of the bond matrix (D0 = 2).  Each step stacks
 * two tensors along z; the left/right leg pairs are truncated to
 * Nx = min(Dx^2, Dcut) by one isometry from the environment of the two left
 * legs (Gram matrix of the stacked pair over its other legs), the
 * front/back pairs likewise by one from the two front legs; then the axes
 * rotate so that the steps block z, x, y, z, ...  Normalisation by max|T|
 * after each step; ln Z / V = ln n0 + sum_k 2^-k ln n_k + 2^-N ln Tr T_N,
 * Tr T = sum T[x,x,y,y,z,z], for the periodic Lx x Ly x Lz lattice with
 * Lz = 2^ceil(N/3), Lx = 2^ceil((N-1)/3), Ly = 2^floor(N/3).
 * model: TRG_ISING only (else TRG_ENOTSUP); beta > 0 and finite, h finite,
 * Dcut >= 1, 0 <= nsteps <= 300 (else TRG_EINVAL).  The precision settings
 * of the context apply.  Outputs f = -(ln Z / V) / beta and ln Z / V (either
 * pointer may be NULL, not both).  The kept eigenvalues of step k's two
 * isometries are available as trg_get_spectrum steps 2k-1 (x) and 2k (y).
 * The context's 2D state is cleared (trg_coarse_grain then needs a new
 * trg_init_tensor).  Device memory: about 8 (Dx^2 Dy^4 Dz^2 + 3 Dcut D^6)
 * bytes for the largest step.  Errors: TRG_ENOMEM, TRG_ENUMERIC (norm or
 * trace not positive, eigensolver), TRG_ECUDA.
 */
int trg_solve3d(trg_ctx* ctx, int model, double beta, double h, int Dcut, int nsteps, double* f_out,
                double* lnz_per_site);

/* Kept eigenvalues of M at half-step `step` (1-based): the squared singular
 * values that the SVD helper of the coarse-graining listing (Sec. 2) ranks
 * to truncate, M being a Gram matrix.  Descending, written to
 * out[0..min(cap,n)-1] (host, caller-owned; out may be NULL to query n);
 * *n_out = number kept.  Untruncated steps (U = I) report n_out = 0.
 * TRG_EINVAL for a step outside 1..half-steps done. */
int trg_get_spectrum(trg_ctx* ctx, int step, double* out, int cap, int* n_out);

/* Current solve state: half-steps done, (Dx, Dy), and sum_k 2^-k ln n_k. */
int trg_get_state(trg_ctx* ctx, int* steps, int* Dx, int* Dy, double* lognorm);

/* Copy the current (normalised) tensor to host memory of cap doubles. */
int trg_get_tensor(trg_ctx* ctx, double* T_host, size_t cap);

/* ------------------------------------------- components (device buffers) */
/*
 * Environment of the x half-step (Sec. 2, the environment einsum of the
 * coarse-graining listing):
 *   M[(i,j),(k,l)] = sum t[j,a,b,e] t[i,e,c,d] t[l,a,b,f] t[k,f,c,d],
 * t: device, (Dx,Dy,Dx,Dy) row-major; M: device, (Dx*Dx) x (Dx*Dx) row-major.
 * Uses the context's precision mode and workspace.
 */
int trg_environment(trg_ctx* ctx, const double* t_dev, int Dx, int Dy, double* M_dev);

/*
 * Isometry from a symmetric PSD environment (the SVD helper of the listing:
 * leading Dn = min(n, Dcut) left singular vectors of M, n = Dx*Dx; with
 * TRG_TRUNC_MULTIPLET Dn may be lower).  M_dev: device, n x n row-major.
 * U_dev: device, n x Dn row-major (capacity n*min(n,Dcut) doubles);
 * lam_host: host, capacity min(n,Dcut) (nullable); *dn_out = Dn.
 * If Dn == n the identity is returned and lam is not computed (*dn_out = n,
 * lam_host untouched).
 */
int trg_isometry(trg_ctx* ctx, const double* M_dev, int n, int Dcut,
                 double* U_dev, double* lam_host, int* dn_out);

/*
 * Contraction of the x half-step (Sec. 2, the U.T.T.U einsum):
 *   Tx[i,j,k,l] = sum U[a,b,i] t[b,j,d,c] t[a,c,e,l] U[e,d,k],
 * t: device (Dx,Dy,Dx,Dy); U: device (Dx,Dx,Dn); Tx: device (Dn,Dy,Dn,Dy).
 * The D^5 intermediates are never formed whole: the free index j is
 * processed in slices sized to the workspace bound.
 */
int trg_contract(trg_ctx* ctx, const double* t_dev, const double* U_dev,
                 int Dx, int Dy, int Dn, double* Tx_dev);

/*
 * Plain matrix product C = A B in the context's precision mode (the kernel
 * every contraction above is built on).  Row-major device matrices:
 * A (M x K, leading dimension lda >= K), B (K x N, ldb >= N),
 * C (M x N, ldc >= N); C is overwritten.  M, N, K >= 1; in TRG_SPLIT_BF16
 * mode K <= 131072.
 */
int trg_gemm(trg_ctx* ctx, int M, int N, int K, const double* A_dev, int lda, const double* B_dev, int ldb,
             double* C_dev, int ldc);

/*
 * Allocation-free split-precision product C = A B (no counterpart in the
 * paper; an addition for callers that must not allocate device memory while
 * they run -- e.g. a serving process that handed all memory to its own pool
 * at start-up, or code where a cudaMalloc would synchronise the device -- and
 * for callers that hold no context).
 *
 * Same arithmetic and layouts as trg_gemm in TRG_SPLIT_BF16 mode with
 * `slices` BF16 slices (2..5), on the CURRENT CUDA device and on `stream`
 * (a cudaStream_t, NULL = default stream).  It calls no cudaMalloc, cudaFree
 * or other allocating routine: its scratch (offset tables, exponents, slices,
 * a status word) is a fixed 64 MiB device array inside the library, held by
 * every GPU that loads the library until the process exits.  Sizes whose
 * scratch exceeds 64 MiB -- about S*(M+N)*K*2 bytes plus 16*(M+N+K) -- are
 * rejected with TRG_EINVAL (use trg_gemm for them).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call shares the one array: calls that overlap on the GPU (other
 *     threads, other streams) race and corrupt each other's results.
 *   - Every call copies its status word to the host and synchronises
 *     `stream` before it returns, so it blocks until its own work is done.
 *   - M and N above 2^30 or K above 131072 are rejected with TRG_EINVAL.
 * Returns TRG_OK, TRG_EINVAL, TRG_ENOTSUP (not a GB300), TRG_ETIMEOUT or
 * TRG_ECUDA.
 */
int trg_gemm_noalloc(int M, int N, int K, const double* A_dev, int lda, const double* B_dev, int ldb,
                     double* C_dev, int ldc, int slices, void* stream);

/* ------------------------------------------------ batches and serving --- */
/*
 * Many independent free-energy solves on one GPU (the paper's runs are
 * independent solves per coupling: Sec. 3.2 sweeps T and D, Sec. 3.3 sweeps
 * T).  Each slot is a worker thread owning one context and one CUDA stream;
 * a solve's tensors stay on the device until it finishes.  Requests queue
 * FIFO and start when a slot is free and their estimated device memory
 * (trg_solve_bytes) fits in what the HBM budget has left, so new requests
 * are admitted while others run and their work overlaps on the device.
 * Results do not depend on what else runs (same kernels, same arithmetic,
 * no shared buffers).
 */
typedef struct trg_solve_spec {
    int model;          /* TRG_ISING (D0 = 2) or TRG_XY (D0 odd) */
    double beta, h;
    int D0;
    int Dcut;
    int nsteps;         /* half-steps */
    int precision;      /* TRG_FP64 or TRG_SPLIT_BF16 */
    int split_slices;   /* 2..5 in TRG_SPLIT_BF16 */
    int trunc;          /* trg_trunc */
    uint64_t seed;      /* subspace-iteration start (0 = default) */
} trg_solve_spec;

typedef struct trg_solve_result {
    int status;             /* trg_status of the solve */
    double f;               /* free energy per site */
    double lnz_per_site;
    double seconds_queued;  /* submit -> start */
    double seconds_run;     /* start -> finish */
    int slot;               /* worker slot that ran it */
} trg_solve_result;

/* In dry-run mode a request with this seed reports TRG_ENUMERIC (host-side
 * fault injection for tests of the scheduler; no effect on real solves). */
#define TRG_DRY_RUN_FAIL_SEED 0xFA17FA17ull

typedef struct trg_server_config {
    int slots;                     /* concurrent solves (worker threads / streams), 1..256 */
    size_t hbm_budget_bytes;       /* admission budget for the running solves' memory */
    size_t workspace_bytes;        /* contraction workspace per solve (default 1 GiB) */
    int dry_run;                   /* 1: no GPU work, slots sleep (tests of the scheduler) */
    double dry_run_seconds_per_step;
    int policy;                    /* TRG_SERVE_FIFO (default) or TRG_SERVE_SHORTEST_FIRST */
    double max_wait_s;             /* shortest-first: a request queued this long goes next
                                      (no starvation); default 60 */
} trg_server_config;

/* Admission order.  FIFO: the oldest queued request starts when a slot is
 * free and its memory fits.  SHORTEST_FIRST: among the queued requests whose
 * memory fits, the one with the least estimated work (half-steps x Dcut^7,
 * the D^7 product's share) starts, unless the oldest has waited max_wait_s. */
enum { TRG_SERVE_FIFO = 0, TRG_SERVE_SHORTEST_FIRST = 1 };

typedef struct trg_serve_stats {
    uint64_t submitted, completed, failed, cancelled, running, queued;
    size_t bytes_in_use, peak_bytes;     /* admitted estimates, now and at most */
    double p50_latency_s, p99_latency_s, max_latency_s;   /* submit -> finish */
    double solves_per_s;                 /* finished / (first submit .. last finish) */
} trg_serve_stats;

typedef struct trg_server trg_server;

int trg_server_config_default(trg_server_config* cfg);
int trg_solve_spec_default(trg_solve_spec* spec);
/* Admission estimate (bytes) of one solve; workspace_bytes 0 = 1 GiB. */
size_t trg_solve_bytes(const trg_solve_spec* spec, size_t workspace_bytes);

int trg_serve_create(trg_server** out, int device, const trg_server_config* cfg);
/* Queue a solve.  TRG_EINVAL for a bad spec, TRG_ENOMEM if its estimate
 * exceeds the whole budget (it could never start). */
int trg_serve_submit(trg_server* server, const trg_solve_spec* spec, uint64_t* ticket);
/* TRG_OK and *out filled when done, TRG_EAGAIN while queued or running,
 * TRG_ECANCELED after a cancel. */
int trg_serve_poll(trg_server* server, uint64_t ticket, trg_solve_result* out);
/* Block until done (timeout_s < 0: no limit); TRG_ETIMEOUT on expiry. */
int trg_serve_wait(trg_server* server, uint64_t ticket, double timeout_s, trg_solve_result* out);
/* Cancel a queued request (TRG_ESTATE if it already started). */
int trg_serve_cancel(trg_server* server, uint64_t ticket);
int trg_serve_get_stats(trg_server* server, trg_serve_stats* out);
/* Stop: queued requests are dropped, running ones finish first. */
int trg_serve_destroy(trg_server* server);

/* Run n solves through a temporary server (cfg NULL = defaults); blocks.
 * Returns the first failing status (each result carries its own). */
int trg_batch_run(int device, const trg_solve_spec* specs, int n, const trg_server_config* cfg,
                  trg_solve_result* results);

/* ------------------------------------------------------- profiling ----- */
/* Phases of a half-step, timed with CUDA events on the context's stream. */
typedef enum trg_phase {
    TRG_PHASE_ENV = 0,    /* environment products (P, Q, M) */
    TRG_PHASE_EIG = 1,    /* isometry: subspace iteration + Cholesky-QR + Rayleigh-Ritz */
    TRG_PHASE_X1 = 2,     /* X1 = U.t        (D^6) */
    TRG_PHASE_X2 = 3,     /* X2 = X1.t       (D^7, the dominant product) */
    TRG_PHASE_X3 = 4,     /* Tx = X2.U       (D^6) */
    TRG_PHASE_NORM = 5,   /* max-abs normalisation and log-norm */
    TRG_PHASE_MMA = 6,    /* split mode: the tensor-core kernels alone (all products) */
    TRG_PHASE_MMA_X2 = 7, /* split mode: the tensor-core kernel launches of the X2 product alone */
    TRG_PHASE_COUNT = 8
} trg_phase;

typedef struct trg_phase_stats {
    double ms;          /* summed event time of the phase's timed regions */
    uint64_t calls;     /* timed regions (one per product / normalisation) */
    double flops;       /* algorithmic FLOPs: 2*M*N*K per product, FP64-equivalent */
    double mma_flops;   /* tensor-core FLOPs issued (split mode: slice products x 2MNK) */
} trg_phase_stats;

/* Enable (on != 0) or disable phase timing; enabling resets the counters.
 * Timing inserts event records around every product; it adds no sync. */
int trg_profile_enable(trg_ctx* ctx, int on);

/* Synchronise the stream and read the accumulated statistics of a phase. */
int trg_profile_read(trg_ctx* ctx, int phase, trg_phase_stats* out);

/* Diagnostic counters since trg_create: out[0] subspace iterations,
 * out[1] Rayleigh-Ritz solves, out[2] FP32 Jacobi sweeps, out[3] FP64
 * Jacobi sweeps (sweeps that rotated; after the FP64 refinement of the
 * eigenbasis usually none), out[4] Cholesky-QR column repairs, out[5] second
 * Cholesky-QR passes left out between power steps, out[6] product shapes
 * whose launch choice this context timed (autotune); n <= 8 entries. */
int trg_get_counters(const trg_ctx* ctx, uint64_t* out, int n);

/* ------------------------------------------------------------ misc ----- */
const char* trg_status_string(int status);
const char* trg_last_error(const trg_ctx* ctx);
/* Number of the library's own kernel launches issued by this context. */
uint64_t trg_launch_count(const trg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TRG_H */
