// The C ABI of libtrg (include/trg.h): context, solve state machine and the
// half-step driver (Sec. 2 and Fig. 1 of the paper: x half-step, y half-step
// as the x half-step of the rotated tensor, normalisation, periodic trace).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>

#include "internal.h"

namespace trg {

[[noreturn]] void fail(int status, const std::string& msg) { throw Error{status, msg}; }

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
    if (e == cudaSuccess) return;
    const char* base = std::strrchr(file, '/');
    std::string m = std::string(what) + ": " + cudaGetErrorString(e) + " (" + (base ? base + 1 : file) + ":" +
                    std::to_string(line) + ")";
    if (e == cudaErrorMemoryAllocation) throw Error{TRG_ENOMEM, m};
    throw Error{TRG_ECUDA, m};
}

void* Ctx::raw_alloc(size_t bytes) {
    void* p = nullptr;
    if (alloc_fn) {
        p = alloc_fn(bytes, (void*)stream, alloc_user);
        if (!p) fail(TRG_ENOMEM, "allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(TRG_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        }
    }
    return p;
}

void Ctx::raw_free(void* p, size_t bytes) {
    if (!p) return;
    if (free_fn) free_fn(p, bytes, (void*)stream, alloc_user);
    else cudaFree(p);
}

void Ctx::ensure(Buf& b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return;
    if (b.p) {
        // the old buffer may still be read by queued work
        TRG_CUDA(cudaStreamSynchronize(stream));
        raw_free(b.p, b.bytes);
        b.p = nullptr;
        b.bytes = 0;
    }
    const size_t sz = std::max<size_t>(bytes, 256);
    b.p = raw_alloc(sz);
    b.bytes = sz;
}

void Ctx::release(Buf& b) {
    raw_free(b.p, b.bytes);
    b.p = nullptr;
    b.bytes = 0;
}

cudaEvent_t Ctx::get_event() {
    if (!event_pool.empty()) {
        cudaEvent_t e = event_pool.back();
        event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    TRG_CUDA(cudaEventCreate(&e));
    return e;
}

int Ctx::region_begin(int p) {
    if (!prof) return -1;
    cudaEvent_t a = get_event(), b = get_event();
    TRG_CUDA(cudaEventRecord(a, stream));
    ph[p].pending.emplace_back(a, b);
    return p;
}

void Ctx::region_end(int token, double flops, double mma_flops) {
    if (token < 0) return;
    TRG_CUDA(cudaEventRecord(ph[token].pending.back().second, stream));
    ph[token].calls += 1;
    ph[token].flops += flops;
    ph[token].mma_flops += mma_flops;
}

void Ctx::collect_timings() {
    TRG_CUDA(cudaStreamSynchronize(stream));
    for (auto& acc : ph) {
        for (auto& pr : acc.pending) {
            float ms = 0.f;
            TRG_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
            acc.ms += ms;
            event_pool.push_back(pr.first);
            event_pool.push_back(pr.second);
        }
        acc.pending.clear();
    }
}

static View4 contiguous_view(double* p, int64_t n0, int64_t n1, int64_t n2, int64_t n3) {
    View4 v;
    v.p = p;
    v.n[0] = n0; v.n[1] = n1; v.n[2] = n2; v.n[3] = n3;
    v.s[3] = 1; v.s[2] = n3; v.s[1] = n2 * n3; v.s[0] = n1 * n2 * n3;
    return v;
}

// The part of a half-step before its contraction: orientation, environment,
// isometry.  Step k (1-based): odd = x, even = y.
static HalfPlan half_step_prepare(Ctx& ctx, int dcut) {
    HalfPlan p;
    p.k = ctx.steps + 1;
    p.xdir = (p.k % 2) == 1;
    p.precision = precision_for_step(ctx, p.k, (int64_t)ctx.Dx * ctx.Dy);
    const int64_t Dx = ctx.Dx, Dy = ctx.Dy;
    View4 t = contiguous_view(ctx.T.as<double>(), Dx, Dy, Dx, Dy);
    p.r = t;
    if (!p.xdir) {
        // R = permute(T, (1, 2, 3, 0)): R[p0,p1,p2,p3] = T[p3,p0,p1,p2]
        p.r.n[0] = t.n[1]; p.r.n[1] = t.n[2]; p.r.n[2] = t.n[3]; p.r.n[3] = t.n[0];
        p.r.s[0] = t.s[1]; p.r.s[1] = t.s[2]; p.r.s[2] = t.s[3]; p.r.s[3] = t.s[0];
    }
    const int64_t rx = p.r.n[0];
    const int64_t n = rx * rx;
    const int64_t dn_max = std::min<int64_t>(n, dcut);

    ctx.ensure(ctx.M, (size_t)(n * n) * sizeof(double));
    ctx.ensure(ctx.U, (size_t)(n * dn_max) * sizeof(double));
    ctx.phase = TRG_PHASE_ENV;
    environment(ctx, p.r, ctx.M.as<double>(), p.precision);

    p.dn = dn_max;
    ctx.phase = TRG_PHASE_EIG;
    {
        const int tok = ctx.region_begin(TRG_PHASE_EIG);
        if (dn_max == n) {
            launch_identity(ctx, ctx.U.as<double>(), n);
        } else {
            p.dn = isometry(ctx, ctx.M.as<double>(), n, dcut, ctx.U.as<double>(), p.lam, p.k, p.precision);
        }
        ctx.region_end(tok, 0.0, 0.0);
    }
    return p;
}

// Output O (dn, ry, dn, ry) of the x formulas, written in place of the coarse
// tensor (Dx', Dy', Dx', Dy') at `base`.
static View4 half_step_out_view(const Ctx& ctx, const HalfPlan& p, double* base) {
    const int64_t dn = p.dn, ry = p.r.n[1];
    if (p.xdir) return contiguous_view(base, dn, ctx.Dy, dn, ctx.Dy);
    // Txy = permute(O, (3, 0, 1, 2)) has shape (ry, dn, ry, dn) = (Dx, dn, Dx, dn)
    View4 txy = contiguous_view(base, ctx.Dx, dn, ctx.Dx, dn), o;
    o.p = txy.p;
    o.n[0] = dn; o.n[1] = ry; o.n[2] = dn; o.n[3] = ry;
    o.s[0] = txy.s[1]; o.s[1] = txy.s[2]; o.s[2] = txy.s[3]; o.s[3] = txy.s[0];
    return o;
}

static int64_t half_step_out_elems(const Ctx& ctx, const HalfPlan& p) {
    const int64_t newDx = p.xdir ? p.dn : ctx.Dx, newDy = p.xdir ? ctx.Dy : p.dn;
    return newDx * newDy * newDx * newDy;
}

// Normalise the coarse tensor in Tnext (and the impure one) and make it the
// current tensor.
static void half_step_finish(Ctx& ctx, HalfPlan& p) {
    const int64_t n_out = half_step_out_elems(ctx, p);
    {
        const int tok = ctx.region_begin(TRG_PHASE_NORM);
        launch_normalise(ctx, ctx.Tnext.as<double>(), n_out, p.k, false);
        // the impure tensor is divided by the same n_k
        if (ctx.have_impure) launch_scale_by_last_norm(ctx, ctx.Timp_next.as<double>(), n_out);
        ctx.region_end(tok, 0.0, 0.0);
    }
    const int st = read_status(ctx);
    if (st & ST_BAD_NORM) fail(TRG_ENUMERIC, "non-positive or non-finite norm at half-step " + std::to_string(p.k));
    std::swap(ctx.T, ctx.Tnext);
    if (ctx.have_impure) std::swap(ctx.Timp, ctx.Timp_next);
    ctx.Dx = (int)(p.xdir ? p.dn : ctx.Dx);
    ctx.Dy = (int)(p.xdir ? ctx.Dy : p.dn);
    ctx.steps = p.k;
    ctx.spectra.push_back(std::move(p.lam));
}

// One directional blocking.
static void half_step(Ctx& ctx, int dcut) {
    HalfPlan p = half_step_prepare(ctx, dcut);
    const int64_t n_out = half_step_out_elems(ctx, p);
    ctx.ensure(ctx.Tnext, (size_t)n_out * sizeof(double));
    contract(ctx, p.r, p.r, ctx.U.as<double>(), p.dn, half_step_out_view(ctx, p, ctx.Tnext.as<double>()),
             p.precision);
    if (ctx.have_impure) {
        // the impurity in the upper and in the lower tensor of the pair, same
        // isometry (from the pure environment), then the mean of the two
        View4 ri = contiguous_view(ctx.Timp.as<double>(), ctx.Dx, ctx.Dy, ctx.Dx, ctx.Dy);
        for (int q = 0; q < 4; ++q) { ri.n[q] = p.r.n[q]; ri.s[q] = p.r.s[q]; }
        ctx.ensure(ctx.Timp_next, (size_t)n_out * sizeof(double));
        ctx.ensure(ctx.Timp_tmp, (size_t)n_out * sizeof(double));
        contract(ctx, ri, p.r, ctx.U.as<double>(), p.dn, half_step_out_view(ctx, p, ctx.Timp_next.as<double>()),
                 p.precision);
        contract(ctx, p.r, ri, ctx.U.as<double>(), p.dn, half_step_out_view(ctx, p, ctx.Timp_tmp.as<double>()),
                 p.precision);
        launch_mean2(ctx, ctx.Timp_next.as<double>(), ctx.Timp_tmp.as<double>(), n_out);
    }
    half_step_finish(ctx, p);
}

static void reset_solve(Ctx& ctx) {
    // a solve depends on its own inputs only, whatever the context ran before
    ctx.eig_hint[0] = ctx.eig_hint[1] = Ctx::EigHint();
    ctx.have_tensor = false;
    ctx.have_impure = false;
    ctx.shard_pending = false;
    ctx.model = -1;
    ctx.steps = 0;
    ctx.spectra.clear();
    TRG_CUDA(cudaMemsetAsync(ctx.scal.p, 0, SC_COUNT * sizeof(double), ctx.stream));
    TRG_CUDA(cudaMemsetAsync(ctx.status.p, 0, sizeof(int), ctx.stream));
}

static void finish_init(Ctx& ctx, int Dx, int Dy, double beta) {
    launch_normalise(ctx, ctx.T.as<double>(), (int64_t)Dx * Dy * Dx * Dy, 0, true);
    const int st = read_status(ctx);
    if (st & ST_BAD_NORM) fail(TRG_ENUMERIC, "initial tensor has no positive norm");
    ctx.Dx = Dx;
    ctx.Dy = Dy;
    ctx.beta = beta;
    ctx.have_tensor = true;
}

}  // namespace trg

using trg::Ctx;
using trg::Error;

#define TRG_GUARD_BEGIN try {
#define TRG_GUARD_END(ctxp)                                                      \
    }                                                                            \
    catch (const Error& e) {                                                     \
        if (ctxp) (ctxp)->last_error = e.msg;                                    \
        return e.status;                                                         \
    }                                                                            \
    catch (const std::bad_alloc&) {                                              \
        if (ctxp) (ctxp)->last_error = "host allocation failed";                \
        return TRG_ENOMEM;                                                       \
    }                                                                            \
    catch (const std::exception& e) {                                            \
        if (ctxp) (ctxp)->last_error = e.what();                                 \
        return TRG_ECUDA;                                                        \
    }

static int bad(trg_ctx* ctx, int status, const char* msg) {
    if (ctx) ctx->last_error = msg;
    return status;
}

extern "C" {

int trg_config_default(trg_config* cfg) {
    if (!cfg) return TRG_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->precision = TRG_FP64;
    cfg->split_slices = 4;
    cfg->split_from_step = 0;
    // half-steps on tensors with Dx Dy <= 16 run in FP64: those of a model's
    // first three half-steps (bond dimensions 2 to 4), whose norms weigh 1/2,
    // 1/4 and 1/8 in ln Z / V; their split products carried most of the split
    // path's error in f (about 5x at Dcut 64) and in FP64 they cost nothing
    cfg->fp64_max_dd = 16;
    cfg->trunc = TRG_TRUNC_PAPER;
    cfg->gap_tol = 1e-6;
    cfg->oversample = 24;
    cfg->eig_tol = 1e-12;
    cfg->eig_max_iter = 300;
    cfg->seed = 0x5EEDull;
    cfg->workspace_bytes = 0;
    cfg->mma_pairs = 1;
    cfg->fused_slices = 1;
    cfg->env_slices = 0;
    cfg->autotune = 1;
    return TRG_OK;
}

static int validate_config(const trg_config& c) {
    if (c.precision != TRG_FP64 && c.precision != TRG_SPLIT_BF16) return TRG_EINVAL;
    if (c.split_slices < 2 || c.split_slices > 5) return TRG_EINVAL;
    if (c.env_slices != 0 && (c.env_slices < 2 || c.env_slices > 5)) return TRG_EINVAL;
    if (c.autotune != 0 && c.autotune != 1) return TRG_EINVAL;
    if (c.split_from_step < 0 || c.fp64_max_dd < 0) return TRG_EINVAL;
    if (c.mma_pairs != 0 && c.mma_pairs != 1) return TRG_EINVAL;
    if (c.fused_slices < 0 || c.fused_slices > 2) return TRG_EINVAL;
    if (c.trunc != TRG_TRUNC_PAPER && c.trunc != TRG_TRUNC_MULTIPLET) return TRG_EINVAL;
    if (!(c.gap_tol >= 0.0) || !(c.eig_tol > 0.0) || c.oversample < 1 || c.eig_max_iter < 1) return TRG_EINVAL;
    return TRG_OK;
}

int trg_create(trg_ctx** out, int device, const trg_config* cfg) {
    if (!out) return TRG_EINVAL;
    *out = nullptr;
    trg_ctx* ctx = new (std::nothrow) trg_ctx();
    if (!ctx) return TRG_ENOMEM;
    TRG_GUARD_BEGIN
    if (cfg) ctx->cfg = *cfg;
    else trg_config_default(&ctx->cfg);
    if (validate_config(ctx->cfg) != TRG_OK) { delete ctx; return TRG_EINVAL; }
    int ndev = 0;
    TRG_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) { delete ctx; return TRG_EINVAL; }
    TRG_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    TRG_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3) {
        delete ctx;
        return TRG_ENOTSUP;
    }
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    ctx->stream = nullptr;
    ctx->ensure(ctx->scal, trg::SC_COUNT * sizeof(double));
    ctx->ensure(ctx->status, 64);
    TRG_CUDA(cudaMemset(ctx->scal.p, 0, trg::SC_COUNT * sizeof(double)));
    TRG_CUDA(cudaMemset(ctx->status.p, 0, 64));
    *out = ctx;
    return TRG_OK;
    }
    catch (const Error& e) {
        int st = e.status;
        delete ctx;
        return st;
    }
}

int trg_destroy(trg_ctx* ctx) {
    if (!ctx) return TRG_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    Ctx& c = *ctx;
    for (trg::Buf* b : {&c.T, &c.Tnext, &c.M, &c.U, &c.scal, &c.status, &c.ws, &c.envP, &c.envQ, &c.eig,
                        &c.eig_small, &c.flags, &c.split_ws, &c.f64_partial, &c.ksplit_ws, &c.bslices, &c.cons_ef, &c.Timp, &c.Timp_next,
                        &c.Timp_tmp, &c.eig_slices})
        c.release(*b);
    for (trg::Buf& b : c.s3) c.release(b);
    for (auto& kv : c.tables) c.release(kv.second);
    c.tables.clear();
    try {
        c.collect_timings();   // a context whose stream has failed still frees its resources
    } catch (const trg::Error&) {
    }
    for (cudaEvent_t e : c.event_pool) cudaEventDestroy(e);
    delete ctx;
    return TRG_OK;
}

int trg_set_stream(trg_ctx* ctx, void* stream) {
    if (!ctx) return TRG_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return TRG_OK;
}

int trg_set_allocator(trg_ctx* ctx, trg_alloc_fn alloc, trg_free_fn free_fn, void* user) {
    if (!ctx || (!alloc) != (!free_fn)) return TRG_EINVAL;
    // only the two always-present scalar buffers exist at this point: move them
    if (ctx->T.p || ctx->M.p || !ctx->tables.empty())
        return bad(ctx, TRG_ESTATE, "trg_set_allocator must come before any other call");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->release(ctx->scal);
    ctx->release(ctx->status);
    ctx->alloc_fn = alloc;
    ctx->free_fn = free_fn;
    ctx->alloc_user = user;
    ctx->ensure(ctx->scal, trg::SC_COUNT * sizeof(double));
    ctx->ensure(ctx->status, 64);
    TRG_CUDA(cudaMemsetAsync(ctx->scal.p, 0, trg::SC_COUNT * sizeof(double), ctx->stream));
    TRG_CUDA(cudaMemsetAsync(ctx->status.p, 0, 64, ctx->stream));
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_set_wait_limit(trg_ctx* ctx, uint64_t acc_wait_ns) {
    if (!ctx) return TRG_EINVAL;
    ctx->acc_wait_ns = acc_wait_ns;
    return TRG_OK;
}

int trg_set_precision(trg_ctx* ctx, int precision, int split_slices, int split_from_step) {
    if (!ctx) return TRG_EINVAL;
    trg_config c = ctx->cfg;
    c.precision = precision;
    c.split_slices = split_slices;
    c.split_from_step = split_from_step;
    if (validate_config(c) != TRG_OK) return bad(ctx, TRG_EINVAL, "invalid precision settings");
    ctx->cfg = c;
    return TRG_OK;
}

int trg_init_tensor(trg_ctx* ctx, int model, double beta, double h, int D0) {
    if (!ctx) return TRG_EINVAL;
    if (!(beta > 0.0) || !std::isfinite(beta) || !std::isfinite(h))
        return bad(ctx, TRG_EINVAL, "beta must be positive and finite, h finite");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    if (model == TRG_ISING) {
        if (D0 != 2) return bad(ctx, TRG_EINVAL, "Ising: D0 must be 2");
        trg::reset_solve(*ctx);
        ctx->ensure(ctx->T, 16 * sizeof(double));
        trg::launch_init_ising(*ctx, ctx->T.as<double>(), beta, h);
        trg::finish_init(*ctx, 2, 2, beta);
        ctx->model = TRG_ISING; ctx->d0 = 2; ctx->h_field = h;
    } else if (model == TRG_XY) {
        if (D0 < 1 || D0 % 2 == 0 || D0 > 41) return bad(ctx, TRG_EINVAL, "XY: D0 must be odd, 1..41");
        trg::reset_solve(*ctx);
        const size_t n = (size_t)D0 * D0 * D0 * D0;
        ctx->ensure(ctx->T, n * sizeof(double));
        trg::launch_init_xy(*ctx, ctx->T.as<double>(), D0, beta, h);
        trg::finish_init(*ctx, D0, D0, beta);
        ctx->model = TRG_XY; ctx->d0 = D0; ctx->h_field = h;
    } else if (model == TRG_POTTS) {
        if (D0 < 2 || D0 > 8) return bad(ctx, TRG_EINVAL, "Potts: D0 = q must be 2..8");
        trg::reset_solve(*ctx);
        const size_t n = (size_t)D0 * D0 * D0 * D0;
        ctx->ensure(ctx->T, n * sizeof(double));
        trg::launch_init_potts(*ctx, ctx->T.as<double>(), D0, beta, h);
        trg::finish_init(*ctx, D0, D0, beta);
        ctx->model = TRG_POTTS; ctx->d0 = D0; ctx->h_field = h;
    } else {
        return bad(ctx, TRG_EINVAL, "unknown model");
    }
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_init_tensor_raw(trg_ctx* ctx, const double* T_host, int Dx, int Dy, double beta) {
    if (!ctx) return TRG_EINVAL;
    if (!T_host || Dx < 1 || Dy < 1 || Dx > 4096 || Dy > 4096)
        return bad(ctx, TRG_EINVAL, "init_tensor_raw: bad tensor");
    if (!(beta > 0.0) || !std::isfinite(beta)) return bad(ctx, TRG_EINVAL, "beta must be positive and finite");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    trg::reset_solve(*ctx);
    const size_t n = (size_t)Dx * Dy * Dx * Dy;
    ctx->ensure(ctx->T, n * sizeof(double));
    TRG_CUDA(cudaMemcpyAsync(ctx->T.p, T_host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    trg::finish_init(*ctx, Dx, Dy, beta);
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_init_impure(trg_ctx* ctx) {
    if (!ctx) return TRG_EINVAL;
    if (!ctx->have_tensor || ctx->steps != 0 || ctx->model < 0)
        return bad(ctx, TRG_ESTATE, "init_impure needs a fresh trg_init_tensor (model tensor, no half-steps yet)");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    const int d0 = ctx->d0;
    const size_t n = (size_t)d0 * d0 * d0 * d0;
    ctx->ensure(ctx->Timp, n * sizeof(double));
    if (ctx->model == TRG_ISING) trg::launch_init_ising(*ctx, ctx->Timp.as<double>(), ctx->beta, ctx->h_field, 1);
    else if (ctx->model == TRG_XY) trg::launch_init_xy(*ctx, ctx->Timp.as<double>(), d0, ctx->beta, ctx->h_field, 1);
    else trg::launch_init_potts(*ctx, ctx->Timp.as<double>(), d0, ctx->beta, ctx->h_field, 1);
    // the pure tensor was divided by n0: so is the impure one
    trg::launch_scale_by_exp_neg(*ctx, ctx->Timp.as<double>(), (int64_t)n, ctx->scal.as<double>() + trg::SC_LN_N0);
    ctx->have_impure = true;
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_init_impure_raw(trg_ctx* ctx, const double* Timp_host) {
    if (!ctx) return TRG_EINVAL;
    if (!Timp_host) return bad(ctx, TRG_EINVAL, "init_impure_raw: no tensor");
    if (!ctx->have_tensor || ctx->steps != 0)
        return bad(ctx, TRG_ESTATE, "init_impure_raw needs a fresh initial tensor (no half-steps yet)");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    const size_t n = (size_t)ctx->Dx * ctx->Dy * ctx->Dx * ctx->Dy;
    ctx->ensure(ctx->Timp, n * sizeof(double));
    TRG_CUDA(cudaMemcpyAsync(ctx->Timp.p, Timp_host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    trg::launch_scale_by_exp_neg(*ctx, ctx->Timp.as<double>(), (int64_t)n, ctx->scal.as<double>() + trg::SC_LN_N0);
    TRG_CUDA(cudaStreamSynchronize(ctx->stream));   // the host buffer may go after return
    ctx->have_impure = true;
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_expectation(trg_ctx* ctx, double* value_out) {
    if (!ctx) return TRG_EINVAL;
    if (!value_out) return bad(ctx, TRG_EINVAL, "no output");
    if (!ctx->have_tensor || !ctx->have_impure) return bad(ctx, TRG_ESTATE, "expectation without an impure tensor");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    double* scal = ctx->scal.as<double>();
    trg::launch_trace(*ctx, ctx->T.as<double>(), ctx->Dx, ctx->Dy, scal + trg::SC_TRACE);
    trg::launch_trace_signed(*ctx, ctx->Timp.as<double>(), ctx->Dx, ctx->Dy, scal + trg::SC_TRACE_IMP);
    double h[trg::SC_COUNT];
    TRG_CUDA(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    TRG_CUDA(cudaStreamSynchronize(ctx->stream));
    if (trg::read_status(*ctx) & trg::ST_BAD_TRACE) return bad(ctx, TRG_ENUMERIC, "non-positive trace");
    *value_out = h[trg::SC_TRACE_IMP] / h[trg::SC_TRACE];
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_coarse_grain(trg_ctx* ctx, int Dcut, int nsteps) {
    if (!ctx) return TRG_EINVAL;
    if (!ctx->have_tensor) return bad(ctx, TRG_ESTATE, "coarse_grain before init_tensor");
    if (Dcut < 1 || nsteps < 0) return bad(ctx, TRG_EINVAL, "Dcut >= 1 and nsteps >= 0 required");
    if (ctx->steps + nsteps > 1000) return bad(ctx, TRG_EINVAL, "more than 1000 half-steps");
    if (ctx->shard_pending) return bad(ctx, TRG_ESTATE, "coarse_grain between trg_shard_begin and trg_shard_finish");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    for (int i = 0; i < nsteps; ++i) trg::half_step(*ctx, Dcut);
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_shard_extent(trg_ctx* ctx, int* nj_out) {
    if (!ctx || !nj_out) return TRG_EINVAL;
    if (!ctx->have_tensor) return bad(ctx, TRG_ESTATE, "shard_extent before init_tensor");
    *nj_out = ((ctx->steps + 1) % 2 == 1) ? ctx->Dy : ctx->Dx;
    return TRG_OK;
}

int trg_shard_begin(trg_ctx* ctx, int Dcut, int j_begin, int j_end, double* slab_dev, size_t slab_cap,
                    int* dn_out) {
    if (!ctx) return TRG_EINVAL;
    if (!ctx->have_tensor) return bad(ctx, TRG_ESTATE, "shard_begin before init_tensor");
    if (ctx->shard_pending) return bad(ctx, TRG_ESTATE, "shard_begin twice without shard_finish");
    if (ctx->have_impure) return bad(ctx, TRG_ENOTSUP, "a split half-step does not carry an impure tensor");
    if (Dcut < 1 || !dn_out || (!slab_dev && j_end > j_begin)) return bad(ctx, TRG_EINVAL, "shard_begin: bad arguments");
    if (ctx->steps + 1 > 1000) return bad(ctx, TRG_EINVAL, "more than 1000 half-steps");
    const int nj = ((ctx->steps + 1) % 2 == 1) ? ctx->Dy : ctx->Dx;
    if (j_begin < 0 || j_begin > j_end || j_end > nj) return bad(ctx, TRG_EINVAL, "shard_begin: j range outside 0..extent");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    trg::HalfPlan p = trg::half_step_prepare(*ctx, Dcut);
    const int64_t ry = p.r.n[1], dn = p.dn;
    if ((size_t)(j_end - j_begin) * (size_t)(dn * dn * ry) > slab_cap)
        return bad(ctx, TRG_EINVAL, "shard_begin: slab capacity below (j_end - j_begin) Dn^2 extent doubles");
    if (j_end > j_begin) {
        // the slab S[jj][i][k][l] of the x formulas' output O[i, j_begin + jj, k, l]
        trg::View4 o;
        o.p = slab_dev;
        o.n[0] = dn; o.n[1] = ry; o.n[2] = dn; o.n[3] = ry;
        o.s[0] = dn * ry; o.s[1] = dn * dn * ry; o.s[2] = ry; o.s[3] = 1;
        trg::contract(*ctx, p.r, p.r, ctx->U.as<double>(), dn, o, p.precision, j_begin, j_end, j_begin);
    }
    ctx->shard = std::move(p);
    ctx->shard_pending = true;
    *dn_out = (int)dn;
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_shard_finish(trg_ctx* ctx, const double* gathered_dev, int j_rows) {
    if (!ctx) return TRG_EINVAL;
    if (!ctx->shard_pending) return bad(ctx, TRG_ESTATE, "shard_finish without shard_begin");
    const int64_t ry = ctx->shard.r.n[1], dn = ctx->shard.dn;
    if (!gathered_dev || j_rows < ry) return bad(ctx, TRG_EINVAL, "shard_finish: need all j rows of the gathered output");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    ctx->shard_pending = false;
    trg::HalfPlan p = std::move(ctx->shard);
    const int64_t n_out = trg::half_step_out_elems(*ctx, p);
    ctx->ensure(ctx->Tnext, (size_t)n_out * sizeof(double));
    // gathered G[j][i][k][l] (rows j >= the extent are padding) -> the coarse tensor
    trg::View4 g;
    g.p = const_cast<double*>(gathered_dev);
    g.n[0] = dn; g.n[1] = ry; g.n[2] = dn; g.n[3] = ry;
    g.s[0] = dn * ry; g.s[1] = dn * dn * ry; g.s[2] = ry; g.s[3] = 1;
    trg::launch_copy_strided(*ctx, g, trg::half_step_out_view(*ctx, p, ctx->Tnext.as<double>()));
    trg::half_step_finish(*ctx, p);
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_free_energy(trg_ctx* ctx, double* f_out, double* lnz_per_site) {
    if (!ctx) return TRG_EINVAL;
    if (!ctx->have_tensor) return bad(ctx, TRG_ESTATE, "free_energy before init_tensor");
    if (!f_out && !lnz_per_site) return bad(ctx, TRG_EINVAL, "no output");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    double* scal = ctx->scal.as<double>();
    trg::launch_trace(*ctx, ctx->T.as<double>(), ctx->Dx, ctx->Dy, scal + trg::SC_TRACE);
    double h[trg::SC_COUNT];
    TRG_CUDA(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    TRG_CUDA(cudaStreamSynchronize(ctx->stream));
    if (trg::read_status(*ctx) & trg::ST_BAD_TRACE) return bad(ctx, TRG_ENUMERIC, "non-positive trace");
    const double lnz = h[trg::SC_LN_N0] + h[trg::SC_LOGNORM] + std::ldexp(std::log(h[trg::SC_TRACE]), -ctx->steps);
    if (lnz_per_site) *lnz_per_site = lnz;
    if (f_out) *f_out = -lnz / ctx->beta;
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_solve3d(trg_ctx* ctx, int model, double beta, double h, int Dcut, int nsteps, double* f_out,
                double* lnz_per_site) {
    if (!ctx) return TRG_EINVAL;
    if (model != TRG_ISING) return bad(ctx, TRG_ENOTSUP, "solve3d: the cubic-lattice path has the Ising model only");
    if (!(beta > 0.0) || !std::isfinite(beta) || !std::isfinite(h))
        return bad(ctx, TRG_EINVAL, "solve3d: beta > 0 and finite h required");
    if (Dcut < 1 || nsteps < 0 || nsteps > 300) return bad(ctx, TRG_EINVAL, "solve3d: Dcut >= 1, 0 <= nsteps <= 300");
    if (!f_out && !lnz_per_site) return bad(ctx, TRG_EINVAL, "no output");
    TRG_GUARD_BEGIN
    trg::Ctx& c = *ctx;
    TRG_CUDA(cudaSetDevice(c.device));
    reset_solve(c);
    c.ensure(c.T, 64 * sizeof(double));
    trg::launch_init_ising3d(c, c.T.as<double>(), beta, h);
    trg::launch_normalise(c, c.T.as<double>(), 64, 0, true);
    if (trg::read_status(c) & trg::ST_BAD_NORM) return bad(ctx, TRG_ENUMERIC, "initial tensor has no positive norm");
    auto contiguous = [](double* p, const int64_t* n) {
        trg::View6 v;
        v.p = p;
        int64_t stride = 1;
        for (int i = 5; i >= 0; --i) { v.n[i] = n[i]; v.s[i] = stride; stride *= n[i]; }
        return v;
    };
    int64_t dims[6] = {2, 2, 2, 2, 2, 2};
    trg::View6 v = contiguous(c.T.as<double>(), dims);
    for (int k = 1; k <= nsteps; ++k) {
        const int64_t Dx = v.n[0], Dy = v.n[2], Dz = v.n[4];
        const int64_t Nx = std::min<int64_t>(Dx * Dx, Dcut), Ny = std::min<int64_t>(Dy * Dy, Dcut);
        c.ensure(c.Tnext, (size_t)(Nx * Nx * Ny * Ny * Dz * Dz) * sizeof(double));
        std::vector<double> lx, ly;
        const auto kept = trg::step3(c, v, Dcut, k, c.Tnext.as<double>(), trg::precision_for_step(c, k, Dx * Dy * Dz), lx, ly);
        const int64_t kx = kept.first, ky = kept.second;
        c.phase = TRG_PHASE_NORM;
        trg::launch_normalise(c, c.Tnext.as<double>(), kx * kx * ky * ky * Dz * Dz, k, false);
        if (trg::read_status(c) & trg::ST_BAD_NORM)
            return bad(ctx, TRG_ENUMERIC, ("non-positive or non-finite norm at step " + std::to_string(k)).c_str());
        std::swap(c.T, c.Tnext);
        // the next axis to block into the z slot: a rotation of the view
        const int64_t out_dims[6] = {kx, kx, ky, ky, Dz, Dz};
        const trg::View6 w = contiguous(c.T.as<double>(), out_dims);
        for (int i = 0; i < 6; ++i) { v.n[i] = w.n[(i + 2) % 6]; v.s[i] = w.s[(i + 2) % 6]; }
        v.p = w.p;
        c.spectra.push_back(lx);
        c.spectra.push_back(ly);
    }
    double* scal = c.scal.as<double>();
    trg::launch_trace3(c, v, scal + trg::SC_TRACE);
    double hs[trg::SC_COUNT];
    TRG_CUDA(cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, c.stream));
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    if (trg::read_status(c) & trg::ST_BAD_TRACE) return bad(ctx, TRG_ENUMERIC, "non-positive trace");
    const double lnz = hs[trg::SC_LN_N0] + hs[trg::SC_LOGNORM] + std::ldexp(std::log(hs[trg::SC_TRACE]), -nsteps);
    if (lnz_per_site) *lnz_per_site = lnz;
    if (f_out) *f_out = -lnz / beta;
    c.have_tensor = false;   // the 2D state does not survive a cubic-lattice solve
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_get_spectrum(trg_ctx* ctx, int step, double* out, int cap, int* n_out) {
    if (!ctx || !n_out) return TRG_EINVAL;
    if (step < 1 || step > (int)ctx->spectra.size()) return bad(ctx, TRG_EINVAL, "no such half-step");
    const std::vector<double>& s = ctx->spectra[(size_t)step - 1];
    *n_out = (int)s.size();
    if (out && cap > 0) std::memcpy(out, s.data(), sizeof(double) * (size_t)std::min<int>(cap, (int)s.size()));
    return TRG_OK;
}

int trg_get_state(trg_ctx* ctx, int* steps, int* Dx, int* Dy, double* lognorm) {
    if (!ctx) return TRG_EINVAL;
    TRG_GUARD_BEGIN
    if (steps) *steps = ctx->steps;
    if (Dx) *Dx = ctx->Dx;
    if (Dy) *Dy = ctx->Dy;
    if (lognorm) {
        TRG_CUDA(cudaMemcpyAsync(lognorm, ctx->scal.as<double>() + trg::SC_LOGNORM, sizeof(double),
                                 cudaMemcpyDeviceToHost, ctx->stream));
        TRG_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_get_tensor(trg_ctx* ctx, double* T_host, size_t cap) {
    if (!ctx || !T_host) return TRG_EINVAL;
    if (!ctx->have_tensor) return bad(ctx, TRG_ESTATE, "no tensor");
    const size_t n = (size_t)ctx->Dx * ctx->Dy * ctx->Dx * ctx->Dy;
    if (cap < n) return bad(ctx, TRG_EINVAL, "buffer too small");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaMemcpyAsync(T_host, ctx->T.p, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    TRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_environment(trg_ctx* ctx, const double* t_dev, int Dx, int Dy, double* M_dev) {
    if (!ctx) return TRG_EINVAL;
    if (!t_dev || !M_dev || Dx < 1 || Dy < 1) return bad(ctx, TRG_EINVAL, "environment: bad arguments");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    trg::View4 t = trg::contiguous_view(const_cast<double*>(t_dev), Dx, Dy, Dx, Dy);
    ctx->phase = TRG_PHASE_ENV;
    trg::environment(*ctx, t, M_dev, ctx->cfg.precision);
    TRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_isometry(trg_ctx* ctx, const double* M_dev, int n, int Dcut, double* U_dev, double* lam_host, int* dn_out) {
    if (!ctx) return TRG_EINVAL;
    if (!M_dev || !U_dev || !dn_out || n < 1 || Dcut < 1) return bad(ctx, TRG_EINVAL, "isometry: bad arguments");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    const int dn_max = std::min(n, Dcut);
    if (dn_max == n) {
        trg::launch_identity(*ctx, U_dev, n);
        *dn_out = n;
    } else {
        std::vector<double> lam;
        ctx->eig_hint[1] = trg::Ctx::EigHint();   // a component call starts from scratch
        ctx->phase = TRG_PHASE_EIG;
        const int dn = trg::isometry(*ctx, M_dev, n, Dcut, U_dev, lam, 1, ctx->cfg.precision);
        *dn_out = dn;
        if (lam_host) std::memcpy(lam_host, lam.data(), sizeof(double) * (size_t)dn);
    }
    TRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_contract(trg_ctx* ctx, const double* t_dev, const double* U_dev, int Dx, int Dy, int Dn, double* Tx_dev) {
    if (!ctx) return TRG_EINVAL;
    if (!t_dev || !U_dev || !Tx_dev || Dx < 1 || Dy < 1 || Dn < 1 || Dn > Dx * Dx)
        return bad(ctx, TRG_EINVAL, "contract: bad arguments");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    trg::View4 t = trg::contiguous_view(const_cast<double*>(t_dev), Dx, Dy, Dx, Dy);
    trg::View4 o = trg::contiguous_view(Tx_dev, Dn, Dy, Dn, Dy);
    ctx->phase = TRG_PHASE_X1;
    trg::contract(*ctx, t, t, U_dev, Dn, o, ctx->cfg.precision);
    TRG_CUDA(cudaStreamSynchronize(ctx->stream));
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_gemm(trg_ctx* ctx, int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
             int ldc) {
    if (!ctx) return TRG_EINVAL;
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < N || ldc < N)
        return bad(ctx, TRG_EINVAL, "gemm: bad arguments");
    TRG_GUARD_BEGIN
    TRG_CUDA(cudaSetDevice(ctx->device));
    trg::GemmDesc g;
    g.M = M; g.N = N; g.K = K;
    g.A.base = A; g.A.off_r = ctx->table({{M, lda}}); g.A.off_c = ctx->table({{K, 1}}); g.A.c_fast = true;
    g.B.base = B; g.B.off_r = ctx->table({{K, ldb}}); g.B.off_c = ctx->table({{N, 1}}); g.B.c_fast = true;
    g.C = C; g.c_m = ctx->table({{M, ldc}}); g.c_n = ctx->table({{N, 1}}); g.beta = 0.0;
    ctx->phase = TRG_PHASE_X2;
    // a status left by an earlier call is not this product's
    TRG_CUDA(cudaMemsetAsync(ctx->status.p, 0, sizeof(int), ctx->stream));
    trg::gemm(*ctx, g, ctx->cfg.precision);
    TRG_CUDA(cudaStreamSynchronize(ctx->stream));
    if (trg::read_status(*ctx) & trg::ST_TIMEOUT) return bad(ctx, TRG_ETIMEOUT, "gemm: device wait timed out");
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_profile_enable(trg_ctx* ctx, int on) {
    if (!ctx) return TRG_EINVAL;
    TRG_GUARD_BEGIN
    ctx->collect_timings();
    for (auto& acc : ctx->ph) { acc.ms = 0.0; acc.flops = 0.0; acc.mma_flops = 0.0; acc.calls = 0; }
    ctx->prof = on != 0;
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

int trg_profile_read(trg_ctx* ctx, int phase, trg_phase_stats* out) {
    if (!ctx || !out || phase < 0 || phase >= TRG_PHASE_COUNT) return TRG_EINVAL;
    TRG_GUARD_BEGIN
    ctx->collect_timings();
    const auto& a = ctx->ph[phase];
    out->ms = a.ms;
    out->calls = a.calls;
    out->flops = a.flops;
    out->mma_flops = a.mma_flops;
    return TRG_OK;
    TRG_GUARD_END(ctx)
}

const char* trg_status_string(int status) {
    switch (status) {
        case TRG_OK: return "ok";
        case TRG_EINVAL: return "invalid argument";
        case TRG_ESTATE: return "call out of order";
        case TRG_ENOMEM: return "out of memory";
        case TRG_ENUMERIC: return "numerical failure";
        case TRG_ETIMEOUT: return "device wait timed out";
        case TRG_ECUDA: return "CUDA error";
        case TRG_ENOTSUP: return "not supported";
        case TRG_EAGAIN: return "not finished yet";
        case TRG_ECANCELED: return "cancelled";
        default: return "unknown status";
    }
}

const char* trg_last_error(const trg_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

uint64_t trg_launch_count(const trg_ctx* ctx) { return ctx ? ctx->launches : 0; }

int trg_get_counters(const trg_ctx* ctx, uint64_t* out, int n) {
    if (!ctx || !out || n < 0 || n > 8) return TRG_EINVAL;
    for (int i = 0; i < n; ++i) out[i] = ctx->counters[i];
    return TRG_OK;
}

}  // extern "C"
