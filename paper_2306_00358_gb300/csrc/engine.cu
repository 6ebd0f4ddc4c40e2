// Solve engine behind trg_batch_run and trg_serve_*: many independent
// free-energy solves (different models, couplings, Dcut, step counts) on one
// GPU at the same time.
//
// Each slot is a worker thread that owns one library context with its own
// CUDA stream; its tensors stay resident on the device for the whole solve.
// Requests wait in a FIFO queue and are admitted when a slot is free and their
// estimated device memory fits in what the HBM budget has left; a slot that
// finishes takes the next request at once, so solves that arrive while others
// run overlap on the device (continuous batching).  Kernels are deterministic
// and a solve never shares buffers with another, so each result is bit for bit
// the same alone and in a mix.  In dry-run mode the slots only sleep for a
// duration derived from the request: the queue, admission, cancellation and
// statistics logic can then be exercised without a GPU.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

// Device bytes one solve can hold at its largest half-step: tensors, the
// environment and its two intermediates, isometry, subspace-iteration blocks,
// the contraction workspace and the split-GEMM scratch.  An upper bound.
size_t estimate_bytes(const trg_solve_spec& s, size_t workspace_cap) {
    const double d0 = (s.model == TRG_ISING) ? 2 : std::max(1, s.D0);
    const double D = std::max<double>(d0, std::min<double>(s.Dcut, std::max(d0 * d0, (double)s.Dcut)));
    const double D2 = D * D, D4 = D2 * D2;
    const double m = std::min<double>({D2, s.Dcut + 24.0, 112.0});
    double bytes = 0;
    bytes += 2 * D4 * 8;                       // T, Tnext
    bytes += 3 * D4 * 8;                       // M, P, Q
    bytes += D2 * D * 8;                       // U
    bytes += 4 * D2 * m * 8 + 4 * m * m * 8;   // Q, Y, Z, QW; small blocks
    const double ws_full = 2 * D4 * D * 8;     // X1 + X2 for all j
    const double ws = std::min<double>(ws_full, (double)workspace_cap);
    bytes += ws;
    if (s.precision == TRG_SPLIT_BF16) {
        // slices of the largest product (X1 slice as A, t as B) plus exponents
        const double jb = std::max(1.0, std::floor(ws / std::max(1.0, 2 * D * D * D2 * 8)));
        const double rows_a = std::min(D, jb) * D * D + 128, rows_b = D2 + 128;
        bytes += (double)std::max(2, s.split_slices) * (rows_a + rows_b) * (D2 + 32) * 2 + (rows_a + rows_b) * 4;
        bytes += (double)std::max(2, s.split_slices) * (D2 + 256) * (D2 + 32) * 2;   // M sliced for the isometry
        // the contraction's operands shared by its j-blocks (t as B, U twice)
        const double S_ = std::max(2, s.split_slices);
        bytes += S_ * (D2 + 128) * (D2 + 32) * 2 +          // t as the D^7 product's B
                 S_ * (D2 + 256) * (D + 32) * 2 +           // U as X1's A (D Dn rows, K = D)
                 S_ * (D + 128) * (D2 + 32) * 2 +           // U as the last product's B
                 3 * (D2 + 256) * 4 + 3 * 256.0;            // their exponents, alignment
        // split-K parts of the isometry's products: at most 152 x 128 rows x m
        bytes += 152.0 * 128 * m * 8;
    }
    bytes += 64.0 * 1024 * 1024;               // tables, scalars, allocator slack
    return (size_t)bytes;
}

// Estimated work of a solve: half-steps x D^7 (the D^7 product dominates).
double estimate_work(const trg_solve_spec& s) {
    const double d = std::max(1, s.Dcut);
    return (double)std::max(1, s.nsteps) * d * d * d * d * d * d * d;
}

struct Request {
    uint64_t ticket = 0;
    trg_solve_spec spec{};
    size_t bytes = 0;
    double work = 0.0;
    Clock::time_point t_submit, t_start, t_end;
    enum { QUEUED, RUNNING, DONE, CANCELLED } state = QUEUED;
    trg_solve_result result{};
};

int validate_spec(const trg_solve_spec& s) {
    if (s.model != TRG_ISING && s.model != TRG_XY && s.model != TRG_POTTS) return TRG_EINVAL;
    if (!(s.beta > 0.0) || !std::isfinite(s.beta) || !std::isfinite(s.h)) return TRG_EINVAL;
    if (s.Dcut < 1 || s.nsteps < 0 || s.nsteps > 1000) return TRG_EINVAL;
    if (s.precision != TRG_FP64 && s.precision != TRG_SPLIT_BF16) return TRG_EINVAL;
    if (s.precision == TRG_SPLIT_BF16 && (s.split_slices < 2 || s.split_slices > 5)) return TRG_EINVAL;
    if (s.trunc != TRG_TRUNC_PAPER && s.trunc != TRG_TRUNC_MULTIPLET) return TRG_EINVAL;
    if (s.model == TRG_ISING && s.D0 != 2) return TRG_EINVAL;
    if (s.model == TRG_XY && (s.D0 < 1 || s.D0 % 2 == 0 || s.D0 > 41)) return TRG_EINVAL;
    if (s.model == TRG_POTTS && (s.D0 < 2 || s.D0 > 8)) return TRG_EINVAL;
    return TRG_OK;
}

}  // namespace

struct trg_server {
    int device = 0;
    trg_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<uint64_t, Request*> all;
    std::vector<std::thread> workers;
    uint64_t next_ticket = 1;
    size_t in_use = 0, peak = 0;
    bool stopping = false;
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, running = 0;
    std::vector<double> latencies;
    Clock::time_point t_first_submit, t_last_done;
    bool any_submitted = false;

    void run_request(trg_ctx*& ctx, Request* r);
    void worker_main(int slot);
};

void trg_server::run_request(trg_ctx*& ctx, Request* r) {
    const trg_solve_spec& s = r->spec;
    trg_solve_result& res = r->result;
    if (cfg.dry_run) {
        // host-only executor: sleep for a duration shaped like the solve's cost
        const double d = std::min<double>(s.Dcut, 64);
        const double t = cfg.dry_run_seconds_per_step * s.nsteps * (d / 16.0) * (d / 16.0);
        std::this_thread::sleep_for(std::chrono::duration<double>(t));
        // host-side fault injection for tests: this seed makes the solve fail
        res.status = (s.seed == TRG_DRY_RUN_FAIL_SEED) ? TRG_ENUMERIC : TRG_OK;
        res.f = -(double)r->ticket;   // recognisable stand-in value
        res.lnz_per_site = 0.0;
        return;
    }
    if (!ctx) {
        trg_config c;
        trg_config_default(&c);
        c.workspace_bytes = cfg.workspace_bytes;
        int st = trg_create(&ctx, device, &c);
        if (st != TRG_OK) { res.status = st; ctx = nullptr; return; }
        cudaStream_t stream = nullptr;
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
            res.status = TRG_ECUDA;
            trg_destroy(ctx);
            ctx = nullptr;
            return;
        }
        trg_set_stream(ctx, stream);
    }
    int st = trg_set_precision(ctx, s.precision, s.precision == TRG_SPLIT_BF16 ? s.split_slices : 4, 0);
    if (st == TRG_OK) {
        ctx->cfg.trunc = s.trunc;
        ctx->cfg.seed = s.seed ? s.seed : 0x5EEDull;
        st = trg_init_tensor(ctx, s.model, s.beta, s.h, s.D0);
    }
    if (st == TRG_OK) st = trg_coarse_grain(ctx, s.Dcut, s.nsteps);
    if (st == TRG_OK) st = trg_free_energy(ctx, &res.f, &res.lnz_per_site);
    res.status = st;
    // give the device memory back so the budget accounting stays true
    trg::trim_buffers(*ctx);
}

void trg_server::worker_main(int slot) {
    trg_ctx* ctx = nullptr;
    if (!cfg.dry_run) cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // the request this slot takes (queue.end() while none may start)
        auto pick = [&]() {
            if (queue.empty()) return queue.end();
            if (cfg.policy == TRG_SERVE_FIFO ||
                secs(queue.front()->t_submit, Clock::now()) >= cfg.max_wait_s) {
                // FIFO, or the oldest request has waited long enough: the head
                // of the queue starts when its memory fits; the rest wait
                return in_use + queue.front()->bytes <= cfg.hbm_budget_bytes ? queue.begin() : queue.end();
            }
            // shortest first among those that fit (the oldest of equal work)
            auto best = queue.end();
            for (auto it = queue.begin(); it != queue.end(); ++it)
                if (in_use + (*it)->bytes <= cfg.hbm_budget_bytes && (best == queue.end() || (*it)->work < (*best)->work))
                    best = it;
            return best;
        };
        std::deque<Request*>::iterator it;
        // waits are bounded so that the starvation guard is re-checked
        while (!stopping && (it = pick()) == queue.end())
            cv_work.wait_for(lk, std::chrono::milliseconds(100));
        if (stopping) break;
        Request* r = *it;
        queue.erase(it);
        r->state = Request::RUNNING;
        r->t_start = Clock::now();
        in_use += r->bytes;
        peak = std::max(peak, in_use);
        ++running;
        lk.unlock();

        run_request(ctx, r);

        lk.lock();
        r->t_end = Clock::now();
        in_use -= r->bytes;
        --running;
        r->state = Request::DONE;
        r->result.slot = slot;
        r->result.seconds_queued = secs(r->t_submit, r->t_start);
        r->result.seconds_run = secs(r->t_start, r->t_end);
        if (r->result.status == TRG_OK) ++completed;
        else ++failed;
        latencies.push_back(secs(r->t_submit, r->t_end));
        t_last_done = r->t_end;
        cv_done.notify_all();
        cv_work.notify_all();
    }
    lk.unlock();
    if (ctx) {
        cudaStream_t stream = ctx->stream;
        trg_destroy(ctx);
        if (stream) cudaStreamDestroy(stream);
    }
}

namespace trg {

void trim_buffers(Ctx& c) {
    cudaStreamSynchronize(c.stream);
    for (Buf* b : {&c.T, &c.Tnext, &c.M, &c.U, &c.ws, &c.envP, &c.envQ, &c.eig, &c.eig_small, &c.flags,
                   &c.split_ws, &c.f64_partial, &c.ksplit_ws, &c.bslices, &c.cons_ef, &c.eig_slices, &c.Timp,
                   &c.Timp_next, &c.Timp_tmp})
        c.release(*b);
    for (Buf& b : c.s3) c.release(b);
    for (auto& kv : c.tables) c.release(kv.second);
    c.tables.clear();
    c.have_tensor = false;
}

}  // namespace trg

extern "C" {

int trg_server_config_default(trg_server_config* cfg) {
    if (!cfg) return TRG_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->slots = 8;
    cfg->hbm_budget_bytes = (size_t)150 << 30;   // 150 GB
    cfg->workspace_bytes = (size_t)1 << 30;
    cfg->dry_run = 0;
    cfg->dry_run_seconds_per_step = 1e-3;
    cfg->policy = TRG_SERVE_FIFO;
    cfg->max_wait_s = 60.0;
    return TRG_OK;
}

int trg_solve_spec_default(trg_solve_spec* s) {
    if (!s) return TRG_EINVAL;
    std::memset(s, 0, sizeof(*s));
    s->model = TRG_ISING;
    s->beta = 0.44;
    s->D0 = 2;
    s->Dcut = 16;
    s->nsteps = 40;
    s->precision = TRG_SPLIT_BF16;
    s->split_slices = 4;
    s->trunc = TRG_TRUNC_PAPER;
    return TRG_OK;
}

size_t trg_solve_bytes(const trg_solve_spec* spec, size_t workspace_bytes) {
    if (!spec) return 0;
    return estimate_bytes(*spec, workspace_bytes ? workspace_bytes : ((size_t)1 << 30));
}

int trg_serve_create(trg_server** out, int device, const trg_server_config* cfg) {
    if (!out) return TRG_EINVAL;
    *out = nullptr;
    trg_server_config c;
    if (cfg) c = *cfg;
    else trg_server_config_default(&c);
    if (c.slots < 1 || c.slots > 256 || c.hbm_budget_bytes == 0) return TRG_EINVAL;
    if (c.policy != TRG_SERVE_FIFO && c.policy != TRG_SERVE_SHORTEST_FIRST) return TRG_EINVAL;
    if (!(c.max_wait_s >= 0.0)) return TRG_EINVAL;
    if (c.workspace_bytes == 0) c.workspace_bytes = (size_t)1 << 30;
    if (!c.dry_run) {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return TRG_ECUDA; }
        if (device < 0 || device >= ndev) return TRG_EINVAL;
    }
    trg_server* s = new (std::nothrow) trg_server();
    if (!s) return TRG_ENOMEM;
    s->device = device;
    s->cfg = c;
    try {
        for (int i = 0; i < c.slots; ++i) s->workers.emplace_back([s, i] { s->worker_main(i); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stopping = true;
        }
        s->cv_work.notify_all();
        for (auto& t : s->workers) t.join();
        delete s;
        return TRG_ENOMEM;
    }
    *out = s;
    return TRG_OK;
}

int trg_serve_submit(trg_server* s, const trg_solve_spec* spec, uint64_t* ticket) {
    if (!s || !spec || !ticket) return TRG_EINVAL;
    const int v = validate_spec(*spec);
    if (v != TRG_OK) return v;
    Request* r = new (std::nothrow) Request();
    if (!r) return TRG_ENOMEM;
    r->spec = *spec;
    r->bytes = estimate_bytes(*spec, s->cfg.workspace_bytes);
    r->work = estimate_work(*spec);
    if (r->bytes > s->cfg.hbm_budget_bytes) {   // could never be admitted
        delete r;
        return TRG_ENOMEM;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) { delete r; return TRG_ESTATE; }
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    if (!s->any_submitted) { s->t_first_submit = r->t_submit; s->any_submitted = true; }
    s->queue.push_back(r);
    s->all[r->ticket] = r;
    ++s->submitted;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return TRG_OK;
}

int trg_serve_poll(trg_server* s, uint64_t ticket, trg_solve_result* out) {
    if (!s) return TRG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return TRG_EINVAL;
    Request* r = it->second;
    if (r->state == Request::CANCELLED) return TRG_ECANCELED;
    if (r->state != Request::DONE) return TRG_EAGAIN;
    if (out) *out = r->result;
    return TRG_OK;
}

int trg_serve_wait(trg_server* s, uint64_t ticket, double timeout_s, trg_solve_result* out) {
    if (!s) return TRG_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return TRG_EINVAL;
    Request* r = it->second;
    auto ready = [&] { return r->state == Request::DONE || r->state == Request::CANCELLED; };
    if (timeout_s < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return TRG_ETIMEOUT;
    if (r->state == Request::CANCELLED) return TRG_ECANCELED;
    if (out) *out = r->result;
    return TRG_OK;
}

int trg_serve_cancel(trg_server* s, uint64_t ticket) {
    if (!s) return TRG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return TRG_EINVAL;
    Request* r = it->second;
    if (r->state != Request::QUEUED) return TRG_ESTATE;   // running solves finish
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
    r->state = Request::CANCELLED;
    ++s->cancelled;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    return TRG_OK;
}

int trg_serve_get_stats(trg_server* s, trg_serve_stats* out) {
    if (!s || !out) return TRG_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->cancelled = s->cancelled;
    out->running = s->running;
    out->queued = s->queue.size();
    out->bytes_in_use = s->in_use;
    out->peak_bytes = s->peak;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto q = [&](double p) {
            const double pos = p * (double)(v.size() - 1);
            const size_t lo = (size_t)std::floor(pos), hi = std::min(v.size() - 1, lo + 1);
            return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);
        };
        out->p50_latency_s = q(0.50);
        out->p99_latency_s = q(0.99);
        out->max_latency_s = v.back();
        const double span = secs(s->t_first_submit, s->t_last_done);
        out->solves_per_s = span > 0 ? (double)(s->completed + s->failed) / span : 0.0;
    }
    return TRG_OK;
}

int trg_serve_destroy(trg_server* s) {
    if (!s) return TRG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;   // queued requests are dropped; running ones finish first
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->all) delete kv.second;
    delete s;
    return TRG_OK;
}

int trg_batch_run(int device, const trg_solve_spec* specs, int n, const trg_server_config* cfg,
                  trg_solve_result* results) {
    if (!specs || !results || n < 0) return TRG_EINVAL;
    trg_server* s = nullptr;
    int st = trg_serve_create(&s, device, cfg);
    if (st != TRG_OK) return st;
    std::vector<uint64_t> tickets((size_t)n, 0);
    int first_err = TRG_OK;
    for (int i = 0; i < n; ++i) {
        st = trg_serve_submit(s, &specs[i], &tickets[(size_t)i]);
        if (st != TRG_OK) {
            std::memset(&results[i], 0, sizeof(results[i]));
            results[i].status = st;
            if (first_err == TRG_OK) first_err = st;
        }
    }
    for (int i = 0; i < n; ++i) {
        if (!tickets[(size_t)i]) continue;
        trg_serve_wait(s, tickets[(size_t)i], -1.0, &results[i]);
        if (results[i].status != TRG_OK && first_err == TRG_OK) first_err = results[i].status;
    }
    trg_serve_destroy(s);
    return first_err;
}

}  // extern "C"
