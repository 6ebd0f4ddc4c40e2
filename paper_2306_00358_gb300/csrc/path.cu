// The HOTRG half-step as flattened matrix products (Sec. 2, coarse-graining
// listing): environment M, U.T.T.U contraction, plus the offset tables that
// turn the index wiring (and the y-direction rotation) into plain GEMMs.
#include <algorithm>
#include <cstring>
#include <sstream>

#include "internal.h"

namespace trg {

std::vector<int64_t> build_table(const std::vector<std::pair<int64_t, int64_t>>& modes) {
    int64_t total = 1;
    for (auto& m : modes) total *= m.first;
    std::vector<int64_t> out((size_t)std::max<int64_t>(total, 0));
    if (total <= 0) return out;
    std::vector<int64_t> idx(modes.size(), 0);
    for (int64_t e = 0; e < total; ++e) {
        int64_t off = 0;
        for (size_t q = 0; q < modes.size(); ++q) off += idx[q] * modes[q].second;
        out[(size_t)e] = off;
        for (int q = (int)modes.size() - 1; q >= 0; --q) {
            if (++idx[(size_t)q] < modes[(size_t)q].first) break;
            idx[(size_t)q] = 0;
        }
    }
    return out;
}

const int64_t* Ctx::table(const std::vector<std::pair<int64_t, int64_t>>& modes) {
    std::ostringstream key;
    for (auto& m : modes) key << m.first << ':' << m.second << ';';
    auto it = tables.find(key.str());
    if (it != tables.end()) return it->second.as<int64_t>();
    std::vector<int64_t> h = build_table(modes);
    Buf b;
    ensure(b, std::max<size_t>(8, h.size() * sizeof(int64_t)));
    if (!h.empty())
        TRG_CUDA(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    // the host vector dies here: wait for the copy (tables are built once per shape)
    TRG_CUDA(cudaStreamSynchronize(stream));
    tables[key.str()] = b;
    return b.as<int64_t>();
}

using Modes = std::vector<std::pair<int64_t, int64_t>>;

static bool unit_first_stride(const Modes& m) {
    // consecutive flat indices are adjacent iff the fastest mode has stride 1
    return !m.empty() && m.back().second == 1 && m.back().first > 1;
}

static Gather gather(Ctx& ctx, const double* base, const Modes& rows, const Modes& cols) {
    Gather g;
    g.base = base;
    g.off_r = ctx.table(rows);
    g.off_c = ctx.table(cols);
    g.c_fast = unit_first_stride(cols);
    g.c_identity = cols.size() == 1 && cols[0].second == 1;
    return g;
}

void gemm_split(Ctx& ctx, const GemmDesc& g);  // split_gemm.cu

void gemm(Ctx& ctx, const GemmDesc& g, int precision) {
    // products inside the isometry are timed as part of that phase
    const int tok = (ctx.phase == TRG_PHASE_EIG) ? -1 : ctx.region_begin(ctx.phase);
    if (precision == TRG_FP64) gemm_f64(ctx, g);
    else if (precision == TRG_SPLIT_BF16) gemm_split(ctx, g);
    else fail(TRG_EINVAL, "unknown precision mode");
    ctx.region_end(tok, 2.0 * (double)g.M * (double)g.N * (double)g.K, 0.0);
}

int slices_now(const Ctx& ctx) {
    const bool env = ctx.phase == TRG_PHASE_ENV || ctx.phase == TRG_PHASE_EIG;
    return (env && ctx.cfg.env_slices) ? ctx.cfg.env_slices : ctx.cfg.split_slices;
}

int precision_for_step(const Ctx& ctx, int step, int64_t dd) {
    if (ctx.cfg.precision == TRG_FP64) return TRG_FP64;
    if (step - 1 < ctx.cfg.split_from_step || dd <= ctx.cfg.fp64_max_dd) return TRG_FP64;
    return ctx.cfg.precision;
}

// M[(i,j),(k,l)] = sum_{e,f} Q[i,e,k,f] P[j,e,l,f],
// P[j,e,l,f] = sum_{a,b} t[j,a,b,e] t[l,a,b,f]   (upper pair, bond e / f)
// Q[i,e,k,f] = sum_{c,d} t[i,e,c,d] t[k,f,c,d]   (lower pair)
void environment(Ctx& ctx, const View4& t, double* M, int precision) {
    const int64_t Dx = t.n[0], Dy = t.n[1];
    const int64_t* s = t.s;
    const int64_t DD = Dx * Dy;
    ctx.ensure(ctx.envP, (size_t)(DD * DD) * sizeof(double));
    ctx.ensure(ctx.envQ, (size_t)(DD * DD) * sizeof(double));
    double* P = ctx.envP.as<double>();
    double* Q = ctx.envQ.as<double>();

    {   // P: rows (j,e), k (a,b), cols (l,f)
        const Modes r = {{Dx, s[0]}, {Dy, s[3]}}, k = {{Dy, s[1]}, {Dx, s[2]}};
        GemmDesc g;
        g.M = DD; g.N = DD; g.K = DD;
        g.A = gather(ctx, t.p, r, k);
        g.B = gather(ctx, t.p, k, r);
        g.C = P; g.c_m = ctx.table({{DD, DD}}); g.c_n = ctx.table({{DD, 1}});
        g.beta = 0.0;
        g.gram = true;          // P = A A^T (the SYRK of the environment)
        gemm(ctx, g, precision);
    }
    {   // Q: rows (i,e), k (c,d), cols (k,f)
        const Modes r = {{Dx, s[0]}, {Dy, s[1]}}, k = {{Dx, s[2]}, {Dy, s[3]}};
        GemmDesc g;
        g.M = DD; g.N = DD; g.K = DD;
        g.A = gather(ctx, t.p, r, k);
        g.B = gather(ctx, t.p, k, r);
        g.C = Q; g.c_m = ctx.table({{DD, DD}}); g.c_n = ctx.table({{DD, 1}});
        g.beta = 0.0;
        g.gram = true;          // Q = A A^T
        gemm(ctx, g, precision);
    }
    {   // M: rows (i,k), k (e,f), cols (j,l); stored M[(i,j),(k,l)]
        GemmDesc g;
        g.M = Dx * Dx; g.N = Dx * Dx; g.K = Dy * Dy;
        g.A = gather(ctx, Q, {{Dx, Dy * DD}, {Dx, Dy}}, {{Dy, DD}, {Dy, 1}});
        g.B = gather(ctx, P, {{Dy, DD}, {Dy, 1}}, {{Dx, Dy * DD}, {Dx, Dy}});
        g.C = M;
        g.c_m = ctx.table({{Dx, Dx * Dx * Dx}, {Dx, Dx}});
        g.c_n = ctx.table({{Dx, Dx * Dx}, {Dx, 1}});
        g.beta = 0.0;
        gemm(ctx, g, precision);
    }
}

// Tx[i,j,k,l] = sum U[a,b,i] t[b,j,d,c] t'[a,c,e,l] U[e,d,k], in slices of j
// (t = top, t' = bottom of the blocked pair):
//   X1[(jj,i,d),(c,a)] = sum_b U[a,b,i] t[b,j0+jj,d,c]          (D^6)
//   X2[(jj,i,l),(e,d)] = sum_{c,a} X1[(jj,i,d),(c,a)] t'[a,c,e,l] (D^7)
//   O[i,j0+jj,k,l]     = sum_{e,d} X2[(jj,i,l),(e,d)] U[e,d,k]    (D^6)
// The summed pair of each product is ordered with the producer's row index
// fastest ((c,a) and (e,d)), so a producer warp, whose lanes are adjacent
// rows, writes adjacent elements of its consumer's rows.  In split mode each
// producer either records the exponent fields of its consumer's rows (the
// consumer then skips the exponent pass over the D^5 intermediate) or, when
// the bond dimensions tile (32, 64, 128), writes the consumer's slices.
void contract(Ctx& ctx, const View4& top, const View4& bottom, const double* U, int64_t Dn, const View4& out,
              int precision, int64_t j_begin, int64_t j_end, int64_t j_out0) {
    const View4& t = top;
    if (bottom.n[0] != top.n[0] || bottom.n[1] != top.n[1] || bottom.n[2] != top.n[2] || bottom.n[3] != top.n[3])
        fail(TRG_EINVAL, "contract: the two tensors of a pair differ in shape");
    const int64_t Dx = t.n[0], Dy = t.n[1];
    const int64_t* s = t.s;
    const int64_t* sb = bottom.s;
    const int64_t* o = out.s;
    const int64_t DD = Dx * Dy;
    const bool split = precision == TRG_SPLIT_BF16;
    if (j_end < 0) j_end = Dy;
    if (j_begin < 0 || j_begin > j_end || j_end > Dy || j_out0 > j_begin)
        fail(TRG_EINVAL, "contract: bad j range");
    // Fused hand-over (split mode): when a consumer row of the next product is
    // Dx x Dx elements of one 128 x 128 output tile, the producer writes the
    // next product's A slices directly (bit-identical to slicing its FP64
    // output).  Done for X2 -> O: the D^7 product is tensor-bound, so the
    // heavier epilogue hides behind its MMAs and the slicing pass over X2
    // disappears.  X1 (K = Dx) is bound by its epilogue already; it keeps the
    // FP64 hand-over, whose epilogue is half as long as the slicing one.
    // fused_slices = 2 hands X1 over as slices too (same results, slower here).
    auto tiles_ok = [](int64_t v) { return v == 32 || v == 64 || v == 128; };
    const bool fuse = split && ctx.cfg.fused_slices >= 1 && tiles_ok(Dx);
    const bool fuse1 = split && ctx.cfg.fused_slices == 2 && tiles_ok(Dx) && tiles_ok(Dy);
    const int S = ctx.cfg.split_slices;
    const size_t ws_cap = ctx.cfg.workspace_bytes ? ctx.cfg.workspace_bytes : ((size_t)4 << 30);
    // bytes per j of each intermediate: FP64, or S BF16 slices (+ padding rows)
    const size_t elem = (fuse || fuse1) ? (size_t)std::max(8, 2 * S) : 8;
    const size_t per_j = (size_t)(2 * Dn * Dx * DD) * elem;
    int64_t jb = std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(1, j_end - j_begin), (int64_t)(ws_cap / per_j)));
    const int64_t rows2 = jb * Dn * Dx, rows3 = jb * Dn * Dy;   // A rows of the two consumers
    size_t r1 = (size_t)(rows2 * DD) * 8, r2 = (size_t)(rows3 * Dx * Dx) * 8;
    if (fuse1) r1 = std::max(r1, (size_t)S * split_rows_padded(ctx, rows2) * split_k_padded(DD) * 2);
    if (fuse) r2 = std::max(r2, (size_t)S * split_rows_padded(ctx, rows3) * split_k_padded(Dx * Dx) * 2);
    r1 = (r1 + 255) & ~(size_t)255;
    ctx.ensure(ctx.ws, r1 + r2);
    double* X1 = ctx.ws.as<double>();
    double* X2 = (double*)(ctx.ws.as<uint8_t>() + r1);
    int* ef2 = nullptr;
    int* ef3 = nullptr;
    if (split) {
        ctx.ensure(ctx.cons_ef, (size_t)(rows2 + rows3) * sizeof(int));
        ef2 = ctx.cons_ef.as<int>();
        ef3 = ef2 + rows2;
    }

    // Operands that are the same for every j-block -- U as X1's A, the
    // bottom tensor as the D^7 product's B, U as the last product's B -- are
    // sliced once, before the first block, when there are several blocks.
    const Gather a1 = gather(ctx, U, {{Dn, 1}, {Dx, Dx * Dn}}, {{Dx, Dn}});
    const Gather b2 = gather(ctx, bottom.p, {{Dy, sb[1]}, {Dx, sb[0]}}, {{Dy, sb[3]}, {Dx, sb[2]}});
    const Gather b3 = gather(ctx, U, {{Dx, Dx * Dn}, {Dx, Dn}}, {{Dn, 1}});
    struct Pre { const uint16_t* s = nullptr; const int* e = nullptr; } p1, p2, p3;
    if (split && j_end - j_begin > jb) {
        auto bytes = [](int64_t rows, int64_t k, int S_) {
            const size_t sl = ((size_t)S_ * rows * split_k_padded(k) * 2 + 255) & ~(size_t)255;
            return sl + (((size_t)rows * sizeof(int) + 255) & ~(size_t)255);
        };
        const int64_t r1 = split_rows_padded(ctx, Dx * Dn), r2 = split_cols_padded(DD), r3 = split_cols_padded(Dn);
        const size_t n1 = bytes(r1, Dx, S), n2 = bytes(r2, DD, S), n3 = bytes(r3, Dx * Dx, S);
        ctx.ensure(ctx.bslices, n1 + n2 + n3);
        uint8_t* base = ctx.bslices.as<uint8_t>();
        auto place = [&](uint8_t* at, int64_t rows, int64_t k, Pre& p) {
            const size_t sl = ((size_t)S * rows * split_k_padded(k) * 2 + 255) & ~(size_t)255;
            p.s = (const uint16_t*)at;
            p.e = (const int*)(at + sl);
        };
        place(base, r1, Dx, p1);
        place(base + n1, r2, DD, p2);
        place(base + n1 + n2, r3, Dx * Dx, p3);
        ctx.phase = TRG_PHASE_X1;
        int tok = ctx.region_begin(TRG_PHASE_X1);
        split_slice_operand(ctx, a1, Dx * Dn, Dx, const_cast<uint16_t*>(p1.s), const_cast<int*>(p1.e));
        ctx.region_end(tok, 0.0, 0.0);
        ctx.phase = TRG_PHASE_X2;
        tok = ctx.region_begin(TRG_PHASE_X2);
        split_slice_b(ctx, b2, DD, DD, const_cast<uint16_t*>(p2.s), const_cast<int*>(p2.e));
        ctx.region_end(tok, 0.0, 0.0);
        ctx.phase = TRG_PHASE_X3;
        tok = ctx.region_begin(TRG_PHASE_X3);
        split_slice_b(ctx, b3, Dx * Dx, Dn, const_cast<uint16_t*>(p3.s), const_cast<int*>(p3.e));
        ctx.region_end(tok, 0.0, 0.0);
    }

    for (int64_t j0 = j_begin; j0 < j_end; j0 += jb) {
        const int64_t jn = std::min(jb, j_end - j0);
        const int64_t M2 = jn * Dn * Dx, M3 = jn * Dn * Dy;       // rows of this block's X2 / O products
        {   // X1[(jj,i,d),(c,a)] = sum_b U[a,b,i] t[b,j0+jj,d,c]: rows (i,a), a fastest,
            // so a warp's lanes hold adjacent a (adjacent in X1, one consumer row)
            ctx.phase = TRG_PHASE_X1;
            GemmDesc g;
            g.M = Dx * Dn; g.N = jn * DD; g.K = Dx;
            g.A = a1;
            g.a_slices = p1.s;
            g.a_e = p1.e;
            g.B = gather(ctx, t.p + j0 * s[1], {{Dx, s[0]}}, {{jb, s[1]}, {Dx, s[2]}, {Dy, s[3]}});
            // consumer row of element ((i,a),(jj,d,c)) is (jj,i,d), its column c Dx + a
            g.cons_m = ctx.table({{Dn, Dx}, {Dx, 0}});
            g.cons_n = ctx.table({{jb, Dn * Dx}, {Dx, 1}, {Dy, 0}});
            if (fuse1) {
                g.C = nullptr;
                g.cs_out = (uint16_t*)X1;
                g.cs_mp = split_rows_padded(ctx, M2);
                g.cs_kp = split_k_padded(DD);
                g.cs_e = ef2;
                g.ck_m = ctx.table({{Dn, 0}, {Dx, 1}});
                g.ck_n = ctx.table({{jb, 0}, {Dx, 0}, {Dy, Dx}});
                g.ck_stride = Dx;
                g.rows_per_crow = (int)Dx;
                g.cols_per_crow = (int)Dy;
            } else {
                g.C = X1;
                g.c_m = ctx.table({{Dn, Dx * DD}, {Dx, 1}});
                g.c_n = ctx.table({{jb, Dn * Dx * DD}, {Dx, DD}, {Dy, Dx}});
                g.c_rows_fast = Dy % 32 == 0;
                g.c_col_stride = Dx;
                if (split) {
                    TRG_CUDA(cudaMemsetAsync(ef2, 0, (size_t)rows2 * sizeof(int), ctx.stream));
                    g.cons_ef = ef2;
                } else {
                    g.cons_m = g.cons_n = nullptr;
                }
            }
            gemm(ctx, g, precision);
        }
        {   // X2[(jj,i,l),(e,d)] = sum_{c,a} X1[(jj,i,d),(c,a)] t[a,c,e,l]  (the D^7 product):
            // rows (jj,i,d), d fastest; columns (l,e), e fastest
            ctx.phase = TRG_PHASE_X2;
            GemmDesc g;
            g.M = M2; g.N = DD; g.K = DD;
            g.A = gather(ctx, X1, {{jb * Dn * Dx, DD}}, {{DD, 1}});
            g.B = b2;
            g.b_slices = p2.s;
            g.b_e = p2.e;
            // consumer row of element ((jj,i,d),(l,e)) is (jj,i,l), its column e Dx + d
            g.cons_m = ctx.table({{jb * Dn, Dy}, {Dx, 0}});
            g.cons_n = ctx.table({{Dy, 1}, {Dx, 0}});
            if (fuse1) {
                g.a_slices = (const uint16_t*)X1;
                g.a_e = ef2;
            } else if (split) {
                g.a_ef = ef2;
            }
            if (fuse) {
                g.C = nullptr;
                g.cs_out = (uint16_t*)X2;
                g.cs_mp = split_rows_padded(ctx, M3);
                g.cs_kp = split_k_padded(Dx * Dx);
                g.cs_e = ef3;
                g.ck_m = ctx.table({{jb * Dn, 0}, {Dx, 1}});
                g.ck_n = ctx.table({{Dy, 0}, {Dx, Dx}});
                g.ck_stride = Dx;
                g.rows_per_crow = (int)Dx;
                g.cols_per_crow = (int)Dx;
            } else {
                g.C = X2;
                g.c_m = ctx.table({{jb * Dn, Dy * Dx * Dx}, {Dx, 1}});
                g.c_n = ctx.table({{Dy, Dx * Dx}, {Dx, Dx}});
                g.c_rows_fast = Dx % 32 == 0;
                g.c_col_stride = Dx;
                if (split) {
                    TRG_CUDA(cudaMemsetAsync(ef3, 0, (size_t)rows3 * sizeof(int), ctx.stream));
                    g.cons_ef = ef3;
                } else {
                    g.cons_m = g.cons_n = nullptr;
                }
            }
            gemm(ctx, g, precision);
        }
        {   // O[i,j0+jj,k,l] = sum_{e,d} X2[(jj,i,l),(e,d)] U[e,d,k]
            ctx.phase = TRG_PHASE_X3;
            GemmDesc g;
            g.M = M3; g.N = Dn; g.K = Dx * Dx;
            g.A = gather(ctx, X2, {{jb * Dn * Dy, Dx * Dx}}, {{Dx * Dx, 1}});
            g.B = b3;
            g.b_slices = p3.s;
            g.b_e = p3.e;
            g.C = out.p + (j0 - j_out0) * o[1];
            g.c_m = ctx.table({{jb, o[1]}, {Dn, o[0]}, {Dy, o[3]}});
            g.c_n = ctx.table({{Dn, o[2]}});
            if (fuse) {
                g.a_slices = (const uint16_t*)X2;
                g.a_e = ef3;
            } else if (split) {
                g.a_ef = ef3;
            }
            gemm(ctx, g, precision);
        }
    }
}

}  // namespace trg
