// The blocking step on the cubic lattice, the direction the paper leaves to
// future work (Sec. 1, Sec. 4).  It is the 2D variant of Sec. 2 (the
// coarse-graining listing) with a third pair of legs: the tensor
// t[x, x', y, y', z, z'] (left, right, front, back, down, up) is stacked
// along z with a copy of itself, the left/right pairs are truncated by one
// isometry U_x taken from the environment of the two left legs, the
// front/back pairs by U_y from the two front legs, and the next axis is
// brought into the z slot by a rotation of the view (no copy).  Every
// product is one split (or FP64) GEMM over offset tables.
#include <algorithm>

#include "internal.h"

namespace trg {

namespace {

using Modes = std::vector<std::pair<int64_t, int64_t>>;

int64_t count(const Modes& m) {
    int64_t n = 1;
    for (auto& x : m) n *= x.first;
    return n;
}

// C[rows, cols] (+)= sum_k A[rows, k] B[k, cols]; every operand a strided
// multi-index given as (size, stride) modes, first mode slowest.
void product(Ctx& ctx, const double* A, const Modes& ar, const Modes& ak, const double* B, const Modes& bk,
             const Modes& bc, double* C, const Modes& cr, const Modes& cc, int precision) {
    GemmDesc g;
    g.M = count(ar);
    g.K = count(ak);
    g.N = count(bc);
    if (count(bk) != g.K || count(cr) != g.M || count(cc) != g.N) fail(TRG_EINVAL, "product: mode sizes differ");
    g.A.base = A;
    g.A.off_r = ctx.table(ar);
    g.A.off_c = ctx.table(ak);
    g.A.c_fast = !ak.empty() && ak.back().second == 1 && ak.back().first > 1;
    g.A.c_identity = ak.size() == 1 && ak[0].second == 1;
    g.B.base = B;
    g.B.off_r = ctx.table(bk);
    g.B.off_c = ctx.table(bc);
    g.B.c_fast = !bc.empty() && bc.back().second == 1 && bc.back().first > 1;
    g.B.c_identity = bc.size() == 1 && bc[0].second == 1;
    g.C = C;
    g.c_m = ctx.table(cr);
    g.c_n = ctx.table(cc);
    g.beta = 0.0;
    gemm(ctx, g, precision);
}

// Environment of the pair of legs `a` (0: left, 2: front) of the z-stacked
// pair, rows and columns (lower leg, upper leg):
//   M[(a1,a2),(b1,b2)] = sum_{m,n} P1[(a1,m),(b1,n)] P2[(a2,m),(b2,n)],
//   P1 = the lower tensor over its legs other than `a` and its up leg m,
//   P2 = the upper tensor over its legs other than `a` and its down leg m.
void environment_pair(Ctx& ctx, const View6& t, int a, double* P1, double* P2, double* M, int precision) {
    const int64_t Da = t.n[a], Dz = t.n[4];
    const int64_t* s = t.s;
    Modes k1, k2;   // summed legs of P1 (all but a and 5) and of P2 (all but a and 4)
    for (int leg = 0; leg < 6; ++leg) {
        if (leg == a) continue;
        if (leg != 5) k1.push_back({t.n[leg], s[leg]});
        if (leg != 4) k2.push_back({t.n[leg], s[leg]});
    }
    const int64_t R = Da * Dz;
    product(ctx, t.p, {{Da, s[a]}, {Dz, s[5]}}, k1, t.p, k1, {{Da, s[a]}, {Dz, s[5]}}, P1, {{R, R}}, {{R, 1}},
            precision);
    product(ctx, t.p, {{Da, s[a]}, {Dz, s[4]}}, k2, t.p, k2, {{Da, s[a]}, {Dz, s[4]}}, P2, {{R, R}}, {{R, 1}},
            precision);
    // rows (a1, b1), K (m, n), cols (a2, b2); stored M[(a1,a2),(b1,b2)]
    product(ctx, P1, {{Da, Dz * R}, {Da, Dz}}, {{Dz, R}, {Dz, 1}}, P2, {{Dz, R}, {Dz, 1}}, {{Da, Dz * R}, {Da, Dz}},
            M, {{Da, Da * Da * Da}, {Da, Da}}, {{Da, Da * Da}, {Da, 1}}, precision);
}

}  // namespace

// One z step.  Products, with Nx = min(Dx^2, Dcut) and Ny = min(Dy^2, Dcut):
//   A[X,x2,x1',y1,y1',z,m]   = sum_x1  U_x[(x1,x2),X]   t[x1,x1',y1,y1',z,m]
//   W[x2,x1',m,X',y2,y2',z'] = sum_x2' U_x[(x1',x2'),X'] t[x2,x2',y2,y2',m,z']
// (U_x on the upper tensor's right leg, with the lower tensor's right leg x1'
// still open), then for each X (bounding the intermediates to D^7):
//   C[(y1,y1',z),(X',y2,y2',z')] = sum_{x2,x1',m} A[X,...] W[...]        (the D^10 part, K = D^3)
//   D[(y1',z,X',y2',z'),Y]       = sum_{y1,y2} C U_y[(y1,y2),Y]
//   out[X,X',Y,Y',z,z']          = sum_{y1',y2'} D U_y[(y1',y2'),Y']
std::pair<int64_t, int64_t> step3(Ctx& ctx, const View6& t, int dcut, int step, double* out, int precision,
                                  std::vector<double>& lam_x, std::vector<double>& lam_y) {
    const int64_t Dx = t.n[0], Dy = t.n[2], Dz = t.n[4];
    if (t.n[1] != Dx || t.n[3] != Dy || t.n[5] != Dz) fail(TRG_EINVAL, "step3: paired legs differ in size");
    const int64_t* s = t.s;
    const int64_t nx = Dx * Dx, ny = Dy * Dy;
    const int64_t Nx = std::min<int64_t>(nx, dcut), Ny = std::min<int64_t>(ny, dcut);

    // environments and isometries
    ctx.phase = TRG_PHASE_ENV;
    const int64_t R = std::max(Dx, Dy) * Dz;
    ctx.ensure(ctx.s3[0], (size_t)(R * R) * sizeof(double));
    ctx.ensure(ctx.s3[1], (size_t)(R * R) * sizeof(double));
    ctx.ensure(ctx.s3[4], (size_t)(nx * nx) * sizeof(double));
    ctx.ensure(ctx.s3[5], (size_t)(ny * ny) * sizeof(double));
    ctx.ensure(ctx.s3[2], (size_t)(nx * Nx) * sizeof(double));
    ctx.ensure(ctx.s3[3], (size_t)(ny * Ny) * sizeof(double));
    double* P1 = ctx.s3[0].as<double>();
    double* P2 = ctx.s3[1].as<double>();
    double* Mx = ctx.s3[4].as<double>();
    double* My = ctx.s3[5].as<double>();
    double* Ux = ctx.s3[2].as<double>();
    double* Uy = ctx.s3[3].as<double>();
    int64_t kx = Nx, ky = Ny;
    ctx.phase = TRG_PHASE_EIG;
    if (Nx == nx) {
        launch_identity(ctx, Ux, nx);
    } else {
        ctx.phase = TRG_PHASE_ENV;
        environment_pair(ctx, t, 0, P1, P2, Mx, precision);
        ctx.phase = TRG_PHASE_EIG;
        std::vector<double> lam;
        kx = isometry(ctx, Mx, nx, dcut, Ux, lam, 2 * step, precision);
        lam_x = lam;
    }
    if (Ny == ny) {
        launch_identity(ctx, Uy, ny);
    } else {
        ctx.phase = TRG_PHASE_ENV;
        environment_pair(ctx, t, 2, P1, P2, My, precision);
        ctx.phase = TRG_PHASE_EIG;
        std::vector<double> lam;
        ky = isometry(ctx, My, ny, dcut, Uy, lam, 2 * step + 1, precision);
        lam_y = lam;
    }
    // the isometries are row-major (n x kept); a multiplet rule may keep
    // fewer vectors than Dcut
    const int64_t ldx = kx, ldy = ky;

    // contraction
    const int64_t L = Dx * Dy * Dy * Dz * Dz;          // columns of A per (X, x2)
    const int64_t nw = kx * Dy * Dy * Dz;              // (X', y2, y2', z'): columns of W and C
    const int64_t rcx = Dy * Dy * Dz;                  // (y1, y1', z): rows of C
    const int64_t rd = Dy * Dz * kx * Dy * Dz;         // rows of D
    ctx.ensure(ctx.s3[6], (size_t)(kx * Dx * L) * sizeof(double));
    ctx.ensure(ctx.s3[7], (size_t)(Dx * Dx * Dz * nw) * sizeof(double));
    ctx.ensure(ctx.s3[8], (size_t)(rcx * nw) * sizeof(double));
    ctx.ensure(ctx.s3[9], (size_t)(rd * ky) * sizeof(double));
    double* A = ctx.s3[6].as<double>();
    double* W = ctx.s3[7].as<double>();
    double* C = ctx.s3[8].as<double>();
    double* D = ctx.s3[9].as<double>();

    ctx.phase = TRG_PHASE_X1;
    // A: rows (X, x2), K x1, cols (x1', y1, y1', z, m)
    product(ctx, Ux, {{kx, 1}, {Dx, ldx}}, {{Dx, Dx * ldx}}, t.p, {{Dx, s[0]}},
            {{Dx, s[1]}, {Dy, s[2]}, {Dy, s[3]}, {Dz, s[4]}, {Dz, s[5]}}, A, {{kx * Dx, L}}, {{L, 1}}, precision);
    // W, stored [x2][x1'][m][X'][y2][y2'][z']: rows (x1', X'), K x2', cols (x2, y2, y2', m, z')
    const int64_t w_m = nw, w_x1 = Dz * nw, w_x2 = Dx * Dz * nw;
    product(ctx, Ux, {{Dx, Dx * ldx}, {kx, 1}}, {{Dx, ldx}}, t.p, {{Dx, s[1]}},
            {{Dx, s[0]}, {Dy, s[2]}, {Dy, s[3]}, {Dz, s[4]}, {Dz, s[5]}}, W, {{Dx, w_x1}, {kx, Dy * Dy * Dz}},
            {{Dx, w_x2}, {Dy, Dy * Dz}, {Dy, Dz}, {Dz, w_m}, {Dz, 1}}, precision);
    const int64_t out_x = kx * ky * ky * Dz * Dz;      // output stride of X
    for (int64_t X = 0; X < kx; ++X) {
        const double* AX = A + X * Dx * L;
        ctx.phase = TRG_PHASE_X2;
        // C: rows (y1, y1', z), K (x2, x1', m), cols (X', y2, y2', z') (contiguous in W)
        product(ctx, AX, {{Dy, Dy * Dz * Dz}, {Dy, Dz * Dz}, {Dz, Dz}}, {{Dx, L}, {Dx, Dy * Dy * Dz * Dz}, {Dz, 1}}, W,
                {{Dx, w_x2}, {Dx, w_x1}, {Dz, w_m}}, {{nw, 1}}, C, {{rcx, nw}}, {{nw, 1}}, precision);
        ctx.phase = TRG_PHASE_X3;
        // D: rows (y1', z, X', y2', z'), K (y1, y2), cols Y
        product(ctx, C, {{Dy, Dz * nw}, {Dz, nw}, {kx, Dy * Dy * Dz}, {Dy, Dz}, {Dz, 1}},
                {{Dy, Dy * Dz * nw}, {Dy, Dy * Dz}}, Uy, {{Dy, Dy * ldy}, {Dy, ldy}}, {{ky, 1}}, D, {{rd, ky}},
                {{ky, 1}}, precision);
        // out: rows (X', Y, z, z'), K (y1', y2'), cols Y'
        const int64_t dz = kx * Dy * Dz * ky;           // stride of z in D
        product(ctx, D, {{kx, Dy * Dz * ky}, {ky, 1}, {Dz, dz}, {Dz, ky}}, {{Dy, Dz * dz}, {Dy, Dz * ky}}, Uy,
                {{Dy, Dy * ldy}, {Dy, ldy}}, {{ky, 1}}, out + X * out_x,
                {{kx, ky * ky * Dz * Dz}, {ky, ky * Dz * Dz}, {Dz, Dz}, {Dz, 1}}, {{ky, Dz * Dz}}, precision);
    }
    return {kx, ky};
}

}  // namespace trg
