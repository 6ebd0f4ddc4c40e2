/*
 * Cyclic Jacobi eigensolver for a real symmetric matrix, FP64.
 *
 * ORACLE / TEST INFRASTRUCTURE ONLY.  Nothing in the GPU product path may
 * link, load or call this file; it exists so that tests and the CPU baseline
 * can check the CUDA path against an independent, obviously correct
 * computation.  It shares no code with the CUDA library.
 *
 * What it computes: the eigendecomposition A = V diag(w) V^T of the
 * environment matrix M of the HOTRG step.  The paper (Sec. 2, the SVD helper
 * of the coarse-graining listing) takes the SVD of M and keeps the leading
 * left singular vectors; M is a Gram matrix (symmetric positive
 * semi-definite), so its SVD and its eigendecomposition coincide and the
 * leading left singular vectors are the eigenvectors of the largest
 * eigenvalues.
 *
 * Method: the classical cyclic-by-row Jacobi iteration (Jacobi 1846; see
 * Golub & Van Loan, "Matrix Computations", sec. 8.5).  Each sweep visits every
 * off-diagonal pair (p, q), p < q, once and applies the plane rotation that
 * annihilates a[p][q]:
 *     tau = (a_qq - a_pp) / (2 a_pq),
 *     t   = sign(tau) / (|tau| + sqrt(1 + tau^2))     (the smaller root),
 *     c   = 1 / sqrt(1 + t^2),  s = t c,
 * A <- J^T A J and V <- V J with J the identity except J_pp = J_qq = c,
 * J_pq = s, J_qp = -s.  Sweeps stop when the off-diagonal Frobenius norm is
 * at most tol times the Frobenius norm of A (or after max_sweeps).
 *
 * A rotation is skipped when |a_pq| <= tol * sqrt(|a_pp a_qq|) (the
 * relative-accuracy threshold of Demmel & Veselic, SIAM J. Matrix Anal. Appl.
 * 13 (1992) 1204) or when a_pq is below 1e-300 times ||A||_F; a sweep that
 * performs no rotation also ends the iteration.  The environment matrices
 * are strongly graded (eigenvalues over many decades), and the threshold
 * keeps the small eigenvalues accurate without rotating on rounding noise.
 *
 * No blocking, no parallel ordering: one rotation at a time, in order.
 * Eigenvectors are accumulated as the rows of V^T (contiguous updates).
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

static double off_norm2(int n, const double *a) {
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j) s += a[(size_t)i * n + j] * a[(size_t)i * n + j];
    return s;
}

static double frob_norm2(int n, const double *a) {
    double s = 0.0;
    for (size_t i = 0; i < (size_t)n * n; ++i) s += a[i] * a[i];
    return s;
}

/*
 * n        matrix order (n >= 1)
 * a        n*n row-major symmetric matrix; overwritten (diagonalised)
 * w        out: n eigenvalues, in the order of the diagonal (unsorted)
 * vt       out: n*n row-major; ROW k is the eigenvector of w[k]
 * tol      relative stopping tolerance on the off-diagonal norm
 * max_sweeps  upper bound on sweeps
 * sweeps_out  out (nullable): sweeps performed
 * returns  0 on convergence, 1 if max_sweeps was reached first, -1 on bad args
 */
int oracle_jacobi_eigh(int n, double *a, double *w, double *vt, double tol,
                       int max_sweeps, int *sweeps_out) {
    if (n < 1 || !a || !w || !vt || max_sweeps < 0) return -1;
    memset(vt, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) vt[(size_t)i * n + i] = 1.0;

    const double fro2 = frob_norm2(n, a);
    const double floor_abs = 1e-300 * sqrt(fro2);
    int sweep = 0;
    int status = 1;
    for (; sweep <= max_sweeps; ++sweep) {
        double off2 = off_norm2(n, a);
        if (off2 <= tol * tol * fro2) { status = 0; break; }
        if (sweep == max_sweeps) break;
        long rotations = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                const double app = a[(size_t)p * n + p];
                const double aqq = a[(size_t)q * n + q];
                if (fabs(apq) <= floor_abs || fabs(apq) <= tol * sqrt(fabs(app * aqq))) continue;
                ++rotations;
                const double tau = (aqq - app) / (2.0 * apq);
                double t;
                if (tau >= 0.0)
                    t = 1.0 / (tau + sqrt(1.0 + tau * tau));
                else
                    t = -1.0 / (-tau + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                /* columns p and q of A J (all rows) */
                for (int k = 0; k < n; ++k) {
                    const double akp = a[(size_t)k * n + p];
                    const double akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                /* rows p and q of J^T (A J) */
                for (int k = 0; k < n; ++k) {
                    const double apk = a[(size_t)p * n + k];
                    const double aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                /* the rotation annihilates a_pq exactly in exact arithmetic */
                a[(size_t)p * n + q] = 0.0;
                a[(size_t)q * n + p] = 0.0;
                /* V <- V J, i.e. rows p and q of V^T */
                for (int k = 0; k < n; ++k) {
                    const double vpk = vt[(size_t)p * n + k];
                    const double vqk = vt[(size_t)q * n + k];
                    vt[(size_t)p * n + k] = c * vpk - s * vqk;
                    vt[(size_t)q * n + k] = s * vpk + c * vqk;
                }
            }
        }
        if (rotations == 0) { status = 0; ++sweep; break; }
    }
    for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
    if (sweeps_out) *sweeps_out = sweep;
    return status;
}
