/*
 * Oracle (test infrastructure only): singular values of C - zI by a plain
 * one-sided (Hestenes) Jacobi SVD in IEEE double precision.
 *
 * The quantity is the one that defines the epsilon-pseudospectrum (Sec. 1,
 * eqs. (defSquare)/(defSquareSVD)): sigma_min(C - zI), with membership
 * sigma_min < eps (strict).  Nothing here follows the paper's algorithms; it
 * is the plain definition: form A = C - zI from the ORIGINAL dense matrix C
 * (never from a Schur factor), orthogonalise its columns by complex plane
 * rotations until every pair satisfies |a_i^H a_j| <= tol*||a_i||*||a_j||
 * (a column below tol*||A||_F, rounding noise, counts as orthogonal to all:
 * see rotate_pair), and read the singular values off as the column norms.
 *
 * No LAPACK, no BLAS, no code shared with the CUDA library.  Rotations use a
 * round-robin (tournament) pair ordering so that the n/2 pairs of a round are
 * disjoint and can run on separate OpenMP threads; the ordering does not
 * change the result being computed (the SVD), only the rounding path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double *re, *im; /* column-major m x n planes */
    int64_t m, n;
} ormat;

/* inner products of columns i and j: alpha = ||a_i||^2, beta = ||a_j||^2,
 * gamma = a_i^H a_j (complex) */
static void col_dots(const ormat *A, int64_t i, int64_t j, double *alpha, double *beta,
                     double *gr, double *gi) {
    const double *ar = A->re + i * A->m, *ai = A->im + i * A->m;
    const double *br = A->re + j * A->m, *bi = A->im + j * A->m;
    double sa = 0, sb = 0, sr = 0, si = 0;
    for (int64_t k = 0; k < A->m; k++) {
        sa += ar[k] * ar[k] + ai[k] * ai[k];
        sb += br[k] * br[k] + bi[k] * bi[k];
        /* conj(a) * b */
        sr += ar[k] * br[k] + ai[k] * bi[k];
        si += ar[k] * bi[k] - ai[k] * br[k];
    }
    *alpha = sa; *beta = sb; *gr = sr; *gi = si;
}

/* One Hestenes rotation on the column pair (i, j).  Returns the pair's
 * relative off-orthogonality |gamma|/sqrt(alpha*beta) before the rotation, or
 * 0 for a pair that counts as orthogonal.
 *
 * A column whose squared norm is at most small2 = (tol ||A||_F)^2 counts as
 * orthogonal to every other.  Such a column is rounding noise: floating point
 * cannot orthogonalise it further (a rotation shrinks it by about one
 * rounding unit at a time, or leaves its direction noise), so the sweeps
 * would stall short of the test.  Setting it to zero would move every
 * singular value by at most its norm (Weyl's bound for a rank-one change),
 * tol ||A||_F, which is the absolute accuracy the oracle is held to.  Every
 * column is A Q e_j for a unitary Q, so its norm is at least sigma_min; the
 * rule therefore acts only where sigma_min(C - zI) <= tol ||C - zI||_F. */
static double rotate_pair(ormat *A, int64_t i, int64_t j, double tol, double small2) {
    double alpha, beta, gr, gi;
    col_dots(A, i, j, &alpha, &beta, &gr, &gi);
    double g = hypot(gr, gi);
    if (alpha == 0.0 || beta == 0.0 || g == 0.0) return 0.0;
    if (alpha <= small2 || beta <= small2) return 0.0;
    double rel = g / sqrt(alpha) / sqrt(beta);
    if (rel <= tol) return rel;
    /* Gram of the pair [[alpha, gamma],[conj(gamma), beta]].  Scale column j
     * by exp(-i*phi) (gamma = g*exp(i*phi)) to make the off-diagonal real,
     * then a real symmetric Jacobi rotation [[c, s], [-s, c]] diagonalises it:
     * zeta = (beta - alpha)/(2g), t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)). */
    double er = gr / g, ei = -gi / g; /* exp(-i*phi) */
    double zeta = (beta - alpha) / (2.0 * g);
    double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    double c = 1.0 / sqrt(1.0 + t * t);
    double s = c * t;
    double *ar = A->re + i * A->m, *ai = A->im + i * A->m;
    double *br = A->re + j * A->m, *bi = A->im + j * A->m;
    for (int64_t k = 0; k < A->m; k++) {
        /* b' = exp(-i*phi) * b */
        double pr = er * br[k] - ei * bi[k];
        double pi = er * bi[k] + ei * br[k];
        double xr = ar[k], xi = ai[k];
        ar[k] = c * xr - s * pr;
        ai[k] = c * xi - s * pi;
        br[k] = s * xr + c * pr;
        bi[k] = s * xi + c * pi;
    }
    return rel;
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Jacobi SVD of the m x n matrix held in A (overwritten).  Writes the n
 * singular values in ascending order and returns the number of sweeps; *off
 * receives the largest relative off-orthogonality seen in the final sweep.
 * nthreads > 1 parallelises the disjoint pairs of each round.  max_rounds >= 0
 * stops after that many rounds (a timing sample; the values are then not the
 * converged ones); -1 = no limit. */
static int jacobi_sweeps(ormat *A, double tol, int max_sweeps, int nthreads, double *sigma,
                         double *off, int64_t max_rounds) {
    int64_t n = A->n;
    int64_t np = (n % 2) ? n + 1 : n; /* odd n: one dummy column sits out */
    int64_t *ring = (int64_t *)malloc(sizeof(int64_t) * np);
    for (int64_t k = 0; k < np; k++) ring[k] = k;
    /* ||A||_F^2, which the rotations keep */
    double fro2 = 0.0;
    for (int64_t k = 0; k < A->m * n; k++) fro2 += A->re[k] * A->re[k] + A->im[k] * A->im[k];
    const double small2 = tol * tol * fro2;
    int sweep = 0;
    double worst = 0.0;
    int64_t rounds_done = 0;
    for (sweep = 0; sweep < max_sweeps; sweep++) {
        worst = 0.0;
        for (int64_t round = 0; round < np - 1; round++) {
            if (max_rounds >= 0 && rounds_done >= max_rounds) break;
            rounds_done++;
            double wr = 0.0;
            int64_t half = np / 2;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) reduction(max : wr) schedule(static) if (nthreads > 1)
#endif
            for (int64_t q = 0; q < half; q++) {
                int64_t a = ring[q], b = ring[np - 1 - q];
                if (a >= n || b >= n) continue;
                int64_t i = a < b ? a : b, j = a < b ? b : a;
                double rel = rotate_pair(A, i, j, tol, small2);
                if (rel > wr) wr = rel;
            }
            if (wr > worst) worst = wr;
            /* tournament rotation: element 0 fixed, the others shift by one */
            int64_t last = ring[np - 1];
            for (int64_t k = np - 1; k > 1; k--) ring[k] = ring[k - 1];
            ring[1] = last;
        }
        if (max_rounds >= 0 && rounds_done >= max_rounds) break;
        if (worst <= tol) { sweep++; break; }
    }
    free(ring);
    for (int64_t k = 0; k < n; k++) {
        const double *ar = A->re + k * A->m, *ai = A->im + k * A->m;
        double s = 0;
        for (int64_t r = 0; r < A->m; r++) s += ar[r] * ar[r] + ai[r] * ai[r];
        sigma[k] = sqrt(s);
    }
    qsort(sigma, (size_t)n, sizeof(double), cmp_double);
    *off = worst;
    return sweep;
}

/* Full singular spectrum of (C - z I) for one z.
 *   C       : interleaved complex (re, im) column-major, m x n, leading dim ldc
 *   sigma   : n doubles out, ascending
 *   off     : final relative off-orthogonality (the oracle's own residual)
 *   returns : number of sweeps used, or -1 if max_sweeps was hit unconverged */
int oracle_svd_shifted(const double *C, int64_t ldc, int64_t m, int64_t n, double zr, double zi,
                       double *sigma, double *off, int nthreads) {
    ormat A;
    A.m = m; A.n = n;
    A.re = (double *)malloc(sizeof(double) * m * n);
    A.im = (double *)malloc(sizeof(double) * m * n);
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++) {
            A.re[j * m + i] = C[2 * (j * ldc + i)];
            A.im[j * m + i] = C[2 * (j * ldc + i) + 1];
        }
    for (int64_t j = 0; j < n && j < m; j++) { A.re[j * m + j] -= zr; A.im[j * m + j] -= zi; }
    double tol = (double)m * 2.220446049250313e-16;
    int max_sweeps = 60;
    int sweeps = jacobi_sweeps(&A, tol, max_sweeps, nthreads, sigma, off, -1);
    free(A.re); free(A.im);
    return (*off <= tol) ? sweeps : -1;
}

/* Timing sample of the oracle for matrices where one point takes hours: the
 * first `rounds` rounds (each n/2 disjoint pair rotations, about 1/(n-1) of a
 * sweep) of the Jacobi iteration above on C - zI, with nothing else changed.
 * A full point takes sweeps * (n - 1 + n % 2) rounds, with sweeps as
 * returned by oracle_svd_shifted.  Returns 0. */
int oracle_jacobi_rounds(const double *C, int64_t ldc, int64_t m, int64_t n, double zr, double zi,
                         int64_t rounds, int nthreads) {
    ormat A;
    A.m = m; A.n = n;
    A.re = (double *)malloc(sizeof(double) * m * n);
    A.im = (double *)malloc(sizeof(double) * m * n);
    double *sigma = (double *)malloc(sizeof(double) * n);
    double off;
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++) {
            A.re[j * m + i] = C[2 * (j * ldc + i)];
            A.im[j * m + i] = C[2 * (j * ldc + i) + 1];
        }
    for (int64_t j = 0; j < n && j < m; j++) { A.re[j * m + j] -= zr; A.im[j * m + j] -= zi; }
    jacobi_sweeps(&A, (double)m * 2.220446049250313e-16, 60, nthreads, sigma, &off, rounds);
    free(A.re); free(A.im); free(sigma);
    return 0;
}

/* sigma_min(C - z_p I) for npts shifts.  Points are spread over OpenMP
 * threads when there are at least as many points as threads; otherwise each
 * point uses all threads inside its Jacobi rounds.  Returns the number of
 * points that did not converge within the sweep cap. */
int oracle_sigma_min_grid(const double *C, int64_t ldc, int64_t m, int64_t n, const double *z,
                          int64_t npts, double *sigma_min, double *off, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    int bad = 0;
    if (npts >= nthreads) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1) reduction(+ : bad)
#endif
        for (int64_t p = 0; p < npts; p++) {
            double *sig = (double *)malloc(sizeof(double) * n);
            int s = oracle_svd_shifted(C, ldc, m, n, z[2 * p], z[2 * p + 1], sig, &off[p], 1);
            sigma_min[p] = sig[0];
            if (s < 0) bad++;
            free(sig);
        }
    } else {
        double *sig = (double *)malloc(sizeof(double) * n);
        for (int64_t p = 0; p < npts; p++) {
            int s = oracle_svd_shifted(C, ldc, m, n, z[2 * p], z[2 * p + 1], sig, &off[p], nthreads);
            sigma_min[p] = sig[0];
            if (s < 0) bad++;
        }
        free(sig);
    }
    return bad;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
