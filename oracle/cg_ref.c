/*
 * Oracle (TEST INFRASTRUCTURE ONLY): plain FP64 conjugate gradients for the
 * homogeneous diffusion inpainting system, for frames too large for a sparse
 * direct solve.  Called through ctypes by tests, the smoke check and the CPU
 * baseline of the benchmark; never by the library.
 *
 * Problem (paper Sec. 2, Eq. eq:homdiff / eq:ls): A u = b with
 * A = C - (I - C) L, b = C f, L the 5-point Laplacian with reflecting image
 * boundaries ((L u)_p = sum over in-image 4-neighbours q of (u_q - u_p)).
 * Known rows fix u_p = f_p.  Eliminating them leaves the symmetric positive
 * definite system on the unknown pixels U
 *     deg(p) u_p - sum_{q in N(p) cap U} u_q = sum_{q in N(p) cap K} f_q ,
 * which is solved here by textbook CG (Saad, Iterative Methods for Sparse
 * Linear Systems, the CG algorithm of Ch. 6) from u0 = C f, stopping when the
 * true residual satisfies ||b - A u|| <= tol * ||b - A u0|| (the relative
 * residual of the paper's Sec. 4-5 with reference u0 = C f).  Every 64
 * iterations the recursively updated residual is replaced by the true one.
 *
 * Layout: channel-planar, row-major (C, H, W) doubles; mask (H, W) bytes,
 * nonzero = known.  One mask is shared by all channels.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* y = (A_UU x) on unknown pixels, 0 on known ones; x is 0 on known pixels. */
static void apply_auu(int H, int W, const unsigned char *known, const double *x, double *y)
{
    #pragma omp parallel for schedule(static)
    for (int yy = 0; yy < H; ++yy) {
        for (int xx = 0; xx < W; ++xx) {
            long p = (long)yy * W + xx;
            if (known[p]) { y[p] = 0.0; continue; }
            double s = 0.0;
            int deg = 0;
            if (yy > 0)     { s += x[p - W]; ++deg; }
            if (yy < H - 1) { s += x[p + W]; ++deg; }
            if (xx > 0)     { s += x[p - 1]; ++deg; }
            if (xx < W - 1) { s += x[p + 1]; ++deg; }
            y[p] = deg * x[p] - s;
        }
    }
}

/* r = b - A u on unknown pixels (0 on known ones, where u = f is imposed). */
static void true_residual(int H, int W, const unsigned char *known, const double *u, double *r)
{
    #pragma omp parallel for schedule(static)
    for (int yy = 0; yy < H; ++yy) {
        for (int xx = 0; xx < W; ++xx) {
            long p = (long)yy * W + xx;
            if (known[p]) { r[p] = 0.0; continue; }
            double s = 0.0;
            if (yy > 0)     s += u[p - W] - u[p];
            if (yy < H - 1) s += u[p + W] - u[p];
            if (xx > 0)     s += u[p - 1] - u[p];
            if (xx < W - 1) s += u[p + 1] - u[p];
            r[p] = s;   /* b_p = 0 and (A u)_p = -(L u)_p on unknown pixels */
        }
    }
}

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    #pragma omp parallel for reduction(+:s) schedule(static)
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/*
 * Solve all C channels.  f: (C,H,W) known values (read where mask != 0).
 * u: (C,H,W) output.  iters / relres: per-channel outputs (may be NULL).
 * Returns 0 on success, 1 if some channel hit max_iter, -1 on bad input,
 * -2 on allocation failure, -3 for an empty mask.
 */
int oracle_cg_solve(int H, int W, int C, const unsigned char *mask, const double *f,
                    double *u, double tol, int max_iter, int *iters, double *relres)
{
    if (H <= 0 || W <= 0 || C <= 0 || !mask || !f || !u) return -1;
    long N = (long)H * W;
    long nknown = 0;
    for (long p = 0; p < N; ++p) nknown += mask[p] != 0;
    if (nknown == 0) return -3;
    unsigned char *known = (unsigned char *)malloc((size_t)N);
    double *r = (double *)malloc(sizeof(double) * N);
    double *d = (double *)malloc(sizeof(double) * N);
    double *q = (double *)malloc(sizeof(double) * N);
    if (!known || !r || !d || !q) { free(known); free(r); free(d); free(q); return -2; }
    for (long p = 0; p < N; ++p) known[p] = mask[p] != 0;

    int status = 0;
    for (int c = 0; c < C; ++c) {
        const double *fc = f + (long)c * N;
        double *uc = u + (long)c * N;
        for (long p = 0; p < N; ++p) uc[p] = known[p] ? fc[p] : 0.0;   /* u0 = C f */
        true_residual(H, W, known, uc, r);
        double rr = dot(N, r, r);
        double ref = sqrt(rr);
        double scale = ref > 0.0 ? ref : 1.0;
        memcpy(d, r, sizeof(double) * N);
        int it = 0;
        while (sqrt(rr) > tol * scale && it < max_iter) {
            apply_auu(H, W, known, d, q);
            double dq = dot(N, d, q);
            if (!(dq > 0.0)) break;
            double alpha = rr / dq;
            #pragma omp parallel for schedule(static)
            for (long p = 0; p < N; ++p) { uc[p] += alpha * d[p]; r[p] -= alpha * q[p]; }
            ++it;
            if (it % 64 == 0) true_residual(H, W, known, uc, r);
            double rr_new = dot(N, r, r);
            double beta = rr_new / rr;
            #pragma omp parallel for schedule(static)
            for (long p = 0; p < N; ++p) d[p] = r[p] + beta * d[p];
            rr = rr_new;
            /* the stop test must hold for the true residual */
            if (sqrt(rr) <= tol * scale && it % 64 != 0) {
                true_residual(H, W, known, uc, r);
                rr = dot(N, r, r);
                if (sqrt(rr) > tol * scale) memcpy(d, r, sizeof(double) * N);
            }
        }
        true_residual(H, W, known, uc, r);
        double fin = sqrt(dot(N, r, r)) / scale;
        if (iters) iters[c] = it;
        if (relres) relres[c] = fin;
        if (fin > tol) status = 1;
    }
    free(known); free(r); free(d); free(q);
    return status;
}

/* Number of OpenMP threads the solver uses (1 without OpenMP). */
int oracle_cg_threads(void)
{
    int n = 1;
    #pragma omp parallel
    {
        #pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
