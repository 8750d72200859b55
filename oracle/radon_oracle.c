/*
 * Exact, slow FP64 reference for the discrete parallel-beam Radon transform
 * A and its adjoint A^T, for TEST INFRASTRUCTURE ONLY.  Nothing in the
 * product path links or calls this file: only tests/, the smoke check and the
 * CPU-baseline leg of bench.py do.  It shares no code, header or table with
 * the CUDA library.
 *
 * What it computes (Sec. 2.1 Eq. radon_transform, Sec. 2.2 Eq. fourier_sum
 * and Eq. nufft; adjoint Sec. 3 Eq. transpose), read as a discrete operator:
 *
 *   pixel centres   x_n = (ix - N/2, iy - N/2), image stored f[iy*N + ix]
 *   angles          theta_a (radians, caller-supplied)
 *   projection      s_n(a) = x cos(theta_a) + y sin(theta_a)    (Eq. line_eqn)
 *   detector bins   t_i = i - D/2,  i = 0..D-1   (D even)
 *   radial freqs    k_m = m/D,  m = -D/2..D/2,  nu_m = 1/2 at |m| = D/2
 *
 *   stage 1 (Fourier-slice theorem, Eq. fourier_radon, as an exact NUDFT):
 *       c(a,m) = sum_n f_n exp(-2 pi i m s_n(a) / D)
 *   stage 2 (inverse of the row transform of Eq. nufft, first line):
 *       y(a,i) = (1/D) Re sum_m nu_m c(a,m) exp(+2 pi i m t_i / D)
 *
 * Equivalently y(a,i) = sum_n f_n K_D(t_i - s_n(a)) with the Dirichlet kernel
 *       K_D(u) = (1/D) [ sin(pi u (D-1)/D) / sin(pi u / D) + cos(pi u) ],
 * K_D(0) = 1.  The sampled entry points use that closed form; the full
 * operators use the two-stage NUDFT.  The two routes are independent
 * formulations of the same operator and the tests hold them to each other.
 *
 * The adjoint is the exact transpose:
 *       x_n = sum_a sum_i y(a,i) K_D(t_i - s_n(a))
 * computed as a row DFT  g(a,m) = (nu_m/D) sum_i y(a,i) exp(-2 pi i m t_i/D)
 * followed by an exact back-summation  x_n = Re sum_{a,m} g(a,m) exp(+2 pi i m s_n(a)/D).
 *
 * The complex exponential over m is advanced by a rotation recurrence that is
 * re-seeded from sin/cos every RESEED steps, which keeps its FP64 drift far
 * below 1e-12 for the lengths used here.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define RESEED 16

static const double PI = 3.14159265358979323846264338327950288;

static double nu_m(int m, int D)
{
    return (2 * m == D || 2 * m == -D) ? 0.5 : 1.0;
}

/* exp(2 pi i k / D) for integer k, taken exactly from a table mod D */
static void unit_table(int D, double *cr, double *ci)
{
    for (int k = 0; k < D; ++k) {
        cr[k] = cos(2.0 * PI * (double)k / (double)D);
        ci[k] = sin(2.0 * PI * (double)k / (double)D);
    }
}

static int mod_int(long long v, int D)
{
    long long r = v % D;
    return (int)(r < 0 ? r + D : r);
}

int oracle_check_geometry(int N, int A, int D)
{
    if (N < 1 || A < 1 || D < 2 || (D & 1)) return -1;
    return 0;
}

/* y[A][D] = A f, f[N][N]; exact two-stage NUDFT.  delta: rotation-axis
 * offset, the projection of x_n lands at detector coordinate s_n + delta
 * (Sec. 4.1, Fourier-shift correction of the axis). */
int oracle_radon_fwd_shift(int N, int A, int D, const double *theta, double delta,
                           const double *f, double *y)
{
    if (oracle_check_geometry(N, A, D)) return -1;
    const int M = D + 1; /* m = -D/2 .. D/2 */
    double *cr_t = (double *)malloc(sizeof(double) * D);
    double *ci_t = (double *)malloc(sizeof(double) * D);
    unit_table(D, cr_t, ci_t);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < A; ++a) {
        double *cre = (double *)calloc(M, sizeof(double));
        double *cim = (double *)calloc(M, sizeof(double));
        if (!cre || !cim) { err = 1; free(cre); free(cim); continue; }
        const double ct = cos(theta[a]), st = sin(theta[a]);
        /* stage 1: c(a,m) = sum_n f_n exp(-2 pi i m s_n / D) */
        for (int iy = 0; iy < N; ++iy) {
            for (int ix = 0; ix < N; ++ix) {
                const double fn = f[(size_t)iy * N + ix];
                if (fn == 0.0) continue;
                const double s = (ix - N / 2) * ct + (iy - N / 2) * st;
                const double ph = -2.0 * PI * s / (double)D;
                const double sr = cos(ph), si = sin(ph);
                double zr = 0.0, zi = 0.0;
                for (int j = 0; j < M; ++j) {
                    const int m = j - D / 2;
                    if (j % RESEED == 0) { zr = cos(ph * m); zi = sin(ph * m); }
                    cre[j] += fn * zr;
                    cim[j] += fn * zi;
                    const double nr = zr * sr - zi * si;
                    zi = zr * si + zi * sr;
                    zr = nr;
                }
            }
        }
        /* stage 2: y(a,i) = (1/D) Re sum_m nu_m c(a,m) exp(2 pi i m (t_i - delta) / D) */
        for (int j = 0; j < M; ++j) {  /* c(a,m) *= exp(-2 pi i m delta / D) */
            const double ph = -2.0 * PI * (j - D / 2) * delta / (double)D;
            const double pr = cos(ph), pi = sin(ph);
            const double nr = cre[j] * pr - cim[j] * pi;
            cim[j] = cre[j] * pi + cim[j] * pr;
            cre[j] = nr;
        }
        for (int i = 0; i < D; ++i) {
            const int t = i - D / 2;
            double acc = 0.0;
            for (int j = 0; j < M; ++j) {
                const int m = j - D / 2;
                const int k = mod_int((long long)m * t, D);
                acc += nu_m(m, D) * (cre[j] * cr_t[k] - cim[j] * ci_t[k]);
            }
            y[(size_t)a * D + i] = acc / (double)D;
        }
        free(cre);
        free(cim);
    }
    free(cr_t);
    free(ci_t);
    return err ? -2 : 0;
}

/* x[N][N] = A^T y, y[A][D]; row DFT then exact back-summation. */
int oracle_radon_adj_shift(int N, int A, int D, const double *theta, double delta,
                           const double *y, double *x)
{
    if (oracle_check_geometry(N, A, D)) return -1;
    const int M = D + 1;
    double *cr_t = (double *)malloc(sizeof(double) * D);
    double *ci_t = (double *)malloc(sizeof(double) * D);
    double *gr = (double *)malloc(sizeof(double) * (size_t)A * M);
    double *gi = (double *)malloc(sizeof(double) * (size_t)A * M);
    double *ct = (double *)malloc(sizeof(double) * A);
    double *st = (double *)malloc(sizeof(double) * A);
    if (!cr_t || !ci_t || !gr || !gi || !ct || !st) {
        free(cr_t); free(ci_t); free(gr); free(gi); free(ct); free(st);
        return -2;
    }
    unit_table(D, cr_t, ci_t);
    for (int a = 0; a < A; ++a) { ct[a] = cos(theta[a]); st[a] = sin(theta[a]); }
    /* g(a,m) = (nu_m / D) sum_i y(a,i) exp(-2 pi i m t_i / D) */
#pragma omp parallel for
    for (int a = 0; a < A; ++a) {
        for (int j = 0; j < M; ++j) {
            const int m = j - D / 2;
            double sr = 0.0, si = 0.0;
            for (int i = 0; i < D; ++i) {
                const int k = mod_int(-(long long)m * (i - D / 2), D);
                const double v = y[(size_t)a * D + i];
                sr += v * cr_t[k];
                si += v * ci_t[k];
            }
            /* times exp(+2 pi i m delta / D): the transpose of the forward shift */
            const double ph = 2.0 * PI * m * delta / (double)D;
            const double pr = cos(ph), pim = sin(ph);
            gr[(size_t)a * M + j] = nu_m(m, D) * (sr * pr - si * pim) / (double)D;
            gi[(size_t)a * M + j] = nu_m(m, D) * (sr * pim + si * pr) / (double)D;
        }
    }
    /* x_n = Re sum_a sum_m g(a,m) exp(+2 pi i m s_n(a) / D) */
#pragma omp parallel for schedule(dynamic, 4)
    for (int n = 0; n < N * N; ++n) {
        const int ix = n % N, iy = n / N;
        double acc = 0.0;
        for (int a = 0; a < A; ++a) {
            const double s = (ix - N / 2) * ct[a] + (iy - N / 2) * st[a];
            const double ph = 2.0 * PI * s / (double)D;
            const double sr = cos(ph), si = sin(ph);
            double zr = 0.0, zi = 0.0;
            const double *gra = gr + (size_t)a * M, *gia = gi + (size_t)a * M;
            for (int j = 0; j < M; ++j) {
                const int m = j - D / 2;
                if (j % RESEED == 0) { zr = cos(ph * m); zi = sin(ph * m); }
                acc += gra[j] * zr - gia[j] * zi;
                const double nr = zr * sr - zi * si;
                zi = zr * si + zi * sr;
                zr = nr;
            }
        }
        x[n] = acc;
    }
    free(cr_t); free(ci_t); free(gr); free(gi); free(ct); free(st);
    return 0;
}

/* Dirichlet kernel K_D(u) of the band-limited detector model; D-periodic. */
double oracle_dirichlet(int D, double u)
{
    double r = fmod(u, (double)D);
    if (r > 0.5 * D) r -= D;
    if (r < -0.5 * D) r += D;
    if (r == 0.0) return 1.0;
    const double num = sin(PI * r * (double)(D - 1) / (double)D);
    const double den = sin(PI * r / (double)D);
    return (num / den + cos(PI * r)) / (double)D;
}

/* y(a_k, i_k) for K sampled sinogram entries, by the closed form. */
int oracle_radon_fwd_at_shift(int N, int A, int D, const double *theta, double delta,
                              const double *f, int K, const int *a_idx,
                              const int *i_idx, double *out)
{
    if (oracle_check_geometry(N, A, D)) return -1;
    for (int k = 0; k < K; ++k)
        if (a_idx[k] < 0 || a_idx[k] >= A || i_idx[k] < 0 || i_idx[k] >= D)
            return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        const double ct = cos(theta[a_idx[k]]), st = sin(theta[a_idx[k]]);
        const double t = i_idx[k] - D / 2 - delta;
        double acc = 0.0;
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                const double fn = f[(size_t)iy * N + ix];
                if (fn == 0.0) continue;
                const double s = (ix - N / 2) * ct + (iy - N / 2) * st;
                acc += fn * oracle_dirichlet(D, t - s);
            }
        out[k] = acc;
    }
    return 0;
}

/* x(pix_k) for K sampled pixels of A^T y, by the closed form. */
int oracle_radon_adj_at_shift(int N, int A, int D, const double *theta, double delta,
                              const double *y, int K, const int *pix_idx,
                              double *out)
{
    if (oracle_check_geometry(N, A, D)) return -1;
    for (int k = 0; k < K; ++k)
        if (pix_idx[k] < 0 || pix_idx[k] >= N * N) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        const int ix = pix_idx[k] % N, iy = pix_idx[k] / N;
        double acc = 0.0;
        for (int a = 0; a < A; ++a) {
            const double s = (ix - N / 2) * cos(theta[a]) + (iy - N / 2) * sin(theta[a]);
            for (int i = 0; i < D; ++i)
                acc += y[(size_t)a * D + i] * oracle_dirichlet(D, (i - D / 2) - delta - s);
        }
        out[k] = acc;
    }
    return 0;
}

/* Unshifted forms (rotation axis at the detector centre). */
int oracle_radon_fwd(int N, int A, int D, const double *theta, const double *f, double *y)
{
    return oracle_radon_fwd_shift(N, A, D, theta, 0.0, f, y);
}

int oracle_radon_adj(int N, int A, int D, const double *theta, const double *y, double *x)
{
    return oracle_radon_adj_shift(N, A, D, theta, 0.0, y, x);
}

/* Batched forms over B slices (each slice is an independent 2D problem). */
int oracle_radon_fwd_batch(int B, int N, int A, int D, const double *theta, double delta,
                           const double *f, double *y)
{
    for (int b = 0; b < B; ++b) {
        int rc = oracle_radon_fwd_shift(N, A, D, theta, delta, f + (size_t)b * N * N,
                                        y + (size_t)b * A * D);
        if (rc) return rc;
    }
    return 0;
}

int oracle_radon_adj_batch(int B, int N, int A, int D, const double *theta, double delta,
                           const double *y, double *x)
{
    for (int b = 0; b < B; ++b) {
        int rc = oracle_radon_adj_shift(N, A, D, theta, delta, y + (size_t)b * A * D,
                                        x + (size_t)b * N * N);
        if (rc) return rc;
    }
    return 0;
}
