/*
 * FP64 CPU oracle for the batched complex-to-complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, call or
 * load this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * What it computes (paper Sec. II-A, the DFT definition):
 *     forward  X[k] = sum_{n=0}^{N-1} x[n] * W_N^{n k},  W_N = exp(-2 pi i / N),
 *              unnormalised;
 *     inverse  x[n] = (1/N) sum_{k} X[k] * exp(+2 pi i n k / N)
 *              (the paper defines only the forward transform; the inverse is
 *               read as the 1/N-scaled conjugate-sign transform so that
 *               inverse(forward(x)) = x).
 *
 * Two independent routines compute it:
 *   oracle_dft   the definition written out, O(N^2), for any N >= 1; the
 *                exponent n*k is reduced exactly modulo N in integer
 *                arithmetic before the angle is formed.
 *   oracle_fft   a plain recursive radix-2 decimation-in-time FFT for N a
 *                power of two (the Cooley-Tukey split of Eq. 1 with N1 = 2):
 *                even/odd halves are transformed recursively and combined as
 *                y[k] = E[k] + w^k O[k], y[k + N/2] = E[k] - w^k O[k],
 *                with w^k = exp(sign * 2 pi i k / N) evaluated directly by
 *                cos/sin for every k (no recurrence, no table).
 *
 * Data layout: interleaved complex, x[2*n] = Re, x[2*n+1] = Im, in double.
 * Batched entry points take `batch` contiguous transforms of N points each.
 * direction: -1 = forward (unnormalised), +1 = inverse (scaled by 1/N).
 * Return value: 0 on success, -1 on an invalid argument.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const double kTwoPi = 6.283185307179586476925286766559;

static int is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

/* exp(sign * 2 pi i * e / N) with e reduced exactly into [0, N). */
static void unit_root(int64_t N, int64_t e, int sign, double *re, double *im) {
    int64_t r = e % N;
    if (r < 0) r += N;
    double theta = (double)sign * kTwoPi * (double)r / (double)N;
    *re = cos(theta);
    *im = sin(theta);
}

/* ---------------------------------------------------------------------- */
/* Definition: O(N^2) DFT.                                                 */
/* ---------------------------------------------------------------------- */
int oracle_dft(int64_t N, const double *x, double *y, int direction) {
    if (N < 1 || (direction != -1 && direction != 1) || !x || !y) return -1;
    double *acc = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    if (!acc) return -1;
    for (int64_t k = 0; k < N; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t n = 0; n < N; ++n) {
            double wr, wi;
            /* (n*k) mod N computed without overflow for N <= 2^31 */
            int64_t e = (int64_t)(((__int128)n * (__int128)k) % N);
            unit_root(N, e, direction, &wr, &wi);
            double xr = x[2 * n], xi = x[2 * n + 1];
            sr += xr * wr - xi * wi;
            si += xr * wi + xi * wr;
        }
        acc[2 * k] = sr;
        acc[2 * k + 1] = si;
    }
    double s = (direction == 1) ? 1.0 / (double)N : 1.0;
    for (int64_t k = 0; k < 2 * N; ++k) y[k] = acc[k] * s;
    free(acc);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Recursive radix-2 DIT FFT.                                              */
/* ---------------------------------------------------------------------- */
/* y[0..N) (interleaved) <- unnormalised DFT (sign) of x[0], x[s], x[2s], ... */
static void fft_rec(int64_t N, const double *x, int64_t stride, double *y,
                    int sign) {
    if (N == 1) {
        y[0] = x[0];
        y[1] = x[1];
        return;
    }
    int64_t h = N / 2;
    fft_rec(h, x, 2 * stride, y, sign);                  /* E -> y[0..h)  */
    fft_rec(h, x + 2 * stride, 2 * stride, y + 2 * h, sign); /* O -> y[h..N) */
    for (int64_t k = 0; k < h; ++k) {
        double wr, wi;
        unit_root(N, k, sign, &wr, &wi);
        double er = y[2 * k], ei = y[2 * k + 1];
        double orr = y[2 * (k + h)], oi = y[2 * (k + h) + 1];
        double tr = wr * orr - wi * oi;
        double ti = wr * oi + wi * orr;
        y[2 * k] = er + tr;
        y[2 * k + 1] = ei + ti;
        y[2 * (k + h)] = er - tr;
        y[2 * (k + h) + 1] = ei - ti;
    }
}

int oracle_fft(int64_t N, const double *x, double *y, int direction) {
    if (!is_pow2(N) || (direction != -1 && direction != 1) || !x || !y)
        return -1;
    double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    if (!tmp) return -1;
    fft_rec(N, x, 1, tmp, direction);
    double s = (direction == 1) ? 1.0 / (double)N : 1.0;
    for (int64_t k = 0; k < 2 * N; ++k) y[k] = tmp[k] * s;
    free(tmp);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Batched drivers (a batch of independent transforms, paper Sec. II-D).   */
/* ---------------------------------------------------------------------- */
typedef struct {
    int64_t N, b0, b1;
    const double *xd;
    const float *xf;
    double *y;
    int direction;
    int rc;
} job_t;

static void *batch_worker(void *arg) {
    job_t *j = (job_t *)arg;
    double *in = NULL;
    if (j->xf) {
        in = (double *)malloc(sizeof(double) * 2 * (size_t)j->N);
        if (!in) { j->rc = -1; return NULL; }
    }
    for (int64_t b = j->b0; b < j->b1; ++b) {
        const double *src;
        if (j->xf) {
            const float *f = j->xf + (size_t)(2 * j->N * b);
            for (int64_t i = 0; i < 2 * j->N; ++i) in[i] = (double)f[i];
            src = in;
        } else {
            src = j->xd + (size_t)(2 * j->N * b);
        }
        if (oracle_fft(j->N, src, j->y + (size_t)(2 * j->N * b), j->direction)) {
            j->rc = -1;
            break;
        }
    }
    free(in);
    return NULL;
}

static int run_batch(int64_t N, int64_t batch, const double *xd, const float *xf,
                     double *y, int direction, int nthreads) {
    if (!is_pow2(N) || batch < 0 || (direction != -1 && direction != 1) || !y)
        return -1;
    if (batch == 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > batch) nthreads = (int)batch;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].N = N;
        jobs[t].b0 = batch * t / nthreads;
        jobs[t].b1 = batch * (t + 1) / nthreads;
        jobs[t].xd = xd;
        jobs[t].xf = xf;
        jobs[t].y = y;
        jobs[t].direction = direction;
        jobs[t].rc = 0;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, batch_worker, &jobs[t]) != 0) {
            jobs[t].rc = -1;
            rc = -1;
            break;
        }
        started = t;
    }
    batch_worker(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].rc) rc = -1;
    free(jobs);
    free(th);
    return rc;
}

int oracle_fft_batch(int64_t N, int64_t batch, const double *x, double *y,
                     int direction, int nthreads) {
    if (!x) return -1;
    return run_batch(N, batch, x, NULL, y, direction, nthreads);
}

/* float32 input widened exactly to double before the transform. */
int oracle_fft_batch_f32(int64_t N, int64_t batch, const float *x, double *y,
                         int direction, int nthreads) {
    if (!x) return -1;
    return run_batch(N, batch, NULL, x, y, direction, nthreads);
}
