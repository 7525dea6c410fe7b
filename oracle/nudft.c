/*
 * Direct FP64 evaluation of the oracle's Fourier slice step (test
 * infrastructure only; never linked into the CUDA library).
 *
 * Forward (Algorithm 1 step 3, eq. Inv_op / inv_GFST): for every kept
 * stretched-time frequency f_k and trace h with squared offset r2[h],
 *
 *   Y[k][h] = sum_{s in {0,1}} w_s[h] * sum_l X[k][l][j_s[h]]
 *                                 * exp(-i 2 pi f_k q_l r2[h])
 *
 * i.e. the 2D spectrum of the stretched model read at k_q = f_k r^2 in the
 * two azimuth slices around theta_h, with the DFT along q evaluated exactly
 * at that non-uniform k_q.  Adjoint (the transpose used by Algorithm 2):
 *
 *   Xa[k][l][j_s[h]] += w_s[h] * exp(+i 2 pi f_k q_l r2[h]) * Y[k][h].
 *
 * Complex arrays are interleaved (re, im) doubles; X is [nk][nq][nth],
 * Y is [nk][ntr].  Each bin is independent, so bins run in parallel.
 */
#include <math.h>
#include <stddef.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

void oracle_slice_forward(int nk, int nq, int nth, int ntr,
                          const double *f, const double *q, const double *r2,
                          const long long *j0, const long long *j1,
                          const double *w0, const double *w1,
                          const double *X, double *Y)
{
    long long k;
#pragma omp parallel for schedule(dynamic, 2)
    for (k = 0; k < nk; ++k) {
        const double *Xk = X + 2 * (size_t)k * nq * nth;
        for (int h = 0; h < ntr; ++h) {
            double re = 0.0, im = 0.0;
            const size_t a = (size_t)j0[h], b = (size_t)j1[h];
            for (int l = 0; l < nq; ++l) {
                const double ph = -2.0 * M_PI * f[k] * q[l] * r2[h];
                const double c = cos(ph), s = sin(ph);
                const double *xa = Xk + 2 * ((size_t)l * nth + a);
                const double *xb = Xk + 2 * ((size_t)l * nth + b);
                const double xr = w0[h] * xa[0] + w1[h] * xb[0];
                const double xi = w0[h] * xa[1] + w1[h] * xb[1];
                re += xr * c - xi * s;
                im += xr * s + xi * c;
            }
            Y[2 * ((size_t)k * ntr + h)] = re;
            Y[2 * ((size_t)k * ntr + h) + 1] = im;
        }
    }
}

void oracle_slice_adjoint(int nk, int nq, int nth, int ntr,
                          const double *f, const double *q, const double *r2,
                          const long long *j0, const long long *j1,
                          const double *w0, const double *w1,
                          const double *Y, double *X)
{
    long long k;
#pragma omp parallel for schedule(dynamic, 2)
    for (k = 0; k < nk; ++k) {
        double *Xk = X + 2 * (size_t)k * nq * nth;
        for (size_t i = 0; i < 2 * (size_t)nq * nth; ++i) Xk[i] = 0.0;
        for (int h = 0; h < ntr; ++h) {
            const double yr = Y[2 * ((size_t)k * ntr + h)];
            const double yi = Y[2 * ((size_t)k * ntr + h) + 1];
            const size_t a = (size_t)j0[h], b = (size_t)j1[h];
            for (int l = 0; l < nq; ++l) {
                const double ph = 2.0 * M_PI * f[k] * q[l] * r2[h];
                const double c = cos(ph), s = sin(ph);
                const double vr = yr * c - yi * s;
                const double vi = yr * s + yi * c;
                double *xa = Xk + 2 * ((size_t)l * nth + a);
                double *xb = Xk + 2 * ((size_t)l * nth + b);
                xa[0] += w0[h] * vr;
                xa[1] += w0[h] * vi;
                xb[0] += w1[h] * vr;
                xb[1] += w1[h] * vi;
            }
        }
    }
}

#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of threads the parallel loops above use (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
