/*
 * Oracle — test infrastructure only.  Nothing in the product path may link or call this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * The sparse Fourier transform by its definition (eq. 1.1, Sec. 1):
 *
 *     u_i = sum_j exp(sign * 2 pi i  x_i . k_j / N) f_j ,   i in I, j in J,
 *
 * with sign = +1 for the forward transform and sign = -1 for its adjoint (the adjoint of
 * eq. 1.1 swaps the roles of the point sets and conjugates the kernel).  Plain FP64: the
 * phase r = x.k/N is reduced to [0,1) by subtracting floor(r) (exact), then sin and cos
 * of 2 pi r come from the C library.  The sum over j is compensated (Neumaier), and the
 * targets are split across OpenMP threads.
 *
 * Arrays: x [nx][dim] and k [nk][dim] row-major doubles; f and u are complex numbers
 * stored as interleaved (re, im) doubles, f [nrhs][nk] and u [nrhs][nx].
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

/* Neumaier compensated accumulation of one term into (s, c). */
static inline void acc(double *s, double *c, double v) {
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else                     *c += (v - t) + *s;
    *s = t;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_direct(int dim, double N, int64_t nx, const double *x, int64_t nk,
                   const double *k, int nrhs, const double *f, double *u, int sign,
                   int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < nx; ++i) {
        for (int r = 0; r < nrhs; ++r) {
            const double *fr = f + 2 * (int64_t)r * nk;
            double sre = 0, cre = 0, sim = 0, cim = 0;
            for (int64_t j = 0; j < nk; ++j) {
                double dot = 0.0;
                for (int d = 0; d < dim; ++d) dot += x[i * dim + d] * k[j * dim + d];
                double ph = dot / N;
                ph -= floor(ph);
                double a = TWO_PI * ph;
                double cs = cos(a), sn = (double)sign * sin(a);
                double fre = fr[2 * j], fim = fr[2 * j + 1];
                acc(&sre, &cre, cs * fre);
                acc(&sre, &cre, -sn * fim);
                acc(&sim, &cim, cs * fim);
                acc(&sim, &cim, sn * fre);
            }
            u[2 * ((int64_t)r * nx + i)] = sre + cre;
            u[2 * ((int64_t)r * nx + i) + 1] = sim + cim;
        }
    }
}
