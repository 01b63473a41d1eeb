/*
 * ivis_oracle.c -- plain, slow FP64 CPU oracle for the Classic3D data term.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. It shares no code
 * with the CUDA path.
 *
 * It evaluates the simplified visibility equation of Sect. 2.1 (the
 * coplanar / small-angle form, w-term and n-term neglected) as the direct
 * non-uniform DFT it defines, and its adjoint, term by term with one sin/cos
 * per (visibility, pixel) term, and likewise the full equation (Eq. 1, with
 * the w-term and 1/n; functions *_w at the end). No fast transform, no
 * table, no recurrence.
 *
 *   V~_j = sum_{q,p} f[q,p] exp(-2 pi i (u_j l_p + v_j m_q))             (forward)
 *   a[q,p] = sum_j c_j exp(+2 pi i (u_j l_p + v_j m_q))                   (adjoint)
 *
 * with l_p = (p - nb/2) * cell and m_q = (q - nb/2) * cell (pixel origin of
 * the pointing window at pixel nb/2; l along columns, m along rows).
 * Complex arrays are interleaved (re, im) doubles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559

/* Forward: model visibilities of the real image f (nb x nb, row-major [q][p])
 * at m points (u, v) in wavelengths. Zero pixels contribute nothing and are
 * skipped (the sum is unchanged). */
void ivo_forward(int nb, double cell, const double *f, int64_t m,
                 const double *u, const double *v, double *out)
{
    int64_t nnz = 0;
    for (int64_t t = 0; t < (int64_t)nb * nb; ++t)
        if (f[t] != 0.0) ++nnz;
    double *val = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    double *lp = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    double *mq = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    int64_t c = 0;
    for (int q = 0; q < nb; ++q)
        for (int p = 0; p < nb; ++p) {
            double a = f[(int64_t)q * nb + p];
            if (a == 0.0) continue;
            val[c] = a;
            lp[c] = (p - nb / 2) * cell;
            mq[c] = (q - nb / 2) * cell;
            ++c;
        }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < m; ++j) {
        double re = 0.0, im = 0.0;
        for (int64_t t = 0; t < nnz; ++t) {
            double ph = -TWO_PI * (u[j] * lp[t] + v[j] * mq[t]);
            re += val[t] * cos(ph);
            im += val[t] * sin(ph);
        }
        out[2 * j] = re;
        out[2 * j + 1] = im;
    }
    free(val); free(lp); free(mq);
}

/* Adjoint at a list of window pixels (q_t, p_t): out[t] = sum_j c_j e^{+2 pi i(...)}. */
void ivo_adjoint_pixels(int nb, double cell, int64_t m, const double *u, const double *v,
                        const double *cvis, int64_t npix, const int32_t *qs,
                        const int32_t *ps, double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < npix; ++t) {
        double l = (ps[t] - nb / 2) * cell;
        double mm = (qs[t] - nb / 2) * cell;
        double re = 0.0, im = 0.0;
        for (int64_t j = 0; j < m; ++j) {
            double ph = TWO_PI * (u[j] * l + v[j] * mm);
            double cs = cos(ph), sn = sin(ph);
            re += cvis[2 * j] * cs - cvis[2 * j + 1] * sn;
            im += cvis[2 * j] * sn + cvis[2 * j + 1] * cs;
        }
        out[2 * t] = re;
        out[2 * t + 1] = im;
    }
}

/* Adjoint over the whole nb x nb window (row-major complex output). */
void ivo_adjoint(int nb, double cell, int64_t m, const double *u, const double *v,
                 const double *cvis, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < nb; ++q) {
        double mm = (q - nb / 2) * cell;
        for (int p = 0; p < nb; ++p) {
            double l = (p - nb / 2) * cell;
            double re = 0.0, im = 0.0;
            for (int64_t j = 0; j < m; ++j) {
                double ph = TWO_PI * (u[j] * l + v[j] * mm);
                double cs = cos(ph), sn = sin(ph);
                re += cvis[2 * j] * cs - cvis[2 * j + 1] * sn;
                im += cvis[2 * j] * sn + cvis[2 * j + 1] * cs;
            }
            out[2 * ((int64_t)q * nb + p)] = re;
            out[2 * ((int64_t)q * nb + p) + 1] = im;
        }
    }
}

/*
 * Full visibility equation of Sect. 2.1 (Eq. 1) with the w-term and the 1/n factor:
 *
 *   V~_j = sum_{q,p} f[q,p] / n_qp exp(-2 pi i (u_j l_p + v_j m_q + w_j (n_qp - 1)))
 *   a[q,p] = 1 / n_qp sum_j c_j exp(+2 pi i (u_j l_p + v_j m_q + w_j (n_qp - 1)))
 *
 * n = sqrt(1 - l^2 - m^2); n - 1 is formed as -(l^2 + m^2) / (1 + n) (no cancellation).
 */
static double n_minus_1(double l, double mm, double *n)
{
    double r2 = l * l + mm * mm;
    *n = sqrt(1.0 - r2);
    return -r2 / (1.0 + *n);
}

void ivo_forward_w(int nb, double cell, const double *f, int64_t m, const double *u,
                   const double *v, const double *w, double *out)
{
    int64_t nnz = 0;
    for (int64_t t = 0; t < (int64_t)nb * nb; ++t)
        if (f[t] != 0.0) ++nnz;
    size_t sz = sizeof(double) * (size_t)(nnz ? nnz : 1);
    double *val = (double *)malloc(sz), *lp = (double *)malloc(sz), *mq = (double *)malloc(sz),
           *nq = (double *)malloc(sz);
    int64_t c = 0;
    for (int q = 0; q < nb; ++q)
        for (int p = 0; p < nb; ++p) {
            double a = f[(int64_t)q * nb + p], n;
            if (a == 0.0) continue;
            lp[c] = (p - nb / 2) * cell;
            mq[c] = (q - nb / 2) * cell;
            nq[c] = n_minus_1(lp[c], mq[c], &n);
            val[c] = a / n;
            ++c;
        }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < m; ++j) {
        double re = 0.0, im = 0.0;
        for (int64_t t = 0; t < nnz; ++t) {
            double ph = -TWO_PI * (u[j] * lp[t] + v[j] * mq[t] + w[j] * nq[t]);
            re += val[t] * cos(ph);
            im += val[t] * sin(ph);
        }
        out[2 * j] = re;
        out[2 * j + 1] = im;
    }
    free(val); free(lp); free(mq); free(nq);
}

void ivo_adjoint_w(int nb, double cell, int64_t m, const double *u, const double *v,
                   const double *w, const double *cvis, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < nb; ++q) {
        double mm = (q - nb / 2) * cell;
        for (int p = 0; p < nb; ++p) {
            double l = (p - nb / 2) * cell, n;
            double nm1 = n_minus_1(l, mm, &n);
            double re = 0.0, im = 0.0;
            for (int64_t j = 0; j < m; ++j) {
                double ph = TWO_PI * (u[j] * l + v[j] * mm + w[j] * nm1);
                double cs = cos(ph), sn = sin(ph);
                re += cvis[2 * j] * cs - cvis[2 * j + 1] * sn;
                im += cvis[2 * j] * sn + cvis[2 * j + 1] * cs;
            }
            out[2 * ((int64_t)q * nb + p)] = re / n;
            out[2 * ((int64_t)q * nb + p) + 1] = im / n;
        }
    }
}

void ivo_adjoint_pixels_w(int nb, double cell, int64_t m, const double *u, const double *v,
                          const double *w, const double *cvis, int64_t npix, const int32_t *qs,
                          const int32_t *ps, double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < npix; ++t) {
        double l = (ps[t] - nb / 2) * cell, mm = (qs[t] - nb / 2) * cell, n;
        double nm1 = n_minus_1(l, mm, &n);
        double re = 0.0, im = 0.0;
        for (int64_t j = 0; j < m; ++j) {
            double ph = TWO_PI * (u[j] * l + v[j] * mm + w[j] * nm1);
            double cs = cos(ph), sn = sin(ph);
            re += cvis[2 * j] * cs - cvis[2 * j + 1] * sn;
            im += cvis[2 * j] * sn + cvis[2 * j + 1] * cs;
        }
        out[2 * t] = re / n;
        out[2 * t + 1] = im / n;
    }
}

int ivo_num_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = 1
#ifdef _OPENMP
            * omp_get_num_threads()
#endif
            ;
    }
    return n;
}
