/* Exact measurement operator and its adjoint by brute force, FP64.
 *
 * TEST INFRASTRUCTURE ONLY: part of the oracle; nothing in the product path
 * links it.
 *
 * Eq. fourier_visibility (Section 2) on a pixel list, with the plain-sum
 * normalisation used throughout the oracle:
 *   degrid: V_k   = sum_p f_p exp(-2 pi i (u_k l_p + v_k m_p + w_k (n_p - 1)))
 *   grid:   d_p   = sum_k V_k exp(+2 pi i (u_k l_p + v_k m_p + w_k (n_p - 1)))
 * The grid form is the adjoint (Eq. dirty_1d in 1-D; the dirty image of
 * Section 5.2 in 3-D).  Each phase is accumulated in turns, reduced to
 * [-1/2, 1/2] and only then multiplied by 2 pi.
 *
 * Layout: uvw is M x 3 (u, v, w in wavelengths); lmn is P x 3 holding
 * (l, m, n - 1); complex arrays are interleaved (re, im) doubles.
 */
#include <math.h>
#include <stdint.h>

static const double TWO_PI = 6.283185307179586476925286766559;

static inline double reduce_turns(double t) { return t - nearbyint(t); }

void oracle_dft_degrid(int64_t M, const double *uvw, int64_t P, const double *lmn,
                       const double *f, double *vis)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < M; ++k) {
        const double u = uvw[3 * k], v = uvw[3 * k + 1], w = uvw[3 * k + 2];
        double re = 0.0, im = 0.0;
        for (int64_t p = 0; p < P; ++p) {
            const double ph = TWO_PI * reduce_turns(u * lmn[3 * p] + v * lmn[3 * p + 1] +
                                                    w * lmn[3 * p + 2]);
            const double c = cos(ph), s = sin(ph);
            const double fr = f[2 * p], fi = f[2 * p + 1];
            /* f * exp(-i ph) */
            re += fr * c + fi * s;
            im += fi * c - fr * s;
        }
        vis[2 * k] = re;
        vis[2 * k + 1] = im;
    }
}

void oracle_dft_grid(int64_t M, const double *uvw, const double *vis, int64_t P,
                     const double *lmn, double *d)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        const double l = lmn[3 * p], m = lmn[3 * p + 1], nm1 = lmn[3 * p + 2];
        double re = 0.0, im = 0.0;
        for (int64_t k = 0; k < M; ++k) {
            const double ph = TWO_PI * reduce_turns(uvw[3 * k] * l + uvw[3 * k + 1] * m +
                                                    uvw[3 * k + 2] * nm1);
            const double c = cos(ph), s = sin(ph);
            const double vr = vis[2 * k], vi = vis[2 * k + 1];
            /* V * exp(+i ph) */
            re += vr * c - vi * s;
            im += vi * c + vr * s;
        }
        d[2 * p] = re;
        d[2 * p + 1] = im;
    }
}
