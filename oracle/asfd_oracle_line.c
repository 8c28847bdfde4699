/*
 * FP64 CPU oracle of the one-dimensional form with explicit source samples.
 *
 * TEST INFRASTRUCTURE ONLY (as asfd_oracle.c): only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * table or constant with the CUDA path.
 *
 * A line source sampled at arbitrary positions: sample n sits at x1[n] on the
 * source axis with height d1[n] and carries the quadrature weight w[n] (its
 * extent along x1, e.g. the projected arc-length step of a tilted facet).
 * The paper's experiments (Sec. 3) are of this kind.  Destination points are
 * x2 = (m - M/2) p2.  With r0 = z0 - d1 and u_I = exp(ik(s x1 + sz d1)),
 * sz = sqrt(1 - s^2) (s = 0: the normally incident plane wave of Sec. 2):
 *
 *   form 7 (Eq. 7):  exp(ik(z0 + x2^2/(2 z0))) / sqrt(i lambda z0)
 *                    * sum_n w u_I u1 exp(ik(-d1 + x1^2/(2 r0))) exp(-ik x1 x2 / r0)
 *   form 5 (Eq. 5):  exp(ik z0) / sqrt(i lambda z0)
 *                    * sum_n w u_I u1 exp(ik(-d1 + x1^2/(2 r0))) exp(-ik x1 x2 / r0)
 *                                     exp(ik x2^2/(2 r0))
 *   form 2 (Eq. 2):  z0 / sqrt(i lambda) * sum_n w u_I u1 exp(ik r) / r^(3/2),
 *                    r = sqrt((x2 - x1)^2 + (z0 - d1)^2)
 *
 * Readings (the paper prints only the 2D forms): the 1D Fresnel prefactor is
 * 1/sqrt(i lambda z0), and the 1D Huygens kernel is the 2D one, z0 exp(ikR)/
 * (i lambda R^2), integrated along the invariant y axis by stationary phase,
 * z0 exp(ikR) / (sqrt(i lambda) R^(3/2)), which is 1/sqrt(i lambda z0) at R = z0.
 * Complex arrays are interleaved (re, im) FP64 pairs.
 */
#include <math.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int m2;            /* destination samples (even)                     */
    double p2;         /* destination pitch [m]                          */
    double lambda;     /* wavelength [m]                                 */
    double z0;         /* distance between source axis and destination   */
    double s;          /* direction cosine of the incident plane wave    */
} asfd_oracle_line_geom;

static const double LINE_PI = 3.14159265358979323846264338327950288;

int asfd_oracle_line(const asfd_oracle_line_geom* g, const double* x1, const double* d1,
                     const double* w, const double* u1, int n, int form, int npts, const int* m,
                     double* out, int nthreads)
{
    if (!g || !x1 || !d1 || !w || !u1 || !m || !out || n < 0 || npts < 0) return -1;
    if (form != 2 && form != 5 && form != 7) return -1;
    if (!(g->s * g->s < 1.0)) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const double k = 2.0 * LINE_PI / g->lambda;
    const double sz = sqrt(1.0 - g->s * g->s);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < npts; ++i) {
        const double x2 = (m[i] - g->m2 / 2) * g->p2;
        double acc_re = 0.0, acc_im = 0.0;
        for (int j = 0; j < n; ++j) {
            const double h = d1[j], x = x1[j];
            const double ph_inc = k * (g->s * x + sz * h);  /* u_I */
            double ph, amp = w[j];
            if (form == 2) {
                const double dx = x2 - x, dz = g->z0 - h;
                const double r = sqrt(dx * dx + dz * dz);
                ph = ph_inc + k * r;
                amp /= r * sqrt(r);
            } else {
                const double r0 = g->z0 - h;
                ph = ph_inc + k * (-h + x * x / (2.0 * r0)) - k * x * x2 / r0;
                if (form == 5) ph += k * x2 * x2 / (2.0 * r0);
            }
            const double c = amp * cos(ph), sn = amp * sin(ph);
            const double ur = u1[2 * j], ui = u1[2 * j + 1];
            acc_re += ur * c - ui * sn;
            acc_im += ur * sn + ui * c;
        }
        /* prefactor: 1/sqrt(i) = exp(-i pi/4) */
        double f, ph0;
        if (form == 2) {
            f = g->z0 / sqrt(g->lambda);
            ph0 = -0.25 * LINE_PI;
        } else {
            f = 1.0 / sqrt(g->lambda * g->z0);
            ph0 = k * g->z0 - 0.25 * LINE_PI;
            if (form == 7) ph0 += k * x2 * x2 / (2.0 * g->z0);
        }
        const double o_re = f * cos(ph0), o_im = f * sin(ph0);
        out[2 * i] = o_re * acc_re - o_im * acc_im;
        out[2 * i + 1] = o_re * acc_im + o_im * acc_re;
    }
    return 0;
}
