/*
 * FP64 CPU oracle for arbitrary-shape-surface Fresnel diffraction.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, table or
 * constant with the CUDA path.
 *
 * What it computes (Shimobaba, Masuda, Ito, "Arbitrary shape surface Fresnel
 * diffraction", Sec. 2):
 *
 *   u(x2) = exp(ik(z0 + |x2|^2/(2 z0))) / (i lambda z0)
 *           * sum_n  p1x p1y * u_I(n) * u1(n)
 *                    * exp(ik(-d1(n) + |x1(n)|^2 / (2 r0(n))))
 *                    * exp(-ik x1(n).x2 / r0(n)),      r0(n) = z0 - d1(n)
 *
 * i.e. the discretised Eq. 7 (the Fourier form obtained from Eq. 5 with the
 * destination-chirp approximation of Eq. 6), which is exactly the sum that
 * the NUFT of Eq. 8 evaluates.  u_I = exp(ik d1) is the normally incident
 * plane wave (Sec. 2, after Eq. 3); a plane wave with direction cosines
 * (sx, sy) gives u_I = exp(ik(sx x + sy y + sz d1)) (geometry fields sx, sy;
 * the incidence extension of the method).  The oracle forms u_I and the
 * exp(-ik d1) factor of Eq. 5 separately, as written, and accumulates every
 * term in FP64 with no table, no kernel and no FFT.
 *
 * Readings where the paper is garbled or silent:
 *  - cross-term sign: Eq. 7 prints "+ik x1.x2/(z0-d1)"; Eqs. 4 and 5 and the
 *    NUFT definition (Eq. 9) carry a minus sign.  The minus sign is used.
 *  - quadrature weight of the integral over x1: the projected area element
 *    p1x*p1y of the uniform source grid.
 *  - coordinates: x1 = ((nx - N1x/2) p1x, (ny - N1y/2) p1y) + (ox, oy),
 *                 x2 = ((mx - M2x/2) p2x, (my - M2y/2) p2y); the offset (ox, oy)
 *                 (zero by default) places a surface off the axis, for sums of
 *                 several surfaces.
 *  - arrays are row-major [y][x], x fastest; complex values are interleaved
 *    (re, im) FP64 pairs.
 *
 * Also Eq. 5 (asfd_oracle_eq5: the destination chirp with r0 per sample) and
 * Eq. 2 (asfd_oracle_eq2: the exact distance of Eq. 3, no Fresnel
 * approximation), for measuring the approximations of Eqs. 4 and 6.
 *
 * Pins (tests/test_oracle_pins.py): single-sample closed form, d1 = 0 at the
 * natural pitch against numpy's FFT, d1 = const against two dense DFT matmuls
 * and against planar single-FFT Fresnel propagation over z0 - c, terraced
 * (piecewise-constant) d1 against a sum of per-terrace FFT propagations, the
 * closed-form Fresnel propagation of a Gaussian beam, linearity, and central
 * finite differences for the gradient routine.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n1x, n1y;      /* source samples along x and y (even)            */
    double p1x, p1y;   /* source pitch [m]                               */
    int m2x, m2y;      /* destination samples (even)                     */
    double p2x, p2y;   /* destination pitch [m]                          */
    double lambda;     /* wavelength [m]                                 */
    double z0;         /* distance between the planes z = 0 and z = z0  */
    double sx, sy;     /* direction cosines of the incident plane wave   */
    double ox, oy;     /* position of the source grid's centre sample    */
} asfd_oracle_geom;

/* Phase of the incident plane wave u_I = exp(ik(sx x + sy y + sz d1)),
 * sz = sqrt(1 - sx^2 - sy^2); normal incidence (sx = sy = 0) gives the
 * exp(ik d1) of Sec. 2. */
static double incident_phase(const asfd_oracle_geom* g, double k, double x, double y, double h)
{
    const double sz = sqrt(1.0 - g->sx * g->sx - g->sy * g->sy);
    return k * (g->sx * x + g->sy * y + sz * h);
}

static int bad_geom(const asfd_oracle_geom* g)
{
    return !(g->sx * g->sx + g->sy * g->sy < 1.0);
}

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int asfd_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Outer factor of Eq. 7 / Eq. 8 at destination point (x2x, x2y):
 * exp(ik(z0 + |x2|^2/(2 z0))) / (i lambda z0). */
static void outer_factor(const asfd_oracle_geom* g, double x2x, double x2y,
                         double* re, double* im)
{
    const double k = 2.0 * ORACLE_PI / g->lambda;
    const double ph = k * (g->z0 + (x2x * x2x + x2y * x2y) / (2.0 * g->z0));
    /* 1/(i a) = -i/a */
    const double a = g->lambda * g->z0;
    *re = sin(ph) / a;
    *im = -cos(ph) / a;
}

/*
 * Eq. 7 evaluated at npts destination points (mx[i], my[i]).
 * u1: [n1y][n1x] complex (interleaved), d1: [n1y][n1x] metres,
 * out: npts complex (interleaved).  Returns 0, or -1 on a bad argument.
 */
int asfd_oracle_eq7(const asfd_oracle_geom* g, const double* u1, const double* d1,
                    int npts, const int* mx, const int* my, double* out, int nthreads)
{
    if (!g || !u1 || !d1 || !mx || !my || !out || npts < 0 || bad_geom(g)) return -1;
    const double k = 2.0 * ORACLE_PI / g->lambda;
    const double w = g->p1x * g->p1y;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < npts; ++i) {
        const double x2x = (mx[i] - g->m2x / 2) * g->p2x;
        const double x2y = (my[i] - g->m2y / 2) * g->p2y;
        double acc_re = 0.0, acc_im = 0.0;
        for (int ny = 0; ny < g->n1y; ++ny) {
            const double x1y = (ny - g->n1y / 2) * g->p1y + g->oy;
            double row_re = 0.0, row_im = 0.0;
            for (int nx = 0; nx < g->n1x; ++nx) {
                const size_t n = (size_t)ny * g->n1x + nx;
                const double x1x = (nx - g->n1x / 2) * g->p1x + g->ox;
                const double h = d1[n];
                const double r0 = g->z0 - h;
                /* incident plane wave u_I */
                const double ph_inc = incident_phase(g, k, x1x, x1y, h);
                /* exp(ik(-d1 + |x1|^2/(2 r0))) */
                const double ph_src = k * (-h + (x1x * x1x + x1y * x1y) / (2.0 * r0));
                /* exp(-ik x1.x2 / r0) */
                const double ph_x = -k * (x1x * x2x + x1y * x2y) / r0;
                const double ph = ph_inc + ph_src + ph_x;
                const double c = cos(ph), s = sin(ph);
                const double ur = u1[2 * n], ui = u1[2 * n + 1];
                row_re += ur * c - ui * s;
                row_im += ur * s + ui * c;
            }
            acc_re += row_re;
            acc_im += row_im;
        }
        acc_re *= w;
        acc_im *= w;
        double o_re, o_im;
        outer_factor(g, x2x, x2y, &o_re, &o_im);
        out[2 * i] = o_re * acc_re - o_im * acc_im;
        out[2 * i + 1] = o_re * acc_im + o_im * acc_re;
    }
    return 0;
}

/*
 * Eq. 5 (Fresnel diffraction from the arbitrary surface before the
 * destination-chirp approximation of Eq. 6) at npts destination points:
 *
 *   u(x2) = exp(ik z0) / (i lambda z0)
 *           * sum_n p1x p1y u_I(n) u1(n) exp(ik(-d1 + |x1|^2/(2 r0)))
 *                   exp(-ik x1.x2 / r0) exp(ik |x2|^2 / (2 r0)),
 *
 * with r0 = z0 - d1(n) in all three exponentials.  The last exponential is
 * printed without "ik" in the paper; it is read as exp(ik|x2|^2/(2 r0)), the
 * term of Eq. 4 it comes from.  Arguments as for asfd_oracle_eq7.
 */
int asfd_oracle_eq5(const asfd_oracle_geom* g, const double* u1, const double* d1,
                    int npts, const int* mx, const int* my, double* out, int nthreads)
{
    if (!g || !u1 || !d1 || !mx || !my || !out || npts < 0 || bad_geom(g)) return -1;
    const double k = 2.0 * ORACLE_PI / g->lambda;
    const double w = g->p1x * g->p1y;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < npts; ++i) {
        const double x2x = (mx[i] - g->m2x / 2) * g->p2x;
        const double x2y = (my[i] - g->m2y / 2) * g->p2y;
        const double x2sq = x2x * x2x + x2y * x2y;
        double acc_re = 0.0, acc_im = 0.0;
        for (int ny = 0; ny < g->n1y; ++ny) {
            const double x1y = (ny - g->n1y / 2) * g->p1y + g->oy;
            double row_re = 0.0, row_im = 0.0;
            for (int nx = 0; nx < g->n1x; ++nx) {
                const size_t n = (size_t)ny * g->n1x + nx;
                const double x1x = (nx - g->n1x / 2) * g->p1x + g->ox;
                const double h = d1[n];
                const double r0 = g->z0 - h;
                const double ph_inc = incident_phase(g, k, x1x, x1y, h);  /* u_I */
                const double ph_src = k * (-h + (x1x * x1x + x1y * x1y) / (2.0 * r0));
                const double ph_x = -k * (x1x * x2x + x1y * x2y) / r0;
                const double ph_dst = k * x2sq / (2.0 * r0);
                const double ph = ph_inc + ph_src + ph_x + ph_dst;
                const double c = cos(ph), s = sin(ph);
                const double ur = u1[2 * n], ui = u1[2 * n + 1];
                row_re += ur * c - ui * s;
                row_im += ur * s + ui * c;
            }
            acc_re += row_re;
            acc_im += row_im;
        }
        acc_re *= w;
        acc_im *= w;
        /* exp(ik z0) / (i lambda z0) */
        const double a = g->lambda * g->z0, ph0 = k * g->z0;
        const double o_re = sin(ph0) / a, o_im = -cos(ph0) / a;
        out[2 * i] = o_re * acc_re - o_im * acc_im;
        out[2 * i + 1] = o_re * acc_im + o_im * acc_re;
    }
    return 0;
}

/*
 * Eq. 2 (Huygens diffraction from the arbitrary surface, no Fresnel
 * approximation) at npts destination points:
 *
 *   u(x2) = z0 / (i lambda) * sum_n p1x p1y u_I(n) u1(n) exp(ik r) / r^2,
 *   r = sqrt(|x2 - x1|^2 + (z0 - d1)^2)                       (Eq. 3),
 *
 * with u_I = exp(ik d1).  Arguments as for asfd_oracle_eq7.
 */
int asfd_oracle_eq2(const asfd_oracle_geom* g, const double* u1, const double* d1,
                    int npts, const int* mx, const int* my, double* out, int nthreads)
{
    if (!g || !u1 || !d1 || !mx || !my || !out || npts < 0 || bad_geom(g)) return -1;
    const double k = 2.0 * ORACLE_PI / g->lambda;
    const double w = g->p1x * g->p1y;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < npts; ++i) {
        const double x2x = (mx[i] - g->m2x / 2) * g->p2x;
        const double x2y = (my[i] - g->m2y / 2) * g->p2y;
        double acc_re = 0.0, acc_im = 0.0;
        for (int ny = 0; ny < g->n1y; ++ny) {
            const double x1y = (ny - g->n1y / 2) * g->p1y + g->oy;
            double row_re = 0.0, row_im = 0.0;
            for (int nx = 0; nx < g->n1x; ++nx) {
                const size_t n = (size_t)ny * g->n1x + nx;
                const double x1x = (nx - g->n1x / 2) * g->p1x + g->ox;
                const double h = d1[n];
                const double dx = x2x - x1x, dy = x2y - x1y, dz = g->z0 - h;
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double r = sqrt(r2);
                const double ph = incident_phase(g, k, x1x, x1y, h) + k * r;
                const double c = cos(ph) / r2, s = sin(ph) / r2;
                const double ur = u1[2 * n], ui = u1[2 * n + 1];
                row_re += ur * c - ui * s;
                row_im += ur * s + ui * c;
            }
            acc_re += row_re;
            acc_im += row_im;
        }
        /* z0 / (i lambda) = -i z0 / lambda */
        const double f = w * g->z0 / g->lambda;
        out[2 * i] = f * acc_im;
        out[2 * i + 1] = -f * acc_re;
    }
    return 0;
}

/*
 * Gradients of a real loss L(u2) through Eq. 7, for the adjoint checks.
 *
 * gu2: npts complex values dL/dRe(u2) + i dL/dIm(u2) at the points
 * (mx[i], my[i]).  Writes, for every source sample n,
 *   gu1[n] = sum_i conj(K_in) gu2[i]                  (complex, may be NULL)
 *   gd1[n] = Re sum_i conj(gu2[i]) dK_in/dd1(n) u1[n]  (real,    may be NULL)
 * where K_in is the coefficient of u1[n] in u2 at point i (Eq. 7), so that
 * dL = Re sum_n conj(gu1[n]) du1[n] + sum_n gd1[n] dd1[n].
 * The d1-derivative of the phase of Eq. 7 is written out term by term:
 *   d/dd1 [k(sx x + sy y + sz d1) + k(-d1 + |x1|^2/(2 r0)) - k x1.x2/r0]
 *     = k sz - k + k|x1|^2/(2 r0^2) - k x1.x2/r0^2      (dr0/dd1 = -1).
 */
int asfd_oracle_eq7_grad(const asfd_oracle_geom* g, const double* u1, const double* d1,
                         int npts, const int* mx, const int* my, const double* gu2,
                         double* gu1, double* gd1, int nthreads)
{
    if (!g || !u1 || !d1 || !mx || !my || !gu2 || npts < 0 || bad_geom(g)) return -1;
    const double k = 2.0 * ORACLE_PI / g->lambda;
    const double w = g->p1x * g->p1y;
    const int nsrc = g->n1x * g->n1y;
    set_threads(nthreads);
    /* precompute conj(O_i) * gu2[i] once per point: the outer factor does not
     * depend on n */
    double* og = (double*)malloc(sizeof(double) * 2 * (size_t)(npts > 0 ? npts : 1));
    if (!og) return -1;
    for (int i = 0; i < npts; ++i) {
        const double x2x = (mx[i] - g->m2x / 2) * g->p2x;
        const double x2y = (my[i] - g->m2y / 2) * g->p2y;
        double o_re, o_im;
        outer_factor(g, x2x, x2y, &o_re, &o_im);
        /* conj(O) * gu2 */
        og[2 * i] = o_re * gu2[2 * i] + o_im * gu2[2 * i + 1];
        og[2 * i + 1] = o_re * gu2[2 * i + 1] - o_im * gu2[2 * i];
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int n = 0; n < nsrc; ++n) {
        const int nx = n % g->n1x, ny = n / g->n1x;
        const double x1x = (nx - g->n1x / 2) * g->p1x + g->ox;
        const double x1y = (ny - g->n1y / 2) * g->p1y + g->oy;
        const double h = d1[n];
        const double r0 = g->z0 - h;
        const double ph_inc = incident_phase(g, k, x1x, x1y, h);
        const double ph_src = k * (-h + (x1x * x1x + x1y * x1y) / (2.0 * r0));
        const double sz = sqrt(1.0 - g->sx * g->sx - g->sy * g->sy);
        const double dph_common = k * sz - k + k * (x1x * x1x + x1y * x1y) / (2.0 * r0 * r0);
        /* S = sum_i conj(O_i) gu2_i exp(-i ph_i)  and
         * D = sum_i conj(O_i) gu2_i exp(-i ph_i) * dph_i/dd1 */
        double s_re = 0.0, s_im = 0.0, d_re = 0.0, d_im = 0.0;
        for (int i = 0; i < npts; ++i) {
            const double x2x = (mx[i] - g->m2x / 2) * g->p2x;
            const double x2y = (my[i] - g->m2y / 2) * g->p2y;
            const double ph_x = -k * (x1x * x2x + x1y * x2y) / r0;
            const double ph = ph_inc + ph_src + ph_x;
            const double dph = dph_common - k * (x1x * x2x + x1y * x2y) / (r0 * r0);
            const double c = cos(ph), s = sin(ph);
            /* og_i * exp(-i ph) */
            const double t_re = og[2 * i] * c + og[2 * i + 1] * s;
            const double t_im = og[2 * i + 1] * c - og[2 * i] * s;
            s_re += t_re;
            s_im += t_im;
            d_re += t_re * dph;
            d_im += t_im * dph;
        }
        /* gu1[n] = w * S  (conj(K) = conj(O) w exp(-i ph)) */
        if (gu1) {
            gu1[2 * n] = w * s_re;
            gu1[2 * n + 1] = w * s_im;
        }
        /* dK/dd1 u1 = K u1 * i dph  ->  conj(gu2) dK/dd1 u1 = conj(conj(K) gu2) * i dph * u1
         * Re(conj(T) * i * u1) summed with weight dph = Re(conj(D) * i * u1) * w */
        if (gd1) {
            const double ur = u1[2 * n], ui = u1[2 * n + 1];
            /* conj(D) * i * u = (d_re - i d_im) * (i ur - ui) -> real part */
            gd1[n] = w * (d_re * (-ui) + d_im * ur);
        }
    }
    free(og);
    return 0;
}
