// Direct (O(N^2 M^2)) evaluation of the diffraction sums at destination
// points, on the GPU: Eq. 7 (the Fourier form the NUFFT computes), Eq. 5 (the
// destination chirp with r0 = z0 - d1 per sample, before the approximation of
// Eq. 6) and Eq. 2 (the Huygens sum with the exact distance of Eq. 3, before
// the Fresnel expansion of Eq. 4).  They measure what those approximations
// cost at 2D scale and serve as a fast reference on sampled points.
//
// Phases are carried in half-turns (k L = pi (2 L / lambda)) and formed in
// FP64 per (sample, point) pair from FP64 per-sample terms, reduced modulo 2
// exactly (h - 2 rint(h/2)) and evaluated with sincospif on the reduced
// fraction; products with u1 are FP32 and the sums are accumulated in FP64.
//   Eq. 7: h = |x1|^2/(lambda r0) - 2 x1.x2/(lambda r0) + 2 (s.x1 + (sz - 1) d1)/lambda
//          (the last term is u_I exp(-ik d1) for a plane wave with direction
//          cosines (sx, sy, sz); zero at normal incidence)
//   Eq. 5: h = the Eq. 7 phase + |x2|^2/(lambda r0)
//   Eq. 2: h = 2 (s.x1 + sz d1 + r)/lambda, amplitude 1/r^2, r = |(x2 - x1, z0 - d1)|
// Outer factors: p1x p1y exp(ik(z0 + |x2|^2/(2 z0)))/(i lambda z0) (Eq. 7),
// p1x p1y exp(ik z0)/(i lambda z0) (Eq. 5), p1x p1y z0/(i lambda) (Eq. 2).
#include <cmath>
#include <string>

#include "asfd_impl.cuh"

namespace asfd {

namespace {

constexpr int kDirectThreads = 256;
constexpr int kDirectPoints = 8;  // destination points per block (shares the sample loads)

struct DirectGeom {
    int n1x, n1y, m2x, m2y;
    double p1x, p1y, p2x, p2y, lambda, z0;
    double sx, sy, sz;  // incident plane wave direction cosines
    double ox, oy;      // source grid offset
};

// The four FP64 terms of one source sample, 32-byte aligned (one load).
struct alignas(32) DirectTerms {
    double x, y, z, w;
};

// per sample: Eq. 5/7 {|x1|^2/(lambda r0) + 2 (s.x1 + (sz - 1) d1)/lambda,
// 2 x1x/(lambda r0), 2 x1y/(lambda r0), 1/(lambda r0)} (the first term carries
// u_I exp(-ik d1), 1 at normal incidence); Eq. 2 {x1x, x1y, z0 - d1,
// 2 (s.x1 + sz d1)/lambda} (the phase of u_I)
__global__ void direct_prep_kernel(DirectGeom g, const double* __restrict__ d1, int form,
                                   DirectTerms* __restrict__ out)
{
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (size_t)g.n1x * g.n1y) return;
    const int nx = (int)(n % g.n1x), ny = (int)(n / g.n1x);
    const double x = (nx - g.n1x / 2) * g.p1x + g.ox, y = (ny - g.n1y / 2) * g.p1y + g.oy;
    const double h = d1[n];
    const double lin = g.sx * x + g.sy * y;
    if (form == 2) {
        out[n] = DirectTerms{x, y, g.z0 - h, 2.0 * (lin + g.sz * h) / g.lambda};
    } else {
        const double inv = 1.0 / (g.lambda * (g.z0 - h));
        const double inc = 2.0 * (lin + (g.sz - 1.0) * h) / g.lambda;
        out[n] = DirectTerms{(x * x + y * y) * inv + inc, 2.0 * x * inv, 2.0 * y * inv, inv};
    }
}

__device__ __forceinline__ float reduce_halfturns(double h)
{
    return (float)(h - 2.0 * rint(0.5 * h));
}

template <int FORM>
__global__ void __launch_bounds__(kDirectThreads)
direct_sum_kernel(DirectGeom g, const DirectTerms* __restrict__ s, const float2* __restrict__ u1,
                  int npts, const int* __restrict__ mx, const int* __restrict__ my,
                  float2* __restrict__ out)
{
    __shared__ double red[2][kDirectPoints][kDirectThreads / 32];
    const int p0 = blockIdx.x * kDirectPoints;
    double x2x[kDirectPoints], x2y[kDirectPoints], x2sq[kDirectPoints];
#pragma unroll
    for (int j = 0; j < kDirectPoints; ++j) {
        const int i = min(p0 + j, npts - 1);
        x2x[j] = (mx[i] - g.m2x / 2) * g.p2x;
        x2y[j] = (my[i] - g.m2y / 2) * g.p2y;
        x2sq[j] = x2x[j] * x2x[j] + x2y[j] * x2y[j];
    }
    double accr[kDirectPoints], acci[kDirectPoints];
#pragma unroll
    for (int j = 0; j < kDirectPoints; ++j) accr[j] = acci[j] = 0.0;
    const size_t total = (size_t)g.n1x * g.n1y;
    for (size_t n = threadIdx.x; n < total; n += kDirectThreads) {
        const DirectTerms t = s[n];
        const float2 u = __ldg(&u1[n]);
#pragma unroll
        for (int j = 0; j < kDirectPoints; ++j) {
            float amp = 1.0f;
            double h;
            if constexpr (FORM == 2) {
                const double dx = x2x[j] - t.x, dy = x2y[j] - t.y;
                const double r2 = fma(dx, dx, fma(dy, dy, t.z * t.z));
                h = fma(2.0 / g.lambda, sqrt(r2), t.w);
                amp = (float)(1.0 / r2);
            } else {
                h = t.x - fma(t.y, x2x[j], t.z * x2y[j]);
                if constexpr (FORM == 5) h = fma(t.w, x2sq[j], h);
            }
            float sn, cs;
            sincospif(reduce_halfturns(h), &sn, &cs);
            const float re = (u.x * cs - u.y * sn) * amp, im = (u.x * sn + u.y * cs) * amp;
            accr[j] += (double)re;
            acci[j] += (double)im;
        }
    }
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
    for (int j = 0; j < kDirectPoints; ++j) {
        double a = accr[j], b = acci[j];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            red[0][j][warp] = a;
            red[1][j][warp] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < kDirectPoints && p0 + (int)threadIdx.x < npts) {
        const int j = threadIdx.x;
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kDirectThreads / 32; ++w) {
            a += red[0][j][w];
            b += red[1][j][w];
        }
        // outer factor o = f * exp(i pi ph) / i = f (sin(pi ph) - i cos(pi ph))
        const double wgt = g.p1x * g.p1y;
        double f, ph;
        if (FORM == 2) {
            f = wgt * g.z0 / g.lambda;
            ph = 0.0;
        } else {
            f = wgt / (g.lambda * g.z0);
            ph = 2.0 * g.z0 / g.lambda;
            if (FORM == 7) ph += x2sq[j] / (g.lambda * g.z0);
        }
        ph -= 2.0 * rint(0.5 * ph);
        double sp, cp;
        sincospi(ph, &sp, &cp);
        const double ore = f * sp, oim = -f * cp;
        out[p0 + j] = make_float2((float)(ore * a - oim * b), (float)(ore * b + oim * a));
    }
}

}  // namespace

asfd_status direct_sum(const asfd_params* p, const double* d1, const float2* u1, int form,
                       int npts, const int* mx, const int* my, float2* out, cudaStream_t st)
{
    if (!p || !d1 || !u1 || npts < 0)
        return fail(ASFD_ERR_ARG, "NULL argument or negative point count");
    if (npts > 0 && (!mx || !my || !out)) return fail(ASFD_ERR_ARG, "NULL point or output array");
    if (form != 2 && form != 5 && form != 7)
        return fail(ASFD_ERR_ARG, "form must be 2, 5 or 7 (the paper's Eq. 2, 5 or 7)");
    if (p->n1x < 2 || p->n1y < 2 || p->m2x < 2 || p->m2y < 2 || p->n1x % 2 || p->n1y % 2 ||
        p->m2x % 2 || p->m2y % 2 || p->n1x > 65536 || p->n1y > 65536)
        return fail(ASFD_ERR_ARG, "n1x, n1y, m2x, m2y must be even, >= 2 (n1 <= 65536)");
    const double pos[] = {p->p1x, p->p1y, p->p2x, p->p2y, p->lambda, p->z0};
    for (double x : pos)
        if (!(std::isfinite(x) && x > 0.0))
            return fail(ASFD_ERR_ARG, "pitches, wavelength and z0 must be finite and > 0");
    if (!(std::isfinite(p->incidence_sx) && std::isfinite(p->incidence_sy) &&
          p->incidence_sx * p->incidence_sx + p->incidence_sy * p->incidence_sy < 1.0))
        return fail(ASFD_ERR_ARG, "incidence direction cosines need sx^2 + sy^2 < 1");
    if (!(std::isfinite(p->offset_x) && std::isfinite(p->offset_y)))
        return fail(ASFD_ERR_ARG, "source offsets must be finite");
    if (npts == 0) return ASFD_OK;
    const double sz = std::sqrt(1.0 - p->incidence_sx * p->incidence_sx -
                                p->incidence_sy * p->incidence_sy);
    DirectGeom g{p->n1x, p->n1y, p->m2x, p->m2y, p->p1x, p->p1y, p->p2x, p->p2y,
                 p->lambda, p->z0, p->incidence_sx, p->incidence_sy, sz, p->offset_x,
                 p->offset_y};
    const size_t n = (size_t)p->n1x * p->n1y;
    DirectTerms* s = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&s), sizeof(DirectTerms) * n, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ASFD_ERR_NOMEM, std::string("per-sample terms: ") + cudaGetErrorString(e));
    }
    direct_prep_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, d1, form, s);
    const unsigned blocks = (unsigned)((npts + kDirectPoints - 1) / kDirectPoints);
    if (form == 2)
        direct_sum_kernel<2><<<blocks, kDirectThreads, 0, st>>>(g, s, u1, npts, mx, my, out);
    else if (form == 5)
        direct_sum_kernel<5><<<blocks, kDirectThreads, 0, st>>>(g, s, u1, npts, mx, my, out);
    else
        direct_sum_kernel<7><<<blocks, kDirectThreads, 0, st>>>(g, s, u1, npts, mx, my, out);
    e = cudaGetLastError();
    const cudaError_t ef = cudaFreeAsync(s, st);
    if (e != cudaSuccess) return cuda_fail(e, "direct_sum_kernel launch");
    if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
    return ASFD_OK;
}

}  // namespace asfd
