// One-dimensional form with explicit source samples (an extension: the
// paper's own experiments, Sec. 3, are line sources sampled along their arc
// length).  Sample j sits at x1[j] with height d1[j] and quadrature weight
// w[j] (its extent along x1); the destination line is x2 = (m - M/2) p2.
// Eq. 7 in one dimension, with r0 = z0 - d1 and the incident plane wave
// u_I = exp(ik(s x1 + sz d1)), sz = sqrt(1 - s^2):
//
//   u2(x2) = exp(ik(z0 + x2^2/(2 z0))) / sqrt(i lambda z0)
//            * sum_j w u_I u1 exp(ik(-d1 + x1^2/(2 r0))) exp(-ik x1 x2 / r0)
//
// (the 1D Fresnel prefactor 1/sqrt(i lambda z0) is a reading; the paper
// prints the 2D forms).  As in 2D this is a type-1 NUFFT at the fine-grid
// coordinate g = x1 p2 nf/(lambda r0): the plan forms, in FP64 and once, each
// sample's prefactor E_j = w exp(i pi h), h = x1^2/(lambda r0) +
// 2 (s x1 + (sz - 1) d1)/lambda half-turns reduced modulo 2, and the
// integer/fraction split of g + nf/2; an execution multiplies u1 by E,
// spreads with the ES kernel (float2 atomic adds into the nf-point line),
// transforms the line with the library's Stockham FFT and applies
// (-1)^m' exp(ik x2^2/(2 z0)) / psi_hat(2 pi m'/nf) and the global factor.
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "asfd_impl.cuh"
#include "sample.cuh"

struct asfd_line_plan_s {
    asfd_line_params prm;
    int device = 0;
    int n = 0, nf = 0, w = 0;
    double beta = 0.0;
    float2* e = nullptr;      // [n] per-sample prefactor (with the weight)
    int* bi = nullptr;        // [n] integer part of g + nf/2 (mod nf)
    float* bf = nullptr;      // [n] fraction
    float2* grid = nullptr;   // [nf]
    float2* c = nullptr;      // [m2] destination table
    double* quad = nullptr;
    unsigned* status = nullptr;
};

namespace asfd {

namespace {

__device__ __forceinline__ double line_reduce(double h) { return h - 2.0 * rint(0.5 * h); }

__global__ void line_prep_kernel(const double* __restrict__ x1, const double* __restrict__ d1,
                                 const double* __restrict__ w, int n, double lambda, double z0,
                                 double p2, int nf, double s, double sz, float2* __restrict__ e,
                                 int* __restrict__ bi, float* __restrict__ bf,
                                 unsigned* __restrict__ status)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double x = x1[j], h = d1[j], wt = w[j];
    if (!isfinite(x) || !isfinite(h) || !isfinite(wt) || !(h < z0)) {
        atomicOr(status, kStatusBadD1);
        e[j] = make_float2(0.f, 0.f);
        bi[j] = 0;
        bf[j] = 0.f;
        return;
    }
    const double r0 = z0 - h;
    const double ph = line_reduce(x * x / (lambda * r0)) + line_reduce(2.0 * (s * x + (sz - 1.0) * h) / lambda);
    double sn, cs;
    sincospi(ph, &sn, &cs);
    e[j] = make_float2((float)(wt * cs), (float)(wt * sn));
    const double g = x * p2 * (double)nf / (lambda * r0) + 0.5 * (double)nf;
    const double gr = g - (double)nf * floor(g / (double)nf);
    int b = (int)floor(gr);
    double f = gr - (double)b;
    if (b >= nf) b -= nf;
    bi[j] = b;
    bf[j] = (float)f;
}

// C[k] = (-1)^m' exp(i pi x2^2/(lambda z0)) / psi_hat(2 pi m'/nf) * exp(ik z0) exp(-i pi/4)
//        / sqrt(lambda z0),  m' = k - m2/2
__global__ void line_dest_kernel(float2* __restrict__ C, int m2, double p2, double lambda,
                                 double z0, int nf, const double* __restrict__ quad, int nq)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m2) return;
    const int mp = k - m2 / 2;
    const double x2 = (double)mp * p2;
    double psi_hat = 0.0;
    for (int i = 0; i < nq; ++i) psi_hat += quad[nq + i] * cospi(2.0 * (double)mp * quad[i] / (double)nf);
    psi_hat *= 2.0;
    const double ph = line_reduce(x2 * x2 / (lambda * z0)) + line_reduce(2.0 * z0 / lambda) - 0.25;
    double sn, cs;
    sincospi(ph, &sn, &cs);
    const double a = ((mp & 1) ? -1.0 : 1.0) / (psi_hat * sqrt(lambda * z0));
    C[k] = make_float2((float)(a * cs), (float)(a * sn));
}

template <int W>
__global__ void __launch_bounds__(256) line_spread_kernel(const float2* __restrict__ u1,
                                                          const float2* __restrict__ e,
                                                          const int* __restrict__ bi,
                                                          const float* __restrict__ bf, int n,
                                                          int nf, float half_w, float two_over_w,
                                                          float beta_log2e, float2* __restrict__ grid)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float2 u = __ldg(&u1[j]), ej = __ldg(&e[j]);
    const float2 c = make_float2(u.x * ej.x - u.y * ej.y, u.x * ej.y + u.y * ej.x);
    const float f = __ldg(&bf[j]) - half_w;
    const float cf = ceilf(f);
    const int l0 = __ldg(&bi[j]) + (int)cf;
    const float dx = cf - f;
    const int mask = nf - 1;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const float wv = es_weight_fast(dx + (float)i - half_w, two_over_w, beta_log2e);
        atomicAdd(&grid[(l0 + i) & mask], make_float2(c.x * wv, c.y * wv));
    }
}

__global__ void line_finish_kernel(const float2* __restrict__ grid, const float2* __restrict__ C,
                                   int m2, int nf, float2* __restrict__ u2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m2) return;
    const float2 b = grid[(k - m2 / 2) & (nf - 1)], c = C[k];
    u2[k] = make_float2(b.x * c.x - b.y * c.y, b.x * c.y + b.y * c.x);
}

void line_free(asfd_line_plan_s* P)
{
    void* bufs[] = {P->e, P->bi, P->bf, P->grid, P->c, P->quad, P->status};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete P;
}

}  // namespace
}  // namespace asfd

using namespace asfd;

extern "C" {

asfd_status asfd_line_plan_create(asfd_line_plan* out, const asfd_line_params* p,
                                  const double* x1_dev, const double* d1_dev, const double* w_dev,
                                  int n, void* stream)
{
    clear_error();
    if (!out || !p || !x1_dev || !d1_dev || !w_dev || n < 1)
        return fail(ASFD_ERR_ARG, "out, params and sample arrays must be non-NULL, n >= 1");
    *out = nullptr;
    if (p->m2 < 2 || p->m2 % 2) return fail(ASFD_ERR_ARG, "m2 must be even and >= 2");
    const double pos[] = {p->p2, p->lambda, p->z0, p->sigma};
    for (double v : pos)
        if (!(std::isfinite(v) && v > 0.0))
            return fail(ASFD_ERR_ARG, "p2, wavelength, z0 and sigma must be finite and > 0");
    if (!(std::isfinite(p->incidence_s) && p->incidence_s * p->incidence_s < 1.0))
        return fail(ASFD_ERR_ARG, "incidence direction cosine needs s^2 < 1");
    if (p->kernel_width < 2 || p->kernel_width > 16)
        return fail(ASFD_ERR_UNSUPPORTED, "kernel_width must be in [2, 16]");
    const double fnf = p->sigma * p->m2;
    const int nf = (int)std::lround(fnf);
    if (std::fabs(fnf - nf) > 1e-9 * fnf || nf < 64 || nf > 16384 || (nf & (nf - 1)))
        return fail(ASFD_ERR_UNSUPPORTED, "sigma*m2 must be a power of two in [64, 16384]");
    if (p->kernel_width >= nf / 2) return fail(ASFD_ERR_UNSUPPORTED, "kernel wider than half the line");
    if (!(std::isfinite(p->es_beta) && p->es_beta >= 0.0))
        return fail(ASFD_ERR_ARG, "es_beta must be finite and >= 0");
    asfd_line_plan_s* P = new (std::nothrow) asfd_line_plan_s();
    if (!P) return fail(ASFD_ERR_NOMEM, "host allocation of the plan failed");
    P->prm = *p;
    P->n = n;
    P->nf = nf;
    P->w = p->kernel_width;
    const double pi = 3.14159265358979323846;
    P->beta = p->es_beta > 0.0 ? p->es_beta
                               : (p->sigma == 2.0 ? 2.30 * p->kernel_width
                                                  : 0.97 * pi * (1.0 - 1.0 / (2.0 * p->sigma)) *
                                                        p->kernel_width);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    asfd_status s = [&]() -> asfd_status {
        ASFD_CUDA(cudaGetDevice(&P->device));
        ASFD_CUDA(cudaMalloc(&P->e, sizeof(float2) * n));
        ASFD_CUDA(cudaMalloc(&P->bi, sizeof(int) * n));
        ASFD_CUDA(cudaMalloc(&P->bf, sizeof(float) * n));
        ASFD_CUDA(cudaMalloc(&P->grid, sizeof(float2) * nf));
        ASFD_CUDA(cudaMalloc(&P->c, sizeof(float2) * p->m2));
        ASFD_CUDA(cudaMalloc(&P->status, sizeof(unsigned)));
        std::vector<double> h;
        const int nq = es_quadrature(P->w, P->beta, h);
        ASFD_CUDA(cudaMalloc(&P->quad, sizeof(double) * h.size()));
        ASFD_CUDA(cudaMemcpyAsync(P->quad, h.data(), sizeof(double) * h.size(),
                                  cudaMemcpyHostToDevice, st));
        ASFD_CUDA(cudaMemsetAsync(P->status, 0, sizeof(unsigned), st));
        const double sz = std::sqrt(1.0 - p->incidence_s * p->incidence_s);
        line_prep_kernel<<<(n + 255) / 256, 256, 0, st>>>(x1_dev, d1_dev, w_dev, n, p->lambda,
                                                           p->z0, p->p2, nf, p->incidence_s, sz,
                                                           P->e, P->bi, P->bf, P->status);
        line_dest_kernel<<<(p->m2 + 255) / 256, 256, 0, st>>>(P->c, p->m2, p->p2, p->lambda,
                                                               p->z0, nf, P->quad, nq);
        ASFD_CUDA(cudaGetLastError());
        unsigned bad = 0;
        ASFD_CUDA(cudaMemcpyAsync(&bad, P->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        ASFD_CUDA(cudaStreamSynchronize(st));
        if (bad)
            return fail(ASFD_ERR_ARG, "x1, d1 and w must be finite and every d1 below z0");
        return ASFD_OK;
    }();
    if (s != ASFD_OK) {
        const std::string msg = asfd_last_error();
        line_free(P);
        return fail(s, msg);
    }
    *out = P;
    return ASFD_OK;
}

asfd_status asfd_line_execute(asfd_line_plan P, const float* u1_dev, float* u2_dev, void* stream)
{
    clear_error();
    if (!P || !u1_dev || !u2_dev) return fail(ASFD_ERR_ARG, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != P->device) {
        const cudaError_t e = cudaSetDevice(P->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    }
    asfd_status s = [&]() -> asfd_status {
        ASFD_CUDA(cudaMemsetAsync(P->grid, 0, sizeof(float2) * P->nf, st));
        const float half_w = 0.5f * (float)P->w;
        const float two_over_w = (float)(2.0 / P->w);
        const float bl2e = (float)(P->beta * 1.4426950408889634074);
        const unsigned blocks = (unsigned)((P->n + 255) / 256);
        const float2* u1 = reinterpret_cast<const float2*>(u1_dev);
        switch (P->w) {
#define ASFD_LW(W)                                                                         \
    case W:                                                                                \
        line_spread_kernel<W><<<blocks, 256, 0, st>>>(u1, P->e, P->bi, P->bf, P->n, P->nf, \
                                                      half_w, two_over_w, bl2e, P->grid);  \
        break;
            ASFD_LW(2) ASFD_LW(3) ASFD_LW(4) ASFD_LW(5) ASFD_LW(6) ASFD_LW(7) ASFD_LW(8)
            ASFD_LW(9) ASFD_LW(10) ASFD_LW(11) ASFD_LW(12) ASFD_LW(13) ASFD_LW(14) ASFD_LW(15)
            ASFD_LW(16)
#undef ASFD_LW
            default: return fail(ASFD_ERR_UNSUPPORTED, "kernel width outside 2..16");
        }
        ASFD_CUDA(cudaGetLastError());
        asfd_status f = launch_fft_lines(P->nf, 1, -1, P->grid, P->grid, st);
        if (f != ASFD_OK) return f;
        line_finish_kernel<<<(P->prm.m2 + 255) / 256, 256, 0, st>>>(
            P->grid, P->c, P->prm.m2, P->nf, reinterpret_cast<float2*>(u2_dev));
        ASFD_CUDA(cudaGetLastError());
        return ASFD_OK;
    }();
    if (dev != P->device && dev >= 0) cudaSetDevice(dev);
    return s;
}

asfd_status asfd_line_destroy(asfd_line_plan P)
{
    clear_error();
    if (!P) return ASFD_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    const int own = P->device;  // P is gone after line_free
    if (dev != own) cudaSetDevice(own);
    line_free(P);
    if (dev != own && dev >= 0) cudaSetDevice(dev);
    return ASFD_OK;
}

}  // extern "C"
