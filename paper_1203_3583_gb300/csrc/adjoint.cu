// Adjoint (type-2) of the forward transform, for gradients of a real loss.
//
// The forward map is u2 = D F S c with c_n = u1_n E_n (E_n = exp(i theta_n),
// the prefactor of Eq. 8), S the spread with the ES kernel at the fine-grid
// position G_n of each sample, F the 2D DFT restricted to the kept bins and D
// the diagonal deconvolution / destination chirp / global factor (Eq. 8).
// Given gu2 = dL/dRe(u2) + i dL/dIm(u2):
//   b~ = F^H D^H gu2          (two inverse-sign FFT passes, fft.cu)
//   I0 = sum_s psi(s - G) b~_s,  I_a = sum_s psi'(s_a - G_a) psi(s_b - G_b) b~_s
//   dL/du1_n = conj(E_n) I0
//   dL/dd1_n = Re[i theta'_n c_n conj(I0)] - sum_a G'_{n,a} Re[c_n conj(I_a)]
// with theta_n = k|x1|^2/(2 r0) = pi a (1 + q) (the incident wave and the
// exp(-ik d1) of Eq. 5 cancel, so their derivatives k and -k do too),
// theta' = pi a (1 + q)^2 / z0 and G'_a = s_a (1 + q)^2 / z0, since
// dq/dd1 = z0 / (z0 - d1)^2 = (1 + q)^2 / z0.  These are the exact
// derivatives of the discrete forward computation, so <A x, y> = <x, A^H y>
// holds to rounding.
#include "asfd_impl.cuh"
#include "sample.cuh"

namespace asfd {

namespace {

struct InterpArgs {
    const float2* u1;
    const float* q;
    const AxisEntry* ax;
    const AxisEntry* ay;
    const AxisPos* px;
    const AxisPos* py;
    const float2* grid;   // b~ in storage coordinates, valid over the band
    float2* gu1;          // may be NULL
    float* gd1;           // may be NULL
    int n1x, n1y;
    int nfx, nfy;
    float half_w, beta_log2e, two_over_w, beta;
    float inv_z0;
};

template <int W>
__global__ void __launch_bounds__(256) interp_grad_kernel(InterpArgs a)
{
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (size_t)a.n1x * a.n1y) return;
    const int nx = (int)(n % a.n1x), ny = (int)(n / a.n1x);
    Raw r;
    r.q = __ldg(&a.q[n]);
    r.u = a.u1 ? __ldg(&a.u1[n]) : make_float2(1.f, 0.f);
    r.ex = a.ax[nx];
    r.ey = a.ay[ny];
    r.px = a.px[nx];
    r.py = a.py[ny];
    int l0x, l0y;
    float dx, dy;
    sample_pos(r.ex, r.ey, r.px, r.py, r.q, a.half_w, l0x, l0y, dx, dy);
    float wx[W], dwx[W], wy[W], dwy[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
        es_weight_deriv_fast(dx + (float)i - a.half_w, a.two_over_w, a.beta_log2e, a.beta, wx[i], dwx[i]);
        es_weight_deriv_fast(dy + (float)i - a.half_w, a.two_over_w, a.beta_log2e, a.beta, wy[i], dwy[i]);
    }
    const int mx = a.nfx - 1, my = a.nfy - 1;
    float2 i0 = make_float2(0.f, 0.f), ix = i0, iy = i0;
#pragma unroll
    for (int b = 0; b < W; ++b) {
        const float2* row = a.grid + (size_t)((l0y + b) & my) * a.nfx;
        float2 s0 = make_float2(0.f, 0.f), sd = s0;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const float2 v = __ldg(&row[(l0x + i) & mx]);
            s0 = fma2(v, wx[i], s0);
            sd = fma2(v, dwx[i], sd);
        }
        i0 = fma2(s0, wy[b], i0);
        ix = fma2(sd, wy[b], ix);
        iy = fma2(s0, dwy[b], iy);
    }
    // E = c / u1 (unit modulus prefactor)
    Raw e1 = r;
    e1.u = make_float2(1.f, 0.f);
    const float2 E = sample_value_fast(e1);
    if (a.gu1) a.gu1[n] = make_float2(E.x * i0.x + E.y * i0.y, E.x * i0.y - E.y * i0.x);
    if (a.gd1) {
        const float2 c = make_float2(r.u.x * E.x - r.u.y * E.y, r.u.x * E.y + r.u.y * E.x);
        const float opq = 1.0f + r.q;
        const float k2 = opq * opq * a.inv_z0;
        const float dtheta = 3.14159265358979f * (r.ex.a + r.ey.a) * k2;
        const float gx = r.ex.s * k2, gy = r.ey.s * k2;
        // Re[i t c conj(I0)] = -t Im[c conj(I0)]
        const float im_c_i0 = c.y * i0.x - c.x * i0.y;
        const float re_c_ix = c.x * ix.x + c.y * ix.y;
        const float re_c_iy = c.x * iy.x + c.y * iy.y;
        a.gd1[n] = -dtheta * im_c_i0 - gx * re_c_ix - gy * re_c_iy;
    }
}

}  // namespace

asfd_status launch_interp_grad(asfd_plan_s* P, const float2* u1, float2* gu1, float* gd1,
                               cudaStream_t st)
{
    InterpArgs a;
    a.u1 = u1;
    a.q = P->q;
    a.ax = P->ax;
    a.ay = P->ay;
    a.px = P->px;
    a.py = P->py;
    a.grid = P->grid;
    a.gu1 = gu1;
    a.gd1 = gd1;
    a.n1x = P->prm.n1x;
    a.n1y = P->prm.n1y;
    a.nfx = P->nfx;
    a.nfy = P->nfy;
    a.half_w = 0.5f * (float)P->w;
    a.beta_log2e = (float)(P->beta * 1.4426950408889634074);
    a.two_over_w = (float)(2.0 / P->w);
    a.beta = (float)P->beta;
    a.inv_z0 = (float)(1.0 / P->prm.z0);
    const size_t n = (size_t)P->prm.n1x * P->prm.n1y;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    cudaError_t e = cudaSuccess;
    switch (P->w) {
#define ASFD_IW(W) case W: interp_grad_kernel<W><<<blocks, 256, 0, st>>>(a); break;
        ASFD_IW(2) ASFD_IW(3) ASFD_IW(4) ASFD_IW(5) ASFD_IW(6) ASFD_IW(7) ASFD_IW(8) ASFD_IW(9)
        ASFD_IW(10) ASFD_IW(11) ASFD_IW(12) ASFD_IW(13) ASFD_IW(14) ASFD_IW(15) ASFD_IW(16)
#undef ASFD_IW
        default: return fail(ASFD_ERR_UNSUPPORTED, "kernel width outside 2..16");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "interp_grad_kernel launch");
    return ASFD_OK;
}

}  // namespace asfd
