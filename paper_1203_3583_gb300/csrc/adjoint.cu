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
// with theta_n = k|x1|^2/(2 r0) + k d1 (sz - 1) = pi a (1 + q) + pi inc_d q/(1 + q)
// (at normal incidence the incident wave and the exp(-ik d1) of Eq. 5
// cancel; a tilted plane wave leaves its depth term, whose derivative is
// k (sz - 1) = pi inc_d / z0), theta' = pi a (1 + q)^2 / z0 + pi inc_d / z0 and
// G'_a = s_a (1 + q)^2 / z0, since
// dq/dd1 = z0 / (z0 - d1)^2 = (1 + q)^2 / z0.  These are the exact
// derivatives of the discrete forward computation, so <A x, y> = <x, A^H y>
// holds to rounding.
#include <algorithm>

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
    float inc_d;          // incident depth phase, half-turns per unit d1/z0
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
    const float2 E = sample_value_fast(e1, a.inc_d);
    if (a.gu1) a.gu1[n] = make_float2(E.x * i0.x + E.y * i0.y, E.x * i0.y - E.y * i0.x);
    if (a.gd1) {
        const float2 c = make_float2(r.u.x * E.x - r.u.y * E.y, r.u.x * E.y + r.u.y * E.x);
        const float opq = 1.0f + r.q;
        const float k2 = opq * opq * a.inv_z0;
        const float dtheta = 3.14159265358979f * ((r.ex.a + r.ey.a) * k2 + a.inc_d * a.inv_z0);
        const float gx = r.ex.s * k2, gy = r.ey.s * k2;
        // Re[i t c conj(I0)] = -t Im[c conj(I0)]
        const float im_c_i0 = c.y * i0.x - c.x * i0.y;
        const float re_c_ix = c.x * ix.x + c.y * ix.y;
        const float re_c_iy = c.x * iy.x + c.y * iy.y;
        a.gd1[n] = -dtheta * im_c_i0 - gx * re_c_ix - gy * re_c_iy;
    }
}

// psi and d psi / dz of the ES kernel for two taps at once (packed FP32x2; the
// MUFU square root and exponential), 1 - u^2 floored at 1e-12 as in
// es_weight_deriv_fast.  neg_c2 = -(2/w)^2; d psi/dz = psi z rsqrt(r) beta neg_c2.
__device__ __forceinline__ void es_weight_deriv2_fast(float2 z, float neg_c2, float beta_log2e,
                                                      float beta_negc2, float2& psi, float2& dpsi)
{
    const float2 t = mul2(z, neg_c2);
    float2 r = fma2v(t, z, make_float2(1.f, 1.f));
    r.x = fmaxf(r.x, 1e-12f);
    r.y = fmaxf(r.y, 1e-12f);
    float2 rs, e;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs.x) : "f"(r.x));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs.y) : "f"(r.y));
    const float2 s = fma2v(r, rs, make_float2(-1.f, -1.f));
    const float2 arg = mul2(s, beta_log2e);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(arg.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(arg.y));
    psi = e;
    const float2 zr = make_float2(z.x * rs.x, z.y * rs.y);
    dpsi = mul2(make_float2(e.x * zr.x, e.y * zr.y), beta_negc2);
}

// Interpolation with a register window (widths up to 7): warp item `it` takes
// 32 consecutive source columns (one per lane) over `rows` consecutive rows.
// Consecutive samples of a column read nearly the same W x W cells of b~, so
// each lane keeps them in registers and, when the first tap row moves down by
// d < W rows, moves the window up and reads only the d new rows; a changed
// first tap column or a larger jump reloads the window.  Sums, outputs and
// arithmetic per sample are those of interp_grad_kernel.
template <int W>
__global__ void __launch_bounds__(128) interp_window_kernel(InterpArgs a, int rows, int items)
{
    const int it = blockIdx.x * 4 + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (it >= items) return;
    const int ncb = (a.n1x + 31) / 32;
    const int nx = (it % ncb) * 32 + lane;
    const int ny0 = (it / ncb) * rows;
    const int nyl = min(ny0 + rows, a.n1y) - 1;
    if (nx >= a.n1x || ny0 > nyl) return;
    const int mx = a.nfx - 1, my = a.nfy - 1;
    const float neg_c2 = -a.two_over_w * a.two_over_w;
    const float beta_negc2 = a.beta * neg_c2;
    const AxisEntry ex = a.ax[nx];
    const AxisPos px = a.px[nx];

    float2 v[W][W];
    int X0 = 0, R0 = 0;
    bool live = false;
    auto load_row = [&](int b, int row) {
        const float2* g = a.grid + (size_t)(row & my) * a.nfx;
#pragma unroll
        for (int i = 0; i < W; ++i) v[b][i] = __ldg(&g[(X0 + i) & mx]);
    };
    size_t n = (size_t)ny0 * a.n1x + nx;
    float qn = __ldg(&a.q[n]);
    float2 un = a.u1 ? __ldg(&a.u1[n]) : make_float2(1.f, 0.f);
    for (int ny = ny0; ny <= nyl; ++ny, n += a.n1x) {
        const float q = qn;
        const float2 u = un;
        if (ny < nyl) {
            qn = __ldg(&a.q[n + a.n1x]);
            if (a.u1) un = __ldg(&a.u1[n + a.n1x]);
        }
        const AxisEntry ey = a.ay[ny];
        int l0x, l0y;
        float dx, dy;
        sample_pos(ex, ey, px, a.py[ny], q, a.half_w, l0x, l0y, dx, dy);
        const int d = l0y - R0;
        if (!live || l0x != X0 || d < 0 || d >= W) {
            X0 = l0x;
            R0 = l0y;
#pragma unroll
            for (int b = 0; b < W; ++b) load_row(b, R0 + b);
            live = true;
        } else if (d == 2) {  // slide down two rows in one move (alpha > 1 takes
                              // 1- and 2-row slides; two 1-row moves copy 12 rows)
#pragma unroll
            for (int b = 0; b + 2 < W; ++b)
#pragma unroll
                for (int i = 0; i < W; ++i) v[b][i] = v[b + 2][i];
            load_row(W - 2, R0 + W);
            load_row(W - 1, R0 + W + 1);
            R0 = l0y;
        } else {
            for (int k = 0; k < d; ++k) {  // slide down one row
#pragma unroll
                for (int b = 0; b + 1 < W; ++b)
#pragma unroll
                    for (int i = 0; i < W; ++i) v[b][i] = v[b + 1][i];
                load_row(W - 1, R0 + W + k);
            }
            R0 = l0y;
        }
        float wx[W], dwx[W], wy[W], dwy[W];
#pragma unroll
        for (int i = 0; i < W; ++i) {
            float2 psi, dpsi;
            es_weight_deriv2_fast(make_float2(dx + (float)i - a.half_w, dy + (float)i - a.half_w),
                                  neg_c2, a.beta_log2e, beta_negc2, psi, dpsi);
            wx[i] = psi.x;
            dwx[i] = dpsi.x;
            wy[i] = psi.y;
            dwy[i] = dpsi.y;
        }
        float2 i0 = make_float2(0.f, 0.f), ixs = i0, iys = i0;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            float2 s0 = make_float2(0.f, 0.f), sd = s0;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                s0 = fma2(v[b][i], wx[i], s0);
                sd = fma2(v[b][i], dwx[i], sd);
            }
            i0 = fma2(s0, wy[b], i0);
            ixs = fma2(sd, wy[b], ixs);
            iys = fma2(s0, dwy[b], iys);
        }
        // E = c / u1 (unit modulus prefactor)
        const float2 E = sample_value_fast(make_float2(1.f, 0.f), ex, ey, q, a.inc_d);
        if (a.gu1) a.gu1[n] = make_float2(E.x * i0.x + E.y * i0.y, E.x * i0.y - E.y * i0.x);
        if (a.gd1) {
            const float2 c = make_float2(u.x * E.x - u.y * E.y, u.x * E.y + u.y * E.x);
            const float opq = 1.0f + q;
            const float k2 = opq * opq * a.inv_z0;
            const float dtheta = 3.14159265358979f * ((ex.a + ey.a) * k2 + a.inc_d * a.inv_z0);
            const float gx = ex.s * k2, gy = ey.s * k2;
            const float im_c_i0 = c.y * i0.x - c.x * i0.y;
            const float re_c_ix = c.x * ixs.x + c.y * ixs.y;
            const float re_c_iy = c.x * iys.x + c.y * iys.y;
            a.gd1[n] = -dtheta * im_c_i0 - gx * re_c_ix - gy * re_c_iy;
        }
    }
}

}  // namespace

asfd_status interp_window_warp_slots(int w, long long* slots)
{
    int dev = 0, sms = 0, per_sm = 0;
    ASFD_CUDA(cudaGetDevice(&dev));
    ASFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const void* k = nullptr;
    switch (w) {
#define ASFD_IWK(W) case W: k = (const void*)interp_window_kernel<W>; break;
        ASFD_IWK(2) ASFD_IWK(3) ASFD_IWK(4) ASFD_IWK(5) ASFD_IWK(6) ASFD_IWK(7)
#undef ASFD_IWK
        default: return fail(ASFD_ERR_UNSUPPORTED, "windowed interpolation widths are 2..7");
    }
    ASFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, 0));
    *slots = (long long)sms * std::max(per_sm, 1) * 4;
    return ASFD_OK;
}

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
    a.inc_d = (float)P->inc_d;
    const size_t n = (size_t)P->prm.n1x * P->prm.n1y;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    cudaError_t e = cudaSuccess;
    if (P->w <= kMaxWindowWidth) {
        // warp items of 32 columns x `rows` rows, in whole waves of the resident warps
        const long long ncb = (P->prm.n1x + 31) / 32;
        long long slots = 0;
        const asfd_status s = interp_window_warp_slots(P->w, &slots);
        if (s != ASFD_OK) return s;
        const int rows = window_run_rows(P->prm.n1y, ncb, slots);
        const int items = (int)(ncb * ((P->prm.n1y + rows - 1) / rows));
        switch (P->w) {
#define ASFD_IWW(W) case W: interp_window_kernel<W><<<(items + 3) / 4, 128, 0, st>>>(a, rows, items); break;
            ASFD_IWW(2) ASFD_IWW(3) ASFD_IWW(4) ASFD_IWW(5) ASFD_IWW(6) ASFD_IWW(7)
#undef ASFD_IWW
            default: break;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "interp_window_kernel launch");
        return ASFD_OK;
    }
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
