// Per-sample arithmetic shared by the spreading (forward) and interpolation
// (adjoint) kernels: the sample's position on the fine grid, its prefactor
// and the exponential-of-semicircle kernel weights.  See spread.cu for the
// phase and position split between the FP64 plan tables and the FP32
// per-sample corrections.
#pragma once

#include "asfd_impl.cuh"

namespace asfd {

// ES kernel psi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)), |z| <= w/2.
__device__ __forceinline__ float es_weight(float z, float two_over_w, float beta_log2e)
{
    const float u = z * two_over_w;
    const float r = fmaxf(1.0f - u * u, 0.0f);
    const float s = r > 0.0f ? r * rsqrtf(r) : 0.0f;
    return exp2f(beta_log2e * (s - 1.0f));
}

// First tap (storage coordinates, not wrapped) and fractional offset of a sample.
__device__ __forceinline__ void sample_pos(const AxisEntry& ex, const AxisEntry& ey,
                                           const AxisPos& px, const AxisPos& py, float q,
                                           float half_w, int& l0x, int& l0y, float& dx, float& dy)
{
    const float fx = px.bf + ex.s * q - half_w;
    const float fy = py.bf + ey.s * q - half_w;
    const float cfx = ceilf(fx), cfy = ceilf(fy);
    l0x = px.bi + (int)cfx;
    l0y = py.bi + (int)cfy;
    dx = cfx - fx;  // in [0, 1): tap i sits at dx + i - w/2 from the sample
    dy = cfy - fy;
}

// Per-sample correction phase in half-turns: the r0 part of the source chirp,
// (a_x + a_y) q, plus the incident wave's depth term inc_d q/(1 + q) (zero at
// normal incidence).
__device__ __forceinline__ float sample_phase(const AxisEntry& ex, const AxisEntry& ey, float q,
                                              float inc_d)
{
    return fmaf(inc_d, __fdividef(q, 1.0f + q), (ex.a + ey.a) * q);
}

// c = u1 E_x E_y exp(i pi (a_x + a_y) q + i pi inc_d q/(1 + q))
__device__ __forceinline__ float2 sample_value(float2 u, const AxisEntry& ex, const AxisEntry& ey,
                                               float q, float inc_d)
{
    float sn, cs;
    sincospif(sample_phase(ex, ey, q, inc_d), &sn, &cs);
    const float2 exy = make_float2(ex.e.x * ey.e.x - ex.e.y * ey.e.y,
                                   ex.e.x * ey.e.y + ex.e.y * ey.e.x);
    const float2 t1 = make_float2(u.x * exy.x - u.y * exy.y, u.x * exy.y + u.y * exy.x);
    return make_float2(t1.x * cs - t1.y * sn, t1.x * sn + t1.y * cs);
}

// acc + v * w on a complex pair (packed FP32x2 FMA)
__device__ __forceinline__ float2 fma2(float2 v, float w, float2 acc)
{
    unsigned long long r;
    const unsigned long long vv = *reinterpret_cast<const unsigned long long*>(&v);
    const unsigned long long aa = *reinterpret_cast<const unsigned long long*>(&acc);
    const float2 ww = make_float2(w, w);
    const unsigned long long wb = *reinterpret_cast<const unsigned long long*>(&ww);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(vv), "l"(wb), "l"(aa));
    return *reinterpret_cast<float2*>(&r);
}

// v * w and a * b + c on complex pairs / FP32 pairs (packed FP32x2)
__device__ __forceinline__ float2 mul2(float2 v, float w)
{
    unsigned long long r;
    const unsigned long long vv = *reinterpret_cast<const unsigned long long*>(&v);
    const float2 ww = make_float2(w, w);
    const unsigned long long wb = *reinterpret_cast<const unsigned long long*>(&ww);
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(vv), "l"(wb));
    return *reinterpret_cast<float2*>(&r);
}

__device__ __forceinline__ float2 fma2v(float2 a, float2 b, float2 c)
{
    unsigned long long r;
    const unsigned long long aa = *reinterpret_cast<const unsigned long long*>(&a);
    const unsigned long long bb = *reinterpret_cast<const unsigned long long*>(&b);
    const unsigned long long cc = *reinterpret_cast<const unsigned long long*>(&c);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(aa), "l"(bb), "l"(cc));
    return *reinterpret_cast<float2*>(&r);
}

// Per-sample inputs, loaded one sample ahead of use.
struct Raw {
    float q;
    float2 u;
    AxisEntry ex, ey;
    AxisPos px, py;
};

template <class Args>
__device__ __forceinline__ Raw load_raw(const Args& a, int nx, int ny)
{
    Raw r;
    const size_t n = (size_t)ny * a.n1x + nx;
    r.q = __ldg(&a.q[n]);
    r.u = __ldg(&a.u1[n]);
    r.ex = a.ax[nx];
    r.ey = a.ay[ny];
    r.px = a.px[nx];
    r.py = a.py[ny];
    return r;
}

// ES weight with the approximate MUFU square root and exponential (relative
// error ~2^-22, far below the kernel's own truncation error).
__device__ __forceinline__ float es_weight_fast(float z, float two_over_w, float beta_log2e)
{
    const float u = z * two_over_w;
    const float r = fmaxf(fmaf(-u, u, 1.0f), 1e-30f);
    float rs, e;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(r));
    const float arg = beta_log2e * fmaf(r, rs, -1.0f);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(arg));
    return e;
}

// c = u1 E_x E_y exp(i pi sample_phase); the correction phase is reduced
// modulo 2 half-turns exactly in FP32, then evaluated with the MUFU sine and
// cosine (absolute error ~4e-7 on [-pi, pi]).
__device__ __forceinline__ float2 sample_value_fast(float2 u, const AxisEntry& ex,
                                                    const AxisEntry& ey, float q, float inc_d)
{
    const float ph = sample_phase(ex, ey, q, inc_d);
    const float red = ph - 2.0f * rintf(0.5f * ph);
    float sn, cs;
    __sincosf(3.14159265358979f * red, &sn, &cs);
    const float2 exy = make_float2(ex.e.x * ey.e.x - ex.e.y * ey.e.y,
                                   ex.e.x * ey.e.y + ex.e.y * ey.e.x);
    const float2 t1 = make_float2(u.x * exy.x - u.y * exy.y, u.x * exy.y + u.y * exy.x);
    return make_float2(t1.x * cs - t1.y * sn, t1.x * sn + t1.y * cs);
}

__device__ __forceinline__ float2 sample_value_fast(const Raw& r, float inc_d)
{
    return sample_value_fast(r.u, r.ex, r.ey, r.q, inc_d);
}

}  // namespace asfd

namespace asfd {

// psi(z) and d psi / dz of the ES kernel at z (fast MUFU forms).  The
// derivative -psi beta (2/w) u / sqrt(1 - u^2) is infinite at the support
// edge, where psi itself is e^-beta; 1 - u^2 is floored at 1e-12 so that the
// edge tap (weight ~e^-beta) stays finite.
__device__ __forceinline__ void es_weight_deriv_fast(float z, float two_over_w, float beta_log2e,
                                                     float beta, float& psi, float& dpsi)
{
    const float u = z * two_over_w;
    const float r = fmaxf(fmaf(-u, u, 1.0f), 1e-12f);
    float rs, e;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(r));
    const float arg = beta_log2e * fmaf(r, rs, -1.0f);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(arg));
    psi = e;
    dpsi = -e * beta * two_over_w * u * rs;
}

}  // namespace asfd

namespace asfd {

// Learned kernel weights: tap a of axis x is sum_k c[0][a][k] t^k with
// t = 2 dx - 1 (monomials on [-1, 1], Horner), likewise y with dy.
template <int W>
__device__ __forceinline__ void table_weights(const float* tab, float dx, float dy, float (&wx)[W],
                                              float (&wy)[W])
{
    static_assert(kLearnCoef == 8, "two float4 per polynomial");
    const float4* t4 = reinterpret_cast<const float4*>(tab);
    const float tx = fmaf(2.0f, dx, -1.0f), ty = fmaf(2.0f, dy, -1.0f);
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const float4 lo = __ldg(&t4[2 * i]), hi = __ldg(&t4[2 * i + 1]);
        float p = hi.w;
        p = fmaf(p, tx, hi.z);
        p = fmaf(p, tx, hi.y);
        p = fmaf(p, tx, hi.x);
        p = fmaf(p, tx, lo.w);
        p = fmaf(p, tx, lo.z);
        p = fmaf(p, tx, lo.y);
        wx[i] = fmaf(p, tx, lo.x);
        const float4 lo2 = __ldg(&t4[2 * (W + i)]), hi2 = __ldg(&t4[2 * (W + i) + 1]);
        float q = hi2.w;
        q = fmaf(q, ty, hi2.z);
        q = fmaf(q, ty, hi2.y);
        q = fmaf(q, ty, hi2.x);
        q = fmaf(q, ty, lo2.w);
        q = fmaf(q, ty, lo2.z);
        q = fmaf(q, ty, lo2.y);
        wy[i] = fmaf(q, ty, lo2.x);
    }
}

}  // namespace asfd
