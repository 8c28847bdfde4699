// Shared-memory Stockham FFT for power-of-two lengths 16..16384 (sm_103a).
//
// NUFFTs combine an interpolation with a uniform FFT (Sec. 2, after Eq. 9);
// this is the uniform FFT.  Each line of length L is processed by L/16
// threads holding 16 complex values in registers.  Passes are radix 16
// (one leading radix-2/4/8 pass when log2 L is not a multiple of 4), in the
// self-sorting Stockham order: pass p with accumulated stride NS reads
// x[j + r L/R], multiplies by W_{NS R}^{r (j mod NS)}, takes an R-point DFT in
// registers and writes X_r to (j/NS) NS R + (j mod NS) + r NS.  The first pass
// reads through a caller loader (global memory, zero fill, gathers) and the
// last pass writes through a caller storer (crop, deconvolution, scatter), so
// a line makes exactly one trip through global memory.  Shared memory is
// padded by one complex per 16 to keep the strided pass writes bank-conflict
// free.  Twiddles come from a table e^{-2 pi i k/L} built in FP64 (radix-16
// passes load four entries per butterfly and form the other eleven by
// products).
#pragma once

#include <cuda_runtime.h>

namespace asfd {

__host__ __device__ constexpr int ilog2_c(int n) { return n <= 1 ? 0 : 1 + ilog2_c(n >> 1); }

// cos and sin of 2 pi j / 16 from the closed forms cos(pi/8) = sqrt(2+sqrt2)/2,
// sin(pi/8) = sqrt(2-sqrt2)/2, cos(pi/4) = sqrt2/2.
__device__ __forceinline__ constexpr float cos16(int j)
{
    constexpr float C1 = 0.923879532511286756f, S1 = 0.382683432365089772f,
                    R2 = 0.707106781186547524f;
    constexpr float t[16] = {1.f, C1, R2, S1, 0.f, -S1, -R2, -C1, -1.f, -C1, -R2, -S1, 0.f, S1, R2, C1};
    return t[j & 15];
}
__device__ __forceinline__ constexpr float sin16(int j) { return cos16(j - 4); }

// Complex arithmetic on packed FP32x2 registers (add/sub/mul/fma .f32x2):
// one instruction per complex add, two per complex multiply, with the same
// IEEE rounding per component as the scalar forms.
__device__ __forceinline__ unsigned long long f2_bits(float2 v)
{
    return *reinterpret_cast<const unsigned long long*>(&v);
}
__device__ __forceinline__ float2 f2_from(unsigned long long r)
{
    return *reinterpret_cast<const float2*>(&r);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(r);
}
__device__ __forceinline__ float2 mul_f2(float2 a, float2 b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(r);
}
__device__ __forceinline__ float2 fma_f2(float2 a, float2 b, float2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)),
        "l"(f2_bits(c)));
    return f2_from(r);
}
// a * b = (a.x b.x - a.y b.y, a.x b.y + a.y b.x): the products a.y b are
// rounded first, then fused into a.x b (as fmaf(a.x, b.x, -(a.y b.y))).
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    const float2 p = mul_f2(make_float2(a.y, a.y), make_float2(b.y, b.x));
    return fma_f2(make_float2(a.x, a.x), b, make_float2(-p.x, p.y));
}
// a * conj(b) = (a.x b.x + a.y b.y, a.y b.x - a.x b.y)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    const float2 p = mul_f2(make_float2(a.y, a.x), make_float2(b.y, b.y));
    return fma_f2(make_float2(a.x, a.y), make_float2(b.x, b.x), make_float2(p.x, -p.y));
}

// d * exp(S * 2 pi i j / 16) with j known at compile time after unrolling.
template <int S>
__device__ __forceinline__ float2 rot16(float2 d, int j)
{
    if (j == 0) return d;
    if (j == 4) return S < 0 ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
    const float c = cos16(j), s = S < 0 ? -sin16(j) : sin16(j);
    // (d.x c - d.y s, d.x s + d.y c)
    const float2 p = mul_f2(make_float2(d.y, d.y), make_float2(s, c));
    return fma_f2(make_float2(d.x, d.x), make_float2(c, s), make_float2(-p.x, p.y));
}

template <int R>
__device__ __forceinline__ constexpr int bitrev_c(int i)
{
    int r = 0;
    for (int b = 1; b < R; b <<= 1) r = (r << 1) | ((i & b) ? 1 : 0);
    return r;
}

// In-register R-point DFT (R = 2, 4, 8, 16), sign S: X_k = sum_r v_r e^{S 2 pi i r k/R}.
// Radix-2 decimation in frequency followed by a compile-time bit reversal.
template <int R, int S>
__device__ __forceinline__ void dft_reg(float2* v)
{
#pragma unroll
    for (int len = R; len >= 2; len >>= 1) {
        const int half = len >> 1;
#pragma unroll
        for (int start = 0; start < R; start += len) {
#pragma unroll
            for (int k = 0; k < half; ++k) {
                const float2 a = v[start + k], b = v[start + k + half];
                v[start + k] = cadd(a, b);
                v[start + k + half] = rot16<S>(csub(a, b), k * (16 / len));
            }
        }
    }
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = v[i];
#pragma unroll
    for (int i = 0; i < R; ++i) v[bitrev_c<R>(i)] = t[i];
}

__device__ __forceinline__ int fft_pad(int i) { return i + (i >> 4); }

template <int L>
struct FftShape {
    static constexpr int E = 16;                        // complex values per thread
    static constexpr int TPL = L / 16;                  // threads per line
    static constexpr int LOG = ilog2_c(L);
    static constexpr int NP = (LOG + 3) / 4;            // passes
    static constexpr int R0 = (LOG % 4 == 0) ? 16 : (1 << (LOG % 4));  // first pass radix
    static constexpr int SMEM = L + L / 16;             // padded complex slots per line
    static_assert(L >= 16 && L <= 16384 && (L & (L - 1)) == 0, "FFT length");
};

// One Stockham pass on the registers v (E/R butterflies of this thread).
template <int L, int R, int NS, int S>
__device__ __forceinline__ void fft_pass_compute(float2 (&v)[16], int t, const float2* __restrict__ tw)
{
    constexpr int TPL = L / 16;
#pragma unroll
    for (int b = 0; b < 16 / R; ++b) {
        const int j = t + b * TPL;
        if (NS > 1) {
            const int k = j % NS;
            constexpr int STEP = L / (NS * R);
            if constexpr (R == 16) {
                // W^(rk) for r = 1..15 from one table entry (r = 1): W^2k, W^4k
                // and W^8k by squaring, the other eleven by products.  The
                // lanes of a warp read one entry each at stride k STEP, which
                // in the middle passes touches a cache line per lane; one such
                // load instead of four takes three quarters of those L1
                // wavefronts away (rows pass 30.7 -> 24.6 us at 2048^2), and
                // the products add a few roundings per twiddle (FFT error
                // 1.4e-7 -> 3.0e-7 relative at length 4096)
                float2 w[16];
                w[1] = __ldg(&tw[k * STEP]);
                w[2] = cmul(w[1], w[1]);
                w[4] = cmul(w[2], w[2]);
                w[8] = cmul(w[4], w[4]);
                w[3] = cmul(w[1], w[2]);
                w[5] = cmul(w[4], w[1]);
                w[6] = cmul(w[4], w[2]);
                w[7] = cmul(w[4], w[3]);
#pragma unroll
                for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
#pragma unroll
                for (int r = 1; r < 16; ++r)
                    v[b * R + r] = S < 0 ? cmul(v[b * R + r], w[r]) : cmulc(v[b * R + r], w[r]);
            } else {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float2 w = __ldg(&tw[r * k * STEP]);
                    v[b * R + r] = S < 0 ? cmul(v[b * R + r], w) : cmulc(v[b * R + r], w);
                }
            }
        }
        dft_reg<R, S>(&v[b * R]);
    }
}

template <int L, int R>
__device__ __forceinline__ void fft_load_smem(float2 (&v)[16], int t, const float2* s)
{
    constexpr int TPL = L / 16;
#pragma unroll
    for (int b = 0; b < 16 / R; ++b) {
        const int j = t + b * TPL;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = s[fft_pad(j + r * (L / R))];
    }
}

template <int L, int R, int NS>
__device__ __forceinline__ void fft_store_smem(const float2 (&v)[16], int t, float2* s)
{
    constexpr int TPL = L / 16;
#pragma unroll
    for (int b = 0; b < 16 / R; ++b) {
        const int j = t + b * TPL;
        const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
        for (int r = 0; r < R; ++r) s[fft_pad(base + r * NS)] = v[b * R + r];
    }
}

// Passes 1..NP-1 (radix 16) after the first; recursion over the pass index.
template <int L, int P, int NS, int S, class Store>
__device__ __forceinline__ void fft_tail(float2 (&v)[16], int t, float2* s, const float2* tw,
                                         Store& st)
{
    constexpr int NP = FftShape<L>::NP;
    constexpr int TPL = L / 16;
    if constexpr (P < NP) {
        fft_load_smem<L, 16>(v, t, s);
        __syncthreads();
        fft_pass_compute<L, 16, NS, S>(v, t, tw);
        if constexpr (P == NP - 1) {
            // last pass: NS * 16 == L and j = t < NS, so X_r goes to t + r L/16
#pragma unroll
            for (int r = 0; r < 16; ++r) st(t + r * TPL, v[r]);
        } else {
            fft_store_smem<L, 16, NS>(v, t, s);
            __syncthreads();
            fft_tail<L, P + 1, NS * 16, S, Store>(v, t, s, tw, st);
        }
    }
}

// Transform one line.  Every thread of the block must call this (it contains
// __syncthreads); t is the thread's index within its line (0..L/16-1), s the
// line's shared-memory slots (FftShape<L>::SMEM complex), ld(i) returns input
// element i, st(i, x) receives output element i.  Every shared-memory read of
// the last pass precedes a block barrier, so the slots may be rewritten as soon
// as this returns.
template <int L, int S, class Load, class Store>
__device__ __forceinline__ void fft_line(int t, float2* s, const float2* __restrict__ tw, Load& ld,
                                         Store& st)
{
    constexpr int R0 = FftShape<L>::R0;
    constexpr int NP = FftShape<L>::NP;
    constexpr int TPL = L / 16;
    float2 v[16];
#pragma unroll
    for (int b = 0; b < 16 / R0; ++b) {
        const int j = t + b * TPL;
#pragma unroll
        for (int r = 0; r < R0; ++r) v[b * R0 + r] = ld(j + r * (L / R0));
    }
    fft_pass_compute<L, R0, 1, S>(v, t, tw);
    if constexpr (NP == 1) {
        // single radix-16 pass (L == 16): output index r
#pragma unroll
        for (int r = 0; r < 16; ++r) st(r, v[r]);
    } else {
        fft_store_smem<L, R0, 1>(v, t, s);
        __syncthreads();
        fft_tail<L, 1, R0, S, Store>(v, t, s, tw, st);
    }
}

}  // namespace asfd
