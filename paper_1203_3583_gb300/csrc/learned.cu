// Learned spreading kernel: a per-source-tile tabulated kernel predicted by a
// small MLP from tile features, with a learned correction of the
// deconvolution, trained on the GPU against a reference field.
//
// Kernel.  Width kLearnW (= 4, against 7 for the ES kernel at the same
// target accuracy).  Tap a of axis x of a sample in source tile t has weight
//   P_{t,x,a}(2 dx - 1) = sum_k table[t][x][a][k] (2 dx - 1)^k,  k <= 7,
// where dx in [0, 1) is the sample's offset from its first tap, likewise y.
// table[t] = base + s * MLP(features[t]); base is a shared trainable table
// (initialised by a least-squares fit of the ES kernel of width 4), the MLP
// has one tanh hidden layer, and s = kLearnOutScale.  The deconvolution is
// the ES width-4 one times 1 + sum_j d_j T_{2j}(2 m'/M) per axis (even
// Chebyshev polynomials of the centred destination index), d trainable.
//
// Features of a source tile (dimensionless, so that a model transfers across
// grid sizes): 1, its mean fine-grid position in x and y relative to the grid
// centre (units of nf/2), its mean sample spacing on the fine grid minus one
// in x and y, and 100 x its mean q = d1/(z0 - d1).
//
// Training step (asfd_learned_train_step): loss L = |u2 - ref|^2 / |ref|^2.
//   forward with the current tables -> u2;  g = dL/du2 = 2 (u2 - ref)/|ref|^2
//   dL/dcorr_x[mx] = Re sum_my conj(g) u2 / corr_x[mx]  (likewise y) -> dL/dd
//   b~ = F^H D^H g (the adjoint FFT passes);  for every tap of every sample
//   v = Re[conj(b~_cell) c_n] and dL/dtable[t][x][a][k] += v P_{t,y,b} t_x^k
//   (likewise y); MLP backward over tiles; Adam update; tables refreshed.
// All of it runs in the kernels of this file and the FFT passes; the host only
// sequences launches and reads back the loss.
#include <cmath>
#include <cstring>
#include <vector>

#include "asfd_impl.cuh"
#include "sample.cuh"

namespace asfd {

namespace {

// ---- features (plan time) ---------------------------------------------------

__global__ void __launch_bounds__(256) features_kernel(const float* q, const AxisEntry* ax,
                                                       const AxisEntry* ay, const double* bux,
                                                       const double* buy, int n1x, int n1y,
                                                       int nstx, int nfx, int nfy, float* feat)
{
    const int t = blockIdx.x;
    const int nx = (t % nstx) * kSrcTile + threadIdx.x % kSrcTile;
    const int ny = (t / nstx) * kSrcTile + threadIdx.x / kSrcTile;
    float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // gx, gy, spacing x, spacing y, q
    float cnt[3] = {0.f, 0.f, 0.f};
    if (nx < n1x && ny < n1y) {
        const size_t n = (size_t)ny * n1x + nx;
        const float qq = q[n];
        const double gx = bux[nx] + (double)(ax[nx].s * qq);
        const double gy = buy[ny] + (double)(ay[ny].s * qq);
        v[0] = (float)((gx - 0.5 * nfx) / (0.5 * nfx));
        v[1] = (float)((gy - 0.5 * nfy) / (0.5 * nfy));
        v[4] = qq;
        cnt[0] = 1.f;
        if (nx + 1 < n1x) {
            v[2] = (float)(bux[nx + 1] + (double)(ax[nx + 1].s * q[n + 1]) - gx);
            cnt[1] = 1.f;
        }
        if (ny + 1 < n1y) {
            v[3] = (float)(buy[ny + 1] + (double)(ay[ny + 1].s * q[n + n1x]) - gy);
            cnt[2] = 1.f;
        }
    }
    __shared__ float red[8][8];
    float acc[8] = {v[0], v[1], v[2], v[3], v[4], cnt[0], cnt[1], cnt[2]};
#pragma unroll
    for (int i = 0; i < 8; ++i)
        for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    if ((threadIdx.x & 31) == 0)
        for (int i = 0; i < 8; ++i) red[threadIdx.x / 32][i] = acc[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < 8; ++w)
            for (int i = 0; i < 8; ++i) s[i] += red[w][i];
        const float c0 = fmaxf(s[5], 1.f), c1 = fmaxf(s[6], 1.f), c2 = fmaxf(s[7], 1.f);
        float* f = feat + (size_t)t * kLearnFeat;
        f[0] = 1.f;
        f[1] = s[0] / c0;
        f[2] = s[1] / c0;
        f[3] = (s[6] > 0.f ? s[2] / c1 : 1.f) - 1.f;
        f[4] = (s[7] > 0.f ? s[3] / c2 : 1.f) - 1.f;
        f[5] = 100.f * s[4] / c0;
    }
}

// ---- MLP forward: features -> hidden -> table --------------------------------

__global__ void __launch_bounds__(kLearnTableSize) mlp_forward_kernel(const float* __restrict__ prm,
                                                                      const float* __restrict__ feat,
                                                                      float* __restrict__ hid,
                                                                      float* __restrict__ tab)
{
    const int t = blockIdx.x, o = threadIdx.x;
    __shared__ float f[kLearnFeat], h[kLearnHidden];
    if (o < kLearnFeat) f[o] = feat[(size_t)t * kLearnFeat + o];
    __syncthreads();
    if (o < kLearnHidden) {
        float s = prm[kLpB1 + o];
        for (int i = 0; i < kLearnFeat; ++i) s = fmaf(prm[kLpW1 + o * kLearnFeat + i], f[i], s);
        const float hv = tanhf(s);
        h[o] = hv;
        hid[(size_t)t * kLearnHidden + o] = hv;
    }
    __syncthreads();
    float s = prm[kLpB2 + o];
    for (int i = 0; i < kLearnHidden; ++i) s = fmaf(prm[kLpW2 + o * kLearnHidden + i], h[i], s);
    tab[(size_t)t * kLearnTableSize + o] = prm[kLpBase + o] + kLearnOutScale * s;
}

// ---- deconvolution correction ----------------------------------------------

// T_{2j}(u) for j = 1..kLearnCheb
__device__ __forceinline__ void cheb_even(float u, float (&T)[kLearnCheb])
{
    float t0 = 1.f, t1 = u;
    for (int n = 2, j = 0; j < kLearnCheb; ++n) {
        const float t2 = 2.f * u * t1 - t0;
        t0 = t1;
        t1 = t2;
        if ((n & 1) == 0) T[j++] = t2;
    }
}

__global__ void deconv_build_kernel(const float* __restrict__ prm, const float2* __restrict__ cb,
                                    float2* __restrict__ c, float* __restrict__ corr, int m, int off)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const float u = 2.f * (float)(k - m / 2) / (float)m;
    float T[kLearnCheb];
    cheb_even(u, T);
    float s = 1.f;
    for (int j = 0; j < kLearnCheb; ++j) s = fmaf(prm[off + j], T[j], s);
    corr[k] = s;
    c[k] = make_float2(cb[k].x * s, cb[k].y * s);
}

// ---- loss --------------------------------------------------------------------

__global__ void loss_reduce_kernel(const float2* __restrict__ u2, const float2* __restrict__ ref,
                                   size_t n, double* red)
{
    double e = 0.0, r = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float2 a = u2[i], b = ref[i];
        const double dx = (double)a.x - b.x, dy = (double)a.y - b.y;
        e += dx * dx + dy * dy;
        r += (double)b.x * b.x + (double)b.y * b.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&red[0], e);
        atomicAdd(&red[1], r);
    }
}

__global__ void residual_kernel(const float2* __restrict__ u2, const float2* __restrict__ ref,
                                size_t n, const double* red, float2* __restrict__ g)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float sc = (float)(2.0 / fmax(red[1], 1e-300));
    const float2 a = u2[i], b = ref[i];
    g[i] = make_float2(sc * (a.x - b.x), sc * (a.y - b.y));
}

// dL/dcorr_x[mx] = Re sum_my conj(g) u2 / corr_x[mx]: blocks of 32 columns x
// 8 thread rows over a slab of destination rows; the slab's column sums are
// added atomically to out (zeroed by the caller)
constexpr int kDeconvSlabs = 64;

__global__ void __launch_bounds__(256) deconv_grad_x_kernel(const float2* __restrict__ g,
                                                            const float2* __restrict__ u2,
                                                            const float* __restrict__ corr,
                                                            int m2x, int m2y, float* __restrict__ out)
{
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int mx = blockIdx.x * 32 + tx;
    const int slab = (m2y + gridDim.y - 1) / gridDim.y;
    const int y0 = blockIdx.y * slab, y1 = min(m2y, y0 + slab);
    float s = 0.f;
    if (mx < m2x)
        for (int my = y0 + ty; my < y1; my += 8) {
            const float2 a = g[(size_t)my * m2x + mx], b = u2[(size_t)my * m2x + mx];
            s += a.x * b.x + a.y * b.y;
        }
    __shared__ float red[8][33];
    red[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && mx < m2x) {
        float t = 0.f;
        for (int r = 0; r < 8; ++r) t += red[r][tx];
        atomicAdd(&out[mx], t / corr[mx]);
    }
}

// dL/dcorr_y[my] (one block per row)
__global__ void deconv_grad_y_kernel(const float2* __restrict__ g, const float2* __restrict__ u2,
                                     const float* __restrict__ corr, int m2x, float* __restrict__ out)
{
    const int my = blockIdx.x;
    float s = 0.f;
    for (int mx = threadIdx.x; mx < m2x; mx += blockDim.x) {
        const float2 a = g[(size_t)my * m2x + mx], b = u2[(size_t)my * m2x + mx];
        s += a.x * b.x + a.y * b.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
        out[my] = t / corr[my];
    }
}

// dL/dd_j = sum_k dL/dcorr[k] T_2j(u_k) (one block per axis)
__global__ void cheb_grad_kernel(const float* __restrict__ gcorr, int m, float* __restrict__ grad)
{
    float s[kLearnCheb];
    for (int j = 0; j < kLearnCheb; ++j) s[j] = 0.f;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const float u = 2.f * (float)(k - m / 2) / (float)m;
        float T[kLearnCheb];
        cheb_even(u, T);
        for (int j = 0; j < kLearnCheb; ++j) s[j] = fmaf(gcorr[k], T[j], s[j]);
    }
    __shared__ float red[kLearnCheb][32];
    for (int j = 0; j < kLearnCheb; ++j) {
        float v = s[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[j][threadIdx.x / 32] = v;
    }
    __syncthreads();
    if (threadIdx.x < kLearnCheb) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[threadIdx.x][w];
        grad[threadIdx.x] = t;
    }
}

// ---- dL/dtable from the adjoint grid ------------------------------------------

struct TGArgs {
    const float2* u1;
    const float* q;
    const AxisEntry* ax;
    const AxisEntry* ay;
    const AxisPos* px;
    const AxisPos* py;
    const float2* grid;   // b~ = F^H D^H g over the band
    const float* tab;
    float* tgrad;
    int n1x, n1y, nstx, nfx, nfy;
    float half_w;
    float inc_d;
};

__global__ void __launch_bounds__(256) table_grad_kernel(TGArgs a)
{
    constexpr int W = kLearnW, K = kLearnCoef;
    const int t = blockIdx.x;
    const int nx = (t % a.nstx) * kSrcTile + threadIdx.x % kSrcTile;
    const int ny = (t / a.nstx) * kSrcTile + threadIdx.x / kSrcTile;
    float gx[W][K], gy[W][K];
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
        for (int k = 0; k < K; ++k) gx[i][k] = gy[i][k] = 0.f;
    if (nx < a.n1x && ny < a.n1y) {
        const Raw r = load_raw(a, nx, ny);
        int l0x, l0y;
        float dx, dy;
        sample_pos(r.ex, r.ey, r.px, r.py, r.q, a.half_w, l0x, l0y, dx, dy);
        const float2 c = sample_value_fast(r, a.inc_d);
        float wx[W], wy[W];
        table_weights<W>(a.tab + (size_t)t * kLearnTableSize, dx, dy, wx, wy);
        const float tx = fmaf(2.f, dx, -1.f), ty = fmaf(2.f, dy, -1.f);
        float ptx[K], pty[K];
        ptx[0] = pty[0] = 1.f;
#pragma unroll
        for (int k = 1; k < K; ++k) {
            ptx[k] = ptx[k - 1] * tx;
            pty[k] = pty[k - 1] * ty;
        }
        const int mx = a.nfx - 1, my = a.nfy - 1;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2* row = a.grid + (size_t)((l0y + b) & my) * a.nfx;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const float2 B = __ldg(&row[(l0x + i) & mx]);
                const float v = B.x * c.x + B.y * c.y;  // Re[conj(B) c]
                const float vx = v * wy[b], vy = v * wx[i];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    gx[i][k] = fmaf(vx, ptx[k], gx[i][k]);
                    gy[b][k] = fmaf(vy, pty[k], gy[b][k]);
                }
            }
        }
    }
    // block reduction of the 2 W K = 64 sums: within each warp a
    // reduce-scatter by recursive halving (at offset o a lane keeps the half
    // of its values selected by lane bit o and adds its partner's copy of
    // that half), after which lane l holds the warp's sums of entries 2l and
    // 2l + 1; then the 8 warps' sums are added in shared memory
    static_assert(2 * W * K == 64, "reduce-scatter of 64 values over 32 lanes");
    float v[64];
#pragma unroll
    for (int i = 0; i < W; ++i)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            v[i * K + k] = gx[i][k];
            v[(W + i) * K + k] = gy[i][k];
        }
    const int lane = threadIdx.x & 31, wid = threadIdx.x / 32;
#pragma unroll
    for (int lvl = 0; lvl < 5; ++lvl) {
        const int o = 16 >> lvl, half = 32 >> lvl;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    __shared__ float red[8][kLearnTableSize];
    red[wid][2 * lane] = v[0];
    red[wid][2 * lane + 1] = v[1];
    __syncthreads();
    if (threadIdx.x < kLearnTableSize) {
        float s = 0.f;
        for (int w2 = 0; w2 < 8; ++w2) s += red[w2][threadIdx.x];
        a.tgrad[(size_t)t * kLearnTableSize + threadIdx.x] = s;
    }
}

// ---- MLP backward over tiles (block-private accumulation, then atomics) --------

__global__ void __launch_bounds__(256) mlp_backward_kernel(const float* __restrict__ prm,
                                                           const float* __restrict__ feat,
                                                           const float* __restrict__ hid,
                                                           const float* __restrict__ tgrad, int ntiles,
                                                           float* __restrict__ grad)
{
    constexpr int O = kLearnTableSize, H = kLearnHidden, F = kLearnFeat;
    __shared__ float gW2[O * H], gb2[O], gbase[O], gW1[H * F], gb1[H];
    __shared__ float dout[O], h[H], f[F], dh[H];
    const int tid = threadIdx.x;
    for (int i = tid; i < O * H; i += blockDim.x) gW2[i] = 0.f;
    for (int i = tid; i < H * F; i += blockDim.x) gW1[i] = 0.f;
    if (tid < O) gb2[tid] = gbase[tid] = 0.f;
    if (tid < H) gb1[tid] = 0.f;
    __syncthreads();
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (tid < O) {
            const float d = tgrad[(size_t)t * O + tid];
            gbase[tid] += d;
            dout[tid] = kLearnOutScale * d;
            gb2[tid] += kLearnOutScale * d;
        }
        if (tid < H) h[tid] = hid[(size_t)t * H + tid];
        if (tid < F) f[tid] = feat[(size_t)t * F + tid];
        __syncthreads();
        for (int i = tid; i < O * H; i += blockDim.x) gW2[i] += dout[i / H] * h[i % H];
        if (tid < H) {
            float s = 0.f;
            for (int o = 0; o < O; ++o) s = fmaf(prm[kLpW2 + o * H + tid], dout[o], s);
            const float d = s * (1.f - h[tid] * h[tid]);
            dh[tid] = d;
            gb1[tid] += d;
        }
        __syncthreads();
        for (int i = tid; i < H * F; i += blockDim.x) gW1[i] += dh[i / F] * f[i % F];
        __syncthreads();
    }
    for (int i = tid; i < O * H; i += blockDim.x) atomicAdd(&grad[kLpW2 + i], gW2[i]);
    for (int i = tid; i < H * F; i += blockDim.x) atomicAdd(&grad[kLpW1 + i], gW1[i]);
    if (tid < O) {
        atomicAdd(&grad[kLpB2 + tid], gb2[tid]);
        atomicAdd(&grad[kLpBase + tid], gbase[tid]);
    }
    if (tid < H) atomicAdd(&grad[kLpB1 + tid], gb1[tid]);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float c1,
                            float c2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---- host helpers ------------------------------------------------------------

// Least-squares fit (FP64 normal equations on Chebyshev nodes) of the ES
// kernel of width kLearnW, tap by tap, by polynomials of degree kLearnDeg in
// t = 2 dx - 1: the initial shared table.
void fit_es_table(double beta, std::vector<float>& table)
{
    constexpr int W = kLearnW, K = kLearnCoef, NP = 256;
    const double pi = 3.14159265358979323846;
    table.assign(kLearnTableSize, 0.f);
    for (int a = 0; a < W; ++a) {
        double A[K][K] = {}, b[K] = {};
        for (int p = 0; p < NP; ++p) {
            const double t = std::cos(pi * (p + 0.5) / NP);
            const double dx = 0.5 * (t + 1.0);
            const double z = dx + a - 0.5 * W;
            const double u = 2.0 * z / W;
            const double psi = std::exp(beta * (std::sqrt(std::max(0.0, 1.0 - u * u)) - 1.0));
            double pw[K];
            pw[0] = 1.0;
            for (int k = 1; k < K; ++k) pw[k] = pw[k - 1] * t;
            for (int i = 0; i < K; ++i) {
                b[i] += pw[i] * psi;
                for (int j = 0; j < K; ++j) A[i][j] += pw[i] * pw[j];
            }
        }
        // Gaussian elimination with partial pivoting
        for (int c = 0; c < K; ++c) {
            int piv = c;
            for (int r = c + 1; r < K; ++r)
                if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
            for (int j = 0; j < K; ++j) std::swap(A[c][j], A[piv][j]);
            std::swap(b[c], b[piv]);
            for (int r = c + 1; r < K; ++r) {
                const double f = A[r][c] / A[c][c];
                for (int j = c; j < K; ++j) A[r][j] -= f * A[c][j];
                b[r] -= f * b[c];
            }
        }
        double x[K];
        for (int c = K - 1; c >= 0; --c) {
            double s = b[c];
            for (int j = c + 1; j < K; ++j) s -= A[c][j] * x[j];
            x[c] = s / A[c][c];
        }
        for (int k = 0; k < K; ++k) {
            table[(0 * W + a) * K + k] = (float)x[k];
            table[(1 * W + a) * K + k] = (float)x[k];
        }
    }
}

}  // namespace

asfd_status learned_features(asfd_plan_s* P, cudaStream_t st)
{
    const int nst = P->nstx * P->nsty;
    features_kernel<<<nst, kSrcTile * kSrcTile, 0, st>>>(P->q, P->ax, P->ay, P->bux, P->buy,
                                                        P->prm.n1x, P->prm.n1y, P->nstx, P->nfx,
                                                        P->nfy, P->lfeat);
    ASFD_CUDA(cudaGetLastError());
    return ASFD_OK;
}

asfd_status learned_refresh(asfd_plan_s* P, cudaStream_t st)
{
    const int nst = P->nstx * P->nsty;
    mlp_forward_kernel<<<nst, kLearnTableSize, 0, st>>>(P->lparams, P->lfeat, P->lhid, P->ltab);
    const int m2x = P->prm.m2x, m2y = P->prm.m2y;
    deconv_build_kernel<<<(m2x + 255) / 256, 256, 0, st>>>(P->lparams, P->cxb, P->cx, P->lcorr, m2x,
                                                           kLpDx);
    deconv_build_kernel<<<(m2y + 255) / 256, 256, 0, st>>>(P->lparams, P->cyb, P->cy,
                                                           P->lcorr + m2x, m2y, kLpDy);
    ASFD_CUDA(cudaGetLastError());
    return ASFD_OK;
}

asfd_status learned_init(asfd_plan_s* P, cudaStream_t st)
{
    const int nst = P->nstx * P->nsty;
    const int mm = P->prm.m2x + P->prm.m2y;
    auto A = [&](void** p, size_t bytes) { return plan_alloc_buffer(P, p, bytes); };
    asfd_status s;
#define LA(ptr, bytes) if ((s = A(reinterpret_cast<void**>(&P->ptr), (bytes))) != ASFD_OK) return s
    LA(ltab, sizeof(float) * nst * kLearnTableSize);
    LA(lfeat, sizeof(float) * nst * kLearnFeat);
    LA(lhid, sizeof(float) * nst * kLearnHidden);
    LA(ltgrad, sizeof(float) * nst * kLearnTableSize);
    LA(lparams, sizeof(float) * kLearnParams);
    LA(lgrad, sizeof(float) * kLearnParams);
    LA(lm, sizeof(float) * kLearnParams);
    LA(lv, sizeof(float) * kLearnParams);
    LA(cxb, sizeof(float2) * P->prm.m2x);
    LA(cyb, sizeof(float2) * P->prm.m2y);
    LA(lcorr, sizeof(float) * mm);
    LA(lcgrad, sizeof(float) * mm);
    LA(lred, sizeof(double) * 2);
#undef LA
    // the ES width-4 deconvolution/chirp tables become the base tables
    ASFD_CUDA(cudaMemcpyAsync(P->cxb, P->cx, sizeof(float2) * P->prm.m2x, cudaMemcpyDeviceToDevice, st));
    ASFD_CUDA(cudaMemcpyAsync(P->cyb, P->cy, sizeof(float2) * P->prm.m2y, cudaMemcpyDeviceToDevice, st));
    // initial parameters: fitted base table, small seeded W1, zero elsewhere
    std::vector<float> h(kLearnParams, 0.f), base;
    fit_es_table(P->beta, base);
    for (int i = 0; i < kLearnTableSize; ++i) h[kLpBase + i] = base[i];
    unsigned long long st64 = 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < kLearnHidden * kLearnFeat; ++i) {
        st64 = st64 * 6364136223846793005ull + 1442695040888963407ull;
        const float u = (float)((st64 >> 40) & 0xFFFFFF) / 16777216.0f;
        h[kLpW1 + i] = 0.5f * (2.f * u - 1.f);
    }
    ASFD_CUDA(cudaMemcpyAsync(P->lparams, h.data(), sizeof(float) * kLearnParams,
                              cudaMemcpyHostToDevice, st));
    ASFD_CUDA(cudaMemsetAsync(P->lm, 0, sizeof(float) * kLearnParams, st));
    ASFD_CUDA(cudaMemsetAsync(P->lv, 0, sizeof(float) * kLearnParams, st));
    P->lstep = 0;
    s = learned_features(P, st);
    if (s != ASFD_OK) return s;
    s = learned_refresh(P, st);
    if (s != ASFD_OK) return s;
    ASFD_CUDA(cudaStreamSynchronize(st));  // h must outlive the copy
    return ASFD_OK;
}

// Forward with the current model, loss against `ref`, and every parameter
// gradient into P->lgrad (no update).
asfd_status learned_gradient(asfd_plan_s* P, const float2* u1, const float2* ref, cudaStream_t st)
{
    const int nst = P->nstx * P->nsty;
    const int m2x = P->prm.m2x, m2y = P->prm.m2y;
    const size_t m = (size_t)m2x * m2y;
    asfd_status s;
    // forward with the current model
    if ((s = learned_refresh(P, st)) != ASFD_OK) return s;
    if ((s = launch_spread(P, u1, st)) != ASFD_OK) return s;
    if ((s = launch_fft_rows(P, st)) != ASFD_OK) return s;
    if ((s = launch_fft_cols(P, P->lu2, st)) != ASFD_OK) return s;
    // loss and its gradient with respect to u2
    ASFD_CUDA(cudaMemsetAsync(P->lred, 0, sizeof(double) * 2, st));
    loss_reduce_kernel<<<512, 256, 0, st>>>(P->lu2, ref, m, P->lred);
    residual_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(P->lu2, ref, m, P->lred, P->lres);
    ASFD_CUDA(cudaMemsetAsync(P->lgrad, 0, sizeof(float) * kLearnParams, st));
    // deconvolution correction gradients
    ASFD_CUDA(cudaMemsetAsync(P->lcgrad, 0, sizeof(float) * m2x, st));
    deconv_grad_x_kernel<<<dim3((m2x + 31) / 32, kDeconvSlabs), 256, 0, st>>>(
        P->lres, P->lu2, P->lcorr, m2x, m2y, P->lcgrad);
    deconv_grad_y_kernel<<<m2y, 256, 0, st>>>(P->lres, P->lu2, P->lcorr + m2x, m2x, P->lcgrad + m2x);
    cheb_grad_kernel<<<1, 256, 0, st>>>(P->lcgrad, m2x, P->lgrad + kLpDx);
    cheb_grad_kernel<<<1, 256, 0, st>>>(P->lcgrad + m2x, m2y, P->lgrad + kLpDy);
    ASFD_CUDA(cudaGetLastError());
    // table gradients through the adjoint grid
    if ((s = launch_fft_cols_adj(P, P->lres, st)) != ASFD_OK) return s;
    if ((s = launch_fft_rows_adj(P, st)) != ASFD_OK) return s;
    TGArgs a;
    a.u1 = u1;
    a.q = P->q;
    a.ax = P->ax;
    a.ay = P->ay;
    a.px = P->px;
    a.py = P->py;
    a.grid = P->grid;
    a.tab = P->ltab;
    a.tgrad = P->ltgrad;
    a.n1x = P->prm.n1x;
    a.n1y = P->prm.n1y;
    a.nstx = P->nstx;
    a.nfx = P->nfx;
    a.nfy = P->nfy;
    a.half_w = 0.5f * kLearnW;
    a.inc_d = (float)P->inc_d;
    table_grad_kernel<<<nst, 256, 0, st>>>(a);
    mlp_backward_kernel<<<nst < 256 ? nst : 256, 256, 0, st>>>(P->lparams, P->lfeat, P->lhid,
                                                                P->ltgrad, nst, P->lgrad);
    ASFD_CUDA(cudaGetLastError());
    return ASFD_OK;
}

asfd_status learned_read_loss(asfd_plan_s* P, double* loss_out, cudaStream_t st)
{
    double red[2];
    ASFD_CUDA(cudaMemcpyAsync(red, P->lred, sizeof(red), cudaMemcpyDeviceToHost, st));
    ASFD_CUDA(cudaStreamSynchronize(st));
    *loss_out = red[0] / (red[1] > 0.0 ? red[1] : 1.0);
    return ASFD_OK;
}

asfd_status learned_train_step(asfd_plan_s* P, const float2* u1, const float2* ref, float lr,
                               double* loss_out, cudaStream_t st)
{
    asfd_status s = learned_gradient(P, u1, ref, st);
    if (s != ASFD_OK) return s;
    // Adam
    ++P->lstep;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)P->lstep), c2 = 1.f - std::pow(b2, (float)P->lstep);
    adam_kernel<<<(kLearnParams + 255) / 256, 256, 0, st>>>(P->lparams, P->lgrad, P->lm, P->lv,
                                                           kLearnParams, lr, b1, b2, c1, c2, 1e-12f);
    ASFD_CUDA(cudaGetLastError());
    if ((s = learned_refresh(P, st)) != ASFD_OK) return s;
    if (loss_out) return learned_read_loss(P, loss_out, st);
    return ASFD_OK;
}

}  // namespace asfd
