// Plan construction: FP64 geometry and phase tables, d1 checks, binning.
//
// All phases are carried in half-turns (units of pi), because
//   k |x|^2 / (2 z) = pi |x|^2 / (lambda z)   and   k z0 = pi (2 z0 / lambda),
// so no inexact multiple of pi enters, and reduction modulo 2 (= 2 pi rad)
// of an FP64 value a is the exact operation a - 2 rint(a/2).  sincospi then
// evaluates the reduced phase.  These are the large phases of Eqs. 5-8: the
// global k z0 (up to ~2e6 rad at the standard workloads), the source chirp
// k|x1|^2/(2 z0) and the destination chirp k|x2|^2/(2 z0) (up to ~5e3 rad).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "asfd_impl.cuh"

namespace asfd {

namespace {

__device__ __forceinline__ double reduce_halfturns(double a) { return a - 2.0 * rint(0.5 * a); }

// Per-axis source table: chirp exp(i pi x^2/(lambda z0)), its unreduced value
// in half-turns, the fine-grid offset alpha x~ and its storage-coordinate split.
// tilt: 2 s / lambda, the incident plane wave's linear phase in half-turns per
// metre along this axis (0 at normal incidence); e = exp(i pi (a + tilt x1)).
// off: position of the centre sample (the grid's offset from the axis, metres).
__global__ void axis_table_kernel(AxisEntry* ae, AxisPos* ap, double* bu, int n, double p,
                                  double lam_z0, double alpha, int nf, double tilt, double off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xt = (double)(i - n / 2) + off / p;  // x1 / p
    const double x1 = xt * p;
    const double a = x1 * x1 / lam_z0;
    double s, c;
    sincospi(reduce_halfturns(a) + reduce_halfturns(tilt * x1), &s, &c);
    const double g = alpha * xt;
    const double B = g + 0.5 * (double)nf;
    const double Br = B - (double)nf * floor(B / (double)nf);
    int bi = (int)floor(Br);
    double bf = Br - (double)bi;
    if (bi >= nf) bi -= nf;
    AxisEntry e;
    e.e = make_float2((float)c, (float)s);
    e.a = (float)a;
    e.s = (float)g;
    ae[i] = e;
    AxisPos q;
    q.bi = bi;
    q.bf = (float)bf;
    ap[i] = q;
    bu[i] = B;
}

// Destination table C[k'] = (-1)^m' exp(i pi x2^2/(lambda z0)) / psi_hat(2 pi m'/nf),
// m' = k' - m/2, times the global factor exp(ik z0) p1x p1y / (i lambda z0)
// when `global` is set.  psi_hat(xi) = 2 sum_i w_i psi(z_i) cos(xi z_i)
// (Gauss-Legendre on [0, w/2], nodes and weighted kernel values in quad).
// A warp per entry: the lanes share the quadrature nodes and their partial
// sums meet in a fixed shuffle tree.
__global__ void dest_table_kernel(float2* C, int m, double p2, double lam_z0, int nf,
                                  const double* quad, int nq, int global, double two_z0_over_lam,
                                  double amp)
{
    const int k = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / 32);
    const int lane = threadIdx.x % 32;
    if (k >= m) return;  // warp-uniform
    const int mp = k - m / 2;
    double ph = 0.0;
    for (int i = lane; i < nq; i += 32)
        ph += quad[nq + i] * cospi(2.0 * (double)mp * quad[i] / (double)nf);
    for (int o = 16; o > 0; o >>= 1) ph += __shfl_xor_sync(0xffffffffu, ph, o);
    if (lane != 0) return;
    ph *= 2.0;
    const double x2 = (double)mp * p2;
    double s, c;
    sincospi(reduce_halfturns(x2 * x2 / lam_z0), &s, &c);
    const double sgn = (mp & 1) ? -1.0 : 1.0;
    double re = sgn * c / ph, im = sgn * s / ph;
    if (global) {
        // exp(i theta) / i * amp = amp (sin theta - i cos theta), theta = k z0
        double gs, gc;
        sincospi(reduce_halfturns(two_z0_over_lam), &gs, &gc);
        const double gre = amp * gs, gim = -amp * gc;
        const double r2 = re * gre - im * gim, i2 = re * gim + im * gre;
        re = r2;
        im = i2;
    }
    C[k] = make_float2((float)re, (float)im);
}

// Checks d1 (finite, below z0) and reduces max |d1|/z0 (in FP32: a bound
// checked against 0.1).
// (grid-stride; the block's maximum goes out with one atomic: per-warp
// atomics on the one word serialise)
__global__ void __launch_bounds__(256) d1_check_kernel(const double* d1, size_t n, double z0,
                                                       float inv_z0, unsigned* status,
                                                       unsigned* maxeps_bits)
{
    float e = 0.f;
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double h = d1[i];
        if (!isfinite(h) || !(h < z0)) bad = true;
        else e = fmaxf(e, (float)fabs(h) * inv_z0);
    }
    if (bad) atomicOr(status, kStatusBadD1);
    for (int o = 16; o > 0; o >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) e = fmaxf(e, red[w]);
        atomicMax(maxeps_bits, __float_as_uint(e));
    }
}

// q = d1 / (z0 - d1), stored FP32: z0 - d1 formed in FP64 (no cancellation
// error), both operands rounded to FP32 and divided there (within 1.5 FP32
// ulp of the FP64 quotient; an FP64 division per sample is slow on this GPU).
__global__ void d1_q_kernel(const double* d1, float* q, size_t n, double z0)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h = d1[i];
    q[i] = __fdiv_rn((float)h, (float)(z0 - h));
}

// Per source tile: bounds of the unreduced storage coordinate alpha x~ (1+q) + nf/2,
// in FP32 (within a few 1e-3 cells: the binning adds a one-cell margin).
__global__ void src_bbox_kernel(const float* q, const AxisEntry* ax, const AxisEntry* ay,
                                const double* bux, const double* buy, int n1x, int n1y, int nstx,
                                float4* bbox)
{
    const int tile = blockIdx.x;
    const int nx = (tile % nstx) * kSrcTile + threadIdx.x % kSrcTile;
    const int ny = (tile / nstx) * kSrcTile + threadIdx.x / kSrcTile;
    float x0 = 3e38f, x1 = -3e38f, y0 = 3e38f, y1 = -3e38f;
    if (nx < n1x && ny < n1y) {
        const float qq = q[(size_t)ny * n1x + nx];
        const float ux = (float)bux[nx] + ax[nx].s * qq;
        const float uy = (float)buy[ny] + ay[ny].s * qq;
        x0 = x1 = ux;
        y0 = y1 = uy;
    }
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    __shared__ float red[4][kSrcTile * kSrcTile / 32];
    const int wid = threadIdx.x / 32;
    if ((threadIdx.x & 31) == 0) {
        red[0][wid] = x0;
        red[1][wid] = x1;
        red[2][wid] = y0;
        red[3][wid] = y1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kSrcTile * kSrcTile / 32; ++w) {
            x0 = fminf(x0, red[0][w]);
            x1 = fmaxf(x1, red[1][w]);
            y0 = fminf(y0, red[2][w]);
            y1 = fmaxf(y1, red[3][w]);
        }
        bbox[tile] = make_float4(x0, x1, y0, y1);
    }
}

// The storage coordinate of a sample is b + (double)(s * q) with b and s
// fixed per column (x) or per row (y); an FP32 product with a fixed factor
// and the FP64 sum with a fixed term are monotone in q, so its extremes over
// a column (row) are those of q, mapped.
__device__ __forceinline__ double2 coord_range(double b, float s, float qlo, float qhi)
{
    const float a0 = s * qlo, a1 = s * qhi;
    return make_double2(b + (double)fminf(a0, a1), b + (double)fmaxf(a0, a1));
}

// Per source column: [min, max] over rows of the unreduced x storage
// coordinate.  Blocks of 32 columns (a lane each) by 8 warps over the rows.
__global__ void __launch_bounds__(256) col_range_kernel(const float* q, const AxisEntry* ax,
                                                        const double* bux, int n1x, int n1y,
                                                        double2* out)
{
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    const int nx = blockIdx.x * 32 + lane;
    float lo = 3e38f, hi = -3e38f;
    if (nx < n1x) {
        for (int ny = w; ny < n1y; ny += 8) {
            const float v = q[(size_t)ny * n1x + nx];
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    }
    __shared__ float red[2][8][32];
    red[0][w][lane] = lo;
    red[1][w][lane] = hi;
    __syncthreads();
    if (w == 0 && nx < n1x) {
        for (int k = 1; k < 8; ++k) {
            lo = fminf(lo, red[0][k][lane]);
            hi = fmaxf(hi, red[1][k][lane]);
        }
        out[nx] = coord_range(bux[nx], ax[nx].s, lo, hi);
    }
}

// Per source row: [min, max] over columns of the unreduced y storage coordinate.
__global__ void row_range_kernel(const float* q, const AxisEntry* ay, const double* buy, int n1x,
                                 double2* out)
{
    const int ny = blockIdx.x;
    float lo = 3e38f, hi = -3e38f;
    for (int nx = threadIdx.x; nx < n1x; nx += blockDim.x) {
        const float v = q[(size_t)ny * n1x + nx];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ float red[2][32];
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x / 32] = lo;
        red[1][threadIdx.x / 32] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) {
            lo = fminf(lo, red[0][w]);
            hi = fmaxf(hi, red[1][w]);
        }
        out[ny] = coord_range(buy[ny], ay[ny].s, lo, hi);
    }
}

// Minimum spacing on the fine grid of neighbouring samples: along x within a
// row and along y within a column (one pair of minima per block).  A thread
// takes one column over a chunk of rows: the FP64 difference of the
// neighbouring columns' base coordinates is formed once, the q terms in
// FP32 (the spacing is ~1 cell, so this is good to ~1e-6 cells).
__global__ void min_step_kernel(const float* q, const AxisEntry* ax, const AxisEntry* ay,
                                const double* bux, const double* buy, int n1x, int n1y,
                                float2* out)
{
    const int nx = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = (n1y + gridDim.y - 1) / gridDim.y;
    const int r0 = blockIdx.y * chunk, r1 = min(n1y, r0 + chunk);
    float mx = 3.0e38f, my = 3.0e38f;
    if (nx < n1x) {
        const bool hasx = nx + 1 < n1x;
        const float sx0 = ax[nx].s, sx1 = hasx ? ax[nx + 1].s : 0.f;
        const float dbx = hasx ? (float)(bux[nx + 1] - bux[nx]) : 0.f;
        for (int ny = r0; ny < r1; ++ny) {
            const size_t i = (size_t)ny * n1x + nx;
            const float qq = q[i];
            if (hasx) mx = fminf(mx, dbx + (sx1 * q[i + 1] - sx0 * qq));
            if (ny + 1 < n1y) {
                const float dby = (float)(buy[ny + 1] - buy[ny]);
                my = fminf(my, dby + (ay[ny + 1].s * q[i + n1x] - ay[ny].s * qq));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fminf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        my = fminf(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    __shared__ float red[2][32];
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x / 32] = mx;
        red[1][threadIdx.x / 32] = my;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) {
            mx = fminf(mx, red[0][w]);
            my = fminf(my, red[1][w]);
        }
        out[blockIdx.y * gridDim.x + blockIdx.x] = make_float2(mx, my);
    }
}

constexpr int kStepBlocks = 1024;

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt)
{
    const double pi = 3.14159265358979323846;
    x.assign(n, 0.0);
    wt.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        wt[i] = wt[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// true when the allocation-failure hook says this allocation must fail
bool injected_failure()
{
    int b = g_alloc_budget.load();
    while (b > 0 && !g_alloc_budget.compare_exchange_weak(b, b - 1)) {
    }
    return b == 0;
}

asfd_status alloc(asfd_plan_s* P, void** p, size_t bytes)
{
    if (injected_failure()) {
        *p = nullptr;
        return fail(ASFD_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) +
                                        " bytes refused by asfd_debug_fail_allocations");
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ASFD_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                        cudaGetErrorString(e));
    }
    P->owned.push_back(DevBuf{*p, bytes});
    P->device_bytes += bytes;
    ++g_live_buffers;
    return ASFD_OK;
}

template <class T>
asfd_status alloc_n(asfd_plan_s* P, T** p, size_t count)
{
    void* v = nullptr;
    asfd_status s = alloc(P, &v, sizeof(T) * (count ? count : 1));
    *p = static_cast<T*>(v);
    return s;
}

void release(asfd_plan_s* P, void* p)
{
    for (size_t i = 0; i < P->owned.size(); ++i) {
        if (P->owned[i].p == p) {
            P->device_bytes -= P->owned[i].bytes;
            cudaFree(p);
            --g_live_buffers;
            P->owned.erase(P->owned.begin() + i);
            return;
        }
    }
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

}  // namespace

asfd_status plan_build_colored(asfd_plan_s* P, bool wraps, cudaStream_t st);

asfd_status plan_alloc_buffer(asfd_plan_s* P, void** p, size_t bytes) { return alloc(P, p, bytes); }

int es_quadrature(int w, double beta, std::vector<double>& h)
{
    const int nq = 160;
    std::vector<double> x, wt;
    h.assign(2 * nq, 0.0);
    gauss_legendre(nq, x, wt);
    const double half = 0.5 * w;
    for (int i = 0; i < nq; ++i) {
        const double z = 0.5 * half * (x[i] + 1.0);
        const double u = z / half;
        const double psi = std::exp(beta * (std::sqrt(std::max(0.0, 1.0 - u * u)) - 1.0));
        h[i] = z;
        h[nq + i] = 0.5 * half * wt[i] * psi;
    }
    return nq;
}

asfd_status plan_validate(const asfd_params* p, int* nfx, int* nfy, double* beta)
{
    if (!p) return fail(ASFD_ERR_ARG, "params is NULL");
    auto even_in = [](int n) { return n >= 2 && n <= 65536 && n % 2 == 0; };
    if (!even_in(p->n1x) || !even_in(p->n1y))
        return fail(ASFD_ERR_ARG, "n1x and n1y must be even and in [2, 65536]");
    if (!even_in(p->m2x) || !even_in(p->m2y))
        return fail(ASFD_ERR_ARG, "m2x and m2y must be even and in [2, 65536]");
    const double pos[] = {p->p1x, p->p1y, p->p2x, p->p2y, p->lambda, p->z0, p->sigma};
    for (double v : pos)
        if (!(std::isfinite(v) && v > 0.0))
            return fail(ASFD_ERR_ARG, "pitches, wavelength, z0 and sigma must be finite and > 0");
    if (p->kernel_width < 2 || p->kernel_width > 16)
        return fail(ASFD_ERR_UNSUPPORTED, "kernel_width must be in [2, 16]");
    if (p->deterministic != 0 && p->deterministic != 1)
        return fail(ASFD_ERR_ARG, "deterministic must be 0 or 1");
    if (p->kind != ASFD_KERNEL_ES && p->kind != ASFD_KERNEL_LEARNED)
        return fail(ASFD_ERR_ARG, "kind must be ASFD_KERNEL_ES or ASFD_KERNEL_LEARNED");
    if (p->kind == ASFD_KERNEL_LEARNED && p->kernel_width != kLearnW)
        return fail(ASFD_ERR_UNSUPPORTED, "the learned kernel has width 4");
    if (!(p->sigma >= 1.25 && p->sigma <= 4.0))
        return fail(ASFD_ERR_UNSUPPORTED, "sigma must be in [1.25, 4]");
    const double fx = p->sigma * p->m2x, fy = p->sigma * p->m2y;
    const int ix = (int)std::lround(fx), iy = (int)std::lround(fy);
    if (std::fabs(fx - ix) > 1e-9 * fx || std::fabs(fy - iy) > 1e-9 * fy || !pow2_in(ix, 64, 16384) ||
        !pow2_in(iy, 64, 16384))
        return fail(ASFD_ERR_UNSUPPORTED,
                    "sigma*m2x and sigma*m2y must be powers of two in [64, 16384]");
    if (p->kernel_width >= ix / 2 || p->kernel_width >= iy / 2)
        return fail(ASFD_ERR_UNSUPPORTED, "kernel wider than half the fine grid");
    if (!(std::isfinite(p->incidence_sx) && std::isfinite(p->incidence_sy) &&
          p->incidence_sx * p->incidence_sx + p->incidence_sy * p->incidence_sy < 1.0))
        return fail(ASFD_ERR_ARG, "incidence direction cosines need sx^2 + sy^2 < 1");
    if (!(std::isfinite(p->es_beta) && p->es_beta >= 0.0))
        return fail(ASFD_ERR_ARG, "es_beta must be finite and >= 0");
    if (!(std::isfinite(p->offset_x) && std::isfinite(p->offset_y)))
        return fail(ASFD_ERR_ARG, "source offsets must be finite");
    const double pi = 3.14159265358979323846;
    double b = p->es_beta;
    if (b == 0.0)
        b = (p->sigma == 2.0) ? 2.30 * p->kernel_width
                              : 0.97 * pi * (1.0 - 1.0 / (2.0 * p->sigma)) * p->kernel_width;
    *nfx = ix;
    *nfy = iy;
    *beta = b;
    return ASFD_OK;
}

asfd_status plan_alloc(asfd_plan_s* P)
{
    const asfd_params& p = P->prm;
    const size_t nsrc = (size_t)p.n1x * p.n1y;
    P->nstx = (p.n1x + kSrcTile - 1) / kSrcTile;
    P->nsty = (p.n1y + kSrcTile - 1) / kSrcTile;
    P->ntx = P->nfx / kTileX;
    P->nty = P->nfy / kTileY;
    asfd_status s;
#define A(ptr, n) if ((s = alloc_n(P, &P->ptr, (n))) != ASFD_OK) return s
    A(ax, p.n1x);
    A(ay, p.n1y);
    A(px, p.n1x);
    A(py, p.n1y);
    A(bux, p.n1x);
    A(buy, p.n1y);
    A(q, nsrc);
    A(cx, p.m2x);
    A(cy, p.m2y);
    A(twx, P->nfx);
    A(twy, P->nfy);
    A(src_bbox, (size_t)P->nstx * P->nsty);
    A(tile_off, (size_t)P->ntx * P->nty + 1);
    A(tile_rect, (size_t)P->ntx * P->nty * (kTileY / kColTileY));
    A(col_range, p.n1x);
    A(row_range, p.n1y);
    A(step_min, kStepBlocks);
    A(status, 2);
#undef A
    return ASFD_OK;
}

WorkLayout work_layout(const asfd_params& p, int nfx, int nfy)
{
    const auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t c = sizeof(float2);
    WorkLayout L;
    size_t o = 0;
    L.grid = o;
    o += up(c * (size_t)nfx * nfy);
    L.rows = o;
    o += up(c * (size_t)nfy * row_buffer_width(p.m2x));
    L.stage_u1 = o;
    o += up(c * (size_t)p.n1x * p.n1y);
    L.stage_u2 = o;
    o += up(c * (size_t)p.m2x * p.m2y);
    if (p.kind == ASFD_KERNEL_LEARNED) {
        L.lu2 = o;
        o += up(c * (size_t)p.m2x * p.m2y);
        L.lres = o;
        o += up(c * (size_t)p.m2x * p.m2y);
    }
    L.total = o;
    return L;
}

asfd_status plan_ensure_work(asfd_plan_s* P, unsigned need)
{
    if (P->ws) return ASFD_OK;  // every work buffer was carved when the workspace was set
    const asfd_params& p = P->prm;
    asfd_status s;
    if ((need & kWorkTransform) && !P->grid) {
        P->band_clean = false;  // fresh memory
        if ((s = alloc_n(P, &P->grid, (size_t)P->nfx * P->nfy)) != ASFD_OK) return s;
        if ((s = alloc_n(P, &P->rows, (size_t)P->nfy * row_buffer_width(p.m2x))) != ASFD_OK) {
            release(P, P->grid);
            P->grid = nullptr;
            return s;
        }
    }
    if ((need & kWorkStaging) && !P->stage_u1) {
        if ((s = alloc_n(P, &P->stage_u1, (size_t)p.n1x * p.n1y)) != ASFD_OK) return s;
        if ((s = alloc_n(P, &P->stage_u2, (size_t)p.m2x * p.m2y)) != ASFD_OK) {
            release(P, P->stage_u1);
            P->stage_u1 = nullptr;
            return s;
        }
    }
    if ((need & kWorkTraining) && P->learned && !P->lu2) {
        if ((s = alloc_n(P, &P->lu2, (size_t)p.m2x * p.m2y)) != ASFD_OK) return s;
        if ((s = alloc_n(P, &P->lres, (size_t)p.m2x * p.m2y)) != ASFD_OK) {
            release(P, P->lu2);
            P->lu2 = nullptr;
            return s;
        }
    }
    return ASFD_OK;
}

asfd_status plan_set_workspace(asfd_plan_s* P, void* ws, size_t bytes)
{
    const WorkLayout L = work_layout(P->prm, P->nfx, P->nfy);
    if (ws) {
        if (bytes < L.total)
            return fail(ASFD_ERR_ARG, "workspace of " + std::to_string(bytes) +
                                          " bytes is smaller than asfd_workspace_bytes() = " +
                                          std::to_string(L.total));
        if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
            return fail(ASFD_ERR_ARG, "workspace must be 256-byte aligned");
        cudaPointerAttributes at{};
        ASFD_CUDA(cudaPointerGetAttributes(&at, ws));
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
            at.device != P->device)
            return fail(ASFD_ERR_ARG, "workspace must be device memory of the plan's device");
    } else if (bytes != 0) {
        return fail(ASFD_ERR_ARG, "a NULL workspace must come with bytes = 0");
    }
    // queued work may still use the buffers being replaced
    ASFD_CUDA(cudaDeviceSynchronize());
    float2** bufs[] = {&P->grid, &P->rows, &P->stage_u1, &P->stage_u2, &P->lu2, &P->lres};
    for (float2** b : bufs) {
        if (*b && !P->ws) release(P, *b);
        *b = nullptr;
    }
    P->ws = static_cast<char*>(ws);
    P->ws_bytes = ws ? bytes : 0;
    P->band_clean = false;
    if (ws) {
        char* base = P->ws;
        P->grid = reinterpret_cast<float2*>(base + L.grid);
        P->rows = reinterpret_cast<float2*>(base + L.rows);
        P->stage_u1 = reinterpret_cast<float2*>(base + L.stage_u1);
        P->stage_u2 = reinterpret_cast<float2*>(base + L.stage_u2);
        if (P->learned) {
            P->lu2 = reinterpret_cast<float2*>(base + L.lu2);
            P->lres = reinterpret_cast<float2*>(base + L.lres);
        }
    }
    return ASFD_OK;
}

asfd_status plan_build_tables(asfd_plan_s* P, cudaStream_t st)
{
    const asfd_params& p = P->prm;
    const double lam_z0 = p.lambda * p.z0;
    P->alpha_x = p.p1x * p.p2x * P->nfx / lam_z0;
    P->alpha_y = p.p1y * p.p2y * P->nfy / lam_z0;
    axis_table_kernel<<<(p.n1x + 255) / 256, 256, 0, st>>>(P->ax, P->px, P->bux, p.n1x, p.p1x,
                                                            lam_z0, P->alpha_x, P->nfx,
                                                            2.0 * p.incidence_sx / p.lambda,
                                                            p.offset_x);
    axis_table_kernel<<<(p.n1y + 255) / 256, 256, 0, st>>>(P->ay, P->py, P->buy, p.n1y, p.p1y,
                                                            lam_z0, P->alpha_y, P->nfy,
                                                            2.0 * p.incidence_sy / p.lambda,
                                                            p.offset_y);
    // the incident wave's depth phase k d1 (sz - 1) (the rest of u_I exp(-ik d1))
    // in half-turns is inc_d d1/z0 = inc_d q/(1 + q)
    {
        const double sz = std::sqrt(1.0 - p.incidence_sx * p.incidence_sx -
                                    p.incidence_sy * p.incidence_sy);
        P->inc_d = 2.0 * p.z0 * (sz - 1.0) / p.lambda;
    }
    ASFD_CUDA(cudaGetLastError());

    // ES kernel values at Gauss-Legendre nodes on [0, w/2]
    std::vector<double> h;
    const int nq = es_quadrature(P->w, P->beta, h);
    if (!P->quad) {
        asfd_status s = alloc_n(P, &P->quad, 2 * nq);
        if (s != ASFD_OK) return s;
    }
    P->nq = nq;
    ASFD_CUDA(cudaMemcpyAsync(P->quad, h.data(), sizeof(double) * 2 * nq, cudaMemcpyHostToDevice, st));
    const double amp = p.p1x * p.p1y / lam_z0;
    dest_table_kernel<<<(p.m2x + 7) / 8, 256, 0, st>>>(P->cx, p.m2x, p.p2x, lam_z0, P->nfx,
                                                            P->quad, nq, 0, 0.0, 0.0);
    dest_table_kernel<<<(p.m2y + 7) / 8, 256, 0, st>>>(P->cy, p.m2y, p.p2y, lam_z0, P->nfy,
                                                            P->quad, nq, 1, 2.0 * p.z0 / p.lambda,
                                                            amp);
    ASFD_CUDA(cudaGetLastError());
    asfd_status s = build_twiddles(P->twx, P->nfx, st);
    if (s != ASFD_OK) return s;
    s = build_twiddles(P->twy, P->nfy, st);
    if (s != ASFD_OK) return s;
    // the host vector h must outlive the async copy
    ASFD_CUDA(cudaStreamSynchronize(st));
    return ASFD_OK;
}

asfd_status plan_build_d1(asfd_plan_s* P, const double* d1, cudaStream_t st)
{
    const asfd_params& p = P->prm;
    const size_t nsrc = (size_t)p.n1x * p.n1y;
    // the band may move: its new cells were never cleared
    P->band_clean = false;
    // 1. validate d1 without touching the plan's tables
    ASFD_CUDA(cudaMemsetAsync(P->status, 0, 2 * sizeof(unsigned), st));
    d1_check_kernel<<<(unsigned)std::min<size_t>((nsrc + 255) / 256, 1216), 256, 0, st>>>(
        d1, nsrc, p.z0, (float)(1.0 / p.z0), P->status, P->status + 1);
    ASFD_CUDA(cudaGetLastError());
    unsigned hs[2] = {0, 0};
    ASFD_CUDA(cudaMemcpyAsync(hs, P->status, sizeof(hs), cudaMemcpyDeviceToHost, st));
    ASFD_CUDA(cudaStreamSynchronize(st));
    if (hs[0] & kStatusBadD1) return fail(ASFD_ERR_ARG, "d1 has a non-finite value or d1 >= z0");
    float me;
    std::memcpy(&me, &hs[1], sizeof(float));
    if (me > 0.1f)
        return fail(ASFD_ERR_UNSUPPORTED, "max |d1|/z0 = " + std::to_string(me) +
                                              " exceeds the supported 0.1");

    // 2. per-sample correction and per-source-tile footprint bounds
    d1_q_kernel<<<(unsigned)((nsrc + 255) / 256), 256, 0, st>>>(d1, P->q, nsrc, p.z0);
    const int nst = P->nstx * P->nsty;
    src_bbox_kernel<<<nst, kSrcTile * kSrcTile, 0, st>>>(P->q, P->ax, P->ay, P->bux, P->buy, p.n1x,
                                                         p.n1y, P->nstx, P->src_bbox);
    ASFD_CUDA(cudaGetLastError());
    std::vector<float> bb(4 * (size_t)nst);
    ASFD_CUDA(cudaMemcpyAsync(bb.data(), P->src_bbox, sizeof(float) * 4 * nst,
                              cudaMemcpyDeviceToHost, st));
    ASFD_CUDA(cudaStreamSynchronize(st));

    // 3. the band (fine-grid tiles that footprints reach) and the wrap flags,
    //    from each source tile's footprint bounds
    const double hw = 0.5 * P->w + 1.0;  // half width plus a one-cell safety margin
    struct Range { int x0, x1, y0, y1; };
    std::vector<Range> rg(nst);
    bool wrapx = false, wrapy = false;
    int bx0 = P->ntx, bx1 = -1, by0 = P->nty, by1 = -1;
    for (int t = 0; t < nst; ++t) {
        const float* b = &bb[4 * (size_t)t];
        Range r;
        r.x0 = (int)std::floor((b[0] - hw) / kTileX);
        r.x1 = (int)std::floor((b[1] + hw) / kTileX);
        r.y0 = (int)std::floor((b[2] - hw) / kTileY);
        r.y1 = (int)std::floor((b[3] + hw) / kTileY);
        // a footprint reaching outside [0, nf) wraps around the periodic grid
        if (b[0] - hw < 0.0 || b[1] + hw > (double)P->nfx) wrapx = true;
        if (b[2] - hw < 0.0 || b[3] + hw > (double)P->nfy) wrapy = true;
        if (r.x1 - r.x0 + 1 >= P->ntx) { r.x0 = 0; r.x1 = P->ntx - 1; }
        if (r.y1 - r.y0 + 1 >= P->nty) { r.y0 = 0; r.y1 = P->nty - 1; }
        if (r.x0 < 0 || r.x1 >= P->ntx) wrapx = true;
        if (r.y0 < 0 || r.y1 >= P->nty) wrapy = true;
        bx0 = std::min(bx0, r.x0);
        bx1 = std::max(bx1, r.x1);
        by0 = std::min(by0, r.y0);
        by1 = std::max(by1, r.y1);
        rg[t] = r;
    }
    if (wrapx) { bx0 = 0; bx1 = P->ntx - 1; }
    if (wrapy) { by0 = 0; by1 = P->nty - 1; }
    P->band_tx0 = bx0;
    P->band_tx1 = bx1 + 1;
    P->band_ty0 = by0;
    P->band_ty1 = by1 + 1;
    P->max_abs_eps = me;
    asfd_status cs = plan_build_colored(P, wrapx || wrapy, st);
    if (cs != ASFD_OK) return cs;
    P->tile_pairs = 0;
    if (!P->colored && !P->dense) {
        // the shared-memory-atomic spread walks, per band tile, the source
        // tiles whose footprints reach it: a CSR list built here
        const int bntx = bx1 - bx0 + 1, bnty = by1 - by0 + 1;
        const int ntiles = bntx * bnty;
        std::vector<int> off(ntiles + 1, 0);
        auto tmod = [](int v, int n) { int m = v % n; return m < 0 ? m + n : m; };
        for (int t = 0; t < nst; ++t) {
            const Range& r = rg[t];
            for (int ty = r.y0; ty <= r.y1; ++ty)
                for (int tx = r.x0; tx <= r.x1; ++tx) {
                    const int i = (tmod(ty, P->nty) - by0) * bntx + (tmod(tx, P->ntx) - bx0);
                    ++off[i + 1];
                }
        }
        for (int i = 0; i < ntiles; ++i) off[i + 1] += off[i];
        std::vector<int> lst(off[ntiles]);
        std::vector<int> fillp(off.begin(), off.end() - 1);
        for (int t = 0; t < nst; ++t) {
            const Range& r = rg[t];
            for (int ty = r.y0; ty <= r.y1; ++ty)
                for (int tx = r.x0; tx <= r.x1; ++tx) {
                    const int i = (tmod(ty, P->nty) - by0) * bntx + (tmod(tx, P->ntx) - bx0);
                    lst[fillp[i]++] = t;
                }
        }
        if (lst.size() > P->tile_src_cap || !P->tile_src) {
            if (P->tile_src) release(P, P->tile_src);
            P->tile_src = nullptr;
            const size_t cap = std::max<size_t>(lst.size() + lst.size() / 4, 1024);
            asfd_status s = alloc_n(P, &P->tile_src, cap);
            if (s != ASFD_OK) { P->tile_src_cap = 0; return s; }
            P->tile_src_cap = cap;
        }
        ASFD_CUDA(cudaMemcpyAsync(P->tile_off, off.data(), sizeof(int) * (ntiles + 1),
                                  cudaMemcpyHostToDevice, st));
        if (!lst.empty())
            ASFD_CUDA(cudaMemcpyAsync(P->tile_src, lst.data(), sizeof(int) * lst.size(),
                                      cudaMemcpyHostToDevice, st));
        ASFD_CUDA(cudaStreamSynchronize(st));
        P->tile_pairs = (long long)lst.size();
    }
    if (P->learned && P->lfeat) {
        cs = learned_features(P, st);
        if (cs != ASFD_OK) return cs;
        return learned_refresh(P, st);
    }
    return ASFD_OK;
}

// Decides whether the conflict-free spreading kernel applies and, if so,
// builds its per-tile source rectangles.  Samples handled in one warp step
// must have disjoint footprints: two samples of one row `sx` columns apart
// are at least sx * min_step_x cells apart, two samples `h` rows apart (any
// columns) at least h * min_step_y - row_spread_y, where row_spread_y bounds
// the variation of the y coordinate along a row.  Both distances must reach
// the kernel width (plus a margin for FP32 rounding of the coordinates).
asfd_status plan_build_colored(asfd_plan_s* P, bool wraps, cudaStream_t st)
{
    const asfd_params& p = P->prm;
    P->colored = false;
    P->windowed = false;
    P->dense = false;
    P->itemtile = false;
    // a column per thread (blocks of 256 columns), rows in chunks, at most
    // kStepBlocks blocks
    static_assert((65536 + 255) / 256 <= kStepBlocks, "n1x <= 65536 fits one row of blocks");
    const int sgx = (p.n1x + 255) / 256;
    const int sgy = std::max(1, std::min(kStepBlocks / sgx, p.n1y));
    min_step_kernel<<<dim3(sgx, sgy), 256, 0, st>>>(P->q, P->ax, P->ay, P->bux, P->buy, p.n1x,
                                                    p.n1y, P->step_min);
    ASFD_CUDA(cudaGetLastError());
    const int nsb = sgx * sgy;
    std::vector<float> sm(2 * (size_t)nsb);
    ASFD_CUDA(cudaMemcpyAsync(sm.data(), P->step_min, sizeof(float) * sm.size(),
                              cudaMemcpyDeviceToHost, st));
    ASFD_CUDA(cudaStreamSynchronize(st));
    double msx = 3e38, msy = 3e38;
    for (int b = 0; b < nsb; ++b) {
        msx = std::min(msx, (double)sm[2 * b]);
        msy = std::min(msy, (double)sm[2 * b + 1]);
    }
    if (p.n1x < 2) msx = 1e30;
    if (p.n1y < 2) msy = 1e30;
    P->min_step_x = msx;
    P->min_step_y = msy;
    P->row_spread_y = 0.0;
    P->col_spread_x = 0.0;
    // the minimum spacing must clear FP32 rounding of the coordinates (~1e-6
    // cells) so that the first tap rows and columns are non-decreasing
    const bool monotone = !wraps && msx > 1e-3 && msy > 1e-3;
    if (monotone && P->w <= kMaxWindowWidth && !p.deterministic) {
        // register windows flushed to the fine grid with float atomics (the
        // fastest path, and the only efficient one for dense maps); runs of
        // dense_rows rows per lane, in whole waves of the resident warps
        const long long ncb = (p.n1x + 31) / 32;
        long long slots = 0;
        const asfd_status s = dense_spread_warp_slots(P->w, p.kind == ASFD_KERNEL_LEARNED, &slots);
        if (s != ASFD_OK) return s;
        const long long rows = window_run_rows(p.n1y, ncb, slots);
        P->dense_rows = (int)rows;
        P->dense_items = (int)(ncb * ((p.n1y + rows - 1) / rows));
        P->dense = true;
        return ASFD_OK;
    }
    if (!monotone || P->w > kMaxRingWidth) return ASFD_OK;

    // atomic-free tiles: row and column extents of the samples' coordinates
    col_range_kernel<<<(p.n1x + 31) / 32, 256, 0, st>>>(P->q, P->ax, P->bux, p.n1x, p.n1y,
                                                         P->col_range);
    row_range_kernel<<<p.n1y, 256, 0, st>>>(P->q, P->ay, P->buy, p.n1x, P->row_range);
    ASFD_CUDA(cudaGetLastError());
    std::vector<double> cr(2 * (size_t)p.n1x), rr(2 * (size_t)p.n1y);
    ASFD_CUDA(cudaMemcpyAsync(cr.data(), P->col_range, sizeof(double) * cr.size(),
                              cudaMemcpyDeviceToHost, st));
    ASFD_CUDA(cudaMemcpyAsync(rr.data(), P->row_range, sizeof(double) * rr.size(),
                              cudaMemcpyDeviceToHost, st));
    ASFD_CUDA(cudaStreamSynchronize(st));
    double spread_y = 0.0, spread_x = 0.0;
    for (int ny = 0; ny < p.n1y; ++ny) spread_y = std::max(spread_y, rr[2 * ny + 1] - rr[2 * ny]);
    for (int nx = 0; nx < p.n1x; ++nx) spread_x = std::max(spread_x, cr[2 * nx + 1] - cr[2 * nx]);
    P->row_spread_y = spread_y;
    P->col_spread_x = spread_x;
    const double margin = 0.01;
    const double sxd = std::ceil((P->w + margin) / msx);
    const double hd = std::ceil((P->w + spread_y + margin) / msy);
    // the register-window tiles also need columns w apart across rows
    const double sxw = std::ceil((P->w + spread_x + margin) / msx);
    // beyond 64 samples between lanes (samples packed far below one cell
    // apart) few lanes find work in a tile and the atomic kernel is faster
    if (!(sxd <= 64.0) || !(hd <= 64.0)) return ASFD_OK;

    // per band tile: source columns whose x range meets the tile's x range
    // widened by half a kernel and a cell, likewise rows (ranges are
    // monotone in the index because the spacing is positive)
    const double hw = 0.5 * P->w + 1.0;
    const int bntx = P->band_tx1 - P->band_tx0;
    const int bnty = (P->band_ty1 - P->band_ty0) * (kTileY / kColTileY);
    std::vector<int> xlo(bntx), xhi(bntx), ylo(bnty), yhi(bnty);
    auto first_hi_ge = [](const std::vector<double>& r, int n, double v) {
        int lo = 0, hi = n;  // first i with r[2i+1] >= v
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (r[2 * mid + 1] >= v) hi = mid; else lo = mid + 1;
        }
        return lo;
    };
    auto first_lo_ge = [](const std::vector<double>& r, int n, double v) {
        int lo = 0, hi = n;  // first i with r[2i] >= v
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (r[2 * mid] >= v) hi = mid; else lo = mid + 1;
        }
        return lo;
    };
    for (int i = 0; i < bntx; ++i) {
        const double o = (double)(P->band_tx0 + i) * kTileX;
        xlo[i] = first_hi_ge(cr, p.n1x, o - hw);
        xhi[i] = first_lo_ge(cr, p.n1x, o + kTileX + hw);
    }
    for (int i = 0; i < bnty; ++i) {
        const double o = (double)P->band_ty0 * kTileY + (double)i * kColTileY;
        ylo[i] = first_hi_ge(rr, p.n1y, o - hw);
        yhi[i] = first_lo_ge(rr, p.n1y, o + kColTileY + hw);
    }
    std::vector<int4> rect((size_t)bntx * bnty);
    for (int j = 0; j < bnty; ++j)
        for (int i = 0; i < bntx; ++i)
            rect[(size_t)j * bntx + i] = make_int4(xlo[i], std::max(xlo[i], xhi[i]), ylo[j],
                                                   std::max(ylo[j], yhi[j]));
    ASFD_CUDA(cudaMemcpyAsync(P->tile_rect, rect.data(), sizeof(int4) * rect.size(),
                              cudaMemcpyHostToDevice, st));
    ASFD_CUDA(cudaStreamSynchronize(st));
    P->sx_min = (int)sxd;
    P->h_min = (int)hd;
    P->colored = true;
    if (P->w <= kMaxWindowWidth) {
        P->sxw_min = (int)sxw;
        P->windowed = true;
    }
    // the faster atomic-free path where it applies (the tiles above stay
    // built: the batched kernel uses them)
    return plan_build_itemtile(P, st);
}

}  // namespace asfd
