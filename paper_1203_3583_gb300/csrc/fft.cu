// Uniform-FFT stages of the type-1 NUFFT (Sec. 2, after Eq. 9) and the
// final scaling of Eq. 8.
//
//   rows:  for each touched fine-grid row, FFT along x (e^{-i}), keeping the
//          M2x centred bins k in [-M2x/2, M2x/2) in the order k + M2x/2.
//          Columns outside the spread band are zero and are not read.
//   cols:  for each kept column, FFT along y over the touched rows (the
//          rest are zero), keep the M2y centred bins and multiply by the
//          separable factor Cx[kx] Cy[ky] that holds the kernel
//          deconvolution 1/psi_hat, the (-1)^k of the centred fine-grid
//          storage, the destination chirp exp(ik|x2|^2/(2 z0)) and, in Cy,
//          the global factor exp(ik z0) p1x p1y / (i lambda z0).
#include <mutex>

#include "asfd_impl.cuh"
#include "fft.cuh"
#include "fft_items.cuh"

namespace asfd {

namespace {

// (4096-point rows: at most 64 registers, four 256-thread blocks per SM)
template <int L>
__global__ void __launch_bounds__(RowCfg<L>::THREADS, L == 4096 ? 4 : 1)
fft_rows_kernel(RowArgs a)
{
    extern __shared__ float2 sm[];
    rows_body<L>(a, blockIdx.x, sm, threadIdx.x);
}

template <int L>
__global__ void __launch_bounds__(ColCfg<L>::THREADS, ColCfgSel<L>::MIN_BLOCKS)
fft_cols_kernel(ColArgs a)
{
    extern __shared__ float2 sm[];
    cols_body<L, ColCfg<L>::LPC>(a, blockIdx.x, sm, threadIdx.x);
}

// Adjoint column pass: h = conj(Cx Cy) gu2 placed at the kept bins, FFT with
// e^{+i} along y, band rows [row0, row0 + nrows) stored to rows[s - row0][kx].
template <int L>
__global__ void __launch_bounds__(ColCfg<L>::THREADS, ColCfgSel<L>::MIN_BLOCKS)
fft_cols_adj_kernel(const float2* __restrict__ g, int m2x, int m2y, const float2* __restrict__ cx,
                    const float2* __restrict__ cy, float2* __restrict__ rows, int row0, int nrows,
                    const float2* __restrict__ tw)
{
    using C = ColCfg<L>;
    extern __shared__ float2 sm[];
    const int c = threadIdx.x % C::LPC, t = threadIdx.x / C::LPC;
    const int col = blockIdx.x * C::LPC + c;
    const bool active = col < m2x;
    const int colc = active ? col : 0;
    const float2 fx = __ldg(&cx[colc]);
    const int half = m2y / 2;
    auto ld = [&](int i) -> float2 {
        int k;
        if (i < half) k = i + half;
        else if (i >= L - half) k = i - (L - half);
        else return make_float2(0.f, 0.f);
        if (!active) return make_float2(0.f, 0.f);
        // conj(fx * cy[k]) * g
        return cmulc(cmulc(__ldg(&g[(size_t)k * m2x + colc]), fx), __ldg(&cy[k]));
    };
    auto st = [&](int i, float2 v) {
        const int rr = i - row0;
        if (active && rr >= 0 && rr < nrows) rows[(size_t)rr * m2x + colc] = v;
    };
    fft_line<L, 1>(t, sm + c * C::LS, tw, ld, st);
}

// Adjoint row pass: band row r of rows[][] placed at the kept bins, FFT with
// e^{+i} along x, band columns [col_lo, col_hi) stored to the fine grid.
template <int L>
__global__ void __launch_bounds__(RowCfg<L>::THREADS)
fft_rows_adj_kernel(const float2* __restrict__ rows, int nrows, int m2x, float2* __restrict__ grid,
                    int row0, int col_lo, int col_hi, const float2* __restrict__ tw)
{
    using C = RowCfg<L>;
    extern __shared__ float2 sm[];
    const int line = threadIdx.x / C::TPL, t = threadIdx.x % C::TPL;
    const int r = blockIdx.x * C::LPC + line;
    const bool active = r < nrows;
    const float2* src = rows + (size_t)(active ? r : 0) * m2x;
    float2* dst = grid + (size_t)(row0 + (active ? r : 0)) * L;
    const int half = m2x / 2;
    auto ld = [&](int i) -> float2 {
        if (!active) return make_float2(0.f, 0.f);
        if (i < half) return __ldg(&src[i + half]);
        if (i >= L - half) return __ldg(&src[i - (L - half)]);
        return make_float2(0.f, 0.f);
    };
    auto st = [&](int i, float2 v) {
        if (active && i >= col_lo && i < col_hi) dst[i] = v;
    };
    fft_line<L, 1>(t, sm + line * C::LS, tw, ld, st);
}

template <int L, int S>
__global__ void __launch_bounds__(RowCfg<L>::THREADS)
fft_lines_kernel(const float2* in, float2* out, int lines, const float2* __restrict__ tw)
{
    using C = RowCfg<L>;
    extern __shared__ float2 sm[];
    const int line = threadIdx.x / C::TPL, t = threadIdx.x % C::TPL;
    const int r = blockIdx.x * C::LPC + line;
    const bool active = r < lines;
    const float2* src = in + (size_t)(active ? r : 0) * L;
    float2* dst = out + (size_t)(active ? r : 0) * L;
    auto ld = [&](int i) -> float2 { return active ? src[i] : make_float2(0.f, 0.f); };
    auto st = [&](int i, float2 v) {
        if (active) dst[i] = v;
    };
    fft_line<L, S>(t, sm + line * C::LS, tw, ld, st);
}

template <class F>
cudaError_t set_smem(F* f, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int L>
cudaError_t rows_L(const RowArgs& a, cudaStream_t st)
{
    using C = RowCfg<L>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] { attr = set_smem(fft_rows_kernel<L>, C::SMEM_BYTES); });
    if (attr != cudaSuccess) return attr;
    const int blocks = (a.nrows + C::LPC - 1) / C::LPC;
    fft_rows_kernel<L><<<blocks, C::THREADS, C::SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

template <int L>
cudaError_t cols_L(const ColArgs& a, cudaStream_t st)
{
    using C = ColCfg<L>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] { attr = set_smem(fft_cols_kernel<L>, C::SMEM_BYTES); });
    if (attr != cudaSuccess) return attr;
    const int blocks = (a.col1 - a.col0 + C::LPC - 1) / C::LPC;
    if (blocks <= 0) return cudaSuccess;
    fft_cols_kernel<L><<<blocks, C::THREADS, C::SMEM_BYTES, st>>>(a);
    return cudaGetLastError();
}

template <int L>
cudaError_t cols_adj_L(const float2* g, int m2x, int m2y, const float2* cx, const float2* cy,
                       float2* rows, int row0, int nrows, const float2* tw, cudaStream_t st)
{
    using C = ColCfg<L>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] { attr = set_smem(fft_cols_adj_kernel<L>, C::SMEM_BYTES); });
    if (attr != cudaSuccess) return attr;
    const int blocks = (m2x + C::LPC - 1) / C::LPC;
    fft_cols_adj_kernel<L><<<blocks, C::THREADS, C::SMEM_BYTES, st>>>(g, m2x, m2y, cx, cy, rows,
                                                                      row0, nrows, tw);
    return cudaGetLastError();
}

template <int L>
cudaError_t rows_adj_L(const float2* rows, int nrows, int m2x, float2* grid, int row0, int col_lo,
                       int col_hi, const float2* tw, cudaStream_t st)
{
    using C = RowCfg<L>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] { attr = set_smem(fft_rows_adj_kernel<L>, C::SMEM_BYTES); });
    if (attr != cudaSuccess) return attr;
    const int blocks = (nrows + C::LPC - 1) / C::LPC;
    fft_rows_adj_kernel<L><<<blocks, C::THREADS, C::SMEM_BYTES, st>>>(rows, nrows, m2x, grid, row0,
                                                                      col_lo, col_hi, tw);
    return cudaGetLastError();
}

template <int L, int S>
cudaError_t lines_L(const float2* in, float2* out, int lines, const float2* tw, cudaStream_t st)
{
    using C = RowCfg<L>;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] { attr = set_smem(fft_lines_kernel<L, S>, C::SMEM_BYTES); });
    if (attr != cudaSuccess) return attr;
    const int blocks = (lines + C::LPC - 1) / C::LPC;
    fft_lines_kernel<L, S><<<blocks, C::THREADS, C::SMEM_BYTES, st>>>(in, out, lines, tw);
    return cudaGetLastError();
}

#define ASFD_FFT_SWITCH(n, CALL)       \
    switch (n) {                       \
        case 16: CALL(16); break;      \
        case 32: CALL(32); break;      \
        case 64: CALL(64); break;      \
        case 128: CALL(128); break;    \
        case 256: CALL(256); break;    \
        case 512: CALL(512); break;    \
        case 1024: CALL(1024); break;  \
        case 2048: CALL(2048); break;  \
        case 4096: CALL(4096); break;  \
        case 8192: CALL(8192); break;  \
        case 16384: CALL(16384); break; \
        default: e = cudaErrorInvalidValue; \
    }

// FP64-built twiddle tables e^{-2 pi i k/L}, one per length, cached per device.
__global__ void twiddle_kernel(float2* tw, int L)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)L, &s, &c);
    tw[k] = make_float2((float)c, (float)-s);
}

}  // namespace

RowArgs make_row_args(const asfd_plan_s* P)
{
    RowArgs a;
    a.grid = P->grid;
    a.row0 = P->band_ty0 * kTileY;
    a.nrows = (P->band_ty1 - P->band_ty0) * kTileY;
    a.col_lo = P->band_tx0 * kTileX;
    a.col_hi = P->band_tx1 * kTileX;
    a.out = P->rows;
    a.m2x = P->prm.m2x;
    a.tw = P->twx;
    a.clear = 0;
    return a;
}

ColArgs make_col_args(const asfd_plan_s* P, float2* u2)
{
    ColArgs a;
    a.rows = P->rows;
    a.row0 = P->band_ty0 * kTileY;
    a.nrows = (P->band_ty1 - P->band_ty0) * kTileY;
    a.m2x = P->prm.m2x;
    a.m2y = P->prm.m2y;
    a.col0 = 0;
    a.col1 = P->prm.m2x;
    a.cx = P->cx;
    a.cy = P->cy;
    a.u2 = u2;
    a.tw = P->twy;
    return a;
}

asfd_status launch_fft_rows(asfd_plan_s* P, cudaStream_t st)
{
    RowArgs a = make_row_args(P);
    if (a.nrows <= 0) return ASFD_OK;
    // for the accumulating (dense) spread the pass leaves the band zero: each
    // thread zeroes the band cells it loaded once its transform is done
    // (2176^2 band at 2048^2: +1.8 us here against 7.5 us for a separate clear)
    a.clear = P->dense ? 1 : 0;
    cudaError_t e = cudaSuccess;
#define ASFD_ROWS(L) e = rows_L<L>(a, st)
    ASFD_FFT_SWITCH(P->nfx, ASFD_ROWS)
#undef ASFD_ROWS
    if (e != cudaSuccess) return cuda_fail(e, "fft_rows_kernel launch");
    P->band_clean = P->dense;
    return ASFD_OK;
}

asfd_status launch_fft_cols(asfd_plan_s* P, float2* u2, cudaStream_t st)
{
    const ColArgs a = make_col_args(P, u2);
    cudaError_t e = cudaSuccess;
#define ASFD_COLS(L) e = cols_L<L>(a, st)
    ASFD_FFT_SWITCH(P->nfy, ASFD_COLS)
#undef ASFD_COLS
    if (e != cudaSuccess) return cuda_fail(e, "fft_cols_kernel launch");
    return ASFD_OK;
}

asfd_status launch_fft_cols_range(asfd_plan_s* P, float2* u2, int col0, int col1,
                                  cudaStream_t st)
{
    ColArgs a = make_col_args(P, u2);
    a.col0 = col0;
    a.col1 = col1;
    cudaError_t e = cudaSuccess;
#define ASFD_COLS(L) e = cols_L<L>(a, st)
    ASFD_FFT_SWITCH(P->nfy, ASFD_COLS)
#undef ASFD_COLS
    if (e != cudaSuccess) return cuda_fail(e, "fft_cols_kernel launch");
    return ASFD_OK;
}

asfd_status launch_fft_rows_band(asfd_plan_s* P, int ty0, int ty1, int tx0, int tx1,
                                 cudaStream_t st)
{
    RowArgs a = make_row_args(P);
    a.row0 = ty0 * kTileY;
    a.nrows = (ty1 - ty0) * kTileY;
    a.col_lo = tx0 * kTileX;
    a.col_hi = tx1 * kTileX;
    if (a.nrows <= 0) return ASFD_OK;
    a.clear = 1;
    cudaError_t e = cudaSuccess;
#define ASFD_ROWS(L) e = rows_L<L>(a, st)
    ASFD_FFT_SWITCH(P->nfx, ASFD_ROWS)
#undef ASFD_ROWS
    if (e != cudaSuccess) return cuda_fail(e, "fft_rows_kernel launch");
    // the given band contains the plan's own band (a sum over several plans)
    P->band_clean = true;
    return ASFD_OK;
}

asfd_status launch_fft_cols_band(asfd_plan_s* P, int ty0, int ty1, float2* u2, cudaStream_t st)
{
    ColArgs a = make_col_args(P, u2);
    a.row0 = ty0 * kTileY;
    a.nrows = (ty1 - ty0) * kTileY;
    cudaError_t e = cudaSuccess;
#define ASFD_COLS(L) e = cols_L<L>(a, st)
    ASFD_FFT_SWITCH(P->nfy, ASFD_COLS)
#undef ASFD_COLS
    if (e != cudaSuccess) return cuda_fail(e, "fft_cols_kernel launch");
    return ASFD_OK;
}

asfd_status launch_fft_cols_adj(asfd_plan_s* P, const float2* g, cudaStream_t st)
{
    const int row0 = P->band_ty0 * kTileY;
    const int nrows = (P->band_ty1 - P->band_ty0) * kTileY;
    cudaError_t e = cudaSuccess;
#define ASFD_CA(L) e = cols_adj_L<L>(g, P->prm.m2x, P->prm.m2y, P->cx, P->cy, P->rows, row0, nrows, P->twy, st)
    ASFD_FFT_SWITCH(P->nfy, ASFD_CA)
#undef ASFD_CA
    if (e != cudaSuccess) return cuda_fail(e, "fft_cols_adj_kernel launch");
    return ASFD_OK;
}

asfd_status launch_fft_rows_adj(asfd_plan_s* P, cudaStream_t st)
{
    const int row0 = P->band_ty0 * kTileY;
    const int nrows = (P->band_ty1 - P->band_ty0) * kTileY;
    const int col_lo = P->band_tx0 * kTileX, col_hi = P->band_tx1 * kTileX;
    if (nrows <= 0) return ASFD_OK;
    cudaError_t e = cudaSuccess;
#define ASFD_RA(L) e = rows_adj_L<L>(P->rows, nrows, P->prm.m2x, P->grid, row0, col_lo, col_hi, P->twx, st)
    ASFD_FFT_SWITCH(P->nfx, ASFD_RA)
#undef ASFD_RA
    P->band_clean = false;  // the band now holds the adjoint grid
    if (e != cudaSuccess) return cuda_fail(e, "fft_rows_adj_kernel launch");
    return ASFD_OK;
}

asfd_status build_twiddles(float2* tw, int L, cudaStream_t st)
{
    twiddle_kernel<<<(L + 255) / 256, 256, 0, st>>>(tw, L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "twiddle_kernel launch");
    return ASFD_OK;
}

asfd_status launch_fft_lines_tw(int n, int lines, int sign, const float2* in, float2* out,
                                const float2* tw, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (sign < 0) {
#define ASFD_LTN(L) e = lines_L<L, -1>(in, out, lines, tw, st)
        ASFD_FFT_SWITCH(n, ASFD_LTN)
#undef ASFD_LTN
    } else {
#define ASFD_LTP(L) e = lines_L<L, 1>(in, out, lines, tw, st)
        ASFD_FFT_SWITCH(n, ASFD_LTP)
#undef ASFD_LTP
    }
    if (e != cudaSuccess) return cuda_fail(e, "fft_lines_kernel launch");
    return ASFD_OK;
}

asfd_status launch_fft_lines(int n, int lines, int sign, const float2* in, float2* out,
                             cudaStream_t st)
{
    if (n < 16 || n > 16384 || (n & (n - 1)) || lines < 0 || (sign != 1 && sign != -1) ||
        (lines > 0 && (!in || !out)))
        return fail(ASFD_ERR_ARG, "asfd_fft_lines: n must be a power of two in [16, 16384], "
                                  "sign +-1, non-NULL buffers");
    if (lines == 0) return ASFD_OK;
    // one twiddle table per (device, length), built on first use
    static std::mutex mu;
    static float2* tables[64][15] = {};
    int dev = 0;
    ASFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(ASFD_ERR_UNSUPPORTED, "device ordinal above 63");
    const int lg = ilog2_c(n);
    float2* tw = nullptr;
    {
        std::lock_guard<std::mutex> g(mu);
        if (!tables[dev][lg]) {
            float2* p = nullptr;
            ASFD_CUDA(cudaMalloc(&p, sizeof(float2) * n));
            asfd_status s = build_twiddles(p, n, st);
            if (s != ASFD_OK) {
                cudaFree(p);
                return s;
            }
            ASFD_CUDA(cudaStreamSynchronize(st));
            tables[dev][lg] = p;
        }
        tw = tables[dev][lg];
    }
    cudaError_t e = cudaSuccess;
    if (sign < 0) {
#define ASFD_LN(L) e = lines_L<L, -1>(in, out, lines, tw, st)
        ASFD_FFT_SWITCH(n, ASFD_LN)
#undef ASFD_LN
    } else {
#define ASFD_LP(L) e = lines_L<L, 1>(in, out, lines, tw, st)
        ASFD_FFT_SWITCH(n, ASFD_LP)
#undef ASFD_LP
    }
    if (e != cudaSuccess) return cuda_fail(e, "fft_lines_kernel launch");
    return ASFD_OK;
}

}  // namespace asfd
