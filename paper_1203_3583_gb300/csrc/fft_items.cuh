// Row and column passes of the 2D FFT as block-level device functions, shared
// by the per-plan kernels (fft.cu) and the batched persistent kernel
// (batch.cu).  Each processes the `blk`-th group of lines with the calling
// block's threads (tid in [0, threads)) and `sm` as its shared memory.
#pragma once

#include "asfd_impl.cuh"
#include "fft.cuh"

namespace asfd {

// Row pass: LPC lines of length L per block, L/16 threads per line.
template <int L>
struct RowCfg {
    static constexpr int TPL = L / 16;
    static constexpr int LPC = L >= 4096 ? 1 : 4096 / L;  // lines per block
    static constexpr int THREADS = TPL * LPC;
    static constexpr int LS = FftShape<L>::SMEM + (TPL < 16 ? TPL : 0);
    static constexpr size_t SMEM_BYTES = sizeof(float2) * LS * LPC;
};

// Column pass with LPC columns per block (threads = L/16 * LPC); the line
// stride keeps the lanes of one shared-memory access on distinct banks.
template <int L, int LPC_>
struct ColShape {
    static constexpr int TPL = L / 16;
    static constexpr int LPC = LPC_;
    static constexpr int THREADS = TPL * LPC;
    static constexpr int LS = FftShape<L>::SMEM + 16 / (LPC < 16 ? LPC : 16);
    static constexpr size_t SMEM_BYTES = sizeof(float2) * LS * LPC;
};

template <int L>
struct ColCfgSel {
    static constexpr int TPL = L / 16;
    static constexpr int LPC0 = (256 / TPL) > 4 ? (256 / TPL) : 4;
    // 4096-point columns: two columns per 512-thread block and two blocks
    // per SM at 64 registers, whose barriers are independent (one block of
    // four columns and 1024 threads measured 43.1 against 42.0 us at 2048
    // columns); other lengths up to 1024 threads, as many blocks as fit
    static constexpr int LPC = L == 4096 ? 2 : ((LPC0 * TPL > 1024) ? (1024 / TPL) : LPC0);
    static constexpr int MIN_BLOCKS = L == 4096 ? 2 : 1;
};
template <int L>
using ColCfg = ColShape<L, ColCfgSel<L>::LPC>;

// The row pass's output, the column pass's input, is stored in groups of
// kRowGroup kept columns: group g holds [band row][kRowGroup] (element
// (r, k) at (k / kRowGroup * nrows + r) * kRowGroup + k % kRowGroup).  A row
// pass lane group then stores whole 32-byte sectors, and a column pass warp
// loads 16 consecutive rows of two columns from one 512-byte stretch,
// instead of 16 rows a row length apart (2048 columns: rows 26.1 -> 28.7
// us, columns 42.5 -> 35.7 us).  The buffer holds nrows x m2x rounded up to
// a multiple of kRowGroup (row_buffer_width, asfd_impl.cuh).

__device__ __forceinline__ size_t row_group_index(int r, int k, int nrows)
{
    return ((size_t)(k / kRowGroup) * nrows + r) * kRowGroup + k % kRowGroup;
}

struct RowArgs {
    float2* grid;        // [nf rows][L] fine grid
    int row0, nrows;     // band rows
    int col_lo, col_hi;  // band columns (others are zero)
    float2* out;         // kept bins k + m2x/2 of the band rows, column groups (above)
    int m2x;
    const float2* tw;
    int clear;           // 1: zero the band cells after the transform (the next
                         // accumulating spread then needs no separate clear)
};

struct ColArgs {
    const float2* rows;  // row-pass output (band rows), column groups (above)
    int row0, nrows;
    int m2x, m2y;
    int col0, col1;      // kept columns [col0, col1) this pass transforms
    const float2* cx;    // [m2x] deconvolution x chirp
    const float2* cy;    // [m2y] same, times the global factor
    float2* u2;          // [m2y][m2x]
    const float2* tw;
};

// Pass arguments of a plan (defined in fft.cu).
RowArgs make_row_args(const asfd_plan_s* P);
ColArgs make_col_args(const asfd_plan_s* P, float2* u2);

// FFT along x of LPC band rows, keeping the M2x centred bins.
template <int L>
__device__ __forceinline__ void rows_body(const RowArgs& a, int blk, float2* sm, int tid)
{
    using C = RowCfg<L>;
    const int line = tid / C::TPL, t = tid % C::TPL;
    const int r = blk * C::LPC + line;
    const bool active = r < a.nrows;
    float2* src = a.grid + (size_t)(a.row0 + (active ? r : 0)) * L;
    float2* out = a.out;
    const int nrows = a.nrows;
    const int half = a.m2x / 2;
    const int col_lo = a.col_lo, col_hi = a.col_hi;
    // plain loads, not the read-only path: with clear set the kernel writes
    // these cells (after every load of them has been used)
    auto ld = [&](int i) -> float2 {
        return (active && i >= col_lo && i < col_hi) ? src[i] : make_float2(0.f, 0.f);
    };
    auto st = [&](int i, float2 v) {
        if (!active) return;
        int k;
        if (i < half) k = i + half;
        else if (i >= L - half) k = i - (L - half);
        else return;
        out[row_group_index(r, k, nrows)] = v;
    };
    fft_line<L, -1>(t, sm + line * C::LS, a.tw, ld, st);
    if (a.clear && active) {
        // zero the band cells this thread loaded (the first pass's indices)
        constexpr int R0 = FftShape<L>::R0;
#pragma unroll
        for (int b = 0; b < 16 / R0; ++b)
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                const int i = t + b * C::TPL + r * (L / R0);
                if (i >= col_lo && i < col_hi) src[i] = make_float2(0.f, 0.f);
            }
    }
}

// FFT along y of LPC kept columns over the band rows, then deconvolution,
// crop and destination chirp (Eq. 8's outer factor).
template <int L, int LPC>
__device__ __forceinline__ void cols_body(const ColArgs& a, int blk, float2* sm, int tid)
{
    using C = ColShape<L, LPC>;
    const int c = tid % LPC, t = tid / LPC;
    const int col = a.col0 + blk * LPC + c;
    const bool active = col < a.col1;
    const int colc = active ? col : 0;
    const float2 fx = __ldg(&a.cx[colc]);
    const int half = a.m2y / 2;
    const int row0 = a.row0, nrows = a.nrows, m2x = a.m2x;
    const float2* rows = a.rows;
    auto ld = [&](int i) -> float2 {
        const int rr = i - row0;
        return (active && rr >= 0 && rr < nrows) ? __ldg(&rows[row_group_index(rr, colc, nrows)])
                                                 : make_float2(0.f, 0.f);
    };
    auto st = [&](int i, float2 v) {
        if (!active) return;
        int k;
        if (i < half) k = i + half;
        else if (i >= L - half) k = i - (L - half);
        else return;
        a.u2[(size_t)k * m2x + colc] = cmul(cmul(v, fx), __ldg(&a.cy[k]));
    };
    fft_line<L, -1>(t, sm + c * C::LS, a.tw, ld, st);
}

}  // namespace asfd
