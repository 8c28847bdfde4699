// Per-sample prefactor fused with the tiled type-1 spread (Sec. 2, Eqs. 7-9).
//
// Sample n = (nx, ny) carries
//   c_n = u1[n] * exp(ik d1) * exp(ik(-d1 + |x1|^2/(2 r0)))
// and sits at the non-uniform frequency t = k p2 x1 / r0 (per axis), i.e. at
// the fine-grid coordinate g = t nf/(2 pi) = alpha x~ (1 + q), with
// alpha = p1 p2 nf/(lambda z0), x~ = n - N/2 and q = d1/(z0 - d1).
//
// Phase split (the large phases are formed and reduced in FP64 by the plan):
//   exp(ik d1) exp(-ik d1) = 1 exactly for the normally incident plane wave,
//   k|x1|^2/(2 r0) = pi a (1 + q),  a = |x1|^2/(lambda z0) = a_x + a_y,
// so c_n = u1 * E_x[nx] E_y[ny] * exp(i pi (a_x + a_y) q), where the tables
// E = exp(i pi a) were built and reduced mod 2 pi in FP64 and only the
// correction pi a q is evaluated per sample, in FP32 with sincospif.  Its
// absolute error is about 2^-23 (a q + a |q|), e.g. 1e-7 rad at a = 500
// half-turns and q = 5e-4; it grows linearly with q, which the plan bounds
// by |d1|/z0 <= 0.1.  Likewise g = (bi + bf) + s q with the FP64-built
// integer/fraction split of alpha x~ + nf/2 and s = alpha x~, so the FP32
// error of g is that of the small term s q (about 1e-7 cells at the standard
// workloads) rather than that of g itself.
//
// Both kernels own fine-grid tiles (storage coordinates, centred: cell index
// = g + nf/2 mod nf): each CTA accumulates in shared memory every tap of
// every sample whose footprint reaches its tile, and writes the tile to
// global memory once.  No global atomics.
//
//  * spread_es_colored_kernel (the fast path): one warp per tile, plain
//    shared-memory read-modify-write without atomics.  The plan proves that
//    the footprints of the 32 samples a warp handles in one step are
//    pairwise disjoint: lanes form 4 row groups x 8 column groups; lanes of
//    one row group take samples of the same source row at least Sx columns
//    apart, row groups take rows at least H apart, where Sx and H follow from
//    the minimum spacing of the samples on the fine grid (the map n -> g is
//    monotone for a non-folding surface).  A __syncwarp separates steps.
//  * spread_es_window_kernel (widths up to kMaxWindowWidth, same lanes):
//    each lane walks its samples down a source column and keeps their taps
//    in a sliding W x W register window, so that shared memory sees about
//    one row of W updates per sample instead of W rows.
//  * spread_es_atomic_kernel (fallback for folding or wrapping maps):
//    256 threads, one sample per thread, shared-memory atomics.
#include "spread.cuh"

namespace asfd {

namespace {

template <int W, bool TAB>
__global__ void __launch_bounds__(256) spread_es_atomic_kernel(SpreadArgs a)
{
    __shared__ float tre[kTileY * kTileX];
    __shared__ float tim[kTileY * kTileX];
    atomic_tile<W, TAB>(a, blockIdx.x, tre, tim, threadIdx.x, blockDim.x);
}

// The dense kernels accumulate with atomic adds into a zero band: clear it
// first unless the previous row pass left it zero, then launch.
template <int W, bool TAB>
cudaError_t launch_dense(const SpreadArgs& a, int tiles, bool clear, cudaStream_t st)
{
    if (clear) {
        const size_t pitch = sizeof(float2) * (size_t)a.nfx;
        const int c0 = a.band_tx0 * kTileX, r0 = a.band_ty0 * kTileY;
        const size_t width = sizeof(float2) * (size_t)a.band_ntx * kTileX;
        const size_t height = (size_t)(tiles / a.band_ntx) * kTileY;
        const cudaError_t e =
            cudaMemset2DAsync(a.grid + (size_t)r0 * a.nfx + c0, pitch, 0, width, height, st);
        if (e != cudaSuccess) return e;
    }
    spread_es_dense_kernel<W, TAB><<<(a.dense_items + kDenseWarps - 1) / kDenseWarps,
                                     32 * kDenseWarps, 0, st>>>(a, a.dense_items);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_w(const SpreadArgs& a, int tiles, bool colored, bool windowed, bool clear,
                     cudaStream_t st)
{
    if constexpr (W <= kMaxWindowWidth) {
        if (a.dense_rows > 0) return launch_dense<W, false>(a, tiles, clear, st);
        if (windowed) {
            spread_es_window_kernel<W, kTileX, kColTileY, false>
                <<<tiles * (kTileY / kColTileY), 32, 0, st>>>(a);
            return cudaGetLastError();
        }
    }
    // widths up to kMaxRingWidth compile without register spills
    if constexpr (W <= kMaxRingWidth) {
        if (colored) {
            spread_es_colored_kernel<W, kTileX, kColTileY, false>
                <<<tiles * (kTileY / kColTileY), 32, 0, st>>>(a);
            return cudaGetLastError();
        }
    }
    spread_es_atomic_kernel<W, false><<<tiles, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_table(const SpreadArgs& a, int tiles, bool colored, bool clear, cudaStream_t st)
{
    if (a.dense_rows > 0) return launch_dense<kLearnW, true>(a, tiles, clear, st);
    if (colored)
        spread_es_colored_kernel<kLearnW, kTileX, kColTileY, true>
            <<<tiles * (kTileY / kColTileY), 32, 0, st>>>(a);
    else
        spread_es_atomic_kernel<kLearnW, true><<<tiles, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

namespace {

asfd_status resident_warps(const void* kernel, long long* slots)
{
    int dev = 0, sms = 0, per_sm = 0;
    ASFD_CUDA(cudaGetDevice(&dev));
    ASFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ASFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * kDenseWarps, 0));
    *slots = (long long)sms * std::max(per_sm, 1) * kDenseWarps;
    return ASFD_OK;
}

}  // namespace

asfd_status dense_spread_warp_slots(int w, bool table, long long* slots)
{
    if (table) return resident_warps((const void*)spread_es_dense_kernel<kLearnW, true>, slots);
    switch (w) {
#define ASFD_SW(W) case W: return resident_warps((const void*)spread_es_dense_kernel<W, false>, slots);
        ASFD_SW(2) ASFD_SW(3) ASFD_SW(4) ASFD_SW(5) ASFD_SW(6) ASFD_SW(7)
#undef ASFD_SW
        default: return fail(ASFD_ERR_UNSUPPORTED, "dense spread widths are 2..7");
    }
}

int window_run_rows(long long n1y, long long ncb, long long slots)
{
    // A run's window starts empty and ends with a flush of all its cells, so
    // runs shorter than about 32 rows pay for that twice as often; uniform
    // items in whole waves avoid a partly filled last wave.
    const auto rows_for = [&](long long waves) {
        const long long runs = std::max<long long>(1, waves * slots / std::max<long long>(ncb, 1));
        return (n1y + runs - 1) / runs;
    };
    long long rows = rows_for(2);
    if (rows < 32) rows = rows_for(1);
    return (int)std::max<long long>(8, std::min<long long>(1024, rows));
}

SpreadArgs make_spread_args(const asfd_plan_s* P, const float2* u1)
{
    SpreadArgs a;
    a.u1 = u1;
    a.q = P->q;
    a.ax = P->ax;
    a.ay = P->ay;
    a.px = P->px;
    a.py = P->py;
    a.tile_off = P->tile_off;
    a.tile_src = P->tile_src;
    a.tile_rect = P->tile_rect;
    a.grid = P->grid;
    a.n1x = P->prm.n1x;
    a.n1y = P->prm.n1y;
    a.nfx = P->nfx;
    a.nfy = P->nfy;
    a.nstx = P->nstx;
    a.band_tx0 = P->band_tx0;
    a.band_ty0 = P->band_ty0;
    a.band_ntx = P->band_tx1 - P->band_tx0;
    a.sx_min = P->sx_min;
    a.h_min = P->h_min;
    a.sxw_min = P->sxw_min;
    a.dense_rows = P->dense ? P->dense_rows : 0;
    a.dense_items = P->dense ? P->dense_items : 0;
    a.inc_d = (float)P->inc_d;
    a.half_w = 0.5f * (float)P->w;
    a.beta_log2e = (float)(P->beta * 1.4426950408889634074);
    a.two_over_w = (float)(2.0 / P->w);
    a.table = P->ltab;
    return a;
}

asfd_status launch_spread_into(asfd_plan_s* P, const float2* u1, float2* grid, cudaStream_t st)
{
    if (!P->dense) return fail(ASFD_ERR_UNSUPPORTED, "accumulating spread needs a dense plan");
    SpreadArgs a = make_spread_args(P, u1);
    a.grid = grid;
    if (a.dense_items <= 0) return ASFD_OK;
    cudaError_t e = cudaSuccess;
    if (P->learned) {
        spread_es_dense_kernel<kLearnW, true><<<(a.dense_items + kDenseWarps - 1) / kDenseWarps,
                                               32 * kDenseWarps, 0, st>>>(a, a.dense_items);
    } else {
        switch (P->w) {
#define ASFD_SI(W) case W: spread_es_dense_kernel<W, false><<<(a.dense_items + kDenseWarps - 1) / kDenseWarps, 32 * kDenseWarps, 0, st>>>(a, a.dense_items); break;
            ASFD_SI(2) ASFD_SI(3) ASFD_SI(4) ASFD_SI(5) ASFD_SI(6) ASFD_SI(7)
#undef ASFD_SI
            default: return fail(ASFD_ERR_UNSUPPORTED, "dense spread widths are 2..7");
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "spread kernel launch");
    return ASFD_OK;
}

asfd_status launch_spread(asfd_plan_s* P, const float2* u1, cudaStream_t st)
{
    const SpreadArgs a = make_spread_args(P, u1);
    const int tiles = (P->band_tx1 - P->band_tx0) * (P->band_ty1 - P->band_ty0);
    if (tiles <= 0) return ASFD_OK;
    const bool colored = P->colored;
    const bool windowed = P->colored && P->windowed;
    // the accumulating (dense) kernels need a zero band; the tile kernels
    // overwrite every band cell
    const bool clear = !P->band_clean;
    P->band_clean = false;
    if (P->itemtile) return launch_spread_itemtile(P, u1, st);
    cudaError_t e;
    if (P->learned) {
        e = launch_table(a, tiles, colored, clear, st);
        if (e != cudaSuccess) return cuda_fail(e, "learned spread kernel launch");
        return ASFD_OK;
    }
    switch (P->w) {
        case 2: e = launch_w<2>(a, tiles, colored, windowed, clear, st); break;
        case 3: e = launch_w<3>(a, tiles, colored, windowed, clear, st); break;
        case 4: e = launch_w<4>(a, tiles, colored, windowed, clear, st); break;
        case 5: e = launch_w<5>(a, tiles, colored, windowed, clear, st); break;
        case 6: e = launch_w<6>(a, tiles, colored, windowed, clear, st); break;
        case 7: e = launch_w<7>(a, tiles, colored, windowed, clear, st); break;
        case 8: e = launch_w<8>(a, tiles, colored, windowed, clear, st); break;
        case 9: e = launch_w<9>(a, tiles, colored, windowed, clear, st); break;
        case 10: e = launch_w<10>(a, tiles, colored, windowed, clear, st); break;
        case 11: e = launch_w<11>(a, tiles, colored, windowed, clear, st); break;
        case 12: e = launch_w<12>(a, tiles, colored, windowed, clear, st); break;
        case 13: e = launch_w<13>(a, tiles, colored, windowed, clear, st); break;
        case 14: e = launch_w<14>(a, tiles, colored, windowed, clear, st); break;
        case 15: e = launch_w<15>(a, tiles, colored, windowed, clear, st); break;
        case 16: e = launch_w<16>(a, tiles, colored, windowed, clear, st); break;
        default: return fail(ASFD_ERR_UNSUPPORTED, "kernel width outside 2..16");
    }
    if (e != cudaSuccess) return cuda_fail(e, "spread kernel launch");
    return ASFD_OK;
}

}  // namespace asfd
