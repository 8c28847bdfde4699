// Spreading kernels shared by the per-plan launches and the batched
// persistent kernel: the argument block, the kernel weights and the
// conflict-free per-warp tile spread.  See spread.cu for the method.
#pragma once

#include "asfd_impl.cuh"
#include "sample.cuh"

namespace asfd {

struct SpreadArgs {
    const float2* u1;
    const float* q;
    const AxisEntry* ax;
    const AxisEntry* ay;
    const AxisPos* px;
    const AxisPos* py;
    const int* tile_off;
    const int* tile_src;
    const int4* tile_rect;
    float2* grid;
    int n1x, n1y;
    int nfx, nfy;
    int nstx;
    int band_tx0, band_ty0, band_ntx;
    int sx_min, h_min;
    int sxw_min;       // column stride of the register-window kernel
    float half_w;      // w/2
    float beta_log2e;  // beta * log2(e)
    float two_over_w;  // 2/w
    const float* table;  // learned kernel: per-source-tile polynomial tables (or NULL)
};

// Kernel weights of the W taps in x and y: the ES kernel, or the learned
// per-source-tile polynomial table of the sample's source tile.
template <int W, bool TAB>
__device__ __forceinline__ void tap_weights(const SpreadArgs& a, int nx, int ny, float dx, float dy,
                                            float (&wx)[W], float (&wy)[W])
{
    if constexpr (TAB) {
        const int tile = (ny / kSrcTile) * a.nstx + nx / kSrcTile;
        table_weights<W>(a.table + (size_t)tile * kLearnTableSize, dx, dy, wx, wy);
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) {
            wx[i] = es_weight_fast(dx + (float)i - a.half_w, a.two_over_w, a.beta_log2e);
            wy[i] = es_weight_fast(dy + (float)i - a.half_w, a.two_over_w, a.beta_log2e);
        }
    }
}

// Conflict-free spreading: one warp per tile, plain shared-memory
// read-modify-write.  Lanes form 4 row groups x 8 column groups; at step
// (j, o) lane (lr, lc) takes sample (x0 + lc sx + o, y0 + lr h + j).  The
// plan's strides make the footprints of the 32 samples of one step pairwise
// disjoint (same row: sx columns apart, different rows: h rows apart), so the
// 49 taps of a lane are loaded, updated and stored as independent operations,
// and a __syncwarp orders consecutive steps.  The inputs of the next step are
// loaded while the current one is processed.
template <int TX, int TY>
struct ColoredTile {
    static constexpr int LD = TX + 4;  // padded row stride (complex slots)
    static constexpr int SLOTS = TY * LD;
};

// One warp spreads every sample of tile t of the band (TX x TY cells) into
// `tile` (ColoredTile<TX, TY>::SLOTS complex slots of shared memory) and
// writes the tile to the fine grid.  All 32 lanes of the warp must call it.
template <int W, int TX, int TY, bool TAB>
__device__ __forceinline__ void colored_tile(const SpreadArgs& a, int t, float2* tile, int lane)
{
    constexpr int LD = ColoredTile<TX, TY>::LD;
    const int ox = (a.band_tx0 + t % a.band_ntx) * TX;
    const int oy = a.band_ty0 * kTileY + (t / a.band_ntx) * TY;

    for (int i = lane; i < TY * LD; i += 32) tile[i] = make_float2(0.f, 0.f);
    __syncwarp();

    const int4 rc = a.tile_rect[t];  // [x, y) columns, [z, w) rows of source samples
    const int rw = rc.y - rc.x, rh = rc.w - rc.z;
    if (rw > 0 && rh > 0) {
        const int lc = lane & 7, lr = lane >> 3;
        const int sx = max(a.sx_min, (rw + 7) / 8);
        const int h = max(a.h_min, (rh + 3) / 4);
        const int nx0 = rc.x + lc * sx, ny0 = rc.z + lr * h;
        const int steps = h * sx;
        int j = 0, o = 0;
        bool v = (nx0 < rc.y) && (ny0 < rc.w);
        Raw cur;
        if (v) cur = load_raw(a, nx0, ny0);
        for (int k = 0; k < steps; ++k) {
            // inputs of step k + 1
            int j2 = j, o2 = o + 1;
            if (o2 == sx) {
                o2 = 0;
                ++j2;
            }
            const bool v2 = (k + 1 < steps) && (nx0 + o2 < rc.y) && (ny0 + j2 < rc.w);
            Raw nxt;
            if (v2) nxt = load_raw(a, nx0 + o2, ny0 + j2);
            if (v) {
                int l0x, l0y;
                float dx, dy;
                sample_pos(cur.ex, cur.ey, cur.px, cur.py, cur.q, a.half_w, l0x, l0y, dx, dy);
                const int cx = l0x - ox, cy = l0y - oy;
                if (cx > -W && cx < TX && cy > -W && cy < TY) {
                    const float2 c = sample_value_fast(cur);
                    float wx[W], wy[W];
                    tap_weights<W, TAB>(a, nx0 + o, ny0 + j, dx, dy, wx, wy);
                    bool colok[W];
#pragma unroll
                    for (int i = 0; i < W; ++i) colok[i] = (unsigned)(cx + i) < (unsigned)TX;
                    // taps of this lane are distinct cells: load all, update, store all
                    float2* base = tile + cy * LD + cx;
                    float2 acc[W][W];
#pragma unroll
                    for (int b = 0; b < W; ++b) {
                        const bool rowok = (unsigned)(cy + b) < (unsigned)TY;
#pragma unroll
                        for (int i = 0; i < W; ++i)
                            acc[b][i] = (rowok && colok[i]) ? base[b * LD + i] : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int b = 0; b < W; ++b) {
                        const float2 cb = make_float2(c.x * wy[b], c.y * wy[b]);
#pragma unroll
                        for (int i = 0; i < W; ++i) acc[b][i] = fma2(cb, wx[i], acc[b][i]);
                    }
#pragma unroll
                    for (int b = 0; b < W; ++b) {
                        const bool rowok = (unsigned)(cy + b) < (unsigned)TY;
#pragma unroll
                        for (int i = 0; i < W; ++i)
                            if (rowok && colok[i]) base[b * LD + i] = acc[b][i];
                    }
                }
            }
            __syncwarp();
            cur = nxt;
            v = v2;
            j = j2;
            o = o2;
        }
    }
    __syncwarp();

    float4* g4 = reinterpret_cast<float4*>(a.grid);
    for (int i = lane; i < TY * (TX / 2); i += 32) {
        const int r = i / (TX / 2), c2 = i % (TX / 2);
        const float2 v0 = tile[r * LD + 2 * c2], v1 = tile[r * LD + 2 * c2 + 1];
        g4[((size_t)(oy + r) * a.nfx + ox) / 2 + c2] = make_float4(v0.x, v0.y, v1.x, v1.y);
    }
}

template <int W, int TX, int TY, bool TAB>
__global__ void __launch_bounds__(32) spread_es_colored_kernel(SpreadArgs a)
{
    __shared__ __align__(16) float2 tile[ColoredTile<TX, TY>::SLOTS];
    colored_tile<W, TX, TY, TAB>(a, blockIdx.x, tile, threadIdx.x);
}

// Register-window spreading: the lanes of colored_tile, but each lane walks
// its samples down source columns (runs of h consecutive rows at a fixed
// column) and accumulates their taps in a W x W window of registers that
// slides down the fine grid with the samples.  A row of the window is added
// to the shared-memory tile only when the next sample's first tap row has
// passed it, so a sample costs about one row of W read-modify-writes instead
// of W rows; the window is flushed whole when the first tap column changes
// and at the end of every run, in a step of its own.
//
// Disjointness of the shared-memory updates of one step: a lane only writes
// rows of the window of its previous step's sample, [R0, R0 + W) with R0 that
// sample's first tap row (a window whose lane found no sample in this step is
// flushed in this step).  Lanes of one row group hold columns at least
// sx * min_step_x - column_spread_x >= w apart (column_spread_x bounds the
// variation of the x coordinate down a column, since the two lanes' windows
// may come from different rows of their runs); lanes of different row groups
// are h rows apart in the same step, h * min_step_y - row_spread_y >= w.
template <int W, int TX, int TY, bool TAB>
__device__ __forceinline__ void window_tile(const SpreadArgs& a, int t, float2* tile, int lane)
{
    constexpr int LD = ColoredTile<TX, TY>::LD;
    const int ox = (a.band_tx0 + t % a.band_ntx) * TX;
    const int oy = a.band_ty0 * kTileY + (t / a.band_ntx) * TY;

    for (int i = lane; i < TY * LD; i += 32) tile[i] = make_float2(0.f, 0.f);
    __syncwarp();

    const int4 rc = a.tile_rect[t];  // [x, y) columns, [z, w) rows of source samples
    const int rw = rc.y - rc.x, rh = rc.w - rc.z;
    if (rw > 0 && rh > 0) {
        const int lc = lane & 7, lr = lane >> 3;
        const int sx = max(a.sxw_min, (rw + 7) / 8);
        const int h = max(a.h_min, (rh + 3) / 4);
        const int nx0 = rc.x + lc * sx, ny0 = rc.z + lr * h;
        const int nsamp = sx * h;

        float2 acc[W][W];
#pragma unroll
        for (int b = 0; b < W; ++b)
#pragma unroll
            for (int i = 0; i < W; ++i) acc[b][i] = make_float2(0.f, 0.f);
        int X0 = 0, R0 = 0;
        bool live = false;

        // add window row b to tile row `row` (tile-relative) at columns X0..
        auto flush_row = [&](int b, int row) {
            if ((unsigned)row < (unsigned)TY) {
                const int cx = X0 - ox;
                float2* p = tile + row * LD + cx;
                float2 v[W];
#pragma unroll
                for (int i = 0; i < W; ++i)
                    v[i] = ((unsigned)(cx + i) < (unsigned)TX) ? p[i] : make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < W; ++i)
                    if ((unsigned)(cx + i) < (unsigned)TX)
                        p[i] = make_float2(v[i].x + acc[b][i].x, v[i].y + acc[b][i].y);
            }
        };
        auto flush_all = [&]() {
#pragma unroll
            for (int b = 0; b < W; ++b) {
                flush_row(b, R0 - oy + b);
#pragma unroll
                for (int i = 0; i < W; ++i) acc[b][i] = make_float2(0.f, 0.f);
            }
        };

        int o = 0, j = 0;
        bool v = (nx0 < rc.y) && (ny0 < rc.w);
        Raw cur;
        if (v) cur = load_raw(a, nx0, ny0);
        for (int s = 0; s < nsamp; ++s) {
            int o2 = o, j2 = j + 1;
            if (j2 == h) {
                j2 = 0;
                ++o2;
            }
            const bool v2 = (s + 1 < nsamp) && (nx0 + o2 < rc.y) && (ny0 + j2 < rc.w);
            Raw nxt;
            if (v2) nxt = load_raw(a, nx0 + o2, ny0 + j2);
            int l0x = 0, l0y = 0;
            float dx = 0.f, dy = 0.f;
            bool hit = false;
            if (v) {
                sample_pos(cur.ex, cur.ey, cur.px, cur.py, cur.q, a.half_w, l0x, l0y, dx, dy);
                const int cx = l0x - ox, cy = l0y - oy;
                hit = cx > -W && cx < TX && cy > -W && cy < TY;
            }
            // A window is written only in the step right after its last
            // sample: a lane whose samples have left the tile flushes now, not
            // at the end of the run, when the lane of the next row group may
            // have come down next to it.
            if (live && (!hit || l0x != X0 || l0y < R0 || l0y - R0 >= W)) {
                flush_all();
                live = false;
            }
            if (hit) {
                const float2 c = sample_value_fast(cur);
                float wx[W], wy[W];
                tap_weights<W, TAB>(a, nx0 + o, ny0 + j, dx, dy, wx, wy);
                if (!live) {
                    X0 = l0x;
                    R0 = l0y;
                    live = true;
                }
                while (R0 < l0y) {  // slide the window down one row
                    flush_row(0, R0 - oy);
#pragma unroll
                    for (int b = 0; b + 1 < W; ++b)
#pragma unroll
                        for (int i = 0; i < W; ++i) acc[b][i] = acc[b + 1][i];
#pragma unroll
                    for (int i = 0; i < W; ++i) acc[W - 1][i] = make_float2(0.f, 0.f);
                    ++R0;
                }
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const float2 cb = make_float2(c.x * wy[b], c.y * wy[b]);
#pragma unroll
                    for (int i = 0; i < W; ++i) acc[b][i] = fma2(cb, wx[i], acc[b][i]);
                }
            }
            __syncwarp();
            if (j == h - 1) {  // end of run: flush in a step of its own
                if (live) flush_all();
                live = false;
                __syncwarp();
            }
            cur = nxt;
            v = v2;
            o = o2;
            j = j2;
        }
    }
    __syncwarp();

    float4* g4 = reinterpret_cast<float4*>(a.grid);
    for (int i = lane; i < TY * (TX / 2); i += 32) {
        const int r = i / (TX / 2), c2 = i % (TX / 2);
        const float2 v0 = tile[r * LD + 2 * c2], v1 = tile[r * LD + 2 * c2 + 1];
        g4[((size_t)(oy + r) * a.nfx + ox) / 2 + c2] = make_float4(v0.x, v0.y, v1.x, v1.y);
    }
}

template <int W, int TX, int TY, bool TAB>
__global__ void __launch_bounds__(32) spread_es_window_kernel(SpreadArgs a)
{
    __shared__ __align__(16) float2 tile[ColoredTile<TX, TY>::SLOTS];
    window_tile<W, TX, TY, TAB>(a, blockIdx.x, tile, threadIdx.x);
}

// Fallback spread of band tile `tile` (kTileX x kTileY) by a whole block:
// one sample per thread, shared-memory float atomics into tre/tim
// (kTileX * kTileY floats each), honouring the periodic wrap of every tap.
template <int W, bool TAB>
__device__ __forceinline__ void atomic_tile(const SpreadArgs& a, int tile, float* tre, float* tim,
                                            int tid, int nthreads)
{
    const int ty = a.band_ty0 + tile / a.band_ntx;
    const int tx = a.band_tx0 + tile % a.band_ntx;
    const int ox = tx * kTileX, oy = ty * kTileY;

    for (int i = tid; i < kTileX * kTileY; i += nthreads) {
        tre[i] = 0.f;
        tim[i] = 0.f;
    }
    __syncthreads();

    const int beg = a.tile_off[tile], end = a.tile_off[tile + 1];
    const int total = (end - beg) * (kSrcTile * kSrcTile);
    const int mx = a.nfx - 1, my = a.nfy - 1;
    for (int idx = tid; idx < total; idx += nthreads) {
        const int s = a.tile_src[beg + idx / (kSrcTile * kSrcTile)];
        const int local = idx % (kSrcTile * kSrcTile);
        const int nx = (s % a.nstx) * kSrcTile + local % kSrcTile;
        const int ny = (s / a.nstx) * kSrcTile + local / kSrcTile;
        if (nx >= a.n1x || ny >= a.n1y) continue;
        const size_t n = (size_t)ny * a.n1x + nx;
        const float q = __ldg(&a.q[n]);
        const AxisEntry ex = a.ax[nx], ey = a.ay[ny];
        const AxisPos px = a.px[nx], py = a.py[ny];
        int l0x, l0y;
        float dx, dy;
        sample_pos(ex, ey, px, py, q, a.half_w, l0x, l0y, dx, dy);
        const int cx0 = (l0x - ox) & mx;  // tile-relative, wrapped to [0, nf)
        const int cy0 = (l0y - oy) & my;
        const bool hitx = (cx0 < kTileX) || (cx0 + W - 1 > mx);
        const bool hity = (cy0 < kTileY) || (cy0 + W - 1 > my);
        if (!(hitx && hity)) continue;
        const float2 c = sample_value(__ldg(&a.u1[n]), ex, ey, q);

        float wx[W], wyv[W];
        if constexpr (TAB) {
            tap_weights<W, true>(a, nx, ny, dx, dy, wx, wyv);
        } else {
#pragma unroll
            for (int i = 0; i < W; ++i) {
                wx[i] = es_weight(dx + (float)i - a.half_w, a.two_over_w, a.beta_log2e);
                wyv[i] = es_weight(dy + (float)i - a.half_w, a.two_over_w, a.beta_log2e);
            }
        }

#pragma unroll
        for (int j = 0; j < W; ++j) {
            int row = cy0 + j;
            if (row > my) row -= a.nfy;
            if (row >= kTileY) continue;
            const float wy = wyv[j];
            const float cr = c.x * wy, ci = c.y * wy;
            float* rre = tre + row * kTileX;
            float* rim = tim + row * kTileX;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                int col = cx0 + i;
                if (col > mx) col -= a.nfx;
                if (col >= kTileX) continue;
                atomicAdd(rre + col, cr * wx[i]);
                atomicAdd(rim + col, ci * wx[i]);
            }
        }
    }
    __syncthreads();

    // write the tile (two cells per float4)
    float4* g4 = reinterpret_cast<float4*>(a.grid);
    for (int i = tid; i < kTileX * kTileY / 2; i += nthreads) {
        const int r = i / (kTileX / 2), c2 = i % (kTileX / 2);
        const int l = r * kTileX + 2 * c2;
        const size_t o = ((size_t)(oy + r) * a.nfx + ox) / 2 + c2;
        g4[o] = make_float4(tre[l], tim[l], tre[l + 1], tim[l + 1]);
    }
}

// Spread arguments of a plan for the field u1.
SpreadArgs make_spread_args(const asfd_plan_s* P, const float2* u1);

}  // namespace asfd
