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
    int dense_rows;    // rows per run of the dense (global-atomic) window kernel (0: not used)
    int dense_items;   // its warp items (32 columns x dense_rows rows each)
    float inc_d;       // incident depth phase, half-turns per unit d1/z0
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
                    const float2 c = sample_value_fast(cur, a.inc_d);
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

// Register-window spreading.  Lanes are those of colored_tile (4 row groups x
// 8 column groups) and, as there, every lane takes one sample per warp step,
// but a lane walks its samples down a source column (a run of h consecutive
// rows at a fixed column) and accumulates their taps in a window of W rows x
// (W + 1) columns of registers that slides down the fine grid with the
// samples.  When the next sample's first tap row is d = 1 or 2 rows lower,
// the d top rows are added to the shared-memory tile and the sample's taps
// are accumulated into the remaining rows moved up by d in the same FMAs
// (row b takes row b + d plus the new taps), so sliding costs no register
// moves; a larger jump, a sample that misses the tile, and the end of a run
// flush the whole window.  The spare column absorbs a first tap column that
// changes by one within the run (the window starts at the smaller of the
// run's first and last sample's first tap column).  A sample is never added
// to the tile directly, so each cell of the tile receives about one
// read-modify-write per sample row instead of one per tap row.
//
// Disjointness of the shared-memory updates of one step: a lane only writes
// rows of the window of its previous step's sample, [R0, R0 + W) with R0 that
// sample's first tap row (a window whose lane found no sample in this step is
// flushed in this step), and only columns covered by its own samples' taps.
// Lanes of one row group hold columns at least
// sx * min_step_x - column_spread_x >= w apart (column_spread_x bounds the
// variation of the x coordinate down a column, since the two lanes' windows
// may come from different rows of their runs); lanes of different row groups
// are h rows apart in the same step, h * min_step_y - row_spread_y >= w.
constexpr int kWindowSpare = 1;  // spare window columns (first tap column drift in a run)

template <int WX, int TX, int TY>
__device__ __forceinline__ void window_flush(float2* tile, int row, int cx, unsigned cmask,
                                             const float2 (&r)[WX])
{
    constexpr int LD = ColoredTile<TX, TY>::LD;
    if ((unsigned)row < (unsigned)TY) {
        float2* p = tile + row * LD;
        float2 v[WX];
#pragma unroll
        for (int i = 0; i < WX; ++i)
            v[i] = ((cmask >> i) & 1u) ? p[cx + i] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < WX; ++i)
            if ((cmask >> i) & 1u) p[cx + i] = make_float2(v[i].x + r[i].x, v[i].y + r[i].y);
    }
}

// a + b on FP32 pairs (packed FP32x2)
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    unsigned long long r;
    const unsigned long long aa = *reinterpret_cast<const unsigned long long*>(&a);
    const unsigned long long bb = *reinterpret_cast<const unsigned long long*>(&b);
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(aa), "l"(bb));
    return *reinterpret_cast<float2*>(&r);
}

// ES weights of two taps at once (packed FP32x2 arithmetic; the square root
// and exponential on the MUFU unit as in es_weight_fast).
__device__ __forceinline__ float2 es_weight2_fast(float2 z, float neg_c2, float beta_log2e)
{
    // r = 1 - (2z/w)^2 = fma(z * neg_c2, z, 1)
    const float2 t = mul2(z, neg_c2);
    float2 r = fma2v(t, z, make_float2(1.f, 1.f));
    r.x = fmaxf(r.x, 1e-30f);
    r.y = fmaxf(r.y, 1e-30f);
    float2 rs, e;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs.x) : "f"(r.x));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs.y) : "f"(r.y));
    const float2 s = fma2v(r, rs, make_float2(-1.f, -1.f));
    const float2 arg = mul2(s, beta_log2e);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(arg.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(arg.y));
    return e;
}

// Adds one sample to a register window whose top row is R0 and whose first
// column is X0: fresh (the window is empty: overwrite every slot), or with
// its first tap row dn = 0, 1 or 2 rows below R0 (the dn top rows go to
// flush(b) first and the rest move up by dn inside the FMAs).  offn is the
// sample's first tap column minus X0 (0, or 1 with a spare column).
template <int W, int WX, class Flush>
__device__ __forceinline__ void window_add(float2 (&acc)[W][WX], bool fresh, int dn, int offn,
                                           float dx, float dy, float2 c, const SpreadArgs& a,
                                           float neg_c2, Flush&& flush)
{
    float wy[W], wxe[WX];
    const float by = dy - a.half_w;
    const float bx = dx - a.half_w - (float)offn;
    const float2 bxy = make_float2(by, bx);
#pragma unroll
    for (int b = 0; b < W; ++b) {
        // tap b's offsets from the sample in y and x, one packed add
        const float2 e = es_weight2_fast(add2(bxy, make_float2((float)b, (float)b)), neg_c2,
                                         a.beta_log2e);
        wy[b] = e.x;
        wxe[b] = e.y;
    }
    if constexpr (WX > W) {
        wxe[W] = es_weight_fast(bx + (float)W, a.two_over_w, a.beta_log2e);
        // tap column i of the sample sits in window column i + offn
        if (offn == 1) wxe[0] = 0.f;
        else wxe[W] = 0.f;
    }
    if (fresh) {
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2 cb = mul2(c, wy[b]);
#pragma unroll
            for (int i = 0; i < WX; ++i) acc[b][i] = mul2(cb, wxe[i]);
        }
    } else if (dn == 0) {
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2 cb = mul2(c, wy[b]);
#pragma unroll
            for (int i = 0; i < WX; ++i) acc[b][i] = fma2(cb, wxe[i], acc[b][i]);
        }
    } else if (dn == 1) {
        flush(0);
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2 cb = mul2(c, wy[b]);
#pragma unroll
            for (int i = 0; i < WX; ++i)
                acc[b][i] = (b + 1 < W) ? fma2(cb, wxe[i], acc[b + 1][i]) : mul2(cb, wxe[i]);
        }
    } else {
        flush(0);
        flush(1);
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2 cb = mul2(c, wy[b]);
#pragma unroll
            for (int i = 0; i < WX; ++i)
                acc[b][i] = (b + 2 < W) ? fma2(cb, wxe[i], acc[b + 2][i]) : mul2(cb, wxe[i]);
        }
    }
}

// window_add with the W x and W y tap weights given (learned tables): the
// window column i takes tap i - offn.
template <int W, int WX, class Flush>
__device__ __forceinline__ void window_add_w(float2 (&acc)[W][WX], bool fresh, int dn, int offn,
                                             const float (&wx)[W], const float (&wy)[W], float2 c,
                                             Flush&& flush)
{
    float wxe[WX];
#pragma unroll
    for (int i = 0; i < WX; ++i) {
        const float lo = (i < W) ? wx[i] : 0.f;
        const float hi = (i >= 1 && i - 1 < W) ? wx[i - 1] : 0.f;
        wxe[i] = offn == 1 ? hi : lo;
    }
    if (fresh) {
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2 cb = mul2(c, wy[b]);
#pragma unroll
            for (int i = 0; i < WX; ++i) acc[b][i] = mul2(cb, wxe[i]);
        }
    } else if (dn == 0) {
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2 cb = mul2(c, wy[b]);
#pragma unroll
            for (int i = 0; i < WX; ++i) acc[b][i] = fma2(cb, wxe[i], acc[b][i]);
        }
    } else if (dn == 1) {
        flush(0);
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2 cb = mul2(c, wy[b]);
#pragma unroll
            for (int i = 0; i < WX; ++i)
                acc[b][i] = (b + 1 < W) ? fma2(cb, wxe[i], acc[b + 1][i]) : mul2(cb, wxe[i]);
        }
    } else {
        flush(0);
        flush(1);
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float2 cb = mul2(c, wy[b]);
#pragma unroll
            for (int i = 0; i < WX; ++i)
                acc[b][i] = (b + 2 < W) ? fma2(cb, wxe[i], acc[b + 2][i]) : mul2(cb, wxe[i]);
        }
    }
}

// Horner evaluation of the learned tap polynomials of one source tile staged
// in shared memory as (x, y) coefficient pairs [tap][coef] (kLearnCoef
// coefficients per tap, in t = 2 d - 1); both axes at once in FP32x2.
template <int W>
__device__ __forceinline__ void table_weights_smem(const float4* tab, float dx, float dy,
                                                   float (&wx)[W], float (&wy)[W])
{
    static_assert(kLearnCoef == 8, "four float4 per tap");
    const float2 t = make_float2(fmaf(2.0f, dx, -1.0f), fmaf(2.0f, dy, -1.0f));
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const float4 c01 = tab[4 * i], c23 = tab[4 * i + 1], c45 = tab[4 * i + 2],
                     c67 = tab[4 * i + 3];
        float2 p = make_float2(c67.z, c67.w);
        p = fma2v(p, t, make_float2(c67.x, c67.y));
        p = fma2v(p, t, make_float2(c45.z, c45.w));
        p = fma2v(p, t, make_float2(c45.x, c45.y));
        p = fma2v(p, t, make_float2(c23.z, c23.w));
        p = fma2v(p, t, make_float2(c23.x, c23.y));
        p = fma2v(p, t, make_float2(c01.z, c01.w));
        p = fma2v(p, t, make_float2(c01.x, c01.y));
        wx[i] = p.x;
        wy[i] = p.y;
    }
}

template <int W, int TX, int TY, bool TAB>
__device__ __forceinline__ void window_tile(const SpreadArgs& a, int t, float2* tile, int lane)
{
    static_assert(!TAB, "the register-window kernel evaluates the ES kernel");
    constexpr int LD = ColoredTile<TX, TY>::LD;
    constexpr int WX = W + kWindowSpare;
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
        const int nyl = min(ny0 + h, rc.w) - 1;  // last source row of this lane's runs
        const int nsamp = sx * h;
        const float neg_c2 = -a.two_over_w * a.two_over_w;

        float2 acc[W][WX];
#pragma unroll
        for (int b = 0; b < W; ++b)
#pragma unroll
            for (int i = 0; i < WX; ++i) acc[b][i] = make_float2(0.f, 0.f);
        int X0 = 0, R0 = 0, maxoff = 0;
        unsigned cmask = 0;
        bool live = false;

        // (a window that is not live holds stale values: the first sample
        // of the next window overwrites every slot)
        auto flush_all = [&]() {
#pragma unroll
            for (int b = 0; b < W; ++b)
                window_flush<WX, TX, TY>(tile, R0 - oy + b, X0 - ox, cmask, acc[b]);
        };
        // window columns X0 .. X0 + W - 1 + maxoff (within the tile)
        auto set_columns = [&](int x0, int mo) {
            X0 = x0;
            maxoff = mo;
            cmask = 0;
#pragma unroll
            for (int i = 0; i < WX; ++i)
                if (i < W + mo && (unsigned)(x0 - ox + i) < (unsigned)TX) cmask |= 1u << i;
        };

        // u1 and q of the samples two steps ahead are loaded in flight; the
        // column's table entries are fixed for a run, the row's are read at use
        int o = 0, j = 0;    // step s: run o, row j
        int oc = 0, jc = 0;  // step s + 2
        auto next_slot = [&](int& oo, int& jj) {
            if (++jj == h) {
                jj = 0;
                ++oo;
            }
        };
        auto slot_ok = [&](int oo, int jj) { return (nx0 + oo < rc.y) && (ny0 + jj <= nyl); };
        next_slot(oc, jc);
        next_slot(oc, jc);
        float qa = 0.f, qb = 0.f;
        float2 ua = make_float2(0.f, 0.f), ub = make_float2(0.f, 0.f);
        if (slot_ok(0, 0)) {
            qa = __ldg(&a.q[(size_t)ny0 * a.n1x + nx0]);
            ua = __ldg(&a.u1[(size_t)ny0 * a.n1x + nx0]);
        }
        if (nsamp > 1) {
            int o1 = 0, j1 = 0;
            next_slot(o1, j1);
            if (slot_ok(o1, j1)) {
                const size_t n = (size_t)(ny0 + j1) * a.n1x + nx0 + o1;
                qb = __ldg(&a.q[n]);
                ub = __ldg(&a.u1[n]);
            }
        }
        AxisEntry ex{};
        AxisPos px{};
        for (int s = 0; s < nsamp; ++s) {
            float qc = 0.f;
            float2 uc = make_float2(0.f, 0.f);
            if (s + 2 < nsamp && slot_ok(oc, jc)) {
                const size_t n = (size_t)(ny0 + jc) * a.n1x + nx0 + oc;
                qc = __ldg(&a.q[n]);
                uc = __ldg(&a.u1[n]);
            }
            const bool v = slot_ok(o, j);
            const int nx = nx0 + o, ny = ny0 + j;
            int l0x = 0, l0y = 0;
            float dx = 0.f, dy = 0.f;
            bool hit = false;
            AxisEntry ey{};
            if (v) {
                if (j == 0) {
                    ex = a.ax[nx];
                    px = a.px[nx];
                }
                ey = a.ay[ny];
                const AxisPos py = a.py[ny];
                sample_pos(ex, ey, px, py, qa, a.half_w, l0x, l0y, dx, dy);
                hit = (l0x - ox) > -W && (l0x - ox) < TX && (l0y - oy) > -W && (l0y - oy) < TY;
                if (j == 0) {
                    // window columns of the run: first tap columns of its first
                    // and last samples
                    const float ql = __ldg(&a.q[(size_t)nyl * a.n1x + nx]);
                    int lx, ly;
                    float fx, fy;
                    sample_pos(ex, a.ay[nyl], px, a.py[nyl], ql, a.half_w, lx, ly, fx, fy);
                    if (kWindowSpare > 0) set_columns(min(l0x, lx), lx != l0x ? 1 : 0);
                    else set_columns(l0x, 0);
                }
            }
            const int off = l0x - X0;
            const int d = l0y - R0;
            if (live && (!hit || off < 0 || off > maxoff || d < 0 || d > 2)) {
                flush_all();
                live = false;
            }
            if (hit) {
                const bool fresh = !live;
                if (fresh) {
                    if (off < 0 || off > maxoff) set_columns(l0x, 0);
                    R0 = l0y;
                    live = true;
                }
                const float2 c = sample_value_fast(ua, ex, ey, qa, a.inc_d);
                window_add<W, WX>(acc, fresh, l0y - R0, l0x - X0, dx, dy, c, a, neg_c2,
                                  [&](int b) {
                                      window_flush<WX, TX, TY>(tile, R0 + b - oy, X0 - ox, cmask,
                                                               acc[b]);
                                  });
                R0 = l0y;
            }
            __syncwarp();
            if (j == h - 1) {  // end of run: flush in a step of its own
                if (live) flush_all();
                live = false;
                __syncwarp();
            }
            qa = qb;
            ua = ub;
            qb = qc;
            ub = uc;
            next_slot(o, j);
            next_slot(oc, jc);
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

// Dense maps (many samples per fine-grid cell, where conflict-free lanes
// would have to be many columns apart): warp item `it` takes 32 consecutive
// source columns (one per lane) over `dense_rows` consecutive rows; each lane
// walks its column with the register window above, and window rows go
// straight to the fine grid with float2 atomic adds (which only need the
// band zeroed beforehand).  Consecutive samples of a column share their
// first tap row about 1/(alpha (1 + q)) times, so a row is flushed about
// alpha times per sample.  Lanes need no step synchronisation beyond the
// warp barrier that publishes each row's table entries.
constexpr int kDenseAhead = 3;  // rows of u1, q and table entries in flight
// The dense item's window has no spare column: a lane whose first tap column
// drifts by one inside its run (the x coordinate moves with q down a
// column, by a fraction of a cell over a run) flushes its window and starts
// a fresh one at the new column.  That costs one full flush per drift, and
// saves a column of taps, FMAs and reductions on every sample.
constexpr int kDenseSpare = 0;
constexpr int kDenseRing = 4;   // ring slots (> kDenseAhead, power of two)
constexpr int kDenseRingBytes = kDenseRing * (32 * (8 + 4) + 32);  // per warp

template <int W, bool TAB = false>
__device__ __forceinline__ void window_atomic_item(const SpreadArgs& a, int it, int lane,
                                                   char* ring, float4* tsm = nullptr)
{
    constexpr int WX = W + kDenseSpare;
    const int ncb = (a.n1x + 31) / 32;
    const int nx = (it % ncb) * 32 + lane;
    const int ny0 = (it / ncb) * a.dense_rows;
    const int nyl = min(ny0 + a.dense_rows, a.n1y) - 1;
    // lanes that stay in the item (without the learned kernel, lanes past
    // the last column return below)
    const int ncols = a.n1x - (it % ncb) * 32;
    const unsigned wmask = (TAB || ncols >= 32) ? 0xffffffffu : ((1u << max(ncols, 0)) - 1u);
    if constexpr (TAB) {
        // learned kernel: the warp's lanes span two source-tile columns and
        // step through the same rows, so the two tiles' polynomial tables
        // are staged in shared memory (tsm: 2 x 4W float4) per tile row
        if (ny0 > nyl || (it % ncb) * 32 >= a.n1x) return;  // warp-uniform
    } else {
        if (nx >= a.n1x || ny0 > nyl) return;
    }
    // (learned kernel: lanes past the last column follow along without flushing)
    const bool lane_on = !TAB || nx < a.n1x;
    const int nxc = (!TAB || lane_on) ? nx : a.n1x - 1;
    const int my = a.nfy - 1;
    const float neg_c2 = -a.two_over_w * a.two_over_w;
    const AxisEntry ex = a.ax[nxc];
    const AxisPos px = a.px[nxc];

    // window columns: first tap columns of the run's first and last samples
    int X0, maxoff;
    {
        int lf, ll, yy;
        float f0, f1;
        sample_pos(ex, a.ay[ny0], px, a.py[ny0], __ldg(&a.q[(size_t)ny0 * a.n1x + nxc]), a.half_w,
                   lf, yy, f0, f1);
        sample_pos(ex, a.ay[nyl], px, a.py[nyl], __ldg(&a.q[(size_t)nyl * a.n1x + nxc]), a.half_w,
                   ll, yy, f0, f1);
        X0 = (kDenseSpare > 0) ? min(lf, ll) : lf;
        maxoff = (kDenseSpare > 0 && lf != ll) ? 1 : 0;
    }
    float2 acc[W][WX];
    int R0 = 0;
    bool live = false;
    auto flush_row = [&](int b) {
        // the plan takes this path only when no footprint wraps around the
        // periodic grid, so the window's columns lie in [0, nfx) and the
        // addresses are one base plus constant offsets; the clamp keeps every
        // address inside the row all the same
        const int xc = min(max(X0, 0), a.nfx - W - maxoff);
        float2* row = a.grid + (size_t)((R0 + b) & my) * a.nfx + xc;
#pragma unroll
        for (int i = 0; i < WX; ++i)
            if (lane_on && i < W + maxoff) atomicAdd(row + i, acc[b][i]);
    };
    // u1 and q of the run's rows are copied asynchronously (cp.async) into a
    // per-lane ring of kDenseRing slots in shared memory, kDenseAhead rows
    // ahead of use, and with them (by lane 0) the row's y table entries,
    // which every lane of the warp reads
    float2* ring_u = reinterpret_cast<float2*>(ring);
    float* ring_q = reinterpret_cast<float*>(ring_u + kDenseRing * 32);
    // the row's y table entries (AxisEntry, AxisPos: 24 of 32 bytes per slot), copied by lane 0
    char* ring_t = reinterpret_cast<char*>(ring_q + kDenseRing * 32);
    auto issue_row = [&](int r) {  // always commits one group (empty past the run)
        if (r <= nyl) {
            const size_t n = (size_t)r * a.n1x + nxc;
            const int slot = (r - ny0) & (kDenseRing - 1);
            const unsigned du = (unsigned)__cvta_generic_to_shared(ring_u + slot * 32 + lane);
            const unsigned dq = (unsigned)__cvta_generic_to_shared(ring_q + slot * 32 + lane);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(du), "l"(a.u1 + n));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dq), "l"(a.q + n));
            if (lane == 0) {
                const unsigned dt = (unsigned)__cvta_generic_to_shared(ring_t + slot * 32);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dt), "l"(a.ay + r));
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dt + 16), "l"(a.py + r));
            }
        }
        asm volatile("cp.async.commit_group;");
    };
#pragma unroll
    for (int r = 0; r < kDenseAhead; ++r) issue_row(ny0 + r);
    int tab_ty = -1;
    const int tcol0 = ((it % ncb) * 32) / kSrcTile;  // first source-tile column of the warp
    // the table float4 this lane stages, loaded one tile row ahead
    const int tcol = min(tcol0 + lane / (4 * W), a.nstx - 1);
    auto load_tab = [&](int ty) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (TAB && lane < 8 * W && ty * kSrcTile < a.n1y)
            v = __ldg(reinterpret_cast<const float4*>(a.table + ((size_t)ty * a.nstx + tcol) *
                                                                   kLearnTableSize) +
                      lane % (4 * W));
        return v;
    };
    float4 tnext = load_tab(ny0 / kSrcTile);
    for (int ny = ny0; ny <= nyl; ++ny) {
        // this lane's copy of row ny has landed once at most kDenseAhead - 1
        // younger groups are pending (lane 0's table copy is visible to the
        // warp after the barrier); then queue row ny + kDenseAhead
        asm volatile("cp.async.wait_group %0;" ::"n"(kDenseAhead - 1));
        __syncwarp(wmask);
        const int slot = (ny - ny0) & (kDenseRing - 1);
        const AxisEntry ey = *reinterpret_cast<const AxisEntry*>(ring_t + slot * 32);
        const AxisPos py = *reinterpret_cast<const AxisPos*>(ring_t + slot * 32 + 16);
        const float q = ring_q[slot * 32 + lane];
        const float2 u = ring_u[slot * 32 + lane];
        issue_row(ny + kDenseAhead);
        int l0x, l0y;
        float dx, dy;
        sample_pos(ex, ey, px, py, q, a.half_w, l0x, l0y, dx, dy);
        const int off = l0x - X0, d = l0y - R0;
        if (live && (off < 0 || off > maxoff || d < 0 || d > 2)) {
#pragma unroll
            for (int b = 0; b < W; ++b) flush_row(b);
            live = false;
        }
        const bool fresh = !live;
        if (fresh) {
            if (off < 0 || off > maxoff) {
                X0 = l0x;
                maxoff = 0;
            }
            R0 = l0y;
            live = true;
        }
        const float2 c = sample_value_fast(u, ex, ey, q, a.inc_d);
        if constexpr (TAB) {
            if (ny / kSrcTile != tab_ty) {  // warp-uniform: every lane is on row ny
                tab_ty = ny / kSrcTile;
                __syncwarp();
                // global layout [axis][tap][coef]; staged as [tap][coef] pairs
                // (x, y) so that the Horner steps read ready FP32x2 operands
                if (lane < 8 * W) {
                    const int e = lane % (4 * W);  // float4 index within the tile's table
                    const float4 v = tnext;
                    const int axis = e / (2 * W), k0 = (e % (2 * W)) * 4;  // tap * 8 + coef
                    float* d = reinterpret_cast<float*>(tsm + (lane / (4 * W)) * (4 * W)) + axis;
                    d[2 * (k0 + 0)] = v.x;
                    d[2 * (k0 + 1)] = v.y;
                    d[2 * (k0 + 2)] = v.z;
                    d[2 * (k0 + 3)] = v.w;
                }
                __syncwarp();
                tnext = load_tab(tab_ty + 1);
            }
            float wx[W], wy[W];
            table_weights_smem<W>(tsm + (nxc / kSrcTile - tcol0) * (4 * W), dx, dy, wx, wy);
            window_add_w<W, WX>(acc, fresh, l0y - R0, l0x - X0, wx, wy, c, flush_row);
        } else {
            window_add<W, WX>(acc, fresh, l0y - R0, l0x - X0, dx, dy, c, a, neg_c2, flush_row);
        }
        R0 = l0y;
    }
    if (live) {
#pragma unroll
        for (int b = 0; b < W; ++b) flush_row(b);
    }
}

// warps (items) per block of the dense spread (blocks of 1 or 2 warps with
// registers capped for more resident warps spilled and ran slower)
constexpr int kDenseWarps = 4;

template <int W, bool TAB = false>
__global__ void __launch_bounds__(32 * kDenseWarps) spread_es_dense_kernel(SpreadArgs a, int items)
{
    __shared__ float4 tsm[kDenseWarps][TAB ? 8 * W : 1];
    __shared__ __align__(16) char ring[kDenseWarps][kDenseRingBytes];
    const int it = blockIdx.x * kDenseWarps + threadIdx.x / 32;
    if (it < items)
        window_atomic_item<W, TAB>(a, it, threadIdx.x % 32, ring[threadIdx.x / 32],
                                   tsm[threadIdx.x / 32]);
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
        const float2 c = sample_value(__ldg(&a.u1[n]), ex, ey, q, a.inc_d);

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
