// Atomic-free spread for monotone maps with at least one fine cell between
// neighbouring samples of a row: per-item shared-memory tiles and an ordered
// gather (the deterministic path, asfd_params.deterministic = 1).
//
// A warp item is that of the default spread (32 consecutive source columns,
// one per lane, over a run of rows), with the same register window per lane
// (spread.cuh, window_add), but a window row leaves the registers into a
// tile of shared memory private to the warp that covers the item's whole
// footprint, instead of going to the fine grid with float atomic adds:
//
//  * All flushes of a step run in one warp-uniform sequence -- for each
//    window row b, for each window column i, every lane that flushes that
//    row adds its cell (row R0 + b, column X0 + i) to the tile, with a warp
//    barrier between the (b, i) phases.  In one phase no two lanes touch the
//    same cell: lanes that flush the same tile row have the same R0, and the
//    plan takes this path only where the first tap columns X0 of the lanes of
//    one step (the same source row, consecutive columns) are strictly
//    increasing, i.e. neighbouring samples of a row are at least one fine
//    cell apart.  So every cell receives its contributions in an order fixed
//    by the inputs.
//  * At the end of its run the warp writes the tile to its slot of a scratch
//    area (the plan's row-FFT buffer, free until the row pass).
//  * The gather kernel forms each band cell of the fine grid as the sum, in a
//    fixed order (run, then column block), of the tiles that cover it; item
//    boxes are products of a per-column-block x range and a per-run y range
//    computed at plan time with the spread's own FP32 position arithmetic.
//
// Results are therefore bit-identical from run to run.  Against the default
// path this costs the tile's read-modify-write phases, the tile write-out
// and the gather, and saves the float atomics.
#include <climits>
#include <vector>

#include "spread.cuh"

namespace asfd {

namespace {

constexpr int kItemWarps = 4;                 // warps (items) per block
constexpr int kItemMaxTileBytes = 18 * 1024;  // shared-memory tile per warp, at most
constexpr int kItemMaxOverlap = 3;            // column blocks (runs) covering one fine column (row)
constexpr int kItemMinRows = 8;               // shortest runs tried

struct ItemArgs {
    SpreadArgs s;
    const int* xbox;  // [ncb][2]: first tap column range of each column block: [lo, hi)
    const int* ybox;  // [nruns][2]: first tap row range of each run
    float2* scratch;  // [items][th][tw]
    int tw, th;       // tile width and height (cells)
};

// First tap row and column of every sample (the spread's arithmetic), folded
// into per-column-block and per-run ranges (min of the first tap, max of the
// first tap + W).  One warp per (column block, run), a lane per column: each
// lane folds its column's rows, the warp folds its lanes, and one lane
// merges the result with four atomics (all samples of a column block meet
// in one entry, so per-sample atomics would serialise).
__global__ void item_box_kernel(SpreadArgs a, int rows, int* xbox, int* ybox)
{
    const int ncb = (a.n1x + 31) / 32, nruns = (a.n1y + rows - 1) / rows;
    const int lane = threadIdx.x % 32;
    const int w = (int)(2.f * a.half_w + 0.5f);
    const int warps = gridDim.x * (blockDim.x / 32);
    for (int item = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; item < ncb * nruns;
         item += warps) {
        const int cb = item % ncb, run = item / ncb;
        const int nx = cb * 32 + lane;
        int xmin = INT_MAX, xmax = INT_MIN, ymin = INT_MAX, ymax = INT_MIN;
        if (nx < a.n1x) {
            const AxisEntry ex = a.ax[nx];
            const AxisPos px = a.px[nx];
            const int ny1 = min((run + 1) * rows, a.n1y);
            for (int ny = run * rows; ny < ny1; ++ny) {
                int l0x, l0y;
                float dx, dy;
                sample_pos(ex, a.ay[ny], px, a.py[ny], __ldg(&a.q[(size_t)ny * a.n1x + nx]),
                           a.half_w, l0x, l0y, dx, dy);
                xmin = min(xmin, l0x);
                xmax = max(xmax, l0x);
                ymin = min(ymin, l0y);
                ymax = max(ymax, l0y);
            }
        }
        xmin = __reduce_min_sync(0xffffffffu, xmin);
        xmax = __reduce_max_sync(0xffffffffu, xmax);
        ymin = __reduce_min_sync(0xffffffffu, ymin);
        ymax = __reduce_max_sync(0xffffffffu, ymax);
        if (lane == 0 && xmin <= xmax) {
            atomicMin(&xbox[2 * cb], xmin);
            atomicMax(&xbox[2 * cb + 1], xmax + w);
            atomicMin(&ybox[2 * run], ymin);
            atomicMax(&ybox[2 * run + 1], ymax + w);
        }
    }
}

__global__ void item_box_init_kernel(int* box, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) box[i] = (i & 1) ? INT_MIN : INT_MAX;
}

template <int W>
__device__ __forceinline__ void item_tile(const ItemArgs& ia, int it, int lane, char* ring,
                                          float2* tile)
{
    const SpreadArgs& a = ia.s;
    const int ncb = (a.n1x + 31) / 32;
    const int cb = it % ncb, run = it / ncb;
    const int nx = cb * 32 + lane;
    const int ny0 = run * a.dense_rows;
    const int nyl = min(ny0 + a.dense_rows, a.n1y) - 1;
    if (ny0 > nyl) return;  // warp-uniform
    // every lane takes part in the warp-uniform phases; lanes past the last
    // column follow the last one without flushing
    const bool lane_on = nx < a.n1x;
    const int nxc = lane_on ? nx : a.n1x - 1;
    constexpr unsigned wmask = 0xffffffffu;
    const int tw = ia.tw, th = ia.th;
    const int xlo = ia.xbox[2 * cb], ylo = ia.ybox[2 * run];

    for (int i = lane; i < tw * th; i += 32) tile[i] = make_float2(0.f, 0.f);
    __syncwarp(wmask);

    const float neg_c2 = -a.two_over_w * a.two_over_w;
    const AxisEntry ex = a.ax[nxc];
    const AxisPos px = a.px[nxc];
    float2 acc[W][W];
    int X0 = 0, R0 = 0;
    bool live = false;
    // rows b < nflush of the window go to the tile, in warp-uniform phases
    // (as many rows as the lane that flushes most: usually one or two)
    auto flush = [&](int nflush) {
        const int nb = __reduce_max_sync(wmask, lane_on ? nflush : 0);
#pragma unroll
        for (int b = 0; b < W; ++b) {
            if (b >= nb) break;  // warp-uniform
            const int r = R0 + b - ylo;
            const bool on = lane_on && b < nflush && (unsigned)r < (unsigned)th;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int c = X0 + i - xlo;
                if (on && (unsigned)c < (unsigned)tw) {
                    float2* p = tile + r * tw + c;
                    const float2 v = *p;
                    *p = make_float2(v.x + acc[b][i].x, v.y + acc[b][i].y);
                }
                __syncwarp(wmask);
            }
        }
    };
    // u1, q and the row's y table entries staged as in the default spread
    float2* ring_u = reinterpret_cast<float2*>(ring);
    float* ring_q = reinterpret_cast<float*>(ring_u + kDenseRing * 32);
    char* ring_t = reinterpret_cast<char*>(ring_q + kDenseRing * 32);
    auto issue_row = [&](int r) {
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
    for (int ny = ny0; ny <= nyl; ++ny) {
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
        const int d = l0y - R0;
        const bool restart = live && (l0x != X0 || d < 0 || d > 2);
        flush(restart ? W : (live ? d : 0));
        const bool fresh = !live || restart;
        if (fresh) {
            X0 = l0x;
            R0 = l0y;
            live = true;
        }
        const float2 c = sample_value_fast(u, ex, ey, q, a.inc_d);
        window_add<W, W>(acc, fresh, l0y - R0, 0, dx, dy, c, a, neg_c2, [](int) {});
        R0 = l0y;
    }
    flush(live ? W : 0);
    // the tile to the item's scratch slot
    float2* out = ia.scratch + (size_t)it * tw * th;
    for (int i = lane; i < tw * th; i += 32) out[i] = tile[i];
}

template <int W>
__global__ void __launch_bounds__(32 * kItemWarps) spread_item_kernel(ItemArgs ia, int items)
{
    extern __shared__ float4 item_smem[];
    const int wid = threadIdx.x / 32;
    char* ring = reinterpret_cast<char*>(item_smem) + wid * kDenseRingBytes;
    float2* tile = reinterpret_cast<float2*>(reinterpret_cast<char*>(item_smem) +
                                             kItemWarps * kDenseRingBytes) +
                   (size_t)wid * ia.tw * ia.th;
    const int it = blockIdx.x * kItemWarps + wid;
    if (it < items) item_tile<W>(ia, it, threadIdx.x % 32, ring, tile);
}

// Band cell (x, y) = sum over the runs and then the column blocks whose item
// boxes cover it of the items' tiles (fixed order).  xmap / ymap: first
// column block (run) and count per band column (row).  A thread forms
// kGatherRows cells of one band column: the column's boxes are looked up
// once, and the rows' tile reads are independent of each other.
constexpr int kGatherRows = 4;

__global__ void __launch_bounds__(128)
item_gather_kernel(const float2* __restrict__ scratch, const int* __restrict__ xbox,
                   const int* __restrict__ ybox, const int* __restrict__ xmap,
                   const int* __restrict__ ymap, int x0, int y0, int bw, int bh, int ncb, int tw,
                   int th, float2* __restrict__ grid, int nfx)
{
    const int bx = blockIdx.x * blockDim.x + threadIdx.x;
    if (bx >= bw) return;
    const int x = x0 + bx;
    const int xm = __ldg(&xmap[bx]);
    const int cb0 = xm & 0xffffff, ncx = xm >> 24;
    int tx[kItemMaxOverlap];
#pragma unroll
    for (int k = 0; k < kItemMaxOverlap; ++k) tx[k] = k < ncx ? x - __ldg(&xbox[2 * (cb0 + k)]) : 0;
    const size_t tile = (size_t)th * tw;
#pragma unroll
    for (int r = 0; r < kGatherRows; ++r) {
        const int by = blockIdx.y * kGatherRows + r;
        if (by >= bh) break;
        const int y = y0 + by;
        const int ym = __ldg(&ymap[by]);
        const int rr0 = ym & 0xffffff, ncy = ym >> 24;
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < kItemMaxOverlap; ++j) {
            if (j < ncy) {
                const int rr = rr0 + j;
                const int ty = y - __ldg(&ybox[2 * rr]);
                const float2* t = scratch + ((size_t)(rr * ncb + cb0) * th + ty) * tw;
#pragma unroll
                for (int k = 0; k < kItemMaxOverlap; ++k) {
                    if (k < ncx) {
                        const float2 v = __ldg(t + k * tile + tx[k]);
                        s.x += v.x;
                        s.y += v.y;
                    }
                }
            }
        }
        grid[(size_t)y * nfx + x] = s;
    }
}

asfd_status item_slots(int w, long long* slots)
{
    int dev = 0, sms = 0, per_sm = 0;
    ASFD_CUDA(cudaGetDevice(&dev));
    ASFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const void* k = nullptr;
    switch (w) {
#define ASFD_IK(W) case W: k = (const void*)spread_item_kernel<W>; break;
        ASFD_IK(2) ASFD_IK(3) ASFD_IK(4) ASFD_IK(5) ASFD_IK(6) ASFD_IK(7)
#undef ASFD_IK
        default: return fail(ASFD_ERR_UNSUPPORTED, "item-tile spread widths are 2..7");
    }
    // resident blocks at the largest tile this path accepts
    const size_t smem = kItemWarps * ((size_t)kDenseRingBytes + kItemMaxTileBytes);
    ASFD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ASFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * kItemWarps, smem));
    *slots = (long long)sms * std::max(per_sm, 1) * kItemWarps;
    return ASFD_OK;
}

}  // namespace

asfd_status plan_build_itemtile(asfd_plan_s* P, cudaStream_t st)
{
    const asfd_params& p = P->prm;
    P->itemtile = false;
    if (P->learned || P->w > kMaxWindowWidth || P->min_step_x < 1.0 + 1e-3) return ASFD_OK;
    const long long ncb = (p.n1x + 31) / 32;
    long long slots = 0;
    asfd_status s = item_slots(P->w, &slots);
    if (s != ASFD_OK) return s;
    const int rows0 = window_run_rows(p.n1y, ncb, slots);
    // tables: per column block, per run (sized for the shortest runs tried)
    // and per fine column / row; each allocated once, a refused one retried
    const long long max_runs = (p.n1y + kItemMinRows - 1) / kItemMinRows;
    const struct {
        int** ptr;
        size_t bytes;
    } tabs[] = {{&P->it_xbox, sizeof(int) * 2 * ncb},
                {&P->it_ybox, sizeof(int) * 2 * max_runs},
                {&P->it_xmap, sizeof(int) * P->nfx},
                {&P->it_ymap, sizeof(int) * P->nfy}};
    for (const auto& t : tabs)
        if (!*t.ptr &&
            (s = plan_alloc_buffer(P, reinterpret_cast<void**>(t.ptr), t.bytes)) != ASFD_OK) {
            *t.ptr = nullptr;
            return s;
        }
    // runs of the wave rule's length, halved until an item's tile fits the
    // shared memory of a warp and all tiles fit the row buffer
    SpreadArgs a = make_spread_args(P, nullptr);
    int rows = rows0, tw = 0, th = 0;
    long long nruns = 0, items = 0;
    std::vector<int> xb(2 * ncb), yb;
    for (;; rows = (rows + 1) / 2) {
        if (rows < kItemMinRows) return ASFD_OK;
        nruns = (p.n1y + rows - 1) / rows;
        items = ncb * nruns;
        item_box_init_kernel<<<(unsigned)((2 * ncb + 255) / 256), 256, 0, st>>>(P->it_xbox,
                                                                               (int)(2 * ncb));
        item_box_init_kernel<<<(unsigned)((2 * nruns + 255) / 256), 256, 0, st>>>(P->it_ybox,
                                                                                 (int)(2 * nruns));
        item_box_kernel<<<(unsigned)std::min<long long>((ncb * nruns + 7) / 8, 4096), 256, 0,
                          st>>>(a, rows, P->it_xbox, P->it_ybox);
        ASFD_CUDA(cudaGetLastError());
        yb.assign(2 * nruns, 0);
        ASFD_CUDA(cudaMemcpyAsync(xb.data(), P->it_xbox, sizeof(int) * xb.size(),
                                  cudaMemcpyDeviceToHost, st));
        ASFD_CUDA(cudaMemcpyAsync(yb.data(), P->it_ybox, sizeof(int) * yb.size(),
                                  cudaMemcpyDeviceToHost, st));
        ASFD_CUDA(cudaStreamSynchronize(st));
        tw = th = 0;
        for (long long c = 0; c < ncb; ++c) tw = std::max(tw, xb[2 * c + 1] - xb[2 * c]);
        for (long long r = 0; r < nruns; ++r) th = std::max(th, yb[2 * r + 1] - yb[2 * r]);
        if (tw <= 0 || th <= 0) return ASFD_OK;
        if ((long long)tw * th * (long long)sizeof(float2) > kItemMaxTileBytes) continue;
        if ((double)items * tw * th > (double)P->nfy * p.m2x) return ASFD_OK;
        break;
    }
    // per band column: the column blocks whose box covers it (consecutive,
    // since the boxes move monotonically with the block); likewise per band row
    const int bx0 = P->band_tx0 * kTileX, bx1 = P->band_tx1 * kTileX;
    const int by0 = P->band_ty0 * kTileY, by1 = P->band_ty1 * kTileY;
    auto build_map = [](const std::vector<int>& box, long long nb, int v0, int v1,
                        std::vector<int>& map) {
        map.assign(v1 - v0, 0);
        long long first = 0;
        for (int v = v0; v < v1; ++v) {
            while (first < nb && box[2 * first + 1] <= v) ++first;
            long long k = first;
            int count = 0;
            while (k < nb && box[2 * k] <= v) {
                if (box[2 * k + 1] <= v) return false;  // not monotone
                ++count;
                ++k;
            }
            if (count > kItemMaxOverlap) return false;
            map[v - v0] = (int)(first | ((long long)count << 24));
        }
        return true;
    };
    // the boxes must move monotonically with the block (run)
    for (long long c = 1; c < ncb; ++c)
        if (xb[2 * c] < xb[2 * c - 2] || xb[2 * c + 1] < xb[2 * c - 1]) return ASFD_OK;
    for (long long r = 1; r < nruns; ++r)
        if (yb[2 * r] < yb[2 * r - 2] || yb[2 * r + 1] < yb[2 * r - 1]) return ASFD_OK;
    std::vector<int> xm, ym;
    if (!build_map(xb, ncb, bx0, bx1, xm) || !build_map(yb, nruns, by0, by1, ym)) return ASFD_OK;
    // every box lies inside the band (the band covers every footprint)
    for (long long c = 0; c < ncb; ++c)
        if (xb[2 * c] < bx0 || xb[2 * c + 1] > bx1) return ASFD_OK;
    for (long long r = 0; r < nruns; ++r)
        if (yb[2 * r] < by0 || yb[2 * r + 1] > by1) return ASFD_OK;
    ASFD_CUDA(cudaMemcpyAsync(P->it_xmap, xm.data(), sizeof(int) * xm.size(), cudaMemcpyHostToDevice, st));
    ASFD_CUDA(cudaMemcpyAsync(P->it_ymap, ym.data(), sizeof(int) * ym.size(), cudaMemcpyHostToDevice, st));
    ASFD_CUDA(cudaStreamSynchronize(st));
    P->it_rows = rows;
    P->it_items = (int)items;
    P->it_ncb = (int)ncb;
    P->it_tw = tw;
    P->it_th = th;
    P->itemtile = true;
    return ASFD_OK;
}

asfd_status launch_spread_itemtile(asfd_plan_s* P, const float2* u1, cudaStream_t st)
{
    ItemArgs ia;
    ia.s = make_spread_args(P, u1);
    ia.s.dense_rows = P->it_rows;
    ia.xbox = P->it_xbox;
    ia.ybox = P->it_ybox;
    ia.scratch = P->rows;  // free until the row pass
    ia.tw = P->it_tw;
    ia.th = P->it_th;
    const size_t smem = kItemWarps * ((size_t)kDenseRingBytes + sizeof(float2) * ia.tw * ia.th);
    const unsigned blocks = (unsigned)((P->it_items + kItemWarps - 1) / kItemWarps);
    switch (P->w) {
#define ASFD_IL(W)                                                                        \
    case W:                                                                               \
        spread_item_kernel<W><<<blocks, 32 * kItemWarps, smem, st>>>(ia, P->it_items);   \
        break;
        ASFD_IL(2) ASFD_IL(3) ASFD_IL(4) ASFD_IL(5) ASFD_IL(6) ASFD_IL(7)
#undef ASFD_IL
        default: return fail(ASFD_ERR_UNSUPPORTED, "item-tile spread widths are 2..7");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "spread_item_kernel launch");
    const int bx0 = P->band_tx0 * kTileX, by0 = P->band_ty0 * kTileY;
    const int bw = (P->band_tx1 - P->band_tx0) * kTileX, bh = (P->band_ty1 - P->band_ty0) * kTileY;
    item_gather_kernel<<<dim3((bw + 127) / 128, (bh + kGatherRows - 1) / kGatherRows), 128, 0, st>>>(
        P->rows, P->it_xbox, P->it_ybox, P->it_xmap, P->it_ymap, bx0, by0, bw, bh, P->it_ncb,
        P->it_tw, P->it_th, P->grid, P->nfx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "item_gather_kernel launch");
    return ASFD_OK;
}

}  // namespace asfd
