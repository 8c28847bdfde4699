// Batched transform: many surfaces (sizes, wavelengths and distances of
// their own), each with its own plan (tables, binning, work buffers), in one
// of two schedules, both replayed from CUDA graphs.
//
// Streams (the default): each surface's three kernels (spread, row FFT,
// column FFT) run in order on one of up to kBatchStreams streams of the
// batch, forked from and joined to the caller's stream; surfaces are dealt
// to the streams largest first, each to the stream with the least work so
// far, so that the small surfaces' kernels fill the SMs the large ones leave
// idle in their tails.  The fork, the launches and the join are captured
// once per set of field pointers and replayed.
//
// Persistent: ONE cooperative kernel over the whole batch, stage-major:
//   stage Z  (when some surface uses the dense spread) clear the bands of
//            those surfaces, then a grid barrier;
//   stage 0  every block takes the shared-memory-atomic tiles of surfaces
//            that need them, then every warp takes (surface, item) items: a
//            conflict-free fine-grid tile, or a dense item (32 source columns
//            whose register windows are flushed with atomic adds);
//   grid barrier (cooperative groups: all blocks are co-resident, as the
//            cooperative launch guarantees, so the barrier cannot deadlock);
//   stage 1  every block takes (surface, row group) items of the row FFT;
//   grid barrier;
//   stage 2  every block takes (surface, column group) items of the column
//            FFT with deconvolution and destination chirp.
// Items of one stage are independent, so the only waits are the two grid
// barriers of the CUDA runtime.  The per-surface argument blocks live in
// device memory and are refreshed from a pinned host copy by a memcpy node of
// the same graph, so one graph launch runs a whole batch for new field
// pointers.  (At 24 surfaces of 256^2..2048^2 the stage barriers leave SMs
// idle while the last items of a stage finish: 1.86 ms against 0.92 ms for
// the stream schedule.)
#include <cooperative_groups.h>

#include <algorithm>
#include <string>
#include <vector>

#include "asfd_impl.cuh"
#include "fft_items.cuh"
#include "spread.cuh"

namespace cg = cooperative_groups;

namespace asfd {

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchWarps = kBatchThreads / 32;
constexpr int kBatchMaxNf = 4096;  // persistent schedule: largest fine grid
constexpr int kBatchStreams = 16;  // stream schedule: streams of a batch
using BTile = ColoredTile<kTileX, kColTileY>;

struct BatchSurf {
    SpreadArgs sa;
    RowArgs ra;
    ColArgs ca;
    int nfx, nfy;
    int windowed;      // conflict-free tiles use the register-window form
    int tile0, ntile;  // first item and count of conflict-free (warp) spread tiles
    int dense0, ndense;  // first item and count of dense (global-atomic) warp items
    int atile0, natile;  // first item and count of atomic (block) spread tiles
    int row0, nrow;    // row-pass items
    int col0, ncol;    // column-pass items
};

// Surface owning item `it` of a stage (items are laid out surface by surface).
template <int Which>
__device__ __forceinline__ int owner(const BatchSurf* S, int n, int it)
{
    int s = 0;
    for (int k = 1; k < n; ++k) {
        const int start = Which == 0   ? S[k].tile0
                          : Which == 1 ? S[k].row0
                          : Which == 2 ? S[k].col0
                          : Which == 3 ? S[k].atile0
                                       : S[k].dense0;
        if (it >= start) s = k;
    }
    return s;
}

// The stages run out of line so that each keeps its own register allocation
// (the kernel's register count is the largest of them).
template <int W>
__device__ __noinline__ void batch_window_tile(const SpreadArgs& a, int t, float2* sm, int lane)
{
    if constexpr (W <= kMaxWindowWidth) window_tile<W, kTileX, kColTileY, false>(a, t, sm, lane);
}

template <int W>
__device__ __noinline__ void batch_colored_tile(const SpreadArgs& a, int t, float2* sm, int lane)
{
    colored_tile<W, kTileX, kColTileY, false>(a, t, sm, lane);
}

template <int W>
__device__ __noinline__ void batch_dense_item(const SpreadArgs& a, int it, int lane, char* ring)
{
    if constexpr (W <= kMaxWindowWidth) window_atomic_item<W>(a, it, lane, ring);
}

template <int L>
__device__ __forceinline__ void batch_row(const BatchSurf& s, int it, float2* sm, int tid)
{
    if constexpr (RowCfg<L>::THREADS == kBatchThreads) rows_body<L>(s.ra, it, sm, tid);
}

template <int L>
__device__ __forceinline__ void batch_col(const BatchSurf& s, int it, float2* sm, int tid)
{
    constexpr int LPC = kBatchThreads / (L / 16);
    if constexpr (LPC >= 1 && LPC * (L / 16) == kBatchThreads) cols_body<L, LPC>(s.ca, it, sm, tid);
}

template <int W>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const BatchSurf* __restrict__ S, int n,
                                                              int ntile, int ndense, int natile,
                                                              int nrow, int ncol)
{
    extern __shared__ __align__(16) float2 sm[];
    cg::grid_group grid = cg::this_grid();
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

    // stage Z: the dense items accumulate with atomics: clear their bands
    if (ndense > 0) {
        const size_t gt = (size_t)blockIdx.x * kBatchThreads + tid;
        const size_t gn = (size_t)gridDim.x * kBatchThreads;
        for (int s = 0; s < n; ++s) {
            if (S[s].ndense == 0) continue;
            const SpreadArgs& a = S[s].sa;
            const int w2 = a.band_ntx * (kTileX / 2);  // float4 per band row
            const size_t total = (size_t)S[s].ra.nrows * w2;
            float4* g4 = reinterpret_cast<float4*>(a.grid + (size_t)S[s].ra.row0 * a.nfx +
                                                   a.band_tx0 * kTileX);
            for (size_t i = gt; i < total; i += gn)
                g4[(i / w2) * (a.nfx / 2) + i % w2] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        grid.sync();
    }

    // stage 0a: spread of surfaces that need the atomic kernel (block items)
    float* tre = reinterpret_cast<float*>(sm);
    float* tim = tre + kTileX * kTileY;
    for (int it = blockIdx.x; it < natile; it += gridDim.x) {
        const int s = owner<3>(S, n, it);
        atomic_tile<W, false>(S[s].sa, it - S[s].atile0, tre, tim, tid, kBatchThreads);
        __syncthreads();
    }
    __syncthreads();

    // stage 0b: conflict-free tiles and dense items (warp items)
    float2* wsm = sm + warp * BTile::SLOTS;
    for (int it = blockIdx.x * kBatchWarps + warp; it < ntile + ndense;
         it += gridDim.x * kBatchWarps) {
        if (it < ntile) {
            const int s = owner<0>(S, n, it);
            if (S[s].windowed) batch_window_tile<W>(S[s].sa, it - S[s].tile0, wsm, lane);
            else batch_colored_tile<W>(S[s].sa, it - S[s].tile0, wsm, lane);
        } else {
            const int s = owner<4>(S, n, it - ntile);
            batch_dense_item<W>(S[s].sa, it - ntile - S[s].dense0, lane,
                                reinterpret_cast<char*>(wsm));
        }
    }
    grid.sync();

    // stage 1: row FFT (block items; the item index is block-uniform)
    for (int it = blockIdx.x; it < nrow; it += gridDim.x) {
        const int s = owner<1>(S, n, it);
        const BatchSurf& b = S[s];
        switch (b.nfx) {
            case 64: batch_row<64>(b, it - b.row0, sm, tid); break;
            case 128: batch_row<128>(b, it - b.row0, sm, tid); break;
            case 256: batch_row<256>(b, it - b.row0, sm, tid); break;
            case 512: batch_row<512>(b, it - b.row0, sm, tid); break;
            case 1024: batch_row<1024>(b, it - b.row0, sm, tid); break;
            case 2048: batch_row<2048>(b, it - b.row0, sm, tid); break;
            case 4096: batch_row<4096>(b, it - b.row0, sm, tid); break;
            default: break;
        }
        __syncthreads();
    }
    grid.sync();

    // stage 2: column FFT + deconvolution + destination chirp
    for (int it = blockIdx.x; it < ncol; it += gridDim.x) {
        const int s = owner<2>(S, n, it);
        const BatchSurf& b = S[s];
        switch (b.nfy) {
            case 64: batch_col<64>(b, it - b.col0, sm, tid); break;
            case 128: batch_col<128>(b, it - b.col0, sm, tid); break;
            case 256: batch_col<256>(b, it - b.col0, sm, tid); break;
            case 512: batch_col<512>(b, it - b.col0, sm, tid); break;
            case 1024: batch_col<1024>(b, it - b.col0, sm, tid); break;
            case 2048: batch_col<2048>(b, it - b.col0, sm, tid); break;
            case 4096: batch_col<4096>(b, it - b.col0, sm, tid); break;
            default: break;
        }
        __syncthreads();
    }
}

size_t batch_smem_bytes()
{
    const size_t spread = sizeof(float2) * (size_t)BTile::SLOTS * kBatchWarps;
    const size_t atomic = 2 * sizeof(float) * kTileX * kTileY;
    const size_t fft = RowCfg<kBatchMaxNf>::SMEM_BYTES;  // largest per-block FFT footprint
    return std::max(std::max(spread, atomic), fft);
}

}  // namespace
}  // namespace asfd

struct asfd_batch_s {
    std::vector<asfd_plan> plans;
    int device = 0;
    int width = 0;
    int schedule = ASFD_BATCH_STREAMS;
    // persistent schedule (when its limits hold)
    bool persistent_ok = false;
    asfd::BatchSurf* host = nullptr;  // pinned
    asfd::BatchSurf* dev = nullptr;
    int ntile = 0, ndense = 0, natile = 0, nrow = 0, ncol = 0;
    int grid_blocks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_ok = false;
    // stream schedule
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
    std::vector<int> order, lane;     // surfaces largest first; stream of each
    cudaGraphExec_t sexec = nullptr;  // for the field pointers in key1 / key2
    std::vector<const float*> key1;
    std::vector<float*> key2;
    bool warm = false;                // a direct run has set the plans' band state
};

namespace asfd {

namespace {

template <int W>
cudaError_t launch_batch(asfd_batch_s* B, cudaStream_t st)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(batch_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)batch_smem_bytes());
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(B->grid_blocks);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = batch_smem_bytes();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const BatchSurf* S = B->dev;
    const int n = (int)B->plans.size();
    return cudaLaunchKernelEx(&cfg, batch_kernel<W>, S, n, B->ntile, B->ndense, B->natile, B->nrow,
                              B->ncol);
}

cudaError_t launch_batch_w(asfd_batch_s* B, cudaStream_t st)
{
    switch (B->width) {
        case 4: return launch_batch<4>(B, st);
        case 5: return launch_batch<5>(B, st);
        case 6: return launch_batch<6>(B, st);
        case 7: return launch_batch<7>(B, st);
        case 8: return launch_batch<8>(B, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int W>
cudaError_t batch_occupancy(int* blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batch_smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<W>,
                                                         kBatchThreads, batch_smem_bytes());
}

cudaError_t batch_occupancy_w(int w, int* blocks_per_sm)
{
    switch (w) {
        case 4: return batch_occupancy<4>(blocks_per_sm);
        case 5: return batch_occupancy<5>(blocks_per_sm);
        case 6: return batch_occupancy<6>(blocks_per_sm);
        case 7: return batch_occupancy<7>(blocks_per_sm);
        case 8: return batch_occupancy<8>(blocks_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

void batch_free(asfd_batch_s* B)
{
    if (B->sexec) cudaGraphExecDestroy(B->sexec);
    for (cudaEvent_t e : B->joins) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    for (cudaStream_t t : B->streams) cudaStreamDestroy(t);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->dev) cudaFree(B->dev);
    if (B->host) cudaFreeHost(B->host);
    for (asfd_plan p : B->plans) asfd_destroy(p);
    delete B;
}

// Streams of the stream schedule and the dealing of surfaces to them.
cudaError_t streams_setup(asfd_batch_s* B)
{
    const int n = (int)B->plans.size();
    const int k = std::min(n, kBatchStreams);
    for (int i = 0; i < k; ++i) {
        cudaStream_t t = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        B->streams.push_back(t);
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        B->joins.push_back(ev);
    }
    cudaError_t e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    // work ~ source samples + the fine-grid band the FFTs transform
    std::vector<double> cost(n), load(k, 0.0);
    for (int i = 0; i < n; ++i) {
        const asfd_plan_s* P = B->plans[i];
        const double band = (double)(P->band_ty1 - P->band_ty0) * kTileY * P->nfx;
        cost[i] = (double)P->prm.n1x * P->prm.n1y + band;
    }
    B->order.resize(n);
    for (int i = 0; i < n; ++i) B->order[i] = i;
    std::stable_sort(B->order.begin(), B->order.end(),
                     [&](int a, int b) { return cost[a] > cost[b]; });
    B->lane.assign(n, 0);
    for (int i : B->order) {
        const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        B->lane[i] = j;
        load[j] += cost[i];
    }
    return cudaSuccess;
}

// Fork from `o`, each surface's three kernels on its stream, join into `o`.
asfd_status streams_enqueue(asfd_batch_s* B, const float* const* u1, float* const* u2,
                            cudaStream_t o)
{
    ASFD_CUDA(cudaEventRecord(B->fork, o));
    for (cudaStream_t t : B->streams) ASFD_CUDA(cudaStreamWaitEvent(t, B->fork, 0));
    for (int i : B->order) {
        asfd_plan_s* P = B->plans[i];
        const cudaStream_t t = B->streams[B->lane[i]];
        asfd_status r = launch_spread(P, reinterpret_cast<const float2*>(u1[i]), t);
        if (r == ASFD_OK) r = launch_fft_rows(P, t);
        if (r == ASFD_OK) r = launch_fft_cols(P, reinterpret_cast<float2*>(u2[i]), t);
        if (r != ASFD_OK) return r;
    }
    for (size_t j = 0; j < B->streams.size(); ++j) {
        ASFD_CUDA(cudaEventRecord(B->joins[j], B->streams[j]));
        ASFD_CUDA(cudaStreamWaitEvent(o, B->joins[j], 0));
    }
    return ASFD_OK;
}

// The stream schedule: the first call runs its launches directly (so that
// the plans' band state is that of a run); later calls replay a graph of the
// same launches, captured again when the field pointers change.
asfd_status streams_execute(asfd_batch_s* B, const float* const* u1, float* const* u2,
                            cudaStream_t st)
{
    const int n = (int)B->plans.size();
    bool same = B->sexec != nullptr;
    for (int i = 0; same && i < n; ++i) same = B->key1[i] == u1[i] && B->key2[i] == u2[i];
    if (same) {
        ASFD_CUDA(cudaGraphLaunch(B->sexec, st));
        return ASFD_OK;
    }
    if (!B->warm) {
        asfd_status r = streams_enqueue(B, u1, u2, st);
        if (r == ASFD_OK) B->warm = true;
        return r;
    }
    if (B->sexec) {
        cudaGraphExecDestroy(B->sexec);
        B->sexec = nullptr;
    }
    // capture on a stream of our own (the caller's may be the legacy
    // default stream, which cannot be captured), then launch on the caller's
    cudaStream_t cap = nullptr;
    ASFD_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    asfd_status r = ASFD_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        r = streams_enqueue(B, u1, u2, cap);
        e = cudaStreamEndCapture(cap, &g);
    }
    if (r == ASFD_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&B->sexec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (r != ASFD_OK) return r;
    if (e != cudaSuccess || !B->sexec) {
        B->sexec = nullptr;
        return cuda_fail(e != cudaSuccess ? e : cudaErrorUnknown, "capture of the batch's streams");
    }
    B->key1.assign(u1, u1 + n);
    B->key2.assign(u2, u2 + n);
    ASFD_CUDA(cudaGraphLaunch(B->sexec, st));
    return ASFD_OK;
}

}  // namespace
}  // namespace asfd

using namespace asfd;

extern "C" {

asfd_status asfd_batch_create(asfd_batch* out, const asfd_params* params,
                              const double* const* d1_devs, int count, void* stream)
{
    clear_error();
    if (!out || !params || !d1_devs || count <= 0)
        return fail(ASFD_ERR_ARG, "out, params and d1 arrays must be non-NULL, count > 0");
    *out = nullptr;
    const int w = params[0].kernel_width;
    bool common = true;
    for (int i = 0; i < count; ++i) {
        if (params[i].kind != ASFD_KERNEL_ES)
            return fail(ASFD_ERR_UNSUPPORTED, "a batch uses the ES kernel");
        if (!d1_devs[i]) return fail(ASFD_ERR_ARG, "d1 pointer is NULL");
        common = common && params[i].kernel_width == w;
    }
    asfd_batch_s* B = new (std::nothrow) asfd_batch_s();
    if (!B) return fail(ASFD_ERR_NOMEM, "host allocation");
    B->width = w;
    // the persistent kernel is instantiated for one common width in 4..8 and
    // fine grids up to kBatchMaxNf
    B->persistent_ok = common && w >= 4 && w <= 8;
    asfd_status s = [&]() -> asfd_status {
        ASFD_CUDA(cudaGetDevice(&B->device));
        for (int i = 0; i < count; ++i) {
            asfd_plan p = nullptr;
            asfd_status r = asfd_plan_create(&p, &params[i], d1_devs[i], stream);
            if (r != ASFD_OK) return r;
            B->plans.push_back(p);
            if (p->nfx > kBatchMaxNf || p->nfy > kBatchMaxNf) B->persistent_ok = false;
            // both schedules read the plans' work buffers
            r = plan_ensure_work(p, kWorkTransform);
            if (r != ASFD_OK) return r;
        }
        ASFD_CUDA(streams_setup(B));
        if (!B->persistent_ok) return ASFD_OK;
        ASFD_CUDA(cudaMallocHost(&B->host, sizeof(BatchSurf) * count));
        ASFD_CUDA(cudaMalloc(&B->dev, sizeof(BatchSurf) * count));
        int nt = 0, nd = 0, na = 0, nr = 0, nc = 0;
        for (int i = 0; i < count; ++i) {
            asfd_plan_s* P = B->plans[i];
            BatchSurf& b = B->host[i];
            b.sa = make_spread_args(P, nullptr);
            b.ra = make_row_args(P);
            b.ca = make_col_args(P, nullptr);
            b.nfx = P->nfx;
            b.nfy = P->nfy;
            b.windowed = P->colored && P->windowed ? 1 : 0;
            const int band_tiles = (P->band_tx1 - P->band_tx0) * (P->band_ty1 - P->band_ty0);
            b.tile0 = nt;
            b.ntile = P->colored ? band_tiles * (kTileY / kColTileY) : 0;
            b.dense0 = nd;
            b.ndense = P->dense ? P->dense_items : 0;
            b.atile0 = na;
            b.natile = (P->colored || P->dense) ? 0 : band_tiles;
            b.row0 = nr;
            const int row_lpc = P->nfx >= 4096 ? 1 : 4096 / P->nfx;  // RowCfg<nfx>::LPC
            b.nrow = (b.ra.nrows + row_lpc - 1) / row_lpc;
            const int col_lpc = kBatchThreads / (P->nfy / 16);
            b.col0 = nc;
            b.ncol = (P->prm.m2x + col_lpc - 1) / col_lpc;
            nt += b.ntile;
            nd += b.ndense;
            na += b.natile;
            nr += b.nrow;
            nc += b.ncol;
        }
        B->ntile = nt;
        B->ndense = nd;
        B->natile = na;
        B->nrow = nr;
        B->ncol = nc;
        int per_sm = 0, sms = 0;
        ASFD_CUDA(batch_occupancy_w(w, &per_sm));
        ASFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device));
        if (per_sm < 1) {
            B->persistent_ok = false;  // the persistent kernel does not fit on an SM
            return ASFD_OK;
        }
        B->grid_blocks = per_sm * sms;
        return ASFD_OK;
    }();
    if (s != ASFD_OK) {
        const std::string msg = asfd_last_error();  // batch_free's plan destroys clear it
        batch_free(B);
        return fail(s, msg);
    }
    *out = B;
    return ASFD_OK;
}

asfd_status asfd_batch_set_schedule(asfd_batch B, int schedule)
{
    clear_error();
    if (!B) return fail(ASFD_ERR_ARG, "batch is NULL");
    if (schedule != ASFD_BATCH_STREAMS && schedule != ASFD_BATCH_PERSISTENT)
        return fail(ASFD_ERR_ARG, "schedule must be ASFD_BATCH_STREAMS or ASFD_BATCH_PERSISTENT");
    if (schedule == ASFD_BATCH_PERSISTENT && !B->persistent_ok)
        return fail(ASFD_ERR_UNSUPPORTED, "the persistent schedule needs one common width in "
                                          "4..8 and fine grids up to 4096");
    if (schedule == B->schedule) return ASFD_OK;
    // the persistent kernel clears the dense surfaces' bands itself and
    // leaves them as the row stage read them; the stream schedule's plans
    // track their band state: start it over
    for (asfd_plan p : B->plans) p->band_clean = false;
    if (B->sexec) cudaGraphExecDestroy(B->sexec);
    B->sexec = nullptr;
    B->warm = false;
    B->schedule = schedule;
    return ASFD_OK;
}

asfd_status asfd_batch_execute(asfd_batch B, const float* const* u1_devs, float* const* u2_devs,
                               void* stream)
{
    clear_error();
    if (!B || !u1_devs || !u2_devs) return fail(ASFD_ERR_ARG, "NULL argument");
    const int n = (int)B->plans.size();
    for (int i = 0; i < n; ++i)
        if (!u1_devs[i] || !u2_devs[i]) return fail(ASFD_ERR_ARG, "NULL field pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int prev = 0;
    ASFD_CUDA(cudaGetDevice(&prev));
    if (prev != B->device) ASFD_CUDA(cudaSetDevice(B->device));
    if (B->schedule == ASFD_BATCH_STREAMS) {
        const asfd_status r = streams_execute(B, u1_devs, u2_devs, st);
        if (prev != B->device) cudaSetDevice(prev);
        return r;
    }
    // the graph's memcpy node reads the pinned host table at launch time;
    // wait until a previous launch has consumed it before rewriting it
    ASFD_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) {
        B->host[i].sa.u1 = reinterpret_cast<const float2*>(u1_devs[i]);
        B->host[i].ca.u2 = reinterpret_cast<float2*>(u2_devs[i]);
    }
    asfd_status s = ASFD_OK;
    if (!B->exec) {
        // capture upload + cooperative launch once; fall back to direct
        // launches if the runtime cannot capture the cooperative kernel
        cudaStream_t cap = nullptr;
        bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            cudaError_t e1 = cudaMemcpyAsync(B->dev, B->host, sizeof(BatchSurf) * n,
                                             cudaMemcpyHostToDevice, cap);
            cudaError_t e2 = launch_batch_w(B, cap);
            cudaGraph_t g = nullptr;
            cudaError_t e3 = cudaStreamEndCapture(cap, &g);
            ok = e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && g;
            if (ok) ok = cudaGraphInstantiate(&B->exec, g, 0) == cudaSuccess;
            if (ok) B->graph = g;
            else if (g) cudaGraphDestroy(g);
        }
        if (cap) cudaStreamDestroy(cap);
        cudaGetLastError();  // clear a failed capture
        B->graph_ok = ok;
        if (!ok) B->exec = nullptr;
    }
    if (B->graph_ok) {
        cudaError_t e = cudaGraphLaunch(B->exec, st);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaGraphLaunch of the batch");
    } else {
        cudaError_t e = cudaMemcpyAsync(B->dev, B->host, sizeof(BatchSurf) * n,
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_batch_w(B, st);
        if (e != cudaSuccess) s = cuda_fail(e, "batch kernel launch");
    }
    if (prev != B->device) cudaSetDevice(prev);
    return s;
}

asfd_status asfd_batch_get_info(asfd_batch B, asfd_batch_info* info)
{
    clear_error();
    if (!B || !info) return fail(ASFD_ERR_ARG, "NULL argument");
    info->surfaces = (int)B->plans.size();
    info->schedule = B->schedule;
    info->persistent_ok = B->persistent_ok ? 1 : 0;
    info->streams = (int)B->streams.size();
    info->blocks = B->grid_blocks;
    info->threads_per_block = kBatchThreads;
    info->spread_items = B->ntile + B->ndense + B->natile;
    info->row_items = B->nrow;
    info->col_items = B->ncol;
    info->graph = B->schedule == ASFD_BATCH_STREAMS ? (B->sexec ? 1 : 0) : (B->graph_ok ? 1 : 0);
    long long src = 0;
    for (asfd_plan p : B->plans) src += (long long)p->prm.n1x * p->prm.n1y;
    info->source_samples = src;
    return ASFD_OK;
}

asfd_status asfd_batch_destroy(asfd_batch B)
{
    clear_error();
    if (!B) return ASFD_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(B->device);
    cudaDeviceSynchronize();
    batch_free(B);
    cudaSetDevice(prev);
    return ASFD_OK;
}

}  // extern "C"
