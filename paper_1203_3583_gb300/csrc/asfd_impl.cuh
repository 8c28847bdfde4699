// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/asfd.h"

namespace asfd {

// Fine-grid tile owned by one CTA of the spreading kernel, and the source
// tile (block of samples) used for binning.
constexpr int kTileX = 64;
constexpr int kTileY = 64;
constexpr int kSrcTile = 16;  // source tiles are kSrcTile x kSrcTile samples
constexpr int kColTileY = 32; // rows of a tile of the conflict-free spreading kernel
constexpr int kMaxRingWidth = 14;  // widest kernel of the conflict-free spreading path (no spills)
constexpr int kMaxWindowWidth = 7;  // widest kernel of the register-window spreading path
constexpr int kHostColBlocks = 4;   // column blocks whose copies to the host overlap the column pass

// Learned spreading kernel: width kLearnW, per-source-tile polynomial of
// degree kLearnDeg per tap and axis in t = 2 dx - 1, an MLP of kLearnFeat
// inputs and kLearnHidden tanh units, and an even Chebyshev correction of
// kLearnCheb terms per axis on the deconvolution.
constexpr int kLearnW = 4;
constexpr int kLearnDeg = 7;
constexpr int kLearnCoef = kLearnDeg + 1;
constexpr int kLearnTableSize = 2 * kLearnW * kLearnCoef;  // [axis][tap][coef]
constexpr int kLearnFeat = 6;
constexpr int kLearnHidden = 32;
constexpr int kLearnCheb = 6;
// parameter vector layout
constexpr int kLpBase = 0;
constexpr int kLpW1 = kLpBase + kLearnTableSize;
constexpr int kLpB1 = kLpW1 + kLearnHidden * kLearnFeat;
constexpr int kLpW2 = kLpB1 + kLearnHidden;
constexpr int kLpB2 = kLpW2 + kLearnTableSize * kLearnHidden;
constexpr int kLpDx = kLpB2 + kLearnTableSize;
constexpr int kLpDy = kLpDx + kLearnCheb;
constexpr int kLearnParams = kLpDy + kLearnCheb;
constexpr float kLearnOutScale = 1e-3f;  // scale of the MLP's per-tile table correction

// Device status word bits (set by kernels, read by asfd_check_device_status).
constexpr unsigned kStatusBadD1 = 1u;       // non-finite d1 or d1 >= z0
constexpr unsigned kStatusRange = 2u;       // |d1|/z0 above the supported bound
constexpr unsigned kStatusTimeout = 4u;     // a bounded wait ran out
constexpr unsigned kStatusIndex = 8u;       // an index check failed (access skipped)

// Per-source-axis table entry (one per nx, and one per ny).
//   e    = exp(i pi x1^2/(lambda z0))   source chirp |x1|^2/(2 z0) of that axis (FP64 -> FP32)
//   a    = x1^2/(lambda z0)             the same phase in half-turns (FP32, unreduced)
//   s    = alpha x~                     fine-grid offset of the sample at d1 = 0
// and, separately, the integer/fraction split of the storage coordinate
//   alpha x~ + nf/2 (mod nf) = bi + bf.
struct AxisEntry {
    float2 e;
    float a;
    float s;
};
struct AxisPos {
    int bi;
    float bf;
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace asfd

struct asfd_plan_s {
    asfd_params prm{};
    int device = 0;
    int nfx = 0, nfy = 0;
    int w = 0;
    double beta = 0.0;
    double alpha_x = 0.0, alpha_y = 0.0;  // fine cells per source sample at d1 = 0
    double inc_d = 0.0;             // incident depth phase in half-turns per unit d1/z0
    double max_abs_eps = 0.0;

    // tables (device)
    asfd::AxisEntry* ax = nullptr;  // [n1x]
    asfd::AxisEntry* ay = nullptr;  // [n1y]
    asfd::AxisPos* px = nullptr;    // [n1x]
    asfd::AxisPos* py = nullptr;    // [n1y]
    double* bux = nullptr;          // unreduced alpha x~ + nf/2 per axis (plan only)
    double* buy = nullptr;
    float* q = nullptr;             // [n1y][n1x]  d1 / (z0 - d1)
    float2* cx = nullptr;           // [m2x] destination chirp * (-1)^m' / psi_hat
    float2* cy = nullptr;           // [m2y] same, times the global factor
    float2* twx = nullptr;          // [nfx] e^{-2 pi i k/nfx}
    float2* twy = nullptr;          // [nfy]
    double* quad = nullptr;         // [2*nq] Gauss-Legendre nodes z_i and w_i psi(z_i) on [0, w/2]
    int nq = 0;

    // binning
    int ntx = 0, nty = 0;           // fine-grid tiles per axis
    int nstx = 0, nsty = 0;         // source tiles per axis
    float4* src_bbox = nullptr;     // per source tile: unreduced footprint bounds (x0, x1, y0, y1)
    int* tile_off = nullptr;        // [band tiles + 1] CSR offsets
    int* tile_src = nullptr;        // CSR source-tile ids
    int band_tx0 = 0, band_tx1 = 0, band_ty0 = 0, band_ty1 = 0;  // band in tiles
    // conflict-free ("colored") spreading: per band tile the rectangle of
    // source samples whose footprints can reach it, and the minimum column
    // and row strides between samples handled in the same warp step
    int4* tile_rect = nullptr;      // per kTileX x kColTileY tile of the band
    double2* col_range = nullptr;   // per source column: [min, max] of the x storage coordinate
    double2* row_range = nullptr;   // per source row:    [min, max] of the y storage coordinate
    float2* step_min = nullptr;     // per block of min_step_kernel: min spacing along x and y
    bool colored = false;
    bool windowed = false;          // register-window kernel applies (w <= kMaxWindowWidth)
    bool dense = false;             // dense map: register windows flushed with global atomics
    int dense_rows = 0, dense_items = 0;
    // atomic-free spread through per-item shared-memory tiles and an ordered
    // gather (deterministic plans whose samples are >= 1 cell apart in x)
    bool itemtile = false;
    int it_rows = 0, it_items = 0, it_ncb = 0, it_tw = 0, it_th = 0;
    int* it_xbox = nullptr;         // [column blocks][2] first tap column range
    int* it_ybox = nullptr;         // [runs][2] first tap row range
    int* it_xmap = nullptr;         // [band columns] first covering block | count << 24
    int* it_ymap = nullptr;         // [band rows] first covering run | count << 24
    int sx_min = 0, h_min = 0, sxw_min = 0;
    double min_step_x = 0.0, min_step_y = 0.0, row_spread_y = 0.0, col_spread_x = 0.0;
    long long tile_pairs = 0;
    size_t tile_src_cap = 0;

    // work buffers: allocated by the plan on first use, or carved from a
    // caller-owned workspace (asfd_set_workspace)
    float2* grid = nullptr;         // [nfy][nfx]
    float2* rows = nullptr;         // [nfy][m2x] row-FFT output (band rows first)
    char* ws = nullptr;             // caller-owned workspace, or NULL
    size_t ws_bytes = 0;
    bool band_clean = false;        // the band of the fine grid is known to be zero
                                    // (left so by the forward row pass, which
                                    // clears each cell it reads)
    unsigned* status = nullptr;     // device status word
    // learned kernel (kind == ASFD_KERNEL_LEARNED)
    bool learned = false;
    float* ltab = nullptr;          // [source tiles][kLearnTableSize] current tables
    float* lfeat = nullptr;         // [source tiles][kLearnFeat]
    float* lhid = nullptr;          // [source tiles][kLearnHidden] hidden activations
    float* ltgrad = nullptr;        // [source tiles][kLearnTableSize] dL/dtable
    float* lparams = nullptr;       // [kLearnParams]
    float* lgrad = nullptr;
    float* lm = nullptr;            // Adam moments
    float* lv = nullptr;
    int lstep = 0;
    float2* cxb = nullptr;          // base deconvolution/chirp tables (ES, width 4)
    float2* cyb = nullptr;
    float* lcorr = nullptr;         // [m2x + m2y] current deconvolution corrections
    float* lcgrad = nullptr;        // [m2x + m2y] dL/dcorrection
    float2* lu2 = nullptr;          // [m2y][m2x] training forward output (work buffer)
    float2* lres = nullptr;         // [m2y][m2x] loss gradient (work buffer)
    double* lred = nullptr;         // [2] loss reductions
    float2* stage_u1 = nullptr;     // staging for asfd_execute_host (work buffer)
    float2* stage_u2 = nullptr;
    // asfd_execute_host: a stream for the device-to-host copies of column
    // blocks and the events that order them after the column pass
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[asfd::kHostColBlocks + 1] = {};

    std::vector<asfd::DevBuf> owned;
    size_t device_bytes = 0;
};

namespace asfd {

// test hooks: allocations of 2D plans still allowed before injected
// failures (-1: off), and device buffers held by all 2D plans
extern std::atomic<int> g_alloc_budget;
extern std::atomic<long long> g_live_buffers;

// error reporting (thread-local message)
asfd_status fail(asfd_status s, const std::string& msg);
asfd_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define ASFD_CUDA(call)                                                   \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return ::asfd::cuda_fail(_e, #call);       \
    } while (0)

// stage launchers (each returns ASFD_OK or an error with a message)
asfd_status launch_spread(asfd_plan_s* P, const float2* u1, cudaStream_t st);
// deterministic item-tile spread (spread_item.cu): plan set-up and launch
asfd_status plan_build_itemtile(asfd_plan_s* P, cudaStream_t st);
asfd_status launch_spread_itemtile(asfd_plan_s* P, const float2* u1, cudaStream_t st);
// dense plans: add the spread of u1 into `grid` (not cleared; another plan's grid)
asfd_status launch_spread_into(asfd_plan_s* P, const float2* u1, float2* grid, cudaStream_t st);
// row / column passes over the band rows [ty0, ty1) (and columns [tx0, tx1)) in tiles
asfd_status launch_fft_rows_band(asfd_plan_s* P, int ty0, int ty1, int tx0, int tx1,
                                 cudaStream_t st);
asfd_status launch_fft_cols_band(asfd_plan_s* P, int ty0, int ty1, float2* u2, cudaStream_t st);
asfd_status multi_execute(asfd_plan_s* const* plans, const float2* const* u1, int count,
                          float2* u2, cudaStream_t st);
asfd_status launch_fft_rows(asfd_plan_s* P, cudaStream_t st);
asfd_status launch_fft_cols(asfd_plan_s* P, float2* u2, cudaStream_t st);
// column pass over the kept columns [col0, col1) only
asfd_status launch_fft_cols_range(asfd_plan_s* P, float2* u2, int col0, int col1,
                                  cudaStream_t st);
asfd_status launch_fft_lines(int n, int lines, int sign, const float2* in, float2* out,
                             cudaStream_t st);
asfd_status launch_fft_cols_adj(asfd_plan_s* P, const float2* g, cudaStream_t st);
asfd_status launch_fft_rows_adj(asfd_plan_s* P, cudaStream_t st);
asfd_status launch_interp_grad(asfd_plan_s* P, const float2* u1, float2* gu1, float* gd1,
                               cudaStream_t st);

// Warp-item scheduling of the column-walking window kernels (dense spread,
// windowed interpolation): warps of the kernel that the current device keeps
// resident at once (SMs x resident blocks x 4 warps), and the rows per run
// that make the items of 32 columns x rows fill whole waves of those slots
// (two waves when the runs stay at least 32 rows long, else one).
asfd_status dense_spread_warp_slots(int w, bool table, long long* slots);
asfd_status interp_window_warp_slots(int w, long long* slots);
int window_run_rows(long long n1y, long long ncb, long long slots);

// plan helpers
asfd_status plan_validate(const asfd_params* p, int* nfx, int* nfy, double* beta);
// Gauss-Legendre nodes z_i on [0, w/2] and weighted ES values w_i psi(z_i) for
// psi_hat(xi) = 2 sum_i w_i psi(z_i) cos(xi z_i); h = [z..., w psi...]; returns nq.
int es_quadrature(int w, double beta, std::vector<double>& h);
asfd_status direct_sum(const asfd_params* p, const double* d1, const float2* u1, int form,
                       int npts, const int* mx, const int* my, float2* out, cudaStream_t st);
asfd_status plan_alloc(asfd_plan_s* P);
asfd_status build_twiddles(float2* tw, int L, cudaStream_t st);
asfd_status plan_build_tables(asfd_plan_s* P, cudaStream_t st);
asfd_status plan_build_d1(asfd_plan_s* P, const double* d1, cudaStream_t st);
asfd_status plan_alloc_buffer(asfd_plan_s* P, void** p, size_t bytes);

// Work buffers (sizes scale with the grids; everything else a plan holds is
// a table).  Byte offsets of each inside a workspace, 256-byte aligned:
// fine grid, row buffer, the host-execute staging of u1 and u2, and for
// learned plans the training output and residual.
// Kept columns per group of the row-FFT buffer's layout (fft_items.cuh), and
// the buffer's row width: m2x rounded up to whole groups.
constexpr int kRowGroup = 4;
inline size_t row_buffer_width(int m2x) { return ((size_t)m2x + kRowGroup - 1) / kRowGroup * kRowGroup; }

struct WorkLayout {
    size_t grid = 0, rows = 0, stage_u1 = 0, stage_u2 = 0, lu2 = 0, lres = 0, total = 0;
};
WorkLayout work_layout(const asfd_params& p, int nfx, int nfy);
enum WorkNeed : unsigned { kWorkTransform = 1u, kWorkStaging = 2u, kWorkTraining = 4u };
// Makes the work buffers in `need` available: carved from the workspace when
// one is set, else allocated by the plan (once).
asfd_status plan_ensure_work(asfd_plan_s* P, unsigned need);
// Attaches a caller-owned workspace (releasing the plan's own work buffers)
// or, with ws == NULL, detaches it.
asfd_status plan_set_workspace(asfd_plan_s* P, void* ws, size_t bytes);
// learned kernel
asfd_status learned_init(asfd_plan_s* P, cudaStream_t st);
asfd_status learned_refresh(asfd_plan_s* P, cudaStream_t st);   // features -> tables, deconvolution
asfd_status learned_features(asfd_plan_s* P, cudaStream_t st);
asfd_status learned_train_step(asfd_plan_s* P, const float2* u1, const float2* ref, float lr,
                               double* loss_out, cudaStream_t st);
asfd_status learned_gradient(asfd_plan_s* P, const float2* u1, const float2* ref, cudaStream_t st);
asfd_status learned_read_loss(asfd_plan_s* P, double* loss_out, cudaStream_t st);

}  // namespace asfd
