/*
 * asfd.h -- C ABI of the arbitrary-shape-surface Fresnel diffraction library
 * (Shimobaba, Masuda, Ito, "Arbitrary shape surface Fresnel diffraction").
 *
 * The library evaluates Eq. 8 of the paper: the Fresnel-approximated Huygens
 * sum from a sampled source surface u1(x1, d1(x1)) to a planar destination,
 * as a non-uniform-to-uniform (type-1) 2D NUFFT.  In its discretised form
 * (Eq. 7, the "Fourier form", with the cross-term sign of Eqs. 4-5 and 9):
 *
 *   u2[m] = exp(ik(z0 + |x2|^2/(2 z0))) / (i lambda z0)
 *           * sum_n p1x p1y u1[n] exp(ik d1[n])
 *                   exp(ik(-d1[n] + |x1[n]|^2 / (2 r0[n])))
 *                   exp(-ik x1[n].x2[m] / r0[n]),     r0 = z0 - d1,
 *
 * with x1 = ((nx - N1x/2) p1x, (ny - N1y/2) p1y) and
 *      x2 = ((mx - M2x/2) p2x, (my - M2y/2) p2y).
 * The incident wave exp(ik d1) is the normally incident plane wave of Sec. 2;
 * asfd_params can tilt it (incidence_sx/sy: exp(ik(sx x + sy y + sz d1))) and
 * move the source grid off the axis (offset_x/y added to x1).
 *
 * Conventions for every entry point:
 *  - Complex arrays are interleaved (re, im) float pairs, row-major [y][x]
 *    with x fastest: u1 is [n1y][n1x], u2 is [m2y][m2x].
 *  - "device" pointers are CUDA global-memory pointers on the device that was
 *    current when the plan was created; "host" pointers are host memory
 *    (page-locked for full copy speed).  All memory passed in is owned by the
 *    caller and only borrowed for the duration of the call (or, for
 *    asynchronous calls, until the work queued on `stream` completes).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is queued asynchronously on it unless stated.
 *  - A plan owns its device tables; its work buffers are its own (allocated
 *    on first use) or carved from a caller-owned workspace
 *    (asfd_set_workspace).  Calls on one plan must not overlap in time (one
 *    stream at a time).
 *  - No exceptions cross the ABI.  Every call returns an asfd_status; a
 *    one-line description of the last failure on the calling thread is
 *    available from asfd_last_error().
 */
#ifndef ASFD_H
#define ASFD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ASFD_OK = 0,
    ASFD_ERR_ARG = 1,          /* invalid argument: sizes, NULL pointers, NaN d1, d1 >= z0 */
    ASFD_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed            */
    ASFD_ERR_NOMEM = 3,        /* device or host allocation failed                        */
    ASFD_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out (reserved: no kernel */
                               /* of this library spins on a device flag, so none sets it) */
    ASFD_ERR_UNSUPPORTED = 5,  /* valid request outside what the library implements       */
    ASFD_ERR_STATE = 6         /* call not valid in the plan's current state              */
} asfd_status;

typedef enum {
    ASFD_KERNEL_ES = 0,        /* exponential-of-semicircle spreading kernel              */
    ASFD_KERNEL_LEARNED = 1    /* per-tile tabulated kernel (see asfd_set_learned_table)  */
} asfd_kernel_kind;

/* Geometry and NUFFT parameters of a plan (SI units). */
typedef struct {
    int n1x, n1y;        /* source samples; even, 2..65536                             */
    double p1x, p1y;     /* source pitch [m], > 0                                       */
    int m2x, m2y;        /* destination samples; even                                   */
    double p2x, p2y;     /* destination pitch [m], > 0                                  */
    double lambda;       /* wavelength [m], > 0                                         */
    double z0;           /* source-to-destination distance [m], > 0                     */
    double sigma;        /* oversampling factor in [1.25, 4]; sigma*m2x and sigma*m2y   */
                         /* must be powers of two in [64, 16384] (typically sigma = 2)  */
    int kernel_width;    /* spreading kernel width w in fine-grid cells, 2..16          */
    double es_beta;      /* ES shape parameter; 0 selects 2.30*w at sigma = 2           */
    asfd_kernel_kind kind;
    int deterministic;   /* 0 (fastest): for monotone maps and ES widths up to 7 the    */
                         /*   spread accumulates register windows into the fine grid   */
                         /*   with float atomic adds, so the last bits of a result may  */
                         /*   differ from run to run; 1: conflict-free shared-memory    */
                         /*   tiles without atomics where the map allows them (results */
                         /*   bit-identical run to run), shared-memory atomics else     */
    double incidence_sx, incidence_sy; /* direction cosines of the incident plane wave */
                         /*   u_I = exp(ik(sx x1 + sy y1 + sz d1)), sz = sqrt(1 - sx^2  */
                         /*   - sy^2), sx^2 + sy^2 < 1; 0, 0: normal incidence, the     */
                         /*   exp(ik d1) of Sec. 2 (incidence is an extension)         */
    double offset_x, offset_y; /* position [m] of the source grid's centre sample     */
                         /*   (n1/2): x1 = (n - n1/2) p1 + offset; 0 puts the grid on   */
                         /*   the axis as in Sec. 2; used to place several surfaces     */
} asfd_params;

typedef struct asfd_plan_s* asfd_plan;

/* Read-only facts about a built plan (for tests and reports). */
typedef struct {
    int nfx, nfy;            /* oversampled (fine) grid size                            */
    int tile_x, tile_y;      /* fine-grid tile of the spreading kernel                  */
    int band_x0, band_x1;    /* touched fine-grid columns [x0, x1) (storage coords)     */
    int band_y0, band_y1;    /* touched fine-grid rows    [y0, y1)                      */
    int spread_tiles;        /* output tiles the spreading kernel processes             */
    long long tile_pairs;    /* (output tile, source tile) pairs in the binning of the  */
                             /*    shared-memory-atomic spread (spread_kind 1; else 0)  */
    double es_beta;          /* ES beta in use                                          */
    double max_abs_eps;      /* max |d1| / z0 over the surface                          */
    size_t device_bytes;     /* device memory owned by the plan                         */
    int spread_kind;         /* 0: conflict-free warp tiles (no atomics) -- used when   */
                             /*    the map n -> g is monotone with positive spacing and */
                             /*    no footprint wraps; 1: shared-memory atomics;        */
                             /*    2: conflict-free warp tiles with a sliding register  */
                             /*    window per lane (ES widths up to 7); 3: dense maps   */
                             /*    (many samples per cell): register windows flushed    */
                             /*    to the fine grid with atomic adds (widths up to 7);  */
                             /*    4: deterministic plans whose samples are at least a  */
                             /*    fine cell apart in x (widths up to 7): register      */
                             /*    windows flushed into per-item shared-memory tiles in */
                             /*    a fixed order, then an ordered gather (no atomics)   */
    int stride_x, stride_y;  /* sample strides between lanes of one warp step (0, 2)    */
    int run_rows;            /* source rows per lane run of the register-window spread  */
                             /*    (spread_kind 3; 0 otherwise)                         */
} asfd_plan_info;

/*
 * Create a plan for the geometry `p` and the height map `d1_dev`
 * (device, FP64, [n1y][n1x], metres, positive toward the destination; read
 * during the call only).  Builds, on the device and in FP64, the per-axis
 * phase and position tables (source chirp |x1|^2/(2 z0) and the fine-grid
 * coordinate of every sample, Sec. 2 Eqs. 4-8), the destination chirp and
 * kernel-deconvolution tables, the per-sample r0 correction, and the binning
 * of samples to fine-grid tiles.  Synchronises `stream` once (binning).
 * Errors: ASFD_ERR_ARG for invalid sizes/pitches, non-finite d1, d1 >= z0;
 * ASFD_ERR_UNSUPPORTED when max |d1|/z0 > 0.1 or a size is out of range;
 * ASFD_ERR_NOMEM / ASFD_ERR_CUDA on allocation or launch failure.
 * On failure *out is set to NULL and nothing is leaked.  The work buffers
 * (fine grid and row buffer) are not allocated here: see asfd_set_workspace.
 */
asfd_status asfd_plan_create(asfd_plan* out, const asfd_params* p, const double* d1_dev,
                             void* stream);

/* Replace the plan's height map (same sizes) and rebuild the d1-dependent
 * tables and binning.  Same errors as asfd_plan_create; the plan is unchanged
 * on failure. */
asfd_status asfd_plan_update_d1(asfd_plan plan, const double* d1_dev, void* stream);

/*
 * Caller-owned work memory.  A plan holds two kinds of device memory: its
 * tables (O(n1x + n1y + m2x + m2y) plus O(tiles); built by asfd_plan_create)
 * and its work buffers, whose sizes scale with the grids of the NUFFT that
 * evaluates Eq. 8 (Sec. 2): the sigma-oversampled fine grid
 * (sigma m2x x sigma m2y complex), the row-FFT output (sigma m2y x m2x
 * complex), the staging of u1 and u2 for asfd_execute_host, and for learned
 * plans the training output and residual (m2x x m2y complex each).
 *
 * asfd_workspace_bytes(p): bytes of a workspace holding every work buffer of
 * a plan with parameters p (each region 256-byte aligned); 0 if p is invalid
 * (asfd_last_error() says why).  Touches no device.
 *
 * asfd_set_workspace(plan, ws_dev, bytes): from now on the plan carves all of
 * its work buffers from ws_dev (device memory of the plan's device, 256-byte
 * aligned, bytes >= asfd_workspace_bytes of the plan's parameters), which the
 * caller owns (e.g. a tensor of PyTorch's caching allocator) and must keep
 * alive, and not use otherwise, while calls on the plan can run.  Work
 * buffers the plan had allocated itself are freed.  With a workspace set, no
 * call on the plan allocates device memory.  ws_dev = NULL with bytes = 0
 * detaches the workspace; the plan then allocates its own work buffers again
 * on first use.  Without a workspace a plan allocates its work buffers at the
 * first call that needs them (asfd_execute, asfd_execute_stage,
 * asfd_execute_host, asfd_adjoint, the learned training calls, and
 * asfd_multi_execute for its first plan): make one such call, or set a
 * workspace, before capturing calls into a CUDA graph.  Synchronises the
 * device (work queued on the old buffers must finish).  Several plans may
 * share one workspace only if their calls never overlap in time.
 * Errors: ASFD_ERR_ARG (NULL plan, too small, misaligned, not device memory
 * of the plan's device, NULL with bytes != 0), ASFD_ERR_CUDA.
 */
size_t asfd_workspace_bytes(const asfd_params* p);
asfd_status asfd_set_workspace(asfd_plan plan, void* ws_dev, size_t bytes);

/*
 * Forward transform, Eq. 8: u2 = outer(x2) * NUFT[u_I u1 exp(ik(-d1 + |x1|^2/(2 r0)))].
 * u1_dev: device [n1y][n1x] complex; u2_dev: device [m2y][m2x] complex.
 * Stages (all CUDA kernels on `stream`): per-sample prefactor fused into the
 * tiled spread onto the sigma-oversampled grid, row FFT with crop, column FFT
 * fused with kernel deconvolution, crop and the destination chirp.
 * Asynchronous (the first call without a workspace allocates the plan's work
 * buffers).  Errors: ASFD_ERR_ARG (NULL), ASFD_ERR_NOMEM (work buffers),
 * ASFD_ERR_CUDA (launch).
 */
asfd_status asfd_execute(asfd_plan plan, const float* u1_dev, float* u2_dev, void* stream);

/*
 * Same transform on HOST buffers, synchronising `stream` before returning.
 * u1_host: [n1y][n1x] complex; u2_host: [m2y][m2x] complex.  A page-locked
 * u1 (cudaHostAlloc, cudaMallocHost, cudaHostRegister, PyTorch's
 * pin_memory) is read by the spread in place, over the host link, while it
 * computes; a pageable u1 is copied to a device copy first.  u2 is formed in
 * a device copy and, when page-locked, copied to the host in column blocks
 * on a stream of the plan while the column pass transforms the next block.
 * The device copies are work buffers of the plan (see asfd_set_workspace).
 * Errors: ASFD_ERR_ARG, ASFD_ERR_NOMEM (work buffers), ASFD_ERR_CUDA.
 */
asfd_status asfd_execute_host(asfd_plan plan, const float* u1_host, float* u2_host, void* stream);

/*
 * asfd_execute_host without the final synchronisation: the copy of u1 to
 * the plan's staging buffer, the transform and the copies of u2 are queued
 * on `stream` (the copies of u2's column blocks on a stream of the plan that
 * `stream` waits for), and the call returns.  u1 is copied by the copy
 * engine, not read in place, so that the SMs stay free for transforms on
 * other streams.  The host buffers must stay valid, u1 unchanged and u2
 * unread, until `stream` reaches this point.  With page-locked buffers the
 * call does not block, so transforms on two plans and two streams overlap
 * one's copies of u2 with the other's upload of u1 and its kernels (the
 * host link carries both directions at once); one plan serves one stream
 * at a time.  A pageable u2 makes the call wait for its copy.
 * Errors: as asfd_execute_host.
 */
asfd_status asfd_execute_host_async(asfd_plan plan, const float* u1_host, float* u2_host,
                                    void* stream);

/*
 * One stage of asfd_execute, for per-kernel timing with events recorded on
 * `stream` between the calls:
 *   stage 0: per-sample prefactor + tiled spread: reads u1_dev, writes the
 *            plan's oversampled grid (u2_dev unused, may be NULL);
 *   stage 1: row FFT + crop: plan grid -> plan row buffer (u1, u2 unused);
 *   stage 2: column FFT + deconvolution + crop + destination chirp:
 *            plan row buffer -> u2_dev (u1 unused).
 * Running stages 0, 1, 2 in order on one stream equals asfd_execute.
 * Errors: ASFD_ERR_ARG (bad stage or missing buffer), ASFD_ERR_CUDA.
 */
asfd_status asfd_execute_stage(asfd_plan plan, int stage, const float* u1_dev, float* u2_dev,
                               void* stream);

/*
 * Adjoint (type-2 NUFFT) of asfd_execute, for gradients of a real loss L(u2)
 * with respect to the source field and the height map (hologram and surface
 * optimisation).  grad_u2_dev: device [m2y][m2x] complex holding
 * dL/dRe(u2) + i dL/dIm(u2).  Writes, for every source sample n,
 *   grad_u1_dev[n] = dL/dRe(u1) + i dL/dIm(u1) = sum_m conj(K_mn) grad_u2[m]
 *   grad_d1_dev[n] = dL/dd1[n]   (FP32, per metre)
 * where K_mn is the coefficient of u1[n] in u2[m] as the forward computes it
 * (Eq. 8 with the plan's kernel): the conjugate transpose of the forward
 * map, and the derivative of that map through the phase k|x1|^2/(2 r0) and
 * the non-uniform frequency k p2 x1 / r0 of each sample.  Stages: column
 * FFT with e^{+i} of conj(deconvolution x chirp) * grad_u2, row FFT with
 * e^{+i}, then one interpolation kernel with the kernel and its derivative.
 * grad_u1_dev and grad_d1_dev may each be NULL (not computed); u1_dev may be
 * NULL only when grad_d1_dev is NULL.  Uses the plan's work buffers (not
 * concurrent with asfd_execute on the same plan).  Asynchronous.
 * Errors: ASFD_ERR_ARG (NULL grad_u2, or grad_d1 without u1), ASFD_ERR_CUDA.
 */
asfd_status asfd_adjoint(asfd_plan plan, const float* u1_dev, const float* grad_u2_dev,
                         float* grad_u1_dev, float* grad_d1_dev, void* stream);

/*
 * Learned spreading kernel (plans created with kind = ASFD_KERNEL_LEARNED and
 * kernel_width = 4).  The ES kernel of the paper's NUFFT step is replaced by
 * a narrower tabulated kernel: for every 16 x 16 block of source samples a
 * small MLP maps dimensionless features of the block (position on the fine
 * grid, local sample spacing, mean d1/(z0 - d1)) to a table of per-tap
 * polynomials of degree 7 in the sample's sub-cell offset, added to a shared
 * base table; the deconvolution is the width-4 ES one times a learned even
 * Chebyshev correction.  The model is a flat vector of
 * asfd_learned_param_count() floats (layout private to the library), trained
 * on the GPU by asfd_learned_train_step.  asfd_execute, asfd_execute_stage
 * and asfd_adjoint use the current model.
 */

/* Number of floats of the learned model (a constant; no errors). */
size_t asfd_learned_param_count(void);

/* Copy the model to host memory (count must equal asfd_learned_param_count()).
 * Synchronous.  Errors: ASFD_ERR_ARG, ASFD_ERR_STATE (not a learned plan). */
asfd_status asfd_learned_get_params(asfd_plan plan, float* params_host, size_t count);

/* Load a model from host memory, reset the optimiser state and rebuild the
 * tables; synchronises `stream`.  Errors: ASFD_ERR_ARG (count, non-finite
 * values), ASFD_ERR_STATE. */
asfd_status asfd_learned_set_params(asfd_plan plan, const float* params_host, size_t count,
                                    void* stream);

/*
 * One Adam step (learning rate lr) on the relative squared error
 * |u2 - ref|^2 / |ref|^2 of the forward transform of u1_dev against
 * ref_u2_dev (device [m2y][m2x] complex, e.g. the ES-kernel transform at a
 * large width, the reference for the learned kernel's error).  Runs the forward,
 * the loss gradient, the adjoint FFT passes, the table, deconvolution and MLP
 * gradients and the update on `stream`.  If loss_host is not NULL the loss
 * before the update is written there (synchronises `stream`).
 * Errors: ASFD_ERR_ARG, ASFD_ERR_STATE, ASFD_ERR_CUDA.
 */
asfd_status asfd_learned_train_step(asfd_plan plan, const float* u1_dev, const float* ref_u2_dev,
                                    float lr, double* loss_host, void* stream);

/* Gradient of the same loss with respect to every model parameter (no
 * update), copied to grad_host (count = asfd_learned_param_count()); the loss
 * goes to loss_host if not NULL.  Synchronises `stream`.  For checking the
 * training kernels against an independent CPU computation.  Errors:
 * ASFD_ERR_ARG (NULL buffers, count not the model size), ASFD_ERR_STATE (not
 * a learned plan), ASFD_ERR_NOMEM (work buffers), ASFD_ERR_CUDA. */
asfd_status asfd_learned_gradient(asfd_plan plan, const float* u1_dev, const float* ref_u2_dev,
                                  float* grad_host, size_t count, double* loss_host, void* stream);

/*
 * Layout of the learned model vector (all float), an interface shared with
 * tools that read or write models.  T = 64 table entries per tile, ordered
 * [axis x, y][tap 0..3][power 0..7] of t = 2 dx - 1; F = 6 features
 * (1, mean fine-grid x and y relative to the grid centre in units of nf/2,
 * mean sample spacing on the fine grid minus 1 in x and y, 100 x mean
 * d1/(z0 - d1)); H = 32 tanh hidden units; C = 6 even Chebyshev terms:
 *   [0, 64)        base table (T)
 *   [64, 256)      W1[H][F]            [256, 288)    b1[H]
 *   [288, 2336)    W2[T][H]            [2336, 2400)  b2[T]
 *   [2400, 2406)   d_x[C]              [2406, 2412)  d_y[C]
 * table(tile) = base + 0.001 (W2 tanh(W1 f + b1) + b2); deconvolution factor
 * per axis = (ES width-4 factor) x (1 + sum_j d_j T_{2j}(2 m'/M)), j = 1..C.
 */

/*
 * Batched transform of many surfaces (each with its own sizes, pitches,
 * wavelength, distance and height map; one plan each), in one of two
 * schedules, both replayed from CUDA graphs:
 *   ASFD_BATCH_STREAMS (default): every surface's three kernels (spread, row
 *     FFT, column FFT with deconvolution and chirp) in order on one of up to
 *     16 streams of the batch, forked from and joined to the caller's stream;
 *     surfaces are dealt to the streams largest first, each to the least
 *     loaded, so that small surfaces fill the SMs that large ones leave idle.
 *     The first call launches directly; later calls replay a graph of the
 *     same launches, captured again when the field pointers change.
 *   ASFD_BATCH_PERSISTENT: ONE persistent cooperative kernel per call: all
 *     spreads, a grid barrier, all row FFTs, a grid barrier, all column FFTs
 *     (one common kernel width in 4..8, fine grids up to 4096).
 */
typedef struct asfd_batch_s* asfd_batch;

enum { ASFD_BATCH_STREAMS = 0, ASFD_BATCH_PERSISTENT = 1 };

typedef struct {
    int surfaces;
    int blocks, threads_per_block;   /* persistent grid (all blocks co-resident)      */
    int spread_items, row_items, col_items;  /* persistent schedule's items         */
    int graph;                       /* 1 when the last call ran from a CUDA graph    */
    long long source_samples;        /* total over the batch                          */
    int schedule;                    /* ASFD_BATCH_STREAMS or ASFD_BATCH_PERSISTENT  */
    int persistent_ok;               /* 1 when the persistent schedule is available   */
    int streams;                     /* streams of the stream schedule                */
} asfd_batch_info;

/*
 * params[count], d1_devs[count] (host arrays; d1 device FP64 [n1y][n1x] each,
 * read during the call).  All surfaces use the ES kernel (else
 * ASFD_ERR_UNSUPPORTED); the persistent schedule is available when they share
 * one width in 4..8 and their fine grids are at most 4096 (in its launch,
 * surfaces whose plan takes the atomic spreading kernel -- folding, wrapping
 * or very densely packed samples -- are spread by whole blocks, the others by
 * single warps).  Creates one plan per surface, with its work buffers, and
 * the batch's streams; the schedule starts as ASFD_BATCH_STREAMS.  Errors as
 * asfd_plan_create.
 */
asfd_status asfd_batch_create(asfd_batch* out, const asfd_params* params,
                              const double* const* d1_devs, int count, void* stream);

/*
 * Transform every surface: u1_devs[i] (device [n1y][n1x] complex of surface
 * i) -> u2_devs[i] (device [m2y][m2x] complex); host arrays of device
 * pointers.  Stream schedule: queued on `stream` (its work forks to the
 * batch's streams and joins back), asynchronous.  Persistent schedule:
 * synchronises `stream` first (the previous launch must have read the
 * pointer table), then queues one graph launch.  One batch serves one
 * stream at a time.  Errors: ASFD_ERR_ARG, ASFD_ERR_CUDA.
 */
asfd_status asfd_batch_execute(asfd_batch batch, const float* const* u1_devs,
                               float* const* u2_devs, void* stream);

/*
 * Choose the schedule of later asfd_batch_execute calls (ASFD_BATCH_STREAMS
 * or ASFD_BATCH_PERSISTENT).  Errors: ASFD_ERR_ARG (NULL batch, unknown
 * schedule), ASFD_ERR_UNSUPPORTED (persistent schedule not available).
 */
asfd_status asfd_batch_set_schedule(asfd_batch batch, int schedule);

asfd_status asfd_batch_get_info(asfd_batch batch, asfd_batch_info* info);

/* Release the batch and its plans (synchronises the device).  NULL accepted. */
asfd_status asfd_batch_destroy(asfd_batch batch);

/* Fill *info.  Errors: ASFD_ERR_ARG. */
asfd_status asfd_get_plan_info(asfd_plan plan, asfd_plan_info* info);

/* Wait for `stream`, then report a device-side failure recorded by the
 * plan's kernels since the last call (bounded waits, index checks), and
 * clear it.  ASFD_OK when none was recorded; else ASFD_ERR_STATE (an index
 * check), ASFD_ERR_TIMEOUT (reserved); ASFD_ERR_ARG (NULL plan),
 * ASFD_ERR_CUDA. */
asfd_status asfd_check_device_status(asfd_plan plan, void* stream);

/* Release the plan and everything it owns (synchronises the device).  NULL is
 * accepted.  Always ASFD_OK. */
asfd_status asfd_destroy(asfd_plan plan);

/* Static description of a status code. */
const char* asfd_status_string(asfd_status s);

/* Description of the last failure on the calling thread ("" if none). */
const char* asfd_last_error(void);

/*
 * Test hooks for the failure paths (no counterpart in the paper; neither
 * call touches the GPU).
 *
 * asfd_debug_fail_allocations(n): the next n device allocations made for 2D
 * plans (asfd_plan_create, asfd_plan_update_d1, learned tables, batch
 * surfaces) succeed and every later one fails with ASFD_ERR_NOMEM without
 * calling the CUDA allocator, until the hook is called again; n < 0 turns it
 * off (the default).  Process-wide.
 *
 * asfd_debug_live_buffers(): the device buffers currently held by all 2D
 * plans of the process (a failed asfd_plan_create must leave it unchanged).
 */
void asfd_debug_fail_allocations(int n);
long long asfd_debug_live_buffers(void);

/*
 * Sum of several surfaces' fields at one destination (e.g. the polygons of
 * a CGH object, each a plan with its own height map, size and position
 * offset_x/y): u2 = sum_i T_i u1_i.  The surfaces must share m2x, m2y, p2x,
 * p2y, lambda, z0, sigma, kernel width and beta, and the source sample area
 * p1x*p1y, and use the default spread (widths up to 7, deterministic = 0,
 * monotone maps without wrap); they are spread into the first plan's fine
 * grid and transformed together (one row and one column pass over the union
 * of their bands).  u1_devs[i]: device complex [n1y_i][n1x_i]; u2_dev:
 * device complex [m2y][m2x].  Uses the first plan's work buffers: no call on
 * it may overlap.  Asynchronous on `stream`.  Errors: ASFD_ERR_ARG
 * (incompatible plans), ASFD_ERR_UNSUPPORTED (not the default spread).
 */
asfd_status asfd_multi_execute(const asfd_plan* plans, const float* const* u1_devs, int count,
                               float* u2_dev, void* stream);

/*
 * One-dimensional form with explicit source samples (an extension; the
 * paper's experiments of Sec. 3 are line sources sampled along their arc
 * length): sample j at x1[j] (metres, any order and spacing) with height
 * d1[j] (< z0) and quadrature weight w[j] (its extent along x1); destination
 * x2 = (m - m2/2) p2.  Computes Eq. 7 in one dimension,
 *   u2(x2) = exp(ik(z0 + x2^2/(2 z0))) / sqrt(i lambda z0)
 *            * sum_j w u_I u1 exp(ik(-d1 + x1^2/(2 r0))) exp(-ik x1 x2/r0),
 * r0 = z0 - d1, u_I = exp(ik(s x1 + sz d1)) (s = incidence_s; s = 0 is the
 * normal incidence of Sec. 2), by a 1D type-1 NUFFT with the ES kernel:
 * FP64 per-sample prefactor and position at plan time, FP32 spread (float2
 * atomic adds), Stockham FFT of sigma*m2 points, deconvolution and chirp.
 */
typedef struct {
    int m2;              /* destination samples; even                            */
    double p2;           /* destination pitch [m]                                */
    double lambda;       /* wavelength [m]                                       */
    double z0;           /* source-axis-to-destination distance [m]              */
    double sigma;        /* oversampling; sigma*m2 a power of two in [64, 16384] */
    int kernel_width;    /* 2..16                                                */
    double es_beta;      /* 0 selects 2.30*w at sigma = 2                        */
    double incidence_s;  /* direction cosine of the incident plane wave, s^2 < 1 */
} asfd_line_params;

typedef struct asfd_line_plan_s* asfd_line_plan;

/* x1_dev, d1_dev, w_dev: device FP64 [n], read during the call only.
 * Synchronises `stream` once (argument check).  Errors: ASFD_ERR_ARG (bad
 * sizes, non-finite samples, d1 >= z0), ASFD_ERR_UNSUPPORTED, ASFD_ERR_NOMEM. */
asfd_status asfd_line_plan_create(asfd_line_plan* out, const asfd_line_params* p,
                                  const double* x1_dev, const double* d1_dev, const double* w_dev,
                                  int n, void* stream);
/* u1_dev: device complex[n] (in the plan's sample order); u2_dev: device
 * complex[m2].  Asynchronous on `stream`; calls on one plan must not overlap.
 * Errors: ASFD_ERR_ARG (NULL), ASFD_ERR_UNSUPPORTED (width), ASFD_ERR_CUDA. */
asfd_status asfd_line_execute(asfd_line_plan plan, const float* u1_dev, float* u2_dev,
                              void* stream);
asfd_status asfd_line_destroy(asfd_line_plan plan);

/*
 * Direct (O(N^2 M^2)) evaluation of the diffraction sums at npts destination
 * points, on the GPU, for measuring the paper's approximations and as a fast
 * reference on sampled points:
 *   form 7: Eq. 7, the Fourier form that asfd_execute evaluates by NUFFT;
 *   form 5: Eq. 5, with r0 = z0 - d1 per sample in the destination chirp
 *           (before the approximation of Eq. 6);
 *   form 2: Eq. 2, the Huygens sum z0/(i lambda) sum u_I u1 exp(ik r)/r^2 with
 *           the exact distance r of Eq. 3 (before the Fresnel expansion of
 *           Eq. 4), u_I = exp(ik d1).
 * All three use the source weight p1x p1y and the centred coordinates of
 * asfd_execute.  p: the geometry fields are used (n1x..z0; the spreading fields
 * are ignored).  d1_dev: device [n1y][n1x] FP64 metres; u1_dev: device
 * [n1y][n1x] complex; mx_dev, my_dev: device int[npts] destination indices;
 * out_dev: device complex[npts].  Phases are formed in FP64 per (sample,
 * point) pair and reduced modulo 2 pi exactly before an FP32 sine/cosine; sums
 * are FP64.  Allocates (stream-ordered) 32 bytes per source sample for the
 * duration of the call.  Asynchronous on `stream`.  Errors: ASFD_ERR_ARG.
 */
asfd_status asfd_direct_sum(const asfd_params* p, const double* d1_dev, const float* u1_dev,
                            int form, int npts, const int* mx_dev, const int* my_dev,
                            float* out_dev, void* stream);

/*
 * Stand-alone batched FFT of the library (the Stockham kernel used by the
 * transform), exposed for unit tests and timing.  in_dev/out_dev: device
 * [lines][n] complex (may alias); n a power of two in [16, 16384];
 * sign = -1 computes X[k] = sum_j x[j] exp(-2 pi i jk/n), +1 the conjugate
 * kernel (no 1/n scaling).  Asynchronous; the first call for a length on a
 * device allocates and fills its twiddle table (and synchronises `stream`).
 * Errors: ASFD_ERR_ARG (n, lines, sign, NULL buffers), ASFD_ERR_UNSUPPORTED
 * (device ordinal above 63), ASFD_ERR_CUDA.
 */
asfd_status asfd_fft_lines(int n, int lines, int sign, const float* in_dev, float* out_dev,
                           void* stream);

/*
 * asfd_fft_lines without any device allocation (the paper has no
 * counterpart; this is a service of the library).  For callers that cannot
 * call cudaMalloc -- e.g. code whose device memory is all handed out up front
 * by a host framework, or latency-critical loops that must avoid the
 * implicit synchronisation of allocation calls -- this variant keeps its
 * twiddle table in a fixed array compiled into the library (16384 complex
 * values, 128 KiB on every GPU that loads the library, held until the
 * process exits) instead of memory allocated on first use.
 *   n: power of two in [16, 16384]; larger n is rejected with ASFD_ERR_ARG
 *      and a message naming the limit.  Other arguments and the result are
 *      exactly as for asfd_fft_lines.
 * Every call looks up the array's device address (cudaGetSymbolAddress) on
 * the current device, so a device reset between calls is harmless; the first
 * call on a device also loads the library's module there, so make that first
 * call before any stream capture.  Every call on a device shares the one array
 * and rewrites the n entries it reads before its transform, so calls that
 * can overlap on the GPU (different streams, or different host threads on
 * one device) race on the table and must be serialised by the caller.
 * Errors: ASFD_ERR_ARG, ASFD_ERR_CUDA.
 */
asfd_status asfd_fft_lines_noalloc(int n, int lines, int sign, const float* in_dev, float* out_dev,
                                   void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ASFD_H */
