// The exported C ABI (include/asfd.h): argument checks, plan lifetime, and
// the forward transform as three kernels on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "asfd_impl.cuh"

namespace asfd {

namespace {
thread_local std::string g_last_error;
}

asfd_status fail(asfd_status s, const std::string& msg)
{
    g_last_error = msg;
    return s;
}

asfd_status cuda_fail(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return ASFD_ERR_CUDA;
}

void clear_error() { g_last_error.clear(); }

std::atomic<int> g_alloc_budget{-1};
std::atomic<long long> g_live_buffers{0};

namespace {

void free_all(asfd_plan_s* P)
{
    for (auto& b : P->owned) cudaFree(b.p);
    g_live_buffers -= (long long)P->owned.size();
    P->owned.clear();
    P->device_bytes = 0;
}

// Runs `fn` with the plan's device current, restoring the caller's device.
template <class F>
asfd_status on_device(int dev, F&& fn)
{
    int prev = 0;
    ASFD_CUDA(cudaGetDevice(&prev));
    if (prev != dev) ASFD_CUDA(cudaSetDevice(dev));
    asfd_status s = fn();
    if (prev != dev) cudaSetDevice(prev);
    return s;
}

// Device address through which kernels on the current device read and write
// the page-locked host memory at p (cudaHostAlloc, cudaMallocHost,
// cudaHostRegister), or NULL for any other memory.
void* mapped_host_address(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

}  // namespace
}  // namespace asfd

using namespace asfd;

extern "C" {

const char* asfd_status_string(asfd_status s)
{
    switch (s) {
        case ASFD_OK: return "ok";
        case ASFD_ERR_ARG: return "invalid argument";
        case ASFD_ERR_CUDA: return "CUDA error";
        case ASFD_ERR_NOMEM: return "out of memory";
        case ASFD_ERR_TIMEOUT: return "device wait timed out";
        case ASFD_ERR_UNSUPPORTED: return "unsupported";
        case ASFD_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char* asfd_last_error(void) { return g_last_error.c_str(); }

void asfd_debug_fail_allocations(int n) { asfd::g_alloc_budget.store(n < 0 ? -1 : n); }

long long asfd_debug_live_buffers(void) { return asfd::g_live_buffers.load(); }

asfd_status asfd_plan_create(asfd_plan* out, const asfd_params* p, const double* d1_dev,
                             void* stream)
{
    clear_error();
    if (!out) return fail(ASFD_ERR_ARG, "out is NULL");
    *out = nullptr;
    int nfx = 0, nfy = 0;
    double beta = 0.0;
    asfd_status s = plan_validate(p, &nfx, &nfy, &beta);
    if (s != ASFD_OK) return s;
    if (!d1_dev) return fail(ASFD_ERR_ARG, "d1 is NULL");
    asfd_plan_s* P = new (std::nothrow) asfd_plan_s();
    if (!P) return fail(ASFD_ERR_NOMEM, "host allocation of the plan failed");
    P->prm = *p;
    P->nfx = nfx;
    P->nfy = nfy;
    P->w = p->kernel_width;
    P->beta = beta;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = [&]() -> asfd_status {
        ASFD_CUDA(cudaGetDevice(&P->device));
        asfd_status r = plan_alloc(P);
        if (r != ASFD_OK) return r;
        r = plan_build_tables(P, st);
        if (r != ASFD_OK) return r;
        r = plan_build_d1(P, d1_dev, st);
        if (r != ASFD_OK) return r;
        if (p->kind == ASFD_KERNEL_LEARNED) {
            P->learned = true;
            return learned_init(P, st);
        }
        return ASFD_OK;
    }();
    if (s != ASFD_OK) {
        free_all(P);
        delete P;
        return s;
    }
    *out = P;
    return ASFD_OK;
}

asfd_status asfd_plan_update_d1(asfd_plan P, const double* d1_dev, void* stream)
{
    clear_error();
    if (!P || !d1_dev) return fail(ASFD_ERR_ARG, "plan or d1 is NULL");
    return on_device(P->device, [&] {
        return plan_build_d1(P, d1_dev, static_cast<cudaStream_t>(stream));
    });
}

asfd_status asfd_execute(asfd_plan P, const float* u1_dev, float* u2_dev, void* stream)
{
    clear_error();
    if (!P || !u1_dev || !u2_dev) return fail(ASFD_ERR_ARG, "plan, u1 or u2 is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return on_device(P->device, [&]() -> asfd_status {
        asfd_status s = plan_ensure_work(P, kWorkTransform);
        if (s != ASFD_OK) return s;
        s = launch_spread(P, reinterpret_cast<const float2*>(u1_dev), st);
        if (s != ASFD_OK) return s;
        s = launch_fft_rows(P, st);
        if (s != ASFD_OK) return s;
        return launch_fft_cols(P, reinterpret_cast<float2*>(u2_dev), st);
    });
}

asfd_status asfd_execute_stage(asfd_plan P, int stage, const float* u1_dev, float* u2_dev,
                               void* stream)
{
    clear_error();
    if (!P) return fail(ASFD_ERR_ARG, "plan is NULL");
    if (stage == 0 && !u1_dev) return fail(ASFD_ERR_ARG, "stage 0 needs u1");
    if (stage == 2 && !u2_dev) return fail(ASFD_ERR_ARG, "stage 2 needs u2");
    if (stage < 0 || stage > 2) return fail(ASFD_ERR_ARG, "stage must be 0, 1 or 2");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return on_device(P->device, [&]() -> asfd_status {
        const asfd_status s = plan_ensure_work(P, kWorkTransform);
        if (s != ASFD_OK) return s;
        if (stage == 0) return launch_spread(P, reinterpret_cast<const float2*>(u1_dev), st);
        if (stage == 1) return launch_fft_rows(P, st);
        return launch_fft_cols(P, reinterpret_cast<float2*>(u2_dev), st);
    });
}

asfd_status asfd_adjoint(asfd_plan P, const float* u1_dev, const float* grad_u2_dev,
                         float* grad_u1_dev, float* grad_d1_dev, void* stream)
{
    clear_error();
    if (!P || !grad_u2_dev) return fail(ASFD_ERR_ARG, "plan or grad_u2 is NULL");
    if (grad_d1_dev && !u1_dev) return fail(ASFD_ERR_ARG, "grad_d1 needs u1");
    if (!grad_u1_dev && !grad_d1_dev) return ASFD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return on_device(P->device, [&]() -> asfd_status {
        asfd_status s = plan_ensure_work(P, kWorkTransform);
        if (s != ASFD_OK) return s;
        s = launch_fft_cols_adj(P, reinterpret_cast<const float2*>(grad_u2_dev), st);
        if (s != ASFD_OK) return s;
        s = launch_fft_rows_adj(P, st);
        if (s != ASFD_OK) return s;
        return launch_interp_grad(P, reinterpret_cast<const float2*>(u1_dev),
                                  reinterpret_cast<float2*>(grad_u1_dev), grad_d1_dev, st);
    });
}

// Queues the host-buffer transform on `stream`; `sync` waits for it.
static asfd_status execute_host(asfd_plan P, const float* u1_host, float* u2_host, void* stream,
                                bool sync)
{
    clear_error();
    if (!P || !u1_host || !u2_host) return fail(ASFD_ERR_ARG, "plan, u1 or u2 is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return on_device(P->device, [&]() -> asfd_status {
        // A synchronous call reads a page-locked u1 in place: the spread
        // reads it over the host link while it computes (as fast as a copy,
        // and hidden behind the spread).  A queued call, and any call with a
        // pageable u1, copies u1 to the plan's staging buffer first: the copy
        // engine then carries the upload and leaves the SMs to transforms
        // running on other streams.  u2 is written to the staging buffer by the column
        // pass, in column blocks, and each block is copied to the host while
        // the next one is transformed (the link takes these copies faster
        // than kernel stores to host memory).  Staging buffers are work
        // buffers (the plan's own, allocated on first use, or the workspace).
        const float2* in = sync ? static_cast<const float2*>(mapped_host_address(u1_host))
                                : nullptr;
        const bool out_locked = mapped_host_address(u2_host) != nullptr;
        const int m2x = P->prm.m2x, m2y = P->prm.m2y;
        const size_t b1 = sizeof(float2) * (size_t)P->prm.n1x * P->prm.n1y;
        const size_t b2 = sizeof(float2) * (size_t)m2x * m2y;
        asfd_status s = plan_ensure_work(P, kWorkTransform | kWorkStaging);
        if (s != ASFD_OK) return s;
        if (!in) {
            ASFD_CUDA(cudaMemcpyAsync(P->stage_u1, u1_host, b1, cudaMemcpyHostToDevice, st));
            in = P->stage_u1;
        }
        s = launch_spread(P, in, st);
        if (s != ASFD_OK) return s;
        s = launch_fft_rows(P, st);
        if (s != ASFD_OK) return s;
        const int nblk = (out_locked && m2x >= 256 * kHostColBlocks) ? kHostColBlocks : 1;
        if (nblk == 1) {
            s = launch_fft_cols(P, P->stage_u2, st);
            if (s != ASFD_OK) return s;
            ASFD_CUDA(cudaMemcpyAsync(u2_host, P->stage_u2, b2, cudaMemcpyDeviceToHost, st));
        } else {
            if (!P->copy_stream) {
                ASFD_CUDA(cudaStreamCreateWithFlags(&P->copy_stream, cudaStreamNonBlocking));
                for (cudaEvent_t& e : P->copy_ev)
                    ASFD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            }
            const size_t pitch = sizeof(float2) * (size_t)m2x;
            // block boundaries on multiples of 64 columns (whole column-pass blocks)
            const int step = (m2x / nblk + 63) / 64 * 64;
            for (int k = 0; k < nblk; ++k) {
                const int c0 = k * step, c1 = std::min(m2x, c0 + step);
                if (c0 >= c1) break;
                s = launch_fft_cols_range(P, P->stage_u2, c0, c1, st);
                if (s != ASFD_OK) return s;
                ASFD_CUDA(cudaEventRecord(P->copy_ev[k], st));
                ASFD_CUDA(cudaStreamWaitEvent(P->copy_stream, P->copy_ev[k], 0));
                ASFD_CUDA(cudaMemcpy2DAsync(reinterpret_cast<float2*>(u2_host) + c0, pitch,
                                            P->stage_u2 + c0, pitch, sizeof(float2) * (c1 - c0),
                                            m2y, cudaMemcpyDeviceToHost, P->copy_stream));
            }
            ASFD_CUDA(cudaEventRecord(P->copy_ev[kHostColBlocks], P->copy_stream));
            ASFD_CUDA(cudaStreamWaitEvent(st, P->copy_ev[kHostColBlocks], 0));
        }
        if (sync) ASFD_CUDA(cudaStreamSynchronize(st));
        return ASFD_OK;
    });
}

asfd_status asfd_execute_host(asfd_plan P, const float* u1_host, float* u2_host, void* stream)
{
    return execute_host(P, u1_host, u2_host, stream, true);
}

asfd_status asfd_execute_host_async(asfd_plan P, const float* u1_host, float* u2_host, void* stream)
{
    return execute_host(P, u1_host, u2_host, stream, false);
}

asfd_status asfd_get_plan_info(asfd_plan P, asfd_plan_info* info)
{
    clear_error();
    if (!P || !info) return fail(ASFD_ERR_ARG, "plan or info is NULL");
    std::memset(info, 0, sizeof(*info));
    info->nfx = P->nfx;
    info->nfy = P->nfy;
    info->tile_x = kTileX;
    info->tile_y = kTileY;
    info->band_x0 = P->band_tx0 * kTileX;
    info->band_x1 = P->band_tx1 * kTileX;
    info->band_y0 = P->band_ty0 * kTileY;
    info->band_y1 = P->band_ty1 * kTileY;
    info->spread_tiles = (P->band_tx1 - P->band_tx0) * (P->band_ty1 - P->band_ty0);
    info->tile_pairs = P->tile_pairs;
    info->es_beta = P->beta;
    info->max_abs_eps = P->max_abs_eps;
    info->device_bytes = P->device_bytes;
    info->spread_kind = P->itemtile ? 4
                      : P->colored ? (P->windowed && !P->learned ? 2 : 0) : (P->dense ? 3 : 1);
    info->stride_x = info->spread_kind == 2 ? P->sxw_min : P->sx_min;
    info->stride_y = P->h_min;
    info->run_rows = P->dense ? P->dense_rows : 0;
    return ASFD_OK;
}

asfd_status asfd_check_device_status(asfd_plan P, void* stream)
{
    clear_error();
    if (!P) return fail(ASFD_ERR_ARG, "plan is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return on_device(P->device, [&]() -> asfd_status {
        unsigned h = 0;
        ASFD_CUDA(cudaMemcpyAsync(&h, P->status, sizeof(h), cudaMemcpyDeviceToHost, st));
        ASFD_CUDA(cudaStreamSynchronize(st));
        if (h == 0) return ASFD_OK;
        ASFD_CUDA(cudaMemsetAsync(P->status, 0, sizeof(unsigned), st));
        ASFD_CUDA(cudaStreamSynchronize(st));
        if (h & kStatusTimeout) return fail(ASFD_ERR_TIMEOUT, "a bounded device wait ran out");
        if (h & kStatusIndex) return fail(ASFD_ERR_STATE, "a device index check failed");
        return fail(ASFD_ERR_ARG, "device status word " + std::to_string(h));
    });
}

size_t asfd_workspace_bytes(const asfd_params* p)
{
    clear_error();
    int nfx = 0, nfy = 0;
    double beta = 0.0;
    if (plan_validate(p, &nfx, &nfy, &beta) != ASFD_OK) return 0;
    return work_layout(*p, nfx, nfy).total;
}

asfd_status asfd_set_workspace(asfd_plan P, void* ws_dev, size_t bytes)
{
    clear_error();
    if (!P) return fail(ASFD_ERR_ARG, "plan is NULL");
    return on_device(P->device, [&] { return plan_set_workspace(P, ws_dev, bytes); });
}

asfd_status asfd_destroy(asfd_plan P)
{
    clear_error();
    if (!P) return ASFD_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(P->device);
    cudaDeviceSynchronize();
    for (cudaEvent_t e : P->copy_ev)
        if (e) cudaEventDestroy(e);
    if (P->copy_stream) cudaStreamDestroy(P->copy_stream);
    free_all(P);
    cudaSetDevice(prev);
    delete P;
    return ASFD_OK;
}

size_t asfd_learned_param_count(void) { return (size_t)kLearnParams; }

asfd_status asfd_learned_get_params(asfd_plan P, float* params_host, size_t count)
{
    clear_error();
    if (!P || !params_host) return fail(ASFD_ERR_ARG, "plan or params is NULL");
    if (!P->learned) return fail(ASFD_ERR_STATE, "plan does not use the learned kernel");
    if (count != (size_t)kLearnParams) return fail(ASFD_ERR_ARG, "count must equal asfd_learned_param_count()");
    return on_device(P->device, [&]() -> asfd_status {
        ASFD_CUDA(cudaMemcpy(params_host, P->lparams, sizeof(float) * kLearnParams, cudaMemcpyDeviceToHost));
        return ASFD_OK;
    });
}

asfd_status asfd_learned_set_params(asfd_plan P, const float* params_host, size_t count, void* stream)
{
    clear_error();
    if (!P || !params_host) return fail(ASFD_ERR_ARG, "plan or params is NULL");
    if (!P->learned) return fail(ASFD_ERR_STATE, "plan does not use the learned kernel");
    if (count != (size_t)kLearnParams) return fail(ASFD_ERR_ARG, "count must equal asfd_learned_param_count()");
    for (size_t i = 0; i < count; ++i)
        if (!std::isfinite(params_host[i])) return fail(ASFD_ERR_ARG, "non-finite parameter");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return on_device(P->device, [&]() -> asfd_status {
        ASFD_CUDA(cudaMemcpyAsync(P->lparams, params_host, sizeof(float) * kLearnParams,
                                  cudaMemcpyHostToDevice, st));
        ASFD_CUDA(cudaMemsetAsync(P->lm, 0, sizeof(float) * kLearnParams, st));
        ASFD_CUDA(cudaMemsetAsync(P->lv, 0, sizeof(float) * kLearnParams, st));
        P->lstep = 0;
        asfd_status s = learned_refresh(P, st);
        if (s != ASFD_OK) return s;
        ASFD_CUDA(cudaStreamSynchronize(st));
        return ASFD_OK;
    });
}

asfd_status asfd_learned_train_step(asfd_plan P, const float* u1_dev, const float* ref_u2_dev,
                                    float lr, double* loss_host, void* stream)
{
    clear_error();
    if (!P || !u1_dev || !ref_u2_dev) return fail(ASFD_ERR_ARG, "plan, u1 or ref is NULL");
    if (!P->learned) return fail(ASFD_ERR_STATE, "plan does not use the learned kernel");
    if (!(lr >= 0.f) || !std::isfinite(lr)) return fail(ASFD_ERR_ARG, "lr must be finite and >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return on_device(P->device, [&]() -> asfd_status {
        const asfd_status s = plan_ensure_work(P, kWorkTransform | kWorkTraining);
        if (s != ASFD_OK) return s;
        return learned_train_step(P, reinterpret_cast<const float2*>(u1_dev),
                                  reinterpret_cast<const float2*>(ref_u2_dev), lr, loss_host, st);
    });
}

asfd_status asfd_learned_gradient(asfd_plan P, const float* u1_dev, const float* ref_u2_dev,
                                  float* grad_host, size_t count, double* loss_host, void* stream)
{
    clear_error();
    if (!P || !u1_dev || !ref_u2_dev || !grad_host) return fail(ASFD_ERR_ARG, "NULL argument");
    if (!P->learned) return fail(ASFD_ERR_STATE, "plan does not use the learned kernel");
    if (count != (size_t)kLearnParams) return fail(ASFD_ERR_ARG, "count must equal asfd_learned_param_count()");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return on_device(P->device, [&]() -> asfd_status {
        asfd_status s = plan_ensure_work(P, kWorkTransform | kWorkTraining);
        if (s != ASFD_OK) return s;
        s = learned_gradient(P, reinterpret_cast<const float2*>(u1_dev),
                                         reinterpret_cast<const float2*>(ref_u2_dev), st);
        if (s != ASFD_OK) return s;
        ASFD_CUDA(cudaMemcpyAsync(grad_host, P->lgrad, sizeof(float) * kLearnParams,
                                  cudaMemcpyDeviceToHost, st));
        if (loss_host) return learned_read_loss(P, loss_host, st);
        ASFD_CUDA(cudaStreamSynchronize(st));
        return ASFD_OK;
    });
}

asfd_status asfd_multi_execute(const asfd_plan* plans, const float* const* u1_devs, int count,
                               float* u2_dev, void* stream)
{
    clear_error();
    if (!plans || !u1_devs || !u2_dev || count < 1)
        return fail(ASFD_ERR_ARG, "plans, u1 array and u2 must be non-NULL, count >= 1");
    for (int i = 0; i < count; ++i)
        if (!plans[i]) return fail(ASFD_ERR_ARG, "plan is NULL");
    return on_device(plans[0]->device, [&]() -> asfd_status {
        const asfd_status s = plan_ensure_work(plans[0], kWorkTransform);
        if (s != ASFD_OK) return s;
        return multi_execute(plans, reinterpret_cast<const float2* const*>(u1_devs), count,
                             reinterpret_cast<float2*>(u2_dev), static_cast<cudaStream_t>(stream));
    });
}

asfd_status asfd_direct_sum(const asfd_params* p, const double* d1_dev, const float* u1_dev,
                            int form, int npts, const int* mx_dev, const int* my_dev,
                            float* out_dev, void* stream)
{
    clear_error();
    return direct_sum(p, d1_dev, reinterpret_cast<const float2*>(u1_dev), form, npts, mx_dev,
                      my_dev, reinterpret_cast<float2*>(out_dev), static_cast<cudaStream_t>(stream));
}

asfd_status asfd_fft_lines(int n, int lines, int sign, const float* in_dev, float* out_dev,
                           void* stream)
{
    clear_error();
    return launch_fft_lines(n, lines, sign, reinterpret_cast<const float2*>(in_dev),
                            reinterpret_cast<float2*>(out_dev), static_cast<cudaStream_t>(stream));
}

}  // extern "C"
