// Probes of the GPU resources that bind the library's kernels: shared-memory
// load and store bandwidth, L2 float2 reduction throughput, packed FP32 FMA
// and MUFU exp2 issue rates.  Each probe is one kernel over every SM that
// exercises a single resource with independent work (no dependency chains
// longer than the unit's pipeline, no bank conflicts, no waits), so that its
// rate, timed by the caller with events, is a measured peak of that resource.
// They change no setting of the GPU.
#include <algorithm>
#include <string>

#include "../../include/asfd_peaks.h"
#include "asfd_impl.cuh"

namespace asfd {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeSmemVec = 2048;  // float4 per block: 32 KiB of shared memory
constexpr int kProbeUnroll = 8;

__device__ __forceinline__ void sink(float* out, float v)
{
    // never true for the probes' finite values; keeps the work observable
    if (v == -1.2345e-30f) out[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kProbeThreads) smem_load_probe(float* out, int iters)
{
    __shared__ float4 buf[kProbeSmemVec];
    for (int i = threadIdx.x; i < kProbeSmemVec; i += kProbeThreads)
        buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    const unsigned base = (unsigned)__cvta_generic_to_shared(buf);
    float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeUnroll; ++k) {
            // consecutive lanes read consecutive float4 (conflict-free); the
            // pattern moves by a warp's width every iteration, so no load
            // repeats an address of the previous iteration and none can be
            // hoisted out of the loop
            const int idx = (threadIdx.x + k * kProbeThreads + it * 32) & (kProbeSmemVec - 1);
            float x, y, z, w;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(x), "=f"(y), "=f"(z), "=f"(w)
                         : "r"(base + 16u * (unsigned)idx));
            ax += x;
            ay += y;
            az += z;
            aw += w;
        }
    }
    sink(out, ax + ay + az + aw);
}

__global__ void __launch_bounds__(kProbeThreads) smem_store_probe(float* out, int iters)
{
    __shared__ float4 buf[kProbeSmemVec];
    const unsigned base = (unsigned)__cvta_generic_to_shared(buf);
    const float v = (float)threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeUnroll; ++k) {
            const int idx = (threadIdx.x + k * kProbeThreads + it * 32) & (kProbeSmemVec - 1);
            asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(base + 16u * (unsigned)idx),
                         "f"(v), "f"(v), "f"(v), "f"(v)
                         : "memory");
        }
    }
    __syncthreads();
    sink(out, reinterpret_cast<float*>(buf)[threadIdx.x]);
}

// float2 reductions (red.global.add.v2.f32, the atomic flush of the default
// spread) over a buffer of n float2 that stays resident in L2; a warp covers
// 32 consecutive float2 per instruction, as a window flush does.
__global__ void __launch_bounds__(kProbeThreads) l2_red_probe(float2* buf, size_t n, int iters)
{
    // the launcher guarantees n >= the number of threads, so one subtraction
    // keeps i in [0, n)
    const size_t stride = (size_t)gridDim.x * kProbeThreads;
    size_t i = (size_t)blockIdx.x * kProbeThreads + threadIdx.x;
    const float2 v = make_float2(1.f, 1.f);
    for (int it = 0; it < iters; ++it) {
        atomicAdd(buf + i, v);
        i += stride;
        if (i >= n) i -= n;
    }
}

__global__ void __launch_bounds__(kProbeThreads) ffma2_probe(float* out, int iters)
{
    unsigned long long acc[kProbeUnroll];
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k) {
        const float2 f = make_float2((float)(threadIdx.x + k), (float)k);
        acc[k] = *reinterpret_cast<const unsigned long long*>(&f);
    }
    const float2 fa = make_float2(0.999f, 1.001f), fb = make_float2(1e-3f, -1e-3f);
    const unsigned long long a = *reinterpret_cast<const unsigned long long*>(&fa);
    const unsigned long long b = *reinterpret_cast<const unsigned long long*>(&fb);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeUnroll; ++k)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[k]) : "l"(a), "l"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k) {
        const float2 f = *reinterpret_cast<const float2*>(&acc[k]);
        s += f.x + f.y;
    }
    sink(out, s);
}

__global__ void __launch_bounds__(kProbeThreads) mufu_ex2_probe(float* out, int iters)
{
    float acc[kProbeUnroll];
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k) acc[k] = -1e-3f * (float)(threadIdx.x % 7 + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeUnroll; ++k)
            asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(acc[k]));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k) s += acc[k];
    sink(out, s);
}

template <class K>
asfd_status probe_grid(K kernel, int* blocks)
{
    int dev = 0, sms = 0, per_sm = 0;
    ASFD_CUDA(cudaGetDevice(&dev));
    ASFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ASFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kProbeThreads, 0));
    *blocks = sms * std::max(per_sm, 1);
    return ASFD_OK;
}

}  // namespace
}  // namespace asfd

using namespace asfd;

extern "C" asfd_status asfd_probe_launch(int kind, int iters, void* scratch_dev,
                                         size_t scratch_bytes, double* work, void* stream)
{
    clear_error();
    if (!work || !scratch_dev || iters < 1 || iters > (1 << 20))
        return fail(ASFD_ERR_ARG, "asfd_probe_launch: work and scratch non-NULL, iters in [1, 2^20]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int blocks = 0;
    asfd_status s = ASFD_OK;
    const double threads_iters = (double)kProbeThreads * (double)iters;
    switch (kind) {
        case ASFD_PROBE_SMEM_LOAD:
        case ASFD_PROBE_SMEM_STORE:
        case ASFD_PROBE_FFMA2:
        case ASFD_PROBE_MUFU_EX2: {
            auto k = kind == ASFD_PROBE_SMEM_LOAD ? smem_load_probe
                   : kind == ASFD_PROBE_SMEM_STORE ? smem_store_probe
                   : kind == ASFD_PROBE_FFMA2 ? ffma2_probe : mufu_ex2_probe;
            if ((s = probe_grid(k, &blocks)) != ASFD_OK) return s;
            if (scratch_bytes < sizeof(float) * (size_t)blocks)
                return fail(ASFD_ERR_ARG, "asfd_probe_launch: scratch needs 4 bytes per block");
            k<<<blocks, kProbeThreads, 0, st>>>(static_cast<float*>(scratch_dev), iters);
            const double per = (double)blocks * threads_iters * kProbeUnroll;
            if (kind == ASFD_PROBE_SMEM_LOAD || kind == ASFD_PROBE_SMEM_STORE) *work = 16.0 * per;
            else if (kind == ASFD_PROBE_FFMA2) *work = 4.0 * per;  // flops: 2 lanes x (mul + add)
            else *work = per;                                       // exp2 evaluations
            break;
        }
        case ASFD_PROBE_L2_RED_V2F32: {
            const size_t n = scratch_bytes / sizeof(float2);
            if (n < 1024) return fail(ASFD_ERR_ARG, "asfd_probe_launch: scratch too small");
            if (reinterpret_cast<uintptr_t>(scratch_dev) % 8)
                return fail(ASFD_ERR_ARG, "asfd_probe_launch: scratch must be 8-byte aligned");
            if ((s = probe_grid(l2_red_probe, &blocks)) != ASFD_OK) return s;
            if (n < (size_t)blocks * kProbeThreads)
                return fail(ASFD_ERR_ARG, "asfd_probe_launch: scratch needs a float2 per thread (" +
                                              std::to_string((size_t)blocks * kProbeThreads * 8) +
                                              " bytes)");
            l2_red_probe<<<blocks, kProbeThreads, 0, st>>>(static_cast<float2*>(scratch_dev), n, iters);
            *work = 8.0 * (double)blocks * threads_iters;  // bytes reduced
            break;
        }
        default:
            return fail(ASFD_ERR_ARG, "asfd_probe_launch: unknown probe kind");
    }
    ASFD_CUDA(cudaGetLastError());
    return ASFD_OK;
}
