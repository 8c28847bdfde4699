// Batched 1D FFT that allocates no device memory.
//
// asfd_fft_lines builds its twiddle table in memory it allocates with
// cudaMalloc the first time a length is used on a device.  Some callers
// cannot allocate device memory at all -- for example code running where
// every allocation must be made up front by a host framework that owns the
// device memory pool, or code that must not trigger the implicit device
// synchronisation of cudaMalloc/cudaFree in a latency-critical loop.  For
// them, asfd_fft_lines_noalloc keeps the table in a fixed array compiled into
// this library instead (kStaticFftMaxLength complex values, 128 KiB per GPU
// that loads the library, held until the process exits).
#include <string>

#include "asfd_impl.cuh"

namespace asfd {

asfd_status launch_fft_lines_tw(int n, int lines, int sign, const float2* in, float2* out,
                                const float2* tw, cudaStream_t st);

namespace {

constexpr int kStaticFftMaxLength = 16384;

// Twiddle scratch shared by every call on a device.  Host code must not use
// the symbol itself as a pointer: its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) float2 g_fft_twiddle_scratch[kStaticFftMaxLength];

// Device address of the scratch array on the current device.  Looked up on
// every call (cudaGetSymbolAddress allocates nothing and is cheap), so a call
// after the device's context was reset and re-created uses the new address.
asfd_status scratch_address(float2** out)
{
    void* p = nullptr;
    ASFD_CUDA(cudaGetSymbolAddress(&p, g_fft_twiddle_scratch));
    *out = static_cast<float2*>(p);
    return ASFD_OK;
}

}  // namespace
}  // namespace asfd

using namespace asfd;

extern "C" asfd_status asfd_fft_lines_noalloc(int n, int lines, int sign, const float* in_dev,
                                              float* out_dev, void* stream)
{
    clear_error();
    if (n < 16 || n > kStaticFftMaxLength || (n & (n - 1)))
        return fail(ASFD_ERR_ARG, "asfd_fft_lines_noalloc: n must be a power of two in [16, " +
                                      std::to_string(kStaticFftMaxLength) + "]");
    if (lines < 0 || (sign != 1 && sign != -1))
        return fail(ASFD_ERR_ARG, "asfd_fft_lines_noalloc: lines >= 0 and sign = +-1");
    if (lines > 0 && (!in_dev || !out_dev))
        return fail(ASFD_ERR_ARG, "asfd_fft_lines_noalloc: NULL buffer");
    if (lines == 0) return ASFD_OK;
    float2* tw = nullptr;
    asfd_status s = scratch_address(&tw);
    if (s != ASFD_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the table of the previous call may be for another length: rewrite all n
    // entries the transform reads, on the same stream, before it runs (the
    // generator is the one asfd_fft_lines uses for its own tables)
    s = build_twiddles(tw, n, st);
    if (s != ASFD_OK) return s;
    return launch_fft_lines_tw(n, lines, sign, reinterpret_cast<const float2*>(in_dev),
                               reinterpret_cast<float2*>(out_dev), tw, st);
}
