/*
 * asfd_peaks.h -- measurement probes of the resources that bound the
 * library's kernels (a service for the throughput report; the paper has no
 * counterpart).
 *
 * The spread, FFT and interpolation kernels of the library are limited by
 * on-chip resources as much as by HBM: shared-memory bandwidth (FFT
 * exchanges), float2 reductions in L2 (the atomic flush of the default
 * spread), packed FP32 FMA issue and MUFU exp2 (kernel evaluation).  Each
 * probe queues ONE kernel on `stream`, over every SM of the current device,
 * that exercises one of these resources with independent operations (no
 * bank conflicts, no long dependency chains, no waits), and returns in *work
 * the amount of work it queued; the caller times the launch with CUDA events
 * recorded on `stream` and divides: work / seconds is the measured peak.
 * The probes change no setting of the GPU.
 *
 *   kind                      work unit      scratch_dev (caller-owned device memory)
 *   ASFD_PROBE_SMEM_LOAD      bytes loaded   >= 4 bytes per block (result sink)
 *   ASFD_PROBE_SMEM_STORE     bytes stored   same
 *   ASFD_PROBE_L2_RED_V2F32   bytes reduced  the reduced buffer (8-byte aligned,
 *                                            one float2 per probe thread or more,
 *                                            i.e. about 3 MiB on 152 SMs; keep it
 *                                            below the L2 size)
 *   ASFD_PROBE_FFMA2          FP32 flops     >= 4 bytes per block
 *   ASFD_PROBE_MUFU_EX2       evaluations    >= 4 bytes per block
 *
 * iters in [1, 2^20] scales the work per thread.  Asynchronous.  Errors:
 * ASFD_ERR_ARG (unknown kind, NULL, scratch too small), ASFD_ERR_CUDA.
 */
#ifndef ASFD_PEAKS_H
#define ASFD_PEAKS_H

#include <stddef.h>

#include "asfd.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ASFD_PROBE_SMEM_LOAD = 0,
    ASFD_PROBE_SMEM_STORE = 1,
    ASFD_PROBE_L2_RED_V2F32 = 2,
    ASFD_PROBE_FFMA2 = 3,
    ASFD_PROBE_MUFU_EX2 = 4
} asfd_probe_kind;

asfd_status asfd_probe_launch(int kind, int iters, void* scratch_dev, size_t scratch_bytes,
                              double* work, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ASFD_PEAKS_H */
