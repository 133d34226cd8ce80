/*
 * tdmrg_bench.h -- measurement entry points of libtdmrg.  The paper has no counterpart: these calls
 * exist so that benchmarks can state the rooflines and launch counts the hot path runs against.
 */
#ifndef TDMRG_BENCH_H
#define TDMRG_BENCH_H

#include <stdint.h>

#include "tdmrg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Number of kernels the context has launched since it was created (host counter, no sync). */
int tdmrg_launch_count(tdmrg_ctx* ctx, int64_t* count);

/* Device allocations the context has made since it was created: number of successful cudaMalloc calls
 * and their total bytes (host counters, no sync).  Lets a caller check that a call allocated nothing. */
int tdmrg_alloc_count(tdmrg_ctx* ctx, int64_t* count, int64_t* bytes);

/* Algorithmic FP64-equivalent flops of one H psi in sector Q as the library computes it: 8 real flops
 * per complex multiply-add of every sector-pair product it issues (stage 1 + stage 2). */
int tdmrg_hpsi_flops(tdmrg_ctx* ctx, int n_up, int n_dn, double* flops);

/* Tensor-core flops one H psi in sector Q issues on the Ozaki path (2 M N K per tcgen05.mma over all
 * tiles, slice pairs and K chunks, padding included); 0 when the context runs FP64. */
int tdmrg_hpsi_tensor_flops(tdmrg_ctx* ctx, int n_up, int n_dn, double* flops);

/* Tile schedule of the persistent tensor-core kernel for plans built from now on (existing plans are
 * dropped and rebuilt on their next use): -1 chosen per GEMM stage by timing when the plan is built
 * (the default), 0 static (CTA b takes tiles b, b + grid, ... of the longest-first list), 1 a device
 * work queue.  Every schedule computes the same exact integer sums, so results are bit-identical.
 * Errors: EINVAL (mode outside -1..1). */
int tdmrg_set_schedule(tdmrg_ctx* ctx, int mode);

/* Sustained FP64 throughput of this device, measured by timing (CUDA events) a register-resident
 * loop of the FP64 tensor MMA (mma.sync m8n8k4 f64) and of scalar DFMA on every SM.  Synchronises
 * the device; takes well under a second.  Results in TFLOP/s. */
int tdmrg_fp64_peak(int device, double* dmma_tflops, double* dfma_tflops);

/* Failure-path check of the bounded device waits: one block on the context's stream polls a device
 * word that nothing sets, at most `spins` times, then records a timeout in the context's status word
 * the way the library's mbarrier and grid-barrier waits do, and returns.  The call synchronises the
 * stream and returns TDMRG_ETIMEOUT (the status is consumed, so the context stays usable).
 * Errors: EINVAL (spins outside 1..2^26), ENOMEM, ECUDA. */
int tdmrg_probe_wait(tdmrg_ctx* ctx, int64_t spins);

#ifdef __cplusplus
}
#endif
#endif /* TDMRG_BENCH_H */
