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

/* FP64 flops (8 per complex multiply-add) of the thin sector-pair products of one H psi in sector Q,
 * i.e. those the tensor path computes on the FP64 warps of its persistent kernel; 0 on an FP64 context. */
int tdmrg_hpsi_thin_flops(tdmrg_ctx* ctx, int n_up, int n_dn, double* flops);

/* Tensor path: sector-pair products whose output block has fewer than `dim` rows or columns run on FP64
 * warps of the persistent tensor kernel instead of tensor tiles (plans built from now on; existing plans
 * are rebuilt on their next use).  Only products whose K over all segments is at most 32 qualify (an
 * FP64 block must not outlast the tensor stage).  dim = 0 puts every product on the tensor tiles.
 * Default 12 (fastest measured at the L=32 m=400, 2x16 m=800 and L=48 m=1000 workloads).
 * Errors: EINVAL (dim outside 0..64). */
int tdmrg_set_thin_dim(tdmrg_ctx* ctx, int dim);

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

/* Tile M of the persistent tensor kernel: 0 (the default) lets the autotuner time M = 64 and M = 128
 * with both schedules per GEMM stage when a plan is built; 64 or 128 fixes it (plans are rebuilt on
 * their next use).  Every choice gives bit-identical products.  Errors: EINVAL. */
int tdmrg_set_tile_m(tdmrg_ctx* ctx, int m);
/* Blocks per SM of the cooperative Lanczos orthogonalisation (1..8, capped by co-residency and by 304
 * blocks; 0 = the default).  Drops the Krylov workspaces.  Errors: EINVAL. */
int tdmrg_set_orth_per_sm(tdmrg_ctx* ctx, int k);
/* The choices of the H psi plan of sector Q: out[0..3] = tile M and schedule (0 static, 1 queue) of
 * stage 1, then of stage 2 (0 / -1 on the FP64 path).  Builds the plan if needed.  Errors: EINVAL, ESTATE. */
int tdmrg_hpsi_tuning(tdmrg_ctx* ctx, int n_up, int n_dn, int32_t* out);

/* Per sector of one block (side 0: left, 1: right), from the last tdmrg_rho_eig[_side] there: the
 * number of sweeps of the FP32 Jacobi seed and the SM cycles its CTA took (host arrays of the side's
 * sector count).  Synchronises the stream.  Errors: EINVAL, ESTATE (no eigendecomposition yet). */
int tdmrg_eig_stats(tdmrg_ctx* ctx, int side, int32_t* sweeps, int64_t* cycles);

#ifdef __cplusplus
}
#endif
#endif /* TDMRG_BENCH_H */
