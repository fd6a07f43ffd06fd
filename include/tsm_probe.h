/*
 * tsm_probe.h -- machine-peak probes behind the roofline denominators.
 *
 * The paper measures its own ceilings with micro-benchmarks (Sec. 1.6: a
 * read-only thread-local-sum kernel for the bandwidth b_s of TSMTTSM, a STREAM
 * "scale" kernel for TSMM, and the FP64 FMA peak).  These probes do the same
 * on the current device.  They are measurements, not part of either product.
 * Each call launches its kernel(s) on `stream`, times them with CUDA events
 * and synchronizes the stream; results are returned through host pointers.
 */
#ifndef TSM_PROBE_H
#define TSM_PROBE_H

#include "tsm.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * FP64 arithmetic peak in GFLOP/s (2 flops per FMA).  mode 0: DFMA on the
 * FP64 pipe in the products' own form (a 4 x 4 or 8 x 4 register tile
 * updated by register outer products, 16 or 32 independent chains per
 * thread), launched with 1, 2 and 4 CTAs of 256 threads per SM; the fastest
 * of the six shapes is reported.  mode 1: FP64 tensor MMA (mma.sync
 * m8n8k4, 2*8*8*4 flops per warp instruction); mode 2: DFMA chains
 * x = x * m + a with compile-time constants m, a (an earlier form of the
 * probe, kept for comparison); both with 4 CTAs of 256 threads per SM.
 * `iters` sets the work (inner iterations per thread at 4 CTAs per SM and
 * 16 chains; the other shapes do the same FMAs per SM).  Each shape: the
 * best of two timed launches after one warm-up launch.  INVALID_VALUE on a
 * bad mode, null output or iters < 1.
 */
tsm_status tsm_probe_fp64(int mode, int64_t iters, double *gflops, tsm_stream_t stream);

/*
 * Memory bandwidth in GB/s over a caller-owned DEVICE buffer of `bytes`
 * bytes (16-byte aligned, multiple of 16).  mode 0: read-only thread-local
 * sum (the TSMTTSM-like stream; loaded bits are folded with integer XOR so
 * the FP64 pipe does not limit it); mode 1: in-place scale x = 1.0 * x (one
 * read and one write stream, TSMM-like; bytes counted twice).  `ilp`
 * independent 16-byte loads in flight per thread (1, 4 or 16: the load
 * parallelism of the paper's Table 1); `blocks` CTAs in total (0 = 8 per SM)
 * of `threads` threads each (0 = 256; otherwise a multiple of 32 in
 * [32, 1024]), which sets the occupancy.  Best of four timed passes.  The
 * buffer's contents are preserved by mode 1.
 */
tsm_status tsm_probe_bandwidth(void *buffer, size_t bytes, int mode, int ilp,
                               int blocks, int threads, double *gbs, tsm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TSM_PROBE_H */
