/*
 * kmerco_peaks.h -- device-rate microbenchmarks that give the countBF
 * update and query their roofline denominators.  The paper has no
 * counterpart: it measures one CPU thread.  The countBF update of Algorithm
 * 3 is a read-modify-write of a 64-bit cell at a hash-chosen (random)
 * position, and the query of Algorithm 5 is a read of such a cell, so the
 * ceilings of both are the rates this GPU sustains for those two access
 * patterns, measured here over buffers of a chosen size (L2-resident, or
 * far larger than L2).
 *
 * Both calls allocate their buffer with cudaMalloc on `device` (-1: the
 * current device), fill it, time the kernel with CUDA events after one
 * untimed warm-up launch, free it and return the rate in *rate (host
 * memory).  The random positions come from a counter-based mix of the
 * thread and iteration indices (SplitMix64's finaliser), so no input is
 * needed.  Errors: KMERCO_EINVAL (bytes below 4 KiB or not a power of two,
 * ops == 0, rate NULL), KMERCO_ENOMEM, KMERCO_ECUDA.
 */
#ifndef KMERCO_PEAKS_H
#define KMERCO_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Random 64-bit read-modify-writes: each operation loads a cell at a random
 * position of a `bytes` buffer (bypassing L1) and issues one atomicCAS that
 * adds 1 to it, the pattern of the atomic update design's first attempt.
 * ops operations are spread over one launch that fills every SM; *rate
 * receives operations per second.
 */
int kmerco_peak_random_cas(uint64_t bytes, uint64_t ops, int device, double *rate);

/*
 * Random 8-byte reads: each operation loads one 64-bit word at a random
 * position of a `bytes` buffer, eight independent loads in flight per
 * thread (the access pattern of the classification query).  *rate receives
 * reads per second.
 */
int kmerco_peak_random_read(uint64_t bytes, uint64_t ops, int device, double *rate);

#ifdef __cplusplus
}
#endif

#endif /* KMERCO_PEAKS_H */
