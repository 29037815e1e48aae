/* pcr_ceilings.h - measurement probes for the roofline of the rasterizer (libpcr_ceilings.so).
 *
 * The rasterizer of arXiv 1908.02681 (Section 2.1) is bound by reading 16-byte points from memory and
 * by 64-bit atomic minima into a framebuffer that lives in L2. These probes measure the two ceilings
 * on the running GPU; the benchmark times them with CUDA events and reports its kernels against them.
 * The paper has no counterpart (it reports frame times only, Table 1).
 *
 * All pointers are caller-owned device memory; calls enqueue one kernel on `stream` and return
 * 0 on success or a nonzero CUDA error code. */
#ifndef PCR_CEILINGS_H_
#define PCR_CEILINGS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* n_ops 64-bit atomics (op 0: min, 1: add) at pseudo-random slots of d_slots[0 .. n_slots), spread
 * uniformly (an integer hash of the operation index), the access pattern of a shuffled point order.
 * d_slots must hold n_slots u64; n_slots >= 1; n_ops < 2^40. */
int pcr_ceiling_random_atomics(uint64_t* d_slots, uint32_t n_slots, uint64_t n_ops, int32_t op, void* stream);

/* Streams n16 16-byte words from d_src with the rasterizer's load instruction and folds them into one
 * u32 per thread, written to d_sink only when the fold hits an impossible value (so nothing is
 * optimised away). d_sink must hold sms * 64 * 256 u32. */
int pcr_ceiling_stream_read(const void* d_src, uint64_t n16, uint32_t* d_sink, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PCR_CEILINGS_H_ */
