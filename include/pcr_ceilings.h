/* pcr_ceilings.h - measurement probes for the roofline of the rasterizer (libpcr_ceilings.so).
 *
 * The rasterizer of arXiv 1908.02681 (Section 2.1) is bound by reading 16-byte points from memory and
 * by 64-bit atomic minima into a framebuffer that lives in L2. These probes measure the two ceilings
 * on the running GPU; the benchmark times them with CUDA events and reports its kernels against them.
 * A third probe measures the FP64 and FP32 fused multiply-add rates that bound the per-point transform.
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

/* The framebuffer operations of the two passes for one view, without the per-point transform: the
 * memory-side floor of Sections 2.1 and 2.2 for the access pattern of that cloud and view.
 *
 * pcr_ceiling_pattern_project writes, for each of the n points (16-B aligned, the rasterizer's layout),
 * d_pix[i] = its pixel (row * width + column) or 0xFFFFFFFF when the FP64 definition culls it, and
 * d_key[i] = its key (40-bit linear depth code << 24 | RGB) or all ones. m12 = rows 0, 1 and 3 of the
 * row-major view-projection; 0 < near < far; width, height in 1..16384.
 *
 * pcr_ceiling_pattern_min does one 64-bit atomic minimum into d_keys[d_pix[i]] per visible fragment
 * (pass 1); with filter = 1 a fragment first reads d_keys[d_pix[i]] and skips the atomic unless its key
 * is smaller (the same minima: a stored key only decreases). pcr_ceiling_pattern_hq reads d_keys[d_pix[i]] per visible fragment and, when the fragment's
 * code lies in the band eps_den * (q - qmin) <= eps_num * (qmin + nq), adds its colour and a count to
 * d_accum[2 p], d_accum[2 p + 1] (pass 2; the sums layout of the framebuffer). Both read 12 B per point
 * and take the points in order, 32 consecutive points per warp step. d_keys: width * height u64;
 * d_accum: 2 * width * height u64. */
int pcr_ceiling_pattern_project(const void* d_points, uint64_t n, const double* m12, double near_, double far_,
                                int32_t width, int32_t height, uint32_t* d_pix, uint64_t* d_key, void* stream);
int pcr_ceiling_pattern_min(const uint32_t* d_pix, const uint64_t* d_key, uint64_t n, uint64_t* d_keys, int32_t filter,
                            void* stream);
int pcr_ceiling_pattern_hq(const uint32_t* d_pix, const uint64_t* d_key, uint64_t n, const uint64_t* d_keys,
                           uint64_t* d_accum, uint32_t eps_num, uint32_t eps_den, uint64_t nq, void* stream);

/* Fused multiply-add throughput of the FP64 (fp64 = 1) or FP32 (fp64 = 0) pipes: sms * 8 blocks of 256
 * threads, each running 16 independent chains of `iters` explicitly rounded fmas. *fmas receives the total
 * number of fmas enqueued (host memory); divide by the kernel's time for the rate. The FP64 rate is what a
 * direct FP64 evaluation of the per-point transform (Sections 1 and 2.1: depth in double precision) is
 * bound by. d_sink must hold sms * 8 * 256 u32; iters >= 1. */
int pcr_ceiling_fma(int32_t fp64, uint32_t iters, uint32_t* d_sink, uint64_t* fmas, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PCR_CEILINGS_H_ */
