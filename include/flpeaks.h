/*
 * flpeaks: roofline ceilings measured on the running GPU, used by the
 * throughput measurements as the denominators of their roofline fractions.
 * Not part of the homomorphic-convolution path (libflashgpu).
 */
#ifndef FLPEAKS_H
#define FLPEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* Butterflies per second of the inverse NTT's lazy Gentleman-Sande
 * butterfly (one Shoup product by a twiddle, a sum and a difference with
 * conditional subtractions, 30-bit residues), issued from registers by
 * every SM (4 CTAs x 256 threads per SM, the register limit, x 16
 * independent chains each), `iters` butterflies per chain, timed with CUDA events on the
 * legacy default stream of the current device after one warm-up launch.
 * This is the ceiling of any kernel built from these butterflies.
 * Returns 0, or -1 (bad argument), -3 (CUDA error), -4 (no memory for the
 * word per CTA the kernel may write). */
int fl_measure_butterfly_rate(int iters, double *butterflies_per_s);

/* Dense flops per second (2 x M x N x K per MMA) of tcgen05.mma
 * cta_group::1 kind::f16 (fp16 A and B, fp32 accumulator in tensor memory)
 * at M = 128, N = n (64, 128 or 256), K = 16: one CTA per SM, one thread of
 * it issuing 4 x `iters` MMAs back to back on operands resident in shared
 * memory, all accumulating into the same tensor-memory columns, timed with
 * CUDA events on the legacy default stream after one warm-up launch.  This
 * is the instruction's own rate, the ceiling of the tensor-core contraction
 * of libflashgpu (fl_he_conv2d_tc), which issues M128 N64 K16.
 * *cycles_per_mma (may be NULL) receives the SM clocks per MMA of the
 * slowest CTA.  Every wait inside the kernel is bounded (2 s).
 * Returns 0, or -1 (n not 64/128/256, iters outside 1..2^20, null result),
 * -2 (the current device is not sm_103), -3 (CUDA error), -4 (no memory for
 * the per-CTA words), -5 (a bounded wait ran out). */
int fl_measure_tc_f16_rate(int n, int iters, double *flops_per_s, double *cycles_per_mma);

#ifdef __cplusplus
}
#endif
#endif /* FLPEAKS_H */
