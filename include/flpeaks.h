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

#ifdef __cplusplus
}
#endif
#endif /* FLPEAKS_H */
