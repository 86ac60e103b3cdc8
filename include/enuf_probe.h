/*
 * enuf_probe.h -- measurement helper of the benchmark, not part of the method
 * and not part of libenuf.so: it is built into libenuf_probe.so, which only
 * the benchmark loads.
 *
 * The single-precision FMA rate of the current device, measured by a kernel
 * of independent fused multiply-add chains, is the peak that the FMA
 * roofline of the spreading and interpolation kernels is reported against
 * (their algorithmic work is p^3 and f p^3 multiply-adds per particle).
 */
#ifndef ENUF_PROBE_H
#define ENUF_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Measured FMA rate in TFLOP/s (2 flops per FMA).  Synchronous: waits for
 * its kernels on cuda_stream (NULL = legacy stream); allocates no device
 * memory; runs for a few milliseconds.  Returns 0, or -1 for a NULL
 * argument and -4 when a CUDA call failed (then enuf_probe_last_error()
 * describes it). */
int enuf_fma_peak_tflops(double* tflops, void* cuda_stream);

/* Description of the last failure of this library on the calling thread. */
const char* enuf_probe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ENUF_PROBE_H */
