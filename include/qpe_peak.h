/*
 * qpe_peak.h - measurement aid beside the QPE library (not part of the
 * paper's method): the FMA throughput of the GPU's FP64 and FP32 units, the
 * denominators of the roofline of the kernels that are bound by plain ALU
 * arithmetic (the fused level kernels). cuBLAS-free: a loop of independent
 * fused multiply-adds in every thread of a full-GPU grid, timed with CUDA
 * events on the given stream.
 */
#ifndef QPE_PEAK_H
#define QPE_PEAK_H

#include <stdint.h>

#include "qpe.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * qpe_measure_fma_peak: FLOP/s of fused multiply-adds (2 flop each) on the
 * FP64 units (fp64 != 0) or the FP32 units (fp64 == 0). Launches a grid of
 * (multiprocessors x 8) CTAs of 256 threads; each thread runs `iters`
 * iterations (1 .. 2^20, else QPE_ERR_ARG) of 8 independent FMA chains. One
 * untimed warm-up launch, then `repeats` (1 .. 100) timed launches on
 * cuda_stream (a cudaStream_t or NULL); *tflops receives the best of them in
 * TFLOP/s. Needs a device scratch of 8 bytes per thread of the grid for the
 * results (which keep the chains from being removed): `scratch` (device
 * pointer of at least *scratch_bytes_needed bytes, QPE_ERR_WORKSPACE if
 * smaller). With scratch NULL the call only sets *scratch_bytes_needed and
 * returns QPE_OK. Synchronises the stream.
 */
qpe_status qpe_measure_fma_peak(int32_t fp64, int32_t iters, int32_t repeats, void* scratch, size_t scratch_bytes,
                                size_t* scratch_bytes_needed, double* tflops, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* QPE_PEAK_H */
