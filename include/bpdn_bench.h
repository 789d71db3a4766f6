/*
 * bpdn_bench.h -- measurement aid of libbpdn (not part of the solver's ABI proper).
 *
 * The paper measures nothing on a GPU; the library states its kernels' rooflines
 * against pipe rates measured on the device it runs on.  This entry point launches
 * one of four arithmetic-pipe loops so that a caller can time it (with CUDA events on
 * cuda_stream) and derive the rate: operations = blocks * threads * iters * ops_per_thread_trip.
 */
#ifndef BPDN_BENCH_H
#define BPDN_BENCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * kind     0: FP32 FMA (fmaf, 2 flops each); 1: packed FP32 pair FMA (fma.rn.f32x2, 4 flops
 *          each); 2: FP64 FMA (2 flops each); 3: FP32 reciprocal square root (special-function
 *          unit, 1 operation each)
 * blocks   >= 1;  threads  a multiple of 32 in [32, 1024];  iters >= 1 trips of the loop
 * d_sink   device float [blocks * threads]: one folded value per thread (written)
 * ops_per_thread_trip  out (host, may be NULL): operations per thread per trip
 * Asynchronous on cuda_stream.  Returns BPDN_EINVAL on bad arguments, BPDN_ECUDA if the
 * launch fails; 0 otherwise.
 */
int bpdn_bench_peak(int32_t kind, int32_t blocks, int32_t threads, int64_t iters, float *d_sink,
                    double *ops_per_thread_trip, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* BPDN_BENCH_H */
