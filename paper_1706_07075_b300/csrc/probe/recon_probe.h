/*
 * librecon_probe: measurement probes for the roofline of the MLEM event pass
 * (bench.py).  They measure the running GPU and have no counterpart in the
 * paper; the reconstruction never calls them.
 *
 * Every probe launches its own kernels on `stream` (a cudaStream_t, NULL =
 * legacy default stream), runs once to warm up and once timed with CUDA events,
 * writes operations per second to *ops_per_s and returns 0 (1: bad argument,
 * 3: CUDA error).  Buffers are caller-owned device memory.
 */
#ifndef RECON_PROBE_H
#define RECON_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Scattered FP32 reductions (red.global.add.f32) into img[0..n_words) at hashed
 * addresses, `runs` consecutive words per hashed address (1: all independent).
 * 148*64*256*256 reductions per run; img is modified. */
int recon_probe_l2_red(float* img, int64_t n_words, int32_t runs, void* stream, double* ops_per_s);

/* FP32 reductions whose lanes share sectors: lanes in groups of `group` (1..32, a
 * divisor of 32); per group and step one hashed 128-byte line of img[0..n_words)
 * (n_words >= 32), lane k of the group adding to word (k*stride) mod 32 of it.
 * *ops_per_s counts element reductions (148*32*256*256 per run); img is modified. */
int recon_probe_red_groups(float* img, int64_t n_words, int32_t group, int32_t stride, void* stream,
                           double* ops_per_s);

/* Scattered 4-byte read-only gathers from img[0..n_words); sink: 148*64*256 floats. */
int recon_probe_gather(const float* img, int64_t n_words, float* sink, void* stream, double* ops_per_s);

/* Steps per second of one scattered gather from lam plus one scattered reduction into C
 * (two images of n_words each: the L2 access pattern of one Siddon piece of the fused
 * pass); C is modified. */
int recon_probe_mixed(const float* lam, float* C, int64_t n_words, float* sink, void* stream, double* steps_per_s);

/* erfcf evaluations per second (FP32 ALU); sink: 148*64*256 floats. */
int recon_probe_erfc(float* sink, void* stream, double* ops_per_s);

/* L2 read bandwidth: coalesced 16-byte reads sweeping img[0..n_words) (n_words a
 * multiple of 4, the buffer L2-resident after the warm-up run) `passes` times;
 * *bytes_per_s = bytes read per second; sink: 148*64*256 floats. */
int recon_probe_l2_stream(const float* img, int64_t n_words, int32_t passes, float* sink, void* stream,
                          double* bytes_per_s);

#ifdef __cplusplus
}
#endif

#endif /* RECON_PROBE_H */
