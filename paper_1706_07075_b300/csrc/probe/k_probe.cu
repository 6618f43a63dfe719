// Hardware probes that measure the roofline denominators of the MLEM event
// pass on the running GPU (not part of the reconstruction): the rate of
// scattered FP32 reductions into an L2-resident image (also with lanes that
// share sectors), the rate of scattered 4-byte gathers from it, and the FP32
// issue rate of the pieces' Gaussian tail evaluation.  Each probe times itself with CUDA events on `stream`
// and returns operations per second.
#include <cstdint>
#include <cuda_runtime.h>

#include "recon_probe.h"

namespace {

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Each thread issues `per_thread` reductions to pseudo-random words of img.
// With `runs` > 1 consecutive reductions of a thread go to consecutive words
// (a run of a Siddon walk along x), else every address is independent.
__global__ void k_red(float* img, uint32_t n_words, int per_thread, int runs)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t h = hash32(t * 0x9e3779b9u + 17u);
    for (int k = 0; k < per_thread; k += runs) {
        h = hash32(h + (uint32_t)k);
        const uint32_t base = h % n_words;
        for (int q = 0; q < runs && k + q < per_thread; ++q) atomicAdd(img + (base + q) % n_words, 1e-7f);
    }
}

__global__ void k_gather(const float* img, uint32_t n_words, int per_thread, float* sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t h = hash32(t * 0x85ebca6bu + 3u);
    float acc = 0.f;
    for (int k = 0; k < per_thread; ++k) {
        h = hash32(h + (uint32_t)k);
        acc += __ldg(img + h % n_words);
    }
    if (acc == 1234.5f) sink[t] = acc;
}

// Reductions whose lanes share 32-byte sectors: the lanes of a warp form groups
// of `group` lanes; each group and step picks one hashed 128-byte line of img
// and lane k of the group adds to word (k * stride) mod 32 of it.  group 1 is
// the scattered case; group 8 with stride 1 puts eight lanes in one sector.
__global__ void k_red_groups(float* img, uint32_t n_lines, int per_thread, int group, int stride)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, warp = t >> 5;
    const uint32_t gid = lane / (uint32_t)group, sub = lane % (uint32_t)group;
    for (int k = 0; k < per_thread; ++k) {
        const uint32_t h = hash32(warp * 7919u + gid * 104729u + (uint32_t)k * 0x9e3779b9u);
        atomicAdd(img + (h % n_lines) * 32u + (sub * (uint32_t)stride) % 32u, 1e-7f);
    }
}

// One scattered gather from `lam` and one scattered reduction into `C` (two
// separate images, as in the fused MLEM pass) per step.
__global__ void k_mixed(const float* lam, float* C, uint32_t n_words, int per_thread, float* sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t h = hash32(t * 0xc2b2ae35u + 11u);
    float acc = 0.f;
    for (int k = 0; k < per_thread; ++k) {
        h = hash32(h + (uint32_t)k);
        acc += __ldg(lam + h % n_words);
        atomicAdd(C + (h >> 7) % n_words, 1e-7f);
    }
    if (acc == 1234.5f) sink[t] = acc;
}

__global__ void k_erfc(int per_thread, float* sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float x = 0.001f * (t & 1023), acc = 0.f;
    for (int k = 0; k < per_thread; ++k) {
        acc += erfcf(x);
        x += 0.0037f;
        if (x > 2.2f) x -= 2.2f;
    }
    if (acc == 1234.5f) sink[t] = acc;
}

// Each thread sums float4s of the buffer at a grid stride, `passes` sweeps.
__global__ void k_l2_stream(const float4* __restrict__ img, long long n4, int passes, float* sink)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    float acc = 0.f;
    for (int p = 0; p < passes; ++p)
        for (long long i = t; i < n4; i += stride) {
            const float4 v = __ldcg(img + i);
            acc += v.x + v.y + v.z + v.w;
        }
    if (acc == 1234.5f) sink[t] = acc;
}

template <class F>
int time_it(cudaStream_t s, F&& launch, double ops, double* out_ops_per_s)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return 3;
    launch();  // warm-up
    cudaEventRecord(a, s);
    launch();
    cudaEventRecord(b, s);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return 3;
    *out_ops_per_s = ops / (ms * 1e-3);
    return 0;
}

}  // namespace

extern "C" int recon_probe_l2_red(float* img, int64_t n_words, int32_t runs, void* stream, double* ops_per_s)
{
    if (!img || n_words <= 0 || n_words >= (1LL << 32) || runs < 1 || !ops_per_s) return 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = 148 * 64, per_thread = 256;
    return time_it(s, [&] { k_red<<<blocks, threads, 0, s>>>(img, (uint32_t)n_words, per_thread, runs); },
                   (double)blocks * threads * per_thread, ops_per_s);
}

extern "C" int recon_probe_red_groups(float* img, int64_t n_words, int32_t group, int32_t stride, void* stream,
                                      double* ops_per_s)
{
    if (!img || n_words < 32 || n_words >= (1LL << 32) || group < 1 || group > 32 || (32 % group) || stride < 1 ||
        stride > 32 || !ops_per_s)
        return 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = 148 * 32, per_thread = 256;
    const uint32_t n_lines = (uint32_t)(n_words / 32);
    return time_it(s, [&] { k_red_groups<<<blocks, threads, 0, s>>>(img, n_lines, per_thread, group, stride); },
                   (double)blocks * threads * per_thread, ops_per_s);
}

extern "C" int recon_probe_gather(const float* img, int64_t n_words, float* sink, void* stream, double* ops_per_s)
{
    if (!img || !sink || n_words <= 0 || n_words >= (1LL << 32) || !ops_per_s) return 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = 148 * 64, per_thread = 256;
    return time_it(s, [&] { k_gather<<<blocks, threads, 0, s>>>(img, (uint32_t)n_words, per_thread, sink); },
                   (double)blocks * threads * per_thread, ops_per_s);
}

extern "C" int recon_probe_mixed(const float* lam, float* C, int64_t n_words, float* sink, void* stream,
                                 double* steps_per_s)
{
    if (!lam || !C || !sink || n_words <= 0 || n_words >= (1LL << 32) || !steps_per_s) return 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = 148 * 64, per_thread = 256;
    return time_it(s, [&] { k_mixed<<<blocks, threads, 0, s>>>(lam, C, (uint32_t)n_words, per_thread, sink); },
                   (double)blocks * threads * per_thread, steps_per_s);
}

extern "C" int recon_probe_erfc(float* sink, void* stream, double* ops_per_s)
{
    if (!sink || !ops_per_s) return 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = 148 * 64, per_thread = 2048;
    return time_it(s, [&] { k_erfc<<<blocks, threads, 0, s>>>(per_thread, sink); },
                   (double)blocks * threads * per_thread, ops_per_s);
}

extern "C" int recon_probe_l2_stream(const float* img, int64_t n_words, int32_t passes, float* sink, void* stream,
                                     double* bytes_per_s)
{
    if (!img || !sink || n_words <= 0 || (n_words & 3) || passes < 1 || !bytes_per_s) return 1;
    if (reinterpret_cast<uintptr_t>(img) % 16) return 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads = 256, blocks = 148 * 64;
    const long long n4 = n_words / 4;
    return time_it(s, [&] { k_l2_stream<<<blocks, threads, 0, s>>>(reinterpret_cast<const float4*>(img), n4, passes,
                                                                  sink); },
                   (double)n_words * 4.0 * passes, bytes_per_s);
}
