// recon_split_regions_noalloc: the TOF-assisted region split for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc.  A process whose device memory belongs
// to another allocator (a framework's caching pool, or an acquisition service
// that reserves all of the GPU's memory when it starts) would see an extra
// allocation fail, or fragment a pool it does not own.  A real-time path
// cannot afford cudaFree, which waits for the whole device, or an allocation
// that may fail half-way through a scan.  This entry point takes only
// caller-owned inputs and outputs; its per-tile counters and prefix sums live
// in one fixed, file-scope device array that every GPU loading this library
// holds until the process exits.
//
// The split itself is the one recon_split_regions performs (Sec. 2.5 of
// arXiv:1706.07075); this file holds a variant of the region-code kernel that
// reads the caller's SoA planes directly and counts into the static array.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "recon.h"
#include "recon_device.cuh"

namespace recon {
void set_thread_error(const std::string& msg);  // recon_api.cu: message for recon_last_error(NULL)
}

using namespace recon;

namespace {

constexpr int kTile = 32768;                        // events per block of the code and scatter kernels
constexpr int kThreads = 256;
constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB per device
constexpr size_t kOffsetsBytes = 1024;              // offsets[R + 2] (R <= 64)

// Counters, prefix sums and offsets of the no-alloc split.  Shared by every
// call on the device; the contents left by the previous call are overwritten.
static __device__ __align__(256) unsigned char g_split_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[256] = {};  // device address of g_split_scratch, per device ordinal

// Largest event count the scratch holds for R regions: offsets, then per
// tile (R + 1) int counts and R int64 bases.
long long max_events_for(int R)
{
    const long long per_tile = 4LL * (R + 1) + 8LL * R;
    return ((long long)(kScratchBytes - kOffsetsBytes - 8) / per_tile) * kTile;
}

// Region code of event i of the caller's SoA planes: the same arithmetic as the
// allocating split (region_code_of in recon_device.cuh).
__device__ __forceinline__ unsigned char region_code_soa(const float* const* pl, long long i, const double* zb, int R,
                                                         double shell)
{
    return region_code_of(pl[0][i], pl[1][i], pl[2][i], pl[3][i], pl[4][i], pl[5][i], pl[6][i], zb, R, shell);
}

struct Planes {
    const float* p[7];
};

struct Bounds {
    double zb[kMaxRegions + 1];
};

// Region codes of the caller's SoA events and per-tile member counts, written
// into the static scratch (after the offsets block): counts[tile * (R + 1) + r].
__global__ void __launch_bounds__(kThreads) k_region_codes_soa(Planes pl, long long n, Bounds b, int R, double shell,
                                                               unsigned char* codes)
{
    __shared__ int cnt[kMaxRegions + 1];
    int* counts = reinterpret_cast<int*>(g_split_scratch + kOffsetsBytes);
    for (int r = threadIdx.x; r <= R; r += blockDim.x) cnt[r] = 0;
    __syncthreads();
    const long long t0 = (long long)blockIdx.x * kTile;
    const long long t1 = min(t0 + kTile, n);
    for (long long i = t0 + threadIdx.x; i < t1; i += blockDim.x) {
        unsigned char c = region_code_soa(pl.p, i, b.zb, R, shell);
        codes[i] = c;
        if (c == 0xFE) atomicAdd(&cnt[R], 1);
        else if (c != 0xFF) {
            atomicAdd(&cnt[c & 0x7F], 1);
            if (c & 0x80) atomicAdd(&cnt[(c & 0x7F) + 1], 1);
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r <= R; r += blockDim.x) counts[(long long)blockIdx.x * (R + 1) + r] = cnt[r];
}

recon_status fail(recon_status s, const char* msg)
{
    set_thread_error(msg);
    return s;
}

// Device address of the static scratch on the current device, looked up once.
recon_status scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(RECON_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= 256) return fail(RECON_ECUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_split_scratch);
        if (e != cudaSuccess || !p) {
            char buf[160];
            snprintf(buf, sizeof buf, "cudaGetSymbolAddress of the split scratch failed: %s", cudaGetErrorString(e));
            cudaGetLastError();
            return fail(RECON_ECUDA, buf);
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RECON_OK;
}

// The call launches kernels that read `p` and write through it, so it must be
// device (or managed) memory of the current device: a host pointer, pinned or
// not, is rejected here instead of faulting in a kernel.
recon_status check_device_pointer(const void* p, const char* what)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    char buf[200];
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(buf, sizeof buf, "%s is not a device pointer (%s)", what, cudaGetErrorString(e));
        return fail(RECON_EINVAL, buf);
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
        snprintf(buf, sizeof buf, "%s must be device memory (got %s memory)", what,
                 at.type == cudaMemoryTypeHost ? "page-locked host" : "unregistered host");
        return fail(RECON_EINVAL, buf);
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(RECON_ECUDA, "cudaGetDevice failed");
    }
    if (at.type == cudaMemoryTypeDevice && at.device != dev) {
        snprintf(buf, sizeof buf, "%s lives on device %d, not on the current device %d", what, at.device, dev);
        return fail(RECON_EINVAL, buf);
    }
    return RECON_OK;
}

}  // namespace

extern "C" recon_status recon_split_regions_noalloc(const recon_grid* grid, const recon_events* events,
                                                    int32_t n_regions, const recon_region* regions, double shell_mm,
                                                    uint8_t* code_out, int64_t* offsets_out, int32_t* idx_out,
                                                    int64_t idx_capacity, void* cuda_stream)
{
    set_thread_error("");
    if (!grid || !events || !regions || !offsets_out) return fail(RECON_EINVAL, "NULL grid, events, regions or offsets_out");
    if (grid->nz <= 0 || !(grid->vz > 0) || !std::isfinite(grid->vz) || !std::isfinite(grid->oz))
        return fail(RECON_EINVAL, "invalid grid");
    if (events->fmt != RECON_EV_F32_SOA || !events->on_device)
        return fail(RECON_EINVAL, "events must be F32 SoA planes in device memory");
    const long long n = events->n;
    const int R = n_regions;
    if (R < 1 || R > kMaxRegions) return fail(RECON_EINVAL, "n_regions must be in [1, 64]");
    if (!(shell_mm >= 0) || !std::isfinite(shell_mm)) return fail(RECON_EINVAL, "shell_mm must be >= 0");
    for (int r = 0; r < R; ++r) {
        if (regions[r].z_lo < 0 || regions[r].z_hi > grid->nz || regions[r].z_lo >= regions[r].z_hi)
            return fail(RECON_EINVAL, "region slice range outside the grid or empty");
        if (r + 1 < R && regions[r + 1].z_lo != regions[r].z_hi) return fail(RECON_EINVAL, "regions must be consecutive");
        if ((double)(regions[r].z_hi - regions[r].z_lo) * grid->vz < 2.0 * shell_mm)
            return fail(RECON_EINVAL, "region core thinner than 2 * shell_mm");
    }
    if (n < 0) return fail(RECON_EINVAL, "event count is negative");
    if (n >= (1LL << 31)) return fail(RECON_EINVAL, "event count must stay below 2^31");
    const long long n_max = max_events_for(R);
    if (n > n_max) {
        char buf[200];
        snprintf(buf, sizeof buf, "%lld events exceed the no-alloc scratch limit of %lld events for %d regions", n,
                 n_max, R);
        return fail(RECON_EINVAL, buf);
    }
    if (n > 0) {
        for (int k = 0; k < 7; ++k)
            if (!events->planes[k]) return fail(RECON_EINVAL, "event plane pointer is NULL");
        if (!code_out) return fail(RECON_EINVAL, "code_out is NULL");
        static const char* kPlaneNames[7] = {"event plane x1", "event plane y1", "event plane z1", "event plane x2",
                                             "event plane y2", "event plane z2", "event plane d"};
        for (int k = 0; k < 7; ++k) {
            recon_status ps = check_device_pointer(events->planes[k], kPlaneNames[k]);
            if (ps != RECON_OK) return ps;
        }
        recon_status ps = check_device_pointer(code_out, "code_out");
        if (ps != RECON_OK) return ps;
        if (idx_out) {
            ps = check_device_pointer(idx_out, "idx_out");
            if (ps != RECON_OK) return ps;
        }
    }
    if (idx_capacity < 0) return fail(RECON_EINVAL, "idx_capacity is negative");
    if (n == 0) {
        for (int r = 0; r <= R; ++r) offsets_out[r] = 0;
        return RECON_OK;
    }
    void* scratch = nullptr;
    recon_status s = scratch_address(&scratch);
    if (s != RECON_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    long long* d_offsets = static_cast<long long*>(scratch);
    int* d_counts = reinterpret_cast<int*>(static_cast<unsigned char*>(scratch) + kOffsetsBytes);
    const long long tiles = (n + kTile - 1) / kTile;
    long long* d_base = reinterpret_cast<long long*>(static_cast<unsigned char*>(scratch) + kOffsetsBytes +
                                                     ((size_t)tiles * (R + 1) * 4 + 7) / 8 * 8);

    Planes pl;
    for (int k = 0; k < 7; ++k) pl.p[k] = static_cast<const float*>(events->planes[k]);
    Bounds b;
    for (int r = 0; r < R; ++r) b.zb[r] = grid->oz + (double)regions[r].z_lo * grid->vz;
    b.zb[R] = grid->oz + (double)regions[R - 1].z_hi * grid->vz;

    char buf[200];
    auto cuda_fail = [&](cudaError_t e, const char* what) {
        snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
        cudaGetLastError();
        return fail(RECON_ECUDA, buf);
    };
    cudaError_t e = cudaMemsetAsync(scratch, 0, kOffsetsBytes + (size_t)tiles * (R + 1) * 4, st);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the scratch");
    k_region_codes_soa<<<(unsigned)tiles, kThreads, 0, st>>>(pl, n, b, R, shell_mm, code_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_region_codes_soa");
    if ((e = launch_region_scan(d_counts, (int)tiles, R, d_offsets, d_base, st)) != cudaSuccess)
        return cuda_fail(e, "region scan");
    long long h_off[kMaxRegions + 2];
    if ((e = cudaMemcpyAsync(h_off, d_offsets, sizeof(long long) * (R + 2), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "reading the offsets");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (h_off[R + 1] != 0) return fail(RECON_EINVAL, "events fall in three or more regions");
    if (h_off[R] > idx_capacity) {
        snprintf(buf, sizeof buf, "idx_out holds %lld entries but the split needs %lld", (long long)idx_capacity,
                 h_off[R]);
        return fail(RECON_EINVAL, buf);
    }
    if (h_off[R] > 0) {
        if (!idx_out) return fail(RECON_EINVAL, "idx_out is NULL");
        if ((e = launch_region_scatter(code_out, n, R, d_base, kTile, idx_out, st)) != cudaSuccess)
            return cuda_fail(e, "region scatter");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    for (int r = 0; r <= R; ++r) offsets_out[r] = h_off[r];
    return RECON_OK;
}
