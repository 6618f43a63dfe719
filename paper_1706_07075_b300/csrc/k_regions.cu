// TOF-assisted division of the events into body regions (Sec. 2.5 and
// Fig. 4 of arXiv:1706.07075).
//
// Each event's TOF-estimated annihilation z is
//     z_tof = (z1 + z2) * 0.5 + (d * dz) / D,   D = sqrt((dx*dx + dy*dy) + dz*dz),
// evaluated in FP64 with every operation rounded on its own (no fused
// multiply-add), so that the assignment is reproducible bit for bit.  Region
// r takes the event iff z_b[r] - shell <= z_tof < z_b[r+1] + shell (the 6 mm
// outer shell of Sec. 2.5), so with cores at least 2*shell wide an event
// feeds one or two neighbouring regions.  Code per event: 0xFF none, r, or
// r | 0x80 for regions r and r+1.
//
// Binning is a stable counting sort: per-tile counts, an exclusive scan over
// (region, tile), then each tile writes its members in ascending event order.
#include <algorithm>

#include "recon_device.cuh"

namespace recon {

namespace {

constexpr int kSplitThreads = 256;

__device__ __forceinline__ void event_z_inputs(const float4* ev, const int4* pk, double L, long long i, double& x1,
                                               double& y1, double& z1, double& x2, double& y2, double& z2,
                                               double& d)
{
    if (ev) {
        float4 a = ev[2 * i], b = ev[2 * i + 1];
        x1 = a.x; y1 = a.y; z1 = a.z; d = a.w;
        x2 = b.x; y2 = b.y; z2 = b.z;
    } else {
        int4 r = pk[i];
        x1 = __dmul_rn((double)(short)(r.x & 0xFFFF), L);
        y1 = __dmul_rn((double)(short)(r.x >> 16), L);
        z1 = __dmul_rn((double)(short)(r.y & 0xFFFF), L);
        x2 = __dmul_rn((double)(short)(r.y >> 16), L);
        y2 = __dmul_rn((double)(short)(r.z & 0xFFFF), L);
        z2 = __dmul_rn((double)(short)(r.z >> 16), L);
        d = (double)__half2float(__ushort_as_half((unsigned short)(r.w & 0xFFFF)));
    }
}

__device__ __forceinline__ uint8_t region_code(const float4* ev, const int4* pk, double L, long long i,
                                               const double* zb, int R, double shell)
{
    double x1, y1, z1, x2, y2, z2, d;
    event_z_inputs(ev, pk, L, i, x1, y1, z1, x2, y2, z2, d);
    return region_code_of(x1, y1, z1, x2, y2, z2, d, zb, R, shell);
}

struct Bounds {
    double zb[kMaxRegions + 1];
};

__device__ __forceinline__ bool member(uint8_t c, int r)
{
    if (c >= 0xFE) return false;
    const int f = c & 0x7F;
    return f == r || ((c & 0x80) && f + 1 == r);
}

// Codes and per-tile member counts; counts[tile * (R + 1) + r].  A code 0xFE
// (three or more regions) is counted in slot R so the host can reject it.
__global__ void __launch_bounds__(kSplitThreads) k_region_codes(const float4* ev, const int4* pk, double L, long long n,
                                                                Bounds b, int R, double shell, uint8_t* codes,
                                                                int* counts, int tile)
{
    __shared__ int cnt[kMaxRegions + 1];
    for (int r = threadIdx.x; r <= R; r += blockDim.x) cnt[r] = 0;
    __syncthreads();
    const long long t0 = (long long)blockIdx.x * tile;
    const long long t1 = min(t0 + tile, n);
    for (long long i = t0 + threadIdx.x; i < t1; i += blockDim.x) {
        uint8_t c = region_code(ev, pk, L, i, b.zb, R, shell);
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

// Exclusive block scan of ints; returns the exclusive prefix, total in *tot.
__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int* tot)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    const int warp_base = wid > 0 ? sh[wid - 1] : 0;
    *tot = sh[nw - 1];
    __syncthreads();
    return warp_base + x - v;
}

// offsets[r] = start of region r in the binned list (offsets[R] = total,
// offsets[R+1] = events in three or more regions); base[tile * R + r] = where
// tile's members of region r go.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_region_scan(const int* counts, int n_tiles, int R, long long* offsets,
                                                      long long* base)
{
    __shared__ int sh[32];
    __shared__ long long shb[32];
    long long running = 0;
    for (int r = 0; r < R; ++r) {
        if (threadIdx.x == 0) offsets[r] = running;
        for (int t0 = 0; t0 < n_tiles; t0 += blockDim.x) {
            const int t = t0 + threadIdx.x;
            const int v = t < n_tiles ? counts[(long long)t * (R + 1) + r] : 0;
            int tot;
            const int ex = block_exclusive_scan(v, sh, &tot);
            if (t < n_tiles) base[(long long)t * R + r] = running + ex;
            running += tot;
        }
    }
    if (threadIdx.x == 0) offsets[R] = running;
    long long bad = 0;
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) bad += counts[(long long)t * (R + 1) + R];
    bad = warp_sum(bad);
    if ((threadIdx.x & 31) == 0) shb[threadIdx.x >> 5] = bad;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += shb[w];
        offsets[R + 1] = b;
    }
}

// Each tile writes the indices of its members of each region in ascending
// event order (rounds of blockDim events; a block scan per round and region).
__global__ void __launch_bounds__(kSplitThreads) k_region_scatter(const uint8_t* codes, long long n, int R,
                                                                  const long long* base, int tile, int* idx)
{
    __shared__ int sh[32];
    const long long t0 = (long long)blockIdx.x * tile;
    const long long t1 = min(t0 + tile, n);
    for (int r = 0; r < R; ++r) {
        long long pos = base[(long long)blockIdx.x * R + r];
        for (long long i0 = t0; i0 < t1; i0 += blockDim.x) {
            const long long i = i0 + threadIdx.x;
            const int f = (i < t1 && member(codes[i], r)) ? 1 : 0;
            int tot;
            const int ex = block_exclusive_scan(f, sh, &tot);
            if (f) idx[pos + ex] = (int)i;
            pos += tot;
        }
    }
}

// Region-ordered copy of the events with w_i halved for events fed to two
// regions, so the summed slabs count every event once.
__global__ void k_region_gather(const float4* ev, const int4* pk, const uint8_t* codes, const int* idx,
                                long long total, float4* out, int4* out_pk)
{
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (long long)gridDim.x * blockDim.x) {
        const int i = idx[p];
        const float f = (codes[i] & 0x80) ? 0.5f : 1.f;
        if (ev) {
            float4 a = ev[2 * (long long)i], b = ev[2 * (long long)i + 1];
            b.w *= f;
            out[2 * p] = a;
            out[2 * p + 1] = b;
        } else {
            int4 r = pk[i];
            float w = __half2float(__ushort_as_half((unsigned short)((unsigned)r.w >> 16))) * f;
            r.w = (int)(((unsigned)r.w & 0xFFFFu) | ((unsigned)__half_as_ushort(__float2half_rn(w)) << 16));
            out_pk[p] = r;
        }
    }
}

}  // namespace

cudaError_t launch_region_codes(const float4* ev_f32, const int4* ev_packed, double lattice, long long n,
                                const double* z_bounds, int n_regions, double shell, uint8_t* codes,
                                int* block_counts, int tile, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    Bounds b;
    for (int r = 0; r <= n_regions; ++r) b.zb[r] = z_bounds[r];
    const long long tiles = (n + tile - 1) / tile;
    k_region_codes<<<(unsigned)tiles, kSplitThreads, 0, st>>>(ev_f32, ev_packed, lattice, n, b, n_regions, shell,
                                                              codes, block_counts, tile);
    return cudaGetLastError();
}

cudaError_t launch_region_scan(const int* block_counts, int n_tiles, int n_regions, long long* offsets,
                               long long* block_base, cudaStream_t st)
{
    k_region_scan<<<1, 1024, 0, st>>>(block_counts, n_tiles, n_regions, offsets, block_base);
    return cudaGetLastError();
}

cudaError_t launch_region_scatter(const uint8_t* codes, long long n, int n_regions, const long long* block_base,
                                  int tile, int* idx, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long long tiles = (n + tile - 1) / tile;
    k_region_scatter<<<(unsigned)tiles, kSplitThreads, 0, st>>>(codes, n, n_regions, block_base, tile, idx);
    return cudaGetLastError();
}

cudaError_t launch_region_gather(const float4* ev_f32, const int4* ev_packed, const uint8_t* codes,
                                 const int* idx, long long total, float4* out_f32, int4* out_packed,
                                 cudaStream_t st)
{
    if (total <= 0) return cudaSuccess;
    long long blocks = std::min((total + 255) / 256, 148LL * 32);
    k_region_gather<<<(unsigned)blocks, 256, 0, st>>>(ev_f32, ev_packed, codes, idx, total, out_f32, out_packed);
    return cudaGetLastError();
}

}  // namespace recon
