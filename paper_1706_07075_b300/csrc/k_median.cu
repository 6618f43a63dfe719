// Median-filter sieve between MLEM iterations (Sec. 2.4): each voxel takes the
// median of its 3 x 3 x 3 neighbourhood, neighbours outside the grid (or the
// region's slab) counting as zero, which lowers border voxels as Sec. 4
// describes for divided images.  Optionally voxels outside the mask {s > 0}
// are set to zero and a BF16 copy is written.
//
// Selection: the 14th smallest of 27 values by forgetful selection (M.
// McGuire, "A fast, small-radius GPU median filter", ShaderX6, 2008): keep a
// working set of 15 values; each round moves the set's minimum and maximum to
// its ends with compare-exchanges, drops both (neither can be the median: at
// least 14 values lie on the other side of each) and takes in one new value;
// after the last value the middle of the final three is the median.  Pure
// min/max, so the result is one of the inputs, bit for bit.
//
// Layout: a thread owns one (x, y) column of a block of 32 x 8 columns and
// walks kZChunk consecutive slices of one region, keeping the three 3 x 3
// planes of the current neighbourhood in registers; each step loads one new
// plane (9 values, coalesced along x across the warp).
#include "recon_device.cuh"

namespace recon {

namespace {

constexpr int kMedTx = 32, kMedTy = 8, kZChunk = 16;

__device__ __forceinline__ void cswap(float& a, float& b)
{
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}

// Median of v[0..26] (values are finite and not NaN).
__device__ __forceinline__ float median27(const float (&v)[27])
{
    float w[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) w[i] = v[i];
#pragma unroll
    for (int k = 15; k >= 3; --k) {
#pragma unroll
        for (int i = 1; i < k; ++i) cswap(w[0], w[i]);           // minimum to w[0]
#pragma unroll
        for (int i = 1; i < k - 1; ++i) cswap(w[i], w[k - 1]);   // maximum to w[k-1]
        if (k > 3) w[0] = v[15 + (15 - k)];                      // drop both, take the next value
    }
    return w[1];
}

__device__ __forceinline__ void load_plane(const float* __restrict__ img, int nx, int ny, int nz, int x, int y, int z,
                                           float (&p)[9])
{
    const bool zin = z >= 0 && z < nz;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int xx = x + dx, yy = y + dy;
            const bool in = zin && xx >= 0 && xx < nx && yy >= 0 && yy < ny;
            p[(dy + 1) * 3 + (dx + 1)] = in ? __ldg(img + ((long long)z * ny + yy) * nx + xx) : 0.f;
        }
    }
}

__global__ void __launch_bounds__(kMedTx * kMedTy) k_median3(const float* __restrict__ in, float* __restrict__ out,
                                                             const float* __restrict__ s32,
                                                             uint16_t* __restrict__ bf16,
                                                             const long long* __restrict__ reg_vox, int nx, int ny,
                                                             int x_tiles)
{
    const int r = blockIdx.z;
    const long long lo = reg_vox[r];
    const long long nxy = (long long)nx * ny;
    const int nz = (int)((reg_vox[r + 1] - lo) / nxy);
    const int x = (blockIdx.x % x_tiles) * kMedTx + threadIdx.x;
    const int y = (blockIdx.x / x_tiles) * kMedTy + threadIdx.y;
    const int z0 = blockIdx.y * kZChunk;
    if (x >= nx || y >= ny || z0 >= nz) return;
    const float* img = in + lo;
    float a[9], b[9], c[9];
    load_plane(img, nx, ny, nz, x, y, z0 - 1, a);
    load_plane(img, nx, ny, nz, x, y, z0, b);
    const int z1 = min(z0 + kZChunk, nz);
    for (int z = z0; z < z1; ++z) {
        load_plane(img, nx, ny, nz, x, y, z + 1, c);
        float v[27];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            v[i] = a[i];
            v[9 + i] = b[i];
            v[18 + i] = c[i];
        }
        const long long j = lo + (long long)z * nxy + (long long)y * nx + x;
        float m = median27(v);
        if (s32 && !(s32[j] > 0.f)) m = 0.f;
        out[j] = m;
        if (bf16) bf16[j] = __bfloat16_as_ushort(__float2bfloat16_rn(m));
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            a[i] = b[i];
            b[i] = c[i];
        }
    }
}

}  // namespace

cudaError_t launch_median3(const float* in, float* out, const float* s32, uint16_t* bf16, const long long* reg_vox,
                           int n_regions, int nx, int ny, int max_nz, cudaStream_t st)
{
    if (n_regions <= 0 || max_nz <= 0 || nx <= 0 || ny <= 0) return cudaSuccess;
    const int x_tiles = (nx + kMedTx - 1) / kMedTx, y_tiles = (ny + kMedTy - 1) / kMedTy;
    const long long xy_blocks = (long long)x_tiles * y_tiles;
    const long long z_chunks = (max_nz + kZChunk - 1) / kZChunk;
    if (xy_blocks > 0x7fffffffLL || z_chunks > 65535 || n_regions > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)xy_blocks, (unsigned)z_chunks, (unsigned)n_regions);
    k_median3<<<grid, dim3(kMedTx, kMedTy), 0, st>>>(in, out, s32, bf16, reg_vox, nx, ny, x_tiles);
    return cudaGetLastError();
}

}  // namespace recon
