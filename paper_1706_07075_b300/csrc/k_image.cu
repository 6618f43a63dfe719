// Image-side kernels: sensitivity backprojection, start image, the
// multiplicative update with its FP64 conservation sums, the per-iteration
// finalisation, event ingest into the resident layout, and the stitch of
// region slabs (Sec. 2.4 and Sec. 2.5 of arXiv:1706.07075).
#include <algorithm>

#include "recon_device.cuh"

namespace recon {

namespace {

constexpr int kImgThreads = 256;

// s_j += L_lj: the chord of each LOR's line through the grid, no TOF
// (sensitivity, Sec. 2.4 "sensitive matrix"), computed and accumulated in FP64.
// The walk is the incremental Siddon walk of the event pass written in double:
// clip the line M + t u to the grid box (slab method), find the voxel at the
// entry point, then cross the nearest voxel plane at each step, plane positions
// taken as first + m * step per axis, each axis crossed only as often as the
// grid has voxels left in that direction.  In FP32 a crossing t = (X - M) / u_k
// carries ulp(|X - M|) / |u_k| of rounding, which on a 2.4 m grid moves up to
// ~1 mm of chord between neighbouring voxels for lines nearly parallel to a
// plane; the sensitivity is computed once per scanner and grid, so it takes
// FP64 throughout.
__global__ void __launch_bounds__(256) k_sensitivity(const float* __restrict__ lor, long long n, GridD g,
                                                     double* __restrict__ s)
{
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    double p1[3], p2[3];
    for (int k = 0; k < 3; ++k) {
        p1[k] = lor[(long long)k * n + l];
        p2[k] = lor[(long long)(3 + k) * n + l];
    }
    const double dx = p1[0] - p2[0], dy = p1[1] - p2[1], dz = p1[2] - p2[2];
    const double D = sqrt(dx * dx + dy * dy + dz * dz);
    if (!(D > 0.0) || !(D < 1e300)) return;
    const double u[3] = {dx / D, dy / D, dz / D};
    const double c[3] = {0.5 * (p1[0] + p2[0]), 0.5 * (p1[1] + p2[1]), 0.5 * (p1[2] + p2[2])};
    const double lo[3] = {g.ox, g.oy, g.oz};
    const double v[3] = {g.vx, g.vy, g.vz};
    const int nn[3] = {g.nx, g.ny, g.nz};
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    double a = -inf, b = inf;
    for (int k = 0; k < 3; ++k) {
        const double hi = lo[k] + (double)nn[k] * v[k];
        if (u[k] == 0.0) {
            if (!(c[k] >= lo[k] && c[k] < hi)) return;
        } else {
            const double t0 = (lo[k] - c[k]) / u[k], t1 = (hi - c[k]) / u[k];
            a = fmax(a, fmin(t0, t1));
            b = fmin(b, fmax(t0, t1));
        }
    }
    if (!(a < b)) return;
    int idx[3], step[3];
    double tnext[3], dt[3], rem[3];
    for (int k = 0; k < 3; ++k) {
        const double x = fma(a, u[k], c[k]);
        const double fi = fmin(fmax(floor((x - lo[k]) / v[k]), 0.0), (double)(nn[k] - 1));
        const int i = (int)fi;
        idx[k] = i;
        if (u[k] > 0.0) {
            step[k] = 1;
            tnext[k] = (lo[k] + (double)(i + 1) * v[k] - c[k]) / u[k];
            dt[k] = v[k] / u[k];
            rem[k] = (double)(nn[k] - 1 - i);
        } else if (u[k] < 0.0) {
            step[k] = -1;
            tnext[k] = (lo[k] + (double)i * v[k] - c[k]) / u[k];
            dt[k] = -v[k] / u[k];
            rem[k] = (double)i;
        } else {
            step[k] = 0;
            tnext[k] = inf;
            dt[k] = 0.0;
            rem[k] = 0.0;
        }
        if (rem[k] <= 0.0) tnext[k] = inf;
    }
    const double t_first[3] = {tnext[0], tnext[1], tnext[2]};
    double m[3] = {0.0, 0.0, 0.0};
    long long j = idx[0] + (long long)g.nx * (idx[1] + (long long)g.ny * idx[2]);
    const long long sl[3] = {step[0], (long long)step[1] * g.nx, (long long)step[2] * g.nx * g.ny};
    double tau = a;
    const int max_steps = g.nx + g.ny + g.nz + 2;
    for (int it = 0; it < max_steps; ++it) {
        const double tmin = fmin(tnext[0], fmin(tnext[1], tnext[2]));
        const double tn = fmax(fmin(tmin, b), tau);
#ifdef RECON_BOUNDS_CHECK
        if (!index_ok(j, (long long)g.nx * g.ny * g.nz)) break;
#endif
        if (tn > tau) atomicAdd(s + j, tn - tau);
        if (tmin >= b) break;
        tau = tn;
        const int k = tnext[0] == tmin ? 0 : (tnext[1] == tmin ? 1 : 2);
        j += sl[k];
        m[k] += 1.0;
        tnext[k] = m[k] < rem[k] ? fma(m[k], dt[k], t_first[k]) : inf;
    }
}

// FP32 copy of s and per-block FP64 sums of s over the mask s > 0.
__global__ void __launch_bounds__(kImgThreads) k_sens_finish(const double* __restrict__ s64, long long n,
                                                             float* __restrict__ s32, double* __restrict__ part)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        double v = s64[j];
        s32[j] = (float)v;
        if (v > 0.0) acc += v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_fill_masked(float* __restrict__ lam, const float* __restrict__ s, long long n, float value)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        lam[j] = s[j] > 0.f ? value : 0.f;
}

// lambda_j <- lambda_j C_j / s_j on {s_j > 0}, else 0; C_j <- 0.  Blocks are
// assigned per region; each block leaves the FP64 sum of s_j lambda_j of its
// voxels in part[region * bpr + block_in_region].
__global__ void __launch_bounds__(kImgThreads) k_update(float* __restrict__ lam, float* __restrict__ C,
                                                        const float* __restrict__ s, uint16_t* __restrict__ lam_bf16,
                                                        const long long* __restrict__ reg_vox, int bpr,
                                                        double* __restrict__ part, float scale)
{
    __shared__ double sh[32];
    const int r = blockIdx.x / bpr, b = blockIdx.x % bpr;
    const long long lo = reg_vox[r], hi = reg_vox[r + 1];
    double acc = 0.0;
    for (long long j = lo + (long long)b * blockDim.x + threadIdx.x; j < hi; j += (long long)bpr * blockDim.x) {
        float sj = s[j];
        float v = 0.f;
        if (sj > 0.f) v = lam[j] * C[j] * scale / sj;   // scale = 1 (MLEM) or B (OSEM: s / B)
        lam[j] = v;
        C[j] = 0.f;
        if (lam_bf16) lam_bf16[j] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        acc += (double)sj * (double)v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// hist[(k * R + r) * 2 + {0,1}] = {N_eff, sum_j s_j lambda_j} of region r after
// iteration k = *iter; then ++*iter.  One block; fixed summation order.
// The pass slots (pass_slots x R) are cleared after reading, ready for the
// next iteration's pass.
__global__ void k_finalize(double* __restrict__ pass_part, int pass_slots, const double* __restrict__ upd_part,
                           int bpr, int R, double* __restrict__ hist, int* __restrict__ iter, int max_iter)
{
    __shared__ double sh[32];
    const int k = *iter;
    for (int r = 0; r < R; ++r) {
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < pass_slots; i += blockDim.x) {
            a += pass_part[(long long)i * R + r];
            pass_part[(long long)i * R + r] = 0.0;
        }
        for (int i = threadIdx.x; i < bpr; i += blockDim.x) b += upd_part[(long long)r * bpr + i];
        a = block_sum(a, sh);
        b = block_sum(b, sh);
        if (threadIdx.x == 0 && k < max_iter) {
            hist[((long long)k * R + r) * 2 + 0] = a;
            hist[((long long)k * R + r) * 2 + 1] = b;
        }
    }
    if (threadIdx.x == 0) *iter = k + 1;
}

__global__ void k_to_bf16(const float* __restrict__ src, uint16_t* __restrict__ dst, long long n)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        dst[j] = __bfloat16_as_ushort(__float2bfloat16_rn(src[j]));
}

struct Planes7 {
    const float* p[7];
};

// Caller's SoA planes (x1,y1,z1,x2,y2,z2,d) -> resident (x1,y1,z1,d),(x2,y2,z2,w).
__global__ void k_ingest_f32(Planes7 pl, const float* __restrict__ weight, long long n, float4* __restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float w = weight ? weight[i] : 1.f;
        out[2 * i] = make_float4(pl.p[0][i], pl.p[1][i], pl.p[2][i], pl.p[6][i]);
        out[2 * i + 1] = make_float4(pl.p[3][i], pl.p[4][i], pl.p[5][i], w);
    }
}

// Packed records: keep the endpoints and d, put the FP16 weight in the pad.
__global__ void k_ingest_packed(const int4* __restrict__ rec, const float* __restrict__ weight, long long n,
                                int4* __restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int4 r = rec[i];
        float w = weight ? weight[i] : 1.f;
        unsigned hw = __half_as_ushort(__float2half_rn(w));
        r.w = (int)(((unsigned)r.w & 0xFFFFu) | (hw << 16));
        out[i] = r;
    }
}

__global__ void __launch_bounds__(kImgThreads) k_reduce_weights(const float4* __restrict__ ev,
                                                                const int4* __restrict__ pk, long long n,
                                                                double* __restrict__ part)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (ev) acc += (double)ev[2 * i + 1].w;
        else acc += (double)__half2float(__ushort_as_half((unsigned short)((unsigned)pk[i].w >> 16)));
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// Per-event weights w_i of the resident records into out[n].
__global__ void k_event_weights(const float4* __restrict__ ev, const int4* __restrict__ pk, long long n,
                                float* __restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = ev ? ev[2 * i + 1].w : __half2float(__ushort_as_half((unsigned short)((unsigned)pk[i].w >> 16)));
}

struct StitchTable {
    int n;
    long long vox[kMaxRegions + 1];
    int lo[kMaxRegions], hi[kMaxRegions];
};

// Whole-body image = sum over regions of each slab image at its place
// (Sec. 2.5: the nine images are summed into one volume).
__global__ void k_stitch(const float* __restrict__ slabs, StitchTable t, int nx, int ny, int nz, float* __restrict__ out)
{
    const long long plane = (long long)nx * ny;
    const long long n = plane * nz;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(j / plane);
        const long long in_plane = j - (long long)k * plane;
        float acc = 0.f;
        for (int r = 0; r < t.n; ++r)
            if (k >= t.lo[r] && k < t.hi[r]) acc += slabs[t.vox[r] + (long long)(k - t.lo[r]) * plane + in_plane];
        out[j] = acc;
    }
}

int grid_for(long long n, int threads, int cap = 148 * 32)
{
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

cudaError_t launch_sensitivity(const float* lor6, long long n, const GridD& g, double* s_acc, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_sensitivity<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(lor6, n, g, s_acc);
    return cudaGetLastError();
}

cudaError_t launch_sens_finish(const double* s64, long long n_vox, float* s32, double* partial, int blocks,
                               cudaStream_t st)
{
    k_sens_finish<<<blocks, kImgThreads, 0, st>>>(s64, n_vox, s32, partial);
    return cudaGetLastError();
}

cudaError_t launch_fill_masked(float* lam, const float* s32, long long n_vox, float value, cudaStream_t st)
{
    if (n_vox <= 0) return cudaSuccess;
    k_fill_masked<<<grid_for(n_vox, kImgThreads), kImgThreads, 0, st>>>(lam, s32, n_vox, value);
    return cudaGetLastError();
}

int update_blocks(long long n_vox)
{
    long long b = (n_vox + 4 * kImgThreads - 1) / (4 * kImgThreads);
    return (int)std::max(1LL, std::min(b, 148LL * 8));
}

cudaError_t launch_update(float* lam, float* C, const float* s32, uint16_t* lam_bf16, const long long* reg_vox,
                          int n_regions, double* partial, int blocks_per_region, cudaStream_t st, float scale)
{
    k_update<<<n_regions * blocks_per_region, kImgThreads, 0, st>>>(lam, C, s32, lam_bf16, reg_vox,
                                                                   blocks_per_region, partial, scale);
    return cudaGetLastError();
}

cudaError_t launch_finalize(double* pass_partial, int pass_slots, const double* upd_partial,
                            int upd_blocks_per_region, int n_regions, double* hist, int* iter_counter,
                            int max_iter, cudaStream_t st)
{
    k_finalize<<<1, 256, 0, st>>>(pass_partial, pass_slots, upd_partial, upd_blocks_per_region, n_regions, hist,
                                  iter_counter, max_iter);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, uint16_t* dst, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_to_bf16<<<grid_for(n, kImgThreads), kImgThreads, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_ingest_f32(const float* const* planes, const float* weight, long long n, float4* out,
                              cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    Planes7 pl;
    for (int k = 0; k < 7; ++k) pl.p[k] = planes[k];
    k_ingest_f32<<<grid_for(n, kImgThreads), kImgThreads, 0, st>>>(pl, weight, n, out);
    return cudaGetLastError();
}

cudaError_t launch_ingest_packed(const int4* rec, const float* weight, long long n, int4* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_ingest_packed<<<grid_for(n, kImgThreads), kImgThreads, 0, st>>>(rec, weight, n, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_weights(const float4* ev_f32, const int4* ev_packed, long long n, double* partial,
                                  int blocks, cudaStream_t st)
{
    k_reduce_weights<<<blocks, kImgThreads, 0, st>>>(ev_f32, ev_packed, n, partial);
    return cudaGetLastError();
}

cudaError_t launch_stitch(const float* slabs, const long long* reg_vox, const int* slab_lo, const int* slab_hi,
                          int n_regions, int nx, int ny, int nz, float* out, cudaStream_t st)
{
    StitchTable t;
    t.n = n_regions;
    for (int r = 0; r <= n_regions; ++r) t.vox[r] = reg_vox[r];
    for (int r = 0; r < n_regions; ++r) {
        t.lo[r] = slab_lo[r];
        t.hi[r] = slab_hi[r];
    }
    long long n = (long long)nx * ny * nz;
    k_stitch<<<grid_for(n, kImgThreads), kImgThreads, 0, st>>>(slabs, t, nx, ny, nz, out);
    return cudaGetLastError();
}

cudaError_t launch_event_weights(const float4* ev_f32, const int4* ev_packed, long long n, float* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_event_weights<<<grid_for(n, kImgThreads), kImgThreads, 0, st>>>(ev_f32, ev_packed, n, out);
    return cudaGetLastError();
}

// Out-of-range voxel indices the walks of this file skipped since the last call
// (bounds-checked build; 0 otherwise).
unsigned long long oob_count_image() { return oob_take(); }

}  // namespace recon
