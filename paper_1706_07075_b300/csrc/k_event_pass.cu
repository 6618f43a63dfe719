// The MLEM event pass (Sec. 2.4: list-mode TOF-weighted MLEM):
//   p_i = sum_j a_ij lambda_j            forward projection (gather)
//   r_i = w_i / p_i  (events with p_i = 0 are skipped)
//   C_j += a_ij r_i                      backprojection (FP32 reductions)
// fused in one kernel: one thread walks one event, the event's record and
// walk setup staying in registers between the two sweeps.  The second sweep
// either walks the line again or, with a piece cache, replays the voxel
// indices and masses the first sweep left in shared memory (no second Siddon
// walk, no second erfc per piece).  The same kernel body, with the pass kind
// as a template argument, gives the standalone forward and backward
// projectors.
//
// Work distribution: either a flat grid (one event per thread) or a
// persistent grid of (SMs x blocks_per_sm) blocks in which each warp takes
// `chunk` consecutive events at a time from a global counter.  Events of the
// batched (region-divided) form are stored region by region; a thread looks
// its region up in a shared-memory table of event ranges and slab grids.
#include <algorithm>
#include <type_traits>

#include "recon_device.cuh"

namespace recon {

namespace {

struct SharedTable {
    int n;
    long long ev_begin[kMaxRegions + 1];
    GridDev grid[kMaxRegions];
};

__device__ __forceinline__ int find_region(const SharedTable& t, long long i)
{
    int r = 0;
    while (r + 1 < t.n && i >= t.ev_begin[r + 1]) ++r;
    return r;
}

// Adds a warp's N_eff weights to the block's per-region sums: one shared-memory
// atomic per warp when its weighted lanes share a region (always for an undivided
// pass), else one per lane.  All 32 lanes of the warp must call it (w = 0 for a
// lane without an event).
__device__ __forceinline__ void add_neff(float* neff, int r, float w)
{
    const int r0 = __shfl_sync(0xffffffffu, r, 0);
    if (__all_sync(0xffffffffu, r == r0 || w == 0.f)) {
        float s = w;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0 && s != 0.f) atomicAdd(&neff[r0], s);
    } else if (w != 0.f) {
        atomicAdd(&neff[r], w);
    }
}

template <int Fmt>
__device__ __forceinline__ Event load_event(const PassArgs& a, long long i)
{
    if (Fmt == FMT_F32) return load_event_f32(static_cast<const float4*>(a.events), i);
    return load_event_packed(static_cast<const int4*>(a.events), i, a.lattice);
}

// Per-thread cache of one walk's pieces in shared memory, laid out
// [piece][thread] so that a warp's accesses fall in distinct banks.
struct PieceCache {
    int* j;
    float* a;
    int cap;     // pieces per thread (0: no cache)
    int stride;  // blockDim.x
};

// One event of the exact projector over images in the brick layout (one grid,
// FP32 gathers): the same pieces and masses as the linear pass, with gathers and
// FP32 reductions at brick-layout indices.  A 32-byte sector holds a 2x2x2 brick,
// so the nearby lines of a warp's events share sectors more often than in rows
// of 8 voxels: fewer L2 requests per reduction and more L1 hits per gather.
// (Merging a lane's consecutive visits of one 16-byte brick half into one
// red.global.add.v4.f32, or caching the half for the gathers, cost more
// instructions than it saved.)
template <class TailF>
__device__ __forceinline__ float do_event_brick(const PassArgs& a, const Event& e, const GridDev& g,
                                                const TailF& tail)
{
    Line ln;
    Walk w;
    w.valid = false;
    if (event_line(e, ln)) w = make_walk(g, ln, -a.tof.half_window, a.tof.half_window);
    if constexpr (TailF::kSigmaUnits) scale_walk(w, tail.inv_sigma());
    const float hin = a.tof.half_inv_norm * TailF::kMassScale;
    const BrickIndex bi(w, a.brick_bx, a.brick_by);
    // a region's slab: its grid's voxel offset is the slab's place in the brick copies
    const float* const lb = a.lam + g.vox_offset;
    float p = 0.f;
    walk_index<true>(g, tail, w, bi, [&](int q, float m) { p = fmaf(m, __ldg(lb + q), p); });
    p *= hin;
    if (!(p > 0.f)) return 0.f;
    const float r = e.w / p * hin;
    float* const Cb = a.C + g.vox_offset;
    walk_index<true>(g, tail, w, bi, [&](int q, float m) { atomicAdd(Cb + q, m * r); });
    return e.w;
}

// One event; returns the weight it adds to N_eff (0 when p_i = 0).
template <int Kind, int Fmt, bool Cached, bool Brick, class TailF>
__device__ __forceinline__ float do_event(const PassArgs& a, const SharedTable& t, long long i, bool bf16,
                                          const PieceCache& pc, const TailF& tail, int& region)
{
    region = find_region(t, i);
    const GridDev& g = t.grid[region];
    Event e = load_event<Fmt>(a, i);
    if constexpr (Brick) return do_event_brick(a, e, g, tail);
    Line ln;
    Walk w;
    w.valid = false;
    if (event_line(e, ln)) w = make_walk(g, ln, -a.tof.half_window, a.tof.half_window);
    if constexpr (TailF::kSigmaUnits) scale_walk(w, tail.inv_sigma());
    // the walk hands over 2 [Phi(b) - Phi(a)] / kMassScale per piece; half_inv_norm
    // times kMassScale turns it into the TOF mass, applied once to p_i and once to r_i
    const float hin = a.tof.half_inv_norm * TailF::kMassScale;
    float* const Cb = a.C + g.vox_offset;
    if (Kind == PASS_BACK) {
        const float r = a.r_in[i] * hin;
        if (r != 0.f) walk<true>(g, a.tof, tail, w, [&](int j, float m) { atomicAdd(Cb + j, m * r); });
        return 0.f;
    }
    float p = 0.f;
    int cnt = 0;
    const int tid = threadIdx.x;
    const float* const lb = a.lam + g.vox_offset;
    const unsigned short* const hb = reinterpret_cast<const unsigned short*>(a.lam_bf16) + g.vox_offset;
    // the gather precision is uniform over the launch: one walk per form, so that
    // the piece loop carries no select between them
    auto forward = [&](auto gather) {
        walk<true>(g, a.tof, tail, w, [&](int j, float m) {
            p = fmaf(m, gather(j), p);
            if (Cached && Kind == PASS_FUSED) {
                if (cnt < pc.cap) {
                    pc.j[cnt * pc.stride + tid] = j;
                    pc.a[cnt * pc.stride + tid] = m;
                }
                ++cnt;
            }
        });
    };
    if (bf16)
        forward([&](int j) { return __uint_as_float(((unsigned)__ldg(hb + j)) << 16); });
    else
        forward([&](int j) { return __ldg(lb + j); });
    p *= hin;
    if (Kind == PASS_FORWARD) {
        a.p_out[i] = p;
        return 0.f;
    }
    if (!(p > 0.f)) return 0.f;
    const float r = e.w / p * hin;
    if (Cached && cnt <= pc.cap) {
        for (int k = 0; k < cnt; ++k) atomicAdd(Cb + pc.j[k * pc.stride + tid], pc.a[k * pc.stride + tid] * r);
    } else {
        walk<true>(g, a.tof, tail, w, [&](int j, float m) { atomicAdd(Cb + j, m * r); });
    }
    return e.w;
}

template <int TailK>
struct TailOf {
    using type = typename std::conditional<
        TailK == TAIL_FIT, TailFit,
        typename std::conditional<TailK == TAIL_ERFC, TailErfc,
                                  typename std::conditional<TailK == TAIL_SERIES4, TailSeries4,
                                                            TailSeries>::type>::type>::type;
};

template <int Kind, int Fmt, bool Persistent, bool Cached, int TailK, bool Brick = false>
__global__ void __launch_bounds__(256) k_event_pass(PassArgs a, RegionTable tbl, int chunk, int cap)
{
    __shared__ SharedTable t;
    __shared__ float neff[kMaxRegions];
    extern __shared__ unsigned char dyn_smem[];
    PieceCache pc;
    pc.cap = Cached ? cap : 0;
    pc.stride = blockDim.x;
    pc.j = reinterpret_cast<int*>(dyn_smem);
    pc.a = reinterpret_cast<float*>(dyn_smem) + (size_t)pc.cap * blockDim.x;
    if (threadIdx.x == 0) t.n = tbl.n;
    for (int k = threadIdx.x; k <= tbl.n; k += blockDim.x) t.ev_begin[k] = tbl.ev_begin[k];
    for (int k = threadIdx.x; k < tbl.n; k += blockDim.x) {
        t.grid[k] = tbl.grid[k];
        neff[k] = 0.f;
    }
    __syncthreads();
    using TailF = typename TailOf<TailK>::type;
    TailF tail;
    tail.inv_sigma_sqrt2 = a.tof.inv_sigma_sqrt2;
    const bool bf16 = a.lam_bf16 != nullptr;
    const int lane = threadIdx.x & 31;
    if (Persistent) {
        for (;;) {
            unsigned long long start = 0;
            if (lane == 0) start = atomicAdd(a.work, (unsigned long long)chunk);
            start = __shfl_sync(0xffffffffu, start, 0);
            if ((long long)start >= a.n) break;
            const long long end = min((long long)start + chunk, a.n);
            for (long long i = (long long)start + lane; i < end; i += 32) {
                int r;
                float w = do_event<Kind, Fmt, Cached, Brick>(a, t, i, bf16, pc, tail, r);
                if (Kind == PASS_FUSED && w != 0.f) atomicAdd(&neff[r], w);
            }
        }
    } else {
        const unsigned long long b =
            a.block_mul > 1 ? (unsigned long long)blockIdx.x * a.block_mul % gridDim.x : blockIdx.x;
        const long long i = (long long)b * blockDim.x + threadIdx.x;
        int r = 0;
        float w = 0.f;
        if (i < a.n) w = do_event<Kind, Fmt, Cached, Brick>(a, t, i, bf16, pc, tail, r);
        if (Kind == PASS_FUSED) add_neff(neff, r, w);
    }
    if (Kind == PASS_FUSED) {
        // fold the block's N_eff into one of kNeffSlots slots per region; the
        // weights are 1 or 1/2, so the FP64 sums are exact in any order
        __syncthreads();
        for (int k = threadIdx.x; k < t.n; k += blockDim.x)
            if (neff[k] != 0.f) atomicAdd(a.partial + (blockIdx.x % kNeffSlots) * t.n + k, (double)neff[k]);
    }
}

// ------------------------------------------------------------------------
// Sampled TOF kernel (Sec. 2.3, the paper's own projector): sample k of event
// i sits at c + t_k u on the line, c = M + d u the TOF point, and adds its
// weight w_k (unit sum over k) to the one voxel that contains it.  The voxel
// decision is made per axis in voxel units, one IEEE rounding per operation:
//     A = (c - o) * (1/v),  B = u * (1/v),  voxel = floor(fma(t_k, B, A)),
// with u = (P1 - P2) * (1/|P1 - P2|) and |P1 - P2| from an fma chain.
// Samples outside the grid are dropped.  Consecutive samples in the same
// voxel are merged, so a voxel costs one gather and one reduction however
// many samples it holds.

// FP32 reductions of one event's backward sweep, two consecutive visits of
// memory-adjacent voxels of one aligned 8-byte pair sent as one
// red.global.add.v2.f32 (one L2 request instead of two).  Indices are absolute
// (image base + slab offset + voxel); flush() sends what is still pending.
struct PairedRed {
    float* base;
    long long pj = -1;
    float pv = 0.f;
    __device__ __forceinline__ void add(long long aj, float v)
    {
        if (pj >= 0 && ((aj == pj + 1 && !(pj & 1)) || (aj + 1 == pj && !(aj & 1)))) {
            const long long lo = aj < pj ? aj : pj;
            const float vlo = aj < pj ? v : pv, vhi = aj < pj ? pv : v;
            asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(base + lo), "f"(vlo), "f"(vhi) : "memory");
            pj = -1;
            return;
        }
        if (pj >= 0) atomicAdd(base + pj, pv);
        pj = aj;
        pv = v;
    }
    __device__ __forceinline__ void flush()
    {
        if (pj >= 0) atomicAdd(base + pj, pv);
        pj = -1;
    }
};

struct LutLine {
    float ax, ay, az, bx, by, bz;
    bool valid;
};

__device__ __forceinline__ LutLine lut_line(const GridDev& g, const Event& e)
{
    LutLine l;
    const float dx = __fsub_rn(e.p1.x, e.p2.x), dy = __fsub_rn(e.p1.y, e.p2.y), dz = __fsub_rn(e.p1.z, e.p2.z);
    const float D = __fsqrt_rn(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
    l.valid = D > 0.f;
    const float inv = __frcp_rn(D);
    const float ux = __fmul_rn(dx, inv), uy = __fmul_rn(dy, inv), uz = __fmul_rn(dz, inv);
    const float mx = __fmul_rn(0.5f, __fadd_rn(e.p1.x, e.p2.x));
    const float my = __fmul_rn(0.5f, __fadd_rn(e.p1.y, e.p2.y));
    const float mz = __fmul_rn(0.5f, __fadd_rn(e.p1.z, e.p2.z));
    const float ivx = __frcp_rn(g.vx), ivy = __frcp_rn(g.vy), ivz = __frcp_rn(g.vz);
    l.ax = __fmul_rn(__fsub_rn(__fmaf_rn(e.d, ux, mx), g.ox), ivx);
    l.ay = __fmul_rn(__fsub_rn(__fmaf_rn(e.d, uy, my), g.oy), ivy);
    l.az = __fmul_rn(__fsub_rn(__fmaf_rn(e.d, uz, mz), g.oz), ivz);
    l.bx = __fmul_rn(ux, ivx);
    l.by = __fmul_rn(uy, ivy);
    l.bz = __fmul_rn(uz, ivz);
    // a NaN sample position would convert to voxel 0: drop lines with a
    // non-finite coefficient instead
    l.valid = l.valid && isfinite(l.ax) && isfinite(l.ay) && isfinite(l.az) && isfinite(l.bx) &&
              isfinite(l.by) && isfinite(l.bz);
    return l;
}

// Visit (voxel, summed weight) of every run of consecutive samples that share
// a voxel inside the grid.  NS > 0: the sample count known at compile time (the
// loop unrolls and the table entries become constant operands); 0: lut.n.
// Samples of one line; consecutive samples in one voxel are merged into one visit
// (voxel index, summed weight).  Brick: the index is the voxel's place in the brick
// layout (bx, by bricks per row and plane) instead of the linear one.
template <int NS, bool Brick = false, class Visit>
__device__ __forceinline__ void lut_walk(const GridDev& g, const LutH& lut, const LutLine& l, Visit&& visit,
                                         int bx = 0, int by = 0)
{
    if (!l.valid) return;
    int prev = -1;
    float acc = 0.f;
    const int n = NS > 0 ? NS : lut.n;
#pragma unroll
    for (int k = 0; k < n; ++k) {
        const float2 s = lut.s[k];
        // floor to an integer in one conversion; a value beyond the int range
        // saturates, so the unsigned range test drops it like any sample outside
        const int ix = __float2int_rd(__fmaf_rn(s.x, l.bx, l.ax));
        const int iy = __float2int_rd(__fmaf_rn(s.x, l.by, l.ay));
        const int iz = __float2int_rd(__fmaf_rn(s.x, l.bz, l.az));
        const bool in = (unsigned)ix < (unsigned)g.nx && (unsigned)iy < (unsigned)g.ny && (unsigned)iz < (unsigned)g.nz;
        int j = -1;
        if (in) j = Brick ? brick_index(ix, iy, iz, bx, by) : ix + g.nx * (iy + g.ny * iz);
        if (j != prev) {
            if (prev >= 0) visit(prev, acc);
            prev = j;
            acc = 0.f;
        }
        acc += s.y;
    }
    if (prev >= 0) visit(prev, acc);
}

// Fused pass over an image in the brick layout (one grid, FP32 gathers): the same
// visits and weights as the linear pass, gathers and FP32 reductions at
// brick-layout indices (see do_event_brick).
template <int Fmt, int NS>
__device__ __forceinline__ float do_event_lut_brick(const PassArgs& a, const SharedTable& t, long long i,
                                                    int& region)
{
    region = 0;
    const GridDev& g = t.grid[0];
    const Event e = load_event<Fmt>(a, i);
    const LutLine l = lut_line(g, e);
    const float* const lb = a.lam;
    float p = 0.f;
    lut_walk<NS, true>(
        g, a.lut, l, [&](int q, float w) { p = fmaf(w, __ldg(lb + q), p); }, a.brick_bx, a.brick_by);
    if (!(p > 0.f)) return 0.f;
    const float r = e.w / p;
    float* const Cb = a.C;
    lut_walk<NS, true>(
        g, a.lut, l, [&](int q, float w) { atomicAdd(Cb + q, w * r); }, a.brick_bx, a.brick_by);
    return e.w;
}

template <int Kind, int Fmt, int NS>
__device__ __forceinline__ float do_event_lut(const PassArgs& a, const SharedTable& t, long long i, bool bf16,
                                              int& region)
{
    region = find_region(t, i);
    const GridDev& g = t.grid[region];
    const Event e = load_event<Fmt>(a, i);
    const LutLine l = lut_line(g, e);
    float* const Cb = a.C + g.vox_offset;
    if (Kind == PASS_BACK) {
        const float r = a.r_in[i];
        if (r != 0.f) lut_walk<NS>(g, a.lut, l, [&](int j, float w) { atomicAdd(Cb + j, w * r); });
        return 0.f;
    }
    const float* const lb = a.lam + g.vox_offset;
    const unsigned short* const hb = reinterpret_cast<const unsigned short*>(a.lam_bf16) + g.vox_offset;
    float p = 0.f;
    if (bf16)
        lut_walk<NS>(g, a.lut, l,
                     [&](int j, float w) { p = fmaf(w, __uint_as_float(((unsigned)__ldg(hb + j)) << 16), p); });
    else
        lut_walk<NS>(g, a.lut, l, [&](int j, float w) { p = fmaf(w, __ldg(lb + j), p); });
    if (Kind == PASS_FORWARD) {
        a.p_out[i] = p;
        return 0.f;
    }
    if (!(p > 0.f)) return 0.f;
    const float r = e.w / p;
    PairedRed pr{a.C};
    lut_walk<NS>(g, a.lut, l, [&](int j, float w) { pr.add(g.vox_offset + j, w * r); });
    pr.flush();
    return e.w;
}

template <int Kind, int Fmt, int NS, bool Brick = false>
__global__ void __launch_bounds__(256) k_lut_pass(PassArgs a, RegionTable tbl)
{
    __shared__ SharedTable t;
    __shared__ float neff[kMaxRegions];
    if (threadIdx.x == 0) t.n = tbl.n;
    for (int k = threadIdx.x; k <= tbl.n; k += blockDim.x) t.ev_begin[k] = tbl.ev_begin[k];
    for (int k = threadIdx.x; k < tbl.n; k += blockDim.x) {
        t.grid[k] = tbl.grid[k];
        neff[k] = 0.f;
    }
    __syncthreads();
    const unsigned long long b =
        a.block_mul > 1 ? (unsigned long long)blockIdx.x * a.block_mul % gridDim.x : blockIdx.x;
    const long long i = (long long)b * blockDim.x + threadIdx.x;
    int r = 0;
    float w = 0.f;
    if (i < a.n) {
        if constexpr (Brick) w = do_event_lut_brick<Fmt, NS>(a, t, i, r);
        else w = do_event_lut<Kind, Fmt, NS>(a, t, i, a.lam_bf16 != nullptr, r);
    }
    if (Kind == PASS_FUSED) add_neff(neff, r, w);
    if (Kind == PASS_FUSED) {
        __syncthreads();
        for (int k = threadIdx.x; k < t.n; k += blockDim.x)
            if (neff[k] != 0.f) atomicAdd(a.partial + (blockIdx.x % kNeffSlots) * t.n + k, (double)neff[k]);
    }
}

template <int Kind, int Fmt>
cudaError_t launch_lut(const LaunchCfg& cfg, const PassArgs& a, const RegionTable& tbl, cudaStream_t s)
{
    if (a.lut.n < 1 || a.lut.n > kMaxLutSamples) return cudaErrorInvalidValue;
    const long long blocks = (a.n + cfg.threads - 1) / cfg.threads;
    if (blocks == 0) return cudaSuccess;
    if (a.brick_bx > 0) {
        // brick layout: fused pass over one grid with FP32 gathers only
        if (Kind != PASS_FUSED || tbl.n != 1 || a.lam_bf16 || tbl.grid[0].vox_offset != 0)
            return cudaErrorInvalidValue;
        if (a.lut.n == 32) k_lut_pass<PASS_FUSED, Fmt, 32, true><<<(unsigned)blocks, cfg.threads, 0, s>>>(a, tbl);
        else k_lut_pass<PASS_FUSED, Fmt, 0, true><<<(unsigned)blocks, cfg.threads, 0, s>>>(a, tbl);
        return cudaGetLastError();
    }
    if (a.lut.n == 32) k_lut_pass<Kind, Fmt, 32><<<(unsigned)blocks, cfg.threads, 0, s>>>(a, tbl);
    else if (a.lut.n == 15) k_lut_pass<Kind, Fmt, 15><<<(unsigned)blocks, cfg.threads, 0, s>>>(a, tbl);
    else k_lut_pass<Kind, Fmt, 0><<<(unsigned)blocks, cfg.threads, 0, s>>>(a, tbl);
    return cudaGetLastError();
}

constexpr int kMaxCacheBytes = 200 * 1024;

template <int Kind, int Fmt, bool Persistent, bool Cached, int TailK>
cudaError_t launch_variant(int blocks, const LaunchCfg& cfg, const PassArgs& a, const RegionTable& tbl,
                           cudaStream_t s)
{
    auto kern = k_event_pass<Kind, Fmt, Persistent, Cached, TailK>;
    size_t smem = 0;
    if (Cached) {
        smem = (size_t)cfg.cache * cfg.threads * 8;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, cfg.threads, smem, s>>>(a, tbl, cfg.chunk, cfg.cache);
    return cudaGetLastError();
}

template <int Kind, int Fmt, int TailK>
cudaError_t launch_tail(int blocks, const LaunchCfg& cfg, const PassArgs& a, const RegionTable& tbl, cudaStream_t s)
{
    const bool persistent = cfg.blocks_per_sm > 0;
    if (a.brick_bx > 0) {
        // brick layout: fused pass, FP32 gathers, flat grid, no piece cache; each grid's
        // voxel offset is its slab's offset in the brick copies
        if (Kind != PASS_FUSED || tbl.n < 1 || a.lam_bf16 || persistent || cfg.cache > 0)
            return cudaErrorInvalidValue;
        if constexpr (Kind == PASS_FUSED) {
            k_event_pass<PASS_FUSED, Fmt, false, false, TailK, true><<<blocks, cfg.threads, 0, s>>>(a, tbl, cfg.chunk,
                                                                                                   cfg.cache);
            return cudaGetLastError();
        }
    }
    if constexpr (Kind == PASS_FUSED) {
        if (cfg.cache > 0) {
            if (persistent) return launch_variant<Kind, Fmt, true, true, TailK>(blocks, cfg, a, tbl, s);
            return launch_variant<Kind, Fmt, false, true, TailK>(blocks, cfg, a, tbl, s);
        }
    }
    if (persistent) return launch_variant<Kind, Fmt, true, false, TailK>(blocks, cfg, a, tbl, s);
    return launch_variant<Kind, Fmt, false, false, TailK>(blocks, cfg, a, tbl, s);
}

template <int Kind, int Fmt>
cudaError_t launch_kind(const LaunchCfg& cfg, const PassArgs& a, const RegionTable& tbl, int num_sms,
                        cudaStream_t s)
{
    if (a.lut.n > 0) return launch_lut<Kind, Fmt>(cfg, a, tbl, s);
    const int blocks = pass_blocks(cfg, a.n, num_sms);
    if (blocks == 0) return cudaSuccess;
    if ((size_t)cfg.cache * cfg.threads * 8 > (size_t)kMaxCacheBytes) return cudaErrorInvalidValue;
    if (cfg.tail == TAIL_FIT) return launch_tail<Kind, Fmt, TAIL_FIT>(blocks, cfg, a, tbl, s);
    if (cfg.tail == TAIL_SERIES) return launch_tail<Kind, Fmt, TAIL_SERIES>(blocks, cfg, a, tbl, s);
    if (cfg.tail == TAIL_SERIES4) return launch_tail<Kind, Fmt, TAIL_SERIES4>(blocks, cfg, a, tbl, s);
    return launch_tail<Kind, Fmt, TAIL_ERFC>(blocks, cfg, a, tbl, s);
}

// Linear image -> brick copy (x fastest in the linear image).
__global__ void k_to_bricks(const float* __restrict__ lin, float* __restrict__ br, int nx, int ny, int nz, int bx,
                            int by)
{
    const long long n = (long long)nx * ny * nz;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(j % nx);
        const long long rest = j / nx;
        const int iy = (int)(rest % ny), iz = (int)(rest / ny);
        br[brick_index(ix, iy, iz, bx, by)] = lin[j];
    }
}

// lin += brick copy; the brick copy is cleared for the next pass.
__global__ void k_from_bricks_add(float* __restrict__ br, float* __restrict__ lin, int nx, int ny, int nz, int bx,
                                  int by)
{
    const long long n = (long long)nx * ny * nz;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(j % nx);
        const long long rest = j / nx;
        const int iy = (int)(rest % ny), iz = (int)(rest / ny);
        const int q = brick_index(ix, iy, iz, bx, by);
        lin[j] += br[q];
        br[q] = 0.f;
    }
}

unsigned brick_blocks(long long n)
{
    const long long b = (n + 255) / 256;
    return (unsigned)std::max(1LL, std::min(b, 148LL * 32));
}

}  // namespace

long long brick_voxels(int nx, int ny, int nz)
{
    return 8LL * ((nx + 1) / 2) * ((ny + 1) / 2) * ((nz + 1) / 2);
}

cudaError_t launch_to_bricks(const float* lin, float* br, int nx, int ny, int nz, cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    if (n <= 0) return cudaSuccess;
    k_to_bricks<<<brick_blocks(n), 256, 0, s>>>(lin, br, nx, ny, nz, (nx + 1) / 2, (ny + 1) / 2);
    return cudaGetLastError();
}

cudaError_t launch_from_bricks_add(float* br, float* lin, int nx, int ny, int nz, cudaStream_t s)
{
    const long long n = (long long)nx * ny * nz;
    if (n <= 0) return cudaSuccess;
    k_from_bricks_add<<<brick_blocks(n), 256, 0, s>>>(br, lin, nx, ny, nz, (nx + 1) / 2, (ny + 1) / 2);
    return cudaGetLastError();
}

int pass_blocks(const LaunchCfg& cfg, long long n, int num_sms)
{
    if (n <= 0) return 0;
    if (cfg.blocks_per_sm > 0) {
        long long want = (long long)num_sms * cfg.blocks_per_sm;
        long long warps_needed = (n + cfg.chunk - 1) / cfg.chunk;
        long long blocks_needed = (warps_needed + cfg.threads / 32 - 1) / (cfg.threads / 32);
        return (int)std::max(1LL, std::min(want, blocks_needed));
    }
    return (int)((n + cfg.threads - 1) / cfg.threads);
}

cudaError_t launch_pass(PassKind kind, EventFmt fmt, const LaunchCfg& cfg, const PassArgs& a,
                        const RegionTable& tbl, int num_sms, cudaStream_t s)
{
    if (fmt == FMT_F32) {
        if (kind == PASS_FUSED) return launch_kind<PASS_FUSED, FMT_F32>(cfg, a, tbl, num_sms, s);
        if (kind == PASS_FORWARD) return launch_kind<PASS_FORWARD, FMT_F32>(cfg, a, tbl, num_sms, s);
        return launch_kind<PASS_BACK, FMT_F32>(cfg, a, tbl, num_sms, s);
    }
    if (kind == PASS_FUSED) return launch_kind<PASS_FUSED, FMT_PACKED>(cfg, a, tbl, num_sms, s);
    if (kind == PASS_FORWARD) return launch_kind<PASS_FORWARD, FMT_PACKED>(cfg, a, tbl, num_sms, s);
    return launch_kind<PASS_BACK, FMT_PACKED>(cfg, a, tbl, num_sms, s);
}

// Out-of-range voxel indices the walks of this file skipped since the last call
// (bounds-checked build; 0 otherwise).
unsigned long long oob_count_event_pass() { return oob_take(); }

}  // namespace recon
