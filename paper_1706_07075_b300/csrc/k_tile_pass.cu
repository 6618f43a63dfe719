// Shared-memory tiled MLEM event pass (Sec. 2.4 with the TOF kernel of Sec.
// 2.3), for grids where an event's TOF window spans a few tens of voxels.
//
// Events are binned once by the cell of their TOF point c = M + d u (cells of
// CS^3 voxels).  Every event of a cell has its TOF window, clipped to the
// grid, inside the cell's tile: the cell widened by a halo of H_k voxels per
// axis, H_k >= K sigma max|u_k| / v_k (events that would leave the tile go to
// a fallback list processed by the global-memory pass).  One block per cell
// loads the tile of lambda into shared memory, zeroes a tile of C, runs the
// cell's events with gathers and reductions in shared memory only, and adds
// its C tile into the global C with one coalesced pass of reductions.  The
// scattered per-piece traffic, which bounds the global-memory pass at the L2,
// stays on the SM.
//
// Within a block each event is walked by 8 lanes: lane l takes the l-th of 8
// equal parts of the clipped window, walks its few Siddon pieces keeping
// (voxel, mass) in registers, the 8 partial sums of p_i meet by shuffles, and
// the backprojection replays the registers (no second walk, no second erfc).
// A voxel split between two lanes gets two partial masses whose sum is its
// mass.
#include <algorithm>
#include <type_traits>

#include "recon_device.cuh"

namespace recon {

namespace {

constexpr int kLanesPerEvent = 8;
constexpr int kTileThreads = 1024;
constexpr int kLanePieces = 12;   // pieces a lane keeps in registers (geometric bound checked on the host)
constexpr unsigned kCellNone = 0xFFFFFFFFu;      // window misses the grid: contributes nothing
constexpr unsigned kCellFallback = 0xFFFFFFFEu;  // window leaves its cell's tile: global-memory pass

template <int Fmt>
__device__ __forceinline__ Event load_ev(const void* ev, long long i, float lattice)
{
    if (Fmt == FMT_F32) return load_event_f32(static_cast<const float4*>(ev), i);
    return load_event_packed(static_cast<const int4*>(ev), i, lattice);
}

// Tile of cell (cx, cy, cz): voxel ranges [lo, hi) per axis, clipped to the grid.
__device__ __forceinline__ void tile_range(const TileH& t, int cx, int cy, int cz, int lo[3], int hi[3])
{
    const int c[3] = {cx, cy, cz};
    const int n[3] = {t.nx, t.ny, t.nz};
    const int h[3] = {t.hx, t.hy, t.hz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = max(0, c[k] * t.cs - h[k]);
        hi[k] = min(n[k], (c[k] + 1) * t.cs + h[k]);
    }
}

// Cell code of each event (kCellNone / kCellFallback / cell id) and per-cell counts.
template <int Fmt>
__global__ void k_cell_codes(const void* __restrict__ ev, long long n, float lattice, TileH t, float half_window,
                             unsigned* __restrict__ code, unsigned* __restrict__ counts,
                             unsigned* __restrict__ rank, unsigned long long* __restrict__ n_fallback)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Event e = load_ev<Fmt>(ev, i, lattice);
    Line ln;
    unsigned out = kCellNone;
    if (event_line(e, ln)) {
        const float cc[3] = {ln.c.x, ln.c.y, ln.c.z}, uu[3] = {ln.u.x, ln.u.y, ln.u.z};
        const float o[3] = {t.ox, t.oy, t.oz}, v[3] = {t.vx, t.vy, t.vz};
        const int nn[3] = {t.nx, t.ny, t.nz}, nc[3] = {t.ncx, t.ncy, t.ncz};
        bool miss = false, fits = true;
        int cell[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float glo = o[k], ghi = o[k] + (float)nn[k] * v[k];
            const float ext = half_window * fabsf(uu[k]);
            const float wlo = fmaxf(cc[k] - ext, glo), whi = fminf(cc[k] + ext, ghi);
            miss = miss || !(wlo <= whi);
            const float f = floorf((cc[k] - glo) / (v[k] * (float)t.cs));
            cell[k] = (int)fminf(fmaxf(f, 0.f), (float)(nc[k] - 1));
        }
        if (!miss) {
            int lo[3], hi[3];
            tile_range(t, cell[0], cell[1], cell[2], lo, hi);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float glo = o[k], ghi = o[k] + (float)nn[k] * v[k];
                const float ext = half_window * fabsf(uu[k]);
                const float wlo = fmaxf(cc[k] - ext, glo), whi = fminf(cc[k] + ext, ghi);
                // the part of the window inside the grid must stay inside the tile, with a
                // margin of 1/8 voxel where the tile ends before the grid does
                const float tlo = o[k] + (float)lo[k] * v[k], thi = o[k] + (float)hi[k] * v[k];
                const float m = 0.125f * v[k];
                if (lo[k] > 0 && !(wlo >= tlo + m)) fits = false;
                if (hi[k] < nn[k] && !(whi <= thi - m)) fits = false;
            }
            out = fits ? (unsigned)cell[0] + (unsigned)t.ncx * ((unsigned)cell[1] + (unsigned)t.ncy * (unsigned)cell[2])
                       : kCellFallback;
            if (fits && t.dir_az * t.dir_pol > 1) {
                // direction bin of the undirected line: u and -u are one line, so fold
                // to ux >= 0; azimuth over (-pi/2, pi/2], polar over uz in [-1, 1]
                const float sgn = uu[0] < 0.f ? -1.f : 1.f;
                const float ux = sgn * uu[0], uy = sgn * uu[1], uz = sgn * uu[2];
                const float az = atan2f(uy, ux) * 0.318309886f + 0.5f;            // [0, 1]
                const int ia = min(t.dir_az - 1, max(0, (int)(az * (float)t.dir_az)));
                const int ip = min(t.dir_pol - 1, max(0, (int)((uz + 1.f) * 0.5f * (float)t.dir_pol)));
                out = out * (unsigned)(t.dir_az * t.dir_pol) + (unsigned)(ia * t.dir_pol + ip);
            }
        }
    }
    if (out == kCellNone) out = t.none_code;   // kept in a last bucket, or left out
    code[i] = out;
    // the count before this event's increment is its place within its cell, so the
    // scatter needs no second atomic
    if (out < kCellFallback) rank[i] = atomicAdd(counts + out, 1u);
    else if (out == kCellFallback) atomicAdd(n_fallback, 1ull);
}

// ---------------------------------------------------------------- scan
// Exclusive scan of n unsigned counts into int64 offsets, three phases:
// per-block scans of kScanItems values, a scan of the block totals (one block,
// sequential chunks), then the block offsets added back.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanItems = kScanThreads * kScanPer;

__device__ __forceinline__ long long block_scan_excl(long long v, long long* sh, long long* total)
{
    // inclusive warp scan, then across warps
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    const long long before = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(const unsigned* __restrict__ in, long long n,
                                                              long long* __restrict__ out,
                                                              long long* __restrict__ block_sums)
{
    __shared__ long long sh[32];
    const long long base = (long long)blockIdx.x * kScanItems + (long long)threadIdx.x * kScanPer;
    long long v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < n ? (long long)in[base + k] : 0;
        s += v[k];
    }
    long long total;
    long long run = block_scan_excl(s, sh, &total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_totals(long long* __restrict__ sums, long long nb,
                                                              long long* __restrict__ grand)
{
    __shared__ long long sh[32];
    long long carry = 0;
    for (long long lo = 0; lo < nb; lo += kScanThreads) {
        const long long i = lo + threadIdx.x;
        const long long v = i < nb ? sums[i] : 0;
        long long total;
        const long long before = block_scan_excl(v, sh, &total);
        if (i < nb) sums[i] = carry + before;
        carry += total;
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(long long* __restrict__ out, long long n, const long long* __restrict__ sums)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / kScanItems];
}

// ------------------------------------------------------ list and scatter

// Cells with at least min_events events go to the list; the events of smaller
// cells (too few to pay for loading and flushing a tile) join the fallback:
// their count is zeroed, so their range in the scan is empty.
__global__ void k_cell_list(unsigned* __restrict__ counts, long long n_cells, unsigned min_events,
                            unsigned* __restrict__ list, unsigned* __restrict__ n_list,
                            unsigned long long* __restrict__ n_fallback)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    const unsigned k = counts[c];
    if (k == 0) return;
    if (k >= min_events) {
        list[atomicAdd(n_list, 1u)] = (unsigned)c;
    } else {
        counts[c] = 0;
        atomicAdd(n_fallback, (unsigned long long)k);
    }
}

template <int Fmt>
__global__ void k_cell_scatter(const void* __restrict__ ev, long long n, const unsigned* __restrict__ code,
                               const long long* __restrict__ begin, const unsigned* __restrict__ rank,
                               void* __restrict__ ev_cell, void* __restrict__ ev_fb,
                               unsigned long long* __restrict__ fb_cursor)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned c = code[i];
    long long pos;
    void* dst;
    if (c < kCellFallback && begin[c + 1] > begin[c]) {
        pos = begin[c] + rank[i];
        dst = ev_cell;
    } else if (c != kCellNone) {
        pos = (long long)atomicAdd(fb_cursor, 1ull);
        dst = ev_fb;
    } else {
        return;
    }
    if (Fmt == FMT_F32) {
        const float4* s = static_cast<const float4*>(ev) + 2 * i;
        float4* d = static_cast<float4*>(dst) + 2 * pos;
        d[0] = s[0];
        d[1] = s[1];
    } else {
        static_cast<int4*>(dst)[pos] = static_cast<const int4*>(ev)[i];
    }
}

// ------------------------------------------------------------ tiled pass

// Incremental form of `walk` (recon_device.cuh): one piece per call.
struct LaneWalk {
    int j;
    float mx, my, mz, tx, ty, tz, tau;
    Tail cur;
    bool done;
};

template <class TailF>
__device__ __forceinline__ void lw_init(LaneWalk& s, const Walk& w, const TailF& tail)
{
    s.done = !w.valid;
    s.j = w.j0;
    s.mx = s.my = s.mz = 0.f;
    s.tx = w.t0x;
    s.ty = w.t0y;
    s.tz = w.t0z;
    s.tau = w.tau_in;
    s.cur = tail(w.tau_in);
}

// Piece of the current voxel: index j and 2 [Phi(b) - Phi(a)]; then advance.
template <class TailF>
__device__ __forceinline__ void lw_step(LaneWalk& s, const Walk& w, const TailF& tail, int& j, float& a)
{
    const float inf = __int_as_float(0x7f800000);
    const float tmin = fminf(s.tx, fminf(s.ty, s.tz));
    const bool last = tmin >= w.tau_out;
    const float tn = fmaxf(fminf(tmin, w.tau_out), s.tau);
    const Tail nxt = tail(tn);
    a = (nxt.s - s.cur.s) + (s.cur.g - nxt.g);
    s.cur = nxt;
    j = s.j;
    s.done = last;
    s.tau = tn;
    const bool bx = s.tx == tmin;
    const bool by = !bx && s.ty == tmin;
    const bool bz = !bx && !by;
    s.j += bx ? w.sxl : (by ? w.syl : w.szl);
    s.mx += bx ? 1.f : 0.f;
    s.my += by ? 1.f : 0.f;
    s.mz += bz ? 1.f : 0.f;
    const float nx_ = s.mx < w.rx ? fmaf(s.mx, w.dtx, w.t0x) : inf;
    const float ny_ = s.my < w.ry ? fmaf(s.my, w.dty, w.t0y) : inf;
    const float nz_ = s.mz < w.rz ? fmaf(s.mz, w.dtz, w.t0z) : inf;
    s.tx = bx ? nx_ : s.tx;
    s.ty = by ? ny_ : s.ty;
    s.tz = bz ? nz_ : s.tz;
}

template <int Fmt, bool Fit, int Threads, int Lanes>
__global__ void __launch_bounds__(Threads, 1) k_tile_pass(PassArgs a, TileH t, const unsigned* __restrict__ list,
                                                          const long long* __restrict__ begin)
{
    extern __shared__ float smem[];
    __shared__ float neff_s;
    const unsigned cell = list[blockIdx.x];
    const int cx = (int)(cell % (unsigned)t.ncx);
    const int cy = (int)((cell / (unsigned)t.ncx) % (unsigned)t.ncy);
    const int cz = (int)(cell / ((unsigned)t.ncx * (unsigned)t.ncy));
    int lo[3], hi[3];
    tile_range(t, cx, cy, cz, lo, hi);
    const int Tx = hi[0] - lo[0], Ty = hi[1] - lo[1], Tz = hi[2] - lo[2];
    const int nt = Tx * Ty * Tz;
    float* lam_s = smem;
    float* C_s = smem + nt;
    // tile of lambda: one row (x run) per warp at a time, every copy asynchronous
    // (cp.async) so that all of them are in flight together
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = Threads / 32;
    for (int row = warp; row < Ty * Tz; row += kWarps) {
        const int y = row % Ty, z = row / Ty;
        const float* src = a.lam + (long long)lo[0] + (long long)t.nx * ((lo[1] + y) + (long long)t.ny * (lo[2] + z));
        float* dst = lam_s + row * Tx;
        for (int x = lane; x < Tx; x += 32) {
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst + x);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src + x) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int k = threadIdx.x; k < nt; k += Threads) C_s[k] = 0.f;
    if (threadIdx.x == 0) neff_s = 0.f;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();

    GridDev tg;
    tg.nx = Tx;
    tg.ny = Ty;
    tg.nz = Tz;
    tg.vx = t.vx;
    tg.vy = t.vy;
    tg.vz = t.vz;
    tg.ox = t.ox + (float)lo[0] * t.vx;
    tg.oy = t.oy + (float)lo[1] * t.vy;
    tg.oz = t.oz + (float)lo[2] * t.vz;
    tg.vox_offset = 0;
    using TailF = typename std::conditional<Fit, TailFit, TailErfc>::type;
    TailF tail;
    tail.inv_sigma_sqrt2 = a.tof.inv_sigma_sqrt2;
    const float hw = a.tof.half_window, hin = a.tof.half_inv_norm;
    const long long e0 = begin[cell], e1 = begin[cell + 1];
    float my_neff = 0.f;   // this thread's share of the block's N_eff

    if (Lanes == 1) {
        // one thread per event: forward sweep gathering from the lambda tile, backward
        // sweep reducing into the C tile
        for (long long i = e0 + threadIdx.x; i < e1; i += Threads) {
            const Event e = load_ev<Fmt>(a.events, i, a.lattice);
            Line ln;
            if (!event_line(e, ln)) continue;
            const Walk w = make_walk(tg, ln, -hw, hw);
            float p = 0.f;
            walk<true>(tg, a.tof, tail, w, [&](int j, float m) { p = fmaf(m, lam_s[j], p); });
            p *= hin;
            if (!(p > 0.f)) continue;
            const float r = e.w / p * hin;
            walk<true>(tg, a.tof, tail, w, [&](int j, float m) { atomicAdd(C_s + j, m * r); });
            my_neff += e.w;
        }
    }
    const int lane8 = threadIdx.x & (kLanesPerEvent - 1);
    const int group = threadIdx.x / kLanesPerEvent;
    constexpr int kGroups = Threads / kLanesPerEvent;

    for (long long base = e0; Lanes == kLanesPerEvent && base < e1; base += kGroups) {
        const long long i = base + group;
        const bool have = i < e1;
        Event e;
        e.w = 0.f;
        Walk w;
        w.valid = false;
        if (have) {
            e = load_ev<Fmt>(a.events, i, a.lattice);
            Line ln;
            if (event_line(e, ln)) {
                const Walk whole = make_walk(tg, ln, -hw, hw);
                if (whole.valid) {
                    const float T = whole.tau_out - whole.tau_in;
                    const float ta = whole.tau_in + T * (0.125f * (float)lane8);
                    const float tb = lane8 == kLanesPerEvent - 1 ? whole.tau_out
                                                                 : whole.tau_in + T * (0.125f * (float)(lane8 + 1));
                    if (ta < tb) w = make_walk(tg, ln, ta, tb);
                }
            }
        }
        // forward: this lane's pieces, kept in registers
        int js[kLanePieces];
        float ms[kLanePieces];
        int cnt = 0;
        float p = 0.f;
        LaneWalk s;
        s.done = true;
        if (w.valid) lw_init(s, w, tail);
#pragma unroll
        for (int q = 0; q < kLanePieces; ++q) {
            js[q] = 0;
            ms[q] = 0.f;
            if (!s.done) {
                int j;
                float m;
                lw_step(s, w, tail, j, m);
                js[q] = j;
                ms[q] = m;
                p = fmaf(m, lam_s[j], p);
                cnt = q + 1;
            }
        }
        const bool over = !s.done;
        for (int guard = Tx + Ty + Tz + 2; !s.done && guard > 0; --guard) {
            int j;
            float m;
            lw_step(s, w, tail, j, m);
            p = fmaf(m, lam_s[j], p);
        }
        // the 8 lanes of an event add their parts (xor butterfly: the same sum in every lane)
        p += __shfl_xor_sync(0xffffffffu, p, 1);
        p += __shfl_xor_sync(0xffffffffu, p, 2);
        p += __shfl_xor_sync(0xffffffffu, p, 4);
        p *= hin;
        if (have && p > 0.f) {
            const float r = e.w / p * hin;
#pragma unroll
            for (int q = 0; q < kLanePieces; ++q)
                if (q < cnt) atomicAdd(C_s + js[q], ms[q] * r);
            if (over) {
                // rare: more pieces than registers; walk again past the cached ones
                lw_init(s, w, tail);
                int q = 0;
                for (int guard = Tx + Ty + Tz + 2; !s.done && guard > 0; --guard, ++q) {
                    int j;
                    float m;
                    lw_step(s, w, tail, j, m);
                    if (q >= kLanePieces) atomicAdd(C_s + j, m * r);
                }
            }
            if (lane8 == 0) my_neff += e.w;
        }
    }
    // one shared atomic per warp for N_eff (every thread of the block gets here)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_neff += __shfl_xor_sync(0xffffffffu, my_neff, o);
    if (lane == 0 && my_neff != 0.f) atomicAdd(&neff_s, my_neff);
    __syncthreads();
    // C tile into the image: rows again, consecutive lanes on consecutive voxels
    for (int row = warp; row < Ty * Tz; row += kWarps) {
        const int y = row % Ty, z = row / Ty;
        float* dst = a.C + (long long)lo[0] + (long long)t.nx * ((lo[1] + y) + (long long)t.ny * (lo[2] + z));
        const float* src = C_s + row * Tx;
        for (int x = lane; x < Tx; x += 32) {
            const float v = src[x];
            if (v != 0.f) atomicAdd(dst + x, v);
        }
    }
    if (threadIdx.x == 0 && neff_s != 0.f) atomicAdd(a.partial + (blockIdx.x % kNeffSlots), (double)neff_s);
}

}  // namespace

cudaError_t launch_cell_codes(const void* ev, int fmt, long long n, float lattice, const TileH& t, float half_window,
                              unsigned* code, unsigned* counts, unsigned* rank, unsigned long long* n_fallback,
                              cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    if (fmt == FMT_F32)
        k_cell_codes<FMT_F32><<<(unsigned)blocks, 256, 0, st>>>(ev, n, lattice, t, half_window, code, counts, rank,
                                                               n_fallback);
    else
        k_cell_codes<FMT_PACKED><<<(unsigned)blocks, 256, 0, st>>>(ev, n, lattice, t, half_window, code, counts,
                                                                  rank, n_fallback);
    return cudaGetLastError();
}

long long scan_scratch_elems(long long n_cells) { return (n_cells + kScanItems - 1) / kScanItems + 1; }

cudaError_t launch_cell_scan(const unsigned* counts, long long n_cells, long long* begin, long long* block_sums,
                             cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    const long long nb = (n_cells + kScanItems - 1) / kScanItems;
    if (nb > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, st>>>(counts, n_cells, begin, block_sums);
    k_scan_totals<<<1, kScanThreads, 0, st>>>(block_sums, nb, begin + n_cells);
    k_scan_add<<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(begin, n_cells, block_sums);
    return cudaGetLastError();
}

cudaError_t launch_cell_list(unsigned* counts, long long n_cells, unsigned min_events, unsigned* list,
                             unsigned* n_list, unsigned long long* n_fallback, cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    k_cell_list<<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(counts, n_cells, min_events, list, n_list,
                                                                   n_fallback);
    return cudaGetLastError();
}

cudaError_t launch_cell_scatter(const void* ev, int fmt, long long n, const unsigned* code, const long long* begin,
                                const unsigned* rank, void* ev_cell, void* ev_fb, unsigned long long* fb_cursor,
                                cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    if (fmt == FMT_F32)
        k_cell_scatter<FMT_F32><<<(unsigned)blocks, 256, 0, st>>>(ev, n, code, begin, rank, ev_cell, ev_fb,
                                                                 fb_cursor);
    else
        k_cell_scatter<FMT_PACKED><<<(unsigned)blocks, 256, 0, st>>>(ev, n, code, begin, rank, ev_cell, ev_fb,
                                                                    fb_cursor);
    return cudaGetLastError();
}

size_t tile_smem_bytes(const TileH& t)
{
    const long long tx = std::min<long long>(t.nx, t.cs + 2LL * t.hx);
    const long long ty = std::min<long long>(t.ny, t.cs + 2LL * t.hy);
    const long long tz = std::min<long long>(t.nz, t.cs + 2LL * t.hz);
    return (size_t)(2 * tx * ty * tz) * sizeof(float);
}

template <int Fmt, bool Fit, int Threads, int Lanes>
cudaError_t launch_tile_variant(const PassArgs& a, const TileH& t, const unsigned* list, unsigned n_list,
                                const long long* begin, cudaStream_t st)
{
    auto kern = k_tile_pass<Fmt, Fit, Threads, Lanes>;
    const size_t smem = tile_smem_bytes(t);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<n_list, Threads, smem, st>>>(a, t, list, begin);
    return cudaGetLastError();
}

template <int Lanes>
cudaError_t launch_tile_lanes(const PassArgs& a, const TileH& t, const unsigned* list, unsigned n_list,
                              const long long* begin, bool fit, cudaStream_t st)
{
    if (a.lattice > 0.f) {
        if (fit) return launch_tile_variant<FMT_PACKED, true, kTileThreads, Lanes>(a, t, list, n_list, begin, st);
        return launch_tile_variant<FMT_PACKED, false, kTileThreads, Lanes>(a, t, list, n_list, begin, st);
    }
    if (fit) return launch_tile_variant<FMT_F32, true, kTileThreads, Lanes>(a, t, list, n_list, begin, st);
    return launch_tile_variant<FMT_F32, false, kTileThreads, Lanes>(a, t, list, n_list, begin, st);
}

cudaError_t launch_tile_pass(const PassArgs& a, const TileH& t, const unsigned* list, unsigned n_list,
                             const long long* begin, int tail, int lanes, cudaStream_t st)
{
    if (n_list == 0) return cudaSuccess;
    if (tile_smem_bytes(t) > 227 * 1024) return cudaErrorInvalidValue;
    const bool fit = tail == TAIL_FIT;
    if (lanes == 1) return launch_tile_lanes<1>(a, t, list, n_list, begin, fit, st);
    return launch_tile_lanes<kLanesPerEvent>(a, t, list, n_list, begin, fit, st);
}

// Out-of-range voxel indices the walks of this file skipped since the last call
// (bounds-checked build; 0 otherwise).
unsigned long long oob_count_tile_pass() { return oob_take(); }

}  // namespace recon
