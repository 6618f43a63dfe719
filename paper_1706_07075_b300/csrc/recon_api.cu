// C-ABI of librecon (include/recon.h): contexts, device-resident state,
// stream-ordered execution with per-iteration CUDA graphs, the launch
// autotuner and the region-divided reconstruction of Sec. 2.5.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "recon.h"
#include "recon_kernels.h"

using namespace recon;

namespace {

thread_local std::string g_create_error;

// A named NVTX range over a scope: entry points and their phases show up on a
// profiler's timeline (no cost beyond a test when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// Host-side fault injection (recon_debug_fail_alloc): when positive, the
// countdown-th device allocation from now on fails as if the device were out of
// memory.  Nothing is allocated for the failing request and no GPU work is done.
std::atomic<long long> g_fail_alloc_countdown{0};

// Grow b to at least `bytes`.  The new allocation is made before the old one is
// released, so a failed growth leaves b (and whatever it holds) as it was.
cudaError_t ensure(DevBuf& b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return cudaSuccess;
    if (g_fail_alloc_countdown.load() > 0 && g_fail_alloc_countdown.fetch_sub(1) == 1)
        return cudaErrorMemoryAllocation;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return e;
    if (b.p) cudaFree(b.p);
    b.p = p;
    b.bytes = bytes;
    return cudaSuccess;
}

void release(DevBuf& b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// Region division prepared for the batched reconstruction: the split, the
// slab layout and each region's start value, valid for one (events,
// sensitivity, division) combination.
struct RegionPrep {
    bool valid = false;
    long long ev_gen = -1, sens_gen = -1;
    std::vector<recon_region> regions;
    double margin = 0, shell = 0;
    int fmt = -1;
    std::vector<long long> off;   // region event offsets (R + 2 entries from the split)
    std::vector<int> lo, hi;      // slab slice ranges
    std::vector<long long> rv;    // slab voxel offsets (R + 1)
    std::vector<float> start;     // uniform start value per region
    int order = -1;               // event order the split read (context tile_mode)
};

// Cell binning of the resident events for the shared-memory tiled pass, valid
// for one (events, grid, kernel window) combination.
struct TilePrep {
    bool valid = false;
    long long ev_gen = -1;
    double half_window = 0;
    int min_events = 0;
    TileH th{};
    long long n_cells = 0;
    unsigned n_list = 0;
    long long n_fb = 0;
    long long n_binned = 0;
    int mode = 0;
    int subsets = 1;
    // cell codes, ranks and counts of the event order computed during a streamed
    // upload (stream_pass), for this event generation, cell geometry and window
    long long codes_gen = -1;
    TileH codes_th{};
    double codes_hw = 0;
    DevBuf code, counts, rank, begin, scratch, list, ev_cell, ev_fb, misc;
};

}  // namespace

struct recon_ctx {
    recon_geometry geom{};
    recon_grid grid{};
    double fwhm_ps = 0, sigma_mm = 0, k_sigma = 3.0;
    int lut_n = 0;   // samples of the sampled TOF kernel; 0: exact projector
    bool median = false;  // median-filter sieve after every iteration
    int subsets = 1;      // OSEM subsets of recon_mlem (1: MLEM)
    int start_mode = 0;   // 0: uniform start image, 1: starting backprojection
    int device = 0, num_sms = 148;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    cudaStream_t copy_stream = nullptr;            // host-to-device copies of the streamed first pass
    cudaEvent_t copied[2] = {nullptr, nullptr};    // staging half k holds chunk data
    cudaEvent_t drained[2] = {nullptr, nullptr};   // staging half k has been ingested
    cudaEvent_t ready = nullptr;                   // prior work on ctx->stream done
    std::string err;
    long long n_vox = 0;

    // whole-grid images
    DevBuf s64, s32, lam, C, lam_bf16;
    bool have_sens = false;
    double sens_total = 0;

    // resident events
    DevBuf ev, staging;
    int fmt = FMT_F32;
    long long n_ev = 0;
    double lattice = 0;
    bool have_ev = false;
    double w_total = 0;
    long long ev_generation = 0;

    // per-call scratch
    DevBuf pass_partial, upd_partial, work, iter, hist, reg_vox, red_partial, vec, med, mu, keep, counter;

    // options
    bool bf16 = false, timing = false, graphs = true, autotune = true;
    bool bricks = false;  // sampled pass of recon_mlem over 2x2x2-brick copies of lambda and C
    DevBuf lam_brick, C_brick;
    bool user_cfg = false;
    LaunchCfg cfg{192, 0, 0, 0, TAIL_SERIES};
    LaunchCfg last_cfg{192, 0, 0, 0, TAIL_SERIES};
    std::map<std::tuple<long long, int, long long, int>, LaunchCfg> tuned;
    // image layout the autotuner chose for recon_mlem per (events, format, voxels):
    // lanes 0 = the cell-ordered global-memory pass, 1 or 8 = the shared-memory tiled
    // pass with that many threads per event; with the launch it was timed with
    struct LayoutChoice {
        int lanes;
        LaunchCfg cfg;
    };
    std::map<std::tuple<long long, int, long long>, LayoutChoice> layout_tuned;
    int last_tiling = 0, last_lanes = 1;   // layout of the last event pass (recon_get_launch)
    recon_stats stats{};

    // per-iteration graph
    cudaGraphExec_t gexec = nullptr;
    std::string gkey;

    // region division
    DevBuf codes, counts, offsets, base, idx, ev_reg, lam_reg, C_reg, s_reg, bf16_reg, reg_vox_reg;
    RegionPrep region_prep;
    long long sens_generation = 0;

    // shared-memory tiled pass (plain MLEM with the exact projector)
    int region_first = 0, region_count = 0;  // recon_mlem_regions reconstructs this block (count 0: all)
    int tile_mode = 2;    // 0 load order, 1 shared-memory tiles, 2 cell order (default)
    int tile_min_events = 256;  // cells with fewer events take the global-memory pass
    int tile_lanes = 1;         // threads per event in the tiled pass (1 or 8)
    int order_cell = 4;         // cell edge (voxels) of the cell-ordered pass
    int order_dir_az = 16, order_dir_pol = 8;  // direction bins within a cell
    TilePrep tile_prep;
};

namespace {

recon_status fail(recon_ctx* c, recon_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

recon_status fail_cuda(recon_ctx* c, cudaError_t e, const char* what, int line)
{
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s (recon_api.cu:%d)", (int)e, cudaGetErrorString(e), what, line);
    cudaGetLastError();  // clear a sticky launch error where possible
    return fail(c, e == cudaErrorMemoryAllocation ? RECON_ENOMEM : RECON_ECUDA, buf);
}

#define CK(x)                                                        \
    do {                                                             \
        cudaError_t e_ = (x);                                        \
        if (e_ != cudaSuccess) return fail_cuda(ctx, e_, #x, __LINE__); \
    } while (0)

#define CHECK_CTX()                                           \
    do {                                                      \
        if (!ctx) return RECON_EINVAL;                        \
        ctx->err.clear();                                     \
        cudaError_t e0_ = cudaSetDevice(ctx->device);         \
        if (e0_ != cudaSuccess) return fail_cuda(ctx, e0_, "cudaSetDevice", __LINE__); \
    } while (0)

bool is_finite(double x) { return std::isfinite(x); }

TofH make_tof(const recon_ctx* c)
{
    TofH t;
    t.half_window = (float)(c->k_sigma * c->sigma_mm);
    t.inv_sigma_sqrt2 = (float)(1.0 / (c->sigma_mm * std::sqrt(2.0)));
    t.half_inv_norm = (float)(0.5 / std::erf(c->k_sigma / std::sqrt(2.0)));
    return t;
}

// Sampled TOF kernel (Sec. 2.3): offsets at the midpoints of lut_n equal
// intervals of [-K sigma, K sigma], weights exp(-t^2 / (2 sigma^2)) scaled to
// sum to one; offsets and weights computed in FP64, rounded once to FP32.
LutH make_lut(const recon_ctx* c)
{
    LutH l;
    memset(&l, 0, sizeof l);
    l.n = c->lut_n;
    if (l.n <= 0) return l;
    const double half = c->k_sigma * c->sigma_mm;
    const double step = 2.0 * half / l.n;
    double t[kMaxLutSamples], w[kMaxLutSamples], total = 0.0;
    for (int k = 0; k < l.n; ++k) {
        t[k] = -half + (k + 0.5) * step;
        const double z = t[k] / c->sigma_mm;
        w[k] = std::exp(-0.5 * z * z);
        total += w[k];
    }
    for (int k = 0; k < l.n; ++k) l.s[k] = make_float2((float)t[k], (float)(w[k] / total));
    return l;
}

GridH grid_h(const recon_grid& g, int z_lo = 0, int z_hi = -1, long long vox_offset = 0)
{
    if (z_hi < 0) z_hi = g.nz;
    GridH h;
    h.nx = g.nx;
    h.ny = g.ny;
    h.nz = z_hi - z_lo;
    h.vx = (float)g.vx;
    h.vy = (float)g.vy;
    h.vz = (float)g.vz;
    h.ox = (float)g.ox;
    h.oy = (float)g.oy;
    h.oz = (float)(g.oz + (double)z_lo * g.vz);
    h.vox_offset = vox_offset;
    return h;
}

int reduce_blocks(long long n) { return (int)std::max(1LL, std::min((n + 1023) / 1024, 592LL)); }

// Sum of `blocks` doubles left by a reduction kernel (synchronises the stream).
recon_status host_sum(recon_ctx* ctx, const double* dev, int blocks, double* out)
{
    std::vector<double> h(blocks);
    CK(cudaMemcpyAsync(h.data(), dev, sizeof(double) * blocks, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double s = 0;
    for (double v : h) s += v;
    *out = s;
    return RECON_OK;
}

void invalidate_graph(recon_ctx* ctx)
{
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    ctx->gkey.clear();
}

// Every device buffer a context owns (released by recon_destroy, counted by
// recon_get_info).
std::vector<DevBuf*> device_buffers(recon_ctx* ctx)
{
    return {&ctx->s64, &ctx->s32, &ctx->lam, &ctx->C, &ctx->lam_bf16, &ctx->lam_brick, &ctx->C_brick,
            &ctx->ev, &ctx->staging,
            &ctx->pass_partial, &ctx->upd_partial, &ctx->work, &ctx->iter, &ctx->hist, &ctx->reg_vox,
            &ctx->red_partial, &ctx->vec, &ctx->med, &ctx->mu, &ctx->keep, &ctx->counter, &ctx->codes,
            &ctx->counts, &ctx->offsets, &ctx->base, &ctx->idx,
            &ctx->ev_reg, &ctx->lam_reg, &ctx->C_reg, &ctx->s_reg, &ctx->bf16_reg, &ctx->reg_vox_reg,
            &ctx->tile_prep.code, &ctx->tile_prep.counts, &ctx->tile_prep.rank, &ctx->tile_prep.begin,
            &ctx->tile_prep.scratch, &ctx->tile_prep.list, &ctx->tile_prep.ev_cell, &ctx->tile_prep.ev_fb,
            &ctx->tile_prep.misc};
}

recon_status validate_events(recon_ctx* ctx, const recon_events* e)
{
    if (!e) return fail(ctx, RECON_EINVAL, "events is NULL");
    if (e->fmt != RECON_EV_F32_SOA && e->fmt != RECON_EV_PACKED_I16_F16)
        return fail(ctx, RECON_EINVAL, "unknown event format");
    if (e->n < 0) return fail(ctx, RECON_EINVAL, "event count is negative");
    if (e->n > (1LL << 34)) return fail(ctx, RECON_EINVAL, "event count too large");
    if (e->n > 0) {
        const int np = e->fmt == RECON_EV_F32_SOA ? 7 : 1;
        for (int k = 0; k < np; ++k)
            if (!e->planes[k]) return fail(ctx, RECON_EINVAL, "event plane pointer is NULL");
        if (e->fmt == RECON_EV_PACKED_I16_F16) {
            if (!(e->lattice_mm > 0) || !is_finite(e->lattice_mm)) return fail(ctx, RECON_EINVAL, "lattice_mm must be > 0");
            if (reinterpret_cast<uintptr_t>(e->planes[0]) % 16) return fail(ctx, RECON_EINVAL, "packed records must be 16-byte aligned");
        }
    }
    return RECON_OK;
}

// After the resident events (or their weights) change: new generation (drops
// graphs and cached region copies) and the weight total sum_i w_i.
recon_status events_changed_sum(recon_ctx* ctx);

// The resident events were rewritten: caches keyed on them go, and their total
// weight is summed again.  If that fails the context holds no events.
recon_status events_changed(recon_ctx* ctx)
{
    ctx->ev_generation++;
    invalidate_graph(ctx);
    recon_status s = events_changed_sum(ctx);
    if (s != RECON_OK) {
        ctx->have_ev = false;
        ctx->n_ev = 0;
        ctx->ev_generation++;
    }
    return s;
}

recon_status events_changed_sum(recon_ctx* ctx)
{
    ctx->w_total = 0;
    const long long n = ctx->n_ev;
    if (n > 0) {
        const bool packed = ctx->fmt == FMT_PACKED;
        const int b = reduce_blocks(n);
        CK(ensure(ctx->red_partial, sizeof(double) * 1024));
        CK(launch_reduce_weights(packed ? nullptr : ctx->ev.as<float4>(), packed ? ctx->ev.as<int4>() : nullptr, n,
                                 ctx->red_partial.as<double>(), b, ctx->stream));
        ctx->stats.kernel_launches += 1;
        recon_status s = host_sum(ctx, ctx->red_partial.as<double>(), b, &ctx->w_total);
        if (s != RECON_OK) return s;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return RECON_OK;
}

// Copy events into the resident layout (chunked through a staging buffer when
// they live on the host).
recon_status load_events(recon_ctx* ctx, const recon_events* e)
{
    recon_status s = validate_events(ctx, e);
    if (s != RECON_OK) return s;
    const long long n = e->n;
    const bool packed = e->fmt == RECON_EV_PACKED_I16_F16;
    const size_t rec = packed ? 16 : 32;
    // the resident events are replaced: until the new ones are in, the context holds none
    ctx->have_ev = false;
    ctx->n_ev = 0;
    ctx->ev_generation++;
    invalidate_graph(ctx);
    CK(ensure(ctx->ev, (size_t)n * rec));
    if (n > 0) {
        if (e->on_device) {
            if (packed)
                CK(launch_ingest_packed(static_cast<const int4*>(e->planes[0]), e->weight, n, ctx->ev.as<int4>(),
                                        ctx->stream));
            else
                CK(launch_ingest_f32(reinterpret_cast<const float* const*>(e->planes), e->weight, n,
                                     ctx->ev.as<float4>(), ctx->stream));
            ctx->stats.kernel_launches += 1;
        } else {
            const long long chunk = std::min(n, 1LL << 23);
            const size_t per = packed ? 16 + 4 : 8 * 4;
            CK(ensure(ctx->staging, (size_t)chunk * per));
            for (long long lo = 0; lo < n; lo += chunk) {
                const long long m = std::min(chunk, n - lo);
                if (packed) {
                    int4* st = ctx->staging.as<int4>();
                    float* wst = reinterpret_cast<float*>(st + chunk);
                    CK(cudaMemcpyAsync(st, static_cast<const int4*>(e->planes[0]) + lo, (size_t)m * 16,
                                       cudaMemcpyHostToDevice, ctx->stream));
                    if (e->weight)
                        CK(cudaMemcpyAsync(wst, e->weight + lo, (size_t)m * 4, cudaMemcpyHostToDevice, ctx->stream));
                    CK(launch_ingest_packed(st, e->weight ? wst : nullptr, m, ctx->ev.as<int4>() + lo, ctx->stream));
                } else {
                    float* st = ctx->staging.as<float>();
                    const float* pl[7];
                    for (int k = 0; k < 7; ++k) {
                        CK(cudaMemcpyAsync(st + (size_t)k * chunk, static_cast<const float*>(e->planes[k]) + lo,
                                           (size_t)m * 4, cudaMemcpyHostToDevice, ctx->stream));
                        pl[k] = st + (size_t)k * chunk;
                    }
                    float* wst = st + (size_t)7 * chunk;
                    if (e->weight)
                        CK(cudaMemcpyAsync(wst, e->weight + lo, (size_t)m * 4, cudaMemcpyHostToDevice, ctx->stream));
                    CK(launch_ingest_f32(pl, e->weight ? wst : nullptr, m, ctx->ev.as<float4>() + 2 * lo,
                                         ctx->stream));
                }
                ctx->stats.kernel_launches += 1;
            }
        }
    }
    ctx->fmt = packed ? FMT_PACKED : FMT_F32;
    ctx->lattice = packed ? e->lattice_mm : 0.0;
    ctx->n_ev = n;
    ctx->have_ev = true;
    return events_changed(ctx);   // drops the events again if their weights cannot be summed
}

recon_status finish_sensitivity(recon_ctx* ctx)
{
    const int b = reduce_blocks(ctx->n_vox);
    CK(ensure(ctx->red_partial, sizeof(double) * 1024));
    CK(launch_sens_finish(ctx->s64.as<double>(), ctx->n_vox, ctx->s32.as<float>(), ctx->red_partial.as<double>(), b,
                          ctx->stream));
    ctx->stats.kernel_launches += 1;
    recon_status s = host_sum(ctx, ctx->red_partial.as<double>(), b, &ctx->sens_total);
    if (s != RECON_OK) return s;
    ctx->have_sens = true;
    ctx->sens_generation++;
    invalidate_graph(ctx);
    return RECON_OK;
}

// The midpoint series for the piece masses holds its error bound (below 1e-7 of the
// window mass) for pieces up to ~0.4 sigma; a piece is at most a voxel diagonal long.
bool series_ok(const recon_ctx* c)
{
    const double diag = std::sqrt(c->grid.vx * c->grid.vx + c->grid.vy * c->grid.vy + c->grid.vz * c->grid.vz);
    return c->sigma_mm > 0 && diag <= 0.5 * c->sigma_mm;
}

// The series through h^4 drops He_6(m) h^6 / 322560, at most 96 h^6 / 322560 of a
// piece's mass (|He_6| <= 96 on [0, 3]): below 1.2e-6 for pieces up to 0.4 sigma.
bool series4_ok(const recon_ctx* c)
{
    const double diag = std::sqrt(c->grid.vx * c->grid.vx + c->grid.vy * c->grid.vy + c->grid.vz * c->grid.vz);
    return c->sigma_mm > 0 && diag <= 0.4 * c->sigma_mm && c->k_sigma <= 3.0;
}

LaunchCfg default_cfg(const recon_ctx* c)
{
    return series_ok(c) ? LaunchCfg{192, 0, 0, 0, TAIL_SERIES} : LaunchCfg{128, 0, 0, 0, TAIL_FIT};
}

bool valid_cfg(const recon_launch* c)
{
    if (!c) return false;
    if (c->threads_per_block < 32 || c->threads_per_block > 256 || c->threads_per_block % 32) return false;
    if (c->blocks_per_sm < 0 || c->blocks_per_sm > 32) return false;
    if (c->blocks_per_sm > 0 && (c->chunk_events < 32 || c->chunk_events % 32 || c->chunk_events > (1 << 20)))
        return false;
    if (c->cached_pieces != 0 && (c->cached_pieces < 8 || c->cached_pieces > 256)) return false;
    if ((long long)c->cached_pieces * c->threads_per_block * 8 > 200 * 1024) return false;
    if (c->tail_eval < TAIL_FIT || c->tail_eval > TAIL_SERIES4) return false;
    if (c->reduction != 0 && c->reduction != 1) return false;
    if (c->reduction == 1 && (c->blocks_per_sm != 0 || c->cached_pieces != 0)) return false;
    return true;
}

// The brick copies of a table's slabs (2x2x2 bricks per slab, slabs one after the
// other): bt is t with each grid's voxel offset replaced by its slab's offset in the
// copies; returns the brick voxels of all slabs.
long long brick_table(const RegionTable& t, RegionTable& bt)
{
    bt = t;
    long long off = 0;
    for (int r = 0; r < t.n; ++r) {
        bt.grid[r].vox_offset = off;
        off += brick_voxels(t.grid[r].nx, t.grid[r].ny, t.grid[r].nz);
    }
    return off;
}

// lambda of every slab into its brick copy, and the brick copies of C added into C.
cudaError_t to_bricks_all(const float* lin, float* br, const RegionTable& t, const RegionTable& bt, cudaStream_t s)
{
    for (int r = 0; r < t.n; ++r) {
        const cudaError_t e = launch_to_bricks(lin + t.grid[r].vox_offset, br + bt.grid[r].vox_offset, t.grid[r].nx,
                                               t.grid[r].ny, t.grid[r].nz, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t from_bricks_add_all(float* br, float* lin, const RegionTable& t, const RegionTable& bt, cudaStream_t s)
{
    for (int r = 0; r < t.n; ++r) {
        const cudaError_t e = launch_from_bricks_add(br + bt.grid[r].vox_offset, lin + t.grid[r].vox_offset,
                                                     t.grid[r].nx, t.grid[r].ny, t.grid[r].nz, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

RegionTable single_table(const recon_ctx* ctx)
{
    RegionTable t;
    memset(&t, 0, sizeof t);
    t.n = 1;
    t.ev_begin[0] = 0;
    t.ev_begin[1] = ctx->n_ev;
    t.grid[0] = grid_h(ctx->grid);
    return t;
}

PassArgs base_args(recon_ctx* ctx, const void* events, long long n)
{
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.events = events;
    a.n = n;
    a.lattice = (float)ctx->lattice;
    a.tof = make_tof(ctx);
    a.lut = make_lut(ctx);
    return a;
}

// Time one fused pass per candidate launch and keep the fastest.  The pass
// accumulates into C, which the caller clears afterwards; lambda is untouched.
// A multiplier coprime with the number of blocks, near 0.618 of it: block b of
// a flat grid then takes block (b * m) mod n of the event list, so blocks that
// run at the same time work on events far apart in the list (for region-ordered
// events: on different regions).  1 for tiny grids.
unsigned spread_multiplier(long long blocks)
{
    if (blocks < 16 || blocks > 0x7fffffffLL) return 1;
    auto gcd = [](unsigned long long x, unsigned long long y) {
        while (y) {
            const unsigned long long t = x % y;
            x = y;
            y = t;
        }
        return x;
    };
    unsigned long long m = (unsigned long long)(0.6180339887 * (double)blocks) | 1ULL;
    while (gcd(m, (unsigned long long)blocks) != 1) m += 2;
    return (unsigned)m;
}

recon_status autotune(recon_ctx* ctx, PassArgs a, const RegionTable& tbl, LaunchCfg* best)
{
    NvtxRange nvtx_range("autotune");
    // sampled projector: threads per block, and the linear image (x-pair vector
    // reductions) or the brick copies
    const std::vector<LaunchCfg> lut_cands = {
        {128, 0, 0, 0, TAIL_FIT, 0}, {192, 0, 0, 0, TAIL_FIT, 0}, {256, 0, 0, 0, TAIL_FIT, 0},
        {128, 0, 0, 0, TAIL_FIT, 1}, {192, 0, 0, 0, TAIL_FIT, 1}, {256, 0, 0, 0, TAIL_FIT, 1},
    };
    // exact projector: flat and persistent grids, walking twice or replaying a
    // shared-memory piece cache, piece-mass forms, reduction forms
    const std::vector<LaunchCfg> exact_cands = {
        {128, 0, 0, 0, TAIL_FIT}, {256, 0, 0, 0, TAIL_FIT}, {96, 0, 0, 0, TAIL_FIT},
        {192, 0, 0, 0, TAIL_FIT}, {128, 8, 64, 0, TAIL_FIT}, {64, 0, 0, 64, TAIL_FIT},
        {128, 0, 0, 0, TAIL_ERFC}, {256, 0, 0, 0, TAIL_ERFC}, {128, 0, 0, 0, TAIL_SERIES},
        {256, 0, 0, 0, TAIL_SERIES}, {192, 0, 0, 0, TAIL_SERIES},
        {128, 0, 0, 0, TAIL_SERIES4}, {192, 0, 0, 0, TAIL_SERIES4},
        // brick copies of lambda and C (a 2x2x2 brick per 32-byte sector)
        {128, 0, 0, 0, TAIL_SERIES4, 1}, {192, 0, 0, 0, TAIL_SERIES4, 1}, {256, 0, 0, 0, TAIL_SERIES4, 1},
        {128, 0, 0, 0, TAIL_SERIES, 1}, {192, 0, 0, 0, TAIL_SERIES, 1},
        {128, 0, 0, 0, TAIL_FIT, 1},
    };
    const std::vector<LaunchCfg>& cands = a.lut.n > 0 ? lut_cands : exact_cands;
    // the brick form needs FP32 gathers (and one grid for the sampled projector); its
    // candidates are timed with the copy kernels around the pass
    const bool brick_ok = !a.lam_bf16 && (tbl.n == 1 ? tbl.grid[0].vox_offset == 0 : a.lut.n == 0);
    RegionTable btbl;
    const long long nb = brick_table(tbl, btbl);
    if (brick_ok) {
        CK(ensure(ctx->lam_brick, sizeof(float) * (size_t)nb));
        CK(ensure(ctx->C_brick, sizeof(float) * (size_t)nb));
        CK(cudaMemsetAsync(ctx->C_brick.p, 0, sizeof(float) * (size_t)nb, ctx->stream));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    *best = default_cfg(ctx);
    CK(ensure(ctx->pass_partial, sizeof(double) * kNeffSlots * tbl.n));
    a.partial = ctx->pass_partial.as<double>();
    // block_mul == 1 marks a cell-ordered event list: each candidate spreads its own grid
    const bool spread = a.block_mul == 1;
    for (const LaunchCfg& c : cands) {
        // the persistent work queue takes events in list order, which a spread list must not
        if (spread && c.blocks_per_sm > 0) continue;
        if (a.lut.n == 0 && c.tail == TAIL_SERIES && !series_ok(ctx)) continue;
        if (a.lut.n == 0 && c.tail == TAIL_SERIES4 && !series4_ok(ctx)) continue;
        if (c.reduction == 1 && !brick_ok) continue;
        float ms_min = 1e30f;
        PassArgs ac = a;
        if (spread) ac.block_mul = spread_multiplier(pass_blocks(c, a.n, ctx->num_sms));
        PassArgs ab = ac;
        if (c.reduction == 1) {
            ab.lam = ctx->lam_brick.as<float>();
            ab.C = ctx->C_brick.as<float>();
            ab.brick_bx = (tbl.grid[0].nx + 1) / 2;
            ab.brick_by = (tbl.grid[0].ny + 1) / 2;
        }
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaMemsetAsync(ctx->work.p, 0, 8, ctx->stream));
            CK(cudaEventRecord(e0, ctx->stream));
            if (c.reduction == 1) CK(to_bricks_all(ac.lam, ctx->lam_brick.as<float>(), tbl, btbl, ctx->stream));
            CK(launch_pass(PASS_FUSED, (EventFmt)ctx->fmt, c, c.reduction == 1 ? ab : ac,
                           c.reduction == 1 ? btbl : tbl, ctx->num_sms, ctx->stream));
            if (c.reduction == 1) CK(from_bricks_add_all(ab.C, ac.C, tbl, btbl, ctx->stream));
            CK(cudaEventRecord(e1, ctx->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            ms_min = std::min(ms_min, ms);
            ctx->stats.kernel_launches += c.reduction == 1 ? 1 + 2 * tbl.n : 1;
        }
        if (ms_min < best_ms) {
            best_ms = ms_min;
            *best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->stats.autotune_runs += 1;
    return RECON_OK;
}

struct IterPlan {
    PassArgs a;
    RegionTable tbl;
    LaunchCfg cfg;
    float* lam;
    float* C;
    const float* s32;
    uint16_t* bf16;
    long long* reg_vox_dev;
    int n_regions;
    int upd_bpr;
    int pass_blocks;
    double* hist;
    int* iter;
    int hist_cap;
    float* med;      // median-filter output (nullptr: no sieve); copied back into lam
    long long med_vox;
    int max_nz;
    int subsets;     // OSEM subsets (1: MLEM); single-region plans only
    size_t rec_bytes;
    bool bricks = false;  // the sampled pass runs over the context's brick copies of lam and C
    // shared-memory tiled pass (single region, MLEM, exact projector)
    bool tiled = false;
    TileH th{};
    const unsigned* list = nullptr;
    unsigned n_list = 0;
    const long long* tbegin = nullptr;
    const void* ev_cell = nullptr;
    const void* ev_fb = nullptr;
    long long n_fb = 0;
    long long n_cell_events = 0;
    int tile_mode = 0;   // 1 shared-memory tiles, 2 cell-ordered global pass
    int lanes = 1;       // threads per event of the shared-memory tiled pass (1 or 8)
};

// The fused event pass of one (sub-)iteration: the tiled pass over the binned
// events plus the global-memory pass over the fallback events, or the
// global-memory pass alone.
recon_status launch_event_pass_layout(recon_ctx* ctx, const IterPlan& p, const PassArgs& a, const RegionTable& t)
{
    if (!p.tiled) {
        if (p.cfg.blocks_per_sm > 0) CK(cudaMemsetAsync(ctx->work.p, 0, 8, ctx->stream));
        CK(launch_pass(PASS_FUSED, (EventFmt)ctx->fmt, p.cfg, a, t, ctx->num_sms, ctx->stream));
        return RECON_OK;
    }
    PassArgs at = a;
    at.events = p.ev_cell;
    if (p.tile_mode == 2) {
        // cell-ordered events through the global-memory pass, cells spread over blocks;
        // an OSEM subset is the same block of the ordered copy (binned block by block)
        RegionTable tc = t;
        at.events = static_cast<const char*>(p.ev_cell) +
                    (static_cast<const char*>(a.events) - static_cast<const char*>(p.a.events));
        at.n = a.n;
        tc.ev_begin[1] = a.n;
        at.block_mul = spread_multiplier(pass_blocks(p.cfg, at.n, ctx->num_sms));
        if (p.cfg.blocks_per_sm > 0) CK(cudaMemsetAsync(ctx->work.p, 0, 8, ctx->stream));
        CK(launch_pass(PASS_FUSED, (EventFmt)ctx->fmt, p.cfg, at, tc, ctx->num_sms, ctx->stream));
    } else {
        CK(launch_tile_pass(at, p.th, p.list, p.n_list, p.tbegin, p.cfg.tail, p.lanes, ctx->stream));
    }
    if (p.n_fb > 0) {
        PassArgs af = a;
        af.events = p.ev_fb;
        af.n = p.n_fb;
        RegionTable tf = t;
        tf.ev_begin[1] = p.n_fb;
        if (p.cfg.blocks_per_sm > 0) CK(cudaMemsetAsync(ctx->work.p, 0, 8, ctx->stream));
        CK(launch_pass(PASS_FUSED, (EventFmt)ctx->fmt, p.cfg, af, tf, ctx->num_sms, ctx->stream));
    }
    return RECON_OK;
}

// The event pass in the image layout of the plan: with bricks, lambda is copied into
// the brick layout first (each region's slab into its own brick copy), the pass
// reduces into the brick copies of C, and those are added into C (and cleared)
// afterwards.
recon_status launch_event_pass(recon_ctx* ctx, const IterPlan& p, const PassArgs& a, const RegionTable& t)
{
    if (!p.bricks) return launch_event_pass_layout(ctx, p, a, t);
    RegionTable bt;
    brick_table(t, bt);
    CK(to_bricks_all(a.lam, ctx->lam_brick.as<float>(), t, bt, ctx->stream));
    PassArgs ab = a;
    ab.lam = ctx->lam_brick.as<float>();
    ab.C = ctx->C_brick.as<float>();
    ab.brick_bx = (t.grid[0].nx + 1) / 2;
    ab.brick_by = (t.grid[0].ny + 1) / 2;
    recon_status s = launch_event_pass_layout(ctx, p, ab, bt);
    if (s != RECON_OK) return s;
    CK(from_bricks_add_all(ctx->C_brick.as<float>(), a.C, t, bt, ctx->stream));
    return RECON_OK;
}

// Pass arguments of sub-iteration b: events of block b of the list.
void subset_args(const IterPlan& p, int b, PassArgs& a, RegionTable& t)
{
    a = p.a;
    t = p.tbl;
    if (p.subsets <= 1) return;
    const long long n = p.a.n, lo = b * n / p.subsets, hi = (b + 1) * n / p.subsets;
    a.events = static_cast<const char*>(p.a.events) + (size_t)lo * p.rec_bytes;
    a.n = hi - lo;
    t.ev_begin[1] = hi - lo;
}

// Sieve (Sec. 2.4): lam -> median -> lam, after the update.
recon_status enqueue_sieve(recon_ctx* ctx, const IterPlan& p)
{
    if (!p.med) return RECON_OK;
    CK(launch_median3(p.lam, p.med, p.s32, p.bf16, p.reg_vox_dev, p.n_regions, ctx->grid.nx, ctx->grid.ny, p.max_nz,
                      ctx->stream));
    CK(cudaMemcpyAsync(p.lam, p.med, sizeof(float) * (size_t)p.med_vox, cudaMemcpyDeviceToDevice, ctx->stream));
    return RECON_OK;
}

recon_status enqueue_iteration(recon_ctx* ctx, const IterPlan& p)
{
    for (int b = 0; b < p.subsets; ++b) {
        PassArgs a;
        RegionTable t;
        subset_args(p, b, a, t);
        recon_status sp = launch_event_pass(ctx, p, a, t);
        if (sp != RECON_OK) return sp;
        CK(launch_update(p.lam, p.C, p.s32, p.bf16, p.reg_vox_dev, p.n_regions, ctx->upd_partial.as<double>(),
                         p.upd_bpr, ctx->stream, (float)p.subsets));
        if (b == p.subsets - 1) {
            recon_status sv = enqueue_sieve(ctx, p);
            if (sv != RECON_OK) return sv;
        }
        CK(launch_finalize(p.a.partial, kNeffSlots, ctx->upd_partial.as<double>(), p.upd_bpr, p.n_regions, p.hist,
                           p.iter, p.hist_cap, ctx->stream));
    }
    return RECON_OK;
}

std::string plan_key(const recon_ctx* ctx, const IterPlan& p)
{
    char buf[512];
    snprintf(buf, sizeof buf, "%p %lld %d %d %d %d %d %p %p %p %p %p %d %d %d %p %p %d %p %lld %d %a %a %a",
             p.a.events, p.a.n, ctx->fmt, p.cfg.threads, p.cfg.blocks_per_sm, p.cfg.chunk, p.cfg.cache * 2 + p.cfg.tail, (void*)p.lam, (void*)p.C,
             (const void*)p.s32, (void*)p.bf16, (void*)p.reg_vox_dev, p.n_regions, p.upd_bpr, p.pass_blocks,
             (void*)p.hist, (void*)p.iter, p.hist_cap, (void*)ctx->stream, ctx->ev_generation, p.tbl.n,
             (double)p.a.tof.half_window, (double)p.a.tof.inv_sigma_sqrt2, (double)p.a.lattice);
    std::string k(buf);
    snprintf(buf, sizeof buf, " lut %d med %p %lld %d sub %d tile %d %d %p %u %p %p %lld %lld %d bm %u br %d %p %p",
             p.a.lut.n, (void*)p.med, p.med_vox, p.max_nz, p.subsets, (int)p.tiled, p.tile_mode, (const void*)p.list,
             p.n_list, p.ev_cell, p.ev_fb, p.n_fb, p.n_cell_events, p.lanes, p.a.block_mul, (int)p.bricks,
             ctx->lam_brick.p, ctx->C_brick.p);
    k += buf;
    for (int r = 0; r < p.tbl.n; ++r) {
        snprintf(buf, sizeof buf, "|%lld %d %a %lld", p.tbl.ev_begin[r + 1], p.tbl.grid[r].nz,
                 (double)p.tbl.grid[r].oz, p.tbl.grid[r].vox_offset);
        k += buf;
    }
    return k;
}

// Run n_iter iterations of the plan: graph replay, or direct launches (timing).
recon_status run_iterations(recon_ctx* ctx, const IterPlan& p, int n_iter, bool reset_counter = true)
{
    NvtxRange nvtx_range("iterations");
    if (reset_counter) CK(cudaMemsetAsync(p.iter, 0, sizeof(int), ctx->stream));
    if (n_iter == 0) return RECON_OK;
    const bool legacy = ctx->stream == nullptr || ctx->stream == cudaStreamLegacy || ctx->stream == cudaStreamPerThread;
    if (ctx->timing || !ctx->graphs || legacy) {
        std::vector<cudaEvent_t> evs;
        const int B = p.subsets;
        if (ctx->timing) {
            evs.resize(3 * (size_t)n_iter * B);
            for (auto& e : evs) CK(cudaEventCreate(&e));
        }
        for (int k = 0; k < n_iter; ++k) {
            for (int b = 0; b < B; ++b) {
                const size_t e = (size_t)k * B + b;
                PassArgs a;
                RegionTable t;
                subset_args(p, b, a, t);
                if (ctx->timing) CK(cudaEventRecord(evs[3 * e], ctx->stream));
                recon_status sp = launch_event_pass(ctx, p, a, t);
                if (sp != RECON_OK) return sp;
                if (ctx->timing) CK(cudaEventRecord(evs[3 * e + 1], ctx->stream));
                CK(launch_update(p.lam, p.C, p.s32, p.bf16, p.reg_vox_dev, p.n_regions,
                                 ctx->upd_partial.as<double>(), p.upd_bpr, ctx->stream, (float)B));
                if (b == B - 1) {
                    recon_status sv = enqueue_sieve(ctx, p);
                    if (sv != RECON_OK) return sv;
                }
                if (ctx->timing) CK(cudaEventRecord(evs[3 * e + 2], ctx->stream));
                CK(launch_finalize(p.a.partial, kNeffSlots, ctx->upd_partial.as<double>(), p.upd_bpr, p.n_regions,
                                   p.hist, p.iter, p.hist_cap, ctx->stream));
                ctx->stats.kernel_launches += (a.n > 0 ? 3 : 2) + (p.med && b == B - 1 ? 1 : 0) +
                                              (p.tiled && p.n_fb > 0 ? 1 : 0) + (p.bricks ? 2 * p.tbl.n : 0);
            }
        }
        if (ctx->timing) {
            CK(cudaStreamSynchronize(ctx->stream));
            for (size_t e = 0; e < (size_t)n_iter * B; ++e) {
                float a = 0, b = 0;
                CK(cudaEventElapsedTime(&a, evs[3 * e], evs[3 * e + 1]));
                CK(cudaEventElapsedTime(&b, evs[3 * e + 1], evs[3 * e + 2]));
                ctx->stats.pass_ms += a;
                ctx->stats.update_ms += b;
                ctx->stats.pass_launches += 1;
            }
            for (auto& e : evs) cudaEventDestroy(e);
        }
        return RECON_OK;
    }
    const std::string key = plan_key(ctx, p);
    if (!ctx->gexec || key != ctx->gkey) {
        invalidate_graph(ctx);
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        recon_status s = enqueue_iteration(ctx, p);
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(ctx->stream, &g);
        if (s != RECON_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (ee != cudaSuccess) return fail_cuda(ctx, ee, "cudaStreamEndCapture", __LINE__);
        cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            ctx->gexec = nullptr;
            return fail_cuda(ctx, ei, "cudaGraphInstantiate", __LINE__);
        }
        ctx->gkey = key;
    }
    for (int k = 0; k < n_iter; ++k) {
        CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
        ctx->stats.kernel_launches += (long long)p.subsets * ((p.pass_blocks > 0 ? 3 : 2) + (p.bricks ? 2 * p.tbl.n : 0)) +
                                      (p.med ? 1 : 0) + (p.tiled && p.n_fb > 0 ? 1 : 0);
    }
    return RECON_OK;
}

// Autotuner cache key: event count, format, voxels, and in the last field the
// number of regions, whether the list is spread-ordered (cell- or region-ordered lists
// are tuned apart from lists in load order) and the sampled projector's sample count.
std::tuple<long long, int, long long, int> tune_key(const recon_ctx* ctx, const PassArgs& a, const RegionTable& tbl)
{
    return std::make_tuple(a.n, ctx->fmt, ctx->n_vox, tbl.n + (a.block_mul == 1 ? (1 << 20) : 0) + (a.lut.n << 22));
}

// The launch choose_cfg would pick, without running the autotuner.
LaunchCfg tuned_or_default(recon_ctx* ctx, const PassArgs& a, const RegionTable& tbl)
{
    if (ctx->user_cfg) return ctx->cfg;
    if (!ctx->autotune || a.n < (1LL << 20)) return default_cfg(ctx);
    auto it = ctx->tuned.find(tune_key(ctx, a, tbl));
    return it != ctx->tuned.end() ? it->second : default_cfg(ctx);
}

LaunchCfg choose_cfg(recon_ctx* ctx, const PassArgs& a, const RegionTable& tbl, recon_status* st)
{
    *st = RECON_OK;
    if (ctx->user_cfg) return ctx->cfg;
    if (!ctx->autotune || a.n < (1LL << 20)) return default_cfg(ctx);
    auto key = tune_key(ctx, a, tbl);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) return it->second;
    LaunchCfg best;
    *st = autotune(ctx, a, tbl, &best);
    if (*st != RECON_OK) return default_cfg(ctx);
    ctx->tuned[key] = best;
    return best;
}

recon_status validate_regions(recon_ctx* ctx, int R, const recon_region* regions, double margin_mm, double shell_mm)
{
    if (R < 1 || R > kMaxRegions) return fail(ctx, RECON_EINVAL, "n_regions must be in [1, 64]");
    if (!regions) return fail(ctx, RECON_EINVAL, "regions is NULL");
    if (!(margin_mm >= 0) || !is_finite(margin_mm)) return fail(ctx, RECON_EINVAL, "margin_mm must be >= 0");
    if (!(shell_mm >= 0) || !is_finite(shell_mm)) return fail(ctx, RECON_EINVAL, "shell_mm must be >= 0");
    for (int r = 0; r < R; ++r) {
        const recon_region& g = regions[r];
        if (g.z_lo < 0 || g.z_hi > ctx->grid.nz || g.z_lo >= g.z_hi)
            return fail(ctx, RECON_EINVAL, "region slice range outside the grid or empty");
        if (r + 1 < R && regions[r + 1].z_lo != g.z_hi) return fail(ctx, RECON_EINVAL, "regions must be consecutive");
        if ((double)(g.z_hi - g.z_lo) * ctx->grid.vz < 2.0 * shell_mm)
            return fail(ctx, RECON_EINVAL, "region core thinner than 2 * shell_mm");
    }
    return RECON_OK;
}

// Split the resident events; leaves codes, idx and offsets (host copy in
// h_offsets, R+2 entries) in the context.
recon_status split_internal(recon_ctx* ctx, int R, const recon_region* regions, double shell_mm,
                            std::vector<long long>& h_offsets, const void* ev = nullptr, long long n_ev = -1)
{
    if (!ev) ev = ctx->ev.p;
    const long long n = n_ev >= 0 ? n_ev : ctx->n_ev;
    if (n >= (1LL << 31)) return fail(ctx, RECON_EINVAL, "region division takes fewer than 2^31 events");
    std::vector<double> zb(R + 1);
    for (int r = 0; r < R; ++r) zb[r] = ctx->grid.oz + (double)regions[r].z_lo * ctx->grid.vz;
    zb[R] = ctx->grid.oz + (double)regions[R - 1].z_hi * ctx->grid.vz;
    const int tile = 4096;
    const long long tiles = std::max(1LL, (n + tile - 1) / tile);
    CK(ensure(ctx->codes, (size_t)n));
    CK(ensure(ctx->counts, sizeof(int) * (size_t)tiles * (R + 1)));
    CK(ensure(ctx->offsets, sizeof(long long) * (R + 2)));
    CK(ensure(ctx->base, sizeof(long long) * (size_t)tiles * R));
    CK(cudaMemsetAsync(ctx->counts.p, 0, sizeof(int) * (size_t)tiles * (R + 1), ctx->stream));
    const bool packed = ctx->fmt == FMT_PACKED;
    CK(launch_region_codes(packed ? nullptr : static_cast<const float4*>(ev), packed ? static_cast<const int4*>(ev)
                                                                                    : nullptr,
                           ctx->lattice, n, zb.data(), R, shell_mm, ctx->codes.as<uint8_t>(), ctx->counts.as<int>(),
                           tile, ctx->stream));
    CK(launch_region_scan(ctx->counts.as<int>(), (int)tiles, R, ctx->offsets.as<long long>(),
                          ctx->base.as<long long>(), ctx->stream));
    ctx->stats.kernel_launches += n > 0 ? 2 : 1;
    h_offsets.assign(R + 2, 0);
    CK(cudaMemcpyAsync(h_offsets.data(), ctx->offsets.p, sizeof(long long) * (R + 2), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h_offsets[R + 1] != 0) return fail(ctx, RECON_EINVAL, "events fall in three or more regions");
    CK(ensure(ctx->idx, sizeof(int) * (size_t)std::max(1LL, h_offsets[R])));
    CK(launch_region_scatter(ctx->codes.as<uint8_t>(), n, R, ctx->base.as<long long>(), tile, ctx->idx.as<int>(),
                             ctx->stream));
    if (n > 0) ctx->stats.kernel_launches += 1;
    return RECON_OK;
}

void slab_ranges(const recon_ctx* ctx, int R, const recon_region* regions, double margin_mm, std::vector<int>& lo,
                 std::vector<int>& hi)
{
    const int m = (int)std::ceil(margin_mm / ctx->grid.vz - 1e-12);
    lo.resize(R);
    hi.resize(R);
    for (int r = 0; r < R; ++r) {
        lo[r] = std::max(0, regions[r].z_lo - m);
        hi[r] = std::min(ctx->grid.nz, regions[r].z_hi + m);
    }
}

}  // namespace

// ======================================================================= API

extern "C" {

recon_status recon_create(const recon_geometry* geom, const recon_grid* grid, double tof_fwhm_ps, recon_ctx** out)
{
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return RECON_EINVAL;
    }
    *out = nullptr;
    if (!geom || !grid) {
        g_create_error = "geometry or grid is NULL";
        return RECON_EINVAL;
    }
    if (!(geom->radius_mm > 0) || !(geom->axial_len_mm > 0) || !is_finite(geom->radius_mm) ||
        !is_finite(geom->axial_len_mm) || !(geom->max_axial_angle_deg > 0) || !(geom->max_axial_angle_deg <= 90)) {
        g_create_error = "invalid geometry";
        return RECON_EINVAL;
    }
    if (grid->nx <= 0 || grid->ny <= 0 || grid->nz <= 0 || !(grid->vx > 0) || !(grid->vy > 0) || !(grid->vz > 0) ||
        !is_finite(grid->vx) || !is_finite(grid->vy) || !is_finite(grid->vz) || !is_finite(grid->ox) || !is_finite(grid->oy) ||
        !is_finite(grid->oz)) {
        g_create_error = "invalid grid";
        return RECON_EINVAL;
    }
    const long long nv = (long long)grid->nx * grid->ny * grid->nz;
    if (nv >= (1LL << 31) - 1) {
        g_create_error = "grid has 2^31 voxels or more";
        return RECON_EINVAL;
    }
    if (!(tof_fwhm_ps > 0) || !is_finite(tof_fwhm_ps)) {
        g_create_error = "tof_fwhm_ps must be > 0";
        return RECON_EINVAL;
    }
    recon_ctx* ctx = new (std::nothrow) recon_ctx();
    if (!ctx) {
        g_create_error = "out of host memory";
        return RECON_ENOMEM;
    }
    ctx->geom = *geom;
    ctx->grid = *grid;
    ctx->fwhm_ps = tof_fwhm_ps;
    // sigma along the LOR: d = c (t2 - t1)/2, FWHM = 2 sqrt(2 ln 2) sigma
    ctx->sigma_mm = 0.5 * 0.299792458 * tof_fwhm_ps / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    ctx->n_vox = nv;
    auto bail = [&](cudaError_t e, const char* what) {
        char buf[256];
        snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
        g_create_error = buf;
        recon_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? RECON_ENOMEM : RECON_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&ctx->device)) != cudaSuccess) return bail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess)
        return bail(e, "cudaDeviceGetAttribute");
    if ((e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(e, "cudaStreamCreateWithFlags");
    ctx->stream = ctx->own_stream;
    if ((e = ensure(ctx->s64, sizeof(double) * nv)) != cudaSuccess) return bail(e, "allocating s");
    if ((e = ensure(ctx->s32, sizeof(float) * nv)) != cudaSuccess) return bail(e, "allocating s");
    if ((e = ensure(ctx->lam, sizeof(float) * nv)) != cudaSuccess) return bail(e, "allocating lambda");
    if ((e = ensure(ctx->C, sizeof(float) * nv)) != cudaSuccess) return bail(e, "allocating C");
    if ((e = ensure(ctx->work, 64)) != cudaSuccess) return bail(e, "allocating work counter");
    if ((e = ensure(ctx->iter, 64)) != cudaSuccess) return bail(e, "allocating iteration counter");
    if ((e = cudaMemsetAsync(ctx->s64.p, 0, sizeof(double) * nv, ctx->stream)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(ctx->s32.p, 0, sizeof(float) * nv, ctx->stream)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(ctx->lam.p, 0, sizeof(float) * nv, ctx->stream)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(ctx->C.p, 0, sizeof(float) * nv, ctx->stream)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) return bail(e, "cudaStreamSynchronize");
    *out = ctx;
    return RECON_OK;
}

void recon_destroy(recon_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    invalidate_graph(ctx);
    for (DevBuf* b : device_buffers(ctx)) release(*b);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (int k = 0; k < 2; ++k) {
        if (ctx->copied[k]) cudaEventDestroy(ctx->copied[k]);
        if (ctx->drained[k]) cudaEventDestroy(ctx->drained[k]);
    }
    if (ctx->ready) cudaEventDestroy(ctx->ready);
    delete ctx;
}

const char* recon_last_error(const recon_ctx* ctx)
{
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

}  // extern "C"

namespace recon {
// Message reported by recon_last_error(NULL) for calls that have no context.
void set_thread_error(const std::string& msg) { g_create_error = msg; }
}  // namespace recon

extern "C" {

recon_status recon_set_stream(recon_ctx* ctx, void* cuda_stream)
{
    CHECK_CTX();
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->own_stream;
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_set_kernel_window(recon_ctx* ctx, double k_sigma)
{
    CHECK_CTX();
    if (!(k_sigma >= 0.5 && k_sigma <= 8.0)) return fail(ctx, RECON_EINVAL, "k_sigma must be in [0.5, 8]");
    ctx->k_sigma = k_sigma;
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_set_projector(recon_ctx* ctx, int32_t projector, int32_t n_samples)
{
    CHECK_CTX();
    if (projector == RECON_PROJ_EXACT) {
        ctx->lut_n = 0;
    } else if (projector == RECON_PROJ_SAMPLED) {
        if (n_samples < 1 || n_samples > RECON_MAX_TOF_SAMPLES)
            return fail(ctx, RECON_EINVAL, "n_samples must be in [1, RECON_MAX_TOF_SAMPLES]");
        ctx->lut_n = n_samples;
    } else {
        return fail(ctx, RECON_EINVAL, "unknown projector");
    }
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_set_start_image(recon_ctx* ctx, int32_t mode)
{
    CHECK_CTX();
    if (mode != 0 && mode != 1) return fail(ctx, RECON_EINVAL, "mode must be 0 or 1");
    ctx->start_mode = mode;
    return RECON_OK;
}

recon_status recon_set_subsets(recon_ctx* ctx, int32_t n_subsets)
{
    CHECK_CTX();
    if (n_subsets < 1 || n_subsets > 1024) return fail(ctx, RECON_EINVAL, "n_subsets must be in [1, 1024]");
    ctx->subsets = n_subsets;
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_set_event_order(recon_ctx* ctx, int32_t order, int32_t azimuth_bins, int32_t polar_bins)
{
    CHECK_CTX();
    if (order < -1 || order > 64) return fail(ctx, RECON_EINVAL, "order must be in [-1, 64]");
    if (azimuth_bins < 1 || azimuth_bins > 64 || polar_bins < 1 || polar_bins > 64)
        return fail(ctx, RECON_EINVAL, "direction bins must be in [1, 64]");
    ctx->order_dir_az = azimuth_bins;
    ctx->order_dir_pol = polar_bins;
    ctx->tile_mode = order != 0 ? 2 : 0;
    ctx->order_cell = order > 0 ? order : 4;
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_set_tiled_pass(recon_ctx* ctx, int32_t on, int32_t lanes)
{
    CHECK_CTX();
    if (on < 0) return fail(ctx, RECON_EINVAL, "on must be >= 0");
    if (lanes != 1 && lanes != 8) return fail(ctx, RECON_EINVAL, "lanes must be 1 or 8");
    ctx->tile_mode = on != 0 ? 1 : 2;
    ctx->tile_min_events = on > 1 ? on : 256;
    ctx->tile_lanes = lanes == 8 ? 8 : 1;
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_set_median_filter(recon_ctx* ctx, int32_t on)
{
    CHECK_CTX();
    ctx->median = on != 0;
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_median_filter(recon_ctx* ctx, const float* image_in, float* image_out)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_median_filter");
    if (!image_in || !image_out) return fail(ctx, RECON_EINVAL, "image_in and image_out are required");
    const size_t bytes = sizeof(float) * (size_t)ctx->n_vox;
    // staged through context scratch (vec: input, med: output), so in and out may alias
    CK(ensure(ctx->med, bytes));
    CK(ensure(ctx->vec, bytes));
    CK(cudaMemcpyAsync(ctx->vec.p, image_in, bytes, cudaMemcpyDefault, ctx->stream));
    const long long rv[2] = {0, ctx->n_vox};
    CK(ensure(ctx->reg_vox, sizeof rv));
    CK(cudaMemcpyAsync(ctx->reg_vox.p, rv, sizeof rv, cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_median3(ctx->vec.as<float>(), ctx->med.as<float>(), nullptr, nullptr, ctx->reg_vox.as<long long>(), 1,
                      ctx->grid.nx, ctx->grid.ny, ctx->grid.nz, ctx->stream));
    CK(cudaMemcpyAsync(image_out, ctx->med.p, bytes, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->stats.kernel_launches += 1;
    return RECON_OK;
}

recon_status recon_get_tof_samples(const recon_ctx* ctx, int32_t capacity, float* offsets_mm, float* weights,
                                   int32_t* n_out)
{
    if (!ctx || !n_out) return RECON_EINVAL;
    const LutH l = make_lut(ctx);
    *n_out = l.n;
    if (l.n > capacity) return RECON_EINVAL;
    for (int k = 0; k < l.n; ++k) {
        if (offsets_mm) offsets_mm[k] = l.s[k].x;
        if (weights) weights[k] = l.s[k].y;
    }
    return RECON_OK;
}

recon_status recon_set_gather_bf16(recon_ctx* ctx, int32_t on)
{
    CHECK_CTX();
    if (on != 0) CK(ensure(ctx->lam_bf16, sizeof(uint16_t) * ctx->n_vox));
    ctx->bf16 = on != 0;
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_set_brick_layout(recon_ctx* ctx, int32_t on)
{
    CHECK_CTX();
    if (on != 0 && on != 1) return fail(ctx, RECON_EINVAL, "on must be 0 or 1");
    if (on && brick_voxels(ctx->grid.nx, ctx->grid.ny, ctx->grid.nz) > 0x7fffffffLL)
        return fail(ctx, RECON_EINVAL, "grid too large for the brick layout (2^31 voxels)");
    ctx->bricks = on != 0;
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_set_launch(recon_ctx* ctx, const recon_launch* cfg)
{
    CHECK_CTX();
    if (!cfg) {
        ctx->user_cfg = false;
        return RECON_OK;
    }
    if (!valid_cfg(cfg)) return fail(ctx, RECON_EINVAL, "invalid launch configuration");
    ctx->user_cfg = true;
    ctx->cfg = LaunchCfg{cfg->threads_per_block, cfg->blocks_per_sm, cfg->blocks_per_sm > 0 ? cfg->chunk_events : 0,
                         cfg->cached_pieces, cfg->tail_eval, cfg->reduction};
    return RECON_OK;
}

recon_status recon_get_launch(const recon_ctx* ctx, recon_launch* out)
{
    if (!ctx || !out) return RECON_EINVAL;
    out->threads_per_block = ctx->last_cfg.threads;
    out->blocks_per_sm = ctx->last_cfg.blocks_per_sm;
    out->chunk_events = ctx->last_cfg.chunk;
    out->cached_pieces = ctx->last_cfg.cache;
    out->tail_eval = ctx->last_cfg.tail;
    out->reduction = ctx->last_cfg.reduction;
    out->image_tiling = ctx->last_tiling;
    out->lanes_per_event = ctx->last_lanes;
    return RECON_OK;
}

recon_status recon_set_timing(recon_ctx* ctx, int32_t on)
{
    CHECK_CTX();
    ctx->timing = on != 0;
    return RECON_OK;
}

recon_status recon_set_graphs(recon_ctx* ctx, int32_t on)
{
    CHECK_CTX();
    ctx->graphs = on != 0;
    return RECON_OK;
}

recon_status recon_debug_bounds_violations(int64_t* count_out)
{
    if (!count_out) return RECON_EINVAL;
#ifdef RECON_BOUNDS_CHECK
    const unsigned long long c =
        oob_count_event_pass() + oob_count_tile_pass() + oob_count_preprocess() + oob_count_image();
    *count_out = (int64_t)c;
#else
    *count_out = -1;
#endif
    return RECON_OK;
}

recon_status recon_debug_fail_alloc(int64_t n)
{
    if (n < 0) return RECON_EINVAL;
    g_fail_alloc_countdown.store(n);
    return RECON_OK;
}

recon_status recon_set_autotune(recon_ctx* ctx, int32_t on)
{
    CHECK_CTX();
    ctx->autotune = on != 0;
    return RECON_OK;
}

recon_status recon_get_info(const recon_ctx* ctx, recon_info* out)
{
    if (ctx && out) {
        long long bytes = 0;
        for (DevBuf* b : device_buffers(const_cast<recon_ctx*>(ctx))) bytes += (long long)b->bytes;
        out->device_bytes = bytes;
    }
    if (!ctx || !out) return RECON_EINVAL;
    out->sigma_mm = ctx->sigma_mm;
    out->k_sigma = ctx->k_sigma;
    out->n_vox = ctx->n_vox;
    out->n_events_resident = ctx->have_ev ? ctx->n_ev : 0;
    out->has_sensitivity = ctx->have_sens ? 1 : 0;
    out->num_sms = ctx->num_sms;
    out->sens_total = ctx->sens_total;
    const TilePrep& tp = ctx->tile_prep;
    const bool tv = tp.valid && tp.ev_gen == ctx->ev_generation;
    out->tile_cells = tv ? (int64_t)tp.n_list : 0;
    out->tile_events = tv ? ctx->n_ev - tp.n_fb : 0;
    out->tile_fallback_events = tv ? tp.n_fb : 0;
    out->tile_cell_voxels = tv ? tp.th.cs : 0;
    out->tile_halo[0] = tv ? tp.th.hx : 0;
    out->tile_halo[1] = tv ? tp.th.hy : 0;
    out->tile_halo[2] = tv ? tp.th.hz : 0;
    out->subsets = ctx->subsets;
    out->lut_samples = ctx->lut_n;
    return RECON_OK;
}

recon_status recon_get_stats(const recon_ctx* ctx, recon_stats* out)
{
    if (!ctx || !out) return RECON_EINVAL;
    *out = ctx->stats;
    return RECON_OK;
}

recon_status recon_reset_stats(recon_ctx* ctx)
{
    if (!ctx) return RECON_EINVAL;
    ctx->stats = recon_stats{};
    return RECON_OK;
}

recon_status recon_sensitivity(recon_ctx* ctx, const float* lor, int64_t n, int32_t on_device, double* sens_out)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_sensitivity");
    if (n < 0) return fail(ctx, RECON_EINVAL, "n is negative");
    if (n > 0 && !lor) return fail(ctx, RECON_EINVAL, "lor is NULL");
    // the image is rewritten: until it is complete the context has none
    ctx->have_sens = false;
    ctx->sens_generation++;
    invalidate_graph(ctx);
    CK(cudaMemsetAsync(ctx->s64.p, 0, sizeof(double) * ctx->n_vox, ctx->stream));
    const recon_grid& cg = ctx->grid;
    const GridD g{cg.nx, cg.ny, cg.nz, cg.vx, cg.vy, cg.vz, cg.ox, cg.oy, cg.oz};
    if (n > 0) {
        if (on_device) {
            CK(launch_sensitivity(lor, n, g, ctx->s64.as<double>(), ctx->stream));
            ctx->stats.kernel_launches += 1;
        } else {
            const long long chunk = std::min<long long>(n, 1LL << 23);
            CK(ensure(ctx->staging, sizeof(float) * 6 * (size_t)chunk));
            float* st = ctx->staging.as<float>();
            for (long long lo = 0; lo < n; lo += chunk) {
                const long long m = std::min(chunk, n - lo);
                for (int k = 0; k < 6; ++k)
                    CK(cudaMemcpyAsync(st + (size_t)k * m, lor + (size_t)k * n + lo, sizeof(float) * m,
                                       cudaMemcpyHostToDevice, ctx->stream));
                CK(launch_sensitivity(st, m, g, ctx->s64.as<double>(), ctx->stream));
                ctx->stats.kernel_launches += 1;
            }
        }
    }
    recon_status s = finish_sensitivity(ctx);
    if (s != RECON_OK) return s;
    if (sens_out) CK(cudaMemcpyAsync(sens_out, ctx->s64.p, sizeof(double) * ctx->n_vox, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RECON_OK;
}

recon_status recon_set_sensitivity(recon_ctx* ctx, const double* sens, int32_t on_device)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_set_sensitivity");
    if (!sens) return fail(ctx, RECON_EINVAL, "sens is NULL");
    ctx->have_sens = false;
    ctx->sens_generation++;
    invalidate_graph(ctx);
    CK(cudaMemcpyAsync(ctx->s64.p, sens, sizeof(double) * ctx->n_vox,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    recon_status s = finish_sensitivity(ctx);
    if (s != RECON_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return RECON_OK;
}

recon_status recon_load_events(recon_ctx* ctx, const recon_events* events)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_load_events");
    return load_events(ctx, events);
}

recon_status recon_preprocess(recon_ctx* ctx, const recon_events* events, const float* mu_map, double z_reject,
                              int32_t apply, float* weight_out, uint8_t* keep_out, int64_t* n_kept)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_preprocess");
    if (!mu_map) return fail(ctx, RECON_EINVAL, "mu_map is NULL");
    if (!(z_reject >= 0.0) || !(z_reject <= 10.0)) return fail(ctx, RECON_EINVAL, "z_reject must be in [0, 10]");
    if (events) {
        recon_status s = load_events(ctx, events);
        if (s != RECON_OK) return s;
    }
    if (!ctx->have_ev) return fail(ctx, RECON_ESTATE, "no events loaded");
    const long long n = ctx->n_ev;
    CK(ensure(ctx->mu, sizeof(float) * (size_t)ctx->n_vox));
    CK(cudaMemcpyAsync(ctx->mu.p, mu_map, sizeof(float) * (size_t)ctx->n_vox, cudaMemcpyDefault, ctx->stream));
    CK(ensure(ctx->counter, sizeof(unsigned long long)));
    CK(cudaMemsetAsync(ctx->counter.p, 0, sizeof(unsigned long long), ctx->stream));
    if (weight_out && n > 0) CK(ensure(ctx->vec, sizeof(float) * (size_t)n));
    if (keep_out && n > 0) CK(ensure(ctx->keep, (size_t)n));
    const float half = (float)(z_reject * ctx->sigma_mm);
    CK(launch_preprocess(ctx->ev.p, ctx->fmt, n, (float)ctx->lattice, grid_h(ctx->grid), ctx->mu.as<float>(), half,
                         apply ? 1 : 0, weight_out ? ctx->vec.as<float>() : nullptr,
                         keep_out ? ctx->keep.as<uint8_t>() : nullptr, ctx->counter.as<unsigned long long>(),
                         ctx->stream));
    ctx->stats.kernel_launches += n > 0 ? 1 : 0;
    if (weight_out && n > 0)
        CK(cudaMemcpyAsync(weight_out, ctx->vec.p, sizeof(float) * (size_t)n, cudaMemcpyDefault, ctx->stream));
    if (keep_out && n > 0) CK(cudaMemcpyAsync(keep_out, ctx->keep.p, (size_t)n, cudaMemcpyDefault, ctx->stream));
    unsigned long long kept = 0;
    CK(cudaMemcpyAsync(&kept, ctx->counter.p, sizeof kept, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (n_kept) *n_kept = (int64_t)kept;
    if (apply) return events_changed(ctx);
    return RECON_OK;
}

recon_status recon_forward(recon_ctx* ctx, const recon_events* events, const float* image, float* p_out)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_forward");
    if (events) {
        recon_status s = load_events(ctx, events);
        if (s != RECON_OK) return s;
    }
    if (!ctx->have_ev) return fail(ctx, RECON_ESTATE, "no events loaded");
    if (!p_out && ctx->n_ev > 0) return fail(ctx, RECON_EINVAL, "p_out is NULL");
    if (image) CK(cudaMemcpyAsync(ctx->lam.p, image, sizeof(float) * ctx->n_vox, cudaMemcpyDefault, ctx->stream));
    if (ctx->n_ev == 0) return RECON_OK;
    CK(ensure(ctx->vec, sizeof(float) * (size_t)ctx->n_ev));
    PassArgs a = base_args(ctx, ctx->ev.p, ctx->n_ev);
    a.lam = ctx->lam.as<float>();
    if (ctx->bf16) {
        CK(launch_to_bf16(ctx->lam.as<float>(), ctx->lam_bf16.as<uint16_t>(), ctx->n_vox, ctx->stream));
        a.lam_bf16 = ctx->lam_bf16.as<uint16_t>();
        ctx->stats.kernel_launches += 1;
    }
    a.p_out = ctx->vec.as<float>();
    LaunchCfg cfg = ctx->user_cfg ? ctx->cfg : default_cfg(ctx);
    CK(ensure(ctx->work, 64));
    a.work = ctx->work.as<unsigned long long>();
    CK(cudaMemsetAsync(ctx->work.p, 0, 8, ctx->stream));
    const RegionTable tbl = single_table(ctx);
    CK(launch_pass(PASS_FORWARD, (EventFmt)ctx->fmt, cfg, a, tbl, ctx->num_sms, ctx->stream));
    ctx->stats.kernel_launches += 1;
    ctx->last_cfg = cfg;
    ctx->last_tiling = 0;
    ctx->last_lanes = 1;
    CK(cudaMemcpyAsync(p_out, ctx->vec.p, sizeof(float) * ctx->n_ev, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RECON_OK;
}

recon_status recon_backproject(recon_ctx* ctx, const recon_events* events, const float* r, float* image_out)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_backproject");
    if (events) {
        recon_status s = load_events(ctx, events);
        if (s != RECON_OK) return s;
    }
    if (!ctx->have_ev) return fail(ctx, RECON_ESTATE, "no events loaded");
    if (!image_out) return fail(ctx, RECON_EINVAL, "image_out is NULL");
    if (!r && ctx->n_ev > 0) return fail(ctx, RECON_EINVAL, "r is NULL");
    CK(cudaMemsetAsync(ctx->C.p, 0, sizeof(float) * ctx->n_vox, ctx->stream));
    if (ctx->n_ev > 0) {
        CK(ensure(ctx->vec, sizeof(float) * (size_t)ctx->n_ev));
        CK(cudaMemcpyAsync(ctx->vec.p, r, sizeof(float) * ctx->n_ev, cudaMemcpyDefault, ctx->stream));
        PassArgs a = base_args(ctx, ctx->ev.p, ctx->n_ev);
        a.C = ctx->C.as<float>();
        a.r_in = ctx->vec.as<float>();
        LaunchCfg cfg = ctx->user_cfg ? ctx->cfg : default_cfg(ctx);
        a.work = ctx->work.as<unsigned long long>();
        CK(cudaMemsetAsync(ctx->work.p, 0, 8, ctx->stream));
        const RegionTable tbl = single_table(ctx);
        CK(launch_pass(PASS_BACK, (EventFmt)ctx->fmt, cfg, a, tbl, ctx->num_sms, ctx->stream));
        ctx->stats.kernel_launches += 1;
        ctx->last_cfg = cfg;
        ctx->last_tiling = 0;
        ctx->last_lanes = 1;
    }
    CK(cudaMemcpyAsync(image_out, ctx->C.p, sizeof(float) * ctx->n_vox, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemsetAsync(ctx->C.p, 0, sizeof(float) * ctx->n_vox, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RECON_OK;
}

// Tile geometry of the shared-memory pass for this context, or false when no
// cell size lets two tiles (lambda and C) fit the shared memory of a block.
// Halo per axis: K sigma |u_k| / v_k voxels plus 1/8 voxel, with |u_z| bounded
// by the scanner's axial acceptance (events beyond it take the fallback pass).
bool tile_params(const recon_ctx* ctx, int mode, TileH* out)
{
    if (mode == 0 || (mode == 1 && (ctx->lut_n > 0 || ctx->subsets != 1))) return false;
    const recon_grid& g = ctx->grid;
    if (mode == 2) {
        // event order only: cells of 3^3 voxels, a halo covering the grid (no fallback)
        TileH t{};
        t.nx = g.nx;
        t.ny = g.ny;
        t.nz = g.nz;
        t.vx = (float)g.vx;
        t.vy = (float)g.vy;
        t.vz = (float)g.vz;
        t.ox = (float)g.ox;
        t.oy = (float)g.oy;
        t.oz = (float)g.oz;
        t.cs = ctx->order_cell;
        t.hx = g.nx;
        t.hy = g.ny;
        t.hz = g.nz;
        t.ncx = (g.nx + t.cs - 1) / t.cs;
        t.ncy = (g.ny + t.cs - 1) / t.cs;
        t.ncz = (g.nz + t.cs - 1) / t.cs;
        t.dir_az = ctx->order_dir_az;
        t.dir_pol = ctx->order_dir_pol;
        const double keys = (double)t.ncx * t.ncy * t.ncz * t.dir_az * t.dir_pol;
        if (keys + 1 >= 4.0e9) return false;
        t.none_code = (unsigned)keys;   // events whose window misses the grid: a last bucket
        *out = t;
        return true;
    }
    const double hw = ctx->k_sigma * ctx->sigma_mm;
    const double sin_max = std::sin(std::min(90.0, std::max(0.0, ctx->geom.max_axial_angle_deg)) * (3.14159265358979323846 / 180.0));
    TileH t{};
    t.nx = g.nx;
    t.ny = g.ny;
    t.nz = g.nz;
    t.vx = (float)g.vx;
    t.vy = (float)g.vy;
    t.vz = (float)g.vz;
    t.ox = (float)g.ox;
    t.oy = (float)g.oy;
    t.oz = (float)g.oz;
    t.hx = (int)std::ceil(hw / g.vx + 0.125);
    t.hy = (int)std::ceil(hw / g.vy + 0.125);
    t.hz = (int)std::ceil(hw * sin_max / g.vz + 0.125);
    t.dir_az = 1;
    t.dir_pol = 1;
    t.none_code = 0xFFFFFFFFu;
    for (int cs = 4; cs >= 2; --cs) {
        t.cs = cs;
        t.ncx = (g.nx + cs - 1) / cs;
        t.ncy = (g.ny + cs - 1) / cs;
        t.ncz = (g.nz + cs - 1) / cs;
        const double cells = (double)t.ncx * t.ncy * t.ncz;
        if (cells >= 4.0e9) continue;
        if (tile_smem_bytes(t) <= (size_t)220 * 1024) {
            *out = t;
            return true;
        }
    }
    return false;
}

// Bin the resident events by cell (cached per event generation and window).
recon_status prepare_tiles(recon_ctx* ctx, int mode)
{
    NvtxRange nvtx_range("event order binning");
    TilePrep& tp = ctx->tile_prep;
    TileH t;
    if (!ctx->have_ev || ctx->n_ev <= 0 || !tile_params(ctx, mode, &t)) {
        tp.valid = false;
        return RECON_OK;
    }
    const double hw = (double)make_tof(ctx).half_window;
    if (tp.valid && tp.ev_gen == ctx->ev_generation && tp.half_window == hw && tp.th.cs == t.cs &&
        tp.th.hx == t.hx && tp.th.hy == t.hy && tp.th.hz == t.hz && tp.th.dir_az == t.dir_az &&
        tp.th.dir_pol == t.dir_pol && tp.min_events == ctx->tile_min_events &&
        tp.mode == mode && tp.subsets == (mode == 2 ? std::max(1, ctx->subsets) : 1))
        return RECON_OK;
    tp.valid = false;
    invalidate_graph(ctx);
    const long long n = ctx->n_ev;
    // keys: cells x direction bins, plus the bucket of events whose window misses the grid
    const long long nc = (long long)t.ncx * t.ncy * t.ncz * t.dir_az * t.dir_pol + (mode == 2 ? 1 : 0);
    const size_t rec = ctx->fmt == FMT_PACKED ? 16 : 32;
    // OSEM: each subset's block of the list is binned on its own, in place, so that
    // the blocks keep their events (every event is binned in the event order)
    const int blocks = mode == 2 ? std::max(1, ctx->subsets) : 1;
    const long long nb_max = (n + blocks - 1) / blocks;
    CK(ensure(tp.code, sizeof(unsigned) * (size_t)std::max(nb_max, 1LL)));
    CK(ensure(tp.counts, sizeof(unsigned) * (size_t)nc));
    CK(ensure(tp.rank, sizeof(unsigned) * (size_t)std::max(nb_max, 1LL)));
    CK(ensure(tp.begin, sizeof(long long) * (size_t)(nc + 1)));
    CK(ensure(tp.scratch, sizeof(long long) * (size_t)scan_scratch_elems(nc)));
    CK(ensure(tp.list, sizeof(unsigned) * (size_t)nc));
    CK(ensure(tp.misc, 64));
    CK(cudaMemsetAsync(tp.misc.p, 0, 64, ctx->stream));
    unsigned long long* n_fb_dev = tp.misc.as<unsigned long long>();
    unsigned long long* fb_cursor = n_fb_dev + 1;
    unsigned* n_list_dev = reinterpret_cast<unsigned*>(n_fb_dev + 2);
    if (mode == 2) {
        CK(ensure(tp.ev_cell, rec * (size_t)n));
        CK(ensure(tp.ev_fb, rec));
        for (int b = 0; b < blocks; ++b) {
            const long long lo = b * n / blocks, hi = (b + 1) * n / blocks;
            if (hi <= lo) continue;
            const void* src = static_cast<const char*>(ctx->ev.p) + (size_t)lo * rec;
            void* dst = static_cast<char*>(tp.ev_cell.p) + (size_t)lo * rec;
            // a streamed upload may have computed the codes already, chunk by chunk
            const bool have_codes = blocks == 1 && tp.codes_gen == ctx->ev_generation && tp.codes_hw == hw &&
                                    tp.codes_th.cs == t.cs && tp.codes_th.ncx == t.ncx && tp.codes_th.ncy == t.ncy &&
                                    tp.codes_th.ncz == t.ncz && tp.codes_th.dir_az == t.dir_az &&
                                    tp.codes_th.dir_pol == t.dir_pol;
            tp.codes_gen = -1;
            if (!have_codes) {
                CK(cudaMemsetAsync(tp.counts.p, 0, sizeof(unsigned) * (size_t)nc, ctx->stream));
                CK(launch_cell_codes(src, ctx->fmt, hi - lo, (float)ctx->lattice, t, (float)hw,
                                     tp.code.as<unsigned>(), tp.counts.as<unsigned>(), tp.rank.as<unsigned>(), n_fb_dev,
                                     ctx->stream));
            }
            CK(launch_cell_scan(tp.counts.as<unsigned>(), nc, tp.begin.as<long long>(), tp.scratch.as<long long>(),
                                ctx->stream));
            CK(launch_cell_scatter(src, ctx->fmt, hi - lo, tp.code.as<unsigned>(), tp.begin.as<long long>(),
                                   tp.rank.as<unsigned>(), dst, tp.ev_fb.p, fb_cursor, ctx->stream));
            ctx->stats.kernel_launches += have_codes ? 4 : 5;
        }
        tp.n_fb = 0;
        tp.n_list = 0;
        tp.n_binned = n;
    } else {
        CK(cudaMemsetAsync(tp.counts.p, 0, sizeof(unsigned) * (size_t)nc, ctx->stream));
        CK(launch_cell_codes(ctx->ev.p, ctx->fmt, n, (float)ctx->lattice, t, (float)hw, tp.code.as<unsigned>(),
                             tp.counts.as<unsigned>(), tp.rank.as<unsigned>(), n_fb_dev, ctx->stream));
        CK(launch_cell_list(tp.counts.as<unsigned>(), nc, (unsigned)ctx->tile_min_events, tp.list.as<unsigned>(),
                            n_list_dev, n_fb_dev, ctx->stream));
        CK(launch_cell_scan(tp.counts.as<unsigned>(), nc, tp.begin.as<long long>(), tp.scratch.as<long long>(),
                            ctx->stream));
        unsigned long long host_misc[3] = {0, 0, 0};
        long long binned = 0;
        CK(cudaMemcpyAsync(host_misc, tp.misc.p, sizeof host_misc, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(&binned, tp.begin.as<long long>() + nc, sizeof binned, cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        tp.n_fb = (long long)host_misc[0];
        tp.n_list = (unsigned)(host_misc[2] & 0xFFFFFFFFu);
        CK(ensure(tp.ev_cell, rec * (size_t)std::max(binned, 1LL)));
        CK(ensure(tp.ev_fb, rec * (size_t)std::max(tp.n_fb, 1LL)));
        CK(launch_cell_scatter(ctx->ev.p, ctx->fmt, n, tp.code.as<unsigned>(), tp.begin.as<long long>(),
                               tp.rank.as<unsigned>(), tp.ev_cell.p, tp.ev_fb.p, fb_cursor, ctx->stream));
        ctx->stats.kernel_launches += 7;
        tp.n_binned = binned;
    }
    tp.th = t;
    tp.mode = mode;
    tp.subsets = blocks;
    tp.min_events = ctx->tile_min_events;
    tp.half_window = hw;
    tp.n_cells = nc;
    tp.ev_gen = ctx->ev_generation;
    tp.valid = true;
    return RECON_OK;
}

// Use the tiled pass in plan p when its binning is ready.
void plan_tiles(recon_ctx* ctx, IterPlan& p)
{
    const TilePrep& tp = ctx->tile_prep;
    p.tiled = tp.valid && tp.ev_gen == ctx->ev_generation && p.n_regions == 1 && tp.subsets == p.subsets &&
              (tp.mode == 2 || (p.subsets == 1 && p.a.lut.n == 0));
    if (!p.tiled) return;
    p.th = tp.th;
    p.list = tp.list.as<unsigned>();
    p.n_list = tp.n_list;
    p.tbegin = tp.begin.as<long long>();
    p.ev_cell = tp.ev_cell.p;
    p.ev_fb = tp.ev_fb.p;
    p.n_fb = tp.n_fb;
    p.n_cell_events = tp.n_binned;
    p.tile_mode = tp.mode;
    p.lanes = ctx->tile_lanes;
}

// Device time of one event pass of plan p (best of two); the pass accumulates
// into C and the N_eff slots, which the caller clears.
recon_status time_event_pass(recon_ctx* ctx, const IterPlan& p, float* ms_out)
{
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        CK(cudaEventRecord(e0, ctx->stream));
        recon_status s = launch_event_pass(ctx, p, p.a, p.tbl);
        if (s != RECON_OK) return s;
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
        ctx->stats.kernel_launches += 1 + (p.tiled && p.n_fb > 0 ? 1 : 0) + (p.bricks ? 2 * p.tbl.n : 0);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = best;
    return RECON_OK;
}

// Host events and n_iter >= 1: the upload is streamed in chunks through two
// staging halves on a copy stream, and the first iteration's event pass runs
// on each chunk as soon as it is resident, so the pass hides under the
// host-to-device copies.  Then the first update runs as usual.
bool can_stream(const recon_ctx* ctx, const recon_events* e, int n_iter)
{
    return e && !e->on_device && !e->weight && e->n > 0 && n_iter >= 1 && ctx->subsets == 1;
}

// Resident-event state for a streamed upload (the data arrive in stream_pass).
recon_status begin_streamed_events(recon_ctx* ctx, const recon_events* e)
{
    recon_status s = validate_events(ctx, e);
    if (s != RECON_OK) return s;
    const bool packed = e->fmt == RECON_EV_PACKED_I16_F16;
    ctx->have_ev = false;
    ctx->n_ev = 0;
    ctx->ev_generation++;
    invalidate_graph(ctx);
    CK(ensure(ctx->ev, (size_t)e->n * (packed ? 16 : 32)));
    ctx->fmt = packed ? FMT_PACKED : FMT_F32;
    ctx->lattice = packed ? e->lattice_mm : 0.0;
    ctx->n_ev = e->n;
    ctx->w_total = (double)e->n;   // unit weights (can_stream excludes caller weights)
    // have_ev is set by recon_mlem once stream_pass has uploaded every chunk
    return RECON_OK;
}

recon_status stream_pass(recon_ctx* ctx, const recon_events* e, const IterPlan& p, bool bin_after)
{
    NvtxRange nvtx_range("streamed first pass");
    if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        if (!ctx->copied[k]) CK(cudaEventCreateWithFlags(&ctx->copied[k], cudaEventDisableTiming));
        if (!ctx->drained[k]) CK(cudaEventCreateWithFlags(&ctx->drained[k], cudaEventDisableTiming));
    }
    if (!ctx->ready) CK(cudaEventCreateWithFlags(&ctx->ready, cudaEventDisableTiming));
    const bool packed = ctx->fmt == FMT_PACKED;
    const long long n = e->n;
    const long long chunk = std::min(n, 1LL << 23);
    const size_t half = (size_t)chunk * (packed ? 16 : 28);
    CK(ensure(ctx->staging, 2 * half));
    // staging may still be read by earlier work on ctx->stream
    CK(cudaEventRecord(ctx->ready, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ready, 0));
    // when iterations in the default event order follow, the events' cell codes are
    // computed chunk by chunk as the chunks arrive (hidden under the copies), so the
    // binning after the upload only scans and scatters
    TilePrep& tp = ctx->tile_prep;
    tp.codes_gen = -1;
    TileH tc{};
    const double hw = (double)make_tof(ctx).half_window;
    const bool codes = bin_after && ctx->tile_mode == 2 && ctx->subsets == 1 && tile_params(ctx, 2, &tc);
    if (codes) {
        const long long nc = (long long)tc.ncx * tc.ncy * tc.ncz * tc.dir_az * tc.dir_pol + 1;
        CK(ensure(tp.code, sizeof(unsigned) * (size_t)n));
        CK(ensure(tp.rank, sizeof(unsigned) * (size_t)n));
        CK(ensure(tp.counts, sizeof(unsigned) * (size_t)nc));
        CK(ensure(tp.misc, 64));
        CK(cudaMemsetAsync(tp.counts.p, 0, sizeof(unsigned) * (size_t)nc, ctx->stream));
        CK(cudaMemsetAsync(tp.misc.p, 0, 64, ctx->stream));
    }
    int q = 0;
    for (long long lo = 0; lo < n; lo += chunk, q ^= 1) {
        const long long m = std::min(chunk, n - lo);
        char* st = static_cast<char*>(ctx->staging.p) + (size_t)q * half;
        if (lo >= 2 * chunk) CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->drained[q], 0));
        const float* pl[7];
        if (packed) {
            CK(cudaMemcpyAsync(st, static_cast<const int4*>(e->planes[0]) + lo, (size_t)m * 16,
                               cudaMemcpyHostToDevice, ctx->copy_stream));
        } else {
            for (int k = 0; k < 7; ++k) {
                float* dst = reinterpret_cast<float*>(st) + (size_t)k * chunk;
                CK(cudaMemcpyAsync(dst, static_cast<const float*>(e->planes[k]) + lo, (size_t)m * 4,
                                   cudaMemcpyHostToDevice, ctx->copy_stream));
                pl[k] = dst;
            }
        }
        CK(cudaEventRecord(ctx->copied[q], ctx->copy_stream));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->copied[q], 0));
        if (packed)
            CK(launch_ingest_packed(reinterpret_cast<const int4*>(st), nullptr, m, ctx->ev.as<int4>() + lo,
                                    ctx->stream));
        else
            CK(launch_ingest_f32(pl, nullptr, m, ctx->ev.as<float4>() + 2 * lo, ctx->stream));
        CK(cudaEventRecord(ctx->drained[q], ctx->stream));
        PassArgs a = p.a;
        RegionTable t = p.tbl;
        a.events = static_cast<const char*>(p.a.events) + (size_t)lo * p.rec_bytes;
        a.n = m;
        t.ev_begin[1] = m;
        if (p.cfg.blocks_per_sm > 0) CK(cudaMemsetAsync(ctx->work.p, 0, 8, ctx->stream));
        CK(launch_pass(PASS_FUSED, (EventFmt)ctx->fmt, p.cfg, a, t, ctx->num_sms, ctx->stream));
        ctx->stats.kernel_launches += 2;
        if (codes) {
            CK(launch_cell_codes(a.events, ctx->fmt, m, (float)ctx->lattice, tc, (float)hw,
                                 tp.code.as<unsigned>() + lo, tp.counts.as<unsigned>(), tp.rank.as<unsigned>() + lo,
                                 tp.misc.as<unsigned long long>(), ctx->stream));
            ctx->stats.kernel_launches += 1;
        }
    }
    if (codes) {
        tp.codes_gen = ctx->ev_generation;
        tp.codes_th = tc;
        tp.codes_hw = hw;
    }
    // first update (the pass above was its event pass)
    CK(cudaMemsetAsync(p.iter, 0, sizeof(int), ctx->stream));
    CK(launch_update(p.lam, p.C, p.s32, p.bf16, p.reg_vox_dev, p.n_regions, ctx->upd_partial.as<double>(), p.upd_bpr,
                     ctx->stream));
    recon_status sv = enqueue_sieve(ctx, p);
    if (sv != RECON_OK) return sv;
    CK(launch_finalize(p.a.partial, kNeffSlots, ctx->upd_partial.as<double>(), p.upd_bpr, p.n_regions, p.hist,
                       p.iter, p.hist_cap, ctx->stream));
    ctx->stats.kernel_launches += 2 + (p.med ? 1 : 0);
    return RECON_OK;
}

}  // extern "C"

namespace {

// recon_event_pass: one event pass instead of n_iter iterations.
struct PassOnly {
    const float* image;   // start from this image (nullable)
    bool from_start;      // start from 1 on {s > 0}
    float* C_out;
    double* n_eff_out;
};

recon_status mlem_impl(recon_ctx* ctx, const recon_events* events, int32_t n_iter, const float* init,
                       float* image_out, double* conservation_out, const PassOnly* po)
{
    if (n_iter < 0) return fail(ctx, RECON_EINVAL, "n_iter is negative");
    if ((long long)n_iter * ctx->subsets > (1LL << 24)) return fail(ctx, RECON_EINVAL, "n_iter x subsets too large");
    const bool streamed =
        !po && can_stream(ctx, events, n_iter) && ctx->have_sens && (init || ctx->start_mode == 0);
    // event order / tiles (mode 2, cell order, is the default)
    const int mode = ctx->tile_mode;
    if (streamed) {
        recon_status s = begin_streamed_events(ctx, events);
        if (s != RECON_OK) return s;
    } else if (events) {
        recon_status s = load_events(ctx, events);
        if (s != RECON_OK) return s;
    }
    if (!ctx->have_sens) return fail(ctx, RECON_ESTATE, "no sensitivity image (call recon_sensitivity first)");
    if (!ctx->have_ev && !streamed) return fail(ctx, RECON_ESTATE, "no events loaded");
    const long long nv = ctx->n_vox;
    if (po) {
        if (po->from_start) {
            CK(launch_fill_masked(ctx->lam.as<float>(), ctx->s32.as<float>(), nv, 1.f, ctx->stream));
            ctx->stats.kernel_launches += 1;
        } else if (po->image) {
            CK(cudaMemcpyAsync(ctx->lam.p, po->image, sizeof(float) * nv, cudaMemcpyDefault, ctx->stream));
        }
    } else if (init) {
        CK(cudaMemcpyAsync(ctx->lam.p, init, sizeof(float) * nv, cudaMemcpyDefault, ctx->stream));
    } else if (ctx->start_mode == 1) {
        // starting backprojection: lambda0 = (sum_i a_ij w_i) / s_j on the mask, from a
        // backward pass with r_i = w_i and the update applied to lambda = 1
        const bool packed = ctx->fmt == FMT_PACKED;
        CK(ensure(ctx->vec, sizeof(float) * (size_t)std::max(1LL, ctx->n_ev)));
        CK(launch_event_weights(packed ? nullptr : ctx->ev.as<float4>(), packed ? ctx->ev.as<int4>() : nullptr,
                                ctx->n_ev, ctx->vec.as<float>(), ctx->stream));
        CK(launch_fill_masked(ctx->lam.as<float>(), ctx->s32.as<float>(), nv, 1.f, ctx->stream));
        CK(cudaMemsetAsync(ctx->C.p, 0, sizeof(float) * nv, ctx->stream));
        PassArgs b = base_args(ctx, ctx->ev.p, ctx->n_ev);
        b.C = ctx->C.as<float>();
        b.r_in = ctx->vec.as<float>();
        const RegionTable bt = single_table(ctx);
        const LaunchCfg bc = ctx->user_cfg ? ctx->cfg : default_cfg(ctx);
        CK(launch_pass(PASS_BACK, (EventFmt)ctx->fmt, bc, b, bt, ctx->num_sms, ctx->stream));
        const int bpr = update_blocks(nv);
        CK(ensure(ctx->upd_partial, sizeof(double) * (size_t)bpr));
        CK(ensure(ctx->reg_vox, sizeof(long long) * 2));
        const long long rv0[2] = {0, nv};
        CK(cudaMemcpyAsync(ctx->reg_vox.p, rv0, sizeof rv0, cudaMemcpyHostToDevice, ctx->stream));
        CK(launch_update(ctx->lam.as<float>(), ctx->C.as<float>(), ctx->s32.as<float>(), nullptr,
                         ctx->reg_vox.as<long long>(), 1, ctx->upd_partial.as<double>(), bpr, ctx->stream));
        ctx->stats.kernel_launches += 4;
    } else {
        const double v = ctx->sens_total > 0 ? ctx->w_total / ctx->sens_total : 0.0;
        CK(launch_fill_masked(ctx->lam.as<float>(), ctx->s32.as<float>(), nv, (float)v, ctx->stream));
        ctx->stats.kernel_launches += 1;
    }
    CK(cudaMemsetAsync(ctx->C.p, 0, sizeof(float) * nv, ctx->stream));
    if (ctx->bf16) {
        CK(ensure(ctx->lam_bf16, sizeof(uint16_t) * nv));
        CK(launch_to_bf16(ctx->lam.as<float>(), ctx->lam_bf16.as<uint16_t>(), nv, ctx->stream));
        ctx->stats.kernel_launches += 1;
    }
    IterPlan p;
    p.a = base_args(ctx, ctx->ev.p, ctx->n_ev);
    p.a.lam = ctx->lam.as<float>();
    p.a.lam_bf16 = ctx->bf16 ? ctx->lam_bf16.as<uint16_t>() : nullptr;
    p.a.C = ctx->C.as<float>();
    p.a.work = ctx->work.as<unsigned long long>();
    p.tbl = single_table(ctx);
    recon_status st;
    CK(ensure(ctx->pass_partial, sizeof(double) * kNeffSlots));
    p.a.partial = ctx->pass_partial.as<double>();
    // a streamed call autotunes only once the events are resident (not before the upload)
    p.cfg = streamed ? tuned_or_default(ctx, p.a, p.tbl) : choose_cfg(ctx, p.a, p.tbl, &st);
    if (!streamed && st != RECON_OK) return st;
    CK(cudaMemsetAsync(ctx->C.p, 0, sizeof(float) * nv, ctx->stream));
    CK(cudaMemsetAsync(ctx->pass_partial.p, 0, sizeof(double) * kNeffSlots, ctx->stream));
    p.pass_blocks = pass_blocks(p.cfg, ctx->n_ev, ctx->num_sms);
    p.upd_bpr = update_blocks(nv);
    CK(ensure(ctx->upd_partial, sizeof(double) * (size_t)p.upd_bpr));
    CK(ensure(ctx->reg_vox, sizeof(long long) * 2));
    const long long rv[2] = {0, nv};
    CK(cudaMemcpyAsync(ctx->reg_vox.p, rv, sizeof rv, cudaMemcpyHostToDevice, ctx->stream));
    p.subsets = ctx->subsets;
    p.rec_bytes = ctx->fmt == FMT_PACKED ? 16 : 32;
    p.hist_cap = std::max(n_iter * p.subsets, 64);
    CK(ensure(ctx->hist, sizeof(double) * 2 * (size_t)p.hist_cap));
    p.hist = ctx->hist.as<double>();
    p.iter = ctx->iter.as<int>();
    p.lam = ctx->lam.as<float>();
    p.C = ctx->C.as<float>();
    p.s32 = ctx->s32.as<float>();
    p.bf16 = ctx->bf16 ? ctx->lam_bf16.as<uint16_t>() : nullptr;
    p.reg_vox_dev = ctx->reg_vox.as<long long>();
    p.n_regions = 1;
    p.med = nullptr;
    p.med_vox = nv;
    p.max_nz = ctx->grid.nz;
    // image layout of the pass: brick copies for the sampled projector when asked
    // for (recon_set_brick_layout), and for the exact projector when the launch
    // says so (its reduction form; not with the shared-memory tiled pass)
    auto set_layout = [&]() -> recon_status {
        const bool exact_bricks = ctx->lut_n == 0 && p.cfg.reduction == 1 && !ctx->bf16 && p.cfg.blocks_per_sm == 0 &&
                                  p.cfg.cache == 0 && !(p.tiled && p.tile_mode == 1);
        const bool lut_bricks = ctx->lut_n > 0 && !ctx->bf16 && (ctx->bricks || p.cfg.reduction == 1);
        p.bricks = lut_bricks || exact_bricks;
        if (p.bricks) {
            const size_t nb = (size_t)brick_voxels(ctx->grid.nx, ctx->grid.ny, ctx->grid.nz);
            CK(ensure(ctx->lam_brick, sizeof(float) * nb));
            CK(ensure(ctx->C_brick, sizeof(float) * nb));
            CK(cudaMemsetAsync(ctx->C_brick.p, 0, sizeof(float) * nb, ctx->stream));
        }
        return RECON_OK;
    };
    {
        recon_status sl = set_layout();
        if (sl != RECON_OK) return sl;
    }
    if (ctx->median) {
        CK(ensure(ctx->med, sizeof(float) * (size_t)nv));
        p.med = ctx->med.as<float>();
    }
    ctx->last_cfg = p.cfg;
    // launch for the event list the iterations will walk (the cell-ordered copy when
    // that order is on); an autotuner run accumulates into C and the N_eff slots, which
    // are cleared again
    auto retune = [&]() -> recon_status {
        PassArgs ta = p.a;
        RegionTable tt = p.tbl;
        if (p.tiled && p.tile_mode == 2) {
            ta.events = p.ev_cell;
            ta.n = p.n_cell_events;
            ta.block_mul = 1;
            tt.ev_begin[1] = p.n_cell_events;
        }
        const long long runs = ctx->stats.autotune_runs;
        recon_status st2;
        LaunchCfg c = choose_cfg(ctx, ta, tt, &st2);
        if (st2 != RECON_OK) return st2;
        if (ctx->stats.autotune_runs != runs) {
            CK(cudaMemsetAsync(ctx->C.p, 0, sizeof(float) * nv, ctx->stream));
            CK(cudaMemsetAsync(ctx->pass_partial.p, 0, sizeof(double) * kNeffSlots, ctx->stream));
        }
        p.cfg = c;
        p.pass_blocks = pass_blocks(p.cfg, ctx->n_ev, ctx->num_sms);
        ctx->last_cfg = c;
        return set_layout();
    };
    // The event list the iterations walk: binned into cell order (the default) or
    // into shared-memory tiles.  With the autotuner on, the first call on a new
    // (events, format, voxels) key of the exact projector also times the tiled pass
    // with 1 and 8 threads per event against the tuned cell-ordered global pass, and
    // keeps the faster layout and its launch for the key.
    auto prepare_layout = [&]() -> recon_status {
        TileH th1;
        const bool can_tile = mode == 2 && ctx->autotune && !ctx->user_cfg && ctx->lut_n == 0 && p.subsets == 1 &&
                              !ctx->bf16 && ctx->n_ev >= (1LL << 20) && tile_params(ctx, 1, &th1);
        const auto lkey = std::make_tuple(ctx->n_ev, ctx->fmt, ctx->n_vox);
        auto it = can_tile ? ctx->layout_tuned.find(lkey) : ctx->layout_tuned.end();
        if (it != ctx->layout_tuned.end() && it->second.lanes > 0) {
            recon_status s1 = prepare_tiles(ctx, 1);
            if (s1 != RECON_OK) return s1;
            plan_tiles(ctx, p);
            p.lanes = it->second.lanes;
            p.cfg = it->second.cfg;
            p.pass_blocks = pass_blocks(p.cfg, ctx->n_ev, ctx->num_sms);
            ctx->last_cfg = p.cfg;
            return set_layout();
        }
        if (mode == 1 || mode == 2) {
            recon_status s1 = prepare_tiles(ctx, mode);
            if (s1 != RECON_OK) return s1;
            plan_tiles(ctx, p);
        }
        recon_status s1 = retune();
        if (s1 != RECON_OK) return s1;
        if (!can_tile || it != ctx->layout_tuned.end()) return RECON_OK;
        const LaunchCfg glob_cfg = p.cfg;
        float t_glob = 0;
        s1 = time_event_pass(ctx, p, &t_glob);
        if (s1 != RECON_OK) return s1;
        s1 = prepare_tiles(ctx, 1);
        if (s1 != RECON_OK) return s1;
        plan_tiles(ctx, p);
        s1 = set_layout();
        if (s1 != RECON_OK) return s1;
        int best = 0;
        float best_t = t_glob;
        if (p.tiled && p.tile_mode == 1) {
            for (int lanes : {1, 8}) {
                p.lanes = lanes;
                float t = 0;
                s1 = time_event_pass(ctx, p, &t);
                if (s1 != RECON_OK) return s1;
                if (t < best_t) {
                    best_t = t;
                    best = lanes;
                }
            }
        }
        ctx->layout_tuned[lkey] = {best, glob_cfg};
        CK(cudaMemsetAsync(ctx->C.p, 0, sizeof(float) * nv, ctx->stream));
        CK(cudaMemsetAsync(ctx->pass_partial.p, 0, sizeof(double) * kNeffSlots, ctx->stream));
        if (best > 0) {
            p.lanes = best;
            return RECON_OK;
        }
        s1 = prepare_tiles(ctx, 2);
        if (s1 != RECON_OK) return s1;
        plan_tiles(ctx, p);
        p.cfg = glob_cfg;
        p.pass_blocks = pass_blocks(p.cfg, ctx->n_ev, ctx->num_sms);
        ctx->last_cfg = p.cfg;
        return set_layout();
    };
    recon_status s;
    if (po) {
        // one pass over the resident events into C; C goes out, N_eff is summed, and
        // C and the N_eff slots are left zero
        s = prepare_layout();
        if (s != RECON_OK) return s;
        ctx->last_tiling = p.tiled && p.tile_mode == 1 ? 1 : 0;
        ctx->last_lanes = ctx->last_tiling ? p.lanes : 1;
        s = launch_event_pass(ctx, p, p.a, p.tbl);
        if (s != RECON_OK) return s;
        ctx->stats.kernel_launches += 1 + (p.tiled && p.n_fb > 0 ? 1 : 0) + (p.bricks ? 2 * p.tbl.n : 0);
        CK(cudaMemcpyAsync(po->C_out, ctx->C.p, sizeof(float) * nv, cudaMemcpyDefault, ctx->stream));
        double n_eff = 0;
        s = host_sum(ctx, ctx->pass_partial.as<double>(), kNeffSlots, &n_eff);
        if (s != RECON_OK) return s;
        if (po->n_eff_out) *po->n_eff_out = n_eff;
        CK(cudaMemsetAsync(ctx->C.p, 0, sizeof(float) * nv, ctx->stream));
        CK(cudaMemsetAsync(ctx->pass_partial.p, 0, sizeof(double) * kNeffSlots, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return RECON_OK;
    }
    if (streamed) {
        s = stream_pass(ctx, events, p, n_iter > 1);
        if (s != RECON_OK) return s;
        ctx->have_ev = true;
        if (n_iter > 1) {
            s = prepare_layout();
            if (s != RECON_OK) return s;
        }
        ctx->last_tiling = p.tiled && p.tile_mode == 1 ? 1 : 0;
        ctx->last_lanes = ctx->last_tiling ? p.lanes : 1;
        s = run_iterations(ctx, p, n_iter - 1, false);
    } else {
        if (n_iter > 0) {
            s = prepare_layout();
            if (s != RECON_OK) return s;
        }
        ctx->last_tiling = p.tiled && p.tile_mode == 1 ? 1 : 0;
        ctx->last_lanes = ctx->last_tiling ? p.lanes : 1;
        s = run_iterations(ctx, p, n_iter);
    }
    if (s != RECON_OK) return s;
    if (image_out) CK(cudaMemcpyAsync(image_out, ctx->lam.p, sizeof(float) * nv, cudaMemcpyDefault, ctx->stream));
    if (conservation_out && n_iter > 0)
        CK(cudaMemcpyAsync(conservation_out, ctx->hist.p, sizeof(double) * 2 * (size_t)n_iter * p.subsets,
                           cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RECON_OK;
}

}  // namespace

extern "C" {

recon_status recon_mlem(recon_ctx* ctx, const recon_events* events, int32_t n_iter, const float* init,
                        float* image_out, double* conservation_out)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_mlem");
    return mlem_impl(ctx, events, n_iter, init, image_out, conservation_out, nullptr);
}

recon_status recon_event_pass(recon_ctx* ctx, const recon_events* events, const float* image, int32_t from_start,
                              float* C_out, double* n_eff_out)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_event_pass");
    if (!C_out) return fail(ctx, RECON_EINVAL, "C_out is NULL");
    if (ctx->subsets != 1) return fail(ctx, RECON_EINVAL, "recon_event_pass runs MLEM passes (one subset)");
    const PassOnly po{image, from_start != 0, C_out, n_eff_out};
    return mlem_impl(ctx, events, 1, nullptr, nullptr, nullptr, &po);
}

recon_status recon_update(recon_ctx* ctx, const float* C_in, float* image_out, double* sum_s_lambda_out)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_update");
    if (!C_in) return fail(ctx, RECON_EINVAL, "C_in is NULL");
    if (!ctx->have_sens) return fail(ctx, RECON_ESTATE, "no sensitivity image (call recon_sensitivity first)");
    const long long nv = ctx->n_vox;
    const int bpr = update_blocks(nv);
    CK(ensure(ctx->upd_partial, sizeof(double) * (size_t)bpr));
    CK(ensure(ctx->reg_vox, sizeof(long long) * 2));
    if (ctx->median) CK(ensure(ctx->med, sizeof(float) * (size_t)nv));
    if (ctx->bf16) CK(ensure(ctx->lam_bf16, sizeof(uint16_t) * nv));
    const long long rv[2] = {0, nv};
    CK(cudaMemcpyAsync(ctx->reg_vox.p, rv, sizeof rv, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->C.p, C_in, sizeof(float) * nv, cudaMemcpyDefault, ctx->stream));
    uint16_t* bf = ctx->bf16 ? ctx->lam_bf16.as<uint16_t>() : nullptr;
    CK(launch_update(ctx->lam.as<float>(), ctx->C.as<float>(), ctx->s32.as<float>(), bf, ctx->reg_vox.as<long long>(), 1,
                     ctx->upd_partial.as<double>(), bpr, ctx->stream));
    ctx->stats.kernel_launches += 1;
    if (ctx->median) {
        CK(launch_median3(ctx->lam.as<float>(), ctx->med.as<float>(), ctx->s32.as<float>(), bf,
                          ctx->reg_vox.as<long long>(), 1, ctx->grid.nx, ctx->grid.ny, ctx->grid.nz, ctx->stream));
        CK(cudaMemcpyAsync(ctx->lam.p, ctx->med.p, sizeof(float) * (size_t)nv, cudaMemcpyDeviceToDevice, ctx->stream));
        ctx->stats.kernel_launches += 1;
    }
    double ssum = 0;
    recon_status s = host_sum(ctx, ctx->upd_partial.as<double>(), bpr, &ssum);
    if (s != RECON_OK) return s;
    if (sum_s_lambda_out) *sum_s_lambda_out = ssum;
    if (image_out) CK(cudaMemcpyAsync(image_out, ctx->lam.p, sizeof(float) * nv, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RECON_OK;
}

recon_status recon_split_regions(recon_ctx* ctx, const recon_events* events, int32_t n_regions,
                                 const recon_region* regions, double margin_mm, double shell_mm,
                                 uint8_t* code_out, int64_t* offsets_out, int32_t* idx_out)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_split_regions");
    recon_status s = validate_regions(ctx, n_regions, regions, margin_mm, shell_mm);
    if (s != RECON_OK) return s;
    if (events) {
        s = load_events(ctx, events);
        if (s != RECON_OK) return s;
    }
    if (!ctx->have_ev) return fail(ctx, RECON_ESTATE, "no events loaded");
    std::vector<long long> off;
    s = split_internal(ctx, n_regions, regions, shell_mm, off);
    if (s != RECON_OK) return s;
    if (code_out && ctx->n_ev > 0)
        CK(cudaMemcpyAsync(code_out, ctx->codes.p, (size_t)ctx->n_ev, cudaMemcpyDefault, ctx->stream));
    if (offsets_out)
        CK(cudaMemcpyAsync(offsets_out, off.data(), sizeof(long long) * (n_regions + 1), cudaMemcpyDefault,
                           ctx->stream));
    if (idx_out && off[n_regions] > 0)
        CK(cudaMemcpyAsync(idx_out, ctx->idx.p, sizeof(int) * (size_t)off[n_regions], cudaMemcpyDefault,
                           ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RECON_OK;
}

recon_status recon_set_region_block(recon_ctx* ctx, int32_t first, int32_t count)
{
    CHECK_CTX();
    if (first < 0 || count < 0 || first + count > kMaxRegions || (count == 0 && first != 0))
        return fail(ctx, RECON_EINVAL, "region block outside [0, 64) (count 0 needs first 0)");
    ctx->region_first = first;
    ctx->region_count = count;
    invalidate_graph(ctx);
    return RECON_OK;
}

recon_status recon_region_slab_voxels(const recon_ctx* ctx, int32_t n_regions, const recon_region* regions,
                                      double margin_mm, int64_t* n_vox_out)
{
    if (!ctx || !n_vox_out) return RECON_EINVAL;
    if (validate_regions(const_cast<recon_ctx*>(ctx), n_regions, regions, margin_mm, 0.0) != RECON_OK)
        return RECON_EINVAL;
    std::vector<int> lo, hi;
    slab_ranges(ctx, n_regions, regions, margin_mm, lo, hi);
    long long t = 0;
    for (int r = 0; r < n_regions; ++r) t += (long long)ctx->grid.nx * ctx->grid.ny * (hi[r] - lo[r]);
    *n_vox_out = t;
    return RECON_OK;
}

recon_status recon_mlem_regions(recon_ctx* ctx, const recon_events* events, int32_t n_regions,
                                const recon_region* regions, double margin_mm, double shell_mm, int32_t n_iter,
                                float* image_out, float* region_images_out, double* conservation_out)
{
    CHECK_CTX();
    NvtxRange nvtx_range("recon_mlem_regions");
    if (n_iter < 0) return fail(ctx, RECON_EINVAL, "n_iter is negative");
    recon_status s = validate_regions(ctx, n_regions, regions, margin_mm, shell_mm);
    if (s != RECON_OK) return s;
    if (events) {
        s = load_events(ctx, events);
        if (s != RECON_OK) return s;
    }
    if (!ctx->have_sens) return fail(ctx, RECON_ESTATE, "no sensitivity image (call recon_sensitivity first)");
    if (!ctx->have_ev) return fail(ctx, RECON_ESTATE, "no events loaded");
    const int R = n_regions;
    const bool packed = ctx->fmt == FMT_PACKED;
    RegionPrep& rp = ctx->region_prep;
    const bool reuse = rp.valid && rp.ev_gen == ctx->ev_generation && rp.sens_gen == ctx->sens_generation &&
                       rp.order == ctx->tile_mode &&
                       rp.margin == margin_mm && rp.shell == shell_mm && rp.fmt == ctx->fmt &&
                       (int)rp.regions.size() == R &&
                       std::equal(rp.regions.begin(), rp.regions.end(), regions, [](const recon_region& a,
                                                                                     const recon_region& b) {
                           return a.z_lo == b.z_lo && a.z_hi == b.z_hi;
                       });
    if (!reuse) {
        // split, region-ordered event copy, slab sensitivities and start values:
        // kept until the events, the sensitivity or the division change.  In cell
        // order the split reads the cell-ordered copy, so each region's events come
        // cell by cell (events whose window misses the grid are left out: they have
        // p_i = 0 and add nothing)
        rp.valid = false;
        const void* src = ctx->ev.p;
        long long n_src = ctx->n_ev;
        if (ctx->tile_mode == 2) {
            s = prepare_tiles(ctx, 2);
            if (s != RECON_OK) return s;
            if (ctx->tile_prep.valid && ctx->tile_prep.n_fb == 0) {
                src = ctx->tile_prep.ev_cell.p;
                n_src = ctx->tile_prep.n_binned;
            }
        }
        s = split_internal(ctx, R, regions, shell_mm, rp.off, src, n_src);
        if (s != RECON_OK) return s;
        const long long total = rp.off[R];
        const size_t rec = packed ? 16 : 32;
        CK(ensure(ctx->ev_reg, rec * (size_t)std::max(1LL, total)));
        CK(launch_region_gather(packed ? nullptr : static_cast<const float4*>(src),
                                packed ? static_cast<const int4*>(src) : nullptr,
                                ctx->codes.as<uint8_t>(), ctx->idx.as<int>(), total,
                                packed ? nullptr : ctx->ev_reg.as<float4>(), packed ? ctx->ev_reg.as<int4>() : nullptr,
                                ctx->stream));
        if (total > 0) ctx->stats.kernel_launches += 1;
        slab_ranges(ctx, R, regions, margin_mm, rp.lo, rp.hi);
        const long long plane = (long long)ctx->grid.nx * ctx->grid.ny;
        rp.rv.assign(R + 1, 0);
        for (int r = 0; r < R; ++r) rp.rv[r + 1] = rp.rv[r] + plane * (rp.hi[r] - rp.lo[r]);
        const long long nvt = rp.rv[R];
        CK(ensure(ctx->lam_reg, sizeof(float) * nvt));
        CK(ensure(ctx->C_reg, sizeof(float) * nvt));
        CK(ensure(ctx->s_reg, sizeof(float) * nvt));
        CK(ensure(ctx->reg_vox_reg, sizeof(long long) * (R + 1)));
        CK(cudaMemcpyAsync(ctx->reg_vox_reg.p, rp.rv.data(), sizeof(long long) * (R + 1), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(ensure(ctx->red_partial, sizeof(double) * 1024 * 2 * R));
        // per-region slab sensitivity (FP32 copy of the global s), sum of s and sum of w
        std::vector<int> bs(R), bw(R);
        double* part = ctx->red_partial.as<double>();
        for (int r = 0; r < R; ++r) {
            const long long nr = rp.rv[r + 1] - rp.rv[r];
            bs[r] = reduce_blocks(nr);
            CK(launch_sens_finish(ctx->s64.as<double>() + rp.lo[r] * plane, nr, ctx->s_reg.as<float>() + rp.rv[r],
                                  part + (size_t)2048 * r, bs[r], ctx->stream));
            const long long ne = rp.off[r + 1] - rp.off[r];
            bw[r] = ne > 0 ? reduce_blocks(ne) : 0;
            if (ne > 0)
                CK(launch_reduce_weights(packed ? nullptr : ctx->ev_reg.as<float4>() + 2 * rp.off[r],
                                         packed ? ctx->ev_reg.as<int4>() + rp.off[r] : nullptr, ne,
                                         part + (size_t)2048 * r + 1024, bw[r], ctx->stream));
            ctx->stats.kernel_launches += ne > 0 ? 2 : 1;
        }
        std::vector<double> h((size_t)2048 * R);
        CK(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        rp.start.assign(R, 0.f);
        for (int r = 0; r < R; ++r) {
            double S = 0, W = 0;
            for (int k = 0; k < bs[r]; ++k) S += h[(size_t)2048 * r + k];
            for (int k = 0; k < bw[r]; ++k) W += h[(size_t)2048 * r + 1024 + k];
            rp.start[r] = (float)(S > 0 ? W / S : 0.0);
        }
        rp.regions.assign(regions, regions + R);
        rp.margin = margin_mm;
        rp.shell = shell_mm;
        rp.fmt = ctx->fmt;
        rp.ev_gen = ctx->ev_generation;
        rp.order = ctx->tile_mode;
        rp.sens_gen = ctx->sens_generation;
        rp.valid = true;
    }
    const std::vector<long long>& off = rp.off;
    const std::vector<int>& lo = rp.lo;
    const std::vector<int>& hi = rp.hi;
    const std::vector<long long>& rv = rp.rv;
    // the block of regions to reconstruct (recon_set_region_block): its events are a
    // contiguous range of the region-ordered copy; the other regions start at 0 and stay 0
    const int b0 = ctx->region_count > 0 ? ctx->region_first : 0;
    const int b1 = ctx->region_count > 0 ? ctx->region_first + ctx->region_count : R;
    if (b1 > R) return fail(ctx, RECON_EINVAL, "the region block reaches past the division's regions");
    const long long total = off[b1] - off[b0];
    const long long nvt = rv[R];
    // start image: uniform on each slab's mask with sum s lambda = sum w of its events
    for (int r = 0; r < R; ++r)
        CK(launch_fill_masked(ctx->lam_reg.as<float>() + rv[r], ctx->s_reg.as<float>() + rv[r], rv[r + 1] - rv[r],
                              r >= b0 && r < b1 ? rp.start[r] : 0.f, ctx->stream));
    ctx->stats.kernel_launches += R;
    CK(cudaMemsetAsync(ctx->C_reg.p, 0, sizeof(float) * nvt, ctx->stream));
    if (ctx->bf16) {
        CK(ensure(ctx->bf16_reg, sizeof(uint16_t) * nvt));
        CK(launch_to_bf16(ctx->lam_reg.as<float>(), ctx->bf16_reg.as<uint16_t>(), nvt, ctx->stream));
        ctx->stats.kernel_launches += 1;
    }

    IterPlan p;
    const size_t rec = ctx->fmt == FMT_PACKED ? 16 : 32;
    p.a = base_args(ctx, static_cast<const char*>(ctx->ev_reg.p) + (size_t)off[b0] * rec, total);
    p.a.lam = ctx->lam_reg.as<float>();
    p.a.lam_bf16 = ctx->bf16 ? ctx->bf16_reg.as<uint16_t>() : nullptr;
    p.a.C = ctx->C_reg.as<float>();
    p.a.work = ctx->work.as<unsigned long long>();
    memset(&p.tbl, 0, sizeof p.tbl);
    p.tbl.n = R;
    for (int r = 0; r <= R; ++r) p.tbl.ev_begin[r] = std::min(std::max(off[r] - off[b0], 0LL), total);
    for (int r = 0; r < R; ++r) p.tbl.grid[r] = grid_h(ctx->grid, lo[r], hi[r], rv[r]);
    CK(ensure(ctx->pass_partial, sizeof(double) * kNeffSlots * R));
    p.a.partial = ctx->pass_partial.as<double>();
    {
        // region-ordered events: tune with the block spreading the pass will use
        PassArgs ta = p.a;
        ta.block_mul = 1;
        p.cfg = choose_cfg(ctx, ta, p.tbl, &s);
    }
    if (s != RECON_OK) return s;
    // the exact projector's brick layout (the launch's reduction form): each slab in its
    // own 2x2x2-brick copy
    p.bricks = ctx->lut_n == 0 && p.cfg.reduction == 1 && !ctx->bf16 && p.cfg.blocks_per_sm == 0 && p.cfg.cache == 0;
    if (p.bricks) {
        RegionTable bt;
        const long long nb = brick_table(p.tbl, bt);
        CK(ensure(ctx->lam_brick, sizeof(float) * (size_t)nb));
        CK(ensure(ctx->C_brick, sizeof(float) * (size_t)nb));
        CK(cudaMemsetAsync(ctx->C_brick.p, 0, sizeof(float) * (size_t)nb, ctx->stream));
    }
    CK(cudaMemsetAsync(ctx->C_reg.p, 0, sizeof(float) * nvt, ctx->stream));
    CK(cudaMemsetAsync(ctx->pass_partial.p, 0, sizeof(double) * kNeffSlots * R, ctx->stream));
    p.pass_blocks = pass_blocks(p.cfg, total, ctx->num_sms);
    p.a.block_mul = p.cfg.blocks_per_sm > 0 ? 0 : spread_multiplier(p.pass_blocks);
    p.upd_bpr = std::max(1, update_blocks(nvt) / R);
    CK(ensure(ctx->upd_partial, sizeof(double) * (size_t)p.upd_bpr * R));
    p.subsets = 1;
    p.rec_bytes = ctx->fmt == FMT_PACKED ? 16 : 32;
    p.hist_cap = std::max(n_iter, 64);
    CK(ensure(ctx->hist, sizeof(double) * 2 * (size_t)p.hist_cap * R));
    p.hist = ctx->hist.as<double>();
    p.iter = ctx->iter.as<int>();
    p.lam = ctx->lam_reg.as<float>();
    p.C = ctx->C_reg.as<float>();
    p.s32 = ctx->s_reg.as<float>();
    p.bf16 = ctx->bf16 ? ctx->bf16_reg.as<uint16_t>() : nullptr;
    p.reg_vox_dev = ctx->reg_vox_reg.as<long long>();
    p.n_regions = R;
    p.med = nullptr;
    p.med_vox = nvt;
    p.max_nz = 0;
    for (int r = 0; r < R; ++r) p.max_nz = std::max(p.max_nz, hi[r] - lo[r]);
    if (ctx->median) {
        CK(ensure(ctx->med, sizeof(float) * (size_t)nvt));
        p.med = ctx->med.as<float>();
    }
    ctx->last_cfg = p.cfg;
    ctx->last_tiling = 0;
    ctx->last_lanes = 1;
    s = run_iterations(ctx, p, n_iter);
    if (s != RECON_OK) return s;
    // stitch into the context's whole-grid image
    CK(launch_stitch(ctx->lam_reg.as<float>(), rv.data(), lo.data(), hi.data(), R, ctx->grid.nx, ctx->grid.ny,
                     ctx->grid.nz, ctx->lam.as<float>(), ctx->stream));
    ctx->stats.kernel_launches += 1;
    if (image_out) CK(cudaMemcpyAsync(image_out, ctx->lam.p, sizeof(float) * ctx->n_vox, cudaMemcpyDefault, ctx->stream));
    if (region_images_out)
        CK(cudaMemcpyAsync(region_images_out, ctx->lam_reg.p, sizeof(float) * nvt, cudaMemcpyDefault, ctx->stream));
    if (conservation_out && n_iter > 0)
        CK(cudaMemcpyAsync(conservation_out, ctx->hist.p, sizeof(double) * 2 * (size_t)n_iter * R, cudaMemcpyDefault,
                           ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RECON_OK;
}

}  // extern "C"
