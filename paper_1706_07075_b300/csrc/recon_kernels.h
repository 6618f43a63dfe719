// Host-visible launch interface of the CUDA kernels (internal to librecon).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace recon {

constexpr int kMaxRegions = 64;
constexpr int kNeffSlots = 32;  // FP64 slots per region that event-pass blocks fold N_eff into

// Grid of one image (or region slab): nx*ny*nz voxels of (vx,vy,vz) mm from
// the low corner (ox,oy,oz); vox_offset places it in a shared image buffer.
struct GridH {
    int nx, ny, nz;
    float vx, vy, vz;
    float ox, oy, oz;
    long long vox_offset;
};

// TOF kernel constants: half_window = K sigma (mm), inv_sigma_sqrt2 =
// 1/(sigma sqrt 2), half_inv_norm = 0.5 / erf(K / sqrt 2).
struct TofH {
    float half_window, inv_sigma_sqrt2, half_inv_norm;
};

// Per-region grid and event range for the batched pass (plain = 1 region).
struct RegionTable {
    int n;
    long long ev_begin[kMaxRegions + 1];
    GridH grid[kMaxRegions];
};

// Sampled TOF kernel (Sec. 2.3): n offsets along the line from the TOF point
// (mm) with unit-sum Gaussian weights, an array of (offset, weight) structs.
// n = 0 selects the exact projector.  Passed by value, so the table sits in
// the kernel's constant parameter bank, where a warp reading sample k
// together gets it as one broadcast.
constexpr int kMaxLutSamples = 64;
struct LutH {
    int n;
    float2 s[kMaxLutSamples];  // (offset mm, weight)
};

// Cell binning of the shared-memory tiled pass: grid (n, v, o), cells of cs^3
// voxels (nc per axis), tile = cell widened by h voxels per axis, clipped to the grid.
struct TileH {
    int nx, ny, nz;
    float vx, vy, vz;
    float ox, oy, oz;
    int cs, hx, hy, hz;
    int ncx, ncy, ncz;
    int dir_az, dir_pol;  // direction bins per cell (azimuth x polar; 1 x 1: none)
    unsigned none_code;   // code of events whose window misses the grid (0xFFFFFFFF: left out)
};

enum EventFmt { FMT_F32 = 0, FMT_PACKED = 1 };
enum PassKind { PASS_FUSED = 0, PASS_FORWARD = 1, PASS_BACK = 2 };
enum TailEval { TAIL_FIT = 0, TAIL_ERFC = 1, TAIL_SERIES = 2, TAIL_SERIES4 = 3 };

struct LaunchCfg {
    int threads;       // threads per block (64, 128, 256)
    int blocks_per_sm; // persistent grid when > 0; flat one-event-per-thread grid when 0
    int chunk;         // events per work-queue grab (persistent), multiple of 32
    int cache;         // pieces per thread kept in shared memory for the backprojection (0: walk twice)
    int tail;          // TailEval: how the Gaussian tails are evaluated
    int reduction;     // 0: the linear image; 1: lambda and C in 2x2x2-brick copies (one brick per
                       // 32-byte sector), gathers and scalar reductions at brick-layout indices
};

struct PassArgs {
    const void* events;          // float4 pairs (FMT_F32) or int4 records (FMT_PACKED)
    long long n;
    float lattice;
    const float* lam;            // FP32 image (gather source unless lam_bf16 is set)
    const uint16_t* lam_bf16;    // optional BF16 copy for the forward gather
    float* C;                    // backprojection accumulator
    float* p_out;                // PASS_FORWARD: p_i
    const float* r_in;           // PASS_BACK: r_i
    double* partial;             // PASS_FUSED: kNeffSlots x regions accumulators of sum w_i over events with
                                 // p_i > 0 (zero before the pass; the finalize reads and clears them)
    unsigned long long* work;    // work-queue counter (persistent launches; zero before the launch)
    TofH tof;
    unsigned block_mul;          // flat grids: block b takes the events of block (b * block_mul) mod grid
                                 // (0 or 1: identity); a multiplier coprime with the grid spreads
                                 // region-ordered events over all regions at any moment
    LutH lut;                    // sampled TOF kernel (lut.n > 0) instead of the exact one
    int brick_bx, brick_by;      // > 0: lam and C are in the 2x2x2-brick layout with these bricks per row
                                 // and plane (fused pass over one grid, FP32 gathers)
};

// Voxels of the 2x2x2-brick layout of an nx x ny x nz grid (8 per brick, the
// bricks padding odd extents), and the copies between it and the linear layout:
// brick <- linear, and linear += brick with the brick copy cleared.
long long brick_voxels(int nx, int ny, int nz);
cudaError_t launch_to_bricks(const float* lin, float* br, int nx, int ny, int nz, cudaStream_t s);
cudaError_t launch_from_bricks_add(float* br, float* lin, int nx, int ny, int nz, cudaStream_t s);

// Number of blocks a pass launch uses.
int pass_blocks(const LaunchCfg& cfg, long long n, int num_sms);
cudaError_t launch_pass(PassKind kind, EventFmt fmt, const LaunchCfg& cfg, const PassArgs& a,
                        const RegionTable& tbl, int num_sms, cudaStream_t s);

// Tiled pass (k_tile_pass.cu).  Binning: code[i] = cell id, 0xFFFFFFFF (window misses
// the grid) or 0xFFFFFFFE (fallback); counts[cell] += 1 (zero before), rank[i] = the
// count before event i's increment (its place within the cell); *n_fallback += 1.
cudaError_t launch_cell_codes(const void* ev, int fmt, long long n, float lattice, const TileH& t, float half_window,
                              unsigned* code, unsigned* counts, unsigned* rank, unsigned long long* n_fallback,
                              cudaStream_t st);
// begin[c] = sum of counts before c (n_cells + 1 entries); block_sums: scratch of
// scan_scratch_elems(n_cells) int64.
long long scan_scratch_elems(long long n_cells);
cudaError_t launch_cell_scan(const unsigned* counts, long long n_cells, long long* begin, long long* block_sums,
                             cudaStream_t st);
// Cells with >= min_events events into list[*n_list]; smaller cells' counts are zeroed
// and added to *n_fallback (run before the scan).  Scatter: event i of a kept cell c to
// ev_cell[begin[c] + rank[i]], the fallback events and those of zeroed cells into
// ev_fb (*fb_cursor zero before).
cudaError_t launch_cell_list(unsigned* counts, long long n_cells, unsigned min_events, unsigned* list,
                             unsigned* n_list, unsigned long long* n_fallback, cudaStream_t st);
cudaError_t launch_cell_scatter(const void* ev, int fmt, long long n, const unsigned* code, const long long* begin,
                                const unsigned* rank, void* ev_cell, void* ev_fb, unsigned long long* fb_cursor,
                                cudaStream_t st);
// One block per listed cell: events [begin[c], begin[c+1]) of ev_cell.  Shared memory:
// 2 x tile_voxels floats.  Accumulates C and N_eff (a.partial, one region) like the fused pass.
size_t tile_smem_bytes(const TileH& t);
// lanes: 1 (one thread per event, two sweeps) or 8 (eight lanes per event, one sweep).
cudaError_t launch_tile_pass(const PassArgs& a, const TileH& t, const unsigned* list, unsigned n_list,
                             const long long* begin, int tail, int lanes, cudaStream_t st);

// Grid in FP64 (the sensitivity walk).
struct GridD {
    int nx, ny, nz;
    double vx, vy, vz;
    double ox, oy, oz;
};

// Sensitivity: s[j] += chord length of each LOR's line through the grid, walked and
// accumulated in FP64.  lor6: six planes of n floats (device).
cudaError_t launch_sensitivity(const float* lor6, long long n, const GridD& g, double* s_acc, cudaStream_t st);

// FP32 copy of s64 and per-block FP64 sums of s over {s > 0} in partial[blocks].
cudaError_t launch_sens_finish(const double* s64, long long n_vox, float* s32, double* partial, int blocks,
                               cudaStream_t st);
// lam = s > 0 ? value : 0 over n voxels.
cudaError_t launch_fill_masked(float* lam, const float* s32, long long n_vox, float value, cudaStream_t st);
// Update per region (reg_vox: device array of region voxel offsets, n_regions+1):
// lam <- s > 0 ? lam * C * scale / s : 0; C <- 0; optional BF16 copy; partial[r * bpr + b] = sum s*lam.
// scale: 1 for MLEM, B for an OSEM sub-iteration over one of B subsets.
int update_blocks(long long n_vox);
cudaError_t launch_update(float* lam, float* C, const float* s32, uint16_t* lam_bf16, const long long* reg_vox,
                          int n_regions, double* partial, int blocks_per_region, cudaStream_t st, float scale = 1.f);
// hist[(k * R + r) * 2 + {0,1}] = {N_eff, sum s lambda} of region r after iteration k = *iter; ++*iter.
cudaError_t launch_finalize(double* pass_partial, int pass_slots, const double* upd_partial,
                            int upd_blocks_per_region, int n_regions, double* hist, int* iter_counter,
                            int max_iter, cudaStream_t st);
// Attenuation weights and TOF scatter rejection per resident event (events:
// F32 float4 pairs or packed int4 records, written when apply != 0); w_out and
// keep_out nullable; *kept += number of kept events.
cudaError_t launch_preprocess(void* events, int fmt, long long n, float lattice, const GridH& g, const float* mu,
                              float half_window, int apply, float* w_out, uint8_t* keep_out,
                              unsigned long long* kept, cudaStream_t st);
cudaError_t launch_to_bf16(const float* src, uint16_t* dst, long long n, cudaStream_t st);
// 3x3x3 median (zero outside each region's slab) of in into out per region
// (reg_vox: device array of n_regions + 1 voxel offsets; slabs nx x ny x nz_r,
// max_nz >= every nz_r); s32 (nullable): zero where s <= 0; bf16 (nullable):
// BF16 copy of out.  in and out must not overlap.
cudaError_t launch_median3(const float* in, float* out, const float* s32, uint16_t* bf16, const long long* reg_vox,
                           int n_regions, int nx, int ny, int max_nz, cudaStream_t st);
// Caller SoA planes (device) -> resident float4 pairs; weight nullable.
cudaError_t launch_ingest_f32(const float* const* planes, const float* weight, long long n, float4* out,
                              cudaStream_t st);
cudaError_t launch_ingest_packed(const int4* rec, const float* weight, long long n, int4* out, cudaStream_t st);
// Event weights of the resident records into out[n] (float).
cudaError_t launch_event_weights(const float4* ev_f32, const int4* ev_packed, long long n, float* out, cudaStream_t st);
// Per-block FP64 sums of the event weights in partial[blocks].
cudaError_t launch_reduce_weights(const float4* ev_f32, const int4* ev_packed, long long n, double* partial,
                                  int blocks, cudaStream_t st);
// Stitch (host arrays reg_vox, slab_lo, slab_hi): out = sum of each slab at its slices.
cudaError_t launch_stitch(const float* slabs, const long long* reg_vox, const int* slab_lo, const int* slab_hi,
                          int n_regions, int nx, int ny, int nz, float* out, cudaStream_t st);

// Region division.  counts: n_tiles * (R + 1) ints; offsets: R + 2 int64
// (offsets[R] = total, offsets[R+1] = events in three or more regions);
// base: n_tiles * R int64.
cudaError_t launch_region_codes(const float4* ev_f32, const int4* ev_packed, double lattice, long long n,
                                const double* z_bounds, int n_regions, double shell, uint8_t* codes,
                                int* block_counts, int tile, cudaStream_t st);
cudaError_t launch_region_scan(const int* block_counts, int n_tiles, int n_regions, long long* offsets,
                               long long* block_base, cudaStream_t st);
cudaError_t launch_region_scatter(const uint8_t* codes, long long n, int n_regions, const long long* block_base,
                                  int tile, int* idx, cudaStream_t st);
cudaError_t launch_region_gather(const float4* ev_f32, const int4* ev_packed, const uint8_t* codes,
                                 const int* idx, long long total, float4* out_f32, int4* out_packed,
                                 cudaStream_t st);

// Bounds-checked build: out-of-range voxel indices skipped by the walks of each
// compiled file since the last call (0 in the normal build).
unsigned long long oob_count_event_pass();
unsigned long long oob_count_tile_pass();
unsigned long long oob_count_preprocess();
unsigned long long oob_count_image();

}  // namespace recon
