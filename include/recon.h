/*
 * librecon: list-mode TOF-weighted MLEM on one NVIDIA B300 (sm_103a).
 *
 * The method is that of arXiv:1706.07075 (RPC-PET whole-body reconstruction):
 * list-mode MLEM with a Gaussian time-of-flight (TOF) kernel along each line
 * of response (Sec. 2.3, 2.4) and the TOF-assisted division of the events
 * into body regions reconstructed independently and summed (Sec. 2.5).  The
 * projector uses exact voxel intersections (Siddon) with the Gaussian
 * integrated over each voxel piece.
 *
 * Conventions used by every call
 * -------------------------------
 * Units: mm and ps.  Image layout: FP32 (sensitivity: FP64), x fastest,
 * linear index ix + nx*(iy + ny*iz).  Voxel (ix,iy,iz) covers the half-open
 * box [o + i*v, o + (i+1)*v) per axis; (ox,oy,oz) is the low corner.
 *
 * Event i: endpoints P1 = (x1,y1,z1), P2 = (x2,y2,z2) and TOF offset d in mm,
 * positive toward P1 (d = c (t2 - t1) / 2), so the most likely annihilation
 * point is M + d u with M = (P1 + P2)/2 and u = (P1 - P2)/|P1 - P2|.
 *
 * Ownership: the caller owns every buffer it passes.  Inputs are copied (host
 * pointers) or read (device pointers) during the call only; outputs are
 * written before the call returns (the call synchronises its stream).  Output
 * pointers may be host or device memory: the copy direction is inferred
 * through unified virtual addressing.  The context owns its device images,
 * its resident copy of the events and the sensitivity image.  Device buffers must
 * be ready when a call is made: a call orders its work only after what is already
 * queued on the context's stream (recon_set_stream), so work on other streams that
 * writes an input or uses an output must be complete (or ordered by the caller).
 *
 * Errors: no call aborts or exits.  Every call returns a recon_status; the
 * message of the last failure is available from recon_last_error().  A CUDA
 * failure inside a call returns RECON_ECUDA.  Calls on one context must not
 * overlap (one host thread at a time); different contexts are independent.
 */
#ifndef RECON_H
#define RECON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct recon_ctx recon_ctx;

typedef enum {
    RECON_OK = 0,
    RECON_EINVAL = 1,   /* bad argument: NULL required pointer, n < 0, bad grid, ... */
    RECON_ENOMEM = 2,   /* a device or host allocation failed */
    RECON_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    RECON_ETIMEOUT = 4, /* a bounded device-side wait expired (reserved) */
    RECON_ESTATE = 5    /* call out of order (e.g. MLEM before the sensitivity image) */
} recon_status;

/* Cylindrical scanner (Sec. 2, 2.1: RPC-PET with a long axial field of view). */
typedef struct {
    double radius_mm;           /* > 0 */
    double axial_len_mm;        /* > 0 */
    double max_axial_angle_deg; /* acceptance, (0, 90]; Sec. 2.1 uses 45 */
} recon_geometry;

/* Image grid: nx*ny*nz voxels of (vx,vy,vz) mm, low corner (ox,oy,oz).
 * nx*ny*nz must stay below 2^31. */
typedef struct {
    int32_t nx, ny, nz;
    double vx, vy, vz;
    double ox, oy, oz;
} recon_grid;

typedef enum {
    RECON_EV_F32_SOA = 0,       /* planes[0..6] = x1,y1,z1,x2,y2,z2,d: n floats each */
    RECON_EV_PACKED_I16_F16 = 1 /* planes[0] = n records of 8 x int16: x1,y1,z1,x2,y2,z2 as
                                   multiples of lattice_mm, the FP16 bits of d, 0 (16 bytes each,
                                   16-byte aligned) */
} recon_event_fmt;

typedef struct {
    int32_t fmt;            /* recon_event_fmt */
    int32_t on_device;      /* 1: planes (and weight) are device pointers; 0: host pointers */
    int64_t n;              /* number of events, >= 0 */
    const void* planes[7];  /* see recon_event_fmt; unused entries ignored */
    double lattice_mm;      /* packed format only: lattice step (> 0), e.g. 0.05 */
    const float* weight;    /* optional per-event weight w_i (NULL: all 1), same residency as planes */
} recon_events;

/* One body region: core slice range [z_lo, z_hi) of the image grid (Sec. 2.5). */
typedef struct {
    int32_t z_lo, z_hi;
} recon_region;

/* Launch configuration of the event pass (chosen by the autotuner unless set). */
typedef struct {
    int32_t threads_per_block; /* multiple of 32 in [32, 256] */
    int32_t blocks_per_sm;     /* > 0 (<= 32): persistent grid of SMs x this with a per-warp work
                                  queue; 0: flat grid, one event per thread */
    int32_t chunk_events;      /* events a warp takes from the queue at a time (multiple of 32) */
    int32_t cached_pieces;     /* 0: the backprojection walks each line again; 8..256: the first
                                  walk keeps up to this many (voxel, mass) pieces per event in shared
                                  memory (8 bytes each, threads_per_block * cached_pieces * 8 <= 200 KB)
                                  and the backprojection replays them */
    int32_t tail_eval;         /* Gaussian mass of each piece from the tails erfc(|tau|/(sigma sqrt 2)) at
                                  its two ends, by 0: t exp(-x^2 + P(t)), t = 1/(1 + x/2), with a fitted
                                  degree-10 P (relative error ~6e-7 at K = 3), 1: CUDA's erfcf; or
                                  2: the Taylor series of the integral about the piece's midpoint through
                                  the h^6 term (Hermite polynomials; error below 1e-7 of the window mass
                                  for pieces up to 0.4 sigma); 3: the same series through the h^4 term
                                  (the omitted term is at most 96 h^6 / 322560 of a piece's mass, 1.2e-6
                                  for pieces up to 0.4 sigma).  Without a fixed launch the library uses
                                  2 only when the voxel diagonal is at most 0.5 sigma, else 0; the
                                  autotuner tries 3 where the diagonal is at most 0.4 sigma and K <= 3 */
    int32_t reduction;         /* the MLEM pass with FP32 gathers (recon_mlem; for the exact projector
                                  also recon_mlem_regions, each slab in its own brick copy): 0 the linear image
                                  (exact projector: scalar FP32 reductions; sampled projector: x-adjacent
                                  pairs as red.global.add.v2.f32); 1 lambda and C in 2x2x2-voxel brick
                                  copies (one 32-byte sector per brick), gathers and scalar FP32
                                  reductions at brick-layout indices, so that the nearby lines of a
                                  warp's events share sectors more often (same visits and weights; the
                                  sums run in another order; for the exact projector only with a flat
                                  grid and no piece cache; for the sampled projector the same as
                                  recon_set_brick_layout(1)).
                                  Other passes use 0 */
    int32_t image_tiling;      /* reported by recon_get_launch, ignored by recon_set_launch: 1 when the
                                  last MLEM pass held lambda and C in shared-memory tiles of the event's
                                  cell (recon_set_tiled_pass, or the autotuner's choice), 0 when it read
                                  and reduced into the global image */
    int32_t lanes_per_event;   /* reported by recon_get_launch, ignored by recon_set_launch: threads per
                                  event of the last MLEM pass (1, or 8 in the tiled pass) */
} recon_launch;

typedef struct {
    double sigma_mm;           /* TOF kernel sigma along the LOR */
    double k_sigma;            /* kernel truncation, in sigmas */
    int64_t n_vox;
    int64_t n_events_resident;
    int32_t has_sensitivity;
    int32_t num_sms;
    double sens_total;         /* sum of s_j over {s_j > 0} */
    /* binning of the resident events (all 0 when the last recon_mlem did not bin them):
     * non-empty tiled cells (shared-memory tiled pass only; 0 for the event order), binned
     * events (including those whose window misses the grid, which contribute nothing),
     * events taking the global-memory fallback pass, cell edge in voxels, tile halo per
     * axis in voxels */
    int64_t tile_cells;
    int64_t tile_events;
    int64_t tile_fallback_events;
    int32_t tile_cell_voxels;
    int32_t tile_halo[3];
    int32_t subsets;           /* OSEM subsets of recon_mlem (1: MLEM); conservation rows per iteration */
    int32_t lut_samples;       /* samples of the sampled projector (0: exact projector) */
    int64_t device_bytes;      /* device memory the context holds now (all its buffers; buffers grow
                                  to the largest call and are kept until recon_destroy) */
} recon_info;

typedef struct {
    int64_t kernel_launches;   /* kernels this context launched (graph nodes counted per replay) */
    int64_t pass_launches;     /* event-pass launches with device timing (timing on) */
    double pass_ms;            /* summed device time of those event passes */
    double update_ms;          /* summed device time of the timed updates */
    int64_t autotune_runs;     /* autotuner searches performed */
} recon_stats;

/* ------------------------------------------------------------------ setup */

/* Create a context on the current CUDA device.  sigma = c * FWHM / (2 * 2 sqrt(2 ln 2))
 * with c = 0.299792458 mm/ps (Sec. 2.5 prints sigma = 19.11 mm for 300 ps); the
 * kernel is truncated at +-3 sigma (the ~3 sigma margin of Sec. 2.5) unless
 * recon_set_kernel_window changes it.  Allocates the device images (about
 * 20 bytes per voxel).  Errors: EINVAL (NULL pointers, non-positive sizes,
 * non-finite values, too many voxels), ENOMEM, ECUDA.  *out is NULL on error. */
recon_status recon_create(const recon_geometry* geom, const recon_grid* grid, double tof_fwhm_ps, recon_ctx** out);

/* Release everything the context owns.  NULL-safe. */
void recon_destroy(recon_ctx* ctx);

/* Message of the last failed call on ctx (ctx NULL: of the last failed recon_create or
 * recon_split_regions_noalloc on this thread).  Valid until the next call on the same
 * context. */
const char* recon_last_error(const recon_ctx* ctx);

/* Stream for all device work of ctx (a cudaStream_t; NULL restores the context's own
 * non-blocking stream).  The caller keeps the stream alive while ctx uses it. */
recon_status recon_set_stream(recon_ctx* ctx, void* cuda_stream);

/* Kernel truncation in sigmas, 0.5 <= k <= 8 (default 3). */
recon_status recon_set_kernel_window(recon_ctx* ctx, double k_sigma);

/* Projector of every later forward, backproject, mlem and mlem_regions call on ctx.
 *
 * RECON_PROJ_EXACT (default; n_samples ignored): the Siddon pieces of the line with
 *   the exact TOF mass [Phi(tau_b/sigma) - Phi(tau_a/sigma)] / (2 Phi(K) - 1) of each
 *   piece (Sec. 2.3, Gaussian kernel truncated at +-K sigma).
 * RECON_PROJ_SAMPLED: the paper's own GPU projector (Sec. 2.3, Fig. 3): n_samples
 *   points equally spaced over [-K sigma, K sigma] around the TOF point (the midpoints
 *   of n_samples equal intervals), weights proportional to the Gaussian and summing to
 *   one, each point deposited in the one voxel that contains it.  Sample k of event i
 *   sits at c + t_k u, c = M + d u; its voxel is decided per axis in FP32 as
 *   floor(fma(t_k, u/v, (c - o)/v)) with the operation order the kernel documents.
 *   Points outside the grid are dropped.  The paper uses 32 samples on its GPU and 15
 *   on its CPU.  The sample table travels in the kernel's constant parameter bank.
 *
 * Errors: EINVAL for an unknown projector or n_samples outside
 * [1, RECON_MAX_TOF_SAMPLES].  The sampled projector runs a flat one-event-per-thread
 * grid with the launch's threads_per_block; the other launch fields do not apply. */
#define RECON_PROJ_EXACT 0
#define RECON_PROJ_SAMPLED 1
#define RECON_MAX_TOF_SAMPLES 64
recon_status recon_set_projector(recon_ctx* ctx, int32_t projector, int32_t n_samples);

/* The sampled projector's table as the kernel uses it: *n_out = sample count (0 for
 * the exact projector); offsets_mm[k] (signed distance from the TOF point along u) and
 * weights[k] for k < *n_out, each nullable, caller-owned host arrays of `capacity`
 * floats.  EINVAL (with *n_out set) when capacity is too small. */
recon_status recon_get_tof_samples(const recon_ctx* ctx, int32_t capacity, float* offsets_mm, float* weights,
                                   int32_t* n_out);

/* Event order of the MLEM pass of recon_mlem (either projector, one subset, at least two
 * iterations for a call that passes events) and of recon_mlem_regions.
 *
 * order = 0: the events as loaded.  order = c in [1, 64]: the resident events are binned
 * once by the cell of c^3 voxels that holds their TOF point and processed cell by cell,
 * with the cells spread over the blocks that run at the same time (block b of the grid
 * takes block (b * m) mod n of the binned list, m coprime with n): a warp's lines start in
 * one cell (nearby voxels), while concurrent blocks work far apart (no hot voxels).
 * order = -1: cells of 4^3 voxels.  azimuth_bins x polar_bins (each in [1, 64]; 1 x 1:
 * none) further split each cell by the direction of the line (folded so that u_x >= 0:
 * azimuth over (-90, 90] degrees, polar over u_z in [-1, 1]), so that a warp's lines also
 * run alike.  Default: order -1 with 16 x 8 direction bins (with the brick copies,
 * 32 x 16 bins make the full-body pass 1.1% faster, but their 4x larger key table costs
 * an end-to-end job more in binning than its iterations gain).  Same arithmetic; the sums run
 * in another order.  The binning costs one copy of the events and is cached with them (a
 * call that passes host events bins them after its first, upload-overlapped pass).
 * Measured on B300, 146 M full-body events, series piece masses: 47.6 ms per pass in load
 * order, 35.5 ms with 3^3-voxel cells (about the same for edges of 1 to 10 voxels),
 * 31.5-31.9 ms with 16 x 8 or 32 x 16 direction bins as well (31.2 ms in the current
 * library, which sums N_eff per warp).  Errors: EINVAL (order
 * outside [-1, 64], bins outside [1, 64]). */
recon_status recon_set_event_order(recon_ctx* ctx, int32_t order, int32_t azimuth_bins, int32_t polar_bins);

/* Shared-memory tiled event pass for recon_mlem (off by default).  A layout choice for
 * the same arithmetic (Sec. 2.3, 2.4), with no counterpart in the paper: the resident
 * events are binned once by the cell (cs^3 voxels) that holds their TOF point; one block
 * per cell holds the cell's tile of lambda and of C (the cell widened by the TOF window,
 * K sigma |u_k| per axis, |u_z| bounded by the scanner's max axial angle) in shared
 * memory, walks the cell's events with eight lanes per event, and adds its C tile into
 * the image.  Events whose window would leave their tile take the global-memory pass.
 * Used for MLEM with the exact projector and one subset when two tiles fit the shared
 * memory of a block (e.g. 4 mm voxels at 300 ps); otherwise every event takes the
 * global-memory pass.  on = 0 returns to the default cell order (recon_set_event_order -1).  A cell is tiled only when it holds at least m events
 * (loading and flushing a tile costs about as much as a few hundred events): on = 1 sets
 * m = 256, on > 1 sets m = on; the events of smaller cells take the global-memory pass.
 * lanes: threads per event, 1 (each thread walks its event twice, forward then back) or
 * 8 (eight lanes split the window and keep their pieces in registers).
 * Measured on B300 with 146 M full-body events it is slower than the global-memory pass
 * (59-88 ms against 48 ms per pass): the lines of a cell's events all cross the cell, so
 * the shared-memory reductions of a block pile onto the same voxels.  It stays available
 * for denser data (more events per cell) and as a tested alternative.
 * The binning costs one copy of the events (32 or 16 bytes each) and is cached until the
 * events, the kernel window or m change.  recon_get_info reports the binning.  Errors:
 * EINVAL (on < 0, lanes not 1 or 8). */
recon_status recon_set_tiled_pass(recon_ctx* ctx, int32_t on, int32_t lanes);

/* Start image of recon_mlem when init is NULL.  mode 0 (default): uniform on {s_j > 0}
 * with sum_j s_j lambda_j = sum_i w_i.  mode 1: the starting backprojection that seeds
 * the paper's MLEM (Sec. 3.5.4, Table 2), read as lambda0_j = (sum_i a_ij w_i) / s_j on
 * {s_j > 0} (the events' TOF-weighted backprojection over the sensitivity; the paper does
 * not give its normalisation).  Mode 1 needs all events before the first iteration, so a
 * call with host events then uploads them first instead of overlapping the upload with the
 * first pass.  Errors: EINVAL (mode not 0 or 1). */
recon_status recon_set_start_image(recon_ctx* ctx, int32_t mode);

/* List-mode OSEM for recon_mlem (OSEM is named in the title of Sec. 2.4; the paper
 * itself reconstructs with MLEM).  n_subsets = B > 1: each iteration runs B
 * sub-iterations; sub-iteration b uses the events of block b of the list,
 * [b n / B, (b+1) n / B) (list-mode events arrive in random order, so the blocks are
 * random partitions), and updates lambda_j <- lambda_j C_j^b / (s_j / B).  B = 1 (the
 * default) is MLEM.  recon_mlem_regions always runs MLEM.  The median sieve, when on,
 * runs once per iteration, after the last subset.  Errors: EINVAL (B outside
 * [1, 1024]). */
recon_status recon_set_subsets(recon_ctx* ctx, int32_t n_subsets);

/* Median-filter sieve between iterations (Sec. 2.4; Sec. 4 on its effect at the
 * borders of divided images).  on = 1: after every iteration's update of recon_mlem
 * and recon_mlem_regions, lambda is replaced by its 3 x 3 x 3 median (the 14th
 * smallest of the 27 values, neighbours outside the grid or the region's slab
 * counting as 0) and voxels with s_j = 0 are set to 0.  The conservation history
 * keeps N_eff and sum_j s_j lambda_j of the update, before the filter (the filter does
 * not conserve counts).  Off by default. */
recon_status recon_set_median_filter(recon_ctx* ctx, int32_t on);

/* One 3 x 3 x 3 median filter of image_in into image_out over the context's grid,
 * zero outside the grid, no mask (nx*ny*nz floats each, host or device; they may
 * alias).  Values must not be NaN.  Errors: EINVAL (NULL pointer), ENOMEM, ECUDA. */
recon_status recon_median_filter(recon_ctx* ctx, const float* image_in, float* image_out);

/* Forward gather from a BF16 copy of the image (1) or the FP32 image (0, default).
 * Backprojection always accumulates in FP32. */
recon_status recon_set_gather_bf16(recon_ctx* ctx, int32_t on);

/* Image layout of the sampled projector's MLEM pass (recon_mlem with RECON_PROJ_SAMPLED,
 * FP32 gathers): 0 (default) the linear layout; 1 copies of lambda and C in 2x2x2-voxel
 * bricks, one 32-byte sector per brick, so that the samples of a warp's nearby lines share
 * sectors more often (fewer L2 requests, more L1 hits).  Each pass then
 * copies lambda into the bricks before and adds the brick copy of C into C after.  Same
 * visits and weights as the linear pass; the sums run in another order.  Not used by the
 * exact projector, with BF16 gathers, by recon_mlem_regions or by the first pass of a
 * call that streams host events.  Costs two device images of 8 ceil(nx/2) ceil(ny/2)
 * ceil(nz/2) floats.  EINVAL if on is not 0 or 1, or that count exceeds 2^31. */
recon_status recon_set_brick_layout(recon_ctx* ctx, int32_t on);

/* Fix the event-pass launch (NULL: return to the autotuner).  EINVAL if invalid. */
recon_status recon_set_launch(recon_ctx* ctx, const recon_launch* cfg);
/* The launch the last event pass used. */
recon_status recon_get_launch(const recon_ctx* ctx, recon_launch* out);

/* Per-call device timing of event passes and updates into recon_stats (off by default).
 * While on, iterations are launched one by one with CUDA events around each kernel. */
recon_status recon_set_timing(recon_ctx* ctx, int32_t on);
/* Capture each MLEM iteration in a CUDA graph and replay it (1, default) or launch
 * kernels directly (0). */
recon_status recon_set_graphs(recon_ctx* ctx, int32_t on);
/* Let recon_mlem / recon_mlem_regions search launch configurations of the event pass
 * on the resident events the first time they meet a new (event count, format, voxel
 * count, region count, event order, projector) with at least 2^20 events (1, default),
 * or use the default launch (0).  Candidates: threads per block,
 * flat or persistent grid, piece cache, piece-mass form and reduction form (scalar
 * into the linear image, or into 2x2x2-brick copies of lambda and C; the latter with FP32
 * gathers, one brick copy per region slab), 19 in all, each timed over two passes (the
 * brick candidates with their copy kernels).  For the sampled projector: 128, 192 or 256
 * threads per block, each with the linear image or the brick copies.  recon_mlem in the default event order
 * then also times the shared-memory tiled pass (recon_set_tiled_pass) with 1 and 8
 * threads per event against the best of those, where tiles fit (exact projector, one
 * subset, FP32 gathers), and keeps the faster image layout for the key.  C and the
 * N_eff sums are cleared afterwards, so the search changes no result;
 * recon_get_launch reports every chosen dimension. */
recon_status recon_set_autotune(recon_ctx* ctx, int32_t on);

/* Failure injection for testing how callers and the library handle an exhausted
 * device (the paper has no counterpart).  n > 0: the n-th device allocation the
 * library attempts from now on (n = 1: the next one), in any context and on any
 * thread, fails as if the device were out of memory: nothing is allocated and the
 * call that needed it returns RECON_ENOMEM with a message naming the allocation.
 * n = 0 disarms.  Only the host side is affected: no kernel runs or faults for it.
 * A call that fails this way leaves the context usable: a buffer that could not grow
 * keeps its old allocation, and state that was being replaced (resident events, the
 * sensitivity image, cached binnings and graphs) is dropped, so later calls rebuild
 * it or return RECON_ESTATE.  The device allocations of recon_split_regions_noalloc
 * do not exist and are not counted.  Errors: EINVAL (n < 0). */
recon_status recon_debug_fail_alloc(int64_t n);

/* Out-of-range accesses caught by the bounds-checked build of this library
 * (librecon_check.so, compiled with RECON_BOUNDS_CHECK; the paper has no counterpart):
 * every voxel index a walk produces (event passes, the tiled pass, pre-processing, the
 * sensitivity) is checked against its image before use, and an index outside is counted
 * and its walk ended instead of reading or writing out of range.  *count_out receives
 * the number counted on the current device since the last call (and clears it), or -1
 * in the normal build, which has no checks.  The check build stands in for a memory
 * sanitizer, with no trap and no fault.  Errors: EINVAL (NULL count_out). */
recon_status recon_debug_bounds_violations(int64_t* count_out);

recon_status recon_get_info(const recon_ctx* ctx, recon_info* out);
recon_status recon_get_stats(const recon_ctx* ctx, recon_stats* out);
recon_status recon_reset_stats(recon_ctx* ctx);

/* ------------------------------------------------------------ sensitivity */

/* Sensitivity image s_j = sum_l L_lj: the full chord length (mm) of each of the n
 * lines through voxel j, no TOF, accumulated in FP64 (Sec. 2.4, the "sensitive
 * matrix").  lor: 6 planes x1,y1,z1,x2,y2,z2 of n floats each, contiguous
 * (plane k at lor + k*n); host (on_device = 0) or device (1).  sens_out: NULL or
 * nx*ny*nz doubles (host or device) receiving s.  The mask {s_j > 0} is the
 * support of every later image.  Errors: EINVAL (n < 0, NULL lor with n > 0). */
recon_status recon_sensitivity(recon_ctx* ctx, const float* lor, int64_t n, int32_t on_device, double* sens_out);

/* Use a given sensitivity image (nx*ny*nz doubles, host or device per on_device). */
recon_status recon_set_sensitivity(recon_ctx* ctx, const double* sens, int32_t on_device);

/* ------------------------------------------------------------------ events */

/* Copy the events into the context's resident device layout (32 bytes per event for
 * the F32 format, 16 for the packed one); they stay resident for later calls that pass
 * events = NULL.  Errors: EINVAL (bad format, n < 0, NULL planes, lattice <= 0),
 * ENOMEM. */
recon_status recon_load_events(recon_ctx* ctx, const recon_events* events);

/* Event pre-processing (Sec. 2.2, 2.4), one pass over the events on the GPU.
 *
 * Attenuation correction (Sec. 2.4): w_i = exp(sum_j mu_j L_ij), the integral of the
 *   attenuation map along the event's whole LOR inside the grid (L_ij: Siddon chord
 *   of the LOR in voxel j), i.e. inversely proportional to the probability that the
 *   photon pair escapes attenuation.
 * TOF scatter rejection (Sec. 2.2, Fig. 2): with z_reject > 0 an event is kept iff
 *   the stretch of its LOR within z_reject * sigma of the TOF point meets a body voxel
 *   (mu_j > 0) over a positive length; z_reject = 1.96 is the paper's 95% confidence.
 *   Rejected events get w_i = 0.  z_reject = 0 keeps every event.
 *
 * events: NULL = the resident events, else loaded first (and kept resident).
 * mu_map: nx*ny*nz floats (1/mm, >= 0, host or device).
 * apply = 1: multiply the resident events' weights by w_i in place (rejected events
 *   then weigh 0; the packed format stores the product in FP16, relative rounding
 *   ~5e-4), so later recon_mlem / recon_mlem_regions calls with events = NULL use
 *   them; apply = 0 leaves the events unchanged.
 * weight_out (n floats), keep_out (n bytes, 1 = kept), n_kept: nullable outputs, host
 * or device.  Errors: EINVAL (NULL mu_map, z_reject outside [0, 10]), ESTATE (no
 * events), ENOMEM, ECUDA. */
recon_status recon_preprocess(recon_ctx* ctx, const recon_events* events, const float* mu_map, double z_reject,
                              int32_t apply, float* weight_out, uint8_t* keep_out, int64_t* n_kept);

/* ---------------------------------------------------------------- projector */

/* Forward projection p_i = sum_j a_ij lambda_j (Sec. 2.3/2.4) with
 * a_ij = [Phi(tau_b/sigma) - Phi(tau_a/sigma)] / (2 Phi(K) - 1) over the piece
 * [tau_a, tau_b] of the LOR inside voxel j and inside +-K sigma of the TOF point
 * (RECON_PROJ_EXACT), or the summed weights of the samples in voxel j
 * (RECON_PROJ_SAMPLED; see recon_set_projector).
 * events: NULL = the resident events, else loaded first (and kept resident).
 * image: nx*ny*nz floats (host or device); NULL = the context's current image.
 * p_out: n floats (host or device).  Errors: EINVAL, ESTATE (no events). */
recon_status recon_forward(recon_ctx* ctx, const recon_events* events, const float* image, float* p_out);

/* Backprojection C_j = sum_i a_ij r_i of per-event values r (n floats, host or
 * device) into image_out (nx*ny*nz floats, host or device). */
recon_status recon_backproject(recon_ctx* ctx, const recon_events* events, const float* r, float* image_out);

/* -------------------------------------------------------------------- MLEM */

/* n_iter iterations of list-mode TOF-MLEM (Sec. 2.4):
 *     p_i = sum_j a_ij lambda_j;  C_j = sum_{i: p_i > 0} a_ij w_i / p_i;
 *     lambda_j <- lambda_j C_j / s_j on {s_j > 0}, 0 elsewhere.
 * Start image: init (nx*ny*nz floats, host or device) if not NULL, else uniform on
 * {s_j > 0} with sum_j s_j lambda_j = sum_i w_i.  image_out: NULL or nx*ny*nz floats
 * receiving the final image (the image also stays in the context).
 * conservation_out: NULL or n_iter x 2 doubles {N_eff, sum_j s_j lambda_j} after each
 * iteration, FP64 sums (N_eff = sum of w_i over events with p_i > 0); the two agree up
 * to FP32 rounding of the image (count conservation).  With B OSEM subsets
 * (recon_set_subsets) there are n_iter x B rows, one per sub-iteration, and
 * sum_j s_j lambda_j = B N_eff of that subset.
 * Errors: EINVAL (n_iter < 0, n_iter x B > 2^24), ESTATE (no sensitivity image or no
 * events). */
recon_status recon_mlem(recon_ctx* ctx, const recon_events* events, int32_t n_iter, const float* init,
                        float* image_out, double* conservation_out);

/* ------------------------------------------------ one iteration, in parts */

/* One MLEM event pass (Sec. 2.4) over the resident events, for callers that combine
 * the passes of several contexts before the update: ranks of a job whose events are
 * sharded over GPUs sum their C images (one all-reduce per iteration) and each then
 * calls recon_update with the sum.
 *     p_i = sum_k a_ik lambda_k,   C_j = sum_{i: p_i > 0} a_ij w_i / p_i.
 * events: NULL = the resident events, else loaded first (and kept resident).
 * lambda: with from_start = 1 the image 1 on {s_j > 0} (MLEM's first update from any
 * uniform start gives the same image, so the ranks need not agree on a start value);
 * else `image` (nx*ny*nz floats, host or device) when not NULL, else the context's
 * current image.  The image stays in the context for recon_update.
 * C_out: nx*ny*nz floats (host or device) receiving C.  n_eff_out (nullable): FP64 sum
 * of w_i over the events with p_i > 0.  Projector, event order, launch and BF16
 * gathers as for recon_mlem.  Errors: EINVAL (NULL C_out, OSEM subsets set), ESTATE
 * (no events or no sensitivity image). */
recon_status recon_event_pass(recon_ctx* ctx, const recon_events* events, const float* image, int32_t from_start,
                              float* C_out, double* n_eff_out);

/* The MLEM update of the context's image from a correction image (Sec. 2.4):
 * lambda_j <- lambda_j C_j / s_j on {s_j > 0}, 0 elsewhere, followed by the median
 * sieve when it is on (recon_set_median_filter).
 * C_in: nx*ny*nz floats (host or device), e.g. the sum of the ranks' recon_event_pass
 * outputs.  image_out (nullable): nx*ny*nz floats (host or device) receiving the new
 * image.  sum_s_lambda_out (nullable): sum_j s_j lambda_j in FP64, before the sieve.
 * Errors: EINVAL (NULL C_in), ESTATE (no sensitivity image). */
recon_status recon_update(recon_ctx* ctx, const float* C_in, float* image_out, double* sum_s_lambda_out);

/* ------------------------------------------------------ region division */

/* TOF-assisted division into body regions (Sec. 2.5, Fig. 4).  Regions are
 * consecutive core slice ranges (regions[r].z_hi == regions[r+1].z_lo) inside
 * [0, nz), each at least 2*shell_mm thick; core boundaries z_b[r] = oz + z_lo*vz.
 * Each event's TOF-estimated z, z_tof = (z1+z2)*0.5 + (d*dz)/D with
 * D = sqrt((dx*dx + dy*dy) + dz*dz) in FP64 rounded per operation, decides the
 * regions: r takes the event iff z_b[r] - shell <= z_tof < z_b[r+1] + shell.
 * events: NULL = the resident events (in the order they were loaded), else loaded
 * first (and kept resident).
 * Outputs (host or device, each nullable):
 *   code_out:    n bytes; 0xFF no region, r one region, r|0x80 regions r and r+1;
 *   offsets_out: n_regions+1 int64, start of each region's list in idx_out;
 *   idx_out:     offsets_out[n_regions] int32 event indices, ascending within a region.
 * 1 <= n_regions <= 64, n < 2^31.  margin_mm is only validated here (>= 0).
 * Errors: EINVAL, ESTATE (no events). */
recon_status recon_split_regions(recon_ctx* ctx, const recon_events* events, int32_t n_regions,
                                 const recon_region* regions, double margin_mm, double shell_mm,
                                 uint8_t* code_out, int64_t* offsets_out, int32_t* idx_out);

/* Region-divided reconstruction (Sec. 2.5): split as recon_split_regions (events:
 * NULL = the resident events), give each event fed to two regions the weight w_i/2,
 * reconstruct every region on its slab of slices [z_lo - m, z_hi + m) clipped to the
 * grid, m = ceil(margin_mm / vz), with the global sensitivity restricted to the slab,
 * and the start image uniform on each slab's {s_j > 0} with sum s lambda = the sum of
 * its events' weights; then sum the slabs into image_out
 * (nx*ny*nz floats, nullable).  All regions run in one event-pass launch per
 * iteration.  region_images_out: NULL or the concatenated slab images (region order,
 * each nx*ny*slab_nz floats; total from recon_region_slab_voxels).
 * conservation_out: NULL or n_iter x n_regions x 2 doubles {N_eff, sum s lambda}.
 * Errors: EINVAL, ESTATE (no sensitivity image or no events). */
recon_status recon_mlem_regions(recon_ctx* ctx, const recon_events* events, int32_t n_regions,
                                const recon_region* regions, double margin_mm, double shell_mm, int32_t n_iter,
                                float* image_out, float* region_images_out, double* conservation_out);

/* Block of regions for later recon_mlem_regions calls: only regions [first, first +
 * count) of the division are reconstructed (count = 0, first = 0: all, the default).
 * The split still uses every region, so an event shared with a region outside the
 * block keeps its weight 1/2 (Sec. 2.5); the pass walks only the block's events, the
 * other regions' slab images start and stay at 0, and image_out holds the block's
 * slabs only.  For jobs whose regions are divided over ranks: the sum of the ranks'
 * images is the whole-body image.  Errors: EINVAL (block outside [0, 64), or count 0
 * with first != 0; a block past the division's last region fails in
 * recon_mlem_regions). */
recon_status recon_set_region_block(recon_ctx* ctx, int32_t first, int32_t count);

/* Total voxels of the region slabs of a division (for sizing region_images_out). */
recon_status recon_region_slab_voxels(const recon_ctx* ctx, int32_t n_regions, const recon_region* regions,
                                      double margin_mm, int64_t* n_vox_out);

/* ------------------------------------------------- allocation-free split */

/* The paper has no counterpart of this call: it is a service for callers that cannot
 * allocate device memory.  A process whose GPU memory belongs to another allocator (a
 * framework's caching pool, or an acquisition service that reserves all of the GPU's
 * memory when it starts) would see an extra cudaMalloc fail or fragment a pool it does
 * not own; a real-time path cannot afford cudaFree, which waits for the whole device, or
 * an allocation that may fail half-way through a scan.
 *
 * Same split as recon_split_regions (same codes, offsets and ascending index lists),
 * with no context and no cudaMalloc/cudaFree: the caller passes device inputs and
 * outputs, and the per-tile counters live in one 8 MiB static device array that every
 * GPU loading this library keeps until the process exits.
 *   grid:        only nz, vz and oz are used (the z boundaries z_b[r] = oz + z_lo*vz).
 *   events:      fmt RECON_EV_F32_SOA with on_device = 1 (the weight is ignored); each
 *                plane holds n floats in device memory of the current device.
 *   code_out:    n bytes, device.      idx_out: idx_capacity int32, device.
 *   offsets_out: n_regions+1 int64, host.
 *   cuda_stream: the stream to run on (NULL: the legacy default stream).  The call
 *                reads the offsets back to the host and synchronises that stream
 *                before it returns.
 * Limit: n <= 32768 * floor((8 MiB - 1032 B) / (12 * n_regions + 4)) events and n < 2^31
 * (any n below 2^31 for up to 10 regions, about 356 M events for 64); larger n returns
 * RECON_EINVAL with a message.  Every event plane, code_out and idx_out must be device
 * (or managed) memory of the current device: host memory, page-locked or not, returns
 * RECON_EINVAL before any kernel runs.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and each overwrites what the previous call left there, so
 * calls that overlap on the GPU (other host threads, other streams) race and must be
 * serialised by the caller.  Errors: EINVAL (arguments, memory residency, limit, idx_out
 * too small), ECUDA; the message is available from recon_last_error(NULL). */
recon_status recon_split_regions_noalloc(const recon_grid* grid, const recon_events* events, int32_t n_regions,
                                         const recon_region* regions, double shell_mm, uint8_t* code_out,
                                         int64_t* offsets_out, int32_t* idx_out, int64_t idx_capacity,
                                         void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RECON_H */
