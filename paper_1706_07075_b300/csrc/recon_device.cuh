// Device-side building blocks of the list-mode TOF-MLEM projector for sm_103a.
//
// Geometry (Sec. 2.3 of arXiv:1706.07075, "TOF kernel"; exact voxel
// intersections after Siddon): event i has endpoints P1, P2, unit direction
// u = (P1 - P2)/|P1 - P2|, midpoint M and TOF offset d, so the most likely
// annihilation point is c = M + d u.  The walker parameterises the line by
// tau = t - d, the signed distance from c, which keeps every kernel argument
// small (|tau| <= K sigma) and FP32-precise.  Voxel (ix,iy,iz) is the
// half-open box [o + i v, o + (i+1) v); linear index ix + nx (iy + ny iz).
//
// System element of a voxel piece [tau_a, tau_b] (Sec. 2.3: Gaussian kernel
// whose weights sum to one; truncated at +-K sigma and renormalised):
//     a = [Phi(tau_b/sigma) - Phi(tau_a/sigma)] / (2 Phi(K) - 1).
// It is evaluated from signed tails g(tau) = sign(tau) erfc(|tau|/(sigma
// sqrt 2)):  Phi(b) - Phi(a) = ((s_b - s_a) + (g_a - g_b)) / 2, which keeps
// full FP32 relative precision in both tails of the window.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "recon_kernels.h"
#include "tail_fit.h"

namespace recon {

// Bounds-checked build (RECON_BOUNDS_CHECK, librecon_check.so): every voxel index a
// walk produces is checked against its image before it is used; an index outside is
// counted here and its walk ends, so nothing is read or written out of range.  One
// counter per compiled file (internal linkage); oob_take() reads and clears it.
#ifdef RECON_BOUNDS_CHECK
static __device__ unsigned long long g_oob_count;
static inline unsigned long long oob_take()
{
    unsigned long long v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_oob_count, sizeof v) != cudaSuccess) v = ~0ULL;
    cudaMemcpyToSymbol(g_oob_count, &zero, sizeof zero);
    return v;
}
__device__ __forceinline__ bool index_ok(long long j, long long limit)
{
    if (j >= 0 && j < limit) return true;
    atomicAdd(&g_oob_count, 1ULL);
    return false;
}
#else
static inline unsigned long long oob_take() { return 0; }
#endif

using GridDev = GridH;
using TofDev = TofH;

// Event as the walker sees it.
struct Event {
    float3 p1, p2;
    float d, w;
};

// Resident F32 layout: two float4 per event, (x1,y1,z1,d) and (x2,y2,z2,w),
// so a thread's event arrives in two 16-byte loads and a warp's in 1 KB.
__device__ __forceinline__ Event load_event_f32(const float4* __restrict__ ev, long long i)
{
    float4 a = __ldg(ev + 2 * i);
    float4 b = __ldg(ev + 2 * i + 1);
    Event e;
    e.p1 = make_float3(a.x, a.y, a.z);
    e.p2 = make_float3(b.x, b.y, b.z);
    e.d = a.w;
    e.w = b.w;
    return e;
}

// Packed layout: 16 bytes per event, int16 endpoints on a lattice, FP16 d,
// FP16 weight: one 16-byte load per thread.
__device__ __forceinline__ Event load_event_packed(const int4* __restrict__ ev, long long i, float lattice)
{
    int4 r = __ldg(ev + i);
    Event e;
    e.p1 = make_float3((float)(short)(r.x & 0xFFFF) * lattice, (float)(short)(r.x >> 16) * lattice,
                       (float)(short)(r.y & 0xFFFF) * lattice);
    e.p2 = make_float3((float)(short)(r.y >> 16) * lattice, (float)(short)(r.z & 0xFFFF) * lattice,
                       (float)(short)(r.z >> 16) * lattice);
    e.d = __half2float(__ushort_as_half((unsigned short)(r.w & 0xFFFF)));
    e.w = __half2float(__ushort_as_half((unsigned short)((unsigned)r.w >> 16)));
    return e;
}

// Signed tail of the Gaussian at tau: g = sign(tau) * erfc(|tau| / (sigma sqrt 2)).
struct Tail {
    float g, s;
};

// Tail from CUDA's erfcf.
struct TailErfc {
    static constexpr bool kPiecewise = false;
    static constexpr bool kSigmaUnits = false;
    static constexpr float kMassScale = 1.f;
    float inv_sigma_sqrt2;
    __device__ __forceinline__ Tail operator()(float tau) const
    {
        Tail t;
        t.s = copysignf(1.f, tau);
        t.g = copysignf(erfcf(fabsf(tau) * inv_sigma_sqrt2), tau);
        return t;
    }
};

// Tail from the fitted-exponent form of erfc (Press et al., Numerical
// Recipes, Sec. 6.2): erfc(x) ~ t exp(-x^2 + P(t)), t = 1/(1 + x/2), with a
// degree-10 polynomial P fitted for 0 <= x <= 8/sqrt 2 by gen_tail_fit.py
// (tail_fit.h).  -x^2 is split into a rounded product and its FMA remainder
// so the large exponent keeps its precision.  Relative error about 6e-7 for
// K = 3 (2e-6 at K = 8), from ~20 FP32 operations and two MUFU operations.
struct TailFit {
    static constexpr bool kPiecewise = false;
    static constexpr bool kSigmaUnits = false;
    static constexpr float kMassScale = 1.f;
    float inv_sigma_sqrt2;
    __device__ __forceinline__ Tail operator()(float tau) const
    {
        const float x = fabsf(tau) * inv_sigma_sqrt2;
        const float t = __fdividef(1.f, fmaf(0.5f, x, 1.f));
        const float s = fmaf(t, kTailFitInvHalf, -kTailFitMidOverHalf);
        const float p = tail_fit_poly(s);
        const float e_hi = -x * x;
        const float e_lo = fmaf(-x, x, -e_hi);
        const float f = t * __expf(e_hi + p) * (1.f + e_lo);
        Tail r;
        r.s = copysignf(1.f, tau);
        r.g = copysignf(f, tau);
        return r;
    }
};

// 2^x by the PTX instruction ex2.approx.ftz.f32 (documented maximum relative error
// about 2^-22 over the range used here; subnormal results flush to zero).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Piece mass from the Taylor expansion of the Gaussian integral about the
// piece's midpoint (derivatives of phi are Hermite polynomials He_n times phi):
//   Phi(b) - Phi(a) = h phi(m) [1 + He_2(m) h^2/24 + He_4(m) h^4/1920
//                               + He_6(m) h^6/322560 + ...]
// with h = b - a and m = (a + b)/2 in sigma units.  For pieces up to 0.4 sigma
// (4 mm voxels at 300 ps: at most 0.36 sigma) the first omitted term is below
// 1e-7 of the piece's mass over the +-3 sigma window.  One exponential per
// piece and no carried boundary value; walk() calls piece() instead of
// differencing two tails.
// Through6 = false stops at the h^4 term: the omitted He_6(m) h^6 / 322560 is at
// most 96 (0.36)^6 / 322560 = 6.5e-7 of the piece's own mass for 4 mm voxels
// (|He_6| <= 96 on [0, 3]), about the FP32 rounding of the sum.
//
// The walk runs in sigma units for this form (kSigmaUnits: the event pass scales
// the walk's crossings by 1/sigma once per event), and the polynomials are written
// in M = a + b = 2m, Q = M^2 = 4 m^2, so that each coefficient is one chain of
// FMAs:  He_2(m)/24 = Q/96 - 1/24,  He_4(m)/1920 = Q^2/30720 - Q/1280 + 1/640,
// He_6(m)/322560 = Q^3/20643840 - Q^2/344064 + Q/28672 - 1/21504, and
// exp(-m^2/2) = 2^(-Q log2(e) / 8).  piece() returns h P exp(-m^2/2); the factor
// sqrt(2/pi) that makes it 2 [Phi(b) - Phi(a)], what the tail forms return, is
// kMassScale, applied once per event with the window normalisation.
template <bool Through6>
struct TailSeriesT {
    static constexpr bool kPiecewise = true;
    static constexpr bool kSigmaUnits = true;
    static constexpr float kMassScale = 0.7978845608f;   // sqrt(2/pi)
    float inv_sigma_sqrt2;
    __device__ __forceinline__ Tail operator()(float) const { return Tail{0.f, 0.f}; }
    __device__ __forceinline__ float inv_sigma() const { return inv_sigma_sqrt2 * 1.41421356f; }
    __device__ __forceinline__ float piece(float ta, float tb) const
    {
        const float h = tb - ta;
        const float M = ta + tb;
        const float Q = M * M;
        const float h2 = h * h;
        const float c1 = fmaf(Q, 1.f / 96.f, -1.f / 24.f);
        const float c2 = fmaf(fmaf(Q, 1.f / 30720.f, -1.f / 1280.f), Q, 1.f / 640.f);
        float poly;
        if constexpr (Through6) {
            const float c3 = fmaf(fmaf(fmaf(Q, 1.f / 20643840.f, -1.f / 344064.f), Q, 1.f / 28672.f), Q,
                                  -1.f / 21504.f);
            poly = fmaf(h2, fmaf(h2, fmaf(h2, c3, c2), c1), 1.f);
        } else {
            poly = fmaf(h2, fmaf(h2, c2, c1), 1.f);
        }
        return h * poly * ex2_approx(Q * -0.18033688011f);   // log2(e) / 8
    }
};
using TailSeries = TailSeriesT<true>;
using TailSeries4 = TailSeriesT<false>;

// Per-event walk state after clipping the line to the grid box and the TOF
// window.  Everything the two sweeps (forward, back) need is here.
struct Walk {
    float tau_in, tau_out;    // clipped parameter range (relative to c)
    int j0;                   // linear index of the start voxel
    int sxl, syl, szl;        // linear-index step per axis (+-1, +-nx, +-nx*ny, or 0)
    float t0x, t0y, t0z;      // tau of the first plane crossing per axis (inf if none inside the grid)
    float dtx, dty, dtz;      // tau between successive crossings per axis
    float rx, ry, rz;         // crossings per axis that stay inside the grid
    int ix0, iy0, iz0;        // start voxel per axis
    bool valid;
};

// tau_out lowered to the first crossing past each axis's budget, computed as the
// walk computes its crossings: after r_k crossings on axis k the walk's next
// crossing there is fmaf(r_k, dt_k, t0_k), and fmaf is monotone in its first
// argument (dt_k > 0), so every crossing past the budget lies at or beyond tau_out
// and the walk ends before it steps out of the grid.  This replaces a budget test
// per piece and axis.  Within the grid the exit crossing and the clipped tau_out
// agree up to rounding.  An axis with no crossing has t0 = inf; a NaN exit (an
// infinite spacing) is ignored by fminf, and such an axis is stepped at most once.
__device__ __forceinline__ void clip_to_budgets(Walk& w)
{
    const float ex = w.rx > 0.f ? fmaf(w.rx, w.dtx, w.t0x) : w.t0x;
    const float ey = w.ry > 0.f ? fmaf(w.ry, w.dty, w.t0y) : w.t0y;
    const float ez = w.rz > 0.f ? fmaf(w.rz, w.dtz, w.t0z) : w.t0z;
    w.tau_out = fminf(w.tau_out, fminf(ex, fminf(ey, ez)));
}

// The walk's parameter rescaled by s (tau -> s tau): clip range, first crossings
// and crossing spacings; infinities stay infinite.  The voxel sequence and the
// crossing counts do not change; the budget clip is taken again on the scaled
// values, which the walk then steps with.
__device__ __forceinline__ void scale_walk(Walk& w, float s)
{
    w.tau_in *= s;
    w.tau_out *= s;
    w.t0x *= s;
    w.t0y *= s;
    w.t0z *= s;
    w.dtx *= s;
    w.dty *= s;
    w.dtz *= s;
    clip_to_budgets(w);
}

// The TOF point c = M + d u of an event as an unevaluated sum c + c_lo of two
// FP32 numbers.  FP32 alone rounds c to ulp(|c|), ~6e-5 mm at 1 m; a line nearly
// parallel to a voxel plane that passes closer than that to the plane would land
// on the wrong side of it for much of its window.  The pair keeps c to ~1e-11 mm
// relative to the planes (error-free sums and products, Dekker and Knuth; the
// __f*_rn intrinsics keep the compiler from fusing them).
struct Line {
    float3 c, c_lo, u;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// c + c_lo = (p1 + p2) / 2 + d u along one axis.
__device__ __forceinline__ void tof_point_axis(float p1, float p2, float d, float u, float& c, float& c_lo)
{
    float s, es;
    two_sum(p1, p2, s, es);                                // p1 + p2 = s + es exactly
    const float du = __fmul_rn(d, u);
    const float edu = __fmaf_rn(d, u, -du);                // d u = du + edu exactly
    float h, eh;
    two_sum(__fmul_rn(0.5f, s), du, h, eh);                // halving is exact
    c = h;
    c_lo = __fadd_rn(eh, __fadd_rn(__fmul_rn(0.5f, es), edu));
}

// Line of an event: u = (P1 - P2)/|P1 - P2| and the TOF point c = M + d u as a
// pair; returns false for a degenerate LOR.
__device__ __forceinline__ bool event_line(const Event& e, Line& l)
{
    const float dx = e.p1.x - e.p2.x, dy = e.p1.y - e.p2.y, dz = e.p1.z - e.p2.z;
    const float D = sqrtf(dx * dx + dy * dy + dz * dz);
    if (!(D > 0.f) || !(D < 1e30f) || !(fabsf(e.d) < 1e30f)) return false;
    const float inv = 1.f / D;
    l.u = make_float3(dx * inv, dy * inv, dz * inv);
    tof_point_axis(e.p1.x, e.p2.x, e.d, l.u.x, l.c.x, l.c_lo.x);
    tof_point_axis(e.p1.y, e.p2.y, e.d, l.u.y, l.c.y, l.c_lo.y);
    tof_point_axis(e.p1.z, e.p2.z, e.d, l.u.z, l.c.z, l.c_lo.z);
    return true;
}

// Set up the walk of segment [tau_lo, tau_hi] of the line through c + c_lo
// with unit direction u (tau measured from the TOF point).  Slab method for the
// box, then the start voxel and the first crossing on each axis.  Every plane
// position enters as (plane - c) - c_lo, a difference of nearby numbers, so the
// side of a plane and the crossings keep the precision of the pair; the start
// voxel is first estimated, then corrected by the sign of the position relative
// to the estimated voxel's planes.  The first crossing is expressed relative to
// c once, and later crossings as first + m * step, so plane positions carry no
// accumulated rounding.  Each axis may be crossed only as often as the grid has
// voxels left in that direction, so every index the walk produces lies inside
// the grid whatever the rounding.
__device__ __forceinline__ Walk make_walk(const GridDev& g, const Line& l, float tau_lo, float tau_hi)
{
    Walk w;
    float a = tau_lo, b = tau_hi;
    const float lo[3] = {g.ox, g.oy, g.oz};
    const float v[3] = {g.vx, g.vy, g.vz};
    const int n[3] = {g.nx, g.ny, g.nz};
    const float cc[3] = {l.c.x, l.c.y, l.c.z};
    const float cl[3] = {l.c_lo.x, l.c_lo.y, l.c_lo.z};
    const float uu[3] = {l.u.x, l.u.y, l.u.z};
    float inv_u[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        inv_u[k] = 1.f / uu[k];
        const float hi = lo[k] + (float)n[k] * v[k];
        if (uu[k] == 0.f) {
            ok = ok && ((cc[k] - lo[k]) + cl[k] >= 0.f) && ((cc[k] - hi) + cl[k] < 0.f);
        } else {
            const float t0 = ((lo[k] - cc[k]) - cl[k]) * inv_u[k];
            const float t1 = ((hi - cc[k]) - cl[k]) * inv_u[k];
            a = fmaxf(a, fminf(t0, t1));
            b = fminf(b, fmaxf(t0, t1));
        }
    }
    w.valid = ok && (a < b);
    w.tau_in = a;
    w.tau_out = b;
    int idx[3], step[3];
    float t0[3], dt[3], rem[3];
    const float inf = __int_as_float(0x7f800000);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // estimate of the start voxel (an approximate division is enough: the
        // correction below decides it), then the position at tau_in relative to the
        // lower plane of that voxel: one voxel down or up when it lies outside [0, v)
        const float x = fmaf(a, uu[k], cc[k]);
        float fi = floorf(__fdividef(x - lo[k], v[k]));
        fi = fminf(fmaxf(fi, 0.f), (float)(n[k] - 1));   // also maps NaN of an invalid walk to 0
        const float xl = lo[k] + fi * v[k];
        const float r = fmaf(a, uu[k], (cc[k] - xl) + cl[k]);
        fi += (r < 0.f && fi > 0.f) ? -1.f : ((r >= v[k] && fi < (float)(n[k] - 1)) ? 1.f : 0.f);
        const int i = (int)fi;
        idx[k] = i;
        if (uu[k] > 0.f) {
            step[k] = 1;
            t0[k] = (((lo[k] + (float)(i + 1) * v[k]) - cc[k]) - cl[k]) * inv_u[k];
            dt[k] = v[k] * inv_u[k];
            rem[k] = (float)(n[k] - 1 - i);
        } else if (uu[k] < 0.f) {
            step[k] = -1;
            t0[k] = (((lo[k] + (float)i * v[k]) - cc[k]) - cl[k]) * inv_u[k];
            dt[k] = -v[k] * inv_u[k];
            rem[k] = (float)i;
        } else {
            step[k] = 0;
            t0[k] = inf;
            dt[k] = 0.f;
            rem[k] = 0.f;
        }
        if (rem[k] <= 0.f) t0[k] = inf;
    }
    w.j0 = idx[0] + g.nx * (idx[1] + g.ny * idx[2]);
    w.ix0 = idx[0];
    w.iy0 = idx[1];
    w.iz0 = idx[2];
    w.sxl = step[0];
    w.syl = step[1] * g.nx;
    w.szl = step[2] * g.nx * g.ny;
    w.t0x = t0[0]; w.t0y = t0[1]; w.t0z = t0[2];
    w.dtx = dt[0]; w.dty = dt[1]; w.dtz = dt[2];
    w.rx = rem[0]; w.ry = rem[1]; w.rz = rem[2];
    clip_to_budgets(w);
    return w;
}

// Index of the current voxel as the walk steps: the linear index
// ix + nx (iy + ny iz), stepped by +-1, +-nx, +-nx ny.
struct LinearIndex {
    static constexpr bool kBudgetTests = true;
    int j, sx, sy, sz;
    __device__ __forceinline__ explicit LinearIndex(const Walk& w) : j(w.j0), sx(w.sxl), sy(w.syl), sz(w.szl) {}
    __device__ __forceinline__ int get() const { return j; }
    __device__ __forceinline__ static long long limit(const GridDev& g) { return (long long)g.nx * g.ny * g.nz; }
    __device__ __forceinline__ void step(bool bx, bool by, bool) { j += bx ? sx : (by ? sy : sz); }
};

// 2x2x2-voxel bricks: with bx = ceil(nx/2) and by = ceil(ny/2) bricks per row and
// per plane, brick (ix/2, iy/2, iz/2) holds its 8 voxels contiguously in the order
// (ix & 1) + 2 (iy & 1) + 4 (iz & 1): one 32-byte sector, split by the z parity into
// two 16-byte halves.  Every index of a voxel inside the grid is below
// 8 bx by ceil(nz/2).
__device__ __forceinline__ int brick_index(int ix, int iy, int iz, int bx, int by)
{
    return ((((iz >> 1) * by + (iy >> 1)) * bx + (ix >> 1)) << 3) | ((iz & 1) << 2) | ((iy & 1) << 1) | (ix & 1);
}

// Index of the current voxel in the brick layout as the walk steps.  A step along
// an axis either stays in the brick (the voxel's parity bit on that axis flips:
// +-1, +-2, +-4) or enters the neighbouring brick (the brick index moves by one
// brick, the bit flips back): +-(8 stride - unit) with stride 1, bx, bx by.  The
// two alternate along an axis, so each axis keeps the delta of its next step and
// the sum of both, and a step swaps the delta for sum - delta.
struct BrickIndex {
    static constexpr bool kBudgetTests = false;
    int q, dx, dy, dz, ax, ay, az;
    __device__ __forceinline__ static void axis(int bit, int dir, int unit, int stride, int& d, int& a)
    {
        const int inner = dir * unit, cross = dir * (8 * stride - unit);
        d = dir == 0 ? 0 : ((bit != 0) == (dir > 0) ? cross : inner);
        a = inner + cross;
    }
    __device__ __forceinline__ BrickIndex(const Walk& w, int bx, int by)
    {
        q = brick_index(w.ix0, w.iy0, w.iz0, bx, by);
        const int sx = w.sxl > 0 ? 1 : (w.sxl < 0 ? -1 : 0);
        const int sy = w.syl > 0 ? 1 : (w.syl < 0 ? -1 : 0);
        const int sz = w.szl > 0 ? 1 : (w.szl < 0 ? -1 : 0);
        axis(w.ix0 & 1, sx, 1, 1, dx, ax);
        axis(w.iy0 & 1, sy, 2, bx, dy, ay);
        axis(w.iz0 & 1, sz, 4, bx * by, dz, az);
    }
    __device__ __forceinline__ int get() const { return q; }
    __device__ __forceinline__ static long long limit(const GridDev& g)
    {
        return 8LL * ((g.nx + 1) / 2) * ((g.ny + 1) / 2) * ((g.nz + 1) / 2);
    }
    __device__ __forceinline__ void step(bool bx, bool by, bool bz)
    {
        q += bx ? dx : (by ? dy : dz);
        dx = bx ? ax - dx : dx;
        dy = by ? ay - dy : dy;
        dz = bz ? az - dz : dz;
    }
};

// Siddon walk over the voxel pieces of a prepared Walk.  `visit(j, a)` gets
// the voxel's index (linear or brick, from the Index stepper) and, with Weighted =
// true, the piece's tail difference a = (s_b - s_a) + (g_a - g_b) = 2 [Phi(b) -
// Phi(a)] (tails from `tail`): the TOF mass is tof.half_inv_norm * a, a factor the
// callers apply once per event instead of once per piece.  With Weighted = false,
// a is the piece length in mm (sensitivity).  Each step crosses the nearest
// plane; the axis update is written without branches so that the lanes of a
// warp, which cross different axes, stay converged.  The walk ends at tau_out (an
// axis with no crossing left inside the grid has its next crossing at +inf),
// after at most nx + ny + nz + 2 pieces.
template <bool Weighted, class TailF, class Index, class Visit>
__device__ __forceinline__ void walk_index(const GridDev& g, const TailF& tail, const Walk& w, Index idx,
                                           Visit&& visit)
{
    if (!w.valid) return;
    float mx = 0.f, my = 0.f, mz = 0.f;
    float tx = w.t0x, ty = w.t0y, tz = w.t0z;
    float tau = w.tau_in;
    Tail cur{0.f, 0.f};
    if (Weighted && !TailF::kPiecewise) cur = tail(tau);
    const int max_steps = g.nx + g.ny + g.nz + 2;
    for (int step = 0; step < max_steps; ++step) {
        const float tmin = fminf(tx, fminf(ty, tz));
        const bool last = tmin >= w.tau_out;
        const float tn = fmaxf(fminf(tmin, w.tau_out), tau);
        float a;
        if (Weighted) {
            if constexpr (TailF::kPiecewise) {
                a = tail.piece(tau, tn);
            } else {
                const Tail nxt = tail(tn);
                a = (nxt.s - cur.s) + (cur.g - nxt.g);
                cur = nxt;
            }
        } else {
            a = tn - tau;
        }
#ifdef RECON_BOUNDS_CHECK
        if (!index_ok(idx.get(), Index::limit(g))) break;
#endif
        visit(idx.get(), a);
        if (last) break;
        tau = tn;
        const bool bx = tx == tmin;
        const bool by = !bx && ty == tmin;
        const bool bz = !bx && !by;
        idx.step(bx, by, bz);
        mx += bx ? 1.f : 0.f;
        my += by ? 1.f : 0.f;
        mz += bz ? 1.f : 0.f;
        if constexpr (Index::kBudgetTests) {
            // an axis past its budget gets no further crossing (redundant with the
            // clip of tau_out; measured faster in the linear-layout pass)
            const float inf = __int_as_float(0x7f800000);
            const float nx_ = mx < w.rx ? fmaf(mx, w.dtx, w.t0x) : inf;
            const float ny_ = my < w.ry ? fmaf(my, w.dty, w.t0y) : inf;
            const float nz_ = mz < w.rz ? fmaf(mz, w.dtz, w.t0z) : inf;
            tx = bx ? nx_ : tx;
            ty = by ? ny_ : ty;
            tz = bz ? nz_ : tz;
        } else {
            // no budget test: tau_out was clipped to the first crossing past each
            // axis's budget (clip_to_budgets), so the walk ends before it
            tx = bx ? fmaf(mx, w.dtx, w.t0x) : tx;
            ty = by ? fmaf(my, w.dty, w.t0y) : ty;
            tz = bz ? fmaf(mz, w.dtz, w.t0z) : tz;
        }
    }
}

// The walk over linear voxel indices.
template <bool Weighted, class TailF, class Visit>
__device__ __forceinline__ void walk(const GridDev& g, const TofDev&, const TailF& tail, const Walk& w,
                                     Visit&& visit)
{
    walk_index<Weighted>(g, tail, w, LinearIndex(w), visit);
}

// Region code of one event (Sec. 2.5, Fig. 4): the TOF-estimated annihilation z,
//     z_tof = (z1 + z2) * 0.5 + (d * dz) / D,   D = sqrt((dx*dx + dy*dy) + dz*dz),
// in FP64 with every operation rounded on its own (no fused multiply-add), then
// the regions r with z_b[r] - shell <= z_tof < z_b[r+1] + shell.  Returns 0xFF
// (none), r (one region), r | 0x80 (regions r and r+1) or 0xFE (three or more).
// The inputs are the event's values converted exactly to FP64.
__device__ __forceinline__ uint8_t region_code_of(double x1, double y1, double z1, double x2, double y2, double z2,
                                                  double d, const double* zb, int R, double shell)
{
    const double dx = __dsub_rn(x1, x2);
    const double dy = __dsub_rn(y1, y2);
    const double dz = __dsub_rn(z1, z2);
    const double D = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    const double z = __dadd_rn(__dmul_rn(__dadd_rn(z1, z2), 0.5), __ddiv_rn(__dmul_rn(d, dz), D));
    int first = -1, count = 0;
    for (int r = 0; r < R; ++r) {
        if (__dsub_rn(zb[r], shell) <= z && z < __dadd_rn(zb[r + 1], shell)) {
            if (first < 0) first = r;
            ++count;
        }
    }
    if (count == 0) return 0xFF;
    if (count == 1) return (uint8_t)first;
    if (count == 2) return (uint8_t)(first | 0x80);
    return 0xFE;
}

// Warp-wide sum.
template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of a double; result valid in thread 0.  `sh` holds 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < (int)((blockDim.x + 31) >> 5) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

}  // namespace recon
