/*
 * FP64 CPU oracle for list-mode TOF-weighted MLEM (arXiv:1706.07075).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * load it.  It shares no source, header, table or constant with the CUDA
 * library; the two meet only at the seeded inputs.
 *
 * What is computed, with the passage each part follows:
 *
 *   Line of response (LOR) of event i: endpoints P1, P2 (mm), D = |P1 - P2|,
 *   u = (P1 - P2) / D, M = (P1 + P2) / 2.  A point on the LOR is M + t u; t is
 *   in mm.  The TOF offset d (mm, positive toward P1) places the most likely
 *   annihilation point at t = d (Sec. 2.3: the TOF kernel is centred on the
 *   measured coincidence time difference).
 *
 *   Siddon ray tracing: the exact intersection of the LOR with every voxel,
 *   found by collecting all plane crossings inside the clipped parameter range,
 *   sorting them and taking each consecutive pair as one voxel segment whose
 *   voxel is the one containing the segment's midpoint (Siddon 1985).  Voxel
 *   (ix,iy,iz) is the half-open box [o + i v, o + (i+1) v); linear index
 *   ix + nx (iy + ny iz).
 *
 *   TOF kernel (Sec. 2.3): a Gaussian of 300 ps FWHM along the LOR whose
 *   weights sum to one.  Reading used here: the Gaussian truncated at +-K sigma
 *   (K = 3, the "approximately 3 sigma" margin of Sec. 2.5) and renormalised,
 *   integrated exactly over each voxel segment:
 *       a_ij = [Phi((t_b - d)/sigma) - Phi((t_a - d)/sigma)] / (2 Phi(K) - 1)
 *   over the segment [t_a, t_b] clipped to [d - K sigma, d + K sigma].
 *
 *   sigma (Sec. 2.5, which prints sigma = 19.11 mm for 300 ps FWHM):
 *       sigma = c * FWHM_t / (2 * 2 sqrt(2 ln 2)),   c = 299.792458 mm/ns.
 *
 *   Forward projection p_i = sum_j a_ij lambda_j, backprojection
 *   C_j = sum_i a_ij r_i, and the sensitivity image s_j = sum_l L_lj (full
 *   chord length, no TOF) over the sensitivity LORs: the list-mode MLEM of
 *   Sec. 2.4 (Shepp & Vardi 1982 in list-mode form).  The update itself and the
 *   iteration loop live in oracle/mlem.py.
 *
 *   Pre-processing (Sec. 2.2, 2.4): attenuation weights exp(sum mu L) along
 *   each LOR and TOF scatter rejection against the body (mu > 0) at 95%
 *   confidence; see oracle_preprocess.
 *
 *   TOF-assisted division into body regions (Sec. 2.5, Fig. 4): the
 *   TOF-estimated annihilation z of each event decides the region(s) it feeds;
 *   each region also takes the events from a 6 mm outer shell on both axial
 *   sides, so an event feeds one or two regions.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off (see oracle/build.py).
 * -ffp-contract=off matters for oracle_region_codes, whose result must be
 * reproduced bit for bit: every operation there is rounded on its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    int32_t nx, ny, nz;
    double vx, vy, vz;
    double ox, oy, oz;
} og_grid;

/* ---------------------------------------------------------------- constants */

double oracle_tof_sigma_mm(double fwhm_ps)
{
    const double c_mm_per_ps = 0.299792458;                  /* speed of light */
    const double fwhm_to_sigma = 2.0 * sqrt(2.0 * log(2.0)); /* FWHM / sigma */
    /* d = c (t2 - t1) / 2, so a timing FWHM maps to c/2 times it along the LOR */
    return 0.5 * c_mm_per_ps * fwhm_ps / fwhm_to_sigma;
}

/* Standard normal cumulative distribution function. */
static double Phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Mass of the +-K sigma truncated, renormalised Gaussian on [ta, tb] (both
 * already inside the window), centred at d. */
double oracle_tof_weight(double ta, double tb, double d, double sigma, double K)
{
    double norm = 2.0 * Phi(K) - 1.0;
    return (Phi((tb - d) / sigma) - Phi((ta - d) / sigma)) / norm;
}

/* ------------------------------------------------------------- geometry */

static double axis_origin(const og_grid *g, int k) { return k == 0 ? g->ox : (k == 1 ? g->oy : g->oz); }
static double axis_voxel(const og_grid *g, int k) { return k == 0 ? g->vx : (k == 1 ? g->vy : g->vz); }
static int32_t axis_count(const og_grid *g, int k) { return k == 0 ? g->nx : (k == 1 ? g->ny : g->nz); }

/* LOR from P1 to P2: midpoint M, unit direction u = (P1 - P2)/D.  Returns D. */
static double make_line(const double p1[3], const double p2[3], double M[3], double u[3])
{
    double d[3], D;
    for (int k = 0; k < 3; ++k) d[k] = p1[k] - p2[k];
    D = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) {
        M[k] = 0.5 * (p1[k] + p2[k]);
        u[k] = D > 0.0 ? d[k] / D : 0.0;
    }
    return D;
}

/* Range of t over which M + t u lies in the grid box (half-open on every
 * axis the line is parallel to).  Returns 0 when the line misses the box. */
static int box_range(const og_grid *g, const double M[3], const double u[3], double *t_in, double *t_out)
{
    double a = -INFINITY, b = INFINITY;
    for (int k = 0; k < 3; ++k) {
        double lo = axis_origin(g, k);
        double hi = lo + axis_count(g, k) * axis_voxel(g, k);
        if (u[k] == 0.0) {
            if (!(M[k] >= lo && M[k] < hi)) return 0;
            continue;
        }
        double t0 = (lo - M[k]) / u[k], t1 = (hi - M[k]) / u[k];
        if (t0 > t1) { double s = t0; t0 = t1; t1 = s; }
        if (t0 > a) a = t0;
        if (t1 < b) b = t1;
    }
    *t_in = a;
    *t_out = b;
    return a < b;
}

static int cmp_double(const void *x, const void *y)
{
    double a = *(const double *)x, b = *(const double *)y;
    return (a > b) - (a < b);
}

/* Upper bound on the number of parameters trace_line may collect. */
static int64_t crossing_capacity(const og_grid *g) { return (int64_t)g->nx + g->ny + g->nz + 8; }

/*
 * Siddon tracing of the LOR P1-P2 restricted to t in [t_lo, t_hi].
 * Writes up to `cap` segments (voxel index, t_a, t_b), in increasing t, and
 * returns their number; returns -1 when cap is too small.  `scratch` must
 * hold crossing_capacity(g) doubles.  Zero-length segments are dropped.
 */
static int64_t trace_line(const og_grid *g, const double p1[3], const double p2[3], double t_lo, double t_hi,
                          int64_t cap, int64_t *vox, double *ta, double *tb, double *scratch)
{
    double M[3], u[3], a, b;
    if (make_line(p1, p2, M, u) <= 0.0) return 0;
    if (!box_range(g, M, u, &a, &b)) return 0;
    if (t_lo > a) a = t_lo;
    if (t_hi < b) b = t_hi;
    if (!(a < b)) return 0;

    int64_t n = 0;
    scratch[n++] = a;
    scratch[n++] = b;
    for (int k = 0; k < 3; ++k) {
        if (u[k] == 0.0) continue;
        double o = axis_origin(g, k), v = axis_voxel(g, k);
        int32_t nk = axis_count(g, k);
        double xa = M[k] + a * u[k], xb = M[k] + b * u[k];
        double xlo = xa < xb ? xa : xb, xhi = xa < xb ? xb : xa;
        int64_t jlo = (int64_t)floor((xlo - o) / v) - 1, jhi = (int64_t)ceil((xhi - o) / v) + 1;
        if (jlo < 0) jlo = 0;
        if (jhi > nk) jhi = nk;
        for (int64_t j = jlo; j <= jhi; ++j) {
            double t = (o + (double)j * v - M[k]) / u[k];
            if (t > a && t < b) scratch[n++] = t;
        }
    }
    qsort(scratch, (size_t)n, sizeof(double), cmp_double);

    int64_t count = 0;
    for (int64_t m = 0; m + 1 < n; ++m) {
        double t0 = scratch[m], t1 = scratch[m + 1];
        if (!(t1 > t0)) continue;
        double tm = 0.5 * (t0 + t1);
        int64_t idx[3];
        int inside = 1;
        for (int k = 0; k < 3; ++k) {
            double x = M[k] + tm * u[k];
            idx[k] = (int64_t)floor((x - axis_origin(g, k)) / axis_voxel(g, k));
            if (idx[k] < 0 || idx[k] >= axis_count(g, k)) inside = 0;
        }
        if (!inside) continue; /* a rounding sliver at the box face */
        if (count >= cap) return -1;
        vox[count] = idx[0] + (int64_t)g->nx * (idx[1] + (int64_t)g->ny * idx[2]);
        ta[count] = t0;
        tb[count] = t1;
        ++count;
    }
    return count;
}

/* Exported tracer for tests: segments of P1-P2 in [t_lo, t_hi]. */
int64_t oracle_trace(const og_grid *g, const double *p1, const double *p2, double t_lo, double t_hi, int64_t cap,
                     int64_t *vox, double *ta, double *tb)
{
    double *scratch = (double *)malloc(sizeof(double) * (size_t)crossing_capacity(g));
    if (!scratch) return -2;
    int64_t n = trace_line(g, p1, p2, t_lo, t_hi, cap, vox, ta, tb, scratch);
    free(scratch);
    return n;
}

/* --------------------------------------------------- system matrix rows */

typedef struct {
    double *scratch, *ta, *tb;
    int64_t *vox;
    int64_t cap;
} row_buf;

static int row_buf_init(row_buf *rb, const og_grid *g)
{
    rb->cap = crossing_capacity(g);
    rb->scratch = (double *)malloc(sizeof(double) * (size_t)rb->cap);
    rb->ta = (double *)malloc(sizeof(double) * (size_t)rb->cap);
    rb->tb = (double *)malloc(sizeof(double) * (size_t)rb->cap);
    rb->vox = (int64_t *)malloc(sizeof(int64_t) * (size_t)rb->cap);
    return rb->scratch && rb->ta && rb->tb && rb->vox;
}

static void row_buf_free(row_buf *rb)
{
    free(rb->scratch);
    free(rb->ta);
    free(rb->tb);
    free(rb->vox);
}

/* Event i of the seven FP64 planes x1,y1,z1,x2,y2,z2,d. */
static void event_at(const double *const ev[7], int64_t i, double p1[3], double p2[3], double *d)
{
    p1[0] = ev[0][i]; p1[1] = ev[1][i]; p1[2] = ev[2][i];
    p2[0] = ev[3][i]; p2[1] = ev[4][i]; p2[2] = ev[5][i];
    *d = ev[6][i];
}

/* Segments of event i inside its TOF window. */
static int64_t event_segments(const og_grid *g, const double *const ev[7], int64_t i, double sigma, double K,
                              row_buf *rb, double *d_out)
{
    double p1[3], p2[3], d;
    event_at(ev, i, p1, p2, &d);
    *d_out = d;
    return trace_line(g, p1, p2, d - K * sigma, d + K * sigma, rb->cap, rb->vox, rb->ta, rb->tb, rb->scratch);
}

/* Sparse row a_i. of one event: voxel indices and TOF-weighted elements. */
int64_t oracle_system_row(const og_grid *g, const double *const ev[7], int64_t i, double sigma, double K,
                          int64_t cap, int64_t *vox, double *a)
{
    row_buf rb;
    if (!row_buf_init(&rb, g)) { row_buf_free(&rb); return -2; }
    double d;
    int64_t n = event_segments(g, ev, i, sigma, K, &rb, &d);
    if (n > cap) n = -1;
    for (int64_t m = 0; m < n; ++m) {
        vox[m] = rb.vox[m];
        a[m] = oracle_tof_weight(rb.ta[m], rb.tb[m], d, sigma, K);
    }
    row_buf_free(&rb);
    return n;
}

/* Forward projection p_i = sum_j a_ij lambda_j for events [i0, i1).
 * Returns 0, or -2 on allocation failure, -1 on a row overflow. */
int oracle_forward(const og_grid *g, const double *const ev[7], int64_t i0, int64_t i1, double sigma, double K,
                   const double *lambda, double *p_out)
{
    row_buf rb;
    if (!row_buf_init(&rb, g)) { row_buf_free(&rb); return -2; }
    int rc = 0;
    for (int64_t i = i0; i < i1; ++i) {
        double d, p = 0.0;
        int64_t n = event_segments(g, ev, i, sigma, K, &rb, &d);
        if (n < 0) { rc = -1; n = 0; }
        for (int64_t m = 0; m < n; ++m) p += oracle_tof_weight(rb.ta[m], rb.tb[m], d, sigma, K) * lambda[rb.vox[m]];
        p_out[i] = p;
    }
    row_buf_free(&rb);
    return rc;
}

/* Backprojection C_j += sum_i a_ij r_i for events [i0, i1) into `C_acc`. */
int oracle_backproject(const og_grid *g, const double *const ev[7], int64_t i0, int64_t i1, double sigma, double K,
                       const double *r, double *C_acc)
{
    row_buf rb;
    if (!row_buf_init(&rb, g)) { row_buf_free(&rb); return -2; }
    int rc = 0;
    for (int64_t i = i0; i < i1; ++i) {
        if (r[i] == 0.0) continue;
        double d;
        int64_t n = event_segments(g, ev, i, sigma, K, &rb, &d);
        if (n < 0) { rc = -1; n = 0; }
        for (int64_t m = 0; m < n; ++m) C_acc[rb.vox[m]] += oracle_tof_weight(rb.ta[m], rb.tb[m], d, sigma, K) * r[i];
    }
    row_buf_free(&rb);
    return rc;
}

/* Number of voxel segments (nonzero-length) of events [i0, i1) inside their
 * TOF windows: the work unit of the projector. */
int64_t oracle_count_visits(const og_grid *g, const double *const ev[7], int64_t i0, int64_t i1, double sigma,
                            double K)
{
    row_buf rb;
    if (!row_buf_init(&rb, g)) { row_buf_free(&rb); return -2; }
    int64_t total = 0;
    for (int64_t i = i0; i < i1; ++i) {
        double d;
        int64_t n = event_segments(g, ev, i, sigma, K, &rb, &d);
        if (n > 0) total += n;
    }
    row_buf_free(&rb);
    return total;
}

/* Sensitivity s_j += sum_l L_lj: full chord lengths (mm) of LORs [l0, l1)
 * given as six FP64 planes x1,y1,z1,x2,y2,z2. */
int oracle_sensitivity(const og_grid *g, const double *const lor[6], int64_t l0, int64_t l1, double *s_acc)
{
    row_buf rb;
    if (!row_buf_init(&rb, g)) { row_buf_free(&rb); return -2; }
    int rc = 0;
    for (int64_t l = l0; l < l1; ++l) {
        double p1[3] = {lor[0][l], lor[1][l], lor[2][l]};
        double p2[3] = {lor[3][l], lor[4][l], lor[5][l]};
        int64_t n = trace_line(g, p1, p2, -INFINITY, INFINITY, rb.cap, rb.vox, rb.ta, rb.tb, rb.scratch);
        if (n < 0) { rc = -1; n = 0; }
        for (int64_t m = 0; m < n; ++m) s_acc[rb.vox[m]] += rb.tb[m] - rb.ta[m];
    }
    row_buf_free(&rb);
    return rc;
}

/* ------------------------- pre-processing: attenuation and TOF rejection */

/*
 * Attenuation correction (Sec. 2.4): each event carries a weight inversely
 * proportional to the probability that its photon pair escapes the body,
 *     w_i = exp( integral of mu along the LOR ) = exp( sum_j mu_j L_ij ),
 * with L_ij the chord of the LOR in voxel j (mu in 1/mm, the mu-map on the
 * image grid).  Reading: "the probability of being attenuated" is read as the
 * survival probability exp(-integral mu), the usual attenuation correction
 * factor; the weight multiplies the event's count in the update.
 *
 * TOF scatter rejection (Sec. 2.2, Fig. 2): an event is rejected when its
 * TOF point lies outside the body at 95% confidence.  Reading: the body is
 * the set of voxels with mu_j > 0; the event is kept iff the interval
 * [d - z sigma, d + z sigma] of the line (z = 1.96 for 95%, two-sided) meets a
 * body voxel over a piece of positive length.  z <= 0 keeps every event.
 *
 * Per event i in [i0, i1): w_out[i] = exp(sum mu L) if kept, else 0;
 * keep_out[i] = 1 or 0.  Returns the number of kept events, or -1 on a
 * buffer error.
 */
int64_t oracle_preprocess(const og_grid *g, const double *const ev[7], int64_t i0, int64_t i1, const double *mu,
                          double sigma, double z, double *w_out, uint8_t *keep_out)
{
    row_buf rb;
    if (!row_buf_init(&rb, g)) { row_buf_free(&rb); return -1; }
    int64_t kept = 0;
    for (int64_t i = i0; i < i1; ++i) {
        double p1[3], p2[3], d;
        event_at(ev, i, p1, p2, &d);
        int64_t n = trace_line(g, p1, p2, -INFINITY, INFINITY, rb.cap, rb.vox, rb.ta, rb.tb, rb.scratch);
        if (n < 0) { row_buf_free(&rb); return -1; }
        double line_mu = 0.0;
        for (int64_t m = 0; m < n; ++m) line_mu += mu[rb.vox[m]] * (rb.tb[m] - rb.ta[m]);
        int keep = 1;
        if (z > 0.0) {
            keep = 0;
            const double lo = d - z * sigma, hi = d + z * sigma;
            for (int64_t m = 0; m < n && !keep; ++m) {
                const double a = rb.ta[m] > lo ? rb.ta[m] : lo;
                const double b = rb.tb[m] < hi ? rb.tb[m] : hi;
                if (mu[rb.vox[m]] > 0.0 && b > a) keep = 1;
            }
        }
        w_out[i] = keep ? exp(line_mu) : 0.0;
        keep_out[i] = (uint8_t)keep;
        kept += keep;
    }
    row_buf_free(&rb);
    return kept;
}

/* --------------------------------------- sampled TOF kernel (Sec. 2.3) */

/*
 * The paper's own projector: N samples equally spaced across the TOF kernel,
 * centred on the TOF point, each carrying its Gaussian weight, the weights
 * summing to one; each sample deposits its weight in the voxel that contains
 * it ("direct technique for voxel filling").  Reading: the samples sit at the
 * centres of N equal cells covering [-K sigma, K sigma]:
 *     t_k = -K sigma + (k + 1/2) 2 K sigma / N,   w_k = phi(t_k/sigma) / sum_m phi(t_m/sigma).
 */
void oracle_lut_samples(int32_t N, double sigma, double K, double *t, double *w)
{
    double sum = 0.0;
    for (int32_t k = 0; k < N; ++k) {
        t[k] = -K * sigma + (k + 0.5) * (2.0 * K * sigma / N);
        w[k] = exp(-0.5 * (t[k] / sigma) * (t[k] / sigma));
        sum += w[k];
    }
    for (int32_t k = 0; k < N; ++k) w[k] /= sum;
}

/*
 * Voxel of the sample at offset t (mm) along event i's line, decided in FP64
 * from the event's values (Sec. 2.3, "direct technique for voxel filling": the
 * sample's weight goes to the voxel that contains it):
 *     u = (P1 - P2) / |P1 - P2|,  c = M + d u,  x = c + t u,
 *     voxel = floor((x - o) / v) per axis, -1 outside the grid.
 * *margin (nullable) receives how close the decision came to another outcome:
 * the distance, in voxels, from (x - o) / v to the nearest integer over the axes
 * on which the sample lies within the grid's extent widened by one voxel (a
 * sample outside the grid by more than that on any axis gets a margin of 1).
 */
static int64_t lut_voxel(const og_grid *g, const double e[7], double t, double *margin)
{
    const double dx = e[0] - e[3], dy = e[1] - e[4], dz = e[2] - e[5];
    const double D = sqrt(dx * dx + dy * dy + dz * dz);
    if (margin) *margin = 1.0;
    if (!(D > 0.0)) return -1;
    const double u[3] = {dx / D, dy / D, dz / D};
    int64_t idx[3];
    int inside = 1;
    double near = 1.0;
    for (int k = 0; k < 3; ++k) {
        const double m = 0.5 * (e[k] + e[k + 3]);
        const double x = m + (e[6] + t) * u[k];          /* c + t u along axis k */
        const double q = (x - axis_origin(g, k)) / axis_voxel(g, k);
        const double f = floor(q);
        const int32_t n = axis_count(g, k);
        if (!(f >= 0.0) || !(f < (double)n)) inside = 0;
        if (q < -1.0 || q > (double)n + 1.0) {            /* far outside on this axis */
            near = 1.0;
            if (margin) *margin = 1.0;
            return -1;
        }
        const double dist = fmin(q - f, f + 1.0 - q);
        if (dist < near) near = dist;
        idx[k] = (int64_t)f;
    }
    if (margin) *margin = near;
    if (!inside) return -1;
    return idx[0] + (int64_t)g->nx * (idx[1] + (int64_t)g->ny * idx[2]);
}

static void event_values(const double *const ev[7], int64_t i, double e[7])
{
    for (int k = 0; k < 7; ++k) e[k] = ev[k][i];
}

/* p_i = sum_k w_k lambda(voxel of sample k), events [i0, i1); t[k], w[k] from
 * oracle_lut_samples. */
int oracle_forward_lut(const og_grid *g, const double *const ev[7], int64_t i0, int64_t i1, int32_t N,
                       const double *w, const double *t, const double *lambda, double *p_out)
{
    for (int64_t i = i0; i < i1; ++i) {
        double e[7];
        event_values(ev, i, e);
        double p = 0.0;
        for (int32_t k = 0; k < N; ++k) {
            int64_t j = lut_voxel(g, e, t[k], NULL);
            if (j >= 0) p += w[k] * lambda[j];
        }
        p_out[i] = p;
    }
    return 0;
}

/* C_j += sum_k w_k r_i over the samples of events [i0, i1) falling in voxel j. */
int oracle_backproject_lut(const og_grid *g, const double *const ev[7], int64_t i0, int64_t i1, int32_t N,
                           const double *w, const double *t, const double *r, double *C_acc)
{
    for (int64_t i = i0; i < i1; ++i) {
        if (r[i] == 0.0) continue;
        double e[7];
        event_values(ev, i, e);
        for (int32_t k = 0; k < N; ++k) {
            int64_t j = lut_voxel(g, e, t[k], NULL);
            if (j >= 0) C_acc[j] += w[k] * r[i];
        }
    }
    return 0;
}

/* Per event of [i0, i1): the number of its N samples whose position lies within
 * eps voxels of a voxel plane (or of the grid's boundary), where a computation
 * in lower precision could decide the voxel, or inside versus outside,
 * differently from this one. */
int oracle_lut_ambiguous(const og_grid *g, const double *const ev[7], int64_t i0, int64_t i1, int32_t N,
                         const double *t, double eps, int32_t *count_out)
{
    for (int64_t i = i0; i < i1; ++i) {
        double e[7];
        event_values(ev, i, e);
        int32_t c = 0;
        for (int32_t k = 0; k < N; ++k) {
            double margin = 1.0;
            lut_voxel(g, e, t[k], &margin);
            if (margin < eps) ++c;
        }
        count_out[i] = c;
    }
    return 0;
}

/* ------------------------------------------------ TOF-assisted division */

/*
 * TOF-estimated annihilation z of each event and the region(s) it feeds
 * (Sec. 2.5).  z_bounds[0..R] are the core boundaries of the R regions along
 * z (increasing).  Region r takes event i iff
 *     z_bounds[r] - shell <= z_tof < z_bounds[r+1] + shell.
 * z_tof is the z of M + d u, evaluated with one rounding per operation in the
 * order written below.  Result per event: 0xFF if no region takes it, else the
 * lowest region r, with bit 7 set when region r+1 takes it too.  Returns the
 * number of events taken by three or more regions (0 when the cores are at
 * least 2*shell wide); those are coded 0xFE.  R must not exceed 64.
 */
int64_t oracle_region_codes(const double *const ev[7], int64_t i0, int64_t i1, int32_t R, const double *z_bounds,
                            double shell, uint8_t *code, double *z_tof_out)
{
    int64_t bad = 0;
    for (int64_t i = i0; i < i1; ++i) {
        double dx = ev[0][i] - ev[3][i];
        double dy = ev[1][i] - ev[4][i];
        double dz = ev[2][i] - ev[5][i];
        double D = sqrt((dx * dx + dy * dy) + dz * dz);
        double z = (ev[2][i] + ev[5][i]) * 0.5 + (ev[6][i] * dz) / D;
        if (z_tof_out) z_tof_out[i] = z;
        int first = -1, count = 0;
        for (int32_t r = 0; r < R; ++r) {
            if (z_bounds[r] - shell <= z && z < z_bounds[r + 1] + shell) {
                if (first < 0) first = r;
                ++count;
            }
        }
        if (count == 0) code[i] = 0xFF;
        else if (count == 1) code[i] = (uint8_t)first;
        else if (count == 2) code[i] = (uint8_t)(first | 0x80);
        else { code[i] = 0xFE; ++bad; }
    }
    return bad;
}
