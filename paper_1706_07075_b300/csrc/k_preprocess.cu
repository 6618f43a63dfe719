// Event pre-processing on the GPU (Sec. 2.2 and 2.4), one thread per event:
//   attenuation correction: w_i = exp(sum_j mu_j L_ij), the integral of the
//     attenuation map along the whole LOR inside the grid (Siddon pieces L_ij);
//     the weight is inversely proportional to the pair's survival probability;
//   TOF scatter rejection: the event is kept iff the part of its line within
//     +-z sigma of the TOF point (z = 1.96: 95% confidence) meets a body voxel
//     (mu_j > 0) over a piece of positive length; rejected events get w_i = 0.
// Optionally the resident event weights are multiplied by w_i in place, so
// the MLEM update counts each event w_i times.
#include "recon_device.cuh"

namespace recon {

namespace {

template <int Fmt>
__global__ void __launch_bounds__(256) k_preprocess(void* events, long long n, float lattice, GridDev g,
                                                    const float* __restrict__ mu, float half_window, int apply,
                                                    float* __restrict__ w_out, uint8_t* __restrict__ keep_out,
                                                    unsigned long long* __restrict__ kept)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false;
    if (i < n) {
        const Event e = Fmt == FMT_F32 ? load_event_f32(static_cast<const float4*>(events), i)
                                       : load_event_packed(static_cast<const int4*>(events), i, lattice);
        Line ln;
        float line_mu = 0.f, comp = 0.f;
        keep = !(half_window > 0.f);
        if (event_line(e, ln)) {
            TofDev tof{};
            TailErfc tail{};
            const Walk whole = make_walk(g, ln, -1e30f, 1e30f);
            // a long LOR crosses hundreds of body voxels: compensated (two-sum)
            // accumulation keeps the integral to ~1 ulp instead of ~n/2 ulp
            walk<false>(g, tof, tail, whole, [&](int j, float L) {
                const float x = __fmul_rn(__ldg(mu + j), L);
                const float t = __fadd_rn(line_mu, x);
                const float z = __fsub_rn(t, line_mu);
                comp = __fadd_rn(comp, __fadd_rn(__fsub_rn(line_mu, __fsub_rn(t, z)), __fsub_rn(x, z)));
                line_mu = t;
            });
            line_mu = __fadd_rn(line_mu, comp);
            if (half_window > 0.f) {
                const Walk win = make_walk(g, ln, -half_window, half_window);
                walk<false>(g, tof, tail, win, [&](int j, float L) {
                    if (L > 0.f && __ldg(mu + j) > 0.f) keep = true;
                });
            }
        }
        const float w = keep ? expf(line_mu) : 0.f;
        if (w_out) w_out[i] = w;
        if (keep_out) keep_out[i] = keep ? 1 : 0;
        if (apply) {
            if (Fmt == FMT_F32) {
                float4* rec = static_cast<float4*>(events) + 2 * i + 1;
                rec->w = e.w * w;
            } else {
                int4* rec = static_cast<int4*>(events) + i;
                const unsigned short h = __half_as_ushort(__float2half_rn(e.w * w));
                rec->w = (int)(((unsigned)h << 16) | ((unsigned)rec->w & 0xFFFFu));
            }
        }
    }
    const unsigned b = __ballot_sync(0xffffffffu, keep);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(kept, (unsigned long long)__popc(b));
}

}  // namespace

cudaError_t launch_preprocess(void* events, int fmt, long long n, float lattice, const GridH& g, const float* mu,
                              float half_window, int apply, float* w_out, uint8_t* keep_out,
                              unsigned long long* kept, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    if (fmt == FMT_F32)
        k_preprocess<FMT_F32><<<(unsigned)blocks, 256, 0, st>>>(events, n, lattice, g, mu, half_window, apply, w_out,
                                                               keep_out, kept);
    else
        k_preprocess<FMT_PACKED><<<(unsigned)blocks, 256, 0, st>>>(events, n, lattice, g, mu, half_window, apply,
                                                                  w_out, keep_out, kept);
    return cudaGetLastError();
}

// Out-of-range voxel indices the walks of this file skipped since the last call
// (bounds-checked build; 0 otherwise).
unsigned long long oob_count_preprocess() { return oob_take(); }

}  // namespace recon
