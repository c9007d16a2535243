// Trajectory tables (FP64 argument, FP32/int32 output): bins and phases of the matched
// filter (eq. standard-GRFT-TD's n(c, t_m); eqs. H-DFM and pre-DFM), the range phase of
// r0, and the dechirp matrix of the fine stage (Def. 1 / Alg. 2).  O(#hypotheses x M)
// work, never per r0: FP64 is scarce on GB300 and stays out of every inner loop.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace grft {

namespace {

__global__ void k_bins_phases(RadarD R, const double *__restrict__ v, const double *__restrict__ a,
                              int nh, int32_t *__restrict__ rho, float2 *__restrict__ w) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)nh * R.M) return;
    int h = (int)(i / R.M), m = (int)(i % R.M);
    double t = slow_time(m, R.prf);
    double d = displacement(v[h], a[h], t);
    rho[i] = bin_shift(d, R.dr, R.inv_dr);
    w[i] = range_phase(d, R.lambda);
}

// Plain grid: hypothesis h = vi * na + ai (global index h0 + local).  One thread per pulse m
// and group of PT_GROUP hypotheses: t = m / PRF (an FP64 division) once for the group, and
// the phase's cycle count 2 d / lambda as d x (2 / lambda) (within two ulps of the divided
// one, far below the FP32 phase's resolution), and the bin's quotient d / dr as a product
// with the rounded reciprocal, divided only where that could change the bin (bin_shift):
// FP64 throughput is what bounds this kernel on GB300.  The bins are those of the
// definition's IEEE operations.
constexpr int PT_GROUP = 8;
__global__ void k_plain_tables(RadarD R, double v0, double dv, double a0, double da, int na,
                               long h0, int nh, double two_over_lambda, int32_t *__restrict__ rho,
                               float2 *__restrict__ w) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ngrp = (nh + PT_GROUP - 1) / PT_GROUP;
    if (i >= (long)ngrp * R.M) return;
    const int g = (int)(i / R.M), m = (int)(i % R.M);
    const double t = slow_time(m, R.prf);
    const double tt = __dmul_rn(t, t);
#pragma unroll 2
    for (int j = 0; j < PT_GROUP; ++j) {
        const int hl = g * PT_GROUP + j;
        if (hl >= nh) break;
        const long h = h0 + hl;
        const double v = axis_value(v0, dv, (int)(h / na));
        const double a = axis_value(a0, da, (int)(h % na));
        // displacement(v, a, t) with t t shared: (v t) + ((0.5 a)(t t))
        const double d = __dadd_rn(__dmul_rn(v, t), __dmul_rn(__dmul_rn(0.5, a), tt));
        const long o = (long)hl * R.M + m;
        rho[o] = bin_shift(d, R.dr, R.inv_dr);
        const double u = __dmul_rn(d, two_over_lambda);
        const double f = __dsub_rn(u, rint(u));
        float s, c;
        sincospif(2.0f * (float)f, &s, &c);
        w[o] = make_float2(c, s);
    }
}

// Coarse cells c = i * na_c + l: bins of the coarse trajectory and H_pre-DFM.
__global__ void k_coarse_tables(RadarD R, grft_dsgrid g, Rate3 rate, int cell_begin, int cell_count,
                                int32_t *__restrict__ rho, float2 *__restrict__ w) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)cell_count * R.M) return;
    int c = cell_begin + (int)(idx / R.M), m = (int)(idx % R.M);
    const int cw = c % rate.count;              // P = 3: (i na_c + l) nb_c + w
    c /= rate.count;
    double vc = axis_value(g.vc.start, g.vc.step, c / g.ac.count);
    double ac = axis_value(g.ac.start, g.ac.step, c % g.ac.count);
    double t = slow_time(m, R.prf);
    double d = rate.on ? displacement3(vc, ac, axis_value(rate.start, rate.step, cw), t) : displacement(vc, ac, t);
    rho[idx] = bin_shift(d, R.dr, R.inv_dr);
    w[idx] = range_phase(d, R.lambda);
}

__global__ void k_range_phase(RadarD R, int r0_begin, int r0_count, float2 *__restrict__ e0) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= r0_count) return;
    e0[j] = range_phase(__dmul_rn((double)(r0_begin + j), R.dr), R.lambda);
}

__device__ __forceinline__ float2 dechirp_value(const RadarD &R, const grft_dsgrid &g, int m, int f,
                                                const Rate3 &rate) {
    const int u = f % rate.Fb;                  // P = 3: f = (k Fa + q) Fb + u
    f /= rate.Fb;
    int k = f / g.Fa, q = f % g.Fa;
    double dv = fine_offset(g.vc.step, g.Fv, k);
    double da = fine_offset(g.ac.step, g.Fa, q);
    double t = slow_time(m, R.prf);
    const double d = rate.on ? displacement3(dv, da, fine_offset(rate.step, rate.Fb, u), t) : displacement(dv, da, t);
    return range_phase(d, R.lambda);
}

// D[m][f], f = k * Fa + q (H_DFM of the fine offsets, Def. 1).
__global__ void k_dechirp(RadarD R, grft_dsgrid g, float2 *__restrict__ D) {
    int F = g.Fv * g.Fa;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)R.M * F) return;
    int m = (int)(i / F), f = (int)(i % F);
    D[i] = dechirp_value(R, g, m, f, Rate3{false, 0.0, 0.0, 1, 1});
}

__device__ __forceinline__ uint16_t to_bits(float x, bool fp16) {
    if (fp16) return __half_as_ushort(__float2half_rn(x));
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float from_bits(uint16_t b, bool fp16) {
    if (fp16) return __half2float(__ushort_as_half(b));
    return __bfloat162float(__ushort_as_bfloat16(b));
}

// Real-GEMM operand B' of the 4M complex product, K-major, rows n' = 2 f + ri (ri = 0
// real output, 1 imaginary output), columns k' = (m / 32) * 64 + kri * 32 + m % 32
// (kri = 0 multiplies Re Z, 1 multiplies Im Z):
//   (ri, kri) = (0,0): Re D   (0,1): -Im D   (1,0): Im D   (1,1): Re D
// split as hi = round(x), lo = round(x - hi) in BF16 or FP16.  Pulses m >= M and fine
// hypotheses f >= F (padding up to Fpad) are zero.
__global__ void k_dechirp_split(RadarD R, grft_dsgrid g, Rate3 rate, int Mpad, int Fpad, int fp16,
                                uint16_t *__restrict__ Bhi, uint16_t *__restrict__ Blo) {
    int F = g.Fv * g.Fa * rate.Fb;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;     // over Fpad * Mpad
    if (i >= (long)Fpad * Mpad) return;
    int f = (int)(i / Mpad), m = (int)(i % Mpad);
    float2 d = (m < R.M && f < F) ? dechirp_value(R, g, m, f, rate) : make_float2(0.f, 0.f);
    float vals[2][2] = {{d.x, -d.y}, {d.y, d.x}};
    long kk = (long)(m / 32) * 64 + (m % 32);
    for (int ri = 0; ri < 2; ++ri) {
        long row = (long)(2 * f + ri) * (2L * Mpad);
        for (int kri = 0; kri < 2; ++kri) {
            float x = vals[ri][kri];
            uint16_t hb = to_bits(x, fp16 != 0);
            float hi = from_bits(hb, fp16 != 0);
            uint16_t lb = to_bits(x - hi, fp16 != 0);
            Bhi[row + kk + kri * 32] = hb;
            Blo[row + kk + kri * 32] = lb;
        }
    }
}

// B operand of the pair form: rows 2 s and 2 s + 1 of each plane hold Re D and Im D of slot
// s's first hypothesis (pair_slot3) over the pulses, K-major with the pulses contiguous;
// slots s >= S (padding up to Spad) and pulses m >= M are zero.
__global__ void k_dechirp_pair(RadarD R, grft_dsgrid g, Rate3 rate, int Mrow, int Spad, int fp16,
                               uint16_t *__restrict__ Bhi, uint16_t *__restrict__ Blo) {
    const int S = pair_slot_count3(g.Fv, g.Fa, rate.Fb);
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // over Spad * Mrow, pulses fastest
    if (i >= (long)Spad * Mrow) return;
    const int s = (int)(i / Mrow), m = (int)(i % Mrow);
    float2 d = make_float2(0.f, 0.f);
    if (m < R.M && s < S) {
        int f, fm;
        pair_slot3(s, g.Fv, g.Fa, rate.Fb, f, fm);         // f: the full fine index
        d = dechirp_value(R, g, m, f, rate);
    }
    const float vals[2] = {d.x, d.y};
    for (int ri = 0; ri < 2; ++ri) {
        const uint16_t hb = to_bits(vals[ri], fp16 != 0);
        const float hi = from_bits(hb, fp16 != 0);
        const long o = (long)(2 * s + ri) * Mrow + m;
        Bhi[o] = hb;
        Blo[o] = to_bits(vals[ri] - hi, fp16 != 0);
    }
}

inline unsigned blocks_for(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int launch_bins_phases(const Ctx &c, const RadarD &R, const double *v, const double *a, int nh,
                       int32_t *rho, grft_c32 *w) {
    long n = (long)nh * R.M;
    if (n == 0) return GRFT_OK;
    KernelTimer kt(c, GRFT_KERNEL_TABLES);
    k_bins_phases<<<blocks_for(n, 256), 256, 0, c.stream>>>(R, v, a, nh, rho, (float2 *)w);
    return check_launch();
}

int launch_plain_tables(const Ctx &c, const RadarD &R, const grft_grid &g, long h0, int nh,
                        int32_t *rho, float2 *w) {
    const long n = (long)((nh + PT_GROUP - 1) / PT_GROUP) * R.M;
    if (n == 0) return GRFT_OK;
    KernelTimer kt(c, GRFT_KERNEL_TABLES);
    k_plain_tables<<<blocks_for(n, 256), 256, 0, c.stream>>>(R, g.v.start, g.v.step, g.a.start, g.a.step,
                                                              g.a.count, h0, nh, 2.0 / R.lambda, rho, w);
    return check_launch();
}

int launch_coarse_tables(const Ctx &c, const RadarD &R, const grft_dsgrid &g, int cell_begin,
                         int cell_count, int32_t *rho, float2 *w, const Rate3 &rate) {
    long n = (long)cell_count * R.M;
    if (n == 0) return GRFT_OK;
    KernelTimer kt(c, GRFT_KERNEL_TABLES);
    k_coarse_tables<<<blocks_for(n, 256), 256, 0, c.stream>>>(R, g, rate, cell_begin, cell_count, rho, w);
    return check_launch();
}

int launch_range_phase(const Ctx &c, const RadarD &R, int r0_begin, int r0_count, float2 *e0) {
    if (r0_count == 0) return GRFT_OK;
    KernelTimer kt(c, GRFT_KERNEL_TABLES);
    k_range_phase<<<blocks_for(r0_count, 256), 256, 0, c.stream>>>(R, r0_begin, r0_count, e0);
    return check_launch();
}

int launch_dechirp(const Ctx &c, const RadarD &R, const grft_dsgrid &g, float2 *D) {
    long n = (long)R.M * g.Fv * g.Fa;
    KernelTimer kt(c, GRFT_KERNEL_TABLES);
    k_dechirp<<<blocks_for(n, 256), 256, 0, c.stream>>>(R, g, D);
    return check_launch();
}

int launch_dechirp_split(const Ctx &c, const RadarD &R, const grft_dsgrid &g, int Mpad, int Fpad,
                         bool fp16, uint16_t *Bhi, uint16_t *Blo, const Rate3 &rate) {
    long n = (long)Fpad * Mpad;
    KernelTimer kt(c, GRFT_KERNEL_TABLES);
    k_dechirp_split<<<blocks_for(n, 256), 256, 0, c.stream>>>(R, g, rate, Mpad, Fpad, fp16 ? 1 : 0, Bhi, Blo);
    return check_launch();
}

int launch_dechirp_pair(const Ctx &c, const RadarD &R, const grft_dsgrid &g, int Mrow, int Spad, bool fp16,
                        uint16_t *Bhi, uint16_t *Blo, const Rate3 &rate) {
    const long n = (long)Spad * Mrow;
    KernelTimer kt(c, GRFT_KERNEL_TABLES);
    k_dechirp_pair<<<blocks_for(n, 256), 256, 0, c.stream>>>(R, g, rate, Mrow, Spad, fp16 ? 1 : 0, Bhi, Blo);
    return check_launch();
}

}  // namespace grft
