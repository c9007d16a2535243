// Fine Doppler-migration correction in the FFT form of the GFT (Def. 1, Alg. 2): per coarse
// cell, range bin and fine acceleration, the coarse-corrected slow-time sequence is
// multiplied by the acceleration dechirp and transformed over pulses; each transform bin is
// one fine velocity.  This needs a fine velocity step of one Doppler bin of an L-point
// transform, dv = lambda PRF / (2 L) (L a power of two, L >= M, zero padded past M); the
// fine offset k - Fv/2 is then the transform bin (k - Fv/2) mod L and the output equals the
// dense contraction of kernel b on the same hypotheses:
//   Y(n0; c, k, q) = e0(n0) sum_m Zc[m][n0] chirp_q(m) exp(+j 2 pi (k - Fv/2) m / L),
//   Zc[m][n0] = s[m][n0 + rho_c(m)] w_c(m),  chirp_q(m) = exp(j 4 pi (da_q t_m^2 / 2) / lambda).
// FP32 SIMT.  One warp per range bin (a CTA holds 16 consecutive bins of one cell): the
// lane gathers its P = L/32 pulses m = lane + 32 n1 once and keeps them in registers for
// all Fa accelerations.  The L-point transform (positive exponent) is split as L = P x 32:
// a P-point decimation-in-frequency DFT over n1 in registers (radix 2, twiddles from a
// shared table of exp(j 2 pi t / L)) leaving bin f1 at position bitrev(f1), the twiddle
// exp(j 2 pi lane f1 / L), then a 32-point decimation-in-frequency transform across the
// lanes by shuffles, which leaves lane l holding the bins f1 + P bitrev5(l).  Only the Fv
// bins of the fine grid are written.
#include "internal.cuh"

namespace grft {

namespace {

constexpr int GF_WARPS = 16;                   // range bins per CTA, one warp each
constexpr int GF_THREADS = 32 * GF_WARPS;

constexpr int bitrev(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}
constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// chirp[q][m] = exp(j 4 pi (da_q t_m^2 / 2) / lambda) for m < M, zero for M <= m < L.
__global__ void k_gft_chirp(RadarD R, grft_dsgrid g, int L, float2 *__restrict__ chirp) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)g.Fa * L) return;
    const int q = (int)(i / L), m = (int)(i % L);
    if (m >= R.M) {
        chirp[i] = make_float2(0.f, 0.f);
        return;
    }
    const double da = fine_offset(g.ac.step, g.Fa, q);
    chirp[i] = range_phase(displacement(0.0, da, slow_time(m, R.prf)), R.lambda);
}

// Radix-2 decimation in frequency over the P values of a lane, in place, twiddles
// exp(j 2 pi k / len) = tw[k L / len]: afterwards a[i] = sum_n a[n] exp(+j 2 pi n f / P)
// with f = bitrev(i) (no register permutation: every index is a compile-time constant).
template <int P, int L>
__device__ __forceinline__ void dft_regs_dif(float2 (&a)[P], const float2 *__restrict__ tw) {
#pragma unroll
    for (int len = P; len >= 2; len >>= 1) {
#pragma unroll
        for (int i = 0; i < P; i += len) {
#pragma unroll
            for (int k = 0; k < len / 2; ++k) {
                const float2 u = a[i + k], v = a[i + k + len / 2];
                a[i + k] = cadd(u, v);
                a[i + k + len / 2] = k ? cmul(csub(u, v), tw[k * (L / len)]) : csub(u, v);
            }
        }
    }
}

// FROM_Z: the pulses come from a coarse output Z[cell][M][r0_count] (src = Z; rho and w
// unused); otherwise they are gathered from the echo (src = echo) as s[m][n0 + rho] w.
// e0 == nullptr: Y carries no range phase.
template <int P, bool FROM_Z>
__global__ __launch_bounds__(GF_THREADS) void k_gft_fft(const float2 *__restrict__ src, int M, int N,
                                                      const int32_t *__restrict__ rho,
                                                      const float2 *__restrict__ w,
                                                      const float2 *__restrict__ chirp,
                                                      const float2 *__restrict__ e0, int r0_begin,
                                                      int r0_count, DsOut out) {
    constexpr int L = 32 * P;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ float2 s_tw[L];                  // exp(j 2 pi t / L)
    __shared__ float2 s_tl[P][32];              // exp(j 2 pi l f1 / L) at [f1][l]: lanes read consecutive words
    for (int t = threadIdx.x; t < L; t += GF_THREADS) {
        float sn, cs;
        sincospif(2.0f * (float)t / (float)L, &sn, &cs);   // 2t/L is exact (L a power of two)
        s_tw[t] = make_float2(cs, sn);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < L; t += GF_THREADS) s_tl[t / 32][t % 32] = s_tw[(t % 32) * (t / 32)];

    const int cl = blockIdx.y;                  // cell within the call
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * GF_WARPS + warp; // range bin within [r0_begin, r0_begin + r0_count)
    const bool jok = j < r0_count;              // warp-uniform
    const long tab = (long)cl * M;
    float2 x[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) {
        const int m = 32 * n1 + lane;
        float2 v = make_float2(0.f, 0.f);
        if (jok && m < M) {
            if (FROM_Z) {
                v = __ldg(src + (tab + m) * r0_count + j);
            } else {
                const int n = r0_begin + j + rho[tab + m];
                if ((unsigned)n < (unsigned)N) v = cmul(__ldg(src + (long)m * N + n), w[tab + m]);
            }
        }
        x[n1] = v;
    }
    const int c = out.cell_begin + cl;
    const int iv = c / out.na_c - out.i0, il = c % out.na_c;
    const int Fv = out.Fv, Fa = out.Fa;
    const int na_full = out.na_c * Fa;
    const float2 ej = (jok && e0) ? e0[j] : make_float2(1.f, 0.f);
    const int f2 = (int)(__brev((unsigned)lane) >> 27);   // bin index across lanes after the DIF
    // twiddles of the cross-lane stages h = 16, 8, 4, 2: exp(j 2 pi (l mod h) / 2h)
    float2 tdif[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int h = 16 >> s;
        tdif[s] = s_tw[(lane & (h - 1)) * (16 / h) * P];
    }
    __syncthreads();                            // s_tl complete

    for (int q = 0; q < Fa; ++q) {
        float2 y[P];
        const float2 *cq = chirp + (long)q * L + lane;
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) y[n1] = cmul(x[n1], __ldg(cq + 32 * n1));
        dft_regs_dif<P, L>(y, s_tw);             // y[i] = bin f1 = bitrev(i) of the P-point DFT
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int f1 = bitrev(i, ilog2(P));
            float2 v = f1 ? cmul(y[i], s_tl[f1][lane]) : y[i];
#pragma unroll
            for (int s = 0; s < 5; ++s) {          // DIF over lanes: pairs (l, l + h), h = 16 >> s
                const int h = 16 >> s;
                const float2 o = make_float2(__shfl_xor_sync(FULL, v.x, h), __shfl_xor_sync(FULL, v.y, h));
                if (lane & h)
                    v = h > 1 ? cmul(csub(o, v), tdif[s < 4 ? s : 0]) : csub(o, v);
                else
                    v = cadd(v, o);
            }
            y[i] = v;
        }
        if (!jok) continue;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            int k = bitrev(i, ilog2(P)) + P * f2 + Fv / 2;   // transform bin f = (k - Fv/2) mod L
            if (k >= L) k -= L;
            if (k < Fv) {
                const long o = ((long)(iv * Fv + k) * na_full + (il * Fa + q)) * r0_count + j;
                if (out.Y) out.Y[o] = cmul(ej, y[i]);
                if (out.P) out.P[o] = y[i].x * y[i].x + y[i].y * y[i].y;
            }
        }
    }
}

}  // namespace

int launch_gft_chirp(const Ctx &c, const RadarD &R, const grft_dsgrid &g, int L, float2 *chirp) {
    const long n = (long)g.Fa * L;
    KernelTimer kt(c, GRFT_KERNEL_TABLES);
    k_gft_chirp<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(R, g, L, chirp);
    return check_launch();
}

template <bool FROM_Z>
static int launch_gft(const Ctx &c, const RadarD &R, const float2 *src, const grft_dsgrid &g, int cell_count,
                      const int32_t *rho, const float2 *w, const float2 *chirp, const float2 *e0, int L,
                      const DsOut &out) {
    if (cell_count == 0 || g.r0_count == 0) return GRFT_OK;
    const dim3 grid((g.r0_count + GF_WARPS - 1) / GF_WARPS, cell_count);
    KernelTimer kt(c, GRFT_KERNEL_CONTRACT_FFT);
    switch (L) {
    case 64:
        k_gft_fft<2, FROM_Z><<<grid, GF_THREADS, 0, c.stream>>>(src, R.M, R.N, rho, w, chirp, e0, g.r0_begin,
                                                                g.r0_count, out);
        break;
    case 128:
        k_gft_fft<4, FROM_Z><<<grid, GF_THREADS, 0, c.stream>>>(src, R.M, R.N, rho, w, chirp, e0, g.r0_begin,
                                                                g.r0_count, out);
        break;
    case 256:
        k_gft_fft<8, FROM_Z><<<grid, GF_THREADS, 0, c.stream>>>(src, R.M, R.N, rho, w, chirp, e0, g.r0_begin,
                                                                g.r0_count, out);
        break;
    case 512:
        k_gft_fft<16, FROM_Z><<<grid, GF_THREADS, 0, c.stream>>>(src, R.M, R.N, rho, w, chirp, e0, g.r0_begin,
                                                                 g.r0_count, out);
        break;
    default:
        return GRFT_EUNSUPPORTED;
    }
    return check_launch();
}

int launch_ds_fft(const Ctx &c, const RadarD &R, const float2 *echo, const grft_dsgrid &g, int cell_count,
                  const int32_t *rho, const float2 *w, const float2 *chirp, const float2 *e0, int L,
                  const DsOut &out) {
    return launch_gft<false>(c, R, echo, g, cell_count, rho, w, chirp, e0, L, out);
}

int launch_ds_fft_z(const Ctx &c, const RadarD &R, const float2 *Z, const grft_dsgrid &g, int cell_count,
                    const float2 *chirp, int L, const DsOut &out) {
    return launch_gft<true>(c, R, Z, g, cell_count, nullptr, nullptr, chirp, nullptr, L, out);
}

}  // namespace grft
