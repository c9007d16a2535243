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
// bins of the fine grid are written, staged per acceleration in shared memory so that each
// (velocity bin, acceleration) row of the CTA's 16 range bins is stored as one contiguous run.
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

// (u - v) exp(j 2 pi k / len) for compile-time k, len: the quarter turn j and the eighth
// turns (+-1 + j) / sqrt(2) without a general complex product or a table read.
template <int K, int LEN, int L>
__device__ __forceinline__ float2 dif_twiddle(float2 d, const float2 *__restrict__ tw) {
    constexpr float R2 = 0.70710678118654752f;
    if (K == 0) return d;
    if (4 * K == LEN) return make_float2(-d.y, d.x);
    if (8 * K == LEN) return make_float2((d.x - d.y) * R2, (d.x + d.y) * R2);
    if (8 * K == 3 * LEN) return make_float2(-(d.x + d.y) * R2, (d.x - d.y) * R2);
    return cmul(d, tw[K * (L / LEN)]);
}

template <int P, int L, int LEN, int I, int K>
struct DifStage {                               // butterflies k = K..LEN/2-1 of group I of span LEN
    static __device__ __forceinline__ void run(float2 (&a)[P], const float2 *__restrict__ tw) {
        if constexpr (K < LEN / 2) {
            const float2 u = a[I + K], v = a[I + K + LEN / 2];
            a[I + K] = cadd(u, v);
            a[I + K + LEN / 2] = dif_twiddle<K, LEN, L>(csub(u, v), tw);
            DifStage<P, L, LEN, I, K + 1>::run(a, tw);
        }
    }
};

template <int P, int L, int LEN, int I>
struct DifGroups {                              // groups I, I + LEN, ... of span LEN
    static __device__ __forceinline__ void run(float2 (&a)[P], const float2 *__restrict__ tw) {
        if constexpr (I < P) {
            DifStage<P, L, LEN, I, 0>::run(a, tw);
            DifGroups<P, L, LEN, I + LEN>::run(a, tw);
        }
    }
};

template <int P, int L, int LEN>
struct DifAll {                                 // spans LEN, LEN/2, ..., 2
    static __device__ __forceinline__ void run(float2 (&a)[P], const float2 *__restrict__ tw) {
        if constexpr (LEN >= 2) {
            DifGroups<P, L, LEN, 0>::run(a, tw);
            DifAll<P, L, LEN / 2>::run(a, tw);
        }
    }
};

// Radix-2 decimation in frequency over the P values of a lane, in place, twiddles
// exp(j 2 pi k / len) = tw[k L / len] (or exact for the quarter and eighth turns):
// afterwards a[i] = sum_n a[n] exp(+j 2 pi n f / P) with f = bitrev(i) (no register
// permutation: every index is a compile-time constant).
template <int P, int L>
__device__ __forceinline__ void dft_regs_dif(float2 (&a)[P], const float2 *__restrict__ tw) {
    DifAll<P, L, P>::run(a, tw);
}

// Output staging of one acceleration: transform bin f = f1 + P f2 of range bin jj (one per
// warp) at slot = f2 + 32 f1, address 17 slot + 16 (slot / 32) + jj = 17 f2 + 560 f1 + jj.
// A warp's writes (f1 fixed, f2 = all 32 values) fall in 32 banks (17 is odd); a warp's
// reads (16 range bins of two consecutive bins f, f + 1, i.e. slots 32 apart) fall 16
// banks apart.
template <int P>
constexpr int gf_stage_words() { return 17 * 32 * P + 16 * P; }
// Pulse tile of the staged form: [GF_WARPS][L + 1] complex (row padding: the fill's 16
// range bins of one pulse fall in distinct banks; a warp's reads of one row are contiguous).
template <int P>
constexpr int gf_tile_words() { return 2 * GF_WARPS * (32 * P + 1); }

// STAGE (worth it when most transform bins are kept): the CTA's pulses are loaded once into
// a shared tile with coalesced reads (16 consecutive range bins per pulse), and each
// acceleration's kept bins are staged in shared memory and written as one contiguous run
// of 16 range bins per (velocity bin, acceleration) row.  Otherwise each lane gathers its
// pulses into registers and stores its kept bins directly (2 MB apart in the output).
// FROM_Z: the pulses come from a coarse output Z[cell][M][r0_count] (src = Z; rho and w
// unused); otherwise they are gathered from the echo (src = echo) as s[m][n0 + rho] w.
// e0 == nullptr: Y carries no range phase.
template <int P, bool FROM_Z, bool STAGE>
__global__ __launch_bounds__(GF_THREADS, STAGE ? 2 : 1) void k_gft_fft(
    const float2 *__restrict__ src, int M, int N, const int32_t *__restrict__ rho, const float2 *__restrict__ w,
    const float2 *__restrict__ chirp, const float2 *__restrict__ e0, int r0_begin, int r0_count, DsOut out) {
    constexpr int L = 32 * P;
    constexpr int XS = L + 1;                   // tile row stride (complex)
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ float gf_dyn[];           // STAGE: pulse tile, then the output stage
    __shared__ float2 s_tw[L];                  // exp(j 2 pi t / L)
    __shared__ float2 s_tl[P][32];              // exp(j 2 pi l f1 / L) at [f1][l]: lanes read consecutive words
    for (int t = threadIdx.x; t < L; t += GF_THREADS) {
        float sn, cs;
        sincospif(2.0f * (float)t / (float)L, &sn, &cs);   // 2t/L is exact (L a power of two)
        s_tw[t] = make_float2(cs, sn);
    }
    const int cl = blockIdx.y;                  // cell within the call
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = blockIdx.x * GF_WARPS;
    const int j = j0 + warp;                    // range bin within [r0_begin, r0_begin + r0_count)
    const bool jok = j < r0_count;              // warp-uniform
    const long tab = (long)cl * M;
    float2 *s_x = (float2 *)gf_dyn;             // STAGE: [GF_WARPS][XS]
    float *gf_stage = gf_dyn + gf_tile_words<P>();
    float2 x[STAGE ? 1 : P];
    if (STAGE) {
        for (int t = threadIdx.x; t < L * GF_WARPS; t += GF_THREADS) {
            const int m = t / GF_WARPS, jj = t % GF_WARPS, jt = j0 + jj;
            float2 v = make_float2(0.f, 0.f);
            if (m < M && jt < r0_count) {
                if (FROM_Z) {
                    v = __ldg(src + (tab + m) * r0_count + jt);
                } else {
                    const int n = r0_begin + jt + rho[tab + m];
                    if ((unsigned)n < (unsigned)N) v = cmul(__ldg(src + (long)m * N + n), w[tab + m]);
                }
            }
            s_x[jj * XS + m] = v;
        }
    } else {
#pragma unroll
        for (int n1 = 0; n1 < (STAGE ? 1 : P); ++n1) {
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
    }
    __syncthreads();                            // s_tw (and the tile) complete
    for (int t = threadIdx.x; t < L; t += GF_THREADS) s_tl[t / 32][t % 32] = s_tw[(t % 32) * (t / 32)];
    const int c = out.cell_begin + cl;
    const int iv = c / out.na_c - out.i0, il = c % out.na_c;
    const int Fv = out.Fv, Fa = out.Fa;
    const int na_full = out.na_c * Fa;
    const float2 ej = (jok && e0) ? e0[j] : make_float2(1.f, 0.f);
    const int f2 = (int)(__brev((unsigned)lane) >> 27);   // bin index across lanes after the DIF
    // Cross-lane stages h = 16, 8, 4, 2, 1: the pair (l, l + h) becomes (v + o, (o - v) t),
    // t = exp(j 2 pi (l mod h) / 2h); written uniformly as u = o + sg v, v = u tw with
    // sg = +1, tw = 1 on the lower lane and sg = -1, tw = t on the upper one.
    float2 tdif[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int h = 16 >> s;
        tdif[s] = (lane & h) ? s_tw[(lane & (h - 1)) * (16 / h) * P] : make_float2(1.f, 0.f);
    }
    __syncthreads();                            // s_tl complete

    for (int q = 0; q < Fa; ++q) {
        float2 y[P];
        const float2 *cq = chirp + (long)q * L + lane;
        if (STAGE) {
            const float2 *xr = s_x + warp * XS + lane;
#pragma unroll
            for (int n1 = 0; n1 < P; ++n1) y[n1] = cmul(xr[32 * n1], __ldg(cq + 32 * n1));
        } else {
#pragma unroll
            for (int n1 = 0; n1 < (STAGE ? 1 : P); ++n1) y[n1] = cmul(x[n1], __ldg(cq + 32 * n1));
        }
        dft_regs_dif<P, L>(y, s_tw);             // y[i] = bin f1 = bitrev(i) of the P-point DFT
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int f1 = bitrev(i, ilog2(P));
            float2 v = f1 ? cmul(y[i], s_tl[f1][lane]) : y[i];
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const int h = 16 >> s;
                const float2 o = make_float2(__shfl_xor_sync(FULL, v.x, h), __shfl_xor_sync(FULL, v.y, h));
                const float sg = (lane & h) ? -1.f : 1.f;
                const float2 u = make_float2(fmaf(sg, v.x, o.x), fmaf(sg, v.y, o.y));
                v = s < 4 ? cmul(u, tdif[s < 4 ? s : 0]) : u;
            }
            y[i] = v;
        }
        if (!STAGE) {
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
            continue;
        }
        __syncthreads();                        // the previous acceleration's write-out is done
        // bin f = f1 + P f2 of this warp's range bin at 17 f2 + 560 f1 + warp
        if (jok) {
            const int base = 17 * f2 + warp;
            if (Fv == L) {                      // every bin kept (the keystone grid): no index test
                if (out.Y) {
#pragma unroll
                    for (int i = 0; i < P; ++i)
                        ((float2 *)gf_stage)[base + 560 * bitrev(i, ilog2(P))] = cmul(ej, y[i]);
                } else {
#pragma unroll
                    for (int i = 0; i < P; ++i)
                        gf_stage[base + 560 * bitrev(i, ilog2(P))] = y[i].x * y[i].x + y[i].y * y[i].y;
                }
            } else {
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const int f1 = bitrev(i, ilog2(P));
                    int k = f1 + P * f2 + Fv / 2;   // kept index: f = (k - Fv/2) mod L
                    if (k >= L) k -= L;
                    if (k < Fv) {
                        const int a = base + 560 * f1;
                        if (out.Y)
                            ((float2 *)gf_stage)[a] = cmul(ej, y[i]);
                        else
                            gf_stage[a] = y[i].x * y[i].x + y[i].y * y[i].y;
                    }
                }
            }
        }
        __syncthreads();
        // write-out: thread (k0 = tid / 16, jj = tid % 16) stores bins k = k0, k0 + 32, ...
        // of range bin j0 + jj: 16 consecutive threads write 64 contiguous bytes.  The staged
        // bin f = f1 + P f2 (f2 < 32) sits at 17 f2 + 560 f1 + jj; the loop steps f by KSTEP = 32,
        // a multiple of P, so f1 = f mod P is fixed and f2 steps by 32 / P (mod 32).
        {
            static_assert((GF_THREADS / GF_WARPS) % P == 0 && L / P == 32, "write-out steps whole f2 rows");
            constexpr int F2STEP = (GF_THREADS / GF_WARPS) / P;
            const int jj = threadIdx.x & (GF_WARPS - 1), k0 = threadIdx.x / GF_WARPS;
            const int jo = j0 + jj;
            if (jo < r0_count) {
                constexpr int KSTEP = GF_THREADS / GF_WARPS;
                const long ostep = (long)KSTEP * na_full * r0_count;
                long o = ((long)(iv * Fv + k0) * na_full + (il * Fa + q)) * r0_count + jo;
                int f = k0 - Fv / 2;
                if (f < 0) f += L;
                const int afix = 560 * (f % P) + jj;
                int f2 = f / P;
                if (out.Y) {
                    for (int k = k0; k < Fv; k += KSTEP, o += ostep) {
                        const float2 v = ((const float2 *)gf_stage)[afix + 17 * f2];
                        out.Y[o] = v;
                        if (out.P) out.P[o] = v.x * v.x + v.y * v.y;   // |e0 y|^2 = |y|^2 (|e0| = 1)
                        f2 = (f2 + F2STEP) & 31;
                    }
                } else {
                    for (int k = k0; k < Fv; k += KSTEP, o += ostep) {
                        out.P[o] = gf_stage[afix + 17 * f2];
                        f2 = (f2 + F2STEP) & 31;
                    }
                }
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

template <int P, bool FROM_Z, bool STAGE>
static int launch_gft_p(const Ctx &c, const dim3 &grid, const RadarD &R, const float2 *src, const grft_dsgrid &g,
                        const int32_t *rho, const float2 *w, const float2 *chirp, const float2 *e0,
                        const DsOut &out) {
    constexpr int most = 4 * (gf_tile_words<P>() + 2 * gf_stage_words<P>());   // float2 staging
    static bool attr[64] = {false};
    if (c.device >= 64) return GRFT_EUNSUPPORTED;
    if (!attr[c.device]) {
        if (cudaFuncSetAttribute(k_gft_fft<P, FROM_Z, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, most) !=
            cudaSuccess)
            return GRFT_ECUDA;
        attr[c.device] = true;
    }
    const size_t smem = STAGE ? 4 * (size_t)(gf_tile_words<P>() + (out.Y ? 2 : 1) * gf_stage_words<P>()) : 0;
    k_gft_fft<P, FROM_Z, STAGE><<<grid, GF_THREADS, smem, c.stream>>>(src, R.M, R.N, rho, w, chirp, e0, g.r0_begin,
                                                               g.r0_count, out);
    return check_launch();
}

template <bool FROM_Z>
static int launch_gft(const Ctx &c, const RadarD &R, const float2 *src, const grft_dsgrid &g, int cell_count,
                      const int32_t *rho, const float2 *w, const float2 *chirp, const float2 *e0, int L,
                      const DsOut &out) {
    if (cell_count == 0 || g.r0_count == 0) return GRFT_OK;
    const dim3 grid((g.r0_count + GF_WARPS - 1) / GF_WARPS, cell_count);
    KernelTimer kt(c, GRFT_KERNEL_CONTRACT_FFT);
    const bool stage = 2 * g.Fv >= L;
#define GF_CASE(PP)                                                                                \
    case 32 * PP:                                                                                  \
        return stage ? launch_gft_p<PP, FROM_Z, true>(c, grid, R, src, g, rho, w, chirp, e0, out)  \
                     : launch_gft_p<PP, FROM_Z, false>(c, grid, R, src, g, rho, w, chirp, e0, out);
    switch (L) {
        GF_CASE(2)
        GF_CASE(4)
        GF_CASE(8)
        GF_CASE(16)
    default:
        return GRFT_EUNSUPPORTED;
    }
#undef GF_CASE
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
