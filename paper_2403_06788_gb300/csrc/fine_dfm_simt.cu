// Fine Doppler-migration correction in FP32 SIMT (the correctness twin of the tensor-core
// path): per coarse cell a complex contraction over pulses (GFT of Def. 1 / Alg. 2 as a
// dense product with the dechirp matrix, Alg. 3):
//   Y(n0; c, f) = e0(n0) * sum_m Zc[m][n0] * D[m][f],  Zc[m][n0] = s[m][n0 + rho_c(m)] w_c(m)
// Zc is gathered on the fly from the echo (or read from a materialised Z).
// CTA tile: 128 bins x 64 fine hypotheses, 256 threads, thread tile 8 bins x 4 hypotheses,
// pulses staged 16 at a time in shared memory ([m][n0] and [m][f], both contiguous in the
// thread's direction).
#include "internal.cuh"

namespace grft {

namespace {

constexpr int SM_BN = 128;   // bins per CTA
constexpr int SM_BF = 64;    // fine hypotheses per CTA
constexpr int SM_BK = 16;    // pulses per stage
constexpr int SM_TN = 8;
constexpr int SM_TF = 4;

__global__ __launch_bounds__(256) void k_ds_simt(
    const float2 *__restrict__ echo, const float2 *__restrict__ Z, int M, int N,
    const int32_t *__restrict__ rho_c, const float2 *__restrict__ w_c,
    const float2 *__restrict__ D, const float2 *__restrict__ e0, int r0_begin, int r0_count,
    int F, DsOut out) {
    __shared__ alignas(16) float2 sA[SM_BK][SM_BN];
    __shared__ alignas(16) float2 sB[SM_BK][SM_BF];

    const int cl = blockIdx.z;
    const int jt = blockIdx.x * SM_BN;
    const int ft = blockIdx.y * SM_BF;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;

    float2 acc[SM_TN][SM_TF];
#pragma unroll
    for (int a = 0; a < SM_TN; ++a)
#pragma unroll
        for (int b = 0; b < SM_TF; ++b) acc[a][b] = make_float2(0.f, 0.f);

    for (int m0 = 0; m0 < M; m0 += SM_BK) {
        for (int i = threadIdx.x; i < SM_BK * SM_BN; i += 256) {
            const int mm = i / SM_BN, jn = i % SM_BN;
            const int m = m0 + mm, j = jt + jn;
            float2 v = make_float2(0.f, 0.f);
            if (m < M && j < r0_count) {
                const long o = (long)cl * M + m;
                if (Z) {
                    v = Z[o * r0_count + j];
                } else {
                    const int n = r0_begin + j + rho_c[o];
                    if ((unsigned)n < (unsigned)N) v = cmul(__ldg(echo + (long)m * N + n), w_c[o]);
                }
            }
            sA[mm][jn] = v;
        }
        for (int i = threadIdx.x; i < SM_BK * SM_BF; i += 256) {
            const int mm = i / SM_BF, fn = i % SM_BF;
            const int m = m0 + mm, f = ft + fn;
            sB[mm][fn] = (m < M && f < F) ? D[(long)m * F + f] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int mm = 0; mm < SM_BK; ++mm) {
            float2 a[SM_TN], b[SM_TF];
            const float4 *pa = reinterpret_cast<const float4 *>(&sA[mm][tx * SM_TN]);
#pragma unroll
            for (int q = 0; q < SM_TN / 2; ++q) {
                float4 t = pa[q];
                a[2 * q] = make_float2(t.x, t.y);
                a[2 * q + 1] = make_float2(t.z, t.w);
            }
            const float4 *pb = reinterpret_cast<const float4 *>(&sB[mm][ty * SM_TF]);
#pragma unroll
            for (int q = 0; q < SM_TF / 2; ++q) {
                float4 t = pb[q];
                b[2 * q] = make_float2(t.x, t.y);
                b[2 * q + 1] = make_float2(t.z, t.w);
            }
#pragma unroll
            for (int x = 0; x < SM_TN; ++x)
#pragma unroll
                for (int y = 0; y < SM_TF; ++y) {
                    acc[x][y].x = fmaf(a[x].x, b[y].x, fmaf(-a[x].y, b[y].y, acc[x][y].x));
                    acc[x][y].y = fmaf(a[x].x, b[y].y, fmaf(a[x].y, b[y].x, acc[x][y].y));
                }
        }
        __syncthreads();
    }

    // epilogue: canonical v-slab layout
    const int c = out.cell_begin + cl;
    const int iv = c / out.na_c - out.i0, il = c % out.na_c;
    const int na_full = out.na_c * out.Fa;
#pragma unroll
    for (int y = 0; y < SM_TF; ++y) {
        const int f = ft + ty * SM_TF + y;
        if (f >= F) break;
        const int k = f / out.Fa, q = f % out.Fa;
        const long rowo = ((long)(iv * out.Fv + k) * na_full + (il * out.Fa + q)) * r0_count;
#pragma unroll
        for (int x = 0; x < SM_TN; ++x) {
            const int j = jt + tx * SM_TN + x;
            if (j >= r0_count) break;
            const float2 v = acc[x][y];
            if (out.Y) out.Y[rowo + j] = cmul(e0[j], v);
            if (out.P) out.P[rowo + j] = v.x * v.x + v.y * v.y;
        }
    }
}

// The pair form in FP32 (the slots of pair_slot: a fine hypothesis and its mirror, whose
// dechirp row is the conjugate): per slot and bin the four real sums A = sum Zr Dr,
// E = sum Zi Dr, C = sum Zr Di, B = sum Zi Di, kept as the pairs (A, E) and (C, B) of two
// paired FMAs per pulse with the gathered sample (Zr, Zi) as it lies in shared memory and the
// slot's (Dr, Dr) and (Di, Di); then Y(f) = (A - B) + j (C + E), Y(f') = (A + B) + j (E - C).
// Two FP32 FMAs per hypothesis and pulse, where the complex form takes four.
// CTA tile: 128 bins x 64 slots, 256 threads, thread tile 8 bins x 4 slots.
constexpr int SP_BS = 64;    // slots per CTA

__device__ __forceinline__ void ffma2p(uint64_t &acc, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ float2 unpack2p(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

__global__ __launch_bounds__(256) void k_ds_simt_pair(
    const float2 *__restrict__ echo, const float2 *__restrict__ Z, int M, int N,
    const int32_t *__restrict__ rho_c, const float2 *__restrict__ w_c,
    const float2 *__restrict__ D, const float2 *__restrict__ e0, int r0_begin, int r0_count,
    int F, int S, DsOut out) {
    __shared__ alignas(16) float2 sA[SM_BK][SM_BN];
    __shared__ alignas(16) float4 sB[SM_BK][SP_BS];      // (Dr, Dr, Di, Di) of each slot's first hypothesis
    __shared__ int s_f[SP_BS], s_fm[SP_BS];
    static_assert(SM_BN == 16 * SM_TN && SP_BS == 16 * SM_TF, "16 x 16 threads over the tile");

    const int cl = blockIdx.z;
    const int jt = blockIdx.x * SM_BN;
    const int st = blockIdx.y * SP_BS;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    if (threadIdx.x < SP_BS) {
        int f = -1, fm = -1;
        if (st + threadIdx.x < S) pair_slot(st + threadIdx.x, out.Fv, out.Fa, f, fm);
        s_f[threadIdx.x] = f;
        s_fm[threadIdx.x] = fm;
    }

    uint64_t ae[SM_TN][SM_TF], cb[SM_TN][SM_TF];
#pragma unroll
    for (int a = 0; a < SM_TN; ++a)
#pragma unroll
        for (int b = 0; b < SM_TF; ++b) ae[a][b] = cb[a][b] = 0ull;

    __syncthreads();
    // Staging, double-buffered through registers: the next stage's samples (echo value and
    // coarse phase, multiplied when stored) and dechirp entries are loaded before the current
    // stage is accumulated.  Thread i of the CTA stages elements i, i + 256, ... of each tile.
    constexpr int NA = SM_BK * SM_BN / 256, NB = SM_BK * SP_BS / 256;
    float2 ra[NA], rw[NA], rb[NB];
    auto fetch = [&](int m0) {
#pragma unroll
        for (int u = 0; u < NA; ++u) {
            const int i = threadIdx.x + 256 * u;
            const int mm = i / SM_BN, jn = i % SM_BN;
            const int m = m0 + mm, j = jt + jn;
            float2 v = make_float2(0.f, 0.f), wv = make_float2(1.f, 0.f);
            if (m < M && j < r0_count) {
                const long o = (long)cl * M + m;
                if (Z) {
                    v = Z[o * r0_count + j];
                } else {
                    const int n = r0_begin + j + rho_c[o];
                    if ((unsigned)n < (unsigned)N) {
                        v = __ldg(echo + (long)m * N + n);
                        wv = w_c[o];
                    }
                }
            }
            ra[u] = v;
            rw[u] = wv;
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int i = threadIdx.x + 256 * u;
            const int mm = i / SP_BS, sn = i % SP_BS;
            const int m = m0 + mm, f = s_f[sn];
            rb[u] = (m < M && f >= 0) ? D[(long)m * F + f] : make_float2(0.f, 0.f);
        }
    };
    // sA holds each thread's SM_TN bins as SM_TN / 2 16-byte words spread over the row: bin
    // pair q of thread tx at word q * 16 + tx, so the 16 threads of a row read 256
    // consecutive bytes per load (their bins tx * SM_TN .. lie 64 bytes apart, which would
    // put four of every eight threads of a load phase on the same banks)
    auto store = [&]() {
#pragma unroll
        for (int u = 0; u < NA; ++u) {
            const int i = threadIdx.x + 256 * u;
            const int jn = i % SM_BN;
            sA[i / SM_BN][((jn % SM_TN) >> 1) * (SM_BN / SM_TN * 2) + (jn / SM_TN) * 2 + (jn & 1)] =
                Z ? ra[u] : cmul(ra[u], rw[u]);
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int i = threadIdx.x + 256 * u;
            sB[i / SP_BS][i % SP_BS] = make_float4(rb[u].x, rb[u].x, rb[u].y, rb[u].y);
        }
    };
    fetch(0);
    store();
    __syncthreads();
    for (int m0 = 0; m0 < M; m0 += SM_BK) {
        if (m0 + SM_BK < M) fetch(m0 + SM_BK);
#pragma unroll 2
        for (int mm = 0; mm < SM_BK; ++mm) {
            uint64_t a[SM_TN];
            ulonglong2 b[SM_TF];
            const ulonglong2 *pa = reinterpret_cast<const ulonglong2 *>(&sA[mm][tx * 2]);
#pragma unroll
            for (int q = 0; q < SM_TN / 2; ++q) {
                const ulonglong2 t = pa[q * (SM_BN / SM_TN)];
                a[2 * q] = t.x;
                a[2 * q + 1] = t.y;
            }
            const ulonglong2 *pb = reinterpret_cast<const ulonglong2 *>(&sB[mm][ty * SM_TF]);
#pragma unroll
            for (int y = 0; y < SM_TF; ++y) b[y] = pb[y];
#pragma unroll
            for (int x = 0; x < SM_TN; ++x)
#pragma unroll
                for (int y = 0; y < SM_TF; ++y) {
                    ffma2p(ae[x][y], a[x], b[y].x);     // (A, E) += (Zr, Zi) (Dr, Dr)
                    ffma2p(cb[x][y], a[x], b[y].y);     // (C, B) += (Zr, Zi) (Di, Di)
                }
        }
        __syncthreads();
        if (m0 + SM_BK < M) {
            store();
            __syncthreads();
        }
    }

    // epilogue: both hypotheses of each slot, canonical v-slab layout
    const int c = out.cell_begin + cl;
    const int iv = c / out.na_c - out.i0, il = c % out.na_c;
    const int na_full = out.na_c * out.Fa;
#pragma unroll
    for (int y = 0; y < SM_TF; ++y) {
        const int sn = ty * SM_TF + y;
        const int f = s_f[sn], fm = s_fm[sn];
        if (f < 0) continue;
        const long rf = ((long)(iv * out.Fv + f / out.Fa) * na_full + (il * out.Fa + f % out.Fa)) * r0_count;
        const long rm =
            fm < 0 ? -1 : ((long)(iv * out.Fv + fm / out.Fa) * na_full + (il * out.Fa + fm % out.Fa)) * r0_count;
#pragma unroll
        for (int x = 0; x < SM_TN; ++x) {
            const int j = jt + tx * SM_TN + x;
            if (j >= r0_count) break;
            const float2 AE = unpack2p(ae[x][y]), CB = unpack2p(cb[x][y]);
            const float2 yf = make_float2(AE.x - CB.y, CB.x + AE.y);     // (A - B, C + E)
            const float2 ym = make_float2(AE.x + CB.y, AE.y - CB.x);     // (A + B, E - C)
            if (out.Y) out.Y[rf + j] = cmul(e0[j], yf);
            if (out.P) out.P[rf + j] = yf.x * yf.x + yf.y * yf.y;
            if (rm >= 0) {
                if (out.Y) out.Y[rm + j] = cmul(e0[j], ym);
                if (out.P) out.P[rm + j] = ym.x * ym.x + ym.y * ym.y;
            }
        }
    }
}

}  // namespace

int launch_ds_simt(const Ctx &c, const RadarD &R, const float2 *echo, const float2 *Z,
                   const grft_dsgrid &g, int cell_count, const int32_t *rho, const float2 *w,
                   const float2 *D, const float2 *e0, const DsOut &out) {
    if (cell_count == 0 || g.r0_count == 0) return GRFT_OK;
    const int F = g.Fv * g.Fa;
    KernelTimer kt(c, GRFT_KERNEL_CONTRACT_FP32);
    if (ds_pair_form(kNoRate)) {             // the pair form (DSGRFT_PAIR=0: the complex form)
        const int S = pair_slot_count(g.Fv, g.Fa);
        dim3 grid((g.r0_count + SM_BN - 1) / SM_BN, (S + SP_BS - 1) / SP_BS, cell_count);
        k_ds_simt_pair<<<grid, 256, 0, c.stream>>>(echo, Z, R.M, R.N, rho, w, D, e0, g.r0_begin, g.r0_count,
                                                   F, S, out);
        return check_launch();
    }
    dim3 grid((g.r0_count + SM_BN - 1) / SM_BN, (F + SM_BF - 1) / SM_BF, cell_count);
    k_ds_simt<<<grid, 256, 0, c.stream>>>(echo, Z, R.M, R.N, rho, w, D, e0, g.r0_begin, g.r0_count,
                                          F, out);
    return check_launch();
}

}  // namespace grft
