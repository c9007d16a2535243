// Plain (single-scale) TD-GRFT (Sec. III-A, eq. standard-GRFT-TD; Table III row TD-GRFT):
//   Y[h][n0] = e0(n0) * sum_m s[m][n0 + rho_h(m)] * w_h(m)
// FP32 SIMT.  A CTA owns a group of PL_H hypotheses and a tile of PL_THREADS*PL_J range
// bins; each thread accumulates PL_J bins (32 apart, so warp accesses are contiguous) for
// all PL_H hypotheses.  Bins and
// phases come from a per-chunk table (FP64-built).  Consecutive hypotheses of a group are
// neighbouring accelerations, whose bin shift is nearly always the same at a given pulse:
// the echo samples are reloaded only when the (CTA-uniform) shift changes, so the inner
// loop is FFMA-bound rather than load-bound.
#include <climits>

#include "internal.cuh"

namespace grft {

namespace {

constexpr int PL_THREADS = 256;
constexpr int PL_J = 4;
constexpr int PL_H = 8;
constexpr int PL_MCHUNK = 128;
constexpr int PL_TILE = PL_THREADS * PL_J;

__global__ __launch_bounds__(PL_THREADS, 2) void k_plain(
    const float2 *__restrict__ echo, int M, int N, const int32_t *__restrict__ rho_tab,
    const float2 *__restrict__ w_tab, int nh, int r0_begin, int r0_count,
    const float2 *__restrict__ e0, float2 *__restrict__ Y, float *__restrict__ P) {
    __shared__ int s_rho[PL_MCHUNK][PL_H];
    __shared__ float2 s_w[PL_MCHUNK][PL_H];

    const int h0 = blockIdx.y * PL_H;
    const int nhl = min(PL_H, nh - h0);
    // bins of this thread: j0 + 32 q, q = 0..PL_J-1 (a warp covers 128 consecutive bins, so
    // every load and store instruction of the warp is one contiguous 256-byte run)
    const int j0 = blockIdx.x * PL_TILE + (threadIdx.x >> 5) * (32 * PL_J) + (threadIdx.x & 31);
    const int n0 = r0_begin + j0;

    float2 acc[PL_H][PL_J];
#pragma unroll
    for (int h = 0; h < PL_H; ++h)
#pragma unroll
        for (int j = 0; j < PL_J; ++j) acc[h][j] = make_float2(0.f, 0.f);

    for (int mc = 0; mc < M; mc += PL_MCHUNK) {
        const int mn = min(PL_MCHUNK, M - mc);
        __syncthreads();
        for (int i = threadIdx.x; i < PL_H * PL_MCHUNK; i += PL_THREADS) {
            int h = i / PL_MCHUNK, mm = i % PL_MCHUNK;
            bool ok = h < nhl && mm < mn;
            long o = (long)(h0 + h) * M + mc + mm;
            s_rho[mm][h] = ok ? rho_tab[o] : 0;
            s_w[mm][h] = ok ? w_tab[o] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        auto load_row = [&](int mm, int r, float2 (&v)[PL_J]) {
            const float2 *row = echo + (long)(mc + mm) * N;
            const int base = n0 + r;
#pragma unroll
            for (int j = 0; j < PL_J; ++j) {
                const int n = base + 32 * j;
                v[j] = ((unsigned)n < (unsigned)N) ? __ldg(row + n) : make_float2(0.f, 0.f);
            }
        };
        // two pulses of look-ahead: the samples of pulses mm+1 and mm+2 (at the first
        // hypothesis' shift) are in flight while pulse mm is accumulated
        int r1 = s_rho[0][0], r2 = mn > 1 ? s_rho[1][0] : 0;
        float2 pre1[PL_J], pre2[PL_J];
        load_row(0, r1, pre1);
        if (mn > 1) load_row(1, r2, pre2);
        for (int mm = 0; mm < mn; ++mm) {
            int prev = r1;
            float2 sv[PL_J];
#pragma unroll
            for (int j = 0; j < PL_J; ++j) {
                sv[j] = pre1[j];
                pre1[j] = pre2[j];
            }
            r1 = r2;
            if (mm + 2 < mn) {
                r2 = s_rho[mm + 2][0];
                load_row(mm + 2, r2, pre2);
            }
#pragma unroll
            for (int h = 0; h < PL_H; ++h) {
                const int r = s_rho[mm][h];
                if (r != prev) {             // CTA-uniform branch
                    prev = r;
                    load_row(mm, r, sv);
                }
                const float2 w = s_w[mm][h];
#pragma unroll
                for (int j = 0; j < PL_J; ++j) {
                    acc[h][j].x = fmaf(sv[j].x, w.x, fmaf(-sv[j].y, w.y, acc[h][j].x));
                    acc[h][j].y = fmaf(sv[j].x, w.y, fmaf(sv[j].y, w.x, acc[h][j].y));
                }
            }
        }
    }

#pragma unroll
    for (int j = 0; j < PL_J; ++j) {
        const int jj = j0 + 32 * j;
        if (jj >= r0_count) break;
        const float2 e = e0[jj];
#pragma unroll
        for (int h = 0; h < PL_H; ++h) {
            if (h >= nhl) break;
            const long o = (long)(h0 + h) * r0_count + jj;
            if (Y) Y[o] = cmul(e, acc[h][j]);
            if (P) P[o] = acc[h][j].x * acc[h][j].x + acc[h][j].y * acc[h][j].y;
        }
    }
}

}  // namespace

// Y and P point at hypothesis h0 of the full output; the table holds hypotheses h0..h0+nh-1.
int launch_plain(const Ctx &c, const RadarD &R, const float2 *echo, const grft_grid &g, long h0,
                 int nh, const int32_t *rho, const float2 *w, const float2 *e0, float2 *Y,
                 float *P) {
    if (nh == 0 || g.r0_count == 0) return GRFT_OK;
    dim3 grid((g.r0_count + PL_TILE - 1) / PL_TILE, (nh + PL_H - 1) / PL_H);
    float2 *Yc = Y ? Y + h0 * g.r0_count : nullptr;
    float *Pc = P ? P + h0 * g.r0_count : nullptr;
    KernelTimer kt(c, GRFT_KERNEL_PLAIN);
    k_plain<<<grid, PL_THREADS, 0, c.stream>>>(echo, R.M, R.N, rho, w, nh, g.r0_begin, g.r0_count,
                                               e0, Yc, Pc);
    return check_launch();
}

}  // namespace grft
