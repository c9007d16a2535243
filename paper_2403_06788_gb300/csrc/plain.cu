// Plain (single-scale) TD-GRFT (Sec. III-A, eq. standard-GRFT-TD; Table III row TD-GRFT):
//   Y[h][n0] = e0(n0) * sum_m s[m][n0 + rho_h(m)] * w_h(m)
// FP32 SIMT.  A CTA owns a group of PL_H hypotheses and a tile of PL_THREADS*PL_J range
// bins; each thread accumulates PL_J bins (32 apart, so warp accesses are contiguous) for
// all PL_H hypotheses (8 x 4 by default; 8 x 2 and 16 x 2 selectable).  Bins and phases come from a per-chunk table (FP64-built).
// Consecutive hypotheses of a group are neighbouring accelerations, whose bin shift is
// nearly always the same at a given pulse: a per-pulse flag marks the pulses where all of
// them share the first one's shift (one row of samples, no per-hypothesis check); at the
// others the samples are reloaded when the (CTA-uniform) shift changes.  The complex
// multiply-adds run as paired FP32 FMAs (fma.rn.f32x2 over a pair of hypotheses, the
// phases staged in shared memory), which round exactly as the scalar form and halve the
// FMA instruction count.
#include <climits>
#include <cstdlib>

#include "internal.cuh"

namespace grft {

namespace {

constexpr int PL_THREADS = 256;
constexpr int PL_MCHUNK = 128;

// Paired FP32 arithmetic (two independent IEEE fma.rn per instruction).
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 unpack2(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ void ffma2(uint64_t &acc, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}

// PL_H hypotheses per CTA, PL_J bins per thread: a gathered sample serves PL_H hypotheses
// (the L2 gathers per FMA fall as PL_H grows) and the accumulators take 2 PL_H PL_J registers.
// The paired FMAs pair two hypotheses (h, h + 1) of one bin: the real parts of both in one
// accumulator pair and the imaginary parts in another, against the pair's phases (re_h,
// re_h+1) and (im_h, im_h+1), one 16-byte shared word per hypothesis pair and pulse.  Per
// output component the FMAs and their order are those of the scalar form
//   re += (-s.im) w.im, re += s.re w.re;   im += s.im w.re, im += s.re w.im.
template <int PL_H, int PL_J>
__global__ __launch_bounds__(PL_THREADS, PL_J == 2 && PL_H == 8 ? 3 : 2) void k_plain(
    const float2 *__restrict__ echo, int M, int N, const int32_t *__restrict__ rho_tab,
    const float2 *__restrict__ w_tab, int nh, int r0_begin, int r0_count,
    const float2 *__restrict__ e0, float2 *__restrict__ Y, float *__restrict__ P) {
    static_assert(PL_H % 2 == 0, "hypotheses are paired");
    constexpr int PL_TILE = PL_THREADS * PL_J;
    constexpr int H2 = PL_H / 2;
    __shared__ int s_rho[PL_MCHUNK][PL_H];
    __shared__ alignas(16) float s_w[PL_MCHUNK][H2][4];   // (re h, re h+1, im h, im h+1)
    __shared__ int s_same[PL_MCHUNK];            // every hypothesis of the group shifts like the first
    __shared__ int s_same3[PL_MCHUNK];           // ... at pulses mm, mm + 1 and mm + 2
    __shared__ int s_rng[2];                     // least and greatest shift of the chunk

    const int h0 = blockIdx.y * PL_H;
    const int nhl = min(PL_H, nh - h0);
    // bins of this thread: j0 + 32 q, q = 0..PL_J-1 (a warp covers 32 PL_J consecutive bins,
    // so every load and store instruction of the warp is one contiguous 256-byte run)
    const int j0 = blockIdx.x * PL_TILE + (threadIdx.x >> 5) * (32 * PL_J) + (threadIdx.x & 31);
    const int n0 = r0_begin + j0;
    const int n0_tile = r0_begin + blockIdx.x * PL_TILE;   // first bin of the CTA's tile

    uint64_t are[H2][PL_J], aim[H2][PL_J];     // (re h, re h+1) and (im h, im h+1)
#pragma unroll
    for (int h = 0; h < H2; ++h)
#pragma unroll
        for (int j = 0; j < PL_J; ++j) are[h][j] = aim[h][j] = 0ull;

    for (int mc = 0; mc < M; mc += PL_MCHUNK) {
        const int mn = min(PL_MCHUNK, M - mc);
        __syncthreads();
        for (int i = threadIdx.x; i < PL_H * PL_MCHUNK; i += PL_THREADS) {
            const int h = i % PL_H, mm = i / PL_H;
            bool ok = h < nhl && mm < mn;
            long o = (long)(h0 + h) * M + mc + mm;
            const float2 wv = ok ? w_tab[o] : make_float2(0.f, 0.f);
            s_rho[mm][h] = ok ? rho_tab[o] : 0;
            s_w[mm][h >> 1][h & 1] = wv.x;
            s_w[mm][h >> 1][2 + (h & 1)] = wv.y;
        }
        if (threadIdx.x == 0) {
            s_rng[0] = INT_MAX;
            s_rng[1] = INT_MIN;
        }
        __syncthreads();
        if (threadIdx.x < PL_MCHUNK) {          // PL_MCHUNK <= PL_THREADS: one thread per pulse
            int same = 1, lo = s_rho[threadIdx.x][0], hi = lo;
#pragma unroll
            for (int h = 1; h < PL_H; ++h) {
                const int r = s_rho[threadIdx.x][h];
                same &= r == s_rho[threadIdx.x][0];
                lo = min(lo, r);
                hi = max(hi, r);
            }
            s_same[threadIdx.x] = same;
            int same3 = same;
#pragma unroll
            for (int k = 1; k < 3; ++k) {
                const int mk = min((int)threadIdx.x + k, PL_MCHUNK - 1);
#pragma unroll
                for (int h = 1; h < PL_H; ++h) same3 &= s_rho[mk][h] == s_rho[mk][0];
            }
            s_same3[threadIdx.x] = same3;
            lo = __reduce_min_sync(0xffffffffu, lo);
            hi = __reduce_max_sync(0xffffffffu, hi);
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&s_rng[0], lo);
                atomicMax(&s_rng[1], hi);
            }
        }
        __syncthreads();
        // block-uniform: every gather of the tile's bins at every shift of the chunk is inside
        // the echo (the unused table slots hold shift 0, which only widens the range)
        const bool inside = n0_tile + s_rng[0] >= 0 && n0_tile + PL_TILE - 1 + s_rng[1] < N;
        auto load_row = [&](int mm, int r, float2 (&v)[PL_J]) {
            const float2 *row = echo + (long)(mc + mm) * N + (n0 + r);
            if (inside) {
#pragma unroll
                for (int j = 0; j < PL_J; ++j) v[j] = __ldg(row + 32 * j);
            } else {
                const int base = n0 + r;
#pragma unroll
                for (int j = 0; j < PL_J; ++j)
                    v[j] = ((unsigned)(base + 32 * j) < (unsigned)N) ? __ldg(row + 32 * j) : make_float2(0.f, 0.f);
            }
        };
        // the four paired FMAs of hypothesis pair h2 and bin j: samples (re, re'), (im, im'),
        // (-im, -im') of the pair's two hypotheses, phases w = ((re h, re h+1), (im h, im h+1))
        auto mac = [&](int h2, int j, uint64_t sr, uint64_t si, uint64_t sn, const ulonglong2 &w) {
            ffma2(are[h2][j], sn, w.y);
            ffma2(aim[h2][j], si, w.x);
            ffma2(are[h2][j], sr, w.x);
            ffma2(aim[h2][j], sr, w.y);
        };
        // pulse mm whose hypotheses all take the samples in sv0
        auto pulse_same = [&](int mm, const float2 (&sv0)[PL_J]) {
            const ulonglong2 *wp = reinterpret_cast<const ulonglong2 *>(&s_w[mm][0][0]);
            // (re, re), (im, im) and (-im, -im) of every sample, reused by all hypotheses
            uint64_t sr[PL_J], si[PL_J], sn[PL_J];
#pragma unroll
            for (int j = 0; j < PL_J; ++j) {
                sr[j] = pack2(sv0[j].x, sv0[j].x);
                si[j] = pack2(sv0[j].y, sv0[j].y);
                sn[j] = pack2(-sv0[j].y, -sv0[j].y);
            }
#pragma unroll
            for (int h2 = 0; h2 < H2; ++h2) {
                const ulonglong2 w = wp[h2];
#pragma unroll
                for (int j = 0; j < PL_J; ++j) mac(h2, j, sr[j], si[j], sn[j], w);
            }
        };
        // pulse mm whose samples at the first hypothesis' shift are in sv0
        auto pulse = [&](int mm, const float2 (&sv0)[PL_J]) {
            if (s_same[mm]) {                // CTA-uniform: one row of samples for all hypotheses
                pulse_same(mm, sv0);
                return;
            }
            const ulonglong2 *wp = reinterpret_cast<const ulonglong2 *>(&s_w[mm][0][0]);
            int prev = s_rho[mm][0];
            float2 cur[PL_J];
#pragma unroll
            for (int j = 0; j < PL_J; ++j) cur[j] = sv0[j];
#pragma unroll
            for (int h2 = 0; h2 < H2; ++h2) {
                float2 sa[PL_J];
                const int ra = s_rho[mm][2 * h2], rb = s_rho[mm][2 * h2 + 1];
                if (ra != prev) {            // CTA-uniform branches
                    prev = ra;
                    load_row(mm, ra, cur);
                }
#pragma unroll
                for (int j = 0; j < PL_J; ++j) sa[j] = cur[j];
                if (rb != prev) {
                    prev = rb;
                    load_row(mm, rb, cur);
                }
                const ulonglong2 w = wp[h2];
#pragma unroll
                for (int j = 0; j < PL_J; ++j)
                    mac(h2, j, pack2(sa[j].x, cur[j].x), pack2(sa[j].y, cur[j].y),
                        pack2(-sa[j].y, -cur[j].y), w);
            }
        };
        // two pulses of look-ahead over three buffers in rotation: the samples of pulses mm+1
        // and mm+2 are in flight while pulse mm is accumulated, and no buffer is copied
        float2 b0[PL_J], b1[PL_J], b2[PL_J];
        load_row(0, s_rho[0][0], b0);
        if (mn > 1) load_row(1, s_rho[1][0], b1);
        for (int mm = 0; mm < mn; mm += 3) {
            if (inside && mm + 4 < mn && s_same3[mm]) {    // CTA-uniform: three pulses, no branch
                const float2 *row = echo + (long)(mc + mm) * N + n0;
#pragma unroll
                for (int j = 0; j < PL_J; ++j) b2[j] = __ldg(row + 2L * N + s_rho[mm + 2][0] + 32 * j);
                pulse_same(mm, b0);
#pragma unroll
                for (int j = 0; j < PL_J; ++j) b0[j] = __ldg(row + 3L * N + s_rho[mm + 3][0] + 32 * j);
                pulse_same(mm + 1, b1);
#pragma unroll
                for (int j = 0; j < PL_J; ++j) b1[j] = __ldg(row + 4L * N + s_rho[mm + 4][0] + 32 * j);
                pulse_same(mm + 2, b2);
                continue;
            }
            if (mm + 2 < mn) load_row(mm + 2, s_rho[mm + 2][0], b2);
            pulse(mm, b0);
            if (mm + 1 >= mn) break;
            if (mm + 3 < mn) load_row(mm + 3, s_rho[mm + 3][0], b0);
            pulse(mm + 1, b1);
            if (mm + 2 >= mn) break;
            if (mm + 4 < mn) load_row(mm + 4, s_rho[mm + 4][0], b1);
            pulse(mm + 2, b2);
        }
    }

#pragma unroll
    for (int j = 0; j < PL_J; ++j) {
        const int jj = j0 + 32 * j;
        if (jj >= r0_count) break;
        const float2 e = e0[jj];
#pragma unroll
        for (int h2 = 0; h2 < H2; ++h2) {
            const float2 re = unpack2(are[h2][j]), im = unpack2(aim[h2][j]);
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int h = 2 * h2 + t;
                if (h >= nhl) break;
                const float2 a = t ? make_float2(re.y, im.y) : make_float2(re.x, im.x);
                const long o = (long)(h0 + h) * r0_count + jj;
                if (Y) Y[o] = cmul(e, a);
                if (P) P[o] = a.x * a.x + a.y * a.y;
            }
        }
    }
}

template <int PL_H, int PL_J>
int launch_plain_shape(const Ctx &c, const RadarD &R, const float2 *echo, const grft_grid &g, int nh,
                       const int32_t *rho, const float2 *w, const float2 *e0, float2 *Yc, float *Pc) {
    constexpr int PL_TILE = PL_THREADS * PL_J;
    dim3 grid((g.r0_count + PL_TILE - 1) / PL_TILE, (nh + PL_H - 1) / PL_H);
    KernelTimer kt(c, GRFT_KERNEL_PLAIN);
    k_plain<PL_H, PL_J><<<grid, PL_THREADS, 0, c.stream>>>(echo, R.M, R.N, rho, w, nh, g.r0_begin, g.r0_count, e0,
                                                          Yc, Pc);
    return check_launch();
}

// Tile shape of k_plain (hypotheses x bins per thread): 8 x 4 at two CTAs per SM by
// default; DSGRFT_PLAIN_SHAPE=8x2 (three CTAs per SM) or 16x2 selects the others (the same
// arithmetic per output, so the same results bit for bit).  For 2^39 hypothesis-pulses:
// 8 x 4 101.9 ms, 8 x 2 104.7, 16 x 2 105.2 (whole calls, tables included): neither the L2
// gathers, which 16 x 2 halves per FMA, nor the occupancy bounds the kernel much.
int plain_shape() {
    static const int v = [] {
        const char *e = getenv("DSGRFT_PLAIN_SHAPE");
        if (e && e[0] == '1') return 2;
        if (e && e[0] == '8' && e[2] == '2') return 0;
        return 1;
    }();
    return v;
}

}  // namespace

// Y and P point at hypothesis h0 of the full output; the table holds hypotheses h0..h0+nh-1.
// Each output's sum runs over the pulses in the same order with the same FMAs whatever the
// group it falls in (a partial last group included), so the shape and the chunking do not
// change any result.
int launch_plain(const Ctx &c, const RadarD &R, const float2 *echo, const grft_grid &g, long h0,
                 int nh, const int32_t *rho, const float2 *w, const float2 *e0, float2 *Y,
                 float *P) {
    if (nh == 0 || g.r0_count == 0) return GRFT_OK;
    float2 *Yc = Y ? Y + h0 * g.r0_count : nullptr;
    float *Pc = P ? P + h0 * g.r0_count : nullptr;
    switch (plain_shape()) {
    case 0: return launch_plain_shape<8, 2>(c, R, echo, g, nh, rho, w, e0, Yc, Pc);
    case 2: return launch_plain_shape<16, 2>(c, R, echo, g, nh, rho, w, e0, Yc, Pc);
    default: return launch_plain_shape<8, 4>(c, R, echo, g, nh, rho, w, e0, Yc, Pc);
    }
}

}  // namespace grft
