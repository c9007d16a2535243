// |Y|^2 detection: CA-CFAR along r0 (or a fixed LRT threshold, eq. LRT), a 3x3x3 local
// maximum over (v, a, r0), and the K strongest detections (Alg. 3's threshold scan plus
// the on-grid estimate of eq. MLE-GRFT-FD).
//
// k_cfar: one CTA per 4096-bin row segment.  The segment and a halo of guard+train+1
// bins are staged in shared memory (all loads in flight at once, float4 where aligned,
// padded one float per 16 so that a warp's 16-bin-strided reads hit distinct banks); each
// thread scans 16 consecutive bins with a sliding training-window sum held in registers.  Cells that pass
// the threshold test compare themselves with their 26 neighbours and are appended to a
// candidate list with a warp-aggregated atomic (one atomicAdd per warp via __ballot_sync).
// HBM-bound: P is read once.
// k_cfar_tma (rows of a multiple of 32 bins) / k_cfar_pipe (any other row length) /
// k_cfar_warp (fallback): the default 2-guard / 16-train test, one warp per 1024-bin chunk
// (below).
// k_topk: one CTA.  Up to 8192 candidates are sorted in shared memory (bitonic, by power
// descending, index ascending); beyond that a 4-pass radix select over the power bits
// finds the K-th largest value first and only the survivors are sorted.
#include <cstdint>
#include <cstdlib>

#include "internal.cuh"
#include "tma.cuh"

namespace grft {

namespace {

constexpr int CF_THREADS = 256;
constexpr int CF_PER = 16;
constexpr int CF_SEG = CF_THREADS * CF_PER;
constexpr int CF_MAXHALO = 80;
constexpr int TOPK_SORT = 8192;
constexpr int TOPK_THREADS = 1024;
constexpr long CAND_CAP = 1L << 22;

struct CfarParams {
    int nv, na, nr0, guard, train, mode;
    int v_lo, v_hi;           // rows of v in [v_lo, v_hi) may be detections; the others are neighbours only
    long long idx_off;        // added to a candidate's linear index in this map (global index of a slab)
    float fixed;
    float alpha[2 * 64 + 1];   // pfa^(-1/Nt) - 1 for Nt = 0..2*train
};

__device__ __forceinline__ int window_count(int lo, int hi, int nr0) {
    lo = max(lo, 0);
    hi = min(hi, nr0 - 1);
    return hi >= lo ? hi - lo + 1 : 0;
}

// Shared-memory slot of staged position i >= 0: one pad float after every 16, so that the
// lanes of a warp, each scanning 16 consecutive bins, read distinct banks.
__device__ __forceinline__ int cf_slot(int i) { return i + (i >> 4); }
constexpr int CF_STAGE = CF_SEG + 2 * CF_MAXHALO;

__global__ __launch_bounds__(CF_THREADS) void k_cfar(const float *__restrict__ P, CfarParams cp,
                                                     int nseg, int *__restrict__ count,
                                                     float *__restrict__ cand_p,
                                                     int64_t *__restrict__ cand_i, int *status) {
    // staged position of bin n is n - seg0 + CF_MAXHALO (always >= 0)
    __shared__ float sv[CF_STAGE + CF_STAGE / 16 + 1];
    const long row = blockIdx.x / nseg;
    const int seg0 = (int)(blockIdx.x % nseg) * CF_SEG;
    const int G = cp.guard, T = cp.train, nr0 = cp.nr0;
    const int halo = G + T + 1;
    const float *prow = P + row * nr0;
    const int nb = seg0 + threadIdx.x * CF_PER;     // first bin of this thread
    const int sb = CF_MAXHALO - seg0;               // staged position of bin n is n + sb
    // every load of the segment is issued before any is used (one memory latency per CTA)
    float x[CF_PER];
    const bool vec = ((((uintptr_t)(prow + nb)) & 15) == 0) && nb + CF_PER <= nr0;
    if (vec) {
        const float4 *src = reinterpret_cast<const float4 *>(prow + nb);
#pragma unroll
        for (int q = 0; q < CF_PER / 4; ++q) {
            const float4 t = __ldcs(src + q);
            x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < CF_PER; ++q) x[q] = (nb + q < nr0) ? __ldcs(prow + nb + q) : 0.f;
    }
    float hl = 0.f, hr = 0.f;                      // halo bins left of / right of the segment
    if (threadIdx.x < halo) {
        const int nl = seg0 - halo + threadIdx.x, nrr = seg0 + CF_SEG + threadIdx.x;
        hl = (nl >= 0 && nl < nr0) ? __ldg(prow + nl) : 0.f;
        hr = (nrr < nr0) ? __ldg(prow + nrr) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < CF_PER; ++q) sv[cf_slot(nb + q + sb)] = x[q];
    if (threadIdx.x < halo) {
        sv[cf_slot(CF_MAXHALO - halo + threadIdx.x)] = hl;
        sv[cf_slot(CF_MAXHALO + CF_SEG + threadIdx.x)] = hr;
    }
    __syncthreads();
#define SV(n) sv[cf_slot((n) + sb)]

    const int vi = (int)(row / cp.na), ai = (int)(row % cp.na);
    // all 16 bins' training windows inside the row: the training-cell count is 2T
    const bool interior = nb - G - T >= 0 && nb + CF_PER - 1 + G + T < nr0;
    const float alpha_in = cp.alpha[2 * T];
    float L = 0.f, Rr = 0.f;
    if (cp.mode == 0) {
        for (int j = nb - G - T; j <= nb - G - 1; ++j) L += SV(j);
        for (int j = nb + G + 1; j <= nb + G + T; ++j) Rr += SV(j);
    }
    // threshold test of the 16 bins (hot, unrolled): a bit per passing bin
    unsigned pmask = 0;
#pragma unroll
    for (int q = 0; q < CF_PER; ++q) {
        const int n = nb + q;
        if (q > 0 && cp.mode == 0) {
            L += SV(n - G - 1) - SV(n - G - T - 1);
            Rr += SV(n + G + T) - SV(n + G);
        }
        const float p = x[q];
        bool pass;
        if (cp.mode == 0) {
            if (interior) {
                pass = p > alpha_in * (L + Rr);
            } else {
                const int nt = window_count(n - G - T, n - G - 1, nr0) + window_count(n + G + 1, n + G + T, nr0);
                pass = nt > 0 && p > cp.alpha[nt] * (L + Rr);
            }
        } else {
            pass = p > cp.fixed;
        }
        if (pass && n < nr0) pmask |= 1u << q;
    }
    if (vi < cp.v_lo || vi >= cp.v_hi) pmask = 0;   // a halo row: its cells are neighbours only
    // local-maximum test and append (rare, compact): only warps with a candidate enter,
    // and every lane of such a warp runs all 16 iterations so the ballot is convergent
    if (__any_sync(0xffffffffu, pmask != 0)) {
#pragma unroll 1
        for (int q = 0; q < CF_PER; ++q) {
            const int n = nb + q;
            bool pass = (pmask >> q) & 1u;
            float p = 0.f;
            if (pass) {
                p = SV(n);
                const long me = row * nr0 + n;
                for (int dv = -1; dv <= 1 && pass; ++dv)
                    for (int da = -1; da <= 1 && pass; ++da)
                        for (int dn = -1; dn <= 1 && pass; ++dn) {
                            if (!dv && !da && !dn) continue;
                            const int v2 = vi + dv, a2 = ai + da, n2 = n + dn;
                            if (v2 < 0 || v2 >= cp.nv || a2 < 0 || a2 >= cp.na || n2 < 0 || n2 >= nr0) continue;
                            const long o = ((long)v2 * cp.na + a2) * nr0 + n2;
                            const float po = (dv == 0 && da == 0) ? SV(n2) : __ldg(P + o);
                            if (po > p || (po == p && o < me)) pass = false;
                        }
            }
            // warp-aggregated append
            const unsigned ballot = __ballot_sync(0xffffffffu, pass);
            if (ballot) {
                const int lane = threadIdx.x & 31;
                int base = 0;
                if (lane == __ffs(ballot) - 1) base = atomicAdd(count, __popc(ballot));
                base = __shfl_sync(0xffffffffu, base, __ffs(ballot) - 1);
                if (pass) {
                    const long pos = (long)base + __popc(ballot & ((1u << lane) - 1));
                    if (pos < CAND_CAP) {
                        cand_p[pos] = p;
                        cand_i[pos] = row * nr0 + n + cp.idx_off;
                    } else {
                        latch_error(status, GRFT_EOVERFLOW);
                    }
                }
            }
        }
    }
#undef SV
}

// Local-maximum test over the 26 (v, a, r0) neighbours (ties: the lower linear index
// wins) and warp-aggregated append of the survivors.  Called by all 32 lanes; `pass` is the
// lane's threshold result for cell (row, n) of power p.
__device__ __forceinline__ void cfar_append(bool pass, const float *__restrict__ P, const CfarParams &cp,
                                            long row, int n, float p, int *__restrict__ count,
                                            float *__restrict__ cand_p, int64_t *__restrict__ cand_i,
                                            int *status) {
    const int nr0 = cp.nr0;
    if (pass) {
        const int vi = (int)(row / cp.na), ai = (int)(row % cp.na);
        if (vi < cp.v_lo || vi >= cp.v_hi) pass = false;   // a halo row: neighbours only
        const long me = row * nr0 + n;
        for (int dv = -1; dv <= 1 && pass; ++dv)
            for (int da = -1; da <= 1 && pass; ++da)
                for (int dn = -1; dn <= 1 && pass; ++dn) {
                    if (!dv && !da && !dn) continue;
                    const int v2 = vi + dv, a2 = ai + da, n2 = n + dn;
                    if (v2 < 0 || v2 >= cp.nv || a2 < 0 || a2 >= cp.na || n2 < 0 || n2 >= nr0) continue;
                    const long o = ((long)v2 * cp.na + a2) * nr0 + n2;
                    const float po = __ldg(P + o);
                    if (po > p || (po == p && o < me)) pass = false;
                }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, pass);
    if (!ballot) return;
    const int lane = threadIdx.x & 31;
    int b0 = 0;
    if (lane == __ffs(ballot) - 1) b0 = atomicAdd(count, __popc(ballot));
    b0 = __shfl_sync(0xffffffffu, b0, __ffs(ballot) - 1);
    if (pass) {
        const long pos = (long)b0 + __popc(ballot & ((1u << lane) - 1));
        if (pos < CAND_CAP) {
            cand_p[pos] = p;
            cand_i[pos] = row * nr0 + n + cp.idx_off;
        } else {
            latch_error(status, GRFT_EOVERFLOW);
        }
    }
}

// Specialisation for compile-time guard/train counts (the default 2/16), one warp per
// 1024-bin chunk of a row: lane l holds bins [32 l, 32 l + 32) of the chunk in registers
// and the G+T bins on either side of them (zeros outside the row), and slides one sum over
// both training windows across its 32 bins: four adds, a multiply and a compare per cell.
// Bins outside the row are zero, so that sum is the sum over the available training cells
// at the row ends too, and since alpha(Nt) = pfa^(-1/Nt) - 1 falls as Nt grows, a cell
// with a clipped window can only pass if it passes with the full-window alpha: the scan
// uses that one alpha, and only cells that pass are re-tested (clipped windows summed
// again with their own alpha) and compared with their 26 neighbours; they are rare.
constexpr int CW_LANE = 32;                     // bins per lane
constexpr int CW_CHUNK = 32 * CW_LANE;          // bins per warp
constexpr int CW_THREADS = 256;

// The CFAR test of chunk [c0, c0 + 1024) of row `row`: x = the lane's bins c0 + 32 l + q,
// hl / hr = bins c0 + 32 l - H + k and c0 + 32 l + 32 + k.  Called by all 32 lanes.
template <int G, int T>
__device__ __forceinline__ void cfar_chunk(const float (&x)[CW_LANE], const float (&hl)[G + T],
                                           const float (&hr)[G + T], const float *__restrict__ P,
                                           const CfarParams &cp, long row, int c0, int *__restrict__ count,
                                           float *__restrict__ cand_p, int64_t *__restrict__ cand_i,
                                           int *status) {
    constexpr int H = G + T;                    // reach of the window on either side
    static_assert(H >= 1 && H <= CW_LANE, "window reach within one neighbour lane");
    constexpr unsigned FULL = 0xffffffffu;
    auto at = [&](int c) -> float {             // bin nb + c; c is a constant after unrolling
        return c < 0 ? hl[c < 0 ? H + c : 0]
                     : (c < CW_LANE ? x[c < CW_LANE ? c : 0] : hr[c - CW_LANE < H ? c - CW_LANE : 0]);
    };
    const float alpha_in = cp.alpha[2 * T];
    float S0 = 0.f;
#pragma unroll
    for (int c = -H; c <= -G - 1; ++c) S0 += at(c);
#pragma unroll
    for (int c = G + 1; c <= H; ++c) S0 += at(c);
    bool hit = false;
    {
        float S = S0;
#pragma unroll
        for (int q = 0; q < CW_LANE; ++q) {
            if (q > 0) S += (at(q - G - 1) - at(q - H - 1)) + (at(q + H) - at(q + G));
            hit |= x[q] > alpha_in * S;
        }
    }
    if (!__any_sync(FULL, hit)) return;

    // rare: the same scan again, keeping which cells passed
    const int lane = threadIdx.x & 31;
    const int nr0 = cp.nr0;
    const float *prow = P + row * nr0;
    const int nb = c0 + lane * CW_LANE;
    unsigned pmask = 0;
    {
        float S = S0;
#pragma unroll
        for (int q = 0; q < CW_LANE; ++q) {
            if (q > 0) S += (at(q - G - 1) - at(q - H - 1)) + (at(q + H) - at(q + G));
            pmask |= (x[q] > alpha_in * S ? 1u : 0u) << q;
        }
    }
    unsigned any = __reduce_or_sync(FULL, pmask);
    while (any) {                               // warp-uniform loop over the passing offsets
        const int q = __ffs(any) - 1;
        any &= any - 1;
        const int n = nb + q;
        bool pass = ((pmask >> q) & 1u) && n < nr0;
        float p = 0.f;
        if (pass) {
            p = __ldg(prow + n);
            if (n < H || n >= nr0 - H) {        // clipped window: its own count and alpha
                float Ls = 0.f, Rs = 0.f;
                for (int j = max(n - H, 0); j <= n - G - 1; ++j) Ls += __ldg(prow + j);
                for (int j = n + G + 1; j <= min(n + H, nr0 - 1); ++j) Rs += __ldg(prow + j);
                const int nt = window_count(n - H, n - G - 1, nr0) + window_count(n + G + 1, n + H, nr0);
                pass = nt > 0 && p > cp.alpha[nt] * (Ls + Rs);
            }
        }
        cfar_append(pass, P, cp, row, n, p, count, cand_p, cand_i, status);
    }
}

// Any row length and alignment: each warp takes one chunk.  A whole chunk of a 16-byte
// aligned row is read as float4 runs per lane; any other chunk (rows whose length is not a
// multiple of 4 bins start at any 4-byte offset) is read coalesced, each load instruction
// one contiguous 128-byte run of the warp (bin c0 + 32 q + lane), and turned into the lane's
// 32 consecutive bins through a warp-private shared tile (4 pad floats per 32: conflict-free
// on both sides, 16-byte aligned runs for the reads).  The neighbouring bins come from the
// adjacent lanes by shuffles (lanes 0 and 31 load theirs).
constexpr int CW_TILE = CW_CHUNK + CW_CHUNK / 8;   // floats of a warp's tile
template <int G, int T>
__global__ __launch_bounds__(CW_THREADS, 2) void k_cfar_warp(const float *__restrict__ P, CfarParams cp,
                                                           int nch, long rows, int *__restrict__ count,
                                                           float *__restrict__ cand_p,
                                                           int64_t *__restrict__ cand_i, int *status) {
    constexpr int H = G + T;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ alignas(16) float s_tile[CW_THREADS / 32][CW_TILE];
    const int lane = threadIdx.x & 31;
    const long gw = (long)blockIdx.x * (CW_THREADS / 32) + (threadIdx.x >> 5);
    if (gw >= rows * nch) return;               // whole warp (no CTA-wide barrier below)
    const long row = gw / nch;
    const int nr0 = cp.nr0;
    const float *prow = P + row * nr0;
    const int c0 = (int)(gw % nch) * CW_CHUNK;
    const int nb = c0 + lane * CW_LANE;
    float x[CW_LANE];
    if (c0 + CW_CHUNK <= nr0 && ((((uintptr_t)(prow + c0)) & 15) == 0)) {     // warp-uniform
        const float4 *src = reinterpret_cast<const float4 *>(prow + nb);
#pragma unroll
        for (int q = 0; q < CW_LANE / 4; ++q) {
            const float4 t = __ldg(src + q);
            x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
        }
    } else {
        float *st = s_tile[threadIdx.x >> 5];
#pragma unroll
        for (int q = 0; q < CW_LANE; ++q) {     // bin c0 + 32 q + lane -> slot 36 q + lane
            const int b = c0 + 32 * q + lane;
            st[36 * q + lane] = b < nr0 ? __ldg(prow + b) : 0.f;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < CW_LANE / 4; ++q) {  // bins nb .. nb + 31 -> slots 36 lane + 0 .. 31
            const float4 t = *reinterpret_cast<const float4 *>(st + 36 * lane + 4 * q);
            x[4 * q] = t.x; x[4 * q + 1] = t.y; x[4 * q + 2] = t.z; x[4 * q + 3] = t.w;
        }
    }
    float hl[H], hr[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
        const int nl = nb - H + k, nr = nb + CW_LANE + k;
        const float vl = __shfl_up_sync(FULL, x[CW_LANE - H + k], 1);
        const float vr = __shfl_down_sync(FULL, x[k], 1);
        hl[k] = lane != 0 ? vl : ((nl >= 0 && nl < nr0) ? __ldg(prow + nl) : 0.f);
        hr[k] = lane != 31 ? vr : (nr < nr0 ? __ldg(prow + nr) : 0.f);
    }
    cfar_chunk<G, T>(x, hl, hr, P, cp, row, c0, count, cand_p, cand_i, status);
}

// Fewer than 2^31 chunks (rows at any 4-byte offset; A16: 16-byte aligned rows, nr0 % 4 ==
// 0, copied in 16-byte units, else in 4-byte units): persistent warps walk
// the chunks gw, gw + W, ... (W warps in the grid) with a CP_STAGES-deep pipeline of
// asynchronous copies into shared memory, so that two chunks per warp are in flight while
// one is tested.  Each lane copies its own 128 bytes (eight 16-byte cp.async whose
// positions are XOR-swizzled by lane, so reads are free of bank conflicts); lanes 0 and 31
// also copy the 20 bins before and after the chunk (zero-filled outside the row).  After
// the wait and a warp barrier every lane reads its bins and, from its neighbours' slots,
// the G+T bins on either side.
constexpr int CP_STAGES = 3;
constexpr int CP_HALO = 20;                               // >= G + T, multiple of 4
constexpr int CP_SEG = 32 * CW_LANE;                      // floats of the 32 lanes' slots
constexpr int CP_STAGE_FLOATS = CP_SEG + 2 * CP_HALO;     // + left and right halo slots
constexpr size_t CP_SMEM = (size_t)(CW_THREADS / 32) * CP_STAGES * CP_STAGE_FLOATS * sizeof(float);

__device__ __forceinline__ void cp_async16(float *dst, const float *src, int bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(float *dst, const float *src, int bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 16-byte chunk c (0..7) of lane l's slot inside a stage
__device__ __forceinline__ int cp_pos(int l, int c) { return l * CW_LANE + 4 * (c ^ (l & 7)); }

template <int G, int T, bool A16>
__global__ __launch_bounds__(CW_THREADS, 2) void k_cfar_pipe(const float *__restrict__ P, CfarParams cp,
                                                           int nch, int items, int *__restrict__ count,
                                                           float *__restrict__ cand_p,
                                                           int64_t *__restrict__ cand_i, int *status) {
    constexpr int H = G + T;
    static_assert(H <= CP_HALO && CP_HALO % 4 == 0 && CP_HALO <= 4 * 5, "halo copy");
    extern __shared__ float4 cf_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *wbase = reinterpret_cast<float *>(cf_smem) + (size_t)warp * CP_STAGES * CP_STAGE_FLOATS;
    const int gw = blockIdx.x * (CW_THREADS / 32) + warp;
    const int W = gridDim.x * (CW_THREADS / 32);
    const int nr0 = cp.nr0;
    // halo copies: lane 0 the CP_HALO bins before the chunk, lane 31 those after it
    const bool hlane = lane == 0 || lane == 31;
    const int hoff = lane == 0 ? -CP_HALO : CW_CHUNK;
    const int hslot = CP_SEG + (lane == 0 ? 0 : CP_HALO);

    auto prefetch = [&](int i, int stage) {
        float *st = wbase + stage * CP_STAGE_FLOATS;
        if (i < items) {
            const unsigned row = (unsigned)i / (unsigned)nch;
            const int c0 = (int)((unsigned)i - row * (unsigned)nch) * CW_CHUNK;
            const float *prow = P + (size_t)row * nr0;
            const int nb = c0 + lane * CW_LANE;
            if constexpr (!A16) {
                // rows at any 4-byte offset: 4-byte copies, each instruction one contiguous
                // 128-byte run of the warp (bin c0 + 32 q + lane into its owner lane q's
                // slot), and the halo bins one per lane (lanes 0..19, both sides)
#pragma unroll
                for (int q = 0; q < CW_LANE; ++q) {
                    const int b = c0 + 32 * q + lane;
                    const bool in = b < nr0;
                    cp_async4(st + cp_pos(q, lane >> 2) + (lane & 3), in ? prow + b : prow, in ? 4 : 0);
                }
                if (lane < CP_HALO) {
                    const int bl = c0 - CP_HALO + lane, br = c0 + CW_CHUNK + lane;
                    const bool il = bl >= 0 && bl < nr0, ir = br < nr0;
                    cp_async4(st + CP_SEG + lane, il ? prow + bl : prow, il ? 4 : 0);
                    cp_async4(st + CP_SEG + CP_HALO + lane, ir ? prow + br : prow, ir ? 4 : 0);
                }
            } else if (c0 + CW_CHUNK <= nr0) {
#pragma unroll
                for (int c = 0; c < CW_LANE / 4; ++c) cp_async16(st + cp_pos(lane, c), prow + nb + 4 * c, 16);
            } else {
#pragma unroll
                for (int c = 0; c < CW_LANE / 4; ++c) {
                    const int b = nb + 4 * c;
                    const bool in = b < nr0;             // nr0 % 4 == 0: whole 16-byte runs
                    cp_async16(st + cp_pos(lane, c), in ? prow + b : prow, in ? 16 : 0);
                }
            }
            if (A16 && hlane) {
#pragma unroll
                for (int c = 0; c < CP_HALO / 4; ++c) {
                    const int b = c0 + hoff + 4 * c;
                    const bool in = b >= 0 && b < nr0;
                    cp_async16(st + hslot + 4 * c, in ? prow + b : prow, in ? 16 : 0);
                }
            }
        }
        cp_async_commit();                      // one group per item, empty past the end
    };

#pragma unroll
    for (int t = 0; t < CP_STAGES - 1; ++t) prefetch(gw + t * W, t);
    for (int t = 0;; ++t) {
        const int i = gw + t * W;               // items + W < 2^31 (host check)
        if (i >= items) break;                  // warp-uniform
        const float *st = wbase + (t % CP_STAGES) * CP_STAGE_FLOATS;
        cp_async_wait<CP_STAGES - 2>();         // this lane's copies of item t have landed
        __syncwarp();                           // ... and every lane's
        float x[CW_LANE];
#pragma unroll
        for (int c = 0; c < CW_LANE / 4; ++c) {
            const float4 v = *reinterpret_cast<const float4 *>(st + cp_pos(lane, c));
            x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
        }
        // bins before the lane's: chunks 3..7 of lane l-1 (its bins 12..31), or the left
        // halo slot for lane 0; bins after: chunks 0..4 of lane l+1, or the right slot
        float lv[CP_HALO], rv[CP_HALO];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float4 a = *reinterpret_cast<const float4 *>(
                st + (lane == 0 ? CP_SEG + 4 * c : cp_pos(lane - 1, 3 + c)));
            const float4 b = *reinterpret_cast<const float4 *>(
                st + (lane == 31 ? CP_SEG + CP_HALO + 4 * c : cp_pos(lane + 1, c)));
            lv[4 * c] = a.x; lv[4 * c + 1] = a.y; lv[4 * c + 2] = a.z; lv[4 * c + 3] = a.w;
            rv[4 * c] = b.x; rv[4 * c + 1] = b.y; rv[4 * c + 2] = b.z; rv[4 * c + 3] = b.w;
        }
        float hl[H], hr[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            hl[k] = lv[CP_HALO - H + k];
            hr[k] = rv[k];
        }
        __syncwarp();                           // all reads of this stage done before it is refilled
        prefetch(gw + (t + CP_STAGES - 1) * W, (t + CP_STAGES - 1) % CP_STAGES);
        const unsigned row = (unsigned)i / (unsigned)nch;
        cfar_chunk<G, T>(x, hl, hr, P, cp, (long)row, (int)((unsigned)i - row * (unsigned)nch) * CW_CHUNK,
                         count, cand_p, cand_i, status);
    }
    cp_async_wait<0>();
}

// Rows of a multiple of 32 bins: the same pipeline with each chunk moved by one tensor-map
// copy.  The chunk's 1024 bins, viewed as 32 lines of 32 floats (a 3-D map {32, nr0/32,
// rows}), land with the 128-byte swizzle, which is exactly the cp_pos layout above (16-byte
// unit c of line l at c ^ (l & 7)); the 20 bins on either side come from a 2-D map {nr0,
// rows} whose boxes past the row's ends are zero-filled by the copy engine.  Lane 0 issues
// the three copies of a chunk on the stage's mbarrier; every wait is bounded (a wait that
// runs out latches GRFT_ETIMEOUT, and the warp waits, again bounded, for the copies it
// still has in flight before it leaves).
constexpr size_t CT_CHUNK_BYTES = CW_CHUNK * sizeof(float);                      // 4096
constexpr size_t CT_HALO_BYTES = 2 * CP_HALO * sizeof(float);                     // 160 copied per chunk
constexpr size_t CT_HALO_SLOT = 128;                                              // a copy's destination: 128-byte aligned
constexpr size_t CT_SMEM = 1024 + (size_t)(CW_THREADS / 32) * CP_STAGES * (CT_CHUNK_BYTES + 2 * CT_HALO_SLOT);

template <int G, int T>
__global__ __launch_bounds__(CW_THREADS, 2) void k_cfar_tma(const __grid_constant__ CUtensorMap mapc,
                                                          const __grid_constant__ CUtensorMap maph, CfarParams cp,
                                                          int nch, int items, int *__restrict__ count,
                                                          float *__restrict__ cand_p, int64_t *__restrict__ cand_i,
                                                          int *status, uint64_t limit, const float *__restrict__ P) {
    constexpr int H = G + T;
    constexpr int WARPS = CW_THREADS / 32;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(H <= CP_HALO && CP_HALO % 4 == 0 && CP_HALO <= 4 * 5, "halo copy");
    extern __shared__ unsigned char ct_raw[];
    __shared__ alignas(8) uint64_t bars[WARPS][CP_STAGES];
    unsigned char *base = (unsigned char *)(((uintptr_t)ct_raw + 1023) & ~(uintptr_t)1023);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *chunks = reinterpret_cast<float *>(base) + (size_t)warp * CP_STAGES * CW_CHUNK;
    // per (warp, stage): the left halo at a 128-byte slot, the right one at the next
    unsigned char *halos = base + (size_t)WARPS * CP_STAGES * CT_CHUNK_BYTES +
                           (size_t)warp * CP_STAGES * 2 * CT_HALO_SLOT;
    uint64_t *bar = bars[warp];
    if (lane == 0) {
        for (int st = 0; st < CP_STAGES; ++st) mbar_init(&bar[st], 1);
        fence_mbarrier_init();
    }
    __syncwarp();
    const int gw = blockIdx.x * WARPS + warp;
    const int W = gridDim.x * WARPS;

    auto prefetch = [&](int i, int stage) {
        if (lane == 0 && i < items) {
            const unsigned row = (unsigned)i / (unsigned)nch;
            const int c0 = (int)((unsigned)i - row * (unsigned)nch) * CW_CHUNK;
            mbar_arrive_expect_tx(&bar[stage], (uint32_t)(CT_CHUNK_BYTES + CT_HALO_BYTES));
            tma_load_3d(chunks + stage * CW_CHUNK, &mapc, 0, c0 / 32, (int)row, &bar[stage]);
            unsigned char *hs = halos + stage * 2 * CT_HALO_SLOT;
            tma_load_2d(hs, &maph, c0 - CP_HALO, (int)row, &bar[stage]);
            tma_load_2d(hs + CT_HALO_SLOT, &maph, c0 + CW_CHUNK, (int)row, &bar[stage]);
        }
    };

#pragma unroll
    for (int t = 0; t < CP_STAGES - 1; ++t) prefetch(gw + t * W, t);
    int t = 0;
    bool ok = true;
    for (;; ++t) {
        const int i = gw + t * W;               // items + W < 2^31 (host check)
        if (i >= items) break;                  // warp-uniform
        const int stage = t % CP_STAGES;
        const uint32_t parity = (uint32_t)(t / CP_STAGES) & 1u;
        int good = 1;
        if (lane == 0) good = mbar_wait(&bar[stage], parity, limit) ? 1 : 0;
        good = __shfl_sync(FULL, good, 0);
        if (!good) {
            if (lane == 0) latch_error(status, GRFT_ETIMEOUT);
            ok = false;
            break;
        }
        mbar_try_wait(&bar[stage], parity);     // completed: every lane acquires the copied data
        const float *st = chunks + stage * CW_CHUNK;
        const float *hsl = reinterpret_cast<const float *>(halos + stage * 2 * CT_HALO_SLOT);
        const float *hsr = reinterpret_cast<const float *>(halos + stage * 2 * CT_HALO_SLOT + CT_HALO_SLOT);
        float x[CW_LANE];
#pragma unroll
        for (int c = 0; c < CW_LANE / 4; ++c) {
            const float4 v = *reinterpret_cast<const float4 *>(st + cp_pos(lane, c));
            x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
        }
        float lv[CP_HALO], rv[CP_HALO];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float4 a = *reinterpret_cast<const float4 *>(lane == 0 ? hsl + 4 * c : st + cp_pos(lane - 1, 3 + c));
            const float4 b = *reinterpret_cast<const float4 *>(lane == 31 ? hsr + 4 * c : st + cp_pos(lane + 1, c));
            lv[4 * c] = a.x; lv[4 * c + 1] = a.y; lv[4 * c + 2] = a.z; lv[4 * c + 3] = a.w;
            rv[4 * c] = b.x; rv[4 * c + 1] = b.y; rv[4 * c + 2] = b.z; rv[4 * c + 3] = b.w;
        }
        float hl[H], hr[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            hl[k] = lv[CP_HALO - H + k];
            hr[k] = rv[k];
        }
        __syncwarp();                           // all reads of this stage done before it is refilled
        prefetch(gw + (t + CP_STAGES - 1) * W, (t + CP_STAGES - 1) % CP_STAGES);
        const unsigned row = (unsigned)i / (unsigned)nch;
        cfar_chunk<G, T>(x, hl, hr, P, cp, (long)row, (int)((unsigned)i - row * (unsigned)nch) * CW_CHUNK,
                         count, cand_p, cand_i, status);
    }
    if (!ok && lane == 0) {                     // copies still in flight: items t .. t + STAGES - 2
        for (int u = t; u < t + CP_STAGES - 1; ++u)
            if (gw + u * W < items) mbar_wait(&bar[u % CP_STAGES], (uint32_t)(u / CP_STAGES) & 1u, limit);
    }
    __syncwarp();
}

__device__ __forceinline__ bool before(float pa, int64_t ia, float pb, int64_t ib) {
    return pa > pb || (pa == pb && ia < ib);
}

__device__ void bitonic_sort(float *kp, int64_t *ki, int n) {   // n power of two
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool asc = (i & size) == 0;   // "ascending" in the before() order
                    const bool sw = asc ? before(kp[j], ki[j], kp[i], ki[i])
                                        : before(kp[i], ki[i], kp[j], ki[j]);
                    if (sw) {
                        float tp = kp[i]; kp[i] = kp[j]; kp[j] = tp;
                        int64_t ti = ki[i]; ki[i] = ki[j]; ki[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
}

struct TopkParams {
    int nv, na, nr0, K;
    int has_axes;
    int r0_begin;
    double dr, v0, dv, a0, da;
};

__global__ __launch_bounds__(TOPK_THREADS) void k_topk(const int *__restrict__ count,
                                                       const float *__restrict__ cand_p,
                                                       const int64_t *__restrict__ cand_i,
                                                       TopkParams tp, grft_det *__restrict__ out,
                                                       int32_t *__restrict__ n_out, int *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t *ki = reinterpret_cast<int64_t *>(smem);
    float *kp = reinterpret_cast<float *>(smem + sizeof(int64_t) * TOPK_SORT);
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_mask, s_remaining, s_n;

    const int total = *count;
    const int n = (int)min((long)total, CAND_CAP);
    const int K = tp.K;
    if (threadIdx.x == 0) {
        s_prefix = 0;
        s_mask = 0;
        s_remaining = (unsigned)K;
        s_n = 0;
    }
    __syncthreads();
    if (n > TOPK_SORT) {
        // radix select of the K-th largest power (power >= 0, so its bits order like uints)
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 24 - 8 * pass;
            for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            const unsigned pre = s_prefix, msk = s_mask;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const unsigned b = __float_as_uint(cand_p[i]);
                if ((b & msk) == pre) atomicAdd(&hist[(b >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned rem = s_remaining, cum = 0;
                int d = 255;
                for (; d > 0; --d) {
                    if (cum + hist[d] >= rem) break;
                    cum += hist[d];
                }
                s_remaining = rem - cum;
                s_prefix = pre | ((unsigned)d << shift);
                s_mask = msk | (255u << shift);
            }
            __syncthreads();
        }
        const unsigned thr = s_prefix;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned b = __float_as_uint(cand_p[i]);
            if (b >= thr) {
                const unsigned pos = atomicAdd(&s_n, 1u);
                if (pos < (unsigned)TOPK_SORT) {
                    kp[pos] = cand_p[i];
                    ki[pos] = cand_i[i];
                }
            }
        }
        __syncthreads();
        if (s_n > (unsigned)TOPK_SORT && threadIdx.x == 0) latch_error(status, GRFT_EOVERFLOW);
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            kp[i] = cand_p[i];
            ki[i] = cand_i[i];
        }
        if (threadIdx.x == 0) s_n = (unsigned)n;
    }
    __syncthreads();
    const int m = (int)min(s_n, (unsigned)TOPK_SORT);
    int np2 = 1;
    while (np2 < m) np2 <<= 1;
    for (int i = m + threadIdx.x; i < np2; i += blockDim.x) {
        kp[i] = -1.0f;
        ki[i] = INT64_MAX;
    }
    __syncthreads();
    if (np2 > 1) bitonic_sort(kp, ki, np2);
    const int nw = min(K, m);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) {
        grft_det d;
        const int64_t idx = ki[i];
        d.idx = idx;
        d.n0 = (int)(idx % tp.nr0);
        d.ai = (int)((idx / tp.nr0) % tp.na);
        d.vi = (int)(idx / ((int64_t)tp.nr0 * tp.na));
        d.p = kp[i];
        if (tp.has_axes) {
            d.r0_m = __dmul_rn((double)(tp.r0_begin + d.n0), tp.dr);
            d.v = axis_value(tp.v0, tp.dv, d.vi);
            d.a = axis_value(tp.a0, tp.da, d.ai);
        } else {
            d.r0_m = d.v = d.a = 0.0;
        }
        out[i] = d;
    }
    if (threadIdx.x == 0) *n_out = total;
}

// Merge of detection lists (the top-K lists of the slabs or ranks a map was split into; each
// list sorted or not): the records of every list, up to min(K_in, totals[l]) from list l, are
// sorted by power descending, index ascending (a bitonic sort in shared memory of the power,
// the index and the record's position) and the first K written.  Linear indices are unique
// across the lists, so the order is total and the result is the top K of the union.
__global__ __launch_bounds__(TOPK_THREADS) void k_merge_dets(const grft_det *__restrict__ in,
                                                             const int32_t *__restrict__ totals, int L, int K_in,
                                                             int K, grft_det *__restrict__ out,
                                                             int32_t *__restrict__ n_out, int *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    int64_t *ki = reinterpret_cast<int64_t *>(smem);
    float *kp = reinterpret_cast<float *>(smem + sizeof(int64_t) * TOPK_SORT);
    int *kpos = reinterpret_cast<int *>(smem + (sizeof(int64_t) + sizeof(float)) * TOPK_SORT);
    __shared__ int s_off[TOPK_THREADS + 1];
    __shared__ long long s_total;
    if (threadIdx.x == 0) {                  // list offsets (L <= TOPK_THREADS, checked by the launcher)
        int off = 0;
        long long tot = 0;
        for (int l = 0; l < L; ++l) {
            s_off[l] = off;
            const int t = totals[l] > 0 ? totals[l] : 0;
            off += t < K_in ? t : K_in;
            tot += t;
        }
        s_off[L] = off;
        s_total = tot;
        if (off > TOPK_SORT) latch_error(status, GRFT_EOVERFLOW);
    }
    __syncthreads();
    const int m = min(s_off[L], TOPK_SORT);
    for (int l = 0; l < L; ++l)
        for (int i = threadIdx.x; s_off[l] + i < min(s_off[l + 1], m); i += blockDim.x) {
            const int slot = s_off[l] + i;
            const grft_det &d = in[(long)l * K_in + i];
            kp[slot] = d.p;
            ki[slot] = d.idx;
            kpos[slot] = l * K_in + i;
        }
    int np2 = 1;
    while (np2 < m) np2 <<= 1;
    for (int i = m + threadIdx.x; i < np2; i += blockDim.x) {
        kp[i] = -1.0f;
        ki[i] = INT64_MAX;
        kpos[i] = -1;
    }
    __syncthreads();
    for (int size = 2; size <= np2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < np2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool asc = (i & size) == 0;
                    const bool sw = asc ? before(kp[j], ki[j], kp[i], ki[i]) : before(kp[i], ki[i], kp[j], ki[j]);
                    if (sw) {
                        const float tp = kp[i]; kp[i] = kp[j]; kp[j] = tp;
                        const int64_t ti = ki[i]; ki[i] = ki[j]; ki[j] = ti;
                        const int tq = kpos[i]; kpos[i] = kpos[j]; kpos[j] = tq;
                    }
                }
            }
            __syncthreads();
        }
    const int nw = min(K, m);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) out[i] = in[kpos[i]];
    if (threadIdx.x == 0) *n_out = (int32_t)min(s_total, (long long)0x7fffffff);
}

}  // namespace

namespace {

struct DetectWs {
    int *count;
    int64_t *cand_i;
    float *cand_p;
};

bool detect_ws(const Ctx &c, DetectWs &w) {
    const size_t need = 256 + (size_t)CAND_CAP * (sizeof(float) + sizeof(int64_t));
    unsigned char *ws = (unsigned char *)workspace(c, need, WS_DETECT);
    if (!ws) return false;
    w.count = (int *)ws;
    w.cand_i = (int64_t *)(ws + 256);
    w.cand_p = (float *)(ws + 256 + CAND_CAP * sizeof(int64_t));
    return true;
}

bool cfar_ok(const grft_cfar &cfar) {
    if (cfar.guard < 0 || cfar.train < 0 || cfar.guard + cfar.train + 1 > CF_MAXHALO || cfar.train > 64)
        return false;
    return !(cfar.mode == 0 && !(cfar.pfa > 0.0 && cfar.pfa < 1.0));
}

}  // namespace

int launch_detect_begin(const Ctx &c) {
    DetectWs w;
    if (!detect_ws(c, w)) return GRFT_ENOMEM;
    return cudaMemsetAsync(w.count, 0, sizeof(int), c.stream) == cudaSuccess ? GRFT_OK : GRFT_ECUDA;
}

int launch_detect_scan(const Ctx &c, const float *P, int nv, int na, int nr0, int v_lo, int v_hi,
                       long long idx_off, const grft_cfar &cfar) {
    if (!cfar_ok(cfar)) return GRFT_EINVAL;
    DetectWs w;
    if (!detect_ws(c, w)) return GRFT_ENOMEM;
    int *count = w.count;
    int64_t *cand_i = w.cand_i;
    float *cand_p = w.cand_p;

    CfarParams cp;
    cp.nv = nv; cp.na = na; cp.nr0 = nr0; cp.guard = cfar.guard; cp.train = cfar.train;
    cp.mode = cfar.mode; cp.fixed = cfar.fixed_thresh;
    cp.v_lo = v_lo; cp.v_hi = v_hi; cp.idx_off = idx_off;
    for (int i = 0; i <= 2 * 64; ++i) {
        cp.alpha[i] = (i == 0 || cfar.mode != 0) ? 0.f : (float)(pow(cfar.pfa, -1.0 / i) - 1.0);
    }
    const long rows = (long)nv * na;
    const int nseg = (nr0 + CF_SEG - 1) / CF_SEG;
    if (rows > 0 && nr0 > 0 && v_hi > v_lo) {
        KernelTimer kt(c, GRFT_KERNEL_CFAR);
        if (cfar.mode == 0 && cfar.guard == 2 && cfar.train == 16) {
            const int nch = (nr0 + CW_CHUNK - 1) / CW_CHUNK;
            const long warps = rows * nch;
            const long blocks = (warps + CW_THREADS / 32 - 1) / (CW_THREADS / 32);
            if (blocks > 0x7fffffffL) return GRFT_EINVAL;
            static bool pipe_attr[64] = {false}, pipe4_attr[64] = {false}, tma_attr[64] = {false};
            const bool fits = c.device < 64 && warps + 2L * c.num_sms * (CW_THREADS / 32) * CP_STAGES < 0x7fffffffL;
            // DSGRFT_CFAR_WARP (read per call) forces the fallback kernel, which the tests compare
            const bool force_warp = getenv("DSGRFT_CFAR_WARP") != nullptr;
            const bool aligned = !force_warp && fits && (nr0 % 4) == 0 && (((uintptr_t)P) & 15) == 0;
            const bool pipe4 = !force_warp && fits && !aligned && (((uintptr_t)P) & 3) == 0;
            CUtensorMap mapc, maph;
            bool use_tma = aligned && (nr0 % 32) == 0;
            if (use_tma) {
                const uint64_t dims[3] = {32, (uint64_t)nr0 / 32, (uint64_t)rows};
                const uint64_t strides[2] = {128, (uint64_t)nr0 * sizeof(float)};
                const uint32_t box[3] = {32, 32, 1};
                use_tma = encode_tma_3d(&mapc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (void *)P, dims, strides, box,
                                        CU_TENSOR_MAP_SWIZZLE_128B) &&
                          encode_tma_2d(&maph, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (void *)P, (uint64_t)nr0,
                                        (uint64_t)rows, (uint64_t)nr0 * sizeof(float), CP_HALO, 1,
                                        CU_TENSOR_MAP_SWIZZLE_NONE);
            }
            if (use_tma && !tma_attr[c.device]) {
                if (cudaFuncSetAttribute(k_cfar_tma<2, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CT_SMEM) != cudaSuccess)
                    return GRFT_ECUDA;
                tma_attr[c.device] = true;
            }
            if (aligned && !pipe_attr[c.device]) {
                if (cudaFuncSetAttribute(k_cfar_pipe<2, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CP_SMEM) != cudaSuccess)
                    return GRFT_ECUDA;
                pipe_attr[c.device] = true;
            }
            if (pipe4 && !pipe4_attr[c.device]) {
                if (cudaFuncSetAttribute(k_cfar_pipe<2, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CP_SMEM) != cudaSuccess)
                    return GRFT_ECUDA;
                pipe4_attr[c.device] = true;
            }
            if (use_tma) {
                const long pblocks = blocks < 2L * c.num_sms ? blocks : 2L * c.num_sms;
                k_cfar_tma<2, 16><<<(unsigned)pblocks, CW_THREADS, CT_SMEM, c.stream>>>(
                    mapc, maph, cp, nch, (int)warps, count, cand_p, cand_i, c.status, c.wait_limit, P);
            } else if (aligned || pipe4) {
                const long pblocks = blocks < 2L * c.num_sms ? blocks : 2L * c.num_sms;
                if (aligned)
                    k_cfar_pipe<2, 16, true><<<(unsigned)pblocks, CW_THREADS, CP_SMEM, c.stream>>>(
                        P, cp, nch, (int)warps, count, cand_p, cand_i, c.status);
                else
                    k_cfar_pipe<2, 16, false><<<(unsigned)pblocks, CW_THREADS, CP_SMEM, c.stream>>>(
                        P, cp, nch, (int)warps, count, cand_p, cand_i, c.status);
            } else {
                k_cfar_warp<2, 16><<<(unsigned)blocks, CW_THREADS, 0, c.stream>>>(P, cp, nch, rows, count, cand_p,
                                                                                  cand_i, c.status);
            }
        } else
            k_cfar<<<(unsigned)(rows * nseg), CF_THREADS, 0, c.stream>>>(P, cp, nseg, count, cand_p, cand_i,
                                                                        c.status);
        int e = check_launch();
        if (e) return e;
    }
    return GRFT_OK;
}

int launch_detect_select(const Ctx &c, int na, int nr0, const grft_grid *axes, double dr, int K, grft_det *out,
                         int32_t *n_out) {
    if (K < 0 || K > TOPK_SORT) return GRFT_EINVAL;
    DetectWs w;
    if (!detect_ws(c, w)) return GRFT_ENOMEM;
    TopkParams tp;
    tp.nv = 0; tp.na = na; tp.nr0 = nr0; tp.K = K;
    tp.has_axes = axes != nullptr;
    tp.r0_begin = axes ? axes->r0_begin : 0;
    tp.dr = dr;
    tp.v0 = axes ? axes->v.start : 0.0; tp.dv = axes ? axes->v.step : 0.0;
    tp.a0 = axes ? axes->a.start : 0.0; tp.da = axes ? axes->a.step : 0.0;
    const size_t smem = (size_t)TOPK_SORT * (sizeof(int64_t) + sizeof(float));
    static bool attr_set[64] = {false};
    if (c.device < 64 && !attr_set[c.device]) {
        if (cudaFuncSetAttribute(k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return GRFT_ECUDA;
        attr_set[c.device] = true;
    }
    KernelTimer kt(c, GRFT_KERNEL_TOPK);
    k_topk<<<1, TOPK_THREADS, smem, c.stream>>>(w.count, w.cand_p, w.cand_i, tp, out, n_out, c.status);
    return check_launch();
}

int launch_detect_merge(const Ctx &c, const grft_det *lists, const int32_t *totals, int n_lists, int K_in, int K,
                        grft_det *out, int32_t *n_out) {
    if (n_lists <= 0 || n_lists > TOPK_THREADS || K_in < 0 || K < 0 || K > TOPK_SORT ||
        (long)n_lists * K_in > TOPK_SORT)
        return GRFT_EINVAL;
    const size_t smem = (size_t)TOPK_SORT * (sizeof(int64_t) + sizeof(float) + sizeof(int));
    static bool attr_set[64] = {false};
    if (c.device < 64 && !attr_set[c.device]) {
        if (cudaFuncSetAttribute(k_merge_dets, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return GRFT_ECUDA;
        attr_set[c.device] = true;
    }
    KernelTimer kt(c, GRFT_KERNEL_TOPK);
    k_merge_dets<<<1, TOPK_THREADS, smem, c.stream>>>(lists, totals, n_lists, K_in, K, out, n_out, c.status);
    return check_launch();
}

int launch_detect(const Ctx &c, const float *P, int nv, int na, int nr0, const grft_cfar &cfar,
                  const grft_grid *axes, double dr, int K, grft_det *out, int32_t *n_out) {
    if (!cfar_ok(cfar) || K < 0 || K > TOPK_SORT) return GRFT_EINVAL;
    int e;
    if ((e = launch_detect_begin(c))) return e;
    if ((e = launch_detect_scan(c, P, nv, na, nr0, 0, nv, 0, cfar))) return e;
    return launch_detect_select(c, na, nr0, axes, dr, K, out, n_out);
}

}  // namespace grft
