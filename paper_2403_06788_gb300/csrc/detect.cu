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
// k_topk: one CTA.  Up to 8192 candidates are sorted in shared memory (bitonic, by power
// descending, index ascending); beyond that a 4-pass radix select over the power bits
// finds the K-th largest value first and only the survivors are sorted.
#include <cstdint>

#include "internal.cuh"

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
                        cand_i[pos] = row * nr0 + n;
                    } else {
                        latch_error(status, GRFT_EOVERFLOW);
                    }
                }
            }
        }
    }
#undef SV
}

// Specialisation for compile-time guard/train counts (the default 2/16): the positions
// read around the thread's 16 bins are known at compile time, so reads inside the thread's
// own bins come from registers and the others use immediate shared-memory offsets.
template <int G, int T>
__global__ __launch_bounds__(CF_THREADS, 4) void k_cfar_fixed(const float *__restrict__ P, CfarParams cp,
                                                           int nseg, int *__restrict__ count,
                                                           float *__restrict__ cand_p,
                                                           int64_t *__restrict__ cand_i, int *status) {
    static_assert(G + T + 1 <= CF_MAXHALO && CF_MAXHALO % 16 == 0, "halo");
    constexpr int HALO = G + T + 1;
    __shared__ float sv[CF_STAGE + CF_STAGE / 16 + 1];
    const long row = blockIdx.x / nseg;
    const int seg0 = (int)(blockIdx.x % nseg) * CF_SEG;
    const int nr0 = cp.nr0;
    const float *prow = P + row * nr0;
    const int nb = seg0 + threadIdx.x * CF_PER;
    const int sb = CF_MAXHALO - seg0;
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
    float hl = 0.f, hr = 0.f;
    if (threadIdx.x < HALO) {
        const int nl = seg0 - HALO + threadIdx.x, nrr = seg0 + CF_SEG + threadIdx.x;
        hl = (nl >= 0 && nl < nr0) ? __ldg(prow + nl) : 0.f;
        hr = (nrr < nr0) ? __ldg(prow + nrr) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < CF_PER; ++q) sv[cf_slot(nb + q + sb)] = x[q];
    if (threadIdx.x < HALO) {
        sv[cf_slot(CF_MAXHALO - HALO + threadIdx.x)] = hl;
        sv[cf_slot(CF_MAXHALO + CF_SEG + threadIdx.x)] = hr;
    }
    __syncthreads();
    // staged position of bin nb + c is 16 (threadIdx.x + CF_MAXHALO/16) + c
    const float *base = sv + 17 * (threadIdx.x + CF_MAXHALO / 16);
    auto at = [&](int c) -> float {   // value of bin nb + c (c compile-time after unrolling)
        return (c >= 0 && c < CF_PER) ? x[c < 0 ? 0 : (c >= CF_PER ? CF_PER - 1 : c)]
                                      : base[c + (c >> 4)];
    };

    const int vi = (int)(row / cp.na), ai = (int)(row % cp.na);
    const bool interior = nb - G - T >= 0 && nb + CF_PER - 1 + G + T < nr0;
    const float alpha_in = cp.alpha[2 * T];
    float L = 0.f, Rr = 0.f;
#pragma unroll
    for (int c = -G - T; c <= -G - 1; ++c) L += at(c);
#pragma unroll
    for (int c = G + 1; c <= G + T; ++c) Rr += at(c);
    unsigned pmask = 0;
#pragma unroll
    for (int q = 0; q < CF_PER; ++q) {
        const int n = nb + q;
        if (q > 0) {
            L += at(q - G - 1) - at(q - G - T - 1);
            Rr += at(q + G + T) - at(q + G);
        }
        const float p = x[q];
        bool pass;
        if (interior) {
            pass = p > alpha_in * (L + Rr);
        } else {
            const int nt = window_count(n - G - T, n - G - 1, nr0) + window_count(n + G + 1, n + G + T, nr0);
            pass = nt > 0 && p > cp.alpha[nt] * (L + Rr);
        }
        if (pass && n < nr0) pmask |= 1u << q;
    }
    if (__any_sync(0xffffffffu, pmask != 0)) {
#pragma unroll 1
        for (int q = 0; q < CF_PER; ++q) {
            const int n = nb + q;
            bool pass = (pmask >> q) & 1u;
            float p = 0.f;
            if (pass) {
                p = sv[cf_slot(n + sb)];
                const long me = row * nr0 + n;
                for (int dv = -1; dv <= 1 && pass; ++dv)
                    for (int da = -1; da <= 1 && pass; ++da)
                        for (int dn = -1; dn <= 1 && pass; ++dn) {
                            if (!dv && !da && !dn) continue;
                            const int v2 = vi + dv, a2 = ai + da, n2 = n + dn;
                            if (v2 < 0 || v2 >= cp.nv || a2 < 0 || a2 >= cp.na || n2 < 0 || n2 >= nr0) continue;
                            const long o = ((long)v2 * cp.na + a2) * nr0 + n2;
                            const float po = (dv == 0 && da == 0) ? sv[cf_slot(n2 + sb)] : __ldg(P + o);
                            if (po > p || (po == p && o < me)) pass = false;
                        }
            }
            const unsigned ballot = __ballot_sync(0xffffffffu, pass);
            if (ballot) {
                const int lane = threadIdx.x & 31;
                int b0 = 0;
                if (lane == __ffs(ballot) - 1) b0 = atomicAdd(count, __popc(ballot));
                b0 = __shfl_sync(0xffffffffu, b0, __ffs(ballot) - 1);
                if (pass) {
                    const long pos = (long)b0 + __popc(ballot & ((1u << lane) - 1));
                    if (pos < CAND_CAP) {
                        cand_p[pos] = p;
                        cand_i[pos] = row * nr0 + n;
                    } else {
                        latch_error(status, GRFT_EOVERFLOW);
                    }
                }
            }
        }
    }
}

// (p, idx) ordering: larger p first, then smaller idx.
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

}  // namespace

int launch_detect(const Ctx &c, const float *P, int nv, int na, int nr0, const grft_cfar &cfar,
                  const grft_grid *axes, double dr, int K, grft_det *out, int32_t *n_out) {
    if (cfar.guard < 0 || cfar.train < 0 || cfar.guard + cfar.train + 1 > CF_MAXHALO ||
        cfar.train > 64 || K < 0 || K > TOPK_SORT)
        return GRFT_EINVAL;
    if (cfar.mode == 0 && !(cfar.pfa > 0.0 && cfar.pfa < 1.0)) return GRFT_EINVAL;
    const size_t need = 256 + (size_t)CAND_CAP * (sizeof(float) + sizeof(int64_t));
    unsigned char *ws = (unsigned char *)workspace(c, need);
    if (!ws) return GRFT_ENOMEM;
    int *count = (int *)ws;
    int64_t *cand_i = (int64_t *)(ws + 256);
    float *cand_p = (float *)(ws + 256 + CAND_CAP * sizeof(int64_t));
    if (cudaMemsetAsync(count, 0, sizeof(int), c.stream) != cudaSuccess) return GRFT_ECUDA;

    CfarParams cp;
    cp.nv = nv; cp.na = na; cp.nr0 = nr0; cp.guard = cfar.guard; cp.train = cfar.train;
    cp.mode = cfar.mode; cp.fixed = cfar.fixed_thresh;
    for (int i = 0; i <= 2 * 64; ++i) {
        cp.alpha[i] = (i == 0 || cfar.mode != 0) ? 0.f : (float)(pow(cfar.pfa, -1.0 / i) - 1.0);
    }
    const long rows = (long)nv * na;
    const int nseg = (nr0 + CF_SEG - 1) / CF_SEG;
    if (rows > 0 && nr0 > 0) {
        KernelTimer kt(c, GRFT_KERNEL_CFAR);
        if (cfar.mode == 0 && cfar.guard == 2 && cfar.train == 16)
            k_cfar_fixed<2, 16><<<(unsigned)(rows * nseg), CF_THREADS, 0, c.stream>>>(P, cp, nseg, count, cand_p,
                                                                                    cand_i, c.status);
        else
            k_cfar<<<(unsigned)(rows * nseg), CF_THREADS, 0, c.stream>>>(P, cp, nseg, count, cand_p, cand_i,
                                                                        c.status);
        int e = check_launch();
        if (e) return e;
    }
    TopkParams tp;
    tp.nv = nv; tp.na = na; tp.nr0 = nr0; tp.K = K;
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
    k_topk<<<1, TOPK_THREADS, smem, c.stream>>>(count, cand_p, cand_i, tp, out, n_out, c.status);
    return check_launch();
}

}  // namespace grft
