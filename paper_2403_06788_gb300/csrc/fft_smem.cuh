// Transforms of power-of-two length over complex FP32 data in shared memory, done by a
// whole CTA of NT threads (every thread calls; each pass ends in __syncthreads): radix-4
// passes of two radix-2 stages each, plus one radix-2 stage when log2 n is odd.  `cols`
// transforms of the same length, stride `ld` apart, run together: one barrier per pass for
// all of them.
#pragma once

#include "internal.cuh"

namespace grft {

__device__ __forceinline__ float2 cadd2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub2(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

__device__ __forceinline__ unsigned brev_bits(unsigned x, int bits) { return bits ? __brev(x) >> (32 - bits) : 0u; }

// Twiddles laid out per stage span: the butterflies of span h read tw[h + r] =
// exp(+j pi r / h), r < h, so consecutive butterflies read consecutive words (no bank
// conflicts, unlike one table read at stride n / 2h).  n entries serve every length <= n.
template <int NT>
__device__ __forceinline__ void build_twiddles(float2 *tw, int n) {
    for (int t = threadIdx.x; t < n; t += NT) {
        if (t == 0) {
            tw[0] = make_float2(1.f, 0.f);
            continue;
        }
        const int h = 1 << (31 - __clz(t)), r = t - h;
        float sn, cs;
        sincospif((float)r / (float)h, &sn, &cs);           // r / h exact (h a power of two)
        tw[t] = make_float2(cs, sn);
    }
}

// Forward decimation in frequency, in place: natural order in, bit-reversed order out
// (exponent -).  Radix-2 stage of span h = 2^lh: butterfly b pairs i = (b >> lh) 2h +
// (b & (h - 1)) with i + h, then multiplies the difference by conj(tw[h + r]).  Two
// consecutive stages (spans h, h/2) run as one radix-4 pass over the quad
// i, i + h/2, i + h, i + 3h/2 (one barrier per pass); a leading radix-2 stage when log2 n
// is odd.
template <int NT>
__device__ __forceinline__ void fft_dif_fwd(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    const int half = 1 << (logn - 1);
    int lh = logn - 1;
    if (logn & 1) {                             // radix-2 stage of span n/2
        const int h = 1 << lh;
        for (int t = threadIdx.x; t < cols * half; t += NT) {
            const int col = t >> (logn - 1), b = t & (half - 1);
            float2 *xc = x + (long)col * ld;
            const float2 u = xc[b], v = xc[b + h];
            xc[b] = cadd2(u, v);
            xc[b + h] = cmul(csub2(u, v), conj2(tw[h + b]));
        }
        __syncthreads();
        --lh;
    }
    if (logn < 2) return;
    const int quarter = 1 << (logn - 2);
    for (; lh >= 1; lh -= 2) {                  // spans h = 2^lh and h/2
        const int h = 1 << lh, g = h >> 1;
        for (int t = threadIdx.x; t < cols * quarter; t += NT) {
            const int col = t >> (logn - 2), b = t & (quarter - 1);
            float2 *xc = x + (long)col * ld;
            const int r = b & (g - 1), i = ((b >> (lh - 1)) << (lh + 1)) + r;
            const float2 x0 = xc[i], x1 = xc[i + g], x2 = xc[i + h], x3 = xc[i + h + g];
            const float2 a0 = cadd2(x0, x2), a2 = cmul(csub2(x0, x2), conj2(tw[h + r]));
            const float2 a1 = cadd2(x1, x3), a3 = cmul(csub2(x1, x3), conj2(tw[h + r + g]));
            const float2 wg = conj2(tw[g + r]);
            xc[i] = cadd2(a0, a1);
            xc[i + g] = cmul(csub2(a0, a1), wg);
            xc[i + h] = cadd2(a2, a3);
            xc[i + h + g] = cmul(csub2(a2, a3), wg);
        }
        __syncthreads();
    }
}

// Inverse decimation in time, in place: bit-reversed order in, natural order out
// (exponent +, unscaled).  Radix-2 stage of span h: x[i + h] is multiplied by tw[h + r]
// before the butterfly.  Stages h, 2h run as one radix-4 pass over i, i + h, i + 2h, i + 3h;
// a trailing radix-2 stage when log2 n is odd.
template <int NT>
__device__ __forceinline__ void fft_dit_inv(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    const int half = 1 << (logn - 1);
    int lh = 0;
    if (logn >= 2) {
        const int quarter = 1 << (logn - 2);
        for (; lh + 1 < logn; lh += 2) {        // spans h = 2^lh and 2h
            const int h = 1 << lh, h2 = h << 1;
            for (int t = threadIdx.x; t < cols * quarter; t += NT) {
                const int col = t >> (logn - 2), b = t & (quarter - 1);
                float2 *xc = x + (long)col * ld;
                const int r = b & (h - 1), i = ((b >> lh) << (lh + 2)) + r;
                const float2 wh = tw[h + r];
                const float2 x0 = xc[i], x1 = cmul(xc[i + h], wh), x2 = xc[i + h2], x3 = cmul(xc[i + h2 + h], wh);
                const float2 a0 = cadd2(x0, x1), a1 = csub2(x0, x1), a2 = cadd2(x2, x3), a3 = csub2(x2, x3);
                const float2 b2 = cmul(a2, tw[h2 + r]), b3 = cmul(a3, tw[h2 + r + h]);
                xc[i] = cadd2(a0, b2);
                xc[i + h2] = csub2(a0, b2);
                xc[i + h] = cadd2(a1, b3);
                xc[i + h2 + h] = csub2(a1, b3);
            }
            __syncthreads();
        }
    }
    if (lh < logn) {                            // radix-2 stage of span n/2
        const int h = 1 << lh;
        for (int t = threadIdx.x; t < cols * half; t += NT) {
            const int col = t >> (logn - 1), b = t & (half - 1);
            float2 *xc = x + (long)col * ld;
            const float2 u = xc[b], v = cmul(xc[b + h], tw[h + b]);
            xc[b] = cadd2(u, v);
            xc[b + h] = csub2(u, v);
        }
        __syncthreads();
    }
}

}  // namespace grft
