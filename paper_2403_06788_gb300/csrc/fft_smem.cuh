// Radix-2 transforms of power-of-two length over complex FP32 data in shared memory, done
// by a whole CTA of NT threads (every thread calls; each stage ends in __syncthreads).
// `cols` transforms of the same length, stride `ld` apart, run together: one barrier per
// stage for all of them.
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
// (exponent -).  Span h = 2^lh: butterfly b pairs i = (b >> lh) 2h + (b & (h - 1)) with i + h.
template <int NT>
__device__ __forceinline__ void fft_dif_fwd(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    const int half = 1 << (logn - 1);
    const int total = cols * half;
    for (int lh = logn - 1; lh >= 0; --lh) {
        const int h = 1 << lh;
        for (int t = threadIdx.x; t < total; t += NT) {
            const int col = t >> (logn - 1), b = t & (half - 1);
            float2 *xc = x + (long)col * ld;
            const int r = b & (h - 1), i = ((b >> lh) << (lh + 1)) + r;
            const float2 u = xc[i], v = xc[i + h];
            xc[i] = cadd2(u, v);
            xc[i + h] = cmul(csub2(u, v), conj2(tw[h + r]));
        }
        __syncthreads();
    }
}

// Inverse decimation in time, in place: bit-reversed order in, natural order out
// (exponent +, unscaled).
template <int NT>
__device__ __forceinline__ void fft_dit_inv(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    const int half = 1 << (logn - 1);
    const int total = cols * half;
    for (int lh = 0; lh < logn; ++lh) {
        const int h = 1 << lh;
        for (int t = threadIdx.x; t < total; t += NT) {
            const int col = t >> (logn - 1), b = t & (half - 1);
            float2 *xc = x + (long)col * ld;
            const int r = b & (h - 1), i = ((b >> lh) << (lh + 1)) + r;
            const float2 u = xc[i], v = cmul(xc[i + h], tw[h + r]);
            xc[i] = cadd2(u, v);
            xc[i + h] = csub2(u, v);
        }
        __syncthreads();
    }
}

}  // namespace grft
