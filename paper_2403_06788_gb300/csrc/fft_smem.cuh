// Transforms of power-of-two length over complex FP32 data in shared memory, done by a whole
// CTA of NT threads (every thread calls).  The radix-2 stages are taken MAXNS (4, or 3 to
// halve the registers) at a time: a thread loads the 2^MAXNS elements that those stages
// combine, runs the stages in registers and stores them back, so a length-2^L transform
// costs ceil(L / MAXNS) passes, each ending in one __syncthreads.  `cols` transforms of the
// same length, `ld` elements apart, run together.
//
// Layout: element e of a column sits at column offset fpad(e) = e + e/16 (one unused slot
// after every 16), so that in the first pass, where a thread reads 2^MAXNS consecutive
// elements, the lanes of a half-warp fall on distinct banks; `ld` >= fft_padded(n).
#pragma once

#include "internal.cuh"

namespace grft {

__device__ __forceinline__ float2 cadd2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub2(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

__device__ __forceinline__ unsigned brev_bits(unsigned x, int bits) { return bits ? __brev(x) >> (32 - bits) : 0u; }

__host__ __device__ __forceinline__ int fpad(int e) { return e + (e >> 4); }
__host__ __device__ constexpr int fft_padded(int n) { return n + (n >> 4); }

// Twiddles laid out per stage span: the butterflies of span h read tw[h + r] =
// exp(+j pi r / h), r < h, so consecutive butterflies read consecutive words.  n entries
// serve every length <= n.  (Unpadded.)
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

// One pass of NS (<= 4) radix-2 stages with spans h0, 2 h0, .., h0 2^(NS-1), h0 = 2^s0.
// Group g of a column holds the elements i0 + h0 q, q < 2^NS, with r0 = g mod h0 and
// i0 = (g / h0) 2^NS h0 + r0; the butterfly of span h = h0 2^u pairs q and q + 2^u (bit u
// of q clear) and takes the twiddle of r = r0 + h0 (q mod 2^u).
//   DIF (forward, exponent -): stages in decreasing span; (a, b) -> (a + b, (a - b) conj(w)).
//   DIT (inverse, exponent +): stages in increasing span; b w, then (a + b w, a - b w).
template <int NT, int NS, bool DIF>
__device__ __forceinline__ void fft_pass(float2 *x, int cols, int ld, const float2 *tw, int logn, int s0) {
    constexpr int G = 1 << NS;
    const int h0 = 1 << s0;
    const int lper = logn - NS;                 // log2 of the groups per column
    for (int t = threadIdx.x; t < (cols << lper); t += NT) {
        const int col = t >> lper, g = t & ((1 << lper) - 1);
        float2 *xc = x + (long)col * ld;
        const int r0 = g & (h0 - 1);
        const int i0 = ((g >> s0) << (s0 + NS)) + r0;
        float2 v[G];
#pragma unroll
        for (int q = 0; q < G; ++q) v[q] = xc[fpad(i0 + (q << s0))];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const int u = DIF ? NS - 1 - k : k;
            const int h = h0 << u;
            float2 w[G / 2];
#pragma unroll
            for (int a = 0; a < (1 << u); ++a) w[a] = tw[h + r0 + (a << s0)];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                if (q & (1 << u)) continue;
                const float2 a = v[q], b = v[q + (1 << u)];
                const float2 wq = w[q & ((1 << u) - 1)];
                if (DIF) {
                    v[q] = cadd2(a, b);
                    v[q + (1 << u)] = cmul(csub2(a, b), conj2(wq));
                } else {
                    const float2 y = cmul(b, wq);
                    v[q] = cadd2(a, y);
                    v[q + (1 << u)] = csub2(a, y);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < G; ++q) xc[fpad(i0 + (q << s0))] = v[q];
    }
}

template <int NT, bool DIF, int MAXNS>
__device__ __forceinline__ void fft_pass_any(float2 *x, int cols, int ld, const float2 *tw, int logn, int s0) {
    switch (logn - s0 < MAXNS ? logn - s0 : MAXNS) {
        case 4: if constexpr (MAXNS >= 4) fft_pass<NT, 4, DIF>(x, cols, ld, tw, logn, s0); break;
        case 3: fft_pass<NT, 3, DIF>(x, cols, ld, tw, logn, s0); break;
        case 2: fft_pass<NT, 2, DIF>(x, cols, ld, tw, logn, s0); break;
        default: fft_pass<NT, 1, DIF>(x, cols, ld, tw, logn, s0); break;
    }
    __syncthreads();
}

// Forward decimation in frequency, in place: natural order in, bit-reversed order out
// (exponent -).  Passes of up to MAXNS (3 or 4) stages from the largest spans down (MAXNS 3
// halves the registers a thread holds).
template <int NT, int MAXNS = 4>
__device__ __forceinline__ void fft_dif_fwd(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    static_assert(MAXNS == 3 || MAXNS == 4, "stages per pass");
    if (logn < 1) return;
    for (int s0 = ((logn - 1) / MAXNS) * MAXNS; s0 >= 0; s0 -= MAXNS)
        fft_pass_any<NT, true, MAXNS>(x, cols, ld, tw, logn, s0);
}

// Inverse decimation in time, in place: bit-reversed order in, natural order out (exponent
// +, unscaled).  Passes of up to MAXNS stages from span 1 up.
template <int NT, int MAXNS = 4>
__device__ __forceinline__ void fft_dit_inv(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    static_assert(MAXNS == 3 || MAXNS == 4, "stages per pass");
    for (int s0 = 0; s0 < logn; s0 += MAXNS) fft_pass_any<NT, false, MAXNS>(x, cols, ld, tw, logn, s0);
}

}  // namespace grft
