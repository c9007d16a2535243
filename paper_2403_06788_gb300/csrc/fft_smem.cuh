// Transforms of power-of-two length (up to 2^13) over complex FP32 data in shared memory,
// done by a whole CTA of NT threads (every thread calls).  The radix-2 stages are taken four
// at a time: a thread loads the 16 elements that those stages combine, runs the stages in
// registers and stores them back, so a length-2^L transform costs ceil(L / 4) passes, each
// ending in one __syncthreads.  `cols` transforms of the same length, `ld` elements apart,
// run together.
//
// Layout: element e of a column sits at column offset fpad(e) = e + e/16 (one unused slot
// after every 16), so that in the first pass, where a thread reads up to 16 consecutive
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

// One pass of NS (<= 4) radix-2 stages with spans h0, 2 h0, .., h0 2^(NS-1), h0 = 2^S0.
// Group g of a column holds the elements i0 + h0 q, q < 2^NS, with r0 = g mod h0 and
// i0 = (g / h0) 2^NS h0 + r0; the butterfly of span h = h0 2^u pairs q and q + 2^u (bit u
// of q clear) and takes the twiddle of r = r0 + h0 (q mod 2^u).
//   DIF (forward, exponent -): stages in decreasing span; (a, b) -> (a + b, (a - b) conj(w)).
//   DIT (inverse, exponent +): stages in increasing span; b w, then (a + b w, a - b w).
// S0 is a compile-time constant (0, 4, 8 or 12), so element q of a group sits at a base
// plus an immediate offset, and so does twiddle a of a stage (tw[h + r0 + a h0]):
//   h0 = 1: i0 = 2^NS g is a multiple of 2^NS (at most 16), so i0 mod 16 + q < 16 and
//           fpad(i0 + q) = fpad(i0) + q for q < 2^NS;
//   h0 >= 16: q h0 is a multiple of 16, so fpad(i0 + q h0) = fpad(i0) + q (h0 + h0 / 16).
template <int NT, int NS, int S0, bool DIF>
__device__ __forceinline__ void fft_pass(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    constexpr int G = 1 << NS;
    constexpr int h0 = 1 << S0;
    constexpr int step = h0 == 1 ? 1 : h0 + h0 / 16;   // padded distance of consecutive q
    static_assert(h0 == 1 || h0 % 16 == 0, "passes start at span 1 or a multiple of 16");
    const int lper = logn - NS;                 // log2 of the groups per column
    for (int t = threadIdx.x; t < (cols << lper); t += NT) {
        const int col = t >> lper, g = t & ((1 << lper) - 1);
        const int r0 = g & (h0 - 1);
        const int i0 = ((g >> S0) << (S0 + NS)) + r0;
        float2 *xg = x + (long)col * ld + fpad(i0);
        float2 v[G];
#pragma unroll
        for (int q = 0; q < G; ++q) v[q] = xg[q * step];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const int u = DIF ? NS - 1 - k : k;
            const int h = h0 << u;
            const float2 *twg = tw + h + r0;
            float2 w[G / 2];
#pragma unroll
            for (int a = 0; a < (1 << u); ++a) w[a] = twg[a * h0];
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
        for (int q = 0; q < G; ++q) xg[q * step] = v[q];
    }
}

// The pass starting at stage S0: NS = min(4, logn - S0) stages, then the CTA barrier.
template <int NT, bool DIF, int S0>
__device__ __forceinline__ void fft_pass_at(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    const int ns = logn - S0 < 4 ? logn - S0 : 4;
    if (ns == 4) {
        fft_pass<NT, 4, S0, DIF>(x, cols, ld, tw, logn);
    } else if (ns == 3) {
        fft_pass<NT, 3, S0, DIF>(x, cols, ld, tw, logn);
    } else if (ns == 2) {
        fft_pass<NT, 2, S0, DIF>(x, cols, ld, tw, logn);
    } else {
        fft_pass<NT, 1, S0, DIF>(x, cols, ld, tw, logn);
    }
    __syncthreads();
}

// Forward decimation in frequency, in place: natural order in, bit-reversed order out
// (exponent -).  Passes of up to four stages (pass starts 0, 4, 8, 12) from the largest
// spans down; lengths up to 2^13.
template <int NT>
__device__ __forceinline__ void fft_dif_fwd(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    if (logn < 1) return;
    if (logn > 12) fft_pass_at<NT, true, 12>(x, cols, ld, tw, logn);
    if (logn > 8) fft_pass_at<NT, true, 8>(x, cols, ld, tw, logn);
    if (logn > 4) fft_pass_at<NT, true, 4>(x, cols, ld, tw, logn);
    fft_pass_at<NT, true, 0>(x, cols, ld, tw, logn);
}

// Inverse decimation in time, in place: bit-reversed order in, natural order out (exponent
// +, unscaled).  Passes of up to four stages from span 1 up; lengths up to 2^13.
template <int NT>
__device__ __forceinline__ void fft_dit_inv(float2 *x, int cols, int ld, const float2 *tw, int logn) {
    if (logn < 1) return;
    fft_pass_at<NT, false, 0>(x, cols, ld, tw, logn);
    if (logn > 4) fft_pass_at<NT, false, 4>(x, cols, ld, tw, logn);
    if (logn > 8) fft_pass_at<NT, false, 8>(x, cols, ld, tw, logn);
    if (logn > 12) fft_pass_at<NT, false, 12>(x, cols, ld, tw, logn);
}

}  // namespace grft
