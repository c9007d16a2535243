// Frequency-domain coarse range-migration correction, the mGIFT of Def. 2 with eq. H-RM and
// eq. pre-DFM (Alg. 1), for N a power of two:
//   S[m][k]    = sum_n s[m][n] exp(-j 2 pi k n / N)                          (range spectrum)
//   Z[c][m][j] = (1/N) sum_k S[m][k] exp(+j 2 pi k (n + delta) / N) * w_c(m),   n = r0_begin + j
// with delta = d_c(t_m) / dr (FP64), k in [-N/2, N/2) (baseband) or in [0, N) (the paper's
// positive band f_k = k f_s / N): the band-limited circular advance of each range profile
// by delta bins.  Two kernels, both one persistent CTA per row at a time
// with the N samples in shared memory:
//   k_range_fft  forward decimation in frequency of each pulse row; the spectrum is stored
//                in bit-reversed order (nothing is permuted);
//   k_rm_fd      per (cell, pulse): the spectrum times the ramp exp(j 2 pi k frac(delta) / N)
//                (two small per-row tables: a coarse and a fine factor, plus exp(-j pi f)),
//                inverse decimation in time from the bit-reversed order to natural order,
//                then the integer part of delta as an index offset when the range
//                window [r0_begin, r0_begin + r0_count) is written (times w_c and 1/N).
// Twiddles (one table per stage span) are built once per CTA with sincospif; the
// transforms are those of fft_smem.cuh.
#include "fft_smem.cuh"

namespace grft {

namespace {

constexpr int FD_THREADS = 512;
constexpr int FD_RPI = 2;                      // rows per iteration of k_rm_fd (N <= 4096)

__global__ __launch_bounds__(FD_THREADS, 2) void k_range_fft(const float2 *__restrict__ echo, int M, int N,
                                                        int logN, float2 *__restrict__ S) {
    extern __shared__ float2 fd_smem[];
    float2 *x = fd_smem, *tw = fd_smem + fft_padded(N);      // x padded (fft_smem.cuh)
    build_twiddles<FD_THREADS>(tw, N);
    for (int m = blockIdx.x; m < M; m += gridDim.x) {
        __syncthreads();
        for (int n = threadIdx.x; n < N; n += FD_THREADS) x[fpad(n)] = __ldg(echo + (long)m * N + n);
        __syncthreads();
        fft_dif_fwd<FD_THREADS>(x, 1, fft_padded(N), tw, logN);
        for (int p = threadIdx.x; p < N; p += FD_THREADS) S[(long)m * N + p] = x[fpad(p)];   // bit-reversed order
    }
}

__global__ __launch_bounds__(FD_THREADS, 2) void k_rm_fd(RadarD R, grft_dsgrid g, int cell_begin, int cell_count,
                                                    int logN, int positive, int rpi, const float2 *__restrict__ S,
                                                    const float2 *__restrict__ w_c, float2 *__restrict__ Z) {
    // rpi (1 or FD_RPI) rows per iteration: their transforms run together (at N = 4096 one
    // row has 256 groups of 16 elements, two rows keep all 512 threads busy in every pass)
    extern __shared__ float2 fd_smem[];
    const int N = R.N, Np = fft_padded(N);
    float2 *x = fd_smem, *tw = fd_smem + (long)rpi * Np;      // rpi padded rows (fft_smem.cuh), twiddles
    __shared__ float2 s_hi[FD_RPI][128], s_lo[FD_RPI][64];   // ramp factors exp(j 2 pi u f / N), u = 64 u_hi + u_lo
    const int lhi = logN > 6 ? logN - 6 : 0;    // bits of u_hi
    __shared__ long s_I[FD_RPI];                // integer advance of each row
    __shared__ float s_f[FD_RPI];               // fractional advance of each row
    __shared__ float2 s_c0[FD_RPI];             // exp(-j pi f) (baseband) or 1
    __shared__ int s_m[FD_RPI];                 // pulse of each row
    build_twiddles<FD_THREADS>(tw, N);
    const long rows = (long)cell_count * R.M;
    const float inv_n = 1.0f / (float)N;        // exact: N a power of two
    for (long row0 = (long)blockIdx.x * rpi; row0 < rows; row0 += (long)gridDim.x * rpi) {
        const int nr = (int)(rows - row0 < rpi ? rows - row0 : rpi);
        __syncthreads();                        // the previous rows' reads of x and the row tables are done
        if (threadIdx.x < nr) {                 // delta = d_c(t_m) / dr in FP64, one thread per row
            const long row = row0 + threadIdx.x;
            const int cl = (int)(row / R.M), m = (int)(row - (long)cl * R.M);
            const int c = cell_begin + cl;
            const double vc = axis_value(g.vc.start, g.vc.step, c / g.ac.count);
            const double ac = axis_value(g.ac.start, g.ac.step, c % g.ac.count);
            const double delta = __ddiv_rn(displacement(vc, ac, slow_time(m, R.prf)), R.dr);
            const double fl = floor(delta);
            const float f = (float)__dsub_rn(delta, fl);   // fractional advance in [0, 1)
            s_I[threadIdx.x] = (long)fl;        // integer advance
            s_f[threadIdx.x] = f;
            s_m[threadIdx.x] = m;
            float sn0, cs0;
            sincospif(positive ? 0.0f : -f, &sn0, &cs0);   // baseband: exp(-j pi f), k = u - N/2
            s_c0[threadIdx.x] = make_float2(cs0, sn0);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nr * (128 + 64); t += FD_THREADS) {
            const int r = t / (128 + 64), u = t - r * (128 + 64);
            const float f = s_f[r];
            float sn, cs;
            if (u < 128) {                      // stored at the bit-reversed position (see below)
                if (u >= (1 << lhi)) continue;
                sincospif(2.0f * (float)(64 * u) * f / (float)N, &sn, &cs);
                s_hi[r][brev_bits((unsigned)u, lhi)] = make_float2(cs, sn);
            } else {
                sincospif(2.0f * (float)(u - 128) * f / (float)N, &sn, &cs);
                s_lo[r][u - 128] = make_float2(cs, sn);
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < (nr << logN); t += FD_THREADS) {
            const int r = t >> logN, p = t & (N - 1);
            const int k = (int)brev_bits((unsigned)p, logN);        // natural frequency of slot p
            const int u = positive ? k : (k < N / 2 ? k + N / 2 : k - N / 2);   // positive: k; else signed k + N/2
            // u >> 6 is the bit reversal of the low lhi bits of p (up to the top bit the
            // baseband offset flips), so the table slot brev(u >> 6) is consecutive over a
            // warp's slots: conflict-free; u & 63 is the same for the whole warp (broadcast)
            const float2 ramp = cmul(s_c0[r], cmul(s_hi[r][brev_bits((unsigned)(u >> 6), lhi)], s_lo[r][u & 63]));
            x[(long)r * Np + fpad(p)] = cmul(__ldg(S + (long)s_m[r] * N + p), ramp);
        }
        __syncthreads();
        fft_dit_inv<FD_THREADS>(x, nr, Np, tw, logN);
        for (int r = 0; r < nr; ++r) {
            const long row = row0 + r;
            const float2 wm = w_c[row];         // w_c[cl][m] with row = cl M + m
            const float2 sc = make_float2(wm.x * inv_n, wm.y * inv_n);
            const long I = s_I[r];
            const float2 *xr = x + (long)r * Np;
            float2 *zrow = Z + row * g.r0_count;
            for (int j = threadIdx.x; j < g.r0_count; j += FD_THREADS) {
                const int n = (int)(((long)g.r0_begin + j + I) & (N - 1));   // mod N (a power of two)
                zrow[j] = cmul(xr[fpad(n)], sc);
            }
        }
    }
}

}  // namespace

// rpi padded rows and the twiddles
size_t fd_smem_bytes(int N, int rpi) { return ((size_t)rpi * fft_padded(N) + N) * sizeof(float2); }
static int fd_rows_per_iter(int N) { return N <= 4096 ? FD_RPI : 1; }

int launch_range_fft(const Ctx &c, const RadarD &R, const float2 *echo, float2 *S) {
    int logN = 0;
    while ((1 << logN) < R.N) ++logN;
    const size_t smem = fd_smem_bytes(R.N, 1);
    static bool attr[64] = {false};
    if (c.device >= 64) return GRFT_EUNSUPPORTED;
    if (!attr[c.device]) {                      // once per device, for the largest N served
        const int most = (int)fd_smem_bytes(8192, 1);   // >= fd_smem_bytes(4096, FD_RPI)
        if (cudaFuncSetAttribute(k_range_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, most) != cudaSuccess ||
            cudaFuncSetAttribute(k_rm_fd, cudaFuncAttributeMaxDynamicSharedMemorySize, most) != cudaSuccess)
            return GRFT_ECUDA;
        attr[c.device] = true;
    }
    const int grid = R.M < 2 * c.num_sms ? R.M : 2 * c.num_sms;
    KernelTimer kt(c, GRFT_KERNEL_COARSE_RM);
    k_range_fft<<<grid, FD_THREADS, smem, c.stream>>>(echo, R.M, R.N, logN, S);
    return check_launch();
}

int launch_rm_fd(const Ctx &c, const RadarD &R, const grft_dsgrid &g, int cell_begin, int cell_count,
                 const float2 *S, const float2 *w, float2 *Z, bool positive) {
    int logN = 0;
    while ((1 << logN) < R.N) ++logN;
    const long rows = (long)cell_count * R.M;
    if (rows == 0) return GRFT_OK;
    const int rpi = fd_rows_per_iter(R.N);
    const long iters = (rows + rpi - 1) / rpi;
    const long cap = 2L * c.num_sms * 4;        // persistent: a few CTAs per SM
    const int grid = (int)(iters < cap ? iters : cap);
    KernelTimer kt(c, GRFT_KERNEL_COARSE_RM);
    k_rm_fd<<<grid, FD_THREADS, fd_smem_bytes(R.N, rpi), c.stream>>>(R, g, cell_begin, cell_count, logN,
                                                                      positive ? 1 : 0, rpi, S, w, Z);
    return check_launch();
}

}  // namespace grft
