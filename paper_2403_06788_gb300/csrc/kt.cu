// Keystone-transform branch, DS-KT-MFP (Sec. III-B eq. Echo-after-KT; Cor. 1 / Prop. 3 /
// Alg. 4), for power-of-two M (16..2048) and N (4..8192).
//
// k_keystone: per range-frequency slot p (frequency k = bitrev(p), signed k_s, the layout
// k_range_fft leaves), the slow-time column y[m] is resampled at t = fbar t',
// fbar = f_c / (f_c + f_k) = 1 + eps, f_k / f_c = k_s lambda / (2 N dr), as a band-limited
// periodic sequence:
//   Y[l] = sum_m y[m] exp(-j 2 pi l m / M),   l in [-M/2, M/2)
//   y_KT[m'] = (1/M) sum_l Y[l] exp(+j 2 pi fbar l m' / M)
// The second sum is a chirp-z transform (Bluestein): with alpha = fbar / M and
// l m' = (l^2 + m'^2 - (m' - l)^2) / 2,
//   y_KT[m'] = (1/M) c(m') sum_l [Y[l] c(l)] conj(c(m' - l)),   c(x) = exp(j pi alpha x^2),
// a linear convolution evaluated as a circular one of length P = 2M by three P-point
// transforms.  A CTA takes `cols` adjacent slots (one 32-byte sector per pulse row) and runs
// all their transforms together in shared memory.  The chirp angle alpha x^2 (in half
// turns) is x^2 / M mod 2 in integers plus eps x^2 / M in compensated FP32, reduced, then
// an FP32 sincospi.
//
// k_rm_kt: per (cell, pulse), the coarse correction of the post-KT spectra, H_KT,RM of
// eq. H-MFP-RM with the cell's q V_a and c_2,c = a_c / 2:
//   exp(+j 2 pi k_s (fbar vq t - c_2,c t^2) / (N dr))
//     = exp(+j 2 pi k_s D / N) * exp(+j 2 pi E_k delta1),
//   delta1 = vq t / dr, D = delta1 - c_2,c t^2 / dr, E_k = k_s eps_k / N,
// i.e. the band-limited advance by D bins (fractional part f as a ramp, integer part as an
// index offset on output, as in k_rm_fd) times a small dispersive factor, one sincospi of
// k_s f / N + E_k delta1 turns per element; then the inverse transform, the range window,
// times H_pre-DFM = exp(j 4 pi c_2,c t^2 / lambda) and 1/N.
#include "fft_smem.cuh"

namespace grft {

namespace {

constexpr int KT_THREADS = 512;
constexpr int KT_RPI = 2;                      // rows per iteration of k_rm_kt (N <= 4096)

// eps = fbar - 1 of slot p in FP64.
__device__ __forceinline__ double kt_eps(int p, int logN, int N, double lam_2ndr) {
    const int k = (int)brev_bits((unsigned)p, logN);
    const int ks = k < N / 2 ? k : k - N;
    const double u = __dmul_rn((double)ks, lam_2ndr);        // f_k / f_c
    return -__ddiv_rn(u, __dadd_rn(1.0, u));                  // fbar - 1
}

// exp(j pi (1 + eps) x^2 / M) for |x| <= 3M/2, M = 2^logM <= 2048, in FP32 without loss:
// x^2 < 2^24 and X = x^2 / M are exact; x^2 / M mod 2 is exact in integers; eps = hi + lo
// (an FP32 pair) and the rounding error of hi X is recovered exactly by an FMA; the large
// part hi X is reduced mod 2 exactly before the small terms are added.
__device__ __forceinline__ float2 kt_chirp(int x, int logM, float2 eps) {
    const int xx = x * x;
    const int M = 1 << logM;
    const float inv_m = 1.0f / (float)M;
    const float X = (float)xx * inv_m;
    const float base = (float)(xx & (2 * M - 1)) * inv_m;              // [0, 2)
    const float p = eps.x * X;
    const float perr = fmaf(eps.x, X, -p);
    float h = base + (p - 2.0f * rintf(0.5f * p));
    h += fmaf(eps.y, X, perr);
    h -= 2.0f * rintf(0.5f * h);                                       // [-1, 1]
    float s, c;
    sincospif(h, &s, &c);
    return make_float2(c, s);
}

__global__ __launch_bounds__(KT_THREADS, 2) void k_keystone(const float2 *__restrict__ S, int M, int N, int logM,
                                                       int logN, int cols, double lam_2ndr,
                                                       float2 *__restrict__ Skt) {
    extern __shared__ float2 kt_smem[];
    const int P = 2 * M, logP = logM + 1, Pp = fft_padded(P);   // columns padded (fft_smem.cuh)
    float2 *b0 = kt_smem;                       // [cols][Pp]: Doppler spectrum, then the chirp kernel
    float2 *b1 = kt_smem + (long)cols * Pp;     // [cols][Pp]: chirped spectrum, then the product
    float2 *tw = kt_smem + 2L * cols * Pp;      // [P]
    __shared__ float2 s_eps[4];                 // eps of each column as an FP32 pair (hi, lo)
    build_twiddles<KT_THREADS>(tw, P);
    const float scale = 1.0f / (float)((long)M * P);          // exact: a power of two
    const int groups = N / cols;
    for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
        const int p0 = grp * cols;
        __syncthreads();                        // the previous group is done with b0, b1, s_eps
        if (threadIdx.x < cols) {
            const double eps = kt_eps(p0 + threadIdx.x, logN, N, lam_2ndr);
            const float hi = (float)eps;
            s_eps[threadIdx.x] = make_float2(hi, (float)__dsub_rn(eps, (double)hi));
        }
        for (int t = threadIdx.x; t < cols * M; t += KT_THREADS) {
            const int col = t % cols, m = t / cols;
            b0[(long)col * Pp + fpad(m)] = __ldg(S + (long)m * N + p0 + col);
        }
        __syncthreads();
        fft_dif_fwd<KT_THREADS>(b0, cols, Pp, tw, logM);      // Y[l] at b0[bitrev_M(l mod M)]
        for (int t = threadIdx.x; t < cols * P; t += KT_THREADS) {
            const int col = t >> logP, i = t & (P - 1);
            float2 v = make_float2(0.f, 0.f);
            if (i < M) {
                const int l = i - M / 2;
                const int at = (int)brev_bits((unsigned)(l & (M - 1)), logM);
                v = cmul(b0[(long)col * Pp + fpad(at)], kt_chirp(l, logM, s_eps[col]));
            }
            b1[(long)col * Pp + fpad(i)] = v;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cols * P; t += KT_THREADS) {
            const int col = t >> logP, e = t & (P - 1);
            float2 g = make_float2(0.f, 0.f);                  // e = M: never used by the convolution
            if (e != M) g = conj2(kt_chirp((e < M ? e : e - P) + M / 2, logM, s_eps[col]));
            b0[(long)col * Pp + fpad(e)] = g;
        }
        __syncthreads();
        fft_dif_fwd<KT_THREADS>(kt_smem, 2 * cols, Pp, tw, logP);  // kernel and sequence together
        for (int t = threadIdx.x; t < cols * P; t += KT_THREADS) {
            const long o = (long)(t >> logP) * Pp + fpad(t & (P - 1));
            b1[o] = cmul(b0[o], b1[o]);
        }
        __syncthreads();
        fft_dit_inv<KT_THREADS>(b1, cols, Pp, tw, logP);
        for (int t = threadIdx.x; t < cols * M; t += KT_THREADS) {
            const int col = t % cols, m = t / cols;
            const float2 v = cmul(b1[(long)col * Pp + fpad(m)], kt_chirp(m, logM, s_eps[col]));
            Skt[(long)m * N + p0 + col] = make_float2(v.x * scale, v.y * scale);
        }
    }
}

__global__ __launch_bounds__(KT_THREADS, 2) void k_rm_kt(RadarD R, grft_dsgrid g, int cell_begin, int cell_count,
                                                    int logN, double lam_2ndr, int rpi,
                                                    const float2 *__restrict__ Skt, float2 *__restrict__ Z) {
    // rpi (1 or KT_RPI) rows per iteration, their transforms run together (as in k_rm_fd)
    extern __shared__ float2 kt_smem[];
    const int N = R.N, Np = fft_padded(N);
    float2 *x = kt_smem, *tw = kt_smem + (long)rpi * Np;     // rpi padded rows (fft_smem.cuh), twiddles
    __shared__ long s_I[KT_RPI];                // integer advance of each row
    __shared__ float s_f[KT_RPI], s_d1[KT_RPI]; // fractional advance, delta1
    __shared__ float2 s_w[KT_RPI];              // H_pre-DFM of each row
    __shared__ int s_m[KT_RPI];                 // pulse of each row
    build_twiddles<KT_THREADS>(tw, N);
    const long rows = (long)cell_count * R.M;
    const float inv_n = 1.0f / (float)N;        // exact: N a power of two
    const float l2n = (float)lam_2ndr;          // f_k / f_c per unit of k_s
    for (long row0 = (long)blockIdx.x * rpi; row0 < rows; row0 += (long)gridDim.x * rpi) {
        const int nr = (int)(rows - row0 < rpi ? rows - row0 : rpi);
        __syncthreads();                        // the previous rows' reads of x and the row scalars are done
        if (threadIdx.x < nr) {                 // one thread per row, FP64
            const long row = row0 + threadIdx.x;
            const int cl = (int)(row / R.M), m = (int)(row - (long)cl * R.M);
            const int c = cell_begin + cl;
            const double vq = axis_value(g.vc.start, g.vc.step, c / g.ac.count);
            const double ac = axis_value(g.ac.start, g.ac.step, c % g.ac.count);
            const double t = slow_time(m, R.prf);
            const double d1 = __ddiv_rn(__dmul_rn(vq, t), R.dr);
            const double q2 = displacement(0.0, ac, t);                    // c_2,c t^2
            const double D = __dsub_rn(d1, __ddiv_rn(q2, R.dr));
            const double fl = floor(D);
            s_I[threadIdx.x] = (long)fl;
            s_f[threadIdx.x] = (float)__dsub_rn(D, fl);
            s_d1[threadIdx.x] = (float)d1;
            s_w[threadIdx.x] = range_phase(q2, R.lambda);
            s_m[threadIdx.x] = m;
        }
        __syncthreads();
        for (int tt = threadIdx.x; tt < (nr << logN); tt += KT_THREADS) {
            const int r = tt >> logN, p = tt & (N - 1);
            const int k = (int)brev_bits((unsigned)p, logN);
            const int ks = k < N / 2 ? k : k - N;
            // E_k = k_s eps_k / N with eps_k = fbar - 1 = -u / (1 + u), u = f_k / f_c (|u| < 1e-2):
            // FP32 here; its relative error enters the phase as E_k delta1 (well under 1e-6 turns)
            const float u = (float)ks * l2n;
            const float E = (float)ks * __fdividef(-u, 1.0f + u) * inv_n;
            // turns of the ramp: k_s f / N (|.| <= 1/2) + the dispersive E_k delta1 (small)
            const float phi = fmaf(E, s_d1[r], (float)ks * s_f[r] * inv_n);
            float sn, cs;
            sincospif(2.0f * phi, &sn, &cs);
            x[(long)r * Np + fpad(p)] = cmul(__ldg(Skt + (long)s_m[r] * N + p), make_float2(cs, sn));
        }
        __syncthreads();
        fft_dit_inv<KT_THREADS>(x, nr, Np, tw, logN);
        for (int r = 0; r < nr; ++r) {
            const long row = row0 + r;
            const float2 sc = make_float2(s_w[r].x * inv_n, s_w[r].y * inv_n);
            const long I = s_I[r];
            const float2 *xr = x + (long)r * Np;
            float2 *zrow = Z + row * g.r0_count;
            for (int j = threadIdx.x; j < g.r0_count; j += KT_THREADS) {
                const int n = (int)(((long)g.r0_begin + j + I) & (N - 1));   // mod N (a power of two)
                zrow[j] = cmul(xr[fpad(n)], sc);
            }
        }
    }
}

int ilog2_exact(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace

int kt_columns(int M) { return M <= 1024 ? 4 : 2; }

size_t kt_smem_bytes(int M) {
    return ((size_t)2 * kt_columns(M) * fft_padded(2 * M) + 2 * (size_t)M) * sizeof(float2);
}

// rpi padded rows and the twiddles
size_t rm_kt_smem_bytes(int N, int rpi) { return ((size_t)rpi * fft_padded(N) + N) * sizeof(float2); }
static int kt_rows_per_iter(int N) { return N <= 4096 ? KT_RPI : 1; }

static int kt_set_attributes(const Ctx &c) {
    static bool done[64] = {false};
    if (c.device >= 64) return GRFT_EUNSUPPORTED;
    if (!done[c.device]) {                      // once per device, for the largest sizes served
        if (cudaFuncSetAttribute(k_keystone, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kt_smem_bytes(2048)) != cudaSuccess ||
            cudaFuncSetAttribute(k_rm_kt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)rm_kt_smem_bytes(8192, 1)) != cudaSuccess)   // >= (4096, KT_RPI)
            return GRFT_ECUDA;
        done[c.device] = true;
    }
    return GRFT_OK;
}

static double lam_over_2ndr(const RadarD &R) { return R.lambda / (2.0 * R.N * R.dr); }

int launch_keystone(const Ctx &c, const RadarD &R, const float2 *S, float2 *Skt) {
    int e = kt_set_attributes(c);
    if (e) return e;
    const int cols = kt_columns(R.M);
    const int groups = R.N / cols;
    const int cap = 4 * c.num_sms;
    const int grid = groups < cap ? groups : cap;
    KernelTimer kt(c, GRFT_KERNEL_KEYSTONE);
    k_keystone<<<grid, KT_THREADS, kt_smem_bytes(R.M), c.stream>>>(S, R.M, R.N, ilog2_exact(R.M),
                                                                    ilog2_exact(R.N), cols, lam_over_2ndr(R), Skt);
    return check_launch();
}

int launch_rm_kt(const Ctx &c, const RadarD &R, const grft_dsgrid &g, int cell_begin, int cell_count,
                 const float2 *Skt, float2 *Z) {
    int e = kt_set_attributes(c);
    if (e) return e;
    const long rows = (long)cell_count * R.M;
    if (rows == 0) return GRFT_OK;
    const int rpi = kt_rows_per_iter(R.N);
    const long iters = (rows + rpi - 1) / rpi;
    const long cap = 2L * c.num_sms * 4;
    const int grid = (int)(iters < cap ? iters : cap);
    KernelTimer kt(c, GRFT_KERNEL_COARSE_RM);
    k_rm_kt<<<grid, KT_THREADS, rm_kt_smem_bytes(R.N, rpi), c.stream>>>(R, g, cell_begin, cell_count,
                                                                         ilog2_exact(R.N), lam_over_2ndr(R), rpi,
                                                                         Skt, Z);
    return check_launch();
}

}  // namespace grft
