/*
 * dsgrft.h - C ABI of libdsgrft.so: the GRFT / DS-GRFT coherent sum over motion
 * hypotheses on one GB300 (sm_103a), after arXiv 2403.06788.
 *
 * The statistic (Sec. III-A, eq. standard-GRFT-TD, with the range phase of the full
 * trajectory; eq. slant range with P = 2):
 *
 *     Y(r0, v, a) = sum_{m=0}^{M-1} s[m][n0 + rho(v,a,m)] * exp(+j 4 pi r(t_m) / lambda)
 *
 *   t_m = m / PRF,  r(t) = r0 + v t + a t^2 / 2,  r0 = n0 * dr,  lambda = c / f_c,
 *   d   = (v*t) + ((0.5*a)*(t*t))   (IEEE FP64, each operation rounded once),
 *   rho = floor(d/dr + 0.5)         (nearest bin, ties toward +inf), and gathered samples
 *   whose bin falls outside [0, N) contribute zero.
 *
 * Conventions shared by every call
 *   - All array arguments are DEVICE pointers owned by the caller, unless stated
 *     otherwise; parameter structs are HOST pointers read during the call only.
 *   - Complex data is interleaved complex64 (grft_c32).  The echo is s[M][N], range
 *     fastest.  Hypothesis outputs are row-major [v][a][r0] (r0 fastest).
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and is
 *     asynchronous; no call synchronises the host except grft_sync_status().
 *   - Every call returns GRFT_OK (0) or a negative status.  Argument errors are found on
 *     the host before anything is enqueued.  Device-side conditions (a bounded wait that
 *     gave up, a candidate-buffer overflow) are latched in a per-device flag that
 *     grft_sync_status() returns and clears.  No call exits the process or throws.
 *   - Internal workspace (tables, candidate buffers) is allocated by the library on first
 *     use per device and grown when a larger problem needs it; grow events synchronise
 *     the device, so make the first call of a given size before any stream capture.
 *     Calls that share a device must not run concurrently on different streams.
 *   - Calls run on the CUDA device that is current in the calling thread.
 */
#ifndef DSGRFT_H_
#define DSGRFT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRFT_ABI_VERSION 1

/* ---------------------------------------------------------------- status codes */
enum {
    GRFT_OK = 0,
    GRFT_EINVAL = -1,       /* null pointer, bad shape, grid or parameter */
    GRFT_ENOMEM = -2,       /* workspace allocation failed */
    GRFT_ECUDA = -3,        /* CUDA runtime / launch error */
    GRFT_ETIMEOUT = -4,     /* a bounded device-side wait ran out (kernel returned early) */
    GRFT_EUNSUPPORTED = -5, /* device is not sm_103 / precision not available */
    GRFT_EOVERFLOW = -6     /* detection candidate buffer overflowed; top-K is incomplete */
};

/* ---------------------------------------------------------------- parameter types */
typedef struct { float re, im; } grft_c32;

/* Uniform axis: value_i = start + i * step, i = 0..count-1 (FP64 as written). */
typedef struct { double start, step; int32_t count, reserved; } grft_axis;

/* Radar / CPI parameters (Sec. II-A): M pulses, N range bins of dr = c/(2 f_s) metres. */
typedef struct {
    int32_t M, N;
    double fc_hz;   /* carrier frequency f_c */
    double prf_hz;  /* pulse repetition frequency; t_m = m / prf */
    double dr_m;    /* range bin */
    double c_mps;   /* propagation speed (3e8) */
} grft_radar;

/* Single-scale grid (Sec. III-C, eq. delta-Beta-1): r0 bins [r0_begin, r0_begin+r0_count). */
typedef struct { int32_t r0_begin, r0_count; grft_axis v, a; } grft_grid;

/* Dual-scale grid (Sec. IV-B, eqs. Partition-Parameter, Space_c_c, Space_c_f).
 * Coarse centres v_c(i) = vc.start + i vc.step, a_c(l) likewise; fine offsets
 * dv_k = (k - Fv/2) vc.step / Fv, da_q = (q - Fa/2) ac.step / Fa (half-open cells).
 * Coarse cell index c = i * ac.count + l; fine index f = k * Fa + q. */
typedef struct { int32_t r0_begin, r0_count; grft_axis vc, ac; int32_t Fv, Fa; } grft_dsgrid;

typedef enum {
    GRFT_FP32 = 0,   /* FP32 SIMT contraction (FFMA) */
    GRFT_BF16X3 = 1, /* tcgen05 tensor cores, hi/lo-split BF16 operands, 3 products, FP32 accumulate */
    GRFT_FP16X3 = 2, /* tcgen05 tensor cores, hi/lo-split FP16 operands, 3 products, FP32 accumulate */
    GRFT_FP16X1 = 3, /* tcgen05 tensor cores, FP16 operands (one rounding each), 1 product, FP32
                        accumulate: not the split form; within the 2e-3-of-peak bound of the split
                        path on the benchmark workloads (measured errors in the tests) */
    GRFT_FP16X2 = 4  /* tcgen05 tensor cores, FP16, hi/lo split of the gathered echo operand and the
                        dechirp rounded once, 2 products (hi*hi + lo*hi), FP32 accumulate */
} grft_precision;

typedef enum { GRFT_GATHER_NEAREST = 0, GRFT_GATHER_LINEAR = 1 } grft_gather;

/* Detector: mode 0 = CA-CFAR along r0 (guard/train cells each side, false-alarm rate pfa);
 * mode 1 = fixed threshold P > fixed_thresh (eq. LRT squared).  Both add a 3x3x3 local
 * maximum test over (v, a, r0). */
typedef struct { int32_t guard, train; double pfa; float fixed_thresh; int32_t mode; } grft_cfar;

/* One detection: linear index (vi*na + ai)*nr0 + n0, grid indices, power and the
 * on-grid estimate (Alg. 3: c0 = r0, c1 = v, c2 = a). */
typedef struct { int64_t idx; int32_t n0, vi, ai; float p; double r0_m, v, a; } grft_det;

/* One CPI of a batched DS-GRFT launch. */
typedef struct {
    const grft_c32 *echo; /* [M][N] */
    float *P;             /* [nv][na][r0_count] canonical layout, nullable if Y given */
    grft_c32 *Y;          /* same layout, nullable */
    int32_t M, N;
    int32_t r0_begin, r0_count;
} grft_batch_item;

/* ---------------------------------------------------------------- library */
int grft_version(void);
const char *grft_status_string(int status);

/* Synchronise `stream`, return (and clear) the device-side status latched by earlier
 * calls on this device: GRFT_OK, GRFT_ETIMEOUT or GRFT_EOVERFLOW. */
int grft_sync_status(void *stream);

/* Bounded-wait limit of the warp-specialised kernels, in SM clock cycles (0 restores the
 * default of about one second).  A wait that exceeds it makes the kernel latch
 * GRFT_ETIMEOUT and return early with partial output. */
int grft_set_wait_limit(uint64_t cycles);

/* Free this device's cached workspace (the next call reallocates it). */
int grft_release_workspace(void);

/* Release everything the library holds for the current device: the workspaces, the side
 * stream and events of the split/contraction pipeline, and pending timing events (timing
 * is switched off).  Synchronises the device; the next call sets up what it needs again. */
int grft_shutdown(void);

/* Per-kernel timing on the GPU (tracing): while enabled, every kernel the library launches
 * outside stream capture is bracketed by a pair of CUDA events recorded on the call's
 * stream.  grft_timing(1) enables and clears the totals, grft_timing(0) disables;
 * grft_timing_get synchronises the recorded events and returns, for one kernel class, the
 * number of launches and their summed duration in milliseconds. */
enum {
    GRFT_KERNEL_TABLES = 0,        /* bins, phases, dechirp operands (tables.cu) */
    GRFT_KERNEL_PLAIN = 1,         /* plain GRFT */
    GRFT_KERNEL_COARSE_RM = 2,     /* standalone coarse-RM gather (TMA) */
    GRFT_KERNEL_SPLIT = 3,         /* split coarse-RM operand of the tensor-core path */
    GRFT_KERNEL_CONTRACT = 4,      /* tensor-core fine-DFM contraction */
    GRFT_KERNEL_CONTRACT_FP32 = 5, /* FP32 SIMT fine-DFM contraction */
    GRFT_KERNEL_CFAR = 6,
    GRFT_KERNEL_TOPK = 7,
    GRFT_KERNEL_ADJOINT = 8,       /* trajectory sum, adjoint, refinement */
    GRFT_KERNEL_CONTRACT_FFT = 9,  /* FFT form of the fine stage (dsgrft_fine_dfm_fft, dskt_fine_dfm_fft) */
    GRFT_KERNEL_KEYSTONE = 10,     /* keystone transform (dskt_keystone) */
    GRFT_KERNEL_COUNT = 11
};
int grft_timing(int enable);
int grft_timing_get(int kernel, int32_t *launches, double *total_ms);

/* Failure-path self test: one CTA waits on a barrier that nothing completes, for `cycles`
 * SM cycles (0 = the current wait limit), then latches GRFT_ETIMEOUT and returns; read it
 * with grft_sync_status().  The context stays usable. */
int grft_selftest_wait(uint64_t cycles, void *stream);

/* ---------------------------------------------------------------- the hot path */

/* Trajectory tables (eq. standard-GRFT-TD's n(c,t_m); eqs. H-DFM / pre-DFM phases).
 * For nh explicit (v[h], a[h]) pairs (device FP64 arrays): rho[h][m] = floor(d/dr + 0.5)
 * (int32, bit-exact to the FP64 definition) and w[h][m] = exp(j 4 pi d / lambda). */
int grft_bins_phases(const grft_radar *radar, const double *v, const double *a, int32_t nh,
                     int32_t *rho, grft_c32 *w, void *stream);

/* Plain (single-scale) TD-GRFT over the whole grid (Sec. III-A eq. standard-GRFT-TD;
 * Table III row TD-GRFT).  Y[v][a][r0_count] (complex, nullable) and/or
 * P[v][a][r0_count] = |Y|^2 (nullable; at least one given).  FP32 SIMT. */
int grft_plain(const grft_radar *radar, const grft_c32 *echo, const grft_grid *grid,
               grft_c32 *Y, float *P, void *stream);

/* Size of the fixed device scratch of grft_plain_static (8 MiB). */
#define GRFT_PLAIN_STATIC_SCRATCH_BYTES (8u << 20)

/* grft_plain without any device allocation (the paper has no counterpart; this is for
 * callers that cannot call cudaMalloc, e.g. a processing loop with a fixed memory budget
 * that must not grow or wait on an allocator, or a process whose device memory belongs to
 * another pool).  Same arguments, results and output layout as grft_plain (bit-identical); the
 * bin/phase tables live in a fixed array of GRFT_PLAIN_STATIC_SCRATCH_BYTES inside the
 * library image (held by every GPU that loads the library until the process exits)
 * instead of the library workspace, and the grid is processed in chunks that fit it.
 *   - Size limit: returns GRFT_EINVAL, before enqueueing anything, if
 *     r0_count * 8 (rounded up to 256) + 8 * M * 12 + 512 > GRFT_PLAIN_STATIC_SCRATCH_BYTES
 *     (the range phases plus one group of 8 hypotheses' tables must fit).
 *   - Set-up: the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before any
 *     stream capture.
 *   - Every call on a device shares the one array: calls that overlap on the GPU (other
 *     streams, other threads) race on it and must be serialised by the caller.  Each call
 *     writes the part it reads, so nothing needs to be cleared between calls. */
int grft_plain_static(const grft_radar *radar, const grft_c32 *echo, const grft_grid *grid,
                      grft_c32 *Y, float *P, void *stream);

/* Coarse range-migration correction, time-domain mGIFT (Def. 2 + eq. pre-DFM, Alg. 1):
 *   Z[c - cell_begin][m][j] = s[m][r0_begin + j + rho_c(m)] * exp(j 4 pi d_c(t_m) / lambda)
 * for coarse cells c in [cell_begin, cell_begin + cell_count), j in [0, r0_count).
 * The echo rows are staged through shared memory by TMA. */
int dsgrft_coarse_rm(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                     int32_t cell_begin, int32_t cell_count, grft_c32 *Z, void *stream);

/* Coarse range-migration correction in the frequency domain, the mGIFT of Def. 2 with
 * eq. H-RM and eq. pre-DFM (Alg. 1): per pulse the range spectrum S[m][k] (N-point DFT)
 * times exp(j 2 pi k delta / N), delta = d_c(t_m) / dr, k in [-N/2, N/2), inverse DFT,
 * times the coarse phase:
 *   Z[c - cell_begin][m][j] = (1/N) sum_k S[m][k] exp(j 2 pi k (r0_begin + j + delta) / N)
 *                             * exp(j 4 pi d_c(t_m) / lambda)
 * the band-limited circular advance of each range profile by delta bins (no rounding of
 * the bin shift).  Same output layout as dsgrft_coarse_rm, so dsgrft_fine_dfm with Z given
 * runs the fine stage on it.  N must be a power of two <= 8192 (else GRFT_EUNSUPPORTED,
 * nothing enqueued).  FP32 transforms, FP64 delta and phases. */
int dsgrft_coarse_rm_fd(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                        int32_t cell_begin, int32_t cell_count, grft_c32 *Z, void *stream);

/* The range frequencies the spectrum index k stands for: baseband k in [-N/2, N/2), or the
 * paper's discrete band f_k = k f_s / N, k = 0..N-1, of eq. Rx-OFDM-Fre1 (the echo of
 * eq. received signal, asinc envelope with its linear phase). */
typedef enum { GRFT_BAND_BASEBAND = 0, GRFT_BAND_POSITIVE = 1 } grft_band;

/* dsgrft_coarse_rm_fd with the band chosen (GRFT_BAND_BASEBAND is dsgrft_coarse_rm_fd):
 * over the positive band k runs over [0, N) in the ramp exp(j 2 pi k delta / N). */
int dsgrft_coarse_rm_fd_ex(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                           int32_t cell_begin, int32_t cell_count, grft_band band, grft_c32 *Z, void *stream);

/* Fine stage on Z of dsgrft_coarse_rm_fd_ex with the same band (Prop. 1): dsgrft_fine_dfm with
 * Z given and the fine offsets of H_DFM scaled by 1 + B_r / (2 f_c), B_r = c / (2 dr), for the
 * positive band (1 for baseband): after a positive-band coarse stage the residual range term
 * c_f t^p of a cell leaves the phase -(4 pi / lambda) (1 + B_r / (2 f_c)) c_f t^p at the peak
 * bin.  (Prop. 1 prints kappa = 1 - B_r / (2 f_c), the factor of the keystone branch, Cor. 1,
 * whose residual range term has the opposite sign.)  Output layout, hypotheses' labels and
 * precisions as dsgrft_fine_dfm. */
int dsgrft_fine_dfm_fd(const grft_radar *radar, const grft_c32 *Z, const grft_dsgrid *grid, int32_t cell_begin,
                       int32_t cell_count, grft_band band, grft_precision precision, grft_c32 *Y, float *P,
                       void *stream);

/* Fine Doppler-migration correction, the GFT of Def. 1 / Alg. 2 as a dense contraction
 * against the dechirp matrix D[m][f] = exp(j 4 pi (dv_k t_m + da_q t_m^2 / 2) / lambda):
 *   Y(n0; c, f) = exp(j 4 pi n0 dr / lambda) * sum_m Zc[m][n0] D[m][f]          (Alg. 3)
 * Z = NULL: Zc is gathered on the fly from `echo` (fused with dsgrft_coarse_rm);
 * Z given: Z is the [cell_count][M][r0_count] output of dsgrft_coarse_rm for the same cells.
 * Output layout (Y and P, either nullable, not both): a v-slab of the canonical DS layout,
 *   [(i - i0) * Fv + k][l * Fa + q][n0 - r0_begin],  i0 = cell_begin / ac.count,
 * covering coarse v rows i0 .. (cell_begin + cell_count - 1) / ac.count; cells outside the
 * range are left untouched.  precision: GRFT_FP32 (SIMT) or a split tensor-core mode. */
int dsgrft_fine_dfm(const grft_radar *radar, const grft_c32 *Z, const grft_c32 *echo,
                    const grft_dsgrid *grid, int32_t cell_begin, int32_t cell_count,
                    grft_precision precision, grft_c32 *Y, float *P, void *stream);

/* Fine Doppler-migration correction in the FFT form of the GFT (Def. 1, Alg. 2): per cell,
 * range bin and fine acceleration, the coarse-corrected pulses are multiplied by the
 * acceleration dechirp exp(j 4 pi (da_q t_m^2 / 2) / lambda) and transformed over slow
 * time; transform bin (k - Fv/2) mod L is fine velocity k.  The grid's fine velocity step
 * vc.step / Fv must be one Doppler bin of an L-point transform, lambda PRF / (2 L), with
 * L = 256 or 512, M <= L (zero padded), Fv <= L and Fv even; otherwise GRFT_EUNSUPPORTED
 * is returned before anything is enqueued.  Same hypotheses, output layout and argument
 * meaning as dsgrft_fine_dfm with Z = NULL (the gather is fused); FP32 SIMT arithmetic,
 * equal to the dense form to FP32 rounding. */
int dsgrft_fine_dfm_fft(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                        int32_t cell_begin, int32_t cell_count, grft_c32 *Y, float *P, void *stream);

/* ---------------------------------------------------------------- keystone branch (DS-KT-MFP)
 *
 * The dual-scale KT-MFP detector of Sec. III-B (eqs. velocity_Amb, Echo-after-KT, H-MFP,
 * H-MFP-RM, KT-GRFT-GRFT) and Sec. IV (eq. Partition-Parameter-c1, Cor. 1, Prop. 3,
 * Alg. 4), P = 2.  A KT grid is a grft_dsgrid whose coarse velocity axis is the folding
 * factor: vc.step = V_a = lambda PRF / 2 (relative tolerance 1e-9) and vc.start = q_min V_a
 * (q_min an integer within 1e-6), so cell (i, l) is (q = q_min + i, a_c = ac value l); the
 * fine velocity is the baseband velocity c'_1 = (k - Fv/2) V_a / Fv on Fv = L transform
 * bins; the fine acceleration is (q - Fa/2) ac.step / Fa as in the DS-GRFT grid (kappa = 1).
 * Any other grid returns GRFT_EINVAL.  Sizes: M and N powers of two, 16 <= M <= 2048,
 * 4 <= N <= 8192, else GRFT_EUNSUPPORTED (before anything is enqueued). */

/* Range spectra and keystone transform (eq. Echo-after-KT).  echo: [M][N] device.  Skt:
 * [M][N] device, written: range-frequency slot p of pulse row m' holds y_KT(f_k, t_m') for
 * the frequency index k = bitrev_log2(N)(p) (signed k - N for k >= N/2, f_k = k f_s / N,
 * f_s = c / (2 dr)), where the slow-time column of each frequency is resampled at
 * t = fbar t', fbar = f_c / (f_c + f_k), as a band-limited periodic sequence of M samples
 * (Doppler index in [-M/2, M/2)).  Uses the library workspace for the range spectra. */
int dskt_keystone(const grft_radar *radar, const grft_c32 *echo, grft_c32 *Skt, void *stream);

/* Coarse stage (Cor. 1: the mGIFT with H_KT,RM and the KT-MFP H_pre-DFM) for the cells
 * [cell_begin, cell_begin + cell_count) of a KT grid, from Skt of dskt_keystone:
 *   Z[c][m][j] = (1/N) sum_k Skt[m][k] exp(j 2 pi k_s (fbar_k q V_a t_m - (a_c/2) t_m^2) / (N dr))
 *                      exp(j 2 pi k_s n / N) exp(j 4 pi (a_c/2) t_m^2 / lambda),
 * n = r0_begin + j; Z is [cell_count][M][r0_count] device (the layout of dsgrft_coarse_rm). */
int dskt_coarse_rm(const grft_radar *radar, const grft_c32 *Skt, const grft_dsgrid *grid,
                   int32_t cell_begin, int32_t cell_count, grft_c32 *Z, void *stream);

/* Fine stage (Prop. 3, the GFT of Def. 1 in its FFT form, Alg. 2) on Z of dskt_coarse_rm:
 *   Y(n0; c, k, q) = sum_m Z[c][m][n0] exp(j 4 pi ((k - Fv/2) (V_a / Fv) t_m + da_q t_m^2 / 2) / lambda)
 * (no range phase of n0, as in eq. KT-GRFT-GRFT), with L = Fv in {64, 128, 256, 512} and
 * M <= L, else GRFT_EUNSUPPORTED; cell_count <= 65535.  Output layout and Y / P semantics
 * are those of dsgrft_fine_dfm (a v-slab of the canonical layout starting at coarse row
 * cell_begin / ac.count).  FP32 SIMT. */
int dskt_fine_dfm_fft(const grft_radar *radar, const grft_c32 *Z, const grft_dsgrid *grid,
                      int32_t cell_begin, int32_t cell_count, grft_c32 *Y, float *P, void *stream);

/* The whole DS-KT-MFP map of Alg. 4 on one echo: dskt_keystone, then dskt_coarse_rm and
 * dskt_fine_dfm_fft over all cells, in chunks of whole folding-factor rows sized to the
 * library's split budget.  Y [nq Fv][nac Fa][r0_count] and/or P (same layout) device.
 * Uses the library workspace (Skt, the range spectra / coarse output, the chirp table). */
int dskt_mfp(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid, grft_c32 *Y,
             float *P, void *stream);

/* ---------------------------------------------------------------- P = 3 (acceleration rate)
 *
 * DS-GRFT with the third-order motion model r(t) = r0 + v t + a t^2 / 2 + b t^3 / 6 (Sec. II
 * eq. slant range, c_3 = b / 6; Alg. 3 extended to P = 3).  Coarse centres vc x ac x bc, fine
 * offsets (k - Fv/2) vc.step / Fv, (q - Fa/2) ac.step / Fa, (u - Fb/2) bc.step / Fb; cell
 * c = (i ac.count + l) bc.count + w, fine f = (k Fa + q) Fb + u.  Bins are
 * floor(d / dr + 0.5) with d = ((v t) + ((0.5 a)(t t))) + ((b / 6)((t t) t)) in FP64, each
 * operation rounded once. */
typedef struct {
    int32_t r0_begin, r0_count;
    grft_axis vc, ac, bc;
    int32_t Fv, Fa, Fb;
} grft_dsgrid3;

/* The fused coarse gather + fine contraction of dsgrft_fine_dfm (Z = NULL) for a P = 3 grid,
 * on the tensor cores (GRFT_BF16X3, GRFT_FP16X3, GRFT_FP16X2, GRFT_FP16X1; GRFT_FP32 returns
 * GRFT_EUNSUPPORTED):
 *   Y(n0; c, f) = exp(j 4 pi n0 dr / lambda) sum_m s[m][n0 + rho_c(m)] w_c(m) D[m][f],
 *   D[m][f] = exp(j 4 pi d(dv_k, da_q, db_u, t_m) / lambda).
 * Output (Y and P, either nullable, not both): the v-slab of the layout
 *   [(i - i0) Fv + k][l Fa + q][w Fb + u][n0 - r0_begin],  i0 = cell_begin / (ac.count bc.count);
 * cells outside [cell_begin, cell_begin + cell_count) are left untouched.  Fv Fa Fb <= 2^20,
 * cell_count <= 65535. */
int dsgrft3_fine_dfm(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid3 *grid,
                     int32_t cell_begin, int32_t cell_count, grft_precision precision, grft_c32 *Y, float *P,
                     void *stream);

/* Many CPIs (uneven M, N) in one persistent launch (graph-capturable after a first
 * uncaptured call of the same shape).  radar's M and N are ignored (per item); grid's
 * r0 fields are ignored (per item).  items is a HOST array of at most 256 entries; its
 * pointers are device pointers.  Tensor-core precisions only. */
int dsgrft_fine_dfm_batched(const grft_radar *radar, const grft_dsgrid *grid,
                            const grft_batch_item *items, int32_t n_items,
                            grft_precision precision, void *stream);

/* CA-CFAR / fixed threshold + 3x3x3 local maximum + top-K (eq. LRT; Alg. 3's threshold
 * scan) over P[nv][na][nr0].  Writes min(K, total) records to out[] sorted by power
 * (descending, ties by lower index) and the total number of detections to *n_out (both
 * device memory).  axes (host, nullable) maps indices to the estimate (r0_m =
 * (axes->r0_begin + n0) * dr_m, v = v.start + vi v.step, a likewise); NULL leaves the
 * estimate fields zero.  K <= 8192. */
int detect_peaks(const float *P, int32_t nv, int32_t na, int32_t nr0, const grft_cfar *cfar,
                 const grft_grid *axes, double dr_m, int32_t K, grft_det *out, int32_t *n_out,
                 void *stream);

/* detect_peaks over a map that is computed and scanned in slabs of whole v rows, so that the
 * whole map never has to exist at once (Alg. 3's threshold scan over every hypothesis of a
 * grid too large to hold):
 *   detect_peaks_begin clears the device's candidate list;
 *   detect_peaks_add scans one slab P[nv][na][nr0] (device) whose row r is v row v_base + r of
 *     the whole map: only rows [v_lo, v_hi) may be detections, the other rows serve as the
 *     neighbours of the 3x3x3 local maximum (a slab passes the rows bordering it on either
 *     side, where they exist, as such halo rows); the candidates' linear indices are those of
 *     the whole map, (v * na + a) * nr0 + n0;
 *   detect_peaks_end writes the top K of every candidate added since begin, exactly as
 *     detect_peaks would for the whole map (same records, same order, same total).
 * The candidate list belongs to the device: no other detection call may run on that device
 * between begin and end.  Candidates beyond 2^22 set GRFT_EOVERFLOW (grft_sync_status). */
int detect_peaks_begin(void *stream);
int detect_peaks_add(const float *P, int32_t nv, int32_t na, int32_t nr0, int32_t v_lo, int32_t v_hi,
                     int64_t v_base, const grft_cfar *cfar, void *stream);
int detect_peaks_end(int32_t na, int32_t nr0, const grft_grid *axes, double dr_m, int32_t K, grft_det *out,
                     int32_t *n_out, void *stream);

/* Top K of the union of detection lists: n_lists lists of K_in records each (device memory,
 * list l holding its min(K_in, totals[l]) strongest records, e.g. the top K_in of each slab
 * or of each GPU a grid was split over, gathered into one buffer), sorted by power
 * descending, ties by lower linear index.  Indices are unique across the lists (they index
 * one map), so with K_in >= K the result is the top K of the whole map, and *n_out is the
 * sum of totals[] (the whole map's total).  n_lists * K_in <= 8192, n_lists <= 1024;
 * more records than that set GRFT_EOVERFLOW (grft_sync_status).  This is the merge step of
 * a grid searched on several GPUs (each searches its own coarse cells; only these lists
 * cross between them). */
int detect_merge(const grft_det *lists, const int32_t *totals, int32_t n_lists, int32_t K_in, int32_t K,
                 grft_det *out, int32_t *n_out, void *stream);

/* DS-GRFT with detection over the whole dual-scale grid (Alg. 3: coarse RM correction, fine
 * DFM contraction, threshold scan, estimates), streamed one coarse-v row of cells at a time:
 * the power map of cells [i * ac.count, (i + 1) * ac.count) (Fv v rows) is computed as in
 * dsgrft_fine_dfm into one of two library-owned slab buffers, with the neighbouring slabs'
 * border rows as halos, and scanned by detect_peaks_add; the whole map P is never held.
 * Output: the top K detections of the whole map (records as detect_peaks with the plain
 * grid of the same hypotheses as axes: v = vc.start - vc.step / 2 + vi vc.step / Fv, a
 * likewise) and the total count, in device memory; identical to dsgrft_fine_dfm over every
 * cell followed by detect_peaks.  Device memory: two slabs of (Fv + 2) x ac.count Fa x
 * r0_count floats (workspace, kept until grft_release_workspace).  K <= 8192.  Capturable
 * in a CUDA graph after one uncaptured call of the same shape. */
int dsgrft_detect(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                  grft_precision precision, const grft_cfar *cfar, int32_t K, grft_det *out, int32_t *n_out,
                  void *stream);

/* Coherent sum along K continuous trajectories theta[k] = (r0_m, v, a) (device FP64
 * [K][3]) and its adjoint (no counterpart in the paper; gather: nearest bin or linear
 * interpolation between bins):
 *   P[k] = |Y_k|^2, Y[k] (each nullable),
 *   grad_theta[k][j] = gP[k] * dP_k/dtheta_j (nullable; gP = grad_P or ones),
 *   grad_s[m][n] += sum_k gP[k] * 2 Y_k conj(dY_k/ds[m][n])  (nullable; the
 *                   d/dRe + j d/dIm convention of torch.autograd; accumulated, unordered).
 * Phases are recomputed from FP64 ranges, never stored. */
int dsgrft_backward(const grft_radar *radar, const grft_c32 *echo, int32_t K, const double *theta,
                    grft_gather gather, const float *grad_P, float *P, grft_c32 *Y,
                    double *grad_theta, grft_c32 *grad_s, void *stream);

/* Sub-grid gradient-ascent refinement of K detections, one launch: with cell = the host
 * array (c_r0, c_v, c_a) of grid steps, g = dP/dtheta and eta = 0.5 / max_j |cell_j g_j|,
 * repeat `steps` times: theta' = theta + eta cell^2 . g; accept if P(theta') >= P(theta),
 * else halve eta.  theta (device [K][3]) is updated in place, P_out[k] gets the final power. */
int dsgrft_refine(const grft_radar *radar, const grft_c32 *echo, int32_t K, double *theta,
                  const double *cell, int32_t steps, grft_gather gather, float *P_out,
                  void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DSGRFT_H_ */
