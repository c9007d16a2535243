// Internal declarations shared by the translation units of libdsgrft.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/dsgrft.h"

namespace grft {

// --------------------------------------------------------------------------- device math
// Bin and phase of a displacement, written with explicit round-to-nearest FP64
// intrinsics so that no operation is contracted into an FMA: the bins are bit-identical
// to the IEEE definition d = (v*t) + ((0.5*a)*(t*t)), rho = floor(d/dr + 0.5).
__device__ __forceinline__ double slow_time(int m, double prf) { return __ddiv_rn((double)m, prf); }

__device__ __forceinline__ double displacement(double v, double a, double t) {
    double vt = __dmul_rn(v, t);
    double ha = __dmul_rn(0.5, a);
    double tt = __dmul_rn(t, t);
    return __dadd_rn(vt, __dmul_rn(ha, tt));
}

// P = 3: d + (b / 6) ((t t) t), the acceleration-rate term added last.
__device__ __forceinline__ double displacement3(double v, double a, double b, double t) {
    const double tt = __dmul_rn(t, t);
    return __dadd_rn(displacement(v, a, t), __dmul_rn(__ddiv_rn(b, 6.0), __dmul_rn(tt, t)));
}

// The range bin of displacement d: floor(d / dr + 1/2), with d / dr the correctly rounded
// FP64 quotient.  The quotient is first taken as p = d x inv_dr (inv_dr = 1 / dr rounded):
// p lies within 3 units in the last place of the rounded quotient q, so x = p + 1/2 and
// q + 1/2 (each rounded) have the same floor unless an integer lies between them, which
// needs x within 2^-50 |p| + 2^-53 of that integer.  Only then (about one entry in 10^12 of
// random displacements, and every exact half-bin tie) is the division carried out.  The
// host form (tests) is the same operations; it needs FMA contraction off.
__host__ __device__ __forceinline__ int bin_shift(double d, double dr, double inv_dr) {
#ifdef __CUDA_ARCH__
    const double p = __dmul_rn(d, inv_dr);
    const double x = __dadd_rn(p, 0.5);
#else
    const double p = d * inv_dr;
    const double x = p + 0.5;
#endif
    if (fabs(x - rint(x)) > fabs(p) * 0x1p-48 + 0x1p-44) return (int)floor(x);
#ifdef __CUDA_ARCH__
    return (int)floor(__dadd_rn(__ddiv_rn(d, dr), 0.5));
#else
    return (int)floor(d / dr + 0.5);
#endif
}

// exp(+j 4 pi x / lambda): FP64 cycle count 2x/lambda, reduced to [-1/2, 1/2] in FP64,
// then an FP32 sincospi of the reduced angle.
__device__ __forceinline__ float2 range_phase(double x, double lambda) {
    double u = __ddiv_rn(__dmul_rn(2.0, x), lambda);
    double f = __dsub_rn(u, rint(u));
    float s, c;
    sincospif(2.0f * (float)f, &s, &c);
    return make_float2(c, s);
}

// Axis value start + i*step and the dual-scale fine offset (k - F/2) * (step_c / F).
__device__ __forceinline__ double axis_value(double start, double step, int i) {
    return __dadd_rn(start, __dmul_rn((double)i, step));
}
__device__ __forceinline__ double fine_offset(double step_c, int F, int k) {
    double off = __dmul_rn((double)(2 * k - F), 0.5);
    return __dmul_rn(off, __ddiv_rn(step_c, (double)F));
}

__device__ __forceinline__ float2 cmul(float2 x, float2 y) {
    return make_float2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}

// Latch the first device-side error of this device (0 = no error).
__device__ __forceinline__ void latch_error(int *status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// The acceleration-rate axis of a P = 3 dual-scale grid (coarse centres start + w step, w <
// count; Fb fine offsets (u - Fb/2) step / Fb).  A coarse cell index c of such a grid is
// (i na_c + l) count + w and a fine index (k Fa + q) Fb + u.  on == false is P = 2 (count 1,
// Fb 1): every formula reduces to the P = 2 one.
struct Rate3 {
    bool on;
    double start, step;
    int count, Fb;
};
constexpr Rate3 kNoRate{false, 0.0, 0.0, 1, 1};

// Pairs of mirrored fine hypotheses.  The fine offsets (2k - F)/2 x step/F of k and F - k
// are exact negatives, so the dechirp rows of hypothesis (k, q) and of its mirror
// (Fv - k, Fa - q), k, q >= 1, are complex conjugates: D[m][f'] = conj(D[m][f]) (the
// displacement, and with it the phase, changes sign).  One contraction of the gathered
// operand's real and imaginary parts against Re D[m][f] and Im D[m][f] gives both sums:
//   A = sum Zr Dr, B = sum Zi Di, C = sum Zr Di, E = sum Zi Dr,
//   Y(f) = (A - B) + j (C + E),  Y(f') = (A + B) + j (E - C).
// The slots list every hypothesis once, with its mirror where it has one: slots [0, Fa) are
// k = 0 (no mirror), [Fa, Fa + Fv - 1) are q = 0, k >= 1 (no mirror), and the rest walk the
// k, q >= 1 rectangle of R = Fv - 1 rows and C = Fa - 1 columns in row-major order up to its
// middle (the mirror of linear index l is R C - 1 - l; the middle one, when R C is odd, is
// its own mirror: the zero offset).
__host__ __device__ inline int pair_slot_count(int Fv, int Fa) {
    const long rc = (long)(Fv - 1) * (Fa - 1);
    return Fa + (Fv - 1) + (int)((rc + 1) / 2);
}
// Hypothesis f = k Fa + q of slot s and its mirror fm (-1 if none or itself).
__host__ __device__ inline void pair_slot(int s, int Fv, int Fa, int &f, int &fm) {
    fm = -1;
    if (s < Fa) {
        f = s;
        return;
    }
    s -= Fa;
    if (s < Fv - 1) {
        f = (s + 1) * Fa;
        return;
    }
    s -= Fv - 1;
    const int C = Fa - 1;
    const long lm = (long)(Fv - 1) * C - 1 - s;
    f = (s / C + 1) * Fa + (s % C + 1);
    if (lm != s) fm = (int)(lm / C + 1) * Fa + (int)(lm % C + 1);
}

// P = 3 grids with Fb >= 2 rate offsets: the mirror of hypothesis (k, q, u) is (Fv - k,
// Fa - q, Fb - u) for k, q, u >= 1 (all three offsets change sign).  The slots list first
// the hypotheses without a mirror (k = 0: Fa Fb of them; q = 0, k >= 1: (Fv - 1) Fb; u = 0,
// k, q >= 1: (Fv - 1)(Fa - 1)), then walk the k, q, u >= 1 box in row-major order up to its
// middle.  f is the full fine index (k Fa + q) Fb + u.  Fb <= 1 is the P = 2 rule (the rate
// axis is a single zero offset) with f = (k Fa + q) Fb.
__host__ __device__ inline int pair_slot_count3(int Fv, int Fa, int Fb) {
    if (Fb <= 1) return pair_slot_count(Fv, Fa);
    const long box = (long)(Fv - 1) * (Fa - 1) * (Fb - 1);
    return Fa * Fb + (Fv - 1) * Fb + (Fv - 1) * (Fa - 1) + (int)((box + 1) / 2);
}
__host__ __device__ inline void pair_slot3(int s, int Fv, int Fa, int Fb, int &f, int &fm) {
    if (Fb <= 1) {
        pair_slot(s, Fv, Fa, f, fm);
        f *= Fb;
        if (fm >= 0) fm *= Fb;
        return;
    }
    fm = -1;
    if (s < Fa * Fb) {                         // k = 0
        f = s;
        return;
    }
    s -= Fa * Fb;
    if (s < (Fv - 1) * Fb) {                   // q = 0, k >= 1
        f = (s / Fb + 1) * Fa * Fb + s % Fb;
        return;
    }
    s -= (Fv - 1) * Fb;
    const int C = Fa - 1, D = Fb - 1;
    if (s < (Fv - 1) * C) {                    // u = 0, k, q >= 1
        f = ((s / C + 1) * Fa + s % C + 1) * Fb;
        return;
    }
    s -= (Fv - 1) * C;
    const long lm = (long)(Fv - 1) * C * D - 1 - s;
    auto full = [&](long l) {
        const int u = (int)(l % D) + 1, kq = (int)(l / D);
        return ((kq / C + 1) * Fa + kq % C + 1) * Fb + u;
    };
    f = full(s);
    if (lm != s) fm = full(lm);
}

// --------------------------------------------------------------------------- host side
struct RadarD {     // radar constants as the kernels use them
    int M, N;
    double prf, dr, lambda;
    double inv_dr;   // 1 / dr, rounded (bin_shift)
};

inline RadarD radar_d(const grft_radar &r) {
    RadarD d;
    d.M = r.M;
    d.N = r.N;
    d.prf = r.prf_hz;
    d.dr = r.dr_m;
    d.lambda = r.c_mps / r.fc_hz;
    d.inv_dr = 1.0 / r.dr_m;
    return d;
}

struct Ctx {                  // per-call device context
    int device;
    cudaStream_t stream;
    int *status;              // device status word (latched errors)
    uint64_t wait_limit;      // bounded-wait limit in SM cycles
    int num_sms;
};

// Workspace of this device, grown to at least `bytes` (synchronises the device when it
// grows).  Returns nullptr on allocation failure.
// Per-device workspaces, grown on demand (a grow synchronises the device).  Slot 0 serves
// the transforms (plain GRFT, coarse stages, fine stages), slot 1 the detection, so that a
// detection and a transform of another CPI may run at the same time on two streams; slot 2
// holds the slab buffers of the streamed detector.
void release_pipe(int dev);   // side stream and events of the split/contraction pipeline
constexpr int WS_SLOTS = 3;
constexpr int WS_TRANSFORM = 0, WS_DETECT = 1, WS_SLAB = 2;
void *workspace(const Ctx &ctx, size_t bytes, int slot = WS_TRANSFORM);

// Launchers (each returns a grft status; they only enqueue work).
int launch_bins_phases(const Ctx &, const RadarD &, const double *v, const double *a, int nh,
                       int32_t *rho, grft_c32 *w);
int launch_plain_tables(const Ctx &, const RadarD &, const grft_grid &, long h0, int nh,
                        int32_t *rho, float2 *w);
int launch_coarse_tables(const Ctx &, const RadarD &, const grft_dsgrid &, int cell_begin,
                         int cell_count, int32_t *rho, float2 *w, const Rate3 &rate = kNoRate);
int launch_range_phase(const Ctx &, const RadarD &, int r0_begin, int r0_count, float2 *e0);
int launch_dechirp(const Ctx &, const RadarD &, const grft_dsgrid &, float2 *D);
// Dechirp matrix in the K-major real-GEMM operand layout of the tensor-core kernel.
int launch_dechirp_split(const Ctx &, const RadarD &, const grft_dsgrid &, int Mpad, int Fpad,
                         bool fp16, uint16_t *Bhi, uint16_t *Blo, const Rate3 &rate = kNoRate);
// The pair form's dechirp operand (pair_slot): rows 2 s and 2 s + 1 hold Re D and Im D of
// the slot's first hypothesis over the pulses (K-major, pulses contiguous, Mrow =
// pair_mrow(M) per row), hi and lo planes of [2 Spad][Mrow]; padding slots and pulses are zero.
int launch_dechirp_pair(const Ctx &, const RadarD &, const grft_dsgrid &, int Mrow, int Spad, bool fp16,
                        uint16_t *Bhi, uint16_t *Blo, const Rate3 &rate = kNoRate);
// Whether the tensor-core contraction of a grid runs in the pair form: P = 2 grids, a P = 3
// grid whose one fine rate offset is zero, and P = 3 grids with Fb >= 2 rate offsets
// (pair_slot3); DSGRFT_PAIR=0 selects the 4M form.
bool ds_pair_form(const Rate3 &rate);
// Pulses per row of the pair form's dechirp operand: its stages take 64 pulses.
inline int pair_mrow(int M) { return (M + 63) / 64 * 64; }
// Tile width (B rows, two per slot) of the pair form's contraction: of 256, 224 and 192 the
// one with the fewest tiles (each tile loads the gathered operand again and has its own
// epilogue: the kernel's time follows the tile count more than the columns), then the
// fewest columns.  552 slots (the 64 x 16 fine grid): 224 (5 tiles of 112 slots, against
// 5 of 128 at 256); 8352 slots (256 x 64): 256 (66 tiles; 192 would take 87).
inline int pair_bn(int slots) {
    int best = 256;
    long best_tiles = (slots + 127) / 128, best_cols = best_tiles * 256;
    for (int bn : {224, 192}) {
        const long tiles = (slots + bn / 2 - 1) / (bn / 2), cols = tiles * bn;
        if (tiles < best_tiles || (tiles == best_tiles && cols < best_cols)) {
            best = bn;
            best_tiles = tiles;
            best_cols = cols;
        }
    }
    return best;
}

int launch_plain(const Ctx &, const RadarD &, const float2 *echo, const grft_grid &, long h0,
                 int nh, const int32_t *rho, const float2 *w, const float2 *e0, float2 *Y,
                 float *P);

int launch_coarse_rm(const Ctx &, const RadarD &, const float2 *echo, const grft_dsgrid &,
                     int cell_count, const int32_t *rho, const float2 *w, float2 *Z);

struct DsOut {           // output placement of a DS call (v-slab of the canonical layout)
    float2 *Y;
    float *P;
    int cell_begin;      // first coarse cell of the call
    int i0;              // first coarse v row of the slab
    int na_c;            // coarse a count
    int Fv, Fa;
};

// Frequency-domain coarse stage (coarse_rm_fd.cu): range spectra S[M][N] (bit-reversed
// order), then Z[cell][m][j] for the cells.  N a power of two <= 8192.
int launch_range_fft(const Ctx &, const RadarD &, const float2 *echo, float2 *S);
int launch_rm_fd(const Ctx &, const RadarD &, const grft_dsgrid &, int cell_begin, int cell_count,
                 const float2 *S, const float2 *w, float2 *Z, bool positive);   // positive: k in [0, N)

// FFT form of the fine stage (fine_dfm_fft.cu): chirp[Fa][L], then the transform kernel.
int launch_gft_chirp(const Ctx &, const RadarD &, const grft_dsgrid &, int L, float2 *chirp);
int launch_ds_fft(const Ctx &, const RadarD &, const float2 *echo, const grft_dsgrid &, int cell_count,
                  const int32_t *rho, const float2 *w, const float2 *chirp, const float2 *e0, int L,
                  const DsOut &out);

// The same transform on a coarse output Z[cell][M][r0_count], without a range phase.
int launch_ds_fft_z(const Ctx &, const RadarD &, const float2 *Z, const grft_dsgrid &, int cell_count,
                    const float2 *chirp, int L, const DsOut &out);

// Keystone branch (kt.cu): Skt[M][N] (slot order of launch_range_fft) from the range spectra,
// then the coarse H_KT,RM stage Z[cell][m][j].  M, N powers of two, M <= 2048, N <= 8192.
int launch_keystone(const Ctx &, const RadarD &, const float2 *S, float2 *Skt);
int launch_rm_kt(const Ctx &, const RadarD &, const grft_dsgrid &, int cell_begin, int cell_count,
                 const float2 *Skt, float2 *Z);

int launch_ds_simt(const Ctx &, const RadarD &, const float2 *echo, const float2 *Z,
                   const grft_dsgrid &, int cell_count, const int32_t *rho, const float2 *w,
                   const float2 *D, const float2 *e0, const DsOut &out);

// One CPI (or one call's cell range) for the tensor-core DS path.
struct DsTcItem {
    const float2 *echo;      // [M][N] (or nullptr when Z is given)
    const float2 *Z;         // [cells][M][r0_count] materialised coarse-RM output, or nullptr
    float *P;                // outputs, canonical v-slab layout (either may be null)
    float2 *Y;
    const float2 *e0;        // e0[j] = range phase of bin r0_begin + j
    int M, N, r0_begin, r0_count;
    int cell_begin, cell_count, i0;
};
int ds_tc_r0_pad(int r0_count);
// Argument checks shared by the entry points: positive sizes, finite positive radar
// parameters, a non-empty axis with finite start and step.
inline bool radar_ok(const grft_radar *r) {
    return r && r->M > 0 && r->N > 0 && std::isfinite(r->fc_hz) && r->fc_hz > 0 &&
           std::isfinite(r->prf_hz) && r->prf_hz > 0 && std::isfinite(r->dr_m) && r->dr_m > 0 &&
           std::isfinite(r->c_mps) && r->c_mps > 0;
}
inline bool axis_ok(const grft_axis &a) { return a.count > 0 && std::isfinite(a.start) && std::isfinite(a.step); }

// Operand format and products per real MAC of a tensor-core precision (3: hi*hi + hi*lo +
// lo*hi; 2: hi*hi + lo*hi with the dechirp rounded once; 1: hi*hi).
inline bool precision_fp16(grft_precision p) {
    return p == GRFT_FP16X3 || p == GRFT_FP16X1 || p == GRFT_FP16X2;
}
inline int precision_nprod(grft_precision p) { return p == GRFT_FP16X1 ? 1 : (p == GRFT_FP16X2 ? 2 : 3); }
// Split coarse-RM pre-pass + tensor-core contraction for a list of items, in rounds whose
// split operand (at most z_rows_cap rows of 2*Mpad 16-bit values per plane) fits one
// buffer.  Tables rho/w are indexed [cell - tab_cell0][Mtab]; B planes are [2 Fpad][2 Mpad].
// Buffers (Zhi[i], Zlo[i]) of z_rows_cap rows each: with two, the split of one round is
// written into one while the contraction of the previous round reads the other; with one
// (Zhi[1] == nullptr) rounds run one after the other on the caller's stream.
constexpr int DS_TC_MAX_ITEMS = 64;    // CPIs per tensor-core launch (kernel-parameter table)
int launch_ds_tc(const Ctx &, const DsTcItem *items, int n_items, const grft_dsgrid &g,
                 const int32_t *rho, const float2 *w, int tab_cell0, int Mtab, const uint16_t *Bhi,
                 const uint16_t *Blo, int Mpad, bool fp16, int nprod, uint16_t *const Zhi[2],
                 uint16_t *const Zlo[2], long z_rows_cap,    // nprod: 3, 2 or 1 products per real MAC
                 const Rate3 &rate = kNoRate);

int launch_detect(const Ctx &, const float *P, int nv, int na, int nr0, const grft_cfar &cfar,
                  const grft_grid *axes, double dr, int K, grft_det *out, int32_t *n_out);
// The same in three phases (a detection over a map computed in slabs): begin clears the
// per-device candidate list; scan appends the candidates of rows [v_lo, v_hi) of one slab
// of nv rows (the other rows are neighbours only), with idx_off added to their linear
// indices; select sorts every candidate appended since begin into the top K.
int launch_detect_begin(const Ctx &);
int launch_detect_scan(const Ctx &, const float *P, int nv, int na, int nr0, int v_lo, int v_hi, long long idx_off,
                       const grft_cfar &cfar);
int launch_detect_select(const Ctx &, int na, int nr0, const grft_grid *axes, double dr, int K, grft_det *out,
                         int32_t *n_out);
// The top K of the union of n_lists detection lists of K_in records each (device memory).
int launch_detect_merge(const Ctx &, const grft_det *lists, const int32_t *totals, int n_lists, int K_in, int K,
                        grft_det *out, int32_t *n_out);

int launch_backward(const Ctx &, const RadarD &, const float2 *echo, int K, const double *theta,
                    int gather, const float *gP, float *P, float2 *Y, double *g, float2 *gs);

int launch_refine(const Ctx &, const RadarD &, const float2 *echo, int K, double *theta,
                  const double cell[3], int steps, int gather, float *P);

int check_launch();   // GRFT_OK or GRFT_ECUDA from cudaGetLastError

// Records a CUDA-event pair around the launches in its scope when timing is enabled
// (grft_timing) and the stream is not being captured.
class KernelTimer {
  public:
    KernelTimer(const Ctx &c, int kernel);
    ~KernelTimer();
    KernelTimer(const KernelTimer &) = delete;
    KernelTimer &operator=(const KernelTimer &) = delete;

  private:
    cudaStream_t stream_;
    int kernel_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

}  // namespace grft
