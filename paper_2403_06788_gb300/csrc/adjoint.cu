// Coherent sum along continuous trajectories and its hand-written adjoint (an addition
// to the paper, which stops at the on-grid estimate of eq. MLE-GRFT-FD):
//   r_m = r0 + v t_m + a t_m^2 / 2,  x_m = r_m / dr
//   nearest: s~ = s[m][floor(x + 0.5)];  linear: s~ = (1-phi) s[m][n] + phi s[m][n+1]
//   Y = sum_m s~ exp(j 4 pi r_m / lambda),  P = |Y|^2
//   dY/dth_j = sum_m [ (ds~/dx)(dr/dth_j)/dr + j (4 pi/lambda)(dr/dth_j) s~ ] exp(j4pi r_m/lambda)
//   dP/dth_j = 2 Re(conj(Y) dY/dth_j);  grad_s[m][n] += gP * 2 Y conj(weight * exp(...))
// Ranges, bins and phases are recomputed in FP64 per pulse (never stored); the per-pulse
// terms are FP32 and their sums are accumulated in FP64 (a few thousand additions per
// trajectory).  One CTA per trajectory: a strided loop over pulses, then a block reduction.
#include "internal.cuh"

namespace grft {

namespace {

constexpr int AD_THREADS = 256;

struct Sums {
    // Y.re, Y.im, dY0.re, dY0.im, dY1.re, dY1.im, dY2.re, dY2.im, accumulated in FP64.
    // dY0 omits the term j (4 pi/lambda) Y of dY/dr0: Re(conj(Y) j c Y) = 0 exactly, and in
    // finite precision that large term would swamp the small real part that remains.
    double v[8];
};

__device__ __forceinline__ float2 echo_at(const float2 *__restrict__ s, int N, int m, long n) {
    return (n >= 0 && n < N) ? __ldg(s + (long)m * N + n) : make_float2(0.f, 0.f);
}

// Partial sums of this thread over pulses m = threadIdx.x, +blockDim.x, ...
__device__ Sums traj_partial(const RadarD &R, const float2 *__restrict__ s, const double th[3],
                             int gather) {
    Sums acc;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc.v[i] = 0.0;
    const float k4 = (float)(4.0 * 3.141592653589793 / R.lambda);
    const float inv_dr = (float)(1.0 / R.dr);
    for (int m = threadIdx.x; m < R.M; m += blockDim.x) {
        const double t = slow_time(m, R.prf);
        const double r = __dadd_rn(th[0], displacement(th[1], th[2], t));
        const double x = __ddiv_rn(r, R.dr);
        float2 st, ds = make_float2(0.f, 0.f);
        if (gather == GRFT_GATHER_NEAREST) {
            st = echo_at(s, R.N, m, (long)floor(__dadd_rn(x, 0.5)));
        } else {
            const double fl = floor(x);
            const float phi = (float)__dsub_rn(x, fl);
            const float2 s0 = echo_at(s, R.N, m, (long)fl), s1 = echo_at(s, R.N, m, (long)fl + 1);
            st = make_float2((1.f - phi) * s0.x + phi * s1.x, (1.f - phi) * s0.y + phi * s1.y);
            ds = make_float2(s1.x - s0.x, s1.y - s0.y);
        }
        const float2 w = range_phase(r, R.lambda);
        const float2 sw = cmul(st, w);
        acc.v[0] += sw.x;
        acc.v[1] += sw.y;
        const float tf = (float)t;
        const float drdth[3] = {1.f, tf, 0.5f * tf * tf};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float c = drdth[j] * inv_dr, q = j == 0 ? 0.f : k4 * drdth[j];
            const float2 term = make_float2(ds.x * c - q * st.y, ds.y * c + q * st.x);
            const float2 tw = cmul(term, w);
            acc.v[2 + 2 * j] += tw.x;
            acc.v[3 + 2 * j] += tw.y;
        }
    }
    return acc;
}

// Block-wide sum of the 8 partials; every thread gets the total.
__device__ Sums block_sum(Sums a) {
    __shared__ double red[AD_THREADS / 32][8];
    __shared__ double tot[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        double x = a.v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        a.v[i] = x;
    }
    const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 8; ++i) red[w][i] = a.v[i];
    __syncthreads();
    if (threadIdx.x < 8) {
        double x = 0.0;
        for (int q = 0; q < (int)(blockDim.x / 32); ++q) x += red[q][threadIdx.x];
        tot[threadIdx.x] = x;
    }
    __syncthreads();
    Sums r;
#pragma unroll
    for (int i = 0; i < 8; ++i) r.v[i] = tot[i];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void power_and_grad(const Sums &S, double &P, double g[3]) {
    P = S.v[0] * S.v[0] + S.v[1] * S.v[1];
#pragma unroll
    for (int j = 0; j < 3; ++j) g[j] = 2.0 * (S.v[0] * S.v[2 + 2 * j] + S.v[1] * S.v[3 + 2 * j]);
}

__global__ __launch_bounds__(AD_THREADS) void k_backward(RadarD R, const float2 *__restrict__ s,
                                                         const double *__restrict__ theta, int gather,
                                                         const float *__restrict__ gP,
                                                         float *__restrict__ P, float2 *__restrict__ Y,
                                                         double *__restrict__ g, float2 *grad_s) {
    const int k = blockIdx.x;
    const double th[3] = {theta[3 * k], theta[3 * k + 1], theta[3 * k + 2]};
    const Sums S = block_sum(traj_partial(R, s, th, gather));
    const float scale = gP ? gP[k] : 1.f;
    if (threadIdx.x == 0) {
        double p;
        double gr[3];
        power_and_grad(S, p, gr);
        if (P) P[k] = (float)p;
        if (Y) Y[k] = make_float2((float)S.v[0], (float)S.v[1]);
        if (g)
            for (int j = 0; j < 3; ++j) g[3 * k + j] = scale * gr[j];
    }
    if (!grad_s) return;
    const float2 Yk = make_float2((float)S.v[0], (float)S.v[1]);
    for (int m = threadIdx.x; m < R.M; m += blockDim.x) {
        const double t = slow_time(m, R.prf);
        const double r = __dadd_rn(th[0], displacement(th[1], th[2], t));
        const double x = __ddiv_rn(r, R.dr);
        const float2 w = range_phase(r, R.lambda);
        const float2 yw = cmul(Yk, make_float2(w.x, -w.y));    // Y conj(w)
        long nn[2];
        float wt[2];
        int cnt;
        if (gather == GRFT_GATHER_NEAREST) {
            nn[0] = (long)floor(__dadd_rn(x, 0.5));
            wt[0] = 1.f;
            cnt = 1;
        } else {
            const double fl = floor(x);
            const float phi = (float)__dsub_rn(x, fl);
            nn[0] = (long)fl;
            wt[0] = 1.f - phi;
            nn[1] = (long)fl + 1;
            wt[1] = phi;
            cnt = 2;
        }
        for (int q = 0; q < cnt; ++q) {
            if (nn[q] < 0 || nn[q] >= R.N) continue;
            float2 *dst = grad_s + (long)m * R.N + nn[q];
            const float c = 2.f * scale * wt[q];
            atomicAdd(&dst->x, c * yw.x);
            atomicAdd(&dst->y, c * yw.y);
        }
    }
}

__global__ __launch_bounds__(AD_THREADS) void k_refine(RadarD R, const float2 *__restrict__ s,
                                                       double *__restrict__ theta, double c0, double c1,
                                                       double c2, int steps, int gather,
                                                       float *__restrict__ P_out) {
    const int k = blockIdx.x;
    const double cell[3] = {c0, c1, c2};
    double th[3] = {theta[3 * k], theta[3 * k + 1], theta[3 * k + 2]};
    double P;
    double g[3];
    power_and_grad(block_sum(traj_partial(R, s, th, gather)), P, g);
    double gmax = 0.0;
    for (int j = 0; j < 3; ++j) gmax = fmax(gmax, fabs(cell[j] * g[j]));
    if (gmax > 0.0) {
        double eta = 0.5 / gmax;
        for (int it = 0; it < steps; ++it) {
            double tn[3];
            for (int j = 0; j < 3; ++j) tn[j] = th[j] + eta * cell[j] * cell[j] * g[j];
            double Pn;
            double gn[3];
            power_and_grad(block_sum(traj_partial(R, s, tn, gather)), Pn, gn);
            if (Pn >= P) {       // block-uniform decision (every thread holds the same sums)
                for (int j = 0; j < 3; ++j) {
                    th[j] = tn[j];
                    g[j] = gn[j];
                }
                P = Pn;
            } else {
                eta *= 0.5;
            }
        }
    }
    if (threadIdx.x == 0) {
        for (int j = 0; j < 3; ++j) theta[3 * k + j] = th[j];
        P_out[k] = (float)P;
    }
}

}  // namespace

int launch_backward(const Ctx &c, const RadarD &R, const float2 *echo, int K, const double *theta,
                    int gather, const float *gP, float *P, float2 *Y, double *g, float2 *gs) {
    if (K == 0) return GRFT_OK;
    KernelTimer kt(c, GRFT_KERNEL_ADJOINT);
    k_backward<<<K, AD_THREADS, 0, c.stream>>>(R, echo, theta, gather, gP, P, Y, g, gs);
    return check_launch();
}

int launch_refine(const Ctx &c, const RadarD &R, const float2 *echo, int K, double *theta,
                  const double cell[3], int steps, int gather, float *P) {
    if (K == 0) return GRFT_OK;
    KernelTimer kt(c, GRFT_KERNEL_ADJOINT);
    k_refine<<<K, AD_THREADS, 0, c.stream>>>(R, echo, theta, cell[0], cell[1], cell[2], steps, gather, P);
    return check_launch();
}

}  // namespace grft
