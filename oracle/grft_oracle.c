/*
 * FP64 CPU oracle for the GRFT / DS-GRFT coherent sum, CA-CFAR peak picking and the
 * trajectory adjoint.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg call it; the library never does.  It shares no code,
 * header or table with the CUDA path.
 *
 * Every sum is written out literally in the order the paper states it; there is no
 * blocking, no fusion and no reuse across hypotheses beyond precomputing, per motion
 * hypothesis, the bin and phase of each pulse.
 *
 * Conventions (paper Sec. II, eq. slant range with P = 2; Sec. III-A eq. standard-GRFT-TD):
 *   t_m  = m / PRF, m = 0..M-1
 *   d    = (v*t) + ((0.5*a)*(t*t))     displacement after t_m, every operation rounded once
 *   rho  = floor(d/dr + 0.5)           bin shift (round half up); gathered bin n0 + rho
 *   r    = n0*dr + d                   range of the hypothesis at t_m
 *   phase(r) = exp(+j 4 pi r / lambda), lambda = c / f_c, evaluated from the cycle count
 *              u = 2 r / lambda reduced to u - rint(u)
 *   Samples gathered from outside [0, N) contribute zero.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t M, N;
    double fc, prf, dr, c;
} orc_radar;

typedef struct {
    double re, im;
} cplx;

static inline cplx cmul(cplx x, cplx y) {
    cplx z = {x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re};
    return z;
}

static inline double slow_time(const orc_radar *R, int m) { return (double)m / R->prf; }

/* Displacement of the polynomial trajectory after t (eq. slant range minus c_0). */
static inline double displacement(double v, double a, double t) {
    double vt = v * t;
    double ha = 0.5 * a;
    double tt = t * t;
    double at = ha * tt;
    return vt + at;
}

/* Nearest bin of a displacement: round(d/dr), ties toward +inf (eq. standard-GRFT-TD). */
static inline int32_t bin_shift(double d, double dr) {
    double x = d / dr;
    return (int32_t)floor(x + 0.5);
}

/* exp(+j 4 pi x / lambda) for a range x (the matched phase of eqs. H-DFM, pre-DFM). */
static inline cplx range_phase(double x, double lambda) {
    double u = (2.0 * x) / lambda;
    double f = u - nearbyint(u);
    double ang = 2.0 * M_PI * f;
    cplx z = {cos(ang), sin(ang)};
    return z;
}

static inline cplx echo_at(const float *s, const orc_radar *R, int m, long n) {
    cplx z = {0.0, 0.0};
    if (n >= 0 && n < R->N) {
        const float *p = s + 2 * ((long)m * R->N + n);
        z.re = (double)p[0];
        z.im = (double)p[1];
    }
    return z;
}

/* Thread count of a call: nthreads > 0 as given, else the process default (the OpenMP
 * maximum seen before any call set a count), so that a one-thread call does not pin the
 * later ones. */
static int default_threads(void) {
#ifdef _OPENMP
    static int d = 0;
    if (d == 0) d = omp_get_max_threads();
    return d;
#else
    return 1;
#endif
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : default_threads());
#else
    (void)nthreads;
#endif
}

int orc_num_threads(void) { return default_threads(); }

/* Bin shifts and phases for explicit (v, a) pairs: rho[h][m], w[h][m] = exp(j4pi d/lambda). */
int orc_bins_phases(const orc_radar *R, const double *v, const double *a, int nh, int32_t *rho,
                    double *w) {
    double lambda = R->c / R->fc;
    for (int h = 0; h < nh; ++h) {
        for (int m = 0; m < R->M; ++m) {
            double t = slow_time(R, m);
            double d = displacement(v[h], a[h], t);
            rho[(long)h * R->M + m] = bin_shift(d, R->dr);
            cplx p = range_phase(d, lambda);
            w[2 * ((long)h * R->M + m)] = p.re;
            w[2 * ((long)h * R->M + m) + 1] = p.im;
        }
    }
    return 0;
}

/*
 * TD-GRFT (eq. standard-GRFT-TD, with the range phase of the full trajectory):
 *   Y(n0, v, a) = sum_m s[m][n0 + rho(v,a,m)] exp(j 4 pi (n0 dr + d(v,a,t_m)) / lambda)
 * for rows (vi[i], ai[i]) of the plain grid and n0 in [r0_begin, r0_begin + r0_count).
 * Y is [nrows][r0_count] complex (interleaved doubles).
 */
int orc_grft_plain_rows(const orc_radar *R, const float *s, int32_t r0_begin, int32_t r0_count,
                        double v0, double dv, double a0, double da, const int32_t *vi,
                        const int32_t *ai, int nrows, double *Y, int nthreads) {
    set_threads(nthreads);
    double lambda = R->c / R->fc;
    int M = R->M;
#pragma omp parallel
    {
        int32_t *rho = (int32_t *)malloc(sizeof(int32_t) * M);
        double *dis = (double *)malloc(sizeof(double) * M);
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < nrows; ++i) {
            double v = v0 + (double)vi[i] * dv;
            double a = a0 + (double)ai[i] * da;
            for (int m = 0; m < M; ++m) {
                double t = slow_time(R, m);
                dis[m] = displacement(v, a, t);
                rho[m] = bin_shift(dis[m], R->dr);
            }
            for (int j = 0; j < r0_count; ++j) {
                int n0 = r0_begin + j;
                cplx acc = {0.0, 0.0};
                for (int m = 0; m < M; ++m) {
                    cplx sv = echo_at(s, R, m, (long)n0 + rho[m]);
                    cplx ph = range_phase((double)n0 * R->dr + dis[m], lambda);
                    cplx p = cmul(sv, ph);
                    acc.re += p.re;
                    acc.im += p.im;
                }
                Y[2 * ((long)i * r0_count + j)] = acc.re;
                Y[2 * ((long)i * r0_count + j) + 1] = acc.im;
            }
        }
        free(rho);
        free(dis);
    }
    return 0;
}

/* Coarse centre and fine offset of the dual-scale grid (eqs. Partition-Parameter,
 * Space_c_c, Space_c_f; half-open fine grid (k - F/2) step_c / F). */
static inline double coarse_value(double start, double step, int i) { return start + (double)i * step; }
static inline double fine_offset(double step_c, int F, int k) {
    double off = (double)(2 * k - F) * 0.5;
    return off * (step_c / (double)F);
}

/*
 * mGIFT in the time domain (Alg. 1 restated with a gather; eq. pre-DFM):
 *   Z[c][m][n0] = s[m][n0 + rho_c(m)] exp(j 4 pi d_c(t_m) / lambda)
 * for coarse cells c = i*na_c + l in [cell_begin, cell_begin + cell_count).
 */
int orc_coarse_rm(const orc_radar *R, const float *s, int32_t r0_begin, int32_t r0_count,
                  double vc0, double dvc, int32_t nvc, double ac0, double dac, int32_t nac,
                  int32_t cell_begin, int32_t cell_count, double *Z, int nthreads) {
    set_threads(nthreads);
    (void)nvc;
    double lambda = R->c / R->fc;
    int M = R->M;
#pragma omp parallel for schedule(dynamic, 1)
    for (int cc = 0; cc < cell_count; ++cc) {
        int c = cell_begin + cc;
        int i = c / nac, l = c % nac;
        double vc = coarse_value(vc0, dvc, i), ac = coarse_value(ac0, dac, l);
        for (int m = 0; m < M; ++m) {
            double t = slow_time(R, m);
            double d = displacement(vc, ac, t);
            int32_t rho = bin_shift(d, R->dr);
            cplx w = range_phase(d, lambda);
            for (int j = 0; j < r0_count; ++j) {
                cplx sv = echo_at(s, R, m, (long)r0_begin + j + rho);
                cplx z = cmul(sv, w);
                long o = ((long)cc * M + m) * r0_count + j;
                Z[2 * o] = z.re;
                Z[2 * o + 1] = z.im;
            }
        }
    }
    return 0;
}

/*
 * DS-GRFT (Alg. 3: mGIFT over the coarse cell, then GFT over the fine offsets; Prop. 2):
 *   Y(n0; c, k, q) = exp(j 4 pi n0 dr / lambda)
 *        * sum_m s[m][n0 + rho_c(m)] exp(j 4 pi d(v_c, a_c, t_m)/lambda) exp(j 4 pi d(dv_k, da_q, t_m)/lambda)
 * i.e. the RM is corrected with the coarse trajectory only, and the phase is the
 * product H_pre-DFM(c_c) * H_DFM(c_f) (kappa = 1 in this time-domain form).
 * Rows are (cell[i], fine[i]) with fine = k*Fa + q.  Y is [nrows][r0_count] complex.
 */
int orc_dsgrft_rows(const orc_radar *R, const float *s, int32_t r0_begin, int32_t r0_count,
                    double vc0, double dvc, int32_t nvc, double ac0, double dac, int32_t nac,
                    int32_t Fv, int32_t Fa, const int32_t *cell, const int32_t *fine, int nrows,
                    double *Y, int nthreads) {
    set_threads(nthreads);
    (void)nvc;
    double lambda = R->c / R->fc;
    int M = R->M;
#pragma omp parallel
    {
        int32_t *rho = (int32_t *)malloc(sizeof(int32_t) * M);
        cplx *w = (cplx *)malloc(sizeof(cplx) * M);
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < nrows; ++i) {
            int c = cell[i], f = fine[i];
            int iv = c / nac, il = c % nac;
            int k = f / Fa, q = f % Fa;
            double vc = coarse_value(vc0, dvc, iv), ac = coarse_value(ac0, dac, il);
            double fv = fine_offset(dvc, Fv, k), fa = fine_offset(dac, Fa, q);
            for (int m = 0; m < M; ++m) {
                double t = slow_time(R, m);
                double dc = displacement(vc, ac, t);
                double df = displacement(fv, fa, t);
                rho[m] = bin_shift(dc, R->dr);
                w[m] = cmul(range_phase(dc, lambda), range_phase(df, lambda));
            }
            for (int j = 0; j < r0_count; ++j) {
                int n0 = r0_begin + j;
                cplx acc = {0.0, 0.0};
                for (int m = 0; m < M; ++m) {
                    cplx p = cmul(echo_at(s, R, m, (long)n0 + rho[m]), w[m]);
                    acc.re += p.re;
                    acc.im += p.im;
                }
                cplx y = cmul(range_phase((double)n0 * R->dr, lambda), acc);
                Y[2 * ((long)i * r0_count + j)] = y.re;
                Y[2 * ((long)i * r0_count + j) + 1] = y.im;
            }
        }
        free(rho);
        free(w);
    }
    return 0;
}

/*
 * CA-CFAR along r0 plus a 3x3x3 local-maximum test, then the K largest (LRT test of
 * eq. LRT with a cell-averaging threshold; Alg. 3's threshold scan).
 * P is [nv][na][nr0] (double).  For a cell n of row (v, a):
 *   training cells: [n-G-T, n-G-1] and [n+G+1, n+G+T], clipped to [0, nr0); Nt = count
 *   mode 0: detect if Nt > 0 and P > (pfa^(-1/Nt) - 1) * sum(training)
 *           (= alpha * mean with alpha = Nt (pfa^(-1/Nt) - 1))
 *   mode 1: detect if P > fixed_thresh
 *   and (both modes) (P, -index) exceeds that of each of the up-to-26 neighbours
 *   (n+-1, v+-1, a+-1, clipped).  index = (v*na + a)*nr0 + n.
 * The detections are ranked by P descending, ties by lower index; the first K are
 * returned.  Returns the total number of detections (which may exceed K).
 */
static int cmp_det(const void *x, const void *y) {
    const double *a = (const double *)x, *b = (const double *)y;
    if (a[0] > b[0]) return -1;
    if (a[0] < b[0]) return 1;
    if (a[1] < b[1]) return -1;
    if (a[1] > b[1]) return 1;
    return 0;
}

long orc_cfar_detect(const double *P, int32_t nv, int32_t na, int32_t nr0, int32_t guard,
                     int32_t train, double pfa, double fixed_thresh, int32_t mode, int32_t K,
                     int64_t *out_idx, double *out_p, int nthreads) {
    set_threads(nthreads);
    long total = (long)nv * na * nr0;
    char *hit = (char *)calloc((size_t)total, 1);
#pragma omp parallel for schedule(dynamic, 16)
    for (long row = 0; row < (long)nv * na; ++row) {
        int vi = (int)(row / na), ai = (int)(row % na);
        const double *pr = P + row * nr0;
        for (int n = 0; n < nr0; ++n) {
            int pass;
            if (mode == 0) {
                double sum = 0.0;
                int nt = 0;
                for (int j = n - guard - train; j <= n - guard - 1; ++j)
                    if (j >= 0 && j < nr0) { sum += pr[j]; ++nt; }
                for (int j = n + guard + 1; j <= n + guard + train; ++j)
                    if (j >= 0 && j < nr0) { sum += pr[j]; ++nt; }
                pass = nt > 0 && pr[n] > (pow(pfa, -1.0 / (double)nt) - 1.0) * sum;
            } else {
                pass = pr[n] > fixed_thresh;
            }
            if (!pass) continue;
            long me = row * nr0 + n;
            int ismax = 1;
            for (int dvv = -1; dvv <= 1 && ismax; ++dvv)
                for (int daa = -1; daa <= 1 && ismax; ++daa)
                    for (int dn = -1; dn <= 1 && ismax; ++dn) {
                        if (!dvv && !daa && !dn) continue;
                        int v2 = vi + dvv, a2 = ai + daa, n2 = n + dn;
                        if (v2 < 0 || v2 >= nv || a2 < 0 || a2 >= na || n2 < 0 || n2 >= nr0) continue;
                        long o = ((long)v2 * na + a2) * nr0 + n2;
                        if (P[o] > pr[n] || (P[o] == pr[n] && o < me)) ismax = 0;
                    }
            if (ismax) hit[me] = 1;
        }
    }
    long cnt = 0;
    for (long i = 0; i < total; ++i) cnt += hit[i];
    double *list = (double *)malloc(sizeof(double) * 2 * (cnt ? cnt : 1));
    long j = 0;
    for (long i = 0; i < total; ++i)
        if (hit[i]) { list[2 * j] = P[i]; list[2 * j + 1] = (double)i; ++j; }
    qsort(list, (size_t)cnt, 2 * sizeof(double), cmp_det);
    for (long i = 0; i < cnt && i < K; ++i) {
        out_p[i] = list[2 * i];
        out_idx[i] = (int64_t)list[2 * i + 1];
    }
    free(list);
    free(hit);
    return cnt;
}

/*
 * Coherent sum along a continuous trajectory theta = (r0 [m], v, a) and its adjoint.
 *   r_m = r0 + d(v, a, t_m),  x_m = r_m / dr
 *   nearest (mode 0): s~_m = s[m][floor(x_m + 0.5)]
 *   linear  (mode 1): s~_m = (1 - phi) s[m][n] + phi s[m][n+1], n = floor(x_m), phi = x_m - n
 *   Y = sum_m s~_m exp(j 4 pi r_m / lambda),   P = |Y|^2
 *   dY/dtheta_j = sum_m [ (ds~/dx) (dr/dtheta_j)/dr + s~_m j (4 pi / lambda) dr/dtheta_j ] exp(j4pi r_m/lambda)
 *   with dr/dtheta = (1, t, t^2/2);  dP/dtheta_j = 2 Re(conj(Y) dY/dtheta_j)
 *   grad_s[m][n] += gP * 2 Y conj(weight * exp(j4pi r_m/lambda))   (the d/dRe + j d/dIm convention)
 * Outputs per detection: P[k], Y[k] (complex), g[k][3].  grad_s may be NULL; gP may be NULL (ones).
 */
static void traj_eval(const orc_radar *R, const float *s, const double *th, int mode, cplx *Yo,
                      cplx dY[3]) {
    double lambda = R->c / R->fc;
    double k4 = 4.0 * M_PI / lambda;
    cplx Y = {0, 0};
    cplx d[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int m = 0; m < R->M; ++m) {
        double t = slow_time(R, m);
        double r = th[0] + displacement(th[1], th[2], t);
        double x = r / R->dr;
        cplx st, ds = {0, 0};
        if (mode == 0) {
            st = echo_at(s, R, m, (long)floor(x + 0.5));
        } else {
            double fl = floor(x);
            double phi = x - fl;
            cplx s0 = echo_at(s, R, m, (long)fl), s1 = echo_at(s, R, m, (long)fl + 1);
            st.re = (1.0 - phi) * s0.re + phi * s1.re;
            st.im = (1.0 - phi) * s0.im + phi * s1.im;
            ds.re = s1.re - s0.re;
            ds.im = s1.im - s0.im;
        }
        cplx w = range_phase(r, lambda);
        cplx sw = cmul(st, w);
        Y.re += sw.re;
        Y.im += sw.im;
        double drdth[3] = {1.0, t, 0.5 * t * t};
        for (int j = 0; j < 3; ++j) {
            /* (ds/dx)(dr/dth)/dr + s * j k4 dr/dth */
            cplx term = {ds.re * drdth[j] / R->dr - st.im * k4 * drdth[j],
                         ds.im * drdth[j] / R->dr + st.re * k4 * drdth[j]};
            cplx tw = cmul(term, w);
            d[j].re += tw.re;
            d[j].im += tw.im;
        }
    }
    *Yo = Y;
    for (int j = 0; j < 3; ++j) dY[j] = d[j];
}

int orc_trajectory_grad(const orc_radar *R, const float *s, int32_t K, const double *theta,
                        int32_t mode, const double *gP, double *P, double *Y, double *g,
                        double *grad_s, int nthreads) {
    set_threads(nthreads);
    double lambda = R->c / R->fc;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        cplx Yk, dY[3];
        traj_eval(R, s, theta + 3 * k, mode, &Yk, dY);
        if (P) P[k] = Yk.re * Yk.re + Yk.im * Yk.im;
        if (Y) { Y[2 * k] = Yk.re; Y[2 * k + 1] = Yk.im; }
        if (g)
            for (int j = 0; j < 3; ++j) g[3 * k + j] = 2.0 * (Yk.re * dY[j].re + Yk.im * dY[j].im);
    }
    if (grad_s) {
        /* serial scatter so that the accumulation order is fixed */
        for (int k = 0; k < K; ++k) {
            cplx Yk, dY[3];
            const double *th = theta + 3 * k;
            traj_eval(R, s, th, mode, &Yk, dY);
            double scale = 2.0 * (gP ? gP[k] : 1.0);
            for (int m = 0; m < R->M; ++m) {
                double t = slow_time(R, m);
                double r = th[0] + displacement(th[1], th[2], t);
                double x = r / R->dr;
                cplx w = range_phase(r, lambda);
                cplx cw = {w.re, -w.im};
                cplx yw = cmul(Yk, cw);
                long nn[2];
                double wt[2];
                int cnt;
                if (mode == 0) { nn[0] = (long)floor(x + 0.5); wt[0] = 1.0; cnt = 1; }
                else {
                    double fl = floor(x), phi = x - fl;
                    nn[0] = (long)fl; wt[0] = 1.0 - phi; nn[1] = (long)fl + 1; wt[1] = phi; cnt = 2;
                }
                for (int q = 0; q < cnt; ++q) {
                    if (nn[q] < 0 || nn[q] >= R->N) continue;
                    long o = (long)m * R->N + nn[q];
                    grad_s[2 * o] += scale * wt[q] * yw.re;
                    grad_s[2 * o + 1] += scale * wt[q] * yw.im;
                }
            }
        }
    }
    return 0;
}

/*
 * Sub-grid gradient-ascent refinement of K detections (an addition to the paper's
 * on-grid estimate of Alg. 3 / eq. MLE-GRFT-FD):
 *   cell = (cr, cv, ca) scale of each coordinate (one fine grid step)
 *   g = dP/dtheta at theta;  eta = 0.5 / max_j |cell_j g_j|   (first step <= 0.5 cell)
 *   repeat `steps` times:  theta' = theta + eta cell^2 . g
 *       if P(theta') >= P(theta): accept (theta, P, g updated)  else: eta = eta / 2
 * theta_io is updated in place; P_out gets the final power.
 */
int orc_refine(const orc_radar *R, const float *s, int32_t K, double *theta_io, const double *cell,
               int32_t steps, int32_t mode, double *P_out, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k) {
        double *th = theta_io + 3 * k;
        cplx Y, dY[3];
        traj_eval(R, s, th, mode, &Y, dY);
        double P = Y.re * Y.re + Y.im * Y.im;
        double g[3];
        for (int j = 0; j < 3; ++j) g[j] = 2.0 * (Y.re * dY[j].re + Y.im * dY[j].im);
        double gmax = 0.0;
        for (int j = 0; j < 3; ++j) {
            double z = fabs(cell[j] * g[j]);
            if (z > gmax) gmax = z;
        }
        if (gmax > 0.0) {
            double eta = 0.5 / gmax;
            for (int it = 0; it < steps; ++it) {
                double tn[3];
                for (int j = 0; j < 3; ++j) tn[j] = th[j] + eta * cell[j] * cell[j] * g[j];
                cplx Yn, dYn[3];
                traj_eval(R, s, tn, mode, &Yn, dYn);
                double Pn = Yn.re * Yn.re + Yn.im * Yn.im;
                if (Pn >= P) {
                    for (int j = 0; j < 3; ++j) {
                        th[j] = tn[j];
                        g[j] = 2.0 * (Yn.re * dYn[j].re + Yn.im * dYn[j].im);
                    }
                    P = Pn;
                } else {
                    eta *= 0.5;
                }
            }
        }
        P_out[k] = P;
    }
    return 0;
}
