// Coarse range-migration correction, the time-domain form of mGIFT (Def. 2, eq. pre-DFM,
// Alg. 1):  Z[c][m][j] = s[m][r0_begin + j + rho_c(m)] * w_c(m).
//
// For one pulse the gather is a contiguous row segment shifted by rho_c(m), so each CTA
// stages its rows with 2-D TMA loads into shared memory: one box of CR_SEG + 2 complex
// samples per (row, 128-bin segment), its x coordinate rounded down to an even sample so
// that x * 8 bytes stays 16-byte aligned; the remainder (0 or 1) is applied when reading
// shared memory.  Out-of-range columns (negative or >= N) are zero-filled by the TMA
// unit, which is exactly the "outside [0, N) contributes zero" rule.  The phase multiply
// happens on the way out; Z is written with coalesced 8-byte stores.  HBM-bound on the
// Z write (the echo stays L2-resident).  Rows of odd length (N odd) cannot be described
// to the TMA unit (16-byte stride rule) and take a plain-load path.
#include "internal.cuh"
#include "tma.cuh"

namespace grft {

namespace {

constexpr int CR_THREADS = 128;
constexpr int CR_ROWS = 8;       // pulses per CTA
constexpr int CR_SEG = 128;      // bins per TMA box (plus 2)
constexpr int CR_NSEG = 4;       // segments per CTA -> 512 bins
constexpr int CR_BOX = CR_SEG + 2;
constexpr int CR_PITCH = 144;    // box padded to 1152 B: every TMA destination 128-byte aligned
constexpr int CR_COLS = CR_SEG * CR_NSEG;
static_assert((CR_PITCH * 8) % 128 == 0 && CR_PITCH >= CR_BOX, "TMA smem destinations need 128 B alignment");

__global__ __launch_bounds__(CR_THREADS) void k_coarse_rm_tma(
    const __grid_constant__ CUtensorMap tmap, int M, int N, const int32_t *__restrict__ rho_c,
    const float2 *__restrict__ w_c, int r0_begin, int r0_count, float2 *__restrict__ Z,
    int *status, uint64_t wait_limit) {
    __shared__ alignas(128) float2 buf[CR_ROWS][CR_NSEG][CR_PITCH];
    __shared__ alignas(8) uint64_t bar;
    __shared__ int s_off[CR_ROWS];
    __shared__ float2 s_w[CR_ROWS];

    const int cl = blockIdx.z;
    const int m0 = blockIdx.y * CR_ROWS;
    const int j0 = blockIdx.x * CR_COLS;
    const int rows = min(CR_ROWS, M - m0);

    if (threadIdx.x == 0) {
        tma_prefetch_desc(&tmap);
        mbar_init(&bar, 1);
        fence_mbarrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (uint32_t)(rows * CR_NSEG * CR_BOX * sizeof(float2)));
        for (int r = 0; r < rows; ++r) {
            const long o = (long)cl * M + m0 + r;
            const int x = r0_begin + j0 + rho_c[o];
            const int xe = x & ~1;          // floor to even (two's complement, also for x < 0)
            s_off[r] = x - xe;
            s_w[r] = w_c[o];
            for (int sg = 0; sg < CR_NSEG; ++sg)
                tma_load_2d(&buf[r][sg][0], &tmap, xe + sg * CR_SEG, m0 + r, &bar);
        }
    }
    __syncthreads();   // s_off / s_w visible
    if (!mbar_wait(&bar, 0, wait_limit)) {
        if (threadIdx.x == 0) latch_error(status, GRFT_ETIMEOUT);
        // give the copies in flight one more bounded wait before shared memory is released
        mbar_wait(&bar, 0, wait_limit);
        return;
    }
    for (int r = 0; r < rows; ++r) {
        const int off = s_off[r];
        const float2 w = s_w[r];
        float2 *zrow = Z + ((long)cl * M + m0 + r) * r0_count;
#pragma unroll
        for (int q = 0; q < CR_COLS / CR_THREADS; ++q) {
            const int jn = q * CR_THREADS + threadIdx.x;
            const int j = j0 + jn;
            if (j < r0_count) {
                const float2 sv = buf[r][jn / CR_SEG][jn % CR_SEG + off];
                zrow[j] = cmul(sv, w);
            }
        }
    }
}

// Plain-load variant (any N): same output.
__global__ __launch_bounds__(256) void k_coarse_rm_ld(const float2 *__restrict__ echo, int M, int N,
                                                      const int32_t *__restrict__ rho_c,
                                                      const float2 *__restrict__ w_c, int r0_begin,
                                                      int r0_count, float2 *__restrict__ Z) {
    const int cl = blockIdx.z;
    const int m = blockIdx.y;
    const long o = (long)cl * M + m;
    const int rho = rho_c[o];
    const float2 w = w_c[o];
    const float2 *row = echo + (long)m * N;
    float2 *zrow = Z + o * r0_count;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < r0_count; j += gridDim.x * blockDim.x) {
        const int n = r0_begin + j + rho;
        const float2 sv = ((unsigned)n < (unsigned)N) ? __ldg(row + n) : make_float2(0.f, 0.f);
        zrow[j] = cmul(sv, w);
    }
}

}  // namespace

int launch_coarse_rm(const Ctx &c, const RadarD &R, const float2 *echo, const grft_dsgrid &g,
                     int cell_count, const int32_t *rho, const float2 *w, float2 *Z) {
    if (cell_count == 0 || g.r0_count == 0) return GRFT_OK;
    const bool tma_ok = (R.N % 2 == 0) && (((uintptr_t)echo & 15) == 0);
    if (tma_ok) {
        CUtensorMap map;
        if (encode_tma_2d(&map, CU_TENSOR_MAP_DATA_TYPE_INT64, (void *)echo, (uint64_t)R.N,
                          (uint64_t)R.M, (uint64_t)R.N * 8, CR_BOX, 1, CU_TENSOR_MAP_SWIZZLE_NONE)) {
            dim3 grid((g.r0_count + CR_COLS - 1) / CR_COLS, (R.M + CR_ROWS - 1) / CR_ROWS, cell_count);
            KernelTimer kt(c, GRFT_KERNEL_COARSE_RM);
            k_coarse_rm_tma<<<grid, CR_THREADS, 0, c.stream>>>(map, R.M, R.N, rho, w, g.r0_begin,
                                                               g.r0_count, Z, c.status, c.wait_limit);
            return check_launch();
        }
    }
    dim3 grid((g.r0_count + 255) / 256 < 8 ? (g.r0_count + 255) / 256 : 8, R.M, cell_count);
    KernelTimer kt(c, GRFT_KERNEL_COARSE_RM);
    k_coarse_rm_ld<<<grid, 256, 0, c.stream>>>(echo, R.M, R.N, rho, w, g.r0_begin, g.r0_count, Z);
    return check_launch();
}

}  // namespace grft
