// Fine Doppler-migration correction on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// Per coarse cell (Alg. 3) the GFT of Def. 1 / Alg. 2 is a dense complex contraction over
// pulses against the shared dechirp matrix D[m][f] (eq. H-DFM of the fine offsets):
//   Y(n0; c, f) = e0(n0) * sum_m Zc[m][n0] D[m][f],   Zc[m][n0] = s[m][n0 + rho_c(m)] w_c(m)
// It runs as one real GEMM (the "4M" form) with K' = 2M and N' = 2F:
//   [Re Zc | Im Zc] (rows n0)  x  [[Re D, Im D], [-Im D, Re D]]  =  [Re Y~ | Im Y~]
// and each real operand x is split as hi = round16(x), lo = round16(x - hi) (BF16 or FP16),
// accumulating hi*hi + hi*lo + lo*hi in FP32 (three tcgen05.mma per K step).
//
// Kernel organisation (one persistent CTA per SM, 320 threads):
//   warp 0      TMA producer: the split dechirp operand tiles (K-major, 128-byte swizzle)
//   warp 1      TMEM allocation and the single MMA-issuing thread
//   warps 2..5  A producers: gather the coarse-cell echo rows (L2-resident), multiply by the
//               coarse phase w_c(m), split hi/lo and write the 128-byte-swizzled K-major
//               A tile (row = range bin) straight from registers
//   warps 6..9  epilogue: TMEM -> registers (tcgen05.ld 32x32b), |Y|^2 (and Y = e0 * Y~),
//               coalesced stores along r0 (one TMEM lane = one range bin)
// Tile: 128 bins x 256 real columns (128 fine hypotheses) x 64 real k (32 pulses) per
// stage; a 2-stage shared-memory ring (96 KB per stage) and two TMEM accumulators of 256
// columns so that the epilogue of one tile overlaps the main loop of the next.  Every
// mbarrier wait is bounded: a wait that runs out latches GRFT_ETIMEOUT, the CTA unwinds
// (draining its own TMA copies and MMAs with a bounded wait) and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"
#include "tma.cuh"

namespace grft {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BN = 256;                     // real columns per tile
constexpr int TC_BK = 64;                      // real k per stage (32 pulses x re/im)
constexpr int TC_STAGES = 2;
constexpr int TC_THREADS = 320;
constexpr uint32_t TC_A_BYTES = TC_BM * 128;   // 16 KB
constexpr uint32_t TC_B_BYTES = TC_BN * 128;   // 32 KB
constexpr uint32_t TC_STAGE_BYTES = 2 * TC_A_BYTES + 2 * TC_B_BYTES;
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr uint64_t TC_DRAIN_LIMIT = 4000000000ull;   // bounded drain on the unwind path
constexpr int TC_TAB_MAX = 2048;                     // pulses whose bins/phases fit in shared memory
constexpr uint32_t TC_TAB_BYTES = TC_TAB_MAX * (4 + 8);
constexpr size_t TC_SMEM_BYTES = (size_t)TC_STAGES * TC_STAGE_BYTES + TC_TAB_BYTES + 1024;

struct TcParams {
    const float2 *echo;
    const float2 *Z;
    const int32_t *rho;
    const float2 *w;
    const float2 *e0;
    int M, N, Mpad, KT;
    int r0_begin, r0_count;
    int F, tiles_m, tiles_n, total_tiles;
    DsOut out;
    int *status;
    uint64_t wait_limit;
    uint32_t idesc;
    int fp16;
};

// ----------------------------------------------------------------------- tcgen05 wrappers
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused, K-major swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ----------------------------------------------------------------------- operand split
__device__ __forceinline__ void split2(float x0, float x1, bool fp16, uint32_t &hi, uint32_t &lo) {
    if (fp16) {
        const __half2 h = __floats2half2_rn(x0, x1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Named barrier among `count` threads (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// A wait done by lane 0 of a warp, combined with the CTA abort flag and broadcast, so that
// the whole warp takes the same decision (keeps .sync.aligned operations converged).
// Returns false if the wait ran out or the CTA is unwinding; lane 0 then latches the error.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, uint64_t limit,
                                          volatile int *abort_flag, int *status) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        ok = (!*abort_flag && mbar_wait(bar, parity, limit)) ? 1 : 0;
        if (!ok) {
            latch_error(status, GRFT_ETIMEOUT);
            *abort_flag = 1;
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    return ok != 0;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_ds_tc(const __grid_constant__ CUtensorMap mapBhi, const __grid_constant__ CUtensorMap mapBlo,
            const TcParams p) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ alignas(8) uint64_t full_a[TC_STAGES], full_b[TC_STAGES], empty[TC_STAGES];
    __shared__ alignas(8) uint64_t tmem_full[2], tmem_empty[2], drain_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_flag;
    __shared__ long s_rowoff[128];

    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        tma_prefetch_desc(&mapBhi);
        tma_prefetch_desc(&mapBlo);
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full_a[s], 128);
            mbar_init(&full_b[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tmem_full[b], 1);
            mbar_init(&tmem_empty[b], 128);
        }
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        fence_mbarrier_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_holder;
    const uint64_t lim = p.wait_limit;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer (B)
        if (lane == 0) {
            int it = 0;
            int last_it = -1;            // last issued stage use (its stage is last_it % TC_STAGES)
            for (int tile = blockIdx.x; tile < p.total_tiles && !abort_flag; tile += gridDim.x) {
                const int nt = tile % p.tiles_n;
                for (int kt = 0; kt < p.KT; ++kt, ++it) {
                    const int s = it % TC_STAGES;
                    if (!mbar_wait(&empty[s], ((it / TC_STAGES) & 1) ^ 1, lim)) {
                        latch_error(p.status, GRFT_ETIMEOUT);
                        abort_flag = 1;
                        break;
                    }
                    unsigned char *st = smem + s * TC_STAGE_BYTES;
                    mbar_arrive_expect_tx(&full_b[s], 2 * TC_B_BYTES);
                    tma_load_2d(st + 2 * TC_A_BYTES, &mapBhi, kt * TC_BK, nt * TC_BN, &full_b[s]);
                    tma_load_2d(st + 2 * TC_A_BYTES + TC_B_BYTES, &mapBlo, kt * TC_BK, nt * TC_BN,
                                &full_b[s]);
                    last_it = it;
                }
            }
            // drain: every issued load has landed before shared memory can be released (the
            // last use of each stage is last_it and, if issued, last_it - 1)
            for (int u = last_it; u >= 0 && u >= last_it - (TC_STAGES - 1); --u)
                mbar_wait(&full_b[u % TC_STAGES], (u / TC_STAGES) & 1, TC_DRAIN_LIMIT);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int it = 0, tcount = 0;
            bool issued_any = false;
            for (int tile = blockIdx.x; tile < p.total_tiles && !abort_flag; tile += gridDim.x, ++tcount) {
                const int b = tcount & 1;
                if (!mbar_wait(&tmem_empty[b], ((tcount >> 1) & 1) ^ 1, lim)) {
                    latch_error(p.status, GRFT_ETIMEOUT);
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(b * TC_BN);
                bool ok = true;
                for (int kt = 0; kt < p.KT; ++kt, ++it) {
                    const int s = it % TC_STAGES;
                    const uint32_t ph = (it / TC_STAGES) & 1;
                    if (!mbar_wait(&full_a[s], ph, lim) || !mbar_wait(&full_b[s], ph, lim)) {
                        latch_error(p.status, GRFT_ETIMEOUT);
                        abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * TC_STAGE_BYTES;
                    const uint32_t a_hi = st, a_lo = st + TC_A_BYTES;
                    const uint32_t b_hi = st + 2 * TC_A_BYTES, b_lo = b_hi + TC_B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk) {
                        const uint32_t off = kk * 32;   // 16 elements x 2 bytes inside the swizzle row
                        umma_f16(d_tmem, umma_desc(a_hi + off), umma_desc(b_hi + off), p.idesc,
                                 (kt > 0 || kk > 0) ? 1u : 0u);
                        umma_f16(d_tmem, umma_desc(a_hi + off), umma_desc(b_lo + off), p.idesc, 1u);
                        umma_f16(d_tmem, umma_desc(a_lo + off), umma_desc(b_hi + off), p.idesc, 1u);
                    }
                    issued_any = true;
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&tmem_full[b]);
            }
            if (issued_any) {   // drain the MMAs in flight before TMEM is freed
                umma_commit(&drain_bar);
                mbar_wait(&drain_bar, 0, TC_DRAIN_LIMIT);
            }
        }
    } else if (warp < 6) {
        // ------------------------------------------------------------ A producers
        // Thread r owns tile row r (one range bin).  The cell's bins and phases are staged in
        // shared memory once per tile; the 32 echo samples of stage k+1 are requested before
        // stage k is converted, so the L2 latency of the gather overlaps the conversion.
        // Every producer warp runs every tile iteration (also after an abort) so that the
        // named barriers always see all 128 threads.
        const int r = threadIdx.x - 64;
        const bool fp16 = p.fp16 != 0;
        const uint32_t swz = (uint32_t)(r & 7);
        int *s_rho = reinterpret_cast<int *>(smem + TC_STAGES * TC_STAGE_BYTES);
        float2 *s_w = reinterpret_cast<float2 *>(smem + TC_STAGES * TC_STAGE_BYTES + TC_TAB_MAX * 4);
        const bool tab_smem = p.M <= TC_TAB_MAX;
        bool aborted = false;
        int it = 0;
        for (int tile = blockIdx.x; tile < p.total_tiles; tile += gridDim.x) {
            const int nt_m = tile / p.tiles_n;
            const int mt = nt_m % p.tiles_m;
            const int cl = nt_m / p.tiles_m;
            const int j = mt * TC_BM + r;                  // local r0 index
            const bool jok = j < p.r0_count;
            const long tab = (long)cl * p.M;
            const int nbase = p.r0_begin + j;
            named_bar_sync(1, 128);                        // previous tile's table no longer read
            const int *rho_t = p.rho + tab;
            const float2 *w_t = p.w + tab;
            if (!p.Z && tab_smem) {
                if (!aborted)
                    for (int m = r; m < p.M; m += 128) {
                        s_rho[m] = __ldg(p.rho + tab + m);
                        s_w[m] = __ldg(p.w + tab + m);
                    }
                rho_t = s_rho;
                w_t = s_w;
            }
            named_bar_sync(1, 128);
            if (aborted) continue;

            float2 cur[32];
            auto load_stage = [&](int kt, float2 (&v)[32]) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int m = kt * 32 + i;
                    float2 x = make_float2(0.f, 0.f);
                    if (m < p.M && jok) {
                        if (p.Z) {
                            x = __ldg(p.Z + (tab + m) * p.r0_count + j);
                        } else {
                            const int n = nbase + rho_t[m];
                            if ((unsigned)n < (unsigned)p.N) x = __ldg(p.echo + (long)m * p.N + n);
                        }
                    }
                    v[i] = x;
                }
            };
            load_stage(0, cur);
            for (int kt = 0; kt < p.KT; ++kt, ++it) {
                float2 nxt[32];
                if (kt + 1 < p.KT) {
                    load_stage(kt + 1, nxt);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) nxt[i] = make_float2(0.f, 0.f);
                }
                const int s = it % TC_STAGES;
                if (!warp_wait(&empty[s], ((it / TC_STAGES) & 1) ^ 1, lim, &abort_flag, p.status)) {
                    aborted = true;
                    break;
                }
                const uint32_t a_hi = sbase + s * TC_STAGE_BYTES + r * 128;
                const uint32_t a_lo = a_hi + TC_A_BYTES;
#pragma unroll
                for (int g = 0; g < 4; ++g) {       // 8 pulses per 16-byte chunk
                    float re[8], im[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int m = kt * 32 + g * 8 + i;
                        float2 v = cur[g * 8 + i];
                        if (!p.Z && m < p.M) v = cmul(v, w_t[m]);
                        re[i] = v.x;
                        im[i] = v.y;
                    }
                    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        split2(re[2 * q], re[2 * q + 1], fp16, rh[q], rl[q]);
                        split2(im[2 * q], im[2 * q + 1], fp16, ih[q], il[q]);
                    }
                    const uint32_t cre = ((uint32_t)g ^ swz) << 4;         // chunk g     (Re)
                    const uint32_t cim = ((uint32_t)(g + 4) ^ swz) << 4;   // chunk g + 4 (Im)
                    st_shared_v4(a_hi + cre, rh[0], rh[1], rh[2], rh[3]);
                    st_shared_v4(a_lo + cre, rl[0], rl[1], rl[2], rl[3]);
                    st_shared_v4(a_hi + cim, ih[0], ih[1], ih[2], ih[3]);
                    st_shared_v4(a_lo + cim, il[0], il[1], il[2], il[3]);
                }
                fence_proxy_async_shared();
                mbar_arrive(&full_a[s]);
#pragma unroll
                for (int i = 0; i < 32; ++i) cur[i] = nxt[i];
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // Thread (warp q4, lane) owns TMEM lane r = 32 q4 + lane = tile row (range bin).
        // Per tile the 128 output row offsets (one per fine hypothesis of the tile) go to a
        // shared table; stores are streaming (evict-first) so that the output does not push
        // the echo and the dechirp operand out of L2.
        const int q4 = warp & 3;
        const int r = q4 * 32 + lane;
        const int er = threadIdx.x - 192;        // 0..127 over the epilogue warps
        const DsOut o = p.out;
        const int na_full = o.na_c * o.Fa;
        bool aborted = false;
        int tcount = 0;
        for (int tile = blockIdx.x; tile < p.total_tiles; tile += gridDim.x, ++tcount) {
            const int b = tcount & 1;
            const int nt = tile % p.tiles_n;
            const int nt_m = tile / p.tiles_n;
            const int mt = nt_m % p.tiles_m;
            const int cl = nt_m / p.tiles_m;
            const int c = o.cell_begin + cl;
            const int iv = c / o.na_c - o.i0, il = c % o.na_c;
            named_bar_sync(2, 128);                  // previous tile's offsets no longer read
            if (!aborted) {
                const int f = nt * (TC_BN / 2) + er;
                long off = -1;
                if (f < p.F) {
                    const int k = f / o.Fa, q = f % o.Fa;
                    off = ((long)(iv * o.Fv + k) * na_full + (il * o.Fa + q)) * p.r0_count;
                }
                s_rowoff[er] = off;
            }
            named_bar_sync(2, 128);
            if (aborted) continue;
            if (!warp_wait(&tmem_full[b], (tcount >> 1) & 1, lim, &abort_flag, p.status)) {
                aborted = true;
                continue;
            }
            tc_fence_after();
            const int j = mt * TC_BM + r;
            const bool jok = j < p.r0_count;
            const float2 e = (jok && o.Y) ? p.e0[j] : make_float2(1.f, 0.f);
            const uint32_t taddr0 = tmem_base + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * TC_BN);
#pragma unroll 1
            for (int ch = 0; ch < TC_BN / 32; ++ch) {
                uint32_t v[32];
                __syncwarp();
                tmem_ld32(taddr0 + ch * 32, v);
                if (jok) {
#pragma unroll
                    for (int pp = 0; pp < 16; ++pp) {
                        const long ro = s_rowoff[ch * 16 + pp];
                        if (ro >= 0) {
                            const float yr = __uint_as_float(v[2 * pp]);
                            const float yi = __uint_as_float(v[2 * pp + 1]);
                            if (o.P) __stcs(o.P + ro + j, yr * yr + yi * yi);
                            if (o.Y) __stcs(o.Y + ro + j, make_float2(e.x * yr - e.y * yi, e.x * yi + e.y * yr));
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&tmem_empty[b]);
        }
    }

    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

int launch_ds_tc(const Ctx &c, const RadarD &R, const float2 *echo, const float2 *Z,
                 const grft_dsgrid &g, int cell_count, const int32_t *rho, const float2 *w,
                 const uint16_t *Bhi, const uint16_t *Blo, int Mpad, bool fp16, const float2 *e0,
                 const DsOut &out) {
    if (cell_count == 0 || g.r0_count == 0) return GRFT_OK;
    const int F = g.Fv * g.Fa;
    const int Fpad = (F + 127) / 128 * 128;
    CUtensorMap mh, ml;
    const uint64_t kdim = 2ull * Mpad, ndim = 2ull * Fpad;
    if (!encode_tma_2d(&mh, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Bhi, kdim, ndim, kdim * 2, TC_BK,
                       TC_BN, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_tma_2d(&ml, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Blo, kdim, ndim, kdim * 2, TC_BK,
                       TC_BN, CU_TENSOR_MAP_SWIZZLE_128B))
        return GRFT_ECUDA;
    TcParams p;
    p.echo = echo;
    p.Z = Z;
    p.rho = rho;
    p.w = w;
    p.e0 = e0;
    p.M = R.M;
    p.N = R.N;
    p.Mpad = Mpad;
    p.KT = Mpad / 32;
    p.r0_begin = g.r0_begin;
    p.r0_count = g.r0_count;
    p.F = F;
    p.tiles_m = (g.r0_count + TC_BM - 1) / TC_BM;
    p.tiles_n = Fpad / 128;
    const long total = (long)cell_count * p.tiles_m * p.tiles_n;
    if (total > 0x7fffffffL) return GRFT_EINVAL;
    p.total_tiles = (int)total;
    p.out = out;
    p.status = c.status;
    p.wait_limit = c.wait_limit;
    p.fp16 = fp16 ? 1 : 0;
    const uint32_t fmt = fp16 ? 0u : 1u;   // kind::f16 operand format: 0 = F16, 1 = BF16
    p.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
              ((uint32_t)(TC_BM >> 4) << 24);
    const size_t smem = TC_SMEM_BYTES;
    static bool attr_set[64] = {false};
    if (c.device < 64 && !attr_set[c.device]) {
        if (cudaFuncSetAttribute(k_ds_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return GRFT_ECUDA;
        attr_set[c.device] = true;
    }
    const int grid = (int)(total < c.num_sms ? total : c.num_sms);
    k_ds_tc<<<grid, TC_THREADS, smem, c.stream>>>(mh, ml, p);
    return check_launch();
}

}  // namespace grft
