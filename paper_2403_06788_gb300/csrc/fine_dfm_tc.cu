// The dual-scale cascade on the tensor cores (Alg. 3): coarse range-migration correction
// in split form (kernel a) feeding the fine Doppler-migration contraction on the
// 5th-generation tensor cores (kernel b).
//
// Per coarse cell the GFT of Def. 1 / Alg. 2 is a dense complex contraction over pulses
// against the dechirp matrix D[m][f] (eq. H-DFM of the fine offsets) shared by every cell:
//   Y(n0; c, f) = e0(n0) * sum_m Zc[m][n0] D[m][f],   Zc[m][n0] = s[m][n0 + rho_c(m)] w_c(m)
// It runs as one real GEMM (the "4M" form) with K' = 2M and N' = 2F:
//   [Re Zc | Im Zc] (rows n0)  x  [[Re D, Im D], [-Im D, Re D]]  =  [Re Y~ | Im Y~]
// and each real operand x is split as hi = round16(x), lo = round16(x - hi) (BF16 or FP16),
// accumulating hi*hi + hi*lo + lo*hi in FP32 (three tcgen05.mma per K step).  The
// two-product FP16 mode (NP = 2) splits the gathered operand only and rounds the dechirp
// once: hi*hi + lo*hi, two tcgen05.mma per K step, no lo plane of the dechirp loaded.  The
// single-product FP16 mode (NP = 1) keeps only hi*hi: one tcgen05.mma per K step, no lo
// planes loaded or written.
//
// k_coarse_split (kernel a, the mGIFT of Alg. 1 in the time domain): one CTA per (cell,
//   128-bin tile), consecutive CTAs on the same bin tile of consecutive cells.  It gathers
//   every bin's samples at n0 + rho_c(m) from the L2-resident window of the echo (one
//   contiguous run of bins per pulse and warp), multiplies by the coarse phase
//   w_c(m), splits hi/lo, transposes through a warp-private shared tile and writes the
//   K-major operand Zs[cell][bin][k'] (two 16-bit planes) as whole 128-byte lines; the TMA
//   loads of kernel b apply the 128-byte swizzle.  Done once per (cell, bin) instead of once
//   per fine-hypothesis tile.
// k_ds_tc (kernel b): one persistent CTA per SM, 192 threads:
//   warp 0      TMA producer: Zs tile (A, 128 x 64) and dechirp tile (B, 256 x 64), hi and
//               lo planes, 128-byte swizzle, into a 2-stage ring (96 KB per stage)
//   warp 1      TMEM allocation (two 128 x 256 FP32 accumulators) and the single thread that
//               issues tcgen05.mma.cta_group::1.kind::f16 (M=128, N=256, K=16)
//   warps 2..5  epilogue: tcgen05.ld 32x32b (one TMEM lane = one range bin), |Y|^2 and
//               e0 * Y~, evict-first stores along r0
// The tiles of one (cell, bin tile) for consecutive fine-hypothesis tiles go to
// consecutive CTAs, so the A tile is read from HBM once and from L2 by the others.
// Every mbarrier wait is bounded: a wait that runs out latches GRFT_ETIMEOUT, the CTA
// unwinds (draining its TMA copies and MMAs with a bounded wait) and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.cuh"
#include "tma.cuh"

namespace grft {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;                      // real k per stage (32 pulses x re/im)
constexpr int TC_THREADS = 192;
constexpr uint64_t TC_DRAIN_LIMIT = 4000000000ull;   // bounded drain on the unwind path
// Tile-shape variants of kernel b (chosen per problem shape by the autotuner):
// BN real columns per tile (BN/2 fine hypotheses) and ST pipeline stages.
// ... and BK real k per stage: 64 (128-byte swizzle rows) or 32 (64-byte swizzle rows, so
// twice the stages fit the same shared memory).
// Planes (hi, lo) of the gathered operand A and of the dechirp operand B per product count.
constexpr int tc_planes_a(int NP) { return NP >= 2 ? 2 : 1; }
constexpr int tc_planes_b(int NP) { return NP == 3 ? 2 : 1; }
constexpr size_t tc_smem_bytes(int BN, int ST, int BK, int NP) {
    return (size_t)ST * (tc_planes_a(NP) * (size_t)TC_BM * BK * 2 + tc_planes_b(NP) * (size_t)BN * BK * 2) + 1024;
}

constexpr int SP_THREADS = 128;             // 4 warps x 32 range bins = one 128-bin tile
constexpr int SP_TAB_MAX = 2048;            // pulses whose bins and phases are staged in shared memory
constexpr int SP_TR_WORDS = (SP_THREADS / 32) * 2 * 32 * 8;   // uint4 words of the warp tiles (32 KB)

constexpr int TC_MAX_ITEMS = DS_TC_MAX_ITEMS;        // CPIs per launch (kernel-parameter table)
constexpr int TC_ROUNDS = 1;                         // rounds beyond what the buffer forces (1: none)
constexpr long TC_MIN_ROUND_ROWS = 65536;            // 512 bin tiles: several GEMM waves per round

// One CPI (or one call's cell range) inside a launch.
struct TcItem {
    const float2 *echo;     // [M][N], or nullptr when Z is given
    const float2 *Z;        // [cells][M][r0_count] (gathered and phased), or nullptr
    float *P;               // output planes (canonical v-slab layout), either may be null
    float2 *Y;
    const float2 *e0;       // e0[j] = range phase of bin r0_begin + j
    int M, N, KT;
    int r0_begin, r0_count, tiles_m, r0_pad;
    int cell0, ncell;       // absolute coarse cells [cell0, cell0 + ncell) of this launch
    int i0;                 // first coarse v row of the output slab
    long zrow0;             // first row of this item in the launch's split operand
    int cta0, tile0;        // first split CTA / first GEMM tile of this item
};

struct TcBatch {
    const int32_t *rho;     // coarse bins   [cell - tab_cell0][Mtab]
    const float2 *w;        // coarse phases [cell - tab_cell0][Mtab]
    int tab_cell0, Mtab;
    int zld;                // row length of the split operand (elements) = 2 * Mpad
    int n_items, total_ctas, total_tiles;
    int tiles_n, F, Fv, Fa, na_c;
    int Fb, nb_c;           // acceleration-rate axis (P = 3); 1, 1 for P = 2
    int fp16;
    int nprod;              // 3: hi*hi + hi*lo + lo*hi; 2: hi*hi + lo*hi; 1: hi*hi only
    int slots;              // pair form: slots of mirrored hypotheses (pair_slot); 0 in the 4M form
    uint32_t idesc;
    int *status;
    uint64_t wait_limit;
    TcItem it[TC_MAX_ITEMS];
};

// Item of a CTA / tile index: the last item whose prefix start is <= idx (items are few
// and the scan is uniform across the CTA).
__device__ __forceinline__ int find_item_cta(const TcBatch &b, int idx) {
    int i = 0;
    while (i + 1 < b.n_items && b.it[i + 1].cta0 <= idx) ++i;
    return i;
}
__device__ __forceinline__ int find_item_tile(const TcBatch &b, int idx) {
    int i = 0;
    while (i + 1 < b.n_items && b.it[i + 1].tile0 <= idx) ++i;
    return i;
}

// Coordinates of a work unit: one tile (item, cell, bin tile mt, hypothesis tile nt).
__device__ __forceinline__ const TcItem &decode_unit(const TcBatch &b, int unit, int &nt, int &mt, int &cl) {
    const TcItem &p = b.it[find_item_tile(b, unit)];
    const int local = unit - p.tile0;
    nt = local % b.tiles_n;
    const int rest = local / b.tiles_n;
    mt = rest % p.tiles_m;
    cl = rest / p.tiles_m;
    return p;
}

// ----------------------------------------------------------------------- tcgen05 wrappers
// Shared-memory matrix descriptor of a K-major tile whose rows are BK 16-bit values (BK = 64:
// 128-byte rows, 128-byte swizzle; BK = 32: 64-byte rows, 64-byte swizzle), 8-row groups
// packed back to back.
template <int BK>
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    static_assert(BK == 64 || BK == 32, "row of 128 or 64 bytes");
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused, K-major swizzled)
    d |= (uint64_t)((8 * BK * 2) >> 4) << 32;   // stride byte offset: 8 rows
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)(BK == 64 ? 2 : 4) << 61;    // 128-byte or 64-byte swizzle
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

// Named barrier among `count` threads (id 1; 0 is __syncthreads).
__device__ __forceinline__ void named_bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// A wait done by lane 0 of a warp, combined with the CTA abort flag and broadcast, so that
// the whole warp takes the same decision (keeps .sync.aligned operations converged).
// Returns false if the wait ran out or the CTA is unwinding; lane 0 then latches the error.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, uint64_t limit,
                                          volatile int *abort_flag, int *status, unsigned sleep_ns) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        ok = (!*abort_flag && mbar_wait_backoff(bar, parity, limit, sleep_ns)) ? 1 : 0;
        if (!ok) {
            latch_error(status, GRFT_ETIMEOUT);
            *abort_flag = 1;
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    return ok != 0;
}

// =========================================================================== kernel a
// L2 policies of kernel a: the split operand streams through L2 (evict first) so that the
// echo rows every cell gathers from stay resident (evict last).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void st_global_v4_hint(uint16_t *dst, uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                                  uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(dst), "r"(a), "r"(b), "r"(c),
                 "r"(d), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ float2 ld_global_nc_hint(const float2 *src, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(src), "l"(pol));
    return v;
}

__global__ void __launch_bounds__(SP_THREADS, 4) k_coarse_split(const __grid_constant__ TcBatch B,
                                                             const __grid_constant__ CUtensorMap mapZhi,
                                                             const __grid_constant__ CUtensorMap mapZlo,
                                                             int tab_cap) {
    // One CTA per (item, cell, 128-bin tile), four warps; warp w owns the 32 bins 32w + lane of
    // the tile and every pulse, taken in sub-steps of 8 pulses.  A lane's gathers for one pulse
    // are consecutive bins of the echo row (the warp reads one 256-byte run per pulse).  The
    // converted values pass through a warp-private shared tile [plane][32 rows][8 chunks of
    // 16 bytes] (chunk index XOR row % 8: conflict-free on both sides) and leave, once the four
    // sub-steps of a 32-pulse stage are in, as whole 128-byte lines of the K-major operand rows
    // (k' = (m/32)*64 + (re|im)*32 + m%32), written by one tensor-map store per plane and
    // stage (the tile's chunk XOR row % 8 order is the copy's 128-byte swizzle).  The cell's
    // bins and phases are staged in shared memory; the next sub-step's samples are requested
    // before the current one is converted.
    extern __shared__ uint4 sp_smem[];          // [warps][2 planes][32][8] (1024-byte aligned), then w[tab_cap], rho[tab_cap]
    __shared__ int s_rng[2];                    // least and greatest bin shift of the cell
    uint4 *const tiles = reinterpret_cast<uint4 *>((reinterpret_cast<uintptr_t>(sp_smem) + 1023) & ~(uintptr_t)1023);
    float2 *s_w = reinterpret_cast<float2 *>(tiles + SP_TR_WORDS);
    int *s_rho = reinterpret_cast<int *>(s_w + tab_cap);
    const TcItem &p = B.it[find_item_cta(B, blockIdx.x)];
    const int local = blockIdx.x - p.cta0;
    // consecutive CTAs take the same bin tile of consecutive cells: the CTAs in flight gather
    // from one window of the echo (the tile's bins plus the cells' shifts), which stays in L2
    // even where the whole echo does not
    const int cl = local % p.ncell;
    const int mt = local / p.ncell;
    const int c = p.cell0 + cl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool fp16 = B.fp16 != 0;
    const int j0 = mt * TC_BM;
    const int j = j0 + warp * 32 + lane;
    const bool jok = j < p.r0_count;
    const long tab = (long)(c - B.tab_cell0) * B.Mtab;
    const long ztab = (long)(c - B.tab_cell0) * p.M;     // cell offset inside Z (M pulses per cell)
    const int nbase = p.r0_begin + j;
    const bool tab_smem = !p.Z && p.M <= tab_cap;
    if (tab_smem) {
        if (tid == 0) {
            s_rng[0] = 0x7fffffff;
            s_rng[1] = -0x7fffffff - 1;
        }
        __syncthreads();
        int lo = 0x7fffffff, hi = -0x7fffffff - 1;
        for (int m = tid; m < p.M; m += SP_THREADS) {
            const int rr = __ldg(B.rho + tab + m);
            s_rho[m] = rr;
            s_w[m] = __ldg(B.w + tab + m);
            lo = min(lo, rr);
            hi = max(hi, rr);
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (lane == 0) {
            atomicMin(&s_rng[0], lo);
            atomicMax(&s_rng[1], hi);
        }
        __syncthreads();
    }
    const int *rho_t = tab_smem ? s_rho : B.rho + tab;
    const float2 *w_t = tab_smem ? s_w : B.w + tab;
    uint4 *tr = tiles + warp * 512;              // this warp's tile: hi plane, then lo plane
    const size_t row0 = (size_t)p.zrow0 + (size_t)cl * p.r0_pad + j0 + warp * 32;
    const uint64_t pol_z = l2_policy_evict_first();
    const bool with_lo = B.nprod >= 2;          // block-uniform
    const int S = 4 * p.KT;                     // sub-steps of 8 pulses (even)

    // Convert sub-step s (pulses 8s..8s+7 of this lane's bin; phase already applied), place
    // it in the warp tile, and after the fourth sub-step of a stage write the stage's lines.
    auto put = [&](int s, const float (&re)[8], const float (&im)[8]) {
        const int g = s & 3, kt = s >> 2, sw = lane & 7;
        uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            split2(re[2 * q], re[2 * q + 1], fp16, rh[q], rl[q]);
            split2(im[2 * q], im[2 * q + 1], fp16, ih[q], il[q]);
        }
        if (g == 0) {                            // the previous stage's copies have read the tile
            if (lane == 0) bulk_wait_read<0>();
            __syncwarp();
        }
        tr[lane * 8 + (g ^ sw)] = make_uint4(rh[0], rh[1], rh[2], rh[3]);
        tr[lane * 8 + ((4 + g) ^ sw)] = make_uint4(ih[0], ih[1], ih[2], ih[3]);
        if (with_lo) {
            tr[256 + lane * 8 + (g ^ sw)] = make_uint4(rl[0], rl[1], rl[2], rl[3]);
            tr[256 + lane * 8 + ((4 + g) ^ sw)] = make_uint4(il[0], il[1], il[2], il[3]);
        }
        if (g == 3) {
            // the stage's 32 rows x 128 bytes per plane, one tensor-map store each
            fence_proxy_async_shared();
            __syncwarp();
            if (lane == 0) {
                tma_store_2d_hint(&mapZhi, tr, kt * TC_BK, (int)row0, pol_z);
                if (with_lo) tma_store_2d_hint(&mapZlo, tr + 256, kt * TC_BK, (int)row0, pol_z);
                bulk_commit();
            }
        }
    };
    // every copy has completed before the CTA's shared memory goes
    auto finish = [&]() {
        if (lane == 0) bulk_wait<0>();
        __syncwarp();
    };

    // Fast path (block-uniform): the tables are staged, every bin of the tile is inside the
    // r0 range and every gathered bin is inside the echo, so the loop over the whole sub-steps
    // of 8 pulses carries no bound checks; the sub-steps past the last whole one (a pulse
    // count that is not a multiple of 32) follow with the pulse check, writing zeros past the
    // last pulse as the operand's K padding must hold.
    if (tab_smem && j0 + TC_BM <= p.r0_count && p.r0_begin + j0 + s_rng[0] >= 0 &&
        p.r0_begin + j0 + TC_BM - 1 + s_rng[1] < p.N) {
        const float2 *src = p.echo + nbase;
        const long N = p.N;
        const uint64_t pol_e = l2_policy_evict_last();
        auto ld = [&](int s, float2 (&v)[8]) {
            const int m0 = s * 8;
            const float2 *rowp = src + (long)m0 * N;
#pragma unroll
            for (int i = 0; i < 8; ++i, rowp += N) v[i] = ld_global_nc_hint(rowp + s_rho[m0 + i], pol_e);
        };
        auto cv = [&](int s, const float2 (&v)[8]) {
            const int m0 = s * 8;
            float re[8], im[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 x = cmul(v[i], s_w[m0 + i]);
                re[i] = x.x;
                im[i] = x.y;
            }
            put(s, re, im);
        };
        float2 va[8], vb[8];
        if (p.M == 32 * p.KT) {                 // whole 32-pulse groups: every sub-step is whole
            float2 vc[8], vd[8];
            ld(0, va);
            ld(1, vb);
            for (int s = 0; s < S; s += 4) {    // four buffers, two sub-steps ahead (S % 4 == 0)
                ld(s + 2, vc);
                ld(s + 3, vd);
                cv(s, va);
                cv(s + 1, vb);
                if (s + 4 < S) {
                    ld(s + 4, va);
                    ld(s + 5, vb);
                }
                cv(s + 2, vc);
                cv(s + 3, vd);
            }
            finish();
            return;
        }
        const int Sw = p.M / 8;                 // whole sub-steps
        if (Sw > 0) ld(0, va);
        int s = 0;
        for (; s + 1 < Sw; s += 2) {            // the two buffers alternate
            ld(s + 1, vb);
            cv(s, va);
            if (s + 2 < Sw) ld(s + 2, va);
            cv(s + 1, vb);
        }
        if (s < Sw) cv(s++, va);                // an odd count: the last whole one is in va
        for (; s < S; ++s) {                    // at most four: the partial one, then zeros
            const int m0 = s * 8;
            const float2 *rowp = src + (long)m0 * N;
            float re[8], im[8];
#pragma unroll
            for (int i = 0; i < 8; ++i, rowp += N) {
                float2 x = make_float2(0.f, 0.f);
                if (m0 + i < p.M) x = cmul(ld_global_nc_hint(rowp + s_rho[m0 + i], pol_e), s_w[m0 + i]);
                re[i] = x.x;
                im[i] = x.y;
            }
            put(s, re, im);
        }
        finish();
        return;
    }

    // General path (edge tiles, materialised Z, partial pulse groups, tables in global memory)
    auto load8 = [&](int s, float2 (&v)[8]) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = s * 8 + i;
            float2 x = make_float2(0.f, 0.f);
            if (m < p.M && jok) {
                if (p.Z) {
                    x = __ldg(p.Z + (ztab + m) * p.r0_count + j);
                } else {
                    const int n = nbase + rho_t[m];
                    if ((unsigned)n < (unsigned)p.N) x = __ldg(p.echo + (long)m * p.N + n);
                }
            }
            v[i] = x;
        }
    };
    auto cv8 = [&](int s, const float2 (&v)[8]) {
        float re[8], im[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = s * 8 + i;
            float2 x = v[i];
            if (!p.Z && m < p.M) x = cmul(x, w_t[m]);
            re[i] = x.x;
            im[i] = x.y;
        }
        put(s, re, im);
    };
    float2 va[8], vb[8];
    load8(0, va);
    for (int s = 0; s < S; s += 2) {
        load8(s + 1, vb);
        cv8(s, va);
        if (s + 2 < S) load8(s + 2, va);
        cv8(s + 1, vb);
    }
    finish();
}

// =========================================================================== kernel b
template <int BN, int ST, int BK, int NP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_ds_tc(const __grid_constant__ CUtensorMap mapAhi, const __grid_constant__ CUtensorMap mapAlo,
            const __grid_constant__ CUtensorMap mapBhi, const __grid_constant__ CUtensorMap mapBlo,
            const __grid_constant__ TcBatch B) {
    constexpr int TC_BN = BN;                          // real columns per tile
    constexpr int TC_STAGES = ST;
    constexpr uint32_t TC_A_BYTES = TC_BM * BK * 2;    // per plane
    constexpr uint32_t TC_B_BYTES = BN * BK * 2;       // per plane
    constexpr uint32_t TC_STAGE_BYTES = tc_planes_a(NP) * TC_A_BYTES + tc_planes_b(NP) * TC_B_BYTES;
    constexpr uint32_t TC_B_OFF = tc_planes_a(NP) * TC_A_BYTES;   // B planes follow the A planes
    constexpr int KSUB = 64 / BK;                      // stages per 32-pulse group
    constexpr uint32_t TC_TMEM_COLS = 2 * BN;          // two accumulators
    static_assert(BN % 32 == 0 && BN <= 256 && TC_TMEM_COLS >= 32, "tile");
    static_assert(NP >= 1 && NP <= 3, "three, two or one products per K step");
    extern __shared__ unsigned char smem_raw[];
    __shared__ alignas(8) uint64_t full[TC_STAGES], empty[TC_STAGES];
    __shared__ alignas(8) uint64_t tmem_full[2], tmem_empty[2], drain_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_flag;
    __shared__ long s_rowoff[128];

    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int cid = (int)blockIdx.x, ncl = (int)gridDim.x;

    if (threadIdx.x == 0) {
        tma_prefetch_desc(&mapAhi);
        tma_prefetch_desc(&mapAlo);
        tma_prefetch_desc(&mapBhi);
        tma_prefetch_desc(&mapBlo);
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
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
    const uint64_t lim = B.wait_limit;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer (A and B)
        if (lane == 0) {
            int it = 0;
            int last_it = -1;
            for (int tile = cid; tile < B.total_tiles && !abort_flag; tile += ncl) {
                int nt, mt, cl;
                const TcItem &p = decode_unit(B, tile, nt, mt, cl);
                const int arow = (int)(p.zrow0 + (long)cl * p.r0_pad + mt * TC_BM);
                for (int kt = 0; kt < p.KT * KSUB; ++kt, ++it) {
                    const int s = it % TC_STAGES;
                    if (!mbar_wait_backoff(&empty[s], ((it / TC_STAGES) & 1) ^ 1, lim, 32)) {
                        latch_error(B.status, GRFT_ETIMEOUT);
                        abort_flag = 1;
                        break;
                    }
                    unsigned char *st = smem + s * TC_STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[s], TC_STAGE_BYTES);
                    tma_load_2d(st, &mapAhi, kt * BK, arow, &full[s]);
                    if (NP >= 2) tma_load_2d(st + TC_A_BYTES, &mapAlo, kt * BK, arow, &full[s]);
                    tma_load_2d(st + TC_B_OFF, &mapBhi, kt * BK, nt * TC_BN, &full[s]);
                    if (NP == 3) tma_load_2d(st + TC_B_OFF + TC_B_BYTES, &mapBlo, kt * BK, nt * TC_BN, &full[s]);
                    last_it = it;
                }
            }
            // drain: every issued load has landed before shared memory can be released (the
            // last use of each stage is last_it and, if issued, last_it - 1)
            for (int u = last_it; u >= 0 && u >= last_it - (TC_STAGES - 1); --u)
                mbar_wait(&full[u % TC_STAGES], (u / TC_STAGES) & 1, TC_DRAIN_LIMIT);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int it = 0, tcount = 0;
            bool issued_any = false;
            for (int tile = cid; tile < B.total_tiles && !abort_flag; tile += ncl, ++tcount) {
                const int b = tcount & 1;
                const int KT = B.it[find_item_tile(B, tile)].KT * KSUB;
                if (!mbar_wait(&tmem_empty[b], ((tcount >> 1) & 1) ^ 1, lim)) {
                    latch_error(B.status, GRFT_ETIMEOUT);
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(b * TC_BN);
                bool ok = true;
                for (int kt = 0; kt < KT; ++kt, ++it) {
                    const int s = it % TC_STAGES;
                    if (!mbar_wait(&full[s], (it / TC_STAGES) & 1, lim)) {
                        latch_error(B.status, GRFT_ETIMEOUT);
                        abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * TC_STAGE_BYTES;
                    const uint32_t a_hi = st, a_lo = st + TC_A_BYTES;
                    const uint32_t b_hi = st + TC_B_OFF, b_lo = b_hi + TC_B_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t off = kk * 32;   // 16 elements x 2 bytes inside the swizzle row
                        umma_f16(d_tmem, umma_desc<BK>(a_hi + off), umma_desc<BK>(b_hi + off), B.idesc,
                                 (kt > 0 || kk > 0) ? 1u : 0u);
                        if (NP == 3)
                            umma_f16(d_tmem, umma_desc<BK>(a_hi + off), umma_desc<BK>(b_lo + off), B.idesc, 1u);
                        if (NP >= 2)
                            umma_f16(d_tmem, umma_desc<BK>(a_lo + off), umma_desc<BK>(b_hi + off), B.idesc, 1u);
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
    } else {
        // ------------------------------------------------------------ epilogue
        // Thread (warp q4, lane) owns TMEM lane r = 32 q4 + lane = tile row (range bin).
        // Per tile the 128 output row offsets (one per fine hypothesis of the tile) go to a
        // shared table; stores are evict-first so that the 4 GB output does not push the
        // operands out of L2.  Every epilogue warp runs every tile iteration (also after an
        // abort) so that the named barrier always sees all 128 threads.
        const int q4 = warp & 3;
        const int r = q4 * 32 + lane;
        const int er = threadIdx.x - 64;         // 0..127 over the epilogue warps
        const int na_full = B.na_c * B.Fa;
        const int nb_full = B.nb_c * B.Fb;
        bool aborted = false;
        int tcount = 0;
        for (int tile = cid; tile < B.total_tiles; tile += ncl, ++tcount) {
            const int b = tcount & 1;
            int nt, mt, cl;
            const TcItem &p = decode_unit(B, tile, nt, mt, cl);
            const int c = p.cell0 + cl;
            const int iw = c % B.nb_c, c2 = c / B.nb_c;      // P = 3: c = (i na_c + l) nb_c + w
            const int iv = c2 / B.na_c - p.i0, il = c2 % B.na_c;
            named_bar_sync(1, 128);                  // previous tile's offsets no longer read
            if (!aborted) {
                const int f = nt * (TC_BN / 2) + er;
                long off = -1;
                if (f < B.F) {                       // f = (k Fa + q) Fb + u
                    const int u = f % B.Fb, f2 = f / B.Fb;
                    const int k = f2 / B.Fa, q = f2 % B.Fa;
                    off = (((long)(iv * B.Fv + k) * na_full + (il * B.Fa + q)) * nb_full + (iw * B.Fb + u)) *
                          p.r0_count;
                }
                s_rowoff[er] = off;
            }
            named_bar_sync(1, 128);
            if (aborted) continue;
            if (!warp_wait(&tmem_full[b], (tcount >> 1) & 1, lim, &abort_flag, B.status, 256)) {
                aborted = true;
                continue;
            }
            tc_fence_after();
            const int j = mt * TC_BM + r;
            const bool jok = j < p.r0_count;
            float *const P = p.P;
            float2 *const Y = p.Y;
            const float2 e = (jok && Y) ? p.e0[j] : make_float2(1.f, 0.f);
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
                            if (P) __stcs(P + ro + j, yr * yr + yi * yi);
                            if (Y) __stcs(Y + ro + j, make_float2(e.x * yr - e.y * yi, e.x * yi + e.y * yr));
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

// =========================================================================== kernel b, pair form
// The contraction in the pair form (see pair_slot): tile = 64 range bins x 128 slots.  The A
// tile interleaves each bin's real and imaginary parts (row 2 b: Re Z of bin b, row 2 b + 1:
// Im Z): per stage of 64 pulses two sub-tiles of 32 pulses (64-byte rows, 64-byte swizzle),
// each one box of the split operand through a 3-D tensor map (x: the 32 pulses of one part,
// y: 2 g + part, both parts, z: the operand row = bin).  The B tile holds Re D and Im D of the
// slots' hypotheses (rows 2 s, 2 s + 1) over the stage's 64 pulses (128-byte rows).  One
// tcgen05.mma (M=128, N=256, K=16) per product and 16 pulses leaves, per bin and slot,
// A = Zr Dr and C = Zr Di in TMEM lane 2 b and E = Zi Dr, B = Zi Di in lane 2 b + 1; the
// epilogue swaps half of them between the two lanes by a shuffle and writes Y (and |Y|^2)
// of each slot's hypothesis and its mirror: a complex MAC of a mirrored pair costs two real
// MACs of one hypothesis in the 4M form.
constexpr int PR_BINS = 64;                               // range bins per tile
constexpr int PR_BK = 64;                                 // pulses per stage (128-byte rows, 128-byte swizzle)
// B rows per tile BN (BN / 2 slots): 256, 224 or 192, whichever pads the slot count least
// (pair_bn); the MMA's N and the tensor work of a tile scale with it.
constexpr uint32_t PR_A_BYTES = 2 * PR_BINS * PR_BK * 2;  // per plane (128 rows: re, im of 64 bins): 16 KB
constexpr uint32_t pr_b_bytes(int BN) { return (uint32_t)BN * PR_BK * 2; }   // per plane: BN rows of 128 bytes
constexpr size_t pr_stage_bytes(int NP, int BN) {
    return (size_t)tc_planes_a(NP) * PR_A_BYTES + (size_t)tc_planes_b(NP) * pr_b_bytes(BN);
}
constexpr size_t pr_smem_bytes(int ST, int NP, int BN) { return (size_t)ST * pr_stage_bytes(NP, BN) + 1024; }

__device__ __forceinline__ const TcItem &decode_pair_unit(const TcBatch &b, int unit, int &nt, int &mt, int &cl) {
    const TcItem &p = b.it[find_item_tile(b, unit)];
    const int local = unit - p.tile0;
    const int tm = (p.r0_count + PR_BINS - 1) / PR_BINS;
    nt = local % b.tiles_n;
    const int rest = local / b.tiles_n;
    mt = rest % tm;
    cl = rest / tm;
    return p;
}

// Output row offset (canonical layout, bin 0) of fine hypothesis f = (k Fa + q) Fb + u of
// cell c, or -1.
__device__ __forceinline__ long pair_row_offset(const TcBatch &B, const TcItem &p, int c, int f) {
    if (f < 0) return -1;
    const int iw = c % B.nb_c, c2 = c / B.nb_c;
    const int iv = c2 / B.na_c - p.i0, il = c2 % B.na_c;
    const int u = f % B.Fb, kq = f / B.Fb;
    const int k = kq / B.Fa, q = kq % B.Fa;
    const long na_full = (long)B.na_c * B.Fa, nb_full = (long)B.nb_c * B.Fb;
    return (((long)(iv * B.Fv + k) * na_full + (il * B.Fa + q)) * nb_full + (long)iw * B.Fb + u) * p.r0_count;
}

constexpr int PR_EPI_WARPS = 12;                          // three per TMEM lane quarter (ds_m512: 8 -> 3.21 ms, 12 -> 3.12, 16 -> 3.14)
constexpr int PR_EPI_PER_Q = PR_EPI_WARPS / 4;            // warps sharing one lane quarter
constexpr int PR_THREADS = 64 + 32 * PR_EPI_WARPS;        // producer, MMA issuer, epilogue
static_assert(PR_EPI_WARPS % 4 == 0 && PR_EPI_WARPS <= 16, "whole lane quarters");

template <int ST, int NP, int BN>
__global__ void __launch_bounds__(PR_THREADS, 1)
    k_ds_pair(const __grid_constant__ CUtensorMap mapAhi, const __grid_constant__ CUtensorMap mapAlo,
              const __grid_constant__ CUtensorMap mapBhi, const __grid_constant__ CUtensorMap mapBlo,
              const __grid_constant__ TcBatch B) {
    constexpr uint32_t STAGE = (uint32_t)pr_stage_bytes(NP, BN);
    constexpr uint32_t B_OFF = tc_planes_a(NP) * PR_A_BYTES;
    constexpr uint32_t PR_B_BYTES = pr_b_bytes(BN);
    constexpr uint32_t TMEM_COLS = 512;                    // two accumulators of BN columns (a power of 2)
    constexpr int SL = BN / 2;                             // slots per tile
    constexpr int NCH = BN / 32;                           // 32-column chunks per tile
    static_assert(NP >= 1 && NP <= 3, "three, two or one products per K step");
    static_assert(BN % 32 == 0 && BN >= 128 && BN <= 256 && STAGE % 1024 == 0, "pair tile");
    extern __shared__ unsigned char smem_raw[];
    __shared__ alignas(8) uint64_t full[ST], empty[ST];
    __shared__ alignas(8) uint64_t tmem_full[2], tmem_empty[2], drain_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_flag;
    __shared__ volatile int s_fail;                        // an epilogue wait gave up (epilogue-uniform)
    __shared__ long s_off_f[128], s_off_m[128];            // output rows of each slot's pair

    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int cid = (int)blockIdx.x, ncl = (int)gridDim.x;

    if (threadIdx.x == 0) {
        tma_prefetch_desc(&mapAhi);
        tma_prefetch_desc(&mapAlo);
        tma_prefetch_desc(&mapBhi);
        tma_prefetch_desc(&mapBlo);
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tmem_full[b], 1);
            mbar_init(&tmem_empty[b], 32 * PR_EPI_WARPS);
        }
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        s_fail = 0;
        fence_mbarrier_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_holder;
    const uint64_t lim = B.wait_limit;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int it = 0, last_it = -1;
            for (int tile = cid; tile < B.total_tiles && !abort_flag; tile += ncl) {
                int nt, mt, cl;
                const TcItem &p = decode_pair_unit(B, tile, nt, mt, cl);
                const int arow = (int)(p.zrow0 + (long)cl * p.r0_pad + mt * PR_BINS);
                for (int kt = 0; kt < (p.KT + 1) / 2; ++kt, ++it) {     // 64-pulse stages
                    const int s = it % ST;
                    if (!mbar_wait_backoff(&empty[s], ((it / ST) & 1) ^ 1, lim, 32)) {
                        latch_error(B.status, GRFT_ETIMEOUT);
                        abort_flag = 1;
                        break;
                    }
                    unsigned char *st = smem + s * STAGE;
                    // the second 32-pulse group of the stage exists unless the pulse count ends
                    // in the first (then its A sub-tile is neither loaded nor used)
                    const bool has1 = 2 * kt + 1 < p.KT;
                    mbar_arrive_expect_tx(&full[s], STAGE - (has1 ? 0u : tc_planes_a(NP) * (PR_A_BYTES / 2)));
                    tma_load_3d(st, &mapAhi, 0, 4 * kt, arow, &full[s]);              // Re, Im Z, group 2 kt
                    if (has1) tma_load_3d(st + PR_A_BYTES / 2, &mapAhi, 0, 4 * kt + 2, arow, &full[s]);
                    if (NP >= 2) {
                        tma_load_3d(st + PR_A_BYTES, &mapAlo, 0, 4 * kt, arow, &full[s]);
                        if (has1) tma_load_3d(st + PR_A_BYTES + PR_A_BYTES / 2, &mapAlo, 0, 4 * kt + 2, arow, &full[s]);
                    }
                    tma_load_2d(st + B_OFF, &mapBhi, kt * PR_BK, nt * BN, &full[s]);
                    if (NP == 3) tma_load_2d(st + B_OFF + PR_B_BYTES, &mapBlo, kt * PR_BK, nt * BN, &full[s]);
                    last_it = it;
                }
            }
            for (int u = last_it; u >= 0 && u >= last_it - (ST - 1); --u)
                mbar_wait(&full[u % ST], (u / ST) & 1, TC_DRAIN_LIMIT);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int it = 0, tcount = 0;
            bool issued_any = false;
            for (int tile = cid; tile < B.total_tiles && !abort_flag; tile += ncl, ++tcount) {
                const int b = tcount & 1;
                const int KG = B.it[find_item_tile(B, tile)].KT;             // 32-pulse groups
                const int KT = (KG + 1) / 2;                                // 64-pulse stages
                if (!mbar_wait(&tmem_empty[b], ((tcount >> 1) & 1) ^ 1, lim)) {
                    latch_error(B.status, GRFT_ETIMEOUT);
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
                bool ok = true;
                for (int kt = 0; kt < KT; ++kt, ++it) {
                    const int s = it % ST;
                    if (!mbar_wait(&full[s], (it / ST) & 1, lim)) {
                        latch_error(B.status, GRFT_ETIMEOUT);
                        abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + s * STAGE;
                    const uint32_t a_hi = st, a_lo = st + PR_A_BYTES;
                    const uint32_t b_hi = st + B_OFF, b_lo = b_hi + PR_B_BYTES;
                    const int nkk = 2 * kt + 1 < KG ? 4 : 2;   // K steps of 16 pulses in the stage
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        if (kk >= nkk) break;
                        // A: sub-tile kk / 2 (64-byte rows), 16 pulses at (kk % 2) x 32 bytes;
                        // B: 16 pulses at kk x 32 bytes of the 128-byte row
                        const uint32_t ao = (kk >> 1) * (PR_A_BYTES / 2) + (kk & 1) * 32, bo = kk * 32;
                        umma_f16(d_tmem, umma_desc<32>(a_hi + ao), umma_desc<64>(b_hi + bo), B.idesc,
                                 (kt > 0 || kk > 0) ? 1u : 0u);
                        if (NP == 3)
                            umma_f16(d_tmem, umma_desc<32>(a_hi + ao), umma_desc<64>(b_lo + bo), B.idesc, 1u);
                        if (NP >= 2)
                            umma_f16(d_tmem, umma_desc<32>(a_lo + ao), umma_desc<64>(b_hi + bo), B.idesc, 1u);
                    }
                    issued_any = true;
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&tmem_full[b]);
            }
            if (issued_any) {
                umma_commit(&drain_bar);
                mbar_wait(&drain_bar, 0, TC_DRAIN_LIMIT);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // PR_EPI_WARPS warps, PR_EPI_PER_Q per TMEM lane quarter (warp w reads lanes 32 (w mod
        // 4) .. + 31), warp part p of the quarter the tile's 32-column chunks [ceil(p NCH /
        // PR_EPI_PER_Q), ceil((p + 1) NCH / PR_EPI_PER_Q)).  Thread (warp,
        // lane) owns TMEM lane r = 32 q4 + lane: the real part (even lane) or the imaginary
        // part (odd lane) of bin r / 2.  Per 32-column chunk (16 slots) the even lane keeps
        // slots 0-7 and hands its columns of slots 8-15 to the odd lane, which keeps 8-15 and
        // hands its columns of 0-7 back (one shuffle per value).  With X the lane's own pair
        // of a slot and W the received one, the even lane holds (A, C) = X, (E, B) = W and the
        // odd lane the reverse, so
        //   U = (X0 - W1)^2 + (X1 + W0)^2,  V = (X0 + W1)^2 + (X1 - W0)^2
        // are |Y(f)|^2, |Y(f')|^2 on the even lane and |Y(f')|^2, |Y(f)|^2 on the odd lane.  The
        // named barriers run once per tile and are reached by every epilogue thread: a wait
        // that gives up is made known through s_fail before the barrier after it.
        constexpr int NT = 32 * PR_EPI_WARPS;
        const int q4 = warp & 3;
        const int part = (warp - 2) >> 2;         // 0 .. PR_EPI_PER_Q - 1
        const int ch0 = (part * NCH + PR_EPI_PER_Q - 1) / PR_EPI_PER_Q;
        const int ch1 = ((part + 1) * NCH + PR_EPI_PER_Q - 1) / PR_EPI_PER_Q;
        const int r = q4 * 32 + lane;
        const bool odd = (lane & 1) != 0;
        const int er = threadIdx.x - 64;          // 0..NT-1 over the epilogue warps
        bool aborted = false;
        int tcount = 0;
        for (int tile = cid; tile < B.total_tiles; tile += ncl, ++tcount) {
            const int b = tcount & 1;
            int nt, mt, cl;
            const TcItem &p = decode_pair_unit(B, tile, nt, mt, cl);
            const int c = p.cell0 + cl;
            named_bar_sync(1, NT);                // the previous tile's offsets are read
            if (!aborted && er < 2 * SL) {        // thread er: slot er mod SL, hypothesis or mirror
                const int sl = er < SL ? er : er - SL;
                const int slot = nt * SL + sl;
                int f = -1, fm = -1;
                if (slot < B.slots) pair_slot3(slot, B.Fv, B.Fa, B.Fb, f, fm);
                if (er < SL)
                    s_off_f[sl] = pair_row_offset(B, p, c, f);
                else
                    s_off_m[sl] = pair_row_offset(B, p, c, fm);
            }
            named_bar_sync(1, NT);
            if (aborted) continue;
            if (!warp_wait(&tmem_full[b], (tcount >> 1) & 1, lim, &abort_flag, B.status, 256) && lane == 0)
                s_fail = 1;
            named_bar_sync(1, NT);
            if (s_fail) {                          // every epilogue warp stops here
                aborted = true;
                continue;
            }
            tc_fence_after();
            const int j = mt * PR_BINS + (r >> 1);
            const bool jok = j < p.r0_count;
            float *const P = p.P;
            float2 *const Y = p.Y;
            const float2 e = (jok && Y) ? p.e0[j] : make_float2(1.f, 0.f);
            // P only, rows of an even bin count, P 8-byte aligned: bin pairs (warp-uniform)
            const bool p2 = P && !Y && (p.r0_count & 1) == 0 && (((uintptr_t)P) & 7) == 0;
            const bool ob = (lane & 2) != 0;      // this lane's bin r / 2 is odd
            const uint32_t taddr0 = tmem_base + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * BN);
#pragma unroll 1
            for (int ch = ch0; ch < ch1; ++ch) {
                uint32_t v[32];
                __syncwarp();
                tmem_ld32(taddr0 + ch * 32, v);
                // own columns: 0-15 (even lane) or 16-31 (odd lane); the other half is swapped
                float X[16], W[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float lo = __uint_as_float(v[i]), hi = __uint_as_float(v[16 + i]);
                    X[i] = odd ? hi : lo;
                    W[i] = __shfl_xor_sync(0xffffffffu, odd ? lo : hi, 1);
                }
                if (p2) {
                    // lanes L and L ^ 2 hold bins b and b ^ 1 (b = r / 2) of the same two rows:
                    // the lane of the even bin writes the U row's two bins, the other the V
                    // row's (one shuffle, one 8-byte store per lane and slot)
#pragma unroll
                    for (int pp = 0; pp < 8; ++pp) {
                        const int sl = ch * 16 + (odd ? 8 + pp : pp);
                        const float x0 = X[2 * pp], x1 = X[2 * pp + 1], w0 = W[2 * pp], w1 = W[2 * pp + 1];
                        const long of = s_off_f[sl], om = s_off_m[sl];
                        const long ou = odd ? om : of, ov = odd ? of : om;
                        const float ur = x0 - w1, ui = x1 + w0, vr = x0 + w1, vi = x1 - w0;
                        const float U = ur * ur + ui * ui, V = vr * vr + vi * vi;
                        const float recv = __shfl_xor_sync(0xffffffffu, ob ? U : V, 2);
                        const long row = ob ? ov : ou;
                        if (jok && row >= 0)
                            __stcs(reinterpret_cast<float2 *>(P + row + (ob ? j - 1 : j)),
                                   ob ? make_float2(recv, V) : make_float2(U, recv));
                    }
                } else if (jok) {
#pragma unroll
                    for (int pp = 0; pp < 8; ++pp) {
                        const int sl = ch * 16 + (odd ? 8 + pp : pp);
                        const float x0 = X[2 * pp], x1 = X[2 * pp + 1], w0 = W[2 * pp], w1 = W[2 * pp + 1];
                        const long of = s_off_f[sl], om = s_off_m[sl];
                        const long ou = odd ? om : of, ov = odd ? of : om;   // rows of U and V
                        if (P) {
                            const float ur = x0 - w1, ui = x1 + w0, vr = x0 + w1, vi = x1 - w0;
                            if (ou >= 0) __stcs(P + ou + j, ur * ur + ui * ui);
                            if (ov >= 0) __stcs(P + ov + j, vr * vr + vi * vi);
                        }
                        if (Y) {                   // Y(f) and Y(f') from (A, B, C, E)
                            const float A = odd ? w0 : x0, Cc = odd ? w1 : x1;
                            const float E = odd ? x0 : w0, Bb = odd ? x1 : w1;
                            if (of >= 0) {
                                const float yr = A - Bb, yi = Cc + E;
                                __stcs(Y + of + j, make_float2(e.x * yr - e.y * yi, e.x * yi + e.y * yr));
                            }
                            if (om >= 0) {
                                const float yr = A + Bb, yi = E - Cc;
                                __stcs(Y + om + j, make_float2(e.x * yr - e.y * yi, e.x * yi + e.y * yr));
                            }
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

bool set_smem_attr(const void *fn, size_t bytes, int device, bool *done) {
    if (device < 64 && done[device]) return true;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return false;
    if (device < 64) done[device] = true;
    return true;
}

}  // namespace

int ds_tc_r0_pad(int r0_count) { return (r0_count + TC_BM - 1) / TC_BM * TC_BM; }

namespace {

// ------------------------------------------------------------------------ autotuner
// Tile-shape choice per problem bucket (Mpad, Fpad, largest r0 tile count rounded up to a
// power of two, FP16 or BF16): the first uncaptured call of a bucket times every variant
// of kernel b on its first round (the split operand is already in place and kernel b is
// idempotent, so the timed reruns change nothing) and keeps the fastest.  The choice is
// cached per process and, if DSGRFT_TUNE_CACHE names a file, appended to it as JSON lines
// {"Mpad":..,"Fpad":..,"r0":..,"fp16":..,"variant":..} that later processes read back.
// DSGRFT_AUTOTUNE=0 disables timing (the default variant is used); DSGRFT_TILE_VARIANT=v
// forces variant v.  Variants give
// bit-identical results: only the N tiling changes, not the order of the K accumulation.
constexpr int TC_VARIANTS = 3;     // (BN, stages, BK): see launch_gemm_variant
using TuneKey = std::tuple<int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
bool g_tune_loaded = false;

const char *tune_path() {
    const char *p = getenv("DSGRFT_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}
bool tune_enabled() {
    const char *p = getenv("DSGRFT_AUTOTUNE");
    return !(p && p[0] == '0');
}
int json_int(const char *line, const char *key) {
    const char *q = strstr(line, key);
    return q ? atoi(q + strlen(key)) : -1;
}
void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = tune_path();
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        const int a = json_int(line, "\"Mpad\":"), b = json_int(line, "\"Fpad\":");
        const int r = json_int(line, "\"r0\":"), h = json_int(line, "\"fp16\":");
        const int v = json_int(line, "\"variant\":");
        if (a > 0 && b > 0 && r > 0 && h >= 0 && v >= 0 && v < TC_VARIANTS) g_tune[TuneKey(a, b, r, h)] = v;
    }
    fclose(f);
}
int tune_lookup(const TuneKey &k) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(k);
    return it == g_tune.end() ? -1 : it->second;
}
void tune_store(const TuneKey &k, int v) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[k] = v;
    const char *path = tune_path();
    if (!path) return;
    if (FILE *f = fopen(path, "a")) {
        fprintf(f, "{\"Mpad\":%d,\"Fpad\":%d,\"r0\":%d,\"fp16\":%d,\"variant\":%d}\n", std::get<0>(k),
                std::get<1>(k), std::get<2>(k), std::get<3>(k), v);
        fclose(f);
    }
}

// Time each variant (one warm run, one timed run) with CUDA events on the call's stream.
template <class Run>
int tune_variant(const Ctx &c, const TcBatch &, Run run) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c.stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1;
    }
    // One untimed run of each shape, then two timed passes in opposite orders: the sum per
    // shape cancels a drift of the clock (the GPU warms towards its power cap) that a single
    // pass in a fixed order would charge to the later shapes.
    bool ok[TC_VARIANTS];
    float tot[TC_VARIANTS];
    for (int v = 0; v < TC_VARIANTS; ++v) {
        ok[v] = run(v) == GRFT_OK;
        tot[v] = 0.f;
    }
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < TC_VARIANTS; ++i) {
            const int v = pass ? TC_VARIANTS - 1 - i : i;
            if (!ok[v]) continue;
            cudaEventRecord(e0, c.stream);
            const int rc = run(v);
            cudaEventRecord(e1, c.stream);
            float ms = 0.f;
            if (rc != GRFT_OK || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                ok[v] = false;
            else
                tot[v] += ms;
        }
    int best = 0;
    float best_ms = 3.4e38f;
    for (int v = 0; v < TC_VARIANTS; ++v)
        if (ok[v] && tot[v] < best_ms) {
            best_ms = tot[v];
            best = v;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

template <int BN, int ST, int BK, int NP>
int launch_gemm(const Ctx &c, const TcBatch &b, const uint16_t *Zhi, const uint16_t *Zlo, long zrows,
                const uint16_t *Bhi, const uint16_t *Blo, int Mpad, int Fpad) {
    static bool attr[64] = {false};
    const size_t smem = tc_smem_bytes(BN, ST, BK, NP);
    static_assert(tc_smem_bytes(BN, ST, BK, NP) <= 227 * 1024, "shared memory");
    if (!set_smem_attr((const void *)k_ds_tc<BN, ST, BK, NP>, smem, c.device, attr)) return GRFT_ECUDA;
    const uint64_t kdim = 2ull * Mpad;
    const CUtensorMapSwizzle sw = BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    CUtensorMap mzh, mzl, mbh, mbl;
    if (!encode_tma_2d(&mzh, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Zhi, kdim, (uint64_t)zrows, kdim * 2, BK,
                       TC_BM, sw) ||
        !encode_tma_2d(&mzl, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Zlo, kdim, (uint64_t)zrows, kdim * 2, BK,
                       TC_BM, sw) ||
        !encode_tma_2d(&mbh, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Bhi, kdim, 2ull * Fpad, kdim * 2, BK, BN,
                       sw) ||
        !encode_tma_2d(&mbl, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Blo, kdim, 2ull * Fpad, kdim * 2, BK, BN,
                       sw))
        return GRFT_ECUDA;
    TcBatch bb = b;
    bb.tiles_n = 2 * Fpad / BN;
    long units = 0;
    for (int i = 0; i < bb.n_items; ++i) {
        bb.it[i].tile0 = (int)units;
        units += (long)bb.it[i].ncell * bb.it[i].tiles_m * bb.tiles_n;
    }
    if (units > 0x7fffffffL) return GRFT_EINVAL;
    bb.total_tiles = (int)units;
    const uint32_t fmt = bb.fp16 ? 0u : 1u;   // kind::f16 operand format: 0 = F16, 1 = BF16
    bb.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
               ((uint32_t)(TC_BM >> 4) << 24);
    const int slots = c.num_sms;              // one persistent CTA per SM
    const int grid = bb.total_tiles < slots ? bb.total_tiles : slots;
    KernelTimer kt(c, GRFT_KERNEL_CONTRACT);
    k_ds_tc<BN, ST, BK, NP><<<grid, TC_THREADS, smem, c.stream>>>(mzh, mzl, mbh, mbl, bb);
    return check_launch();
}

int launch_gemm_variant(int variant, const Ctx &c, const TcBatch &b, const uint16_t *Zhi, const uint16_t *Zlo,
                        long zrows, const uint16_t *Bhi, const uint16_t *Blo, int Mpad, int Fpad) {
    // The BK = 32 shapes fill shared memory to its 227 KB limit with stages: the more bytes in
    // flight, the more of the L2 latency the ring hides (the loads run at 42 % of the L2-to-SM
    // bandwidth; the pipe waits on their latency, not their rate).
    if (b.nprod == 2) {   // lo plane of A only: 64 KB (BK 64) or 32 KB (BK 32) per stage of 256 columns
        switch (variant) {
            case 1: return launch_gemm<128, 4, 64, 2>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Fpad);
            case 2: return launch_gemm<256, 7, 32, 2>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Fpad);
            default: return launch_gemm<256, 3, 64, 2>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Fpad);
        }
    }
    if (b.nprod == 1) {   // no lo planes: twice the stages in the same shared memory
        switch (variant) {
            case 1: return launch_gemm<128, 6, 64, 1>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Fpad);
            case 2: return launch_gemm<256, 9, 32, 1>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Fpad);
            default: return launch_gemm<256, 4, 64, 1>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Fpad);
        }
    }
    switch (variant) {
        case 1: return launch_gemm<128, 3, 64, 3>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Fpad);
        case 2: return launch_gemm<256, 4, 32, 3>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Fpad);
        default: return launch_gemm<256, 2, 64, 3>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Fpad);
    }
}

// The pair form: one shape per product count and tile width, filling shared memory with
// stages of 64 pulses (3 stages with two products, 2 with three, 4 with one).  Spad is the
// slot count of the dechirp operand (a multiple of 128, at least the tiles' slots).
template <int ST, int NP, int BN>
int launch_pair(const Ctx &c, const TcBatch &b, const uint16_t *Zhi, const uint16_t *Zlo, long zrows,
                const uint16_t *Bhi, const uint16_t *Blo, int Mpad, int Spad) {
    static bool attr[64] = {false};
    const size_t smem = pr_smem_bytes(ST, NP, BN);
    static_assert(pr_smem_bytes(ST, NP, BN) <= 227 * 1024 - 2048, "shared memory (with the static part)");
    const int tiles_n = (b.slots + BN / 2 - 1) / (BN / 2);
    if (tiles_n * (BN / 2) > Spad) return GRFT_EINVAL;
    if (!set_smem_attr((const void *)k_ds_pair<ST, NP, BN>, smem, c.device, attr)) return GRFT_ECUDA;
    // A: the split operand seen as [row][2 Mpad / 32 runs][32 pulses] (run y = 2 g + part); a
    // box of both parts of one group and 64 rows lands as 128 rows (bin, part) of 64 bytes
    const uint64_t dims[3] = {32, 2ull * (uint64_t)(Mpad / 32), (uint64_t)zrows};
    const uint64_t strides[2] = {64, 4ull * (uint64_t)Mpad};
    const uint32_t box[3] = {32, 2, (uint32_t)PR_BINS};
    CUtensorMap mzh, mzl, mbh, mbl;
    if (!encode_tma_3d(&mzh, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Zhi, dims, strides, box,
                       CU_TENSOR_MAP_SWIZZLE_64B) ||
        !encode_tma_3d(&mzl, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Zlo, dims, strides, box,
                       CU_TENSOR_MAP_SWIZZLE_64B) ||
        !encode_tma_2d(&mbh, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Bhi, (uint64_t)pair_mrow(Mpad), 2ull * Spad,
                       (uint64_t)pair_mrow(Mpad) * 2, PR_BK, BN, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_tma_2d(&mbl, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Blo, (uint64_t)pair_mrow(Mpad), 2ull * Spad,
                       (uint64_t)pair_mrow(Mpad) * 2, PR_BK, BN, CU_TENSOR_MAP_SWIZZLE_128B))
        return GRFT_ECUDA;
    TcBatch bb = b;
    bb.tiles_n = tiles_n;
    long units = 0;
    for (int i = 0; i < bb.n_items; ++i) {
        bb.it[i].tile0 = (int)units;
        units += (long)bb.it[i].ncell * ((bb.it[i].r0_count + PR_BINS - 1) / PR_BINS) * bb.tiles_n;
    }
    if (units > 0x7fffffffL) return GRFT_EINVAL;
    bb.total_tiles = (int)units;
    const uint32_t fmt = bb.fp16 ? 0u : 1u;   // kind::f16 operand format: 0 = F16, 1 = BF16
    bb.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const int grid = bb.total_tiles < c.num_sms ? bb.total_tiles : c.num_sms;
    if (grid <= 0) return GRFT_OK;
    KernelTimer kt(c, GRFT_KERNEL_CONTRACT);
    k_ds_pair<ST, NP, BN><<<grid, PR_THREADS, smem, c.stream>>>(mzh, mzl, mbh, mbl, bb);
    return check_launch();
}

template <int BN>
int launch_pair_nprod(const Ctx &c, const TcBatch &b, const uint16_t *Zhi, const uint16_t *Zlo, long zrows,
                      const uint16_t *Bhi, const uint16_t *Blo, int Mpad, int Spad) {
    if (b.nprod == 1) return launch_pair<4, 1, BN>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Spad);
    if (b.nprod == 2) return launch_pair<3, 2, BN>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Spad);
    return launch_pair<2, 3, BN>(c, b, Zhi, Zlo, zrows, Bhi, Blo, Mpad, Spad);
}

// One round = the split kernel over every (item, cell, bin tile) of the batch, then the
// persistent GEMM over every (item, cell, bin tile, hypothesis tile).
struct Round {
    TcBatch b;
    long rows;
};

int launch_split(const Ctx &c, const TcBatch &b, uint16_t *Zhi, uint16_t *Zlo, long zrows) {
    // shared memory: the warp tiles (1024-byte aligned for the 128-byte swizzle), then the
    // bins and phases of a cell (largest M of the round, up to SP_TAB_MAX; larger items read
    // their tables from global memory)
    static bool attr[64] = {false};
    int cap = 0;
    for (int i = 0; i < b.n_items; ++i) cap = b.it[i].M > cap ? b.it[i].M : cap;
    if (cap > SP_TAB_MAX) cap = SP_TAB_MAX;
    const size_t most = 1024 + SP_TR_WORDS * sizeof(uint4) + (size_t)SP_TAB_MAX * (sizeof(float2) + sizeof(int));
    const size_t bytes = 1024 + SP_TR_WORDS * sizeof(uint4) + (size_t)cap * (sizeof(float2) + sizeof(int));
    if (c.device >= 64 || !set_smem_attr((const void *)k_coarse_split, most, c.device, attr)) return GRFT_ECUDA;
    // the operand planes as [rows][zld] 16-bit elements; a box of 64 elements (one 32-pulse
    // stage: re and im parts) x 32 rows is one warp tile
    CUtensorMap mh, ml;
    if (zrows <= 0 || zrows > 0x7fffffffL) return GRFT_EINVAL;
    if (!encode_tma_2d(&mh, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)Zhi, (uint64_t)b.zld, (uint64_t)zrows,
                       (uint64_t)b.zld * 2, TC_BK, 32, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !encode_tma_2d(&ml, CU_TENSOR_MAP_DATA_TYPE_UINT16, (void *)(Zlo ? Zlo : Zhi), (uint64_t)b.zld,
                       (uint64_t)zrows, (uint64_t)b.zld * 2, TC_BK, 32, CU_TENSOR_MAP_SWIZZLE_128B))
        return GRFT_ECUDA;
    KernelTimer kt(c, GRFT_KERNEL_SPLIT);
    k_coarse_split<<<b.total_ctas, SP_THREADS, bytes, c.stream>>>(b, mh, ml, cap);
    return check_launch();
}

int launch_round_gemm(const Ctx &c, const Round &rd, int Mpad, int Fpad, const uint16_t *Bhi,
                      const uint16_t *Blo, uint16_t *Zhi, uint16_t *Zlo, int &variant, const TuneKey &key) {
    if (rd.b.slots > 0) {   // pair form (one shape per product count)
        const int Spad = (rd.b.slots + 127) / 128 * 128;     // the dechirp operand's slots
        int bn = pair_bn(rd.b.slots);
        if (const char *e = getenv("DSGRFT_PAIR_BN")) bn = atoi(e);   // explicit width (experiments)
        switch (bn) {
            case 224: return launch_pair_nprod<224>(c, rd.b, Zhi, Zlo, rd.rows, Bhi, Blo, Mpad, Spad);
            case 192: return launch_pair_nprod<192>(c, rd.b, Zhi, Zlo, rd.rows, Bhi, Blo, Mpad, Spad);
            default: return launch_pair_nprod<256>(c, rd.b, Zhi, Zlo, rd.rows, Bhi, Blo, Mpad, Spad);
        }
    }
    if (variant < 0) {   // autotune: time the tile shapes on this round of cells, keep the fastest
        variant = tune_variant(c, rd.b, [&](int v) {
            return launch_gemm_variant(v, c, rd.b, Zhi, Zlo, rd.rows, Bhi, Blo, Mpad, Fpad);
        });
        if (variant < 0) return GRFT_ECUDA;
        tune_store(key, variant);
    }
    return launch_gemm_variant(variant, c, rd.b, Zhi, Zlo, rd.rows, Bhi, Blo, Mpad, Fpad);
}

// Side stream and events of the split/contraction pipeline, created once per device.
struct Pipe {
    bool init = false;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, split_done[2] = {nullptr, nullptr}, gemm_done[2] = {nullptr, nullptr};
};
Pipe g_pipe[64];
std::mutex g_pipe_mu;

Pipe *get_pipe(int dev) {
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    Pipe &p = g_pipe[dev];
    if (!p.init) {
        if (cudaStreamCreateWithFlags(&p.side, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        cudaEvent_t *evs[5] = {&p.fork, &p.split_done[0], &p.split_done[1], &p.gemm_done[0], &p.gemm_done[1]};
        for (cudaEvent_t *e : evs)
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        p.init = true;
    }
    return &p;
}

}  // namespace

// Destroys the side stream and events of the split/contraction pipeline of a device (the
// next call that needs them creates them again).  The device must be idle.
void release_pipe(int dev) {
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    Pipe &p = g_pipe[dev];
    if (!p.init) return;
    cudaEvent_t evs[5] = {p.fork, p.split_done[0], p.split_done[1], p.gemm_done[0], p.gemm_done[1]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (p.side) cudaStreamDestroy(p.side);
    p = Pipe();
}

int launch_ds_tc(const Ctx &c, const DsTcItem *items, int n_items, const grft_dsgrid &g,
                 const int32_t *rho, const float2 *w, int tab_cell0, int Mtab, const uint16_t *Bhi,
                 const uint16_t *Blo, int Mpad, bool fp16, int nprod, uint16_t *const Zhi[2],
                 uint16_t *const Zlo[2], long z_rows_cap, const Rate3 &rate) {
    const int F = g.Fv * g.Fa * rate.Fb;
    const int Fpad = (F + 127) / 128 * 128;
    TcBatch b;
    b.rho = rho;
    b.w = w;
    b.tab_cell0 = tab_cell0;
    b.Mtab = Mtab;
    b.zld = 2 * Mpad;
    b.tiles_n = Fpad / 128;          // 256-column tiles; launch_gemm recounts for its variant
    b.F = F;
    b.Fv = g.Fv;
    b.Fa = g.Fa;
    b.na_c = g.ac.count;
    b.Fb = rate.Fb;
    b.nb_c = rate.count;
    b.fp16 = fp16 ? 1 : 0;
    b.nprod = nprod;
    b.slots = ds_pair_form(rate) ? pair_slot_count3(g.Fv, g.Fa, rate.Fb) : 0;
    b.idesc = 0;                     // set per variant by launch_gemm
    b.status = c.status;
    b.wait_limit = c.wait_limit;
    auto reset = [&]() {
        b.n_items = 0;
        b.total_ctas = 0;
        b.total_tiles = 0;
    };
    reset();
    int rmax = 1;
    long total_rows = 0;
    for (int i = 0; i < n_items; ++i) {
        const int tm = (items[i].r0_count + TC_BM - 1) / TC_BM;
        while (rmax < tm) rmax <<= 1;
        if (items[i].cell_count > 0) total_rows += (long)items[i].cell_count * tm * TC_BM;
    }
    // precision bucket: 0 split BF16, 1 split FP16, 3 single-product FP16, 5 two-product FP16
    const TuneKey key(Mpad, Fpad, rmax, (fp16 ? 1 : 0) + (nprod == 1 ? 2 : 0) + (nprod == 2 ? 4 : 0));
    int variant = tune_lookup(key);
    if (variant < 0 && !tune_enabled()) variant = 0;
    if (const char *fv = getenv("DSGRFT_TILE_VARIANT")) {   // explicit choice (tests, experiments)
        const int v = atoi(fv);
        if (v >= 0 && v < TC_VARIANTS) variant = v;
    }
    // Rounds of about 1/TC_ROUNDS of the work (whole cells, at least TC_MIN_ROUND_ROWS rows,
    // within the buffer), so that the split of round r+1 runs beside the contraction of
    // round r.  DSGRFT_ROUNDS overrides the target count (1: split, then contract).
    int n_rounds = TC_ROUNDS;
    if (const char *nr = getenv("DSGRFT_ROUNDS")) {
        const int v = atoi(nr);
        if (v >= 1 && v <= 1024) n_rounds = v;
    }
    long round_rows = (total_rows + n_rounds - 1) / n_rounds;
    if (n_rounds > 1 && round_rows < TC_MIN_ROUND_ROWS) round_rows = TC_MIN_ROUND_ROWS;
    if (round_rows > z_rows_cap) round_rows = z_rows_cap;
    std::vector<Round> rounds;
    long rows_used = 0;
    auto flush = [&]() {
        if (b.n_items > 0) rounds.push_back(Round{b, rows_used});
        reset();
        rows_used = 0;
    };
    for (int i = 0; i < n_items; ++i) {
        const DsTcItem &d = items[i];
        if (d.cell_count <= 0 || d.r0_count <= 0) continue;
        const int tiles_m = (d.r0_count + TC_BM - 1) / TC_BM;
        const int r0_pad = tiles_m * TC_BM;
        if (r0_pad > z_rows_cap || d.M > Mtab || (d.M + 31) / 32 * 32 > Mpad) return GRFT_EINVAL;
        int cell = d.cell_begin;
        const int cell_end = d.cell_begin + d.cell_count;
        while (cell < cell_end) {
            const long lim = round_rows < r0_pad ? r0_pad : round_rows;
            long fit = (lim - rows_used) / r0_pad;
            if (fit <= 0 || b.n_items == TC_MAX_ITEMS) {
                flush();
                continue;
            }
            const int take = (int)(fit < cell_end - cell ? fit : cell_end - cell);
            const long ctas = (long)take * tiles_m;
            const long tiles = ctas * b.tiles_n;
            if ((long)b.total_tiles + tiles > 0x7fffffffL) return GRFT_EINVAL;
            TcItem &t = b.it[b.n_items++];
            t.echo = d.echo;
            t.Z = d.Z;
            t.P = d.P;
            t.Y = d.Y;
            t.e0 = d.e0;
            t.M = d.M;
            t.N = d.N;
            t.KT = (d.M + 31) / 32;
            t.r0_begin = d.r0_begin;
            t.r0_count = d.r0_count;
            t.tiles_m = tiles_m;
            t.r0_pad = r0_pad;
            t.cell0 = cell;
            t.ncell = take;
            t.i0 = d.i0;
            t.zrow0 = rows_used;
            t.cta0 = b.total_ctas;
            t.tile0 = b.total_tiles;
            b.total_ctas += (int)ctas;
            b.total_tiles += (int)tiles;
            rows_used += (long)take * r0_pad;
            cell += take;
        }
    }
    flush();
    if (rounds.empty()) return GRFT_OK;
    int e;
    static const bool overlap = [] {             // DSGRFT_OVERLAP=0: every round on the caller's stream
        const char *e = getenv("DSGRFT_OVERLAP");
        return !(e && e[0] == '0');
    }();
    if (rounds.size() == 1 || !Zhi[1] || !Zlo[1] || !overlap) {   // rounds in sequence on the caller's stream
        for (const Round &rd : rounds) {
            if ((e = launch_split(c, rd.b, Zhi[0], Zlo[0], rd.rows))) return e;
            if ((e = launch_round_gemm(c, rd, Mpad, Fpad, Bhi, Blo, Zhi[0], Zlo[0], variant, key))) return e;
        }
        return GRFT_OK;
    }
    // Pipeline: splits on the side stream into alternating buffers, contractions on the
    // caller's stream; events order each buffer's reuse.
    Pipe *pp = get_pipe(c.device);
    if (!pp) return GRFT_ECUDA;
    Ctx cs = c;
    cs.stream = pp->side;
    if (cudaEventRecord(pp->fork, c.stream) != cudaSuccess ||
        cudaStreamWaitEvent(pp->side, pp->fork, 0) != cudaSuccess)
        return GRFT_ECUDA;
    for (size_t r = 0; r < rounds.size(); ++r) {
        const int buf = (int)(r & 1);
        if (r >= 2 && cudaStreamWaitEvent(pp->side, pp->gemm_done[buf], 0) != cudaSuccess) return GRFT_ECUDA;
        if ((e = launch_split(cs, rounds[r].b, Zhi[buf], Zlo[buf], rounds[r].rows))) return e;
        if (cudaEventRecord(pp->split_done[buf], pp->side) != cudaSuccess ||
            cudaStreamWaitEvent(c.stream, pp->split_done[buf], 0) != cudaSuccess)
            return GRFT_ECUDA;
        if ((e = launch_round_gemm(c, rounds[r], Mpad, Fpad, Bhi, Blo, Zhi[buf], Zlo[buf], variant, key)))
            return e;
        if (cudaEventRecord(pp->gemm_done[buf], c.stream) != cudaSuccess) return GRFT_ECUDA;
    }
    return GRFT_OK;
}

}  // namespace grft
