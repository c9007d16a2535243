// C ABI of libdsgrft.so: argument checks, per-device state (status word, workspace) and
// the sequencing of table builders and kernels on the caller's stream.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "tma.cuh"

namespace grft {

bool ds_pair_form(const Rate3 &rate) {
    static const bool on = [] {
        const char *e = getenv("DSGRFT_PAIR");
        return !(e && e[0] == '0');
    }();
    // P = 2; P = 3 whose rate axis is one zero offset (the P = 2 pairs); P = 3 with Fb >= 2
    // rate offsets (mirrors on all three axes).  A single nonzero rate offset has no mirror.
    return on && (!rate.on || (rate.Fb == 1 && rate.step == 0.0) || rate.Fb >= 2);
}

namespace {

constexpr int MAX_DEV = 64;
constexpr uint64_t DEFAULT_WAIT_LIMIT = 2000000000ull;   // ~1 s of SM cycles
constexpr size_t PLAIN_TABLE_BUDGET = 256ull << 20;
constexpr size_t SPLIT_OPERAND_DEFAULT = 16ull << 30;  // both planes of the split coarse-RM output

// Workspace budget of the split operand of the tensor-core DS path (both planes).  The
// environment variable DSGRFT_SPLIT_BUDGET_BYTES overrides it (read once; smaller values
// make large problems run in more rounds, which the tests use to exercise chunking).
size_t split_budget() {
    static size_t v = [] {
        const char *e = getenv("DSGRFT_SPLIT_BUDGET_BYTES");
        if (e && *e) {
            const unsigned long long x = strtoull(e, nullptr, 10);
            if (x > 0) return (size_t)x;
        }
        return SPLIT_OPERAND_DEFAULT;
    }();
    return v;
}

// Rows per split-operand buffer.  If the whole operand (total_rows) fits the budget in one
// buffer of two planes, one buffer holding all of it (one round); otherwise two buffers of
// a quarter of the budget each, so that the split of one round can be written while the
// contraction of the previous one reads the other.  At least min_rows (one cell or item).
long split_rows(long total_rows, long min_rows, long row_bytes, int &nbuf, bool force_two = false) {
    const long budget_rows = (long)(split_budget() / (2 * (size_t)row_bytes));
    if (!force_two && total_rows <= budget_rows) {
        nbuf = 1;
        return total_rows > min_rows ? total_rows : min_rows;
    }
    nbuf = 2;
    long rows = budget_rows / 2;
    if (min_rows > 0 && rows > min_rows) rows = rows / min_rows * min_rows;   // whole cells
    if (rows > total_rows) rows = total_rows;
    return rows > min_rows ? rows : min_rows;
}

struct DevState {
    bool init = false;
    int *status = nullptr;
    void *ws[WS_SLOTS] = {};                   // one workspace per operation class
    size_t ws_size[WS_SLOTS] = {};
    int num_sms = 0;
    int cc = 0;
};

DevState g_dev[MAX_DEV];
std::mutex g_mu;
uint64_t g_wait_limit = DEFAULT_WAIT_LIMIT;

int make_ctx(void *stream, Ctx &c) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return GRFT_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &d = g_dev[dev];
    if (!d.init) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return GRFT_ECUDA;
        d.cc = major * 10 + minor;
        if (cudaMalloc(&d.status, 256) != cudaSuccess) return GRFT_ENOMEM;
        if (cudaMemset(d.status, 0, 256) != cudaSuccess) return GRFT_ECUDA;
        d.init = true;
    }
    if (d.cc != 103) return GRFT_EUNSUPPORTED;   // the library is built for sm_103a only
    c.device = dev;
    c.stream = (cudaStream_t)stream;
    c.status = d.status;
    c.wait_limit = g_wait_limit;
    c.num_sms = d.num_sms;
    return GRFT_OK;
}

bool dsgrid_ok(const grft_dsgrid *g, const grft_radar *r) {
    return g && axis_ok(g->vc) && axis_ok(g->ac) && g->Fv > 0 && g->Fa > 0 && g->r0_count > 0 &&
           g->r0_begin >= 0 && (long)g->r0_begin + g->r0_count <= (long)r->N &&
           (long)g->vc.count * g->ac.count <= 0x7fffffffL && (long)g->Fv * g->Fa <= (1L << 20);
}

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

}  // namespace

void *workspace(const Ctx &ctx, size_t bytes, int slot) {
    if (slot < 0 || slot >= WS_SLOTS) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &d = g_dev[ctx.device];
    if (bytes <= d.ws_size[slot]) return d.ws[slot];
    if (d.ws[slot]) {
        cudaDeviceSynchronize();
        cudaFree(d.ws[slot]);
        d.ws[slot] = nullptr;
        d.ws_size[slot] = 0;
    }
    size_t want = align_up(bytes, 64ull << 20);
    if (cudaMalloc(&d.ws[slot], want) != cudaSuccess) {
        cudaGetLastError();
        d.ws[slot] = nullptr;
        return nullptr;
    }
    d.ws_size[slot] = want;
    return d.ws[slot];
}

namespace {
struct TimingRec {
    int kernel;
    cudaEvent_t a, b;
};
std::mutex g_timing_mu;
bool g_timing_on = false;
std::vector<TimingRec> g_timing_pending;
int g_timing_count[GRFT_KERNEL_COUNT] = {0};
double g_timing_ms[GRFT_KERNEL_COUNT] = {0.0};

void timing_drain_locked() {
    for (const TimingRec &r : g_timing_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_timing_count[r.kernel] += 1;
            g_timing_ms[r.kernel] += ms;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_timing_pending.clear();
}
}  // namespace

KernelTimer::KernelTimer(const Ctx &c, int kernel) : stream_(c.stream), kernel_(kernel) {
    {
        std::lock_guard<std::mutex> lk(g_timing_mu);
        if (!g_timing_on) return;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream_, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaEventCreate(&a_) != cudaSuccess) {
        a_ = nullptr;
        return;
    }
    if (cudaEventCreate(&b_) != cudaSuccess) {
        cudaEventDestroy(a_);
        a_ = b_ = nullptr;
        return;
    }
    cudaEventRecord(a_, stream_);
}

KernelTimer::~KernelTimer() {
    if (!a_) return;
    cudaEventRecord(b_, stream_);
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_timing_pending.push_back(TimingRec{kernel_, a_, b_});
}

int check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GRFT_OK : GRFT_ECUDA;
}

bool encode_tma_2d(CUtensorMap *map, CUtensorMapDataType dtype, void *base, uint64_t dim0,
                   uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1,
                   CUtensorMapSwizzle swizzle) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !ptr)
            return false;
        fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    cuuint64_t dims[2] = {dim0, dim1};
    cuuint64_t strides[1] = {stride1_bytes};
    cuuint32_t box[2] = {box0, box1};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, dtype, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_tma_3d(CUtensorMap *map, CUtensorMapDataType dtype, void *base, const uint64_t dims[3],
                   const uint64_t strides_bytes[2], const uint32_t box[3], CUtensorMapSwizzle swizzle) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !ptr)
            return false;
        fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    }
    cuuint64_t d[3] = {dims[0], dims[1], dims[2]};
    cuuint64_t st[2] = {strides_bytes[0], strides_bytes[1]};
    cuuint32_t bx[3] = {box[0], box[1], box[2]};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, dtype, 3, base, d, st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {

// Waits on an mbarrier phase that nothing completes, bounded by `limit` SM cycles: the
// timeout path of every warp-specialised kernel, exercised without any copy or MMA in flight.
__global__ void k_selftest_wait(int *status, uint64_t limit) {
    __shared__ alignas(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbarrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit)) latch_error(status, GRFT_ETIMEOUT);
}

}  // namespace

}  // namespace grft

using namespace grft;

extern "C" {

int grft_timing(int enable) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    timing_drain_locked();
    for (int i = 0; i < GRFT_KERNEL_COUNT; ++i) {
        g_timing_count[i] = 0;
        g_timing_ms[i] = 0.0;
    }
    g_timing_on = enable != 0;
    return GRFT_OK;
}

int grft_timing_get(int kernel, int32_t *launches, double *total_ms) {
    if (kernel < 0 || kernel >= GRFT_KERNEL_COUNT || !launches || !total_ms) return GRFT_EINVAL;
    std::lock_guard<std::mutex> lk(g_timing_mu);
    timing_drain_locked();
    *launches = g_timing_count[kernel];
    *total_ms = g_timing_ms[kernel];
    return GRFT_OK;
}

int grft_selftest_wait(uint64_t cycles, void *stream) {
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    k_selftest_wait<<<1, 32, 0, c.stream>>>(c.status, cycles ? cycles : c.wait_limit);
    return check_launch();
}

int grft_version(void) { return GRFT_ABI_VERSION; }

const char *grft_status_string(int s) {
    switch (s) {
        case GRFT_OK: return "ok";
        case GRFT_EINVAL: return "invalid argument";
        case GRFT_ENOMEM: return "out of device memory";
        case GRFT_ECUDA: return "CUDA error";
        case GRFT_ETIMEOUT: return "bounded device wait ran out";
        case GRFT_EUNSUPPORTED: return "unsupported device or precision";
        case GRFT_EOVERFLOW: return "detection candidate buffer overflow";
        default: return "unknown status";
    }
}

int grft_sync_status(void *stream) {
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return GRFT_ECUDA;
    int h = 0;
    if (cudaMemcpy(&h, c.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GRFT_ECUDA;
    if (h != 0 && cudaMemset(c.status, 0, sizeof(int)) != cudaSuccess) return GRFT_ECUDA;
    return h;
}

int grft_shutdown(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return GRFT_ECUDA;
    int e = grft_release_workspace();
    if (e) return e;
    release_pipe(dev);
    std::lock_guard<std::mutex> lk(g_timing_mu);
    for (const TimingRec &r : g_timing_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_timing_pending.clear();
    g_timing_on = false;
    return GRFT_OK;
}

int grft_set_wait_limit(uint64_t cycles) {
    g_wait_limit = cycles ? cycles : DEFAULT_WAIT_LIMIT;
    return GRFT_OK;
}

int grft_release_workspace(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return GRFT_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &d = g_dev[dev];
    if ((d.ws[0] || d.ws[1]) && cudaDeviceSynchronize() != cudaSuccess) return GRFT_ECUDA;
    for (int i = 0; i < WS_SLOTS; ++i) {
        if (d.ws[i]) cudaFree(d.ws[i]);
        d.ws[i] = nullptr;
        d.ws_size[i] = 0;
    }
    return GRFT_OK;
}

int grft_bins_phases(const grft_radar *radar, const double *v, const double *a, int32_t nh,
                     int32_t *rho, grft_c32 *w, void *stream) {
    if (!radar_ok(radar) || nh < 0 || (nh > 0 && (!v || !a || !rho || !w))) return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    return launch_bins_phases(c, radar_d(*radar), v, a, nh, rho, w);
}

int grft_plain(const grft_radar *radar, const grft_c32 *echo, const grft_grid *grid, grft_c32 *Y,
               float *P, void *stream) {
    if (!radar_ok(radar) || !echo || !grid || (!Y && !P) || !axis_ok(grid->v) || !axis_ok(grid->a) ||
        grid->r0_count <= 0 || grid->r0_begin < 0 || (long)grid->r0_begin + grid->r0_count > radar->N)
        return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    const RadarD R = radar_d(*radar);
    const long nh_total = (long)grid->v.count * grid->a.count;
    long chunk = (long)(PLAIN_TABLE_BUDGET / ((size_t)R.M * (sizeof(int32_t) + sizeof(float2))));
    chunk = chunk / 16 * 16;
    if (chunk < 8) chunk = 8;
    if (chunk > (1L << 18)) chunk = 1L << 18;
    if (chunk > nh_total) chunk = nh_total;
    const size_t e0_bytes = align_up((size_t)grid->r0_count * sizeof(float2));
    const size_t rho_bytes = align_up((size_t)chunk * R.M * sizeof(int32_t));
    const size_t w_bytes = align_up((size_t)chunk * R.M * sizeof(float2));
    unsigned char *ws = (unsigned char *)workspace(c, e0_bytes + rho_bytes + w_bytes);
    if (!ws) return GRFT_ENOMEM;
    float2 *e0 = (float2 *)ws;
    int32_t *rho = (int32_t *)(ws + e0_bytes);
    float2 *w = (float2 *)(ws + e0_bytes + rho_bytes);
    if ((e = launch_range_phase(c, R, grid->r0_begin, grid->r0_count, e0))) return e;
    for (long h0 = 0; h0 < nh_total; h0 += chunk) {
        const int nh = (int)(nh_total - h0 < chunk ? nh_total - h0 : chunk);
        if ((e = launch_plain_tables(c, R, *grid, h0, nh, rho, w))) return e;
        if ((e = launch_plain(c, R, (const float2 *)echo, *grid, h0, nh, rho, w, e0, (float2 *)Y, P)))
            return e;
    }
    return GRFT_OK;
}

int dsgrft_coarse_rm(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                     int32_t cell_begin, int32_t cell_count, grft_c32 *Z, void *stream) {
    if (!radar_ok(radar) || !echo || !Z || !dsgrid_ok(grid, radar) || cell_begin < 0 ||
        cell_count < 0 || (long)cell_begin + cell_count > (long)grid->vc.count * grid->ac.count ||
        cell_count > 65535)
        return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    const RadarD R = radar_d(*radar);
    const size_t rho_bytes = align_up((size_t)cell_count * R.M * sizeof(int32_t));
    const size_t w_bytes = align_up((size_t)cell_count * R.M * sizeof(float2));
    unsigned char *ws = (unsigned char *)workspace(c, rho_bytes + w_bytes);
    if (!ws) return GRFT_ENOMEM;
    int32_t *rho = (int32_t *)ws;
    float2 *w = (float2 *)(ws + rho_bytes);
    if ((e = launch_coarse_tables(c, R, *grid, cell_begin, cell_count, rho, w))) return e;
    return launch_coarse_rm(c, R, (const float2 *)echo, *grid, cell_count, rho, w, (float2 *)Z);
}

namespace {

// Bytes of one plane of the dechirp operand D (the split modes keep a hi and a lo plane of
// [2 Fpad][2 Mpad] 16-bit values; the FP32 contraction one [M][F] complex plane).
size_t dechirp_plane_bytes(const RadarD &R, const grft_dsgrid &g, const Rate3 &rate, bool tc) {
    const int F = g.Fv * g.Fa * rate.Fb;
    const int Fpad = (F + 127) / 128 * 128;
    const int Mpad = (R.M + 31) / 32 * 32;
    return tc ? align_up((size_t)2 * Fpad * 2 * Mpad * sizeof(uint16_t)) : align_up((size_t)R.M * F * sizeof(float2));
}

// D of the fine offsets of grid (eq. H-DFM) in the layout of the precision: two planes of
// dechirp_plane_bytes at dst for the tensor-core modes (the pair form's [2 Spad][Mpad]
// layout where ds_pair_form holds, which fits the 4M form's [2 Fpad][2 Mpad]), one for FP32.
int fill_dechirp(const Ctx &c, const RadarD &R, const grft_dsgrid &g, const Rate3 &rate, grft_precision precision,
                 unsigned char *dst) {
    const bool tc = precision != GRFT_FP32;
    if (!tc) return launch_dechirp(c, R, g, (float2 *)dst);
    const int F = g.Fv * g.Fa * rate.Fb;
    const int Fpad = (F + 127) / 128 * 128;
    const int Mpad = (R.M + 31) / 32 * 32;
    const size_t d_bytes = dechirp_plane_bytes(R, g, rate, true);
    if (ds_pair_form(rate)) {   // [2 Spad][pair_mrow(M)] per plane: within d_bytes (Spad <= Fpad, Mrow <= 2 Mpad)
        const int Spad = (pair_slot_count3(g.Fv, g.Fa, rate.Fb) + 127) / 128 * 128;
        return launch_dechirp_pair(c, R, g, pair_mrow(R.M), Spad, precision_fp16(precision), (uint16_t *)dst,
                                   (uint16_t *)(dst + d_bytes), rate);
    }
    return launch_dechirp_split(c, R, g, Mpad, Fpad, precision_fp16(precision), (uint16_t *)dst,
                                (uint16_t *)(dst + d_bytes), rate);
}

// The fine stage of dsgrft_fine_dfm (rate off) and dsgrft3_fine_dfm (P = 3, rate on): the
// arguments are checked by the callers.  dechirp (nullable): D already in place, as
// fill_dechirp writes it for this radar, grid, rate and precision (it is not recomputed).
int fine_dfm_impl(const grft_radar *radar, const grft_c32 *Z, const grft_c32 *echo, const grft_dsgrid *grid,
                  const Rate3 &rate, int32_t cell_begin, int32_t cell_count, grft_precision precision,
                  grft_c32 *Y, float *P, void *stream, const unsigned char *dechirp = nullptr) {
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    const RadarD R = radar_d(*radar);
    const int Mpad = (R.M + 31) / 32 * 32;
    const bool tc = precision != GRFT_FP32;
    const size_t rho_bytes = align_up((size_t)cell_count * R.M * sizeof(int32_t));
    const size_t w_bytes = align_up((size_t)cell_count * R.M * sizeof(float2));
    const size_t e0_bytes = align_up((size_t)grid->r0_count * sizeof(float2));
    const size_t d_bytes = dechirp_plane_bytes(R, *grid, rate, tc);
    // split operand: as many whole cells as fit the budget (at least one)
    const long row_bytes = 2L * Mpad * (long)sizeof(uint16_t);
    const long r0_pad = tc ? ds_tc_r0_pad(grid->r0_count) : 0;
    long z_rows = 0;                 // rows per operand buffer (two 16-bit planes each)
    int nbuf = 1;
    if (tc) z_rows = split_rows(r0_pad * cell_count, r0_pad, row_bytes, nbuf);
    const size_t z_plane = align_up((size_t)z_rows * row_bytes);
    unsigned char *ws = (unsigned char *)workspace(
        c, rho_bytes + w_bytes + e0_bytes + (tc ? 2 * d_bytes + 2 * nbuf * z_plane : d_bytes));
    if (!ws) return GRFT_ENOMEM;
    int32_t *rho = (int32_t *)ws;
    float2 *w = (float2 *)(ws + rho_bytes);
    float2 *e0 = (float2 *)(ws + rho_bytes + w_bytes);
    unsigned char *dptr = ws + rho_bytes + w_bytes + e0_bytes;
    if (!Z && (e = launch_coarse_tables(c, R, *grid, cell_begin, cell_count, rho, w, rate))) return e;
    if ((e = launch_range_phase(c, R, grid->r0_begin, grid->r0_count, e0))) return e;
    if (!tc) {                       // P = 2 only (the callers refuse FP32 for P = 3)
        DsOut out;
        out.Y = (float2 *)Y;
        out.P = P;
        out.cell_begin = cell_begin;
        out.i0 = cell_begin / grid->ac.count;
        out.na_c = grid->ac.count;
        out.Fv = grid->Fv;
        out.Fa = grid->Fa;
        float2 *D = (float2 *)dptr;
        if (dechirp)
            D = (float2 *)dechirp;
        else if ((e = fill_dechirp(c, R, *grid, rate, precision, dptr)))
            return e;
        return launch_ds_simt(c, R, (const float2 *)echo, (const float2 *)Z, *grid, cell_count, rho, w,
                              D, e0, out);
    }
    const unsigned char *dsrc = dechirp ? dechirp : dptr;
    const uint16_t *Bhi = (const uint16_t *)dsrc, *Blo = (const uint16_t *)(dsrc + d_bytes);
    unsigned char *zp = dptr + 2 * d_bytes;
    uint16_t *const Zhi[2] = {(uint16_t *)zp, nbuf > 1 ? (uint16_t *)(zp + 2 * z_plane) : nullptr};
    uint16_t *const Zlo[2] = {(uint16_t *)(zp + z_plane), nbuf > 1 ? (uint16_t *)(zp + 3 * z_plane) : nullptr};
    const bool fp16 = precision_fp16(precision);
    const int nprod = precision_nprod(precision);
    if (!dechirp && (e = fill_dechirp(c, R, *grid, rate, precision, dptr))) return e;
    DsTcItem it;
    it.echo = (const float2 *)echo;
    it.Z = (const float2 *)Z;
    it.P = P;
    it.Y = (float2 *)Y;
    it.e0 = e0;
    it.M = R.M;
    it.N = R.N;
    it.r0_begin = grid->r0_begin;
    it.r0_count = grid->r0_count;
    it.cell_begin = cell_begin;
    it.cell_count = cell_count;
    it.i0 = cell_begin / (grid->ac.count * rate.count);
    return launch_ds_tc(c, &it, 1, *grid, rho, w, cell_begin, R.M, Bhi, Blo, Mpad, fp16, nprod, Zhi, Zlo, z_rows,
                        rate);
}

bool precision_ok(grft_precision p) {
    return p == GRFT_FP32 || p == GRFT_BF16X3 || p == GRFT_FP16X3 || p == GRFT_FP16X1 || p == GRFT_FP16X2;
}

}  // namespace

int dsgrft_fine_dfm(const grft_radar *radar, const grft_c32 *Z, const grft_c32 *echo,
                    const grft_dsgrid *grid, int32_t cell_begin, int32_t cell_count,
                    grft_precision precision, grft_c32 *Y, float *P, void *stream) {
    if (!radar_ok(radar) || (!Z && !echo) || (!Y && !P) || !dsgrid_ok(grid, radar) ||
        cell_begin < 0 || cell_count < 0 ||
        (long)cell_begin + cell_count > (long)grid->vc.count * grid->ac.count || cell_count > 65535)
        return GRFT_EINVAL;
    if (!precision_ok(precision)) return GRFT_EINVAL;
    return fine_dfm_impl(radar, Z, echo, grid, kNoRate, cell_begin, cell_count, precision, Y, P, stream);
}

int dsgrft3_fine_dfm(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid3 *grid3, int32_t cell_begin,
                     int32_t cell_count, grft_precision precision, grft_c32 *Y, float *P, void *stream) {
    if (!radar_ok(radar) || !echo || (!Y && !P) || !grid3 || !axis_ok(grid3->bc) || grid3->Fb <= 0)
        return GRFT_EINVAL;
    grft_dsgrid g;
    g.r0_begin = grid3->r0_begin;
    g.r0_count = grid3->r0_count;
    g.vc = grid3->vc;
    g.ac = grid3->ac;
    g.Fv = grid3->Fv;
    g.Fa = grid3->Fa;
    if (!dsgrid_ok(&g, radar) || (long)g.Fv * g.Fa * grid3->Fb > (1L << 20) || cell_begin < 0 || cell_count < 0 ||
        (long)cell_begin + cell_count > (long)g.vc.count * g.ac.count * grid3->bc.count || cell_count > 65535)
        return GRFT_EINVAL;
    if (!precision_ok(precision)) return GRFT_EINVAL;
    if (precision == GRFT_FP32) return GRFT_EUNSUPPORTED;     // the tensor-core path only
    const Rate3 rate{true, grid3->bc.start, grid3->bc.step, grid3->bc.count, grid3->Fb};
    return fine_dfm_impl(radar, nullptr, echo, &g, rate, cell_begin, cell_count, precision, Y, P, stream);
}

int dsgrft_coarse_rm_fd_ex(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                           int32_t cell_begin, int32_t cell_count, grft_band band, grft_c32 *Z, void *stream) {
    if (!radar_ok(radar) || !echo || !Z || !dsgrid_ok(grid, radar) || cell_begin < 0 || cell_count < 0 ||
        (long)cell_begin + cell_count > (long)grid->vc.count * grid->ac.count ||
        (band != GRFT_BAND_BASEBAND && band != GRFT_BAND_POSITIVE))
        return GRFT_EINVAL;
    const int N = radar->N;
    if (N < 2 || N > 8192 || (N & (N - 1)) != 0) return GRFT_EUNSUPPORTED;
    if (cell_count == 0) return GRFT_OK;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    const RadarD R = radar_d(*radar);
    const size_t rho_bytes = align_up((size_t)cell_count * R.M * sizeof(int32_t));
    const size_t w_bytes = align_up((size_t)cell_count * R.M * sizeof(float2));
    const size_t s_bytes = align_up((size_t)R.M * N * sizeof(float2));
    unsigned char *ws = (unsigned char *)workspace(c, rho_bytes + w_bytes + s_bytes);
    if (!ws) return GRFT_ENOMEM;
    int32_t *rho = (int32_t *)ws;
    float2 *w = (float2 *)(ws + rho_bytes);
    float2 *S = (float2 *)(ws + rho_bytes + w_bytes);
    if ((e = launch_coarse_tables(c, R, *grid, cell_begin, cell_count, rho, w))) return e;
    if ((e = launch_range_fft(c, R, (const float2 *)echo, S))) return e;
    return launch_rm_fd(c, R, *grid, cell_begin, cell_count, S, w, (float2 *)Z, band == GRFT_BAND_POSITIVE);
}

int dsgrft_coarse_rm_fd(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                        int32_t cell_begin, int32_t cell_count, grft_c32 *Z, void *stream) {
    return dsgrft_coarse_rm_fd_ex(radar, echo, grid, cell_begin, cell_count, GRFT_BAND_BASEBAND, Z, stream);
}

int dsgrft_fine_dfm_fd(const grft_radar *radar, const grft_c32 *Z, const grft_dsgrid *grid, int32_t cell_begin,
                       int32_t cell_count, grft_band band, grft_precision precision, grft_c32 *Y, float *P,
                       void *stream) {
    if (!radar_ok(radar) || !Z || !grid || (band != GRFT_BAND_BASEBAND && band != GRFT_BAND_POSITIVE))
        return GRFT_EINVAL;
    grft_dsgrid g = *grid;
    if (band == GRFT_BAND_POSITIVE) {        // fine offsets scaled by 1 + B_r / (2 f_c), B_r = c / (2 dr)
        const double s = 1.0 + radar->c_mps / (2.0 * radar->dr_m) / (2.0 * radar->fc_hz);
        g.vc.step *= s;
        g.ac.step *= s;
    }
    return dsgrft_fine_dfm(radar, Z, nullptr, &g, cell_begin, cell_count, precision, Y, P, stream);
}

int dsgrft_fine_dfm_fft(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                        int32_t cell_begin, int32_t cell_count, grft_c32 *Y, float *P, void *stream) {
    if (!radar_ok(radar) || !echo || (!Y && !P) || !dsgrid_ok(grid, radar) || cell_begin < 0 ||
        cell_count < 0 || (long)cell_begin + cell_count > (long)grid->vc.count * grid->ac.count ||
        cell_count > 65535)
        return GRFT_EINVAL;
    // transform length: the fine velocity step must be lambda PRF / (2 L) exactly
    const double Lr = radar->c_mps * radar->prf_hz * grid->Fv / (2.0 * radar->fc_hz * grid->vc.step);
    const int L = (int)std::lround(Lr);
    if (!std::isfinite(Lr) || (L != 256 && L != 512) || std::fabs(Lr - L) > 1e-6 * L || radar->M > L ||
        grid->Fv > L || (grid->Fv % 2) != 0)
        return GRFT_EUNSUPPORTED;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    const RadarD R = radar_d(*radar);
    const size_t rho_bytes = align_up((size_t)cell_count * R.M * sizeof(int32_t));
    const size_t w_bytes = align_up((size_t)cell_count * R.M * sizeof(float2));
    const size_t e0_bytes = align_up((size_t)grid->r0_count * sizeof(float2));
    const size_t ch_bytes = align_up((size_t)grid->Fa * L * sizeof(float2));
    unsigned char *ws = (unsigned char *)workspace(c, rho_bytes + w_bytes + e0_bytes + ch_bytes);
    if (!ws) return GRFT_ENOMEM;
    int32_t *rho = (int32_t *)ws;
    float2 *w = (float2 *)(ws + rho_bytes);
    float2 *e0 = (float2 *)(ws + rho_bytes + w_bytes);
    float2 *chirp = (float2 *)(ws + rho_bytes + w_bytes + e0_bytes);
    if ((e = launch_coarse_tables(c, R, *grid, cell_begin, cell_count, rho, w))) return e;
    if ((e = launch_range_phase(c, R, grid->r0_begin, grid->r0_count, e0))) return e;
    if ((e = launch_gft_chirp(c, R, *grid, L, chirp))) return e;
    DsOut out;
    out.Y = (float2 *)Y;
    out.P = P;
    out.cell_begin = cell_begin;
    out.i0 = cell_begin / grid->ac.count;
    out.na_c = grid->ac.count;
    out.Fv = grid->Fv;
    out.Fa = grid->Fa;
    return launch_ds_fft(c, R, (const float2 *)echo, *grid, cell_count, rho, w, chirp, e0, L, out);
}

namespace {

bool pow2_in(int x, int lo, int hi) { return x >= lo && x <= hi && (x & (x - 1)) == 0; }

// A KT grid: coarse velocity axis = folding factor q, vc.step = V_a, vc.start = q_min V_a.
bool ktgrid_ok(const grft_dsgrid *g, const grft_radar *r) {
    if (!dsgrid_ok(g, r)) return false;
    const double va = r->c_mps / r->fc_hz * r->prf_hz / 2.0;
    const double q = g->vc.start / va;
    return std::fabs(g->vc.step - va) <= 1e-9 * va && std::fabs(q - std::rint(q)) <= 1e-6;
}

int kt_sizes(const grft_radar *r) {
    return pow2_in(r->M, 16, 2048) && pow2_in(r->N, 4, 8192) ? GRFT_OK : GRFT_EUNSUPPORTED;
}

bool cells_ok(const grft_dsgrid *g, int32_t cell_begin, int32_t cell_count) {
    return cell_begin >= 0 && cell_count >= 0 &&
           (long)cell_begin + cell_count <= (long)g->vc.count * g->ac.count;
}

// Fine stage of a KT grid: transform length L = Fv, M <= L.
int kt_fine_length(const grft_radar *r, const grft_dsgrid *g) {
    const int L = g->Fv;
    return (L == 64 || L == 128 || L == 256 || L == 512) && r->M <= L ? L : 0;
}

int kt_fine(const Ctx &c, const RadarD &R, const float2 *Z, const grft_dsgrid &g, int cell_begin, int cell_count,
            int L, const float2 *chirp, float2 *Y, float *P) {
    DsOut out;
    out.Y = Y;
    out.P = P;
    out.cell_begin = cell_begin;
    out.i0 = cell_begin / g.ac.count;
    out.na_c = g.ac.count;
    out.Fv = g.Fv;
    out.Fa = g.Fa;
    return launch_ds_fft_z(c, R, Z, g, cell_count, chirp, L, out);
}

}  // namespace

int dskt_keystone(const grft_radar *radar, const grft_c32 *echo, grft_c32 *Skt, void *stream) {
    if (!radar_ok(radar) || !echo || !Skt) return GRFT_EINVAL;
    int e = kt_sizes(radar);
    if (e) return e;
    Ctx c;
    if ((e = make_ctx(stream, c))) return e;
    const RadarD R = radar_d(*radar);
    float2 *S = (float2 *)workspace(c, (size_t)R.M * R.N * sizeof(float2));
    if (!S) return GRFT_ENOMEM;
    if ((e = launch_range_fft(c, R, (const float2 *)echo, S))) return e;
    return launch_keystone(c, R, S, (float2 *)Skt);
}

int dskt_coarse_rm(const grft_radar *radar, const grft_c32 *Skt, const grft_dsgrid *grid, int32_t cell_begin,
                   int32_t cell_count, grft_c32 *Z, void *stream) {
    if (!radar_ok(radar) || !Skt || !Z || !ktgrid_ok(grid, radar) || !cells_ok(grid, cell_begin, cell_count))
        return GRFT_EINVAL;
    int e = kt_sizes(radar);
    if (e) return e;
    if (cell_count == 0) return GRFT_OK;
    Ctx c;
    if ((e = make_ctx(stream, c))) return e;
    return launch_rm_kt(c, radar_d(*radar), *grid, cell_begin, cell_count, (const float2 *)Skt, (float2 *)Z);
}

int dskt_fine_dfm_fft(const grft_radar *radar, const grft_c32 *Z, const grft_dsgrid *grid, int32_t cell_begin,
                      int32_t cell_count, grft_c32 *Y, float *P, void *stream) {
    if (!radar_ok(radar) || !Z || (!Y && !P) || !ktgrid_ok(grid, radar) || !cells_ok(grid, cell_begin, cell_count) ||
        cell_count > 65535)
        return GRFT_EINVAL;
    int e = kt_sizes(radar);
    if (e) return e;
    const int L = kt_fine_length(radar, grid);
    if (!L) return GRFT_EUNSUPPORTED;
    if (cell_count == 0) return GRFT_OK;
    Ctx c;
    if ((e = make_ctx(stream, c))) return e;
    const RadarD R = radar_d(*radar);
    float2 *chirp = (float2 *)workspace(c, (size_t)grid->Fa * L * sizeof(float2));
    if (!chirp) return GRFT_ENOMEM;
    if ((e = launch_gft_chirp(c, R, *grid, L, chirp))) return e;
    return kt_fine(c, R, (const float2 *)Z, *grid, cell_begin, cell_count, L, chirp, (float2 *)Y, P);
}

int dskt_mfp(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid, grft_c32 *Y, float *P,
             void *stream) {
    if (!radar_ok(radar) || !echo || (!Y && !P) || !ktgrid_ok(grid, radar)) return GRFT_EINVAL;
    int e = kt_sizes(radar);
    if (e) return e;
    const int L = kt_fine_length(radar, grid);
    if (!L) return GRFT_EUNSUPPORTED;
    Ctx c;
    if ((e = make_ctx(stream, c))) return e;
    const RadarD R = radar_d(*radar);
    const int nac = grid->ac.count;
    // whole folding-factor rows per chunk, the coarse output within the split budget
    const size_t row_bytes = (size_t)nac * R.M * grid->r0_count * sizeof(float2);
    long rows = (long)(split_budget() / row_bytes);
    if (rows < 1) rows = 1;
    if (rows > grid->vc.count) rows = grid->vc.count;
    if (rows * nac > 65535) rows = 65535 / nac;
    if (rows < 1) return GRFT_EUNSUPPORTED;
    const size_t ch_bytes = align_up((size_t)grid->Fa * L * sizeof(float2));
    const size_t kt_bytes = align_up((size_t)R.M * R.N * sizeof(float2));
    size_t z_bytes = align_up((size_t)rows * row_bytes);
    if (z_bytes < kt_bytes) z_bytes = kt_bytes;                 // the range spectra share it
    unsigned char *ws = (unsigned char *)workspace(c, ch_bytes + kt_bytes + z_bytes);
    if (!ws) return GRFT_ENOMEM;
    float2 *chirp = (float2 *)ws;
    float2 *Skt = (float2 *)(ws + ch_bytes);
    float2 *Z = (float2 *)(ws + ch_bytes + kt_bytes);
    if ((e = launch_range_fft(c, R, (const float2 *)echo, Z))) return e;
    if ((e = launch_keystone(c, R, Z, Skt))) return e;
    if ((e = launch_gft_chirp(c, R, *grid, L, chirp))) return e;
    const long slab = (long)grid->Fv * nac * grid->Fa * grid->r0_count;   // outputs per coarse row
    for (int i0 = 0; i0 < grid->vc.count; i0 += (int)rows) {
        const int n = (int)(i0 + rows <= grid->vc.count ? rows : grid->vc.count - i0);
        const int cb = i0 * nac, cc = n * nac;
        if ((e = launch_rm_kt(c, R, *grid, cb, cc, Skt, Z))) return e;
        if ((e = kt_fine(c, R, Z, *grid, cb, cc, L, chirp, Y ? (float2 *)Y + i0 * slab : nullptr,
                         P ? P + i0 * slab : nullptr)))
            return e;
    }
    return GRFT_OK;
}

int dsgrft_fine_dfm_batched(const grft_radar *radar, const grft_dsgrid *grid,
                            const grft_batch_item *items, int32_t n_items, grft_precision precision,
                            void *stream) {
    if (!radar || !grid || !items || n_items <= 0 || n_items > 256) return GRFT_EINVAL;
    if (precision != GRFT_BF16X3 && precision != GRFT_FP16X3 && precision != GRFT_FP16X1 &&
        precision != GRFT_FP16X2)
        return GRFT_EINVAL;
    int Mmax = 0, Nmax = 0;
    long rpad_max = 0;
    for (int i = 0; i < n_items; ++i) {
        const grft_batch_item &b = items[i];
        if (!b.echo || (!b.P && !b.Y) || b.M <= 0 || b.N <= 0 || b.r0_begin < 0 || b.r0_count <= 0 ||
            (long)b.r0_begin + b.r0_count > b.N)
            return GRFT_EINVAL;
        if (b.M > Mmax) Mmax = b.M;
        if (b.N > Nmax) Nmax = b.N;
        if (ds_tc_r0_pad(b.r0_count) > rpad_max) rpad_max = ds_tc_r0_pad(b.r0_count);
    }
    grft_radar rmax = *radar;
    rmax.M = Mmax;
    rmax.N = Nmax;
    grft_dsgrid g = *grid;
    g.r0_begin = 0;
    g.r0_count = Nmax;
    if (!radar_ok(&rmax) || !dsgrid_ok(&g, &rmax)) return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    const RadarD R = radar_d(rmax);            // tables for Mmax pulses and bins [0, Nmax)
    const int ncell = g.vc.count * g.ac.count;
    const int F = g.Fv * g.Fa;
    const int Fpad = (F + 127) / 128 * 128;
    const int Mpad = (Mmax + 31) / 32 * 32;
    const size_t rho_bytes = align_up((size_t)ncell * Mmax * sizeof(int32_t));
    const size_t w_bytes = align_up((size_t)ncell * Mmax * sizeof(float2));
    const size_t e0_bytes = align_up((size_t)Nmax * sizeof(float2));
    const size_t d_bytes = align_up((size_t)2 * Fpad * 2 * Mpad * sizeof(uint16_t));
    const long row_bytes = 2L * Mpad * (long)sizeof(uint16_t);
    long total_rows = 0;
    for (int i = 0; i < n_items; ++i) total_rows += (long)ncell * ds_tc_r0_pad(items[i].r0_count);
    int nbuf = 1;
    // more items than one launch holds: rounds are forced, so keep two buffers
    long z_rows = split_rows(total_rows, rpad_max, row_bytes, nbuf, n_items > DS_TC_MAX_ITEMS);
    const size_t z_plane = align_up((size_t)z_rows * row_bytes);
    unsigned char *ws =
        (unsigned char *)workspace(c, rho_bytes + w_bytes + e0_bytes + 2 * d_bytes + 2 * nbuf * z_plane);
    if (!ws) return GRFT_ENOMEM;
    int32_t *rho = (int32_t *)ws;
    float2 *w = (float2 *)(ws + rho_bytes);
    float2 *e0 = (float2 *)(ws + rho_bytes + w_bytes);
    unsigned char *dptr = ws + rho_bytes + w_bytes + e0_bytes;
    uint16_t *Bhi = (uint16_t *)dptr, *Blo = (uint16_t *)(dptr + d_bytes);
    unsigned char *zp = dptr + 2 * d_bytes;
    uint16_t *const Zhi[2] = {(uint16_t *)zp, nbuf > 1 ? (uint16_t *)(zp + 2 * z_plane) : nullptr};
    uint16_t *const Zlo[2] = {(uint16_t *)(zp + z_plane), nbuf > 1 ? (uint16_t *)(zp + 3 * z_plane) : nullptr};
    const bool fp16 = precision_fp16(precision);
    const int nprod = precision_nprod(precision);
    if ((e = launch_coarse_tables(c, R, g, 0, ncell, rho, w))) return e;
    if ((e = launch_range_phase(c, R, 0, Nmax, e0))) return e;
    if ((e = fill_dechirp(c, R, g, kNoRate, precision, (unsigned char *)Bhi))) return e;
    (void)Blo;
    (void)fp16;
    DsTcItem list[256];
    for (int i = 0; i < n_items; ++i) {
        const grft_batch_item &b = items[i];
        DsTcItem &it = list[i];
        it.echo = (const float2 *)b.echo;
        it.Z = nullptr;
        it.P = b.P;
        it.Y = (float2 *)b.Y;
        it.e0 = e0 + b.r0_begin;
        it.M = b.M;
        it.N = b.N;
        it.r0_begin = b.r0_begin;
        it.r0_count = b.r0_count;
        it.cell_begin = 0;
        it.cell_count = ncell;
        it.i0 = 0;
    }
    return launch_ds_tc(c, list, n_items, g, rho, w, 0, Mmax, Bhi, Blo, Mpad, fp16, nprod, Zhi, Zlo, z_rows);
}

int detect_peaks(const float *P, int32_t nv, int32_t na, int32_t nr0, const grft_cfar *cfar,
                 const grft_grid *axes, double dr_m, int32_t K, grft_det *out, int32_t *n_out,
                 void *stream) {
    if (!P || !cfar || !n_out || nv <= 0 || na <= 0 || nr0 <= 0 || K < 0 || (K > 0 && !out))
        return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    return launch_detect(c, P, nv, na, nr0, *cfar, axes, dr_m, K, out, n_out);
}

int detect_peaks_begin(void *stream) {
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    return launch_detect_begin(c);
}

int detect_peaks_add(const float *P, int32_t nv, int32_t na, int32_t nr0, int32_t v_lo, int32_t v_hi,
                     int64_t v_base, const grft_cfar *cfar, void *stream) {
    if (!P || !cfar || nv <= 0 || na <= 0 || nr0 <= 0 || v_lo < 0 || v_hi > nv || v_lo > v_hi || v_base < 0 ||
        (v_base + (int64_t)nv) * na * (int64_t)nr0 >= ((int64_t)1 << 62))
        return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    return launch_detect_scan(c, P, nv, na, nr0, v_lo, v_hi, (long long)v_base * na * nr0, *cfar);
}

int detect_peaks_end(int32_t na, int32_t nr0, const grft_grid *axes, double dr_m, int32_t K, grft_det *out,
                     int32_t *n_out, void *stream) {
    if (!n_out || na <= 0 || nr0 <= 0 || K < 0 || (K > 0 && !out)) return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    return launch_detect_select(c, na, nr0, axes, dr_m, K, out, n_out);
}

int detect_merge(const grft_det *lists, const int32_t *totals, int32_t n_lists, int32_t K_in, int32_t K,
                 grft_det *out, int32_t *n_out, void *stream) {
    if (!lists || !totals || !n_out || n_lists <= 0 || K_in < 0 || K < 0 || (K > 0 && !out)) return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    return launch_detect_merge(c, lists, totals, n_lists, K_in, K, out, n_out);
}

int dsgrft_detect(const grft_radar *radar, const grft_c32 *echo, const grft_dsgrid *grid,
                  grft_precision precision, const grft_cfar *cfar, int32_t K, grft_det *out, int32_t *n_out,
                  void *stream) {
    if (!radar_ok(radar) || !echo || !dsgrid_ok(grid, radar) || !precision_ok(precision) || !cfar || !n_out ||
        K < 0 || (K > 0 && !out))
        return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    const int nac = grid->ac.count, nvc = grid->vc.count, Fv = grid->Fv;
    const long na = (long)nac * grid->Fa, nr0 = grid->r0_count;
    if (na > 0x7fffffffL) return GRFT_EINVAL;
    const size_t row = (size_t)na * nr0;              // floats per fine-v row of the map
    const size_t slab = (size_t)(Fv + 2) * row;       // one coarse-v row of cells + a halo row each side
    // the dechirp operand is the same for every slab: computed once, after the two slabs
    const RadarD R = radar_d(*radar);
    const size_t d_bytes = dechirp_plane_bytes(R, *grid, kNoRate, precision != GRFT_FP32);
    const size_t slab_bytes = align_up(2 * slab * sizeof(float));
    unsigned char *ws = (unsigned char *)workspace(c, slab_bytes + 2 * d_bytes, WS_SLAB);
    if (!ws) return GRFT_ENOMEM;
    float *buf = (float *)ws;
    unsigned char *D = ws + slab_bytes;
    float *B[2] = {buf, buf + slab};
    if ((e = fill_dechirp(c, R, *grid, kNoRate, precision, D))) return e;
    auto slab_map = [&](int i, float *dst) {          // the power map of coarse-v row i
        return fine_dfm_impl(radar, nullptr, echo, grid, kNoRate, i * nac, nac, precision, nullptr, dst, stream, D);
    };
    if ((e = launch_detect_begin(c))) return e;
    if ((e = slab_map(0, B[0] + row))) return e;
    for (int i = 0; i < nvc; ++i) {
        float *cur = B[i & 1], *nxt = B[(i + 1) & 1];
        const bool has_next = i + 1 < nvc;
        if (has_next) {
            // slab i + 1 (it may overwrite nxt: the scan of slab i - 1 that read nxt is ordered
            // before it on the stream), then the halo rows that slabs i and i + 1 share
            if ((e = slab_map(i + 1, nxt + row))) return e;
            if (cudaMemcpyAsync(cur + (size_t)(Fv + 1) * row, nxt + row, row * sizeof(float),
                                cudaMemcpyDeviceToDevice, c.stream) != cudaSuccess ||
                cudaMemcpyAsync(nxt, cur + (size_t)Fv * row, row * sizeof(float), cudaMemcpyDeviceToDevice,
                                c.stream) != cudaSuccess)
                return GRFT_ECUDA;
        }
        const int v_lo = i > 0 ? 1 : 0;                // row 0 of cur is the previous slab's last row
        const float *P = i > 0 ? cur : cur + row;
        const int nv = Fv + v_lo + (has_next ? 1 : 0);
        const long long v_base = (long long)i * Fv - v_lo;
        if ((e = launch_detect_scan(c, P, nv, (int)na, (int)nr0, v_lo, v_lo + Fv, v_base * na * nr0, *cfar)))
            return e;
    }
    grft_grid axes = {};                              // the plain grid of the same hypotheses
    axes.r0_begin = grid->r0_begin;
    axes.r0_count = grid->r0_count;
    axes.v.start = grid->vc.start - 0.5 * grid->vc.step;
    axes.v.step = grid->vc.step / Fv;
    axes.v.count = nvc * Fv;
    axes.a.start = grid->ac.start - 0.5 * grid->ac.step;
    axes.a.step = grid->ac.step / grid->Fa;
    axes.a.count = (int32_t)na;
    return launch_detect_select(c, (int)na, (int)nr0, &axes, radar->dr_m, K, out, n_out);
}

int dsgrft_backward(const grft_radar *radar, const grft_c32 *echo, int32_t K, const double *theta,
                    grft_gather gather, const float *grad_P, float *P, grft_c32 *Y,
                    double *grad_theta, grft_c32 *grad_s, void *stream) {
    if (!radar_ok(radar) || !echo || K < 0 || (K > 0 && !theta) ||
        (gather != GRFT_GATHER_NEAREST && gather != GRFT_GATHER_LINEAR))
        return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    return launch_backward(c, radar_d(*radar), (const float2 *)echo, K, theta, (int)gather, grad_P, P,
                           (float2 *)Y, grad_theta, (float2 *)grad_s);
}

int dsgrft_refine(const grft_radar *radar, const grft_c32 *echo, int32_t K, double *theta,
                  const double *cell, int32_t steps, grft_gather gather, float *P_out,
                  void *stream) {
    if (!radar_ok(radar) || !echo || K < 0 || (K > 0 && (!theta || !P_out)) || !cell || steps < 0 ||
        (gather != GRFT_GATHER_NEAREST && gather != GRFT_GATHER_LINEAR))
        return GRFT_EINVAL;
    for (int j = 0; j < 3; ++j)
        if (!std::isfinite(cell[j]) || cell[j] <= 0) return GRFT_EINVAL;
    Ctx c;
    int e = make_ctx(stream, c);
    if (e) return e;
    return launch_refine(c, radar_d(*radar), (const float2 *)echo, K, theta, cell, steps, (int)gather,
                         P_out);
}

}  // extern "C"
