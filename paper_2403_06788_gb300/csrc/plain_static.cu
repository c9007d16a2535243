// grft_plain_static: plain GRFT that allocates no device memory.
//
// Who needs it: callers that must not call cudaMalloc (or any allocating routine) once
// they are running, such as a radar processing loop that owns a fixed memory budget and
// must not wait on an allocator, or a process whose device memory is managed by someone
// else's pool.  grft_plain() takes its bin/phase tables from
// a library workspace that is allocated (and grown) on first use; this variant keeps them
// in a fixed array that is part of the library image instead, so that the only memory it
// touches is the caller's (echo, Y, P) and that array.
//
// The array holds the range phases e0(n0) and the per-pulse bin shifts and phases of a
// chunk of hypotheses; the grid is processed chunk by chunk with the same kernels as
// grft_plain(), so the results are bit-identical to grft_plain().  Everything in the array
// is written before it is read in each call, so nothing has to start at zero.
#include "internal.cuh"

namespace grft {

namespace {

constexpr size_t kStaticScratchBytes = GRFT_PLAIN_STATIC_SCRATCH_BYTES;

// Device-resident scratch, allocated with the module; every GPU that loads the library
// holds it until the process exits.
static __device__ __align__(256) unsigned char g_plain_scratch[kStaticScratchBytes];

constexpr int kMaxDev = 64;
void *g_scratch_addr[kMaxDev] = {nullptr};   // device address of g_plain_scratch per device

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

}  // namespace grft

using namespace grft;

extern "C" int grft_plain_static(const grft_radar *radar, const grft_c32 *echo, const grft_grid *grid,
                                 grft_c32 *Y, float *P, void *stream) {
    if (!radar_ok(radar) || !echo || !grid || (!Y && !P) || !axis_ok(grid->v) || !axis_ok(grid->a) ||
        grid->r0_count <= 0 || grid->r0_begin < 0 || (long)grid->r0_begin + grid->r0_count > radar->N)
        return GRFT_EINVAL;
    // size limits of the fixed scratch: the range phases plus at least one group of 8
    // hypotheses' tables must fit
    const size_t e0_bytes = align256((size_t)grid->r0_count * sizeof(float2));
    const size_t per_hyp = (size_t)radar->M * (sizeof(int32_t) + sizeof(float2));
    if (e0_bytes + 8 * per_hyp + 512 > kStaticScratchBytes) return GRFT_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return GRFT_ECUDA;
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return GRFT_ECUDA;
    if (major * 10 + minor != 103) return GRFT_EUNSUPPORTED;
    // set-up, once per device, with that device current: the host-side name of the array is
    // not a device address, so fetch the address the kernels must use
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_plain_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return GRFT_ECUDA;
        }
        g_scratch_addr[dev] = ptr;
    }
    unsigned char *base = static_cast<unsigned char *>(g_scratch_addr[dev]);

    Ctx c;
    c.device = dev;
    c.stream = (cudaStream_t)stream;
    c.status = nullptr;          // these kernels have no device-side waits to report
    c.wait_limit = 0;
    c.num_sms = 0;
    const RadarD R = radar_d(*radar);
    const long nh_total = (long)grid->v.count * grid->a.count;
    long chunk = (long)((kStaticScratchBytes - e0_bytes - 512) / per_hyp);
    chunk = chunk >= 16 ? chunk / 16 * 16 : chunk / 8 * 8;   // at least 8 (checked above)
    if (chunk > (1L << 18)) chunk = 1L << 18;   // the launch limit grft_plain applies (grid y <= 65535)
    if (chunk > nh_total) chunk = nh_total;
    float2 *e0 = reinterpret_cast<float2 *>(base);
    int32_t *rho = reinterpret_cast<int32_t *>(base + e0_bytes);
    float2 *w = reinterpret_cast<float2 *>(base + e0_bytes + align256((size_t)chunk * R.M * sizeof(int32_t)));
    int e;
    if ((e = launch_range_phase(c, R, grid->r0_begin, grid->r0_count, e0))) return e;
    for (long h0 = 0; h0 < nh_total; h0 += chunk) {
        const int nh = (int)(nh_total - h0 < chunk ? nh_total - h0 : chunk);
        if ((e = launch_plain_tables(c, R, *grid, h0, nh, rho, w))) return e;
        if ((e = launch_plain(c, R, (const float2 *)echo, *grid, h0, nh, rho, w, e0, (float2 *)Y, P)))
            return e;
    }
    return GRFT_OK;
}
