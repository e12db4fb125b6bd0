// vgrid_trace_noalloc: tau per ray without allocating device memory.
//
// Some callers cannot call cudaMalloc: their device memory belongs to another
// allocator with a fixed budget, or they run latency-bound loops that must
// not take the implicit device synchronisation of cudaMalloc/cudaFree. For
// them the work buffers of the traversal (start cells, work counter,
// counters, ray-set descriptor) live in one file-scope device array of fixed
// size instead of buffers allocated per grid. The array exists once per
// device that loads the library and stays until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"
#include "kernels.h"
#include "vgrid.h"

namespace {

// layout of the scratch array
constexpr size_t kQueueOff = 0;     // unsigned long long work counter
constexpr size_t kStatsOff = 64;    // StatsDev
constexpr size_t kSetOff = 256;     // RaySetDev
constexpr size_t kStartOff = 512;   // RayPrep start record per ray
static_assert(sizeof(StatsDev) <= kSetOff - kStatsOff, "stats slot");
static_assert(sizeof(RaySetDev) <= kStartOff - kSetOff, "ray-set slot");
static_assert(sizeof(RayPrep) == 64, "start record");
static_assert(kStartOff + sizeof(RayPrep) * (size_t)VGRID_NOALLOC_MAX_RAYS == (size_t)VGRID_NOALLOC_SCRATCH_BYTES, "size");

static __device__ __align__(256) unsigned char vg_noalloc_scratch[VGRID_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices];

// Device address of the scratch array on the current device (looked up once
// per device; the host-side name of the array is not a device address).
cudaError_t scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, vg_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

int fail(int code, const std::string &m) {
    vg::set_error(m);  // read back through vgrid_last_error()
    return code;
}

}  // namespace

extern "C" int vgrid_trace_noalloc(vgrid_t *g, const double *origin, const double *dir, int64_t N, int precision,
                                   void *tau, int32_t *ray_status, vgrid_stream_t stream) {
    vg::GridView v;
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (vg::grid_view(g, &v) != 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    if (precision != VGRID_FP64 && precision != VGRID_FP32_RECHECK && precision != VGRID_FP32_EXACT)
        return fail(VGRID_ERR_ARG, "bad precision");
    if (N < 0 || (N > 0 && (!origin || !dir || !tau))) return fail(VGRID_ERR_ARG, "bad rays or tau");
    if (N > VGRID_NOALLOC_MAX_RAYS)
        return fail(VGRID_ERR_ARG, "N = " + std::to_string(N) + " exceeds VGRID_NOALLOC_MAX_RAYS = " +
                                       std::to_string(VGRID_NOALLOC_MAX_RAYS));
    if (N == 0) return VGRID_OK;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return fail(VGRID_ERR_CUDA, "no CUDA device");
    if (prev != v.device && cudaSetDevice(v.device) != cudaSuccess) return fail(VGRID_ERR_CUDA, "cudaSetDevice");
    int rc = VGRID_OK;
    do {
        unsigned char *base = nullptr;
        cudaError_t e = scratch_address(v.device, &base);
        if (e != cudaSuccess) {
            rc = fail(VGRID_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            break;
        }
        auto *queue = reinterpret_cast<unsigned long long *>(base + kQueueOff);
        auto *stats = reinterpret_cast<StatsDev *>(base + kStatsOff);
        auto *dset = reinterpret_cast<RaySetDev *>(base + kSetOff);
        auto *start = reinterpret_cast<RayPrep *>(base + kStartOff);
        cudaStream_t s = (cudaStream_t)stream;
        const int fp64 = precision == VGRID_FP64;
        RaySetDev set{origin, dir, tau, ray_status, start, N, 0, 0, 0};
        // clears the counter and statistics left by the previous call
        if ((e = vg::launch_prepare(dset, set, queue, stats, s)) != cudaSuccess ||
            (e = vg::launch_locate(v.d_desc, dset, 1, N, fp64 ? vg::PREP_FP64 : vg::PREP_FP32, nullptr, v.sms,
                                   s)) != cudaSuccess) {
            rc = fail(VGRID_ERR_CUDA, cudaGetErrorString(e));
            break;
        }
        if (fp64) v.lanes_per_ray = v.fp64_lanes_per_ray;
        if (precision == VGRID_FP32_EXACT) v.lanes_per_ray = 1;  // its kernels take one lane per ray
        vg::KernelSet ks{};
        switch (v.lanes_per_ray) {
            case 1: vg::kernel_table_lpr1(ks); break;
            case 2: vg::kernel_table_lpr2(ks); break;
            case 8: vg::kernel_table_lpr8(ks); break;
            default: vg::kernel_table_lpr4(ks); break;
        }
        const void *fn = ks.fn[precision == VGRID_FP32_EXACT ? 2 : fp64][vg::MODE_TAU];
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, v.block, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        if (v.blocks_per_sm > 0 && v.blocks_per_sm < per_sm) per_sm = v.blocks_per_sm;
        int64_t blocks = (int64_t)per_sm * v.sms;
        const int64_t need = (N * v.lanes_per_ray + v.block - 1) / v.block;
        if (need < blocks) blocks = need;
        vg::TraceArgs a{};
        a.grids = v.d_desc;
        a.sets = dset;
        a.nsets = 1;
        a.total = N;
        a.queue = queue;
        a.stats = stats;
        a.g1 = v.hd;
        a.s1 = set;
        void *args[] = {&a};
        e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(v.block), args, 0, s);
        if (e != cudaSuccess) rc = fail(VGRID_ERR_CUDA, std::string("cudaLaunchKernel: ") + cudaGetErrorString(e));
    } while (0);
    if (prev != v.device) cudaSetDevice(prev);
    return rc;
}

