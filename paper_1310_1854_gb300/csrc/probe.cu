// Bandwidth ceilings of the memory level that serves the traversal, measured
// on the device in the calling process (no device setting is changed).
//
//  * stream: every thread reads 32-byte pairs (one 256-bit load each, the
//    load the traversal uses) of a buffer, strided over the whole grid, for
//    a number of passes; a buffer smaller than L2 stays there after the
//    first pass, so the later passes measure L2 read bandwidth.
//  * chase: every thread follows a chain of 288-byte blocks (nine 32-byte
//    pairs, the size of an average cell block of the float32 traversal),
//    reading all nine pairs of a block and taking the next block's index
//    from the data of its first pair, so each block waits for the previous
//    one as a cell of the traversal waits for the winner of the last one.
//    Blocks are chosen by a multiplicative hash over the buffer (random
//    positions), at full occupancy.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.h"
#include "kernels.h"
#include "vgrid.h"

namespace {

__device__ __forceinline__ void ld_pair(const float4 *p, uint4 &a, uint4 &b) {
    asm volatile("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                 : "l"(p));
}

__global__ void fill_kernel(uint32_t *p, int64_t n, uint32_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 0x9E3779B1u ^ seed;
        x ^= x >> 15;
        x *= 0x2C1B3C6Du;
        x ^= x >> 12;
        p[i] = x;
    }
}

// pairs: number of 32-byte pairs in the buffer
__global__ void __launch_bounds__(256) stream_kernel(const float4 *buf, int64_t pairs, int passes, uint32_t *sink) {
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; p++) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pairs; i += 4 * stride) {
            uint4 a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int64_t j = i + u * stride;
                if (j < pairs) ld_pair(buf + 2 * j, a[u], b[u]);
                else a[u] = b[u] = make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) acc ^= a[u].x ^ a[u].y ^ a[u].z ^ a[u].w ^ b[u].x ^ b[u].y ^ b[u].z ^ b[u].w;
        }
    }
    if (acc == 0x12345678u) sink[0] = acc;  // keeps the loads
}

constexpr int kChasePairs = 9;  // 288-byte blocks

__global__ void __launch_bounds__(256) chase_kernel(const float4 *buf, int64_t nblocks, int steps, uint32_t *sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    uint64_t blk = ((uint64_t)(tid * 0x9E3779B1u) * (uint64_t)nblocks) >> 32;
    for (int s = 0; s < steps; s++) {
        const float4 *p = buf + 2 * kChasePairs * (int64_t)blk;
        uint4 a[kChasePairs], b[kChasePairs];
#pragma unroll
        for (int u = 0; u < kChasePairs; u++) ld_pair(p + 2 * u, a[u], b[u]);
#pragma unroll
        for (int u = 0; u < kChasePairs; u++) acc ^= a[u].y ^ a[u].z ^ b[u].x ^ b[u].w;
        // the next block depends on this block's data
        const uint32_t h = (a[0].x ^ (uint32_t)s) * 0x9E3779B1u + tid;
        blk = ((uint64_t)h * (uint64_t)nblocks) >> 32;
    }
    if (acc == 0x12345678u) sink[0] = acc;
}

int fail(int code, const std::string &m) {
    vg::set_error(m);
    return code;
}

}  // namespace

extern "C" int vgrid_probe_l2(int64_t bytes, int mode, double *gbs, vgrid_stream_t stream) {
    if (!gbs) return fail(VGRID_ERR_ARG, "gbs is NULL");
    if (mode != 0 && mode != 1) return fail(VGRID_ERR_ARG, "mode must be 0 (stream) or 1 (chase)");
    if (bytes < (int64_t)(1 << 20) || bytes > ((int64_t)1 << 32))
        return fail(VGRID_ERR_ARG, "bytes must lie in [1 MiB, 4 GiB]");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(VGRID_ERR_CUDA, "no CUDA device");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t unit = mode == 0 ? 32 : 32 * kChasePairs;
    const int64_t units = bytes / unit;
    void *buf = nullptr;
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = VGRID_OK;
    do {
        if (cudaMalloc(&buf, (size_t)(units * unit)) != cudaSuccess || cudaMalloc(&sink, 64) != cudaSuccess) {
            rc = fail(VGRID_ERR_NOMEM, "probe buffer");
            break;
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = fail(VGRID_ERR_CUDA, "cudaEventCreate");
            break;
        }
        const int64_t words = units * unit / 4;
        fill_kernel<<<std::min<int64_t>((words + 255) / 256, (int64_t)sms * 32), 256, 0, s>>>((uint32_t *)buf, words,
                                                                                             0x5bd1e995u);
        int per_sm = 1;
        const void *fn = mode == 0 ? (const void *)stream_kernel : (const void *)chase_kernel;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
        const int blocks = per_sm * sms;
        // about 8 GB per timed launch of the stream probe (a few hundred
        // microseconds from L2), so that launch and tail costs do not count
        const int passes = mode == 0 ? (int)std::min<int64_t>(4096, std::max<int64_t>(4, 8000000000LL / (units * unit))) : 0;
        const int steps = mode == 1 ? 64 : 0;
        double moved = 0;
        float ms = 0;
        for (int rep = 0; rep < 2; rep++) {  // the first launch warms L2 and the clocks
            cudaEventRecord(e0, s);
            if (mode == 0) {
                stream_kernel<<<blocks, 256, 0, s>>>((const float4 *)buf, units, passes, sink);
                moved = (double)passes * (double)(units * unit);
            } else {
                chase_kernel<<<blocks, 256, 0, s>>>((const float4 *)buf, units, steps, sink);
                moved = (double)blocks * 256.0 * steps * (double)unit;
            }
            cudaEventRecord(e1, s);
        }
        vg::count_launches(3);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = fail(VGRID_ERR_CUDA, std::string("probe: ") + cudaGetErrorString(e));
            break;
        }
        *gbs = moved / (ms * 1e-3) / 1e9;
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (buf) cudaFree(buf);
    return rc;
}
