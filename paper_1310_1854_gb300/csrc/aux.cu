// Auxiliary kernels of libvgrid: start-cell location (C(r), Sect. 2.3),
// per-call set-up, density reordering and the prefix sum that turns
// per-ray segment counts into offsets.
#include <algorithm>
#include <atomic>

#include "kernels.h"
#include "trace.cuh"

namespace vg {

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// Write the ray-set descriptor and clear the work counter and statistics
// (one thread; the descriptor travels as a kernel argument, so the call is
// stream-ordered and needs no host staging buffer). stats may be NULL.
__global__ void prepare_kernel(RaySetDev *d_set, RaySetDev set, unsigned long long *queue, StatsDev *stats) {
    if (d_set) *d_set = set;
    *queue = 0ull;
    if (!stats) return;  // counters keep adding up (host-pipelined chunks)
    unsigned long long *s = reinterpret_cast<unsigned long long *>(stats);
    for (int i = 0; i < (int)(sizeof(StatsDev) / sizeof(unsigned long long)); i++) s[i] = 0ull;
}

__global__ void put_grid_kernel(GridDev *d, GridDev g) { *d = g; }

cudaError_t launch_put_grid(GridDev *d, const GridDev &g, cudaStream_t s) {
    put_grid_kernel<<<1, 1, 0, s>>>(d, g);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_prepare(RaySetDev *d_set, const RaySetDev &set, unsigned long long *queue, StatsDev *stats,
                           cudaStream_t s) {
    prepare_kernel<<<1, 1, 0, s>>>(d_set, set, queue, stats);
    count_launches(1);
    return cudaGetLastError();
}

// Start records for every ray of every set. PREP_CELL32 / PREP_CELL64: C(r0)
// only, written as the caller's id to out_caller (no start record), with
// float32 (rechecked) or float64 distances;
// PREP_FP32: float32 form (cell, direction check, wall exit of Eq. 5 and the
// float pairs of origin and direction); PREP_FP64: float64 form (cell and
// direction check). The caller's id of the cell goes to out_caller if given.
// Held to five blocks of 256 threads per SM (48 registers, a few spilled):
// the kernel waits on its loads, and the extra warps hide more of that wait
// than the spilled bytes cost.
__global__ void __launch_bounds__(256, 5) locate_kernel(const GridDev *grids, const RaySetDev *sets, int nsets,
                                                     int64_t total, int prep, int32_t *out_caller, uint8_t *bin,
                                                     uint32_t *hist) {
    __shared__ uint32_t s_hist[kOrderBins];
    if (bin) {
        for (int b = threadIdx.x; b < kOrderBins; b += blockDim.x) s_hist[b] = 0u;
        __syncthreads();
    }
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int set = find_set(sets, nsets, w);
        const RaySetDev &rs = sets[set];
        const int64_t li = w - rs.first;
        const GridDev *gp = grids + rs.grid;
        const double *o = rs.origin + 3 * li;
        const LocPt P = loc_point(__ldg(o), __ldg(o + 1), __ldg(o + 2));
        // float32 distances with the proven float64 fallback give exactly the
        // float64 argmin, so both traversal forms start that way; only
        // vgrid_locate's float64 mode (PREP_CELL64) scans in float64
        int m = locate_point<true>(gp, P, prep != PREP_CELL64, nullptr);
        if (out_caller) out_caller[w] = m >= 0 ? __ldg(&gp->perm[m]) : -1;
        if (prep == PREP_CELL32 || prep == PREP_CELL64) continue;
        RayPrep *out = rs.start + li;
        const double *d = rs.dir + 3 * li;
        const double k[3] = {__ldg(d), __ldg(d + 1), __ldg(d + 2)};
        RayPrep p;
        for (int c = 0; c < 3; c++) {
            p.r0_hi[c] = P.h[c];
            p.r0_lo[c] = P.l[c];
            split_pair(k[c], p.k_hi[c], p.k_lo[c]);
        }
        // |k.k - 1| <= 2.000001e-6, in float32 from the pairs (error below
        // 1e-6) unless that is too close to call, then in float64
        float kkf = 0.0f;
        for (int c = 0; c < 3; c++)
            kkf = __fmaf_rn(p.k_hi[c], p.k_hi[c], __fmaf_rn(2.0f * p.k_hi[c], p.k_lo[c], kkf));
        const float dev = fabsf(__fsub_rn(kkf, 1.0f));
        bool unit;
        if (dev <= 1.000001e-6f) {
            unit = true;
        } else if (dev > 3.000001e-6f || !(dev == dev)) {
            unit = false;
        } else {
            const double kk = __dadd_rn(__dadd_rn(__dmul_rn(k[0], k[0]), __dmul_rn(k[1], k[1])), __dmul_rn(k[2], k[2]));
            unit = fabs(kk - 1.0) <= 2.000001e-6;
        }
        if (!unit) m = -2;
        const bool fp64 = prep == PREP_FP64;  // the float64 form needs the cell only
        if (fp64 && !bin) {
            out->cell = m;
            continue;
        }
        // the float32 traversal starts from the cell's relative block
        p.cell = m >= 0 && !fp64 ? __float_as_int(__ldg(&gp->site[m]).w) : m;
        // distance to the wall ahead (Eq. 5 for the walls the ray faces), as
        // a float pair: q1 = n/k rounded, the exact remainder n - q1 k by
        // fma, then q2 = remainder / k (relative error a few 2^-48); in a
        // spherical domain the sphere's exit from the origin in float64,
        // split into a float pair
        float th = 3.0e38f, tl = 0.0f;
        int wid = -1;
        if (gp->domain == VGRID_DOMAIN_SPHERE) {
            split_pair(sphere_exit64(gp, P.x, k), th, tl);
            wid = kSphereWall;
        }
        for (int c = 0; c < 3 && gp->domain != VGRID_DOMAIN_SPHERE; c++) {
            const uint64_t kb = dbits(k[c]);
            if ((kb << 1) == 0) continue;  // k_c = +-0
            const bool up = (kb >> 63) == 0;
            float nh, nl;
            split_pair(__dsub_rn(up ? gp->hi[c] : gp->lo[c], P.x[c]), nh, nl);
            const float kh = p.k_hi[c], kl = p.k_lo[c];
            const float q1 = __fdiv_rn(nh, kh);
            float rem = __fmaf_rn(-q1, kh, nh);
            rem = __fadd_rn(rem, __fmaf_rn(-q1, kl, nl));
            const float q2 = __fdiv_rn(rem, kh);
            float h, l;
            two_sum(q1, q2, h, l);
            if (h < th || (h == th && l < tl)) {
                th = h;
                tl = l;
                wid = up ? -(2 * c + 2) : -(2 * c + 1);
            }
        }
        if (!(th >= 0.0f) || th > 1.0e38f) {  // start on the boundary facing out (or k = 0)
            th = 0.0f;
            tl = 0.0f;
        } else if (th == 0.0f && tl < 0.0f) {
            tl = 0.0f;
        }
        p.wall = wid;
        p.tmax_hi = th;
        p.tmax_lo = tl;
        if (fp64) {
            out->cell = m;
        } else {
            const float4 *src = reinterpret_cast<const float4 *>(&p);
            float4 *dst = reinterpret_cast<float4 *>(out);
            for (int q = 0; q < 4; q++) dst[q] = src[q];
        }
        if (bin) {
            // estimated crossings: (sites per volume)^(1/3) integrated along
            // the in-box segment [0, t_max] with 8 midpoint samples
            int b = 0;
            if (m >= 0 && th > 0.0f) {
                const float dt = th * 0.125f;
                float acc = 0.0f;
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const float t = (i + 0.5f) * dt;
                    int idx = 0;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        const float x = __fmaf_rn(t, p.k_hi[c], P.h[c]);
                        const int ic = __float2int_rz(__fmul_rn(__fsub_rn(x, gp->flo_hi[c]), gp->dscale[c]));
                        idx = idx * gp->ddim[c] + max(0, min(ic, gp->ddim[c] - 1));
                    }
                    acc += __ldg(gp->dens + idx);
                }
                const int S = max(1, gp->ospatial), NL = kOrderBins / S;
                const float Q = S == 1 ? 4.0f : 2.0f;  // bins per octave of the estimate
                const int lb = max(0, min(NL - 1, __float2int_rz(Q * __log2f(1.0f + acc * dt))));
                b = lb * S + (S > 1 ? (int)(((int64_t)m * S) / gp->M) : 0);
            }
            bin[w] = (uint8_t)b;
            atomicAdd(&s_hist[b], 1u);
        }
    }
    if (bin) {
        __syncthreads();
        for (int b = threadIdx.x; b < kOrderBins; b += blockDim.x)
            if (s_hist[b]) atomicAdd(&hist[b], s_hist[b]);
    }
}

cudaError_t launch_locate_ordered(const GridDev *grids, const RaySetDev *sets, int nsets, int64_t total,
                                  const RayOrder &ord, int prep, int sms, cudaStream_t s) {
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    blocks = blocks < (int64_t)sms * 16 ? blocks : (int64_t)sms * 16;
    locate_kernel<<<(unsigned)blocks, 256, 0, s>>>(grids, sets, nsets, total, prep, nullptr, ord.bin, ord.hist);
    count_launches(1);
    return cudaGetLastError();
}

// cursor[b] = number of rays in longer bins (the longest bin goes first)
__global__ void order_scan_kernel(uint32_t *hist) {
    __shared__ uint32_t h[kOrderBins];
    const int b = threadIdx.x;
    h[b] = hist[b];
    __syncthreads();
    uint32_t sum = 0u;
    for (int q = b + 1; q < kOrderBins; q++) sum += h[q];
    hist[kOrderBins + b] = sum;
}

// order[cursor[bin[w]]++] = w in tiles of 2048 rays per block: ranks within
// the tile from shared-memory counters, then one global atomic per bin and
// tile reserves the tile's range (the order inside a bin is arbitrary)
constexpr int kScatterThreads = 256, kScatterPer = 8;
__global__ void __launch_bounds__(kScatterThreads) order_scatter_kernel(const uint8_t *__restrict__ bin,
                                                                        int64_t total, uint32_t *cursor,
                                                                        int32_t *__restrict__ order) {
    __shared__ uint32_t s_cnt[kOrderBins], s_base[kOrderBins];
    const int64_t tile = (int64_t)kScatterThreads * kScatterPer;
    for (int64_t t0 = blockIdx.x * tile; t0 < total; t0 += (int64_t)gridDim.x * tile) {
        if (threadIdx.x < kOrderBins) s_cnt[threadIdx.x] = 0u;
        __syncthreads();
        int b[kScatterPer];
        uint32_t r[kScatterPer];
#pragma unroll
        for (int j = 0; j < kScatterPer; j++) {
            const int64_t w = t0 + (int64_t)j * kScatterThreads + threadIdx.x;
            b[j] = w < total ? (int)__ldg(bin + w) : -1;
            r[j] = b[j] >= 0 ? atomicAdd(&s_cnt[b[j]], 1u) : 0u;
        }
        __syncthreads();
        if (threadIdx.x < kOrderBins)
            s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&cursor[threadIdx.x], s_cnt[threadIdx.x]) : 0u;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kScatterPer; j++) {
            const int64_t w = t0 + (int64_t)j * kScatterThreads + threadIdx.x;
            if (b[j] >= 0) order[s_base[b[j]] + r[j]] = (int32_t)w;
        }
        __syncthreads();
    }
}

cudaError_t launch_order(const RayOrder &ord, int64_t total, int sms, cudaStream_t s) {
    if (total <= 0) return cudaSuccess;
    order_scan_kernel<<<1, kOrderBins, 0, s>>>(ord.hist);
    count_launches(1);
    const int64_t tile = (int64_t)kScatterThreads * kScatterPer;
    int64_t blocks = (total + tile - 1) / tile;
    blocks = blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8;
    order_scatter_kernel<<<(unsigned)blocks, kScatterThreads, 0, s>>>(ord.bin, total, ord.hist + kOrderBins,
                                                                     ord.order);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_locate(const GridDev *grids, const RaySetDev *sets, int nsets, int64_t total, int prep,
                          int32_t *out_caller, int sms, cudaStream_t s) {
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    blocks = blocks < (int64_t)sms * 16 ? blocks : (int64_t)sms * 16;
    locate_kernel<<<(unsigned)blocks, 256, 0, s>>>(grids, sets, nsets, total, prep, out_caller, nullptr, nullptr);
    count_launches(1);
    return cudaGetLastError();
}

// rho (caller order) into the headers of both forms of the cell blocks
__global__ void permute_density_kernel(const float *__restrict__ rho_caller, const int32_t *__restrict__ perm,
                                       const float4 *__restrict__ site, int64_t M, float4 *cells, float4 *rel) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = __float_as_int(__ldg(&site[i]).w);
        const float v = __ldg(&rho_caller[__ldg(&perm[i])]);
        float4 *h1 = rel + f + 1;
        h1->y = v;
        cells[__float_as_int(h1->w)].z = v;
    }
}

cudaError_t launch_permute_density(const float *rho_caller, const int32_t *perm, const float4 *site, int64_t M,
                                   float4 *cells, float4 *rel, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    int64_t blocks = (M + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    permute_density_kernel<<<(unsigned)blocks, 256, 0, s>>>(rho_caller, perm, site, M, cells, rel);
    count_launches(1);
    return cudaGetLastError();
}

// Rays that start outside the box move to where they enter it: the slab
// test gives the parameter interval [t_in, t_out] in which the line is
// inside every slab; a ray with t_in <= t_out and t_out >= 0 starts at
// r0 + max(t_in, 0) k, clamped into the closed box against rounding. Rays
// inside are copied unchanged, rays that miss keep their outside origin.
// In a spherical domain a ray outside the ball (q = o.o - R^2 > 0, o = r0 -
// c) that meets it ahead (b = k.o < 0, b^2 - q >= 0) starts epsilon past the
// smaller root, q / (sqrt(b^2 - q) - b) + epsilon (no digits cancel), every
// operation rounded to nearest in this order.
__global__ void enter_kernel(const double *__restrict__ origin, const double *__restrict__ dir, int64_t N,
                             const GridDev *gp, double *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double r[3], k[3];
        bool in = true;
        for (int c = 0; c < 3; c++) {
            r[c] = origin[3 * i + c];
            k[c] = dir[3 * i + c];
            in = in && r[c] >= gp->lo[c] && r[c] <= gp->hi[c];
        }
        if (gp->domain == VGRID_DOMAIN_SPHERE) {
            double o[3];
            for (int c = 0; c < 3; c++) o[c] = __dsub_rn(r[c], gp->sph[c]);
            const double q = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(o[0], o[0]), __dmul_rn(o[1], o[1])),
                                                 __dmul_rn(o[2], o[2])),
                                       __dmul_rn(gp->sph[3], gp->sph[3]));
            if (q > 0.0) {
                const double b = __dadd_rn(__dadd_rn(__dmul_rn(k[0], o[0]), __dmul_rn(k[1], o[1])), __dmul_rn(k[2], o[2]));
                const double disc = __dsub_rn(__dmul_rn(b, b), q);
                if (b < 0.0 && disc >= 0.0) {
                    const double t = __dadd_rn(__ddiv_rn(q, __dsub_rn(__dsqrt_rn(disc), b)), gp->eps64);
                    for (int c = 0; c < 3; c++) r[c] = __dadd_rn(r[c], __dmul_rn(t, k[c]));
                }
            }
        } else if (!in) {
            double t_in = -1e300, t_out = 1e300;
            bool miss = false;
            for (int c = 0; c < 3; c++) {
                if (k[c] != 0.0) {
                    const double t1 = (gp->lo[c] - r[c]) / k[c], t2 = (gp->hi[c] - r[c]) / k[c];
                    t_in = fmax(t_in, fmin(t1, t2));
                    t_out = fmin(t_out, fmax(t1, t2));
                } else if (r[c] < gp->lo[c] || r[c] > gp->hi[c]) {
                    miss = true;
                }
            }
            if (!miss && t_in <= t_out && t_out >= 0.0) {
                const double t = fmax(t_in, 0.0);
                for (int c = 0; c < 3; c++) r[c] = fmin(fmax(__fma_rn(t, k[c], r[c]), gp->lo[c]), gp->hi[c]);
            }
        }
        for (int c = 0; c < 3; c++) out[3 * i + c] = r[c];
    }
}

cudaError_t launch_enter(const double *origin, const double *dir, int64_t N, const GridDev *gp, double *out, int sms,
                         cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    int64_t blocks = (N + 255) / 256;
    blocks = blocks < (int64_t)sms * 16 ? blocks : (int64_t)sms * 16;
    enter_kernel<<<(unsigned)blocks, 256, 0, s>>>(origin, dir, N, gp, out);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// exclusive prefix sum over int64 (three passes: tiles, tile totals, fix-up)
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *warp_sums, int64_t &block_total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    block_total = warp_sums[(blockDim.x >> 5) - 1];
    const int64_t before = wid > 0 ? warp_sums[wid - 1] : 0;
    const int64_t r = before + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(int64_t *data, int64_t n, int64_t *tile_sums) {
    __shared__ int64_t ws[32];
    const int64_t base = blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = base + i < n ? data[base + i] : 0;
        sum += v[i];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(sum, ws, total);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (base + i < n) data[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int64_t *tile_sums, int64_t ntiles, int64_t *out_total) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += kScanThreads) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = i < ntiles ? tile_sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, ws, total);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_fix_kernel(int64_t *data, int64_t n, const int64_t *tile_sums) {
    const int64_t add = tile_sums[blockIdx.x];
    const int64_t base = blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int i = 0; i < kScanItems; i++)
        if (base + i < n) data[base + i] += add;
}

// Chunked segments -> CSR, in the order of the destination so that the
// stores are coalesced: (1) chunks per ray, ceil(n / kSegChunk), scanned into
// coff; (2) each used chunk c of ray r at position k is entered as
// inv[coff[r] + k] = c; (3) kSegChunk threads per destination chunk copy its
// slots to the ray's offset plus kSegChunk * k. The number of chunks the
// traversal took and the total are read on the device: when the total
// exceeds the caller's capacity (some chunks were never stored) steps 2 and
// 3 do nothing, and only the offsets go back.
__global__ void chunk_counts_kernel(const int64_t *off, int64_t N, int64_t *ccount) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x)
        ccount[r] = (__ldg(off + r + 1) - __ldg(off + r) + kSegChunk - 1) / kSegChunk;
}

__global__ void chunk_invert_kernel(const int2 *meta, const unsigned long long *cursor, int64_t chunk_cap,
                                    const int64_t *off, int64_t N, int64_t cap, const int64_t *coff, int32_t *inv) {
    if (__ldg(off + N) > cap) return;
    const int64_t nchunks = min((int64_t)*cursor, chunk_cap);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int2 m = __ldg(meta + c);
        if (m.x >= 0) inv[__ldg(coff + m.x) + m.y] = (int32_t)c;  // -1: handed to a warp, not used
    }
}

template <bool FP64>
__global__ void __launch_bounds__(256) compact_segments_kernel(const int64_t *off, const int64_t *coff, int64_t N,
                                                               int64_t cap, const int32_t *inv, const int2 *meta,
                                                               const void *slots, int32_t *cell, void *len) {
    if (__ldg(off + N) > cap) return;
    const int64_t nd = __ldg(coff + N);  // destination chunks
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nd * kSegChunk; t += stride) {
        const int32_t c = __ldg(inv + t / kSegChunk);
        const int2 m = __ldg(meta + c);
        const int64_t o = __ldg(off + m.x), n = __ldg(off + m.x + 1) - o;
        const int64_t j = (int64_t)m.y * kSegChunk + (t & (kSegChunk - 1));
        if (j >= n) continue;
        const int64_t at = (int64_t)c * kSegChunk + (t & (kSegChunk - 1));
        if (FP64) {
            const int4 v = __ldcs(reinterpret_cast<const int4 *>(slots) + at);
            cell[o + j] = v.x;
            reinterpret_cast<double *>(len)[o + j] = __hiloint2double(v.w, v.z);
        } else {
            const int2 v = __ldcs(reinterpret_cast<const int2 *>(slots) + at);
            cell[o + j] = v.x;
            reinterpret_cast<float *>(len)[o + j] = __int_as_float(v.y);
        }
    }
}

static int grid_for(int64_t threads, int sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, (int64_t)sms * 8));
}

cudaError_t launch_compact_segments(const int64_t *off, int64_t N, int64_t chunk_cap, const unsigned long long *cursor,
                                    const int2 *meta, const void *slots, bool fp64, int64_t cap, int64_t *coff,
                                    int64_t *scan_tmp, int32_t *inv, int32_t *cell, void *len, int sms,
                                    cudaStream_t s) {
    if (N <= 0 || chunk_cap <= 0 || !cell || !len) return cudaSuccess;
    chunk_counts_kernel<<<grid_for(N, sms), 256, 0, s>>>(off, N, coff);
    count_launches(1);
    cudaError_t e = launch_exclusive_scan(coff, N, scan_tmp, s);
    if (e != cudaSuccess) return e;
    chunk_invert_kernel<<<grid_for(chunk_cap, sms), 256, 0, s>>>(meta, cursor, chunk_cap, off, N, cap, coff, inv);
    count_launches(1);
    // destination chunks: coff[N] (read on the device), at most chunk_cap
    if (fp64)
        compact_segments_kernel<true><<<grid_for(chunk_cap * kSegChunk, sms), 256, 0, s>>>(off, coff, N, cap, inv,
                                                                                           meta, slots, cell, len);
    else
        compact_segments_kernel<false><<<grid_for(chunk_cap * kSegChunk, sms), 256, 0, s>>>(off, coff, N, cap, inv,
                                                                                            meta, slots, cell, len);
    count_launches(1);
    return cudaGetLastError();
}

// exact float64 sum of two floats? (the TwoSum error term is zero)
__device__ __forceinline__ bool exact_sum(double a, double b) {
    const double s = __dadd_rn(a, b), bb = __dsub_rn(s, a);
    return __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb)) == 0.0;
}

// One thread per cell: the records of its absolute block get n = p_j - p_m
// in float64 (site coordinates are floats, so n is exact unless their
// exponents lie far apart; then the flag sends the kernel back to the float
// coordinates, as it does for p_j + p_m).
__global__ void build_rec64_kernel(const float4 *site, const float4 *rel, const float4 *cells, int64_t M,
                                   float4 *rec64) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        const float4 sm = site[m];
        const int A = __float_as_int(rel[__float_as_int(sm.w) + 1].w);
        const int cnt = __float_as_int(cells[A].y);
        rec64[2 * (int64_t)A] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec64[2 * (int64_t)A + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        const double pm[3] = {(double)sm.x, (double)sm.y, (double)sm.z};
        for (int p = 1; p <= cnt; p++) {
            const float4 q = cells[A + p];
            const int w = __float_as_int(q.w);
            double n[3] = {0.0, 0.0, 0.0};
            int flag = 0;
            if (w >= 0) {
                const double pj[3] = {(double)q.x, (double)q.y, (double)q.z};
                for (int c = 0; c < 3; c++) {
                    n[c] = __dsub_rn(pj[c], pm[c]);
                    if (!exact_sum(pj[c], -pm[c]) || !exact_sum(pj[c], pm[c])) flag = 1;
                }
            }
            const int64_t at = 2 * ((int64_t)A + p);
            rec64[at] = make_float4(__int_as_float(__double2loint(n[0])), __int_as_float(__double2hiint(n[0])),
                                    __int_as_float(__double2loint(n[1])), __int_as_float(__double2hiint(n[1])));
            rec64[at + 1] = make_float4(__int_as_float(__double2loint(n[2])), __int_as_float(__double2hiint(n[2])),
                                        __int_as_float(w), __int_as_float(flag));
        }
    }
}

cudaError_t launch_build_rec64(const float4 *site, const float4 *rel, const float4 *cells, int64_t M, int64_t nrec,
                               float4 *rec64, int sms, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    (void)nrec;
    const int blocks = (int)std::min<int64_t>((M + 127) / 128, (int64_t)sms * 16);
    build_rec64_kernel<<<blocks, 128, 0, s>>>(site, rel, cells, M, rec64);
    count_launches(1);
    return cudaGetLastError();
}

// 8 lanes per ray striding over its segments (coalesced reads of the
// lists); the term is (dL/dtau_r kappa) l, as the traversal's adjoint forms it
__global__ void segments_grad_kernel(const int64_t *off, const int32_t *cell, const float *len, int64_t N,
                                     const float *g, float kappa, float *out) {
    const int i = threadIdx.x & 7;
    const int64_t groups = (int64_t)gridDim.x * blockDim.x / 8;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 8; r < N; r += groups) {
        const float gk = __ldg(g + r) * kappa;
        const int64_t a = __ldg(off + r), b = __ldg(off + r + 1);
        for (int64_t k = a + i; k < b; k += 8) atomicAdd(out + __ldg(cell + k), gk * __ldg(len + k));
    }
}

cudaError_t launch_segments_grad(const int64_t *off, const int32_t *cell, const float *len, int64_t N, const float *g,
                                 float kappa, float *out, int sms, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((N * 8 + 255) / 256, (int64_t)sms * 8));
    segments_grad_kernel<<<blocks, 256, 0, s>>>(off, cell, len, N, g, kappa, out);
    count_launches(1);
    return cudaGetLastError();
}

int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t launch_exclusive_scan(int64_t *data, int64_t n, int64_t *tmp, cudaStream_t s) {
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) {
        return cudaMemsetAsync(data, 0, sizeof(int64_t), s);
    }
    scan_tiles_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(data, n, tmp);
    count_launches(1);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(tmp, tiles, data + n);
    count_launches(1);
    scan_fix_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(data, n, tmp);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vg
