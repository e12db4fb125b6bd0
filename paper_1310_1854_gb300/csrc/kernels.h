// Kernel tables and host-callable launch helpers of libvgrid (internal).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace vg {

enum { MODE_TAU = 0, MODE_SEGS = 1, MODE_GRAD = 2, MODE_INTERACT = 3, NUM_MODES = 4 };

// Segment lists in one traversal. A ray's segments go, in path order, into
// chunks of kSegChunk slots of a work buffer; each chunk records its ray and
// its position in that ray's list, so once the counts have been scanned a
// compaction kernel can copy every chunk to its place in the CSR arrays
// independently of the others. Chunks are handed to the lanes of a warp from
// a page of kSegPage chunks that the warp takes from one global cursor, so
// the cursor sees one atomic per kSegPage chunks. A slot is int2 (cell,
// float32 length) or int4 (cell, 0, float64 length as low and high words).
constexpr int kSegChunk = 8;
constexpr int kSegPage = 32;  // >= 32: one ballot's requests always fit in what is left plus one page

struct TraceArgs {
    const GridDev *grids;     // one descriptor per grid
    const RaySetDev *sets;    // one per (grid, rays) set
    int32_t nsets;
    int64_t total;            // rays over all sets
    unsigned long long *queue;
    StatsDev *stats;
    // segment mode
    int64_t *seg_off;         // segment count per ray (scanned afterwards)
    void *seg_slots;          // chunk slots (kSegChunk per chunk)
    int2 *chunk_meta;         // per chunk: (ray, position in the ray's list); ray -1: unused
    unsigned long long *chunk_cursor;  // chunks handed out (zeroed by the caller)
    int64_t chunk_cap;        // chunks in the buffer; segments beyond are counted, not stored
    const float *dL_dtau;
    float *dL_drho;
    // interaction mode
    const float *tau_int;     // optical depth at which each ray interacts
    const float *weight;      // package weight per ray (nullable: 1)
    int32_t *int_cell;        // caller id of the interaction cell, -1 if the ray escapes
    float *int_s;             // distance from the origin to the interaction point (or the exit)
    float *absorbed;          // per cell (caller ids), accumulated; nullable
    // single-grid launches read the grid and the ray set from here (kernel
    // parameter space) instead of from `grids` / `sets`
    GridDev g1;
    RaySetDev s1;
    const int32_t *order;     // nullable: queue position -> ray (longest predicted first)
};


// fn[fp64][mode]: single-grid trace kernels of one lanes-per-ray value
// (nullptr if absent); batch: the float32 tau kernel over many grids
struct KernelSet {
    // fn[0]: float32 form, fn[1]: float64 form, fn[2]: float32 form with
    // exact lengths (one lane per ray only)
    const void *fn[3][NUM_MODES];
    const void *batch;
};

void kernel_table_lpr1(KernelSet &k);
void kernel_table_lpr2(KernelSet &k);
void kernel_table_lpr4(KernelSet &k);
void kernel_table_lpr8(KernelSet &k);

// auxiliary kernels (aux.cu)
// kernels launched by this library in this process (every launch helper
// adds the kernels it launched)
void count_launches(int64_t n);
int64_t launches_so_far();

cudaError_t launch_put_grid(GridDev *d, const GridDev &g, cudaStream_t s);
cudaError_t launch_enter(const double *origin, const double *dir, int64_t N, const GridDev *gp, double *out, int sms,
                         cudaStream_t s);
cudaError_t launch_prepare(RaySetDev *d_set, const RaySetDev &set, unsigned long long *queue, StatsDev *stats,
                           cudaStream_t s);
// what the start-cell kernel writes per ray (see locate_kernel)
enum { PREP_CELL32 = 0, PREP_FP32 = 1, PREP_FP64 = 2, PREP_CELL64 = 3 };
// Longest-predicted-first ray order. A persistent launch ends when its last
// ray does, so long rays handed out late leave most lanes idle at the end;
// handing the longest out first fixes that. The start-cell kernel estimates
// each ray's crossings (sum of the coarse (sites per volume)^(1/3) grid at 8
// points of its in-box segment, times the segment length) and counts rays
// per bin; a scan and a scatter turn the bins into the permutation the
// traversal takes its rays from, highest bin first. For a grid whose blocks
// fit in L2 the bin is the quarter-octave of the estimate; for a larger one
// it is (half-octave of the estimate, one of 16 ranges of the start cell's
// Morton index), so that the rays in flight at a time start in one part of
// the grid and share more of L2.
constexpr int kOrderBins = 256;
struct RayOrder {
    uint8_t *bin;     // per ray
    uint32_t *hist;   // kOrderBins counts, then kOrderBins cursors (zeroed by the caller)
    int32_t *order;   // queue position -> ray
};
// the start records (PREP_FP32 or PREP_FP64) plus the bins and their counts
cudaError_t launch_locate_ordered(const GridDev *grids, const RaySetDev *sets, int nsets, int64_t total,
                                  const RayOrder &ord, int prep, int sms, cudaStream_t s);
// bins -> permutation (scan of the counts, longest bin first, and scatter)
cudaError_t launch_order(const RayOrder &ord, int64_t total, int sms, cudaStream_t s);
cudaError_t launch_locate(const GridDev *grids, const RaySetDev *sets, int nsets, int64_t total, int prep,
                          int32_t *out_caller, int sms, cudaStream_t s);
cudaError_t launch_permute_density(const float *rho_caller, const int32_t *perm, const float4 *site, int64_t M,
                                   float4 *cells, float4 *rel, cudaStream_t s);
// the float64 form's table of exact differences (GridDev::rec64) for the
// nrec entries of `cells`
cudaError_t launch_build_rec64(const float4 *site, const float4 *rel, const float4 *cells, int64_t M, int64_t nrec,
                               float4 *rec64, int sms, cudaStream_t s);
// copy the segments of the chunks the traversal took (read from the chunk
// cursor on the device, at most chunk_cap; see kSegChunk) of rays 0..N-1
// into the CSR arrays at the scanned offsets off[0..N], unless off[N]
// exceeds cap (then nothing is written); coff holds N+1 and inv chunk_cap
// values of scratch, scan_tmp scan_tmp_elems(N)
cudaError_t launch_compact_segments(const int64_t *off, int64_t N, int64_t chunk_cap, const unsigned long long *cursor,
                                    const int2 *meta, const void *slots, bool fp64, int64_t cap, int64_t *coff,
                                    int64_t *scan_tmp, int32_t *inv, int32_t *cell, void *len, int sms,
                                    cudaStream_t s);
// adjoint from segment lists: out[cell[k]] += g[r] * kappa * len[k] for the
// segments k of every ray r (CSR offsets off[0..N])
cudaError_t launch_segments_grad(const int64_t *off, const int32_t *cell, const float *len, int64_t N, const float *g,
                                 float kappa, float *out, int sms, cudaStream_t s);
// exclusive scan of counts[0..n-1] (int64) into off[0..n]; tmp holds
// scan_tmp_elems(n) int64 values
int64_t scan_tmp_elems(int64_t n);
cudaError_t launch_exclusive_scan(int64_t *counts_to_off, int64_t n, int64_t *tmp, cudaStream_t s);

}  // namespace vg
