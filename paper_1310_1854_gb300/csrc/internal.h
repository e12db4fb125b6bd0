// Internal declarations shared by the host builder, the C-ABI layer and the
// CUDA kernels of libvgrid. Not part of the public interface (include/vgrid.h).
#pragma once

#include <vector_types.h>

#include <cstdint>
#include <string>
#include <functional>
#include <vector>

namespace vg {

// Host results of the cell construction, in the library's internal cell order.
struct CellsOut {
    std::vector<int64_t> off;   // CSR offsets, M + 1
    std::vector<int32_t> idx;   // neighbour ids (internal) and walls -1..-6
    std::vector<double> vol;    // cell volumes
    std::vector<double> bbox;   // 6 per cell
};

struct BlocksOut {
    int32_t dim[3];
    std::vector<int64_t> off;   // K + 1
    std::vector<int32_t> idx;   // internal cell ids
};

int build_cells(const double *sites, int64_t M, const double *box, int threads, CellsOut &out, std::string &err);
int build_cells_into(const double *sites, int64_t M, const double *box, int threads, const std::vector<int32_t> *ids,
                     std::vector<std::vector<int32_t>> &nbr, double *volume, double *bbox, std::string &err);
void cells_to_csr(const std::vector<std::vector<int32_t>> &nbr, CellsOut &out);
// GPU construction (build_gpu.cu); cells the device could not hold are rebuilt
// on the host. Returns 0, or -1 with err set.
int build_cells_gpu(const double *sites, int64_t M, const double *box, int threads, CellsOut &out, std::string &err,
                    int64_t *host_fallback_cells);
// cells sorted by the Morton code of their site (21 bits per axis); the
// sorted codes go to *codes if given
void morton_order(const double *sites, int64_t M, const double *box, std::vector<int32_t> &perm,
                  std::vector<uint64_t> *codes = nullptr, int threads = 0);
// fn(begin, end) over [0, n) split into contiguous ranges on up to `threads`
// host threads (0: all cores); ranges of fewer than `grain` items stay on
// one thread
void parallel_for(int64_t n, int threads, int64_t grain, const std::function<void(int64_t, int64_t)> &fn);
void build_blocks(const double *box, const std::vector<double> &bbox, int64_t M, double blocks_per_site,
                  BlocksOut &out, int threads = 0);

}  // namespace vg

// ---------------------------------------------------------------------------
// Device-side view of one grid. Plain data, passed by value to kernels or
// stored in an array for batched launches. Cells are in the library's
// internal (Morton) order.
//
// cells    absolute cell blocks (float64 form and rechecks), float4: cell i
//          starts at A_i with a header (bits of the caller's id, bits of the
//          neighbour count c, rho, bits of F_i) followed by c records (x, y, z
//          of the neighbour's site, bits of the neighbour's offset A_j, or of
//          a wall id -1..-6).
// rel      relative cell blocks (float32 form), float4: cell i starts at F_i
//          (even) with (x, y, z of p_i, bits of the record count c4) and
//          (bits of the caller's id, rho, N1max, bits of A_i), followed by c4
//          records: (fl(p_j - p_i) as float32, bits of F_j) for every cell
//          neighbour j, then NaN records up to c4 = max(4, an even count).
//          N1max bounds |fl(p_j - p_i)|_1 over the records from above.
// site[i]  float4 (x, y, z, bits of F_i): positions for C(r) and ray starts.
// perm[i]  caller's id of internal cell i.
// blk_off, blk_rec  block lists of Sect. 2.3: for every block, records
//          (x, y, z of a site, bits of its internal id) of the cells whose
//          bounding box overlaps the block.
// ---------------------------------------------------------------------------
struct GridDev {
    const float4 *site;
    const float4 *cells;
    const float4 *rel;
    const int32_t *perm;
    const int32_t *blk_off;
    const float4 *blk_rec;
    // float64 form: per entry of `cells`, 32 bytes (two float4) holding the
    // record's n = p_j - p_m as three doubles, its id (neighbour's offset in
    // `cells`, or wall id) and a flag set where n or p_j + p_m is not exact
    // in float64 (then the record is evaluated from its float coordinates)
    const float4 *rec64;
    double lo[3], hi[3];      // domain box
    double bscale[3];         // blocks per unit length along each axis
    int64_t lokey[3], hikey[3];        // order keys of lo and hi (exact box test)
    float flo_hi[3], flo_lo[3];        // lo as float pairs
    float fbscale[3];                  // bscale in float32
    float fbw[3];                      // block width in float32; block (i, j, k) has the
                                       // centre flo_hi + (i + 1/2) fbw (float32 operations),
                                       // and its list is ordered by distance from it
    const float *dens;                 // coarse grid of (sites per unit volume)^(1/3), for the ray order
    int32_t ddim[3];                   // its cells per axis
    float dscale[3];                   // its cells per unit length
    int32_t ospatial;                  // ray order: start-cell ranges per length bin (1: length only)
    int32_t bdim[3];
    int32_t M;
    float kappa;
    int32_t zmax;             // zero-length steps in a row before the epsilon nudge
    double eps64;             // epsilon nudge, float64 path
    double eps32;             // epsilon nudge, float32 path
    double scale;             // max |coordinate| of the box + diagonal
    int64_t max_steps;
    int32_t domain;           // VGRID_DOMAIN_BOX or VGRID_DOMAIN_SPHERE
    int32_t pad1;
    double sph[4];            // spherical domain: centre and radius
};

// Per-ray record written by the start-cell kernel (full warps, where the
// float64 set-up is cheap) and read once by the traversal kernel when the
// ray starts (64 bytes).
struct RayPrep {
    int32_t cell;             // start cell: internal id (float64 form), offset of its relative
                              // block (float32 form); -1 outside the box, -2 direction not unit
    int32_t wall;             // wall the ray leaves through (Eq. 5), -1..-6
    float tmax_hi, tmax_lo;   // distance to that wall, as a float pair
    float r0_hi[3], r0_lo[3]; // origin as float pairs
    float k_hi[3], k_lo[3];   // direction as float pairs
};

// A batch work descriptor: rays of one grid.
struct RaySetDev {
    const double *origin;
    const double *dir;
    void *tau;                // float (float32 form) or double (float64 form), nullable
    int32_t *status;          // nullable
    RayPrep *start;           // per-ray start records - work buffer
    int64_t n;
    int64_t first;            // global index of the first ray of this set
    int32_t grid;             // index into the GridDev array
    int32_t pad;
};

// Counters accumulated on the device; mirrors vgrid_stats.
struct StatsDev {
    unsigned long long rays, crossings, decisions, rechecks, fallbacks, zero_steps, step_limit, outside, bad_dir;
};


// What the allocation-free entry point (noalloc.cu) needs from a grid.
struct vgrid;
namespace vg {
struct GridView {
    int device;
    int sms;
    const GridDev *d_desc;
    GridDev hd;  // host copy of *d_desc
    int lanes_per_ray, block, blocks_per_sm, fp64_lanes_per_ray;
};
int grid_view(const struct vgrid *g, GridView *out);  // 0, or -1 for a host-only grid
void set_error(const std::string &msg);              // message for vgrid_last_error()
}  // namespace vg
