/*
 * vgrid - straight-path traversal of 3D Voronoi grids on one GPU.
 *
 * The method is that of Camps, Baes & Saftly (2013), "Using 3D Voronoi grids
 * in radiative transfer simulations", Sect. 2: a ray (photon package) with
 * start r0 inside a cuboidal domain D and unit direction k is followed cell by
 * cell; in the current cell m the exit is the nearest bisector plane ahead of
 * the ray among the cell's neighbours (Eq. 1-4) or a domain wall (Eq. 5);
 * every crossing yields a segment (cell, length) and the optical depth is
 * tau = sum over segments of kappa * rho_cell * length.
 *
 * Conventions for every entry point
 *  - Return value: VGRID_OK (0) or a negative VGRID_ERR_* code. The message of
 *    the most recent failure on the calling thread is vgrid_last_error().
 *  - "device" pointers are CUDA global-memory pointers on the device that was
 *    current when the grid was created; "host" pointers are ordinary memory.
 *    The caller owns every buffer it passes and must keep it alive until the
 *    work on `stream` has finished. The library owns a vgrid_t and its device
 *    copies and frees them in vgrid_destroy().
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream). Calls on one vgrid_t share its work buffers, so they must be
 *    issued on one stream (or otherwise serialised).
 *  - Cell ids in every input and output are the caller's site indices
 *    0..M-1. Domain walls are -1 (x = xmin), -2 (x = xmax), -3 (y = ymin),
 *    -4 (y = ymax), -5 (z = zmin), -6 (z = zmax), as in Sect. 2.2 item 3.
 *  - There is no CPU fallback: without a usable CUDA device the calls fail
 *    with VGRID_ERR_CUDA.
 */
#ifndef VGRID_H
#define VGRID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vgrid vgrid_t;
typedef struct vgrid_batch vgrid_batch_t;
typedef struct CUstream_st *vgrid_stream_t; /* same type as cudaStream_t */

enum {
    VGRID_OK = 0,
    VGRID_ERR_ARG = -1,        /* bad argument (null, size, non-finite, not unit) */
    VGRID_ERR_DUP_SITE = -2,   /* two sites coincide (after float32 rounding) */
    VGRID_ERR_OUTSIDE = -3,    /* a site, or a ray start, lies outside the domain */
    VGRID_ERR_CAPACITY = -4,   /* segment buffer too small; seg_off holds the sizes */
    VGRID_ERR_STEP_LIMIT = -5, /* some rays hit the step limit (see ray_status) */
    VGRID_ERR_CUDA = -6,       /* CUDA runtime failure or no device */
    VGRID_ERR_NOMEM = -7,      /* host or device allocation failed */
    VGRID_ERR_BUILD = -8       /* the neighbour construction failed for a cell */
};

/* arithmetic of the exit search */
enum {
    VGRID_FP64 = 0,         /* Eq. 1-5 in float64, as written */
    VGRID_FP32_RECHECK = 1, /* float32 plane tests with error bounds; a crossing
                               whose two nearest exits are not separated by the
                               bounds is recomputed in float64. A crossing's
                               length is num/den in float32, its end point
                               placed to within about 12 u N^2 / (n.k) (u =
                               2^-24, N the cell's largest |n|_1) */
    VGRID_FP32_EXACT = 2    /* the decisions of VGRID_FP32_RECHECK, and each
                               crossing's length from the exact site
                               difference in float-pair arithmetic (within a
                               few u); float32 results as FP32_RECHECK's.
                               vgrid_trace, vgrid_trace_host and
                               vgrid_trace_noalloc take it, with one lane per
                               ray (the launch's lanes_per_ray is not used) */
};

/* what vgrid_trace writes */
enum {
    VGRID_TAU = 0,      /* tau per ray */
    VGRID_SEGMENTS = 1, /* tau per ray and the segment list of every ray */
    VGRID_ENTER = 0x100 /* flag, OR it in: a ray starting outside the domain
                           first moves to where it enters the box (the
                           nearest boundary point along +k, slab test) and is
                           traced from there; rays that miss the box stay
                           VGRID_RAY_OUTSIDE (Sect. 2.2 notes the method is
                           easily adjusted for rays that originate outside the
                           domain) */
};

/* per-ray status codes written to ray_status */
enum {
    VGRID_RAY_OK = 0,
    VGRID_RAY_OUTSIDE = 1,   /* start point outside the domain: no path */
    VGRID_RAY_STEP_LIMIT = 2, /* the path was cut at opts.max_steps decisions */
    VGRID_RAY_BAD_DIR = 3     /* |dir| differs from 1 by more than 1e-6: not traced */
};

typedef struct {
    int32_t threads;           /* host threads for the build; 0 = all cores */
    int32_t round_sites;       /* 1: round sites to float32; 0: reject sites that are
                                  not exactly representable in float32 */
    int32_t reorder;           /* 1 (default): store cells along a Morton curve */
    double blocks_per_site;    /* locate block grid: blocks per site (default 8) */
    int64_t max_steps;         /* exit decisions per ray before VGRID_RAY_STEP_LIMIT
                                  (default 100,000) */
    int32_t host_only;         /* 1: build the neighbour lists, volumes and block
                                  lists on the host but copy nothing to a device;
                                  only vgrid_info, vgrid_get_neighbors,
                                  vgrid_get_cells and vgrid_destroy accept such a
                                  grid (no GPU needed) */
    int32_t gpu_build;         /* 1: construct the cells on the current GPU (one
                                  thread per cell; cells that exceed its fixed
                                  capacities are rebuilt on the host) */
    int32_t zero_run_max;      /* zero-length steps in a row that a path may take
                                  (a ray through an edge or vertex of several
                                  cells); one more moves the point on by epsilon
                                  and locates its cell again, as a decision without
                                  any exit does (Sect. 2.2). Default 4; 0 nudges
                                  after every zero-length step. Epsilon is
                                  1e-12 |Dmax - Dmin| in the float64 form and
                                  1e-6 |Dmax - Dmin| in the float32 form. */
    int32_t domain;            /* VGRID_DOMAIN_BOX (default): the domain is bbox.
                                  VGRID_DOMAIN_SPHERE: the ball `sphere` inside
                                  bbox (Sect. 2.2: the method carries over to
                                  other domain geometries). Every site must lie
                                  in the closed ball ((dx dx + dy dy) + dz dz <=
                                  R R in float64, else VGRID_ERR_OUTSIDE). The
                                  cells keep the neighbour lists, volumes and
                                  bounding boxes of bbox's clipping (a face that
                                  lies outside the ball is never reached: the
                                  path leaves the domain first); a point outside
                                  the ball is outside the domain, and a path ends
                                  where it leaves the ball: the larger root s of
                                  |r + s k - c|^2 = R^2 (wall id -7), in float64
                                  from the current point in the float64 form, once
                                  per ray from the origin in the float32 form.
                                  With VGRID_ENTER a ray outside the ball that
                                  meets it ahead starts 1e-12 |Dmax - Dmin| past
                                  its entry point. */
    double sphere[4];          /* VGRID_DOMAIN_SPHERE: centre x, y, z and radius
                                  R > 0; the ball must lie in bbox */
} vgrid_opts;

/* domains (vgrid_opts.domain) */
enum { VGRID_DOMAIN_BOX = 0, VGRID_DOMAIN_SPHERE = 1 };

typedef struct {
    int64_t rays;          /* rays traced */
    int64_t crossings;     /* segments of positive length */
    int64_t decisions;     /* exit decisions (crossings, zero-length steps, wall exit) */
    int64_t rechecks;      /* float64 rechecks of float32 decisions */
    int64_t fallbacks;     /* epsilon nudges followed by a new C(r) (Sect. 2.2) */
    int64_t zero_steps;    /* zero-length steps */
    int64_t step_limit;    /* rays cut at max_steps */
    int64_t outside;       /* rays starting outside the domain */
} vgrid_stats;

typedef struct {
    int64_t M;             /* sites */
    int64_t nnz;           /* neighbour entries including walls */
    int64_t block_entries; /* entries of all block lists */
    int32_t block_dim[3];  /* locate block grid */
    double box[6];         /* xmin, ymin, zmin, xmax, ymax, zmax */
    double build_seconds;  /* host time of vgrid_create */
    int64_t device_bytes;  /* device memory held by the grid */
    int64_t host_fallback_cells; /* gpu_build: cells rebuilt on the host */
    double phase_seconds[6];   /* vgrid_create by phase: checks and duplicates,
                                  cell order, cells (host or GPU), block lists,
                                  device layout, copies to the device */
    int64_t rel_bytes;     /* bytes of the cell blocks the float32 traversal
                              reads (the part that must stay in L2 for it to
                              run from L2) */
} vgrid_info_t;

/* launch shape of the traversal kernels */
typedef struct {
    int32_t lanes_per_ray;      /* 1, 2, 4 or 8 lanes cooperate on one ray (default 1) */
    int32_t block;              /* threads per block (multiple of 32, 32..256; default 128) */
    int32_t blocks_per_sm;      /* persistent blocks per SM; 0 = as many as fit */
    int32_t fp64_lanes_per_ray; /* lanes per ray of the float64 form; 0 = lanes_per_ray (default 1) */
    int32_t order;              /* order in which the traversal takes the rays:
                                   1 = longest estimated path first (crossings estimated
                                   from a coarse site-density grid along each ray),
                                   -1 = the caller's order, 0 (default) = longest first
                                   when there are at least two rays per resident lane.
                                   Results do not depend on it; the time does: a
                                   persistent launch lasts until its last ray ends.
                                   Used by vgrid_trace (both forms), vgrid_trace_host,
                                   vgrid_trace_grad and vgrid_interact; a batch orders
                                   all its work items together only with order = 1
                                   (that interleaves its grids, which then share L2). */
} vgrid_launch;

/* Kernels this library has launched in this process so far (every call
 * adds the kernels it enqueued; a replayed batch graph adds those it holds). */
int64_t vgrid_kernel_launches(void);

/* Message of the last failed call on this thread ("" if none). */
const char *vgrid_last_error(void);

/* Fill *opts with the defaults. */
void vgrid_default_opts(vgrid_opts *opts);

/*
 * Build a grid (Sect. 2.2 setup items 1-3 and the block lists of Sect. 2.3).
 *   sites  host, M x 3 float64 (x, y, z per site), all inside the closed box.
 *   bbox   host, 6 float64: xmin, ymin, zmin, xmax, ymax, zmax.
 *   opts   host, nullable (defaults).
 * On the host: the cell of every site is cut from the box by the bisector
 * half-spaces of nearby sites (Sect. 2.1), giving neighbour lists with walls,
 * cell volumes and bounding boxes; the bounding boxes fill a regular block grid
 * of candidate lists for C(r) (Sect. 2.3). The lists, the sites (float32) and
 * a default density rho = 1, kappa = 1 are then copied to the current device.
 * Errors: VGRID_ERR_ARG, VGRID_ERR_OUTSIDE (site outside box),
 * VGRID_ERR_DUP_SITE, VGRID_ERR_BUILD, VGRID_ERR_NOMEM, VGRID_ERR_CUDA.
 */
int vgrid_create(const double *sites, int64_t M, const double bbox[6], const vgrid_opts *opts, vgrid_t **out);

/* Free the grid and its device memory. NULL is accepted. */
int vgrid_destroy(vgrid_t *g);

/* Sizes and build facts. */
int vgrid_info(const vgrid_t *g, vgrid_info_t *info);

/*
 * Host copies of the neighbour lists (Sect. 2.2 item 3) in the caller's ids:
 * off host int64[M+1], idx host int32[info.nnz] (walls negative, ascending
 * within a cell). Either pointer may be NULL to skip it.
 */
int vgrid_get_neighbors(const vgrid_t *g, int64_t *off, int32_t *idx);

/* Host copies of cell volumes (host float64[M]) and bounding boxes
 * (host float64[M*6]); either may be NULL. */
int vgrid_get_cells(const vgrid_t *g, double *volume, double *bbox);

/*
 * Set the density per cell, rho (device float32[M], caller ids), and the
 * opacity kappa used in tau = sum kappa rho l. The values are copied into the
 * grid's own cell order on `stream`; later changes to rho are not seen.
 */
int vgrid_set_density(vgrid_t *g, const float *rho, float kappa, vgrid_stream_t stream);

/*
 * C(r) of Sect. 2.3 for N points: pts device float64[N*3]; cell device
 * int32[N] receives the nearest site (caller id), or -1 for points outside the
 * closed box. precision: VGRID_FP64 (distances in float64) or
 * VGRID_FP32_RECHECK (float32 distances; near-equal candidates are compared
 * again in float64). Exact ties go to the lowest site index.
 */
int vgrid_locate(vgrid_t *g, const double *pts, int64_t N, int precision, int32_t *cell, vgrid_stream_t stream);

/*
 * Trace N rays to the domain boundary (Sect. 2.2).
 *   origin, dir   device float64[N*3]; every dir must have unit length
 *                 within 1e-6 (checked on the device: such a ray gets tau 0,
 *                 no segments and status VGRID_RAY_BAD_DIR).
 *   precision     VGRID_FP64, VGRID_FP32_RECHECK or VGRID_FP32_EXACT (the
 *                 latter's tau and lengths are float32, as FP32_RECHECK's).
 *   output        VGRID_TAU or VGRID_SEGMENTS, optionally | VGRID_ENTER
 *                 (segments, tau and lengths then start at the entry point;
 *                 needs a work buffer of N*3 doubles, grown like the others).
 *   tau           device float64[N] (FP64) or float32[N] (FP32_RECHECK);
 *                 nullable in segment mode.
 *   seg_off       device int64[N+1] (segment mode): exclusive prefix sum of
 *                 the per-ray segment counts; seg_off[N] is the total.
 *   seg_cell      device int32[seg_capacity]: cell id of each segment.
 *   seg_len       device float64 (FP64) or float32 (FP32_RECHECK)
 *                 [seg_capacity]: segment lengths.
 *   ray_status    device int32[N] or NULL: VGRID_RAY_* per ray.
 *   stats         host or NULL: counters of this call (synchronises `stream`).
 * Segment mode traces once: each ray appends its segments to chunks of 8 in
 * a work buffer of the library, the counts are scanned into seg_off, and a
 * copy kernel moves the chunks into seg_cell / seg_len in ray order (the
 * copy compares the total with seg_capacity on the device and writes
 * nothing if it does not fit); the call reads the total back and
 * synchronises once, at its end. If seg_capacity is too small it returns
 * VGRID_ERR_CAPACITY with seg_off filled so the caller can size the buffers
 * and call again (seg_capacity = 0 only counts). The work buffer holds
 * ceil(seg_capacity/8) + min(N, seg_capacity) + 32 x (warps of the launch)
 * chunks of 8 slots of 8 (FP32_RECHECK) or 16 (FP64) bytes plus 12 bytes
 * of records each, and 8 bytes per ray; N is at most 2^31 - 1 in segment
 * mode.
 * Rays that start outside the domain get tau = 0, no segments and status
 * VGRID_RAY_OUTSIDE (not an error). Whenever the call reads its counters back
 * (stats non-NULL, or segment mode) it returns VGRID_ERR_ARG if some
 * direction was not a unit vector and VGRID_ERR_STEP_LIMIT if some ray was
 * cut at max_steps, after writing every output; in tau mode without stats
 * the call does not synchronise and those rays show only in ray_status.
 * The first call with more rays than any earlier call on this grid
 * allocates larger work buffers: a 64-byte start record per ray, and with
 * the ray order (vgrid_launch.order) 5 more bytes per ray; segment mode adds
 * the scan's scratch and the chunk buffer above.
 */
int vgrid_trace(vgrid_t *g, const double *origin, const double *dir, int64_t N, int precision, int output,
                void *tau, int64_t *seg_off, int32_t *seg_cell, void *seg_len, int64_t seg_capacity,
                int32_t *ray_status, vgrid_stats *stats, vgrid_stream_t stream);

/*
 * tau of N rays held in HOST memory (Sect. 2.2 as vgrid_trace, VGRID_TAU
 * output), with the copies overlapped with the traversal. Each chunk of
 * rays goes through one of two device slots that alternate across chunks and
 * calls: its origins and directions are copied in on a copy stream as soon
 * as the slot's previous traversal is done, its start records (and ray
 * order) are prepared on a third stream once they are in, so that this runs
 * beside the previous chunk's traversal, and it is traced on `stream`.
 * If tau (and ray_status, when given) are page-locked host memory mapped
 * into the device's address space (cudaHostAlloc and pinned tensors are,
 * with unified addressing), the traversal writes them directly; otherwise
 * they are copied out from the slot on a second copy stream. Consecutive
 * calls therefore overlap: the next call's rays go in while this call's
 * traversal runs. Host buffers should be page-locked for the copies to
 * overlap; pageable buffers work, serialised.
 *   origin, dir   host float64[N*3], unit directions as for vgrid_trace
 *   precision     VGRID_FP64, VGRID_FP32_RECHECK or VGRID_FP32_EXACT
 *   tau           host float64[N] (FP64) or float32[N] (the float32 forms)
 *   ray_status    host int32[N] or NULL
 *   chunk         rays per chunk; 0 = N. A traversal launch lasts at least
 *                 as long as its longest ray, so chunks only pay off for rays
 *                 that do not fit on the device at once.
 *   stats         host or NULL: counters summed over all chunks; the call
 *                 then synchronises `stream` before it returns.
 * Without stats the call returns once everything is queued: the results are
 * in host memory when `stream` has been synchronised, and the host buffers
 * must stay untouched until then. The first call with a larger chunk than
 * before synchronises the device and allocates two device slots (125 bytes
 * per ray each: rays, result, status, start record, order); the first call
 * creates three streams. A call with stats prepares its start records on
 * `stream`, after the previous traversal.
 */
int vgrid_trace_host(vgrid_t *g, const double *origin, const double *dir, int64_t N, int precision, void *tau,
                     int32_t *ray_status, int64_t chunk, vgrid_stats *stats, vgrid_stream_t stream);

/*
 * Adjoint of tau = sum kappa rho l (the optical depth along the path of
 * Sect. 2.2, linear in the cell densities) with respect to rho: for every ray
 * r and every segment (c, l) of its path, dL_drho[c] += dL_dtau[r] * kappa * l.
 * The path is the one vgrid_trace finds with VGRID_FP32_RECHECK, and kappa
 * is the grid's current one (vgrid_set_density).
 *   dL_dtau  device float32[N]; dL_drho device float32[M], accumulated into
 *   (caller ids; zero it first for a plain gradient).
 */
int vgrid_trace_grad(vgrid_t *g, const double *origin, const double *dir, int64_t N, const float *dL_dtau,
                     float *dL_drho, vgrid_stream_t stream);

/*
 * The same adjoint (tau = sum kappa rho l over the path of Sect. 2.2) from
 * the segment lists that vgrid_trace returned (VGRID_SEGMENTS with
 * VGRID_FP32_RECHECK), without tracing again: for every
 * ray r and every k in [seg_off[r], seg_off[r+1]),
 * dL_drho[seg_cell[k]] += dL_dtau[r] * kappa * seg_len[k].
 * Each term is the product vgrid_trace_grad adds; the order of the float32
 * atomic sums differs.
 *   seg_off  device int64[N+1]; seg_cell device int32 and seg_len device
 *            float32, seg_off[N] entries each (caller ids, as returned).
 *   dL_dtau  device float32[N]; dL_drho device float32[M], accumulated into.
 *   kappa    the opacity that the tau of these lists was computed with (the
 *            lists do not depend on it, and the grid may hold another one
 *            by now).
 * One pass over the lists (about 8 bytes read and one atomic per segment).
 * Errors: VGRID_ERR_ARG (also for a kappa that is not finite).
 */
int vgrid_segments_grad(vgrid_t *g, const int64_t *seg_off, const int32_t *seg_cell, const float *seg_len, int64_t N,
                        const float *dL_dtau, float kappa, float *dL_drho, vgrid_stream_t stream);

/*
 * Interaction sampling along the path: the Monte Carlo step that consumes
 * the traversal in the paper's radiative-transfer code (Sect. 3.1, 3.4:
 * photon packages are shot through the grid and their absorption is booked
 * in the cells they cross). Ray r carries an optical depth tau_int[r]
 * (typically -ln of a uniform deviate, drawn by the caller) and a weight
 * w[r]; it is traced (float32 form, as vgrid_trace) until the running
 * tau = sum kappa rho l reaches tau_int[r] inside some cell.
 *   tau_int   device float32[N]
 *   weight    device float32[N] or NULL (all 1)
 *   cell      device int32[N]: the cell where the ray interacts (caller id),
 *             -1 if it leaves the domain first (or starts outside / is cut)
 *   s         device float32[N]: distance from the origin to the interaction
 *             point, or the in-domain path length if it leaves first
 *   absorbed  device float32[M] or NULL, accumulated into: for every cell
 *             crossed before the interaction, w (exp(-tau_in) - exp(-tau_out))
 *             where tau_in, tau_out are the running tau entering and leaving
 *             the cell (capped at tau_int), i.e. the part of the package the
 *             cell removes.
 */
int vgrid_interact(vgrid_t *g, const double *origin, const double *dir, int64_t N, const float *tau_int,
                   const float *weight, int32_t *cell, float *s, float *absorbed, vgrid_stream_t stream);

/* Launch shape used by this grid's traversal kernels (NULL resets to the
 * built-in default). */
int vgrid_set_launch(vgrid_t *g, const vgrid_launch *launch);
int vgrid_get_launch(const vgrid_t *g, vgrid_launch *launch);

/*
 * Many grids in one launch (uneven sizes and ray counts): the traversal of
 * Sect. 2.2 for every set, as vgrid_trace computes it in its float32 form,
 * with one work queue over all sets. Each set names a
 * grid and its rays; tau (device float32[n]) and status (device int32[n],
 * nullable) receive the results of VGRID_FP32_RECHECK tracing.
 */
typedef struct {
    const vgrid_t *grid;
    const double *origin; /* device float64[n*3] */
    const double *dir;    /* device float64[n*3] */
    int64_t n;
    float *tau;           /* device float32[n] */
    int32_t *status;      /* device int32[n] or NULL */
} vgrid_rayset;

/*
 * Prepare a batch: copies the per-grid descriptors to the device and sizes
 * its work buffers. The rays and outputs named in `sets` must stay valid for
 * every later vgrid_batch_run. launch may be NULL (built-in default).
 */
int vgrid_batch_create(const vgrid_rayset *sets, int32_t G, const vgrid_launch *launch, vgrid_batch_t **out);

/*
 * Run the batch on `stream`: one locate launch and one persistent traversal
 * launch over all (grid, ray) work items. With use_graph = 1 the sequence is
 * captured into a CUDA graph on the first call and replayed afterwards.
 */
int vgrid_batch_run(vgrid_batch_t *b, int use_graph, vgrid_stats *stats, vgrid_stream_t stream);

/*
 * Launch shape of a batch (lanes per ray, block, blocks per SM, ray order;
 * fp64_lanes_per_ray is unused). NULL resets to the built-in default. A
 * graph captured by vgrid_batch_run holds the old shape and is dropped; the
 * next graph run captures again. Results do not depend on the shape. The
 * first setting with order = 1 allocates the order's buffers (5 bytes per
 * ray and the bin counts). Errors: VGRID_ERR_ARG, VGRID_ERR_NOMEM.
 */
int vgrid_batch_set_launch(vgrid_batch_t *b, const vgrid_launch *launch);
int vgrid_batch_get_launch(const vgrid_batch_t *b, vgrid_launch *launch);

int vgrid_batch_destroy(vgrid_batch_t *b);

/*
 * Device-time accounting for benchmarks. With enable = 1, every later
 * vgrid_trace / vgrid_trace_grad call on this grid records CUDA events on its
 * stream around the start-cell launch (C(r0) for all rays) and around each
 * traversal launch, without synchronising. vgrid_read_timing waits for those
 * events, returns the summed milliseconds and the number of traversal
 * launches since the previous read, and clears the record. Timing adds no
 * work to the kernels themselves.
 */
int vgrid_enable_timing(vgrid_t *g, int enable);
int vgrid_read_timing(vgrid_t *g, double *locate_ms, double *trace_ms, int64_t *launches);

/*
 * Tau per ray with no device allocation, for callers that cannot call
 * cudaMalloc: code whose device memory is handed out by another allocator
 * under a fixed budget, or latency-bound loops that must not take the
 * implicit device synchronisation cudaMalloc/cudaFree can cause. The paper
 * has no counterpart; this is a variant of vgrid_trace in VGRID_TAU mode.
 *
 * Same arguments and results as vgrid_trace with output VGRID_TAU (tau is
 * float64[N] for VGRID_FP64, float32[N] for the float32 forms; ray_status
 * nullable), but its work buffers (start cells, work counter, counters) live
 * in one fixed device array of VGRID_NOALLOC_SCRATCH_BYTES inside the
 * library, which every GPU that loads the library holds until the process
 * exits. N above VGRID_NOALLOC_MAX_RAYS is rejected with VGRID_ERR_ARG before
 * anything is enqueued. The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress, with the grid's device current);
 * make that first call before any stream capture. All calls share the one
 * array: the call clears what must start at zero, but calls that overlap on
 * the GPU (other streams, other threads, other grids on the same device)
 * race on it and must be serialised by the caller. No counters are returned
 * and nothing is synchronised.
 */
/*
 * Measurement helper (no counterpart in the paper): a read-bandwidth ceiling
 * of the memory level that serves the traversal, measured on the current
 * device, for roofline figures. It allocates a buffer of `bytes` (1 MiB to
 * 4 GiB; below the L2 size it stays in L2 after the first pass), fills it,
 * runs the probe once to warm it and once timed on `stream`, frees the
 * buffer and returns the read rate in *gbs (1e9 bytes per second).
 *   mode 0  stream: 256-bit loads of 32-byte pairs over the whole buffer,
 *           repeated for about 8 GB.
 *   mode 1  chase: each thread reads 288-byte blocks (nine 32-byte pairs,
 *           the size of an average cell block of the float32 traversal) at
 *           random positions, the next block's index taken from the data of
 *           the previous one, at full occupancy.
 * Synchronises `stream`. Errors: VGRID_ERR_ARG, VGRID_ERR_NOMEM, VGRID_ERR_CUDA.
 */
int vgrid_probe_l2(int64_t bytes, int mode, double *gbs, vgrid_stream_t stream);

#define VGRID_NOALLOC_MAX_RAYS (1 << 18)
#define VGRID_NOALLOC_SCRATCH_BYTES (512 + 64 * VGRID_NOALLOC_MAX_RAYS)
int vgrid_trace_noalloc(vgrid_t *g, const double *origin, const double *dir, int64_t N, int precision, void *tau,
                        int32_t *ray_status, vgrid_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* VGRID_H */
