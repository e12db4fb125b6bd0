// C-ABI of libvgrid (declared in include/vgrid.h): grid construction and
// upload, C(r), traversal in the float64 and float32-with-recheck forms,
// segment lists, the adjoint, and batched launches over many grids.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <string>
#include <vector>

#include "fsplit.h"
#include "internal.h"
#include "kernels.h"
#include "vgrid.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define VG_CUDA(call)                                                                                 \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return fail(VGRID_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

const vg::KernelSet &kernels(int lpr) {
    static vg::KernelSet t1, t2, t4, t8;
    static bool init = [] {
        vg::kernel_table_lpr1(t1);
        vg::kernel_table_lpr2(t2);
        vg::kernel_table_lpr4(t4);
        vg::kernel_table_lpr8(t8);
        return true;
    }();
    (void)init;
    switch (lpr) {
        case 1: return t1;
        case 2: return t2;
        case 8: return t8;
        default: return t4;
    }
}

bool valid_lpr(int l) { return l == 1 || l == 2 || l == 4 || l == 8; }

template <class T>
int dmalloc(T **p, size_t n, int64_t &total) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) return fail(VGRID_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    total += (int64_t)(n * sizeof(T));
    return VGRID_OK;
}

}  // namespace

struct vgrid {
    int device = 0;
    int sms = 1;
    int64_t M = 0;
    vgrid_opts opts{};
    vgrid_launch launch{1, 128, 0, 1, 0};
    GridDev hd{};
    GridDev *d_desc = nullptr;
    float4 *d_site = nullptr;
    float4 *d_cells = nullptr;
    float4 *d_rec64 = nullptr;       // float64 form: exact differences per entry of d_cells
    float4 *d_rel = nullptr;
    int32_t *d_perm = nullptr;
    int32_t *d_blk_off = nullptr;
    float4 *d_blk_rec = nullptr;
    float *d_dens = nullptr;         // coarse density grid for the ray order
    std::vector<int32_t> perm, inv;  // internal -> caller, caller -> internal
    vg::CellsOut cells;              // internal order
    vg::BlocksOut blocks;
    // work buffers
    unsigned long long *d_queue = nullptr;
    StatsDev *d_stats = nullptr;
    RaySetDev *d_set = nullptr;
    RayPrep *d_start = nullptr;
    int64_t start_cap = 0;
    int64_t *d_scan = nullptr;
    int64_t scan_cap = 0;
    double *d_entry = nullptr;   // entry points of VGRID_ENTER calls
    int64_t entry_cap = 0;
    // segment mode: chunk slots, each chunk's (ray, position), the cursor
    int4 *d_slots = nullptr;     // slots of 8 (float32) or 16 (float64) bytes
    int64_t slot_bytes = 0;
    int2 *d_chunk_meta = nullptr;
    int32_t *d_chunk_inv = nullptr;  // destination chunk -> chunk
    int64_t meta_cap = 0;
    int64_t *d_coff = nullptr;       // chunks per ray, scanned
    int64_t coff_cap = 0;
    unsigned long long *d_cursor = nullptr;
    uint8_t *d_bin = nullptr;    // ray order: bins, counts, permutation
    uint32_t *d_hist = nullptr;
    int32_t *d_order = nullptr;
    int64_t order_cap = 0;
    // host-pipelined calls: two device slots of rays and results, two copy
    // streams and their events
    double *d_hin[2] = {nullptr, nullptr};  // chunk origins then directions
    void *d_hout[2] = {nullptr, nullptr};   // chunk tau (8 bytes per ray)
    int32_t *d_hst[2] = {nullptr, nullptr}; // chunk status
    // per slot also the start records, ray order, work counter and set
    // descriptor, so that a chunk's start records can be prepared on s_loc
    // while the previous chunk is traced (the start-cell pass then fills the
    // SMs that the traversal frees in its tail)
    RayPrep *d_hstart[2] = {nullptr, nullptr};
    uint8_t *d_hbin[2] = {nullptr, nullptr};
    int32_t *d_horder[2] = {nullptr, nullptr};
    uint32_t *d_hhist = nullptr;             // per slot 2 kOrderBins
    unsigned long long *d_hqueue = nullptr;  // per slot
    RaySetDev *d_hset = nullptr;             // per slot
    int64_t host_cap = 0;
    int host_slot = 0;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr, s_loc = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_k[2] = {}, ev_out[2] = {}, ev_prep[2] = {};
    double build_seconds = 0;
    double phase_seconds[6] = {0, 0, 0, 0, 0, 0};
    int64_t device_bytes = 0;
    int64_t host_fallback_cells = 0;
    int64_t rel_bytes = 0;           // bytes of the relative cell blocks
    // optional event record: {locate start, locate end} or {trace start, trace end}
    bool timing = false;
    std::vector<std::array<cudaEvent_t, 2>> ev_loc, ev_trace;
    size_t n_loc = 0, n_trace = 0;
};

struct vgrid_batch {
    int device = 0;
    int sms = 1;
    int32_t G = 0;
    int64_t total = 0;
    vgrid_launch launch{1, 128, 0, 1, 0};
    GridDev *d_grids = nullptr;
    RaySetDev *d_sets = nullptr;
    RayPrep *d_start = nullptr;
    unsigned long long *d_queue = nullptr;
    StatsDev *d_stats = nullptr;
    uint8_t *d_bin = nullptr;    // ray order (when used): bins, counts, permutation
    uint32_t *d_hist = nullptr;
    int32_t *d_order = nullptr;
    int64_t graph_kernels = 0;   // kernels in the captured graph
    int ngrids = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
};

extern "C" {

const char *vgrid_last_error(void) { return g_err.c_str(); }

void vgrid_default_opts(vgrid_opts *o) {
    if (!o) return;
    o->threads = 0;
    o->round_sites = 0;
    o->reorder = 1;
    o->blocks_per_site = 8.0;
    o->max_steps = 100000;
    o->host_only = 0;
    o->gpu_build = 0;
    o->zero_run_max = 4;
    o->domain = VGRID_DOMAIN_BOX;
    for (int c = 0; c < 4; c++) o->sphere[c] = 0.0;
}

static void free_events(vgrid_t *g) {
    for (auto *v : {&g->ev_loc, &g->ev_trace})
        for (auto &p : *v) {
            cudaEventDestroy(p[0]);
            cudaEventDestroy(p[1]);
        }
    g->ev_loc.clear();
    g->ev_trace.clear();
    g->n_loc = g->n_trace = 0;
}

// bytes per ray of one host-pipe slot: rays, result, status, start record,
// order bin and permutation
constexpr int64_t kSlotBytesPerRay =
    6 * sizeof(double) + sizeof(double) + sizeof(int32_t) + sizeof(RayPrep) + sizeof(uint8_t) + sizeof(int32_t);

static void free_pipe(vgrid_t *g) {
    for (int k = 0; k < 2; k++) {
        void *ptrs[] = {g->d_hin[k], g->d_hout[k], g->d_hst[k], g->d_hstart[k], g->d_hbin[k], g->d_horder[k]};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        g->d_hin[k] = nullptr;
        g->d_hout[k] = nullptr;
        g->d_hst[k] = nullptr;
        g->d_hstart[k] = nullptr;
        g->d_hbin[k] = nullptr;
        g->d_horder[k] = nullptr;
    }
    g->device_bytes -= g->host_cap * 2 * kSlotBytesPerRay;
    g->host_cap = 0;
}

static void free_grid(vgrid_t *g) {
    if (!g) return;
    free_events(g);
    free_pipe(g);
    for (int k = 0; k < 2; k++) {
        if (g->ev_in[k]) cudaEventDestroy(g->ev_in[k]);
        if (g->ev_k[k]) cudaEventDestroy(g->ev_k[k]);
        if (g->ev_out[k]) cudaEventDestroy(g->ev_out[k]);
    }
    for (int k = 0; k < 2; k++)
        if (g->ev_prep[k]) cudaEventDestroy(g->ev_prep[k]);
    if (g->s_h2d) cudaStreamDestroy(g->s_h2d);
    if (g->s_d2h) cudaStreamDestroy(g->s_d2h);
    if (g->s_loc) cudaStreamDestroy(g->s_loc);
    if (g->d_hhist) cudaFree(g->d_hhist);
    if (g->d_hqueue) cudaFree(g->d_hqueue);
    if (g->d_hset) cudaFree(g->d_hset);
    void *ptrs[] = {g->d_desc,  g->d_site,  g->d_cells, g->d_rec64, g->d_rel,   g->d_dens,  g->d_bin,   g->d_hist,
                    g->d_order, g->d_perm,  g->d_blk_off, g->d_blk_rec, g->d_queue, g->d_stats, g->d_set,
                    g->d_start, g->d_scan,  g->d_entry, g->d_slots, g->d_chunk_meta, g->d_chunk_inv, g->d_coff, g->d_cursor};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete g;
}

int vgrid_create(const double *sites, int64_t M, const double bbox[6], const vgrid_opts *opts, vgrid_t **out) {
    g_err.clear();
    if (!out) return fail(VGRID_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!sites || !bbox) return fail(VGRID_ERR_ARG, "sites or bbox is NULL");
    if (M < 1) return fail(VGRID_ERR_ARG, "need at least one site");
    if (M > (int64_t)1 << 30) return fail(VGRID_ERR_ARG, "too many sites");
    for (int c = 0; c < 3; c++)
        if (!std::isfinite(bbox[c]) || !std::isfinite(bbox[3 + c]) || !(bbox[c] < bbox[3 + c]))
            return fail(VGRID_ERR_ARG, "bbox must be finite with min < max on every axis");
    vgrid_opts o;
    vgrid_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.blocks_per_site > 0)) o.blocks_per_site = 8.0;
    if (o.max_steps <= 0) o.max_steps = 100000;
    if (o.zero_run_max < 0) return fail(VGRID_ERR_ARG, "zero_run_max must be >= 0");
    if (o.domain != VGRID_DOMAIN_BOX && o.domain != VGRID_DOMAIN_SPHERE)
        return fail(VGRID_ERR_ARG, "domain must be VGRID_DOMAIN_BOX or VGRID_DOMAIN_SPHERE");
    if (o.domain == VGRID_DOMAIN_SPHERE) {
        const double R = o.sphere[3];
        if (!(R > 0) || !std::isfinite(R)) return fail(VGRID_ERR_ARG, "sphere radius must be positive and finite");
        for (int c = 0; c < 3; c++)
            if (!std::isfinite(o.sphere[c]) || !(o.sphere[c] - R >= bbox[c]) || !(o.sphere[c] + R <= bbox[3 + c]))
                return fail(VGRID_ERR_ARG, "the sphere must lie inside bbox");
    }
    const auto t0 = std::chrono::steady_clock::now();

    // sites as float32 values (the device stores float4)
    std::vector<double> S(3 * M);
    for (int64_t i = 0; i < 3 * M; i++) {
        const double v = sites[i];
        if (!std::isfinite(v)) return fail(VGRID_ERR_ARG, "site " + std::to_string(i / 3) + " is not finite");
        const double f = (double)(float)v;
        if (f != v && !o.round_sites)
            return fail(VGRID_ERR_ARG, "site " + std::to_string(i / 3) + " is not representable in float32");
        S[i] = f;
    }
    for (int64_t i = 0; i < M; i++)
        for (int c = 0; c < 3; c++)
            if (!(S[3 * i + c] >= bbox[c] && S[3 * i + c] <= bbox[3 + c]))
                return fail(VGRID_ERR_OUTSIDE, "site " + std::to_string(i) + " lies outside the box");
    if (o.domain == VGRID_DOMAIN_SPHERE)
        for (int64_t i = 0; i < M; i++) {
            const double dx = S[3 * i] - o.sphere[0], dy = S[3 * i + 1] - o.sphere[1], dz = S[3 * i + 2] - o.sphere[2];
            if (!((dx * dx + dy * dy) + dz * dz <= o.sphere[3] * o.sphere[3]))
                return fail(VGRID_ERR_OUTSIDE, "site " + std::to_string(i) + " lies outside the sphere");
        }
    // duplicates: coinciding sites share a Morton code, so with the Morton
    // order they sit in one run of equal codes (runs are a few sites long);
    // without it, a lexicographic sort puts them next to each other
    std::vector<int32_t> perm;
    std::vector<uint64_t> codes;
    if (o.reorder) {
        vg::morton_order(S.data(), M, bbox, perm, &codes, o.threads);
        for (int64_t r0 = 0; r0 < M;) {
            int64_t r1 = r0 + 1;
            while (r1 < M && codes[r1] == codes[r0]) r1++;
            for (int64_t a = r0; a < r1; a++)
                for (int64_t b = a + 1; b < r1; b++)
                    if (std::equal(&S[3 * (int64_t)perm[a]], &S[3 * (int64_t)perm[a]] + 3, &S[3 * (int64_t)perm[b]]))
                        return fail(VGRID_ERR_DUP_SITE, "sites " + std::to_string(std::min(perm[a], perm[b])) +
                                                            " and " + std::to_string(std::max(perm[a], perm[b])) +
                                                            " coincide");
            r0 = r1;
        }
    } else {
        std::vector<int32_t> ord(M);
        for (int64_t i = 0; i < M; i++) ord[i] = (int32_t)i;
        std::sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
            return std::lexicographical_compare(&S[3 * (int64_t)a], &S[3 * (int64_t)a] + 3, &S[3 * (int64_t)b],
                                                &S[3 * (int64_t)b] + 3);
        });
        for (int64_t i = 1; i < M; i++)
            if (std::equal(&S[3 * (int64_t)ord[i]], &S[3 * (int64_t)ord[i]] + 3, &S[3 * (int64_t)ord[i - 1]]))
                return fail(VGRID_ERR_DUP_SITE, "sites " + std::to_string(ord[i - 1]) + " and " +
                                                    std::to_string(ord[i]) + " coincide");
        perm.resize(M);
        for (int64_t i = 0; i < M; i++) perm[i] = (int32_t)i;
    }

    const auto t_checked = std::chrono::steady_clock::now();
    vgrid_t *g = new vgrid();
    g->M = M;
    g->opts = o;
    auto lap = [&](int k, std::chrono::steady_clock::time_point &since) {
        const auto now = std::chrono::steady_clock::now();
        g->phase_seconds[k] = std::chrono::duration<double>(now - since).count();
        since = now;
    };
    auto t_lap = t_checked;
    g->phase_seconds[0] = std::chrono::duration<double>(t_checked - t0).count();
    g->perm.swap(perm);
    g->inv.resize(M);
    for (int64_t i = 0; i < M; i++) g->inv[g->perm[i]] = (int32_t)i;
    std::vector<double> Si(3 * M);
    for (int64_t i = 0; i < M; i++)
        for (int c = 0; c < 3; c++) Si[3 * i + c] = S[3 * (int64_t)g->perm[i] + c];

    lap(1, t_lap);
    std::string err;
    if (o.gpu_build && o.host_only) {
        delete g;
        return fail(VGRID_ERR_ARG, "gpu_build and host_only exclude each other");
    }
    const int brc = o.gpu_build ? vg::build_cells_gpu(Si.data(), M, bbox, o.threads, g->cells, err, &g->host_fallback_cells)
                                : vg::build_cells(Si.data(), M, bbox, o.threads, g->cells, err);
    if (brc != 0) {
        delete g;
        return fail(o.gpu_build ? VGRID_ERR_CUDA : VGRID_ERR_BUILD, err);
    }
    lap(2, t_lap);
    vg::build_blocks(bbox, g->cells.bbox, M, o.blocks_per_site, g->blocks, o.threads);
    lap(3, t_lap);
    if ((int64_t)(g->blocks.idx.size() + g->blocks.off.size()) + 2 >= ((int64_t)1 << 31)) {  // with the padding
        delete g;
        return fail(VGRID_ERR_NOMEM, "block lists exceed 2^31 entries; lower blocks_per_site");
    }

    // absolute cell blocks (offsets A): header (caller id, count, rho = 1,
    // F), then one record per neighbour (site of the neighbour, its A) or
    // wall. Relative cell blocks (offsets F, even): (site, record count),
    // (caller id, rho = 1, N1max, A), then one record per cell neighbour
    // (fl(p_j - p_i) in float32, its F), NaN-padded to an even count of
    // records (at least four). N1max bounds |fl(p_j - p_i)|_1 over the
    // records from above.
    std::vector<int64_t> boffs(M + 1, 0), foffs(M + 1, 0);
    std::vector<int32_t> ncell(M, 0);
    vg::parallel_for(M, o.threads, 1 << 14, [&](int64_t b0, int64_t e0) {
        for (int64_t i = b0; i < e0; i++)
            for (int64_t q = g->cells.off[i]; q < g->cells.off[i + 1]; q++) ncell[i] += g->cells.idx[q] >= 0;
    });
    for (int64_t i = 0; i < M; i++) {
        const int64_t b = g->cells.off[i], e = g->cells.off[i + 1];
        boffs[i + 1] = boffs[i] + 1 + (e - b);
        foffs[i + 1] = foffs[i] + 2 + std::max<int64_t>(4, (ncell[i] + 1) & ~(int64_t)1);
    }
    if (boffs[M] + 8 >= ((int64_t)1 << 31) || foffs[M] + 8 >= ((int64_t)1 << 31)) {
        delete g;
        return fail(VGRID_ERR_NOMEM, "cell blocks exceed 2^31 records");
    }
    const int64_t nrec = boffs[M] + 8;   // room past the end for the last block's reads
    const int64_t nrel = foffs[M] + 8;
    g->rel_bytes = nrel * (int64_t)sizeof(float4);
    // every float of both block arrays is written below (in parallel), so
    // they are allocated without the sequential zero fill
    std::unique_ptr<float[]> blocks(new float[4 * nrec]), rel(new float[4 * nrel]);
    std::vector<float> site4(4 * M);
    auto put_int = [](float *dst, int32_t v) { std::memcpy(dst, &v, 4); };
    const float fnan = std::numeric_limits<float>::quiet_NaN();
    // every cell writes only its own blocks and site entry
    vg::parallel_for(M, o.threads, 1 << 12, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; i++) {
        const int64_t b = g->cells.off[i], e = g->cells.off[i + 1];
        const float pi[3] = {(float)Si[3 * i + 0], (float)Si[3 * i + 1], (float)Si[3 * i + 2]};
        float *h = &blocks[4 * boffs[i]];
        put_int(h + 0, g->perm[i]);
        put_int(h + 1, (int32_t)(e - b));
        h[2] = 1.0f;
        put_int(h + 3, (int32_t)foffs[i]);
        float *f = &rel[4 * foffs[i]];
        const int64_t c4 = foffs[i + 1] - foffs[i] - 2;
        f[0] = pi[0];
        f[1] = pi[1];
        f[2] = pi[2];
        put_int(f + 3, (int32_t)c4);
        put_int(f + 4, g->perm[i]);
        f[5] = 1.0f;
        put_int(f + 7, (int32_t)boffs[i]);
        double n1max = 0.0;
        int64_t k = 0;
        for (int64_t q = b; q < e; q++) {
            float *r = &blocks[4 * (boffs[i] + 1 + (q - b))];
            const int32_t j = g->cells.idx[q];
            if (j >= 0) {
                float pj[3];
                for (int c = 0; c < 3; c++) pj[c] = (float)Si[3 * (int64_t)j + c];
                r[0] = pj[0];
                r[1] = pj[1];
                r[2] = pj[2];
                put_int(r + 3, (int32_t)boffs[j]);
                float *rr = &f[4 * (2 + k++)];
                double n1 = 0.0;
                for (int c = 0; c < 3; c++) {
                    volatile float d = pj[c] - pi[c];  // one float32 rounding, as on the device
                    rr[c] = d;
                    n1 += std::fabs((double)rr[c]);
                }
                put_int(rr + 3, (int32_t)foffs[j]);
                n1max = std::max(n1max, n1);
            } else {
                r[0] = r[1] = r[2] = 0.0f;
                put_int(r + 3, j);
            }
        }
        for (; k < c4; k++) {
            float *rr = &f[4 * (2 + k)];
            rr[0] = rr[1] = rr[2] = fnan;
            put_int(rr + 3, -8);
        }
        float n1f = (float)(n1max * (1.0 + 1e-6));
        if ((double)n1f < n1max * (1.0 + 1e-6)) n1f = std::nextafter(n1f, INFINITY);
        f[6] = n1f;
        site4[4 * i + 0] = pi[0];
        site4[4 * i + 1] = pi[1];
        site4[4 * i + 2] = pi[2];
        put_int(&site4[4 * i + 3], (int32_t)foffs[i]);
    }
    });
    for (int64_t r = boffs[M]; r < nrec; r++) {
        blocks[4 * r] = blocks[4 * r + 1] = blocks[4 * r + 2] = 0.0f;
        put_int(&blocks[4 * r + 3], -8);
    }
    for (int64_t r = foffs[M]; r < nrel; r++) {
        rel[4 * r] = rel[4 * r + 1] = rel[4 * r + 2] = fnan;
        put_int(&rel[4 * r + 3], -8);
    }
    // block lists on the device: each padded to an even length with NaN
    // records (id -1), so every list starts on a 32-byte boundary and is read
    // in 256-bit pairs
    const size_t nblk = g->blocks.off.size() - 1;
    std::vector<int32_t> boff(nblk + 1, 0);
    for (size_t i = 0; i < nblk; i++) {
        const int64_t len = g->blocks.off[i + 1] - g->blocks.off[i];
        boff[i + 1] = boff[i] + (int32_t)((len + 1) & ~(int64_t)1);
    }

    // coarse density grid for the ray order: about 2^18 near-cubic cells
    // over the box, each holding (sites per unit volume)^(1/3), which is
    // proportional to the cell faces a ray crosses per unit length
    int32_t ddim[3];
    {
        const double ext[3] = {bbox[3] - bbox[0], bbox[4] - bbox[1], bbox[5] - bbox[2]};
        const double cs = std::cbrt(ext[0] * ext[1] * ext[2] / 262144.0);
        for (int c = 0; c < 3; c++) ddim[c] = (int32_t)std::min<long>(std::max<long>(std::lround(ext[c] / cs), 1), 256);
    }
    std::vector<float> dens((size_t)ddim[0] * ddim[1] * ddim[2], 0.0f);
    {
        std::vector<int64_t> cnt(dens.size(), 0);
        for (int64_t i = 0; i < M; i++) {
            int64_t idx = 0;
            for (int c = 0; c < 3; c++) {
                const double f = (Si[3 * i + c] - bbox[c]) / (bbox[3 + c] - bbox[c]) * ddim[c];
                const int64_t ic = std::min<int64_t>(std::max<int64_t>((int64_t)f, 0), ddim[c] - 1);
                idx = idx * ddim[c] + ic;
            }
            cnt[idx]++;
        }
        const double vol = (bbox[3] - bbox[0]) * (bbox[4] - bbox[1]) * (bbox[5] - bbox[2]) /
                           ((double)ddim[0] * ddim[1] * ddim[2]);
        for (size_t q = 0; q < dens.size(); q++) dens[q] = (float)std::cbrt(std::max(0.25, (double)cnt[q]) / vol);
    }

    lap(4, t_lap);
    if (o.host_only) {
        g->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int c = 0; c < 3; c++) {
            g->hd.lo[c] = bbox[c];
            g->hd.hi[c] = bbox[3 + c];
        }
        g->device = -1;
        *out = g;
        return VGRID_OK;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        delete g;
        return fail(VGRID_ERR_CUDA, "no CUDA device");
    }
    g->device = dev;
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
    int rc = VGRID_OK;
#define VG_ALLOC(p, n)                                              \
    if ((rc = dmalloc(&(p), (size_t)(n), g->device_bytes)) != 0) { \
        free_grid(g);                                               \
        return rc;                                                  \
    }
    VG_ALLOC(g->d_site, M);
    VG_ALLOC(g->d_cells, nrec);
    VG_ALLOC(g->d_rec64, 2 * (size_t)nrec);
    VG_ALLOC(g->d_rel, nrel);
    VG_ALLOC(g->d_perm, M);
    VG_ALLOC(g->d_blk_off, boff.size());
    VG_ALLOC(g->d_blk_rec, (size_t)boff[nblk] + 2);
    VG_ALLOC(g->d_dens, dens.size());
    VG_ALLOC(g->d_desc, 1);
    VG_ALLOC(g->d_queue, 1);
    VG_ALLOC(g->d_stats, 1);
    VG_ALLOC(g->d_set, 1);
#undef VG_ALLOC
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpy(g->d_site, site4.data(), sizeof(float) * 4 * M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_cells, blocks.get(), sizeof(float) * 4 * nrec, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_rel, rel.get(), sizeof(float) * 4 * nrel, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_perm, g->perm.data(), sizeof(int32_t) * M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_blk_off, boff.data(), sizeof(int32_t) * boff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_dens, dens.data(), sizeof(float) * dens.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const float fnan = std::numeric_limits<float>::quiet_NaN();
        // every entry is written below (the lists in parallel, each with its
        // NaN padding, then the two entries past the end), so the buffer is
        // allocated without a fill
        const size_t nbrec = (size_t)boff[nblk] + 2;
        std::unique_ptr<float[]> brec(new float[4 * nbrec]);
        auto put_nan = [&](size_t q) {
            brec[4 * q + 0] = brec[4 * q + 1] = brec[4 * q + 2] = fnan;
            put_int(&brec[4 * q + 3], -1);
        };
        put_nan(nbrec - 2);
        put_nan(nbrec - 1);
        // each list ordered by the sites' distance from its block's centre,
        // flo_hi + (i + 1/2) fbw per axis in float32 (the operations the
        // start-cell search repeats), ties by cell: the search stops once the
        // rest of the list is certainly farther than its best site
        const int32_t *bd = g->blocks.dim;
        float fbw[3], flo[3];
        for (int c = 0; c < 3; c++) {
            fbw[c] = (float)((bbox[3 + c] - bbox[c]) / bd[c]);
            flo[c] = (float)bbox[c];
        }
        vg::parallel_for((int64_t)nblk, o.threads, 1 << 12, [&](int64_t b0, int64_t b1) {
            std::vector<std::pair<double, int32_t>> ord;
            for (int64_t b = b0; b < b1; b++) {
                const int64_t bk[3] = {b / ((int64_t)bd[1] * bd[2]), (b / bd[2]) % bd[1], b % bd[2]};
                double cen[3];
                for (int c = 0; c < 3; c++) {
                    volatile float t = (float)bk[c] + 0.5f;
                    volatile float m = t * fbw[c];
                    cen[c] = (double)(float)(flo[c] + m);
                }
                ord.clear();
                for (int64_t q = g->blocks.off[b]; q < g->blocks.off[b + 1]; q++) {
                    const int32_t c = g->blocks.idx[q];
                    double d2 = 0.0;
                    for (int a = 0; a < 3; a++) {
                        const double d = (double)(float)Si[3 * (int64_t)c + a] - cen[a];
                        d2 += d * d;
                    }
                    ord.emplace_back(d2, c);
                }
                std::sort(ord.begin(), ord.end());
                for (int64_t q = g->blocks.off[b]; q < g->blocks.off[b + 1]; q++) {
                    const int32_t c = ord[(size_t)(q - g->blocks.off[b])].second;
                    float *r = &brec[4 * ((size_t)boff[b] + (size_t)(q - g->blocks.off[b]))];
                    r[0] = (float)Si[3 * (int64_t)c + 0];
                    r[1] = (float)Si[3 * (int64_t)c + 1];
                    r[2] = (float)Si[3 * (int64_t)c + 2];
                    put_int(r + 3, c);
                }
                const size_t len = (size_t)(g->blocks.off[b + 1] - g->blocks.off[b]);
                for (size_t q = (size_t)boff[b] + len; q < (size_t)boff[b + 1]; q++) put_nan(q);
            }
        });
        e = cudaMemcpy(g->d_blk_rec, brec.get(), sizeof(float) * 4 * nbrec, cudaMemcpyHostToDevice);
    }

    if (e == cudaSuccess) {
        e = vg::launch_build_rec64(g->d_site, g->d_rel, g->d_cells, M, nrec, g->d_rec64, g->sms, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }

    GridDev &hd = g->hd;
    hd.site = g->d_site;
    hd.cells = g->d_cells;
    hd.rec64 = g->d_rec64;
    hd.rel = g->d_rel;
    hd.perm = g->d_perm;
    hd.blk_off = g->d_blk_off;
    hd.blk_rec = g->d_blk_rec;
    hd.dens = g->d_dens;
    {
        // ray order: by length alone while the relative blocks fit in half of
        // L2, else by (length, start-cell range) to keep the rays in flight
        // on one part of the grid
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device);
        hd.ospatial = (double)nrel * sizeof(float4) > 0.5 * (double)l2 ? 16 : 1;
    }
    double dmax = 0;
    for (int c = 0; c < 3; c++) {
        hd.lo[c] = bbox[c];
        hd.hi[c] = bbox[3 + c];
        hd.bdim[c] = g->blocks.dim[c];
        hd.bscale[c] = (double)g->blocks.dim[c] / (bbox[3 + c] - bbox[c]);
        hd.lokey[c] = vg::dkey(bbox[c]);
        hd.hikey[c] = vg::dkey(bbox[3 + c]);
        hd.flo_hi[c] = (float)bbox[c];
        hd.flo_lo[c] = (float)(bbox[c] - (double)hd.flo_hi[c]);
        hd.fbscale[c] = (float)hd.bscale[c];
        hd.fbw[c] = (float)((bbox[3 + c] - bbox[c]) / g->blocks.dim[c]);
        hd.ddim[c] = ddim[c];
        hd.dscale[c] = (float)((double)ddim[c] / (bbox[3 + c] - bbox[c]));
        dmax = std::max(dmax, std::max(std::fabs(bbox[c]), std::fabs(bbox[3 + c])));
    }
    const double dx = bbox[3] - bbox[0], dy = bbox[4] - bbox[1], dz = bbox[5] - bbox[2];
    const double diag = std::sqrt(dx * dx + dy * dy + dz * dz);
    hd.M = (int32_t)M;
    hd.kappa = 1.0f;
    hd.eps64 = 1e-12 * diag;
    hd.eps32 = 1e-6 * diag;
    hd.scale = dmax + diag;
    hd.max_steps = o.max_steps;
    hd.zmax = o.zero_run_max;
    hd.domain = o.domain;
    hd.pad1 = 0;
    for (int c = 0; c < 4; c++) hd.sph[c] = o.domain == VGRID_DOMAIN_SPHERE ? o.sphere[c] : 0.0;
    if (e == cudaSuccess) e = cudaMemcpy(g->d_desc, &hd, sizeof(GridDev), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_grid(g);
        return fail(VGRID_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    lap(5, t_lap);
    g->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = g;
    return VGRID_OK;
}

int vgrid_destroy(vgrid_t *g) {
    if (!g) return VGRID_OK;
    if (g->device < 0) {
        delete g;
        return VGRID_OK;
    }
    DeviceGuard dg(g->device);
    free_grid(g);
    return VGRID_OK;
}

int vgrid_info(const vgrid_t *g, vgrid_info_t *info) {
    if (!g || !info) return fail(VGRID_ERR_ARG, "null argument");
    info->M = g->M;
    info->nnz = (int64_t)g->cells.idx.size();
    info->block_entries = (int64_t)g->blocks.idx.size();
    for (int c = 0; c < 3; c++) {
        info->block_dim[c] = g->blocks.dim[c];
        info->box[c] = g->hd.lo[c];
        info->box[3 + c] = g->hd.hi[c];
    }
    info->build_seconds = g->build_seconds;
    for (int k = 0; k < 6; k++) info->phase_seconds[k] = g->phase_seconds[k];
    info->device_bytes = g->device_bytes;
    info->host_fallback_cells = g->host_fallback_cells;
    info->rel_bytes = g->rel_bytes;
    return VGRID_OK;
}

int vgrid_get_neighbors(const vgrid_t *g, int64_t *off, int32_t *idx) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    int64_t pos = 0;
    std::vector<int32_t> tmp;
    for (int64_t c = 0; c < g->M; c++) {
        const int32_t i = g->inv[c];
        const int64_t b = g->cells.off[i], e = g->cells.off[i + 1];
        if (off) off[c] = pos;
        if (idx) {
            tmp.clear();
            for (int64_t q = b; q < e; q++) {
                const int32_t j = g->cells.idx[q];
                tmp.push_back(j >= 0 ? g->perm[j] : j);
            }
            std::sort(tmp.begin(), tmp.end());
            std::copy(tmp.begin(), tmp.end(), idx + pos);
        }
        pos += e - b;
    }
    if (off) off[g->M] = pos;
    return VGRID_OK;
}

int vgrid_get_cells(const vgrid_t *g, double *volume, double *bbox) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    for (int64_t c = 0; c < g->M; c++) {
        const int32_t i = g->inv[c];
        if (volume) volume[c] = g->cells.vol[i];
        if (bbox)
            for (int k = 0; k < 6; k++) bbox[6 * c + k] = g->cells.bbox[6 * (int64_t)i + k];
    }
    return VGRID_OK;
}

int vgrid_set_density(vgrid_t *g, const float *rho, float kappa, vgrid_stream_t stream) {
    if (!g || !rho) return fail(VGRID_ERR_ARG, "null argument");
    if (g->device < 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    if (!std::isfinite(kappa)) return fail(VGRID_ERR_ARG, "kappa is not finite");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    VG_CUDA(vg::launch_permute_density(rho, g->d_perm, g->d_site, g->M, g->d_cells, g->d_rel, s));
    g->hd.kappa = kappa;
    VG_CUDA(vg::launch_put_grid(g->d_desc, g->hd, s));
    return VGRID_OK;
}

int vgrid_set_launch(vgrid_t *g, const vgrid_launch *l) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (!l) {
        g->launch = vgrid_launch{1, 128, 0, 1, 0};
        return VGRID_OK;
    }
    if (!valid_lpr(l->lanes_per_ray)) return fail(VGRID_ERR_ARG, "lanes_per_ray must be 1, 2, 4 or 8");
    if (l->fp64_lanes_per_ray != 0 && !valid_lpr(l->fp64_lanes_per_ray))
        return fail(VGRID_ERR_ARG, "fp64_lanes_per_ray must be 0, 1, 2, 4 or 8");
    if (l->block < 32 || l->block > 256 || l->block % 32) return fail(VGRID_ERR_ARG, "block must be 32..256, multiple of 32");
    if (l->blocks_per_sm < 0) return fail(VGRID_ERR_ARG, "blocks_per_sm must be >= 0");
    if (l->order < -1 || l->order > 1) return fail(VGRID_ERR_ARG, "order must be -1, 0 or 1");
    g->launch = *l;
    return VGRID_OK;
}

int vgrid_get_launch(const vgrid_t *g, vgrid_launch *l) {
    if (!g || !l) return fail(VGRID_ERR_ARG, "null argument");
    *l = g->launch;
    return VGRID_OK;
}

}  // extern "C"

namespace {

// record event pair `which` (0: start cells, 1: traversal) around a launch
cudaEvent_t next_event(vgrid_t *g, int which, int half) {
    auto &v = which == 0 ? g->ev_loc : g->ev_trace;
    size_t &n = which == 0 ? g->n_loc : g->n_trace;
    if (half == 0 && n == v.size()) {
        std::array<cudaEvent_t, 2> p{};
        if (cudaEventCreate(&p[0]) != cudaSuccess || cudaEventCreate(&p[1]) != cudaSuccess) return nullptr;
        v.push_back(p);
    }
    if (half == 0) return v[n][0];
    return v[n++][1];
}

void mark(vgrid_t *g, int which, int half, cudaStream_t s) {
    if (!g->timing) return;
    cudaEvent_t e = next_event(g, which, half);
    if (e) cudaEventRecord(e, s);
}

int ensure_start(vgrid_t *g, int64_t N) {
    if (N <= g->start_cap) return VGRID_OK;
    if (g->d_start) {
        cudaFree(g->d_start);
        g->device_bytes -= g->start_cap * (int64_t)sizeof(RayPrep);
        g->d_start = nullptr;
        g->start_cap = 0;
    }
    int rc = dmalloc(&g->d_start, (size_t)N, g->device_bytes);
    if (rc) return rc;
    g->start_cap = N;
    return VGRID_OK;
}

int ensure_entry(vgrid_t *g, int64_t N) {
    if (N <= g->entry_cap) return VGRID_OK;
    if (g->d_entry) {
        cudaFree(g->d_entry);
        g->device_bytes -= g->entry_cap * 3 * (int64_t)sizeof(double);
        g->d_entry = nullptr;
        g->entry_cap = 0;
    }
    int rc = dmalloc(&g->d_entry, (size_t)(3 * N), g->device_bytes);
    if (rc) return rc;
    g->entry_cap = N;
    return VGRID_OK;
}

int ensure_order(vgrid_t *g, int64_t N) {
    if (!g->d_hist) {
        int rc = dmalloc(&g->d_hist, 2 * vg::kOrderBins, g->device_bytes);
        if (rc) return rc;
    }
    if (N <= g->order_cap) return VGRID_OK;
    if (g->d_bin) cudaFree(g->d_bin);
    if (g->d_order) cudaFree(g->d_order);
    g->device_bytes -= g->order_cap * (int64_t)(sizeof(uint8_t) + sizeof(int32_t));
    g->d_bin = nullptr;
    g->d_order = nullptr;
    g->order_cap = 0;
    int rc = dmalloc(&g->d_bin, (size_t)N, g->device_bytes);
    if (!rc) rc = dmalloc(&g->d_order, (size_t)N, g->device_bytes);
    if (rc) return rc;
    g->order_cap = N;
    return VGRID_OK;
}

int ensure_scan(vgrid_t *g, int64_t N) {
    const int64_t need = vg::scan_tmp_elems(N);
    if (need <= g->scan_cap) return VGRID_OK;
    if (g->d_scan) {
        cudaFree(g->d_scan);
        g->device_bytes -= g->scan_cap * (int64_t)sizeof(int64_t);
        g->d_scan = nullptr;
        g->scan_cap = 0;
    }
    int rc = dmalloc(&g->d_scan, (size_t)need, g->device_bytes);
    if (rc) return rc;
    g->scan_cap = need;
    return VGRID_OK;
}

// chunk pool of segment mode: `chunks` chunks of kSegChunk slots of
// slot_bytes, their (ray, position) records and the inverse map, and the
// chunk offsets of N rays
int ensure_chunks(vgrid_t *g, int64_t N, int64_t chunks, int slot_bytes) {
    if (!g->d_cursor) {
        int rc = dmalloc(&g->d_cursor, 1, g->device_bytes);
        if (rc) return rc;
    }
    if (N + 1 > g->coff_cap) {
        if (g->d_coff) cudaFree(g->d_coff);
        g->device_bytes -= g->coff_cap * (int64_t)sizeof(int64_t);
        g->d_coff = nullptr;
        g->coff_cap = 0;
        int rc = dmalloc(&g->d_coff, (size_t)(N + 1), g->device_bytes);
        if (rc) return rc;
        g->coff_cap = N + 1;
    }
    const int64_t bytes = chunks * vg::kSegChunk * slot_bytes;  // a multiple of 64
    if (bytes > g->slot_bytes) {
        if (g->d_slots) cudaFree(g->d_slots);
        g->device_bytes -= g->slot_bytes;
        g->d_slots = nullptr;
        g->slot_bytes = 0;
        int rc = dmalloc(&g->d_slots, (size_t)(bytes / 16), g->device_bytes);
        if (rc) return rc;
        g->slot_bytes = bytes;
    }
    if (chunks > g->meta_cap) {
        if (g->d_chunk_meta) cudaFree(g->d_chunk_meta);
        if (g->d_chunk_inv) cudaFree(g->d_chunk_inv);
        g->device_bytes -= g->meta_cap * (int64_t)(sizeof(int2) + sizeof(int32_t));
        g->d_chunk_meta = nullptr;
        g->d_chunk_inv = nullptr;
        g->meta_cap = 0;
        int rc = dmalloc(&g->d_chunk_meta, (size_t)chunks, g->device_bytes);
        if (!rc) rc = dmalloc(&g->d_chunk_inv, (size_t)chunks, g->device_bytes);
        if (rc) return rc;
        g->meta_cap = chunks;
    }
    return VGRID_OK;
}

// persistent grid size for a trace kernel
int persistent_blocks(const void *fn, const vgrid_launch &l, int sms, int64_t work_items) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, l.block, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    if (l.blocks_per_sm > 0 && l.blocks_per_sm < per_sm) per_sm = l.blocks_per_sm;
    int64_t blocks = (int64_t)per_sm * sms;
    const int64_t need = (work_items * l.lanes_per_ray + l.block - 1) / l.block;
    if (need < blocks) blocks = need > 0 ? need : 1;
    return (int)blocks;
}

int launch_trace(const void *fn, const vgrid_launch &l, int sms, int64_t total, vg::TraceArgs &a, cudaStream_t s) {
    if (!fn) return fail(VGRID_ERR_ARG, "no kernel for this precision/mode");
    const int blocks = persistent_blocks(fn, l, sms, total);
    void *args[] = {&a};
    VG_CUDA(cudaLaunchKernel(fn, dim3(blocks), dim3(l.block), args, 0, s));
    vg::count_launches(1);
    return VGRID_OK;
}

// resident lanes of a persistent float32 launch
int64_t resident_lanes(vgrid_t *g, const void *fn, const vgrid_launch &l) {
    return (int64_t)persistent_blocks(fn, l, g->sms, INT64_MAX / 16) * l.block / l.lanes_per_ray;
}

// start records (float32 form, or float64 with fp64) for the set in
// g->d_set; with the ray order (see vgrid_launch.order) also the
// permutation, which goes to *order
int locate_start(vgrid_t *g, const void *fn, const vgrid_launch &l, int64_t N, const int32_t **order, cudaStream_t s,
                bool fp64 = false) {
    *order = nullptr;
    const int prep = fp64 ? vg::PREP_FP64 : vg::PREP_FP32;
    const bool want = l.order == 1 || (l.order == 0 && N >= 2 * resident_lanes(g, fn, l));
    if (!want || N > INT32_MAX) {
        VG_CUDA(vg::launch_locate(g->d_desc, g->d_set, 1, N, prep, nullptr, g->sms, s));
        return VGRID_OK;
    }
    int rc = ensure_order(g, N);
    if (rc) return rc;
    const vg::RayOrder ord{g->d_bin, g->d_hist, g->d_order};
    VG_CUDA(cudaMemsetAsync(g->d_hist, 0, 2 * vg::kOrderBins * sizeof(uint32_t), s));
    VG_CUDA(vg::launch_locate_ordered(g->d_desc, g->d_set, 1, N, ord, prep, g->sms, s));
    VG_CUDA(vg::launch_order(ord, N, g->sms, s));
    *order = g->d_order;
    return VGRID_OK;
}

// the kernel table's row for a precision (float32, float64, float32 with
// exact lengths) and the launch shape it runs with
static int precision_row(int precision, vgrid_launch &L) {
    if (precision == VGRID_FP64) {
        if (L.fp64_lanes_per_ray) L.lanes_per_ray = L.fp64_lanes_per_ray;
        return 1;
    }
    if (precision == VGRID_FP32_EXACT) {
        L.lanes_per_ray = 1;
        return 2;
    }
    return 0;
}

// tau (and status) of n device-resident rays on s; the counters restart
// only if reset_stats
int trace_tau_chunk(vgrid_t *g, const double *origin, const double *dir, int64_t n, int precision, void *tau,
                    int32_t *status, bool reset_stats, cudaStream_t s) {
    int rc = ensure_start(g, n);
    if (rc) return rc;
    vgrid_launch L = g->launch;
    const int fp64 = precision == VGRID_FP64;
    const int row = precision_row(precision, L);
    const vg::KernelSet &ks = kernels(L.lanes_per_ray);
    RaySetDev set{origin, dir, tau, status, g->d_start, n, 0, 0, 0};
    VG_CUDA(vg::launch_prepare(g->d_set, set, g->d_queue, reset_stats ? g->d_stats : nullptr, s));
    mark(g, 0, 0, s);
    const int32_t *order = nullptr;
    if ((rc = locate_start(g, ks.fn[row][vg::MODE_TAU], L, n, &order, s, fp64 != 0))) return rc;
    mark(g, 0, 1, s);
    vg::TraceArgs a{};
    a.grids = g->d_desc;
    a.sets = g->d_set;
    a.nsets = 1;
    a.total = n;
    a.queue = g->d_queue;
    a.stats = g->d_stats;
    a.g1 = g->hd;
    a.s1 = set;
    a.order = order;
    mark(g, 1, 0, s);
    if ((rc = launch_trace(ks.fn[row][vg::MODE_TAU], L, g->sms, n, a, s))) return rc;
    mark(g, 1, 1, s);
    return VGRID_OK;
}

// tau (and status) of one chunk of host-resident rays in slot k: its start
// records (and ray order) are prepared on s_loc once its rays are in and the
// slot's previous traversal is done, then it is traced on s. The start-cell
// pass of one chunk can thus run while the previous chunk is traced, in the
// SMs that traversal frees in its tail. The counters are not reset (calls
// that read them take trace_tau_chunk instead).
int trace_chunk_slot(vgrid_t *g, int k, const double *origin, const double *dir, int64_t n, int precision, void *tau,
                     int32_t *status, cudaStream_t s) {
    vgrid_launch L = g->launch;
    const int fp64 = precision == VGRID_FP64;
    const int row = precision_row(precision, L);
    const void *fn = kernels(L.lanes_per_ray).fn[row][vg::MODE_TAU];
    cudaStream_t t = g->s_loc;
    VG_CUDA(cudaStreamWaitEvent(t, g->ev_in[k], 0));
    VG_CUDA(cudaStreamWaitEvent(t, g->ev_k[k], 0));
    RaySetDev set{origin, dir, tau, status, g->d_hstart[k], n, 0, 0, 0};
    VG_CUDA(vg::launch_prepare(g->d_hset + k, set, g->d_hqueue + k, nullptr, t));
    const int prep = fp64 ? vg::PREP_FP64 : vg::PREP_FP32;
    const bool want = n <= INT32_MAX && (L.order == 1 || (L.order == 0 && n >= 2 * resident_lanes(g, fn, L)));
    const int32_t *order = nullptr;
    if (want) {
        const vg::RayOrder ord{g->d_hbin[k], g->d_hhist + 2 * vg::kOrderBins * k, g->d_horder[k]};
        VG_CUDA(cudaMemsetAsync(ord.hist, 0, 2 * vg::kOrderBins * sizeof(uint32_t), t));
        VG_CUDA(vg::launch_locate_ordered(g->d_desc, g->d_hset + k, 1, n, ord, prep, g->sms, t));
        VG_CUDA(vg::launch_order(ord, n, g->sms, t));
        order = ord.order;
    } else {
        VG_CUDA(vg::launch_locate(g->d_desc, g->d_hset + k, 1, n, prep, nullptr, g->sms, t));
    }
    VG_CUDA(cudaEventRecord(g->ev_prep[k], t));
    VG_CUDA(cudaStreamWaitEvent(s, g->ev_prep[k], 0));
    vg::TraceArgs a{};
    a.grids = g->d_desc;
    a.sets = g->d_hset + k;
    a.nsets = 1;
    a.total = n;
    a.queue = g->d_hqueue + k;
    a.stats = g->d_stats;
    a.g1 = g->hd;
    a.s1 = set;
    a.order = order;
    return launch_trace(fn, L, g->sms, n, a, s);
}

int read_stats(StatsDev *d, vgrid_stats *out, cudaStream_t s, StatsDev *host_copy = nullptr) {
    StatsDev h{};
    VG_CUDA(cudaMemcpyAsync(&h, d, sizeof(StatsDev), cudaMemcpyDeviceToHost, s));
    VG_CUDA(cudaStreamSynchronize(s));
    if (out) {
        out->rays = (int64_t)h.rays;
        out->crossings = (int64_t)h.crossings;
        out->decisions = (int64_t)h.decisions;
        out->rechecks = (int64_t)h.rechecks;
        out->fallbacks = (int64_t)h.fallbacks;
        out->zero_steps = (int64_t)h.zero_steps;
        out->step_limit = (int64_t)h.step_limit;
        out->outside = (int64_t)h.outside;
    }
    if (host_copy) *host_copy = h;
    if (h.bad_dir) return fail(VGRID_ERR_ARG, std::to_string(h.bad_dir) + " ray directions are not unit vectors");
    if (h.step_limit) return fail(VGRID_ERR_STEP_LIMIT, std::to_string(h.step_limit) + " rays hit the step limit");
    return VGRID_OK;
}

}  // namespace

extern "C" {

int vgrid_locate(vgrid_t *g, const double *pts, int64_t N, int precision, int32_t *cell, vgrid_stream_t stream) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (g->device < 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    if (N < 0 || (N > 0 && (!pts || !cell))) return fail(VGRID_ERR_ARG, "bad points or output");
    if (precision != VGRID_FP64 && precision != VGRID_FP32_RECHECK) return fail(VGRID_ERR_ARG, "bad precision");
    if (N == 0) return VGRID_OK;
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    // the cells go straight to `cell`: no start records
    RaySetDev set{pts, pts, nullptr, nullptr, nullptr, N, 0, 0, 0};
    VG_CUDA(vg::launch_prepare(g->d_set, set, g->d_queue, g->d_stats, s));
    VG_CUDA(vg::launch_locate(g->d_desc, g->d_set, 1, N,
                              precision == VGRID_FP32_RECHECK ? vg::PREP_CELL32 : vg::PREP_CELL64, cell, g->sms, s));
    return VGRID_OK;
}

int vgrid_trace(vgrid_t *g, const double *origin, const double *dir, int64_t N, int precision, int output, void *tau,
                int64_t *seg_off, int32_t *seg_cell, void *seg_len, int64_t seg_capacity, int32_t *ray_status,
                vgrid_stats *stats, vgrid_stream_t stream) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (g->device < 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    if (precision != VGRID_FP64 && precision != VGRID_FP32_RECHECK && precision != VGRID_FP32_EXACT)
        return fail(VGRID_ERR_ARG, "bad precision");
    const bool enter = (output & VGRID_ENTER) != 0;
    output &= ~VGRID_ENTER;
    if (output != VGRID_TAU && output != VGRID_SEGMENTS) return fail(VGRID_ERR_ARG, "bad output");
    if (N < 0 || (N > 0 && (!origin || !dir))) return fail(VGRID_ERR_ARG, "bad rays");
    if (output == VGRID_TAU && N > 0 && !tau) return fail(VGRID_ERR_ARG, "tau is NULL");
    if (output == VGRID_SEGMENTS && !seg_off) return fail(VGRID_ERR_ARG, "seg_off is NULL");
    if (seg_capacity < 0) return fail(VGRID_ERR_ARG, "negative capacity");
    if (output == VGRID_SEGMENTS && N > INT32_MAX) return fail(VGRID_ERR_ARG, "segment mode takes at most 2^31-1 rays");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) {
        if (output == VGRID_SEGMENTS) VG_CUDA(cudaMemsetAsync(seg_off, 0, sizeof(int64_t), s));
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return VGRID_OK;
    }
    int rc = ensure_start(g, N);
    if (rc) return rc;
    if (enter) {
        if ((rc = ensure_entry(g, N))) return rc;
        VG_CUDA(vg::launch_enter(origin, dir, N, g->d_desc, g->d_entry, g->sms, s));
        origin = g->d_entry;
    }
    const int fp64 = precision == VGRID_FP64;
    vgrid_launch L = g->launch;
    const int row = precision_row(precision, L);
    const vg::KernelSet &ks = kernels(L.lanes_per_ray);
    RaySetDev set{origin, dir, tau, ray_status, g->d_start, N, 0, 0, 0};
    VG_CUDA(vg::launch_prepare(g->d_set, set, g->d_queue, g->d_stats, s));
    mark(g, 0, 0, s);
    const int32_t *order = nullptr;
    {
        const void *fn = ks.fn[row][output == VGRID_TAU ? vg::MODE_TAU : vg::MODE_SEGS];
        if ((rc = locate_start(g, fn, L, N, &order, s, fp64 != 0))) return rc;
    }
    mark(g, 0, 1, s);
    vg::TraceArgs a{};
    a.order = order;
    a.grids = g->d_desc;
    a.sets = g->d_set;
    a.nsets = 1;
    a.total = N;
    a.queue = g->d_queue;
    a.stats = g->d_stats;
    a.g1 = g->hd;
    a.s1 = set;
    if (output == VGRID_TAU) {
        mark(g, 1, 0, s);
        if ((rc = launch_trace(ks.fn[row][vg::MODE_TAU], L, g->sms, N, a, s))) return rc;
        mark(g, 1, 1, s);
        if (stats) return read_stats(g->d_stats, stats, s);
        return VGRID_OK;
    }
    // segment lists in one traversal: each ray's segments go to chunks of
    // the pool, the counts are scanned into seg_off, and the chunks are
    // copied into the caller's arrays. The pool holds every chunk a ray
    // fills or starts (at most cap / kSegChunk + min(N, cap) when the total
    // fits the capacity) plus the page each warp may leave unused, so it
    // never runs out when the segments fit the caller's buffers.
    const void *fn = ks.fn[row][vg::MODE_SEGS];
    int64_t chunks = 0;
    if (seg_capacity > 0) {
        const int64_t warps = (int64_t)persistent_blocks(fn, L, g->sms, N) * L.block / 32;
        chunks = (seg_capacity + vg::kSegChunk - 1) / vg::kSegChunk + std::min(N, seg_capacity) +
                 warps * vg::kSegPage;
        if (chunks > INT32_MAX - 2 * vg::kSegPage)
            return fail(VGRID_ERR_ARG, "seg_capacity too large for one call (split the rays)");
    }
    if ((rc = ensure_scan(g, N))) return rc;
    if ((rc = ensure_chunks(g, N, chunks, fp64 ? 16 : 8))) return rc;
    VG_CUDA(cudaMemsetAsync(g->d_cursor, 0, sizeof(unsigned long long), s));
    a.seg_off = seg_off;
    a.seg_slots = g->d_slots;
    a.chunk_meta = g->d_chunk_meta;
    a.chunk_cursor = g->d_cursor;
    a.chunk_cap = chunks;
    mark(g, 1, 0, s);
    if ((rc = launch_trace(fn, L, g->sms, N, a, s))) return rc;
    mark(g, 1, 1, s);
    VG_CUDA(vg::launch_exclusive_scan(seg_off, N, g->d_scan, s));
    // the copy compares the total with the capacity on the device, so the
    // call synchronises once, at its end
    const bool have = seg_cell && seg_len;
    VG_CUDA(vg::launch_compact_segments(seg_off, N, chunks, g->d_cursor, g->d_chunk_meta, g->d_slots, fp64 != 0,
                                        have ? seg_capacity : 0, g->d_coff, g->d_scan, g->d_chunk_inv, seg_cell,
                                        seg_len, g->sms, s));
    int64_t total = 0;
    unsigned long long taken = 0;
    VG_CUDA(cudaMemcpyAsync(&total, seg_off + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    VG_CUDA(cudaMemcpyAsync(&taken, g->d_cursor, sizeof(taken), cudaMemcpyDeviceToHost, s));
    const int src = read_stats(g->d_stats, stats, s);  // synchronises
    if (total > seg_capacity || (total > 0 && !have))
        return fail(VGRID_ERR_CAPACITY, "segment buffers hold " + std::to_string(seg_capacity) + ", need " +
                                            std::to_string(total));
    if ((int64_t)taken > chunks)  // cannot happen when the total fits (see above)
        return fail(VGRID_ERR_CUDA, "segment chunk pool ran out");
    return src;
}

int vgrid_trace_host(vgrid_t *g, const double *origin, const double *dir, int64_t N, int precision, void *tau,
                     int32_t *ray_status, int64_t chunk, vgrid_stats *stats, vgrid_stream_t stream) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (g->device < 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    if (precision != VGRID_FP64 && precision != VGRID_FP32_RECHECK && precision != VGRID_FP32_EXACT)
        return fail(VGRID_ERR_ARG, "bad precision");
    if (N < 0 || (N > 0 && (!origin || !dir || !tau))) return fail(VGRID_ERR_ARG, "bad rays or tau");
    if (chunk < 0) return fail(VGRID_ERR_ARG, "negative chunk");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return VGRID_OK;
    }
    const int fp64 = precision == VGRID_FP64;
    const size_t tau_sz = fp64 ? sizeof(double) : sizeof(float);
    // one launch per chunk, and a launch lasts at least as long as its
    // longest ray, so by default the whole call is one chunk; the copies then
    // overlap with the traversal of the previous call
    if (chunk == 0) chunk = N;
    chunk = std::min(chunk, N);
    if (chunk > g->host_cap) {
        VG_CUDA(cudaDeviceSynchronize());  // an earlier call may still use the slots
        free_pipe(g);
        for (int k = 0; k < 2; k++) {
            int rc = dmalloc(&g->d_hin[k], (size_t)(6 * chunk), g->device_bytes);
            if (!rc) rc = dmalloc(reinterpret_cast<double **>(&g->d_hout[k]), (size_t)chunk, g->device_bytes);
            if (!rc) rc = dmalloc(&g->d_hst[k], (size_t)chunk, g->device_bytes);
            if (!rc) rc = dmalloc(&g->d_hstart[k], (size_t)chunk, g->device_bytes);
            if (!rc) rc = dmalloc(&g->d_hbin[k], (size_t)chunk, g->device_bytes);
            if (!rc) rc = dmalloc(&g->d_horder[k], (size_t)chunk, g->device_bytes);
            if (rc) {
                free_pipe(g);
                return rc;
            }
        }
        g->host_cap = chunk;
    }
    if (!g->s_h2d) {
        int rc = dmalloc(&g->d_hhist, 2 * 2 * vg::kOrderBins, g->device_bytes);
        if (!rc) rc = dmalloc(&g->d_hqueue, 2, g->device_bytes);
        if (!rc) rc = dmalloc(&g->d_hset, 2, g->device_bytes);
        if (rc) return rc;
        VG_CUDA(cudaStreamCreateWithFlags(&g->s_h2d, cudaStreamNonBlocking));
        VG_CUDA(cudaStreamCreateWithFlags(&g->s_d2h, cudaStreamNonBlocking));
        VG_CUDA(cudaStreamCreateWithFlags(&g->s_loc, cudaStreamNonBlocking));
        for (int k = 0; k < 2; k++) {
            VG_CUDA(cudaEventCreateWithFlags(&g->ev_in[k], cudaEventDisableTiming));
            VG_CUDA(cudaEventCreateWithFlags(&g->ev_k[k], cudaEventDisableTiming));
            VG_CUDA(cudaEventCreateWithFlags(&g->ev_out[k], cudaEventDisableTiming));
            VG_CUDA(cudaEventCreateWithFlags(&g->ev_prep[k], cudaEventDisableTiming));
        }
    }
    // Results go straight into the caller's memory when the device can
    // write it (pinned host memory is mapped into the device's address
    // space): no copy out, and the next call's traversal need not wait for
    // one. Otherwise they go through the slots and a copy out.
    char *tau_dev = nullptr;
    int32_t *st_dev = nullptr;
    {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, tau) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer)
            tau_dev = static_cast<char *>(at.devicePointer);
        if (tau_dev && ray_status) {
            cudaPointerAttributes as{};
            if (cudaPointerGetAttributes(&as, ray_status) == cudaSuccess && as.type == cudaMemoryTypeHost &&
                as.devicePointer)
                st_dev = static_cast<int32_t *>(as.devicePointer);
            else
                tau_dev = nullptr;
        }
        cudaGetLastError();  // a pointer the runtime does not know is not an error here
    }
    const bool direct = tau_dev != nullptr;
    // slots alternate across chunks and calls; a slot's events order its
    // reuse after the traversal and the copy out that last used it
    const int64_t nchunks = (N + chunk - 1) / chunk;
    int k = g->host_slot;
    for (int64_t c = 0; c < nchunks; c++, k ^= 1) {
        const int64_t first = c * chunk, n = std::min(chunk, N - first);
        double *dO = g->d_hin[k], *dD = g->d_hin[k] + 3 * chunk;
        // rays in once the slot's previous traversal is done
        VG_CUDA(cudaStreamWaitEvent(g->s_h2d, g->ev_k[k], 0));
        VG_CUDA(cudaMemcpyAsync(dO, origin + 3 * first, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, g->s_h2d));
        VG_CUDA(cudaMemcpyAsync(dD, dir + 3 * first, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, g->s_h2d));
        VG_CUDA(cudaEventRecord(g->ev_in[k], g->s_h2d));
        // trace once the rays are in and the slot's previous results are out
        VG_CUDA(cudaStreamWaitEvent(s, g->ev_in[k], 0));
        VG_CUDA(cudaStreamWaitEvent(s, g->ev_out[k], 0));
        void *out_tau = direct ? static_cast<void *>(tau_dev + tau_sz * first) : g->d_hout[k];
        int32_t *out_st = direct ? (st_dev ? st_dev + first : nullptr) : (ray_status ? g->d_hst[k] : nullptr);
        // without counters to read, the chunk's start records are prepared
        // beside the previous chunk's traversal (trace_chunk_slot)
        int rc = stats ? trace_tau_chunk(g, dO, dD, n, precision, out_tau, out_st, c == 0, s)
                       : trace_chunk_slot(g, k, dO, dD, n, precision, out_tau, out_st, s);
        if (rc) return rc;
        VG_CUDA(cudaEventRecord(g->ev_k[k], s));
        if (direct) continue;
        // results out
        VG_CUDA(cudaStreamWaitEvent(g->s_d2h, g->ev_k[k], 0));
        VG_CUDA(cudaMemcpyAsync(static_cast<char *>(tau) + tau_sz * first, g->d_hout[k], tau_sz * n,
                                cudaMemcpyDeviceToHost, g->s_d2h));
        if (ray_status)
            VG_CUDA(cudaMemcpyAsync(ray_status + first, g->d_hst[k], sizeof(int32_t) * n, cudaMemcpyDeviceToHost,
                                    g->s_d2h));
        VG_CUDA(cudaEventRecord(g->ev_out[k], g->s_d2h));
    }
    g->host_slot = k;
    // `stream` continues after the last copy out (direct writes are done
    // when the traversal on `stream` is)
    if (!direct) VG_CUDA(cudaStreamWaitEvent(s, g->ev_out[k ^ 1], 0));
    if (stats) return read_stats(g->d_stats, stats, s);  // synchronises
    return VGRID_OK;
}

int vgrid_segments_grad(vgrid_t *g, const int64_t *seg_off, const int32_t *seg_cell, const float *seg_len, int64_t N,
                        const float *dL_dtau, float kappa, float *dL_drho, vgrid_stream_t stream) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (g->device < 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    if (N < 0 || (N > 0 && (!seg_off || !seg_cell || !seg_len || !dL_dtau || !dL_drho)))
        return fail(VGRID_ERR_ARG, "bad arguments");
    if (!std::isfinite(kappa)) return fail(VGRID_ERR_ARG, "kappa is not finite");
    if (N == 0) return VGRID_OK;
    DeviceGuard dg(g->device);
    VG_CUDA(vg::launch_segments_grad(seg_off, seg_cell, seg_len, N, dL_dtau, kappa, dL_drho, g->sms,
                                     (cudaStream_t)stream));
    return VGRID_OK;
}

int vgrid_trace_grad(vgrid_t *g, const double *origin, const double *dir, int64_t N, const float *dL_dtau,
                     float *dL_drho, vgrid_stream_t stream) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (g->device < 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    if (N < 0 || (N > 0 && (!origin || !dir || !dL_dtau || !dL_drho))) return fail(VGRID_ERR_ARG, "bad arguments");
    if (N == 0) return VGRID_OK;
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_start(g, N);
    if (rc) return rc;
    RaySetDev set{origin, dir, nullptr, nullptr, g->d_start, N, 0, 0, 0};
    VG_CUDA(vg::launch_prepare(g->d_set, set, g->d_queue, g->d_stats, s));
    mark(g, 0, 0, s);
    const int32_t *order = nullptr;
    if ((rc = locate_start(g, kernels(g->launch.lanes_per_ray).fn[0][vg::MODE_GRAD], g->launch, N, &order, s))) return rc;
    mark(g, 0, 1, s);
    vg::TraceArgs a{};
    a.order = order;
    a.grids = g->d_desc;
    a.sets = g->d_set;
    a.nsets = 1;
    a.total = N;
    a.queue = g->d_queue;
    a.stats = g->d_stats;
    a.dL_dtau = dL_dtau;
    a.dL_drho = dL_drho;
    a.g1 = g->hd;
    a.s1 = set;
    mark(g, 1, 0, s);
    rc = launch_trace(kernels(g->launch.lanes_per_ray).fn[0][vg::MODE_GRAD], g->launch, g->sms, N, a, s);
    mark(g, 1, 1, s);
    return rc;
}

int64_t vgrid_kernel_launches(void) { return vg::launches_so_far(); }

int vgrid_enable_timing(vgrid_t *g, int enable) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (g->device < 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    DeviceGuard dg(g->device);
    g->timing = enable != 0;
    g->n_loc = g->n_trace = 0;
    return VGRID_OK;
}

int vgrid_read_timing(vgrid_t *g, double *locate_ms, double *trace_ms, int64_t *launches) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (g->device < 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    DeviceGuard dg(g->device);
    double tl = 0, tt = 0;
    for (int which = 0; which < 2; which++) {
        auto &v = which == 0 ? g->ev_loc : g->ev_trace;
        size_t n = which == 0 ? g->n_loc : g->n_trace;
        for (size_t i = 0; i < n; i++) {
            VG_CUDA(cudaEventSynchronize(v[i][1]));
            float ms = 0;
            VG_CUDA(cudaEventElapsedTime(&ms, v[i][0], v[i][1]));
            (which == 0 ? tl : tt) += ms;
        }
    }
    if (locate_ms) *locate_ms = tl;
    if (trace_ms) *trace_ms = tt;
    if (launches) *launches = (int64_t)g->n_trace;
    g->n_loc = g->n_trace = 0;
    return VGRID_OK;
}

int vgrid_interact(vgrid_t *g, const double *origin, const double *dir, int64_t N, const float *tau_int,
                   const float *weight, int32_t *cell, float *s_out, float *absorbed, vgrid_stream_t stream) {
    if (!g) return fail(VGRID_ERR_ARG, "null grid");
    if (g->device < 0) return fail(VGRID_ERR_ARG, "grid was built with host_only");
    if (N < 0 || (N > 0 && (!origin || !dir || !tau_int || !cell || !s_out))) return fail(VGRID_ERR_ARG, "bad arguments");
    if (N == 0) return VGRID_OK;
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_start(g, N);
    if (rc) return rc;
    RaySetDev set{origin, dir, nullptr, nullptr, g->d_start, N, 0, 0, 0};
    VG_CUDA(vg::launch_prepare(g->d_set, set, g->d_queue, g->d_stats, s));
    mark(g, 0, 0, s);
    const int32_t *order = nullptr;
    if ((rc = locate_start(g, kernels(g->launch.lanes_per_ray).fn[0][vg::MODE_INTERACT], g->launch, N, &order, s))) return rc;
    mark(g, 0, 1, s);
    vg::TraceArgs a{};
    a.order = order;
    a.grids = g->d_desc;
    a.sets = g->d_set;
    a.nsets = 1;
    a.total = N;
    a.queue = g->d_queue;
    a.stats = g->d_stats;
    a.tau_int = tau_int;
    a.weight = weight;
    a.int_cell = cell;
    a.int_s = s_out;
    a.absorbed = absorbed;
    a.g1 = g->hd;
    a.s1 = set;
    mark(g, 1, 0, s);
    rc = launch_trace(kernels(g->launch.lanes_per_ray).fn[0][vg::MODE_INTERACT], g->launch, g->sms, N, a, s);
    mark(g, 1, 1, s);
    return rc;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------

static void free_batch(vgrid_batch_t *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    void *ptrs[] = {b->d_grids, b->d_sets, b->d_start, b->d_queue, b->d_stats, b->d_bin, b->d_hist, b->d_order};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete b;
}

static bool valid_batch_launch(const vgrid_launch *l) {
    return valid_lpr(l->lanes_per_ray) && l->block >= 32 && l->block <= 256 && l->block % 32 == 0 &&
           l->blocks_per_sm >= 0 && l->order >= -1 && l->order <= 1;
}

// the ray order's buffers of a batch (bins, counts, permutation)
static int batch_order_buffers(vgrid_batch_t *b) {
    if (b->d_order || b->total <= 0 || b->total > INT32_MAX) return VGRID_OK;
    int64_t bytes = 0;
    int rc;
    if ((rc = dmalloc(&b->d_bin, (size_t)b->total, bytes)) || (rc = dmalloc(&b->d_order, (size_t)b->total, bytes)) ||
        (rc = dmalloc(&b->d_hist, 2 * vg::kOrderBins, bytes)))
        return rc;
    return VGRID_OK;
}

int vgrid_batch_create(const vgrid_rayset *sets, int32_t G, const vgrid_launch *launch, vgrid_batch_t **out) {
    if (!out) return fail(VGRID_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!sets || G < 1) return fail(VGRID_ERR_ARG, "need at least one ray set");
    if (launch && !valid_batch_launch(launch)) return fail(VGRID_ERR_ARG, "bad launch shape");
    const int dev = sets[0].grid ? sets[0].grid->device : 0;
    std::vector<const vgrid_t *> uniq;
    std::vector<GridDev> descs;
    std::vector<RaySetDev> rs(G);
    int64_t total = 0;
    for (int32_t i = 0; i < G; i++) {
        const vgrid_rayset &q = sets[i];
        if (!q.grid || q.grid->device < 0 || q.n < 0 || (q.n > 0 && (!q.origin || !q.dir || !q.tau)))
            return fail(VGRID_ERR_ARG, "bad ray set " + std::to_string(i));
        if (q.grid->device != dev) return fail(VGRID_ERR_ARG, "all grids of a batch must live on one device");
        int gi = (int)(std::find(uniq.begin(), uniq.end(), q.grid) - uniq.begin());
        if (gi == (int)uniq.size()) {
            uniq.push_back(q.grid);
            descs.push_back(q.grid->hd);
        }
        rs[i] = RaySetDev{q.origin, q.dir, q.tau, q.status, nullptr, q.n, total, gi, 0};
        total += q.n;
    }
    DeviceGuard dg(dev);
    vgrid_batch_t *b = new vgrid_batch();
    b->device = dev;
    b->G = G;
    b->total = total;
    b->ngrids = (int)uniq.size();
    if (launch) b->launch = *launch;
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t bytes = 0;
    int rc;
    if ((rc = dmalloc(&b->d_grids, descs.size(), bytes)) || (rc = dmalloc(&b->d_sets, (size_t)G, bytes)) ||
        (rc = dmalloc(&b->d_start, (size_t)std::max<int64_t>(total, 1), bytes)) ||
        (rc = dmalloc(&b->d_queue, 1, bytes)) || (rc = dmalloc(&b->d_stats, 1, bytes))) {
        free_batch(b);
        return rc;
    }
    // longest-first ray order over all work items of the batch, only on
    // request: it interleaves the grids, whose blocks together may not fit
    // in L2, where the caller's order takes them one after another
    if (b->launch.order == 1 && (rc = batch_order_buffers(b))) {
        free_batch(b);
        return rc;
    }
    for (int32_t i = 0; i < G; i++) rs[i].start = b->d_start + rs[i].first;
    cudaError_t e = cudaMemcpy(b->d_grids, descs.data(), sizeof(GridDev) * descs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_sets, rs.data(), sizeof(RaySetDev) * G, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_batch(b);
        return fail(VGRID_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
    }
    *out = b;
    return VGRID_OK;
}

static int batch_issue(vgrid_batch_t *b, cudaStream_t s) {
    RaySetDev none{};
    VG_CUDA(vg::launch_prepare(nullptr, none, b->d_queue, b->d_stats, s));
    vg::TraceArgs a{};
    if (b->launch.order == 1 && b->d_order) {
        const vg::RayOrder ord{b->d_bin, b->d_hist, b->d_order};
        VG_CUDA(cudaMemsetAsync(b->d_hist, 0, 2 * vg::kOrderBins * sizeof(uint32_t), s));
        VG_CUDA(vg::launch_locate_ordered(b->d_grids, b->d_sets, b->G, b->total, ord, vg::PREP_FP32, b->sms, s));
        VG_CUDA(vg::launch_order(ord, b->total, b->sms, s));
        a.order = b->d_order;
    } else {
        VG_CUDA(vg::launch_locate(b->d_grids, b->d_sets, b->G, b->total, vg::PREP_FP32, nullptr, b->sms, s));
    }
    a.grids = b->d_grids;
    a.sets = b->d_sets;
    a.nsets = b->G;
    a.total = b->total;
    a.queue = b->d_queue;
    a.stats = b->d_stats;
    return launch_trace(kernels(b->launch.lanes_per_ray).batch, b->launch, b->sms, b->total, a, s);
}

int vgrid_batch_run(vgrid_batch_t *b, int use_graph, vgrid_stats *stats, vgrid_stream_t stream) {
    if (!b) return fail(VGRID_ERR_ARG, "null batch");
    DeviceGuard dg(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (use_graph) {
        if (!s) return fail(VGRID_ERR_ARG, "graph replay needs a non-default stream");
        if (!b->exec) {
            VG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            const int64_t before = vg::launches_so_far();
            int rc = batch_issue(b, s);
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            b->graph_kernels = vg::launches_so_far() - before;
            vg::count_launches(-b->graph_kernels);  // captured, not launched
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return fail(VGRID_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            b->graph = graph;
            VG_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
        }
        VG_CUDA(cudaGraphLaunch(b->exec, s));
        vg::count_launches(b->graph_kernels);
    } else {
        int rc = batch_issue(b, s);
        if (rc) return rc;
    }
    if (stats) return read_stats(b->d_stats, stats, s);
    return VGRID_OK;
}

int vgrid_batch_set_launch(vgrid_batch_t *b, const vgrid_launch *launch) {
    if (!b) return fail(VGRID_ERR_ARG, "null batch");
    vgrid_launch l{1, 128, 0, 1, 0};
    if (launch) l = *launch;
    if (!valid_batch_launch(&l)) return fail(VGRID_ERR_ARG, "bad launch shape");
    DeviceGuard dg(b->device);
    if (l.order == 1) {
        int rc = batch_order_buffers(b);
        if (rc) return rc;
    }
    b->launch = l;
    // a captured graph holds the old shape: capture again on the next run
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    return VGRID_OK;
}

int vgrid_batch_get_launch(const vgrid_batch_t *b, vgrid_launch *launch) {
    if (!b || !launch) return fail(VGRID_ERR_ARG, "null argument");
    *launch = b->launch;
    return VGRID_OK;
}

int vgrid_batch_destroy(vgrid_batch_t *b) {
    if (!b) return VGRID_OK;
    DeviceGuard dg(b->device);
    free_batch(b);
    return VGRID_OK;
}

}  // extern "C"

namespace vg {

void set_error(const std::string &msg) { g_err = msg; }

int grid_view(const struct vgrid *g, GridView *out) {
    if (!g || g->device < 0) return -1;
    out->device = g->device;
    out->sms = g->sms;
    out->d_desc = g->d_desc;
    out->hd = g->hd;
    out->lanes_per_ray = g->launch.lanes_per_ray;
    out->fp64_lanes_per_ray = g->launch.fp64_lanes_per_ray ? g->launch.fp64_lanes_per_ray : g->launch.lanes_per_ray;
    out->block = g->launch.block;
    out->blocks_per_sm = g->launch.blocks_per_sm;
    return 0;
}

}  // namespace vg
