// GPU construction of the Voronoi cells: the parallel set-up the paper
// names as future work (Sect. 3.6). Same definition as the host builder: the
// cell of site m is the domain box cut by the bisector half-space of every
// site that can reach it (Sect. 2.1, Eq. 1-3); a site farther than twice the
// largest vertex radius cannot, so the search stops once every unvisited
// site is that far (security radius).
//
// Sites are first sorted into a grid of buckets (counting sort; each
// bucket's list is then ordered by site index so the result does not depend
// on atomic order). The grid lines of each axis sit at quantiles of the
// sites' coordinates on that axis, so that where the sites are dense the
// buckets are small: a density that is a product of functions of x, y and z
// gives every bucket about the same number of sites. One thread builds one cell: a convex polyhedron in
// float64 with shared vertices and faces as vertex loops, cut plane by plane
// while the buckets are visited ring by ring around the site, the sites of
// each ring nearest first. Fixed capacities keep the polyhedron in local
// memory; a cell that would overflow them is flagged and rebuilt by the
// host builder.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.h"

namespace vg {
namespace {

constexpr int kNV = 96;    // vertices of the polyhedron
constexpr int kNF = 48;    // faces
constexpr int kNL = 320;   // entries of all face loops
constexpr int kNE = 64;    // crossed edges of one cut
constexpr int kCap = 64;   // neighbour ids written back per cell

struct BucketGrid {
    const double *edge[3];  // grid lines of each axis: dim + 1 non-decreasing values, box bounds at both ends
    int dim[3];
};

struct DPoly {
    double x[kNV], y[kNV], z[kNV];
    int nv;
    int fid[kNF];
    short fbeg[kNF], flen[kNF];
    int nf;
    unsigned char L[kNL];
    int nl;
};

struct Scratch {
    double fv[kNV];
    int fid[kNF];
    short fbeg[kNF], flen[kNF];
    unsigned char L[kNL];
    unsigned char seg_a[kNF], seg_b[kNF];
    int ekey[kNE];
    unsigned char evid[kNE];
    unsigned char remap[kNV];
    double x[kNV], y[kNV], z[kNV];
};

// the bucket of coordinate v along one axis: the largest i < dim with
// edge[i] <= v (0 below the first line)
__device__ __forceinline__ int bucket_coord(double v, const double *edge, int dim) {
    int lo = 0, hi = dim - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(edge + mid) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void bucket_count_kernel(const double *S, int64_t M, BucketGrid bg, int *bidx, int64_t *cnt) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        const int i = bucket_coord(S[3 * m], bg.edge[0], bg.dim[0]);
        const int j = bucket_coord(S[3 * m + 1], bg.edge[1], bg.dim[1]);
        const int k = bucket_coord(S[3 * m + 2], bg.edge[2], bg.dim[2]);
        const int b = (i * bg.dim[1] + j) * bg.dim[2] + k;
        bidx[m] = b;
        atomicAdd(reinterpret_cast<unsigned long long *>(&cnt[b]), 1ull);
    }
}

__global__ void bucket_fill_kernel(const int *bidx, int64_t M, int64_t *cursor, int *bsites) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long at = atomicAdd(reinterpret_cast<unsigned long long *>(&cursor[bidx[m]]), 1ull);
        bsites[at] = (int)m;
    }
}

// order every bucket's list by site index (insertion sort; lists are short)
__global__ void bucket_sort_kernel(const int64_t *off, int64_t K, int *bsites) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < K; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = off[b], e = off[b + 1];
        for (int64_t i = s + 1; i < e; i++) {
            const int v = bsites[i];
            int64_t k = i - 1;
            while (k >= s && bsites[k] > v) {
                bsites[k + 1] = bsites[k];
                k--;
            }
            bsites[k + 1] = v;
        }
    }
}

__device__ void poly_box(DPoly &P, const double *box) {
    P.nv = 8;
    for (int i = 0; i < 8; i++) {
        P.x[i] = (i & 4) ? box[3] : box[0];
        P.y[i] = (i & 2) ? box[4] : box[1];
        P.z[i] = (i & 1) ? box[5] : box[2];
    }
    // counter-clockwise seen from outside; walls -1..-6 = x min, x max, y min, y max, z min, z max
    const unsigned char quad[6][4] = {{0, 1, 3, 2}, {4, 6, 7, 5}, {0, 4, 5, 1}, {2, 3, 7, 6}, {0, 2, 6, 4}, {1, 5, 7, 3}};
    P.nf = 6;
    P.nl = 24;
    for (int w = 0; w < 6; w++) {
        P.fid[w] = -(w + 1);
        P.fbeg[w] = (short)(4 * w);
        P.flen[w] = 4;
        for (int k = 0; k < 4; k++) P.L[4 * w + k] = quad[w][k];
    }
}

__device__ double poly_rmax2(const DPoly &P, double px, double py, double pz) {
    double r2 = 0.0;
    for (int i = 0; i < P.nv; i++) {
        const double dx = P.x[i] - px, dy = P.y[i] - py, dz = P.z[i] - pz;
        r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
    }
    return r2;
}

// A double truncated to float32 with integer operations only (its high word:
// 21 significant bits, relative error below 2^-20; |x| < 2^-126 gives 0).
__device__ __forceinline__ float trunc_float(double x) {
    const int h = __double2hiint(x);
    const int e = (h >> 20) & 0x7ff;
    const int bits = (h & (int)0x80000000) | ((e - 896) << 23) | ((h & 0xfffff) << 3);
    return e > 896 ? __int_as_float(bits) : 0.0f;
}

// Cut P by {x : n.x <= d}. 1: changed, 0: untouched, -1: capacity exceeded
// or topology broken (the caller rebuilds the cell on the host).
// B bounds the error of the float32 screen below: with |n| = 1, every vertex
// and the midpoint inside the box (|coordinate| <= X), truncation and
// float32 rounding leave n.v - d within about 0.76 2^-17 X of its float32
// value, and B = 2^-16 X; the screen returns 0 only where the float64 test
// below would (no vertex above the plane by more than eps << B).
__device__ int poly_cut(DPoly &P, Scratch &W, double nx, double ny, double nz, double d, int id, double eps,
                        float B) {
    {
        // most planes that pass the security radius still miss the cell:
        // tell them apart without the float64 pipe, which a warp pays for
        // all its lanes whenever one of them uses it
        const float fx = trunc_float(nx), fy = trunc_float(ny), fz = trunc_float(nz), fd = trunc_float(d);
        bool maybe = false;
        for (int i = 0; i < P.nv; i++) {
            const float v = __fmaf_rn(fz, trunc_float(P.z[i]), __fmaf_rn(fy, trunc_float(P.y[i]),
                                                                         __fmul_rn(fx, trunc_float(P.x[i]))));
            maybe |= __fsub_rn(v, fd) > -B;
        }
        if (!maybe) return 0;
    }
    // each vertex classified once: above the plane (fv > eps) and strictly
    // below it (fv < -eps) as bits of two 128-bit masks held in registers,
    // so that the face walk below tests the masks and reads fv only at the
    // two ends of an edge the plane cuts
    static_assert(kNV <= 128, "vertex masks hold 128 bits");
    unsigned long long out0 = 0ull, out1 = 0ull, str0 = 0ull, str1 = 0ull;
    for (int i = 0; i < P.nv; i++) {
        const double f = nx * P.x[i] + ny * P.y[i] + nz * P.z[i] - d;
        W.fv[i] = f;
        const unsigned long long bit = 1ull << (i & 63);
        const unsigned long long ob = f > eps ? bit : 0ull, sb = f < -eps ? bit : 0ull;
        if (i < 64) {
            out0 |= ob;
            str0 |= sb;
        } else {
            out1 |= ob;
            str1 |= sb;
        }
    }
    if (!(out0 | out1)) return 0;
    auto is_out = [&](int v) { return ((v < 64 ? out0 >> v : out1 >> (v - 64)) & 1ull) != 0ull; };
    auto is_strict = [&](int v) { return ((v < 64 ? str0 >> v : str1 >> (v - 64)) & 1ull) != 0ull; };
    int ne = 0, nseg = 0, nf2 = 0, nl2 = 0, nv = P.nv;
    for (int f = 0; f < P.nf; f++) {
        const int b = P.fbeg[f], k = P.flen[f];
        int out_count = 0;
        for (int i = 0; i < k; i++) out_count += is_out(P.L[b + i]);
        if (out_count == k) continue;
        if (nf2 >= kNF) return -1;
        const int start = nl2;
        int entry = -1, exit_ = -1;
        for (int i = 0; i < k; i++) {
            const int va = P.L[b + i], vb = P.L[b + (i + 1) % k];
            const bool ao = is_out(va), bo = is_out(vb);
            if (!ao) {
                if (nl2 >= kNL) return -1;
                W.L[nl2++] = (unsigned char)va;
            }
            if (ao != bo) {
                const bool strict = !ao ? is_strict(va) : is_strict(vb);
                int x = !ao ? va : vb;
                if (strict) {
                    // the vertex on edge (va, vb), made once from the lower index
                    const int lo = min(va, vb), hi = max(va, vb);
                    const int key = lo * 256 + hi;
                    x = -1;
                    for (int e = 0; e < ne; e++)
                        if (W.ekey[e] == key) { x = W.evid[e]; break; }
                    if (x < 0) {
                        if (ne >= kNE || nv >= kNV) return -1;
                        const double t = W.fv[lo] / (W.fv[lo] - W.fv[hi]);
                        P.x[nv] = P.x[lo] + t * (P.x[hi] - P.x[lo]);
                        P.y[nv] = P.y[lo] + t * (P.y[hi] - P.y[lo]);
                        P.z[nv] = P.z[lo] + t * (P.z[hi] - P.z[lo]);
                        W.fv[nv] = 0.0;
                        W.ekey[ne] = key;
                        W.evid[ne] = (unsigned char)nv;
                        ne++;
                        x = nv++;
                    }
                    if (nl2 >= kNL) return -1;
                    W.L[nl2++] = (unsigned char)x;
                }
                if (!ao) exit_ = x;
                else entry = x;
            }
        }
        if (entry >= 0 && exit_ >= 0 && entry != exit_) {
            if (nseg >= kNF) return -1;
            W.seg_a[nseg] = (unsigned char)entry;
            W.seg_b[nseg] = (unsigned char)exit_;
            nseg++;
        }
        if (nl2 - start >= 3) {
            W.fid[nf2] = P.fid[f];
            W.fbeg[nf2] = (short)start;
            W.flen[nf2] = (short)(nl2 - start);
            nf2++;
        } else {
            nl2 = start;
        }
    }
    if (nseg > 0) {
        // cap face: chain the cut segments entry -> exit
        const int start = nl2;
        int cur = W.seg_a[0];
        const int first = cur;
        bool ok = true;
        unsigned long long used = 0ull;
        for (int step = 0; step < nseg; step++) {
            int pick = -1;
            for (int i = 0; i < nseg; i++)
                if (!((used >> i) & 1ull) && W.seg_a[i] == cur) { pick = i; break; }
            if (pick < 0) { ok = false; break; }
            used |= 1ull << pick;
            if (nl2 >= kNL) return -1;
            W.L[nl2++] = W.seg_a[pick];
            cur = W.seg_b[pick];
        }
        if (!ok || cur != first) return -1;  // inconsistent topology: leave it to the host
        if (nl2 - start >= 3) {
            if (nf2 >= kNF) return -1;
            W.fid[nf2] = id;
            W.fbeg[nf2] = (short)start;
            W.flen[nf2] = (short)(nl2 - start);
            nf2++;
        } else {
            nl2 = start;
        }
    }
    // compact the vertices that are still referenced
    for (int i = 0; i < nv; i++) W.remap[i] = 255;
    int nv2 = 0;
    for (int i = 0; i < nl2; i++) {
        const int v = W.L[i];
        if (W.remap[v] == 255) {
            W.remap[v] = (unsigned char)nv2;
            W.x[nv2] = P.x[v];
            W.y[nv2] = P.y[v];
            W.z[nv2] = P.z[v];
            nv2++;
        }
        P.L[i] = W.remap[v];
    }
    for (int i = 0; i < nv2; i++) {
        P.x[i] = W.x[i];
        P.y[i] = W.y[i];
        P.z[i] = W.z[i];
    }
    P.nv = nv2;
    P.nl = nl2;
    P.nf = nf2;
    for (int f = 0; f < nf2; f++) {
        P.fid[f] = W.fid[f];
        P.fbeg[f] = W.fbeg[f];
        P.flen[f] = W.flen[f];
    }
    return nf2 >= 4 ? 1 : -1;
}

// Persistent threads: each takes its next cell from a global counter as soon
// as it has finished one, so a thread whose cell needed few cuts does not
// wait for the slowest cell of its block. Eight blocks of 128 per SM (64
// registers): the kernel waits on its local-memory polyhedra and gains more
// from the extra warps than it loses to the few more spills.
__global__ void __launch_bounds__(128, 8) cells_kernel(const double *S, int64_t M, BucketGrid bg, const int64_t *boff,
                                                    const int *bsites, double box0, double box1, double box2,
                                                    double box3, double box4, double box5, double eps, int *out_cnt,
                                                    int *out_nbr, double *out_vol, double *out_bbox, int *out_fail,
                                                    unsigned long long *next, const float4 *Sf, int prefilter) {
    DPoly P;
    Scratch W;
    const double box[6] = {box0, box1, box2, box3, box4, box5};
    double X = 0.0;
    for (int c = 0; c < 6; c++) X = fmax(X, fabs(box[c]));
    const float Bscreen = __fmaf_rn((float)X, 0x1p-16f, 0x1p-120f);  // see poly_cut
    for (int64_t m = (int64_t)atomicAdd(next, 1ull); m < M; m = (int64_t)atomicAdd(next, 1ull)) {
        const double px = S[3 * m], py = S[3 * m + 1], pz = S[3 * m + 2];
        poly_box(P, box);
        double rmax = sqrt(poly_rmax2(P, px, py, pz));
        // Float32 prefilter of the security radius. A warp issues a float64
        // instruction for all its lanes, so the float64 distance of every
        // candidate site costs the whole warp; most candidates lie far out
        // of reach. Site coordinates are float32 values, so their float
        // copies are exact and the float32 squared distance is within 2^-21
        // (relative) of the exact one; a site is dropped only when it
        // exceeds reach^2 (1 + 2^-17), rounded up, where the float64 test
        // drops it as well. Zero or underflowed distances never pass it.
        const float4 pf = Sf[m];
        auto reach2f = [&](double r) {
            const double reach = 2.0 * r + 4.0 * eps;
            return __double2float_ru(reach * reach * (1.0 + 0x1p-17));
        };
        float R2f = reach2f(rmax);
        const int bi = bucket_coord(px, bg.edge[0], bg.dim[0]);
        const int bj = bucket_coord(py, bg.edge[1], bg.dim[1]);
        const int bk = bucket_coord(pz, bg.edge[2], bg.dim[2]);
        const int bc[3] = {bi, bj, bk};
        const double pc[3] = {px, py, pz};
        const int smax = max(bg.dim[0], max(bg.dim[1], bg.dim[2]));
        int fail = 0;
        // each shell's candidates within reach are cut nearest first (up to
        // kBuf at a time, picked by float32 distance, ties by index): the
        // near planes shrink the polyhedron, and with it the reach, so that
        // more of the far candidates drop out before they are cut. The
        // result is the same polyhedron up to rounding; only the work to
        // reach it changes. A candidate is one 64-bit key, the distance's
        // bits above the site index (non-negative floats order as their
        // bits), and the buffer becomes a binary min-heap when it is
        // drained, so each pick costs a walk down the heap rather than a
        // scan of the whole buffer.
        constexpr int kBuf = 384;
        unsigned long long bkey[kBuf];
        int nb = 0;
        auto sift_down = [&](int i, unsigned long long v) {
            for (;;) {
                int c = 2 * i + 1;
                if (c >= nb) break;
                unsigned long long cv = bkey[c];
                if (c + 1 < nb) {
                    const unsigned long long c2 = bkey[c + 1];
                    if (c2 < cv) { cv = c2; c++; }
                }
                if (v <= cv) break;
                bkey[i] = cv;
                i = c;
            }
            bkey[i] = v;
        };
        auto flush = [&]() -> int {
            for (int i = nb / 2 - 1; i >= 0; i--) sift_down(i, bkey[i]);
            while (nb > 0) {
                const unsigned long long top = bkey[0];
                nb--;
                if (nb > 0) sift_down(0, bkey[nb]);
                const float d2k = __uint_as_float((unsigned)(top >> 32));
                const int jj = (int)(unsigned)top;
                if (prefilter && d2k > R2f) {
                    nb = 0;  // the nearest left is out of reach: so are the others
                    break;
                }
                const double qx = S[3 * (int64_t)jj], qy = S[3 * (int64_t)jj + 1], qz = S[3 * (int64_t)jj + 2];
                const double dx = qx - px, dy = qy - py, dz = qz - pz;
                const double dist = sqrt(dx * dx + dy * dy + dz * dz);
                if (dist > 2.0 * rmax + 4.0 * eps) continue;
                const double nx = dx / dist, ny = dy / dist, nz = dz / dist;
                const double d = nx * 0.5 * (qx + px) + ny * 0.5 * (qy + py) + nz * 0.5 * (qz + pz);
                const int rc = poly_cut(P, W, nx, ny, nz, d, jj, eps, Bscreen);
                if (rc < 0) return 1;
                if (rc > 0) {
                    rmax = sqrt(poly_rmax2(P, px, py, pz));
                    R2f = reach2f(rmax);
                }
            }
            return 0;
        };
        for (int s = 0; s <= smax && !fail; s++) {
            for (int di = -s; di <= s && !fail; di++) {
                const int i = bi + di;
                if (i < 0 || i >= bg.dim[0]) continue;
                for (int dj = -s; dj <= s && !fail; dj++) {
                    const int j = bj + dj;
                    if (j < 0 || j >= bg.dim[1]) continue;
                    const bool shell = abs(di) == s || abs(dj) == s;
                    for (int dk = -s; dk <= s && !fail; dk += (shell || s == 0) ? 1 : 2 * s) {
                        const int k = bk + dk;
                        if (k < 0 || k >= bg.dim[2]) continue;
                        const int b = (i * bg.dim[1] + j) * bg.dim[2] + k;
                        for (int64_t q = boff[b]; q < boff[b + 1]; q++) {
                            const int jj = bsites[q];
                            if (jj == (int)m) continue;
                            const float4 qf = Sf[jj];
                            const float fx = __fsub_rn(qf.x, pf.x), fy = __fsub_rn(qf.y, pf.y),
                                        fz = __fsub_rn(qf.z, pf.z);
                            const float d2f = __fmaf_rn(fz, fz, __fmaf_rn(fy, fy, __fmul_rn(fx, fx)));
                            if (prefilter && d2f > R2f) continue;
                            if (nb == kBuf) fail = flush();
                            if (fail) break;
                            bkey[nb++] = ((unsigned long long)__float_as_uint(d2f) << 32) | (unsigned)jj;
                        }
                    }
                }
            }
            if (!fail) fail = flush();
            // every unvisited site lies beyond one of the grid lines that
            // bound rings 0..s (a site in bucket i has edge[i] <= v <
            // edge[i + 1]), so it is at least the smallest gap from the
            // site to those lines away; there are no sites past the last
            // bucket on either side
            double gap = 1e300;
            for (int c = 0; c < 3; c++) {
                if (bc[c] + s + 1 <= bg.dim[c] - 1) gap = fmin(gap, __ldg(bg.edge[c] + bc[c] + s + 1) - pc[c]);
                if (bc[c] - s >= 1) gap = fmin(gap, pc[c] - __ldg(bg.edge[c] + bc[c] - s));
            }
            if (2.0 * rmax + 4.0 * eps < gap) break;
        }
        // faces of positive area -> neighbours; volume as pyramids from the site; bounding box
        static_assert(kNE >= kCap, "the edge keys hold the neighbour list");
        int *const ids = W.ekey;  // free once the cuts are done
        int cnt = 0;
        double vol = 0.0;
        double bb[6] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300};
        for (int f = 0; f < P.nf && !fail; f++) {
            const int b = P.fbeg[f], k = P.flen[f];
            const int v0 = P.L[b];
            double sx = 0, sy = 0, sz = 0, sv = 0;
            for (int t = 1; t + 1 < k; t++) {
                const int v1 = P.L[b + t], v2 = P.L[b + t + 1];
                const double ax = P.x[v1] - P.x[v0], ay = P.y[v1] - P.y[v0], az = P.z[v1] - P.z[v0];
                const double cx = P.x[v2] - P.x[v0], cy = P.y[v2] - P.y[v0], cz = P.z[v2] - P.z[v0];
                const double ux = ay * cz - az * cy, uy = az * cx - ax * cz, uz = ax * cy - ay * cx;
                sx += ux;
                sy += uy;
                sz += uz;
                // signed volume of the tetrahedron (site, v0, v1, v2)
                sv += ((P.x[v0] - px) * ux + (P.y[v0] - py) * uy + (P.z[v0] - pz) * uz) / 6.0;
            }
            vol += fabs(sv);
            const double area2 = sx * sx + sy * sy + sz * sz;
            if (area2 > 0.0) {
                if (cnt >= kCap) { fail = 1; break; }
                ids[cnt++] = P.fid[f];
            }
        }
        for (int i = 0; i < P.nv; i++) {
            bb[0] = fmin(bb[0], P.x[i]);
            bb[1] = fmin(bb[1], P.y[i]);
            bb[2] = fmin(bb[2], P.z[i]);
            bb[3] = fmax(bb[3], P.x[i]);
            bb[4] = fmax(bb[4], P.y[i]);
            bb[5] = fmax(bb[5], P.z[i]);
        }
        // the list in ascending order without repeats (insertion sort: a few
        // dozen ids), as the host's CSR holds it
        for (int a = 1; a < cnt; a++) {
            const int v = ids[a];
            int b = a - 1;
            while (b >= 0 && ids[b] > v) {
                ids[b + 1] = ids[b];
                b--;
            }
            ids[b + 1] = v;
        }
        int u = 0;
        for (int a = 0; a < cnt; a++)
            if (u == 0 || ids[a] != ids[u - 1]) ids[u++] = ids[a];
        for (int a = 0; a < u; a++) out_nbr[m * kCap + a] = ids[a];
        out_cnt[m] = u;
        out_vol[m] = vol;
        for (int c = 0; c < 6; c++) out_bbox[6 * m + c] = bb[c];
        out_fail[m] = fail;
    }
}

// the cells' lists into one CSR array (offsets computed on the host)
__global__ void gather_lists_kernel(const int *nbr, const int *cnt, const int64_t *off, int64_t M, int *idx) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = off[m];
        const int c = cnt[m];
        for (int a = 0; a < c; a++) idx[o + a] = nbr[m * kCap + a];
    }
}

}  // namespace

int build_cells_gpu(const double *S, int64_t M, const double *box, int threads, CellsOut &out, std::string &err,
                    int64_t *host_fallback_cells) {
    const double ext[3] = {box[3] - box[0], box[4] - box[1], box[5] - box[2]};
    const double diag = std::sqrt(ext[0] * ext[0] + ext[1] * ext[1] + ext[2] * ext[2]);
    const double eps = 1e-12 * diag;
    BucketGrid bg;
    const double target = std::max(1.0, 0.5 * (double)M);  // about two sites per bucket
    const double w = std::cbrt(ext[0] * ext[1] * ext[2] / target);
    int64_t K = 1;
    // grid lines at quantiles of each coordinate, from every stride-th site
    // (at most 2^16 of them; deterministic)
    std::vector<double> edges;
    {
        const int64_t stride = std::max<int64_t>(1, M >> 16);
        std::vector<double> v;
        for (int c = 0; c < 3; c++) {
            bg.dim[c] = (int)std::min<long>(std::max<long>(std::lround(ext[c] / w), 1), 512);
            K *= bg.dim[c];
            v.clear();
            for (int64_t m = 0; m < M; m += stride) v.push_back(S[3 * m + c]);
            std::sort(v.begin(), v.end());
            const int64_t n = (int64_t)v.size();
            edges.push_back(box[c]);
            for (int i = 1; i < bg.dim[c]; i++)
                edges.push_back(std::max(edges.back(), std::min(box[3 + c], v[(size_t)(i * n / bg.dim[c])])));
            edges.push_back(box[3 + c]);
        }
    }
    double *dS = nullptr, *dE = nullptr;
    float4 *dSf = nullptr;
    int prefilter = 1;
    int *bidx = nullptr, *bsites = nullptr, *cnt = nullptr, *nbr = nullptr, *fail = nullptr;
    int64_t *boff = nullptr, *cursor = nullptr, *tmp = nullptr, *doff = nullptr;
    int *didx = nullptr;
    double *vol = nullptr, *bbox = nullptr;
    auto cleanup = [&]() {
        void *ptrs[] = {dS, dE, dSf, bidx, bsites, cnt, nbr, fail, boff, cursor, tmp, vol, bbox, doff, didx};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    };
    auto bad = [&](cudaError_t e, const char *what) {
        err = std::string("GPU cell construction: ") + what + ": " + cudaGetErrorString(e);
        cleanup();
        return -1;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&dS, sizeof(double) * 3 * M)) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&bidx, sizeof(int) * M)) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&bsites, sizeof(int) * M)) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&boff, sizeof(int64_t) * (K + 1))) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&cursor, sizeof(int64_t) * (K + 1))) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&tmp, sizeof(int64_t) * scan_tmp_elems(K))) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&cnt, sizeof(int) * M)) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&nbr, sizeof(int) * kCap * M)) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&fail, sizeof(int) * M)) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&vol, sizeof(double) * M)) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMalloc(&bbox, sizeof(double) * 6 * M)) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMemcpy(dS, S, sizeof(double) * 3 * M, cudaMemcpyHostToDevice)) != cudaSuccess) return bad(e, "upload");
    if ((e = cudaMalloc(&dE, sizeof(double) * edges.size())) != cudaSuccess) return bad(e, "alloc");
    if ((e = cudaMemcpy(dE, edges.data(), sizeof(double) * edges.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bad(e, "upload");
    bg.edge[0] = dE;
    bg.edge[1] = dE + bg.dim[0] + 1;
    bg.edge[2] = bg.edge[1] + bg.dim[1] + 1;
    {
        // float copies of the sites; the prefilter's bound needs them exact
        // (sites are float32 values; it is off otherwise)
        std::vector<float4> sf((size_t)M);
        for (int64_t m = 0; m < M; m++) {
            sf[m] = make_float4((float)S[3 * m], (float)S[3 * m + 1], (float)S[3 * m + 2], 0.f);
            if ((double)sf[m].x != S[3 * m] || (double)sf[m].y != S[3 * m + 1] || (double)sf[m].z != S[3 * m + 2])
                prefilter = 0;
        }
        if ((e = cudaMalloc(&dSf, sizeof(float4) * M)) != cudaSuccess) return bad(e, "alloc");
        if ((e = cudaMemcpy(dSf, sf.data(), sizeof(float4) * M, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bad(e, "upload");
    }
    if ((e = cudaMemset(boff, 0, sizeof(int64_t) * (K + 1))) != cudaSuccess) return bad(e, "memset");
    const int blocks = (int)std::min<int64_t>((M + 255) / 256, 65535);
    bucket_count_kernel<<<blocks, 256>>>(dS, M, bg, bidx, boff);
    if ((e = launch_exclusive_scan(boff, K, tmp, 0)) != cudaSuccess) return bad(e, "scan");
    if ((e = cudaMemcpy(cursor, boff, sizeof(int64_t) * (K + 1), cudaMemcpyDeviceToDevice)) != cudaSuccess)
        return bad(e, "copy");
    bucket_fill_kernel<<<blocks, 256>>>(bidx, M, cursor, bsites);
    bucket_sort_kernel<<<(int)std::min<int64_t>((K + 255) / 256, 65535), 256>>>(boff, K, bsites);
    int dev = 0, sms = 1, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cells_kernel, 128, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int cblocks = (int)std::max<int64_t>(1, std::min<int64_t>((M + 127) / 128, (int64_t)per_sm * sms));
    if ((e = cudaMemset(cursor, 0, sizeof(unsigned long long))) != cudaSuccess) return bad(e, "memset");
    cells_kernel<<<cblocks, 128>>>(dS, M, bg, boff, bsites, box[0], box[1], box[2], box[3], box[4], box[5], eps, cnt,
                                   nbr, vol, bbox, fail, reinterpret_cast<unsigned long long *>(cursor), dSf, prefilter);
    count_launches(4);  // bucket count, fill, sort, cells (the scan counts its own)
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bad(e, "cells kernel");
    std::vector<int> hcnt(M), hfail(M);
    out.vol.assign(M, 0.0);
    out.bbox.assign(6 * M, 0.0);
    if ((e = cudaMemcpy(hcnt.data(), cnt, sizeof(int) * M, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(hfail.data(), fail, sizeof(int) * M, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(out.vol.data(), vol, sizeof(double) * M, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(out.bbox.data(), bbox, sizeof(double) * 6 * M, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return bad(e, "download");
    if (std::find(hfail.begin(), hfail.end(), 1) == hfail.end()) {
        // every cell was built here: its list is sorted already, so only the
        // CSR is gathered on the device and read back
        out.off.assign(M + 1, 0);
        for (int64_t m = 0; m < M; m++) out.off[m + 1] = out.off[m] + hcnt[m];
        out.idx.resize(out.off[M]);
        if (host_fallback_cells) *host_fallback_cells = 0;
        if ((e = cudaMalloc(&doff, sizeof(int64_t) * (M + 1))) != cudaSuccess) return bad(e, "alloc");
        if ((e = cudaMalloc(&didx, sizeof(int) * std::max<int64_t>(1, out.off[M]))) != cudaSuccess)
            return bad(e, "alloc");
        if ((e = cudaMemcpy(doff, out.off.data(), sizeof(int64_t) * (M + 1), cudaMemcpyHostToDevice)) != cudaSuccess)
            return bad(e, "upload");
        gather_lists_kernel<<<blocks, 256>>>(nbr, cnt, doff, M, didx);
        count_launches(1);
        if ((e = cudaMemcpy(out.idx.data(), didx, sizeof(int) * out.off[M], cudaMemcpyDeviceToHost)) != cudaSuccess)
            return bad(e, "download");
        cleanup();
        return 0;
    }
    std::vector<int> hnbr((size_t)kCap * M);
    if ((e = cudaMemcpy(hnbr.data(), nbr, sizeof(int) * kCap * M, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return bad(e, "download");
    cleanup();
    // each cell's list sorted and made unique in place (parallel over
    // cells), the failed cells rebuilt on the host, then one CSR
    std::vector<int64_t> len(M, 0);
    parallel_for(M, threads, 1 << 12, [&](int64_t b, int64_t e) {
        for (int64_t m = b; m < e; m++) {
            if (hfail[m]) continue;
            int *row = hnbr.data() + m * kCap;
            std::sort(row, row + hcnt[m]);
            len[m] = std::unique(row, row + hcnt[m]) - row;
        }
    });
    std::vector<int32_t> redo;
    for (int64_t m = 0; m < M; m++)
        if (hfail[m]) redo.push_back((int32_t)m);
    if (host_fallback_cells) *host_fallback_cells = (int64_t)redo.size();
    std::vector<std::vector<int32_t>> lists(redo.empty() ? 0 : M);
    if (!redo.empty()) {
        if (build_cells_into(S, M, box, threads, &redo, lists, out.vol.data(), out.bbox.data(), err) != 0) return -1;
        for (int32_t m : redo) len[m] = (int64_t)lists[m].size();
    }
    out.off.assign(M + 1, 0);
    for (int64_t m = 0; m < M; m++) out.off[m + 1] = out.off[m] + len[m];
    out.idx.resize(out.off[M]);
    parallel_for(M, threads, 1 << 12, [&](int64_t b, int64_t e) {
        for (int64_t m = b; m < e; m++) {
            if (hfail[m]) std::copy(lists[m].begin(), lists[m].end(), out.idx.begin() + out.off[m]);
            else std::copy(hnbr.begin() + m * kCap, hnbr.begin() + m * kCap + len[m], out.idx.begin() + out.off[m]);
        }
    });
    return 0;
}

}  // namespace vg
