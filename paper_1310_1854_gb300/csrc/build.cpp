// Host-side grid construction for vgrid_create.
//
// For every site the Voronoi cell (Sect. 2.1: the points at least as close
// to this site as to any other) is cut out of the domain box by the bisector
// half-spaces of nearby sites (Eq. 1-3 give the plane: normal p_j - p_m
// through the midpoint). Sites are visited in increasing distance from a
// k-d tree ball query; once a site is farther than twice the largest vertex
// radius of the current polyhedron its plane cannot touch the cell, so the
// search stops there. What remains per cell is what the traversal needs
// (Sect. 2.2 item 3): the ids of the sites and walls owning a face, plus the
// volume and bounding box (Sect. 2.3); the polyhedron itself is dropped.
//
// The polyhedron keeps shared vertices and faces as ordered vertex-index
// loops, counter-clockwise seen from outside. A cut classifies every vertex
// once, creates one new vertex per crossed edge, and closes the hole with a
// cap face obtained by chaining the cut segments of the clipped faces.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace vg {

namespace {

// ---------------------------------------------------------------------------
// k-d tree over the sites for ball queries
// ---------------------------------------------------------------------------

struct KdNode {
    double lo[3], hi[3];
    int32_t begin, end;   // range in order[]
    int32_t child;        // index of left child (right = child + 1), -1 for leaves
};

struct KdTree {
    const double *S = nullptr;
    std::vector<int32_t> order;
    std::vector<KdNode> nodes;
    static constexpr int kLeaf = 12;

    void build(const double *sites, int64_t M) {
        S = sites;
        order.resize(M);
        for (int64_t i = 0; i < M; i++) order[i] = (int32_t)i;
        nodes.clear();
        nodes.reserve(4 * (M / kLeaf + 1));
        nodes.push_back(KdNode{});
        split(0, 0, (int32_t)M);
    }

    void split(int32_t ni, int32_t b, int32_t e) {
        KdNode nd;
        for (int c = 0; c < 3; c++) { nd.lo[c] = INFINITY; nd.hi[c] = -INFINITY; }
        for (int32_t i = b; i < e; i++)
            for (int c = 0; c < 3; c++) {
                double v = S[3 * (int64_t)order[i] + c];
                nd.lo[c] = std::min(nd.lo[c], v);
                nd.hi[c] = std::max(nd.hi[c], v);
            }
        nd.begin = b;
        nd.end = e;
        nd.child = -1;
        if (e - b > kLeaf) {
            int ax = 0;
            for (int c = 1; c < 3; c++)
                if (nd.hi[c] - nd.lo[c] > nd.hi[ax] - nd.lo[ax]) ax = c;
            int32_t mid = b + (e - b) / 2;
            std::nth_element(order.begin() + b, order.begin() + mid, order.begin() + e,
                             [&](int32_t x, int32_t y) { return S[3 * (int64_t)x + ax] < S[3 * (int64_t)y + ax]; });
            int32_t l = (int32_t)nodes.size();
            nd.child = l;
            nodes.push_back(KdNode{});
            nodes.push_back(KdNode{});
            nodes[ni] = nd;
            split(l, b, mid);
            split(l + 1, mid, e);
            return;
        }
        nodes[ni] = nd;
    }

    // Typical spacing near q: side of the cube holding one site in q's leaf.
    double local_spacing(const double *q) const {
        int32_t ni = 0;
        while (nodes[ni].child >= 0) {
            const KdNode &a = nodes[nodes[ni].child], &b = nodes[nodes[ni].child + 1];
            double da = box_d2(a, q), db = box_d2(b, q);
            ni = da <= db ? nodes[ni].child : nodes[ni].child + 1;
        }
        const KdNode &l = nodes[ni];
        double v = 1.0;
        int dims = 0;
        for (int c = 0; c < 3; c++) {
            double ext = l.hi[c] - l.lo[c];
            if (ext > 0) { v *= ext; dims++; }
        }
        int n = l.end - l.begin;
        if (dims == 0 || n <= 1) return 0.0;
        return std::pow(v / n, 1.0 / dims);
    }

    static double box_d2(const KdNode &n, const double *q) {
        double d2 = 0;
        for (int c = 0; c < 3; c++) {
            double d = q[c] < n.lo[c] ? n.lo[c] - q[c] : (q[c] > n.hi[c] ? q[c] - n.hi[c] : 0.0);
            d2 += d * d;
        }
        return d2;
    }

    // Sites j != self with r_in^2 < |p_j - q|^2 <= r_out^2, appended as (d2, j).
    void shell(const double *q, int32_t self, double r_in2, double r_out2,
               std::vector<std::pair<double, int32_t>> &out, std::vector<int32_t> &stack) const {
        stack.clear();
        stack.push_back(0);
        while (!stack.empty()) {
            int32_t ni = stack.back();
            stack.pop_back();
            const KdNode &n = nodes[ni];
            if (box_d2(n, q) > r_out2) continue;
            if (n.child >= 0) {
                stack.push_back(n.child);
                stack.push_back(n.child + 1);
                continue;
            }
            for (int32_t i = n.begin; i < n.end; i++) {
                int32_t j = order[i];
                if (j == self) continue;
                const double *p = S + 3 * (int64_t)j;
                double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
                double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 > r_in2 && d2 <= r_out2) out.emplace_back(d2, j);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// convex polyhedron with shared vertices
// ---------------------------------------------------------------------------

struct Plane {
    double n[3];
    double d;   // cell side: n.x <= d
    int32_t id; // site index or wall -1..-6
};

class Poly {
public:
    std::vector<double> V;          // 3 per vertex
    std::vector<Plane> F;           // one plane per face
    std::vector<int32_t> fbeg, flen; // face loops in L
    std::vector<int32_t> L;

    void make_box(const double *box) {
        V.resize(24);
        for (int i = 0; i < 8; i++) {
            V[3 * i + 0] = (i & 4) ? box[3] : box[0];
            V[3 * i + 1] = (i & 2) ? box[4] : box[1];
            V[3 * i + 2] = (i & 1) ? box[5] : box[2];
        }
        // counter-clockwise seen from outside
        static const int quad[6][4] = {{0, 1, 3, 2}, {4, 6, 7, 5}, {0, 4, 5, 1},
                                       {2, 3, 7, 6}, {0, 2, 6, 4}, {1, 5, 7, 3}};
        F.clear();
        fbeg.clear();
        flen.clear();
        L.clear();
        for (int w = 0; w < 6; w++) {
            Plane p{};
            int ax = w / 2, hi = w % 2;
            p.n[ax] = hi ? 1.0 : -1.0;
            p.d = hi ? box[3 + ax] : -box[ax];
            p.id = -(w + 1);
            F.push_back(p);
            fbeg.push_back((int32_t)L.size());
            flen.push_back(4);
            for (int k = 0; k < 4; k++) L.push_back(quad[w][k]);
        }
    }

    int nverts() const { return (int)(V.size() / 3); }

    double rmax(const double *c) const {
        double r2 = 0;
        for (size_t i = 0; i < V.size(); i += 3) {
            double dx = V[i] - c[0], dy = V[i + 1] - c[1], dz = V[i + 2] - c[2];
            r2 = std::max(r2, dx * dx + dy * dy + dz * dz);
        }
        return std::sqrt(r2);
    }

    // Cut by plane P. Returns 1 if the polyhedron changed, 0 if not, -1 if the
    // topology could not be repaired (the caller reports a build failure).
    int cut(const Plane &P, double eps) {
        const int nv = nverts();
        fv_.resize(nv);
        bool any_out = false;
        for (int i = 0; i < nv; i++) {
            const double *x = &V[3 * i];
            fv_[i] = P.n[0] * x[0] + P.n[1] * x[1] + P.n[2] * x[2] - P.d;
            any_out |= fv_[i] > eps;
        }
        if (!any_out) return 0;

        edge_keys_.clear();
        edge_vid_.clear();
        segs_.clear();
        nL_.clear();
        nbeg_.clear();
        nlen_.clear();
        nF_.clear();
        const int nf = (int)F.size();
        for (int f = 0; f < nf; f++) {
            const int32_t *loop = &L[fbeg[f]];
            const int k = flen[f];
            int out_count = 0;
            for (int i = 0; i < k; i++) out_count += fv_[loop[i]] > eps;
            if (out_count == 0) {
                emit_face(F[f], loop, k);
                continue;
            }
            if (out_count == k) continue;
            tmp_.clear();
            int32_t seg_entry = -1, seg_exit = -1;
            for (int i = 0; i < k; i++) {
                int32_t a = loop[i], b = loop[(i + 1) % k];
                bool ao = fv_[a] > eps, bo = fv_[b] > eps;
                if (!ao) tmp_.push_back(a);
                if (ao != bo) {
                    int32_t x;
                    if (!ao) {  // leaving the kept side after a
                        x = fv_[a] < -eps ? edge_vertex(a, b) : a;
                        if (x != a) tmp_.push_back(x);
                        seg_exit = x;
                    } else {    // re-entering before b
                        x = fv_[b] < -eps ? edge_vertex(a, b) : b;
                        if (x != b) tmp_.push_back(x);
                        seg_entry = x;
                    }
                }
            }
            if (seg_entry >= 0 && seg_exit >= 0 && seg_entry != seg_exit) segs_.push_back({seg_entry, seg_exit});
            if (tmp_.size() >= 3) emit_face(F[f], tmp_.data(), (int)tmp_.size());
        }
        // the cap: chain segments entry -> exit of the clipped faces
        if (!segs_.empty()) {
            cap_.clear();
            bool ok = chain_cap();
            if (!ok) sort_cap(P);
            if (cap_.size() >= 3) emit_face(P, cap_.data(), (int)cap_.size());
        }
        F.swap(nF_);
        L.swap(nL_);
        fbeg.swap(nbeg_);
        flen.swap(nlen_);
        compact();
        return F.size() >= 4 ? 1 : -1;
    }

    double face_area(int f) const {
        const int32_t *loop = &L[fbeg[f]];
        int k = flen[f];
        const double *a = &V[3 * loop[0]];
        double s[3] = {0, 0, 0};
        for (int i = 1; i + 1 < k; i++) {
            const double *b = &V[3 * loop[i]], *c = &V[3 * loop[i + 1]];
            double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
            double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
            s[0] += u[1] * w[2] - u[2] * w[1];
            s[1] += u[2] * w[0] - u[0] * w[2];
            s[2] += u[0] * w[1] - u[1] * w[0];
        }
        return 0.5 * std::fabs(s[0] * F[f].n[0] + s[1] * F[f].n[1] + s[2] * F[f].n[2]);
    }

private:
    std::vector<double> fv_;
    std::vector<uint64_t> edge_keys_;
    std::vector<int32_t> edge_vid_;
    std::vector<std::array<int32_t, 2>> segs_;
    std::vector<int32_t> tmp_, cap_, nL_, nbeg_, nlen_, remap_;
    std::vector<Plane> nF_;
    std::vector<double> nV_;

    void emit_face(const Plane &p, const int32_t *loop, int k) {
        nF_.push_back(p);
        nbeg_.push_back((int32_t)nL_.size());
        nlen_.push_back(k);
        nL_.insert(nL_.end(), loop, loop + k);
    }

    // Vertex where the plane crosses edge (a, b); computed once per edge from
    // the endpoint with the smaller index so both faces share it exactly.
    int32_t edge_vertex(int32_t a, int32_t b) {
        int32_t lo = std::min(a, b), hi = std::max(a, b);
        uint64_t key = ((uint64_t)(uint32_t)lo << 32) | (uint32_t)hi;
        for (size_t i = 0; i < edge_keys_.size(); i++)
            if (edge_keys_[i] == key) return edge_vid_[i];
        double t = fv_[lo] / (fv_[lo] - fv_[hi]);
        int32_t id = nverts();
        for (int c = 0; c < 3; c++) V.push_back(V[3 * lo + c] + t * (V[3 * hi + c] - V[3 * lo + c]));
        fv_.push_back(0.0);
        edge_keys_.push_back(key);
        edge_vid_.push_back(id);
        return id;
    }

    bool chain_cap() {
        // each clipped face left the segment entry -> exit on the cut plane;
        // seen from outside the cap runs through them end to start
        const size_t n = segs_.size();
        std::vector<char> used(n, 0);
        int32_t start = segs_[0][0];
        int32_t cur = start;
        for (size_t step = 0; step < n; step++) {
            size_t pick = n;
            for (size_t i = 0; i < n; i++)
                if (!used[i] && segs_[i][0] == cur) { pick = i; break; }
            if (pick == n) return false;
            used[pick] = 1;
            cap_.push_back(segs_[pick][0]);
            cur = segs_[pick][1];
        }
        return cur == start;
    }

    void sort_cap(const Plane &P) {
        // fallback: the distinct cut vertices ordered by angle about their mean
        cap_.clear();
        for (auto &s : segs_)
            for (int e = 0; e < 2; e++)
                if (std::find(cap_.begin(), cap_.end(), s[e]) == cap_.end()) cap_.push_back(s[e]);
        if (cap_.size() < 3) return;
        double c[3] = {0, 0, 0};
        for (int32_t v : cap_)
            for (int k = 0; k < 3; k++) c[k] += V[3 * v + k] / cap_.size();
        double u[3], w[3];
        int ax = std::fabs(P.n[0]) < 0.6 ? 0 : (std::fabs(P.n[1]) < 0.6 ? 1 : 2);
        double e[3] = {0, 0, 0};
        e[ax] = 1;
        u[0] = P.n[1] * e[2] - P.n[2] * e[1];
        u[1] = P.n[2] * e[0] - P.n[0] * e[2];
        u[2] = P.n[0] * e[1] - P.n[1] * e[0];
        w[0] = P.n[1] * u[2] - P.n[2] * u[1];
        w[1] = P.n[2] * u[0] - P.n[0] * u[2];
        w[2] = P.n[0] * u[1] - P.n[1] * u[0];
        std::vector<std::pair<double, int32_t>> a;
        for (int32_t v : cap_) {
            double q[3] = {V[3 * v] - c[0], V[3 * v + 1] - c[1], V[3 * v + 2] - c[2]};
            // counter-clockwise about +n: angle measured from u towards w = n x u
            a.emplace_back(std::atan2(q[0] * w[0] + q[1] * w[1] + q[2] * w[2], q[0] * u[0] + q[1] * u[1] + q[2] * u[2]), v);
        }
        std::sort(a.begin(), a.end());
        cap_.clear();
        for (auto &x : a) cap_.push_back(x.second);
    }

    void compact() {
        const int nv = nverts();
        remap_.assign(nv, -1);
        nV_.clear();
        for (int32_t &v : L) {
            if (remap_[v] < 0) {
                remap_[v] = (int32_t)(nV_.size() / 3);
                nV_.insert(nV_.end(), &V[3 * v], &V[3 * v] + 3);
            }
            v = remap_[v];
        }
        V.swap(nV_);
    }
};

struct CellResult {
    std::vector<int32_t> nbr;
    double vol = 0;
    double bb[6];
    int err = 0;
};

}  // namespace

// ---------------------------------------------------------------------------
// driver
// ---------------------------------------------------------------------------

// Cells of the listed sites (all sites if ids == nullptr): neighbour lists
// into nbr[m], volumes into vol[m], bounding boxes into bbox[6m].
int build_cells_into(const double *S, int64_t M, const double *box, int threads, const std::vector<int32_t> *ids,
                     std::vector<std::vector<int32_t>> &nbr, double *volume, double *bbox_out, std::string &err) {
    KdTree tree;
    tree.build(S, M);
    const double diag = std::sqrt((box[3] - box[0]) * (box[3] - box[0]) + (box[4] - box[1]) * (box[4] - box[1]) +
                                  (box[5] - box[2]) * (box[5] - box[2]));
    const double eps = 1e-12 * diag;
    const double vbox = (box[3] - box[0]) * (box[4] - box[1]) * (box[5] - box[2]);
    const int64_t count = ids ? (int64_t)ids->size() : M;
    std::atomic<int64_t> next{0};
    std::atomic<int64_t> failed{-1};

    auto work = [&]() {
        Poly P;
        std::vector<std::pair<double, int32_t>> cand;
        std::vector<int32_t> stack;
        for (;;) {
            int64_t m0 = next.fetch_add(64);
            if (m0 >= count || failed.load() >= 0) break;
            int64_t m1 = std::min<int64_t>(count, m0 + 64);
            for (int64_t mi = m0; mi < m1; mi++) {
                const int64_t m = ids ? (*ids)[mi] : mi;
                const double *pm = S + 3 * m;
                P.make_box(box);
                double rmax = P.rmax(pm);
                double h = tree.local_spacing(pm);
                if (!(h > 0)) h = std::cbrt(vbox / (double)M);
                double r_in = -1.0, r_out = 2.5 * h;
                bool done = (M == 1);
                while (!done) {
                    cand.clear();
                    tree.shell(pm, (int32_t)m, r_in < 0 ? -1.0 : r_in * r_in, r_out * r_out, cand, stack);
                    std::sort(cand.begin(), cand.end());
                    bool stopped = false;
                    for (auto &c : cand) {
                        double dist = std::sqrt(c.first);
                        if (dist > 2.0 * rmax + 4.0 * eps) { stopped = true; break; }
                        const double *pj = S + 3 * (int64_t)c.second;
                        Plane pl;
                        double nrm[3] = {pj[0] - pm[0], pj[1] - pm[1], pj[2] - pm[2]};
                        for (int k = 0; k < 3; k++) pl.n[k] = nrm[k] / dist;
                        pl.d = pl.n[0] * 0.5 * (pj[0] + pm[0]) + pl.n[1] * 0.5 * (pj[1] + pm[1]) +
                               pl.n[2] * 0.5 * (pj[2] + pm[2]);
                        pl.id = c.second;
                        int rc = P.cut(pl, eps);
                        if (rc < 0) {
                            failed.store(m);
                            return;
                        }
                        if (rc > 0) rmax = P.rmax(pm);
                    }
                    if (stopped || 2.0 * rmax + 4.0 * eps < r_out) break;
                    if (r_out > 2.0 * diag) break;  // every site has been seen
                    // grow geometrically: a cell that is still open has a
                    // box-sized vertex radius, so jumping to 2 rmax would
                    // pull in every site
                    r_in = r_out;
                    r_out = std::min(2.0 * r_out, 2.0 * rmax + 8.0 * eps);
                }
                // faces -> neighbours, volume (pyramids from the site), bounding box
                std::vector<int32_t> &nb = nbr[m];
                nb.clear();
                double vol = 0;
                for (int f = 0; f < (int)P.F.size(); f++) {
                    double a = P.face_area(f);
                    const Plane &pl = P.F[f];
                    double hgt = pl.d - (pl.n[0] * pm[0] + pl.n[1] * pm[1] + pl.n[2] * pm[2]);
                    vol += a * hgt / 3.0;
                    if (a > 0.0) nb.push_back(pl.id);
                }
                std::sort(nb.begin(), nb.end());
                nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
                double *bb = &bbox_out[6 * m];
                for (int c = 0; c < 3; c++) { bb[c] = INFINITY; bb[3 + c] = -INFINITY; }
                for (size_t i = 0; i < P.V.size(); i += 3)
                    for (int c = 0; c < 3; c++) {
                        bb[c] = std::min(bb[c], P.V[i + c]);
                        bb[3 + c] = std::max(bb[3 + c], P.V[i + c]);
                    }
                volume[m] = vol;
            }
        }
    };
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    threads = (int)std::min<int64_t>(threads, std::max<int64_t>(1, count / 64 + 1));
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; t++) pool.emplace_back(work);
    work();
    for (auto &t : pool) t.join();
    if (failed.load() >= 0) {
        err = "cell construction failed for site " + std::to_string(failed.load());
        return -1;
    }
    return 0;
}

void cells_to_csr(const std::vector<std::vector<int32_t>> &nbr, CellsOut &out) {
    const int64_t M = (int64_t)nbr.size();
    out.off.assign(M + 1, 0);
    for (int64_t m = 0; m < M; m++) out.off[m + 1] = out.off[m] + (int64_t)nbr[m].size();
    out.idx.resize(out.off[M]);
    for (int64_t m = 0; m < M; m++) std::copy(nbr[m].begin(), nbr[m].end(), out.idx.begin() + out.off[m]);
}

int build_cells(const double *S, int64_t M, const double *box, int threads, CellsOut &out, std::string &err) {
    std::vector<std::vector<int32_t>> nbr(M);
    out.vol.assign(M, 0.0);
    out.bbox.assign(6 * M, 0.0);
    int rc = build_cells_into(S, M, box, threads, nullptr, nbr, out.vol.data(), out.bbox.data(), err);
    if (rc) return rc;
    cells_to_csr(nbr, out);
    return 0;
}

// Morton order of the sites inside the box (21 bits per axis).
static inline uint64_t spread21(uint64_t x) {
    x &= 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

void parallel_for(int64_t n, int threads, int64_t grain, const std::function<void(int64_t, int64_t)> &fn) {
    if (n <= 0) return;
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    threads = (int)std::max<int64_t>(1, std::min<int64_t>(threads, n / std::max<int64_t>(grain, 1)));
    if (threads == 1) {
        fn(0, n);
        return;
    }
    std::vector<std::thread> pool;
    const int64_t step = (n + threads - 1) / threads;
    for (int t = 1; t < threads; t++) {
        const int64_t b = t * step, e = std::min(n, b + step);
        if (b < e) pool.emplace_back(fn, b, e);
    }
    fn(0, std::min(n, step));
    for (auto &th : pool) th.join();
}

void morton_order(const double *S, int64_t M, const double *box, std::vector<int32_t> &perm,
                  std::vector<uint64_t> *codes, int threads) {
    std::vector<std::pair<uint64_t, int32_t>> key(M);
    parallel_for(M, threads, 1 << 14, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; i++) {
            uint64_t code = 0;
            for (int c = 0; c < 3; c++) {
                double u = (S[3 * i + c] - box[c]) / (box[3 + c] - box[c]);
                u = std::min(std::max(u, 0.0), 1.0);
                uint64_t q = (uint64_t)std::min(u * 2097152.0, 2097151.0);
                code |= spread21(q) << c;
            }
            key[i] = {code, (int32_t)i};
        }
    });
    std::sort(key.begin(), key.end());
    perm.resize(M);
    if (codes) codes->resize(M);
    for (int64_t i = 0; i < M; i++) {
        perm[i] = key[i].second;
        if (codes) (*codes)[i] = key[i].first;
    }
}

// Regular block grid over the box; each block lists the cells whose bounding
// box overlaps it (Sect. 2.3).
void build_blocks(const double *box, const std::vector<double> &bbox, int64_t M, double blocks_per_site,
                  BlocksOut &out, int threads) {
    double ext[3] = {box[3] - box[0], box[4] - box[1], box[5] - box[2]};
    double target = std::max(1.0, blocks_per_site * (double)M);
    double s = std::cbrt(ext[0] * ext[1] * ext[2] / target);
    for (int c = 0; c < 3; c++) {
        long n = std::lround(ext[c] / s);
        out.dim[c] = (int32_t)std::min<long>(std::max<long>(n, 1), 1024);
    }
    const int64_t K = (int64_t)out.dim[0] * out.dim[1] * out.dim[2];
    const double diag = std::sqrt(ext[0] * ext[0] + ext[1] * ext[1] + ext[2] * ext[2]);
    double maxabs = 0.0;
    for (int c = 0; c < 6; c++) maxabs = std::max(maxabs, std::fabs(box[c]));
    // covers the float32 block index on the device (error below
    // 4u |x - lo| + 4u^2 max|coordinate|, u = 2^-24)
    const double pad = 1e-6 * diag + 1e-13 * maxabs;
    auto range = [&](int64_t m, int c, int32_t &a, int32_t &b) {
        double lo = (bbox[6 * m + c] - pad - box[c]) / ext[c] * out.dim[c];
        double hi = (bbox[6 * m + 3 + c] + pad - box[c]) / ext[c] * out.dim[c];
        a = (int32_t)std::max(0.0, std::floor(lo));
        b = (int32_t)std::min((double)out.dim[c] - 1, std::floor(hi));
    };
    // cells per block (parallel over cells, atomic counters), prefix sum,
    // then every cell into the lists of its blocks and each list sorted by
    // cell index, so the lists do not depend on the thread schedule
    std::vector<std::atomic<int64_t>> count(K + 1);
    parallel_for(K + 1, threads, 1 << 16, [&](int64_t b, int64_t e) {
        for (int64_t q = b; q < e; q++) count[q].store(0, std::memory_order_relaxed);
    });
    parallel_for(M, threads, 1 << 12, [&](int64_t b0, int64_t e0) {
        for (int64_t m = b0; m < e0; m++) {
            int32_t a[3], b[3];
            for (int c = 0; c < 3; c++) range(m, c, a[c], b[c]);
            for (int32_t i = a[0]; i <= b[0]; i++)
                for (int32_t j = a[1]; j <= b[1]; j++)
                    for (int32_t k = a[2]; k <= b[2]; k++)
                        count[((int64_t)i * out.dim[1] + j) * out.dim[2] + k + 1].fetch_add(1, std::memory_order_relaxed);
        }
    });
    out.off.resize(K + 1);
    out.off[0] = 0;
    for (int64_t q = 0; q < K; q++) out.off[q + 1] = out.off[q] + count[q + 1].load(std::memory_order_relaxed);
    out.idx.resize(out.off[K]);
    parallel_for(K, threads, 1 << 16, [&](int64_t b, int64_t e) {
        for (int64_t q = b; q < e; q++) count[q].store(out.off[q], std::memory_order_relaxed);  // cursors
    });
    parallel_for(M, threads, 1 << 12, [&](int64_t b0, int64_t e0) {
        for (int64_t m = b0; m < e0; m++) {
            int32_t a[3], b[3];
            for (int c = 0; c < 3; c++) range(m, c, a[c], b[c]);
            for (int32_t i = a[0]; i <= b[0]; i++)
                for (int32_t j = a[1]; j <= b[1]; j++)
                    for (int32_t k = a[2]; k <= b[2]; k++)
                        out.idx[count[((int64_t)i * out.dim[1] + j) * out.dim[2] + k].fetch_add(
                            1, std::memory_order_relaxed)] = (int32_t)m;
        }
    });
    parallel_for(K, threads, 1 << 12, [&](int64_t b, int64_t e) {
        for (int64_t q = b; q < e; q++) std::sort(out.idx.begin() + out.off[q], out.idx.begin() + out.off[q + 1]);
    });
}

}  // namespace vg
