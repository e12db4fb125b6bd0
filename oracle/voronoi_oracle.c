/*
 * CPU oracle for straight-path traversal of 3D Voronoi grids
 * (Camps, Baes & Saftly 2013, "Using 3D Voronoi grids in radiative transfer
 * simulations", Sect. 2).
 *
 * THIS FILE IS TEST INFRASTRUCTURE. It is plain, slow, FP64 C written from
 * the paper's definitions. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the GPU library never does, and
 * the two share no code.
 *
 * Contents
 *   oracle_cells   Voronoi cell of a site by clipping the domain box with the
 *                  bisector half-space of other sites (Sect. 2.1: a cell is the
 *                  set of points at least as close to its site as to any other
 *                  site). Candidates are taken in increasing distance; the
 *                  loop stops once a candidate is farther than twice the
 *                  largest vertex radius (its bisector plane then lies
 *                  entirely outside the cell), or never stops (brute = 1).
 *                  The sites within a shell of radii are found through a
 *                  uniform bucket grid (every site of every bucket that meets
 *                  the shell's bounding cube is tested against the radii), so
 *                  the candidate set and its order are those of a loop over
 *                  all sites.
 *                  Gives the neighbour list (faces of positive area, walls as
 *                  -1..-6), the cell volume and bounding box (Sect. 2.3).
 *   oracle_locate  C(r): nearest site by brute force over all sites,
 *                  negative index outside the domain (Sect. 2.3 steps 1, 4).
 *   Domains: the box, or a sphere inside the box (Sect. 2.2 notes that the
 *                  method carries over to other domain geometries). In a
 *                  spherical domain the cells keep the lists of the box's
 *                  clipping (a face outside the sphere is never reached, as
 *                  the path leaves the domain first), a point is inside when
 *                  its squared distance to the centre is at most R^2, and the
 *                  domain exit is the sphere's: the larger root s of
 *                  |r + s k - c|^2 = R^2 from the current point, in place of
 *                  the box walls' Eq. 5, with the wall id -7.
 *   oracle_trace   the straight-path loop of Sect. 2.2 with the exit-point
 *                  algorithm (steps 1-3), bisector intersection Eq. 1-4,
 *                  wall intersection Eq. 5 and the epsilon nudge when no exit
 *                  is found. Candidates are either the cell's neighbour list
 *                  (the paper's algorithm) or every other site and all six
 *                  walls (the plain definition of the exit; identical result
 *                  because a cell is the intersection of all bisector
 *                  half-spaces).
 *
 * Readings where the paper is silent (numbered as in the design notes):
 *   R2 candidate planes are those with n.k > 0 (Sect. 2.2 sign shortcut);
 *   R3 a numerator that rounds below zero is clamped to zero;
 *   R4 ties are broken by the lexicographic order of (s, id); walls carry
 *      negative ids and so win exact ties;
 *   R5 zero-length steps emit no segment;
 *   R6 epsilon = 1e-12 * |Dmax - Dmin|; more than Z consecutive
 *      zero-length steps also trigger the nudge (Z = 4 by default; a test
 *      may lower it, Z = 0 nudging after every zero-length step);
 *   R9 the current point is updated literally, r <- r + s k.
 * Floating-point contraction is disabled at compile time so that results do
 * not depend on the host's FMA support.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_MAXF 256
#define OR_MAXV 96

/* ------------------------------------------------------------------------ */
/* threads: a plain parallel-for over independent items                      */
/* ------------------------------------------------------------------------ */

typedef void (*or_item_fn)(void *ctx, int64_t i, void *scratch);

typedef struct {
    or_item_fn fn;
    void *ctx;
    int64_t n;
    int64_t next;
    pthread_mutex_t lock;
    size_t scratch_bytes;
    int failed;
} or_pool;

static void *or_worker(void *arg)
{
    or_pool *p = (or_pool *)arg;
    void *scratch = p->scratch_bytes ? malloc(p->scratch_bytes) : NULL;
    if (p->scratch_bytes && !scratch) {
        pthread_mutex_lock(&p->lock);
        p->failed = 1;
        pthread_mutex_unlock(&p->lock);
        return NULL;
    }
    for (;;) {
        int64_t lo, hi;
        pthread_mutex_lock(&p->lock);
        lo = p->next;
        hi = lo + 16;
        if (hi > p->n) hi = p->n;
        p->next = hi;
        pthread_mutex_unlock(&p->lock);
        if (lo >= p->n) break;
        for (int64_t i = lo; i < hi; i++) p->fn(p->ctx, i, scratch);
    }
    free(scratch);
    return NULL;
}

static int or_parallel_for(int64_t n, or_item_fn fn, void *ctx, size_t scratch_bytes, int nthreads)
{
    or_pool p;
    p.fn = fn;
    p.ctx = ctx;
    p.n = n;
    p.next = 0;
    p.scratch_bytes = scratch_bytes;
    p.failed = 0;
    pthread_mutex_init(&p.lock, NULL);
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > n) nthreads = (int)(n > 0 ? n : 1);
    pthread_t th[256];
    int started = 0;
    for (int t = 1; t < nthreads; t++) {
        if (pthread_create(&th[t], NULL, or_worker, &p) == 0) started = t;
        else break;
    }
    or_worker(&p);
    for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&p.lock);
    return p.failed ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* convex polyhedron as a list of planar faces                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int id;          /* neighbour site index, or wall -1..-6 */
    double n[3];     /* unit outward normal: the cell is {x : n.x <= d} */
    double d;
    int nv;
    double v[OR_MAXV][3];
} or_face;

typedef struct {
    int nf;
    or_face f[OR_MAXF];
} or_poly;

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* The box [xmin,xmax] x [ymin,ymax] x [zmin,zmax] as six quadrilaterals.
 * Wall ids: -1 x=xmin, -2 x=xmax, -3 y=ymin, -4 y=ymax, -5 z=zmin, -6 z=zmax. */
static void poly_box(or_poly *P, const double *box)
{
    double c[8][3];
    for (int i = 0; i < 8; i++) {
        c[i][0] = (i & 4) ? box[3] : box[0];
        c[i][1] = (i & 2) ? box[4] : box[1];
        c[i][2] = (i & 1) ? box[5] : box[2];
    }
    static const int quad[6][4] = {
        {0, 1, 3, 2}, {4, 6, 7, 5}, {0, 4, 5, 1}, {2, 3, 7, 6}, {0, 2, 6, 4}, {1, 5, 7, 3}};
    P->nf = 6;
    for (int w = 0; w < 6; w++) {
        or_face *F = &P->f[w];
        int axis = w / 2, hi = w % 2;
        F->id = -(w + 1);
        F->n[0] = F->n[1] = F->n[2] = 0.0;
        F->n[axis] = hi ? 1.0 : -1.0;
        F->d = hi ? box[3 + axis] : -box[axis];
        F->nv = 4;
        for (int k = 0; k < 4; k++) memcpy(F->v[k], c[quad[w][k]], sizeof(double) * 3);
    }
}

/* Clip P by {x : n.x <= d} (n unit). Returns 1 if some vertex lay outside by
 * more than eps, 0 if the plane does not cut, -1 on capacity overflow. */
static int poly_clip(or_poly *P, const double *n, double d, int id, double eps)
{
    int any_out = 0;
    for (int f = 0; f < P->nf && !any_out; f++)
        for (int i = 0; i < P->f[f].nv; i++)
            if (dot3(n, P->f[f].v[i]) - d > eps) { any_out = 1; break; }
    if (!any_out) return 0;

    double cap[OR_MAXV * 4][3];
    int ncap = 0;
    int nf_out = 0;
    for (int f = 0; f < P->nf; f++) {
        or_face *F = &P->f[f];
        double out[OR_MAXV][3];
        int no = 0;
        double fv[OR_MAXV];
        for (int i = 0; i < F->nv; i++) fv[i] = dot3(n, F->v[i]) - d;
        for (int i = 0; i < F->nv; i++) {
            int j = (i + 1) % F->nv;
            const double *a = F->v[i], *b = F->v[j];
            double fa = fv[i], fb = fv[j];
            int a_in = fa <= eps, b_in = fb <= eps;
            if (a_in) {
                if (no >= OR_MAXV) return -1;
                memcpy(out[no++], a, sizeof(double) * 3);
                if (fa >= -eps) {
                    if (ncap >= OR_MAXV * 4) return -1;
                    memcpy(cap[ncap++], a, sizeof(double) * 3);
                }
            }
            if (a_in != b_in && ((a_in && fa < -eps) || (!a_in && fb < -eps))) {
                double t = fa / (fa - fb), x[3];
                for (int c = 0; c < 3; c++) x[c] = a[c] + t * (b[c] - a[c]);
                if (no >= OR_MAXV || ncap >= OR_MAXV * 4) return -1;
                memcpy(out[no++], x, sizeof(double) * 3);
                memcpy(cap[ncap++], x, sizeof(double) * 3);
            }
        }
        if (no >= 3) {
            or_face *G = &P->f[nf_out++];
            if (G != F) { G->id = F->id; memcpy(G->n, F->n, sizeof(F->n)); G->d = F->d; }
            G->nv = no;
            memcpy(G->v, out, sizeof(double) * 3 * no);
        }
    }
    P->nf = nf_out;

    /* the new face: distinct cut points ordered by angle about their centroid */
    double pts[OR_MAXV][3];
    int np = 0;
    for (int i = 0; i < ncap; i++) {
        int dup = 0;
        for (int k = 0; k < np && !dup; k++) {
            double dx = cap[i][0] - pts[k][0], dy = cap[i][1] - pts[k][1], dz = cap[i][2] - pts[k][2];
            if (dx * dx + dy * dy + dz * dz <= 16.0 * eps * eps) dup = 1;
        }
        if (!dup) {
            if (np >= OR_MAXV) return -1;
            memcpy(pts[np++], cap[i], sizeof(double) * 3);
        }
    }
    if (np < 3) return 1;
    if (P->nf >= OR_MAXF) return -1;
    double cen[3] = {0, 0, 0};
    for (int i = 0; i < np; i++)
        for (int c = 0; c < 3; c++) cen[c] += pts[i][c];
    for (int c = 0; c < 3; c++) cen[c] /= np;
    double ax[3] = {0, 0, 0}, u[3], w[3];
    int a = fabs(n[0]) <= fabs(n[1]) ? (fabs(n[0]) <= fabs(n[2]) ? 0 : 2) : (fabs(n[1]) <= fabs(n[2]) ? 1 : 2);
    ax[a] = 1.0;
    cross3(n, ax, u);
    double un = sqrt(dot3(u, u));
    for (int c = 0; c < 3; c++) u[c] /= un;
    cross3(n, u, w);
    double ang[OR_MAXV];
    for (int i = 0; i < np; i++) {
        double q[3] = {pts[i][0] - cen[0], pts[i][1] - cen[1], pts[i][2] - cen[2]};
        ang[i] = atan2(dot3(q, w), dot3(q, u));
    }
    /* insertion sort by angle */
    for (int i = 1; i < np; i++) {
        double ak = ang[i], pk[3];
        memcpy(pk, pts[i], sizeof pk);
        int k = i - 1;
        while (k >= 0 && ang[k] > ak) {
            ang[k + 1] = ang[k];
            memcpy(pts[k + 1], pts[k], sizeof pk);
            k--;
        }
        ang[k + 1] = ak;
        memcpy(pts[k + 1], pk, sizeof pk);
    }
    or_face *F = &P->f[P->nf++];
    F->id = id;
    memcpy(F->n, n, sizeof(double) * 3);
    F->d = d;
    F->nv = np;
    memcpy(F->v, pts, sizeof(double) * 3 * np);
    return 1;
}

static double face_area(const or_face *F)
{
    double s[3] = {0, 0, 0};
    for (int i = 1; i + 1 < F->nv; i++) {
        double a[3], b[3], c[3];
        for (int k = 0; k < 3; k++) {
            a[k] = F->v[i][k] - F->v[0][k];
            b[k] = F->v[i + 1][k] - F->v[0][k];
        }
        cross3(a, b, c);
        for (int k = 0; k < 3; k++) s[k] += c[k];
    }
    return 0.5 * fabs(dot3(s, F->n));
}

static double poly_rmax(const or_poly *P, const double *c)
{
    double r2 = 0.0;
    for (int f = 0; f < P->nf; f++)
        for (int i = 0; i < P->f[f].nv; i++) {
            double dx = P->f[f].v[i][0] - c[0], dy = P->f[f].v[i][1] - c[1], dz = P->f[f].v[i][2] - c[2];
            double q = dx * dx + dy * dy + dz * dz;
            if (q > r2) r2 = q;
        }
    return sqrt(r2);
}

/* ------------------------------------------------------------------------ */
/* cells                                                                    */
/* ------------------------------------------------------------------------ */

/* Uniform bucket grid over the box: bucket b holds the sites
 * ids[start[b] .. start[b+1]-1]; a site's bucket along an axis is
 * floor((x - lo) / h) clamped to [0, n - 1], a non-decreasing function of x,
 * so every site within distance r of a point lies in a bucket between those
 * of the point's coordinates minus and plus r. */
typedef struct {
    int n[3];
    double lo[3], h[3];
    int64_t *start;
    int64_t *ids;
} or_buckets;

static int bucket_coord(const or_buckets *B, int c, double x)
{
    double f = floor((x - B->lo[c]) / B->h[c]);
    if (!(f >= 0.0)) return 0;
    if (f >= (double)(B->n[c] - 1)) return B->n[c] - 1;
    return (int)f;
}

static int buckets_build(or_buckets *B, const double *S, int64_t M, const double *box)
{
    double ext[3], vol = 1.0;
    for (int c = 0; c < 3; c++) {
        ext[c] = box[3 + c] - box[c];
        vol *= ext[c];
    }
    double side = cbrt(2.0 * vol / (double)(M > 0 ? M : 1)); /* about two sites per bucket */
    int64_t nb = 1;
    for (int c = 0; c < 3; c++) {
        double k = floor(ext[c] / side);
        B->n[c] = k < 1.0 ? 1 : (k > 1024.0 ? 1024 : (int)k);
        B->lo[c] = box[c];
        B->h[c] = ext[c] / B->n[c];
        nb *= B->n[c];
    }
    B->start = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    B->ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M > 0 ? M : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
    if (!B->start || !B->ids || !fill) {
        free(fill);
        return -1;
    }
    for (int64_t j = 0; j < M; j++) {
        const double *p = S + 3 * j;
        int64_t b = ((int64_t)bucket_coord(B, 0, p[0]) * B->n[1] + bucket_coord(B, 1, p[1])) * B->n[2] +
                    bucket_coord(B, 2, p[2]);
        B->start[b + 1]++;
    }
    for (int64_t b = 0; b < nb; b++) B->start[b + 1] += B->start[b];
    memcpy(fill, B->start, sizeof(int64_t) * (size_t)nb);
    for (int64_t j = 0; j < M; j++) {
        const double *p = S + 3 * j;
        int64_t b = ((int64_t)bucket_coord(B, 0, p[0]) * B->n[1] + bucket_coord(B, 1, p[1])) * B->n[2] +
                    bucket_coord(B, 2, p[2]);
        B->ids[fill[b]++] = j;
    }
    free(fill);
    return 0;
}

typedef struct {
    const double *S;
    int64_t M;
    const double *box;
    const or_buckets *B;
    const int64_t *cells;
    int brute;
    int maxdeg;
    double eps, area_tol;
    int32_t *nbr;
    int32_t *deg;
    double *area;
    double *vol;
    double *bbox;
    int32_t *err;
} cells_ctx;

typedef struct { double d2; int64_t j; } or_cand;

static int cand_cmp(const void *x, const void *y)
{
    const or_cand *a = (const or_cand *)x, *b = (const or_cand *)y;
    if (a->d2 < b->d2) return -1;
    if (a->d2 > b->d2) return 1;
    return (a->j > b->j) - (a->j < b->j);
}

/* Bisector half-space of sites m and j that contains site m, as a unit
 * normal n and offset d (Eq. 1-3: normal p_j - p_m through the midpoint). */
static void bisector(const double *pm, const double *pj, double *n, double *d)
{
    double v[3] = {pj[0] - pm[0], pj[1] - pm[1], pj[2] - pm[2]};
    double l = sqrt(dot3(v, v));
    double mid[3] = {0.5 * (pj[0] + pm[0]), 0.5 * (pj[1] + pm[1]), 0.5 * (pj[2] + pm[2])};
    for (int c = 0; c < 3; c++) n[c] = v[c] / l;
    *d = dot3(n, mid);
}

static void cell_item(void *vctx, int64_t ci, void *scratch)
{
    cells_ctx *X = (cells_ctx *)vctx;
    int64_t m = X->cells[ci];
    const double *pm = X->S + 3 * m;
    or_poly *P = (or_poly *)scratch;
    or_cand *cand = (or_cand *)((char *)scratch + sizeof(or_poly));
    int32_t *out_nbr = X->nbr + ci * X->maxdeg;
    double *out_area = X->area + ci * X->maxdeg;
    poly_box(P, X->box);

    double lo[3] = {X->box[0], X->box[1], X->box[2]}, hi[3] = {X->box[3], X->box[4], X->box[5]};
    double vbox = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    double r_c = 3.0 * cbrt(vbox / (double)X->M);
    if (!X->brute) {
        /* first shell: three site spacings at the density of the site's own
         * bucket. Where the shells are cut does not change the result: the
         * candidates are still clipped in increasing (distance, index) order
         * up to the first one beyond twice the largest vertex radius. */
        const or_buckets *B = X->B;
        int64_t b = ((int64_t)bucket_coord(B, 0, pm[0]) * B->n[1] + bucket_coord(B, 1, pm[1])) * B->n[2] +
                    bucket_coord(B, 2, pm[2]);
        double nloc = (double)(B->start[b + 1] - B->start[b]);
        r_c = 3.0 * cbrt(B->h[0] * B->h[1] * B->h[2] / (nloc > 1.0 ? nloc : 1.0));
    }
    double r_prev = -1.0;
    int done = 0;
    while (!done) {
        int64_t nc = 0;
        /* the sites with r_prev < d <= r_c (all sites with brute), from the
         * buckets meeting the cube of half side r_c around the site, or from
         * a loop over all sites when that cube spans more buckets than there
         * are sites */
        const or_buckets *B = X->B;
        int b0[3] = {0, 0, 0}, b1[3] = {0, 0, 0};
        double span = 1.0;
        if (!X->brute)
            for (int c = 0; c < 3; c++) {
                b0[c] = bucket_coord(B, c, pm[c] - r_c);
                b1[c] = bucket_coord(B, c, pm[c] + r_c);
                span *= (double)(b1[c] - b0[c] + 1);
            }
        if (X->brute || span > (double)X->M) {
            for (int64_t j = 0; j < X->M; j++) {
                if (j == m) continue;
                const double *pj = X->S + 3 * j;
                double dx = pj[0] - pm[0], dy = pj[1] - pm[1], dz = pj[2] - pm[2];
                double d2 = dx * dx + dy * dy + dz * dz;
                if (!X->brute) {
                    if (r_prev >= 0.0 && d2 <= r_prev * r_prev) continue; /* earlier shell */
                    if (d2 > r_c * r_c) continue;                         /* later shell */
                }
                cand[nc].d2 = d2;
                cand[nc].j = j;
                nc++;
            }
        } else {
            for (int ix = b0[0]; ix <= b1[0]; ix++)
                for (int iy = b0[1]; iy <= b1[1]; iy++)
                    for (int iz = b0[2]; iz <= b1[2]; iz++) {
                        int64_t b = ((int64_t)ix * B->n[1] + iy) * B->n[2] + iz;
                        for (int64_t q = B->start[b]; q < B->start[b + 1]; q++) {
                            int64_t j = B->ids[q];
                            if (j == m) continue;
                            const double *pj = X->S + 3 * j;
                            double dx = pj[0] - pm[0], dy = pj[1] - pm[1], dz = pj[2] - pm[2];
                            double d2 = dx * dx + dy * dy + dz * dz;
                            if (r_prev >= 0.0 && d2 <= r_prev * r_prev) continue; /* earlier shell */
                            if (d2 > r_c * r_c) continue;                         /* later shell */
                            cand[nc].d2 = d2;
                            cand[nc].j = j;
                            nc++;
                        }
                    }
        }
        qsort(cand, (size_t)nc, sizeof(or_cand), cand_cmp);
        double rmax = poly_rmax(P, pm);
        int stopped = 0;
        for (int64_t k = 0; k < nc; k++) {
            double dist = sqrt(cand[k].d2);
            if (!X->brute && dist > 2.0 * rmax + 4.0 * X->eps) { stopped = 1; break; }
            double n[3], d;
            bisector(pm, X->S + 3 * cand[k].j, n, &d);
            int rc = poly_clip(P, n, d, (int)cand[k].j, X->eps);
            if (rc < 0) { X->err[ci] = 1; return; }
            if (rc > 0) rmax = poly_rmax(P, pm);
        }
        if (X->brute || stopped) done = 1;
        else {
            /* every site within r_c has been used; continue only if some site
             * beyond r_c could still cut the cell */
            if (2.0 * rmax + 4.0 * X->eps < r_c) done = 1;
            else {
                r_prev = r_c;
                r_c = 2.0 * r_c; /* the next shell; any radius gives the same order */
                int64_t remaining = 0;
                for (int64_t j = 0; j < X->M && !remaining; j++) {
                    if (j == m) continue;
                    const double *pj = X->S + 3 * j;
                    double dx = pj[0] - pm[0], dy = pj[1] - pm[1], dz = pj[2] - pm[2];
                    if (dx * dx + dy * dy + dz * dz > r_prev * r_prev) remaining = 1;
                }
                if (!remaining) done = 1;
            }
        }
    }

    /* neighbours: faces of positive area; volume as pyramids from the site */
    int nd = 0;
    double vol = 0.0;
    double bb[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int f = 0; f < P->nf; f++) {
        const or_face *F = &P->f[f];
        double a = face_area(F);
        double h = F->d - dot3(F->n, pm);
        vol += a * h / 3.0;
        for (int i = 0; i < F->nv; i++)
            for (int c = 0; c < 3; c++) {
                if (F->v[i][c] < bb[c]) bb[c] = F->v[i][c];
                if (F->v[i][c] > bb[3 + c]) bb[3 + c] = F->v[i][c];
            }
        if (a > X->area_tol) {
            if (nd >= X->maxdeg) { X->err[ci] = 2; return; }
            out_nbr[nd] = F->id;
            out_area[nd] = a;
            nd++;
        }
    }
    /* sort ascending by id for a canonical order */
    for (int i = 1; i < nd; i++) {
        int32_t id = out_nbr[i];
        double a = out_area[i];
        int k = i - 1;
        while (k >= 0 && out_nbr[k] > id) {
            out_nbr[k + 1] = out_nbr[k];
            out_area[k + 1] = out_area[k];
            k--;
        }
        out_nbr[k + 1] = id;
        out_area[k + 1] = a;
    }
    X->deg[ci] = nd;
    X->vol[ci] = vol;
    memcpy(X->bbox + 6 * ci, bb, sizeof bb);
}

/* Voronoi cells of the listed sites. nbr/area are ncells x maxdeg, row ci
 * holding deg[ci] entries. Returns 0, or -1 (capacity / allocation), with
 * err[ci] != 0 marking the failed cells. */
int oracle_cells(const double *sites, int64_t M, const double *box, const int64_t *cells, int64_t ncells,
                 int brute, int maxdeg, double eps, double area_tol, int32_t *nbr, int32_t *deg, double *area,
                 double *vol, double *bbox, int32_t *err, int nthreads)
{
    or_buckets B = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, NULL, NULL};
    memset(err, 0, sizeof(int32_t) * (size_t)ncells);
    if (!brute && buckets_build(&B, sites, M, box) != 0) {
        free(B.start);
        free(B.ids);
        return -1;
    }
    cells_ctx X = {sites, M, box, &B, cells, brute, maxdeg, eps, area_tol, nbr, deg, area, vol, bbox, err};
    size_t scratch = sizeof(or_poly) + sizeof(or_cand) * (size_t)(M > 0 ? M : 1);
    int rc = or_parallel_for(ncells, cell_item, &X, scratch, nthreads);
    free(B.start);
    free(B.ids);
    if (rc != 0) return -1;
    for (int64_t i = 0; i < ncells; i++)
        if (err[i]) return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* locate                                                                   */
/* ------------------------------------------------------------------------ */

/* Nearest site to r (lowest index on exact ties), -1 outside the closed box.
 * If mu is given it receives the relative gap (d2 - d1) / d2 between the
 * nearest and second-nearest site distances (+inf with one site). */
/* Inside the closed domain: the box, and the ball when sph (cx, cy, cz, R)
 * is given. */
static int inside_domain(const double *box, const double *sph, const double *r)
{
    for (int c = 0; c < 3; c++)
        if (!(r[c] >= box[c] && r[c] <= box[3 + c])) return 0;
    if (sph) {
        double dx = r[0] - sph[0], dy = r[1] - sph[1], dz = r[2] - sph[2];
        if (!((dx * dx + dy * dy) + dz * dz <= sph[3] * sph[3])) return 0;
    }
    return 1;
}

/* Exit of r + s k (s >= 0) from the ball (cx, cy, cz, R): with o = r - c,
 * b = k.o and q = o.o - R^2, the larger root of s^2 + 2 b s + q = 0 (k a unit
 * vector), -b + sqrt(b^2 - q), written as -q / (b + sqrt(b^2 - q)) when
 * b > 0 so that no digits cancel. */
static double sphere_exit(const double *sph, const double *r, const double *k)
{
    double o[3];
    for (int c = 0; c < 3; c++) o[c] = r[c] - sph[c];
    double b = (k[0] * o[0] + k[1] * o[1]) + k[2] * o[2];
    double q = ((o[0] * o[0] + o[1] * o[1]) + o[2] * o[2]) - sph[3] * sph[3];
    double disc = b * b - q;
    if (disc < 0.0) disc = 0.0;
    double sq = sqrt(disc);
    double s = b > 0.0 ? -q / (b + sq) : sq - b;
    return s < 0.0 ? 0.0 : s;
}

static int64_t locate_mu(const double *S, int64_t M, const double *box, const double *sph, const double *r,
                         double *mu)
{
    if (!inside_domain(box, sph, r)) return -1;
    int64_t best = -1;
    double bd = INFINITY, sd = INFINITY;
    for (int64_t j = 0; j < M; j++) {
        double dx = r[0] - S[3 * j], dy = r[1] - S[3 * j + 1], dz = r[2] - S[3 * j + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < bd) { sd = bd; bd = d2; best = j; }
        else if (d2 < sd) sd = d2;
    }
    if (mu) *mu = isinf(sd) ? INFINITY : (sqrt(sd) - sqrt(bd)) / sqrt(sd);
    return best;
}

static int64_t locate1(const double *S, int64_t M, const double *box, const double *sph, const double *r)
{
    return locate_mu(S, M, box, sph, r, NULL);
}

typedef struct { const double *S; int64_t M; const double *box, *sph; const double *pts; int64_t *out; } loc_ctx;

static void loc_item(void *vctx, int64_t i, void *scratch)
{
    (void)scratch;
    loc_ctx *X = (loc_ctx *)vctx;
    X->out[i] = locate1(X->S, X->M, X->box, X->sph, X->pts + 3 * i);
}

/* C(r) for N points: index of the nearest site (lowest index on exact ties),
 * -1 for points outside the closed domain (the box, and the ball sphere =
 * (cx, cy, cz, R) unless NULL). */
void oracle_locate(const double *sites, int64_t M, const double *box, const double *sphere, const double *pts,
                   int64_t N, int64_t *out, int nthreads)
{
    loc_ctx X = {sites, M, box, sphere, pts, out};
    or_parallel_for(N, loc_item, &X, 0, nthreads);
}

/* ------------------------------------------------------------------------ */
/* trace                                                                    */
/* ------------------------------------------------------------------------ */

enum { OR_OK = 0, OR_OUTSIDE = 1, OR_STEP_LIMIT = 2, OR_CAPACITY = 3 };

typedef struct {
    const double *S;
    int64_t M;
    const double *box;
    const double *sph;  /* NULL: the box is the domain; else (cx, cy, cz, R) */
    const int64_t *off;
    const int32_t *idx; /* NULL: every site and all walls are candidates */
    const double *rho;
    double kappa;
    const double *org, *dir;
    int64_t cap;
    int32_t *seg_cell;
    double *seg_len;
    int32_t *nseg;
    double *tau, *length, *min_margin;
    int32_t *near_tie, *nfallback, *status;
    int64_t max_steps;
    int zmax;            /* zero-length steps in a row tolerated before the nudge */
    double eps_nudge, tie_rel;
} trace_ctx;

/* One candidate plane: s from Eq. 4 (bisector) or Eq. 5 (wall), or the
 * sphere's exit (id -7). Returns 0 if it is not a candidate (n.k <= 0; the
 * box walls of a spherical domain). */
static int plane_s(const trace_ctx *X, int64_t m, int64_t j, const double *r, const double *k, double *s_out,
                   double *num_out, double *nlen_out)
{
    if (j >= 0) {
        const double *pm = X->S + 3 * m, *pj = X->S + 3 * j;
        double n[3], mid[3], w[3];
        for (int c = 0; c < 3; c++) n[c] = pj[c] - pm[c];          /* Eq. 1 */
        double den = (n[0] * k[0] + n[1] * k[1]) + n[2] * k[2];
        if (!(den > 0.0)) return 0;                                 /* R2 */
        for (int c = 0; c < 3; c++) mid[c] = (pj[c] + pm[c]) * 0.5; /* Eq. 2 */
        for (int c = 0; c < 3; c++) w[c] = mid[c] - r[c];
        double num = (n[0] * w[0] + n[1] * w[1]) + n[2] * w[2];     /* Eq. 4 */
        *num_out = num;
        *nlen_out = sqrt((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
        if (num < 0.0) num = 0.0;                                   /* R3 */
        *s_out = num / den;
        return 1;
    } else if (j == -7) {
        double s = sphere_exit(X->sph, r, k);
        *num_out = s;
        *nlen_out = 1.0;
        *s_out = s;
        return 1;
    } else {
        if (X->sph) return 0;
        int w = (int)(-j - 1), axis = w / 2, hi = w % 2;
        double kc = k[axis];
        if (hi ? !(kc > 0.0) : !(kc < 0.0)) return 0;             /* n.k > 0 */
        double bound = hi ? X->box[3 + axis] : X->box[axis];
        double num = bound - r[axis];                               /* Eq. 5 */
        double s = num / kc;
        *num_out = hi ? num : -num;
        *nlen_out = 1.0;
        if (s < 0.0) s = 0.0;
        *s_out = s;
        return 1;
    }
}

static void trace_item(void *vctx, int64_t i, void *scratch)
{
    (void)scratch;
    trace_ctx *X = (trace_ctx *)vctx;
    const double *k = X->dir + 3 * i;
    double r[3] = {X->org[3 * i], X->org[3 * i + 1], X->org[3 * i + 2]};
    double mu0;
    int64_t m = locate_mu(X->S, X->M, X->box, X->sph, r, &mu0);
    double tau = 0.0, len = 0.0, mmin = INFINITY;
    int32_t ns = 0, nfb = 0, tie = 0, st = OR_OK;
    /* a start point (nearly) equidistant from two sites is a near tie too */
    if (m >= 0 && mu0 <= X->tie_rel) tie = 1;
    if (m < 0) {
        st = OR_OUTSIDE;
        goto out;
    }
    int zrun = 0;
    for (int64_t step = 0;; step++) {
        if (step >= X->max_steps) { st = OR_STEP_LIMIT; break; }
        const double *pm = X->S + 3 * m;
        double best = INFINITY, second = INFINITY, best_num = 0.0, best_nlen = 1.0;
        int64_t best_id = INT64_MAX;
        double hmin2 = INFINITY;
        /* the cell's list (or every site and the six walls), then the
           sphere of a spherical domain */
        int64_t nl = X->idx ? (X->off[m + 1] - X->off[m]) : (X->M + 6);
        int64_t nc = nl + (X->sph ? 1 : 0);
        for (int64_t q = 0; q < nc; q++) {
            int64_t j;
            if (q == nl) j = -7;
            else if (X->idx) j = X->idx[X->off[m] + q];
            else j = q < X->M ? q : -(q - X->M + 1);
            if (j == m) continue;
            if (j >= 0) {
                const double *pj = X->S + 3 * j;
                double dx = pj[0] - pm[0], dy = pj[1] - pm[1], dz = pj[2] - pm[2];
                double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 < hmin2) hmin2 = d2;
            }
            double s, num, nlen;
            if (!plane_s(X, m, j, r, k, &s, &num, &nlen)) continue;
            if (s < best || (s == best && j < best_id)) {                /* R4 */
                second = best;
                best = s;
                best_id = j;
                best_num = num;
                best_nlen = nlen;
            } else if (s < second) {
                second = s;
            }
        }
        if (best_id == INT64_MAX) {
            /* no exit found: nudge over epsilon and relocate (Sect. 2.2) */
            nfb++;
            for (int c = 0; c < 3; c++) r[c] = r[c] + X->eps_nudge * k[c];
            m = locate1(X->S, X->M, X->box, X->sph, r);
            zrun = 0;
            if (m < 0) break;
            continue;
        }
        /* decision margin against the local cell scale h_m */
        double h = 0.5 * sqrt(hmin2);
        double mu = (second - best) / fmax(best, h);
        if (mu < mmin) mmin = mu;
        if (mu <= X->tie_rel || fabs(best_num) <= X->tie_rel * h * best_nlen) tie = 1;
        if (best > 0.0) {
            if (ns < X->cap) {
                X->seg_cell[i * X->cap + ns] = (int32_t)m;
                X->seg_len[i * X->cap + ns] = best;
            } else if (X->cap > 0) {
                st = OR_CAPACITY;
            }
            ns++;
            tau += X->kappa * X->rho[m] * best;
            len += best;
            zrun = 0;
        } else {
            zrun++;
        }
        for (int c = 0; c < 3; c++) r[c] = r[c] + best * k[c];  /* R9 */
        if (best_id < 0) break;
        m = best_id;
        if (zrun > X->zmax) {
            nfb++;
            for (int c = 0; c < 3; c++) r[c] = r[c] + X->eps_nudge * k[c];
            m = locate1(X->S, X->M, X->box, X->sph, r);
            zrun = 0;
            if (m < 0) break;
        }
    }
out:
    X->nseg[i] = ns;
    X->tau[i] = tau;
    X->length[i] = len;
    X->min_margin[i] = mmin;
    X->near_tie[i] = tie;
    X->nfallback[i] = nfb;
    X->status[i] = st;
}

/* Straight paths for N rays (origin, unit direction). With idx == NULL the
 * candidates are all other sites plus the six walls; otherwise the CSR
 * neighbour lists off/idx (walls as -1..-6). With sphere = (cx, cy, cz, R)
 * the domain is that ball (inside the box): its exit replaces the walls. Per ray: segments (cell, length)
 * up to cap, the count, tau = sum kappa rho l, the summed length, the
 * smallest decision margin, a near-tie flag, fallback count, status. More
 * than zmax zero-length steps in a row nudge the point by epsilon and locate
 * it again, as a decision without any exit does (Sect. 2.2). */
void oracle_trace(const double *sites, int64_t M, const double *box, const double *sphere, const int64_t *off,
                  const int32_t *idx,
                  const double *rho, double kappa, const double *org, const double *dir, int64_t N, int64_t cap,
                  int32_t *seg_cell, double *seg_len, int32_t *nseg, double *tau, double *length,
                  double *min_margin, int32_t *near_tie, int32_t *nfallback, int32_t *status, int64_t max_steps,
                  int zmax, double tie_rel, int nthreads)
{
    double dx = box[3] - box[0], dy = box[4] - box[1], dz = box[5] - box[2];
    trace_ctx X;
    X.S = sites;
    X.M = M;
    X.box = box;
    X.sph = sphere;
    X.off = off;
    X.idx = idx;
    X.rho = rho;
    X.kappa = kappa;
    X.org = org;
    X.dir = dir;
    X.cap = cap;
    X.seg_cell = seg_cell;
    X.seg_len = seg_len;
    X.nseg = nseg;
    X.tau = tau;
    X.length = length;
    X.min_margin = min_margin;
    X.near_tie = near_tie;
    X.nfallback = nfallback;
    X.status = status;
    X.max_steps = max_steps;
    X.zmax = zmax < 0 ? 0 : zmax;
    X.eps_nudge = 1e-12 * sqrt(dx * dx + dy * dy + dz * dz); /* R6 */
    X.tie_rel = tie_rel;
    or_parallel_for(N, trace_item, &X, 0, nthreads);
}
