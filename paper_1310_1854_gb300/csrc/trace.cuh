// Device code of the straight-path traversal (Sect. 2.2 of Camps, Baes &
// Saftly 2013) and of C(r) (Sect. 2.3), shared by the kernel instantiations.
//
// Work mapping: a persistent grid of warps; each warp is split into groups of
// LPR lanes, one ray per group. A group takes a new ray from a global counter
// as soon as its ray ends, so rays of very different length do not leave
// lanes idle; with a ray order the counter indexes a permutation that hands
// out the rays with the longest estimated paths first, so that the launch
// does not end waiting for a few long rays started late. Inside a crossing
// the group's lanes stride over the current cell's block (32-byte record
// pairs, one 256-bit load each) and reduce the exit with shuffles.
//
// Cell blocks, in two forms; each crossing reads one contiguous block.
//  * absolute (float64 form, rechecks): cell i owns a run of float4 at A_i:
//    a header (caller's id, neighbour count, rho, F_i) and one record per
//    neighbour (x, y, z of the neighbour's site, and its offset A_j, or a
//    wall id -1..-6); the winner's record holds the next site and block.
//  * relative (float32 form): cell i owns a run at F_i: (x, y, z of p_i,
//    record count), (caller's id, rho, N1max, A_i), then one record per cell
//    neighbour (n~ = fl(p_j - p_i), the neighbour's offset F_j), padded with
//    NaN records to an even count of at least four. Walls are not records
//    there: the wall ahead is one candidate from the ray's start record.
//
// Two arithmetic forms of the exit search (Sect. 2.2, steps 1-3, Eq. 1-5):
//  * float64: Eq. 4 and Eq. 5 evaluated as written, in the same operation
//    order as a plain C implementation with contraction disabled, the
//    current point updated as r <- r + s k.
//  * float32 with recheck: each plane test runs in float32 in the frame of
//    the current site, together with a rigorous bound on its rounding error.
//    The exit is accepted when the upper bound of the winner lies below the
//    lower bound of every other candidate; otherwise that one crossing is
//    recomputed with the float64 form. The ray parameter t is kept as an
//    unevaluated float pair, so no float64 work is needed per crossing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fsplit.h"
#include "internal.h"
#include "kernels.h"
#include "vgrid.h"

namespace vg {

enum { RAY_OK = 0, RAY_OUTSIDE = 1, RAY_STEP_LIMIT = 2, RAY_BAD_DIR = 3 };

constexpr int kNone = 0x7fffffff;                   // "no candidate"
constexpr float kU = 5.9604644775390625e-8f;        // 2^-24, unit roundoff of float32
constexpr float kU2 = 3.552713678800501e-15f;       // 2^-48
constexpr float kCDen = 6.0f * kU;                  // |den~ - den| <= kCDen |n~|_1
constexpr float kCA = 4.0f * kU;                    // |num~ - num| <= |n|_1 (kCA |n|_1 + kCB |r|_1 + 2 e_r)
constexpr float kCB = 8.0f * kU;
constexpr float kDivLo = 0.99999952316284180f;      // 1 - 2^-21: covers 2 ulp of __fdividef
constexpr float kDivHi = 1.00000047683715820f;      // 1 + 2^-21
// __fdividef's 2-ulp bound holds for divisors in [2^-126, 2^126]; above,
// it returns 0 (a valid lower bound, not an upper one). An accepted winner
// has its divisor below 2^125, so that the length divided out of it (by the
// rounded denominator, at most the upper divisor plus twice its error term)
// is in range too.
constexpr float kDivMin = 0x1p-126f;
constexpr float kDivMax = 0x1p125f;


// ---------------------------------------------------------------------------
// float pairs (value = hi + lo)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (hi, lo) += x
__device__ __forceinline__ void ff_add(float &hi, float &lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    e = __fadd_rn(e, lo);
    fast_two_sum(s, e, hi, lo);
}

__device__ __forceinline__ void split_double(double x, float &hi, float &lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(__dsub_rn(x, (double)hi));
}

// The same split with integer operations where they cover x (nearly always)
__device__ __forceinline__ void split_pair(double x, float &hi, float &lo) {
    if (!split_double_int(x, hi, lo)) split_double(x, hi, lo);
}

__device__ __forceinline__ void ff_add_double(float &hi, float &lo, double x) {
    float xh, xl, s, e;
    split_double(x, xh, xl);
    two_sum(hi, xh, s, e);
    e = __fadd_rn(__fadd_rn(e, lo), xl);
    fast_two_sum(s, e, hi, lo);
}

// r = (R0 + t K) - p along one axis, to within 2u|r| + 16 u^2 (|R0| + t + |p|):
// R0_hi - p and t_hi K_hi are formed exactly, the small terms added last.
__device__ __forceinline__ float local_coord(float R0h, float R0l, float Kh, float Kl, float th, float tl, float p) {
    float ah, al;
    two_sum(R0h, -p, ah, al);
    const float bh = __fmul_rn(th, Kh);
    const float bl = __fmaf_rn(th, Kh, -bh);
    float small = __fmaf_rn(th, Kl, R0l);
    small = __fmaf_rn(tl, Kh, small);
    small = __fadd_rn(small, __fadd_rn(al, bl));
    return __fadd_rn(__fadd_rn(ah, bh), small);
}

// a b = p + e exactly (fused multiply-add)
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// (hi, lo) += (xh, xl)
__device__ __forceinline__ void ff_add2(float &hi, float &lo, float xh, float xl) {
    float s, e;
    two_sum(hi, xh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, xl));
    fast_two_sum(s, e, hi, lo);
}

// The length of a crossing through the bisector of the current site p and
// the winner's site q (Eq. 4), for the float32 form with exact lengths:
// n = q - p exactly as float pairs (both are float32 values), r = (R0 + t K)
// - p, w = n/2 - r and the dot products n.w and n.k in float-pair
// arithmetic, then one corrected division. The result is within a few u of
// the exact length unless n.w cancels to a few u^2 |n||w| (a step that
// starts on the plane), where it is within that absolute amount.
__device__ __forceinline__ void exact_length(float4 q, float px, float py, float pz, const float *R0h,
                                             const float *R0l, const float *Kh, const float *Kl, float th, float tl,
                                             float &len_h, float &len_l) {
    const float qc[3] = {q.x, q.y, q.z}, pc[3] = {px, py, pz};
    float numh = 0.f, numl = 0.f, denh = 0.f, denl = 0.f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float nh, nl;
        two_sum(qc[c], -pc[c], nh, nl);                    // n = q - p, exact
        float ah, al, bh, bl, sh, se;
        two_sum(R0h[c], -pc[c], ah, al);                   // R0_hi - p, exact
        two_prod(th, Kh[c], bh, bl);                       // t_hi K_hi, exact
        two_sum(ah, bh, sh, se);
        const float small = __fadd_rn(__fadd_rn(__fadd_rn(al, bl), R0l[c]),
                                      __fmaf_rn(th, Kl[c], __fmul_rn(tl, Kh[c])));
        float rh, rl;
        fast_two_sum(sh, __fadd_rn(se, small), rh, rl);    // r
        float wh, we;
        two_sum(__fmul_rn(0.5f, nh), -rh, wh, we);          // w = n/2 - r
        float wl;
        fast_two_sum(wh, __fadd_rn(we, __fsub_rn(__fmul_rn(0.5f, nl), rl)), wh, wl);
        float ph, pe;
        two_prod(nh, wh, ph, pe);                          // n.w term
        pe = __fadd_rn(pe, __fmaf_rn(nh, wl, __fmul_rn(nl, wh)));
        ff_add2(numh, numl, ph, pe);
        two_prod(nh, Kh[c], ph, pe);                       // n.k term
        pe = __fadd_rn(pe, __fmaf_rn(nh, Kl[c], __fmul_rn(nl, Kh[c])));
        ff_add2(denh, denl, ph, pe);
    }
    const float q1 = __fdiv_rn(numh, denh);
    float rem = __fmaf_rn(-q1, denh, numh);
    rem = __fadd_rn(rem, __fmaf_rn(-q1, denl, numl));
    fast_two_sum(q1, __fdiv_rn(rem, denh), len_h, len_l);
    if (!(len_h > 0.0f)) {
        len_h = 0.0f;
        len_l = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// cell blocks
// ---------------------------------------------------------------------------

struct Hot {
    const float4 *__restrict__ cells;  // absolute cell blocks (float64 form, rechecks)
    const float4 *__restrict__ rel;    // relative cell blocks (float32 form)
    const float4 *__restrict__ site;   // (x, y, z, bits of the relative block offset) per internal cell
};

__device__ __forceinline__ int rec_w(float4 q) { return __float_as_int(q.w); }

// Two consecutive float4 in one 256-bit load (p 32-byte aligned). The lanes of
// a warp read unrelated blocks, so every lane touches its own 32-byte sector:
// one request per sector instead of one per half sector. The data is used
// once by the lane that reads it and almost never found in L1 again (the
// blocks the resident warps read exceed it), so it is not kept there.
__device__ __forceinline__ void ldg_pair(const float4 *p, float4 &a, float4 &b) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}
__device__ __forceinline__ int hdr_caller(float4 h) { return __float_as_int(h.x); }
__device__ __forceinline__ int hdr_count(float4 h) { return __float_as_int(h.y); }

// ---------------------------------------------------------------------------
// float64 exit search (Eq. 4, Eq. 5), lexicographic (s, id) minimum; walls
// keep their negative ids, cells compare by the caller's index on exact ties
// ---------------------------------------------------------------------------

// tie-break key of a record: the wall id, or the caller's id of the cell
__device__ __forceinline__ int key64(const Hot &h, int w) {
    return w < 0 ? w : hdr_caller(__ldg(&h.cells[w]));
}

// FRAC: candidates are compared as fractions s = num / den with den > 0,
// num_a den_b < num_b den_a, two products instead of a division per
// candidate; only the winner's s is divided out, with the same operations
// as the oracle's, so its length is bit-identical. The products round where
// the quotients would, so the choice can differ from a comparison of
// rounded quotients only between candidates whose quotients agree to about
// one ulp (near ties, where either exit is correct to that precision). The
// float64 form uses it; the float32 form's recheck, rare and inlined into a
// kernel whose occupancy is set by its registers, divides per candidate
// (n holds s there and d is unused).
template <bool FRAC>
__device__ __forceinline__ bool better64(const Hot &h, double n, double d, int w, double bn, double bd, int bw,
                                         bool have) {
    if (!have) return true;
    const double l = FRAC ? __dmul_rn(n, bd) : n, r = FRAC ? __dmul_rn(bn, d) : bn;
    if (l < r) return true;
    if (l > r) return false;
    return key64(h, w) < key64(h, bw);
}

// A spherical domain (the ball sph = centre, R inside the box): a point is
// inside when ((dx dx + dy dy) + dz dz) <= R R, and the path leaves it at the
// larger root s of s^2 + 2 b s + q = 0, b = k.o, q = o.o - R^2, o = r - c (k a
// unit vector): -q / (b + sqrt(b^2 - q)) for b > 0, so that no digits cancel,
// else sqrt(b^2 - q) - b; every operation rounded to nearest, in this order.
constexpr int kSphereWall = -7;         // its wall id
constexpr int kSphereWin = 0x40000000;  // exit64's result when the sphere is the exit

__device__ __forceinline__ bool in_sphere(const GridDev *gp, const double *x) {
    const double dx = __dsub_rn(x[0], gp->sph[0]), dy = __dsub_rn(x[1], gp->sph[1]), dz = __dsub_rn(x[2], gp->sph[2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 <= __dmul_rn(gp->sph[3], gp->sph[3]);
}

__device__ __forceinline__ double sphere_exit64(const GridDev *gp, const double *r, const double *k) {
    double o[3];
    for (int c = 0; c < 3; c++) o[c] = __dsub_rn(r[c], gp->sph[c]);
    const double b = __dadd_rn(__dadd_rn(__dmul_rn(k[0], o[0]), __dmul_rn(k[1], o[1])), __dmul_rn(k[2], o[2]));
    const double q = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(o[0], o[0]), __dmul_rn(o[1], o[1])), __dmul_rn(o[2], o[2])),
                               __dmul_rn(gp->sph[3], gp->sph[3]));
    double disc = __dsub_rn(__dmul_rn(b, b), q);
    if (disc < 0.0) disc = 0.0;
    const double sq = __dsqrt_rn(disc);
    const double s = b > 0.0 ? __ddiv_rn(-q, __dadd_rn(b, sq)) : __dsub_rn(sq, b);
    return s < 0.0 ? 0.0 : s;
}

// A wall (Eq. 5) as the fraction num / den; false unless the ray faces it.
// In a spherical domain the box's walls are not part of the boundary.
__device__ __forceinline__ bool wall64(const GridDev *gp, int w, const double *r, const double *k, double &num,
                                      double &den) {
    if (w < -6 || gp->domain == VGRID_DOMAIN_SPHERE) return false;
    const int wi = -w - 1, axis = wi >> 1, hi = wi & 1;
    const double kc = k[axis];
    if (hi ? !(kc > 0.0) : !(kc < 0.0)) return false;
    // (bound - r) / k as a fraction with a positive denominator: the
    // negated difference is the exact negation of the rounded one
    const double bound = hi ? gp->hi[axis] : gp->lo[axis];
    const double v = hi ? __dsub_rn(bound, r[axis]) : __dsub_rn(r[axis], bound);
    num = v < 0.0 ? 0.0 : v;
    den = fabs(kc);
    return true;
}

// One record: bisector of the current site and the record's site (Eq. 1-4),
// or a wall (Eq. 5), as the fraction num / den (num >= 0, den > 0). Returns
// false if it is not a candidate (n.k <= 0).
__device__ __forceinline__ bool plane64(const GridDev *gp, float4 q, double pmx, double pmy, double pmz,
                                        const double *r, const double *k, double &num, double &den) {
    const int w = rec_w(q);
    if (w >= 0) {
        const double px = (double)q.x, py = (double)q.y, pz = (double)q.z;
        const double nx = __dsub_rn(px, pmx), ny = __dsub_rn(py, pmy), nz = __dsub_rn(pz, pmz);
        den = __dadd_rn(__dadd_rn(__dmul_rn(nx, k[0]), __dmul_rn(ny, k[1])), __dmul_rn(nz, k[2]));
        if (!(den > 0.0)) return false;
        const double wx = __dsub_rn(__dmul_rn(__dadd_rn(px, pmx), 0.5), r[0]);
        const double wy = __dsub_rn(__dmul_rn(__dadd_rn(py, pmy), 0.5), r[1]);
        const double wz = __dsub_rn(__dmul_rn(__dadd_rn(pz, pmz), 0.5), r[2]);
        num = __dadd_rn(__dadd_rn(__dmul_rn(nx, wx), __dmul_rn(ny, wy)), __dmul_rn(nz, wz));
        if (num < 0.0) num = 0.0;
        return true;
    }
    return wall64(gp, w, r, k, num, den);
}

// float64 form, one record of the table of exact differences (see
// GridDev::rec64): the same num and den as plane64 on the float record, with
// fewer float64 operations. n = p_j - p_m is stored, and fma(0.5, n, p_m)
// is (p_j + p_m) / 2 exactly, the value plane64 gets by rounding the sum and
// halving it, because the table holds only records whose sum and difference
// are exact; the flagged others go through plane64.
__device__ __forceinline__ bool plane64x(const GridDev *gp, const float4 *crec, float4 xa, float4 xb, double pmx,
                                         double pmy, double pmz, const double *r, const double *k, double &num,
                                         double &den) {
    const int w = __float_as_int(xb.z);
    if (w < 0) return wall64(gp, w, r, k, num, den);
    if (__float_as_int(xb.w) != 0) return plane64(gp, __ldg(crec), pmx, pmy, pmz, r, k, num, den);
    const double nx = __hiloint2double(__float_as_int(xa.y), __float_as_int(xa.x));
    const double ny = __hiloint2double(__float_as_int(xa.w), __float_as_int(xa.z));
    const double nz = __hiloint2double(__float_as_int(xb.y), __float_as_int(xb.x));
    den = __dadd_rn(__dadd_rn(__dmul_rn(nx, k[0]), __dmul_rn(ny, k[1])), __dmul_rn(nz, k[2]));
    if (!(den > 0.0)) return false;
    const double wx = __dsub_rn(__fma_rn(0.5, nx, pmx), r[0]);
    const double wy = __dsub_rn(__fma_rn(0.5, ny, pmy), r[1]);
    const double wz = __dsub_rn(__fma_rn(0.5, nz, pmz), r[2]);
    num = __dadd_rn(__dadd_rn(__dmul_rn(nx, wx), __dmul_rn(ny, wy)), __dmul_rn(nz, wz));
    if (num < 0.0) num = 0.0;
    return true;
}

// Exit of the cell whose records are blk[1..cnt] for the group: the
// lexicographically smallest (s, id); returns the winner's record position
// (1-based), kSphereWin if the exit is a spherical domain's boundary, or 0 if
// there is no candidate, and its s in bs.
// The float64 form's pre-test: false only for a record whose plane
// certainly faces away (n.k <= 0), so that the float64 test can skip it; the
// results are the same bits. The stored n's high words are truncated to
// float32 with integer operations only (21 significant bits, relative error
// below 2^-20; components below 2^-126 become 0) and dotted with k in
// float32. The error against the exact n.k is at most ||n~||_1 (2^-20 +
// 4.1 2^-24) + 3 2^-126; the bound b below is more than three times that,
// so d <= -b leaves n.k < 0 by a margin far above float64's rounding. Walls
// and flagged records always pass.
__device__ __forceinline__ float hi_to_float(int h) {
    const int e = (h >> 20) & 0x7ff;
    const int bits = (h & (int)0x80000000) | ((e - 896) << 23) | ((h & 0xfffff) << 3);
    return e > 896 ? __int_as_float(bits) : 0.0f;
}

__device__ __forceinline__ bool may_face64(float4 xa, float4 xb, const float *kf) {
    if (__float_as_int(xb.z) < 0 || __float_as_int(xb.w) != 0) return true;
    const float nx = hi_to_float(__float_as_int(xa.y));
    const float ny = hi_to_float(__float_as_int(xa.w));
    const float nz = hi_to_float(__float_as_int(xb.y));
    const float d = __fmaf_rn(nz, kf[2], __fmaf_rn(ny, kf[1], __fmul_rn(nx, kf[0])));
    const float b = __fmaf_rn(__fadd_rn(__fadd_rn(fabsf(nx), fabsf(ny)), fabsf(nz)), 0x1p-18f, 0x1p-120f);
    return d > -b;
}

// FRAC (the float64 form) reads the records from x64, the block's entries
// of the table of exact differences (two float4 per entry), and blk only for
// flagged records; otherwise it reads the float records of blk.
template <int LPR, bool FRAC>
__device__ __forceinline__ int exit64(const Hot &h, const GridDev *gp, const float4 *blk, const float4 *x64, int cnt,
                                      double pmx, double pmy, double pmz, const double *r, const double *k,
                                      const float *kf, unsigned gmask, int gl, double &bs) {
    double bn = 0.0, bd = 1.0;
    int bp = 0, bw = 0;
    if (FRAC) {
        // A warp issues a float64 instruction for all its lanes if any needs
        // it, so a lane first marks which of its records may face ahead
        // (float32 pre-test, up to 32 at a time) and then runs the float64
        // test over those alone: the warp's float64 work follows the lane
        // with the most candidates, not the one with the most records.
        for (int base = 1 + gl; base <= cnt; base += 32 * LPR) {
            unsigned m = 0;
            for (int i = 0; i < 32; i++) {
                const int p = base + i * LPR;
                if (p > cnt) break;
                float4 xa, xb;
                ldg_pair(x64 + 2 * p, xa, xb);  // 32-byte entries
                if (may_face64(xa, xb, kf)) m |= 1u << i;
            }
            while (m) {
                const int p = base + (__ffs(m) - 1) * LPR;
                m &= m - 1;
                float4 xa, xb;
                ldg_pair(x64 + 2 * p, xa, xb);
                double n, d;
                if (plane64x(gp, blk + p, xa, xb, pmx, pmy, pmz, r, k, n, d)) {
                    const int w = __float_as_int(xb.z);
                    if (better64<true>(h, n, d, w, bn, bd, bw, bp != 0)) {
                        bn = n;
                        bd = d;
                        bp = p;
                        bw = w;
                    }
                }
            }
        }
    }
    // the float32 form's recheck: every record of blk, s divided out
    for (int p = 1 + gl; !FRAC && p <= cnt; p += LPR) {
        const float4 q = __ldg(blk + p);
        double n, d;
        if (plane64(gp, q, pmx, pmy, pmz, r, k, n, d)) {
            n = __ddiv_rn(n, d);
            if (better64<false>(h, n, d, rec_w(q), bn, bd, bw, bp != 0)) {
                bn = n;
                bp = p;
                bw = rec_w(q);
            }
        }
    }
    // a spherical domain: its exit from r is one more candidate (s / 1)
    if (gp->domain == VGRID_DOMAIN_SPHERE) {
        const double s = sphere_exit64(gp, r, k);
        if (better64<FRAC>(h, s, 1.0, kSphereWall, bn, bd, bw, bp != 0)) {
            bn = s;
            bd = 1.0;
            bp = kSphereWin;
            bw = kSphereWall;
        }
    }
#pragma unroll
    for (int o = 1; o < LPR; o <<= 1) {
        const double on = __shfl_xor_sync(gmask, bn, o);
        const double od = FRAC ? __shfl_xor_sync(gmask, bd, o) : 1.0;
        const int op = __shfl_xor_sync(gmask, bp, o);
        const int ow = __shfl_xor_sync(gmask, bw, o);
        if (op != 0 && better64<FRAC>(h, on, od, ow, bn, bd, bw, bp != 0)) {
            bn = on;
            if (FRAC) bd = od;
            bp = op;
            bw = ow;
        }
    }
    bs = bp == 0 ? 0.0 : (FRAC ? __ddiv_rn(bn, bd) : bn);
    return bp;
}

// ---------------------------------------------------------------------------
// C(r): nearest site among the candidates of r's block (Sect. 2.3)
// ---------------------------------------------------------------------------

// A query point: float64 coordinates and their float pairs.
struct LocPt {
    double x[3];
    float h[3], l[3];
};

__device__ __forceinline__ LocPt loc_point(double x, double y, double z) {
    LocPt P;
    P.x[0] = x;
    P.x[1] = y;
    P.x[2] = z;
    for (int c = 0; c < 3; c++) split_pair(P.x[c], P.h[c], P.l[c]);
    return P;
}

// Closed box test, exact (integer order keys of the float64 values)
__device__ __forceinline__ bool inside(const GridDev *gp, const LocPt &P) {
    bool in = true;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int64_t k = dkey(P.x[c]);
        in = in && !disnan(P.x[c]) && k >= gp->lokey[c] && k <= gp->hikey[c];
    }
    return in && (gp->domain != VGRID_DOMAIN_SPHERE || in_sphere(gp, P.x));
}

// Block of the point, from its float pairs: (x - lo) is formed to within
// 2u|x - lo| + 4u^2 max|coordinate|, so the index may be off only for points
// closer to a block face than the padding of the block lists, and those
// lists name every cell within that padding.
__device__ __forceinline__ int block_of(const GridDev *gp, const LocPt &P, int *i) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float d = __fadd_rn(__fsub_rn(P.h[c], gp->flo_hi[c]), __fsub_rn(P.l[c], gp->flo_lo[c]));
        i[c] = max(0, min(__float2int_rz(__fmul_rn(d, gp->fbscale[c])), gp->bdim[c] - 1));
    }
    return (i[0] * gp->bdim[1] + i[1]) * gp->bdim[2] + i[2];
}

// float64 scan of a block list, distances as ((dx dx + dy dy) + dz dz)
static __device__ __noinline__ int locate64(const GridDev *gp, double x, double y, double z, int beg, int end) {
    const float4 *rec = gp->blk_rec;
    const int32_t *perm = gp->perm;
    int best = -1;
    double bd = 0.0;
    for (int i = beg; i < end; i++) {
        const float4 q = __ldg(&rec[i]);
        const int c = __float_as_int(q.w);
        if (c < 0) continue;  // padding
        const double dx = __dsub_rn(x, (double)q.x), dy = __dsub_rn(y, (double)q.y), dz = __dsub_rn(z, (double)q.z);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (best < 0 || d2 < bd || (d2 == bd && __ldg(&perm[c]) < __ldg(&perm[best]))) {
            bd = d2;
            best = c;
        }
    }
    return best;
}

// Nearest site (internal id), -1 outside the closed box. With fp32 the
// squared distances are float32 and the winner is accepted when
// D2 - E(D2) > D1 + E(D1), E(D) = u (10 D + 4 X sqrt D), X = max |x_c|,
// which bounds the rounding error of a float32 squared distance; otherwise
// the list is rescanned in float64. *rechecked is set when that happened.
// A block's list is ordered by the sites' distance from the block's centre
// c, so the float32 scan can stop early: a site not scanned yet is at least
// as far from c as the last one scanned, s, hence at least |s - c| - |p - c|
// from the point p (triangle inequality). That bound, rounded down with
// margins for the float32 distances (16u relative) and for p's low words
// (4uX), stops the scan once its square exceeds D1, and takes the place of
// D2 when smaller, so the acceptance test above stays rigorous.
// Block lists start on 32-byte boundaries and have an even length (NaN
// records pad them; a NaN distance never wins), so they can be read in pairs
// (PAIRS; the traversal kernel's rare relocation reads them one by one).
template <bool PAIRS>
static __device__ __noinline__ int locate_point(const GridDev *gp, const LocPt P, bool fp32, int *rechecked) {
    if (!inside(gp, P)) return -1;
    int bi[3];
    const int b = block_of(gp, P, bi);
    const int beg = __ldg(&gp->blk_off[b]), end = __ldg(&gp->blk_off[b + 1]);
    if (fp32) {
        const float4 *rec = gp->blk_rec;
        const float xf = P.h[0], yf = P.h[1], zf = P.h[2];
        const float X = fmaxf(fabsf(xf), fmaxf(fabsf(yf), fabsf(zf)));
        float D1 = __int_as_float(0x7f800000), D2 = D1;
        int i1 = -1;
        float cc[3];
#pragma unroll
        for (int c = 0; c < 3; c++)
            cc[c] = __fadd_rn(gp->flo_hi[c], __fmul_rn(__fadd_rn((float)bi[c], 0.5f), gp->fbw[c]));
        float rp;
        {
            const float ex = __fsub_rn(xf, cc[0]), ey = __fsub_rn(yf, cc[1]), ez = __fsub_rn(zf, cc[2]);
            rp = __fsqrt_rn(__fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex))));
        }
        // |p - c| rounded up, plus p's low words: subtracted from the bound
        const float slack = __fadd_ru(__fmul_ru(rp, 1.0f + 16.0f * kU), __fmul_ru(4.0f * kU, X));
        for (int i = beg; i < end; i += 2) {
            float4 q[2];
            if (PAIRS) {
                ldg_pair(rec + i, q[0], q[1]);
            } else {
                q[0] = __ldg(rec + i);
                q[1] = __ldg(rec + i + 1);
            }
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const float dx = __fsub_rn(xf, q[u].x), dy = __fsub_rn(yf, q[u].y), dz = __fsub_rn(zf, q[u].z);
                const float D = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                const bool better = D < D1;
                D2 = better ? D1 : fminf(D2, D);
                i1 = better ? __float_as_int(q[u].w) : i1;
                D1 = fminf(D1, D);
            }
            // the rest of the list is at least lb from p (NaN padding: no stop)
            const float ex = __fsub_rn(q[1].x, cc[0]), ey = __fsub_rn(q[1].y, cc[1]), ez = __fsub_rn(q[1].z, cc[2]);
            const float dl = __fsqrt_rn(__fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex))));
            const float lb = __fsub_rd(__fmul_rd(dl, 1.0f - 16.0f * kU), slack);
            if (lb > 0.0f) {
                const float lb2 = __fmul_rd(lb, lb);
                if (lb2 > D1) {
                    D2 = fminf(D2, lb2);
                    break;
                }
            }
        }
        if (i1 >= 0 && D2 == __int_as_float(0x7f800000)) return i1;  // a single candidate
        const float s1 = sqrtf(D1), s2 = sqrtf(D2);
        const float E1 = 1.0001f * kU * __fmaf_rn(10.0f, D1, 4.0f * X * s1);
        const float E2 = 1.0001f * kU * __fmaf_rn(10.0f, D2, 4.0f * X * s2);
        if (i1 >= 0 && s2 > 8.0f * kU * X && __fsub_rd(D2, E2) > __fadd_ru(D1, E1)) return i1;
        if (rechecked) *rechecked = 1;
    }
    return locate64(gp, P.x[0], P.x[1], P.x[2], beg, end);
}

// ---------------------------------------------------------------------------
// float32 exit search with error bounds (one group)
// ---------------------------------------------------------------------------

struct Cand32 {
    float L1, L2;        // smallest and second smallest lower bound
    int p1;              // record position (1-based) of the smallest, 0 if none
    // one lane per ray: the smallest's plane terms and neighbour offset, kept
    // so that the winner's record is not read again
    float num1, den1;
    int w1;
};

// Terms of the bisector of the current site p (origin of the local frame)
// and a neighbour's site q, from the record's n~ = fl(q - p) (rounded once,
// on the host, exactly as a float32 subtraction here would), with their
// rounding-error bounds (u = 2^-24, r~ within 2u|r| + e_r, N = the cell's
// bound on |n~|_1 from its header):
//   |den~ - n.k|  <= dden = 6u N                    (the rounding of n, three of the dot, K)
//   |num~ - n.w|  <= dnum = N (4u N + 8u |r~|_1 + 2 e_r),   w = n/2 - r
// dden and dnum are the same for every plane of the cell (computed once per
// crossing from N).
struct Plane32 {
    float num, den, dnum, dden;
};

__device__ __forceinline__ Plane32 plane32(float4 q, float rx, float ry, float rz, float dnum, float dden, float Kx,
                                           float Ky, float Kz) {
    Plane32 p;
    const float nx = q.x, ny = q.y, nz = q.z;
    p.den = __fmaf_rn(nz, Kz, __fmaf_rn(ny, Ky, __fmul_rn(nx, Kx)));
    p.dden = dden;
    const float wx = __fmaf_rn(0.5f, nx, -rx), wy = __fmaf_rn(0.5f, ny, -ry), wz = __fmaf_rn(0.5f, nz, -rz);
    p.num = __fmaf_rn(nz, wz, __fmaf_rn(ny, wy, __fmul_rn(nx, wx)));
    p.dnum = dnum;
    return p;
}

// dden carries 2^-126 on top of the rounding bound of den~ (added once per
// crossing), so den_hi = den~ + dden rounded up exceeds 2^-126 for every
// plane that may face ahead: the test den_hi > 2^-126 masks only planes with
// n.k <= 0 (R2), and the NaN records that pad a block (for which it is
// false), and every plane it keeps divides by a normal number, where the
// division's error bound holds. Those planes get the lower bound
// a / den_hi on s (Eq. 4), a = max((num~ - dnum) kDivLo, 0) rounded down in
// one fused multiply-add (dnumK = dnum kDivLo rounded up, once per
// crossing): the factor kDivLo = 1 - 2^-21 taken out of the numerator covers
// the division's 2 ulp (2^-22 relative), so the quotient stays below
// (num~ - dnum) / den_hi (above 2^126 the division returns 0, still a lower
// bound). Branch-free: in a warp some lane nearly always has
// a plane facing ahead, so skipping the numerator for planes facing away (the
// sign shortcut of Sect. 2.2) would only add divergence; a masked result
// costs nothing more. Positions past the count (several lanes per ray) are
// masked by `valid`.
template <bool KEEP>
__device__ __forceinline__ void consider32(int pos, bool valid, float4 q, float rx, float ry, float rz, float dnumK,
                                           float dden, float Kx, float Ky, float Kz, Cand32 &c) {
    const Plane32 p = plane32(q, rx, ry, rz, dnumK, dden, Kx, Ky, Kz);
    const float num_lo = fmaxf(__fmaf_rd(p.num, kDivLo, -dnumK), 0.0f);
    const float den_hi = __fadd_ru(p.den, p.dden);
    float lower;
    if (KEEP) {
        // one lane per ray (every position valid): the divisor clamped at 0
        // masks a plane certainly facing away (den_hi <= 0 and the NaN
        // padding: a / 0 = +inf, 0 / 0 = NaN, and a NaN loses every
        // comparison and min below); 0 < den_hi <= 2^-126 means den~ < 0,
        // a plane facing away too, whatever value it gets can only lower
        // L2 or win without an upper bound (den_lo < 0), which sends the
        // crossing to the float64 recheck
        lower = __fdividef(num_lo, fmaxf(den_hi, 0.0f));
    } else {
        lower = __fdividef(num_lo, den_hi);
        lower = (valid && den_hi > kDivMin) ? lower : __int_as_float(0x7f800000);
    }
    const bool b = lower < c.L1;
    c.L2 = b ? c.L1 : fminf(c.L2, lower);
    if (KEEP) {
        c.num1 = b ? p.num : c.num1;
        c.den1 = b ? p.den : c.den1;
        c.w1 = b ? rec_w(q) : c.w1;
    } else {
        c.p1 = b ? pos : c.p1;
    }
    c.L1 = fminf(c.L1, lower);
}

// Records recs[1..cnt] (cnt even, at least four); lane gl of
// the group takes records gl+1, gl+1+LPR, ... four at a time. With one lane
// per ray the caller loads the first four (f0..f3) together with the header,
// so they do not wait for the count, and no position is ever past the count.
template <int LPR>
__device__ __forceinline__ void exit32(const float4 *recs, int cnt, float4 f0, float4 f1, float4 f2, float4 f3,
                                       float rx, float ry, float rz, float dnumK, float dden, float Kx, float Ky,
                                       float Kz, unsigned gmask, int gl, int gbase, Cand32 &c) {
    c.L1 = __int_as_float(0x7f800000);
    c.L2 = c.L1;
    c.p1 = 0;
    c.num1 = 0.f;
    c.den1 = 1.f;
    c.w1 = 0;
    if (LPR == 1) {
        consider32<true>(1, true, f0, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
        consider32<true>(2, true, f1, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
        consider32<true>(3, true, f2, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
        consider32<true>(4, true, f3, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
        const float nan = __int_as_float(0x7fc00000);
        for (int p = 5; p <= cnt; p += 4) {
            // the last group may hold one pair: the other reads as NaN records
            float4 q0, q1, q2 = make_float4(nan, nan, nan, nan), q3 = q2;
            ldg_pair(recs + p, q0, q1);
            if (p + 2 <= cnt) ldg_pair(recs + p + 2, q2, q3);
            consider32<true>(p, true, q0, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
            consider32<true>(p + 1, true, q1, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
            consider32<true>(p + 2, true, q2, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
            consider32<true>(p + 3, true, q3, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
        }
    } else {
        const float nan = __int_as_float(0x7fc00000);
        const float4 pad = make_float4(nan, nan, nan, __int_as_float(-8));
        for (int p = 1 + gl; p <= cnt; p += 4 * LPR) {
            const int p0 = p, p1 = p + LPR, p2 = p + 2 * LPR, p3 = p + 3 * LPR;
            const float4 q0 = __ldg(recs + p0);
            const float4 q1 = p1 <= cnt ? __ldg(recs + p1) : pad;
            const float4 q2 = p2 <= cnt ? __ldg(recs + p2) : pad;
            const float4 q3 = p3 <= cnt ? __ldg(recs + p3) : pad;
            consider32<false>(p0, true, q0, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
            consider32<false>(p1, p1 <= cnt, q1, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
            consider32<false>(p2, p2 <= cnt, q2, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
            consider32<false>(p3, p3 <= cnt, q3, rx, ry, rz, dnumK, dden, Kx, Ky, Kz, c);
        }
    }
    if (LPR > 1) {
        int win = gl;
#pragma unroll
        for (int o = 1; o < LPR; o <<= 1) {
            const float oL1 = __shfl_xor_sync(gmask, c.L1, o);
            const float oL2 = __shfl_xor_sync(gmask, c.L2, o);
            const int ow = __shfl_xor_sync(gmask, win, o);
            const float nL2 = fminf(fmaxf(c.L1, oL1), fminf(c.L2, oL2));
            if (oL1 < c.L1 || (oL1 == c.L1 && ow < win)) {
                c.L1 = oL1;
                win = ow;
            }
            c.L2 = nL2;
        }
        c.p1 = __shfl_sync(gmask, c.p1, gbase + win);
    }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------

__device__ __forceinline__ int find_set(const RaySetDev *sets, int nsets, int64_t w) {
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&sets[mid].first) <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// BATCH = false: one grid, read from the parameter space (a.g1, a.s1);
// BATCH = true: many grids and ray sets, looked up per ray.
// Register caps of the float32 traversals: the kernel is bound by the L1
// data pipe and load latency, and the warps it keeps in flight set how much
// of that latency is hidden, so each instance is held to the largest count
// that still gives it one more block of 128 threads per SM: 72 (seven
// blocks) for tau, the adjoint and interaction sampling, 80 (six) for
// segment lists (both forms) and the batch. The float64 tau traversal, bound
// by the FP64 pipe, is left alone (80 registers; held to 72 it was slower).
// The per-ray values that a crossing of the float32 form reads once live in
// shared memory, which is what lets the float32 instances fit.
template <bool FP64, int MODE, bool BATCH, bool XL>
constexpr int trace_max_regs() {
    return FP64 ? (MODE == MODE_SEGS ? 80 : 255) : (BATCH || MODE == MODE_SEGS || XL) ? 80 : 72;
}

// XL: the float32 form with exact lengths (one lane per ray): decisions as
// in the float32 form, each crossing's length from exact_length.
template <int LPR, bool FP64, int MODE, bool BATCH, bool XL = false>
__global__ void __launch_bounds__(256) __maxnreg__((trace_max_regs<FP64, MODE, BATCH, XL>())) trace_kernel(TraceArgs a) {
    static_assert(LPR == 1 || LPR == 2 || LPR == 4 || LPR == 8, "lanes per ray");
    static_assert(!XL || (LPR == 1 && !FP64 && !BATCH), "exact lengths: float32 form, one lane per ray");
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LPR - 1);
    const int gbase = lane & ~(LPR - 1);
    const unsigned gmask = ((1u << LPR) - 1u) << gbase;

    // statistics: block counters in shared memory, updated by group leaders
    // once per ray and on rare events, added to the global counters at exit
    __shared__ unsigned long long s_stats[9];
    if (threadIdx.x < 9) s_stats[threadIdx.x] = 0ull;
    __syncthreads();
    enum { S_RAYS, S_CROSS, S_DEC, S_RE, S_FB, S_ZERO, S_LIM, S_OUT, S_BAD };
#define VG_STAT(i, v) atomicAdd(&s_stats[i], (unsigned long long)(v))

    int64_t ray = -1;       // global work index; -1 wants a ray, -2 finished
    int set = 0;
    int64_t li = 0;         // index within the set
    const GridDev *gp = a.grids;  // device copy of the descriptor (cold paths)
    Hot h{a.g1.cells, a.g1.rel, a.g1.site};
    float kappa = a.g1.kappa;
    int max_steps = (int)min(a.g1.max_steps, (int64_t)0x7fffffff);
    // float64 form: current point and direction (and the direction in
    // float32 for the pre-test of the planes)
    double r64[3] = {0, 0, 0}, k64[3] = {0, 0, 0};
    float kf64[3] = {0.f, 0.f, 0.f};
    // float32 form: origin and direction as float pairs, ray parameter t, wall
    // exit. Only the high words of the direction (used by every plane test)
    // and t stay in registers; the origin pairs, the low words of the
    // direction and the wall distance (read once per crossing) are kept per
    // thread in shared memory, and the error terms are formed from the wall
    // distance when needed.
    float Kh[3];
    float th = 0.f, tl = 0.f;
    __shared__ float s_ray[FP64 ? 1 : 11][FP64 ? 1 : 256];
    const int tix = threadIdx.x;
#define R0h_(c) s_ray[(c)][tix]
#define R0l_(c) s_ray[3 + (c)][tix]
#define Kl_(c) s_ray[6 + (c)][tix]
#define tmh_ s_ray[9][tix]
#define tml_ s_ray[10][tix]
    int B = 0;              // block offset of the current cell
    float pmx = 0.f, pmy = 0.f, pmz = 0.f;
    double tau64 = 0.0;
    float tau32 = 0.f, tauc = 0.f;
    float dLr = 0.f;
    float tint = 0.f, wgt = 1.f, att = 1.f;   // interaction mode: tau_int, weight, exp(-tau)
    int nseg = 0, zrun = 0, steps = 0, status = 0;
    // segment mode: the segment of the last step waits in registers until
    // the top of the next iteration, where the warp is converged and takes
    // chunks for its lanes from a shared page [pg, pe)
    using SegLen = typename std::conditional<FP64, double, float>::type;
    bool pend = false;
    int pend_cell = 0, pend_ray = 0;
    SegLen pend_len = 0;
    int cur_chunk = -1;     // chunk of the current ray; -1 none yet, -2 out of chunks
    // the warp's page of chunks [s_page[w][0], s_page[w][1]), kept in shared
    // memory (registers are the scarce resource of this kernel)
    __shared__ int s_page[8][2];
    const int wib = threadIdx.x >> 5;
    if (MODE == MODE_SEGS) {
        if (lane == 0) s_page[wib][0] = s_page[wib][1] = 0;
        __syncwarp();
    }

    for (;;) {
        // ---------------- segment mode: store the last step's segment ----------------
        if (MODE == MODE_SEGS) {
            if (a.chunk_cap > 0) {
                // the pending segment is number j of its ray (nseg is reset
                // only when the next ray starts, further down)
                const int j = nseg - 1;
                const bool want = pend && cur_chunk != -2 && (j & (kSegChunk - 1)) == 0;
                const unsigned wm = __ballot_sync(0xffffffffu, want);
                if (wm) {
                    const int k = __popc(wm);
                    const int rank = __popc(wm & ((1u << lane) - 1u));
                    const int pg = s_page[wib][0], pe = s_page[wib][1];
                    const int left = pe - pg;
                    int base = 0;
                    if (k > left) {
                        // a new page; the cursor may run past the buffer, ids
                        // at or beyond chunk_cap are never stored
                        unsigned long long b = 0;
                        if (lane == 0) b = atomicAdd(a.chunk_cursor, (unsigned long long)kSegPage);
                        b = __shfl_sync(0xffffffffu, b, 0);
                        base = (int)min(b, (unsigned long long)a.chunk_cap);
                    }
                    if (want) {
                        const int nc = rank < left ? pg + rank : base + (rank - left);
                        if (nc < a.chunk_cap) {
                            a.chunk_meta[nc] = make_int2(pend_ray, j / kSegChunk);
                            cur_chunk = nc;
                        } else {
                            cur_chunk = -2;  // the rest of this ray is only counted
                        }
                    }
                    __syncwarp();
                    if (lane == 0) {
                        s_page[wib][0] = k > left ? base + (k - left) : pg + k;
                        if (k > left) s_page[wib][1] = base + kSegPage;
                    }
                    __syncwarp();
                }
                if (pend && cur_chunk >= 0) {
                    const int64_t at = (int64_t)cur_chunk * kSegChunk + (j & (kSegChunk - 1));
                    // streaming stores: the slots are read once, by the
                    // compaction, and should not push the grid out of L2
                    if (FP64) {
                        const double v = (double)pend_len;
                        __stcs(reinterpret_cast<int4 *>(a.seg_slots) + at,
                               make_int4(pend_cell, 0, __double2loint(v), __double2hiint(v)));
                    } else {
                        __stcs(reinterpret_cast<int2 *>(a.seg_slots) + at,
                               make_int2(pend_cell, __float_as_int((float)pend_len)));
                    }
                }
            }
            pend = false;
        }

        // ---------------- fetch new rays (one atomic per warp) ----------------
        const bool need = ray == -1;
        const unsigned needmask = __ballot_sync(0xffffffffu, need && gl == 0);
        if (needmask) {
            const int leader = __ffs(needmask) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(a.queue, (unsigned long long)__popc(needmask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (need) {
                const int rank = __popc(needmask & ((1u << gbase) - 1u));
                const int64_t w = (int64_t)base + rank;
                ray = w < a.total ? (a.order ? (int64_t)__ldg(a.order + w) : w) : -2;
            }
            // only a fetch can leave the warp without work: a lane whose ray
            // ends asks for a new one (ray = -1) before it can finish (-2).
            // The float32 form tests it here, the float64 form after the
            // fetch (its traversal ran 5 % slower with the test here).
            if (!FP64 && !__any_sync(0xffffffffu, ray != -2)) break;
        }
        if (FP64 && !__any_sync(0xffffffffu, ray != -2)) break;

        if (need && ray >= 0) {
            // ---------------- start a ray ----------------
            const RaySetDev *rs = &a.s1;
            li = ray;
            if (BATCH) {
                set = find_set(a.sets, a.nsets, ray);
                rs = &a.sets[set];
                li = ray - rs->first;
                gp = a.grids + rs->grid;
                h.cells = gp->cells;
                h.rel = gp->rel;
                h.site = gp->site;
                kappa = gp->kappa;
                max_steps = (int)min(gp->max_steps, (int64_t)0x7fffffff);
            }
            nseg = 0;
            zrun = 0;
            steps = 0;
            tau64 = 0.0;
            tau32 = 0.f;
            tauc = 0.f;
            th = tl = 0.f;
            if (MODE == MODE_SEGS) cur_chunk = -1;
            if (MODE == MODE_GRAD) dLr = __ldg(&a.dL_dtau[ray]);
            if (MODE == MODE_INTERACT) {
                tint = __ldg(&a.tau_int[ray]);
                wgt = a.weight ? __ldg(&a.weight[ray]) : 1.f;
                att = 1.f;
            }
            // the start record was prepared by the start-cell kernel
            const RayPrep *pr = rs->start + li;
            int m;
            if (FP64) {
                m = pr->cell;
                if (m >= 0) {
                    const double *o = rs->origin + 3 * li;
                    const double *d = rs->dir + 3 * li;
                    for (int c = 0; c < 3; c++) {
                        r64[c] = __ldg(o + c);
                        k64[c] = __ldg(d + c);
                        kf64[c] = __double2float_rn(k64[c]);
                    }
                }
            } else {
                const float4 *p4 = reinterpret_cast<const float4 *>(pr);  // 64-byte aligned
                float4 a0, a1, a2, a3;
                ldg_pair(p4, a0, a1);
                ldg_pair(p4 + 2, a2, a3);
                m = __float_as_int(a0.x);
                tmh_ = a0.z;
                tml_ = a0.w;
                R0h_(0) = a1.x; R0h_(1) = a1.y; R0h_(2) = a1.z;
                R0l_(0) = a1.w; R0l_(1) = a2.x; R0l_(2) = a2.y;
                Kh[0] = a2.z;  Kh[1] = a2.w;  Kh[2] = a3.x;
                Kl_(0) = a3.y;  Kl_(1) = a3.z;  Kl_(2) = a3.w;
            }
            status = m == -2 ? RAY_BAD_DIR : (m < 0 ? RAY_OUTSIDE : RAY_OK);
            if (status == RAY_OK) {
                if (FP64) {
                    const float4 q = __ldg(&h.site[m]);
                    pmx = q.x;
                    pmy = q.y;
                    pmz = q.z;
                    B = rec_w(__ldg(h.rel + rec_w(q) + 1));  // absolute block of the cell
                } else {
                    B = m;  // relative block; the site comes with its header
                }
            }
            if (status != RAY_OK) {
                if (gl == 0) {
                    VG_STAT(S_RAYS, 1);
                    VG_STAT(status == RAY_OUTSIDE ? S_OUT : S_BAD, 1);
                    if (MODE == MODE_TAU || MODE == MODE_SEGS) {
                        if (rs->tau) {
                            if (FP64) ((double *)rs->tau)[li] = 0.0;
                            else ((float *)rs->tau)[li] = 0.f;
                        }
                        if (rs->status) rs->status[li] = status;
                    }
                    if (MODE == MODE_SEGS) a.seg_off[ray] = 0;
                    if (MODE == MODE_INTERACT) {
                        a.int_cell[ray] = -1;
                        a.int_s[ray] = 0.f;
                    }
                }
                ray = -1;
                continue;
            }
        }
        if (ray < 0) continue;

        // ---------------- one exit decision ----------------
        // float64 form: absolute block A (header: caller, count, rho, F);
        // float32 form: relative block F (site and count, then caller, rho,
        // N1max, A).
        const float4 *blk = FP64 ? h.cells + B : h.rel + B;
        float4 hdr, hdr1;
        if (FP64) {
            hdr = __ldg(blk);
            hdr1 = hdr;
        } else {
            ldg_pair(blk, hdr, hdr1);  // relative blocks start on 32-byte boundaries
        }
        const int cnt = FP64 ? hdr_count(hdr) : __float_as_int(hdr.w);
        const int caller = hdr_caller(hdr1);
        const float rho = FP64 ? hdr.z : hdr1.y;
        bool ended = false;
        double s64 = 0.0;      // float64 length (float64 form or recheck)
        bool from64 = FP64;
        float len = 0.f;
        float len_lo = 0.f;    // exact lengths: the low word of the length
        bool found = false;    // an exit was found
        bool to_wall = false;  // ... and it is a wall
        int nextB = 0;         // block offset of the next cell (same form as B)
        float4 qn = make_float4(0.f, 0.f, 0.f, 0.f);  // float64 form: the winner's record
        if (FP64) {
            const int win = exit64<LPR, true>(h, gp, blk, a.g1.rec64 + 2 * (int64_t)B, cnt, (double)pmx, (double)pmy,
                                              (double)pmz, r64, k64, kf64, gmask, gl, s64);
            if (win == kSphereWin) {
                found = true;
                to_wall = true;
            } else if (win > 0) {
                qn = __ldg(blk + win);
                found = true;
                to_wall = rec_w(qn) < 0;
                nextB = rec_w(qn);
            }
        } else {
            const float4 *recs = blk + 1;  // records recs[1..cnt]
            float4 f0{}, f1{}, f2{}, f3{};
            if (LPR == 1) {
                ldg_pair(recs + 1, f0, f1);
                ldg_pair(recs + 3, f2, f3);
            }
            pmx = hdr.x;
            pmy = hdr.y;
            pmz = hdr.z;
            const float rx = local_coord(R0h_(0), R0l_(0), Kh[0], Kl_(0), th, tl, pmx);
            const float ry = local_coord(R0h_(1), R0l_(1), Kh[1], Kl_(1), th, tl, pmy);
            const float rz = local_coord(R0h_(2), R0l_(2), Kh[2], Kl_(2), th, tl, pmz);
            const float r1 = __fadd_rn(__fadd_rn(fabsf(rx), fabsf(ry)), fabsf(rz));
            // the error terms of r and of the wall distance from t_max (no
            // shared-memory reads)
            const float tmax_h = tmh_;
            const float scale = BATCH ? (float)gp->scale : (float)a.g1.scale;
            const float rr = __fmaf_rn(kCB, r1, 2.0f * (16.0f * kU2 * (scale + tmax_h)));
            const float n1m = hdr1.z;  // the cell's bound on |n|_1
            // the rounding bound of den~ plus 2^-126 (see consider32)
            const float dden = __fadd_ru(__fmul_ru(kCDen, n1m), kDivMin);
            const float dnum = __fmul_ru(n1m, __fmaf_ru(kCA, n1m, rr));
            Cand32 c;
            exit32<LPR>(recs, cnt, f0, f1, f2, f3, rx, ry, rz, __fmul_ru(dnum, kDivLo), dden, Kh[0], Kh[1], Kh[2], gmask,
                        gl, gbase, c);
            // the wall ahead is one more candidate: s_w = t_max - t
            float sw, swl;
            two_sum(tmh_, -th, sw, swl);
            sw = __fadd_rn(sw, __fadd_rn(swl, __fsub_rn(tml_, tl)));
            const float Ew = __fmaf_rn(3.0f * kU, fabsf(sw), 16.0f * kU2 * tmax_h);
            const float lw = __fsub_rd(sw, Ew);
            bool wall_wins = false;
            if (lw < c.L1) {
                c.L2 = c.L1;
                c.L1 = lw;
                wall_wins = true;
            } else if (lw < c.L2) {
                c.L2 = lw;
            }
            float upper = __int_as_float(0x7f800000);
            Plane32 w1{0.f, 1.f, 0.f, 0.f};
            float4 qw = make_float4(0.f, 0.f, 0.f, 0.f);
            if (wall_wins) {
                upper = __fadd_ru(sw, Ew);
            } else if (LPR == 1 ? c.L1 < __int_as_float(0x7f800000) : c.p1 > 0) {
                if (LPR == 1) {
                    w1 = Plane32{c.num1, c.den1, dnum, dden};  // kept by the exit search
                    qw.w = __int_as_float(c.w1);
                } else {
                    // the winner's terms again (same operations, same values)
                    qw = __ldg(recs + c.p1);
                    w1 = plane32(qw, rx, ry, rz, dnum, dden, Kh[0], Kh[1], Kh[2]);
                }
                const float den_lo = __fsub_rd(w1.den, w1.dden);
                const float num_hi = fmaxf(__fadd_ru(w1.num, w1.dnum), 0.0f);
                // an upper bound needs the divisor in the division's range;
                // outside it the crossing is not separated (float64 recheck)
                upper = den_lo >= kDivMin && den_lo <= kDivMax ? __fmul_ru(__fdividef(num_hi, den_lo), kDivHi) : upper;
            }
            if (upper < c.L2) {
                found = true;
                if (wall_wins) {
                    len = fmaxf(sw, 0.0f);
                    to_wall = true;
                } else {
                    if (XL) {
                        // the winner's site heads its block
                        const float R0h[3] = {R0h_(0), R0h_(1), R0h_(2)}, R0l[3] = {R0l_(0), R0l_(1), R0l_(2)};
                        const float Kl[3] = {Kl_(0), Kl_(1), Kl_(2)};
                        exact_length(__ldg(h.rel + rec_w(qw)), pmx, pmy, pmz, R0h, R0l, Kh, Kl, th, tl, len, len_lo);
                    } else {
                        // den > dden > 0 here; 2-ulp division (the length only feeds tau and t)
                        len = __fdividef(fmaxf(w1.num, 0.0f), w1.den);
                    }
                    nextB = rec_w(qw);
                }
            } else {
                // float64 recheck of this crossing from r = r0 + t k, on the
                // absolute block of the cell
                if (gl == 0) VG_STAT(S_RE, 1);
                const RaySetDev *rs = BATCH ? &a.sets[set] : &a.s1;
                const double *o = rs->origin + 3 * li;
                const double *d = rs->dir + 3 * li;
                double kd[3], rp[3];
                const double t = __dadd_rn((double)th, (double)tl);
                for (int cc = 0; cc < 3; cc++) {
                    kd[cc] = __ldg(d + cc);
                    rp[cc] = __fma_rn(t, kd[cc], __ldg(o + cc));
                }
                const float4 *ablk = h.cells + rec_w(hdr1);
                const int acnt = hdr_count(__ldg(ablk));
                const int win = exit64<LPR, false>(h, gp, ablk, nullptr, acnt, (double)pmx, (double)pmy, (double)pmz,
                                                   rp, kd, nullptr, gmask, gl, s64);
                if (win == kSphereWin) {
                    found = true;
                    to_wall = true;
                } else if (win > 0) {
                    const float4 qa = __ldg(ablk + win);
                    found = true;
                    to_wall = rec_w(qa) < 0;
                    if (!to_wall) nextB = rec_w(__ldg(h.cells + rec_w(qa)));  // F of the next cell
                }
                len = __double2float_rn(s64);
                from64 = true;
            }
        }
        // interaction mode: the package's attenuation in this cell, and
        // whether it interacts here (the running tau reaches tau_int)
        float dtau_i = 0.f;
        bool passes = true;
        if (MODE == MODE_INTERACT) {
            dtau_i = __fmul_rn(__fmul_rn(kappa, rho), len);
            passes = !(__fsub_rn(tint, tau32) <= __fsub_rn(dtau_i, tauc));
        }
        if (!FP64 && found && !to_wall && !from64 && len > 0.0f && passes && steps + 1 < max_steps) {
            // the common crossing of the float32 form, a positive step into
            // the next cell, apart from the general case below (same
            // operations, fewer branches per crossing)
            if (MODE == MODE_SEGS && gl == 0) {
                pend = true;
                pend_cell = caller;
                pend_ray = (int)ray;
                pend_len = len;
            }
            if (MODE == MODE_GRAD && gl == 0) atomicAdd(&a.dL_drho[caller], dLr * kappa * len);
            if (MODE == MODE_INTERACT) {
                if (gl == 0 && a.absorbed) atomicAdd(&a.absorbed[caller], wgt * att * -expm1f(-dtau_i));
                att = __fmul_rn(att, __expf(-dtau_i));
            }
            steps++;
            nseg++;
            const float y = __fsub_rn(__fmul_rn(__fmul_rn(kappa, rho), len), tauc);
            const float tt = __fadd_rn(tau32, y);
            tauc = __fsub_rn(__fsub_rn(tt, tau32), y);
            tau32 = tt;
            zrun = 0;
            if (XL) ff_add2(th, tl, len, len_lo);
            else ff_add(th, tl, len);
            B = nextB;
            continue;
        }
        bool interacted = false;  // interaction mode: the package interacts in this cell

        steps++;
        bool relocate = false;
        if (!found) {
            relocate = true;  // no exit found (Sect. 2.2): nudge over epsilon and locate again
        } else {
            const bool positive = FP64 ? (s64 > 0.0) : (len > 0.0f);
            if (positive) {
                if (MODE == MODE_SEGS && gl == 0) {
                    pend = true;  // stored at the top of the next iteration
                    pend_cell = caller;
                    pend_ray = (int)ray;
                    if (FP64) pend_len = s64;
                    else pend_len = len;
                }
                if (MODE == MODE_GRAD && gl == 0) atomicAdd(&a.dL_drho[caller], dLr * kappa * len);
                if (MODE == MODE_INTERACT) {
                    // the package is attenuated by exp(-dtau) in this cell; it
                    // interacts here if the running tau reaches tau_int
                    const float krho = __fmul_rn(kappa, rho);
                    const float dtau = __fmul_rn(krho, len);
                    const float left = __fsub_rn(tint, tau32);
                    if (left <= __fsub_rn(dtau, tauc)) {
                        const float part = fmaxf(left, 0.0f);
                        if (gl == 0) {
                            if (a.absorbed) atomicAdd(&a.absorbed[caller], wgt * att * -expm1f(-part));
                            a.int_cell[ray] = caller;
                            const float ds = krho > 0.0f ? fminf(__fdividef(part, krho), len) : 0.0f;
                            a.int_s[ray] = __fadd_rn(__fadd_rn(th, tl), ds);
                        }
                        interacted = true;
                    } else {
                        if (gl == 0 && a.absorbed)
                            atomicAdd(&a.absorbed[caller], wgt * att * -expm1f(-dtau));
                        att = __fmul_rn(att, __expf(-dtau));
                    }
                }
                nseg++;
                if (FP64) {
                    tau64 = __dadd_rn(tau64, __dmul_rn(__dmul_rn((double)kappa, (double)rho), s64));
                } else {
                    // Kahan-compensated sum of kappa rho l
                    const float y = __fsub_rn(__fmul_rn(__fmul_rn(kappa, rho), len), tauc);
                    const float tt = __fadd_rn(tau32, y);
                    tauc = __fsub_rn(__fsub_rn(tt, tau32), y);
                    tau32 = tt;
                }
                zrun = 0;
            } else {
                zrun++;
                if (gl == 0) VG_STAT(S_ZERO, 1);
            }
            if (MODE == MODE_INTERACT && interacted) to_wall = true;  // the path ends here
            // advance the point
            if (FP64) {
                for (int c = 0; c < 3; c++) r64[c] = __dadd_rn(r64[c], __dmul_rn(s64, k64[c]));
            } else if (from64) {
                ff_add_double(th, tl, s64);
            } else if (XL) {
                ff_add2(th, tl, len, len_lo);
            } else {
                ff_add(th, tl, len);
            }
            if (to_wall) {
                ended = true;
            } else {
                if (FP64) {  // the float32 form reads the site from the next block
                    pmx = qn.x;
                    pmy = qn.y;
                    pmz = qn.z;
                }
                B = nextB;
                // more zero-length steps in a row than the grid allows: nudge
                relocate = zrun > 0 && zrun > (BATCH ? gp->zmax : a.g1.zmax);
            }
        }
        if (relocate) {
            if (gl == 0) VG_STAT(S_FB, 1);
            zrun = 0;
            double x[3];
            if (FP64) {
                for (int c = 0; c < 3; c++) r64[c] = __dadd_rn(r64[c], __dmul_rn(gp->eps64, k64[c]));
                for (int c = 0; c < 3; c++) x[c] = r64[c];
            } else {
                ff_add_double(th, tl, gp->eps32);
                const RaySetDev *rs = BATCH ? &a.sets[set] : &a.s1;
                const double t = __dadd_rn((double)th, (double)tl);
                for (int c = 0; c < 3; c++) x[c] = __fma_rn(t, __ldg(rs->dir + 3 * li + c), __ldg(rs->origin + 3 * li + c));
            }
            const int nm = locate_point<false>(gp, loc_point(x[0], x[1], x[2]), !FP64, nullptr);
            if (nm < 0) {
                ended = true;
            } else {
                const float4 q = __ldg(&h.site[nm]);
                pmx = q.x;
                pmy = q.y;
                pmz = q.z;
                B = rec_w(q);
                if (FP64) B = rec_w(__ldg(h.rel + B + 1));  // absolute block of the cell
            }
        }
        if (!ended && steps >= max_steps) {
            ended = true;
            status = RAY_STEP_LIMIT;
            if (gl == 0) VG_STAT(S_LIM, 1);
        }
        if (ended) {
            if (gl == 0) {
                VG_STAT(S_RAYS, 1);
                VG_STAT(S_CROSS, nseg);
                VG_STAT(S_DEC, steps);
                const RaySetDev *rs = BATCH ? &a.sets[set] : &a.s1;
                if (MODE == MODE_TAU || MODE == MODE_SEGS) {
                    if (rs->tau) {
                        if (FP64) ((double *)rs->tau)[li] = tau64;
                        else ((float *)rs->tau)[li] = tau32;
                    }
                    if (rs->status) rs->status[li] = status;
                }
                if (MODE == MODE_SEGS) a.seg_off[ray] = nseg;
                if (MODE == MODE_INTERACT && !interacted) {
                    a.int_cell[ray] = -1;  // escaped (or cut at the step limit)
                    a.int_s[ray] = __fadd_rn(th, tl);
                }
            }
            ray = -1;
        }
    }

    // segment mode: the rest of the warp's page holds no segments
    if (MODE == MODE_SEGS && a.chunk_cap > 0)
        for (int c = s_page[wib][0] + lane; c < s_page[wib][1]; c += 32)
            if (c < a.chunk_cap) a.chunk_meta[c] = make_int2(-1, 0);

    // ---------------- statistics: one global atomic per block and counter ----------------
#undef VG_STAT
#undef R0h_
#undef R0l_
#undef Kl_
#undef tmh_
#undef tml_
    __syncthreads();
    if (threadIdx.x < 9 && s_stats[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(a.stats) + threadIdx.x, s_stats[threadIdx.x]);
}

}  // namespace vg
