// Integer-only helpers for float64 values, shared by host and device code.
//
// GB300's float64 pipe runs at a small fraction of its float32 and integer
// rates, so the start-cell kernel avoids float64 arithmetic for the work it
// does per ray: splitting coordinates into float pairs and comparing them
// with the box.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define VG_HD __host__ __device__ __forceinline__
#else
#define VG_HD inline
#endif

namespace vg {

VG_HD uint64_t dbits(double x) {
    uint64_t t;
    memcpy(&t, &x, 8);
    return t;
}

VG_HD float fbits(uint32_t b) {
    float f;
    memcpy(&f, &b, 4);
    return f;
}

// Float pair of x: hi = fl32(x) and lo = fl32(x - hi), both rounded to
// nearest even, i.e. the values of the two float64 -> float32 conversions of
// that definition (x - hi is exact in float64). The 53-bit significand S of
// x is cut after its top 24 bits: hi takes those (rounded by the 29 bits
// below), lo = sign * fl32(R) * 2^(e-52) with R = S - 2^29 * Sh the signed
// remainder (|R| <= 2^28). Handles x = +-0 and 2^-60 <= |x| < 2^100, where
// hi and lo are normal float32 values; returns false for every other x
// (subnormal, huge, inf, NaN), where the caller converts in float64.
VG_HD bool split_double_int(double x, float &hi, float &lo) {
    const uint64_t t = dbits(x);
    const uint32_t s = (uint32_t)(t >> 63);
    const int E = (int)((t >> 52) & 0x7ff);
    if ((t << 1) == 0) {  // +-0
        hi = fbits(s << 31);
        lo = 0.0f;
        return true;
    }
    const int e = E - 1023;
    if (e < -60 || e >= 100) return false;
    const uint64_t S = (t & 0xfffffffffffffull) | (1ull << 52);
    uint32_t Sh = (uint32_t)(S >> 29);               // 24 bits, in [2^23, 2^24)
    int32_t R = (int32_t)(uint32_t)(S & 0x1fffffffu);  // 29 bits
    if (R > (1 << 28) || (R == (1 << 28) && (Sh & 1u))) {
        Sh += 1u;  // 2^24 carries into the exponent below
        R -= (1 << 29);
    }
    hi = fbits((s << 31) | (((uint32_t)(e + 127) << 23) + (Sh - (1u << 23))));
    const float scale = fbits((uint32_t)(e - 52 + 127) << 23);  // 2^(e-52), normal
    lo = (float)(s ? -R : R) * scale;                          // one rounding (int -> float)
    return true;
}

// Order key of a float64 value: for non-NaN a, b, a <= b exactly when
// dkey(a) <= dkey(b) as signed integers (-0 and +0 share a key).
VG_HD int64_t dkey(double x) {
    int64_t t = (int64_t)dbits(x);
    if (t == INT64_MIN) t = 0;
    return t ^ ((t >> 63) & INT64_MAX);
}

VG_HD bool disnan(double x) { return (dbits(x) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull; }

}  // namespace vg
