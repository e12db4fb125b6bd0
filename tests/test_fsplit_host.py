"""Host checks of the integer float64 helpers the start-cell kernel uses
(csrc/fsplit.h): the float-pair split must give exactly the two float32
conversions of its definition, hi = fl32(x), lo = fl32(x - hi), and the order
keys must order float64 values like the values themselves. The header is
compiled for the host with g++ (the same source the device compiles)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1310_1854_gb300", "csrc")

PROG = r"""
#include "fsplit.h"
#include <cstdio>
#include <cstdlib>
int main(int argc, char **argv) {
    // stdin: count, then doubles as hex bit patterns; stdout per value:
    // ok hi_bits lo_bits key
    long n;
    if (scanf("%ld", &n) != 1) return 2;
    for (long i = 0; i < n; i++) {
        unsigned long long b;
        if (scanf("%llx", &b) != 1) return 2;
        double x;
        memcpy(&x, &b, 8);
        float h = 0.f, l = 0.f;
        const int ok = vg::split_double_int(x, h, l) ? 1 : 0;
        uint32_t hb, lb;
        memcpy(&hb, &h, 4);
        memcpy(&lb, &l, 4);
        printf("%d %08x %08x %lld %d\n", ok, hb, lb, (long long)vg::dkey(x), vg::disnan(x) ? 1 : 0);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("fsplit")
    src = d / "t.cpp"
    src.write_text(PROG)
    exe = d / "t"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)])
    return str(exe)


def run(prog, xs):
    bits = np.asarray(xs, dtype=np.float64).view(np.uint64)
    inp = f"{len(bits)}\n" + "\n".join(f"{int(b):x}" for b in bits) + "\n"
    out = subprocess.run([prog], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [r.split() for r in out if r.strip()]
    ok = np.array([int(r[0]) for r in rows], dtype=bool)
    hi = np.array([int(r[1], 16) for r in rows], dtype=np.uint32).view(np.float32)
    lo = np.array([int(r[2], 16) for r in rows], dtype=np.uint32).view(np.float32)
    key = np.array([int(r[3]) for r in rows], dtype=np.int64)
    nan = np.array([int(r[4]) for r in rows], dtype=bool)
    return ok, hi, lo, key, nan


def samples(n=60000, seed=1310_1854):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2**63, size=n, dtype=np.uint64) | (rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63))
    e = rng.integers(1023 - 70, 1023 + 110, size=n).astype(np.uint64)
    bits = (bits & np.uint64(0x800FFFFFFFFFFFFF)) | (e << np.uint64(52))
    x = bits.view(np.float64)
    # ties and near-ties of float32 rounding: f +- half an ulp, and one
    # float64 ulp either side of those
    f = x.astype(np.float32).astype(np.float64)
    half = np.ldexp(1.0, np.frexp(f)[1] - 25)
    t = np.concatenate([f + half, f - half])
    t = t[np.isfinite(t)]
    near = np.concatenate([t, np.nextafter(t, 0.0), np.nextafter(t, np.inf), f, np.nextafter(f, 0.0)])
    special = np.array([0.0, -0.0, 1.0, -1.0, 0.1, 1.0 / 3.0, 16777215.5, 16777216.5, 2.0**-60, -(2.0**-60),
                        np.nextafter(2.0**100, 0.0), 2.0**100, 2.0**-61, 1e-300, 5e-324, np.inf, -np.inf, np.nan,
                        np.float64(np.float32(3.4028234663852886e38)), np.nextafter(1.0, 0.0), np.nextafter(2.0, 0.0)])
    return np.concatenate([x, near, special])


def test_split_equals_two_conversions(prog):
    x = samples()
    ok, hi, lo, _, _ = run(prog, x)
    fin = np.isfinite(x)
    # covered range: zero and 2^-60 <= |x| < 2^100
    ax = np.abs(x)
    covered = fin & ((ax == 0) | ((ax >= 2.0**-60) & (ax < 2.0**100)))
    assert np.array_equal(ok, covered)
    with np.errstate(over="ignore", invalid="ignore"):
        ref_hi = x.astype(np.float32)
        ref_lo = (x - ref_hi.astype(np.float64)).astype(np.float32)
    assert np.array_equal(hi[ok].view(np.uint32), ref_hi[ok].view(np.uint32))
    assert np.array_equal(lo[ok].view(np.uint32), ref_lo[ok].view(np.uint32))
    # the pair carries x to within 2^-48 |x|
    sel = ok & (ax > 0)
    err = np.abs(hi[sel].astype(np.float64) + lo[sel].astype(np.float64) - x[sel]) / ax[sel]
    assert err.max() <= 2.0**-48


def test_order_keys(prog):
    x = samples(20000)
    x = x[~np.isnan(x)]
    _, _, _, key, nan = run(prog, x)
    assert not nan.any()
    o = np.argsort(x, kind="stable")
    xs, ks = x[o], key[o]
    # keys never decrease along increasing x; equal values share a key
    assert np.all(np.diff(ks) >= 0)
    same = np.diff(xs) == 0
    assert np.all(np.diff(ks)[same] == 0)
    assert np.all(np.diff(ks)[~same] > 0)
    _, _, _, _, nan = run(prog, [np.nan, -np.nan, np.inf, 1.0])
    assert list(nan) == [True, True, False, False]
