"""The checked build (-DVOGE_CHECKED): its index-check helpers on the CPU, and
the checked library itself (built, loaded, every declared symbol exported).

The helpers are compiled for the host with nvcc from the same header the
kernels use, so the test sees the code the kernels run (the device form
differs only in recording the site with atomicCAS).  No kernel runs here."""
import ctypes
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include "voge_device.cuh"
using namespace voge;
static int fails = 0;
#define EXPECT(c) do { if (!(c)) { std::printf("FAIL line %d\n", __LINE__); ++fails; } } while (0)
int main() {
    // in_bounds: [0, n), with negative and huge indices out
    EXPECT(in_bounds(0, 1));
    EXPECT(in_bounds(4, 5));
    EXPECT(!in_bounds(5, 5));
    EXPECT(!in_bounds(-1, 5));
    EXPECT(!in_bounds(0, 0));
    EXPECT(!in_bounds((int64_t)1 << 40, (int64_t)1 << 32));
    EXPECT(in_bounds(((int64_t)1 << 32) - 1, (int64_t)1 << 32));
    // checked_index: in range passes through and records nothing
    int32_t site = 0;
    EXPECT(checked_index(&site, 7, 8, kChkRecord) == 7);
    EXPECT(site == 0);
    // out of range: redirected to 0, the site recorded
    EXPECT(checked_index(&site, 8, 8, kChkRecord) == 0);
    EXPECT(site == kChkRecord);
    // the first failure wins
    EXPECT(checked_index(&site, -3, 8, kChkOutput) == 0);
    EXPECT(site == kChkRecord);
    EXPECT(checked_index(&site, 2, 8, kChkOutput) == 2);
    EXPECT(site == kChkRecord);
    // every site is a distinct non-zero code
    const int32_t sites[] = {kChkTileList, kChkRecord, kChkTile, kChkListRead, kChkOutput, kChkScratch, kChkBin};
    for (int i = 0; i < 7; ++i) {
        EXPECT(sites[i] != 0);
        for (int j = 0; j < i; ++j) EXPECT(sites[i] != sites[j]);
    }
    std::printf(fails ? "failed\n" : "ok\n");
    return fails ? 1 : 0;
}
"""


def test_check_helpers_on_the_host():
    from paper_2205_15401_gb300 import build

    nvcc = build._nvcc()
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "harness.cu"), os.path.join(d, "harness")
        open(src, "w").write(HARNESS)
        inc = os.path.join(ROOT, "paper_2205_15401_gb300", "csrc")
        subprocess.check_call([nvcc, "-std=c++17", "-I", inc, "-o", exe, src])
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


def test_checked_library_builds_and_exports_every_symbol():
    from paper_2205_15401_gb300 import build

    path = build.build(checked=True)
    assert path.endswith("libvoge_checked.so") and os.path.exists(path)
    from test_cabi import declared_symbols

    L = ctypes.CDLL(path)
    for n in declared_symbols():
        assert hasattr(L, n), n
    L.voge_strerror.restype = ctypes.c_char_p
    assert b"checked" in L.voge_strerror(-8)
