"""The host-side expand masks (wdf_internal.h expand_masks, Hacker's Delight section 7-5)
that the consumer kernel uses to move decisions collected in record order to the real
nodes' heap positions: checked against a bit-by-bit deposit on random masks, including
the property the kernel relies on instead of a final mask -- every stray copy the six
steps leave lies outside the mask, where the pass-through bits are all ones."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2511_09376_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "wdf_internal.h"

static uint64_t rng = 0x9E3779B97F4A7C15ull;
static uint64_t next() {  // splitmix64
    uint64_t z = (rng += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int main() {
    const uint64_t nodes63 = (1ull << 63) - 1ull;  // the 63 inner nodes of a depth-6 tree
    for (int trial = 0; trial < 200000; ++trial) {
        uint64_t m = next() & nodes63;
        if (trial % 3 == 1) m &= next();
        if (trial % 3 == 2) m = trial % 64 == 0 ? 0ull : (nodes63 >> (trial % 63));
        int cnt = 0;
        for (int p = 0; p < 64; ++p) cnt += (int)((m >> p) & 1ull);
        const uint64_t x = cnt == 0 ? 0ull : (cnt == 64 ? next() : next() & ((1ull << cnt) - 1ull));
        uint64_t ref = 0ull;
        for (int p = 0, k = 0; p < 64; ++p)
            if ((m >> p) & 1ull) ref |= ((x >> k++) & 1ull) << p;
        uint64_t mv[6];
        wdf::expand_masks(m, mv);
        uint64_t y = x;
        for (int k = 5; k >= 0; --k) y = (y & ~mv[k]) | ((y << (1 << k)) & mv[k]);
        const uint64_t pt = ~m & nodes63;
        if ((y & m) != ref || ((y | pt) & nodes63) != (ref | pt)) {
            std::printf("mismatch m=%llx x=%llx\n", (unsigned long long)m, (unsigned long long)x);
            return 1;
        }
    }
    std::printf("ok\n");
    return 0;
}
"""


def test_expand_masks_against_bitwise_deposit(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "expand.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "expand"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
