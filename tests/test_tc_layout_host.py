"""Host-side checks of the shared tile layout of the tcgen05 kernels
(paper_1808_03374_gb300/csrc/tc_layout.cuh), compiled by nvcc and run on the
CPU (no GPU needed):

- bt_kpos maps the 16 samples of a code word onto K positions 0..15 one to one,
  and bt_sample_of_kpos inverts it;
- bt_swz maps (row < 128, K byte < 128) one to one onto the 16 KB tile;
- bt_swz equals the 128-byte swizzle as the public descriptions state it,
  written here independently of bt_swz: take the unswizzled byte address
  a = 128 r + kk of a tile of 128-byte rows and XOR its bits 7-9 into its bits
  4-6 (CuTe's Swizzle<3, 4, 3>: a ^ ((a & 0x380) >> 3)), and a few offsets
  worked out by hand from the rule "16-byte chunk c of row r lands at chunk
  c XOR (r mod 8) of the same 128-byte row; rows r >= 8 start 1024 bytes per 8
  rows further".
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SOURCE = r'''
#include <cstdio>
#include <vector>
#include "tc_layout.cuh"
using namespace gkl;
int main() {
    int bad = 0;
    std::vector<int> seen(16, 0);
    for (int s = 0; s < 16; ++s) {
        const int k = bt_kpos(s);
        if (k < 0 || k > 15 || seen[k]++) ++bad;
        if (bt_sample_of_kpos(k) != s) ++bad;
    }
    std::vector<int> hit(16384, 0);
    for (int r = 0; r < 128; ++r)
        for (int kk = 0; kk < 128; ++kk) {
            const int o = bt_swz(r, kk);
            if (o < 0 || o >= 16384 || hit[o]++) { ++bad; continue; }
            const int a = 128 * r + kk;                                   // unswizzled address
            if (o != (a ^ ((a & 0x380) >> 3))) ++bad;                      // Swizzle<3, 4, 3>
        }
    // (row, K byte) -> offset, by hand
    const int hand[][3] = {{0, 0, 0},       {0, 17, 17},    {1, 0, 144},    {1, 16, 128},  {1, 31, 143},
                           {2, 32, 128 * 2 + 0}, {3, 48, 384}, {7, 127, 911}, {8, 0, 1024}, {9, 40, 1208},
                           {15, 112, 1920 + 0}, {127, 5, 16373}};
    for (const auto& e : hand)
        if (bt_swz(e[0], e[1]) != e[2]) { printf("hand %d %d -> %d\n", e[0], e[1], bt_swz(e[0], e[1])); ++bad; }
    printf("%d\n", bad);
    return 0;
}
'''


def test_tc_layout_helpers(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "layout_check.cu"
    src.write_text(SOURCE)
    exe = tmp_path / "layout_check"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_1808_03374_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    assert out.strip() == "0"
