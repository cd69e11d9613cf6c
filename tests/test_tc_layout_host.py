"""Host-side checks of the shared tile layout of the tcgen05 kernels
(paper_1808_03374_gb300/csrc/tc_layout.cuh), compiled by nvcc and run on the
CPU (no GPU needed):

- bt_kpos maps the 16 samples of a code word onto K positions 0..15 one to one,
  and bt_sample_of_kpos inverts it;
- bt_swz maps (row < 128, K byte < 128) one to one onto the 16 KB tile, keeps
  each row inside its own 128-byte line and each 16-byte chunk contiguous, and
  permutes the chunks of row r by XOR with r mod 8 (the 128-byte swizzle).
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
            if (o / 128 != (r >> 3) * 8 + (r & 7)) ++bad;                 // row r's own 128-byte line
            if ((o & 15) != (kk & 15)) ++bad;                             // chunks stay contiguous
            if (((o >> 4) & 7) != (((kk >> 4) ^ (r & 7)) & 7)) ++bad;     // chunk c of row r at c ^ (r mod 8)
        }
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
