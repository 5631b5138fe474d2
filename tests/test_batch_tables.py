"""Host logic of the batched march, checked without a GPU.

march_ctas (batch.cuh) splits every instance of a batch into strips of WOUT columns and
row segments of about one common height, tallest first.  A host program built against
the header builds the tables for random and degenerate instance shapes and every wave
count the autotuner tries, and checks that each instance's every strip is covered by its
segments exactly once, with no segment empty or past the lattice.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0704_3444_gb300", "csrc")
OUT = os.path.join(ROOT, "paper_0704_3444_gb300", "_build", "batch_table_probe")

PROBE = r'''
#include "batch.cuh"
#include <cstdio>
#include <random>
using namespace mclb;

template <typename T, int N>
int check(const std::vector<Problem>& probs, int slots) {
    using G = MarchGeom<T, N>;
    int bad = 0;
    for (int waves : MARCH_WAVES) {
        const auto v = march_ctas<T, N>((int)probs.size(), probs.data(), slots, waves);
        for (size_t c = 1; c < v.size(); ++c) bad += v[c - 1].H < v[c].H;      // tallest first
        for (size_t k = 0; k < probs.size(); ++k) {
            const int nx = probs[k].nx, ny = probs[k].ny, ns = (nx + G::WOUT - 1) / G::WOUT;
            std::vector<int> cover((size_t)ns * ny, 0);
            for (const auto& c : v) {
                if (c.inst != (int)k) continue;
                bad += c.H < 1 || c.y0 < 0 || c.y0 + c.H > ny || c.x0 % G::WOUT != 0 || c.x0 >= nx;
                for (int y = c.y0; y < c.y0 + c.H && y < ny; ++y) ++cover[(size_t)(c.x0 / G::WOUT) * ny + y];
            }
            for (int n : cover) bad += n != 1;
        }
    }
    return bad;
}

int main() {
    std::mt19937 rng(11);
    std::vector<Problem> probs;
    const int fixed[][2] = {{1, 1}, {1, 9}, {9, 1}, {2, 7}, {112, 1}, {113, 5}, {224, 224}, {225, 33}, {512, 512}};
    for (auto& s : fixed) { Problem p{}; p.nx = s[0]; p.ny = s[1]; probs.push_back(p); }
    std::uniform_int_distribution<int> d(1, 600);
    for (int k = 0; k < 300; ++k) { Problem p{}; p.nx = d(rng); p.ny = d(rng); probs.push_back(p); }
    int bad = 0;
    for (int slots : {1, 152, 456, 608}) {
        bad += check<float, 2>(probs, slots) + check<float, 3>(probs, slots);
        bad += check<__nv_bfloat16, 3>(probs, slots) + check<double, 2>(probs, slots);
    }
    printf("violations %d\n", bad);
    return bad != 0;
}
'''


def test_march_cta_tables_cover_every_instance_once():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(OUT, exist_ok=True)
    src, exe = os.path.join(OUT, "probe.cu"), os.path.join(OUT, "probe")
    with open(src, "w") as fh:
        fh.write(PROBE)
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I" + CSRC, "-I" + os.path.join(ROOT, "include"), src, "-o", exe, "-lcuda"],
                   check=True, capture_output=True, timeout=900)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "violations 0" in r.stdout, r.stdout + r.stderr
