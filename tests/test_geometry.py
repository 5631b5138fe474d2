"""Compile-time geometry of the single-pass kernel, checked without a GPU.

march.cuh picks, per storage type and N, the strip width, the ring depth and the number
of box-store staging buffers, and derives the shared memory, the resident CTAs per SM and
the register cap from them.  Those constants decide the kernel's speed (two or three
CTAs per SM) and the legality of its TMA boxes, so a host program built against the
header prints them and this test checks the budgets and the picks the measurements rest on.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0704_3444_gb300", "csrc")
OUT = os.path.join(ROOT, "paper_0704_3444_gb300", "_build", "geometry_probe")

PROBE = r'''
#include "march.cuh"
#include <cstdio>
using namespace mclb;
template <typename G, typename T, int N> void pg(const char* nm) {
    printf("%s %d %d %d %d %zu %d %d %d %d %d %d %d\n", nm, N, G::NWC, G::STAGES, G::NB, G::SMEM,
           G::MIN_CTAS, G::MAXREG, G::THREADS, G::WI, G::WOUT, (int)sizeof(T), (int)G::FITS);
}
template <typename T, int N> void pr(const char* nm) {
    pg<MarchGeom<T, N>, T, N>(nm);
    // the batch's narrow alternative, where it exists
    if (has_narrow<T, N>()) {
        char buf[32];
        snprintf(buf, sizeof(buf), "%s-narrow", nm);
        pg<MarchNarrow<T, N>, T, N>(buf);
    }
}
template <typename T> void all(const char* nm) {
    pr<T, 1>(nm); pr<T, 2>(nm); pr<T, 3>(nm); pr<T, 4>(nm);
    pr<T, 5>(nm); pr<T, 6>(nm); pr<T, 7>(nm); pr<T, 8>(nm);
}
int main() { all<double>("fp64"); all<float>("fp32"); all<__nv_bfloat16>("bf16"); all<__half>("fp16"); }
'''


@pytest.fixture(scope="module")
def geometry():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(OUT, exist_ok=True)
    src, exe = os.path.join(OUT, "probe.cu"), os.path.join(OUT, "probe")
    with open(src, "w") as fh:
        fh.write(PROBE)
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I" + CSRC, "-I" + os.path.join(ROOT, "include"), src, "-o", exe, "-lcuda"],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    g = {}
    for line in out.splitlines():
        name, *v = line.split()
        n, nw, ns, nb, smem, ctas, maxreg, threads, wi, wout, size, fits = map(int, v)
        g[(name, n)] = dict(nw=nw, ns=ns, nb=nb, smem=smem, ctas=ctas, maxreg=maxreg,
                            threads=threads, wi=wi, wout=wout, size=size, fits=fits)
    assert sum(1 for (name, _) in g if "narrow" not in name) == 32
    return g


def test_budgets(geometry):
    for (name, n), c in geometry.items():
        assert c["fits"] == 1 and c["smem"] <= 227 * 1024, (name, n)
        # the resident CTAs share the SM's 228 KB (1 KB reserved per CTA) ...
        assert c["ctas"] * (c["smem"] + 1024) <= 228 * 1024, (name, n)
        # ... and each sub-partition's 16K registers
        warps_sp = (c["ctas"] * c["threads"] // 32 + 3) // 4
        assert c["maxreg"] * 32 * warps_sp <= 16384, (name, n)
        assert 3 <= c["ns"] <= 5 and c["nw"] in (2, 4) and c["nb"] in (1, 2)


def test_tma_boxes(geometry):
    for (name, n), c in geometry.items():
        assert c["wi"] <= 256                       # a box dimension is at most 256
        assert (c["wi"] * c["size"]) % 16 == 0      # inner extent a 16-byte multiple
        hx = max(4, 16 // c["size"])                # ghost columns per side
        assert c["wi"] >= c["wout"] + 3 + hx         # written columns, right halo, left ghosts
        if c["size"] == 2:                          # 16-bit: CTA-wide box stores
            assert (c["wout"] * 2) % 16 == 0
        else:                                       # per-warp 28-column box stores
            assert (28 * c["size"]) % 16 == 0


def test_narrow_alternative(geometry):
    """The batch's second strip shape: two compute warps (56 columns) wherever the pick has
    four, the same ring depth, and never fewer resident CTAs than the wide one."""
    for (name, n), c in geometry.items():
        if "narrow" in name:
            continue
        nar = geometry.get((name + "-narrow", n))
        if c["nw"] == 4:
            assert nar is not None, (name, n)
            assert nar["nw"] == 2 and nar["wout"] == 56 and nar["ns"] == c["ns"]
            assert nar["ctas"] >= c["ctas"], (name, n)
        else:
            assert nar is None


def test_measured_picks(geometry):
    """The configurations the recorded measurements were taken with."""
    f5, b5, h5, f3 = geometry[("fp32", 5)], geometry[("bf16", 5)], geometry[("fp16", 5)], geometry[("fp32", 3)]
    assert (f5["nw"], f5["ns"], f5["ctas"]) == (4, 4, 2)
    for c in (b5, h5):
        assert (c["nw"], c["ns"], c["nb"], c["ctas"], c["maxreg"]) == (4, 4, 1, 3, 128)
    assert (f3["nw"], f3["ns"], f3["ctas"]) == (4, 4, 3)
