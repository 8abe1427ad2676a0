"""Host checks of the split column pass's claim order (no GPU needed).

The Navier-Stokes column pass at 4096^2 runs each tile in two parts; CTAs
claim positions from a counter and `split_item` (passes.cuh) maps a position
to (part, tile).  Every wait of a part 1 ends only if each tile's part 0 sits
at an earlier position than its part 1, and the pass is complete only if the
map is a bijection onto the 2 * tiles items.  This compiles the kernel
header's own function into a host program with nvcc and checks both
properties for tile counts 1 .. 1200 and several grid sizes (the lag is
min(grid, tiles), as in the kernel), plus the kernel's workload case (342
tiles of four columns on 152 SMs).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1206_3215_gb300", "csrc")

PROGRAM = r"""
#include "passes.cuh"
#include <cstdio>
#include <vector>
int main()
{
    long bad = 0, cases = 0;
    const int grids[] = {1, 2, 3, 7, 64, 151, 152, 153, 304, 5000};
    for (int tiles = 1; tiles <= 1200; ++tiles)
        for (int grid : grids) {
            const int lag = grid < tiles ? grid : tiles;
            std::vector<int> at0(tiles, -1), at1(tiles, -1);
            for (int p = 0; p < 2 * tiles; ++p) {
                int part = -1, tile = -1;
                pss::split_item(p, tiles, lag, part, tile);
                if (tile < 0 || tile >= tiles || (part != 0 && part != 1)) { ++bad; continue; }
                int &slot = part ? at1[tile] : at0[tile];
                if (slot >= 0) ++bad;  // an item reached twice
                slot = p;
            }
            for (int t = 0; t < tiles; ++t)
                if (at0[t] < 0 || at1[t] < 0 || at1[t] <= at0[t]) ++bad;
            ++cases;
        }
    // the workload's case: part 1 of tile j about one round after its part 0
    const int tiles = 342, lag = 152;
    int worst = 1 << 30;
    for (int p = 0; p < 2 * tiles; ++p) {
        int part, tile;
        pss::split_item(p, tiles, lag, part, tile);
        if (part == 1) {
            int p0 = -1;
            for (int q = 0; q < 2 * tiles; ++q) {
                int pa, ti;
                pss::split_item(q, tiles, lag, pa, ti);
                if (pa == 0 && ti == tile) p0 = q;
            }
            if (p - p0 < worst) worst = p - p0;
        }
    }
    std::printf("%ld %ld %d\n", cases, bad, worst);
    return 0;
}
"""


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_split_claim_order_is_a_bijection_with_part0_first(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "split_order.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "split_order"
    # the header's device code needs the target's intrinsics declared
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                    "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    cases, bad, worst = (int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.split())
    assert cases == 1200 * 10
    assert bad == 0
    # at the workload size part 1 never comes right after its part 0: it is
    # claimed at least a full grid of positions later
    assert worst >= 152
