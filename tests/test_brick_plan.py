"""Host logic of the brick planner (csrc/brick.cu: plan_bricks), which cuts the m^3 rows of
a 3-D operator into one wave of bricks for the brick kernels.  A small program compiled
with nvcc (host code only runs) prints the plan for a range of meshes; the test checks
what the kernels rely on:

* the bricks tile the grid: every row in exactly one brick;
* one wave: at most one brick per SM (152), the CTA's warps cover every brick's 4 x 8
  lane patches, at most 12 planes per brick (the register tile);
* TMA alignment: every brick starts at an x that is a multiple of 4 (16 bytes), every
  class box is a multiple of 4 floats wide with an odd number of 16-byte chunks, and is
  the brick grown by p where the mirrored reads need it;
* the shared memory of the stages and the vector tile fits the 227 KB of a CTA.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
#include "paper_2004_05197_gb300/csrc/brick.cu"
#include <cstdio>
namespace iga {
int fail(int code, const std::string&) { return code; }
int cuda_fail(cudaError_t, const char*) { return -3; }
void count_launch(long long) {}
DevBuf::~DevBuf() {}
int DevBuf::alloc(size_t) { return 0; }
void DevBuf::release() {}
int onthefly_prepare(iga_ops*) { return 0; }
}
int main() {
    const int ms[] = {14, 22, 30, 42, 50, 66, 82, 98};
    for (int P = 1; P <= 2; ++P)
        for (int m : ms) {
            const auto pr = iga::plan_bricks(m, P, P == 2 ? 63 : 14, 152, 12, 31, 227 * 1024);
            std::printf("plan %d %d %zu %d %d %d %d %d\n", m, P, pr.bricks.size(), pr.ns, pr.ncw, pr.ncls,
                        pr.stage_floats, pr.xt_floats);
            for (int c = 0; c < pr.ncls; ++c) std::printf("cls %d %d %d %d\n", c, pr.bx[c], pr.by[c], pr.bz[c]);
            for (const auto& b : pr.bricks)
                std::printf("brick %d %d %d %d %d %d %d %d\n", b.x0, b.y0, b.z0, b.nx, b.ny, b.nz, b.cls, b.warps);
        }
    return 0;
}
"""


def _plans():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "plan.cu"), os.path.join(d, "plan")
    with open(src, "w") as f:
        f.write(PROBE)
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "-I", ROOT,
                           "-I", os.path.join(ROOT, "include"), "-o", exe, src, "-lcuda"],
                          stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    out = subprocess.check_output([exe]).decode().splitlines()
    shutil.rmtree(d, ignore_errors=True)
    plans, cur = [], None
    for line in out:
        f = line.split()
        if f[0] == "plan":
            cur = dict(zip(["m", "P", "n", "ns", "ncw", "ncls", "stage", "xt"], map(int, f[1:])), cls={}, bricks=[])
            plans.append(cur)
        elif f[0] == "cls":
            cur["cls"][int(f[1])] = tuple(map(int, f[2:]))
        else:
            cur["bricks"].append(tuple(map(int, f[1:])))
    return plans


def test_brick_plans_tile_the_grid_in_one_aligned_wave():
    plans = _plans()
    assert len(plans) == 16
    big = [pl for pl in plans if pl["m"] == 98 and pl["P"] == 2][0]
    assert big["n"] > 140 and big["ns"] == 3   # the bench mesh: one brick per SM, three stages
    for pl in plans:
        m, P = pl["m"], pl["P"]
        if pl["n"] == 0:
            continue   # no plan: the row kernels run
        assert pl["n"] == len(pl["bricks"]) <= 152, (m, P)
        cover = np.zeros((m, m, m), dtype=np.int32)
        for x0, y0, z0, nx, ny, nz, cls, warps in pl["bricks"]:
            cover[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx] += 1
            assert x0 % 4 == 0 and 1 <= nz <= 12, (m, P)
            assert warps == ((nx + 3) // 4) * ((ny + 7) // 8) <= pl["ncw"] <= 31, (m, P)
            bx, by, bz = pl["cls"][cls]
            assert bx % 4 == 0 and (bx // 4) % 2 == 1 and bx >= nx + 2 * P, (m, P, bx)
            assert by == ny + 2 * P or by >= ny + 2 * P, (m, P)
            assert bz >= nz + P, (m, P)
            assert bx * by * bz <= pl["stage"] and bx * by * (bz + P) <= pl["xt"], (m, P)
        assert (cover == 1).all(), (m, P)
        assert 1024 + 4 * (pl["ns"] * pl["stage"] + pl["xt"]) <= 227 * 1024, (m, P)
