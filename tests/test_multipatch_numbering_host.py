"""Host logic of the library's multi-patch gluing (csrc/multipatch.cu: the entry order of a
side or face and the orientation codes) against the oracle's rule, which its own tests pin
by hand and by the p = 1 single-patch identities: a small program compiled with nvcc
prints, for 2-D sides and 3-D faces and every orientation code, the local index of every
entry and of its partner; the lists must equal the oracle's."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle.multipatch import oriented, side_indices

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
#include "paper_2004_05197_gb300/csrc/multipatch.cu"
#include <cstdio>
int main() {
    const int m = 5;
    for (int dim = 2; dim <= 3; ++dim) {
        const long long ne = dim == 2 ? m : (long long)m * m;
        for (int side = 0; side < 2 * dim; ++side) {
            std::printf("side %d %d", dim, side);
            for (long long e = 0; e < ne; ++e) std::printf(" %lld", iga::side_index(dim, m, side, e));
            std::printf("\n");
        }
        for (int o = 0; o < (dim == 2 ? 2 : 8); ++o) {
            std::printf("orient %d %d", dim, o);
            for (long long e = 0; e < ne; ++e) std::printf(" %lld", iga::oriented_entry(dim, m, o, e));
            std::printf("\n");
        }
    }
    return 0;
}
"""


def test_library_face_order_and_orientations_equal_the_oracle():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "mp.cu"), os.path.join(d, "mp")
    with open(src, "w") as f:
        f.write(PROBE)
    # the probe runs only the two host functions; the rest of the file links against the library
    from paper_2004_05197_gb300 import build
    build.build()
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a", "-I", ROOT,
                           "-I", os.path.join(ROOT, "include"), "-o", exe, src,
                           "-L", os.path.join(ROOT, "paper_2004_05197_gb300"), "-liga",
                           "-Xlinker", "-rpath=" + os.path.join(ROOT, "paper_2004_05197_gb300")],
                          stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    out = subprocess.check_output([exe]).decode().splitlines()
    shutil.rmtree(d, ignore_errors=True)
    m, seen = 5, 0
    for line in out:
        f = line.split()
        dim, k, vals = int(f[1]), int(f[2]), np.array(list(map(int, f[3:])))
        if f[0] == "side":
            assert np.array_equal(vals, side_indices(m, k, dim)), (dim, k)
        else:
            assert np.array_equal(vals, oriented(m, dim, k)), (dim, k)
        seen += 1
    assert seen == 4 + 2 + 6 + 8
