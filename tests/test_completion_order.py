"""The CUDA path's enumeration of the spatial completion family (kc_cand in the
library's internal header, compiled here into a small host program) follows R11's order:
the same cosine products, in the same order, as the oracle's family, for square, thin and
ragged subdomain shapes, and nothing past the family's end."""
import itertools
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import dd_dlra

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2602_14854_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <cstdlib>
#include "dd_internal.cuh"
int main(int argc, char** argv) {
  const int nx = atoi(argv[1]), ny = atoi(argv[2]), count = atoi(argv[3]);
  for (int j = 0; j < count; ++j) {
    int a = -1, b = -1;
    const bool ok = dd::kc_cand(j, nx, ny, &a, &b);
    printf("%d %d %d\n", ok ? 1 : 0, a, b);
  }
  return 0;
}
"""


class _Sub:
    def __init__(self, nx, ny):
        self.nxk, self.nyk = nx, ny


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("kc_order")
    src = d / "kc_order.cu"
    src.write_text(PROG)
    exe = d / "kc_order"
    r = subprocess.run([nvcc, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    return str(exe)


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 7), (5, 1), (4, 4), (16, 16), (3, 40), (32, 8),
                                   (17, 5), (128, 128)])
def test_spatial_family_order_matches_the_oracle(prog, nx, ny):
    count = min(nx * ny, 160)
    out = subprocess.run([prog, str(nx), str(ny), str(count + 1)], capture_output=True,
                         text=True, timeout=60, check=True).stdout.split("\n")
    pairs = [tuple(int(t) for t in line.split()) for line in out if line.strip()]
    cands = list(itertools.islice(dd_dlra.spatial_candidates(_Sub(nx, ny)), count))
    i, jj = np.arange(nx), np.arange(ny)
    for j, (ok, a, b) in enumerate(pairs[:count]):
        assert ok and 0 <= a < nx and 0 <= b < ny, (j, a, b)
        v = (np.cos(math.pi * b * (jj + 0.5) / ny)[:, None]
             * np.cos(math.pi * a * (i + 0.5) / nx)[None, :]).reshape(-1)
        assert np.array_equal(v, cands[j]), (nx, ny, j, a, b)
    if count == nx * ny:
        assert pairs[count][0] == 0                  # past the end of the family
