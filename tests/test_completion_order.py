"""Host logic of the CUDA path, compiled here from the library's internal header into a
small host program:
- the enumeration of the spatial completion family (kc_cand) follows R11's order: the same
  cosine products, in the same order, as the oracle's family, for square, thin and ragged
  subdomain shapes, and nothing past the family's end;
- the guard on the angular table (orthogonal_prefix_gram): the whole weighted table of a product
  quadrature is mutually orthogonal, and a direction table whose angles are perturbed keeps
  only the leading part that still is."""
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
  if (argc == 4 && argv[1][0] == 'p') {          // p <table file: nc n values> <tol>
    FILE* f = fopen(argv[2], "r");
    int nc = 0, n = 0;
    if (!f || fscanf(f, "%d %d", &nc, &n) != 2) return 2;
    double* t = new double[(size_t)nc * n];
    for (size_t i = 0; i < (size_t)nc * n; ++i)
      if (fscanf(f, "%lf", &t[i]) != 1) return 3;
    fclose(f);
    double* g = new double[(size_t)nc * nc];           // the table's Gram, as the library forms it
    for (int i = 0; i < nc; ++i)
      for (int j = 0; j < nc; ++j) {
        double y = 0.0;
        for (int q = 0; q < n; ++q) y += t[(size_t)i * n + q] * t[(size_t)j * n + q];
        g[(size_t)i * nc + j] = y;
      }
    printf("%d\n", dd::orthogonal_prefix_gram(g, nc, atof(argv[3])));
    delete[] g;
    delete[] t;
    return 0;
  }
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


def _prefix(prog, tmp_path, table):
    path = tmp_path / "table.txt"
    nc, n = table.shape
    path.write_text(f"{nc} {n}\n" + "\n".join(repr(float(x)) for x in table.reshape(-1)))
    out = subprocess.run([prog, "p", str(path), "1e-12"], capture_output=True, text=True,
                         timeout=60, check=True).stdout
    return int(out.strip())


def test_angular_table_orthogonal_prefix(prog, tmp_path):
    from paper_2602_14854_gb300 import inputs
    wl = inputs.config_c0()                               # 8 mu x 16 phi product quadrature
    tab = np.array(list(itertools.islice(dd_dlra.angular_candidates(wl), 64)))
    tab = tab * np.sqrt(wl.w)[None, :]                    # weighted, as the library stores it
    assert _prefix(prog, tmp_path, tab) == tab.shape[0]
    # the same family evaluated on directions whose azimuths are perturbed: no longer an
    # exact quadrature for the products, so the orthogonal run ends early (but not at once)
    rng = np.random.default_rng(3)
    phi = np.arctan2(wl.omega_y, wl.omega_x) + 0.02 * rng.standard_normal(wl.n)
    s = np.hypot(wl.omega_x, wl.omega_y)
    bad = wl.with_(omega_x=s * np.cos(phi), omega_y=s * np.sin(phi))
    tab2 = np.array(list(itertools.islice(dd_dlra.angular_candidates(bad), 64)))
    tab2 = tab2 * np.sqrt(bad.w)[None, :]
    p2 = _prefix(prog, tmp_path, tab2)
    assert 1 <= p2 < tab2.shape[0]
    G = tab2[:p2] @ tab2[:p2].T
    d = np.sqrt(np.diag(G))
    assert np.max(np.abs(G / np.outer(d, d) - np.eye(p2))) <= 1e-12
    g = tab2[:p2 + 1] @ tab2[p2]
    dn = np.sqrt(np.sum(tab2[:p2 + 1] ** 2, axis=1))
    assert np.max(np.abs(g[:p2]) / (dn[:p2] * dn[p2])) > 1e-12   # the first one that is not
