"""The boundary-band layout of the library (csrc/band.cuh), compiled into a
small host program: band_cell and band_offset are inverse bijections between
[0, band_cells) and the model cells within r of a face, and the cells come in
the documented order (z-face planes, then y-face rows, then x-face cells),
written out independently here with numpy."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1603_03971_gb300", "csrc")

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "band.cuh"
int main(int argc, char** argv) {
    const int nx = atoi(argv[1]), ny = atoi(argv[2]), nz = atoi(argv[3]), r = atoi(argv[4]);
    const long long n = rtm::band_cells(nx, ny, nz, r);
    long long hits = 0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                const long long b = rtm::band_offset(x, y, z, nx, ny, nz, r);
                if (b < -1 || b >= n) { printf("BAD offset\n"); return 1; }
                if (b >= 0) hits++;
            }
    if (hits != n) { printf("BAD count %lld %lld\n", hits, n); return 1; }
    printf("%lld\n", n);
    for (long long b = 0; b < n; b++) {
        int x, y, z;
        rtm::band_cell(b, nx, ny, nz, r, x, y, z);
        if (rtm::band_offset(x, y, z, nx, ny, nz, r) != b) { printf("BAD inverse\n"); return 1; }
        printf("%d %d %d\n", z, y, x);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def band_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("band")
    src = d / "band_check.cu"
    src.write_text(PROGRAM)
    exe = d / "band_check"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    return str(exe)


def _documented_order(nx, ny, nz, r):
    cells = []
    for f in range(2 * r):  # z-face planes
        z = f if f < r else f + nz - 2 * r
        cells += [(z, y, x) for y in range(ny) for x in range(nx)]
    for z in range(r, nz - r):  # y-face rows of the other planes
        for f in range(2 * r):
            y = f if f < r else f + ny - 2 * r
            cells += [(z, y, x) for x in range(nx)]
    for z in range(r, nz - r):  # x-face cells of the remaining rows
        for y in range(r, ny - r):
            for f in range(2 * r):
                cells.append((z, y, f if f < r else f + nx - 2 * r))
    return np.array(cells)


@pytest.mark.parametrize("shape,r", [((9, 10, 11), 4), ((17, 18, 20), 8), ((3, 4, 5), 1),
                                     ((12, 9, 10), 4)])
def test_band_layout(band_exe, shape, r):
    nx, ny, nz = shape
    out = subprocess.run([band_exe, str(nx), str(ny), str(nz), str(r)], check=True,
                         capture_output=True, text=True).stdout.split("\n")
    n = int(out[0])
    got = np.array([[int(v) for v in line.split()] for line in out[1:1 + n]])
    want = _documented_order(nx, ny, nz, r)
    assert n == len(want)
    assert np.array_equal(got, want)
    # and they are exactly the cells within r of a face
    z, y, x = want.T
    dist = np.minimum.reduce([z, nz - 1 - z, y, ny - 1 - y, x, nx - 1 - x])
    assert (dist < r).all()
    assert n == nx * ny * nz - (nx - 2 * r) * (ny - 2 * r) * (nz - 2 * r)
