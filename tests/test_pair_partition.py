"""How the paired wavefront cuts a grid into strips and row segments (pair_partition in
csrc/temporal.cuh), host code only: compiled here by nvcc into a small program that prints the
partition for every tile width (128, 192, 256 columns), K = 2 .. 8 and a range of grid sizes,
and checked against what the kernels rely on:

* strips are of an even width (pairs of columns stay 8-byte aligned), every strip but the last
  exactly w wide, and together they cover the nx columns once;
* the tile of a strip, its left halo KL = K rounded up to even (K + 1 at odd K) plus w output
  columns plus K on the right, fits the CTA's columns, so every output column has its full
  dependency cone inside the tile;
* row segments cover the ny rows once, with at most one wave of the CTA slots."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1401_0427_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

DRIVER = r"""
#include <cstdio>
#include "temporal.cuh"
int main() {
  const int cols[3] = {128, 192, 256};
  const int sizes[] = {1, 2, 3, 7, 10, 64, 115, 116, 117, 118, 127, 128, 129, 191, 192, 244, 245, 246, 250, 256,
                       257, 488, 489, 490, 500, 1023, 1024, 2049, 2900, 2901, 3002, 4095, 4096, 8192};
  for (int ci = 0; ci < 3; ++ci)
    for (int K = 2; K <= 8; ++K) {
      if ((cols[ci] - 2 * K - (K & 1)) / 2 < 1) continue;
      for (int nx : sizes)
        for (int ny : {1, 5, 17, 96, 1000, 4096}) {
          const lbm::Partition P = lbm::pair_partition(nx, ny, K, cols[ci], 304);
          std::printf("%d %d %d %d %d %d %d %d\n", cols[ci], K, nx, ny, P.w, P.strips, P.rows_per_cta, P.segments);
        }
    }
  return 0;
}
"""


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc is not available")
    d = tmp_path_factory.mktemp("partition")
    src, exe = d / "partition.cu", d / "partition"
    src.write_text(DRIVER)
    r = subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", INCLUDE, str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return [tuple(int(v) for v in line.split()) for line in out.splitlines()]


def test_strips_are_even_cover_the_width_and_fit_the_tile(rows):
    assert len(rows) > 1000
    for cols, K, nx, ny, w, strips, rows_per_cta, segments in rows:
        kl = K + (K & 1)
        assert w % 2 == 0 and w >= 2, (cols, K, nx, w)
        assert kl + w + K <= cols, (cols, K, nx, w)
        assert strips * w >= nx and (strips - 1) * w < nx, (cols, K, nx, w, strips)


def test_row_segments_cover_the_height_in_one_wave(rows):
    for cols, K, nx, ny, w, strips, rows_per_cta, segments in rows:
        assert rows_per_cta >= 1
        assert segments * rows_per_cta >= ny and (segments - 1) * rows_per_cta < ny, (cols, K, nx, ny)
        assert strips * segments <= max(304, strips), (cols, K, nx, ny, strips, segments)


def test_odd_k_tiles_start_at_even_columns(rows):
    """Strip s starts at s w (even), so its tile starts at s w - KL: even for every K."""
    for cols, K, nx, ny, w, strips, rows_per_cta, segments in rows:
        kl = K + (K & 1)
        assert all((s * w - kl) % 2 == 0 for s in range(strips))
