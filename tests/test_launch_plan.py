"""The launch plan of lbm_sw_step on fused handles (csrc/launch_plan.h), host code only:
compiled here into a small program with the address and undefined-behaviour sanitizers,
and run for every K, both kinds of sides and every step count up to 3000, in the way
lbm_sw_step calls it (plan buffers of 64 launches, called again until n is covered).

Every plan must cover exactly n steps, use only sizes the kernels provide (at most K: K itself,
even sizes, other odd sizes above one only with every side periodic), run the bulk
as launches of K, and use at most one single step (with even fused sizes only, only for an
odd step count)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1401_0427_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "launch_plan.h"
int main() {
  for (int K = 2; K <= 8; ++K)
    for (int odd = 0; odd <= 1; ++odd)
      for (int n = 0; n <= 3000; ++n) {
        std::printf("%d %d %d:", K, odd, n);
        int left = n, plan[64];
        while (left > 0) {
          const int c = lbm::plan_launches(K, odd != 0, left, plan, 64);
          if (c <= 0) { std::printf(" STUCK"); break; }
          for (int i = 0; i < c; ++i) { std::printf(" %d", plan[i]); left -= plan[i]; }
        }
        std::printf("\n");
      }
  return 0;
}
"""


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("plan")
    src, exe = d / "plan.cpp", d / "plan"
    src.write_text(DRIVER)
    flags = ["-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]
    r = subprocess.run([gxx, *flags, "-I", CSRC, str(src), "-o", str(exe)], capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        r = subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], capture_output=True,
                           text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    table = {}
    for line in out.splitlines():
        head, sizes = line.split(":")
        K, odd, n = (int(v) for v in head.split())
        table[(K, odd, n)] = [int(v) if v != "STUCK" else -1 for v in sizes.split()]
    return table


def test_every_plan_covers_its_steps_with_sizes_the_kernels_provide(plans):
    for (K, odd, n), sizes in plans.items():
        assert -1 not in sizes, (K, odd, n)
        assert sum(sizes) == n, (K, odd, n, sizes)
        for k in sizes:
            assert 1 <= k <= K, (K, odd, n, sizes)
            assert k in (1, K) or k % 2 == 0 or odd, (K, odd, n, sizes)


def test_the_bulk_runs_launches_of_k(plans):
    for (K, odd, n), sizes in plans.items():
        tail = [k for k in sizes]
        while tail and tail[0] == K:
            tail.pop(0)
        assert sum(tail) <= K + 8, (K, odd, n, sizes)


def test_at_most_one_single_step(plans):
    for (K, odd, n), sizes in plans.items():
        ones = sizes.count(1)
        assert ones <= 1, (K, odd, n, sizes)
        if ones and K % 2 == 0 and not odd:  # only even fused sizes: an odd count needs it
            assert n % 2 == 1, (K, odd, n, sizes)


@pytest.mark.parametrize("n,want", [(20, [6, 6, 4, 4]), (22, [6, 6, 6, 4]), (8, [4, 4]), (6, [6]), (2, [2]),
                                    (12, [6, 6]), (14, [6, 4, 4])])
def test_known_plans_at_k6(plans, n, want):
    assert plans[(6, 1, n)] == want and plans[(6, 0, n)] == want


def test_long_runs(plans):
    assert plans[(6, 1, 1000)] == [6] * 166 + [4]
    assert plans[(6, 1, 2000)] == [6] * 332 + [4, 4]
    assert plans[(4, 0, 1000)] == [4] * 250
    assert plans[(6, 1, 23)] == [6, 6, 6, 5] and plans[(6, 0, 23)] == [6, 6, 6, 4, 1]
