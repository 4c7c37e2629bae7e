"""Host-side layout of the persistent kernel's work list (batches and server rounds), checked on the CPU.

The persistent stage kernel hands CTA c of G the entries c, c + G, c + 2G, ... of the work list.  The
helpers in csrc/alw_params2d.h reorder an instance-major list so that each CTA takes blocks of R
consecutive entries (cta_blocks) or one contiguous stretch (cta_runs); both must be permutations, and
stage2d_grid must never launch more CTAs than entries or than fit.  A small host program includes the
header and prints the layouts.
"""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1909_13263_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r"""
#include "alw_params2d.h"
#include <cstdio>
#include <cstdlib>
#include <cstring>
int main(int argc, char **argv) {
  if (argc == 4 && !strcmp(argv[1], "grid")) {
    printf("%d\n", alw::stage2d_grid(atoi(argv[2]), atoi(argv[3]), 304));
    return 0;
  }
  const int n = atoi(argv[2]), G = atoi(argv[3]), R = atoi(argv[4]);
  std::vector<int> in(n), out;
  for (int i = 0; i < n; ++i) in[i] = 1000 + i;
  if (!strcmp(argv[1], "runs")) alw::cta_runs(in, G, out);
  else alw::cta_blocks(in, G, R, out);
  for (int v : out) printf("%d ", v);
  printf("\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("worklist")
    src, exe = d / "wl.cpp", d / "wl"
    src.write_text(PROGRAM)
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _layout(prog, mode, n, G, R=1):
    out = subprocess.run([prog, mode, str(n), str(G), str(R)], check=True, capture_output=True, text=True).stdout
    return [int(v) - 1000 for v in out.split()]


@pytest.mark.parametrize("n,G", [(1, 304), (10, 3), (303, 304), (304, 304), (1000, 304), (49460, 304), (7, 7)])
def test_cta_runs_gives_each_cta_one_stretch(prog, n, G):
    lay = _layout(prog, "runs", n, G)
    assert sorted(lay) == list(range(n))
    start = 0
    for c in range(min(G, n)):
        mine = lay[c::G]
        assert mine == list(range(start, start + len(mine)))   # one contiguous stretch, in order
        start += len(mine)


@pytest.mark.parametrize("n,G,R", [(10, 3, 2), (1000, 304, 4), (49460, 304, 4), (5000, 304, 8), (300, 304, 4),
                                   (17, 4, 1)])
def test_cta_blocks_is_a_permutation_of_blocks(prog, n, G, R):
    lay = _layout(prog, "blocks", n, G, R)
    assert sorted(lay) == list(range(n))
    if R == 1:
        assert lay == list(range(n))
    # in the rounds where every block is complete, CTA c takes R consecutive entries per turn
    full_rounds = n // (G * R)
    for c in range(G):
        mine = lay[c::G]
        for r in range(full_rounds):
            block = mine[r * R:(r + 1) * R]
            assert block == list(range(r * G * R + c * R, r * G * R + c * R + R))


def test_stage2d_grid_bounds(prog):
    def grid(ntiles, ctas):
        out = subprocess.run([prog, "grid", str(ntiles), str(ctas)], check=True, capture_output=True, text=True)
        return int(out.stdout)
    assert grid(10, 0) == 10          # never more CTAs than entries
    assert grid(5000, 0) == 304       # as many as fit
    assert grid(5000, 100) == 100     # a requested count below the cap
    assert grid(5000, 1000) == 304    # capped
