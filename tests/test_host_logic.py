"""Host-side checks of decision helpers that the library's host loops and kernels share
(`__host__ __device__` functions in the CUDA headers), compiled by nvcc into a small host
program and run on the CPU: no GPU and no kernel launch.

- `class_q` / `class_rep` / `class_count` (sl_common.cuh): the boundary-distance classes that
  index the fine stencil tables.  Two coordinates may share a table entry only if their
  truncation geometry is the same, i.e. the same distance to each boundary up to the band
  width B; every class has a representative that maps back to it.
- `ir_next_recursive` (sl_launch.h): where a refinement round of mixed precision starts.  The
  inner residual may be handed on only while it is above twice the stop threshold, within four
  orders of magnitude of the last true residual, and for at most max_rec rounds in a row.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1605_04821_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "sl_launch.h"
using namespace sl;
int main() {
  // classes: n, B, then per coordinate i in [1, n-2]: class_q; then class_rep of every class
  const int cases[][2] = {{9, 2}, {17, 4}, {33, 5}, {12, 6}, {7, 4}, {65, 16}};
  for (const auto &c : cases) {
    const int n = c[0], B = c[1];
    std::printf("C %d %d %d", n, B, class_count(n, B));
    for (int i = 1; i <= n - 2; ++i) std::printf(" %d", class_q(i, n, B));
    std::printf(" |");
    for (int q = 0; q < class_count(n, B); ++q) std::printf(" %d", class_rep(q, n, B));
    std::printf("\n");
  }
  // refinement decisions: inner_rr, tol, bn2, rr_true, rec_rounds, max_rec
  const double r[][6] = {
      {3e-24, 1e-12, 1.0, 1e-20, 0, 3},    // below 2 tol ||F|| (4e-24): true residual
      {5e-24, 1e-12, 1.0, 1e-20, 0, 3},    // above it, far above 1e-8 of the last true one
      {0.9e-16, 1e-12, 1.0, 1e-8, 0, 3},   // more than four orders below the last true one
      {1.1e-16, 1e-12, 1.0, 1e-8, 0, 3},   // just within four orders
      {1e-10, 1e-12, 1.0, 1e-8, 3, 3},     // max_rec rounds in a row already
      {1e-10, 1e-12, 1.0, 1e-8, 2, 3},
      {1e-10, 1e-12, 1.0, 1e-8, 0, 0},     // option off
  };
  for (const auto &a : r)
    std::printf("R %d\n", ir_next_recursive(a[0], a[1], a[2], a[3], int(a[4]), int(a[5])) ? 1 : 0);
  return 0;
}
"""


@pytest.fixture(scope="module")
def output(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("hostlogic")
    src, exe = os.path.join(d, "prog.cu"), os.path.join(d, "prog")
    with open(src, "w") as f:
        f.write(PROGRAM)
    r = subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                        "-o", exe, src], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0
    return r.stdout.splitlines()


def test_classes_identify_the_truncation_geometry(output):
    for line in (l for l in output if l.startswith("C ")):
        head, reps = line[2:].split("|")
        vals = [int(v) for v in head.split()]
        n, B, count = vals[:3]
        q = {i: vals[3 + i - 1] for i in range(1, n - 1)}
        rep = [int(v) for v in reps.split()]
        assert len(rep) == count
        # class 0 is the boundary coordinate itself; the interior uses classes 1 .. count-1
        assert set(q.values()) == set(range(1, count))
        geom = {i: (min(i, B), min(n - 1 - i, B)) for i in range(1, n - 1)}
        for i in q:
            for j in q:
                assert (q[i] == q[j]) == (geom[i] == geom[j]), (n, B, i, j)
        assert rep[0] == 0
        for c in range(1, count):
            assert 1 <= rep[c] <= n - 2 and q[rep[c]] == c, (n, B, c, rep[c])


def test_refinement_round_start(output):
    got = [int(l.split()[1]) for l in output if l.startswith("R ")]
    assert got == [0, 1, 0, 1, 0, 1, 0]
