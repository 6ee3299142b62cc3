"""Host checks of the factorised predictor's compile-time enumerations
(csrc/predict_index.cuh): the packed constants and index functions that its
item loops decode must reproduce the mode orderings the tables and probes use
(spatial modes c outermost, then b, then a; space-time modes e outermost), and
the projection axes must take, for every direction d and variable 1 + v', the
right flux entry with the two axes other than d in the order the last step
expects.  A small host program (nvcc, no GPU needed) prints every decoded value;
the expected values are built here from the definitions."""
import os
import shutil
import subprocess
import tempfile

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2211_13295_gb300", "csrc")

PROGRAM = r'''
#include <cstdio>
#include "predict_index.cuh"
using namespace awe;
int main() {
  for (int t = 0; t < 10; ++t)
    printf("tri2 %d %d %d %d %d\n", t, unpack(kTri2P, 2, t), unpack(kTri2Q, 2, t), unpack(kTri2R, 2, t),
           tri2_fast(unpack(kTri2P, 2, t), unpack(kTri2Q, 2, t), unpack(kTri2R, 2, t)));
  for (int b = 0; b < 15; ++b) {
    int a = unpack(kGmA, 2, b), bb = unpack(kGmB, 2, b), c = unpack(kGmC, 2, b), e = unpack(kGmE, 2, b);
    printf("gm %d %d %d %d %d %d %d\n", b, a, bb, c, e, gm_fast(a, bb, c, e), gmidx(a, bb, c, e));
  }
  for (int c = 0; c <= 3; ++c)
    for (int b = 0; b <= 3 - c; ++b) {
      printf("p3 %d %d %d\n", b, c, p3idx(b, c));
      for (int a = 0; a <= 3 - b - c; ++a) printf("s3 %d %d %d %d\n", a, b, c, simplex_idx(3, a, b, c));
    }
  for (int pe = 0; pe < 6; ++pe) printf("p2 %d %d %d %d\n", pe, pair2_p(pe), pair2_e(pe), p2idx(pair2_p(pe), pair2_e(pe)));
  for (int r = 0; r < 9; ++r) printf("c1 %d %d\n", r, unpack(kP1C1, 4, r));
  for (int dv = 0; dv < 12; ++dv)
    printf("dv %d %d %d %d\n", dv, unpack(kP2Row, 4, dv), unpack(kP2Lo, 4, dv), unpack(kP2Swap, 4, dv));
  return 0;
}
'''


@pytest.fixture(scope="module")
def decoded():
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "idx.cu")
        with open(src, "w") as f:
            f.write(PROGRAM)
        exe = os.path.join(d, "idx")
        subprocess.run([nvcc, "-std=c++17", "-I", CSRC, src, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = {}
    for line in out.splitlines():
        k, *vals = line.split()
        rows.setdefault(k, []).append(tuple(int(v) for v in vals))
    return rows


def tri2_order():
    return [(p, q, r) for r in range(3) for q in range(3 - r) for p in range(3 - r - q)]


def gm_order():
    return [(a, b, c, e) for e in range(3) for c in range(3 - e) for b in range(3 - e - c)
            for a in range(3 - e - b - c)]


def test_triples_decode_to_their_enumeration(decoded):
    order = tri2_order()
    for t, p, q, r, fast in decoded["tri2"]:
        assert (p, q, r) == order[t]
        assert fast == t


def test_gmodes_decode_to_the_space_time_enumeration(decoded):
    order = gm_order()
    assert len(decoded["gm"]) == 15
    for b, a, bb, c, e, fast, idx in decoded["gm"]:
        assert (a, bb, c, e) == order[b]
        assert fast == b and idx == b


def test_pair_and_simplex_indices(decoded):
    pairs = [(b, c) for c in range(4) for b in range(4 - c)]
    for b, c, i in decoded["p3"]:
        assert pairs[i] == (b, c)
    modes = [(a, b, c) for c in range(4) for b in range(4 - c) for a in range(4 - b - c)]
    for a, b, c, i in decoded["s3"]:
        assert modes[i] == (a, b, c)
    pe_order = [(p, e) for e in range(3) for p in range(3 - e)]
    for pe, p, e, i in decoded["p2"]:
        assert (p, e) == pe_order[pe] and i == pe


def test_projection_axes_take_the_right_flux_entry(decoded):
    c1 = {r: c for r, c in decoded["c1"]}
    for dv, r, lo, swap in decoded["dv"]:
        d, v = divmod(dv, 4)
        # row sets: 0-2 diagonal momentum flux of direction r, 3-5 off-diagonal
        # (0,1), (0,2), (1,2), 6-8 energy flux of direction r - 6
        if v == 3:
            assert r == 6 + d
        elif v == d:
            assert r == d
        else:
            assert r == 3 + [(0, 1), (0, 2), (1, 2)].index(tuple(sorted((d, v))))
        # P1 contracts an axis other than d; an off-diagonal entry's P1 axis is
        # the one neither of its directions, so both directions share it
        assert c1[r] != d
        if 3 <= r <= 5:
            assert c1[r] == 3 - d - v
        rest = sorted({0, 1, 2} - {c1[r]})        # the two axes P1 leaves, lower first
        assert lo == (d == rest[0])
        c2 = rest[1] if d == rest[0] else rest[0]  # the axis P2 contracts
        assert {c1[r], c2, d} == {0, 1, 2}
        assert swap == (c2 > c1[r])
