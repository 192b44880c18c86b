"""The split-precision GEMM's MMA schedule (`oz_schedule` in csrc/ozaki.h), on CPU.

Per 16-wide K step the GEMM multiplies every pair of A and B digit slices (k, l), 1-based, whose weight
2^(-7(k+l-2)) is kept (k + l <= S + 1): S(S+1)/2 products.  They accumulate into four TMEM regions:
region k+l-2 for the exact groups of one weight each (0, 1, 2), region 3 for the rounded tail.  The
schedule is a compile-time list of MMAs.  Each MMA covers one product, or two products of adjacent B
slices landing in adjacent regions (one N = 2H MMA).  An MMA overwrites its region(s) when it is the
first write of the chunk, else it accumulates.  The checks below derive all of this from that
definition, for every S the kernels instantiate, with and without fusion.  Planted mistakes in a copy of
the header must fail them.  The test compiles the header as host code with nvcc; it runs no GPU code."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2201_01257_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "ozaki.h"
int main() {
  printf("const %d %d %d\n", tamm::kOzMaxOps, tamm::kOzChunkTiles, tamm::kOzTileK);
  for (int S = 3; S <= 8; ++S)
    for (int f = 0; f < 2; ++f) {
      const tamm::OzSched s = tamm::oz_schedule(S, f != 0);
      printf("sched %d %d %d\n", S, f, s.n);
      for (int i = 0; i < s.n; ++i)
        printf("op %d %d %d %d %d\n", s.op[i].a, s.op[i].b, s.op[i].nb, s.op[i].region, s.op[i].first);
    }
  return 0;
}
"""


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    pytest.skip("nvcc not found")


def _schedules(tmp_path, header_dir=None):
    src = tmp_path / "sched.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "sched"
    inc = ([f"-I{header_dir}"] if header_dir else []) + [f"-I{CSRC}"]
    subprocess.run([_nvcc(), "-std=c++17", *inc, "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    consts, scheds, cur = None, {}, None
    for ln in out:
        f = ln.split()
        if not f:
            continue
        if f[0] == "const":
            consts = tuple(int(x) for x in f[1:])
        elif f[0] == "sched":
            cur = scheds.setdefault((int(f[1]), bool(int(f[2]))), [])
        else:
            cur.append(tuple(int(x) for x in f[1:]))
    return consts, scheds


def check_schedule(S, fuse, ops, max_ops):
    """Every kept product exactly once, in its region, fused only as the definition allows, with the
    first-write flags of a chunk's first K step; raises AssertionError on the first violation."""
    assert 0 < len(ops) <= max_ops, (S, fuse, len(ops))
    want = {(k, l) for k in range(1, S + 1) for l in range(1, S + 2 - k)}
    assert len(want) == S * (S + 1) // 2
    seen = []
    written = [False] * 4
    for a, b, nb, region, first in ops:
        assert nb in (1, 2) and 0 <= region <= 3
        assert fuse or nb == 1, "fused MMA in the unfused schedule"
        prods = [(a + 1, b + 1)] + ([(a + 1, b + 2)] if nb == 2 else [])
        for j, (k, l) in enumerate(prods):
            assert (k, l) in want, ("product outside the kept set", S, k, l)
            assert region + j == min(k + l - 2, 3), ("wrong region", S, k, l, region + j)
        regs = [region + j for j in range(nb)]
        if nb == 2:
            assert regs[1] <= 3 and regs[0] <= 2
            assert written[regs[0]] == written[regs[1]], "one flag for two regions of different status"
        assert first == (0 if written[regs[0]] else 1), ("first-write flag", S, fuse, a, b)
        for r in regs:
            written[r] = True
        seen += prods
    assert sorted(seen) == sorted(want), ("products missing or repeated", S, fuse)
    # the exact regions hold products of one weight: region r <= 2 receives exactly the r + 1 products
    # with k + l = r + 2
    for r in range(3):
        assert sum(1 for k, l in seen if min(k + l - 2, 3) == r) == r + 1


def test_schedules_cover_every_kept_product_once(tmp_path):
    (max_ops, chunk_tiles, tile_k), scheds = _schedules(tmp_path)
    assert len(scheds) == 12
    for (S, fuse), ops in scheds.items():
        check_schedule(S, fuse, ops, max_ops)
    # fusion saves MMAs from S = 3 on (products of the exact groups share N = 2H MMAs)
    for S in range(3, 9):
        assert len(scheds[(S, True)]) < len(scheds[(S, False)]) == S * (S + 1) // 2


def test_exact_chunk_bound(tmp_path):
    """The exact groups stay exact over the longest chunk: at most 3 products per element of G2, digits of
    magnitude at most 64, so 3 * K * 64 * 64 < 2^24 for K = the largest chunk."""
    (_, chunk_tiles, tile_k), _ = _schedules(tmp_path)
    assert 3 * chunk_tiles * tile_k * 64 * 64 < 2 ** 24


MUTANTS = {
    # region of (k, l) one weight too high
    "region_off_by_one": ("const int region = k + l - 2 < 3 ? k + l - 2 : 3;",
                          "const int region = k + l - 1 < 3 ? k + l - 1 : 3;"),
    # the last kept product of every row dropped
    "drops_products": ("while (l <= S + 1 - k) {", "while (l <= S - k) {"),
    # a fused pair issued as one product (its second product is skipped)
    "pair_drops_second": ("o.nb = pair ? 2 : 1;", "o.nb = 1;"),
    # B slice index off by one
    "b_slice_off_by_one": ("o.b = l - 1;", "o.b = l;"),
    # every MMA accumulates (no overwrite at a chunk's start)
    "never_first": ("o.first = written[region] ? 0 : 1;", "o.first = 0;"),
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_checks_catch_planted_schedule_mistakes(mutant, tmp_path):
    old, new = MUTANTS[mutant]
    src = open(os.path.join(CSRC, "ozaki.h")).read()
    assert src.count(old) == 1, mutant
    hdr = tmp_path / "hdr"
    hdr.mkdir()
    (hdr / "ozaki.h").write_text(src.replace(old, new))
    (max_ops, _, _), scheds = _schedules(tmp_path, header_dir=str(hdr))
    caught = False
    for (S, fuse), ops in scheds.items():
        try:
            check_schedule(S, fuse, ops, max_ops)
        except AssertionError:
            caught = True
            break
    assert caught, f"planted mistake {mutant!r} was not caught"
