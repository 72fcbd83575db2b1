"""CPU checks of the launcher's host-side arithmetic (no GPU): the shared-
memory carveout request.  The helper is header-only C++; it is compiled here
with the host compiler against the CUDA headers and run on a table of cases."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1007_3818_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

# (bytes the blocks need per SM, shared memory per SM) -> expected percent.
# 233,472 B (228 KB) is the sm_100 family's largest carveout.
SM = 233472
CASES = [
    (3 * (65664 + 1024), SM, 85),   # fused level kernel, 3 CTAs: 196 KB
    (3 * (63104 + 1024), SM, 85),   # tile kernel, 3 CTAs: 196 KB
    (3 * (76784 + 1024), SM, 100),  # over 196 KB: only the largest holds it
    (2 * (71136 + 1024), SM, 71),   # 144.3 KB: 164 KB
    (0, SM, 0),
    (8 * 1024, SM, 3),              # exactly a supported capacity
    (8 * 1024 + 1, SM, 7),          # one byte more: the next one (16 KB)
    (1000, 0, 100),                 # unknown SM size: no preference
]

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include "abi_common.h"
int main(int argc, char** argv) {
    for (int i = 1; i + 1 < argc; i += 2)
        std::printf("%d\n", gamer::carveout_percent(std::atoll(argv[i]), std::atoi(argv[i + 1])));
    return 0;
}
"""


def _capacity_kb(pct, sm):
    """The capacity a percentage selects under the driver's rounding up."""
    caps = [0, 8, 16, 32, 64, 100, 132, 164, 196, 228]
    want = pct * sm / 100.0
    return next(c for c in caps if c * 1024 >= want)


@pytest.fixture(scope="module")
def helper(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("no host C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("carveout")
    src = d / "carveout.cpp"
    src.write_text(PROGRAM)
    exe = d / "carveout"
    subprocess.run([gxx, "-std=c++17", "-O1", f"-I{CSRC}", f"-I{CUDA_INC}",
                    f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)], check=True)
    return exe


def test_carveout_percent_table(helper):
    args = [str(v) for need, sm, _ in CASES for v in (need, sm)]
    out = subprocess.run([str(helper)] + args, check=True, capture_output=True,
                         text=True).stdout.split()
    assert [int(x) for x in out] == [pct for _, _, pct in CASES]


def test_carveout_percent_selects_a_capacity_that_holds_the_blocks(helper):
    """For every need up to the largest capacity, the capacity the returned
    percentage rounds up to holds the blocks and is the smallest that does."""
    needs = list(range(0, SM, 997))
    args = [str(v) for n in needs for v in (n, SM)]
    out = [int(x) for x in subprocess.run([str(helper)] + args, check=True,
                                          capture_output=True, text=True).stdout.split()]
    caps = [0, 8, 16, 32, 64, 100, 132, 164, 196, 228]
    for need, pct in zip(needs, out):
        smallest = next(c for c in caps if c * 1024 >= need)
        got = 228 if pct == 100 else _capacity_kb(pct, SM)
        assert got * 1024 >= need and got == smallest, (need, pct, got, smallest)
