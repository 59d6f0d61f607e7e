"""Host logic of time blocking (depth 2), checked on the CPU.

The header functions the library schedules with are compiled here into a
small host program:
* `set_of`: the field set holding the state after n steps.
* `pair_split`: how fdtd_step splits n steps into a leading single step,
  pairs and trailing single steps.
* `rename_sets`: how the sets are renamed when the depth changes.

The program checks the properties the GPU path relies on:
* Consecutive states never share a set.
* At depth 2 the even states alternate between sets 0 and 1 and the odd
  states use set 2, so a pass reads one set and writes another.
* Every pair starts at an even step.
* The last step of a call is a single step, so the states after the last
  two steps are complete.
* A renaming is a permutation that moves the last two states to where the
  new depth expects them.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1008_2602_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "fdtd_internal.h"
using namespace fdtd;
int main()
{
    int bad = 0;
    for (int d = 1; d <= 2; ++d)
        for (long long n = -1; n < 64; ++n)
            bad += set_of(d, n) == set_of(d, n + 1);                  // a step reads one set, writes another
    for (long long n = 0; n < 64; n += 2) {
        bad += set_of(2, n) == 2 || set_of(2, n + 1) != 2;            // odd states in set 2 only
        bad += set_of(2, n) == set_of(2, n + 2);                       // the pass reads A, writes A'
    }
    for (long long s = 0; s < 12; ++s)
        for (int n = 0; n < 80; ++n) {
            const PairSplit p = pair_split(s, n);
            bad += p.lead + 2 * p.pairs + p.tail != n;                 // every step runs once
            bad += p.lead < 0 || p.pairs < 0 || p.tail < 0 || p.lead > 1 || p.tail > 2;
            bad += p.pairs > 0 && ((s + p.lead) & 1) != 0;             // pairs start at even steps
            bad += n > 0 && p.tail == 0 && p.lead != n;                // the last step is a single one
            bad += (s & 1) == 0 && p.lead != 0;
        }
    for (int d0 = 1; d0 <= 2; ++d0)
        for (int d1 = 1; d1 <= 2; ++d1)
            for (long long n = 0; n < 16; ++n) {
                int perm[3] = {-1, -1, -1};
                rename_sets(d0, d1, n, perm);
                int seen = 0;
                for (int x = 0; x < 3; ++x) {
                    bad += perm[x] < 0 || perm[x] > 2;
                    if (perm[x] >= 0 && perm[x] <= 2) seen |= 1 << perm[x];
                }
                bad += seen != 7;                                      // a permutation
                bad += perm[set_of(d1, n)] != set_of(d0, n);           // state n moves to its new set
                bad += perm[set_of(d1, n - 1)] != set_of(d0, n - 1);   // and state n - 1
                if (d0 == d1) bad += perm[0] != 0 || perm[1] != 1 || perm[2] != 2;
            }
    std::printf("%d\n", bad);
    return bad;
}
"""


def test_pair_schedule_and_set_renaming(tmp_path):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda.h")):
        pytest.skip("g++ and the CUDA headers are needed to compile the host check")
    src = tmp_path / "sched.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "sched"
    subprocess.run([gxx, "-std=c++17", "-I", CSRC, "-I", cuda_inc, "-o", str(exe), str(src)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "0", r.stdout
