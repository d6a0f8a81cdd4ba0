"""The device Philox header on the CPU (no GPU): csrc/philox.cuh compiled as
plain C++ (its CUDA qualifiers defined away), both its forms, Philox4x32-10
from the seed (Salmon et al., SC'11: ten rounds with Weyl key increments)
and from precomputed round keys (the form one-graph handles pass as kernel
parameters), against the oracle's own Philox on random counters and seeds.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import philox4x32_10

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1804_08487_gb300", "csrc")

_PROG = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include <cinttypes>
#include <cstdio>
#include "philox.cuh"
int main() {
  unsigned long long seed;
  unsigned c0, c1, c2, c3;
  while (std::scanf("%llu %u %u %u %u", &seed, &c0, &c1, &c2, &c3) == 5) {
    const cb::Philox4 a = cb::philox4x32_10(c0, c1, c2, c3, seed);
    uint32_t ks[20];
    cb::philox_round_keys(seed, ks);
    const cb::Philox4 b = cb::philox4x32_10_rk(c0, c1, c2, c3, ks);
    std::printf("%u %u %u %u %u %u %u %u\n", a.w0, a.w1, a.w2, a.w3, b.w0, b.w1, b.w2, b.w3);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def header_prog(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("philox_header")
    src, exe = d / "philox_host.cpp", d / "philox_host"
    src.write_text(_PROG)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return exe


def test_round_key_form_equals_seed_form_and_the_oracle(header_prog):
    rng = np.random.default_rng(20180423)
    cases = [(0, 0, 0, 0, 0), (2**64 - 1, 2**32 - 1, 2**32 - 1, 2**32 - 1, 2**32 - 1), (42, 7, 9, 3, 1)]
    for _ in range(200):
        seed = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        cases.append((seed,) + tuple(int(x) for x in rng.integers(0, 2**32, size=4)))
    text = "".join(" ".join(str(v) for v in case) + "\n" for case in cases)
    out = subprocess.run([str(header_prog)], input=text, capture_output=True, text=True, check=True).stdout
    lines = out.strip().splitlines()
    assert len(lines) == len(cases)
    for case, line in zip(cases, lines):
        got = [int(v) for v in line.split()]
        want = [int(v) for v in philox4x32_10(case[1:], case[0])]
        assert got[:4] == want, case     # the seed form
        assert got[4:] == want, case     # the round-key form
