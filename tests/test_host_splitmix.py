"""The CUDA path's own counter-based SplitMix64 (`csrc/splitmix.h`, the start
vector of the set-up's power iteration), compiled with the host C++ compiler:

* stream 0 reproduces SplitMix64's published outputs from state 0;
* its uniforms equal those of the input generator (`workloads`), which the
  oracle uses.  The two are separate implementations of the same published
  definition: the CUDA path and the oracle share no generator code.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_06850_gb300", "csrc")

PUBLISHED = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
IDX = [0, 1, 2, 17, 1000, 123456789, 16974592]

PROG = r"""
#include <cstdio>
#include "splitmix.h"
int main() {
  for (unsigned long long i = 0; i < 3; ++i) std::printf("%llu\n", thermo::splitmix64_at(0, i));
  const unsigned long long idx[] = {0ull, 1ull, 2ull, 17ull, 1000ull, 123456789ull, 16974592ull};
  for (unsigned long long i : idx) std::printf("%.17g\n", thermo::splitmix_u01(101, i));
  return 0;
}
"""


@pytest.fixture(scope="module")
def out(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("splitmix")
    (d / "t.cpp").write_text(PROG)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(d / "t.cpp"), "-o", str(d / "t")], check=True)
    return subprocess.run([str(d / "t")], capture_output=True, text=True, check=True, timeout=60).stdout.split()


def test_stream_zero_is_the_published_sequence(out):
    assert [int(v) for v in out[:3]] == PUBLISHED


def test_uniforms_equal_the_input_generator(out):
    got = np.array([float(v) for v in out[3:]])
    ref = np.array([W.uniform01_at(101, i) for i in IDX])
    np.testing.assert_array_equal(got, ref)
