"""The integer-arithmetic float <-> double conversions of the CUDA path's
Krylov kernels (`csrc/fconv.h`), compiled with the host C++ compiler and
compared bit for bit with the C conversions (IEEE round to nearest, ties to
even) on seeded random encodings of every exponent, on exact ties and on
the edges of the normal float range (including overflow to infinity,
subnormal results, zeros, infinities and NaNs)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_06850_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <cfloat>
#include "fconv.h"
using namespace thermo;
static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t next() {  // SplitMix64
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static long bad = 0, n = 0;
static void check_d(double x) {
  const float a = d2f_int(x), b = (float)x;
  ++n;
  if (fconv_bits(a) != fconv_bits(b) && !(std::isnan(a) && std::isnan(b))) {
    if (bad < 5) std::printf("d2f %a -> %a expected %a\n", x, (double)a, (double)b);
    ++bad;
  }
}
static void check_f(float f) {
  const double a = f2d_int(f), b = (double)f;
  ++n;
  if (fconv_bits(a) != fconv_bits(b) && !(std::isnan(a) && std::isnan(b))) {
    if (bad < 5) std::printf("f2d %a -> %a expected %a\n", (double)f, a, b);
    ++bad;
  }
}
int main() {
  for (int i = 0; i < 4000000; ++i) check_d(fconv_double(next()));          // every exponent
  for (int i = 0; i < 4000000; ++i) {                                      // the float range
    const uint64_t r = next();
    const uint64_t e = 850 + (r % 320);
    check_d(fconv_double((r & 0x800fffffffffffffull) | (e << 52)));
  }
  for (int i = 0; i < 1000000; ++i) {                                      // exact ties and neighbours
    const uint64_t r = next();
    const uint64_t e = 897 + (r % 254);
    const uint64_t m = ((r >> 20) & 0xffffffull) << 29;
    const uint64_t base = (r & 0x8000000000000000ull) | (e << 52) | (m & 0xfffffffffffffull);
    for (int d = -1; d <= 1; ++d) check_d(fconv_double((base | 0x10000000ull) + (uint64_t)(int64_t)d));
  }
  const double edge[] = {0.0, -0.0, FLT_MAX, -FLT_MAX, (double)FLT_MAX * (1 + 0x1p-25), (double)FLT_MAX * (1 + 0x1p-23),
                         FLT_MIN, -FLT_MIN, FLT_MIN * 0.75, 0x1p-149, 0x1p-150, 1e-300, 1e300, INFINITY, -INFINITY, NAN,
                         1.0, 1.0 + 0x1p-24, 1.0 + 0x1p-24 + 0x1p-52, 1.0 + 3 * 0x1p-24};
  for (double x : edge) check_d(x);
  for (int i = 0; i < 4000000; ++i) check_f(fconv_float((uint32_t)next()));
  const float fedge[] = {0.0f, -0.0f, FLT_MIN, 0x1p-149f, FLT_MAX, INFINITY, -INFINITY, NAN};
  for (float f : fedge) check_f(f);
  std::printf("%ld %ld\n", n, bad);
  return 0;
}
"""


@pytest.fixture(scope="module")
def out(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("fconv")
    (d / "t.cpp").write_text(PROG)
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, str(d / "t.cpp"), "-o", str(d / "t")],
                   check=True)
    return subprocess.run([str(d / "t")], capture_output=True, text=True, check=True, timeout=120).stdout


def test_conversions_equal_the_c_conversions(out):
    last = out.strip().splitlines()[-1].split()
    n, bad = int(last[0]), int(last[1])
    assert n > 15_000_000
    assert bad == 0, out
