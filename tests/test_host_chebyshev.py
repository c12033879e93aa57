"""The library's Chebyshev smoother coefficients (`csrc/chebyshev.h`, host code
of the set-up), compiled with the host C++ compiler, against the oracle's
(`oracle.mmg.chebyshev_coefficients`).  The oracle's are pinned to the scaled
Chebyshev polynomial in tests/test_oracle_mmg.py."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import mmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_06850_gb300", "csrc")
CASES = [(1.53, 30.0, 5), (2.0, 30.0, 4), (1.1, 10.0, 8), (0.7, 100.0, 1), (1.9, 30.0, 64)]

PROG = r"""
#include <cstdio>
#include "chebyshev.h"
int main() {
  const double cases[][3] = {%s};
  for (const auto& c : cases) {
    double a[64], b[64];
    const int m = (int)c[2];
    thermo::chebyshev_coefficients(c[0], c[1], m, a, b);
    for (int k = 0; k < m; ++k) std::printf("%%.17g %%.17g\n", a[k], b[k]);
  }
  return 0;
}
""" % ", ".join("{%r, %r, %d}" % c for c in CASES)


def test_library_coefficients_equal_the_oracle(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    (tmp_path / "t.cpp").write_text(PROG)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(tmp_path / "t.cpp"), "-o", str(tmp_path / "t")],
                   check=True)
    out = subprocess.run([str(tmp_path / "t")], capture_output=True, text=True, check=True, timeout=60).stdout
    vals = np.array([float(v) for v in out.split()]).reshape(-1, 2)
    ref = []
    for lmax, ratio, m in CASES:
        a, b = mmg.chebyshev_coefficients(lmax, ratio, m)
        ref += list(zip(a, b))
    np.testing.assert_allclose(vals, np.array(ref), rtol=1e-15, atol=0)
