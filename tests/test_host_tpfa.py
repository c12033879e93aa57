"""The CUDA path's TPFA per-cell arithmetic (`csrc/tpfa.h`: the rows of the
paper's Sec. 2.2 operator, the right-hand side with the design-dependent source
of Sec. 2.1, the mean-temperature adjoint sensitivity of Sec. 2.3), compiled
with the host C++ compiler and compared with the oracle (oracle/tpfa.py,
pinned in tests/test_oracle_tpfa.py) on a ragged grid with Dirichlet faces on
several sides and a non-uniform T_D-weighted right-hand side:

* (A t)_c within 1e-13 of the oracle's assembled product, relative to (|A||t|)_c;
* b and the sensitivity within 1e-12 (relative to their scales).
The two are separate implementations: the oracle assembles sparse matrices,
the kernel evaluates each row from its six neighbours."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import tpfa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_06850_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <vector>
#include "tpfa.h"
using namespace thermo;
int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "rb");
  int n3[3];
  double par[9];
  if (std::fread(n3, sizeof(int), 3, f) != 3 || std::fread(par, sizeof(double), 9, f) != 9) return 1;
  TpfaGrid g{n3[0], n3[1], n3[2], par[0], par[1], par[2]};
  const double p = par[3], kmin = par[4], kmax = par[5], f0 = par[6], TD = par[7];
  const long long M = (long long)g.nx * g.ny * g.nz;
  std::vector<double> kappa(M), t(M), u(M), x(M);
  std::vector<unsigned char> m(M);
  if (std::fread(kappa.data(), 8, M, f) != (size_t)M || std::fread(m.data(), 1, M, f) != (size_t)M ||
      std::fread(t.data(), 8, M, f) != (size_t)M || std::fread(u.data(), 8, M, f) != (size_t)M ||
      std::fread(x.data(), 8, M, f) != (size_t)M) return 2;
  std::fclose(f);
  FILE* o = std::fopen(argv[2], "wb");
  for (long long c = 0; c < M; ++c) {
    double v[3] = {tpfa_row(g, kappa.data(), m.data(), t.data(), c),
                   tpfa_rhs(g, x[c], p, f0, kappa[c], m[c], TD),
                   tpfa_sens(g, kappa.data(), m.data(), x.data(), p, kmin, kmax, f0, TD, t.data(), u.data(), c)};
    std::fwrite(v, 8, 3, o);
  }
  std::fclose(o);
  return 0;
}
"""


def _faces_to_bits(grid, dfaces):
    M = grid[0] * grid[1] * grid[2]
    bits = np.zeros(M, dtype=np.uint8)
    for (axis, side), m in dfaces.items():
        bits[m] |= np.uint8(1 << (2 * axis + side))
    return bits


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("tpfa")
    (d / "t.cpp").write_text(PROG)
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(d / "t.cpp"), "-o", str(d / "t")], check=True)
    return d


@pytest.mark.parametrize("p,TD", [(3.0, 100.0), (1.0, 0.0)])
def test_kernel_arithmetic_matches_oracle(exe, p, TD):
    grid = (7, 5, 6)
    h = (0.3, 0.5, 0.7)
    M = grid[0] * grid[1] * grid[2]
    x = 0.05 + 0.95 * W.uniform01(91, M)
    # Dirichlet faces: the z = 0 patch, the whole +x face and part of the -y face
    dfaces = tpfa.dirichlet_faces(grid, "z0", half_width=0.25)
    cell = np.arange(M)
    i, j, k = cell % grid[0], (cell // grid[0]) % grid[1], cell // (grid[0] * grid[1])
    dfaces[(0, 1)] = i == grid[0] - 1
    dfaces[(1, 0)] = (j == 0) & (k < 3)
    P = tpfa.build(grid, h, x, p, 1e-3, 1.0, 1.0, dfaces, TD=TD)
    t = W.uniform01(92, M) * 50.0
    u = W.uniform01(93, M) - 0.5
    bits = _faces_to_bits(grid, dfaces)
    inp = exe / "in.bin"
    with open(inp, "wb") as f:
        f.write(np.array(grid, dtype=np.int32).tobytes())
        f.write(np.array([*h, p, 1e-3, 1.0, 1.0, TD, 0.0], dtype=np.float64).tobytes())
        f.write(P["kappa"].astype(np.float64).tobytes())
        f.write(bits.tobytes())
        f.write(t.tobytes())
        f.write(u.tobytes())
        f.write(x.tobytes())
    out = exe / "out.bin"
    subprocess.run([str(exe / "t"), str(inp), str(out)], check=True, timeout=60)
    y, b, g = np.fromfile(out, dtype=np.float64).reshape(M, 3).T
    A = P["A"]
    scale = abs(A) @ np.abs(t)
    assert np.max(np.abs(y - A @ t) / scale) <= 1e-13
    np.testing.assert_allclose(b, P["b"], rtol=1e-13, atol=0)
    ref = tpfa.sensitivity(P, t, u)
    assert np.max(np.abs(g - ref)) <= 1e-12 * np.max(np.abs(ref)), np.max(np.abs(g - ref))
