"""Host logic of the fine engines' z decomposition (`csrc/zchunks.h`), compiled
with the host C++ compiler and run on the CPU:

* `zchunk`: the chunks of every (Nz, n) cover the element planes 0..Nz-1 once, in
  order; their lengths differ by at most one; the last chunk also takes the
  closing node plane Nz;
* `balanced_zchunks`: chunks have at least 6 planes (one chunk when Nz < 12).
  The CTAs fill whole waves when a count with few halo planes allows it.  For the
  256^3 benchmark (128 xy tiles; 3 x 152 or 2 x 152 resident CTAs) the count is 7
  for both engines, i.e. 896 CTAs, against 2.25 waves with 32-plane chunks.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_06850_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <initializer_list>
#include "zchunks.h"
using thermo::zchunk;
using thermo::balanced_zchunks;
int main() {
  // coverage of every (Nz, n)
  for (int Nz = 1; Nz <= 300; ++Nz)
    for (int n = 1; n <= Nz; ++n) {
      int next = 0, lmin = 1 << 30, lmax = 0;
      for (int k = 0; k < n; ++k) {
        int zs, ze;
        zchunk(Nz, n, k, zs, ze);
        if (zs != next) { std::printf("GAP %d %d %d\n", Nz, n, k); return 1; }
        const int len = (k == n - 1) ? ze - zs : ze - zs + 1;  // element planes
        if (len < lmin) lmin = len;
        if (len > lmax) lmax = len;
        next = (k == n - 1) ? ze : ze + 1;
        if (k == n - 1 && ze != Nz) { std::printf("LAST %d %d\n", Nz, n); return 1; }
      }
      if (next != Nz || lmax - lmin > 1 || lmin < 1) { std::printf("LEN %d %d\n", Nz, n); return 1; }
    }
  // chunk counts
  for (int Nz = 4; Nz <= 1024; Nz += 4)
    for (long long tiles : {1LL, 8LL, 16LL, 128LL, 1024LL})
      for (long long slots : {304LL, 456LL}) {
        const int n = balanced_zchunks(tiles, slots, Nz);
        if (n < 1 || (Nz >= 12 && Nz / n < 6) || (Nz < 12 && n != 1)) {
          std::printf("COUNT %d %lld %lld %d\n", Nz, tiles, slots, n);
          return 1;
        }
      }
  std::printf("%d %d %d %d\n", balanced_zchunks(128, 456, 256), balanced_zchunks(128, 304, 256),
              balanced_zchunks(1024, 456, 512), balanced_zchunks(8, 456, 64));
  return 0;
}
"""


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("zchunks")
    src = d / "t.cpp"
    src.write_text(PROG)
    exe = d / "t"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return exe


def test_zchunks_cover_and_balance(prog):
    r = subprocess.run([str(prog)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout
    n256_q, n256_d, n512, n64 = (int(v) for v in r.stdout.split())
    assert (n256_q, n256_d) == (7, 7)  # 896 CTAs: 1.96 waves of 456, 2.95 of 304
    assert n512 == 4                   # 4096 CTAs, 8.98 waves; 128-plane chunks
    assert n64 == 10                   # under one wave: as many chunks as 6-plane chunks allow
