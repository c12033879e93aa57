// z decomposition of the fine engines: ragged chunks of node planes, and the
// chunk count that fills whole waves of resident CTAs.  Plain C++ (also
// compiled by the host-logic tests without CUDA).
#pragma once
#include <cmath>

#ifdef __CUDACC__
#define ZCH_HD __host__ __device__ __forceinline__
#else
#define ZCH_HD inline
#endif

namespace thermo {

// z chunk k of n over Nz element planes (lengths differ by at most one plane):
// node planes zs..ze; the last chunk also takes the closing node plane Nz
ZCH_HD void zchunk(int Nz, int n, int k, int& zs, int& ze) {
  zs = (int)(((long long)k * Nz) / n);
  ze = (k == n - 1) ? Nz : (int)(((long long)(k + 1) * Nz) / n) - 1;
}

// Number of ragged z chunks for an engine whose CTAs each own one of `tiles`
// xy tiles and one chunk: the CTAs should fill whole waves of `slots` resident
// CTAs (a last, partly filled wave runs at a fraction of the bandwidth), while
// each chunk re-reads about one halo plane.  Chunks have at least 6 planes.
inline int balanced_zchunks(long long tiles, long long slots, int Nz) {
  int best = 1;
  double best_score = -1.0;
  if (tiles < 1 || slots < 1) return Nz / 8 > 0 ? Nz / 8 : 1;
  for (int n = 1; n <= Nz / 6 || n == 1; ++n) {
    const double waves = (double)(tiles * n) / (double)slots;
    const double fill = waves / std::ceil(waves);
    const double len = (double)Nz / n;
    const double score = fill * len / (len + 1.0);
    if (score > best_score + 1e-12) {
      best_score = score;
      best = n;
    }
  }
  return best;
}

}  // namespace thermo
