// Counter-based SplitMix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): position i of stream `seed`
// uses the state (seed 2^32 + i + 1) times the golden gamma, then the standard
// finaliser; stream 0 is the published sequence from state 0.  Plain C++ (also
// compiled by the host-logic tests without CUDA).
#pragma once

#ifdef __CUDACC__
#define SMX_HD __host__ __device__ __forceinline__
#else
#define SMX_HD inline
#endif

namespace thermo {

SMX_HD unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i) {
  unsigned long long z = (seed * (1ull << 32) + i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// uniform double in [0, 1): the top 53 bits
SMX_HD double splitmix_u01(unsigned long long seed, unsigned long long i) {
  return (double)(splitmix64_at(seed, i) >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace thermo
