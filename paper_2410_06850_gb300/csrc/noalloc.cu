// Deterministic FP64 dot product whose scratch is a file-scope device array:
// the call allocates no memory (no cudaMalloc / cudaFree, no allocating
// library routine), so it can be used by callers that must not allocate.
//
// Reduction order (fixed, independent of timing): block b sums the chunk
// [b*CHUNK, min((b+1)*CHUNK, n)) with a fixed per-thread stride and a fixed
// shared-memory tree, writes partial[b]; the last block to arrive (atomic
// counter) sums partial[0..nb) in index order with the same tree and resets
// the counter to zero.  Equal inputs give bitwise equal results.
#include <cuda_runtime.h>
#include <mutex>
#include <stdio.h>
#include <string.h>

#include "../../include/thermo.h"

namespace {

constexpr int NT = 256;                       // threads per block
constexpr long long CHUNK = 8192;             // elements per block
constexpr int MAX_BLOCKS = 16384;             // partials held in the static scratch
constexpr long long MAX_N = CHUNK * MAX_BLOCKS;  // 134,217,728 elements
constexpr int MAX_DEVICES = 64;

// scratch: [0, MAX_BLOCKS) partial sums, then the arrival counter (as a
// double-sized slot).  The counter starts at zero (zero-initialised at module
// load, zeroed again at the first call on each device) and every completed
// call leaves it at zero.  The partials need no initial value.
static __device__ __align__(256) double nalloc_scratch[MAX_BLOCKS + 32];

struct DevScratch {
  double* partial = nullptr;
  unsigned* counter = nullptr;
  bool ready = false;
};
DevScratch g_dev[MAX_DEVICES];
std::mutex g_mu;

__device__ __forceinline__ double tree_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

__global__ void __launch_bounds__(NT) k_dot_static(const double* __restrict__ x, const double* __restrict__ y,
                                                   long long n, double* __restrict__ partial,
                                                   unsigned* __restrict__ counter, double* __restrict__ out) {
  __shared__ double sh[NT];
  __shared__ bool last;
  const long long lo = (long long)blockIdx.x * CHUNK;
  const long long hi = lo + CHUNK < n ? lo + CHUNK : n;
  double v = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += NT) v = fma(x[i], y[i], v);
  const double s = tree_sum(v, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double w = 0.0;
  for (unsigned i = threadIdx.x; i < gridDim.x; i += NT) w += __ldcg(partial + i);
  const double t = tree_sum(w, sh);
  if (threadIdx.x == 0) {
    *out = t;
    *counter = 0u;  // leave the scratch ready for the next call
  }
}

void put(char* msg, int len, const char* text) {
  if (msg && len > 0) {
    strncpy(msg, text, (size_t)len - 1);
    msg[len - 1] = '\0';
  }
}

}  // namespace

extern "C" thermo_status thermo_dot_noalloc(const double* x, const double* y, long long n, double* result,
                                            void* stream, char* msg, int msg_len) {
  if (n < 0 || (n > 0 && (!x || !y)) || !result) {
    put(msg, msg_len, "thermo_dot_noalloc: n must be >= 0 and x, y (n > 0) and result non-NULL");
    return THERMO_EINVAL;
  }
  if (n > MAX_N) {
    char b[160];
    snprintf(b, sizeof b, "thermo_dot_noalloc: n = %lld exceeds the static scratch limit of %lld elements", n, MAX_N);
    put(msg, msg_len, b);
    return THERMO_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    put(msg, msg_len, "thermo_dot_noalloc: no usable current CUDA device");
    return THERMO_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  DevScratch& d = g_dev[dev];
  {
    // one-time set-up per device: resolve the scratch address, zero the counter
    std::lock_guard<std::mutex> lk(g_mu);
    if (!d.ready) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, nalloc_scratch) != cudaSuccess || !p) {
        put(msg, msg_len, "thermo_dot_noalloc: cudaGetSymbolAddress of the static scratch failed");
        return THERMO_ECUDA;
      }
      d.partial = static_cast<double*>(p);
      d.counter = reinterpret_cast<unsigned*>(d.partial + MAX_BLOCKS);
      if (cudaMemset(d.counter, 0, sizeof(unsigned)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        put(msg, msg_len, "thermo_dot_noalloc: zeroing the static scratch counter failed");
        return THERMO_ECUDA;
      }
      d.ready = true;
    }
  }
  if (n == 0) {
    if (cudaMemsetAsync(result, 0, sizeof(double), st) != cudaSuccess) {
      put(msg, msg_len, "thermo_dot_noalloc: cudaMemsetAsync of the result failed");
      return THERMO_ECUDA;
    }
    return THERMO_OK;
  }
  const unsigned nb = (unsigned)((n + CHUNK - 1) / CHUNK);
  k_dot_static<<<nb, NT, 0, st>>>(x, y, n, d.partial, d.counter, result);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char b[160];
    snprintf(b, sizeof b, "thermo_dot_noalloc: launch failed: %s", cudaGetErrorString(e));
    put(msg, msg_len, b);
    return THERMO_ECUDA;
  }
  return THERMO_OK;
}
