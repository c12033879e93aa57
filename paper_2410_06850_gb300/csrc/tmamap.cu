// Host-side cache of TMA tensor maps (cuTensorMapEncodeTiled through the
// runtime's driver entry point), shared by the fine-grid kernels.
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include <functional>
#include <mutex>
#include <unordered_map>

#include "tma.cuh"

namespace thermo {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

struct MapKey {
  const void* p;
  long long d0, d1, d2;
  int dt, b0, b1;
  bool operator==(const MapKey& o) const {
    return p == o.p && d0 == o.d0 && d1 == o.d1 && d2 == o.d2 && dt == o.dt && b0 == o.b0 && b1 == o.b1;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    size_t h = std::hash<const void*>()(k.p);
    h ^= std::hash<long long>()(k.d0 * 1000003LL + k.d1 * 131LL + k.d2) + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    h ^= std::hash<long long>()((long long)k.dt * 1000000 + k.b0 * 1000 + k.b1) + (h << 6) + (h >> 2);
    return h;
  }
};

// 3-D map of a padded array: dims (d0 elements, d1 rows, d2 planes), dense
// rows of d0 elements, box (b0, b1, 1), zero fill outside.
cudaError_t get_map(CUtensorMap* out, const void* base, CUtensorMapDataType dt, int esize, long long d0,
                           long long d1, long long d2, int b0, int b1) {
  static std::mutex mu;
  static std::unordered_map<MapKey, CUtensorMap, MapKeyHash> cache;
  if (!base) {
    memset(out, 0, sizeof(*out));
    return cudaSuccess;
  }
  const MapKey key{base, d0, d1, d2, (int)dt, b0, b1};
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  const cuuint64_t strides[2] = {(cuuint64_t)(d0 * esize), (cuuint64_t)(d0 * d1 * esize)};
  const cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  CUtensorMap m;
  const CUresult r = fn(&m, dt, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  if (cache.size() > 4096) cache.clear();
  cache.emplace(key, m);
  *out = m;
  return cudaSuccess;
}


}  // namespace thermo
