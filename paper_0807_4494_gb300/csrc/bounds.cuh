// Index checks of the kernels' global accesses, the bounds-checked build that stands in for a
// memory checker.  Built with -DSSHT_DEBUG (paper_0807_4494_gb300/build.py, debug=True), every
// checked access computes its index against the extent of the buffer it touches (the size the host
// allocated or the caller's buffer holds by the API's layout); an index outside [0, n) is counted,
// the first one recorded (kernel, index, extent), and the access skipped, so that a wrong index
// shows up as a record and not as a fault.  Release builds compile the checks away.
//
// The record is a device variable of each translation unit (no relocatable device code); the file
// that includes this header with SSHT_BOUNDS_TU(tag) defines bounds_take_<tag>(), which copies the
// record out and clears it, and ssht_debug_bounds() adds them up.
#pragma once
#include <cuda_runtime.h>

namespace ssht {

struct BoundsRecord {
  unsigned long long count;  // accesses outside their buffer since the last take
  int kernel;                // BoundsSite of the first one
  int pad;
  long long index, extent;   // its index and the buffer's extent, in the access's units
};

// Where a checked access sits (the first failing one is reported by this number).
enum BoundsSite {
  kbNone = 0,
  kbInverseThetaIn = 1, kbInverseThetaOut, kbPhiIn, kbPhiOut, kbForwardThetaIn, kbForwardThetaOut,
  kbAdjointThetaIn, kbAdjointThetaOut, kbPutTile,
  kbPackVIn = 20, kbPackVOut, kbPackAIn, kbPackAOut, kbGemmA, kbGemmX, kbGemmOut,
  kbColumnTable = 40, kbColumnTile, kbLaneTable, kbLaneTile, kbColumnCoef,
  kbPairIn = 60, kbPairOut, kbRealIn, kbRealOut,
  kbSimtIn = 80, kbSimtOut,
};

#if defined(SSHT_DEBUG) && defined(__CUDACC__)
static __device__ BoundsRecord g_bounds;

__device__ __forceinline__ bool in_bounds(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_bounds.count, 1ull) == 0ull) {
    g_bounds.kernel = site;
    g_bounds.index = i;
    g_bounds.extent = n;
  }
  return false;
}

#define SSHT_BOUNDS_TU(tag)                                                                    \
  cudaError_t bounds_take_##tag(BoundsRecord* r) {                                             \
    cudaError_t e = cudaMemcpyFromSymbol(r, g_bounds, sizeof(BoundsRecord));                   \
    if (e != cudaSuccess) return e;                                                            \
    const BoundsRecord zero{};                                                                 \
    return cudaMemcpyToSymbol(g_bounds, &zero, sizeof(BoundsRecord));                          \
  }
#else
__host__ __device__ __forceinline__ bool in_bounds(long long, long long, int) { return true; }

#define SSHT_BOUNDS_TU(tag)                         \
  cudaError_t bounds_take_##tag(BoundsRecord* r) { \
    *r = BoundsRecord{};                            \
    return cudaSuccess;                             \
  }
#endif

// Whether this library was built with the checks.
constexpr bool kBoundsChecked =
#ifdef SSHT_DEBUG
    true;
#else
    false;
#endif

}  // namespace ssht
