// Device-side index checks of the debug build (nvcc -DLBM_DEBUG_BOUNDS).
//
// ck(i, n, site) returns i when 0 <= i < n.  Otherwise, in the debug build,
// it sets `site` in this translation unit's error word and returns 0, so
// the access goes to the array's first element instead of out of bounds: no
// trap, the context stays usable, and the host reads the word afterwards
// (lbm_debug_bounds ORs the words of every translation unit).  Without the
// flag ck is the identity and the word reads 0.
//
// Checked: the von Neumann QR's row and column indices that follow the
// deflation bounds (vn.cu), the optimizer's polynomial-matrix slots, power
// blocks, point-table and K_l-table offsets (optcost.cu), the batched
// step's block records and lane positions (step_impl.cuh), the resident
// batch members' entries (resident.cuh), and the batched init / moments
// blocks (io_dev.cu).
#pragma once
#include <cuda_runtime.h>

namespace lbm {
namespace bounds {

enum Site : unsigned {
  VN_HQR = 1u << 0,       // QR sweep / deflation indices
  VN_HESS = 1u << 1,      // Householder reduction indices
  OPT_SLOT = 1u << 2,     // polynomial-matrix coefficient slot
  OPT_POW = 1u << 3,      // power-of-B block
  OPT_H = 1u << 4,        // H_l index
  OPT_TAB = 1u << 5,      // point-table entry
  OPT_KTAB = 1u << 6,     // K_l table offset
  BATCH_REC = 1u << 7,    // batched step: block record's lattice
  BATCH_LANE = 1u << 8,   // batched step: lane row / chunk inside the lattice
  IO_BLOCK = 1u << 9,     // batched init / moments block
  SELFTEST = 1u << 31,    // lbm_debug_bounds_selftest
};

#ifdef LBM_DEBUG_BOUNDS
static __device__ unsigned int g_word;

__device__ __forceinline__ int ck(int i, int n, unsigned site) {
  if (i < 0 || i >= n) {
    atomicOr(&g_word, site);
    return 0;
  }
  return i;
}
__device__ __forceinline__ long long ck(long long i, long long n, unsigned site) {
  if (i < 0 || i >= n) {
    atomicOr(&g_word, site);
    return 0;
  }
  return i;
}
__device__ __forceinline__ bool ok(bool cond, unsigned site) {
  if (!cond) atomicOr(&g_word, site);
  return cond;
}
// the word of this translation unit (current device), optionally cleared
static inline unsigned read_word(bool reset) {
  unsigned w = 0;
  if (cudaMemcpyFromSymbol(&w, g_word, sizeof(w)) != cudaSuccess) {
    cudaGetLastError();
    return ~0u;
  }
  if (reset) {
    const unsigned z = 0;
    if (cudaMemcpyToSymbol(g_word, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
  }
  return w;
}
constexpr bool kEnabled = true;
#else
__device__ __forceinline__ int ck(int i, int, unsigned) { return i; }
__device__ __forceinline__ long long ck(long long i, long long, unsigned) { return i; }
__device__ __forceinline__ bool ok(bool, unsigned) { return true; }
static inline unsigned read_word(bool) { return 0; }
constexpr bool kEnabled = false;
#endif

}  // namespace bounds
}  // namespace lbm
