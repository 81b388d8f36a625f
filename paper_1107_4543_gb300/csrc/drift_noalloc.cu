// lbm_drift_pop_noalloc: the FP64 conservation-drift reduction over a
// caller-owned population array, with its scratch in a fixed device array
// of this library instead of memory allocated per call or per handle.
//
// For callers that cannot allocate device memory themselves: for example a
// host application whose own allocator already owns the GPU's memory (a
// framework caching allocator holding the whole HBM), or a loop that runs
// under a fixed memory budget where an allocation -- with its implicit
// synchronisation and its failure modes -- is not acceptable.  The caller
// passes the populations and receives the four sums; nothing is allocated.
//
// Scratch: g_noalloc_scratch, (LBM_NOALLOC_MAX_ROWS + 1) x 4 doubles
// (256 KiB + 32 B), a file-scope __device__ array.  Every GPU that loads the
// library holds it until the process exits.  Rows 0..ny-1 receive one
// block's partial sums each; the last 4 doubles receive the result.  Each
// call writes every slot it later reads, so no slot needs clearing between
// calls; the array keeps the last call's contents.  Calls that overlap on
// the GPU (different streams, or different host threads) share the array and
// race: serialize them.
#include <math.h>

#include <mutex>
#include <string>

#include "lbm_internal.h"

#define LBM_NOALLOC_MAX_ROWS 8192
#define LBM_NOALLOC_THREADS 256
#define LBM_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_scratch[(LBM_NOALLOC_MAX_ROWS + 1) * 4];

namespace {

// Host code cannot use the array's name as a device address: look the
// address up once per device, with that device current.
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[LBM_NOALLOC_MAX_DEVICES] = {nullptr};

cudaError_t noalloc_scratch(int dev, double **out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// base populations f^eq(rho0, j0), subtracted population by population
struct Base {
  double f0[9];
};

// one block per row: the row's nodes in a fixed order, then a fixed tree.
// Each node's sums are taken over the deviations f_i - f0_i (exact while
// f_i stays within a factor two of f0_i), as lbm_drift takes them.
__global__ void __launch_bounds__(LBM_NOALLOC_THREADS)
k_drift_rows(const double *__restrict__ f, int nx, int ny, Base base, double *scratch) {
  __shared__ double sh[4][LBM_NOALLOC_THREADS];
  const int y = blockIdx.x;
  const long long plane = (long long)nx * ny;
  double s0 = 0, s1 = 0, s2 = 0, bad = 0;
  for (int x = threadIdx.x; x < nx; x += LBM_NOALLOC_THREADS) {
    const long long n = (long long)y * nx + x;
    double g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const double v = f[i * plane + n];
      if (!isfinite(v)) {
        bad += 1.0;
        g[i] = 0.0;
      } else {
        g[i] = v - base.f0[i];
      }
    }
    s0 += g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
    s1 += g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
    s2 += g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
  }
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  sh[2][threadIdx.x] = s2;
  sh[3][threadIdx.x] = bad;
  __syncthreads();
  for (int w = LBM_NOALLOC_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) scratch[y * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

// one block sums the ny row partials into the result slot
__global__ void __launch_bounds__(LBM_NOALLOC_THREADS)
k_drift_rows_final(int ny, double *scratch) {
  __shared__ double sh[4][LBM_NOALLOC_THREADS];
  double s[4] = {0, 0, 0, 0};
  for (int r = threadIdx.x; r < ny; r += LBM_NOALLOC_THREADS)
    for (int c = 0; c < 4; ++c) s[c] += scratch[r * 4 + c];
  for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int w = LBM_NOALLOC_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) scratch[LBM_NOALLOC_MAX_ROWS * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

extern "C" int lbm_drift_pop_noalloc(const double *f_dev, int nx, int ny, double rho0,
                                     double jx0, double jy0, double out[4], void *stream) {
  if (!f_dev || !out) {
    lbm::set_error("lbm_drift_pop_noalloc: null argument");
    return LBM_EINVAL;
  }
  if (nx < 1 || ny < 1) {
    lbm::set_error("lbm_drift_pop_noalloc: nx and ny must be >= 1");
    return LBM_EINVAL;
  }
  if (ny > LBM_NOALLOC_MAX_ROWS) {
    lbm::set_error("lbm_drift_pop_noalloc: ny = " + std::to_string(ny) +
                   " exceeds the fixed scratch of " + std::to_string(LBM_NOALLOC_MAX_ROWS) +
                   " rows; use lbm_drift on a handle instead");
    return LBM_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && (dev < 0 || dev >= LBM_NOALLOC_MAX_DEVICES)) e = cudaErrorInvalidDevice;
  double *scratch = nullptr;
  if (e == cudaSuccess) e = noalloc_scratch(dev, &scratch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) {
    Base base;
    lbm::host_feq_j(rho0, jx0, jy0, base.f0);
    k_drift_rows<<<ny, LBM_NOALLOC_THREADS, 0, st>>>(f_dev, nx, ny, base, scratch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_drift_rows_final<<<1, LBM_NOALLOC_THREADS, 0, st>>>(ny, scratch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, scratch + LBM_NOALLOC_MAX_ROWS * 4, 4 * sizeof(double),
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    lbm::set_error(std::string("lbm_drift_pop_noalloc: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  return out[3] > 0 ? LBM_EUNSTABLE : LBM_OK;
}
