// Plain FP64 step: fused pull-stream + MRT collide on the full populations.
//
// The collision follows the operation order of a plain matrix-vector
// implementation of section 2.1 (collide_f64), and this file is compiled
// with -fmad=false, so the result is bit-identical to a straightforward
// FP64 CPU implementation of the same definition.  Per node it moves 9 + 9
// doubles (144 B) and performs ~150 FP64 operations; on GB300 the FP64
// units, not HBM, bound it.
#include "lbm_internal.h"

namespace lbm {

__global__ void __launch_bounds__(256)
k_step_f64(const double *__restrict__ src, double *__restrict__ dst, Geom g, F64Params P,
           long long ntasks) {
  constexpr int V = Elem<double>::V;
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long task = warp0; task < ntasks; task += nwarps) {
    LanePos p = lane_pos<V>(g, task, lane);
    double f[9][V];
    pull9<double, false>(src, g, p, 1.0, f);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      double n[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) n[i] = f[i][e];
      collide_f64(n, P);
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i][e] = n[i];
    }
    store9<double, false>(dst, g, p, 1.0, f);
  }
}

cudaError_t launch_step_f64(const Lattice &L, const void *src, void *dst, cudaStream_t st,
                            int block, int grid_cap) {
  const long long nt = L.g.tasks;
  const int wpb = block / 32;
  long long grid = (nt + wpb - 1) / wpb;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  if (grid < 1) grid = 1;
  k_step_f64<<<(unsigned)grid, block, 0, st>>>((const double *)src, (double *)dst, L.g, L.fp,
                                               nt);
  return cudaGetLastError();
}

}  // namespace lbm
