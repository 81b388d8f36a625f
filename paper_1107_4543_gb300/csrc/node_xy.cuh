// (x, y) of node n = y nx + x of an nx-wide lattice, for the grid-stride
// loops of the auxiliary kernels (init, moments, drift, population copies).
// A 64-bit integer division per node kept the FP64 pipe of GB300 busy in
// those FP64-bound kernels (the batched drift measured 68% FP64-pipe
// activity); node indices below 2^31, every node of a lattice of fewer
// nodes, divide in 32 bits instead, with the same quotient.
#pragma once

namespace lbm {

__host__ __device__ __forceinline__ void node_xy(long long n, int nx, int &x, int &y) {
  if (n < 0x7fffffffLL) {
    const unsigned q = (unsigned)n / (unsigned)nx;
    y = (int)q;
    x = (int)((unsigned)n - q * (unsigned)nx);
  } else {
    y = (int)(n / nx);
    x = (int)(n - (long long)y * nx);
  }
}

// The nodes n, n + stride, n + 2 stride, ... of a grid-stride loop, their
// (x, y) advanced by a fixed step instead of a division per node.
struct NodeWalk {
  int x, y, dx, dy, nx;
  __host__ __device__ __forceinline__ NodeWalk(long long n, long long stride, int nx_) : nx(nx_) {
    node_xy(n, nx, x, y);
    dy = (int)(stride / nx);
    dx = (int)(stride - (long long)dy * nx);
  }
  __host__ __device__ __forceinline__ void next() {
    x += dx;
    y += dy;
    if (x >= nx) {
      x -= nx;
      ++y;
    }
  }
};

}  // namespace lbm
