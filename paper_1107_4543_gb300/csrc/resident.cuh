// Batched step for small lattices held in shared memory for all the time
// steps of one launch (section 2.1, Eq. blbs, as the per-step kernels): one
// thread block per member loads the member's nine planes into shared memory,
// runs its n steps there (pull with periodic wrap, collide, store into the
// other buffer, block barrier, swap) and writes the result back once: its
// 9 x nx ny elements cross HBM once in and once out for the whole launch
// instead of in and out at every step.
//
// The arithmetic is the per-step kernels' own (collide_dev for FP32,
// collide_pair for the 16-bit types, the same storage rounding), node by
// node, so a member's result is bit-identical to the per-step path's.
#pragma once
#include <type_traits>

#include "bounds.cuh"
#include "lbm_internal.h"

namespace lbm {

// 512 threads (16 warps) per member; two blocks per SM at the 64-register
// cap (256 threads: 135 against 152 GLUPS on 4,096 lattices of 32^2 - 56^2)
constexpr int kResidentThreads = 512;

template <typename T>
__device__ __forceinline__ uint32_t bits16(const T *p) {
  return (uint32_t) * reinterpret_cast<const unsigned short *>(p);
}

// Node r = y nx + x of the plane arrays A (9 planes of N compact elements):
// the element plane i pulls into (x, y), i.e. the one at (x - c_ix, y - c_iy)
// with periodic wrap.
struct Nbr {
  int r0;          // y * nx
  int xm, x, xp;   // x - 1, x, x + 1 (wrapped)
  int ym, yp;      // (y - 1) nx, (y + 1) nx (wrapped)
  __device__ __forceinline__ int at(int i) const {
    const int cx = CXd(i), cy = CYd(i);
    const int row = cy == 1 ? ym : (cy == -1 ? yp : r0);
    const int col = cx == 1 ? xm : (cx == -1 ? xp : x);
    return row + col;
  }
};

__device__ __forceinline__ Nbr nbr(int x, int y, int nx, int ny) {
  Nbr n;
  n.x = x;
  n.r0 = y * nx;
  n.xm = x == 0 ? nx - 1 : x - 1;
  n.xp = x == nx - 1 ? 0 : x + 1;
  n.ym = (y == 0 ? ny - 1 : y - 1) * nx;
  n.yp = (y == ny - 1 ? 0 : y + 1) * nx;
  return n;
}

// (x, y) of node r, advanced by a fixed stride of (dx, dy) = (stride mod nx,
// stride / nx) nodes without a division per node
struct Walk {
  int x, y, dx, dy, nx;
  __device__ __forceinline__ Walk(int r, int stride, int nx_) : nx(nx_) {
    y = r / nx;
    x = r - y * nx;
    dy = stride / nx;
    dx = stride - dy * nx;
  }
  __device__ __forceinline__ void next() {
    x += dx;
    y += dy;
    if (x >= nx) {
      x -= nx;
      ++y;
    }
  }
};

// idx[b]: the entry block b steps.  Each member takes min(steps, limits[e])
// steps (limits may be null) from buffer parity ^ off and leaves its state
// in the buffer that parity of steps selects, as the per-step launches do.
template <typename T>
__global__ void __launch_bounds__(kResidentThreads, 2)
k_batch_resident(const BatchEntry *__restrict__ ents, const int *__restrict__ idx, int nents,
                 int parity, int steps, const int *__restrict__ limits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int e = idx[blockIdx.x];
  if (!bounds::ok(e >= 0 && e < nents, bounds::BATCH_REC)) return;  // block-uniform
  const BatchEntry &E = ents[e];
  const int nx = E.g.nx, ny = E.g.ny, N = nx * ny;
  int n = steps;
  if (limits != nullptr && limits[e] < n) n = limits[e];
  if (n <= 0) return;  // block-uniform
  const int from = parity ^ E.off;
  const T *src = static_cast<const T *>(E.buf[from]);
  T *dst = static_cast<T *>(E.buf[from ^ (n & 1)]);
  T *A = reinterpret_cast<T *>(smem_raw);
  T *B = A + 9 * N;
  for (int q = threadIdx.x; q < 9 * N; q += blockDim.x) {
    const int i = q / N, r = q - i * N, y = r / nx;
    A[q] = src[(long long)i * E.g.plane + (long long)y * E.g.rstride + (r - y * nx)];
  }
  __syncthreads();
  const DevParams &P = E.dp;
  for (int t = 0; t < n; ++t) {
    if constexpr (sizeof(T) == 4) {
      Walk wk(threadIdx.x, blockDim.x, nx);
      for (int r = threadIdx.x; r < N; r += blockDim.x, wk.next()) {
        const Nbr nb = nbr(wk.x, wk.y, nx, ny);
        float f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = A[i * N + nb.at(i)];
        collide_dev<true, false>(f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], f[8], P);
#pragma unroll
        for (int i = 0; i < 9; ++i) B[i * N + r] = f[i];
      }
    } else {
      // two nodes per thread, one per lane of the packed pair collision
      constexpr bool SCALED = std::is_same<T, __half>::value;
      Walk wk(2 * threadIdx.x, 2 * blockDim.x, nx);
      for (int r0 = 2 * threadIdx.x; r0 < N; r0 += 2 * blockDim.x, wk.next()) {
        const int r1 = r0 + 1 < N ? r0 + 1 : r0;
        // node r0 + 1 is (x + 1, y), or the start of the next row
        const int x1 = wk.x + 1 < nx ? wk.x + 1 : 0;
        const int y1 = wk.x + 1 < nx ? wk.y : wk.y + 1;
        const Nbr n0 = nbr(wk.x, wk.y, nx, ny);
        const Nbr n1 = r1 != r0 ? nbr(x1, y1, nx, ny) : n0;
        F2 f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          float u[2];
          Elem<T>::unpack2(bits16(&A[i * N + n0.at(i)]) | bits16(&A[i * N + n1.at(i)]) << 16, u);
          f[i] = f2(u[0], u[1]);
        }
        collide_pair<SCALED>(f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], f[8],
                             ParamPairs{P});
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          float u[2];
          f2split(f[i], u[0], u[1]);
          const uint32_t w = Elem<T>::pack2(u[0], u[1]);
          reinterpret_cast<unsigned short *>(B)[i * N + r0] = (unsigned short)(w & 0xffffu);
          if (r1 != r0) reinterpret_cast<unsigned short *>(B)[i * N + r1] = (unsigned short)(w >> 16);
        }
      }
    }
    __syncthreads();
    T *tmp = A;
    A = B;
    B = tmp;
  }
  for (int q = threadIdx.x; q < 9 * N; q += blockDim.x) {
    const int i = q / N, r = q - i * N, y = r / nx;
    dst[(long long)i * E.g.plane + (long long)y * E.g.rstride + (r - y * nx)] = A[q];
  }
}

template <typename T>
cudaError_t launch_resident_t(const BatchEntry *ents, const int *idx, int nres, int nents,
                              size_t smem, int parity, long steps, const int *limits,
                              cudaStream_t st) {
  if (nres < 1 || steps < 1) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_batch_resident<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // launches of at most 2^30 steps (the step count is an int on the device)
  const long chunk = 1L << 30;
  for (long done = 0; done < steps; done += chunk) {
    const long k = steps - done < chunk ? steps - done : chunk;
    k_batch_resident<T><<<(unsigned)nres, kResidentThreads, smem, st>>>(
        ents, idx, nents, parity ^ (int)(done & 1), (int)k, limits);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace lbm
