// Field I/O kernels of the deviation storage types (FP32, FP16, BF16):
// equilibrium initialisation from device fields, the largest deviation that
// sets the FP16 storage scale, and the moments.  The FP64 storage type keeps
// the canonical kernels of aux.cu (bit parity with a plain FP64 version).
//
// The equilibrium of section 2.3, f^eq = M^-1 m^eq, equals the second-order
// polynomial  w_i [rho + 3 c_i.j + 9/2 (c_i.j)^2 / rho - 3/2 |j|^2 / rho]
// with weights 4/9, 1/9 (axis) and 1/36 (diagonal).  What is stored is the
// deviation f^eq(rho, j) - f^eq(rho0, j0), formed here from the differences
// rho - rho0, j - j0, jx^2/rho - jx0^2/rho0, jy^2/rho - jy0^2/rho0 and
// jx jy/rho - jx0 jy0/rho0: every term is of the size of the perturbation,
// so nothing of order one is subtracted after rounding, and a node costs
// a few dozen FP64 operations and no division (GB300's FP64 rate is what
// bounds these kernels, not their 60 bytes per node).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "bounds.cuh"
#include "lbm_internal.h"
#include "node_xy.cuh"

namespace lbm {
namespace {

// reference state and its quadratic terms (host-computed)
struct RefState {
  double rho0, jx0, jy0;
  double axx0, ayy0, axy0;  // jx0^2/rho0, jy0^2/rho0, jx0 jy0/rho0
};

RefState make_ref(const AuxView &a) {
  RefState r;
  r.rho0 = a.rho0;
  r.jx0 = a.jx0;
  r.jy0 = a.jy0;
  r.axx0 = a.jx0 * a.jx0 / a.rho0;
  r.ayy0 = a.jy0 * a.jy0 / a.rho0;
  r.axy0 = a.jx0 * a.jy0 / a.rho0;
  return r;
}

__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// f^eq_i(rho, rho u) - f^eq_i(rho0, j0), i = 0..8
__device__ __forceinline__ void feq_deviation(const RefState &R, double r, double u, double v,
                                              double d[9]) {
  const double jx = r * u, jy = r * v;
  const double dr = r - R.rho0;
  const double ex = 3.0 * (jx - R.jx0), ey = 3.0 * (jy - R.jy0);
  // jx^2 / rho = rho u^2 etc.: the fields give u, so no division is needed
  // (GB300's FP64 divide is the costliest step of this FP64-bound kernel)
  const double A = jx * u - R.axx0;
  const double B = jy * v - R.ayy0;
  const double C = jx * v - R.axy0;
  const double t1 = dr + 3.0 * A - 1.5 * B;  // axis x: 9/2 A - 3/2 (A + B)
  const double t2 = dr + 3.0 * B - 1.5 * A;  // axis y
  const double t5 = dr + 3.0 * (A + B);      // diagonals: 9/2 (A + B +- 2C) - 3/2 (A + B)
  const double p = t5 + 9.0 * C, q = t5 - 9.0 * C;
  constexpr double w0 = 4.0 / 9.0, w1 = 1.0 / 9.0, w5 = 1.0 / 36.0;
  d[0] = w0 * (dr - 1.5 * (A + B));
  d[1] = w1 * (t1 + ex);
  d[2] = w1 * (t2 + ey);
  d[3] = w1 * (t1 - ex);
  d[4] = w1 * (t2 - ey);
  d[5] = w5 * (p + ex + ey);
  d[6] = w5 * (q - ex + ey);
  d[7] = w5 * (p - ex - ey);
  d[8] = w5 * (q + ex - ey);
}

template <typename T>
__device__ __forceinline__ T encode(double d, double scale);
template <>
__device__ __forceinline__ float encode<float>(double d, double) {
  return (float)d;
}
template <>
__device__ __forceinline__ __half encode<__half>(double d, double scale) {
  return __float2half_rn((float)(d * scale));
}
template <>
__device__ __forceinline__ __nv_bfloat16 encode<__nv_bfloat16>(double d, double) {
  return __float2bfloat16_rn((float)d);
}
template <>
__device__ __forceinline__ double encode<double>(double d, double) {
  return d;
}

template <typename T>
__device__ __forceinline__ double decode(T s, double inv_scale);
template <>
__device__ __forceinline__ double decode<float>(float s, double) {
  return (double)s;
}
template <>
__device__ __forceinline__ double decode<__half>(__half s, double inv_scale) {
  return (double)__half2float(s) * inv_scale;  // the scale is a power of two
}
template <>
__device__ __forceinline__ double decode<__nv_bfloat16>(__nv_bfloat16 s, double) {
  return (double)__bfloat162float(s);
}
template <>
__device__ __forceinline__ double decode<double>(double s, double) {
  return s;
}

// Population i of node x goes to slot x - c_i, where the next step's pull
// (f_i(x) = P_i(x - c_i)) reads it.  bad counts nodes whose field is not
// finite or has rho <= 0.
// one node of the equilibrium init: the deviations of f^eq(r, (u, v)) into
// the slots the next pull reads; returns whether the field is invalid
template <typename T>
__device__ __forceinline__ bool init_node(const AuxView &a, const RefState &R, int x, int y,
                                          double r, double u, double v) {
  T *buf = static_cast<T *>(a.buf);
  double d[9];
  feq_deviation(R, r, u, v, d);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int xs = wrap(x - CXd(i), a.g.nx), ys = wrap(y - CYd(i), a.g.nyw);
    buf[(long long)i * a.g.plane + (long long)ys * a.g.rstride + xs] = encode<T>(d[i], a.scale);
  }
  return !(r > 0.0) || !isfinite(r) || !isfinite(u) || !isfinite(v);
}

template <typename T>
__global__ void __launch_bounds__(256) k_init_dev(AuxView a, RefState R, const double *rho,
                                                  const double *ux, const double *uy,
                                                  unsigned int *bad) {
  const int nx = a.g.nx, ny = a.g.ny;
  const long long N = (long long)nx * ny;
  unsigned int nbad = 0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int x, y;
    node_xy(n, nx, x, y);
    if (init_node<T>(a, R, x, y, rho[n], ux[n], uy[n])) ++nbad;
  }
  if (bad && nbad) atomicAdd(bad, nbad);
}

__global__ void __launch_bounds__(256) k_maxdev_dev(AuxView a, RefState R, const double *rho,
                                                    const double *ux, const double *uy,
                                                    unsigned int *max_bits) {
  const long long N = (long long)a.g.nx * a.g.ny;
  float m = 0.0f;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    double d[9];
    feq_deviation(R, rho[n], ux[n], uy[n], d);
#pragma unroll
    for (int i = 0; i < 9; ++i) m = fmaxf(m, (float)fabs(d[i]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(max_bits, __float_as_uint(m));
}

// rho = rho0 + sum f', j = j0 + sum c f' of the pre-collision populations
// f_i(x) = P_i(x - c_i); u = j / rho
// rho, u of node (x, y) from its pre-collision populations
template <typename T>
__device__ __forceinline__ void moments_node(const AuxView &a, int x, int y, double inv_scale,
                                             double &r, double &u, double &v) {
  const T *buf = static_cast<const T *>(a.buf);
  double f[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int xs = wrap(x - CXd(i), a.g.nx), ys = wrap(y - CYd(i), a.g.nyw);
    f[i] = decode<T>(buf[(long long)i * a.g.plane + (long long)ys * a.g.rstride + xs], inv_scale);
  }
  r = a.rho0 + (f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8]);
  const double jx = a.jx0 + (f[1] - f[3] + f[5] - f[6] - f[7] + f[8]);
  const double jy = a.jy0 + (f[2] - f[4] + f[5] + f[6] - f[7] - f[8]);
  const double inv = 1.0 / r;
  u = jx * inv;
  v = jy * inv;
}

template <typename T>
__global__ void __launch_bounds__(256) k_moments_dev(AuxView a, double *rho, double *ux,
                                                     double *uy) {
  const int nx = a.g.nx, ny = a.g.ny;
  const long long N = (long long)nx * ny;
  const double inv_scale = 1.0 / a.scale;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int x, y;
    node_xy(n, nx, x, y);
    moments_node<T>(a, x, y, inv_scale, rho[n], ux[n], uy[n]);
  }
}

// Batched forms: block b covers nodes [start, start + count) of member
// blocks[b].member, whose fields sit at poff[member] of the packed arrays
// (rho at `stage`, ux at stage + total, uy at stage + 2 total).  The
// per-node arithmetic is that of the single-lattice kernels.
__device__ __forceinline__ RefState ref_of(const AuxView &a) {
  RefState r;
  r.rho0 = a.rho0;
  r.jx0 = a.jx0;
  r.jy0 = a.jy0;
  r.axx0 = a.jx0 * a.jx0 / a.rho0;
  r.ayy0 = a.jy0 * a.jy0 / a.rho0;
  r.axy0 = a.jx0 * a.jy0 / a.rho0;
  return r;
}

template <typename T>
__device__ __forceinline__ void batch_init_block(const AuxView &a, const IoBlock &B,
                                                 const double *r_, const double *u_,
                                                 const double *v_, unsigned int *bad) {
  const RefState R = ref_of(a);
  unsigned int nbad = 0;
  for (int j = threadIdx.x; j < B.count; j += blockDim.x) {
    const long long n = B.start + j;
    int x, y;
    node_xy(n, a.g.nx, x, y);
    if (init_node<T>(a, R, x, y, r_[n], u_[n], v_[n])) ++nbad;
  }
  if (nbad) atomicAdd(bad + B.member, nbad);
}

__global__ void __launch_bounds__(256) k_batch_init_dev(const AuxView *__restrict__ views,
                                                        const IoBlock *__restrict__ blocks,
                                                        const long long *__restrict__ poff,
                                                        long long total, const double *stage,
                                                        unsigned int *bad, int members) {
  const IoBlock B = blocks[blockIdx.x];
  if (!bounds::ok(B.member >= 0 && B.member < members, bounds::IO_BLOCK)) return;
  if (!bounds::ok(B.start >= 0 && B.count >= 0 &&
                      B.start + B.count <= (long long)views[B.member].g.nx * views[B.member].g.ny &&
                      poff[B.member] + B.start + B.count <= total,
                  bounds::IO_BLOCK))
    return;
  const AuxView &a = views[B.member];
  const double *r = stage + poff[B.member];
  switch (a.dtype) {
    case LBM_F32DEV: batch_init_block<float>(a, B, r, r + total, r + 2 * total, bad); break;
    case LBM_F16DEV: batch_init_block<__half>(a, B, r, r + total, r + 2 * total, bad); break;
    default: batch_init_block<__nv_bfloat16>(a, B, r, r + total, r + 2 * total, bad); break;
  }
}

template <typename T>
__device__ __forceinline__ void batch_moments_block(const AuxView &a, const IoBlock &B,
                                                    double *r_, double *u_, double *v_) {
  const double inv_scale = 1.0 / a.scale;
  for (int j = threadIdx.x; j < B.count; j += blockDim.x) {
    const long long n = B.start + j;
    int x, y;
    node_xy(n, a.g.nx, x, y);
    moments_node<T>(a, x, y, inv_scale, r_[n], u_[n], v_[n]);
  }
}

__global__ void __launch_bounds__(256) k_batch_moments_dev(const AuxView *__restrict__ views,
                                                           const IoBlock *__restrict__ blocks,
                                                           const long long *__restrict__ poff,
                                                           long long total, double *stage,
                                                           int members) {
  const IoBlock B = blocks[blockIdx.x];
  if (!bounds::ok(B.member >= 0 && B.member < members, bounds::IO_BLOCK)) return;
  if (!bounds::ok(B.start >= 0 && B.count >= 0 &&
                      B.start + B.count <= (long long)views[B.member].g.nx * views[B.member].g.ny &&
                      poff[B.member] + B.start + B.count <= total,
                  bounds::IO_BLOCK))
    return;
  const AuxView &a = views[B.member];
  double *r = stage + poff[B.member];
  switch (a.dtype) {
    case LBM_F32DEV: batch_moments_block<float>(a, B, r, r + total, r + 2 * total); break;
    case LBM_F16DEV: batch_moments_block<__half>(a, B, r, r + total, r + 2 * total); break;
    default: batch_moments_block<__nv_bfloat16>(a, B, r, r + total, r + 2 * total); break;
  }
}

unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  long long cap = (long long)sm_count() * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

__global__ void __launch_bounds__(256) k_batch_maxdev_fp16(const AuxView *__restrict__ views,
                                                           const IoBlock *__restrict__ blocks,
                                                           const long long *__restrict__ poff,
                                                           long long total, const double *stage,
                                                           unsigned int *max_bits, int members) {
  const IoBlock B = blocks[blockIdx.x];
  if (!bounds::ok(B.member >= 0 && B.member < members, bounds::IO_BLOCK)) return;
  if (!bounds::ok(B.start >= 0 && B.count >= 0 &&
                      B.start + B.count <= (long long)views[B.member].g.nx * views[B.member].g.ny &&
                      poff[B.member] + B.start + B.count <= total,
                  bounds::IO_BLOCK))
    return;
  const AuxView &a = views[B.member];
  if (a.dtype != LBM_F16DEV) return;  // block-uniform
  const RefState R = ref_of(a);
  const double *r = stage + poff[B.member];
  float m = 0.0f;
  for (int j = threadIdx.x; j < B.count; j += blockDim.x) {
    const long long n = B.start + j;
    double d[9];
    feq_deviation(R, r[n], r[total + n], r[2 * total + n], d);
#pragma unroll
    for (int i = 0; i < 9; ++i) m = fmaxf(m, (float)fabs(d[i]));
  }
  // one atomic per block (a member's blocks all update the same word)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float wmax[8];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
    atomicMax(max_bits + B.member, __float_as_uint(m));
  }
}

__global__ void k_batch_set_scales(AuxView *views0, AuxView *views1, BatchEntry *const *ent,
                                   const unsigned int *max_bits, const double *floor_,
                                   double *scale_out, int members) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= members || views0[k].dtype != LBM_F16DEV || ent[k] == nullptr) return;
  const double m = fmax((double)__uint_as_float(max_bits[k]), floor_[k]);
  const double s = fp16_scale(m);
  views0[k].scale = s;
  views1[k].scale = s;
  ent[k]->dp.scale = (float)s;
  ent[k]->dp.inv_scale = (float)(1.0 / s);
  scale_out[k] = s;
}

}  // namespace

cudaError_t launch_init_dev(const AuxView &a, const double *rho, const double *ux,
                            const double *uy, cudaStream_t st, unsigned int *bad) {
  const long long N = (long long)a.g.nx * a.g.ny;
  if (bad) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
  }
  const RefState R = make_ref(a);
  const unsigned grid = grid_for(N);
  switch (a.dtype) {
    case LBM_F32DEV: k_init_dev<float><<<grid, 256, 0, st>>>(a, R, rho, ux, uy, bad); break;
    case LBM_F16DEV: k_init_dev<__half><<<grid, 256, 0, st>>>(a, R, rho, ux, uy, bad); break;
    case LBM_BF16DEV:
      k_init_dev<__nv_bfloat16><<<grid, 256, 0, st>>>(a, R, rho, ux, uy, bad);
      break;
    case LBM_F64DEV: k_init_dev<double><<<grid, 256, 0, st>>>(a, R, rho, ux, uy, bad); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_maxdev_dev(const AuxView &a, const double *rho, const double *ux,
                              const double *uy, unsigned int *max_bits, cudaStream_t st) {
  const long long N = (long long)a.g.nx * a.g.ny;
  cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  k_maxdev_dev<<<grid_for(N), 256, 0, st>>>(a, make_ref(a), rho, ux, uy, max_bits);
  return cudaGetLastError();
}

cudaError_t launch_batch_fp16_scales(AuxView *views0, AuxView *views1, BatchEntry *const *ent,
                                     const IoBlock *blocks, long long nblocks,
                                     const long long *poff, long long total, const double *stage,
                                     unsigned int *max_bits, const double *floor_,
                                     double *scale_out, int members, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned int) * members, st);
  if (e != cudaSuccess) return e;
  if (nblocks > 0)
    k_batch_maxdev_fp16<<<(unsigned)nblocks, 256, 0, st>>>(views0, blocks, poff, total, stage,
                                                           max_bits, members);
  k_batch_set_scales<<<(members + 127) / 128, 128, 0, st>>>(views0, views1, ent, max_bits, floor_,
                                                            scale_out, members);
  return cudaGetLastError();
}

cudaError_t launch_batch_init_dev(const AuxView *views, const IoBlock *blocks, long long nblocks,
                                  const long long *poff, long long total, const double *stage,
                                  unsigned int *bad, int members, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int) * members, st);
  if (e != cudaSuccess || nblocks < 1) return e;
  k_batch_init_dev<<<(unsigned)nblocks, 256, 0, st>>>(views, blocks, poff, total, stage, bad,
                                                      members);
  return cudaGetLastError();
}

cudaError_t launch_batch_moments_dev(const AuxView *views, const IoBlock *blocks,
                                     long long nblocks, const long long *poff, long long total,
                                     double *stage, int members, cudaStream_t st) {
  if (nblocks < 1) return cudaSuccess;
  k_batch_moments_dev<<<(unsigned)nblocks, 256, 0, st>>>(views, blocks, poff, total, stage,
                                                         members);
  return cudaGetLastError();
}

cudaError_t launch_moments_dev(const AuxView &a, double *rho, double *ux, double *uy,
                               cudaStream_t st) {
  const long long N = (long long)a.g.nx * a.g.ny;
  const unsigned grid = grid_for(N);
  switch (a.dtype) {
    case LBM_F32DEV: k_moments_dev<float><<<grid, 256, 0, st>>>(a, rho, ux, uy); break;
    case LBM_F16DEV: k_moments_dev<__half><<<grid, 256, 0, st>>>(a, rho, ux, uy); break;
    case LBM_BF16DEV: k_moments_dev<__nv_bfloat16><<<grid, 256, 0, st>>>(a, rho, ux, uy); break;
    case LBM_F64DEV: k_moments_dev<double><<<grid, 256, 0, st>>>(a, rho, ux, uy); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Debug-build self-test of the index checks: one checked access with an
// index past its bound, which the check turns into index 0 of a one-element
// array (so nothing outside it is touched) while setting the SELFTEST bit.
__global__ void k_bounds_selftest(unsigned int *one) {
  const int i = bounds::ck(threadIdx.x + 1, 1, bounds::SELFTEST);
  one[i] = 1u;
}

cudaError_t launch_bounds_selftest(unsigned int *one, cudaStream_t st) {
  k_bounds_selftest<<<1, 1, 0, st>>>(one);
  return cudaGetLastError();
}

unsigned bounds_word_io(bool reset) { return bounds::read_word(reset); }

}  // namespace lbm
