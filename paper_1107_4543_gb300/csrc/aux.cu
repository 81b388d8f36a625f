// Auxiliary kernels: equilibrium initialisation, moments, population
// get/set (checkpoint), largest deviation (FP16 scale), and the FP64 drift
// reduction.  None of them is on the per-step path.
//
// Compiled with -fmad=false: for LBM_F64 the equilibrium and the moments
// follow the operation order of a plain matrix-vector implementation
// (f^eq = M^-1 m^eq summed over k = 0..8 left to right; rho, j = rows 0..2 of
// M f), so they are bit-identical to a straightforward FP64 CPU version.
#include <math.h>

#include "lbm_internal.h"
#include "node_xy.cuh"

namespace lbm {

// Lallemand-Luo D2Q9 matrix, rows rho, jx, jy, e, eps, qx, qy, pxx, pxy
// (the paper's moment order, section 2.3), and its row norms.
__host__ __device__ constexpr int mm(int k, int j) {
  constexpr int T[9][9] = {
      {1, 1, 1, 1, 1, 1, 1, 1, 1},     {0, 1, 0, -1, 0, 1, -1, -1, 1},
      {0, 0, 1, 0, -1, 1, 1, -1, -1},  {-4, -1, -1, -1, -1, 2, 2, 2, 2},
      {4, -2, -2, -2, -2, 1, 1, 1, 1}, {0, -2, 0, 2, 0, 1, -1, -1, 1},
      {0, 0, -2, 0, 2, 1, 1, -1, -1},  {0, 1, -1, 1, -1, 0, 0, 0, 0},
      {0, 0, 0, 0, 0, 1, -1, 1, -1}};
  return T[k][j];
}
__host__ __device__ constexpr double dnorm(int k) {
  return k == 0 ? 9.0 : (k <= 2 ? 6.0 : (k <= 4 ? 36.0 : (k <= 6 ? 12.0 : 4.0)));
}

// f^eq = M^-1 m^eq(rho, j), m^eq of section 2.3
__host__ __device__ inline void feq_of_j(double rho, double jx, double jy, double f[9]) {
  const double jsq = jx * jx + jy * jy;
  const double m[9] = {rho, jx, jy, -2.0 * rho + 3.0 * jsq / rho, rho - 3.0 * jsq / rho,
                       -jx, -jy, (jx * jx - jy * jy) / rho, jx * jy / rho};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (mm(k, i) != 0) acc = acc + ((double)mm(k, i) / dnorm(k)) * m[k];
    f[i] = acc;
  }
}

// f^eq(rho, u) with j = rho u formed first, as a plain implementation does
__host__ __device__ inline void feq_canonical(double rho, double ux, double uy, double f[9]) {
  feq_of_j(rho, rho * ux, rho * uy, f);
}

void host_feq_j(double rho, double jx, double jy, double out[9]) {
  feq_of_j(rho, jx, jy, out);
}

__device__ __forceinline__ int wrapi(int a, int n) {
  return a < 0 ? a + n : (a >= n ? a - n : a);
}

__device__ __forceinline__ double load_stored(const AuxView &a, long long idx) {
  switch (a.dtype) {
    case LBM_F64:
    case LBM_F64DEV: return static_cast<const double *>(a.buf)[idx];
    case LBM_F32DEV: return (double)static_cast<const float *>(a.buf)[idx];
    case LBM_F16DEV: return (double)__half2float(static_cast<const __half *>(a.buf)[idx]) / a.scale;
    default: return (double)__bfloat162float(static_cast<const __nv_bfloat16 *>(a.buf)[idx]);
  }
}

// stored representation of population i with full value fv
__device__ __forceinline__ void store_value(const AuxView &a, long long idx, int i, double fv) {
  switch (a.dtype) {
    case LBM_F64: static_cast<double *>(a.buf)[idx] = fv; break;
    case LBM_F64DEV: static_cast<double *>(a.buf)[idx] = fv - a.f0[i]; break;
    case LBM_F32DEV: static_cast<float *>(a.buf)[idx] = (float)(fv - a.f0[i]); break;
    case LBM_F16DEV:
      static_cast<__half *>(a.buf)[idx] = __float2half_rn((float)((fv - a.f0[i]) * a.scale));
      break;
    default:
      static_cast<__nv_bfloat16 *>(a.buf)[idx] = __float2bfloat16_rn((float)(fv - a.f0[i]));
  }
}

// macroscopic field at node (x, y): device arrays, or an analytic field
__device__ __forceinline__ void field_at(const AuxView &a, const double *rho, const double *ux,
                                         const double *uy, int kind, const double *p, int x,
                                         int y, double &r, double &u, double &v) {
  const long long n = (long long)y * a.g.nx + x;
  if (kind == 0) {
    r = rho[n]; u = ux[n]; v = uy[n];
    return;
  }
  const double u0x = a.rho0 > 0 ? a.jx0 / a.rho0 : 0.0, u0y = a.rho0 > 0 ? a.jy0 / a.rho0 : 0.0;
  if (kind == LBM_INIT_GAUSSIAN) {
    const double nxd = a.g.nx, nyd = a.g.ny;
    double dx = fmod((double)x - p[2] + 0.5 * nxd, nxd);
    if (dx < 0) dx += nxd;
    dx -= 0.5 * nxd;
    double dy = fmod((double)y - p[3] + 0.5 * nyd, nyd);
    if (dy < 0) dy += nyd;
    dy -= 0.5 * nyd;
    const double alpha = 0.69314718055994530942 / (p[1] * p[1]);
    r = a.rho0 + p[0] * exp(-alpha * (dx * dx + dy * dy));
    u = u0x; v = u0y;
  } else {  // LBM_INIT_PLANE
    const double c = cos(2.0 * 3.14159265358979323846 * p[1] * (double)x / (double)a.g.nx);
    r = a.rho0 + p[0] * c;
    u = u0x + p[0] * c / (1.7320508075688772935 * a.rho0);
    v = u0y;
  }
}

struct AnalyticParams { double p[8]; };

// f = f^eq(field) at node x.  Population i of node x goes to slot x - c_i,
// where the next step's pull (f_i(x) = P_i(x - c_i)) reads it.
// bad (may be null) counts nodes whose field is not finite or has rho <= 0
__global__ void k_init_eq(AuxView a, const double *rho, const double *ux, const double *uy,
                          int kind, AnalyticParams ap, unsigned int *bad) {
  const long long N = (long long)a.g.nx * a.g.ny;
  unsigned int nbad = 0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int x, y;
    node_xy(n, a.g.nx, x, y);
    double r, u, v, f[9];
    field_at(a, rho, ux, uy, kind, ap.p, x, y, r, u, v);
    if (!(r > 0.0) || !isfinite(r) || !isfinite(u) || !isfinite(v)) ++nbad;
    feq_canonical(r, u, v, f);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int xs = wrapi(x - CXd(i), a.g.nx), ys = wrapi(y - CYd(i), a.g.nyw);
      store_value(a, (long long)i * a.g.plane + (long long)ys * a.g.rstride + xs, i, f[i]);
    }
  }
  if (bad && nbad) atomicAdd(bad, nbad);
}

// Point source: set the pre-collision populations of node (x, y) to fs by
// writing the 9 slots the next step's pull reads for that node.
struct NodePops { double f[9]; };

__global__ void k_force_node(AuxView a, int x, int y, NodePops fs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int xs = wrapi(x - CXd(i), a.g.nx), ys = wrapi(y - CYd(i), a.g.nyw);
    store_value(a, (long long)i * a.g.plane + (long long)ys * a.g.rstride + xs, i, fs.f[i]);
  }
}

cudaError_t launch_force_node(const AuxView &a, int x, int y, const double fs[9],
                              cudaStream_t st) {
  NodePops p;
  for (int i = 0; i < 9; ++i) p.f[i] = fs[i];
  k_force_node<<<1, 32, 0, st>>>(a, x, y, p);
  return cudaGetLastError();
}

// the same, with the nine populations read from device memory (a table the
// host fills before a captured sequence of forced steps)
__global__ void k_force_node_tab(AuxView a, int x, int y, const double *fs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int xs = wrapi(x - CXd(i), a.g.nx), ys = wrapi(y - CYd(i), a.g.nyw);
    store_value(a, (long long)i * a.g.plane + (long long)ys * a.g.rstride + xs, i, fs[i]);
  }
}

cudaError_t launch_force_node_tab(const AuxView &a, int x, int y, const double *fs_dev,
                                  cudaStream_t st) {
  k_force_node_tab<<<1, 32, 0, st>>>(a, x, y, fs_dev);
  return cudaGetLastError();
}

__global__ void k_maxdev_eq(AuxView a, const double *rho, const double *ux, const double *uy,
                            int kind, AnalyticParams ap, unsigned int *max_bits) {
  const long long N = (long long)a.g.nx * a.g.ny;
  float m = 0.0f;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int x, y;
    node_xy(n, a.g.nx, x, y);
    double r, u, v, f[9];
    field_at(a, rho, ux, uy, kind, ap.p, x, y, r, u, v);
    feq_canonical(r, u, v, f);
#pragma unroll
    for (int i = 0; i < 9; ++i) m = fmaxf(m, (float)fabs(f[i] - a.f0[i]));
  }
  atomicMax(max_bits, __float_as_uint(m));
}

// pre-collision populations at node (x, y): f_i(x) = P_i(x - c_i)
__device__ __forceinline__ void gather(const AuxView &a, int x, int y, double f[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int xs = wrapi(x - CXd(i), a.g.nx), ys = wrapi(y - CYd(i), a.g.nyw);
    f[i] = load_stored(a, (long long)i * a.g.plane + (long long)ys * a.g.rstride + xs);
  }
}

__global__ void k_moments(AuxView a, double *rho, double *ux, double *uy) {
  const long long N = (long long)a.g.nx * a.g.ny;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int x, y;
    node_xy(n, a.g.nx, x, y);
    double f[9];
    gather(a, x, y, f);
    double r = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    double jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    double jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    if (a.dtype != LBM_F64) {
      r = a.rho0 + r;
      jx = a.jx0 + jx;
      jy = a.jy0 + jy;
    }
    rho[n] = r;
    ux[n] = jx / r;
    uy[n] = jy / r;
  }
}

__global__ void k_get_pop(AuxView a, double *f) {
  const long long N = (long long)a.g.nx * a.g.ny;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int x, y;
    node_xy(n, a.g.nx, x, y);
    double g[9];
    gather(a, x, y, g);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i * N + n] = a.dtype == LBM_F64 ? g[i] : a.f0[i] + g[i];
  }
}

__global__ void k_set_pop(AuxView a, const double *f) {
  const long long N = (long long)a.g.nx * a.g.ny;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int x, y;
    node_xy(n, a.g.nx, x, y);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int xs = wrapi(x - CXd(i), a.g.nx), ys = wrapi(y - CYd(i), a.g.nyw);
      store_value(a, (long long)i * a.g.plane + (long long)ys * a.g.rstride + xs, i, f[i * N + n]);
    }
  }
}

__global__ void k_maxdev_pop(AuxView a, const double *f, unsigned int *max_bits) {
  const long long N = (long long)a.g.nx * a.g.ny;
  float m = 0.0f;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < 9; ++i) m = fmaxf(m, (float)fabs(f[i * N + n] - a.f0[i]));
  }
  atomicMax(max_bits, __float_as_uint(m));
}

// ------------------------------------------------------------- drift
// Stage 1: a fixed grid of DRIFT_BLOCKS blocks; thread t of block b sums the
// nodes n = b * 256 + t + k * (DRIFT_BLOCKS * 256) in increasing k, then the
// block reduces its 256 partials by a fixed tree.  Stage 2: one block sums
// the DRIFT_BLOCKS partials by a fixed tree.  The order never depends on
// scheduling, so the result is reproducible bit for bit.
constexpr int DRIFT_BLOCKS = 1024;
constexpr int DRIFT_THREADS = 256;
int drift_blocks() { return DRIFT_BLOCKS; }

// s + e = a + b exactly (Knuth's TwoSum; this file is built without FMA
// contraction, which the identity needs)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// float-float accumulator: hi + lo carries about 48 significant bits
struct FF {
  float hi, lo;
  __device__ __forceinline__ void add(float a) {
    float t;
    two_sum(hi, a, hi, t);
    lo += t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Mass and momentum deviations of one node's 9 stored populations (the
// node's own slots, which is all a lattice-wide sum needs), non-finite
// values counted in bad and taken as zero.  FP64 storage sums in FP64; the
// deviation types sum their FP32 values as float-float (GB300 runs FP32 at
// many times its FP64 rate, and the 9-term sums keep ~48 bits).
__device__ __forceinline__ void node_sums(const AuxView &a, long long off, double &r, double &jx,
                                          double &jy, unsigned &bad) {
  if (a.dtype == LBM_F64 || a.dtype == LBM_F64DEV) {
    // deviations from the base populations first: f_i - f0_i is exact while
    // f_i stays within a factor two of f0_i (Sterbenz), so the node's sums
    // round at the size of the perturbation, not at the size of f
    // (LBM_F64DEV stores the deviations themselves)
    const double sub = a.dtype == LBM_F64 ? 1.0 : 0.0;
    double d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const double v = static_cast<const double *>(a.buf)[(long long)i * a.g.plane + off];
      if (!isfinite(v)) { ++bad; d[i] = 0.0; }
      else d[i] = v - sub * a.f0[i];
    }
    r = d[0] + d[1] + d[2] + d[3] + d[4] + d[5] + d[6] + d[7] + d[8];
    jx = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
    jy = d[2] - d[4] + d[5] + d[6] - d[7] - d[8];
    return;
  }
  float f[9];
  const float inv = (float)(1.0 / a.scale);  // a power of two
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const long long idx = (long long)i * a.g.plane + off;
    float v;
    if (a.dtype == LBM_F32DEV) v = static_cast<const float *>(a.buf)[idx];
    else if (a.dtype == LBM_F16DEV) v = __half2float(static_cast<const __half *>(a.buf)[idx]) * inv;
    else v = __bfloat162float(static_cast<const __nv_bfloat16 *>(a.buf)[idx]);
    if (!isfinite(v)) { ++bad; v = 0.0f; }
    f[i] = v;
  }
  FF s0{f[0], 0.0f}, s1{f[1], 0.0f}, s2{f[2], 0.0f};
#pragma unroll
  for (int i = 1; i < 9; ++i) s0.add(f[i]);
  s1.add(-f[3]); s1.add(f[5]); s1.add(-f[6]); s1.add(-f[7]); s1.add(f[8]);
  s2.add(-f[4]); s2.add(f[5]); s2.add(f[6]); s2.add(-f[7]); s2.add(-f[8]);
  r = s0.value();
  jx = s1.value();
  jy = s2.value();
}

__global__ void __launch_bounds__(DRIFT_THREADS) k_drift1(AuxView a, double *partials) {
  __shared__ double sh[4][DRIFT_THREADS];
  const long long N = (long long)a.g.nx * a.g.ny;
  double s0 = 0, s1 = 0, s2 = 0;
  unsigned bad = 0;
  const long long n0 = blockIdx.x * (long long)DRIFT_THREADS + threadIdx.x;
  const long long stride = (long long)DRIFT_BLOCKS * DRIFT_THREADS;
  if (n0 < N) {
    NodeWalk w(n0, stride, a.g.nx);
    for (long long n = n0; n < N; n += stride, w.next()) {
      double r, jx, jy;
      node_sums(a, (long long)w.y * a.g.rstride + w.x, r, jx, jy, bad);
      s0 += r; s1 += jx; s2 += jy;
    }
  }
  sh[0][threadIdx.x] = s0; sh[1][threadIdx.x] = s1;
  sh[2][threadIdx.x] = s2; sh[3][threadIdx.x] = (double)bad;
  __syncthreads();
  for (int w = DRIFT_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) partials[blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(DRIFT_BLOCKS) k_drift2(const double *partials, double *out) {
  __shared__ double sh[4][DRIFT_BLOCKS];
  for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] = partials[threadIdx.x * 4 + c];
  __syncthreads();
  for (int w = DRIFT_BLOCKS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = sh[threadIdx.x][0];
}

// Batched drift: lattice l is reduced by BD_BLOCKS blocks of blockIdx.y = l;
// thread t of block b sums nodes b * 256 + t + k * (BD_BLOCKS * 256) in
// increasing k, each block reduces by a fixed tree, and one warp per lattice
// adds the BD_BLOCKS partials in order: reproducible per lattice, whatever
// the rest of the batch.
constexpr int BD_BLOCKS = 16;

__global__ void __launch_bounds__(DRIFT_THREADS)
k_batch_drift1(const AuxView *__restrict__ views, double *partials) {
  __shared__ double sh[4][DRIFT_THREADS];
  const AuxView &a = views[blockIdx.y];
  const long long N = (long long)a.g.nx * a.g.ny;
  double s0 = 0, s1 = 0, s2 = 0;
  unsigned bad = 0;
  const long long n0 = blockIdx.x * (long long)DRIFT_THREADS + threadIdx.x;
  const long long stride = (long long)BD_BLOCKS * DRIFT_THREADS;
  if (n0 < N) {
    NodeWalk w(n0, stride, a.g.nx);
    for (long long n = n0; n < N; n += stride, w.next()) {
      double r, jx, jy;
      node_sums(a, (long long)w.y * a.g.rstride + w.x, r, jx, jy, bad);
      s0 += r; s1 += jx; s2 += jy;
    }
  }
  sh[0][threadIdx.x] = s0; sh[1][threadIdx.x] = s1;
  sh[2][threadIdx.x] = s2; sh[3][threadIdx.x] = (double)bad;
  __syncthreads();
  for (int w = DRIFT_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 4; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4)
    partials[((long long)blockIdx.y * BD_BLOCKS + blockIdx.x) * 4 + threadIdx.x] =
        sh[threadIdx.x][0];
}

__global__ void k_batch_drift2(const double *partials, int n, double *out) {
  const int l = blockIdx.x * (blockDim.x / 4) + threadIdx.x / 4;
  const int c = threadIdx.x & 3;
  if (l >= n) return;
  double s = 0;
  for (int b = 0; b < BD_BLOCKS; ++b) s += partials[((long long)l * BD_BLOCKS + b) * 4 + c];
  out[l * 4 + c] = s;
}

int batch_drift_partials(int n) { return n * BD_BLOCKS * 4; }

cudaError_t launch_batch_drift(const AuxView *views_dev, int n, double *partials, double *out,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_batch_drift1<<<dim3(BD_BLOCKS, n), DRIFT_THREADS, 0, st>>>(views_dev, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_batch_drift2<<<(n + 63) / 64, 256, 0, st>>>(partials, n, out);
  return cudaGetLastError();
}

// ----------------------------------------------------------- launchers
static unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  long long cap = (long long)sm_count() * 16;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

static AnalyticParams make_ap(const double *p) {
  AnalyticParams ap;
  for (int k = 0; k < 8; ++k) ap.p[k] = p ? p[k] : 0.0;
  return ap;
}

cudaError_t launch_init_eq(const AuxView &a, const double *rho, const double *ux,
                           const double *uy, int kind, const double *params, cudaStream_t st,
                           unsigned int *bad) {
  if (kind == 0 && a.dtype != LBM_F64) return launch_init_dev(a, rho, ux, uy, st, bad);
  const long long N = (long long)a.g.nx * a.g.ny;
  if (bad) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
  }
  k_init_eq<<<grid_for(N), 256, 0, st>>>(a, rho, ux, uy, kind, make_ap(params), bad);
  return cudaGetLastError();
}

cudaError_t launch_maxdev_eq(const AuxView &a, const double *rho, const double *ux,
                             const double *uy, int kind, const double *params,
                             unsigned int *max_bits, cudaStream_t st) {
  if (kind == 0 && a.dtype != LBM_F64) return launch_maxdev_dev(a, rho, ux, uy, max_bits, st);
  const long long N = (long long)a.g.nx * a.g.ny;
  cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  k_maxdev_eq<<<grid_for(N), 256, 0, st>>>(a, rho, ux, uy, kind, make_ap(params), max_bits);
  return cudaGetLastError();
}

cudaError_t launch_moments(const AuxView &a, double *rho, double *ux, double *uy,
                           cudaStream_t st) {
  if (a.dtype != LBM_F64) return launch_moments_dev(a, rho, ux, uy, st);
  const long long N = (long long)a.g.nx * a.g.ny;
  k_moments<<<grid_for(N), 256, 0, st>>>(a, rho, ux, uy);
  return cudaGetLastError();
}

cudaError_t launch_get_pop(const AuxView &a, double *f, cudaStream_t st) {
  const long long N = (long long)a.g.nx * a.g.ny;
  k_get_pop<<<grid_for(N), 256, 0, st>>>(a, f);
  return cudaGetLastError();
}

cudaError_t launch_set_pop(const AuxView &a, const double *f, cudaStream_t st) {
  const long long N = (long long)a.g.nx * a.g.ny;
  k_set_pop<<<grid_for(N), 256, 0, st>>>(a, f);
  return cudaGetLastError();
}

cudaError_t launch_maxdev_pop(const AuxView &a, const double *f, unsigned int *max_bits,
                              cudaStream_t st) {
  const long long N = (long long)a.g.nx * a.g.ny;
  cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  k_maxdev_pop<<<grid_for(N), 256, 0, st>>>(a, f, max_bits);
  return cudaGetLastError();
}

cudaError_t launch_drift(const AuxView &a, double *partials, double *out, cudaStream_t st) {
  k_drift1<<<DRIFT_BLOCKS, DRIFT_THREADS, 0, st>>>(a, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_drift2<<<1, DRIFT_BLOCKS, 0, st>>>(partials, out);
  return cudaGetLastError();
}

// acc[i] += add[i] for i < n (the pipelined batch solves' invalid-field
// totals)
__global__ void k_add_u32(unsigned int *acc, const unsigned int *add, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) acc[i] += add[i];
}

cudaError_t launch_add_u32(unsigned int *acc, const unsigned int *add, int n, cudaStream_t st) {
  if (n < 1) return cudaSuccess;
  k_add_u32<<<(n + 255) / 256, 256, 0, st>>>(acc, add, n);
  return cudaGetLastError();
}

}  // namespace lbm
