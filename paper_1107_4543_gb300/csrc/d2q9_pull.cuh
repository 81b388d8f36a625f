// D2Q9 pull streaming with 128-bit vector I/O (device helpers).
//
// Storage: populations as 9 planes f[i][y][x] of `pitch` elements per row
// (pitch >= nx, a multiple of the vector width), periodic in x and y.  The
// buffer holds the post-collision populations of the previous step, so the
// pre-collision population at node (x, y) is f_i(x, y) = P_i(x - cx_i,
// y - cy_i): the collide-then-stream of section 2.1 (Eq. blbs) written as a
// pull.
//
// Work unit ("task"): one warp takes 32 consecutive chunks of V nodes
// (V * sizeof(T) = 16 bytes, or 8 bytes for BF16); see lane_pos.  Every plane is read with aligned vector loads;
// the +-1 x-shifts are formed from the neighbouring lane's chunk by a warp
// shuffle, and only lanes whose neighbouring chunk is elsewhere make one
// extra scalar load (a cache hit: the neighbouring warp or row loads the
// same line).  Periodic wrap is folded into the row index (y) and into
// those edge loads (x).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

// velocities c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1)
__host__ __device__ constexpr int CXd(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int CYd(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}

// ---------------------------------------------------------- element I/O
// Nodes per vector for the 16-bit storage types: 8 (16-byte vectors) or 4
// (8-byte vectors, half the registers).  Measured on GB300: FP16 streams
// fastest with 8, BF16 (whose 8-wide kernel needs ~180 registers) with 4.
#ifndef LBM_VF16
#define LBM_VF16 8
#endif
#ifndef LBM_VBF16
#define LBM_VBF16 4
#endif

template <int BYTES> struct RawOf;
template <> struct RawOf<16> {
  using type = uint4;
  static __device__ __forceinline__ void words(const uint4 &r, uint32_t *w) {
    w[0] = r.x; w[1] = r.y; w[2] = r.z; w[3] = r.w;
  }
  static __device__ __forceinline__ uint4 make(const uint32_t *w) {
    return make_uint4(w[0], w[1], w[2], w[3]);
  }
  static __device__ __forceinline__ uint4 zero() { return make_uint4(0, 0, 0, 0); }
};
template <> struct RawOf<8> {
  using type = uint2;
  static __device__ __forceinline__ void words(const uint2 &r, uint32_t *w) {
    w[0] = r.x; w[1] = r.y;
  }
  static __device__ __forceinline__ uint2 make(const uint32_t *w) {
    return make_uint2(w[0], w[1]);
  }
  static __device__ __forceinline__ uint2 zero() { return make_uint2(0, 0); }
};

template <typename T> struct Elem;

template <> struct Elem<float> {
  static constexpr int V = 4;
  using C = float;  // compute type
  using R = RawOf<16>;
  static __device__ __forceinline__ void unpack(const uint4 &r, float *o) {
    o[0] = __uint_as_float(r.x); o[1] = __uint_as_float(r.y);
    o[2] = __uint_as_float(r.z); o[3] = __uint_as_float(r.w);
  }
  static __device__ __forceinline__ uint4 pack(const float *v) {
    return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]),
                      __float_as_uint(v[2]), __float_as_uint(v[3]));
  }
  static __device__ __forceinline__ float one(const float *p) { return __ldg(p); }
};

template <> struct Elem<__half> {
  static constexpr int V = LBM_VF16;
  using C = float;
  using R = RawOf<2 * V>;
  static __device__ __forceinline__ void unpack(const typename R::type &r, float *o) {
    uint32_t w[V / 2];
    R::words(r, w);
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
      __half2 h = *reinterpret_cast<const __half2 *>(&w[k]);
      float2 f = __half22float2(h);
      o[2 * k] = f.x; o[2 * k + 1] = f.y;
    }
  }
  static __device__ __forceinline__ typename R::type pack(const float *v) {
    uint32_t w[V / 2];
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
      __half2 h = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
      w[k] = *reinterpret_cast<uint32_t *>(&h);
    }
    return R::make(w);
  }
  static __device__ __forceinline__ float one(const __half *p) {
    return __half2float(__ldg(p));
  }
};

template <> struct Elem<__nv_bfloat16> {
  static constexpr int V = LBM_VBF16;
  using C = float;
  using R = RawOf<2 * V>;
  static __device__ __forceinline__ void unpack(const typename R::type &r, float *o) {
    uint32_t w[V / 2];
    R::words(r, w);
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
      __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w[k]);
      float2 f = __bfloat1622float2(h);
      o[2 * k] = f.x; o[2 * k + 1] = f.y;
    }
  }
  static __device__ __forceinline__ typename R::type pack(const float *v) {
    uint32_t w[V / 2];
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
      __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
      w[k] = *reinterpret_cast<uint32_t *>(&h);
    }
    return R::make(w);
  }
  static __device__ __forceinline__ float one(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
  }
};

template <> struct Elem<double> {
  static constexpr int V = 2;
  using C = double;
  using R = RawOf<16>;
  static __device__ __forceinline__ void unpack(const uint4 &r, double *o) {
    o[0] = __hiloint2double((int)r.y, (int)r.x);
    o[1] = __hiloint2double((int)r.w, (int)r.z);
  }
  static __device__ __forceinline__ uint4 pack(const double *v) {
    return make_uint4((unsigned)__double2loint(v[0]), (unsigned)__double2hiint(v[0]),
                      (unsigned)__double2loint(v[1]), (unsigned)__double2hiint(v[1]));
  }
  static __device__ __forceinline__ double one(const double *p) { return __ldg(p); }
};

// Work mapping: the lattice's rows of cpr = pitch / V chunk slots (the
// ceil(nx / V) real chunks, then the padding up to the 128-byte row pitch)
// form one row-major sequence and warp task k takes slots 32k .. 32k+31.
// Every task then starts on a 128-byte line in all 9 planes (the y-shifted
// rows too, the pitch being whole lines), and a warp may span rows, so
// lanes have work whatever nx is; padding slots are inactive lanes.  A lane
// whose neighbouring chunk is not in the neighbouring lane loads the edge
// element itself.

// geometry of one lattice as the step kernels see it
struct Geom {
  int nx, ny, pitch;
  int nchunks;      // real vectors per row: ceil(nx / V)
  int cpr;          // chunk slots per row: pitch / V (>= nchunks)
  long long plane;  // pitch * ny
  long long tasks;  // warp tasks per step: ceil(cpr * ny / 32)
  // row = slot / cpr as (slot * dmul) >> dshift, exact for slot indices
  // below 2^31 (dshift = 31 + ceil(log2 cpr), dmul = ceil(2^dshift / cpr));
  // small = the lattice's slots (+ one warp) fit
  unsigned long long dmul;
  int dshift;
  int small;
};

// Position of this lane for task `task` of a lattice.
struct LanePos {
  int y, x0;         // row, first node of the chunk
  bool first, last;  // the row's previous / next chunk is not in the previous / next lane
  bool active;       // a real chunk: slot in the lattice and xc < nchunks
};

template <int V>
__device__ __forceinline__ LanePos lane_pos(const Geom &g, long long task, int lane) {
  LanePos p;
  const long long c = task * 32 + lane;
  int y, xc;
  if (g.small) {  // multiply-shift division
    const unsigned cu = (unsigned)c;
    y = (int)(((unsigned long long)cu * g.dmul) >> g.dshift);
    xc = (int)(cu - (unsigned)y * (unsigned)g.cpr);
  } else {
    y = (int)(c / g.cpr);
    xc = (int)(c - (long long)y * g.cpr);
  }
  p.active = y < g.ny && xc < g.nchunks;
  if (!p.active) y = xc = 0;
  p.y = y;
  p.x0 = xc * V;
  p.first = lane == 0 || xc == 0;
  p.last = lane == 31 || xc + 1 == g.nchunks;
  return p;
}

// Pull the 9 pre-collision populations of the V nodes of this lane's chunk
// into out[i][e] (compute type C; storage value times inv_scale when
// SCALED).  All 32 lanes must call it (it shuffles); inactive lanes get
// zeros.  Elements of padding columns (x >= nx) get unspecified values that
// never reach a real node.
//
// Two phases, so that every load of the task is in flight at once: first
// the 9 aligned 16-byte loads and the (predicated) edge loads of the six
// x-shifted planes, then the shuffles that assemble the shifted vectors.
template <typename T, bool SCALED>
__device__ __forceinline__ void pull9(const T *__restrict__ src, const Geom &g,
                                      const LanePos &p,
                                      typename Elem<T>::C inv_scale,
                                      typename Elem<T>::C (&out)[9][Elem<T>::V]) {
  using C = typename Elem<T>::C;
  constexpr int V = Elem<T>::V;
  const int last = g.nx - 1;
  // which element of this chunk is the last real node (or -1)
  const int e_last = (p.x0 <= last && last < p.x0 + V) ? last - p.x0 : -1;
  // edge loads: a lane whose previous chunk is not in the previous lane (or
  // x0 = 0, the wrap) needs x0 - 1 for the planes with cx = +1; one whose
  // next chunk is not in the next lane needs x0 + V for cx = -1; the chunk
  // holding the last node needs column 0 for cx = -1
  const bool need_prev = p.active && p.first;
  const int x_prev = p.x0 == 0 ? last : p.x0 - 1;
  const bool need_next = p.active && p.last && p.x0 + V <= last;
  const bool need_wrap = p.active && e_last >= 0;
  auto sc = [&](C a) -> C { return SCALED ? a * inv_scale : a; };

  using RawT = typename Elem<T>::R::type;
  RawT raw[9];
  C edge[9];
  C wrap0[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cx = CXd(i), cy = CYd(i);
    int ys = p.y - cy;
    ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
    const T *row = src + (long long)i * g.plane + (long long)ys * g.pitch;
    raw[i] = p.active ? __ldg(reinterpret_cast<const RawT *>(row + p.x0)) : Elem<T>::R::zero();
    edge[i] = C(0);
    wrap0[i] = C(0);
    if (cx == 1) {
      if (need_prev) edge[i] = Elem<T>::one(row + x_prev);
    } else if (cx == -1) {
      if (need_next) edge[i] = Elem<T>::one(row + p.x0 + V);
      if (need_wrap) wrap0[i] = Elem<T>::one(row);
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cx = CXd(i);
    C v[V];
    Elem<T>::unpack(raw[i], v);
    if (cx == 0) {
#pragma unroll
      for (int e = 0; e < V; ++e) out[i][e] = sc(v[e]);
    } else if (cx == 1) {
      // node x pulls from x - 1
      C prev = __shfl_up_sync(0xffffffffu, v[V - 1], 1);
      if (need_prev) prev = edge[i];
      out[i][0] = sc(prev);
#pragma unroll
      for (int e = 1; e < V; ++e) out[i][e] = sc(v[e - 1]);
    } else {
      // node x pulls from x + 1 (column 0 for the last real node)
      C next = __shfl_down_sync(0xffffffffu, v[0], 1);
      if (need_next) next = edge[i];
#pragma unroll
      for (int e = 0; e < V - 1; ++e) out[i][e] = sc(v[e + 1]);
      out[i][V - 1] = sc(next);
      if (need_wrap) {
        const C w = sc(wrap0[i]);
#pragma unroll
        for (int e = 0; e < V; ++e)
          if (e == e_last) out[i][e] = w;
      }
    }
  }
}

// Store the 9 post-collision populations of this lane's chunk (aligned
// 16-byte stores; padding columns x >= nx receive unspecified values).
template <typename T, bool SCALED>
__device__ __forceinline__ void store9(T *__restrict__ dst, const Geom &g, const LanePos &p,
                                       typename Elem<T>::C scale,
                                       typename Elem<T>::C (&in)[9][Elem<T>::V]) {
  using C = typename Elem<T>::C;
  constexpr int V = Elem<T>::V;
  if (!p.active) return;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    C v[V];
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = SCALED ? in[i][e] * scale : in[i][e];
    T *row = dst + (long long)i * g.plane + (long long)p.y * g.pitch;
    *reinterpret_cast<typename Elem<T>::R::type *>(row + p.x0) = Elem<T>::pack(v);
  }
}

}  // namespace lbm
