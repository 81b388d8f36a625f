// D2Q9 pull streaming with 128-bit vector I/O (device helpers).
//
// Storage: populations as 9 planes f[i][y][x] of `pitch` elements per row
// (pitch >= nx, a multiple of the vector width), periodic in x and y;
// element (i, y, x) at i * plane + y * rstride + x (Geom): with plane = pitch
// and rstride = 9 pitch, row y of the nine planes lie back to back.  The
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
// (8-byte vectors).  With the packed pull (pull9_packed: shifts on packed
// words, two nodes unpacked at a time) both stream fastest with 8 on GB300:
// 8192^2 FP16 6.46 TB/s, BF16 6.25 TB/s (4-wide: 5.55 and 5.41).
#ifndef LBM_VF16
#define LBM_VF16 8
#endif
#ifndef LBM_VBF16
#define LBM_VBF16 8
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
  // two packed elements <-> two floats (element 2k in the low half)
  static __device__ __forceinline__ void unpack2(uint32_t w, float *o) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
    o[0] = f.x; o[1] = f.y;
  }
  static __device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
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
  static __device__ __forceinline__ void unpack2(uint32_t w, float *o) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
    o[0] = f.x; o[1] = f.y;
  }
  static __device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
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
  int nx, ny, pitch;  // pitch: elements per row of one plane (a multiple of 128 bytes)
  int nchunks;      // real vectors per row: ceil(nx / V)
  int cpr;          // chunk slots per row of the task mapping: pitch / V, or nchunks
  // y extent of the periodic wrap: ny for a whole periodic lattice; 0 for a
  // slab of rows whose neighbouring rows y = -1 and y = ny are stored halo
  // rows (the wrap is then the identity)
  int nyw;
  long long plane;    // offset between planes i and i + 1 (elements)
  long long rstride;  // offset between rows y and y + 1 of one plane (elements)
  // element (i, y, x) lives at i * plane + y * rstride + x
  long long tasks;  // warp tasks per step: ceil(cpr * ny / 32)
  // row = slot / cpr as (slot * dmul) >> dshift, exact for slot indices
  // below 2^31 (dshift = 31 + ceil(log2 cpr), dmul = ceil(2^dshift / cpr));
  // small = the lattice's slots (+ one warp) fit
  unsigned long long dmul;
  int dshift;
  int small;
};

// Geometry of an nx x ny lattice stored V nodes per vector of elements of
// esize bytes (host side; shared with the host-compiled index tests).
inline Geom make_geom(int nx, int ny, int V, int esize) {
  Geom g;
  g.nx = nx;
  g.ny = ny;
  // rows start on 128-byte lines; 16-bit rows on 64-byte halves, which
  // leaves fewer padding lanes in short rows (measured +1.5% on the
  // 512-lattice batch in FP16 and BF16, the kernels being issue-bound)
  const int abytes = esize == 2 ? 64 : 128;
  const int align = V > abytes / esize ? V : abytes / esize;
  g.pitch = (nx + align - 1) / align * align;
  g.nyw = ny;
  g.nchunks = (nx + V - 1) / V;
  // chunk slots per row of the task mapping: whole lines of chunks, so that
  // every task starts on a line; but rows whose padding slots exceed an
  // eighth of the row (short rows: a 40-node FP16 row fills 5 of its 8
  // slots) map their real chunks only, leaving no lane idle, tasks then
  // starting anywhere in a row
  const int slots = g.pitch / V;
  g.cpr = (slots - g.nchunks) * 8 > slots ? g.nchunks : slots;
  // row-interleaved planes: row y of planes 0..8 lie back to back, so the
  // nine rows a warp task streams share DRAM pages (measured +0.6% on the
  // batched step, +2% on one 8192^2 lattice against plane after plane)
  g.plane = g.pitch;
  g.rstride = 9LL * g.pitch;
  g.tasks = ((long long)g.cpr * ny + 31) / 32;
  int k = 31;
  while ((1LL << (k - 31)) < (long long)g.cpr) ++k;  // 31 + ceil(log2 cpr)
  g.dshift = k;
  g.dmul = ((1ULL << k) + (unsigned long long)g.cpr - 1) / (unsigned long long)g.cpr;
  g.small = g.tasks * 32 < (1LL << 31) ? 1 : 0;
  return g;
}

// Position of this lane for task `task` of a lattice.
struct LanePos {
  int y, x0;         // row, first node of the chunk
  bool first, last;  // the row's previous / next chunk is not in the previous / next lane
  bool active;       // a real chunk: slot in the lattice and xc < nchunks
};

template <int V>
__host__ __device__ __forceinline__ LanePos lane_pos(const Geom &g, long long task, int lane) {
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
    ys = ys < 0 ? ys + g.nyw : (ys >= g.nyw ? ys - g.nyw : ys);
    const T *row = src + (long long)i * g.plane + (long long)ys * g.rstride;
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

// The lane holding a row's last real chunk also writes the padding chunk
// after it when its own chunk ends in the middle of a 32-byte sector, so
// that the stores of a row cover whole sectors: a sector written in part
// makes the memory system read the rest before writing it back (measured
// on 100 x 700 FP16 lattices: 26 B read per node against 18).  Padding
// columns hold unspecified values.
// With 16-byte chunks and rows starting on 64-byte boundaries, a row ends
// in the middle of a sector exactly when its chunk count is odd, and the
// pitch (a multiple of four chunks) then has room for the next chunk.
template <typename T>
__device__ __forceinline__ bool fills_sector(const Geom &g, const LanePos &p) {
  constexpr int V = Elem<T>::V;
  static_assert(V * sizeof(T) == 16 || V * sizeof(T) == 8, "16- or 8-byte chunks");
  return V * sizeof(T) == 16 && (g.nchunks & 1) && p.active && p.x0 + V >= g.nx;
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
    T *row = dst + (long long)i * g.plane + (long long)p.y * g.rstride;
    *reinterpret_cast<typename Elem<T>::R::type *>(row + p.x0) = Elem<T>::pack(v);
  }
  if (fills_sector<T>(g, p)) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      T *row = dst + (long long)i * g.plane + (long long)p.y * g.rstride;
      *reinterpret_cast<typename Elem<T>::R::type *>(row + p.x0 + V) = Elem<T>::R::zero();
    }
  }
}

// 16-bit storage types: the same pull with the populations kept packed,
// out[i][k] holding nodes 2k (low half) and 2k + 1 (high half) of this
// lane's chunk.  The +-1 x-shifts are byte permutes of neighbouring words
// (and of the neighbouring lane's edge word), which move the stored bits
// unchanged, so the caller can unpack, collide and repack two nodes at a
// time instead of holding 9 x V floats per lane.
__device__ __forceinline__ uint32_t raw16(const void *p) {
  return (uint32_t)__ldg(static_cast<const unsigned short *>(p));
}

// Where a lane's +-1 x-shifted elements come from when the neighbouring
// lane does not hold them: the previous element for the planes with
// cx = +1 (x_prev: x0 - 1, or column nx - 1 across the wrap), the next one
// for cx = -1, and column 0 for the element of the last real node.
struct EdgeInfo {
  int e_last;  // which element of this chunk is the last real node (or -1)
  int x_prev;
  bool need_prev, need_next, need_wrap;
};

__device__ __forceinline__ EdgeInfo edge_info(const Geom &g, const LanePos &p, int V) {
  EdgeInfo E;
  const int last = g.nx - 1;
  E.e_last = (p.x0 <= last && last < p.x0 + V) ? last - p.x0 : -1;
  E.need_prev = p.active && p.first;
  E.x_prev = p.x0 == 0 ? last : p.x0 - 1;
  E.need_next = p.active && p.last && p.x0 + V <= last;
  E.need_wrap = p.active && E.e_last >= 0;
  return E;
}

// the (predicated) scalar edge loads of plane i; raw16 values
template <typename T>
__device__ __forceinline__ void edge_loads_packed(const T *row, const LanePos &p,
                                                  const EdgeInfo &E, int i, uint32_t &edge,
                                                  uint32_t &wrap0) {
  constexpr int V = Elem<T>::V;
  const int cx = CXd(i);
  edge = 0u;
  wrap0 = 0u;
  if (cx == 1) {
    if (E.need_prev) edge = raw16(row + E.x_prev);
  } else if (cx == -1) {
    if (E.need_next) edge = raw16(row + p.x0 + V);
    if (E.need_wrap) wrap0 = raw16(row);
  }
}

// Second phase of the packed pull: the shifted vectors from this lane's
// chunks (raw), the neighbouring lanes' (shuffles) and the edge values.
template <typename T>
__device__ __forceinline__ void assemble_packed(const typename Elem<T>::R::type (&raw)[9],
                                                const EdgeInfo &E, const uint32_t (&edge)[9],
                                                const uint32_t (&wrap0)[9],
                                                uint32_t (&out)[9][Elem<T>::V / 2]) {
  constexpr int W = Elem<T>::V / 2;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cx = CXd(i);
    uint32_t v[W];
    Elem<T>::R::words(raw[i], v);
    if (cx == 0) {
#pragma unroll
      for (int k = 0; k < W; ++k) out[i][k] = v[k];
    } else if (cx == 1) {
      // node x pulls from x - 1: word k = (high half of v[k-1], low half of v[k])
      uint32_t prevw = __shfl_up_sync(0xffffffffu, v[W - 1], 1);
      if (E.need_prev) prevw = edge[i] << 16;
      out[i][0] = __byte_perm(prevw, v[0], 0x5432);
#pragma unroll
      for (int k = 1; k < W; ++k) out[i][k] = __byte_perm(v[k - 1], v[k], 0x5432);
    } else {
      // node x pulls from x + 1 (column 0 for the last real node)
      uint32_t nextw = __shfl_down_sync(0xffffffffu, v[0], 1);
      if (E.need_next) nextw = edge[i];
#pragma unroll
      for (int k = 0; k < W - 1; ++k) out[i][k] = __byte_perm(v[k], v[k + 1], 0x5432);
      out[i][W - 1] = __byte_perm(v[W - 1], nextw, 0x5432);
      if (E.need_wrap) {
        // the last real node's element takes column 0 (a select per word,
        // so that the array stays in registers)
        const int kw = E.e_last >> 1;
        const uint32_t keep = (E.e_last & 1) ? 0xffffu : 0xffff0000u;
        const uint32_t put = (E.e_last & 1) ? (wrap0[i] << 16) : wrap0[i];
#pragma unroll
        for (int k = 0; k < W; ++k) out[i][k] = k == kw ? ((out[i][k] & keep) | put) : out[i][k];
      }
    }
  }
}

// source row of plane i for destination row y (periodic wrap over nyw rows;
// nyw = 0 for a slab, whose rows -1 and ny are stored halo rows)
__device__ __forceinline__ int src_row(const Geom &g, int y, int i) {
  int ys = y - CYd(i);
  return ys < 0 ? ys + g.nyw : (ys >= g.nyw ? ys - g.nyw : ys);
}

template <typename T>
__device__ __forceinline__ void pull9_packed(const T *__restrict__ src, const Geom &g,
                                             const LanePos &p,
                                             uint32_t (&out)[9][Elem<T>::V / 2]) {
  constexpr int V = Elem<T>::V;
  static_assert(sizeof(T) == 2 && V % 2 == 0, "16-bit storage types only");
  const EdgeInfo E = edge_info(g, p, V);
  using RawT = typename Elem<T>::R::type;
  RawT raw[9];
  uint32_t edge[9], wrap0[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T *row = src + (long long)i * g.plane + (long long)src_row(g, p.y, i) * g.rstride;
    raw[i] = p.active ? __ldg(reinterpret_cast<const RawT *>(row + p.x0)) : Elem<T>::R::zero();
    edge_loads_packed<T>(row, p, E, i, edge[i], wrap0[i]);
  }
  assemble_packed<T>(raw, E, edge, wrap0, out);
}

template <typename T>
__device__ __forceinline__ void store9_packed(T *__restrict__ dst, const Geom &g,
                                              const LanePos &p,
                                              const uint32_t (&in)[9][Elem<T>::V / 2]) {
  if (!p.active) return;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    T *row = dst + (long long)i * g.plane + (long long)p.y * g.rstride;
    if constexpr (Elem<T>::V == 8)
      *reinterpret_cast<uint4 *>(row + p.x0) = make_uint4(in[i][0], in[i][1], in[i][2], in[i][3]);
    else
      *reinterpret_cast<uint2 *>(row + p.x0) = make_uint2(in[i][0], in[i][1]);
  }
  if (fills_sector<T>(g, p)) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      T *row = dst + (long long)i * g.plane + (long long)p.y * g.rstride;
      *reinterpret_cast<typename Elem<T>::R::type *>(row + p.x0 + Elem<T>::V) =
          Elem<T>::R::zero();
    }
  }
}

}  // namespace lbm
