// One periodic lattice split into y-slabs (lbm_slabs_* and lbm_slab_* in
// include/lbm.h).
//
// The periodic lattice of section 2.1 (Eq. blbs with its lattice-closure
// condition) couples row y only to rows y - 1 and y + 1, so whole rows can
// be stepped apart: slab k owns rows [y_k, y_k + rows_k) and stores one halo
// row below its row 0 and one above its last row (create_lattice with
// halo = true; the geometry's y wrap is then the identity and the pull reads
// the halo rows).  A step crosses a slab boundary only through the three
// populations that move across it: those with c_y = +1 (i = 2, 5, 6, the
// "up" set U) leave the last row upwards, those with c_y = -1 (i = 4, 7, 8,
// the "down" set D) leave row 0 downwards.
//
// Storage keeps the post-collision populations P_i at the node that wrote
// them, and node (x, y) pulls P_i(x - c_i).  So after every step
//   halo row -1   (U) <- the lower neighbour's last row (U)
//   halo row rows (D) <- the upper neighbour's row 0    (D)
// ("forward" exchange).  An initialisation (or set_populations) scatters
// f_i(x) into P_i(x - c_i): it fills the slab's own halo slots, which the
// first pull needs, but leaves the slots of its boundary rows that belong to
// the neighbours' nodes; the "reverse" exchange copies them
//   lower neighbour's last row (U) <- halo row -1   (U)
//   upper neighbour's row 0    (D) <- halo row rows (D)
// so that every stored slot is valid again (the drift sums read them).
//
// In one process (lbm_slabs_*) the exchange is a set of device-to-device
// copies (peer copies between devices) on a copy stream per slab,
// overlapped with the interior rows: each step first runs the slab's two
// boundary rows, records an event, then its interior rows; the copies into
// a slab's halo rows wait only for its neighbours' boundary rows.  Across
// processes (lbm_slab_*) each rank packs its outgoing rows into device
// buffers, moves them with its own transport (e.g. NCCL send / recv) and
// unpacks what it received.  Either way a slab's populations are those of
// the unsplit lattice bit for bit: every node runs the same arithmetic on
// the same inputs.
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

namespace {

const int kUp[3] = {2, 5, 6};    // c_y = +1
const int kDown[3] = {4, 7, 8};  // c_y = -1

#define SCK(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));       \
      cudaGetLastError();                                                  \
      return LBM_ECUDA;                                                    \
    }                                                                      \
  } while (0)

#define SREQ(cond, msg)  \
  do {                   \
    if (!(cond)) {       \
      set_error(msg);    \
      return LBM_EINVAL; \
    }                    \
  } while (0)

// address of row y (-1 .. rows) of plane i in buffer `buf` of a slab
char *row_addr(const Lattice &L, void *buf, int y, int i) {
  const long long off = ((long long)9 * y + i) * L.g.pitch;
  return static_cast<char *>(buf) + off * L.esize;
}

size_t row_bytes(const Lattice &L) { return (size_t)L.g.pitch * L.esize; }

// copy 3 plane-rows of a set, each row_bytes long, between two addresses
// given per plane; contiguous planes (5, 6 and 7, 8) go in one copy
template <class Src, class Dst>
cudaError_t copy_set(const int *set, Src src, Dst dst, size_t rb, int dst_dev, int src_dev,
                     cudaStream_t st) {
  for (int j = 0; j < 3;) {
    const int n = (j + 1 < 3 && set[j + 1] == set[j] + 1) ? 2 : 1;
    void *d = dst(j);
    const void *s = src(j);
    cudaError_t e = dst_dev == src_dev
                        ? cudaMemcpyAsync(d, s, n * rb, cudaMemcpyDeviceToDevice, st)
                        : cudaMemcpyPeerAsync(d, dst_dev, s, src_dev, n * rb, st);
    if (e != cudaSuccess) return e;
    j += n;
  }
  return cudaSuccess;
}

// step rows [r0, r0 + nr) of a slab from buffer `from` into the other
cudaError_t launch_rows(lbm_handle h, int from, int r0, int nr, cudaStream_t st) {
  if (nr < 1) return cudaSuccess;
  const Lattice &L = lattice_of(h);
  Lattice S = L;
  S.g = make_geom(L.g.nx, nr, L.V, L.esize);
  S.g.nyw = 0;
  const long long off = (long long)r0 * L.g.rstride * L.esize;
  const void *src = static_cast<const char *>(L.buf[from]) + off;
  void *dst = static_cast<char *>(L.buf[from ^ 1]) + off;
  if (L.dtype == LBM_F64) return launch_step_f64(S, src, dst, st, 256, 0);
  return launch_step_dev(S, src, dst, st, block_of(h), L.variant);
}

}  // namespace

struct lbm_slabs_ctx {
  int nx = 0, ny = 0, dtype = 0, n = 0;
  std::vector<lbm_handle> slab;
  std::vector<int> y0, rows, dev;
  std::vector<cudaStream_t> copy;
  std::vector<cudaEvent_t> ev_bnd, ev_copy;
};

static void slabs_free(lbm_slabs_ctx *s) {
  for (int k = 0; k < (int)s->slab.size(); ++k) {
    DevGuard g(s->dev[k]);
    if (k < (int)s->copy.size() && s->copy[k]) {
      cudaStreamSynchronize(s->copy[k]);
      cudaStreamDestroy(s->copy[k]);
    }
    if (k < (int)s->ev_bnd.size() && s->ev_bnd[k]) cudaEventDestroy(s->ev_bnd[k]);
    if (k < (int)s->ev_copy.size() && s->ev_copy[k]) cudaEventDestroy(s->ev_copy[k]);
    if (s->slab[k]) lbm_destroy(s->slab[k]);
  }
  cudaGetLastError();
  delete s;
}

// forward (after a step) or reverse (after an initialisation) exchange of
// every slab boundary, on the copy streams; slab k's compute stream then
// waits for the copies that touch its buffers
static int slabs_exchange(lbm_slabs_ctx *s, bool reverse) {
  const int n = s->n;
  for (int k = 0; k < n; ++k) {
    DevGuard g(s->dev[k]);
    const int lo = (k + n - 1) % n, hi = (k + 1) % n;
    SCK(cudaStreamWaitEvent(s->copy[k], s->ev_bnd[lo], 0));
    SCK(cudaStreamWaitEvent(s->copy[k], s->ev_bnd[hi], 0));
    SCK(cudaStreamWaitEvent(s->copy[k], s->ev_bnd[k], 0));
  }
  for (int k = 0; k < n; ++k) {
    DevGuard g(s->dev[k]);
    const int lo = (k + n - 1) % n, hi = (k + 1) % n;
    const Lattice &L = lattice_of(s->slab[k]);
    const Lattice &Llo = lattice_of(s->slab[lo]);
    const Lattice &Lhi = lattice_of(s->slab[hi]);
    const size_t rb = row_bytes(L);
    void *mine = L.buf[L.cur];
    void *blo = Llo.buf[Llo.cur];
    void *bhi = Lhi.buf[Lhi.cur];
    const int rk = s->rows[k], rlo = s->rows[lo];
    cudaError_t e;
    if (!reverse) {
      // my halo rows <- the neighbours' boundary rows (copies into slab k)
      e = copy_set(
          kUp, [&](int j) { return row_addr(Llo, blo, rlo - 1, kUp[j]); },
          [&](int j) { return row_addr(L, mine, -1, kUp[j]); }, rb, s->dev[k], s->dev[lo],
          s->copy[k]);
      if (e == cudaSuccess)
        e = copy_set(
            kDown, [&](int j) { return row_addr(Lhi, bhi, 0, kDown[j]); },
            [&](int j) { return row_addr(L, mine, rk, kDown[j]); }, rb, s->dev[k], s->dev[hi],
            s->copy[k]);
    } else {
      // the lower neighbour's last row (U) <- my halo row -1; done by the
      // lower neighbour's copy stream would need the same waits, so slab k
      // writes into its neighbours here, and each boundary slot is written
      // by exactly one slab
      e = copy_set(
          kUp, [&](int j) { return row_addr(L, mine, -1, kUp[j]); },
          [&](int j) { return row_addr(Llo, blo, rlo - 1, kUp[j]); }, rb, s->dev[lo], s->dev[k],
          s->copy[k]);
      if (e == cudaSuccess)
        e = copy_set(
            kDown, [&](int j) { return row_addr(L, mine, rk, kDown[j]); },
            [&](int j) { return row_addr(Lhi, bhi, 0, kDown[j]); }, rb, s->dev[hi], s->dev[k],
            s->copy[k]);
    }
    if (e != cudaSuccess) {
      set_error(std::string("slab halo exchange: ") + cudaGetErrorString(e));
      cudaGetLastError();
      return LBM_ECUDA;
    }
    SCK(cudaEventRecord(s->ev_copy[k], s->copy[k]));
  }
  // a forward exchange writes only into slab k's buffers; a reverse one
  // writes into its neighbours' as well
  for (int k = 0; k < n; ++k) {
    DevGuard g(s->dev[k]);
    const int lo = (k + n - 1) % n, hi = (k + 1) % n;
    cudaStream_t st = stream_of(s->slab[k]);
    SCK(cudaStreamWaitEvent(st, s->ev_copy[k], 0));
    if (reverse) {
      SCK(cudaStreamWaitEvent(st, s->ev_copy[lo], 0));
      SCK(cudaStreamWaitEvent(st, s->ev_copy[hi], 0));
    }
  }
  return LBM_OK;
}

// every slab's compute stream has reached this point (an event per slab on
// its compute stream, used by the next exchange as "boundary rows ready")
static int slabs_mark(lbm_slabs_ctx *s) {
  for (int k = 0; k < s->n; ++k) {
    DevGuard g(s->dev[k]);
    SCK(cudaEventRecord(s->ev_bnd[k], stream_of(s->slab[k])));
  }
  return LBM_OK;
}

extern "C" {

int lbm_slabs_create(int nx, int ny, const double S[9], double rho0, const double u0[2],
                     int storage_dtype, int nslabs, const int *devices, lbm_slabs *out) {
  SREQ(out != nullptr && S != nullptr && u0 != nullptr, "null argument");
  SREQ(nslabs >= 1 && ny >= nslabs, "need 1 <= nslabs <= ny");
  SREQ(storage_dtype == LBM_F64 || storage_dtype == LBM_F32DEV ||
           storage_dtype == LBM_BF16DEV || storage_dtype == LBM_F64DEV,
       "slabs take FP64, FP32, BF16 or FP64-deviation storage (FP16 slabs would need one "
       "storage scale for the whole lattice)");
  int cur_dev = 0;
  SCK(cudaGetDevice(&cur_dev));
  lbm_slabs_ctx *s = new (std::nothrow) lbm_slabs_ctx();
  if (!s) {
    set_error("out of host memory");
    return LBM_ENOMEM;
  }
  s->nx = nx;
  s->ny = ny;
  s->dtype = storage_dtype;
  s->n = nslabs;
  for (int k = 0; k < nslabs; ++k) {
    const int a = (int)((long long)k * ny / nslabs), b = (int)((long long)(k + 1) * ny / nslabs);
    s->y0.push_back(a);
    s->rows.push_back(b - a);
    s->dev.push_back(devices ? devices[k] : cur_dev);
  }
  s->slab.assign(nslabs, nullptr);
  s->copy.assign(nslabs, nullptr);
  s->ev_bnd.assign(nslabs, nullptr);
  s->ev_copy.assign(nslabs, nullptr);
  for (int k = 0; k < nslabs; ++k) {
    DevGuard g(s->dev[k]);
    if (cudaSetDevice(s->dev[k]) != cudaSuccess) {
      cudaGetLastError();
      slabs_free(s);
      set_error("no such device for slab " + std::to_string(k));
      return LBM_EINVAL;
    }
    int rc = create_lattice(nx, s->rows[k], S, rho0, u0, storage_dtype, true, &s->slab[k]);
    if (rc != LBM_OK) {
      s->slab[k] = nullptr;
      slabs_free(s);
      return rc;
    }
    if (cudaStreamCreateWithFlags(&s->copy[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_bnd[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_copy[k], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      slabs_free(s);
      set_error("cannot create the slab streams");
      return LBM_ECUDA;
    }
  }
  // FP64 slabs start from the uniform equilibrium, halo slots included
  // (their creation initialises them); the exchange keeps the boundary
  // slots consistent as for any initialisation
  int rc = slabs_mark(s);
  if (rc == LBM_OK) rc = slabs_exchange(s, true);
  if (rc != LBM_OK) {
    slabs_free(s);
    return rc;
  }
  *out = s;
  return LBM_OK;
}

int lbm_slabs_rows(lbm_slabs s, int k, int *y0, int *rows, int *device) {
  SREQ(s != nullptr && k >= 0 && k < s->n, "no such slab");
  if (y0) *y0 = s->y0[k];
  if (rows) *rows = s->rows[k];
  if (device) *device = s->dev[k];
  return LBM_OK;
}

int lbm_slabs_init_field(lbm_slabs s, const double *rho, const double *ux, const double *uy) {
  SREQ(s && rho && ux && uy, "null argument");
  for (int k = 0; k < s->n; ++k) {
    DevGuard g(s->dev[k]);
    const size_t o = (size_t)s->y0[k] * s->nx;
    int rc = lbm_init_field(s->slab[k], rho + o, ux + o, uy + o);
    if (rc != LBM_OK) {
      set_error("slab " + std::to_string(k) + ": " + lbm_last_error());
      return rc;
    }
  }
  int rc = slabs_mark(s);
  if (rc == LBM_OK) rc = slabs_exchange(s, true);
  return rc;
}

int lbm_slabs_set_populations(lbm_slabs s, const double *f) {
  SREQ(s && f, "null argument");
  const size_t plane = (size_t)s->nx * s->ny;
  for (int k = 0; k < s->n; ++k) {
    DevGuard g(s->dev[k]);
    const size_t n = (size_t)s->rows[k] * s->nx;
    std::vector<double> part;
    try {
      part.resize(9 * n);
    } catch (...) {
      set_error("out of host memory");
      return LBM_ENOMEM;
    }
    for (int i = 0; i < 9; ++i)
      memcpy(part.data() + i * n, f + i * plane + (size_t)s->y0[k] * s->nx, n * sizeof(double));
    int rc = lbm_set_populations(s->slab[k], part.data());
    if (rc != LBM_OK) return rc;
  }
  int rc = slabs_mark(s);
  if (rc == LBM_OK) rc = slabs_exchange(s, true);
  return rc;
}

int lbm_slabs_step(lbm_slabs s, long nsteps) {
  NvtxRange nvtx("lbm_slabs_step");
  SREQ(s != nullptr, "null slabs");
  SREQ(nsteps >= 0, "negative step count");
  for (long t = 0; t < nsteps; ++t) {
    // boundary rows first, then (after the event the exchange waits for)
    // the interior rows, which run beside the halo copies
    for (int k = 0; k < s->n; ++k) {
      DevGuard g(s->dev[k]);
      lbm_handle h = s->slab[k];
      cudaStream_t st = stream_of(h);
      const int r = s->rows[k], from = lattice_of(h).cur;
      SCK(launch_rows(h, from, 0, 1, st));
      if (r > 1) SCK(launch_rows(h, from, r - 1, 1, st));
      SCK(cudaEventRecord(s->ev_bnd[k], st));
      if (r > 2) SCK(launch_rows(h, from, 1, r - 2, st));
      advance_one(h);
    }
    int rc = slabs_exchange(s, false);
    if (rc != LBM_OK) return rc;
  }
  return LBM_OK;
}

int lbm_slabs_moments(lbm_slabs s, double *rho, double *ux, double *uy) {
  SREQ(s && rho && ux && uy, "null argument");
  for (int k = 0; k < s->n; ++k) {
    DevGuard g(s->dev[k]);
    const size_t o = (size_t)s->y0[k] * s->nx;
    int rc = lbm_moments(s->slab[k], rho + o, ux + o, uy + o);
    if (rc != LBM_OK) return rc;
  }
  return LBM_OK;
}

int lbm_slabs_get_populations(lbm_slabs s, double *f) {
  SREQ(s && f, "null argument");
  const size_t plane = (size_t)s->nx * s->ny;
  for (int k = 0; k < s->n; ++k) {
    DevGuard g(s->dev[k]);
    const size_t n = (size_t)s->rows[k] * s->nx;
    std::vector<double> part;
    try {
      part.resize(9 * n);
    } catch (...) {
      set_error("out of host memory");
      return LBM_ENOMEM;
    }
    int rc = lbm_get_populations(s->slab[k], part.data());
    if (rc != LBM_OK) return rc;
    for (int i = 0; i < 9; ++i)
      memcpy(f + i * plane + (size_t)s->y0[k] * s->nx, part.data() + i * n, n * sizeof(double));
  }
  return LBM_OK;
}

int lbm_slabs_drift(lbm_slabs s, double out[4]) {
  SREQ(s && out, "null argument");
  double acc[4] = {0, 0, 0, 0};
  int rc_all = LBM_OK;
  for (int k = 0; k < s->n; ++k) {
    DevGuard g(s->dev[k]);
    double d[4];
    int rc = lbm_drift(s->slab[k], d);
    if (rc != LBM_OK && rc != LBM_EUNSTABLE) return rc;
    if (rc == LBM_EUNSTABLE) rc_all = rc;
    for (int c = 0; c < 4; ++c) acc[c] += d[c];
  }
  for (int c = 0; c < 4; ++c) out[c] = acc[c];
  return rc_all;
}

int lbm_slabs_destroy(lbm_slabs s) {
  if (!s) return LBM_EINVAL;
  slabs_free(s);
  return LBM_OK;
}

// ------------------------------------------------- one slab per process
int lbm_slab_create(int nx, int ny_total, int y0, int rows, const double S[9], double rho0,
                    const double u0[2], int storage_dtype, lbm_handle *out) {
  SREQ(rows >= 1 && y0 >= 0 && y0 + rows <= ny_total, "slab rows outside the lattice");
  SREQ(storage_dtype != LBM_F16DEV,
       "slabs take FP64, FP32 or BF16 storage (FP16 slabs would need one storage scale for "
       "the whole lattice)");
  return create_lattice(nx, rows, S, rho0, u0, storage_dtype, true, out);
}

int lbm_slab_halo_bytes(lbm_handle h, size_t *bytes) {
  SREQ(h && bytes, "null argument");
  SREQ(is_slab(h), "not a slab");
  *bytes = 3 * row_bytes(lattice_of(h));
  return LBM_OK;
}

int lbm_slab_pack(lbm_handle h, int reverse, void *to_below, void *to_above) {
  SREQ(h && to_below && to_above, "null argument");
  SREQ(is_slab(h), "not a slab");
  DevGuard g(device_of(h));
  const Lattice &L = lattice_of(h);
  const size_t rb = row_bytes(L);
  void *buf = L.buf[L.cur];
  const int r = L.g.ny;
  const int *below_set = reverse ? kUp : kDown, *above_set = reverse ? kDown : kUp;
  const int below_row = reverse ? -1 : 0, above_row = reverse ? r : r - 1;
  cudaStream_t st = stream_of(h);
  const int dev = device_of(h);
  cudaError_t e = copy_set(
      below_set, [&](int j) { return row_addr(L, buf, below_row, below_set[j]); },
      [&](int j) { return static_cast<void *>(static_cast<char *>(to_below) + j * rb); }, rb, dev,
      dev, st);
  if (e == cudaSuccess)
    e = copy_set(
        above_set, [&](int j) { return row_addr(L, buf, above_row, above_set[j]); },
        [&](int j) { return static_cast<void *>(static_cast<char *>(to_above) + j * rb); }, rb,
        dev, dev, st);
  if (e != cudaSuccess) {
    set_error(std::string("lbm_slab_pack: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  return LBM_OK;
}

int lbm_slab_unpack(lbm_handle h, int reverse, const void *from_below, const void *from_above) {
  SREQ(h && from_below && from_above, "null argument");
  SREQ(is_slab(h), "not a slab");
  DevGuard g(device_of(h));
  const Lattice &L = lattice_of(h);
  const size_t rb = row_bytes(L);
  void *buf = L.buf[L.cur];
  const int r = L.g.ny;
  // forward: halo row -1 takes U from below, halo row r takes D from above;
  // reverse: row 0 takes D from below, row r - 1 takes U from above
  const int *from_below_set = reverse ? kDown : kUp, *from_above_set = reverse ? kUp : kDown;
  const int below_row = reverse ? 0 : -1, above_row = reverse ? r - 1 : r;
  cudaStream_t st = stream_of(h);
  const int dev = device_of(h);
  cudaError_t e = copy_set(
      from_below_set,
      [&](int j) {
        return static_cast<const void *>(static_cast<const char *>(from_below) + j * rb);
      },
      [&](int j) { return row_addr(L, buf, below_row, from_below_set[j]); }, rb, dev, dev, st);
  if (e == cudaSuccess)
    e = copy_set(
        from_above_set,
        [&](int j) {
          return static_cast<const void *>(static_cast<const char *>(from_above) + j * rb);
        },
        [&](int j) { return row_addr(L, buf, above_row, from_above_set[j]); }, rb, dev, dev, st);
  if (e != cudaSuccess) {
    set_error(std::string("lbm_slab_unpack: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  return LBM_OK;
}

}  // extern "C"
