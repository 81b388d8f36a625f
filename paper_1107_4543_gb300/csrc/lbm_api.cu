// C ABI of liblbm.so (declared in include/lbm.h): lattice handles, the step
// loop (graph-captured chunks of fused step launches), initialisation,
// moments, checkpoints, drift, tuning, host memory.  Batches live in
// batch.cu, the serving scheduler in serve.cu, slabs in slabs.cu.
#include <math.h>
#include <string.h>

#include <stdlib.h>
#include <sys/mman.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_set>
#include <new>
#include <string>
#include <vector>

#include "bounds.cuh"
#include "lbm_internal.h"
#include "runtime.h"

namespace lbm {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

static std::mutex g_alloc_mu;
static lbm_alloc_fn g_alloc = nullptr;
static lbm_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

void *dev_alloc(size_t bytes) {
  if (bytes == 0) bytes = 256;
  lbm_alloc_fn a;
  void *ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
    ctx = g_alloc_ctx;
  }
  if (a) return a(bytes, ctx);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void *p) {
  if (!p) return;
  lbm_free_fn f;
  void *ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    f = g_free;
    ctx = g_alloc_ctx;
  }
  if (f)
    f(p, ctx);
  else
    cudaFree(p);
}

size_t resident_limit(int device) {
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
      cudaSuccess) {
    cudaGetLastError();
    optin = 0;
  }
  size_t lim = (size_t)(optin > 0 ? optin : 0);
  if (const char *v = getenv("LBM_RESIDENT_BYTES")) {
    const size_t cap = (size_t)strtoull(v, nullptr, 10);
    if (cap < lim) lim = cap;
  }
  return lim;
}

int sm_count() {
  int d = 0, n = 0;
  if (cudaGetDevice(&d) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return 148;
  }
  return n;
}

}  // namespace lbm

using namespace lbm;


AuxView lbm::aux_view(const lbm_ctx *h) {
  AuxView a;
  a.g = h->L.g;
  a.dtype = h->L.dtype;
  a.buf = h->L.buf[h->L.cur];
  a.rho0 = h->rho0;
  a.jx0 = h->j0[0];
  a.jy0 = h->j0[1];
  for (int i = 0; i < 9; ++i) a.f0[i] = h->f0[i];
  a.scale = h->qscale;
  return a;
}

// the largest |f'| the point source writes: at its node f^eq(rho0 +
// amplitude sin(...), 0) - f^eq(rho0, 0) peaks at the rest weight 4/9
double lbm::source_maxdev(const lbm_ctx *h) {
  return h->src_on ? 4.0 / 9.0 * fabs(h->s_amp) : 0.0;
}

// The captured step graphs hold the storage scale (the step kernel's
// DevParams, the forced-node kernel's AuxView) by value: a new scale drops
// them, so the next run recaptures.
void lbm::set_scale(lbm_ctx *h, double s) {
  if (s != h->qscale) free_graph(h);
  h->qscale = s;
  h->L.dp.scale = (float)s;
  h->L.dp.inv_scale = (float)(1.0 / s);
}

// stored |f'| * qscale stays near 2^14 (fp16_scale)
void lbm::set_qscale(lbm_ctx *h, double maxabs) { set_scale(h, fp16_scale(maxabs)); }

int lbm::free_graph(lbm_ctx *h) {
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_steps = 0;
  }
  if (h->src_graph) {
    cudaGraphExecDestroy(h->src_graph);
    h->src_graph = nullptr;
  }
  return LBM_OK;
}

// launch variant before (or without) tuning: the 80-register cap (3 blocks
// of 256 per SM), the fastest for every deviation type on GB300
int lbm::default_variant(int) { return 2; }

bool lbm::autotune_enabled() {
  const char *e = getenv("LBM_AUTOTUNE");
  return !(e && e[0] == '0');
}

// Tuner results per (dtype, nx, ny), shared by the handles of a process.
std::mutex lbm::g_tune_mu;
static std::map<std::tuple<int, int, int>, int> g_tune_cache;
// batch choices read from the tuning file, by the hash of the composition
std::map<unsigned long long, int> lbm::g_batch_file_cache;

// Optional tuning file (environment LBM_TUNE_CACHE = path): lines
// "<device> L <dtype>:<nx>:<ny> <variant>" and "<device> B <hash> <variant>"
// are read once per process and appended as new choices are made, so later
// processes on the same GPU model skip the timing runs.  <device> is the GPU
// name and SM count; lines of other devices and malformed lines are
// ignored.  Called with g_tune_mu held.
static const char *tune_file() {
  const char *p = getenv("LBM_TUNE_CACHE");
  return (p && p[0]) ? p : nullptr;
}

static std::string device_tag() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string t = prop.name;
  for (char &c : t)
    if (c == ' ' || c == '\t') c = '_';
  return t + "_sm" + std::to_string(prop.multiProcessorCount);
}

unsigned long long lbm::fnv1a(const std::string &s) {
  unsigned long long h = 1469598103934665603ULL;
  for (unsigned char c : s) {
    h ^= c;
    h *= 1099511628211ULL;
  }
  return h;
}

void lbm::tune_file_load_locked() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char *path = tune_file();
  if (!path) return;
  FILE *fp = fopen(path, "r");
  if (!fp) return;
  const std::string tag = device_tag();
  char dtag[256], kind[4], key[128];
  int v;
  while (fscanf(fp, "%255s %3s %127s %d", dtag, kind, key, &v) == 4) {
    if (tag != dtag) continue;
    if (kind[0] == 'L' && v >= 0 && v < kStepVariants) {
      int dt, nx, ny;
      if (sscanf(key, "%d:%d:%d", &dt, &nx, &ny) == 3) g_tune_cache[std::make_tuple(dt, nx, ny)] = v;
    } else if (kind[0] == 'B' && v >= 0 && v < kBatchVariants) {
      g_batch_file_cache[strtoull(key, nullptr, 16)] = v;
    }
  }
  fclose(fp);
}

void lbm::tune_file_append_locked(const char *kind, const std::string &key, int v) {
  const char *path = tune_file();
  if (!path) return;
  FILE *fp = fopen(path, "a");
  if (!fp) return;
  fprintf(fp, "%s %s %s %d\n", device_tag().c_str(), kind, key.c_str(), v);
  fclose(fp);
}


// repetitions for ~2 ms of traffic per variant at ~6 TB/s
int lbm::tune_reps(double bytes) {
  const int r = (int)(2e-3 * 6e12 / std::max(bytes, 1.0));
  return std::max(2, std::min(200, r));
}

static cudaError_t launch_one(lbm_ctx *h, int from, cudaStream_t st) {
  const void *src = h->L.buf[from];
  void *dst = h->L.buf[from ^ 1];
  if (h->L.dtype == LBM_F64) return launch_step_f64(h->L, src, dst, st, 256, h->grid_cap);
  return launch_step_dev(h->L, src, dst, st, h->block, h->L.variant);
}

// capture `steps` (even) launches starting from buffer 0 into a graph
static int capture_graph(lbm_ctx *h, int steps) {
  free_graph(h);
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = launch_one(h, k & 1, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    set_error(std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  h->graph_steps = steps;
  return LBM_OK;
}

// steps per captured graph of forced steps (even)
constexpr int kSrcGraph = 64;

// capture kSrcGraph forced steps starting from buffer 0: before step k the
// source node's populations are set from src_tab + 9 k (filled by the host
// for each replay), then the step runs
static int capture_src_graph(lbm_ctx *h) {
  if (h->src_graph) {
    cudaGraphExecDestroy(h->src_graph);
    h->src_graph = nullptr;
  }
  if (!h->src_tab) {
    h->src_tab = (double *)dev_alloc(sizeof(double) * 9 * kSrcGraph);
    if (!h->src_tab) {
      set_error("out of device memory for the source table");
      return LBM_ENOMEM;
    }
  }
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < kSrcGraph && e == cudaSuccess; ++k) {
      AuxView a = aux_view(h);
      a.buf = h->L.buf[k & 1];
      e = launch_force_node_tab(a, h->sx, h->sy, h->src_tab + 9 * k, cs);
      if (e == cudaSuccess) e = launch_one(h, k & 1, cs);
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->src_graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    h->src_graph = nullptr;
    set_error(std::string("source graph capture: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  h->src_gx = h->sx;
  h->src_gy = h->sy;
  return LBM_OK;
}

int lbm::ensure_stage(lbm_ctx *h) {
  if (h->stage) return LBM_OK;
  const size_t n = (size_t)h->L.g.nx * h->L.g.ny;
  h->stage = (double *)dev_alloc(3 * n * sizeof(double));
  if (!h->stage) {
    set_error("cannot allocate the field staging buffer");
    return LBM_ENOMEM;
  }
  h->bytes += 3 * n * sizeof(double);
  return LBM_OK;
}

// v = hi + lo with hi = fl32(v), lo = fl32(v - hi)
static void split_rate(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// Time every launch variant of the step kernel on this lattice and keep the
// fastest.  Each trial launch reads the current buffer and writes the idle
// one, so the lattice's state is unchanged.
static int tune_handle(lbm_ctx *h, double *times) {
  if (h->L.dtype == LBM_F64) {
    if (times)
      for (int v = 0; v < kStepVariants; ++v) times[v] = -1.0;
    h->tuned = true;
    return LBM_OK;
  }
  const double bytes = (double)h->L.g.nx * h->L.g.ny * 18.0 * h->L.esize;
  const int reps = tune_reps(bytes);
  const int from = h->L.cur;
  double best = 1e300;
  int bv = h->L.variant;
  for (int v = 0; v < kStepVariants; ++v) {
    double ms = 0;
    int rc = time_launches(h->stream, reps, [&](int) {
      return launch_step_dev(h->L, h->L.buf[from], h->L.buf[from ^ 1], h->stream, h->block, v);
    }, &ms);
    if (rc != LBM_OK) return rc;
    if (times) times[v] = ms;
    if (ms < best) {
      best = ms;
      bv = v;
    }
  }
  if (bv != h->L.variant) {
    h->L.variant = bv;
    free_graph(h);
  }
  h->tuned = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[std::make_tuple(h->L.dtype, h->L.g.nx, h->L.g.ny)] = bv;
  tune_file_append_locked("L", std::to_string(h->L.dtype) + ":" + std::to_string(h->L.g.nx) + ":" +
                                   std::to_string(h->L.g.ny), bv);
  return LBM_OK;
}

// First step of a large lattice: reuse a cached choice or tune now.
static int maybe_autotune(lbm_ctx *h) {
  if (h->tuned || h->L.dtype == LBM_F64) return LBM_OK;
  if ((long long)h->L.g.nx * h->L.g.ny < (1LL << 20) || !autotune_enabled()) {
    h->tuned = true;
    return LBM_OK;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_file_load_locked();
    auto it = g_tune_cache.find(std::make_tuple(h->L.dtype, h->L.g.nx, h->L.g.ny));
    if (it != g_tune_cache.end()) {
      if (it->second != h->L.variant) {
        h->L.variant = it->second;
        free_graph(h);
      }
      h->tuned = true;
      return LBM_OK;
    }
  }
  return tune_handle(h, nullptr);
}

static int check_rates(const double S[9]) {
  static const int conserved[3] = {0, 3, 5};  // rho, jx, jy in LL order
  for (int k = 0; k < 9; ++k) {
    bool cons = (k == conserved[0] || k == conserved[1] || k == conserved[2]);
    if (!isfinite(S[k])) return 0;
    if (!cons && !(S[k] > 0.0 && S[k] <= 2.0)) return 0;
  }
  return 1;
}

// init f = f^eq(field) (kind 0: device arrays; else analytic).  With bad
// set, the init kernel counts invalid nodes there (read after a sync).
static int do_init(lbm_ctx *h, const double *rho, const double *ux, const double *uy, int kind,
                   const double *params, unsigned int *bad = nullptr) {
  if (h->batch) {
    set_error("lattice is a batch member");
    return LBM_EINVAL;
  }
  h->L.cur = 0;
  AuxView a = aux_view(h);
  if (h->L.dtype == LBM_F16DEV) {
    CK(launch_maxdev_eq(a, rho, ux, uy, kind, params, h->maxbits, h->stream));
    unsigned int bits = 0;
    CK(cudaMemcpyAsync(&bits, h->maxbits, sizeof(bits), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    float m;
    memcpy(&m, &bits, sizeof(m));
    set_qscale(h, std::max((double)m, source_maxdev(h)));
    a = aux_view(h);
  }
  CK(launch_init_eq(a, rho, ux, uy, kind, params, h->stream, bad));
  h->t = 0;
  return LBM_OK;
}

extern "C" {

const char *lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_PENDING: return "pending";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "non-finite populations";
    case LBM_ETIMEOUT: return "timed out";
    case LBM_ENOTFOUND: return "unknown request";
    case LBM_ECLOSED: return "server closed";
    default: return "unknown error";
  }
}

const char *lbm_last_error(void) { return g_last_error.c_str(); }

int lbm_debug_bounds(unsigned int *word, int reset) {
  REQUIRE(word != nullptr, "null argument");
  const bool r = reset != 0;
  *word = bounds_word_vn(r) | bounds_word_opt(r) | bounds_word_step_f32(r) |
          bounds_word_step_f16(r) | bounds_word_step_bf16(r) | bounds_word_io(r);
  REQUIRE(bounds::kEnabled, "built without LBM_DEBUG_BOUNDS");
  return LBM_OK;
}

int lbm_debug_bounds_selftest(void) {
  REQUIRE(bounds::kEnabled, "built without LBM_DEBUG_BOUNDS");
  unsigned int *one = (unsigned int *)dev_alloc(sizeof(unsigned int));
  REQUIRE(one != nullptr, "device allocation failed");
  cudaError_t e = launch_bounds_selftest(one, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  dev_free(one);
  CK(e);
  return LBM_OK;
}

// ------------------------------------------------------------ host memory
// Page-locked host arrays on transparent huge pages (lbm_host_alloc): the
// copy engines translate each page of a transfer, and on a GB300 host with
// 64 KiB base pages and 512 MiB huge pages, copies from ordinary
// page-locked memory fell from ~210 to 17 - 80 GB/s once the host had run
// for a while, while a huge-page mapping kept 192 - 211 GB/s.
static std::mutex g_host_mu;
struct HostMap {
  void *base;
  size_t len;
};
static std::map<void *, HostMap> g_host_maps;

static size_t huge_page_bytes() {
  size_t hp = (size_t)2 << 20;
  if (FILE *f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
    unsigned long long v = 0;
    if (fscanf(f, "%llu", &v) == 1 && v >= 4096 && v <= ((size_t)1 << 30)) hp = (size_t)v;
    fclose(f);
  }
  return hp;
}

void *lbm_host_alloc(size_t bytes) {
  if (bytes == 0) bytes = 1;
  const size_t page = (size_t)sysconf(_SC_PAGESIZE);
  const size_t hp = huge_page_bytes();
  // arrays of at least a quarter huge page start on a huge-page boundary
  // and fill whole huge pages; smaller ones stay page-sized
  const size_t unit = bytes >= hp / 4 ? hp : page;
  const size_t len = (bytes + unit - 1) / unit * unit;
  const size_t span = len + (unit > page ? unit : 0);
  void *m = mmap(nullptr, span, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (m == MAP_FAILED) {
    set_error("lbm_host_alloc: mmap failed");
    return nullptr;
  }
  char *base = static_cast<char *>(m);
  char *p = base;
  if (unit > page) {
    p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(base) + unit - 1) / unit * unit);
    if (p > base) munmap(base, (size_t)(p - base));
    const size_t tail = span - (size_t)(p - base) - len;
    if (tail) munmap(p + len, tail);
    madvise(p, len, MADV_HUGEPAGE);  // a hint: ordinary pages where it is refused
  }
  memset(p, 0, len);  // fault the pages in before they are registered
#ifdef MADV_COLLAPSE
  // where faults fell back to base pages, collapse them into huge pages
  // now (Linux 6.1 and later; a refusal leaves the base pages)
  if (unit > page) madvise(p, len, MADV_COLLAPSE);
#else
  if (unit > page) madvise(p, len, 25);  // MADV_COLLAPSE, as above
#endif
  if (cudaHostRegister(p, len, cudaHostRegisterDefault) != cudaSuccess) {
    cudaGetLastError();
    munmap(p, len);
    set_error("lbm_host_alloc: cudaHostRegister failed");
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_host_mu);
  g_host_maps[p] = HostMap{p, len};
  return p;
}

int lbm_host_free(void *p) {
  if (p == nullptr) return LBM_OK;
  HostMap m;
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    auto it = g_host_maps.find(p);
    if (it == g_host_maps.end()) {
      set_error("lbm_host_free: not an lbm_host_alloc array");
      return LBM_EINVAL;
    }
    m = it->second;
    g_host_maps.erase(it);
  }
  cudaError_t e = cudaHostUnregister(m.base);
  munmap(m.base, m.len);
  if (e != cudaSuccess) {
    set_error(std::string("cudaHostUnregister: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  return LBM_OK;
}

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    set_error("allocator and free must both be set or both be NULL");
    return LBM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = alloc ? ctx : nullptr;
  return LBM_OK;
}

}  // extern "C"

namespace lbm {
// lbm_create, or (halo) a slab of ny rows of a larger periodic lattice: its
// buffers get one stored row below row 0 and one above row ny - 1, and the
// geometry's y wrap is the identity (Geom::nyw = 0), so the pull reads the
// neighbouring slabs' rows from those halo rows.
int create_lattice(int nx, int ny, const double S[9], double rho0, const double u0[2],
                   int storage_dtype, bool halo, lbm_handle *out) {
  REQUIRE(out != nullptr && S != nullptr && u0 != nullptr, "null argument");
  // a slab of a larger lattice may be one row high (its halo rows hold the
  // neighbouring rows)
  REQUIRE(nx >= 2 && ny >= (halo ? 1 : 2), "nx and ny must be >= 2");
  REQUIRE((long long)nx * ny <= (1LL << 40), "lattice too large");
  REQUIRE(rho0 > 0.0 && isfinite(rho0), "rho0 must be positive");
  REQUIRE(isfinite(u0[0]) && isfinite(u0[1]), "u0 must be finite");
  REQUIRE(check_rates(S), "rates: non-conserved entries must lie in (0, 2], all finite");
  int esize, V;
  switch (storage_dtype) {
    case LBM_F64:
    case LBM_F64DEV: esize = 8; break;
    case LBM_F32DEV: esize = 4; break;
    case LBM_F16DEV:
    case LBM_BF16DEV: esize = 2; break;
    default: REQUIRE(false, "unknown storage dtype");
  }
  V = vec_nodes(storage_dtype);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  lbm_ctx *h = new (std::nothrow) lbm_ctx();
  if (!h) {
    set_error("out of host memory");
    return LBM_ENOMEM;
  }
  h->device = dev;
  h->L.g = make_geom(nx, ny, V, esize);
  if (halo) h->L.g.nyw = 0;
  h->slab = halo;
  h->L.dtype = storage_dtype;
  h->L.V = V;
  h->L.variant = default_variant(storage_dtype);
  h->L.esize = esize;
  h->L.cur = 0;
  // Lallemand-Luo order (rho, e, eps, jx, qx, jy, qy, pxx, pxy) -> paper
  // order (rho, jx, jy, e, eps, qx, qy, pxx, pxy)
  const int ll_of_paper[9] = {0, 3, 5, 1, 2, 4, 6, 7, 8};
  for (int k = 0; k < 9; ++k) h->S_paper[k] = S[ll_of_paper[k]];
  // The FP32 collision of the deviation types knows the reference state
  // only as FP32 numbers, so the base f^eq(rho0, j0) is built from exactly
  // those values: any mismatch would act as a spurious mean-flow error.
  DevParams &dp = h->L.dp;
  dp.rho0 = (float)rho0;
  dp.jx0 = (float)(rho0 * u0[0]);
  dp.jy0 = (float)(rho0 * u0[1]);
  if (storage_dtype == LBM_F64 || storage_dtype == LBM_F64DEV) {
    h->rho0 = rho0;
    h->j0[0] = rho0 * u0[0];
    h->j0[1] = rho0 * u0[1];
  } else {
    h->rho0 = dp.rho0;
    h->j0[0] = dp.jx0;
    h->j0[1] = dp.jy0;
  }
  host_feq_j(h->rho0, h->j0[0], h->j0[1], h->f0);
  split_rate(h->S_paper[3] / 36.0, dp.k3, dp.l3);
  split_rate(h->S_paper[4] / 36.0, dp.k4, dp.l4);
  split_rate(h->S_paper[5] / 12.0, dp.k5, dp.l5);
  split_rate(h->S_paper[6] / 12.0, dp.k6, dp.l6);
  split_rate(h->S_paper[7] / 4.0, dp.k7, dp.l7);
  split_rate(h->S_paper[8] / 4.0, dp.k8, dp.l8);
  {
    const double jx = dp.jx0, jy = dp.jy0, r = dp.rho0;
    split_rate(jx * jx + jy * jy, dp.q0h, dp.q0l);
    split_rate(jx * jx - jy * jy, dp.d0h, dp.d0l);
    split_rate(jx * jy, dp.x0h, dp.x0l);
    split_rate(1.0 / (r * r), dp.i2h, dp.i2l);
  }
  dp.scale = 1.0f;
  dp.inv_scale = 1.0f;
  {
    // FP64 deviation storage: the reference state and rates in FP64
    DevParams64 &q = h->L.dp64;
    q.rho0 = h->rho0;
    q.jx0 = h->j0[0];
    q.jy0 = h->j0[1];
    q.k3 = h->S_paper[3] / 36.0;
    q.k4 = h->S_paper[4] / 36.0;
    q.k5 = h->S_paper[5] / 12.0;
    q.k6 = h->S_paper[6] / 12.0;
    q.k7 = h->S_paper[7] / 4.0;
    q.k8 = h->S_paper[8] / 4.0;
    q.q0 = q.jx0 * q.jx0 + q.jy0 * q.jy0;
    q.d0 = q.jx0 * q.jx0 - q.jy0 * q.jy0;
    q.x0 = q.jx0 * q.jy0;
    q.i2 = 1.0 / (q.rho0 * q.rho0);
  }
  F64Params &fp = h->L.fp;
  fp.s3 = h->S_paper[3];
  fp.s4 = h->S_paper[4];
  fp.s5 = h->S_paper[5];
  fp.s6 = h->S_paper[6];
  fp.s7 = h->S_paper[7];
  fp.s8 = h->S_paper[8];

  const size_t row_bytes = (size_t)9 * h->L.g.pitch * esize;
  const size_t buf_bytes = row_bytes * (h->L.g.ny + (halo ? 2 : 0));
  for (int k = 0; k < 2; ++k) {
    h->alloc[k] = dev_alloc(buf_bytes);
    h->L.buf[k] = h->alloc[k] && halo ? static_cast<char *>(h->alloc[k]) + row_bytes
                                      : h->alloc[k];
  }
  h->partials = (double *)dev_alloc(sizeof(double) * 4 * drift_blocks());
  h->drift_out = (double *)dev_alloc(sizeof(double) * 4);
  h->maxbits = (unsigned int *)dev_alloc(sizeof(unsigned int));
  if (!h->L.buf[0] || !h->L.buf[1] || !h->partials || !h->drift_out || !h->maxbits) {
    lbm_destroy(h);
    set_error("device allocation failed");
    return LBM_ENOMEM;
  }
  // the step kernels move 16-byte vectors and bulk copies of them
  if ((reinterpret_cast<uintptr_t>(h->alloc[0]) | reinterpret_cast<uintptr_t>(h->alloc[1])) & 255) {
    lbm_destroy(h);
    set_error("the device allocator returned memory not aligned to 256 bytes");
    return LBM_EINVAL;
  }
  h->bytes = 2 * buf_bytes + sizeof(double) * (4 * drift_blocks() + 4) + sizeof(unsigned int);
  if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    lbm_destroy(h);
    set_error("cannot create a stream");
    return LBM_ECUDA;
  }
  h->stream = h->own_stream;
  // start from the uniform equilibrium f^eq(rho0, u0)
  if (cudaMemsetAsync(h->alloc[0], 0, buf_bytes, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->alloc[1], 0, buf_bytes, h->stream) != cudaSuccess) {
    cudaGetLastError();
    lbm_destroy(h);
    set_error("memset failed");
    return LBM_ECUDA;
  }
  if (storage_dtype == LBM_F64) {
    const double p[8] = {0, 1, 0, 0, 0, 0, 0, 0};  // zero-amplitude Gaussian
    int rc = do_init(h, nullptr, nullptr, nullptr, LBM_INIT_GAUSSIAN, p);
    if (rc != LBM_OK) {
      lbm_destroy(h);
      return rc;
    }
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    set_error(std::string("create: ") + cudaGetErrorString(cudaGetLastError()));
    lbm_destroy(h);
    return LBM_ECUDA;
  }
  *out = h;
  return LBM_OK;
}

Lattice &lattice_of(lbm_handle h) { return h->L; }
int block_of(lbm_handle h) { return h->block; }
bool is_slab(lbm_handle h) { return h->slab; }
cudaStream_t stream_of(lbm_handle h) { return h->stream; }
int device_of(lbm_handle h) { return h->device; }
void advance_one(lbm_handle h) {
  h->L.cur ^= 1;
  h->t += 1;
}
}  // namespace lbm

extern "C" {

int lbm_create(int nx, int ny, const double S[9], double rho0, const double u0[2],
               int storage_dtype, lbm_handle *out) {
  return create_lattice(nx, ny, S, rho0, u0, storage_dtype, false, out);
}

int lbm_destroy(lbm_handle h) {
  if (!h) return LBM_EINVAL;
  DevGuard g(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_graph(h);
  dev_free(h->src_tab);
  dev_free(h->alloc[0]);
  dev_free(h->alloc[1]);
  dev_free(h->partials);
  dev_free(h->drift_out);
  dev_free(h->maxbits);
  dev_free(h->stage);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  cudaGetLastError();
  delete h;
  return LBM_OK;
}

int lbm_set_stream(lbm_handle h, void *stream) {
  REQUIRE(h != nullptr, "null handle");
  DevGuard g(h->device);
  CK(cudaStreamSynchronize(h->stream));
  h->stream = stream ? (cudaStream_t)stream : h->own_stream;
  return LBM_OK;
}

int lbm_sync(lbm_handle h) {
  REQUIRE(h != nullptr, "null handle");
  DevGuard g(h->device);
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_init_field_dev(lbm_handle h, const double *rho, const double *ux, const double *uy) {
  REQUIRE(h && rho && ux && uy, "null argument");
  DevGuard g(h->device);
  return do_init(h, rho, ux, uy, 0, nullptr);
}

int lbm_init_field(lbm_handle h, const double *rho, const double *ux, const double *uy) {
  REQUIRE(h && rho && ux && uy, "null argument");
  DevGuard g(h->device);
  const size_t n = (size_t)h->L.g.nx * h->L.g.ny;
  int rc = ensure_stage(h);
  if (rc != LBM_OK) return rc;
  CK(cudaMemcpyAsync(h->stage, rho, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->stage + n, ux, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->stage + 2 * n, uy, n * sizeof(double), cudaMemcpyHostToDevice,
                     h->stream));
  // the fields are validated on the device, inside the init kernel
  rc = do_init(h, h->stage, h->stage + n, h->stage + 2 * n, 0, nullptr, h->maxbits);
  if (rc != LBM_OK) return rc;
  unsigned int bad = 0;
  CK(cudaMemcpyAsync(&bad, h->maxbits, sizeof(bad), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (bad) {
    set_error(std::to_string(bad) + " nodes with non-finite fields or rho <= 0");
    return LBM_EINVAL;
  }
  return LBM_OK;
}

int lbm_init_analytic(lbm_handle h, int kind, const double params[8]) {
  REQUIRE(h && params, "null argument");
  REQUIRE(!h->slab, "analytic fields are defined on whole lattices; give a slab its rows' fields");
  REQUIRE(kind == LBM_INIT_GAUSSIAN || kind == LBM_INIT_PLANE, "unknown init kind");
  for (int k = 0; k < 8; ++k) REQUIRE(isfinite(params[k]), "params must be finite");
  if (kind == LBM_INIT_GAUSSIAN) REQUIRE(params[1] > 0.0, "half-width must be positive");
  DevGuard g(h->device);
  return do_init(h, nullptr, nullptr, nullptr, kind, params);
}

int lbm_step(lbm_handle h, long n) {
  NvtxRange nvtx("lbm_step");
  REQUIRE(h != nullptr, "null handle");
  REQUIRE(n >= 0, "negative step count");
  REQUIRE(!h->slab || n <= 1, "a slab takes one step between halo exchanges");
  REQUIRE(h->batch == nullptr, "lattice is a batch member; step the batch");
  DevGuard g(h->device);
  if (n > 0) {
    int rc = maybe_autotune(h);
    if (rc != LBM_OK) return rc;
  }
  if (h->src_on) {
    // The forcing changes every step.  Runs of kSrcGraph steps from buffer 0
    // replay a captured graph after the host uploads that run's forcing
    // (the same host arithmetic as a single forced step, so both paths give
    // identical populations); other steps are launched one by one.
    const double PI = 3.14159265358979323846;
    auto forcing = [&](long long t, double *fs) {
      const double rho_t = h->rho0 + h->s_amp * sin(2.0 * PI * (double)t / h->s_period);
      host_feq_j(rho_t, 0.0, 0.0, fs);
    };
    while (n > 0) {
      if (h->L.cur == 0 && n >= kSrcGraph) {
        if (!h->src_graph || h->src_gx != h->sx || h->src_gy != h->sy) {
          int rc = capture_src_graph(h);
          if (rc != LBM_OK) return rc;
        }
        double tab[9 * kSrcGraph];
        for (int k = 0; k < kSrcGraph; ++k) forcing(h->t + k, tab + 9 * k);
        // pageable source: the copy is staged before the call returns
        CK(cudaMemcpyAsync(h->src_tab, tab, sizeof(tab), cudaMemcpyHostToDevice, h->stream));
        CK(cudaGraphLaunch(h->src_graph, h->stream));
        n -= kSrcGraph;
        h->t += kSrcGraph;
      } else {
        double fs[9];
        forcing(h->t, fs);
        CK(launch_force_node(aux_view(h), h->sx, h->sy, fs, h->stream));
        CK(launch_one(h, h->L.cur, h->stream));
        h->L.cur ^= 1;
        n -= 1;
        h->t += 1;
      }
    }
    return LBM_OK;
  }
  const int G = 64;  // steps per captured graph (even)
  while (n > 0) {
    if (h->L.cur == 0 && n >= G) {
      if (!h->graph || h->graph_steps != G) {
        int rc = capture_graph(h, G);
        if (rc != LBM_OK) return rc;
      }
      CK(cudaGraphLaunch(h->graph, h->stream));
      n -= G;
      h->t += G;
    } else {
      CK(launch_one(h, h->L.cur, h->stream));
      h->L.cur ^= 1;
      n -= 1;
      h->t += 1;
    }
  }
  return LBM_OK;
}

int lbm_set_source(lbm_handle h, int x, int y, double amplitude, double period) {
  REQUIRE(h != nullptr, "null handle");
  REQUIRE(!h->slab, "no point source on a slab");
  REQUIRE(x >= 0 && x < h->L.g.nx && y >= 0 && y < h->L.g.ny, "source outside the lattice");
  REQUIRE(isfinite(amplitude) && isfinite(period) && period > 0, "bad source amplitude or period");
  REQUIRE(h->batch == nullptr, "lattice is a batch member");
  // FP16: the stored state's scale must leave room for the source (the
  // scale maps the largest deviation near 2^14, FP16's largest is 65504)
  REQUIRE(h->L.dtype != LBM_F16DEV || 4.0 / 9.0 * fabs(amplitude) * h->qscale < 32768.0,
          "source amplitude exceeds the FP16 storage scale of the current state; set the "
          "source before lbm_init_field or lbm_set_populations");
  h->src_on = amplitude != 0.0;
  h->sx = x;
  h->sy = y;
  h->s_amp = amplitude;
  h->s_period = period;
  return LBM_OK;
}

int lbm_set_variant(lbm_handle h, int variant) {
  REQUIRE(h != nullptr, "null handle");
  REQUIRE(variant >= 0 && variant < kStepVariants, "no such launch variant");
  if (h->L.variant != variant) free_graph(h);
  h->L.variant = variant;
  h->tuned = true;
  return LBM_OK;
}

int lbm_tune(lbm_handle h, double *times_ms, int *chosen) {
  REQUIRE(h != nullptr, "null handle");
  REQUIRE(h->batch == nullptr, "lattice is a batch member; tune the batch");
  DevGuard g(h->device);
  int rc = tune_handle(h, times_ms);
  if (rc == LBM_OK && chosen) *chosen = h->L.variant;
  return rc;
}

int lbm_moments_dev(lbm_handle h, double *rho, double *ux, double *uy) {
  REQUIRE(h && rho && ux && uy, "null argument");
  DevGuard g(h->device);
  CK(launch_moments(aux_view(h), rho, ux, uy, h->stream));
  return LBM_OK;
}

int lbm_moments(lbm_handle h, double *rho, double *ux, double *uy) {
  REQUIRE(h && rho && ux && uy, "null argument");
  DevGuard g(h->device);
  int rc = ensure_stage(h);
  if (rc != LBM_OK) return rc;
  const size_t n = (size_t)h->L.g.nx * h->L.g.ny;
  CK(launch_moments(aux_view(h), h->stage, h->stage + n, h->stage + 2 * n, h->stream));
  CK(cudaMemcpyAsync(rho, h->stage, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(ux, h->stage + n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(uy, h->stage + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_get_populations(lbm_handle h, double *f) {
  REQUIRE(h && f, "null argument");
  DevGuard g(h->device);
  const size_t n = (size_t)h->L.g.nx * h->L.g.ny;
  double *tmp = (double *)dev_alloc(9 * n * sizeof(double));
  if (!tmp) {
    set_error("cannot allocate population staging");
    return LBM_ENOMEM;
  }
  cudaError_t e = launch_get_pop(aux_view(h), tmp, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(f, tmp, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(tmp);
  if (e != cudaSuccess) {
    set_error(std::string("get_populations: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  return LBM_OK;
}

int lbm_set_populations(lbm_handle h, const double *f) {
  REQUIRE(h && f, "null argument");
  REQUIRE(h->batch == nullptr, "lattice is a batch member");
  DevGuard g(h->device);
  const size_t n = (size_t)h->L.g.nx * h->L.g.ny;
  for (size_t k = 0; k < 9 * n; ++k) REQUIRE(isfinite(f[k]), "populations must be finite");
  double *tmp = (double *)dev_alloc(9 * n * sizeof(double));
  if (!tmp) {
    set_error("cannot allocate population staging");
    return LBM_ENOMEM;
  }
  h->L.cur = 0;
  cudaError_t e =
      cudaMemcpyAsync(tmp, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && h->L.dtype == LBM_F16DEV) {
    e = launch_maxdev_pop(aux_view(h), tmp, h->maxbits, h->stream);
    unsigned int bits = 0;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&bits, h->maxbits, sizeof(bits), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    float m;
    memcpy(&m, &bits, sizeof(m));
    if (e == cudaSuccess) set_qscale(h, std::max((double)m, source_maxdev(h)));
  }
  if (e == cudaSuccess) e = launch_set_pop(aux_view(h), tmp, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(tmp);
  if (e != cudaSuccess) {
    set_error(std::string("set_populations: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  h->t = 0;
  return LBM_OK;
}

int lbm_drift(lbm_handle h, double out[4]) {
  NvtxRange nvtx("lbm_drift");
  REQUIRE(h && out, "null argument");
  DevGuard g(h->device);
  CK(launch_drift(aux_view(h), h->partials, h->drift_out, h->stream));
  CK(cudaMemcpyAsync(out, h->drift_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return out[3] > 0 ? LBM_EUNSTABLE : LBM_OK;
}

int lbm_info(lbm_handle h, lbm_info_t *out) {
  REQUIRE(h && out, "null argument");
  out->nx = h->L.g.nx;
  out->ny = h->L.g.ny;
  out->pitch = h->L.g.pitch;
  out->dtype = h->L.dtype;
  out->elem_bytes = h->L.esize;
  out->t = h->t;
  out->qscale = h->qscale;
  for (int k = 0; k < 9; ++k) out->S_paper[k] = h->S_paper[k];
  out->device_bytes = h->bytes;
  return LBM_OK;
}

}  // extern "C"

