// Internal to liblbm.so: the lattice handle and the helpers that the
// handle code (lbm_api.cu) and the batch runtime (batch.cu) share.
#pragma once
#include <map>
#include <mutex>
#include <string>

#include "lbm_internal.h"

struct lbm_batch_ctx;

struct lbm_ctx {
  lbm::Lattice L;
  int device = 0;
  double S_paper[9];
  double rho0 = 1.0, j0[2] = {0, 0};  // reference state (FP32-exact for *DEV)
  double f0[9];                       // base populations f^eq(rho0, j0)
  double qscale = 1.0;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  long t = 0;
  double *partials = nullptr, *drift_out = nullptr;
  unsigned int *maxbits = nullptr;
  double *stage = nullptr;  // 3 * N doubles, lazily allocated
  void *alloc[2] = {nullptr, nullptr};  // the buffers' allocations (one halo row
                                        // before L.buf[k] for slabs)
  bool slab = false;  // rows of a larger lattice, with halo rows (slabs.cu)
  size_t bytes = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  // 64-thread blocks for the deviation step: a block retires as soon as its
  // two warps finish, so fewer warp slots sit idle behind a slow warp than
  // with 256-thread blocks (measured +3-4% on batches, +5-7% on one FP16 or
  // BF16 lattice, FP32 8192^2 unchanged); the FP64 step keeps 256
  int block = 64;
  int grid_cap = 0;
  bool tuned = false;
  lbm_batch_ctx *batch = nullptr;
  // acoustic point source (lbm_set_source)
  bool src_on = false;
  int sx = 0, sy = 0;
  double s_amp = 0, s_period = 1;
  // forced steps in graphs: kSrcGraph x (forced node from src_tab[k], step)
  cudaGraphExec_t src_graph = nullptr;
  double *src_tab = nullptr;  // 9 populations per captured step
  int src_gx = -1, src_gy = -1;  // source node the graph was captured for
};

#define CK(call)                                                            \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
      cudaGetLastError();                                                   \
      return LBM_ECUDA;                                                     \
    }                                                                       \
  } while (0)

#define REQUIRE(cond, msg)         \
  do {                             \
    if (!(cond)) {                 \
      set_error(msg);              \
      return LBM_EINVAL;           \
    }                              \
  } while (0)

namespace lbm {

// the handle's drift / I-O view (current buffer, reference state, scale)
AuxView aux_view(const lbm_ctx *h);
// the largest |f'| a point source writes (0 without one)
double source_maxdev(const lbm_ctx *h);
// FP16 storage scale: set it (dropping graphs that hold the old one), or
// choose it from the largest |f'| (fp16_scale)
void set_scale(lbm_ctx *h, double s);
void set_qscale(lbm_ctx *h, double maxabs);
int free_graph(lbm_ctx *h);
// launch variant before (or without) tuning
int default_variant(int dtype);
// the host staging buffer of a handle's field I/O (lazily allocated)
int ensure_stage(lbm_ctx *h);

// tuning: LBM_AUTOTUNE, the optional tuning file (LBM_TUNE_CACHE) and the
// batch choices read from it; g_tune_mu guards the caches and the file
bool autotune_enabled();
unsigned long long fnv1a(const std::string &s);
extern std::mutex g_tune_mu;
extern std::map<unsigned long long, int> g_batch_file_cache;
void tune_file_load_locked();
void tune_file_append_locked(const char *kind, const std::string &key, int v);
// repetitions for ~2 ms of traffic per variant
int tune_reps(double bytes);

// Average duration of `reps` launches produced by `launch(k)` on stream st.
template <typename F>
int time_launches(cudaStream_t st, int reps, F launch, double *ms) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = launch(0);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int k = 0; k < reps && e == cudaSuccess; ++k) e = launch(k);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_error(std::string("tuning: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  *ms = t / reps;
  return LBM_OK;
}

}  // namespace lbm
