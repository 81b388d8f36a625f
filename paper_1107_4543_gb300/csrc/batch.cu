// C ABI of the batches (include/lbm.h): many independent lattices stepped
// together -- per-step launches over a work list of block records, replayed
// from captured graphs, small members held in shared memory for all the
// steps of a call -- their packed host I/O, the pipelined solves, batch
// tuning and drift.
#include <math.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <unordered_set>
#include <vector>

#include "lbm_internal.h"
#include "runtime.h"
#include "slots.h"

using namespace lbm;

// ------------------------------------------------------------ constant slots
// Slots of the batched step's constant tables (const_slots(dtype) per
// storage type and device, step_impl.cuh): a batch group holds one
// contiguous range from its creation to its destruction; a group that finds
// no room (or runs with LBM_CONST_TABLE=0) reads its entries' parameters
// instead.
namespace {
std::mutex g_slot_mu;
std::map<std::pair<int, int>, SlotRanges> g_slots;  // (device, dtype) -> its table's ranges

int slots_reserve(int dev, int dtype, int n) {
  const char *env = getenv("LBM_CONST_TABLE");
  if (env != nullptr && strcmp(env, "0") == 0) return -1;
  std::lock_guard<std::mutex> lk(g_slot_mu);
  auto it = g_slots.find({dev, dtype});
  if (it == g_slots.end())
    it = g_slots.emplace(std::make_pair(dev, dtype), SlotRanges(const_slots(dtype))).first;
  return it->second.reserve(n);
}

void slots_release(int dev, int dtype, int base, int n) {
  std::lock_guard<std::mutex> lk(g_slot_mu);
  auto it = g_slots.find({dev, dtype});
  if (it != g_slots.end()) it->second.release(base, n);
}
}  // namespace

// ------------------------------------------------------------------ batch
struct lbm_batch_ctx {
  std::vector<lbm_ctx *> members;
  int device = 0;
  cudaStream_t stream = nullptr;
  struct Group {
    int dtype;
    int n;
    long long ntasks;
    long long nblocks;
    BatchEntry *ents = nullptr;
    BlockRec *blocks = nullptr;
    int *limits = nullptr;  // per-entry step limits of a ragged generation
    // entries held in shared memory for all the steps of a launch (small
    // lattices; k_batch_resident), which the block records leave out; in
    // three classes by size (up to a third, a half, all of a block's shared
    // memory), one launch each, so that small ones share an SM
    int nres = 0;
    int *res = nullptr;
    int res_count[3] = {0, 0, 0};
    size_t res_smem[3] = {0, 0, 0};  // shared memory of a block of the class
    // the group's slots in its type's constant table (-1: none) and the
    // device staging of their refresh (n x const_slot_bytes(dtype))
    int pbase = -1;
    void *pstage = nullptr;
  };
  std::vector<int> member_group, member_local;  // member -> (group, entry)
  std::vector<int> member_res;                  // member stepped as a resident entry
  bool spent = false;  // a ragged generation ran: members' parities differ
  std::vector<Group> groups;
  bool resident = false;                 // some group has resident entries
  cudaStream_t res_stream = nullptr;     // their launches, beside the batch stream
  cudaEvent_t res_fork = nullptr, res_join = nullptr;
  std::vector<int> offs;                 // member buffer index at creation
  std::vector<cudaStream_t> saved_streams;
  AuxView *views[2] = {nullptr, nullptr}; // drift views at batch parity 0 / 1
  double *dpart = nullptr, *dout = nullptr;
  unsigned int *dflags = nullptr;         // per-member counters (2 per member)
  int parity = 0;                        // steps taken mod 2
  // captured step sequences, keyed by step count, each starting at batch
  // parity 0 (64 steps, and the remainders of longer calls)
  std::map<long, cudaGraphExec_t> graphs;
  int block = 64;                        // threads per block (see lbm_ctx::block)
  int variant = 2;                       // launch variant (tuner)
  bool tuned = false;
  long long nodes = 0;
  // host<->device copies of the batch-level field I/O run on their own
  // stream, member by member, so that they overlap the kernels of the
  // members before (init) or after (moments) them
  cudaStream_t io = nullptr;
  cudaEvent_t io_ev = nullptr;
  // packed host I/O: member k's fields start at poff[k] of a packed array;
  // pstage holds rho, ux, uy of all members (3 x nodes doubles, lazily)
  std::vector<size_t> poff;
  double *pstage = nullptr;
  // pipelined solves (lbm_batch_solve_packed / lbm_batch_wait): two slots,
  // each with device staging for the fields in and the moments out and its
  // own drift sums, so that solve k's upload (copy stream `up`) and solve
  // k-1's download (copy stream `down`) run while the batch stream steps.
  // Events per solve, in stream order: up stream E_UP0 .. E_UP1 (H2D); batch
  // stream E_B0 (upload landed), E_INIT, E_STEP, E_DRIFT, E_MOM; down stream
  // E_DN0 .. E_DN1 (D2H).  They sit in a ring of kRing solves: solve s waits
  // on the events of solve s - 2 (the last user of its slot), and
  // lbm_batch_wait reads the phase times of every solve still in the ring.
  enum { E_UP0, E_UP1, E_B0, E_INIT, E_STEP, E_DRIFT, E_MOM, E_DN0, E_DN1, E_COUNT };
  static constexpr int kRing = 32;
  cudaEvent_t ring[kRing][E_COUNT] = {};
  long long waited = 0;  // solves queued before the last lbm_batch_wait
  // The caller's drift array may be pageable memory, and a copy into
  // pageable memory would block the host until the solve ends (which
  // serialises the next solve's upload behind it): the sums land in a
  // page-locked array of the slot and a host function on the download
  // stream copies them out.
  struct DriftOut {
    double *dst = nullptr;
    const double *src = nullptr;
    size_t bytes = 0;
  };
  struct Slot {
    double *in = nullptr, *out = nullptr;  // 3 x nodes doubles each
    double *dout = nullptr;                // drift sums, 4 per member
    double *hdrift = nullptr;              // page-locked copy of dout
    bool used = false;
  };
  Slot slot[2];
  cudaStream_t up = nullptr, down = nullptr;
  unsigned int *sbad = nullptr;  // per member: this solve's invalid nodes, then the total
  IoBlock *ioblk = nullptr;      // blocks of the batched init / moments launches
  long long nioblk = 0;
  long long *poff_dev = nullptr;  // members' offsets in the packed arrays
  // FP16 members of pipelined solves choose their storage scale on the
  // device: per member the largest |f'| (float bits), the floor (a point
  // source's amplitude), the scale chosen, and the member's batch entry
  bool has16 = false;
  unsigned int *smax = nullptr;
  double *sfloor = nullptr, *sscale = nullptr;
  BatchEntry **sent = nullptr;
  long long solves = 0;          // solves queued since the batch was made
  int last_slot = -1;
  std::vector<double *> pending_drift;  // caller's drift arrays since the last wait
};

static int ensure_io(lbm_batch_ctx *b) {
  if (b->io) return LBM_OK;
  CK(cudaStreamCreateWithFlags(&b->io, cudaStreamNonBlocking));
  cudaError_t e = cudaEventCreateWithFlags(&b->io_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaStreamDestroy(b->io);
    b->io = nullptr;
    CK(e);
  }
  return LBM_OK;
}

static BatchList batch_list(const lbm_batch_ctx::Group &gr) {
  BatchList bl;
  bl.ents = gr.ents;
  bl.n = gr.n;
  bl.blocks = gr.blocks;
  bl.nblocks = gr.nblocks;
  bl.ntasks = gr.ntasks;
  bl.pbase = gr.pbase;
  return bl;
}

// Refresh the groups' constant-table slots from their entries, in the
// order of the batch stream: before any call steps, since the entries may
// have changed (a member's FP16 scale, set on the host or by a solve).
static int batch_upload_pairs(lbm_batch_ctx *b) {
  for (auto &gr : b->groups)
    if (gr.pbase >= 0)
      CK(upload_batch_consts(gr.dtype, gr.ents, gr.n, gr.pbase, gr.pstage, b->stream));
  return LBM_OK;
}

// Launch the resident entries of every group for `steps` steps from batch
// parity `parity` (limits: per-entry step limits of a ragged generation, or
// null) on the side stream, forked from the batch stream; resident_join
// makes the batch stream wait for them.
static int resident_fork(lbm_batch_ctx *b, int parity, long steps, bool ragged) {
  if (!b->resident || steps < 1) return LBM_OK;
  if (!b->res_stream) {
    CK(cudaStreamCreateWithFlags(&b->res_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&b->res_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&b->res_join, cudaEventDisableTiming));
  }
  CK(cudaEventRecord(b->res_fork, b->stream));
  CK(cudaStreamWaitEvent(b->res_stream, b->res_fork, 0));
  for (auto &gr : b->groups)
    for (int c = 0, off = 0; c < 3; off += gr.res_count[c++])
      if (gr.res_count[c] > 0)
        CK(launch_batch_resident(gr.dtype, gr.ents, gr.res + off, gr.res_count[c], gr.n,
                                 gr.res_smem[c], parity, steps, ragged ? gr.limits : nullptr,
                                 b->res_stream));
  CK(cudaEventRecord(b->res_join, b->res_stream));
  return LBM_OK;
}

static int resident_join(lbm_batch_ctx *b) {
  if (b->resident && b->res_join) CK(cudaStreamWaitEvent(b->stream, b->res_join, 0));
  return LBM_OK;
}

static cudaError_t batch_launch_all(lbm_batch_ctx *b, int parity, cudaStream_t st,
                                    int variant) {
  for (auto &gr : b->groups) {
    cudaError_t e = launch_step_batch(gr.dtype, batch_list(gr), parity, st, b->block, variant);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static void batch_drop_graphs(lbm_batch_ctx *b) {
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

// The captured sequence of `steps` batched step launches starting at batch
// parity 0 (captured on first use, kept until the launch variant changes).
static int batch_graph(lbm_batch_ctx *b, long steps, cudaGraphExec_t *out) {
  auto it = b->graphs.find(steps);
  if (it != b->graphs.end()) {
    *out = it->second;
    return LBM_OK;
  }
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t gr = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (long k = 0; k < steps && e == cudaSuccess; ++k)
      e = batch_launch_all(b, (int)(k & 1), cs, b->variant);
    cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, gr, 0);
  if (gr) cudaGraphDestroy(gr);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    set_error(std::string("batch graph capture: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  b->graphs[steps] = ex;
  *out = ex;
  return LBM_OK;
}

static std::map<std::string, int> g_batch_tune_cache;

static std::string batch_key(const lbm_batch_ctx *b) {
  std::string k;
  for (auto *m : b->members)
    k += std::to_string(m->L.dtype) + ":" + std::to_string(m->L.g.nx) + "x" +
         std::to_string(m->L.g.ny) + ",";
  return k;
}

// As tune_handle, for the whole batch: trial launches at the current parity
// write only the idle buffers.
static int tune_batch(lbm_batch_ctx *b, double *times) {
  int urc = batch_upload_pairs(b);
  if (urc != LBM_OK) return urc;
  double bytes = 0;
  for (auto *m : b->members) bytes += (double)m->L.g.nx * m->L.g.ny * 18.0 * m->L.esize;
  const int reps = tune_reps(bytes);
  double best = 1e300;
  int bv = b->variant;
  for (int v = 0; v < kBatchVariants; ++v) {
    double ms = 0;
    int rc = time_launches(b->stream, reps,
                           [&](int) { return batch_launch_all(b, b->parity, b->stream, v); }, &ms);
    if (rc != LBM_OK) return rc;
    if (times) times[v] = ms;
    if (ms < best) {
      best = ms;
      bv = v;
    }
  }
  if (bv != b->variant) {
    b->variant = bv;
    batch_drop_graphs(b);
  }
  b->tuned = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const std::string key = batch_key(b);
  g_batch_tune_cache[key] = bv;
  char hex[32];
  snprintf(hex, sizeof(hex), "%016llx", fnv1a(key));
  tune_file_append_locked("B", hex, bv);
  return LBM_OK;
}

// First step of a large batch: reuse the choice made for a batch of the
// same composition (storage types and sizes, in order) or tune now.
static int maybe_autotune_batch(lbm_batch_ctx *b) {
  if (b->nodes >= (1LL << 20) && autotune_enabled()) {
    int cached = -1;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_file_load_locked();
      const std::string key = batch_key(b);
      auto it = g_batch_tune_cache.find(key);
      if (it != g_batch_tune_cache.end()) {
        cached = it->second;
      } else {
        auto jt = g_batch_file_cache.find(fnv1a(key));
        if (jt != g_batch_file_cache.end()) cached = jt->second;
      }
    }
    if (cached >= 0) {
      b->variant = cached;
    } else {
      int rc = tune_batch(b, nullptr);
      if (rc != LBM_OK) return rc;
    }
  }
  b->tuned = true;
  return LBM_OK;
}

namespace lbm {
// Pin a batch's launch variant (no automatic tuning); -1 leaves it to the
// tuner.  Used by the server, which tunes once and reuses the choice.
void batch_pin_variant(lbm_batch_ctx *b, int variant) {
  if (variant < 0 || variant >= kBatchVariants) return;
  if (b->variant != variant) batch_drop_graphs(b);
  b->variant = variant;
  b->tuned = true;
}
int batch_variant(const lbm_batch_ctx *b) { return b->tuned ? b->variant : -1; }

int batch_step_ragged(lbm_batch_ctx *b, const long *steps, long n) {
  REQUIRE(b != nullptr && steps != nullptr && n >= 0, "bad ragged step arguments");
  REQUIRE(!b->spent && b->parity == 0, "ragged steps need a fresh batch");
  REQUIRE(n <= 0x3fffffffL, "too many steps for one generation");
  DevGuard g(b->device);
  if (n > 0) {
    int rc = batch_upload_pairs(b);
    if (rc == LBM_OK && !b->tuned) rc = maybe_autotune_batch(b);
    if (rc != LBM_OK) return rc;
  }
  const size_t nm = b->members.size();
  std::vector<std::vector<int>> lim(b->groups.size());
  for (size_t gi = 0; gi < b->groups.size(); ++gi) lim[gi].assign(b->groups[gi].n, 0);
  std::vector<long> take(nm);
  for (size_t mi = 0; mi < nm; ++mi) {
    take[mi] = std::max(0L, std::min(steps[mi], n));
    lim[b->member_group[mi]][b->member_local[mi]] = (int)take[mi];
  }
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    CK(cudaMemcpyAsync(b->groups[gi].limits, lim[gi].data(), sizeof(int) * lim[gi].size(),
                       cudaMemcpyHostToDevice, b->stream));
  int rrc = resident_fork(b, 0, n, true);
  if (rrc != LBM_OK) return rrc;
  for (long k = 0; k < n; ++k)
    for (auto &gr : b->groups)
      CK(launch_step_batch(gr.dtype, batch_list(gr), (int)(k & 1), b->stream, b->block,
                           b->variant, gr.limits, (int)k));
  rrc = resident_join(b);
  if (rrc != LBM_OK) return rrc;
  for (size_t mi = 0; mi < nm; ++mi) {
    b->members[mi]->L.cur = b->offs[mi] ^ (int)(take[mi] & 1);
    b->members[mi]->t += take[mi];
  }
  b->spent = true;
  // the host arrays above must outlive the copies
  CK(cudaStreamSynchronize(b->stream));
  return LBM_OK;
}
long long batch_nodes(const lbm_batch_ctx *b) { return b->nodes; }
}  // namespace lbm

static void batch_free(lbm_batch_ctx *b) {
  batch_drop_graphs(b);
  for (auto *st : {b->up, b->down, b->res_stream})
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (auto *ev : {b->res_fork, b->res_join})
    if (ev) cudaEventDestroy(ev);
  for (auto &r : b->ring)
    for (auto &e : r)
      if (e) cudaEventDestroy(e);
  for (auto &sl : b->slot) {
    dev_free(sl.in);
    dev_free(sl.out);
    dev_free(sl.dout);
    if (sl.hdrift) cudaFreeHost(sl.hdrift);
  }
  dev_free(b->sbad);
  dev_free(b->ioblk);
  dev_free(b->poff_dev);
  dev_free(b->smax);
  dev_free(b->sfloor);
  dev_free(b->sscale);
  dev_free(b->sent);
  if (b->io) {
    cudaStreamSynchronize(b->io);
    cudaStreamDestroy(b->io);
    cudaEventDestroy(b->io_ev);
  }
  dev_free(b->pstage);
  for (auto &gr : b->groups) {
    dev_free(gr.ents);
    dev_free(gr.blocks);
    dev_free(gr.limits);
    dev_free(gr.res);
    dev_free(gr.pstage);
    if (gr.pbase >= 0) slots_release(b->device, gr.dtype, gr.pbase, gr.n);
  }
  dev_free(b->views[0]);
  dev_free(b->views[1]);
  dev_free(b->dpart);
  dev_free(b->dout);
  dev_free(b->dflags);
  for (size_t k = 0; k < b->members.size(); ++k) {
    auto *m = b->members[k];
    if (m->batch == b) m->batch = nullptr;
    if (k < b->saved_streams.size()) m->stream = b->saved_streams[k];
  }
  cudaGetLastError();
  delete b;
}

// Refresh the device copies of the members' step parameters (after the
// FP16 storage scale of a member changed).
static int batch_refresh_params(lbm_batch_ctx *b) {
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    auto &gr = b->groups[gi];
    std::vector<BatchEntry> ents((size_t)gr.n);
    CK(cudaMemcpyAsync(ents.data(), gr.ents, sizeof(BatchEntry) * gr.n, cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    for (size_t mi = 0; mi < b->members.size(); ++mi)
      if (b->member_group[mi] == (int)gi) ents[b->member_local[mi]].dp = b->members[mi]->L.dp;
    CK(cudaMemcpyAsync(gr.ents, ents.data(), sizeof(BatchEntry) * gr.n, cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
  }
  const int n = (int)b->members.size();
  for (int par = 0; par < 2; ++par) {
    std::vector<AuxView> v((size_t)n);
    for (int k = 0; k < n; ++k) {
      auto *m = b->members[k];
      v[k] = aux_view(m);
      v[k].buf = m->L.buf[b->offs[k] ^ par];
    }
    CK(cudaMemcpyAsync(b->views[par], v.data(), sizeof(AuxView) * n, cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
  }
  return LBM_OK;
}

// ------------------------------------------------- batch-level host I/O
// Members are visited in copy groups: group g covers members
// [ends[g-1], ends[g]).  A group's copies run on the copy stream while the
// batch stream works on the previous group's members (init) or the copy
// stream downloads a group while the batch stream computes the next one
// (moments).  The staging buffers belong to these synchronous calls alone,
// so uploads need not wait for work already queued on the batch stream.

// init: upload(g) enqueues group g's copies; fields(k, r, u, v) gives member
// k's staged fields.  FP16 members first take their storage scale from the
// new fields (device counters in dflags, one read-back); the others are
// initialised as their group lands.
template <class Upload, class Fields>
static int batch_init_common(lbm_batch_ctx *b, const std::vector<size_t> &ends, Upload upload,
                             Fields fields) {
  NvtxRange nvtx("batch host upload + init");
  int rc = ensure_io(b);
  if (rc != LBM_OK) return rc;
  const size_t nm = b->members.size();
  bool any16 = false;
  size_t k = 0;
  for (size_t gi = 0; gi < ends.size(); ++gi) {
    CK(upload(gi));
    CK(cudaEventRecord(b->io_ev, b->io));
    CK(cudaStreamWaitEvent(b->stream, b->io_ev, 0));
    for (; k < ends[gi]; ++k) {
      auto *m = b->members[k];
      const double *r, *u, *v;
      fields(k, r, u, v);
      if (m->L.dtype == LBM_F16DEV) {
        any16 = true;
        CK(launch_maxdev_eq(aux_view(m), r, u, v, 0, nullptr, b->dflags + k, b->stream));
      } else {
        CK(launch_init_eq(aux_view(m), r, u, v, 0, nullptr, b->stream, b->dflags + nm + k));
      }
    }
  }
  if (any16) {
    std::vector<unsigned int> bits(nm, 0);
    CK(cudaMemcpyAsync(bits.data(), b->dflags, sizeof(unsigned int) * nm, cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    for (size_t j = 0; j < nm; ++j)
      if (b->members[j]->L.dtype == LBM_F16DEV) {
        float mx;
        memcpy(&mx, &bits[j], sizeof(mx));
        set_qscale(b->members[j], std::max((double)mx, source_maxdev(b->members[j])));
      }
    rc = batch_refresh_params(b);
    if (rc != LBM_OK) return rc;
    for (size_t j = 0; j < nm; ++j) {
      auto *m = b->members[j];
      if (m->L.dtype != LBM_F16DEV) continue;
      const double *r, *u, *v;
      fields(j, r, u, v);
      CK(launch_init_eq(aux_view(m), r, u, v, 0, nullptr, b->stream, b->dflags + nm + j));
    }
  }
  // equilibria are in each member's current buffer (the batch's bookkeeping
  // of buffers stays valid); the fields were validated on the device
  std::vector<unsigned int> bad(nm, 0);
  CK(cudaMemcpyAsync(bad.data(), b->dflags + nm, sizeof(unsigned int) * nm,
                     cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  for (auto *m : b->members) m->t = 0;
  for (size_t j = 0; j < nm; ++j)
    if (bad[j]) {
      set_error("member " + std::to_string(j) + ": " + std::to_string(bad[j]) +
                " nodes with non-finite fields or rho <= 0");
      return LBM_EINVAL;
    }
  return LBM_OK;
}

// moments: fields(k, r, u, v) gives member k's staging; download(g)
// enqueues group g's copies to the host
template <class Download, class Fields>
static int batch_moments_common(lbm_batch_ctx *b, const std::vector<size_t> &ends,
                                Download download, Fields fields) {
  NvtxRange nvtx("batch moments + download");
  int rc = ensure_io(b);
  if (rc != LBM_OK) return rc;
  size_t k = 0;
  for (size_t gi = 0; gi < ends.size(); ++gi) {
    for (; k < ends[gi]; ++k) {
      double *r, *u, *v;
      fields(k, r, u, v);
      CK(launch_moments(aux_view(b->members[k]), r, u, v, b->stream));
    }
    CK(cudaEventRecord(b->io_ev, b->stream));
    CK(cudaStreamWaitEvent(b->io, b->io_ev, 0));
    CK(download(gi));
  }
  CK(cudaStreamSynchronize(b->io));
  return LBM_OK;
}

// packed layout: member offsets and the batch-wide staging buffer
static void ensure_poff(lbm_batch_ctx *b) {
  const size_t nm = b->members.size();
  if (b->poff.size() == nm + 1) return;
  b->poff.assign(nm + 1, 0);
  for (size_t k = 0; k < nm; ++k)
    b->poff[k + 1] = b->poff[k] + (size_t)b->members[k]->L.g.nx * b->members[k]->L.g.ny;
}

static int ensure_packed(lbm_batch_ctx *b) {
  if (b->pstage) return LBM_OK;
  const size_t nm = b->members.size();
  ensure_poff(b);
  b->pstage = (double *)dev_alloc(3 * b->poff[nm] * sizeof(double));
  if (!b->pstage) {
    set_error("out of device memory for the packed staging buffer");
    return LBM_ENOMEM;
  }
  return LBM_OK;
}

// copy groups of the packed arrays: consecutive members up to about 2^23
// nodes (64 MiB per field) per group, so that every copy is large (many
// small host copies run far below the link rate on some hosts) while the
// copies still overlap the kernels of the neighbouring group
static std::vector<size_t> packed_groups(const lbm_batch_ctx *b) {
  const size_t kGroupNodes = (size_t)1 << 23;
  const size_t nm = b->members.size();
  std::vector<size_t> ends;
  size_t start = 0;
  for (size_t k = 0; k < nm; ++k)
    if (b->poff[k + 1] - b->poff[start] >= kGroupNodes || k + 1 == nm) {
      ends.push_back(k + 1);
      start = k + 1;
    }
  return ends;
}

extern "C" {

int lbm_batch_create(int n, const lbm_handle *members, lbm_batch *out) {
  REQUIRE(n >= 1 && members && out, "bad batch arguments");
  int dev = members[0] ? members[0]->device : 0;
  for (int k = 0; k < n; ++k) {
    REQUIRE(members[k] != nullptr, "null member");
    REQUIRE(members[k]->L.dtype != LBM_F64 && members[k]->L.dtype != LBM_F64DEV,
            "batches take the 32- and 16-bit deviation storage types");
    REQUIRE(members[k]->batch == nullptr, "lattice already in a batch");
    REQUIRE(!members[k]->slab, "slabs of a split lattice cannot join a batch");
    REQUIRE(members[k]->device == dev, "members on different devices");
    for (int j = 0; j < k; ++j) REQUIRE(members[j] != members[k], "duplicate member");
  }
  DevGuard g(dev);
  lbm_batch_ctx *b = new (std::nothrow) lbm_batch_ctx();
  if (!b) {
    set_error("out of host memory");
    return LBM_ENOMEM;
  }
  b->device = dev;
  b->stream = members[0]->stream;
  for (int k = 0; k < n; ++k) b->members.push_back(members[k]);
  // the batch runs on the first member's stream: finish what the members
  // queued elsewhere (each distinct stream once: a server's members share
  // one), then route their later work to the batch stream
  {
    std::unordered_set<cudaStream_t> done;
    for (auto *m : b->members) {
      if (!done.insert(m->stream).second) continue;
      if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        set_error("member stream failed");
        cudaGetLastError();
        batch_free(b);
        return LBM_ECUDA;
      }
    }
  }
  for (auto *m : b->members) {
    b->saved_streams.push_back(m->stream);
    m->stream = b->stream;
  }
  const int wpb = b->block / 32;
  b->member_group.assign(b->members.size(), -1);
  b->member_local.assign(b->members.size(), -1);
  b->member_res.assign(b->members.size(), 0);
  const size_t res_max = resident_limit(dev);
  for (int dt : {LBM_F32DEV, LBM_F16DEV, LBM_BF16DEV}) {
    std::vector<BatchEntry> ents;
    std::vector<BlockRec> bl;  // the plain grid's blocks
    std::vector<int> res_cls[3];  // resident entries by size class
    size_t res_smem[3] = {0, 0, 0};
    long long t0 = 0;
    {
      size_t nb = 0;  // an upper bound of the records (a server builds ~10^5 per generation)
      for (auto *m : b->members)
        if (m->L.dtype == dt) nb += (size_t)((m->L.g.tasks + wpb - 1) / wpb);
      bl.reserve(nb);
    }
    for (size_t mi = 0; mi < b->members.size(); ++mi) {
      auto *m = b->members[mi];
      if (m->L.dtype != dt) continue;
      b->member_group[mi] = (int)b->groups.size();
      b->member_local[mi] = (int)ents.size();
      BatchEntry e;
      e.g = m->L.g;
      e.dp = m->L.dp;
      e.buf[0] = m->L.buf[0];
      e.buf[1] = m->L.buf[1];
      e.off = m->L.cur;
      const size_t rb = resident_bytes(m->L.g.nx, m->L.g.ny, m->L.esize);
      if (rb <= res_max) {
        b->member_res[mi] = 1;
        const int c = rb <= res_max / 3 ? 0 : (rb <= res_max / 2 ? 1 : 2);
        res_cls[c].push_back((int)ents.size());
        res_smem[c] = std::max(res_smem[c], rb);
        ents.push_back(e);
        continue;
      }
      t0 += m->L.g.tasks;
      for (long long tb = 0; tb < m->L.g.tasks; tb += wpb) {
        BlockRec r;
        r.g = e.g;
        r.buf[0] = e.buf[0];
        r.buf[1] = e.buf[1];
        r.task_base = tb;
        r.lat = (int)ents.size();
        r.off = e.off;
        bl.push_back(r);
      }
      ents.push_back(e);
    }
    if (ents.empty()) continue;
    lbm_batch_ctx::Group gr;
    gr.dtype = dt;
    gr.n = (int)ents.size();
    gr.ntasks = t0;
    gr.nblocks = (long long)bl.size();
    gr.ents = (BatchEntry *)dev_alloc(sizeof(BatchEntry) * ents.size());
    gr.blocks = (BlockRec *)dev_alloc(sizeof(BlockRec) * bl.size());
    gr.limits = (int *)dev_alloc(sizeof(int) * ents.size());
    std::vector<int> res;
    for (int c = 0; c < 3; ++c) {
      res.insert(res.end(), res_cls[c].begin(), res_cls[c].end());
      gr.res_count[c] = (int)res_cls[c].size();
      gr.res_smem[c] = res_smem[c];
    }
    gr.nres = (int)res.size();
    if (gr.nres > 0) {
      gr.res = (int *)dev_alloc(sizeof(int) * res.size());
      b->resident = true;
    }
    if (const_slots(dt) > 0) {
      gr.pbase = slots_reserve(b->device, dt, gr.n);
      if (gr.pbase >= 0) {
        gr.pstage = dev_alloc(const_slot_bytes(dt) * (size_t)gr.n);
        if (!gr.pstage) {
          slots_release(b->device, dt, gr.pbase, gr.n);
          gr.pbase = -1;
        }
      }
    }
    b->groups.push_back(gr);
    if (!gr.ents || !gr.blocks || !gr.limits || (gr.nres > 0 && !gr.res)) {
      set_error("cannot allocate batch tables");
      batch_free(b);
      return LBM_ENOMEM;
    }
    if (cudaMemcpyAsync(gr.ents, ents.data(), sizeof(BatchEntry) * ents.size(),
                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        (!bl.empty() && cudaMemcpyAsync(gr.blocks, bl.data(), sizeof(BlockRec) * bl.size(),
                                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess) ||
        (gr.nres > 0 && cudaMemcpyAsync(gr.res, res.data(), sizeof(int) * res.size(),
                                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess)) {
      set_error("cannot upload batch tables");
      cudaGetLastError();
      batch_free(b);
      return LBM_ECUDA;
    }
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    set_error("batch upload failed");
    cudaGetLastError();
    batch_free(b);
    return LBM_ECUDA;
  }
  for (auto *m : b->members) {
    b->offs.push_back(m->L.cur);
    b->nodes += (long long)m->L.g.nx * m->L.g.ny;
  }
  b->variant = default_variant(b->members[0]->L.dtype);
  // drift views of every member for both batch parities
  {
    const int n = (int)b->members.size();
    std::vector<AuxView> v0, v1;
    for (auto *m : b->members) {
      AuxView a = aux_view(m);
      a.buf = m->L.buf[m->L.cur];
      v0.push_back(a);
      a.buf = m->L.buf[m->L.cur ^ 1];
      v1.push_back(a);
    }
    b->views[0] = (AuxView *)dev_alloc(sizeof(AuxView) * n);
    b->views[1] = (AuxView *)dev_alloc(sizeof(AuxView) * n);
    b->dpart = (double *)dev_alloc(sizeof(double) * batch_drift_partials(n));
    b->dout = (double *)dev_alloc(sizeof(double) * 4 * n);
    b->dflags = (unsigned int *)dev_alloc(sizeof(unsigned int) * 2 * n);
    if (!b->views[0] || !b->views[1] || !b->dpart || !b->dout || !b->dflags ||
        cudaMemcpyAsync(b->views[0], v0.data(), sizeof(AuxView) * n, cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->views[1], v1.data(), sizeof(AuxView) * n, cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
      set_error("cannot set up the batch drift tables");
      cudaGetLastError();
      b->offs.clear();
      batch_free(b);
      return LBM_ENOMEM;
    }
  }
  for (auto *m : b->members) m->batch = b;
  b->parity = 0;
  *out = b;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch b, long n) {
  NvtxRange nvtx("lbm_batch_step");
  REQUIRE(b != nullptr, "null batch");
  REQUIRE(n >= 0, "negative step count");
  DevGuard g(b->device);
  REQUIRE(!b->spent, "batch ran a ragged generation; create a new batch");
  for (size_t k = 0; k < b->members.size(); ++k)
    REQUIRE(b->members[k]->L.cur == (b->offs[k] ^ b->parity),
            "a member was modified outside the batch");
  if (n > 0) {
    int rc = batch_upload_pairs(b);
    if (rc == LBM_OK && !b->tuned) rc = maybe_autotune_batch(b);
    if (rc != LBM_OK) return rc;
  }
  // resident members: all n steps in one launch per storage type, beside
  // the per-step launches of the others
  int rrc = resident_fork(b, b->parity, n, false);
  if (rrc != LBM_OK) return rrc;
  // whole graphs of 64 steps, the remainder as one graph of its own length
  // (both cached), so a call of n steps is a handful of graph launches
  const long G = 64;
  long done = 0;
  if (b->parity == 1 && n > 0) {
    CK(batch_launch_all(b, 1, b->stream, b->variant));
    b->parity = 0;
    n -= 1;
    done += 1;
  }
  while (n > 0) {
    const long k = n >= G ? G : n;
    if (k >= 2) {
      cudaGraphExec_t ex = nullptr;
      int rc = batch_graph(b, k, &ex);
      if (rc != LBM_OK) return rc;
      CK(cudaGraphLaunch(ex, b->stream));
      b->parity = (int)(k & 1);
    } else {
      CK(batch_launch_all(b, 0, b->stream, b->variant));
      b->parity = 1;
    }
    n -= k;
    done += k;
  }
  rrc = resident_join(b);
  if (rrc != LBM_OK) return rrc;
  for (size_t k = 0; k < b->members.size(); ++k) {
    b->members[k]->L.cur = b->offs[k] ^ b->parity;
    b->members[k]->t += done;
  }
  return LBM_OK;
}



int lbm_batch_init_fields(lbm_batch b, const double *const *rho, const double *const *ux,
                          const double *const *uy) {
  REQUIRE(b != nullptr && rho && ux && uy, "null argument");
  REQUIRE(!b->spent, "batch ran a ragged generation; create a new batch");
  DevGuard g(b->device);
  const size_t nm = b->members.size();
  for (size_t k = 0; k < nm; ++k) REQUIRE(rho[k] && ux[k] && uy[k], "null field pointer");
  for (auto *m : b->members) {
    int rc = ensure_stage(m);
    if (rc != LBM_OK) return rc;
  }
  std::vector<size_t> ends(nm);
  for (size_t k = 0; k < nm; ++k) ends[k] = k + 1;  // one copy group per member
  auto fields = [&](size_t k, const double *&r, const double *&u, const double *&v) {
    const size_t n = (size_t)b->members[k]->L.g.nx * b->members[k]->L.g.ny;
    r = b->members[k]->stage;
    u = r + n;
    v = r + 2 * n;
  };
  auto upload = [&](size_t k) -> cudaError_t {
    auto *m = b->members[k];
    const size_t n = (size_t)m->L.g.nx * m->L.g.ny;
    cudaError_t e = cudaMemcpyAsync(m->stage, rho[k], n * sizeof(double),
                                    cudaMemcpyHostToDevice, b->io);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->stage + n, ux[k], n * sizeof(double), cudaMemcpyHostToDevice, b->io);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->stage + 2 * n, uy[k], n * sizeof(double), cudaMemcpyHostToDevice,
                          b->io);
    return e;
  };
  return batch_init_common(b, ends, upload, fields);
}

int lbm_batch_moments(lbm_batch b, double *const *rho, double *const *ux, double *const *uy) {
  REQUIRE(b != nullptr && rho && ux && uy, "null argument");
  DevGuard g(b->device);
  const size_t nm = b->members.size();
  for (size_t k = 0; k < nm; ++k) REQUIRE(rho[k] && ux[k] && uy[k], "null output pointer");
  for (auto *m : b->members) {
    int rc = ensure_stage(m);
    if (rc != LBM_OK) return rc;
  }
  std::vector<size_t> ends(nm);
  for (size_t k = 0; k < nm; ++k) ends[k] = k + 1;
  auto fields = [&](size_t k, double *&r, double *&u, double *&v) {
    const size_t n = (size_t)b->members[k]->L.g.nx * b->members[k]->L.g.ny;
    r = b->members[k]->stage;
    u = r + n;
    v = r + 2 * n;
  };
  auto download = [&](size_t k) -> cudaError_t {
    auto *m = b->members[k];
    const size_t n = (size_t)m->L.g.nx * m->L.g.ny;
    cudaError_t e = cudaMemcpyAsync(rho[k], m->stage, n * sizeof(double),
                                    cudaMemcpyDeviceToHost, b->io);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ux[k], m->stage + n, n * sizeof(double), cudaMemcpyDeviceToHost, b->io);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(uy[k], m->stage + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                          b->io);
    return e;
  };
  return batch_moments_common(b, ends, download, fields);
}

int lbm_batch_size(lbm_batch b, int *members, long long *nodes) {
  REQUIRE(b != nullptr, "null batch");
  if (members) *members = (int)b->members.size();
  if (nodes) *nodes = b->nodes;
  return LBM_OK;
}

int lbm_batch_init_packed(lbm_batch b, const double *rho, const double *ux, const double *uy) {
  REQUIRE(b != nullptr && rho && ux && uy, "null argument");
  REQUIRE(!b->spent, "batch ran a ragged generation; create a new batch");
  DevGuard g(b->device);
  int rc = ensure_packed(b);
  if (rc != LBM_OK) return rc;
  const size_t T = (size_t)b->nodes;
  const std::vector<size_t> ends = packed_groups(b);
  auto fields = [&](size_t k, const double *&r, const double *&u, const double *&v) {
    r = b->pstage + b->poff[k];
    u = r + T;
    v = r + 2 * T;
  };
  auto upload = [&](size_t gi) -> cudaError_t {
    const size_t k0 = gi == 0 ? 0 : ends[gi - 1];
    const size_t o = b->poff[k0], cnt = b->poff[ends[gi]] - o;
    cudaError_t e = cudaSuccess;
    const double *src[3] = {rho, ux, uy};
    for (int c = 0; c < 3 && e == cudaSuccess; ++c)
      e = cudaMemcpyAsync(b->pstage + c * T + o, src[c] + o, cnt * sizeof(double),
                          cudaMemcpyHostToDevice, b->io);
    return e;
  };
  return batch_init_common(b, ends, upload, fields);
}

int lbm_batch_moments_packed(lbm_batch b, double *rho, double *ux, double *uy) {
  REQUIRE(b != nullptr && rho && ux && uy, "null argument");
  DevGuard g(b->device);
  int rc = ensure_packed(b);
  if (rc != LBM_OK) return rc;
  const size_t T = (size_t)b->nodes;
  const std::vector<size_t> ends = packed_groups(b);
  auto fields = [&](size_t k, double *&r, double *&u, double *&v) {
    r = b->pstage + b->poff[k];
    u = r + T;
    v = r + 2 * T;
  };
  auto download = [&](size_t gi) -> cudaError_t {
    const size_t k0 = gi == 0 ? 0 : ends[gi - 1];
    const size_t o = b->poff[k0], cnt = b->poff[ends[gi]] - o;
    cudaError_t e = cudaSuccess;
    double *dst[3] = {rho, ux, uy};
    for (int c = 0; c < 3 && e == cudaSuccess; ++c)
      e = cudaMemcpyAsync(dst[c] + o, b->pstage + c * T + o, cnt * sizeof(double),
                          cudaMemcpyDeviceToHost, b->io);
    return e;
  };
  return batch_moments_common(b, ends, download, fields);
}

// Set up the two solve slots, the copy streams and the invalid-field
// counters on first use.
static int ensure_solve(lbm_batch_ctx *b) {
  if (b->up) return LBM_OK;
  const size_t T = (size_t)b->nodes, nm = b->members.size();
  ensure_poff(b);  // member offsets of the packed arrays
  for (auto &sl : b->slot) {
    sl.in = (double *)dev_alloc(3 * T * sizeof(double));
    sl.out = (double *)dev_alloc(3 * T * sizeof(double));
    sl.dout = (double *)dev_alloc(4 * nm * sizeof(double));
    if (cudaHostAlloc(&sl.hdrift, 4 * nm * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      sl.hdrift = nullptr;
    }
    if (!sl.in || !sl.out || !sl.dout || !sl.hdrift) {
      set_error("out of device memory for the pipelined solve staging");
      return LBM_ENOMEM;
    }
  }
  for (auto &r : b->ring)
    for (auto &e : r) CK(cudaEventCreate(&e));
  b->sbad = (unsigned int *)dev_alloc(2 * nm * sizeof(unsigned int));
  if (!b->sbad) {
    set_error("out of device memory for the solve counters");
    return LBM_ENOMEM;
  }
  // blocks of kIoBlockNodes nodes of one member each, and the members'
  // packed offsets, for the one-launch init and moments
  std::vector<IoBlock> blk;
  for (size_t k = 0; k < nm; ++k) {
    const long long n = (long long)b->members[k]->L.g.nx * b->members[k]->L.g.ny;
    for (long long s0 = 0; s0 < n; s0 += kIoBlockNodes) {
      IoBlock io;
      io.member = (int)k;
      io.count = (int)std::min<long long>(kIoBlockNodes, n - s0);
      io.start = s0;
      blk.push_back(io);
    }
  }
  std::vector<long long> po(b->poff.begin(), b->poff.end());
  b->ioblk = (IoBlock *)dev_alloc(blk.size() * sizeof(IoBlock));
  b->poff_dev = (long long *)dev_alloc(po.size() * sizeof(long long));
  if (!b->ioblk || !b->poff_dev) {
    set_error("out of device memory for the solve tables");
    return LBM_ENOMEM;
  }
  b->nioblk = (long long)blk.size();
  CK(cudaMemcpyAsync(b->ioblk, blk.data(), blk.size() * sizeof(IoBlock), cudaMemcpyHostToDevice,
                     b->stream));
  CK(cudaMemcpyAsync(b->poff_dev, po.data(), po.size() * sizeof(long long),
                     cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemsetAsync(b->sbad, 0, 2 * nm * sizeof(unsigned int), b->stream));
  // FP16 members: their scale tables (entry pointers into the groups'
  // device entry arrays; a point source's amplitude as the floor)
  std::vector<BatchEntry *> ent(nm, nullptr);
  std::vector<double> floor_(nm, 0.0);
  for (size_t k = 0; k < nm; ++k) {
    auto *m = b->members[k];
    if (m->L.dtype != LBM_F16DEV) continue;
    b->has16 = true;
    ent[k] = b->groups[b->member_group[k]].ents + b->member_local[k];
    floor_[k] = source_maxdev(m);
  }
  if (b->has16) {
    b->smax = (unsigned int *)dev_alloc(nm * sizeof(unsigned int));
    b->sfloor = (double *)dev_alloc(nm * sizeof(double));
    b->sscale = (double *)dev_alloc(nm * sizeof(double));
    b->sent = (BatchEntry **)dev_alloc(nm * sizeof(BatchEntry *));
    if (!b->smax || !b->sfloor || !b->sscale || !b->sent) {
      set_error("out of device memory for the FP16 scale tables");
      return LBM_ENOMEM;
    }
    CK(cudaMemcpyAsync(b->sfloor, floor_.data(), nm * sizeof(double), cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaMemcpyAsync(b->sent, ent.data(), nm * sizeof(BatchEntry *), cudaMemcpyHostToDevice,
                       b->stream));
  }
  CK(cudaStreamSynchronize(b->stream));
  cudaStream_t up = nullptr, down = nullptr;
  CK(cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking));
  if (cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking) != cudaSuccess) {
    cudaStreamDestroy(up);
    set_error("cannot create the download stream");
    cudaGetLastError();
    return LBM_ECUDA;
  }
  b->up = up;
  b->down = down;
  return LBM_OK;
}

int lbm_batch_solve_packed(lbm_batch b, long n, const double *rho_in, const double *ux_in,
                           const double *uy_in, double *rho_out, double *ux_out, double *uy_out,
                           double *drift_out) {
  NvtxRange nvtx("lbm_batch_solve_packed");
  REQUIRE(b != nullptr && rho_in && ux_in && uy_in && rho_out && ux_out && uy_out,
          "null argument");
  REQUIRE(n >= 0, "negative step count");
  REQUIRE(!b->spent, "batch ran a ragged generation; create a new batch");
  DevGuard g(b->device);
  int rc = ensure_solve(b);
  if (rc != LBM_OK) return rc;
  using B = lbm_batch_ctx;
  const size_t T = (size_t)b->nodes, nm = b->members.size();
  const int si = (int)(b->solves & 1);
  B::Slot &sl = b->slot[si];
  cudaEvent_t *ev = b->ring[b->solves % B::kRing];
  const cudaEvent_t *back2 = b->ring[(b->solves + B::kRing - 2) % B::kRing];
  const bool reuse = b->solves >= 2;  // the slot was used by solve - 2
  // upload, once the solve two back has initialised from this slot
  if (reuse) CK(cudaStreamWaitEvent(b->up, back2[B::E_INIT], 0));
  CK(cudaEventRecord(ev[B::E_UP0], b->up));
  const double *src[3] = {rho_in, ux_in, uy_in};
  for (int c = 0; c < 3; ++c)
    CK(cudaMemcpyAsync(sl.in + c * T, src[c], T * sizeof(double), cudaMemcpyHostToDevice,
                       b->up));
  CK(cudaEventRecord(ev[B::E_UP1], b->up));
  // equilibrium init of every member from the staged fields (FP16 members
  // first choose their storage scale from them, on the device)
  CK(cudaStreamWaitEvent(b->stream, ev[B::E_UP1], 0));
  CK(cudaEventRecord(ev[B::E_B0], b->stream));
  if (b->has16)
    CK(launch_batch_fp16_scales(b->views[0], b->views[1], b->sent, b->ioblk, b->nioblk,
                                b->poff_dev, (long long)T, sl.in, b->smax, b->sfloor, b->sscale,
                                (int)nm, b->stream));
  CK(launch_batch_init_dev(b->views[b->parity], b->ioblk, b->nioblk, b->poff_dev, (long long)T,
                           sl.in, b->sbad, (int)nm, b->stream));
  CK(launch_add_u32(b->sbad + nm, b->sbad, (int)nm, b->stream));
  for (auto *m : b->members) m->t = 0;
  CK(cudaEventRecord(ev[B::E_INIT], b->stream));
  rc = lbm_batch_step(b, n);
  if (rc != LBM_OK) return rc;
  CK(cudaEventRecord(ev[B::E_STEP], b->stream));
  CK(launch_batch_drift(b->views[b->parity], (int)nm, b->dpart, sl.dout, b->stream));
  CK(cudaEventRecord(ev[B::E_DRIFT], b->stream));
  // moments into this slot's output staging, once the solve two back has
  // downloaded from it
  if (reuse) CK(cudaStreamWaitEvent(b->stream, back2[B::E_DN1], 0));
  CK(launch_batch_moments_dev(b->views[b->parity], b->ioblk, b->nioblk, b->poff_dev,
                              (long long)T, sl.out, (int)nm, b->stream));
  CK(cudaEventRecord(ev[B::E_MOM], b->stream));
  // download
  CK(cudaStreamWaitEvent(b->down, ev[B::E_MOM], 0));
  CK(cudaEventRecord(ev[B::E_DN0], b->down));
  double *dst[3] = {rho_out, ux_out, uy_out};
  for (int c = 0; c < 3; ++c)
    CK(cudaMemcpyAsync(dst[c], sl.out + c * T, T * sizeof(double), cudaMemcpyDeviceToHost,
                       b->down));
  if (drift_out) {
    CK(cudaMemcpyAsync(sl.hdrift, sl.dout, 4 * nm * sizeof(double), cudaMemcpyDeviceToHost,
                       b->down));
    // the host runs ahead of the device by several solves, so each call
    // gets its own payload (freed by the host function); the page-locked
    // array itself is reused only after this stream has passed the host
    // function of the solve two back
    auto *dc = new (std::nothrow) lbm_batch_ctx::DriftOut();
    if (!dc) {
      set_error("out of host memory");
      return LBM_ENOMEM;
    }
    dc->dst = drift_out;
    dc->src = sl.hdrift;
    dc->bytes = 4 * nm * sizeof(double);
    cudaError_t e = cudaLaunchHostFunc(
        b->down,
        [](void *p) {
          auto *d = static_cast<lbm_batch_ctx::DriftOut *>(p);
          memcpy(d->dst, d->src, d->bytes);
          delete d;
        },
        dc);
    if (e != cudaSuccess) {
      delete dc;
      CK(e);
    }
    b->pending_drift.push_back(drift_out);
  }
  CK(cudaEventRecord(ev[B::E_DN1], b->down));
  sl.used = true;
  b->last_slot = si;
  ++b->solves;
  return LBM_OK;
}

int lbm_batch_wait(lbm_batch b, double *phase_ms) {
  REQUIRE(b != nullptr, "null batch");
  DevGuard g(b->device);
  if (b->up) {
    CK(cudaStreamSynchronize(b->up));
    CK(cudaStreamSynchronize(b->stream));
    CK(cudaStreamSynchronize(b->down));
  }
  if (phase_ms) {
    for (int k = 0; k < 6; ++k) phase_ms[k] = 0.0;
    if (b->last_slot >= 0) {
      using B = lbm_batch_ctx;
      const int pairs[6][2] = {{B::E_UP0, B::E_UP1},   {B::E_B0, B::E_INIT},
                               {B::E_INIT, B::E_STEP}, {B::E_STEP, B::E_DRIFT},
                               {B::E_DRIFT, B::E_MOM}, {B::E_DN0, B::E_DN1}};
      // the median over the solves since the previous wait that are still
      // in the event ring (the last one alone when no new solve was queued)
      const long long last = b->solves - 1;
      long long first = std::max(b->waited, b->solves - (long long)B::kRing);
      if (first > last) first = last;
      for (int k = 0; k < 6; ++k) {
        std::vector<double> t;
        for (long long s = first; s <= last; ++s) {
          float ms = 0.0f;
          CK(cudaEventElapsedTime(&ms, b->ring[s % B::kRing][pairs[k][0]],
                                  b->ring[s % B::kRing][pairs[k][1]]));
          t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        const size_t m = t.size();
        phase_ms[k] = m % 2 ? t[m / 2] : 0.5 * (t[m / 2 - 1] + t[m / 2]);
      }
    }
  }
  const size_t nm = b->members.size();
  int rc = LBM_OK;
  if (b->has16 && b->solves > b->waited) {
    // the host copies of the FP16 members' scales follow the last solve's
    std::vector<double> sc(nm, 1.0);
    CK(cudaMemcpy(sc.data(), b->sscale, nm * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < nm; ++k)
      if (b->members[k]->L.dtype == LBM_F16DEV) set_scale(b->members[k], sc[k]);
  }
  if (b->sbad) {
    std::vector<unsigned int> tot(nm, 0);
    CK(cudaMemcpy(tot.data(), b->sbad + nm, nm * sizeof(unsigned int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(b->sbad + nm, 0, nm * sizeof(unsigned int)));
    for (size_t j = 0; j < nm; ++j)
      if (tot[j]) {
        set_error("member " + std::to_string(j) + ": " + std::to_string(tot[j]) +
                  " nodes with non-finite fields or rho <= 0 over the solves since the last wait");
        rc = LBM_EINVAL;
        break;
      }
  }
  if (rc == LBM_OK)
    for (double *d : b->pending_drift)
      for (size_t k = 0; k < nm && rc == LBM_OK; ++k)
        if (d[4 * k + 3] > 0) {
          set_error("member " + std::to_string(k) + " holds non-finite populations");
          rc = LBM_EUNSTABLE;
        }
  b->pending_drift.clear();
  b->waited = b->solves;
  return rc;
}

int lbm_get_variant(lbm_handle h, int *variant) {
  REQUIRE(h != nullptr && variant != nullptr, "null argument");
  *variant = h->L.dtype == LBM_F64 ? 0 : (h->tuned ? h->L.variant : -1);
  return LBM_OK;
}

int lbm_batch_resident(lbm_batch b, int *flags) {
  REQUIRE(b != nullptr && flags != nullptr, "null argument");
  for (size_t k = 0; k < b->members.size(); ++k) flags[k] = b->member_res[k];
  return LBM_OK;
}

int lbm_batch_const_table(lbm_batch b, int *flags) {
  REQUIRE(b != nullptr && flags != nullptr, "null argument");
  for (size_t k = 0; k < b->members.size(); ++k)
    flags[k] = b->groups[b->member_group[k]].pbase >= 0 ? 1 : 0;
  return LBM_OK;
}

int lbm_batch_get_variant(lbm_batch b, int *variant) {
  REQUIRE(b != nullptr && variant != nullptr, "null argument");
  *variant = b->tuned ? b->variant : -1;
  return LBM_OK;
}

int lbm_batch_set_variant(lbm_batch b, int variant) {
  REQUIRE(b != nullptr, "null batch");
  REQUIRE(variant >= 0 && variant < kBatchVariants, "no such launch variant");
  batch_pin_variant(b, variant);
  return LBM_OK;
}

int lbm_batch_tune(lbm_batch b, double *times_ms, int *chosen) {
  REQUIRE(b != nullptr, "null batch");
  DevGuard g(b->device);
  int rc = tune_batch(b, times_ms);
  if (rc == LBM_OK && chosen) *chosen = b->variant;
  return rc;
}

int lbm_batch_drift(lbm_batch b, double *out) {
  NvtxRange nvtx("lbm_batch_drift");
  REQUIRE(b != nullptr && out != nullptr, "null argument");
  REQUIRE(!b->spent, "batch ran a ragged generation; use lbm_drift per member");
  DevGuard g(b->device);
  const int n = (int)b->members.size();
  CK(launch_batch_drift(b->views[b->parity], n, b->dpart, b->dout, b->stream));
  CK(cudaMemcpyAsync(out, b->dout, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  for (int k = 0; k < n; ++k)
    if (out[4 * k + 3] > 0) return LBM_EUNSTABLE;
  return LBM_OK;
}

int lbm_batch_destroy(lbm_batch b) {
  if (!b) return LBM_EINVAL;
  DevGuard g(b->device);
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  return LBM_OK;
}

}  // extern "C"
