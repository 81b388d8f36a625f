// Continuous-batching server for lattice solves (lbm_server_* / lbm_submit /
// lbm_poll in include/lbm.h).
//
// One scheduler thread per server owns the device work.  Each loop it
//   1. admits queued requests -- in arrival order (LBM_SERVE_FIFO) or
//      smallest remaining work first (LBM_SERVE_SHORTEST) -- while the
//      device bytes of the resident lattices plus the request fit in the
//      budget and, if a cap is set, their nodes fit in the resident-node cap
//      (create + initialise on the device);
//   2. steps every resident lattice together for one "generation" of up to
//      chunk_steps steps: one batched launch per step and storage type, in
//      which each lattice takes part until its own step count is reached;
//   3. retires the lattices that are done: moments to host, memory freed,
//      latency stamped.
// Requests that arrive while a generation runs join at the next one, so
// work of different requests overlaps on the device while memory allows.
// Every lattice advances with exactly the arithmetic of a standalone
// handle (same kernel body, same per-lattice parameters), so a result does
// not depend on what else was in the mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum State { QUEUED, RUNNING, DONE, FAILED };

struct Req {
  long long id;
  lbm_request r;
  std::vector<double> fields;  // LBM_INIT_FIELDS: rho, ux, uy copied at submit
  double t_submit = 0, latency = 0;
  State state = QUEUED;
  int err = LBM_OK;
  lbm_handle h = nullptr;
  long remaining = 0;
  size_t bytes = 0;
  std::vector<double> rho, ux, uy;
};

// device bytes of a request's lattice: two population buffers laid out as
// lbm_create lays them out, plus the per-lattice scratch
size_t estimate_bytes(const lbm_request &r) {
  const int esize = r.dtype == LBM_F32DEV ? 4 : 2;
  const Geom g = make_geom(r.nx, r.ny, vec_nodes(r.dtype), esize);
  return 2 * (size_t)g.pitch * (size_t)r.ny * 9 * esize + 64 * 1024;
}

}  // namespace

struct lbm_server_ctx {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req *> queue;
  std::unordered_map<long long, Req *> all;
  std::vector<Req *> running;
  size_t budget = 0, resident_bytes = 0;
  long chunk = 100;
  int device = 0;
  bool stop = false;
  long long next_id = 1;
  std::thread worker;
  cudaStream_t stream = nullptr;
  double *stage = nullptr;  // 3 * max nodes doubles, for fields in and moments out
  size_t stage_nodes = 0;
  lbm_server_stats_t st{};
  int variant = -1;  // step launch variant, tuned on the first large generation
  int policy = LBM_SERVE_FIFO;
  long long max_nodes = 0;  // resident-node cap (0: bytes only)
  long long resident_nodes = 0;
  std::deque<long long> done_ids;  // finished since the last lbm_server_done
};

static int ensure_server_stage(lbm_server_ctx *s, size_t nodes) {
  if (nodes <= s->stage_nodes) return LBM_OK;
  dev_free(s->stage);
  s->stage = (double *)dev_alloc(3 * nodes * sizeof(double));
  s->stage_nodes = s->stage ? nodes : 0;
  return s->stage ? LBM_OK : LBM_ENOMEM;
}

static int admit_one(lbm_server_ctx *s, Req *q) {
  const lbm_request &r = q->r;
  int rc = lbm_create(r.nx, r.ny, r.S, r.rho0, r.u0, r.dtype, &q->h);
  if (rc != LBM_OK) return rc;
  lbm_set_stream(q->h, s->stream);
  if (r.init_kind == LBM_INIT_FIELDS) {
    const size_t n = (size_t)r.nx * r.ny;
    rc = ensure_server_stage(s, n);
    if (rc != LBM_OK) return rc;
    if (cudaMemcpyAsync(s->stage, q->fields.data(), 3 * n * sizeof(double),
                        cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
      cudaGetLastError();
      return LBM_ECUDA;
    }
    rc = lbm_init_field_dev(q->h, s->stage, s->stage + n, s->stage + 2 * n);
    q->fields.clear();
    q->fields.shrink_to_fit();
  } else {
    rc = lbm_init_analytic(q->h, r.init_kind, r.init_params);
  }
  if (rc != LBM_OK) return rc;
  lbm_info_t info;
  lbm_info(q->h, &info);
  q->bytes = info.device_bytes;
  q->remaining = r.steps;
  return LBM_OK;
}

static int retire_one(lbm_server_ctx *s, Req *q) {
  const size_t n = (size_t)q->r.nx * q->r.ny;
  int rc = ensure_server_stage(s, n);
  if (rc != LBM_OK) return rc;
  rc = lbm_moments_dev(q->h, s->stage, s->stage + n, s->stage + 2 * n);
  if (rc != LBM_OK) return rc;
  q->rho.resize(n);
  q->ux.resize(n);
  q->uy.resize(n);
  if (cudaMemcpyAsync(q->rho.data(), s->stage, n * sizeof(double), cudaMemcpyDeviceToHost,
                      s->stream) != cudaSuccess ||
      cudaMemcpyAsync(q->ux.data(), s->stage + n, n * sizeof(double), cudaMemcpyDeviceToHost,
                      s->stream) != cudaSuccess ||
      cudaMemcpyAsync(q->uy.data(), s->stage + 2 * n, n * sizeof(double),
                      cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess) {
    cudaGetLastError();
    return LBM_ECUDA;
  }
  return LBM_OK;
}

static void finish(lbm_server_ctx *s, Req *q, int err) {
  // called with s->mu held
  if (q->h) {
    lbm_destroy(q->h);
    q->h = nullptr;
  }
  if (q->state == RUNNING) {
    s->resident_bytes -= q->bytes;
    s->resident_nodes -= (long long)q->r.nx * q->r.ny;
  }
  q->state = err == LBM_OK ? DONE : FAILED;
  q->err = err;
  q->latency = now_s() - q->t_submit;
  s->done_ids.push_back(q->id);
  if (err == LBM_OK)
    s->st.completed++;
  else
    s->st.failed++;
}

static void worker_loop(lbm_server_ctx *s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Req *> fresh;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stop || !s->queue.empty() || !s->running.empty(); });
      if (s->stop && s->queue.empty() && s->running.empty()) return;
      while (!s->queue.empty()) {
        auto pick = s->queue.begin();
        if (s->policy == LBM_SERVE_SHORTEST)
          pick = std::min_element(s->queue.begin(), s->queue.end(), [](Req *a, Req *b) {
            return (double)a->r.nx * a->r.ny * a->r.steps < (double)b->r.nx * b->r.ny * b->r.steps;
          });
        Req *q = *pick;
        const size_t need = estimate_bytes(q->r);
        const long long nodes = (long long)q->r.nx * q->r.ny;
        if (s->resident_bytes + need > s->budget) break;
        if (s->max_nodes > 0 && s->resident_nodes > 0 && s->resident_nodes + nodes > s->max_nodes)
          break;
        s->queue.erase(pick);
        q->state = RUNNING;
        q->bytes = need;
        s->resident_bytes += need;
        s->resident_nodes += nodes;
        fresh.push_back(q);
      }
    }
    // create and initialise outside the lock (device work)
    for (Req *q : fresh) {
      int rc = admit_one(s, q);
      std::lock_guard<std::mutex> lk(s->mu);
      if (rc != LBM_OK) {
        finish(s, q, rc);
        continue;
      }
      // the reservation was an estimate: keep the true footprint
      s->resident_bytes += q->bytes;
      s->resident_bytes -= estimate_bytes(q->r);
      s->running.push_back(q);
      s->st.admitted++;
    }
    std::vector<Req *> run;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      run = s->running;
      s->st.resident = (int)run.size();
      if (s->st.resident > s->st.peak_resident) s->st.peak_resident = s->st.resident;
      if (s->resident_bytes > s->st.peak_bytes) s->st.peak_bytes = s->resident_bytes;
      s->st.resident_bytes = s->resident_bytes;
    }
    if (run.empty()) continue;
    // a generation lasts up to chunk steps; each lattice stops at its own count
    long n = 0;
    for (Req *q : run) n = std::max(n, q->remaining);
    n = std::min(n, s->chunk);
    std::vector<long> take(run.size());
    for (size_t k = 0; k < run.size(); ++k) take[k] = std::min(run[k]->remaining, n);
    const double t0 = now_s();
    int rc = LBM_OK;
    if (n > 0) {
      lbm::NvtxRange nvtx("serve generation");
      std::vector<lbm_handle> hs;
      for (Req *q : run) hs.push_back(q->h);
      lbm_batch b = nullptr;
      rc = lbm_batch_create((int)hs.size(), hs.data(), &b);
      if (rc == LBM_OK) {
        // tune once, on the first generation whose populations exceed the
        // L2 (2^24 nodes: >= 0.6 GB in 16-bit storage), and keep that choice
        // for every later generation; smaller generations run the default
        // variant (a tuning run that fits in L2 ranks the variants by their
        // cache-resident speed, which is not the HBM-bound speed that the
        // large generations need)
        if (s->variant >= 0) batch_pin_variant(b, s->variant);
        else if (batch_nodes(b) < (1LL << 24)) batch_pin_variant(b, kStepVariants - 1);
        rc = batch_step_ragged(b, take.data(), n);
        if (s->variant < 0 && batch_nodes(b) >= (1LL << 24)) {
          s->variant = batch_variant(b);
          std::lock_guard<std::mutex> lk(s->mu);
          s->st.variant = s->variant;
        }
        lbm_batch_destroy(b);
      }
    }
    double lu = 0;
    for (size_t k = 0; k < run.size(); ++k) lu += (double)run[k]->r.nx * run[k]->r.ny * take[k];
    // retire finished lattices (moments to host)
    std::vector<std::pair<Req *, int>> done;
    for (size_t k = 0; k < run.size(); ++k) {
      Req *q = run[k];
      if (rc != LBM_OK) {
        done.push_back({q, rc});
        continue;
      }
      q->remaining -= take[k];
      if (q->remaining <= 0) done.push_back({q, retire_one(s, q)});
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) cudaGetLastError();
    const double t1 = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.generations++;
    s->st.lattice_updates += lu;
    s->st.busy_s += t1 - t0;
    for (auto &d : done) {
      finish(s, d.first, d.second);
      s->running.erase(std::find(s->running.begin(), s->running.end(), d.first));
    }
    s->st.resident = (int)s->running.size();
    s->st.resident_bytes = s->resident_bytes;
  }
}

extern "C" {

int lbm_server_create(size_t hbm_budget_bytes, long chunk_steps, lbm_server *out) {
  if (!out || hbm_budget_bytes == 0 || chunk_steps < 1) {
    set_error("bad server arguments");
    return LBM_EINVAL;
  }
  lbm_server_ctx *s = new (std::nothrow) lbm_server_ctx();
  if (!s) return LBM_ENOMEM;
  s->budget = hbm_budget_bytes;
  s->chunk = chunk_steps;
  s->st.variant = -1;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    set_error("no usable GPU for the server");
    return LBM_ECUDA;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return LBM_OK;
}

int lbm_server_set_policy(lbm_server s, int policy, long long max_resident_nodes) {
  if (!s || (policy != LBM_SERVE_FIFO && policy != LBM_SERVE_SHORTEST) ||
      max_resident_nodes < 0) {
    set_error("bad server policy");
    return LBM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->policy = policy;
  s->max_nodes = max_resident_nodes;
  return LBM_OK;
}

int lbm_submit(lbm_server s, const lbm_request *req, long long *id) {
  if (!s || !req || !id) {
    set_error("null argument");
    return LBM_EINVAL;
  }
  const lbm_request &r = *req;
  if (r.nx < 2 || r.ny < 2 || r.steps < 0 || r.rho0 <= 0 ||
      (r.dtype != LBM_F32DEV && r.dtype != LBM_F16DEV && r.dtype != LBM_BF16DEV) ||
      (r.init_kind != LBM_INIT_FIELDS && r.init_kind != LBM_INIT_GAUSSIAN &&
       r.init_kind != LBM_INIT_PLANE) ||
      (r.init_kind == LBM_INIT_FIELDS && (!r.rho || !r.ux || !r.uy))) {
    set_error("invalid request");
    return LBM_EINVAL;
  }
  if (estimate_bytes(r) > s->budget) {
    set_error("request alone exceeds the HBM budget");
    return LBM_ENOMEM;
  }
  Req *q = new (std::nothrow) Req();
  if (!q) return LBM_ENOMEM;
  q->r = r;
  if (r.init_kind == LBM_INIT_FIELDS) {
    const size_t n = (size_t)r.nx * r.ny;
    q->fields.resize(3 * n);
    memcpy(q->fields.data(), r.rho, n * sizeof(double));
    memcpy(q->fields.data() + n, r.ux, n * sizeof(double));
    memcpy(q->fields.data() + 2 * n, r.uy, n * sizeof(double));
  }
  q->r.rho = q->r.ux = q->r.uy = nullptr;
  q->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete q;
      set_error("server closed");
      return LBM_ECLOSED;
    }
    q->id = s->next_id++;
    s->all[q->id] = q;
    s->queue.push_back(q);
    s->st.submitted++;
    *id = q->id;
  }
  s->cv.notify_one();
  return LBM_OK;
}

int lbm_poll(lbm_server s, long long id, double *rho, double *ux, double *uy,
             double *latency_s) {
  if (!s) return LBM_EINVAL;
  Req *q = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return LBM_ENOTFOUND;
    q = it->second;
    if (q->state == QUEUED || q->state == RUNNING) return LBM_PENDING;
    s->all.erase(it);
  }
  const size_t n = (size_t)q->r.nx * q->r.ny;
  int rc = q->state == DONE ? LBM_OK : q->err;
  if (rc == LBM_OK) {
    if (rho) memcpy(rho, q->rho.data(), n * sizeof(double));
    if (ux) memcpy(ux, q->ux.data(), n * sizeof(double));
    if (uy) memcpy(uy, q->uy.data(), n * sizeof(double));
  }
  if (latency_s) *latency_s = q->latency;
  delete q;
  return rc;
}

int lbm_server_done(lbm_server s, long long *ids, int cap, int *count) {
  if (!s || !count || cap < 0 || (cap > 0 && !ids)) {
    set_error("bad lbm_server_done arguments");
    return LBM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0;
  while (n < cap && !s->done_ids.empty()) {
    ids[n++] = s->done_ids.front();
    s->done_ids.pop_front();
  }
  *count = n;
  return LBM_OK;
}

int lbm_server_stats(lbm_server s, lbm_server_stats_t *out) {
  if (!s || !out) return LBM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  return LBM_OK;
}

int lbm_server_destroy(lbm_server s) {
  if (!s) return LBM_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // requests never admitted are dropped
    for (Req *q : s->queue) {
      q->state = FAILED;
      q->err = LBM_ECLOSED;
    }
    s->queue.clear();
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto &kv : s->all) delete kv.second;
  dev_free(s->stage);
  if (s->stream) cudaStreamDestroy(s->stream);
  cudaGetLastError();
  delete s;
  return LBM_OK;
}

}  // extern "C"
