// server.cu — serving alignment requests: continuous admission into slots whose work overlaps
// on the device.
//
// A server has max_slots slots.  Each slot is a worker thread with a CUDA stream of its own
// and a workspace (a grid object holding only evaluation buffers).  A free slot admits the
// request at the head of the queue (first come, first served) as soon as the device-memory
// budget allows, binds its workspace to the request's resident reference (the reference's
// device arrays are shared, not copied) and runs the request's whole coarse-to-fine lattice
// search on its stream, every level built on the device from the previous level's argmax
// (the pipeline of align_search_ex, so a request has no host round trip between levels).
// Requests that arrive while others run are admitted as slots and memory free up; the
// launches of all active requests interleave on the device (one stream per slot), so each
// request's host work and the tails of its launches overlap with the others' kernels.  A
// request's result is bit-identical to align_search_ex on its reference alone.
//
// Memory: the budget covers the references and every slot's workspace, which keeps the
// buffers of the largest request it has run (re-allocating between requests would
// synchronise the device under the other slots' work).  When the request at the head of
// the queue fits only without them and nothing runs, idle slots release their workspaces.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "align.h"
#include "align_internal.h"
#include "runtime_internal.h"

using namespace mialign;

namespace {

struct Req {
  uint64_t ticket = 0;
  int32_t ref = 0;
  std::vector<float> xyz;  // host copy
  int64_t nB = 0;
  double c[6], r[6];
  int32_t counts[6];
  int32_t levels = 0;
  size_t bytes = 0;        // device memory estimate of its workspace
  int32_t spill_np = 0;    // key partitions its spill queues serve (0: none; counted in bytes)
  double T[6] = {0, 0, 0, 0, 0, 0};
  float best_mi = 0.0f;
  int32_t status = ALIGN_OK;
  double t_submit = 0, t_start = 0, t_done = 0;
};

struct Ref {
  align_grid* grid = nullptr;
  size_t bytes = 0;
};

struct Slot {
  align_grid* ws = nullptr;      // workspace bound to one reference at a time
  cudaStream_t stream = nullptr;
  size_t held = 0;               // device bytes its workspace may hold (estimate)
  bool busy = false;
  Req* cur = nullptr;
};

int64_t lattice_size(const int32_t m[6]) {
  int64_t P = 1;
  for (int a = 0; a < 6; ++a) P *= m[a];
  return P;
}

}  // namespace

struct align_server {
  int device = 0;
  int n_sm = 0;
  size_t budget = 0;
  int32_t max_slots = 1;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;       // workers: new requests, freed memory or stop
  std::condition_variable cv_done;  // clients: a request finished
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, Req*> done;
  std::unordered_map<uint64_t, int> pending;  // ticket -> 1 while queued or active
  std::vector<Ref> refs;
  size_t ref_bytes = 0;
  std::vector<Slot> slots;
  int32_t n_active = 0;
  size_t peak = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  int64_t stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  size_t used() const {
    size_t u = ref_bytes;
    for (const Slot& sl : slots) u += sl.held;
    return u;
  }
};

namespace {

// Device bytes of a workspace running a request of nB points with lattice counts m on a grid
// whose single-pose table has T slots: the staged points, the pre-rotated tile copies, the
// per-pose buffers of one level, and the per-CTA 64-bit side sums and overflow lists.
size_t request_bytes(int64_t nB, const int32_t m[6], int K, int T, int n_sm, int spill_np) {
  const int64_t P = lattice_size(m);
  const int64_t n_pad = std::max<int64_t>(3, (nB + 1023) / 1024) * 1024;
  int64_t n_rot = (int64_t)m[3] * m[4] * m[5];
  if (n_rot > std::max<int64_t>(1, P / 4)) n_rot = 1;
  const int64_t per_pose = (int64_t)K * K * 4 + 24 + 4 + 48 + 4 + 4 + 4;
  const int64_t per_cta = 2 * (int64_t)T * 8 + (int64_t)eval_shape(0).ovf_cap() * 16;
  // spill queues: spill_np of n_pad runs per CTA (pose pairs'; single poses use half)
  const int64_t spill = spill_np > 1 ? (int64_t)spill_np * ((n_pad + 31) / 32 * 32) * 16 : 0;
  return (size_t)(nB * 12 + n_rot * n_pad * 16 + P * per_pose + (int64_t)n_sm * (per_cta + spill));
}

// A workspace: a grid object that owns only evaluation buffers; the reference arrays it
// reads are bound from a resident reference grid (and never released through it).
align_grid* workspace_create(int device, int n_sm, size_t smem_optin, cudaStream_t stream) {
  align_grid* g = new (std::nothrow) align_grid();
  if (!g) return nullptr;
  g->device = device;
  g->n_sm = n_sm;
  g->smem_optin = smem_optin;
  g->stream = stream;
  return g;
}

void workspace_bind(align_grid* ws, const align_grid* ref) {
  ws->gc = ref->gc;
  std::memcpy(ws->origin, ref->origin, sizeof(ws->origin));
  ws->res_m = ref->res_m;
  ws->V = ref->V;
  std::memcpy(ws->boxA, ref->boxA, sizeof(ws->boxA));
  ws->symA.p = ref->symA.p;  // borrowed
  ws->symA.cap = ref->symA.cap;
  ws->sat.p = ref->sat.p;    // borrowed
  ws->sat.cap = ref->sat.cap;
  ws->has_ref = ref->has_ref;
  ws->table_slots = ref->table_slots;
  for (int i = 0; i < kEvalShapes; ++i) {
    ws->passes_seed[i] = ref->passes_seed[i];
    ws->passes_seed_pair[i] = ref->passes_seed_pair[i];
  }
  ws->passes_seed_cluster = ref->passes_seed_cluster;
  ws->sweep_mode = ref->sweep_mode;
  ws->layout_min = ref->layout_min;
  ws->spill_on = ref->spill_on;
}

// Key partitions learned by a workspace go back to its reference (for the next request).
void workspace_learn(const align_grid* ws, align_grid* ref) {
  for (int i = 0; i < kEvalShapes; ++i) {
    ref->passes_seed[i] = std::max(ref->passes_seed[i], ws->passes_seed[i]);
    ref->passes_seed_pair[i] = std::max(ref->passes_seed_pair[i], ws->passes_seed_pair[i]);
  }
  ref->passes_seed_cluster = std::max(ref->passes_seed_cluster, ws->passes_seed_cluster);
  ref->layout_min = std::max(ref->layout_min, ws->layout_min);
}

void workspace_destroy(align_grid* ws) {
  if (!ws) return;
  ws->symA = DevBuf{};  // the reference's arrays: not ours to free
  ws->sat = DevBuf{};
  align_destroy_grid(ws);
}

// Admit the request at the head of the queue into idle slot k if the budget allows it.
Req* try_admit_locked(align_server* s, size_t k) {
  if (s->queue.empty()) return nullptr;
  Req* r = s->queue.front();
  Slot& me = s->slots[k];
  auto need = [&]() {
    size_t others = s->ref_bytes;
    for (size_t j = 0; j < s->slots.size(); ++j)
      if (j != k) others += s->slots[j].held;
    return others + std::max(me.held, r->bytes);
  };
  if (need() > s->budget) {
    if (s->n_active > 0) return nullptr;  // wait until running requests finish
    // nothing runs: the idle slots' workspaces give way (each fits the budget alone with
    // the references, as align_submit checked)
    for (size_t j = 0; j < s->slots.size(); ++j) {
      Slot& o = s->slots[j];
      if (j == k || o.held == 0 || o.ws == nullptr) continue;
      workspace_destroy(o.ws);
      o.ws = nullptr;
      o.held = 0;
    }
  }
  s->queue.pop_front();
  me.held = std::max(me.held, r->bytes);
  me.busy = true;
  me.cur = r;
  r->t_start = s->now();
  s->n_active += 1;
  s->peak = std::max(s->peak, s->used());
  s->stats[1] += 1;
  s->stats[3] = std::max<int64_t>(s->stats[3], (int64_t)s->n_active);
  s->stats[5] = (int64_t)s->used();
  s->stats[6] = (int64_t)s->peak;
  s->stats[7] = (int64_t)s->queue.size();
  return r;
}

void finish_locked(align_server* s, Req* r, int32_t status) {
  r->status = status;
  r->t_done = s->now();
  s->pending.erase(r->ticket);
  s->done[r->ticket] = r;
  s->stats[2] += 1;
  s->cv_done.notify_all();
}

void worker_main(align_server* s, size_t k) {
  cudaSetDevice(s->device);
  for (;;) {
    Req* r = nullptr;
    align_grid* ref = nullptr;
    align_grid* ws = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        r = try_admit_locked(s, k);
        if (r) break;
        s->cv.wait(lk);
      }
      Slot& me = s->slots[k];
      if (!me.ws) me.ws = workspace_create(s->device, s->n_sm, s->refs[0].grid->smem_optin, me.stream);
      ws = me.ws;
      ref = s->refs[(size_t)r->ref].grid;
      if (ws) {
        workspace_bind(ws, ref);
        ws->spill_on = r->spill_np > 0 ? 1 : 0;  // within the request's memory estimate
        ws->spill_np_max = std::max(2, r->spill_np);
      }
    }
    int32_t st = ALIGN_OK;
    float mi = 0.0f;
    if (!ws) {
      st = report_error(ALIGN_E_OOM, "host allocation failed");
    } else {
      st = align_search_ex(ws, r->nB > 0 ? r->xyz.data() : nullptr, r->nB, 0, r->c, r->r, r->counts, r->levels,
                           r->T, &mi, nullptr);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (ws) workspace_learn(ws, ref);
    r->best_mi = mi;
    if (st == ALIGN_OK) {
      s->stats[0] += r->levels;
      s->stats[4] += (int64_t)r->levels * lattice_size(r->counts);
    }
    Slot& me = s->slots[k];
    me.busy = false;
    me.cur = nullptr;
    s->n_active -= 1;
    finish_locked(s, r, st);
    s->cv.notify_all();  // a slot is free: any waiting worker may admit
  }
}

}  // namespace

extern "C" {

align_status align_server_create(size_t hbm_budget_bytes, int32_t max_slots, align_server** out) {
  if (!out) return report_error(ALIGN_E_INVALID, "out is NULL");
  *out = nullptr;
  if (max_slots < 1 || max_slots > 256) return report_error(ALIGN_E_INVALID, "max_slots must be in 1..256");
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return report_cuda_error(e, "device query");
  std::unique_ptr<align_server> s(new (std::nothrow) align_server());
  if (!s) return report_error(ALIGN_E_OOM, "host allocation failed");
  s->device = dev;
  s->n_sm = n_sm;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->t0 = std::chrono::steady_clock::now();
  s->slots.resize((size_t)max_slots);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      for (Slot& o : s->slots)
        if (o.stream) cudaStreamDestroy(o.stream);
      return report_error(ALIGN_E_CUDA, "creating the slots' streams failed");
    }
  }
  align_server* raw = s.release();
  try {
    for (size_t k = 0; k < raw->slots.size(); ++k) raw->workers.emplace_back(worker_main, raw, k);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(raw->mu);
      raw->stop = true;
      raw->cv.notify_all();
    }
    for (std::thread& t : raw->workers)
      if (t.joinable()) t.join();
    for (Slot& o : raw->slots) cudaStreamDestroy(o.stream);
    delete raw;
    return report_error(ALIGN_E_INTERNAL, "could not start the worker threads");
  }
  *out = raw;
  return ALIGN_OK;
}

align_status align_server_add_reference(align_server* s, const align_grid_desc* desc, const float* xyzA,
                                        int64_t nA, int32_t* ref_id) {
  if (!s || !ref_id) return report_error(ALIGN_E_INVALID, "NULL argument");
  GridConst gc;
  align_status st = check_grid_desc(desc, &gc);
  if (st != ALIGN_OK) return st;
  const int64_t V = (int64_t)gc.X * gc.Y * gc.Z;
  const size_t bytes = (size_t)V + (size_t)(gc.K - 1) * (gc.X + 1) * (gc.Y + 1) * (gc.Z + 1) * 4;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->used() + bytes > s->budget) return report_error(ALIGN_E_OOM, "reference does not fit the memory budget");
  }
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return report_cuda_error(e, "cudaSetDevice");
  align_grid* g = nullptr;
  st = align_create_grid(desc, nullptr, &g);
  if (st != ALIGN_OK) return st;
  st = align_set_reference(g, xyzA, nA, 0);
  if (st == ALIGN_OK) {
    e = cudaStreamSynchronize(g->stream);  // every slot's stream reads the arrays from now on
    if (e != cudaSuccess) st = report_cuda_error(e, "synchronize");
  }
  if (st != ALIGN_OK) {
    align_destroy_grid(g);
    return st;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->refs.push_back(Ref{g, bytes});
  s->ref_bytes += bytes;
  s->peak = std::max(s->peak, s->used());
  *ref_id = (int32_t)s->refs.size() - 1;
  return ALIGN_OK;
}

align_status align_submit(align_server* s, const align_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return report_error(ALIGN_E_INVALID, "NULL argument");
  if (req->nB < 0 || req->nB >= INT32_MAX) return report_error(ALIGN_E_INVALID, "nB out of range");
  if (req->nB > 0 && !req->xyzB) return report_error(ALIGN_E_INVALID, "xyzB is NULL");
  if (req->levels < 0) return report_error(ALIGN_E_INVALID, "levels < 0");
  std::unique_ptr<Req> r(new (std::nothrow) Req());
  if (!r) return report_error(ALIGN_E_OOM, "host allocation failed");
  static const int32_t kDefault[6] = {8, 8, 2, 2, 2, 8};
  bool zero = true;
  for (int a = 0; a < 6; ++a) zero = zero && req->counts[a] == 0;
  for (int a = 0; a < 6; ++a) {
    r->counts[a] = zero ? kDefault[a] : req->counts[a];
    if (r->counts[a] < 1) return report_error(ALIGN_E_INVALID, "counts must be >= 1");
    r->c[a] = req->init[a];
    r->r[a] = req->range[a];
    if (!std::isfinite(r->c[a]) || !std::isfinite(r->r[a]))
      return report_error(ALIGN_E_INVALID, "init and range must be finite");
  }
  if (lattice_size(r->counts) >= (1 << 26)) return report_error(ALIGN_E_INVALID, "lattice too large");
  r->levels = req->levels;
  r->nB = req->nB;
  if (req->nB > 0) r->xyz.assign(req->xyzB, req->xyzB + (size_t)req->nB * 3);
  std::lock_guard<std::mutex> lk(s->mu);
  if (req->ref_id < 0 || req->ref_id >= (int32_t)s->refs.size()) return report_error(ALIGN_E_INVALID, "unknown ref_id");
  r->ref = req->ref_id;
  const align_grid* g = s->refs[(size_t)r->ref].grid;
  // a grid whose single poses already needed key partitions gets spill queues for up to twice
  // as many (a request on a grid that has not needed them sweeps B once per partition)
  const int32_t seed = g->passes_seed[0];
  r->spill_np = g->spill_on && seed >= 2 && seed <= 8 ? std::min(8, 2 * seed) : 0;
  r->bytes = request_bytes(r->nB, r->counts, g->gc.K, g->table_slots, s->n_sm, r->spill_np);
  if (s->ref_bytes + r->bytes > s->budget) return report_error(ALIGN_E_OOM, "request can never fit the memory budget");
  r->ticket = s->next_ticket++;
  r->t_submit = s->now();
  *ticket = r->ticket;
  Req* raw = r.release();
  if (raw->levels == 0) {  // nothing to evaluate: the centre is the answer
    std::memcpy(raw->T, raw->c, sizeof(raw->T));
    raw->t_start = raw->t_submit;
    raw->t_done = raw->t_submit;
    s->done[raw->ticket] = raw;
    s->stats[2] += 1;
    s->cv_done.notify_all();
    return ALIGN_OK;
  }
  s->pending[raw->ticket] = 1;
  s->queue.push_back(raw);
  s->stats[7] = (int64_t)s->queue.size();
  s->cv.notify_all();
  return ALIGN_OK;
}

static void fill_result(const Req* r, align_result* out) {
  std::memcpy(out->T, r->T, sizeof(out->T));
  out->mi = r->best_mi;
  out->status = r->status;
  out->t_submit = r->t_submit;
  out->t_start = r->t_start;
  out->t_done = r->t_done;
}

align_status align_poll(align_server* s, uint64_t ticket, align_result* out) {
  if (!s || !out) return report_error(ALIGN_E_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    if (s->pending.count(ticket)) return ALIGN_NOT_READY;
    return report_error(ALIGN_E_INVALID, "unknown ticket");
  }
  fill_result(it->second, out);
  delete it->second;
  s->done.erase(it);
  return ALIGN_OK;
}

align_status align_wait(align_server* s, uint64_t ticket, int64_t timeout_ms, align_result* out) {
  if (!s || !out) return report_error(ALIGN_E_INVALID, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] { return s->done.count(ticket) || !s->pending.count(ticket); };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return report_error(ALIGN_E_TIMEOUT, "request not done within the timeout");
  }
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return report_error(ALIGN_E_INVALID, "unknown ticket");
  fill_result(it->second, out);
  delete it->second;
  s->done.erase(it);
  return ALIGN_OK;
}

double align_server_now(const align_server* s) { return s ? s->now() : 0.0; }

align_status align_server_stats(align_server* s, int64_t out[8]) {
  if (!s || !out) return report_error(ALIGN_E_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  s->stats[5] = (int64_t)s->used();
  s->stats[6] = (int64_t)s->peak;
  s->stats[7] = (int64_t)s->queue.size();
  for (int i = 0; i < 8; ++i) out[i] = s->stats[i];
  return ALIGN_OK;
}

align_status align_server_destroy(align_server* s) {
  if (!s) return ALIGN_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  for (std::thread& t : s->workers)
    if (t.joinable()) t.join();
  cudaSetDevice(s->device);
  for (Req* r : s->queue) delete r;
  for (auto& kv : s->done) delete kv.second;
  for (Slot& sl : s->slots) {
    workspace_destroy(sl.ws);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  for (Ref& f : s->refs) align_destroy_grid(f.grid);
  delete s;
  return ALIGN_OK;
}

}  // extern "C"
