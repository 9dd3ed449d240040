// server.cu — serving alignment requests with continuous batching.
//
// Worker threads (two, or one with a single slot) each own a batch (align_eval_batch, with
// its own stream and workspace) and run steps: admit queued requests while slots and the
// device memory budget allow (first come, first served; a worker admits only while it
// holds no more requests than the other), evaluate the current lattice level of each of
// its active requests in one batched launch, then advance each request to its next level
// (centre <- best pose, ranges halve, as align_search_ex) and retire the finished ones.
// Requests therefore join and leave between steps, the work of all of a worker's requests
// overlaps in the same launches, and while one worker prepares its next step or reads its
// results back on the host, the other's launches keep the device busy.  Reference scans
// stay resident as grids owned by the server.
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
  int32_t levels = 0, level = 0;
  size_t bytes = 0;        // device memory estimate while active
  DevBuf dev_xyz;          // resident B while active
  bool uploaded = false;
  float best_mi = 0.0f;
  int32_t status = ALIGN_OK;
  double t_submit = 0, t_start = 0, t_done = 0;
  // per-step scratch
  std::vector<double> eta;
  std::vector<float> poses;
  std::vector<float> mi;
  int64_t am = -1;
};

struct Ref {
  align_grid* grid = nullptr;
  size_t bytes = 0;
};

int64_t lattice_size(const int32_t m[6]) {
  int64_t P = 1;
  for (int a = 0; a < 6; ++a) P *= m[a];
  return P;
}

}  // namespace

struct align_server {
  int device = 0;
  size_t budget = 0;
  int32_t max_slots = 1;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;       // worker: new requests or stop
  std::condition_variable cv_done;  // clients: a request finished
  std::deque<Req*> queue;
  std::vector<std::vector<Req*>> active;  // per worker
  int32_t n_active = 0;                  // over all workers
  std::unordered_map<uint64_t, Req*> done;
  std::unordered_map<uint64_t, int> pending;  // ticket -> 1 while queued or active
  std::vector<Ref> refs;
  size_t used = 0, peak = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<align_batch*> batches;  // per worker
  std::vector<std::thread> workers;
  // device buffers of retired requests' points, kept for reuse: freeing device memory
  // synchronises the whole device (the other worker's launches included)
  std::vector<mialign::DevBuf> spare;
  int64_t stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Device bytes a request holds while active: its resident points, the batch's staged
// copy and pre-rotated tiles, and the per-pose buffers of one level.
size_t request_bytes(int64_t nB, const int32_t m[6], int K) {
  const int64_t P = lattice_size(m);
  const int64_t n_pad = std::max<int64_t>(3, (nB + 1023) / 1024) * 1024;
  int64_t n_rot = (int64_t)m[3] * m[4] * m[5];
  if (n_rot > std::max<int64_t>(1, P / 4)) n_rot = 1;
  return (size_t)(nB * 24 + n_rot * n_pad * 16 + P * ((int64_t)K * K * 4 + 24 + 4 + 48 + 4 + 4 + 4));
}

void finish_locked(align_server* s, Req* r, int32_t status) {
  r->status = status;
  r->t_done = s->now();
  s->used -= std::min(s->used, r->bytes);
  if (r->dev_xyz.p) {  // back to the spare buffers (at most max_slots are kept)
    if ((int32_t)s->spare.size() < s->max_slots) s->spare.push_back(r->dev_xyz);
    else r->dev_xyz.release();
    r->dev_xyz = DevBuf{};
  }
  s->pending.erase(r->ticket);
  s->done[r->ticket] = r;
  s->stats[2] += 1;
  s->n_active -= 1;
  s->cv_done.notify_all();
  s->cv.notify_all();  // a slot and memory are free: any worker may admit
}

// Admit queued requests into worker w while the slots and the budget allow and w holds no
// more requests than any other worker.
void admit_locked(align_server* s, size_t w) {
  std::vector<Req*>& mine = s->active[w];
  while (!s->queue.empty() && s->n_active < s->max_slots) {
    size_t least = mine.size();
    for (const auto& other : s->active) least = std::min(least, other.size());
    if (mine.size() > least) break;  // another worker has fewer: it admits next
    Req* r = s->queue.front();
    if (s->used + r->bytes > s->budget && s->n_active > 0) break;  // wait for memory
    s->queue.pop_front();
    s->used += r->bytes;
    s->peak = std::max(s->peak, s->used);
    r->t_start = s->now();
    mine.push_back(r);
    s->n_active += 1;
    s->stats[1] += 1;
  }
  s->stats[3] = std::max<int64_t>(s->stats[3], (int64_t)s->n_active);
  s->stats[5] = (int64_t)s->used;
  s->stats[6] = (int64_t)s->peak;
  s->stats[7] = (int64_t)s->queue.size();
}

void worker_main(align_server* s, size_t w) {
  cudaSetDevice(s->device);
  std::vector<align_pair> pairs;
  for (;;) {
    std::vector<Req*> act;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop) return;
        admit_locked(s, w);
        if (!s->active[w].empty()) break;
        s->cv.wait(lk);
      }
      act = s->active[w];
    }
    // upload the points of newly admitted requests; build every request's lattice level
    int32_t step_status = ALIGN_OK;
    pairs.assign(act.size(), align_pair{});
    for (size_t i = 0; i < act.size(); ++i) {
      Req* r = act[i];
      align_grid* g = s->refs[(size_t)r->ref].grid;
      if (!r->uploaded) {
        if (r->nB > 0) {
          {  // a spare buffer large enough, if there is one
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t k = 0; k < s->spare.size(); ++k)
              if (s->spare[k].cap >= (size_t)r->nB * 12) {
                r->dev_xyz = s->spare[k];
                s->spare.erase(s->spare.begin() + (ptrdiff_t)k);
                break;
              }
          }
          cudaError_t e = r->dev_xyz.ensure((size_t)r->nB * 12);
          if (e == cudaSuccess) e = cudaMemcpy(r->dev_xyz.p, r->xyz.data(), (size_t)r->nB * 12, cudaMemcpyHostToDevice);
          if (e != cudaSuccess) {
            step_status = report_cuda_error(e, "upload request points");
            break;
          }
        }
        r->uploaded = true;
      }
      lattice_poses(g->origin, r->c, r->r, r->counts, r->eta, r->poses);
      const int64_t P = (int64_t)(r->eta.size() / 6);
      r->mi.resize((size_t)P);
      r->am = -1;
      align_pair& q = pairs[i];
      q.grid = g;
      q.xyzB = r->nB > 0 ? r->dev_xyz.as<float>() : nullptr;
      q.nB = r->nB;
      q.poses12 = r->poses.data();
      q.eta6 = nullptr;
      q.P = P;
      q.mi_out = r->mi.data();
      q.argmax_out = &r->am;
    }
    if (step_status == ALIGN_OK)
      step_status = align_eval_batch(s->batches[w], pairs.data(), (int32_t)pairs.size(), ALIGN_XYZ_DEVICE);
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats[0] += 1;
    std::vector<Req*> still;
    for (Req* r : act) {
      if (step_status != ALIGN_OK) {
        finish_locked(s, r, step_status);
        continue;
      }
      s->stats[4] += (int64_t)r->mi.size();
      if (r->am < 0 || r->am >= (int64_t)r->mi.size()) {
        finish_locked(s, r, ALIGN_E_INTERNAL);
        continue;
      }
      r->best_mi = r->mi[(size_t)r->am];
      std::memcpy(r->c, &r->eta[(size_t)r->am * 6], sizeof(r->c));
      for (int a = 0; a < 6; ++a) r->r[a] *= 0.5;
      if (++r->level >= r->levels) finish_locked(s, r, ALIGN_OK);
      else still.push_back(r);
    }
    s->active[w].swap(still);
  }
}

}  // namespace

extern "C" {

align_status align_server_create(size_t hbm_budget_bytes, int32_t max_slots, align_server** out) {
  if (!out) return report_error(ALIGN_E_INVALID, "out is NULL");
  *out = nullptr;
  if (max_slots < 1) return report_error(ALIGN_E_INVALID, "max_slots must be >= 1");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_cuda_error(e, "cudaGetDevice");
  std::unique_ptr<align_server> s(new (std::nothrow) align_server());
  if (!s) return report_error(ALIGN_E_OOM, "host allocation failed");
  s->device = dev;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->t0 = std::chrono::steady_clock::now();
  const size_t n_workers = max_slots > 1 ? 2 : 1;
  for (size_t w = 0; w < n_workers; ++w) {
    align_batch* b = nullptr;
    align_status st = align_batch_create(nullptr, &b);  // its own stream
    if (st != ALIGN_OK) {
      for (align_batch* q : s->batches) align_batch_destroy(q);
      return st;
    }
    s->batches.push_back(b);
  }
  s->active.assign(n_workers, {});
  align_server* raw = s.release();
  try {
    for (size_t w = 0; w < n_workers; ++w) raw->workers.emplace_back(worker_main, raw, w);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(raw->mu);
      raw->stop = true;
      raw->cv.notify_all();
    }
    for (std::thread& t : raw->workers)
      if (t.joinable()) t.join();
    for (align_batch* q : raw->batches) align_batch_destroy(q);
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
    if (s->used + bytes > s->budget) return report_error(ALIGN_E_OOM, "reference does not fit the memory budget");
  }
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return report_cuda_error(e, "cudaSetDevice");
  align_grid* g = nullptr;
  st = align_create_grid(desc, nullptr, &g);
  if (st != ALIGN_OK) return st;
  st = align_set_reference(g, xyzA, nA, 0);
  if (st != ALIGN_OK) {
    align_destroy_grid(g);
    return st;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->refs.push_back(Ref{g, bytes});
  s->used += bytes;
  s->peak = std::max(s->peak, s->used);
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
  r->bytes = request_bytes(r->nB, r->counts, s->refs[(size_t)r->ref].grid->gc.K);
  size_t ref_bytes = 0;
  for (const Ref& f : s->refs) ref_bytes += f.bytes;
  if (ref_bytes + r->bytes > s->budget) return report_error(ALIGN_E_OOM, "request can never fit the memory budget");
  r->ticket = s->next_ticket++;
  r->t_submit = s->now();
  *ticket = r->ticket;
  Req* raw = r.release();
  if (raw->levels == 0) {  // nothing to evaluate: the centre is the answer
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
  std::memcpy(out->T, r->c, sizeof(out->T));
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
  s->stats[5] = (int64_t)s->used;
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
  for (auto& act : s->active)
    for (Req* r : act) {
      r->dev_xyz.release();
      delete r;
    }
  for (auto& kv : s->done) delete kv.second;
  for (DevBuf& b : s->spare) b.release();
  for (Ref& f : s->refs) align_destroy_grid(f.grid);
  for (align_batch* b : s->batches) align_batch_destroy(b);
  delete s;
  return ALIGN_OK;
}

}  // extern "C"
