// Serving loop with continuous batching (see vl.h, "serving").
//
// A worker thread owns the device side.  Submitted queries wait in a FIFO.
// Whenever a launch slot is free, the worker packs the oldest queries whose
// estimated device memory fits the budget into one batch (one persistent
// launch) on that slot's stream; queries arriving meanwhile go into the next
// batch, which runs while earlier ones are still on the GPU.  A finished
// batch (polled with an event, never a device-wide wait) hands each query its
// own result and returns its memory to the budget.  Images and intermediate
// masks stay on the device; only the caller reads results back.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "runtime.h"

using namespace vl;
using Clock = std::chrono::steady_clock;

namespace {

struct Query {
  int64_t ticket = 0;
  const vl_formula* f = nullptr;
  std::vector<vl_image*> imgs;
  int64_t est_bytes = 0;
  Clock::time_point t_submit, t_done;
  vl_status status = VL_ERR_BUSY;  // BUSY until finished
  bool launched = false;
  vl_result* res = nullptr;
};

struct Flight {
  vl_batch* batch = nullptr;
  cudaEvent_t ev = nullptr;
  int slot = 0;
  std::vector<Query*> queries;
  int64_t bytes = 0;
};

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Device bytes one query needs inside a batch (mirrors the batch layout:
// slots, percentile values, select scratch, result masks, tables).
int64_t estimate_bytes(const Plan& P, int H, int W) {
  const int Wp = words_per_row(W);
  const size_t mask = (size_t)H * Wp * 4, px = (size_t)H * W;
  const size_t tiles = (size_t)ccl_tiles_y(H) * ccl_tiles_x(Wp);
  const size_t tstate = tiles * ccl_tile_cap_host(Wp);
  size_t b = align256(mask * (P.n_inter_slots + P.n_root_slots));
  b += (size_t)P.n_scratch_sets *
       (align256(2 * px * 4) + align256(tstate * 4) + align256(tstate));
  b += align256(sizeof(Insn) * P.insns.size()) + align256(sizeof(StepDesc) * P.steps.size()) +
       64 * 1024;
  return (int64_t)b;
}

}  // namespace

struct vl_server {
  uint32_t tag = TAG_SRV;
  vl_context* ctx = nullptr;
  vl_server_config cfg{};
  int64_t budget = 0;
  std::vector<cudaStream_t> streams;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work;  // wakes the worker
  std::condition_variable cv_done;  // wakes waiters
  bool stop = false;
  int64_t next_ticket = 1;
  std::deque<Query*> pending;
  std::map<int64_t, Query*> queries;
  std::vector<Flight> flights;
  std::vector<int> free_slots;
  // statistics
  vl_server_stats st{};
  std::vector<double> lat_ms;

  void run();
  void retire_finished();
  bool launch_one();
};

void vl_server::retire_finished() {
  // under mu
  for (size_t i = 0; i < flights.size();) {
    Flight& fl = flights[i];
    const cudaError_t q = cudaEventQuery(fl.ev);
    if (q == cudaErrorNotReady) { ++i; continue; }
    const auto now = Clock::now();
    std::vector<vl_result*> outs(fl.queries.size(), nullptr);
    if (q == cudaSuccess) batch_release_results(fl.batch, outs.data());
    for (size_t k = 0; k < fl.queries.size(); ++k) {
      Query* qy = fl.queries[k];
      qy->t_done = now;
      if (q != cudaSuccess) {
        qy->status = VL_ERR_CUDA;
        st.failed++;
        continue;
      }
      int32_t word = 0;
      cudaMemcpy(&word, outs[k]->status, sizeof(int32_t), cudaMemcpyDeviceToHost);
      // the batch is done: the result's memory may outlive this server's
      // streams, so release it on the default stream later
      for (auto& blk : outs[k]->keep) blk->stream = nullptr;
      outs[k]->stream = nullptr;
      qy->res = outs[k];
      qy->status = word == 0 ? VL_OK : word == ST_TIMEOUT ? VL_ERR_TIMEOUT : VL_ERR_INTERNAL;
      if (qy->status == VL_OK) {
        st.completed++;
        lat_ms.push_back(std::chrono::duration<double, std::milli>(now - qy->t_submit).count());
      } else {
        st.failed++;
      }
    }
    if (q != cudaSuccess) cudaGetLastError();
    batch_destroy(fl.batch);
    cudaEventDestroy(fl.ev);
    st.bytes_in_use -= fl.bytes;
    free_slots.push_back(fl.slot);
    flights.erase(flights.begin() + i);
    cv_done.notify_all();
  }
}

bool vl_server::launch_one() {
  // under mu; returns true if a batch was launched
  if (free_slots.empty() || pending.empty()) return false;
  std::vector<Query*> take;
  int64_t bytes = 0;
  while (!pending.empty() && (int)take.size() < cfg.max_batch_jobs) {
    Query* q = pending.front();
    if (st.bytes_in_use + bytes + q->est_bytes > budget && !(take.empty() && flights.empty()))
      break;  // wait for memory to come back (a query alone always gets a try)
    take.push_back(q);
    bytes += q->est_bytes;
    pending.pop_front();
  }
  if (take.empty()) return false;
  const int slot = free_slots.back();
  cudaStream_t s = streams[slot];
  std::vector<std::vector<vl_image*>> imgs(take.size());
  std::vector<vl_job> jobs(take.size());
  for (size_t k = 0; k < take.size(); ++k) {
    imgs[k] = take[k]->imgs;
    jobs[k] = vl_job{take[k]->f, imgs[k].data(), (int32_t)imgs[k].size(), 0};
  }
  vl_batch* b = nullptr;
  vl_status rc = batch_build(ctx, jobs.data(), (int)jobs.size(), s, &b);
  if (rc == VL_OK) rc = batch_run(b, s);
  cudaEvent_t ev = nullptr;
  if (rc == VL_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
      cudaEventRecord(ev, s) == cudaSuccess) {
    free_slots.pop_back();
    Flight fl;
    fl.batch = b;
    fl.ev = ev;
    fl.slot = slot;
    fl.queries = take;
    fl.bytes = std::max<int64_t>(bytes, batch_bytes(b));
    st.bytes_in_use += fl.bytes;
    st.peak_bytes = std::max(st.peak_bytes, st.bytes_in_use);
    st.batches++;
    for (Query* q : take) q->launched = true;
    flights.push_back(fl);
    return true;
  }
  // could not launch: out of memory with work in flight -> retry later;
  // otherwise the queries fail
  if (ev) cudaEventDestroy(ev);
  if (b) batch_destroy(b);
  if (rc == VL_ERR_OOM && !flights.empty()) {
    for (auto it = take.rbegin(); it != take.rend(); ++it) pending.push_front(*it);
    return false;
  }
  for (Query* q : take) {
    q->status = rc == VL_OK ? VL_ERR_CUDA : rc;
    q->t_done = Clock::now();
    st.failed++;
  }
  cv_done.notify_all();
  return true;
}

void vl_server::run() {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    retire_finished();
    if (stop && pending.empty() && flights.empty()) break;
    // gather a short window of arrivals before launching a small batch
    if (!pending.empty() && !free_slots.empty() && (int)pending.size() < cfg.max_batch_jobs &&
        cfg.batch_window_us > 0 && !stop) {
      const auto oldest = pending.front()->t_submit;
      const auto ready = oldest + std::chrono::microseconds(cfg.batch_window_us);
      if (Clock::now() < ready && flights.size() > 0) {
        cv_work.wait_until(lk, ready);
        continue;
      }
    }
    bool launched = false;
    {
      std::lock_guard<std::mutex> g(ctx->mu);
      launched = launch_one();
    }
    if (launched) continue;
    // nothing to launch: poll in-flight batches every 50 us, or sleep until
    // a submission arrives
    if (!flights.empty()) cv_work.wait_for(lk, std::chrono::microseconds(50));
    else if (pending.empty() || free_slots.empty()) cv_work.wait_for(lk, std::chrono::milliseconds(5));
  }
}

namespace vl {
void server_destroy(vl_server* s) {
  if (!s || s->tag != TAG_SRV) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    for (Query* q : s->pending) {
      q->status = VL_ERR_CANCELLED;
      s->st.cancelled++;
    }
    s->pending.clear();
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->queries) {
    if (kv.second->res) vl_free(kv.second->res);
    delete kv.second;
  }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  s->tag = TAG_DEAD;
  delete s;
}
}  // namespace vl

extern "C" {

VL_API vl_status vl_server_create(vl_context* ctx, const vl_server_config* cfg, vl_server** out) {
  if (!ctx || ctx->tag != TAG_CTX || !out) return VL_ERR_ARG;
  auto* s = new vl_server();
  s->ctx = ctx;
  if (cfg) s->cfg = *cfg;
  if (s->cfg.max_inflight_batches <= 0) s->cfg.max_inflight_batches = 2;
  if (s->cfg.max_batch_jobs <= 0) s->cfg.max_batch_jobs = 256;
  if (s->cfg.batch_window_us < 0) s->cfg.batch_window_us = 0;
  cudaSetDevice(ctx->device);
  int64_t budget = s->cfg.memory_budget > 0 ? s->cfg.memory_budget : ctx->cfg.memory_budget;
  if (budget <= 0) {
    // the stream-ordered pool keeps what earlier batches freed; hand the
    // free part back first, so that free device memory counts it
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete s;
      return set_err(ctx, VL_ERR_CUDA, "querying free device memory");
    }
    const size_t reserve = std::max<size_t>(total_b / 20, (size_t)2 << 30);
    budget = free_b > reserve ? (int64_t)(free_b - reserve) : (int64_t)(free_b / 2);
  }
  s->budget = budget;
  for (int k = 0; k < s->cfg.max_inflight_batches; ++k) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t t : s->streams) cudaStreamDestroy(t);
      delete s;
      return set_err(ctx, VL_ERR_CUDA, "creating server streams");
    }
    s->streams.push_back(st);
    s->free_slots.push_back(k);
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return VL_OK;
}

VL_API vl_status vl_server_submit(vl_server* s, const vl_formula* f, vl_image* const* imgs,
                                  int32_t n_imgs, int64_t* ticket) {
  if (!s || s->tag != TAG_SRV || !f || f->tag != TAG_FML || !ticket || n_imgs < 1 || !imgs)
    return VL_ERR_ARG;
  // validate now so that a bad query never reaches a batch
  int H = -1, W = -1;
  for (int i = 0; i < n_imgs; ++i) {
    const vl_image* im = imgs[i];
    if (!im || im->tag != TAG_IMG) return set_err(s->ctx, VL_ERR_ARG, "bad image handle");
    if (H < 0) { H = im->H; W = im->W; }
    if (im->H != H || im->W != W) return set_err(s->ctx, VL_ERR_SHAPE, "images must share H x W");
  }
  const Plan& P = f->plan;
  if (n_imgs < (int)P.img_kind.size()) return set_err(s->ctx, VL_ERR_ARG, "too few images");
  for (int i = 0; i < (int)P.img_kind.size(); ++i) {
    if (P.img_kind[i] == 1 && (imgs[i]->is_mask || imgs[i]->C < P.img_channels[i]))
      return set_err(s->ctx, VL_ERR_SHAPE, "image " + std::to_string(i) + " must be a float image");
    if (P.img_kind[i] == 2 && !imgs[i]->is_mask)
      return set_err(s->ctx, VL_ERR_SHAPE, "image " + std::to_string(i) + " must be a mask");
  }
  if (f->pp.group_buffers != s->ctx->pp.group_buffers || f->pp.hmax != s->ctx->pp.hmax)
    return set_err(s->ctx, VL_ERR_ARG, "formula was planned for another tile configuration");
  auto* q = new Query();
  q->f = f;
  q->imgs.assign(imgs, imgs + n_imgs);
  q->est_bytes = estimate_bytes(P, H, W);
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) {
      delete q;
      return VL_ERR_CANCELLED;
    }
    q->ticket = s->next_ticket++;
    s->queries[q->ticket] = q;
    s->pending.push_back(q);
    s->st.submitted++;
    *ticket = q->ticket;
  }
  s->cv_work.notify_all();
  return VL_OK;
}

VL_API vl_status vl_server_wait(vl_server* s, int64_t ticket, int64_t timeout_us, vl_result** out) {
  if (!s || s->tag != TAG_SRV) return VL_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->queries.find(ticket);
  if (it == s->queries.end()) return VL_ERR_ARG;
  Query* q = it->second;
  auto done = [&] { return q->status != VL_ERR_BUSY; };
  if (timeout_us < 0) s->cv_done.wait(lk, done);
  else s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
  if (!done()) return VL_ERR_BUSY;
  const vl_status st = q->status;
  if (out) *out = q->res;
  else if (q->res) vl_free(q->res);
  s->queries.erase(it);
  delete q;
  return st;
}

VL_API vl_status vl_server_cancel(vl_server* s, int64_t ticket) {
  if (!s || s->tag != TAG_SRV) return VL_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->queries.find(ticket);
  if (it == s->queries.end()) return VL_ERR_ARG;
  Query* q = it->second;
  if (q->launched || q->status != VL_ERR_BUSY) return VL_ERR_BUSY;  // too late
  s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), q), s->pending.end());
  q->status = VL_ERR_CANCELLED;
  q->t_done = Clock::now();
  s->st.cancelled++;
  s->cv_done.notify_all();
  return VL_OK;
}

VL_API vl_status vl_server_stats_get(vl_server* s, vl_server_stats* out) {
  if (!s || s->tag != TAG_SRV || !out) return VL_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->st;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
  }
  return VL_OK;
}

}  // extern "C"
