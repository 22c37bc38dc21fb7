// C ABI of the library: contexts, images, formulas, evaluation, results,
// connected components.  See include/vl.h for the contract of each call.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>

#include "runtime.h"
#include "schedule.h"
#include "spec.h"

using namespace vl;

namespace vl {

DevBlock::~DevBlock() {
  if (!ptr) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != device) cudaSetDevice(device);
  if (cudaFreeAsync(ptr, stream) != cudaSuccess) {
    // the stream is gone (its owner destroyed it): free synchronously, and
    // leave no error behind for the caller's next check
    cudaGetLastError();
    cudaFree(ptr);
    cudaGetLastError();
  }
  if (cur != device && cur >= 0) cudaSetDevice(cur);
}

vl_status set_err(vl_context* ctx, vl_status code, const std::string& msg) {
  if (ctx) {
    std::lock_guard<std::mutex> g(ctx->err_mu);
    ctx->err = msg;
  }
  return code;
}

vl_status cuda_err(vl_context* ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear the sticky-free error state of the runtime
  return set_err(ctx, e == cudaErrorMemoryAllocation ? VL_ERR_OOM : VL_ERR_CUDA, m);
}

cudaError_t dev_alloc(vl_context* ctx, size_t bytes, cudaStream_t st, DevBlockPtr* out) {
  auto b = std::make_shared<DevBlock>();
  b->bytes = bytes;
  b->stream = st;
  b->device = ctx->device;
  if (bytes) {
    cudaError_t e = cudaMallocAsync(&b->ptr, bytes, st);
    if (e == cudaErrorMemoryAllocation) {
      // the pool keeps freed memory (its release threshold is unlimited, so
      // graph replays never give memory back); blocks of other sizes can
      // fill the device: hand the free ones back and try once more
      cudaGetLastError();
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
      e = cudaMallocAsync(&b->ptr, bytes, st);
    }
    if (e != cudaSuccess) {
      b->ptr = nullptr;
      return e;
    }
  }
  *out = std::move(b);
  return cudaSuccess;
}

cudaError_t wait_images(vl_image* const* imgs, int n, cudaStream_t st) {
  for (int i = 0; i < n; ++i)
    if (imgs[i] && imgs[i]->ready && imgs[i]->ready->ev) {
      const cudaError_t e = cudaStreamWaitEvent(st, imgs[i]->ready->ev, 0);
      if (e) return e;
    }
  return cudaSuccess;
}

// Order reads of a result on `st` after the work that produced it.
cudaError_t wait_result(const vl_result* r, cudaStream_t st) {
  if (r->done && r->done->ev && st != r->stream) return cudaStreamWaitEvent(st, r->done->ev, 0);
  return cudaSuccess;
}

cudaError_t record_ready(vl_image* im, cudaStream_t st) {
  im->ready = std::make_shared<EventHolder>();
  cudaError_t e = cudaEventCreateWithFlags(&im->ready->ev, cudaEventDisableTiming);
  if (!e) e = cudaEventRecord(im->ready->ev, st);
  return e;
}

}  // namespace vl

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool valid(const void* h, uint32_t tag) {
  return h && *reinterpret_cast<const uint32_t*>(h) == tag;
}

// Check the images of a job against a plan; returns shape in H, W.
vl_status check_job_images(vl_context* ctx, const Plan& P, vl_image* const* imgs, int n_imgs,
                           int* H, int* W, int* D = nullptr) {
  if (n_imgs < (int)P.img_kind.size())
    return set_err(ctx, VL_ERR_ARG, "formula reads image " + std::to_string(P.img_kind.size() - 1) +
                                        " but only " + std::to_string(n_imgs) + " were given");
  if (n_imgs < 1 || !imgs) return set_err(ctx, VL_ERR_ARG, "at least one image is needed");
  int h = -1, w = -1;
  for (int i = 0; i < n_imgs; ++i) {
    const vl_image* im = imgs[i];
    if (!valid(im, TAG_IMG)) return set_err(ctx, VL_ERR_ARG, "bad image handle " + std::to_string(i));
    if (h < 0) { h = im->H; w = im->W; }
    if (im->H != h || im->W != w || im->D != imgs[0]->D)
      return set_err(ctx, VL_ERR_SHAPE, "images of one evaluation must share D x H x W");
    if (i < (int)P.img_kind.size()) {
      if (P.img_kind[i] == 1 && (im->is_mask || im->C < P.img_channels[i]))
        return set_err(ctx, VL_ERR_SHAPE, "image " + std::to_string(i) +
                                              " must be a float image with enough channels");
      if (P.img_kind[i] == 2 && !im->is_mask)
        return set_err(ctx, VL_ERR_SHAPE, "image " + std::to_string(i) + " must be a mask");
    }
  }
  // the component select keys pixels and unseeded components apart: its
  // union-find holds 2 * H * W int32 entries
  if (!P.rz.empty() && (long long)h * w > (1LL << 30))
    return set_err(ctx, VL_ERR_SHAPE, "reachability needs images of at most 2^30 pixels");
  if (imgs[0]->D > 1 && P.conn != 6 && P.conn != 26)
    return set_err(ctx, VL_ERR_SHAPE, "a volume needs a formula compiled with adjacency 6 or 26");
  *H = h;
  *W = w;
  if (D) *D = imgs[0]->D;
  return VL_OK;
}

// Formulas over volumes (adjacency 6 or 26) run in the per-operator form.
inline bool volume_plan(const Plan& P) { return P.conn == 6 || P.conn == 26; }

int ccl_merge_chunks(int H, int Wp, int cth) {
  const long long n = ccl_merge_units(H, Wp, 0, cth);  // one warp each
  const int warps = EXEC_THREADS / 32;
  return (int)std::max<long long>(1, (n + warps - 1) / warps);
}

}  // namespace

// ================================================================ batch ==

struct vl_batch {
  uint32_t tag = TAG_BAT;
  vl_context* ctx = nullptr;
  int n_jobs = 0;
  DevBlockPtr persist;  // root buffers + status words (kept by results)
  DevBlockPtr trans;    // tables, counters, slots, scratch
  size_t counters_off = 0, counters_bytes = 0;
  int32_t* status_base = nullptr;
  int n_status = 0;
  ExecLaunch L{};
  std::vector<vl_result*> results;
  bool released = false;
  std::shared_ptr<EventHolder> done;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  int64_t bytes = 0;
  std::vector<vl_image*> images;        // waited on before every run
  DevBlockPtr trace;                    // optional step timeline
  std::vector<int32_t> trace_meta;      // {job, step, kind} per timeline entry
  // A lone job with a tiny plan runs in the per-operator form captured in
  // the graph instead (the persistent launch's step latencies would
  // dominate it): its plan, images and shape.
  bool plain_form = false;
  int plain_runs = 0;                   // the graph is captured on the second run
  std::shared_ptr<vl::Plan> plain_plan;
  std::vector<vl_image*> plain_imgs;
  int plain_H = 0, plain_W = 0;
  char* plain_roots = nullptr;
};

namespace vl {

int64_t batch_bytes(const vl_batch* b) { return b ? b->bytes : 0; }

vl_status batch_build_per_op(vl_context* ctx, const vl_job& job, int H, int W, cudaStream_t st,
                             vl_batch** out);

vl_status batch_build(vl_context* ctx, const vl_job* jobs, int n_jobs, cudaStream_t st,
                      vl_batch** out, const TileShape* force, bool persistent) {
  if (n_jobs < 1 || !jobs) return set_err(ctx, VL_ERR_ARG, "empty batch");
  struct JobInfo {
    const Plan* P;
    int H, W, Wp, pitch;
    int gty, gtx, cty, ctx_, ctiles, cth;
    std::vector<int> need;
    size_t off_images, off_slotptrs, off_pct, off_slots, off_rz, set_bytes, set_off[3];
    size_t off_roots, off_status, off_planes, off_num;
    int n_table;  // image table: the formula's images, then its number images
    int step_base;
    int formula_idx;
  };
  std::vector<JobInfo> J(n_jobs);
  std::map<const Plan*, int> formula_index;
  std::vector<const Plan*> formulas;
  for (int j = 0; j < n_jobs; ++j) {
    const vl_formula* f = jobs[j].formula;
    if (!valid(f, TAG_FML)) return set_err(ctx, VL_ERR_ARG, "bad formula handle in job " + std::to_string(j));
    if (f->pp.group_buffers != ctx->pp.group_buffers || f->pp.hmax != ctx->pp.hmax)
      return set_err(ctx, VL_ERR_ARG, "formula was planned for another tile configuration");
    if (volume_plan(f->plan))
      return set_err(ctx, VL_ERR_ARG, "job " + std::to_string(j) +
                                          ": formulas over volumes (adjacency 6 or 26) run in the "
                                          "per-operator form (vl_eval)");
    vl_status s = check_job_images(ctx, f->plan, jobs[j].images, jobs[j].n_images, &J[j].H, &J[j].W);
    if (s != VL_OK) return s;
    J[j].P = &f->plan;
    if (!formula_index.count(&f->plan)) {
      formula_index[&f->plan] = (int)formulas.size();
      formulas.push_back(&f->plan);
    }
    J[j].formula_idx = formula_index[&f->plan];
  }
  // ---- layout of the transient block
  size_t off = 0;
  auto take = [&](size_t bytes, size_t a = 256) { off = align_up(off, a); size_t o = off; off += bytes; return o; };
  const size_t off_jobs = take(sizeof(DevJob) * n_jobs);
  std::vector<size_t> f_steps(formulas.size()), f_insns(formulas.size()), f_rz(formulas.size()),
      f_pct(formulas.size()), f_rtab(formulas.size()), f_rvals(formulas.size()),
      f_doff(formulas.size()), f_deps(formulas.size()), f_arith(formulas.size());
  for (size_t k = 0; k < formulas.size(); ++k) {
    const Plan* P = formulas[k];
    f_steps[k] = take(sizeof(StepDesc) * std::max<size_t>(1, P->steps.size()));
    f_insns[k] = take(sizeof(Insn) * std::max<size_t>(1, P->insns.size()));
    f_rz[k] = take(sizeof(RzDesc) * std::max<size_t>(1, P->rz.size()));
    f_pct[k] = take(sizeof(PctDesc) * std::max<size_t>(1, P->pct.size()));
    f_rtab[k] = take(sizeof(RankTab) * std::max<size_t>(1, P->rtab.size()));
    f_rvals[k] = take(sizeof(float) * std::max<size_t>(1, P->rvals.size()));
    f_doff[k] = take(sizeof(int32_t) * std::max<size_t>(1, P->dep_off.size()));
    f_deps[k] = take(sizeof(int32_t) * std::max<size_t>(1, P->deps.size()));
    f_arith[k] = take(sizeof(ArithInsn) * std::max<size_t>(1, P->arith.size()));
  }
  const TileShape ts = force ? *force : pick_tile_shape(ctx, jobs, n_jobs, nullptr, !persistent);
  if (ts.per_op) {
    if (n_jobs != 1 || persistent)
      return set_err(ctx, VL_ERR_ARG, "the per-operator form takes a batch of one job");
    return batch_build_per_op(ctx, jobs[0], J[0].H, J[0].W, st, out);
  }
  if (!tile_shape_fits(ctx, ts)) return set_err(ctx, VL_ERR_ARG, "tile shape does not fit shared memory");
  const int cps = ts.ctas_per_sm > 0 ? std::min(ts.ctas_per_sm, ctx->ctas_per_sm) : ctx->ctas_per_sm;
  int total_steps = 0;
  std::vector<WorkItem> items;
  const int grid = std::max(1, ctx->sm_count * cps);
  for (int j = 0; j < n_jobs; ++j) {
    JobInfo& I = J[j];
    const Plan& P = *I.P;
    I.Wp = words_per_row(I.W);
    I.pitch = 32 * I.Wp;
    I.gty = (I.H + ts.rows - 1) / ts.rows;
    I.gtx = (I.Wp + ts.words - 1) / ts.words;
    // labelling tiles of 16 rows when the job's selects would otherwise
    // leave most of the grid idle (a lone small image, a chain of selects)
    {
      int maxbatch = 0;
      for (const StepDesc& sd : P.steps)
        if (sd.kind == SK_RZ_LOCAL) maxbatch = std::max(maxbatch, sd.rz_cnt);
      const long long t32 = (long long)ccl_tiles_y(I.H) * ccl_tiles_x(I.Wp);
      I.cth = (long long)n_jobs * t32 * maxbatch < grid ? 16 : CCL_TH;
    }
    I.cty = ccl_tiles_y(I.H, 0, I.cth);
    I.ctx_ = ccl_tiles_x(I.Wp);
    I.ctiles = I.cty * I.ctx_;
    I.step_base = total_steps;
    total_steps += (int)P.steps.size();
    for (const StepDesc& s : P.steps) {
      int n = 1;
      switch (s.kind) {
        case SK_PCT: n = s.pct_cnt; break;
        case SK_GROUP: n = I.gty * I.gtx; break;
        case SK_RZ_LOCAL: case SK_RZ_FINAL: n = s.rz_cnt * I.ctiles; break;
        case SK_RZ_MERGE:
          // at most two waves of items per step: the merge is latency-bound,
          // and fewer, longer items tie up fewer CTAs that a critical step
          // could use (one wave, or no cap, measured slower)
          n = s.rz_cnt * std::min(ccl_merge_chunks(I.H, I.Wp, I.cth),
                                  std::max(1, 2 * (grid + s.rz_cnt - 1) / s.rz_cnt));
          break;
        case SK_RANK: n = (int)P.rtab.size() * ((I.H + RANK_ROWS - 1) / RANK_ROWS); break;
        case SK_ARITH: n = (I.H + ARITH_ROWS - 1) / ARITH_ROWS; break;
      }
      I.need.push_back(std::max(1, n));
    }
    // the formula's own images, then its number images
    I.n_table = (int)P.img_kind.size() + P.n_num_images;
    I.off_images = take(sizeof(DevImage) * std::max(1, I.n_table));
    I.off_slotptrs = take(sizeof(uint32_t*) * std::max(1, P.n_inter_slots + P.n_root_slots + P.n_mask_slots));
  }
  // work items: every step split into items of about a tile each (at most
  // 4 x grid items per step), with an estimated time per item, then put in
  // executor order (order_work_items in schedule.cpp: a list-scheduling
  // simulation by bottom level for one job, progress order for several).
  {
    long long subitems = 0;
    for (int j = 0; j < n_jobs; ++j)
      for (size_t s = 0; s < J[j].need.size(); ++s) subitems += J[j].need[s];
    // with work for many waves (thousands of small images), items of short
    // tiles are merged up to ~40 us so that popping stays cheap beside work
    // -- but only as far as the jobs running side by side still offer four
    // items per CTA: the steps of one job mostly wait on each other, and
    // merging the tiles of a step there only serialises them on fewer CTAs
    const bool plenty = subitems > 32LL * grid;
    std::vector<WorkItem> pending;  // every item, step by step
    std::vector<SchedJob> sj(n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
      const Plan& P = *J[j].P;
      sj[j].dep_off = P.dep_off.data();
      sj[j].deps = P.deps.data();
      const double tile_scale = (double)ts.rows * ts.words / (16.0 * 32.0);
      for (size_t si = 0; si < J[j].need.size(); ++si) {
        const StepDesc& sd = P.steps[si];
        const int n = J[j].need[si];
        // estimated microseconds per sub-item (one GB300, two CTAs per SM)
        double sub_us;
        switch (sd.kind) {
          case SK_GROUP: sub_us = (5.0 + 1.3 * sd.insn_cnt) * tile_scale; break;
          case SK_RZ_LOCAL: sub_us = 35.0 * J[j].cth / CCL_TH; break;
          case SK_RZ_MERGE: {
            // a sub-item of a select's merge: its share of the merge units
            // over the 16 warps of a CTA, ~5 us per latency-bound unit
            const long long units = ccl_merge_units(J[j].H, J[j].Wp, 0, J[j].cth);
            const long long per_rz = std::max(1, n / std::max(1, sd.rz_cnt));
            sub_us = 5.0 * std::ceil((double)units / (per_rz * (EXEC_THREADS / 32)));
            break;
          }
          case SK_RZ_FINAL: sub_us = 10.0 * J[j].cth / CCL_TH; break;
          case SK_RANK: sub_us = 50.0; break;
          case SK_ARITH: sub_us = 10.0 + 2.0 * sd.insn_cnt; break;
          default: sub_us = 100.0; break;
        }
        int chunk = std::max(1, (n + 4 * grid - 1) / (4 * grid));
        if (plenty) {
          const double tile_us = sd.kind == SK_GROUP ? 5.0 + 1.0 * sd.insn_cnt
                                 : sd.kind == SK_RZ_FINAL ? 20.0 : 40.0;
          const long long side_by_side = std::max<long long>(1, (long long)n * n_jobs / (4LL * grid));
          chunk = std::max<long long>(chunk, std::min<long long>(
              {(long long)n, (long long)std::ceil(40.0 / tile_us), side_by_side}));
        }
        SchedStep st{(int)pending.size(), 0, sub_us * chunk};
        for (int first = 0; first < n; first += chunk, ++st.n)
          pending.push_back(WorkItem{j, (int)si, first, std::min(chunk, n - first)});
        sj[j].steps.push_back(st);
      }
    }
    if (!order_work_items(sj, pending, grid, &items))
      return set_err(ctx, VL_ERR_INTERNAL, "internal: step order");
  }
  const size_t off_items = take(sizeof(WorkItem) * std::max<size_t>(1, items.size()));
  const size_t off_need = take(sizeof(int32_t) * std::max(1, total_steps));
  // counters: head, done[steps] -- zeroed before every run
  const size_t off_counters = take(sizeof(int32_t) * (1 + total_steps));
  const size_t counters_bytes = sizeof(int32_t) * (1 + total_steps);
  const size_t tables_end = off;
  // buffers
  for (int j = 0; j < n_jobs; ++j) {
    JobInfo& I = J[j];
    const Plan& P = *I.P;
    const size_t mask_bytes = (size_t)I.H * I.Wp * 4;
    const size_t P_px = (size_t)I.H * I.W;
    I.off_pct = take(sizeof(float) * std::max(1, P.n_pct_slots));
    I.off_planes = take(mask_bytes * P.n_planes);
    I.off_num = take(sizeof(float) * (size_t)I.H * I.pitch * P.n_num_images);
    I.off_slots = take(mask_bytes * P.n_inter_slots);
    const size_t tstate = (size_t)I.ctiles * ccl_tile_cap_host(I.Wp, I.cth);
    // select scratch sets: G (2 * P_px keys), tpar, tflag, each 256-byte aligned
    {
      size_t o = 0;
      auto sub = [&](size_t bytes) { o = align_up(o, 256); size_t r = o; o += bytes; return r; };
      I.set_off[0] = sub(2 * P_px * 4);
      I.set_off[1] = sub(tstate * 4);
      I.set_off[2] = sub(tstate);
      I.set_bytes = align_up(o, 256);
      I.off_rz = take(I.set_bytes * (size_t)P.n_scratch_sets);
    }
  }
  const size_t trans_bytes = align_up(off, 256);
  // persistent block: root buffers and status words
  size_t poff = 0;
  auto ptake = [&](size_t bytes) { poff = align_up(poff, 256); size_t o = poff; poff += bytes; return o; };
  const size_t off_status = ptake(sizeof(int32_t) * n_jobs);
  for (int j = 0; j < n_jobs; ++j) {
    JobInfo& I = J[j];
    I.off_roots = ptake((size_t)I.H * I.Wp * 4 * I.P->n_root_slots);
  }
  auto b = std::make_unique<vl_batch>();
  b->ctx = ctx;
  b->n_jobs = n_jobs;
  for (int j = 0; j < n_jobs; ++j)
    for (int i = 0; i < jobs[j].n_images; ++i) b->images.push_back(jobs[j].images[i]);
  std::sort(b->images.begin(), b->images.end());
  b->images.erase(std::unique(b->images.begin(), b->images.end()), b->images.end());
  cudaError_t e = dev_alloc(ctx, trans_bytes, st, &b->trans);
  if (e) return cuda_err(ctx, e, "allocating batch tables and scratch");
  e = dev_alloc(ctx, align_up(poff, 256), st, &b->persist);
  if (e) return cuda_err(ctx, e, "allocating result buffers");
  b->bytes = (int64_t)(trans_bytes + poff);
  char* tb = static_cast<char*>(b->trans->ptr);
  char* pb = static_cast<char*>(b->persist->ptr);
  // ---- host copy of the tables
  std::vector<char> host(tables_end, 0);
  for (size_t k = 0; k < formulas.size(); ++k) {
    const Plan* P = formulas[k];
    if (!P->steps.empty()) std::memcpy(&host[f_steps[k]], P->steps.data(), sizeof(StepDesc) * P->steps.size());
    if (!P->insns.empty()) std::memcpy(&host[f_insns[k]], P->insns.data(), sizeof(Insn) * P->insns.size());
    if (!P->rz.empty()) std::memcpy(&host[f_rz[k]], P->rz.data(), sizeof(RzDesc) * P->rz.size());
    if (!P->pct.empty()) std::memcpy(&host[f_pct[k]], P->pct.data(), sizeof(PctDesc) * P->pct.size());
    if (!P->rtab.empty()) std::memcpy(&host[f_rtab[k]], P->rtab.data(), sizeof(RankTab) * P->rtab.size());
    if (!P->rvals.empty()) std::memcpy(&host[f_rvals[k]], P->rvals.data(), sizeof(float) * P->rvals.size());
    if (!P->dep_off.empty()) std::memcpy(&host[f_doff[k]], P->dep_off.data(), sizeof(int32_t) * P->dep_off.size());
    if (!P->deps.empty()) std::memcpy(&host[f_deps[k]], P->deps.data(), sizeof(int32_t) * P->deps.size());
    if (!P->arith.empty()) std::memcpy(&host[f_arith[k]], P->arith.data(), sizeof(ArithInsn) * P->arith.size());
  }
  DevJob* hj = reinterpret_cast<DevJob*>(&host[off_jobs]);
  int32_t* hneed = reinterpret_cast<int32_t*>(&host[off_need]);
  int32_t* counters_dev = reinterpret_cast<int32_t*>(tb + off_counters);
  int32_t* status_dev = reinterpret_cast<int32_t*>(pb + off_status);
  for (int j = 0; j < n_jobs; ++j) {
    JobInfo& I = J[j];
    const Plan& P = *I.P;
    DevJob d{};
    d.H = I.H; d.W = I.W; d.Wp = I.Wp; d.pitch = I.pitch;
    d.n_steps = (int)P.steps.size();
    d.step_base = I.step_base;
    d.gth = ts.rows; d.gtww = ts.words;
    d.g_tiles_y = I.gty; d.g_tiles_x = I.gtx;
    d.c_tiles_y = I.cty; d.c_tiles_x = I.ctx_;
    d.conn = P.conn;
    d.n_images = I.n_table;
    DevImage* him = reinterpret_cast<DevImage*>(&host[I.off_images]);
    const int n_own = (int)P.img_kind.size();
    for (int i = 0; i < n_own; ++i) {
      const vl_image* im = jobs[j].images[i];
      him[i] = DevImage{im->data, im->mask, im->C, im->is_mask, im->format, 0};
    }
    for (int k = 0; k < P.n_num_images; ++k)
      him[n_own + k] = DevImage{tb + I.off_num + sizeof(float) * (size_t)I.H * I.pitch * k, nullptr,
                                1, 0, PX_F32, 1};
    d.images = reinterpret_cast<const DevImage*>(tb + I.off_images);
    d.arith = reinterpret_cast<const ArithInsn*>(tb + f_arith[I.formula_idx]);
    d.n_arith = (int32_t)P.arith.size();
    d.first_num_image = n_own;
    uint32_t** hs = reinterpret_cast<uint32_t**>(&host[I.off_slotptrs]);
    const size_t mask_bytes = (size_t)I.H * I.Wp * 4;
    for (int s = 0; s < P.n_inter_slots; ++s)
      hs[s] = reinterpret_cast<uint32_t*>(tb + I.off_slots + mask_bytes * s);
    for (int s = 0; s < P.n_root_slots; ++s)
      hs[P.n_inter_slots + s] = reinterpret_cast<uint32_t*>(pb + I.off_roots + mask_bytes * s);
    for (int s = 0; s < P.n_mask_slots; ++s)
      hs[P.n_inter_slots + P.n_root_slots + s] = jobs[j].images[P.mask_slot_image[s]]->mask;
    d.slots = reinterpret_cast<uint32_t* const*>(tb + I.off_slotptrs);
    const int k = I.formula_idx;
    d.insns = reinterpret_cast<const Insn*>(tb + f_insns[k]);
    d.steps = reinterpret_cast<const StepDesc*>(tb + f_steps[k]);
    d.dep_off = reinterpret_cast<const int32_t*>(tb + f_doff[k]);
    d.deps = reinterpret_cast<const int32_t*>(tb + f_deps[k]);
    d.rz = reinterpret_cast<const RzDesc*>(tb + f_rz[k]);
    d.pct = reinterpret_cast<const PctDesc*>(tb + f_pct[k]);
    d.pct_val = reinterpret_cast<float*>(tb + I.off_pct);
    d.rtab = reinterpret_cast<const RankTab*>(tb + f_rtab[k]);
    d.rvals = reinterpret_cast<const float*>(tb + f_rvals[k]);
    d.n_rtab = (int32_t)P.rtab.size();
    d.planes = reinterpret_cast<uint32_t*>(tb + I.off_planes);
    d.rzs = reinterpret_cast<unsigned char*>(tb + I.off_rz);
    d.set_bytes = (int64_t)I.set_bytes;
    d.off_tpar = (int64_t)I.set_off[1];
    d.off_tflag = (int64_t)I.set_off[2];
    d.tile_cap = ccl_tile_cap_host(I.Wp, I.cth);
    d.c_th = I.cth;
    d.status = status_dev + j;
    hj[j] = d;
    for (size_t s = 0; s < I.need.size(); ++s) hneed[I.step_base + s] = I.need[s];
  }
  // items with job-relative steps
  if (!items.empty()) std::memcpy(&host[off_items], items.data(), sizeof(WorkItem) * items.size());
  e = cudaMemcpyAsync(tb, host.data(), tables_end, cudaMemcpyHostToDevice, st);
  if (e) return cuda_err(ctx, e, "uploading batch tables");
  // ---- launch description
  b->counters_off = off_counters;
  b->counters_bytes = counters_bytes;
  b->status_base = status_dev;
  b->n_status = n_jobs;
  ExecLaunch& L = b->L;
  L.jobs = reinterpret_cast<const DevJob*>(tb + off_jobs);
  L.items = reinterpret_cast<const WorkItem*>(tb + off_items);
  L.n_items = (int32_t)items.size();
  L.head = counters_dev;
  L.done = counters_dev + 1;
  L.need = reinterpret_cast<const int32_t*>(tb + off_need);
  L.spin_limit = ctx->cfg.spin_limit != 0 ? ctx->cfg.spin_limit : (1LL << 22);
  L.group_buffers = ctx->nb;
  L.group_bh = ts.rows + 2 * ctx->hmax;
  L.group_bw = ts.words + 2;
  L.grid = std::max(1, std::min<int>(grid, (int)items.size()));
  L.smem_bytes = (int32_t)ctx->exec_smem;
  L.trace = nullptr;
  if (ctx->cfg.trace) {
    e = dev_alloc(ctx, sizeof(unsigned long long) * 4 * std::max(1, total_steps), st, &b->trace);
    if (e) return cuda_err(ctx, e, "allocating the step timeline");
    L.trace = static_cast<unsigned long long*>(b->trace->ptr);
    for (int j = 0; j < n_jobs; ++j)
      for (size_t s2 = 0; s2 < J[j].P->steps.size(); ++s2) {
        b->trace_meta.push_back(j);
        b->trace_meta.push_back((int32_t)s2);
        b->trace_meta.push_back(J[j].P->steps[s2].kind);
      }
  }
  // ---- results
  b->done = std::make_shared<EventHolder>();
  e = cudaEventCreateWithFlags(&b->done->ev, cudaEventDisableTiming);
  if (e) return cuda_err(ctx, e, "creating an event");
  for (int j = 0; j < n_jobs; ++j) {
    JobInfo& I = J[j];
    const Plan& P = *I.P;
    auto* r = new vl_result();
    r->ctx = ctx;
    r->H = I.H; r->W = I.W; r->Wp = I.Wp;
    r->n_roots = P.n_roots;
    const size_t mask_bytes = (size_t)I.H * I.Wp * 4;
    for (int q = 0; q < P.n_roots; ++q)
      r->roots.push_back(reinterpret_cast<uint32_t*>(pb + I.off_roots +
                                                     mask_bytes * (P.root_slot[q] - P.n_inter_slots)));
    r->status = status_dev + j;
    r->stream = st;
    r->done = b->done;
    r->borrowed = true;
    r->keep.push_back(b->persist);
    b->results.push_back(r);
  }
  *out = b.release();
  return VL_OK;
}

// A batch of one job in the per-operator form: result buffers and status
// word only; batch_run captures the kernels into the batch's graph.
vl_status batch_build_per_op(vl_context* ctx, const vl_job& job, int H, int W, cudaStream_t st,
                             vl_batch** out) {
  const Plan& P = job.formula->plan;
  const int Wp = words_per_row(W);
  const size_t mask_bytes = (size_t)H * Wp * 4;
  auto b = std::make_unique<vl_batch>();
  b->ctx = ctx;
  b->n_jobs = 1;
  b->images.assign(job.images, job.images + job.n_images);
  std::sort(b->images.begin(), b->images.end());
  b->images.erase(std::unique(b->images.begin(), b->images.end()), b->images.end());
  cudaError_t e = dev_alloc(ctx, 256 + mask_bytes * P.n_root_slots, st, &b->persist);
  if (e) return cuda_err(ctx, e, "allocating result buffers");
  b->bytes = (int64_t)(256 + mask_bytes * P.n_root_slots);
  char* pb = static_cast<char*>(b->persist->ptr);
  b->status_base = reinterpret_cast<int32_t*>(pb);
  b->n_status = 1;
  b->plain_form = true;
  b->plain_plan = std::make_shared<Plan>(P);
  b->plain_imgs.assign(job.images, job.images + job.n_images);
  b->plain_H = H;
  b->plain_W = W;
  b->plain_roots = pb + 256;
  b->done = std::make_shared<EventHolder>();
  e = cudaEventCreateWithFlags(&b->done->ev, cudaEventDisableTiming);
  if (e) return cuda_err(ctx, e, "creating an event");
  auto* r = new vl_result();
  r->ctx = ctx;
  r->H = H; r->W = W; r->Wp = Wp;
  r->n_roots = P.n_roots;
  for (int q = 0; q < P.n_roots; ++q)
    r->roots.push_back(reinterpret_cast<uint32_t*>(b->plain_roots +
                                                   mask_bytes * (P.root_slot[q] - P.n_inter_slots)));
  r->status = b->status_base;
  r->stream = st;
  r->done = b->done;
  r->borrowed = true;
  r->keep.push_back(b->persist);
  b->results.push_back(r);
  *out = b.release();
  return VL_OK;
}

vl_status batch_run(vl_batch* b, cudaStream_t st) {
  vl_context* ctx = b->ctx;
  cudaError_t e;
  const bool graphs = ctx->cfg.use_graphs && st != nullptr && st != cudaStreamLegacy &&
                      st != cudaStreamPerThread;
  if ((e = wait_images(b->images.data(), (int)b->images.size(), st)))
    return cuda_err(ctx, e, "waiting for image uploads");
  if (b->trace) {  // timeline: start = +inf, the rest 0
    const size_t n = b->trace->bytes / 32;
    if ((e = cudaMemsetAsync(b->trace->ptr, 0, b->trace->bytes, st)) ||
        (e = cudaMemset2DAsync(b->trace->ptr, 32, 0xFF, 8, n, st)))
      return cuda_err(ctx, e, "clearing the step timeline");
  }
  if (b->plain_form) {  // per-operator form, captured like the executor
    if ((e = ccl_configure())) return cuda_err(ctx, e, "setting kernel attributes");
    auto enqueue = [&]() -> vl_status {
      cudaError_t z = cudaMemsetAsync(b->status_base, 0, sizeof(int32_t), st);
      if (z) return cuda_err(ctx, z, "zeroing the status word");
      return plain_enqueue(ctx, *b->plain_plan, b->plain_imgs.data(), b->plain_H, b->plain_W, 1,
                           b->plain_roots, b->status_base, st);
    };
    // a batch run once (a server's) is not worth a capture, and its graph's
    // memory nodes would keep their memory from the pool: capture on the
    // second run
    if (graphs && !b->gexec && b->plain_runs++ > 0) {
      if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)))
        return cuda_err(ctx, e, "beginning graph capture");
      const vl_status s1 = enqueue();
      e = cudaStreamEndCapture(st, &b->graph);
      if (s1 != VL_OK || e) {
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        return s1 != VL_OK ? s1 : cuda_err(ctx, e, "capturing the per-operator graph");
      }
      if ((e = cudaGraphInstantiate(&b->gexec, b->graph, 0)))
        return cuda_err(ctx, e, "instantiating the per-operator graph");
    }
    if (b->gexec) {
      if ((e = cudaGraphLaunch(b->gexec, st))) return cuda_err(ctx, e, "launching the graph");
    } else {
      const vl_status s1 = enqueue();
      if (s1 != VL_OK) return s1;
    }
    if ((e = cudaEventRecord(b->done->ev, st))) return cuda_err(ctx, e, "recording an event");
    for (vl_result* r : b->results) r->stream = st;
    return VL_OK;
  }
  char* tb = static_cast<char*>(b->trans->ptr);
  if (graphs && !b->gexec) {
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e) return cuda_err(ctx, e, "beginning graph capture");
    cudaError_t e1 = cudaMemsetAsync(tb + b->counters_off, 0, b->counters_bytes, st);
    cudaError_t e2 = cudaMemsetAsync(b->status_base, 0, sizeof(int32_t) * b->n_status, st);
    cudaError_t e3 = launch_exec(b->L, st);
    e = cudaStreamEndCapture(st, &b->graph);
    if (e1 || e2 || e3 || e) {
      if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
      return cuda_err(ctx, e1 ? e1 : e2 ? e2 : e3 ? e3 : e, "capturing the executor graph");
    }
    e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
    if (e) return cuda_err(ctx, e, "instantiating the executor graph");
  }
  if (b->gexec) {
    e = cudaGraphLaunch(b->gexec, st);
    if (e) return cuda_err(ctx, e, "launching the executor graph");
  } else {
    if ((e = cudaMemsetAsync(tb + b->counters_off, 0, b->counters_bytes, st)))
      return cuda_err(ctx, e, "zeroing counters");
    if ((e = cudaMemsetAsync(b->status_base, 0, sizeof(int32_t) * b->n_status, st)))
      return cuda_err(ctx, e, "zeroing status words");
    if ((e = launch_exec(b->L, st))) return cuda_err(ctx, e, "launching the executor");
  }
  if ((e = cudaEventRecord(b->done->ev, st))) return cuda_err(ctx, e, "recording an event");
  for (vl_result* r : b->results) r->stream = st;
  return VL_OK;
}

vl_status batch_release_results(vl_batch* b, vl_result** outs) {
  for (size_t j = 0; j < b->results.size(); ++j) {
    vl_result* r = b->results[j];
    r->borrowed = false;
    outs[j] = r;
  }
  b->results.clear();
  b->released = true;
  return VL_OK;
}

vl_status batch_read_status(vl_batch* b, cudaStream_t st, int32_t* first_nonzero) {
  std::vector<int32_t> w(b->n_status);
  cudaError_t e = cudaMemcpyAsync(w.data(), b->status_base, sizeof(int32_t) * w.size(),
                                  cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return cuda_err(b->ctx, e, "reading batch status words");
  *first_nonzero = 0;
  for (int32_t v : w)
    if (v) { *first_nonzero = v; break; }
  return VL_OK;
}

void batch_destroy(vl_batch* b) {
  if (!b) return;
  for (vl_result* r : b->results) {
    r->tag = TAG_DEAD;
    delete r;
  }
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  // the per-operator graph allocated its intermediates through graph memory
  // nodes: give that memory back to the device for the stream-ordered pool
  if (b->plain_form && b->gexec) cudaDeviceGraphMemTrim(b->ctx->device);
  b->tag = TAG_DEAD;
  delete b;
}

}  // namespace vl

// ========================================================== plain form ==

namespace vl {

// The per-operator form of plan P on `st`: one launch per primitive, the
// roots written to `roots` (root slot s at roots + mask_bytes * (s -
// n_inter_slots)), device errors to *status (which the caller clears).
// Intermediate memory comes from the stream-ordered pool and is released in
// stream order before returning; no host synchronisation and no event, so
// the whole sequence can be captured into a CUDA graph (the allocations
// become graph memory nodes, freed inside the graph).
vl_status plain_enqueue(vl_context* ctx, const Plan& P, vl_image* const* imgs, int H, int W, int D,
                        char* roots, int32_t* status, cudaStream_t st) {
  const int Wp = words_per_row(W), pitch = 32 * Wp;
  const bool vol = volume_plan(P);
  MaskGeom g{H, W, Wp};
  if (vol) g.Hs = H / D;
  // labelling tiles of 16 rows when an image has fewer 32-row tiles than SMs
  if (!vol && (long long)ccl_tiles_y(H) * ccl_tiles_x(Wp) < ctx->sm_count) g.cth = 16;
  const size_t mask_bytes = (size_t)H * Wp * 4;
  cudaError_t e;
  auto root_buf = [&](int slot) {
    return reinterpret_cast<uint32_t*>(roots + mask_bytes * (slot - P.n_inter_slots));
  };
  // number terms: one launch per operation into register planes; the
  // compared terms are copied into number images, which follow the
  // formula's own images
  struct Chan { const void* p; int format; };
  const size_t plane_elems = (size_t)H * pitch;
  const int n_own = (int)P.img_kind.size();
  DevBlockPtr numbuf;
  std::vector<Chan> reg_view(kArithMaxRegs, Chan{nullptr, PX_F32});
  if (!P.arith.empty()) {
    const size_t plane_bytes = plane_elems * sizeof(float);
    if ((e = dev_alloc(ctx, plane_bytes * (size_t)(P.arith_regs + P.n_num_images), st, &numbuf)))
      return cuda_err(ctx, e, "allocating number images");
    char* nb = static_cast<char*>(numbuf->ptr);
    for (const ArithInsn& A : P.arith) {
      if (A.op == A_VALUE) {
        const vl_image* im = imgs[A.img];
        reg_view[A.dst] = Chan{static_cast<const char*>(im->data) +
                                   (size_t)A.ch * plane_elems * (im->format == PX_U16 ? 2 : 4),
                               im->format};
      } else if (A.op == A_STORE) {
        e = cudaMemcpyAsync(nb + plane_bytes * (P.arith_regs + A.img), reg_view[A.a].p, plane_bytes,
                            cudaMemcpyDeviceToDevice, st);
      } else {
        float* out = reinterpret_cast<float*>(nb + plane_bytes * A.dst);
        const Chan a = reg_view[A.a];
        const Chan b = A.b == kArithConst ? Chan{nullptr, PX_F32} : reg_view[A.b];
        e = launch_arith(A.op, a.p, a.format, b.p, b.format, A.c, out, H, W, pitch, st);
        reg_view[A.dst] = Chan{out, PX_F32};
      }
      if (e) return cuda_err(ctx, e, "launching a number-term operation");
    }
  }
  auto chan = [&](int img, int ch) -> Chan {
    if (img >= n_own)
      return Chan{static_cast<const char*>(numbuf->ptr) +
                      sizeof(float) * plane_elems * (size_t)(P.arith_regs + img - n_own),
                  PX_F32};
    const vl_image* im = imgs[img];
    return Chan{static_cast<const char*>(im->data) +
                    (size_t)ch * plane_elems * (im->format == PX_U16 ? 2 : 4),
                im->format};
  };
  // percentiles
  DevBlockPtr pct, sel_scratch;
  if (P.n_pct_slots) {
    if ((e = dev_alloc(ctx, sizeof(float) * P.n_pct_slots, st, &pct))) return cuda_err(ctx, e, "allocating percentiles");
    // channels of a million pixels and more take the grid-wide select
    const bool wide = (long long)H * W >= (1LL << 20);
    if (wide && (e = dev_alloc(ctx, select_wide_scratch_bytes(), st, &sel_scratch)))
      return cuda_err(ctx, e, "allocating select scratch");
    for (const PctDesc& d : P.pct) {
      const long long n = (long long)H * W;
      const long long rank = (long long)(d.q * (double)(n - 1));
      const Chan c = chan(d.img, d.ch);
      float* o = static_cast<float*>(pct->ptr) + d.slot;
      e = wide ? launch_select_wide(c.p, c.format, pitch, H, W, rank, o, sel_scratch->ptr, st)
               : launch_select(c.p, c.format, pitch, H, W, rank, o, st);
      if (e) return cuda_err(ctx, e, "launching a percentile select");
    }
  }
  // rho scratch
  DevBlockPtr scratch;
  CclScratch sc{};
  Rz3Scratch sc3{};
  if (!P.rz.empty() && vol) {
    // labels of phi2, a flag per component, the seed voxels, tile state
    const size_t px = (size_t)H * W;
    const size_t tiles = (size_t)ccl_tiles_y(H, g.Hs) * ccl_tiles_x(Wp);
    const int tcap = ccl_tile_cap_host(Wp);
    size_t off = 0;
    auto take = [&](size_t b) { off = align_up(off, 256); size_t o = off; off += b; return o; };
    const size_t oL = take(px * 4), oF = take(px), oS = take(mask_bytes), oP = take(tiles * tcap * 4),
                 oT = take(tiles * tcap);
    if ((e = dev_alloc(ctx, align_up(off, 256), st, &scratch)))
      return cuda_err(ctx, e, "allocating select scratch");
    char* p = static_cast<char*>(scratch->ptr);
    sc3.ccl.G = reinterpret_cast<int32_t*>(p + oL);
    sc3.ccl.tile_cap = tcap;
    sc3.ccl.tpar = reinterpret_cast<int32_t*>(p + oP);
    sc3.ccl.tflag = reinterpret_cast<uint8_t*>(p + oT);
    sc3.F = reinterpret_cast<uint8_t*>(p + oF);
    sc3.seed = reinterpret_cast<uint32_t*>(p + oS);
  } else if (!P.rz.empty()) {
    const size_t px = (size_t)H * W;
    const size_t tiles = (size_t)ccl_tiles_y(H, 0, ccl_rows(g)) * ccl_tiles_x(Wp);
    const int tcap = ccl_tile_cap_host(Wp, ccl_rows(g));
    size_t off = 0;
    auto take = [&](size_t b) { off = align_up(off, 256); size_t o = off; off += b; return o; };
    const size_t oG = take(2 * px * 4), oP = take(tiles * tcap * 4), oT = take(tiles * tcap);
    if ((e = dev_alloc(ctx, align_up(off, 256), st, &scratch)))
      return cuda_err(ctx, e, "allocating select scratch");
    char* p = static_cast<char*>(scratch->ptr);
    sc.G = reinterpret_cast<int32_t*>(p + oG);
    sc.tile_cap = tcap;
    sc.tpar = reinterpret_cast<int32_t*>(p + oP);
    sc.tflag = reinterpret_cast<uint8_t*>(p + oT);
  }
  const int N = (int)P.exec.size();
  std::vector<int> uses(N, 0), root_slot(N, -1);
  for (int i = 0; i < N; ++i) {
    const ENode& x = P.exec[i];
    if (x.a >= 0 && (x.op == E_NOT || x.op == E_NEAR || x.op == E_COPY || x.op == E_AND ||
                     x.op == E_OR || x.op == E_ANDNOT || x.op == E_RZ)) uses[x.a]++;
    if (x.b >= 0 && (x.op == E_AND || x.op == E_OR || x.op == E_ANDNOT || x.op == E_RZ)) uses[x.b]++;
  }
  for (int q = 0; q < P.n_roots; ++q) root_slot[P.exec_roots[q]] = P.root_slot[q];
  std::vector<uint32_t*> val(N, nullptr);
  std::vector<DevBlockPtr> own(N);
  for (int i = 0; i < N; ++i) {
    const ENode& x = P.exec[i];
    if (x.op == E_MASK) { val[i] = imgs[x.img]->mask; continue; }
    if (root_slot[i] >= 0) {
      val[i] = root_buf(root_slot[i]);
    } else {
      if ((e = dev_alloc(ctx, mask_bytes, st, &own[i]))) return cuda_err(ctx, e, "allocating a mask");
      val[i] = static_cast<uint32_t*>(own[i]->ptr);
    }
    uint32_t* o = val[i];
    switch (x.op) {
      case E_TRUE: e = launch_const(g, true, o, st); break;
      case E_FALSE: e = launch_const(g, false, o, st); break;
      case E_THR: {
        const Chan c = chan(x.img, x.ch);
        e = launch_threshold(c.p, c.format, pitch, g, x.t, nullptr, x.lt, o, st);
        break;
      }
      case E_PCT: {
        const Chan c = chan(x.img, x.ch);
        e = launch_threshold(c.p, c.format, pitch, g, 0.f, static_cast<float*>(pct->ptr) + x.pct_slot,
                             x.lt, o, st);
        break;
      }
      case E_NOT: e = launch_not(val[x.a], g, o, st); break;
      case E_AND: e = launch_and(val[x.a], val[x.b], g, o, st); break;
      case E_OR: e = launch_or(val[x.a], val[x.b], g, o, st); break;
      case E_ANDNOT: e = launch_andnot(val[x.a], val[x.b], g, o, st); break;
      case E_NEAR:
        e = vol ? launch_near3(val[x.a], g, P.conn, o, st) : launch_near(val[x.a], g, P.conn, o, st);
        break;
      case E_COPY: e = cudaMemcpyAsync(o, val[x.a], mask_bytes, cudaMemcpyDeviceToDevice, st); break;
      case E_RZ:
        e = vol ? launch_rz3(val[x.a], val[x.b], g, P.conn, sc3, o, status, st)
                : launch_rz(val[x.a], val[x.b], g, P.conn, sc, o, status, st);
        break;
      default: return set_err(ctx, VL_ERR_INTERNAL, "plain form: unknown node");
    }
    if (e) return cuda_err(ctx, e, "launching a plain operator");
    auto release = [&](int v) {
      if (v >= 0 && --uses[v] == 0 && own[v]) { own[v].reset(); }
    };
    const bool bin = x.op == E_AND || x.op == E_OR || x.op == E_ANDNOT || x.op == E_RZ;
    const bool un = x.op == E_NOT || x.op == E_NEAR || x.op == E_COPY;
    if (un || bin) release(x.a);
    if (bin) release(x.b);
  }
  return VL_OK;
}

}  // namespace vl

namespace {

vl_status eval_plain(vl_context* ctx, const vl_formula* f, vl_image* const* imgs, int n_imgs,
                     cudaStream_t st, vl_result** out) {
  const Plan& P = f->plan;
  int H, W, D;
  vl_status s = check_job_images(ctx, P, imgs, n_imgs, &H, &W, &D);
  if (s != VL_OK) return s;
  const int Wp = words_per_row(W);
  const size_t mask_bytes = (size_t)H * Wp * 4;
  cudaError_t e;
  if ((e = wait_images(imgs, n_imgs, st))) return cuda_err(ctx, e, "waiting for image uploads");
  DevBlockPtr persist;
  if ((e = dev_alloc(ctx, align_up(sizeof(int32_t), 256) + mask_bytes * P.n_root_slots, st, &persist)))
    return cuda_err(ctx, e, "allocating results");
  char* pb = static_cast<char*>(persist->ptr);
  int32_t* status = reinterpret_cast<int32_t*>(pb);
  if ((e = cudaMemsetAsync(status, 0, sizeof(int32_t), st))) return cuda_err(ctx, e, "zeroing status");
  s = plain_enqueue(ctx, P, imgs, H, W, D, pb + 256, status, st);
  if (s != VL_OK) return s;
  auto* r = new vl_result();
  r->ctx = ctx;
  r->H = H; r->W = W; r->Wp = Wp;
  r->D = D;
  r->n_roots = P.n_roots;
  for (int q = 0; q < P.n_roots; ++q)
    r->roots.push_back(reinterpret_cast<uint32_t*>(pb + 256 + mask_bytes * (P.root_slot[q] - P.n_inter_slots)));
  r->status = status;
  r->stream = st;
  r->keep.push_back(persist);
  r->done = std::make_shared<EventHolder>();
  if ((e = cudaEventCreateWithFlags(&r->done->ev, cudaEventDisableTiming)) ||
      (e = cudaEventRecord(r->done->ev, st))) {
    delete r;
    return cuda_err(ctx, e, "recording an event");
  }
  *out = r;
  return VL_OK;
}

}  // namespace

// ================================================================= ABI ==

extern "C" {

VL_API void vl_config_default(vl_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->device = 0;
  cfg->exec_mode = VL_EXEC_FUSED;
  cfg->use_graphs = 1;
}

VL_API vl_status vl_context_create(const vl_config* cfg, vl_context** out) {
  if (!out) return VL_ERR_ARG;
  *out = nullptr;
  auto* c = new vl_context();
  vl_config_default(&c->cfg);
  if (cfg) c->cfg = *cfg;
  c->device = c->cfg.device;
  cudaError_t e = cudaSetDevice(c->device);
  if (e) { delete c; cudaGetLastError(); return VL_ERR_CUDA; }
  cudaDeviceProp prop{};
  if ((e = cudaGetDeviceProperties(&prop, c->device))) { delete c; return VL_ERR_CUDA; }
  c->sm_count = prop.multiProcessorCount;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  // a fixed tile shape needs both sides; with neither the autotuner picks
  // per batch among shapes that fit the buffers sized for 32 x 32
  if ((c->cfg.tile_rows > 0) != (c->cfg.tile_words > 0) || c->cfg.tile_rows < 0 ||
      c->cfg.tile_words < 0 || c->cfg.tile_rows > 1024 || c->cfg.tile_words > 256) {
    delete c;
    return VL_ERR_ARG;
  }
  c->gth = c->cfg.tile_rows > 0 ? c->cfg.tile_rows : 32;
  c->gtww = c->cfg.tile_words > 0 ? c->cfg.tile_words : 32;
  c->hmax = 8;
  const int bh = c->gth + 2 * c->hmax, bw = c->gtww + 2;
  const size_t budget = std::max<size_t>(ccl_smem_bytes(), 64 * 1024);
  c->nb = (int)std::min<size_t>(64, budget / ((size_t)bh * bw * 4));
  if (c->nb < 4) { delete c; return VL_ERR_ARG; }
  c->pp.group_buffers = c->nb;
  c->pp.hmax = c->hmax;
  c->exec_smem = exec_smem_bytes(c->nb, bh, bw);
  {
    // room beside the group buffers for staging rank planes, as long as two
    // CTAs still fit on an SM
    int smem_sm = 0, reserved = 0, optin = 0;
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device) ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, c->device) ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device)) {
      cudaGetLastError();
    } else {
      // (less the executor's static shared words and some slack)
      const size_t two = ((size_t)(smem_sm / 2 - reserved - 256)) & ~(size_t)127;
      if (two > c->exec_smem && two <= (size_t)optin) c->exec_smem = two;
    }
  }
  if ((e = exec_configure(c->exec_smem, &c->ctas_per_sm))) { delete c; cudaGetLastError(); return VL_ERR_CUDA; }
  if (c->ctas_per_sm < 2 && c->exec_smem > exec_smem_bytes(c->nb, bh, bw)) {
    // the widened size lost the second CTA on this GPU: fall back
    c->exec_smem = exec_smem_bytes(c->nb, bh, bw);
    if ((e = exec_configure(c->exec_smem, &c->ctas_per_sm))) { delete c; cudaGetLastError(); return VL_ERR_CUDA; }
  }
  if (c->ctas_per_sm < 1) c->ctas_per_sm = 1;
  if ((e = cudaMalloc(&c->ccl_status, sizeof(int32_t)))) { delete c; cudaGetLastError(); return VL_ERR_OOM; }
  if ((e = cudaMemset(c->ccl_status, 0, sizeof(int32_t)))) { cudaFree(c->ccl_status); delete c; return VL_ERR_CUDA; }
  *out = c;
  return VL_OK;
}

VL_API const char* vl_last_error(vl_context* ctx) {
  if (!valid(ctx, TAG_CTX)) return "invalid context";
  std::lock_guard<std::mutex> g(ctx->err_mu);
  return ctx->err.c_str();
}

VL_API void vl_free(void* h) {
  if (!h) return;
  const uint32_t tag = *reinterpret_cast<uint32_t*>(h);
  switch (tag) {
    case TAG_CTX: {
      auto* c = static_cast<vl_context*>(h);
      DeviceGuard dg(c->device);
      if (c->ccl_status) cudaFree(c->ccl_status);
      c->tag = TAG_DEAD;
      delete c;
      break;
    }
    case TAG_IMG: {
      auto* im = static_cast<vl_image*>(h);
      DeviceGuard dg(im->ctx->device);
      im->tag = TAG_DEAD;
      delete im;
      break;
    }
    case TAG_FML: {
      auto* f = static_cast<vl_formula*>(h);
      f->tag = TAG_DEAD;
      delete f;
      break;
    }
    case TAG_RES: {
      auto* r = static_cast<vl_result*>(h);
      if (r->borrowed) return;  // owned by its batch
      DeviceGuard dg(r->ctx->device);
      r->tag = TAG_DEAD;
      delete r;
      break;
    }
    case TAG_BAT: {
      auto* b = static_cast<vl_batch*>(h);
      DeviceGuard dg(b->ctx->device);
      batch_destroy(b);
      break;
    }
    case TAG_SRV:
      server_destroy(static_cast<vl_server*>(h));
      break;
    default:
      break;
  }
}

// ---------------------------------------------------------------- images

// max_rows: 65535 for an image; a volume stores depth x height rows, up to
// 2^20 of them.
static vl_status image_common(vl_context* ctx, int32_t h, int32_t w, int32_t c,
                              int32_t max_rows = 65535) {
  if (!valid(ctx, TAG_CTX)) return VL_ERR_ARG;
  if (h < 1 || w < 1 || c < 1 || h > max_rows || w > 65535 || c > 4096)
    return set_err(ctx, VL_ERR_ARG, "image sides must be in [1, 65535] (a volume's depth x height "
                                    "in [1, 2^20]), channels in [1, 4096]");
  if ((long long)h * w > 0x7FFFFFFFLL)
    return set_err(ctx, VL_ERR_ARG, "image has more than 2^31 - 1 pixels");
  return VL_OK;
}

static vl_status image_create(vl_context* ctx, int32_t h, int32_t w, int32_t channels,
                              const void* data, int format, int32_t data_on_device, void* stream,
                              vl_image** out, int32_t max_rows = 65535) {
  vl_status s = image_common(ctx, h, w, channels, max_rows);
  if (s != VL_OK) return s;
  if (!data || !out) return set_err(ctx, VL_ERR_ARG, "null data or output");
  DeviceGuard dg(ctx->device);
  auto im = std::make_unique<vl_image>();
  im->ctx = ctx;
  im->H = h; im->W = w; im->C = channels;
  im->format = format;
  im->Wp = words_per_row(w);
  im->pitch = 32 * im->Wp;
  const size_t esz = format == PX_U16 ? 2 : 4;
  const size_t bytes = (size_t)channels * h * im->pitch * esz;
  cudaError_t e = dev_alloc(ctx, bytes, S(stream), &im->block);
  if (e) return cuda_err(ctx, e, "allocating an image");
  im->data = im->block->ptr;
  if (im->pitch != w && (e = cudaMemsetAsync(im->data, 0, bytes, S(stream))))
    return cuda_err(ctx, e, "clearing image padding");
  e = cudaMemcpy2DAsync(im->data, (size_t)im->pitch * esz, data, (size_t)w * esz, (size_t)w * esz,
                        (size_t)channels * h,
                        data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        S(stream));
  if (e) return cuda_err(ctx, e, "copying an image");
  if ((e = record_ready(im.get(), S(stream)))) return cuda_err(ctx, e, "recording an event");
  *out = im.release();
  return VL_OK;
}

VL_API vl_status vl_image_create(vl_context* ctx, int32_t h, int32_t w, int32_t channels,
                                 const float* data, int32_t data_on_device, void* stream,
                                 vl_image** out) {
  return image_create(ctx, h, w, channels, data, PX_F32, data_on_device, stream, out);
}

VL_API vl_status vl_image_create_u16(vl_context* ctx, int32_t h, int32_t w, int32_t channels,
                                     const uint16_t* data, int32_t data_on_device, void* stream,
                                     vl_image** out) {
  return image_create(ctx, h, w, channels, data, PX_U16, data_on_device, stream, out);
}

static vl_status mask_create(vl_context* ctx, int32_t h, int32_t w, const uint8_t* data,
                             int32_t data_on_device, void* stream, vl_image** out,
                             int32_t max_rows) {
  vl_status s = image_common(ctx, h, w, 1, max_rows);
  if (s != VL_OK) return s;
  if (!data || !out) return set_err(ctx, VL_ERR_ARG, "null data or output");
  DeviceGuard dg(ctx->device);
  auto im = std::make_unique<vl_image>();
  im->ctx = ctx;
  im->H = h; im->W = w; im->C = 1; im->is_mask = 1;
  im->Wp = words_per_row(w);
  im->pitch = 32 * im->Wp;
  cudaError_t e = dev_alloc(ctx, (size_t)h * im->Wp * 4, S(stream), &im->block);
  if (e) return cuda_err(ctx, e, "allocating a mask");
  im->mask = static_cast<uint32_t*>(im->block->ptr);
  const uint8_t* src = data;
  DevBlockPtr tmp;
  if (!data_on_device) {
    if ((e = dev_alloc(ctx, (size_t)h * w, S(stream), &tmp))) return cuda_err(ctx, e, "allocating staging");
    if ((e = cudaMemcpyAsync(tmp->ptr, data, (size_t)h * w, cudaMemcpyHostToDevice, S(stream))))
      return cuda_err(ctx, e, "copying a mask");
    src = static_cast<const uint8_t*>(tmp->ptr);
  }
  if ((e = launch_pack_u8(src, MaskGeom{h, w, im->Wp}, im->mask, S(stream))))
    return cuda_err(ctx, e, "packing a mask");
  if ((e = record_ready(im.get(), S(stream)))) return cuda_err(ctx, e, "recording an event");
  *out = im.release();
  return VL_OK;
}

VL_API vl_status vl_mask_create(vl_context* ctx, int32_t h, int32_t w, const uint8_t* data,
                                int32_t data_on_device, void* stream, vl_image** out) {
  return mask_create(ctx, h, w, data, data_on_device, stream, out, 65535);
}

VL_API vl_status vl_mask_create_packed(vl_context* ctx, int32_t h, int32_t w, const uint32_t* words,
                                       int32_t data_on_device, void* stream, vl_image** out) {
  vl_status s = image_common(ctx, h, w, 1);
  if (s != VL_OK) return s;
  if (!words || !out) return set_err(ctx, VL_ERR_ARG, "null data or output");
  DeviceGuard dg(ctx->device);
  auto im = std::make_unique<vl_image>();
  im->ctx = ctx;
  im->H = h; im->W = w; im->C = 1; im->is_mask = 1;
  im->Wp = words_per_row(w);
  im->pitch = 32 * im->Wp;
  const size_t bytes = (size_t)h * im->Wp * 4;
  cudaError_t e = dev_alloc(ctx, bytes, S(stream), &im->block);
  if (e) return cuda_err(ctx, e, "allocating a mask");
  im->mask = static_cast<uint32_t*>(im->block->ptr);
  if ((e = cudaMemcpyAsync(im->mask, words, bytes,
                           data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           S(stream))))
    return cuda_err(ctx, e, "copying a mask");
  if ((e = launch_clear_padding(im->mask, MaskGeom{h, w, im->Wp}, S(stream))))
    return cuda_err(ctx, e, "clearing mask padding");
  if ((e = record_ready(im.get(), S(stream)))) return cuda_err(ctx, e, "recording an event");
  *out = im.release();
  return VL_OK;
}

VL_API vl_status vl_image_info(const vl_image* img, int32_t* h, int32_t* w, int32_t* channels,
                               int32_t* is_mask) {
  if (!valid(img, TAG_IMG)) return VL_ERR_ARG;
  if (h) *h = img->H;
  if (w) *w = img->W;
  if (channels) *channels = img->C;
  if (is_mask) *is_mask = img->is_mask;
  return VL_OK;
}

VL_API vl_status vl_image_format(const vl_image* img, int32_t* format) {
  if (!valid(img, TAG_IMG) || img->is_mask) return VL_ERR_ARG;
  if (format) *format = img->format;
  return VL_OK;
}

// Volumes: D slices of h x w stored as one image of D * h rows.
constexpr int32_t kVolumeMaxRows = 1 << 20;

static vl_status volume_common(vl_context* ctx, int32_t d, int32_t h) {
  if (!valid(ctx, TAG_CTX)) return VL_ERR_ARG;
  if (d < 1 || h < 1 || (long long)d * h > kVolumeMaxRows)
    return set_err(ctx, VL_ERR_ARG, "a volume needs depth >= 1 and depth x height <= 2^20");
  return VL_OK;
}

static vl_status as_volume(vl_status s, int32_t d, vl_image** out) {
  if (s == VL_OK) (*out)->D = d;
  return s;
}

VL_API vl_status vl_volume_create(vl_context* ctx, int32_t d, int32_t h, int32_t w, int32_t channels,
                                  const float* data, int32_t data_on_device, void* stream,
                                  vl_image** out) {
  vl_status s = volume_common(ctx, d, h);
  if (s != VL_OK) return s;
  return as_volume(image_create(ctx, d * h, w, channels, data, PX_F32, data_on_device, stream, out,
                                kVolumeMaxRows), d, out);
}

VL_API vl_status vl_volume_create_u16(vl_context* ctx, int32_t d, int32_t h, int32_t w,
                                      int32_t channels, const uint16_t* data,
                                      int32_t data_on_device, void* stream, vl_image** out) {
  vl_status s = volume_common(ctx, d, h);
  if (s != VL_OK) return s;
  return as_volume(image_create(ctx, d * h, w, channels, data, PX_U16, data_on_device, stream, out,
                                kVolumeMaxRows), d, out);
}

VL_API vl_status vl_mask_volume_create(vl_context* ctx, int32_t d, int32_t h, int32_t w,
                                       const uint8_t* data, int32_t data_on_device, void* stream,
                                       vl_image** out) {
  vl_status s = volume_common(ctx, d, h);
  if (s != VL_OK) return s;
  return as_volume(mask_create(ctx, d * h, w, data, data_on_device, stream, out, kVolumeMaxRows), d,
                   out);
}

VL_API vl_status vl_image_depth(const vl_image* img, int32_t* d) {
  if (!valid(img, TAG_IMG) || !d) return VL_ERR_ARG;
  *d = img->D;
  return VL_OK;
}

VL_API vl_status vl_result_depth(const vl_result* r, int32_t* d) {
  if (!valid(r, TAG_RES) || !d) return VL_ERR_ARG;
  *d = r->D;
  return VL_OK;
}

// -------------------------------------------------------------- formulas

static PlanParams default_plan_params() {
  // the tile configuration of a default context: 32 x 32-word group tiles,
  // halo budget 8, buffers that fit the labelling footprint
  PlanParams pp;
  pp.hmax = 8;
  const int bh = 32 + 2 * pp.hmax, bw = 32 + 2;
  const size_t budget = std::max<size_t>(ccl_smem_bytes(), 64 * 1024);
  pp.group_buffers = (int)std::min<size_t>(64, budget / ((size_t)bh * bw * 4));
  return pp;
}

VL_API vl_status vl_formula_compile(vl_context* ctx, const vl_node* nodes, int32_t n_nodes,
                                    const int32_t* roots, int32_t n_roots, int32_t connectivity,
                                    vl_formula** out) {
  if (ctx && !valid(ctx, TAG_CTX)) return VL_ERR_ARG;
  if (!out) return set_err(ctx, VL_ERR_ARG, "null output");
  auto f = std::make_unique<vl_formula>();
  f->ctx = ctx;
  f->pp = ctx ? ctx->pp : default_plan_params();
  std::string err;
  int rc = compile_formula(nodes, n_nodes, roots, n_roots, connectivity, f->pp, &f->plan, &err);
  if (rc != VL_OK) return set_err(ctx, (vl_status)rc, err);
  f->plan_hash = plan_hash(f->plan);
  *out = f.release();
  return VL_OK;
}

VL_API vl_status vl_formula_compile_text(vl_context* ctx, const char* src, int32_t connectivity,
                                         vl_formula** out, char* err_buf, int32_t err_len) {
  if (ctx && !valid(ctx, TAG_CTX)) return VL_ERR_ARG;
  auto report = [&](vl_status s, const std::string& m) {
    if (err_buf && err_len > 0) std::snprintf(err_buf, (size_t)err_len, "%s", m.c_str());
    return s == VL_OK ? VL_OK : set_err(ctx, s, m);
  };
  if (!out || !src) return report(VL_ERR_ARG, "null argument");
  TextSpec spec;
  std::string err;
  if (!parse_spec(src, &spec, &err)) return report(VL_ERR_FORMULA, err);
  auto f = std::make_unique<vl_formula>();
  f->ctx = ctx;
  f->pp = ctx ? ctx->pp : default_plan_params();
  const int rc = compile_formula(spec.nodes.data(), (int32_t)spec.nodes.size(), spec.roots.data(),
                                 (int32_t)spec.roots.size(), connectivity, f->pp, &f->plan, &err);
  if (rc != VL_OK) return report((vl_status)rc, err);
  f->plan_hash = plan_hash(f->plan);
  f->loads = spec.loads;
  f->saves = spec.saves;
  f->sources = spec.sources;
  *out = f.release();
  return report(VL_OK, "");
}

VL_API vl_status vl_formula_spec_names(const vl_formula* f, int32_t which, int32_t* count,
                                       int32_t index, char* buf, int32_t len) {
  if (!valid(f, TAG_FML) || which < 0 || which > 2) return VL_ERR_ARG;
  const std::vector<std::string>& v = which == 0 ? f->loads : which == 1 ? f->saves : f->sources;
  if (count) *count = (int32_t)v.size();
  if (!buf) return VL_OK;
  if (index < 0 || index >= (int32_t)v.size() || len < 1) return VL_ERR_ARG;
  std::snprintf(buf, (size_t)len, "%s", v[index].c_str());
  return VL_OK;
}

VL_API vl_status vl_formula_plan(const vl_formula* f, vl_plan_sizes* sizes, vl_plan_step* steps,
                                 vl_plan_insn* insns, vl_plan_select* selects, vl_plan_pct* pct,
                                 int32_t* root_slots, int32_t* mask_slot_images) {
  if (!valid(f, TAG_FML)) return VL_ERR_ARG;
  const Plan& P = f->plan;
  if (sizes) {
    sizes->n_steps = (int32_t)P.steps.size();
    sizes->n_insns = (int32_t)P.insns.size();
    sizes->n_selects = (int32_t)P.rz.size();
    sizes->n_pct = (int32_t)P.pct.size();
    sizes->n_inter_slots = P.n_inter_slots;
    sizes->n_root_slots = P.n_root_slots;
    sizes->n_mask_slots = P.n_mask_slots;
    sizes->n_roots = P.n_roots;
    sizes->n_rank_tables = (int32_t)P.rtab.size();
    sizes->n_rank_values = (int32_t)P.rvals.size();
    sizes->n_rank_planes = P.n_planes;
    sizes->n_deps = (int32_t)P.deps.size();
  }
  static_assert(sizeof(vl_plan_step) == sizeof(StepDesc), "step layout");
  static_assert(sizeof(vl_plan_insn) == sizeof(Insn), "insn layout");
  static_assert(sizeof(vl_plan_select) == sizeof(RzDesc), "select layout");
  static_assert(sizeof(vl_plan_pct) == sizeof(PctDesc), "pct layout");
  if (steps && !P.steps.empty()) std::memcpy(steps, P.steps.data(), sizeof(StepDesc) * P.steps.size());
  if (insns && !P.insns.empty()) std::memcpy(insns, P.insns.data(), sizeof(Insn) * P.insns.size());
  if (selects && !P.rz.empty()) std::memcpy(selects, P.rz.data(), sizeof(RzDesc) * P.rz.size());
  if (pct && !P.pct.empty()) std::memcpy(pct, P.pct.data(), sizeof(PctDesc) * P.pct.size());
  if (root_slots) for (int r = 0; r < P.n_roots; ++r) root_slots[r] = P.root_slot[r];
  if (mask_slot_images)
    for (int k = 0; k < P.n_mask_slots; ++k) mask_slot_images[k] = P.mask_slot_image[k];
  return VL_OK;
}

VL_API vl_status vl_formula_step_deps(const vl_formula* f, int32_t* dep_off, int32_t* deps) {
  if (!valid(f, TAG_FML)) return VL_ERR_ARG;
  const Plan& P = f->plan;
  if (dep_off && !P.dep_off.empty()) std::memcpy(dep_off, P.dep_off.data(), sizeof(int32_t) * P.dep_off.size());
  if (deps && !P.deps.empty()) std::memcpy(deps, P.deps.data(), sizeof(int32_t) * P.deps.size());
  return VL_OK;
}

VL_API vl_status vl_formula_rank_tables(const vl_formula* f, vl_plan_rank* tables,
                                        float* values) {
  if (!valid(f, TAG_FML)) return VL_ERR_ARG;
  static_assert(sizeof(vl_plan_rank) == sizeof(RankTab), "rank table layout");
  const Plan& P = f->plan;
  if (tables && !P.rtab.empty()) std::memcpy(tables, P.rtab.data(), sizeof(RankTab) * P.rtab.size());
  if (values && !P.rvals.empty()) std::memcpy(values, P.rvals.data(), sizeof(float) * P.rvals.size());
  return VL_OK;
}

VL_API vl_status vl_formula_arith(const vl_formula* f, vl_plan_arith* insns, int32_t* n_insns,
                                  int32_t* n_number_images, int32_t* first_number_image) {
  if (!valid(f, TAG_FML)) return VL_ERR_ARG;
  static_assert(sizeof(vl_plan_arith) == sizeof(ArithInsn), "arithmetic program layout");
  const Plan& P = f->plan;
  if (insns && !P.arith.empty()) std::memcpy(insns, P.arith.data(), sizeof(ArithInsn) * P.arith.size());
  if (n_insns) *n_insns = (int32_t)P.arith.size();
  if (n_number_images) *n_number_images = P.n_num_images;
  if (first_number_image) *first_number_image = (int32_t)P.img_kind.size();
  return VL_OK;
}

VL_API vl_status vl_formula_info(const vl_formula* f, int64_t* n_primitive, int64_t* n_reach,
                                 int32_t* n_roots, int32_t* n_images) {
  if (!valid(f, TAG_FML)) return VL_ERR_ARG;
  if (n_primitive) *n_primitive = f->plan.n_primitive;
  if (n_reach) *n_reach = f->plan.n_reach;
  if (n_roots) *n_roots = f->plan.n_roots;
  if (n_images) *n_images = (int32_t)f->plan.img_kind.size();
  return VL_OK;
}

VL_API vl_status vl_formula_stats_get(const vl_formula* f, vl_formula_stats* st) {
  if (!valid(f, TAG_FML) || !st) return VL_ERR_ARG;
  const Plan& P = f->plan;
  std::memset(st, 0, sizeof(*st));
  st->n_primitive = P.n_primitive;
  st->n_reach = P.n_reach;
  st->n_threshold = P.n_thr;
  st->n_not = P.n_not;
  st->n_and = P.n_and;
  st->n_near = P.n_near;
  st->n_roots = P.n_roots;
  st->n_images = (int32_t)P.img_kind.size();
  st->n_steps = (int32_t)P.steps.size();
  for (const StepDesc& s : P.steps) st->n_groups += s.kind == SK_GROUP;
  st->n_selects = (int32_t)P.rz.size();
  std::map<std::pair<int, int>, int> ch;
  for (const ENode& e : P.exec)
    if (e.op == E_THR || e.op == E_PCT) ch[{e.img, e.ch}] = 1;
  st->n_channels_read = (int32_t)ch.size();
  for (const Insn& in : P.insns) {
    if (insn_op(in) == I_STORE) st->mask_writes++;
    if (insn_op(in) == I_LOAD) st->mask_reads++;
  }
  st->mask_writes += (int64_t)P.rz.size();  // each select writes Z
  st->max_halo = P.max_group_halo;
  st->n_number_images = P.n_num_images;
  return VL_OK;
}

// ------------------------------------------------------------ evaluation

VL_API vl_status vl_eval_mode(vl_context* ctx, const vl_formula* f, vl_image* const* imgs,
                              int32_t n_imgs, int32_t exec_mode, void* stream, vl_result** out) {
  if (!valid(ctx, TAG_CTX) || !out) return VL_ERR_ARG;
  if (!valid(f, TAG_FML)) return set_err(ctx, VL_ERR_ARG, "bad formula handle");
  *out = nullptr;
  if (f->pp.group_buffers != ctx->pp.group_buffers || f->pp.hmax != ctx->pp.hmax)
    return set_err(ctx, VL_ERR_ARG, "formula was planned for another tile configuration");
  DeviceGuard dg(ctx->device);
  if (exec_mode != VL_EXEC_PLAIN && exec_mode != VL_EXEC_FUSED)
    return set_err(ctx, VL_ERR_ARG, "unknown execution form");
  // formulas over volumes have the per-operator form only
  if (exec_mode == VL_EXEC_PLAIN || volume_plan(f->plan))
    return eval_plain(ctx, f, imgs, n_imgs, S(stream), out);
  vl_job job{f, imgs, n_imgs, 0};
  vl_batch* b = nullptr;
  vl_status s = batch_build(ctx, &job, 1, S(stream), &b, nullptr, true);
  if (s != VL_OK) return s;
  s = batch_run(b, S(stream));
  if (s == VL_OK) batch_release_results(b, out);
  batch_destroy(b);
  return s;
}

VL_API vl_status vl_eval(vl_context* ctx, const vl_formula* f, vl_image* const* imgs, int32_t n_imgs,
                         void* stream, vl_result** out) {
  if (!valid(ctx, TAG_CTX)) return VL_ERR_ARG;
  return vl_eval_mode(ctx, f, imgs, n_imgs, ctx->cfg.exec_mode, stream, out);
}

VL_API vl_status vl_eval_batch(vl_context* ctx, const vl_job* jobs, int32_t n_jobs, void* stream,
                               vl_result** outs) {
  if (!valid(ctx, TAG_CTX) || !outs) return VL_ERR_ARG;
  DeviceGuard dg(ctx->device);
  vl_batch* b = nullptr;
  vl_status s = batch_build(ctx, jobs, n_jobs, S(stream), &b);
  if (s != VL_OK) return s;
  s = batch_run(b, S(stream));
  if (s == VL_OK) batch_release_results(b, outs);
  batch_destroy(b);
  return s;
}

VL_API vl_status vl_batch_prepare(vl_context* ctx, const vl_job* jobs, int32_t n_jobs, void* stream,
                                  vl_batch** out) {
  if (!valid(ctx, TAG_CTX) || !out) return VL_ERR_ARG;
  DeviceGuard dg(ctx->device);
  return batch_build(ctx, jobs, n_jobs, S(stream), out);
}

VL_API vl_status vl_batch_run(vl_batch* b, void* stream) {
  if (!valid(b, TAG_BAT)) return VL_ERR_ARG;
  DeviceGuard dg(b->ctx->device);
  return batch_run(b, S(stream));
}

VL_API vl_status vl_batch_result(vl_batch* b, int32_t job, vl_result** out) {
  if (!valid(b, TAG_BAT) || !out || b->released) return VL_ERR_ARG;
  if (job < 0 || job >= (int)b->results.size()) return set_err(b->ctx, VL_ERR_ARG, "job out of range");
  *out = b->results[job];
  return VL_OK;
}

VL_API vl_status vl_batch_trace(const vl_batch* b, int64_t* out, int64_t max_entries,
                                int64_t* n_entries) {
  if (!valid(b, TAG_BAT)) return VL_ERR_ARG;
  if (!b->trace) return set_err(b->ctx, VL_ERR_ARG, "the batch's context was made without trace");
  DeviceGuard dg(b->ctx->device);
  const int64_t n = (int64_t)b->trace_meta.size() / 3;
  if (n_entries) *n_entries = n;
  if (!out) return VL_OK;
  std::vector<unsigned long long> t(4 * (size_t)n);
  cudaError_t e = cudaEventSynchronize(b->done->ev);
  if (!e) e = cudaMemcpy(t.data(), b->trace->ptr, t.size() * 8, cudaMemcpyDeviceToHost);
  if (e) return cuda_err(b->ctx, e, "reading the step timeline");
  for (int64_t i = 0; i < std::min(n, max_entries); ++i) {
    out[7 * i + 0] = b->trace_meta[3 * i + 0];
    out[7 * i + 1] = b->trace_meta[3 * i + 1];
    out[7 * i + 2] = b->trace_meta[3 * i + 2];
    for (int k = 0; k < 4; ++k) out[7 * i + 3 + k] = (int64_t)t[4 * i + k];
  }
  return VL_OK;
}

VL_API vl_status vl_batch_info(const vl_batch* b, int64_t* n_items, int32_t* grid, int64_t* smem) {
  if (!valid(b, TAG_BAT)) return VL_ERR_ARG;
  if (n_items) *n_items = b->L.n_items;
  if (grid) *grid = b->L.grid;
  if (smem) *smem = (int64_t)b->L.smem_bytes;
  return VL_OK;
}

// --------------------------------------------------------------- results

VL_API vl_status vl_result_sync(vl_result* r) {
  if (!valid(r, TAG_RES)) return VL_ERR_ARG;
  DeviceGuard dg(r->ctx->device);
  cudaError_t e = r->done ? cudaEventSynchronize(r->done->ev) : cudaStreamSynchronize(r->stream);
  if (e) return cuda_err(r->ctx, e, "waiting for a result");
  int32_t st = 0;
  if ((e = cudaMemcpy(&st, r->status, sizeof(int32_t), cudaMemcpyDeviceToHost)))
    return cuda_err(r->ctx, e, "reading a status word");
  if (st == ST_TIMEOUT) return set_err(r->ctx, VL_ERR_TIMEOUT, "a device-side wait ran out");
  if (st != 0)
    return set_err(r->ctx, VL_ERR_INTERNAL,
                   "a device-side consistency check failed (status word " + std::to_string(st) + ")");
  return VL_OK;
}

VL_API vl_status vl_result_status_word(vl_result* r, int32_t* word) {
  if (!valid(r, TAG_RES) || !word) return VL_ERR_ARG;
  DeviceGuard dg(r->ctx->device);
  cudaError_t e = r->done ? cudaEventSynchronize(r->done->ev) : cudaStreamSynchronize(r->stream);
  if (!e) e = cudaMemcpy(word, r->status, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e) return cuda_err(r->ctx, e, "reading a status word");
  return VL_OK;
}

VL_API vl_status vl_result_info(const vl_result* r, int32_t* h, int32_t* w, int32_t* wp,
                                int32_t* n_roots) {
  if (!valid(r, TAG_RES)) return VL_ERR_ARG;
  if (h) *h = r->H;
  if (w) *w = r->W;
  if (wp) *wp = r->Wp;
  if (n_roots) *n_roots = r->n_roots;
  return VL_OK;
}

VL_API vl_status vl_result_mask(const vl_result* r, int32_t root, uint32_t* dst, int32_t dst_on_device,
                                void* stream) {
  if (!valid(r, TAG_RES) || !dst) return VL_ERR_ARG;
  if (root < 0 || root >= r->n_roots) return set_err(r->ctx, VL_ERR_ARG, "root out of range");
  DeviceGuard dg(r->ctx->device);
  const size_t bytes = (size_t)r->H * r->Wp * 4;
  cudaError_t e = wait_result(r, S(stream));
  if (!e) e = cudaMemcpyAsync(dst, r->roots[root], bytes,
                                  dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  S(stream));
  if (!e && !dst_on_device) e = cudaStreamSynchronize(S(stream));
  if (e) return cuda_err(r->ctx, e, "copying a result mask");
  return VL_OK;
}

VL_API vl_status vl_result_masks(const vl_result* r, uint32_t* dst, int32_t dst_on_device,
                                 void* stream) {
  if (!valid(r, TAG_RES) || !dst) return VL_ERR_ARG;
  DeviceGuard dg(r->ctx->device);
  const size_t words = (size_t)r->H * r->Wp;
  cudaError_t e = wait_result(r, S(stream));
  for (int q = 0; q < r->n_roots && !e; ++q)
    e = cudaMemcpyAsync(dst + words * q, r->roots[q], words * 4,
                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S(stream));
  if (!e && !dst_on_device) e = cudaStreamSynchronize(S(stream));
  if (e) return cuda_err(r->ctx, e, "copying result masks");
  return VL_OK;
}

VL_API vl_status vl_result_mask_u8(const vl_result* r, int32_t root, uint8_t* dst, int32_t dst_on_device,
                                   void* stream) {
  if (!valid(r, TAG_RES) || !dst) return VL_ERR_ARG;
  if (root < 0 || root >= r->n_roots) return set_err(r->ctx, VL_ERR_ARG, "root out of range");
  DeviceGuard dg(r->ctx->device);
  const MaskGeom g{r->H, r->W, r->Wp};
  cudaError_t e = wait_result(r, S(stream));
  if (e) return cuda_err(r->ctx, e, "ordering after a result");
  if (dst_on_device) {
    if ((e = launch_unpack_u8(r->roots[root], g, dst, S(stream)))) return cuda_err(r->ctx, e, "unpacking");
    return VL_OK;
  }
  DevBlockPtr tmp;
  if ((e = dev_alloc(r->ctx, (size_t)r->H * r->W, S(stream), &tmp))) return cuda_err(r->ctx, e, "staging");
  if ((e = launch_unpack_u8(r->roots[root], g, static_cast<uint8_t*>(tmp->ptr), S(stream))) ||
      (e = cudaMemcpyAsync(dst, tmp->ptr, (size_t)r->H * r->W, cudaMemcpyDeviceToHost, S(stream))) ||
      (e = cudaStreamSynchronize(S(stream))))
    return cuda_err(r->ctx, e, "unpacking a result mask");
  return VL_OK;
}

VL_API vl_status vl_result_device_ptr(const vl_result* r, int32_t root, const uint32_t** ptr) {
  if (!valid(r, TAG_RES) || !ptr) return VL_ERR_ARG;
  if (root < 0 || root >= r->n_roots) return set_err(r->ctx, VL_ERR_ARG, "root out of range");
  *ptr = r->roots[root];
  return VL_OK;
}

// ------------------------------------------------------------------- ccl

VL_API vl_status vl_ccl(vl_context* ctx, const vl_image* mask, int32_t connectivity, int32_t* labels_dev,
                        void* stream) {
  if (!valid(ctx, TAG_CTX)) return VL_ERR_ARG;
  if (!valid(mask, TAG_IMG) || !mask->is_mask) return set_err(ctx, VL_ERR_ARG, "vl_ccl needs a mask image");
  if (!labels_dev) return set_err(ctx, VL_ERR_ARG, "null labels buffer");
  const bool vol = connectivity == 6 || connectivity == 26;
  if (connectivity != 4 && connectivity != 8 && !vol)
    return set_err(ctx, VL_ERR_ARG, "connectivity must be 4 or 8 (images), 6 or 26 (volumes)");
  if (mask->D > 1 && !vol) return set_err(ctx, VL_ERR_ARG, "a volume needs connectivity 6 or 26");
  DeviceGuard dg(ctx->device);
  MaskGeom g{mask->H, mask->W, mask->Wp};
  if (vol) g.Hs = mask->H / mask->D;
  const size_t tiles = (size_t)ccl_tiles_y(mask->H, g.Hs) * ccl_tiles_x(mask->Wp);
  const int tcap = ccl_tile_cap_host(mask->Wp);
  DevBlockPtr tmp;  // per-tile labelling state, released in stream order
  cudaError_t e = dev_alloc(ctx, align_up(tiles * tcap * 4, 256) + tiles * tcap, S(stream), &tmp);
  if (e) return cuda_err(ctx, e, "allocating labelling scratch");
  CclScratch sc{};
  sc.G = labels_dev;
  sc.tile_cap = tcap;
  sc.tpar = static_cast<int32_t*>(tmp->ptr);
  sc.tflag = static_cast<uint8_t*>(tmp->ptr) + align_up(tiles * tcap * 4, 256);
  vl_image* mi = const_cast<vl_image*>(mask);
  e = wait_images(&mi, 1, S(stream));
  if (!e) e = cudaMemsetAsync(ctx->ccl_status, 0, sizeof(int32_t), S(stream));
  if (!e)
    e = vol ? launch_labels3(mask->mask, g, connectivity, sc, ctx->ccl_status, S(stream))
            : launch_ccl_labels(mask->mask, g, connectivity, sc, ctx->ccl_status, S(stream));
  if (e) return cuda_err(ctx, e, "launching connected components");
  return VL_OK;
}

VL_API vl_status vl_ccl_pointer_jumping(vl_context* ctx, const vl_image* mask, int32_t connectivity,
                                        int32_t period, int32_t max_rounds, int32_t* labels_dev,
                                        void* stream, int32_t* iterations) {
  if (!valid(ctx, TAG_CTX)) return VL_ERR_ARG;
  if (!valid(mask, TAG_IMG) || !mask->is_mask) return set_err(ctx, VL_ERR_ARG, "pointer jumping needs a mask image");
  if (!labels_dev) return set_err(ctx, VL_ERR_ARG, "null labels buffer");
  if (connectivity != 4 && connectivity != 8) return set_err(ctx, VL_ERR_ARG, "connectivity must be 4 or 8");
  if (period < 0 || max_rounds < 0) return set_err(ctx, VL_ERR_ARG, "negative period or round limit");
  DeviceGuard dg(ctx->device);
  const size_t n = (size_t)mask->H * mask->W;
  DevBlockPtr tmp;  // second label buffer + termination flag
  cudaError_t e = dev_alloc(ctx, align_up(n * 4, 256) + 256, S(stream), &tmp);
  if (e) return cuda_err(ctx, e, "allocating pointer-jumping scratch");
  int32_t* scratch = static_cast<int32_t*>(tmp->ptr);
  int32_t* flag = reinterpret_cast<int32_t*>(static_cast<char*>(tmp->ptr) + align_up(n * 4, 256));
  vl_image* mi = const_cast<vl_image*>(mask);
  if ((e = wait_images(&mi, 1, S(stream)))) return cuda_err(ctx, e, "waiting for the mask");
  int32_t flag_host = 0;
  int iters = 0;
  bool converged = false;
  e = ccl_pointer_jumping(mask->mask, MaskGeom{mask->H, mask->W, mask->Wp}, connectivity,
                          period ? period : 16, max_rounds ? max_rounds : 65536, labels_dev, scratch,
                          flag, &flag_host, S(stream), &iters, &converged);
  if (e) return cuda_err(ctx, e, "running pointer jumping");
  if (iterations) *iterations = iters;
  if (!converged) return set_err(ctx, VL_ERR_TIMEOUT, "pointer jumping did not converge within the round limit");
  return VL_OK;
}

VL_API vl_status vl_ccl_status(vl_context* ctx, void* stream) {
  if (!valid(ctx, TAG_CTX)) return VL_ERR_ARG;
  DeviceGuard dg(ctx->device);
  int32_t st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, ctx->ccl_status, sizeof(int32_t), cudaMemcpyDeviceToHost, S(stream));
  if (!e) e = cudaStreamSynchronize(S(stream));
  if (e) return cuda_err(ctx, e, "reading the labelling status");
  if (st == ST_TIMEOUT) return VL_ERR_TIMEOUT;
  return st ? VL_ERR_INTERNAL : VL_OK;
}

}  // extern "C"
