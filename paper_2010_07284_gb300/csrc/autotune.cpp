// Tile autotuner: picks the fused-group tile shape and the persistent grid
// of a batch by timing the batch itself, and remembers the winner per batch
// signature.  Why it matters: a step of the executor has one work item per
// tile, so one 2048 x 2048 image in 32 x 32-word tiles gives 128 items for
// 304 resident CTAs (the GPU runs a fraction full and each tile's long
// instruction sequence sets the step's latency), while thousands of small
// images give far more items than CTAs and prefer large tiles with less
// halo.  Nothing here changes results: every shape computes the same masks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <iterator>
#include <set>

#include "runtime.h"

namespace vl {

namespace {

// Candidate shapes, largest first (rows, words).
const TileShape kShapes[] = {{32, 32, 0}, {64, 16, 0}, {32, 16, 0}, {16, 32, 0},
                             {16, 16, 0}, {64, 8, 0},  {32, 8, 0},  {16, 8, 0}};

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ULL;
  return h;
}
uint64_t fnv_int(uint64_t h, int64_t v) { return fnv(h, &v, sizeof v); }

int log2_bucket(int64_t v) {
  int b = 0;
  while (v > 1) { v >>= 1; ++b; }
  return b;
}

bool valid_ctx(const void* h) { return h && *static_cast<const uint32_t*>(h) == TAG_CTX; }

// Signature of a batch: its formulas and the coarse sizes of its images.
bool batch_signature(const vl_context* ctx, const vl_job* jobs, int n, uint64_t* key) {
  std::set<uint64_t> plans;
  int64_t total = 0, max_h = 0, max_wp = 0;
  for (int j = 0; j < n; ++j) {
    const vl_formula* f = jobs[j].formula;
    if (!f || f->tag != TAG_FML || !jobs[j].images || jobs[j].n_images < 1) return false;
    const vl_image* im = jobs[j].images[0];
    if (!im || im->tag != TAG_IMG) return false;
    plans.insert(f->plan_hash);
    total += (int64_t)im->H * im->W;
    max_h = std::max<int64_t>(max_h, im->H);
    max_wp = std::max<int64_t>(max_wp, im->Wp);
  }
  uint64_t h = 1469598103934665603ULL;
  h = fnv_int(h, ctx->sm_count);
  for (uint64_t p : plans) h = fnv_int(h, (int64_t)p);
  h = fnv_int(h, log2_bucket(n));
  h = fnv_int(h, log2_bucket(total));
  h = fnv_int(h, log2_bucket(max_h));
  h = fnv_int(h, log2_bucket(max_wp));
  *key = h;
  return true;
}

int64_t group_tiles(const vl_job* jobs, int n, const TileShape& t) {
  int64_t tiles = 0;
  for (int j = 0; j < n; ++j) {
    const vl_image* im = jobs[j].images[0];
    tiles += (int64_t)((im->H + t.rows - 1) / t.rows) * ((im->Wp + t.words - 1) / t.words);
  }
  return tiles;
}

// The per-operator form is reported as a 0 x 0 tile with 0 CTAs per SM.
vl_tile_choice to_choice(const vl_context* ctx, const TileShape& t, int status, double ms) {
  vl_tile_choice c{};
  c.tile_rows = t.per_op ? 0 : t.rows;
  c.tile_words = t.per_op ? 0 : t.words;
  c.ctas_per_sm = t.per_op ? 0
                  : t.ctas_per_sm > 0 ? std::min(t.ctas_per_sm, ctx->ctas_per_sm) : ctx->ctas_per_sm;
  c.status = status;
  c.ms = ms;
  return c;
}

}  // namespace

uint64_t plan_hash(const Plan& P) {
  uint64_t h = 1469598103934665603ULL;
  h = fnv_int(h, P.conn);
  if (!P.steps.empty()) h = fnv(h, P.steps.data(), sizeof(StepDesc) * P.steps.size());
  if (!P.insns.empty()) h = fnv(h, P.insns.data(), sizeof(Insn) * P.insns.size());
  if (!P.rz.empty()) h = fnv(h, P.rz.data(), sizeof(RzDesc) * P.rz.size());
  if (!P.pct.empty()) h = fnv(h, P.pct.data(), sizeof(PctDesc) * P.pct.size());
  return h;
}

bool tile_shape_fits(const vl_context* ctx, const TileShape& t) {
  if (t.rows < 1 || t.words < 1) return false;
  const size_t bytes = (size_t)ctx->nb * (t.rows + 2 * ctx->hmax) * (t.words + 2) * 4;
  return bytes <= ctx->exec_smem;
}

TileShape pick_tile_shape(vl_context* ctx, const vl_job* jobs, int n_jobs, int* tuned,
                          bool allow_per_op) {
  if (tuned) *tuned = 0;
  if (ctx->cfg.tile_rows > 0 && ctx->cfg.tile_words > 0)
    return TileShape{ctx->cfg.tile_rows, ctx->cfg.tile_words, 0};
  uint64_t key = 0;
  if (batch_signature(ctx, jobs, n_jobs, &key)) {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end() && tile_shape_fits(ctx, it->second) &&
        (allow_per_op || !it->second.per_op)) {
      if (tuned) *tuned = 1;
      return it->second;
    }
  } else {
    return TileShape{};  // batch_build reports the bad handle
  }
  // a lone job with a tiny plan: its per-operator kernels (a handful of
  // launches beats a chain of executor steps)
  if (allow_per_op && n_jobs == 1 && jobs[0].formula->plan.n_primitive <= kTinyPlanPrimitives &&
      !ctx->cfg.trace) {
    TileShape t{};
    t.per_op = true;
    return t;
  }
  // heuristic: the largest shape whose tiles per step fill three quarters
  // of the grid (smaller tiles pay more halo than the last CTAs bring: on
  // a 2048 x 2048 image 32 x 16 tiles, 256 of them, beat 16 x 16 by a fifth)
  const int64_t grid = (int64_t)ctx->sm_count * ctx->ctas_per_sm;
  TileShape last{};
  for (const TileShape& t : kShapes) {
    if (!tile_shape_fits(ctx, t)) continue;
    last = t;
    if (4 * group_tiles(jobs, n_jobs, t) >= 3 * grid) return t;
  }
  return last;
}

}  // namespace vl

using namespace vl;

extern "C" VL_API vl_status vl_autotune(vl_context* ctx, const vl_job* jobs, int32_t n_jobs,
                                        void* stream, int32_t reps, vl_tile_choice* trials,
                                        int32_t max_trials, int32_t* n_trials,
                                        vl_tile_choice* best) {
  if (!valid_ctx(ctx) || !jobs || n_jobs < 1 || !best) return VL_ERR_ARG;
  if (ctx->cfg.tile_rows > 0) return set_err(ctx, VL_ERR_ARG, "the context has a fixed tile shape");
  if (reps < 1) reps = 3;
  uint64_t key = 0;
  if (!batch_signature(ctx, jobs, n_jobs, &key)) return set_err(ctx, VL_ERR_ARG, "bad job handles");
  int prev_dev = -1;
  cudaGetDevice(&prev_dev);
  if (prev_dev != ctx->device) cudaSetDevice(ctx->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  vl_status rc = VL_OK;
  std::vector<vl_tile_choice> all;
  TileShape win{};
  double win_ms = -1;
  cudaError_t ce = cudaEventCreate(&e0);
  if (!ce) ce = cudaEventCreate(&e1);
  if (ce) rc = cuda_err(ctx, ce, "creating timing events");
  DevBlockPtr flush;  // larger than the 129 MB L2
  if (rc == VL_OK && dev_alloc(ctx, (size_t)192 << 20, st, &flush) != cudaSuccess) {
    cudaGetLastError();
    flush.reset();
  }
  std::vector<int> cps_list{ctx->ctas_per_sm};
  if (ctx->ctas_per_sm > 1) cps_list.push_back(1);
  // candidates: every tile shape and CTA count of the persistent executor,
  // and for a batch of one job its per-operator kernels in a graph
  // Besides the fixed shapes, for one job: per tile width, the lowest tile
  // height whose tiles still fit in one wave of the grid (a 2048 x 2048
  // image: 14 x 32 gives 294 tiles, 27 x 16 gives 304, where 16 x 32 gives
  // 256 and leaves 48 CTAs without a tile of each group step).
  std::vector<TileShape> bases(std::begin(kShapes), std::end(kShapes));
  if (n_jobs == 1) {
    const int64_t grid = (int64_t)ctx->sm_count * ctx->ctas_per_sm;
    const vl_image* im = jobs[0].images[0];
    for (int words : {32, 16}) {
      const int64_t tx = (im->Wp + words - 1) / words, per_col = grid / tx;
      if (per_col < 1) continue;
      const int rows = (int)((im->H + per_col - 1) / per_col);
      if (rows < 8 || rows > 64) continue;
      bool dup = false;
      for (const TileShape& b : bases) dup |= b.rows == rows && b.words == words;
      if (!dup) bases.push_back(TileShape{rows, words, 0});
    }
  }
  std::vector<TileShape> cands;
  for (const TileShape& base : bases) {
    if (!tile_shape_fits(ctx, base)) continue;
    for (int cps : cps_list) {
      TileShape t = base;
      t.ctas_per_sm = cps;
      cands.push_back(t);
    }
  }
  if (n_jobs == 1) {
    TileShape t{};
    t.per_op = true;
    cands.push_back(t);
  }
  for (const TileShape& t : cands) {
    if (rc != VL_OK) break;
    {
      vl_batch* b = nullptr;
      vl_status s = batch_build(ctx, jobs, n_jobs, st, &b, &t, !t.per_op);
      double ms = -1;
      // untimed: builds the graph (the per-operator form captures it on its
      // second run), warms up
      if (s == VL_OK) s = batch_run(b, st);
      if (s == VL_OK && t.per_op) s = batch_run(b, st);
      int32_t word = 0;
      if (s == VL_OK) s = batch_read_status(b, st, &word);
      if (s == VL_OK && word) s = (word & 0xFF) == VL_ERR_TIMEOUT ? VL_ERR_TIMEOUT : VL_ERR_INTERNAL;
      if (s == VL_OK) {
        // every timed run starts from a cold L2 (a write larger than the
        // L2 before it), as the batch would in a stream of other work
        double sum = 0;
        cudaError_t e = cudaSuccess;
        for (int r = 0; r < reps && s == VL_OK && !e; ++r) {
          if (flush) e = cudaMemsetAsync(flush->ptr, r & 0xFF, flush->bytes, st);
          if (!e) e = cudaEventRecord(e0, st);
          if (!e) s = batch_run(b, st);
          if (!e && s == VL_OK) e = cudaEventRecord(e1, st);
          if (!e && s == VL_OK) e = cudaEventSynchronize(e1);
          float f = 0;
          if (!e && s == VL_OK) e = cudaEventElapsedTime(&f, e0, e1);
          sum += f;
        }
        if (e) s = cuda_err(ctx, e, "timing a candidate");
        if (s == VL_OK) ms = sum / reps;
      }
      if (b) batch_destroy(b);
      all.push_back(to_choice(ctx, t, s, ms));
      if (s == VL_OK && (win_ms < 0 || ms < win_ms)) {
        win_ms = ms;
        win = t;
      }
      // a CUDA failure other than a full pool leaves the device in an
      // unknown state: stop; a device status (timeout) or OOM only rules
      // this candidate out
      if (s == VL_ERR_CUDA) { rc = s; break; }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (prev_dev >= 0 && prev_dev != ctx->device) cudaSetDevice(prev_dev);
  if (n_trials) *n_trials = (int32_t)all.size();
  if (trials)
    for (int i = 0; i < (int)all.size() && i < max_trials; ++i) trials[i] = all[i];
  if (rc != VL_OK) return rc;
  if (win_ms < 0) return set_err(ctx, VL_ERR_INTERNAL, "no candidate tile shape ran cleanly");
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->tuned[key] = win;
  }
  *best = to_choice(ctx, win, VL_OK, win_ms);
  return VL_OK;
}

extern "C" VL_API vl_status vl_tile_shape(vl_context* ctx, const vl_job* jobs, int32_t n_jobs,
                                          vl_tile_choice* out, int32_t* tuned) {
  if (!valid_ctx(ctx) || !jobs || n_jobs < 1 || !out) return VL_ERR_ARG;
  uint64_t key = 0;
  if (!batch_signature(ctx, jobs, n_jobs, &key)) return set_err(ctx, VL_ERR_ARG, "bad job handles");
  int t = 0;
  const TileShape s = pick_tile_shape(ctx, jobs, n_jobs, &t);
  *out = to_choice(ctx, s, VL_OK, -1);
  if (tuned) *tuned = t;
  return VL_OK;
}

extern "C" VL_API vl_status vl_tune_save(vl_context* ctx, const char* path) {
  if (!valid_ctx(ctx) || !path) return VL_ERR_ARG;
  FILE* fh = std::fopen(path, "w");
  if (!fh) return set_err(ctx, VL_ERR_ARG, std::string("cannot write ") + path);
  std::lock_guard<std::mutex> g(ctx->tune_mu);
  std::fprintf(fh, "vl-tile-table 1 sm_count %d\n", ctx->sm_count);
  for (const auto& kv : ctx->tuned)  // the per-operator form as 0 0 0
    std::fprintf(fh, "%016llx %d %d %d\n", (unsigned long long)kv.first,
                 kv.second.per_op ? 0 : kv.second.rows, kv.second.per_op ? 0 : kv.second.words,
                 kv.second.per_op ? 0 : kv.second.ctas_per_sm);
  const bool ok = std::fclose(fh) == 0;
  return ok ? VL_OK : set_err(ctx, VL_ERR_ARG, std::string("cannot write ") + path);
}

extern "C" VL_API vl_status vl_tune_load(vl_context* ctx, const char* path) {
  if (!valid_ctx(ctx) || !path) return VL_ERR_ARG;
  FILE* fh = std::fopen(path, "r");
  if (!fh) return set_err(ctx, VL_ERR_ARG, std::string("cannot read ") + path);
  int version = 0, sms = 0;
  if (std::fscanf(fh, "vl-tile-table %d sm_count %d", &version, &sms) != 2 || version != 1) {
    std::fclose(fh);
    return set_err(ctx, VL_ERR_ARG, "not a tile table");
  }
  if (sms != ctx->sm_count) {
    std::fclose(fh);
    return set_err(ctx, VL_ERR_ARG, "tile table measured on a GPU with another SM count");
  }
  std::map<uint64_t, TileShape> got;
  unsigned long long key = 0;
  int r = 0, w = 0, c = 0;
  while (std::fscanf(fh, "%llx %d %d %d", &key, &r, &w, &c) == 4) {
    TileShape t{r, w, c};
    if (r == 0 && w == 0 && c == 0) {
      t = TileShape{};
      t.per_op = true;
    } else if (r < 1 || w < 1 || c < 0 || !tile_shape_fits(ctx, t)) {
      std::fclose(fh);
      return set_err(ctx, VL_ERR_ARG, "tile table entry does not fit this context");
    }
    got[(uint64_t)key] = t;
  }
  const bool eof = std::feof(fh) != 0;
  std::fclose(fh);
  if (!eof) return set_err(ctx, VL_ERR_ARG, "malformed tile table");
  std::lock_guard<std::mutex> g(ctx->tune_mu);
  for (const auto& kv : got) ctx->tuned[kv.first] = kv.second;
  return VL_OK;
}
