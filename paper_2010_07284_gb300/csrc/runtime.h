// Runtime objects behind the C ABI handles (internal).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vl.h"
#include "compiler.h"
#include "kernels.h"
#include "vl_internal.h"

namespace vl {

enum : uint32_t {
  TAG_CTX = 0x5643544Bu,
  TAG_IMG = 0x56494D47u,
  TAG_FML = 0x56464D4Cu,
  TAG_RES = 0x56524553u,
  TAG_BAT = 0x56424154u,
  TAG_SRV = 0x56535256u,
  TAG_DEAD = 0xDEADDEADu,
};

// A device allocation released with cudaFreeAsync on `stream` when the last
// owner drops it.
struct DevBlock {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  ~DevBlock();
};
using DevBlockPtr = std::shared_ptr<DevBlock>;

// Shape of the fused-group tiles of one batch and the persistent grid:
// rows x words (32-px words) per tile, CTAs per SM (0 = as many as fit).
struct TileShape {
  int rows = 32, words = 32, ctas_per_sm = 0;
  // a batch of one job: its per-operator kernels captured in the batch's
  // graph instead of the persistent executor (tiles then unused)
  bool per_op = false;
};

}  // namespace vl

struct vl_context {
  uint32_t tag = vl::TAG_CTX;
  vl_config cfg{};
  int device = 0;
  int sm_count = 0;
  int ctas_per_sm = 1;
  size_t exec_smem = 0;
  int gth = 32, gtww = 32, hmax = 8, nb = 14;
  vl::PlanParams pp{};
  int32_t* ccl_status = nullptr;  // device word of vl_ccl
  std::string err;
  std::mutex err_mu;  // guards err
  std::mutex mu;      // serialises launches issued by the server thread
  std::mutex tune_mu;                       // guards tuned
  std::map<uint64_t, vl::TileShape> tuned;  // batch signature -> measured best
};

namespace vl {
struct EventHolder {
  cudaEvent_t ev = nullptr;
  ~EventHolder() {
    if (ev && cudaEventDestroy(ev) != cudaSuccess) cudaGetLastError();
  }
};
}  // namespace vl

struct vl_image {
  uint32_t tag = vl::TAG_IMG;
  vl_context* ctx = nullptr;
  int H = 0, W = 0, C = 0, Wp = 0, pitch = 0;  // H: stored rows (depth * slice rows)
  int D = 1;                // volumes: slices stacked in the H rows (1: an image)
  int is_mask = 0;
  int format = vl::PX_F32;  // number images: PX_F32 or PX_U16 elements
  void* data = nullptr;     // number images: C planes of H x pitch elements
  uint32_t* mask = nullptr;
  vl::DevBlockPtr block;
  std::shared_ptr<vl::EventHolder> ready;  // recorded after the upload
};

struct vl_formula {
  uint32_t tag = vl::TAG_FML;
  vl_context* ctx = nullptr;
  vl::PlanParams pp{};
  vl::Plan plan;
  uint64_t plan_hash = 0;  // of the compiled plan: keys the tuning table
  std::vector<std::string> loads, saves, sources;  // when compiled from a specification text
};

struct vl_result {
  uint32_t tag = vl::TAG_RES;
  vl_context* ctx = nullptr;
  int H = 0, W = 0, Wp = 0;       // H: stored rows (depth * slice rows)
  int D = 1;                      // depth of a volume result
  int n_roots = 0;
  bool borrowed = false;          // owned by a batch
  std::vector<uint32_t*> roots;   // device mask per root
  int32_t* status = nullptr;      // device status word
  cudaStream_t stream = nullptr;
  std::shared_ptr<vl::EventHolder> done;  // recorded after the work
  std::vector<vl::DevBlockPtr> keep;  // memory this result keeps alive
};

struct vl_batch;

namespace vl {

// Helpers shared by api.cpp and server.cpp.
vl_status set_err(vl_context* ctx, vl_status code, const std::string& msg);
vl_status cuda_err(vl_context* ctx, cudaError_t e, const char* what);
cudaError_t dev_alloc(vl_context* ctx, size_t bytes, cudaStream_t st, DevBlockPtr* out);
// Make `st` wait until the uploads of these images are done (images may be
// created on other streams than the one that reads them).
cudaError_t wait_images(vl_image* const* imgs, int n, cudaStream_t st);

// Build a batch (plans, tables, buffers, results) for `jobs`, with the tile
// shape `force` if given, else the one pick_tile_shape chooses.
// `persistent`: always the persistent executor (an explicit request for the
// fused form, and the autotuner's trials); otherwise a lone job with a tiny
// plan takes the per-operator form captured in the batch's graph.
vl_status batch_build(vl_context* ctx, const vl_job* jobs, int n_jobs, cudaStream_t st,
                      vl_batch** out, const TileShape* force = nullptr, bool persistent = false);
// The per-operator form of a plan (one launch per primitive), enqueued on
// `st` without synchronisation or events: roots written at `roots` (root
// slot s at roots + H*Wp*4 * (s - n_inter_slots)), device errors to
// *status; capturable into a CUDA graph.
vl_status plain_enqueue(vl_context* ctx, const Plan& P, vl_image* const* imgs, int H, int W, int D,
                        char* roots, int32_t* status, cudaStream_t st);
// Autotuner (autotune.cpp): the tile shape for a batch -- the fixed shape of
// the context's configuration, else the measured best for the batch's
// signature, else a heuristic.  *tuned is set to 1 when a measurement chose it.
// allow_per_op = false: only shapes of the persistent executor.
TileShape pick_tile_shape(vl_context* ctx, const vl_job* jobs, int n_jobs, int* tuned = nullptr,
                          bool allow_per_op = true);
// Whether the group buffers of this shape fit the executor's shared memory.
bool tile_shape_fits(const vl_context* ctx, const TileShape& t);
uint64_t plan_hash(const Plan& P);
vl_status batch_run(vl_batch* b, cudaStream_t st);
// Hand the batch's results to the caller (they keep the batch memory alive).
vl_status batch_release_results(vl_batch* b, vl_result** outs);
int64_t batch_bytes(const vl_batch* b);
// Copy the batch's status words to the host (synchronises `st`); the first
// nonzero one, or 0, goes to *first_nonzero.
vl_status batch_read_status(vl_batch* b, cudaStream_t st, int32_t* first_nonzero);
void batch_destroy(vl_batch* b);
void server_destroy(vl_server* s);

}  // namespace vl
