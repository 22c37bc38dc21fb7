// Connected component labelling that allocates no memory.
//
// Who needs it: callers that cannot call cudaMalloc.  cudaMalloc (unlike the
// stream-ordered cudaMallocAsync the rest of the library uses) synchronises
// the whole device, which latency-critical loops cannot afford; some
// deployments reserve all device memory at start-up for their own pool, so
// any further allocation fails; and code whose memory belongs to another
// allocator (a framework's caching allocator) must not grow the device
// footprint behind that allocator's back.  Such callers bring their own input
// and output buffers; the little working memory the labelling needs beyond
// them lives in the fixed array below.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds it (kBytes, about 5 MiB) until the process exits.
// Host code must not use the symbol as a pointer -- on the host it is only a
// stand-in -- so every call looks up its device address with
// cudaGetSymbolAddress, with the caller's device current.  The lookup is a
// host-side table read once the module is loaded (it allocates nothing); it
// is repeated on every call instead of cached so that a call made after
// cudaDeviceReset, or under another context of the same device, gets the
// address that is valid now.  The first call on a device loads the module
// and sets the labelling kernels' shared-memory attribute: make it before
// any stream capture.
#include <cuda_runtime.h>

#include "../../include/vl.h"
#include "kernels.h"
#include "vl_internal.h"

namespace {

// Saved per-tile labelling state: one int32 and one byte per entry; a tile
// of Wp words needs CCL_NS * min(32, Wp) * 32 entries.
constexpr size_t kEntries = size_t(1) << 20;
constexpr size_t kStatusBytes = 256;  // the status word, padded
constexpr size_t kBytes = kStatusBytes + kEntries * 4 + kEntries;

__device__ __align__(256) unsigned char g_ccl_scratch[kBytes];

vl_status from_cuda(cudaError_t e) {
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? VL_ERR_OOM : VL_ERR_CUDA;
}

}  // namespace

extern "C" VL_API vl_status vl_ccl_noalloc(const uint32_t* mask_dev, int32_t h, int32_t w,
                                           int32_t connectivity, int32_t* labels_dev,
                                           int32_t wait, void* stream) {
  if (!mask_dev || !labels_dev) return VL_ERR_ARG;
  if (h < 1 || w < 1 || h > 65535 || w > 65535 || (long long)h * w > 0x7FFFFFFFLL)
    return VL_ERR_ARG;
  if (connectivity != 4 && connectivity != 8) return VL_ERR_ARG;
  const int Wp = vl::words_per_row(w);
  const size_t tiles = (size_t)vl::ccl_tiles_y(h) * vl::ccl_tiles_x(Wp);
  const int tcap = vl::ccl_tile_cap_host(Wp);
  if (tiles * (size_t)tcap > kEntries) return VL_ERR_SHAPE;  // beyond the fixed array
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_ccl_scratch);
  if (e) return from_cuda(e);
  unsigned char* base = static_cast<unsigned char*>(p);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int32_t* status = reinterpret_cast<int32_t*>(base);
  vl::CclScratch sc{};
  sc.G = labels_dev;  // the labels double as the union-find array
  sc.tile_cap = tcap;
  sc.tpar = reinterpret_cast<int32_t*>(base + kStatusBytes);
  sc.tflag = base + kStatusBytes + kEntries * 4;
  // the status word keeps the previous call's value: clear it first
  if ((e = cudaMemsetAsync(status, 0, sizeof(int32_t), st))) return from_cuda(e);
  if ((e = vl::launch_ccl_labels(mask_dev, vl::MaskGeom{h, w, Wp}, connectivity, sc, status, st)))
    return from_cuda(e);
  if (!wait) return VL_OK;
  int32_t word = 0;
  if ((e = cudaMemcpyAsync(&word, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st)))
    return from_cuda(e);
  if (word == vl::ST_TIMEOUT) return VL_ERR_TIMEOUT;
  return word ? VL_ERR_INTERNAL : VL_OK;
}
