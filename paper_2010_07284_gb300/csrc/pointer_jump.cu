// Connected components by iterated pointer jumping: the labelling the paper
// runs on the GPU (Sec. 3.3), kept as an in-library comparison for the
// union-find labelling that the model checker uses.
//
// What the method computes (Sec. 3.3): labels are pixel coordinates, here
// the linear index y*W + x (whose order is the lexicographic order of (row,
// column)); background is -1.  A jump gives every set pixel the largest
// label found around the pixel its label names (that pixel included), so
// labels both spread one step and follow each other's pointers.  Jumps
// alone can leave a component with several labels at concave corners, so
// every `period` jumps a repair lets each set pixel raise the label stored
// at the pixel its own label names to the largest label around it; then a
// test asks whether any set pixel still has a set neighbour with another
// label, and the host stops when none has.
//
// Here all of it is one pass kernel with four modes over a shared
// neighbourhood scan: the first jump reads the mask directly (a set pixel
// is its own label, so no initialisation pass runs), the repair raises
// labels in place with atomic maxima (labels only grow, and every label a
// pixel can see belongs to its own component), and the test is a warp vote
// with one flag store per warp.  Each round ends with one device-to-host
// read of the flag: the host-synchronised loop of the paper's design, which
// the persistent union-find executor replaces.
#include "dev_common.cuh"
#include "kernels.h"

namespace vl {

namespace {

constexpr int kPjThreads = 256;
enum PjMode { PJ_FIRST_JUMP = 0, PJ_JUMP = 1, PJ_REPAIR = 2, PJ_TEST = 3, PJ_OWN = 4 };

struct PjGrid {
  const uint32_t* m;
  int H, W, Wp, conn;
  VL_DEV bool set(int y, int x) const {
    return (__ldg(m + (size_t)y * Wp + (x >> 5)) >> (x & 31)) & 1u;
  }
  // label of pixel (y, x): from the mask in the first jump, else from `lab`
  // -- through the read-only cache where the pass does not write `lab`
  // (jumps write the other buffer, the test writes none), through L2 in the
  // in-place repair
  template <bool RO>
  VL_DEV int32_t label(const int32_t* lab, bool from_mask, int y, int x) const {
    if (from_mask) return set(y, x) ? y * W + x : -1;
    return RO ? __ldg(lab + (size_t)y * W + x) : __ldcg(lab + (size_t)y * W + x);
  }
  // largest label over the neighbourhood of (y, x), (y, x) included; with
  // `differs`, also whether a labelled neighbour's label is not `own`
  template <bool RO>
  VL_DEV int32_t scan(const int32_t* lab, bool from_mask, int y, int x, int32_t own,
                      bool* differs) const {
    int32_t best = -1;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = y + dy;
      if (yy < 0 || yy >= H) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx;
        if (xx < 0 || xx >= W || (conn == 4 && dy != 0 && dx != 0)) continue;
        const int32_t l = label<RO>(lab, from_mask, yy, xx);
        best = max(best, l);
        if (differs && l >= 0 && l != own) *differs = true;
      }
    }
    return best;
  }
};

// One pass over every pixel.  cur: labels before the pass (unused by the
// first jump and by PJ_OWN, which only writes every pixel's own label: the
// labels when no jump runs); nxt: labels after a jump, or cur itself for
// the in-place repair; flag: set by the test.
template <int MODE>
__global__ void k_pj_pass(PjGrid g, const int32_t* cur, int32_t* nxt, int32_t* flag) {
  const long long n = (long long)g.H * g.W;
  bool differs = false;
  // (the test stops a thread at its first mismatch: one is enough)
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
       i < n && !(MODE == PJ_TEST && differs); i += (long long)gridDim.x * blockDim.x) {
    int y, x;
    split_index(i, g.W, y, x);
    const int32_t own = (MODE == PJ_FIRST_JUMP || MODE == PJ_OWN) ? (g.set(y, x) ? (int32_t)i : -1)
                        : MODE == PJ_REPAIR ? __ldcg(cur + i) : __ldg(cur + i);
    if (MODE == PJ_OWN) {
      nxt[i] = own;
    } else if (MODE == PJ_JUMP || MODE == PJ_FIRST_JUMP) {
      int32_t out = -1;
      if (own >= 0) {
        int qy, qx;
        split_index(own, g.W, qy, qx);
        out = g.scan<true>(cur, MODE == PJ_FIRST_JUMP, qy, qx, 0, nullptr);
      }
      nxt[i] = out;
    } else if (own >= 0) {
      if (MODE == PJ_REPAIR) {
        // nxt == cur here: raised in place
        const int32_t around = g.scan<false>(cur, false, y, x, 0, nullptr);
        if (around > __ldcg(cur + own)) atomicMax(nxt + own, around);
      } else {
        g.scan<true>(cur, false, y, x, own, &differs);
      }
    }
  }
  if (MODE == PJ_TEST && __any_sync(0xFFFFFFFFu, differs) && (threadIdx.x & 31) == 0) *flag = 1;
}

int pj_grid(long long n) {
  long long b = (n + kPjThreads - 1) / kPjThreads;
  if (b > 152LL * 64) b = 152LL * 64;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t ccl_pointer_jumping(const uint32_t* mask, MaskGeom g, int conn, int period,
                                int max_rounds, int32_t* labels, int32_t* scratch,
                                int32_t* flag_dev, int32_t* flag_host, cudaStream_t st,
                                int* iterations, bool* converged) {
  const long long n = (long long)g.H * g.W;
  const int grid = pj_grid(n);
  const PjGrid pg{mask, g.H, g.W, g.Wp, conn};
  *iterations = 0;
  *converged = false;
  int32_t* cur = labels;
  int32_t* nxt = scratch;
  cudaError_t e = cudaSuccess;
  bool have = false;  // cur holds labels
  auto own_labels = [&]() {
    k_pj_pass<PJ_OWN><<<grid, kPjThreads, 0, st>>>(pg, nullptr, cur, nullptr);
    have = true;
    return cudaGetLastError();
  };
  for (int round = 0; !e && round < max_rounds; ++round) {
    for (int k = 0; k < period && !e; ++k) {
      if (!have) k_pj_pass<PJ_FIRST_JUMP><<<grid, kPjThreads, 0, st>>>(pg, nullptr, nxt, nullptr);
      else k_pj_pass<PJ_JUMP><<<grid, kPjThreads, 0, st>>>(pg, cur, nxt, nullptr);
      e = cudaGetLastError();
      int32_t* t = cur; cur = nxt; nxt = t;
      have = true;
      ++*iterations;
    }
    if (e) break;
    if (!have && (e = own_labels())) break;  // period 0
    k_pj_pass<PJ_REPAIR><<<grid, kPjThreads, 0, st>>>(pg, cur, cur, nullptr);
    if ((e = cudaGetLastError())) break;
    if ((e = cudaMemsetAsync(flag_dev, 0, sizeof(int32_t), st))) break;
    k_pj_pass<PJ_TEST><<<grid, kPjThreads, 0, st>>>(pg, cur, nullptr, flag_dev);
    if ((e = cudaGetLastError())) break;
    if ((e = cudaMemcpyAsync(flag_host, flag_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, st))) break;
    if ((e = cudaStreamSynchronize(st))) break;
    if (*flag_host == 0) { *converged = true; break; }
  }
  if (!e && !have) e = own_labels();  // no round ran
  if (!e && cur != labels)
    e = cudaMemcpyAsync(labels, cur, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st);
  if (!e) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace vl
